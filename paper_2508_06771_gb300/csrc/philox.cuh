// philox.cuh -- counter-based random numbers for the collision kernels.
//
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): ten rounds of two
// 32x32->64-bit multiplies with the published multipliers, the key advanced
// by the published Weyl increments after every round.  Streams are addressed
// by counter (id, step, tag, 0) under key = seed, so every draw is a pure
// function of (seed, particle or pair id, step, use) and no random-number
// array is stored (the paper precomputes such arrays with cupy, Sec. 4.2 and
// Sec. 4.4).
#pragma once
#include <stdint.h>

namespace ltpc {

enum : uint32_t { TAG_PARTICLE = 1u, TAG_PAIR = 2u, TAG_SCATTER = 3u, TAG_SECONDARY = 4u, TAG_PERM = 5u,
                  TAG_RECOMB = 6u };

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               uint32_t k0, uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return make_uint4(c0, c1, c2, c3);
}

// The ten round keys of a seed (key + r x Weyl increment), computed once on
// the host and passed in the kernel's parameter block, so that every round
// XORs with a parameter instead of advancing the key in registers.
struct PhiloxKeys {
    uint32_t k0[10], k1[10];
};

__host__ __device__ inline PhiloxKeys philox_keys(uint64_t seed)
{
    PhiloxKeys K;
    uint32_t a = (uint32_t)seed, b = (uint32_t)(seed >> 32);
    for (int r = 0; r < 10; ++r) {
        K.k0[r] = a;
        K.k1[r] = b;
        a += 0x9E3779B9u;
        b += 0xBB67AE85u;
    }
    return K;
}

__device__ __forceinline__ uint4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                               const PhiloxKeys& K)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c0;
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ K.k0[r];
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ K.k1[r];
        c1 = (uint32_t)p1;
        c3 = (uint32_t)p0;
        c0 = n0;
        c2 = n2;
    }
    return make_uint4(c0, c1, c2, c3);
}

__device__ __forceinline__ uint4 draw(const PhiloxKeys& K, uint32_t id, uint32_t step, uint32_t tag)
{
    return philox4x32_10(id, step, tag, 0u, K);
}

// Block for stream `tag` of id `id` (particle index, or the smaller index of a
// pair) at step `step`.
__device__ __forceinline__ uint4 draw(uint32_t k0, uint32_t k1, uint32_t id, uint32_t step, uint32_t tag)
{
    return philox4x32_10(id, step, tag, 0u, k0, k1);
}

// Uniform variates on (0, 1].  Double: (w + 1/2) 2^-32, exact, in (0, 1).
// Float: ((w >> 8) + 1) 2^-24, exact in binary32, in (0, 1].
template <class T> __device__ __forceinline__ T unif(uint32_t w);
template <> __device__ __forceinline__ double unif<double>(uint32_t w)
{
    return fma((double)w, 0x1p-32, 0x1p-33);
}
// Built from bits, without an integer-to-float conversion:
// ((w >> 8) + 1) 2^-24 = (w >> 9) 2^-23 + (((w >> 8) & 1) + 1) 2^-24, where the
// first term is the mantissa of a float in [1, 2) minus 1 and the sum is exact
// (the result is a multiple of 2^-24 in (0, 1]).
__device__ __forceinline__ float unif24(uint32_t u24)   // u24 = w >> 8
{
    const float hi = __uint_as_float(0x3F800000u | (u24 >> 1)) - 1.0f;
    const float lo = __uint_as_float(0x33800000u + ((u24 & 1u) << 23));   // 2^-24 or 2^-23
    return hi + lo;
}
template <> __device__ __forceinline__ float unif<float>(uint32_t w)
{
    return unif24(w >> 8);
}

// Uniform variate for an angle, on [0, 1): only its distribution matters, not
// that it avoids 0.  binary64 keeps unif (the 1e-12 parity bar needs the same
// value as the FP64 reference); binary32 takes the top 23 bits as the mantissa
// of a float in [1, 2) and subtracts 1 (exact): three instructions instead of
// the eight of unif<float>, and within 2^-23 of it.
template <class T> __device__ __forceinline__ T unif_angle(uint32_t w) { return unif<T>(w); }
template <> __device__ __forceinline__ float unif_angle<float>(uint32_t w)
{
    return __uint_as_float(0x3F800000u | (w >> 9)) - 1.0f;
}

// Range of unif(w) over all w sharing the top 16 bits `hi` (used to decide
// the null-collision candidate test without redrawing the stream).
template <class T> __device__ __forceinline__ void unif_hi16_range(uint32_t hi, T& lo, T& up);
template <> __device__ __forceinline__ void unif_hi16_range<double>(uint32_t hi, double& lo, double& up)
{
    lo = fma((double)(hi << 16), 0x1p-32, 0x1p-33);
    up = fma((double)((hi << 16) | 0xFFFFu), 0x1p-32, 0x1p-33);
}
template <> __device__ __forceinline__ void unif_hi16_range<float>(uint32_t hi, float& lo, float& up)
{
    lo = unif24(hi << 8);
    up = unif24((hi << 8) | 0xFFu);
}

}  // namespace ltpc
