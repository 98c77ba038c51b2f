// bijection.cuh -- the keyed bijection of the bijection pairing mode.
//
// Table 5 pairs consecutive entries of a cell's index list; any random perfect
// matching serves the Takizuka-Abe model (Sec. 4.4).  In the bijection mode a
// cell of n >= BIJ_MIN_N particles puts the particle of id rank r (its index
// among the cell's ids in ascending order) at pairing position pi(r):
//   * [0, n) is embedded in [0, a b), a = ceil(sqrt n), b = ceil(n / a), as
//     x = L b + R;
//   * six Feistel rounds alternate the radix: round i replaces (L, R) by
//     (R, (L + F_i(R)) mod m_i), m_i = a for even i and b for odd i, with
//     F_i(R) = floor(mix(R ^ K_i) m_i / 2^32) and mix a multiply-xorshift-
//     multiply hash;
//   * an image at or above n is mapped again (cycle walking).
// The round keys are six words of two Philox blocks of (seed, cell, step);
// a seventh word rounds the null-collision candidate count (Sec. 4.2 selects
// P_null N particles): n_c = floor(P_null N + U).  The forward map places a
// rank; the inverse finds the rank at a pairing position.  All arithmetic is
// 32-bit integer: a, b <= 256 for n <= 65536, so x < 2^16 and the quotient
// x / b is exact as a multiply-high by ceil(2^32 / b).
#pragma once
#include <stdint.h>

#if defined(__CUDACC__)
#define BIJ_HD __host__ __device__ __forceinline__
#else
#define BIJ_HD static inline
#endif

namespace ltpc {

constexpr uint32_t BIJ_MIN_N = 4097u;   // smaller cells keep the pairing-key sort
constexpr uint32_t BIJ_MAX_N = 65536u;  // largest cell the 32-bit arithmetic covers

struct BijParams {
    uint32_t n, a, b, mb;   // mb = ceil(2^32 / b)
    uint32_t key[6];
};

BIJ_HD uint32_t bij_umulhi(uint32_t x, uint32_t y)
{
#if defined(__CUDA_ARCH__)
    return __umulhi(x, y);
#else
    return (uint32_t)(((uint64_t)x * (uint64_t)y) >> 32);
#endif
}

BIJ_HD uint32_t bij_mix(uint32_t t)
{
    const uint32_t w = t * 0x9E3779B1u;
    return (w ^ (w >> 16)) * 0x85EBCA6Bu;
}

BIJ_HD uint32_t bij_round(uint32_t r, uint32_t key, uint32_t m) { return bij_umulhi(bij_mix(r ^ key), m); }

// t mod m for t < 2m, without a branch: t - m wraps to above t when t < m.
BIJ_HD uint32_t bij_reduce(uint32_t t, uint32_t m)
{
    const uint32_t u = t - m;
#if defined(__CUDA_ARCH__)
    return min(t, u);
#else
    return u < t ? u : t;
#endif
}

// a = ceil(sqrt(n)), b = ceil(n / a), mb = ceil(2^32 / b) (n >= 2).
BIJ_HD void bij_shape(uint32_t n, uint32_t* a, uint32_t* b, uint32_t* mb)
{
    uint32_t s = 1;
    while (s * s < n) ++s;
    *a = s;
    *b = (n + s - 1) / s;
    *mb = 0xFFFFFFFFu / *b + 1u;
}

// One pass of the six rounds over [0, a b).
BIJ_HD uint32_t bij_enc(const BijParams& B, uint32_t x)
{
    uint32_t L = bij_umulhi(x, B.mb);
    uint32_t R = x - L * B.b;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint32_t m = (i & 1) ? B.b : B.a;
        const uint32_t t = bij_reduce(L + bij_round(R, B.key[i], m), m);
        L = R;
        R = t;
    }
    return L * B.b + R;
}

BIJ_HD uint32_t bij_dec(const BijParams& B, uint32_t y)
{
    uint32_t L = bij_umulhi(y, B.mb);
    uint32_t R = y - L * B.b;
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        const uint32_t m = (i & 1) ? B.b : B.a;
        const uint32_t t = bij_reduce(R + m - bij_round(L, B.key[i], m), m);
        R = L;
        L = t;
    }
    return L * B.b + R;
}

// The inverse rounds with each round function read from a table: tab[i][R] =
// bij_round(R, K_i, m_i) for R below the radix of the round's input (b for
// even i, a for odd i), so the six rounds are six byte loads (the values are
// below m_i <= 256).  Same result as bij_dec.
template <class TAB>
BIJ_HD uint32_t bij_dec_tab(const BijParams& B, const TAB& tab, uint32_t y)
{
    uint32_t L = bij_umulhi(y, B.mb);
    uint32_t R = y - L * B.b;
#pragma unroll
    for (int i = 5; i >= 0; --i) {
        const uint32_t m = (i & 1) ? B.b : B.a;
        const uint32_t t = bij_reduce(R + m - (uint32_t)tab(i, L), m);
        R = L;
        L = t;
    }
    return L * B.b + R;
}

// The forward rounds with the same tables (round i reads its input R below b for
// even i, a for odd i, as the inverse does).  Same result as bij_enc.
template <class TAB>
BIJ_HD uint32_t bij_enc_tab(const BijParams& B, const TAB& tab, uint32_t x)
{
    uint32_t L = bij_umulhi(x, B.mb);
    uint32_t R = x - L * B.b;
#pragma unroll
    for (int i = 0; i < 6; ++i) {
        const uint32_t m = (i & 1) ? B.b : B.a;
        const uint32_t t = bij_reduce(L + (uint32_t)tab(i, R), m);
        L = R;
        R = t;
    }
    return L * B.b + R;
}

// pi(r) and its inverse on [0, n) (cycle walking ends: the cycle of r in
// [0, a b) returns to r < n).
BIJ_HD uint32_t bij_forward(const BijParams& B, uint32_t r)
{
    uint32_t y = bij_enc(B, r);
    while (y >= B.n) y = bij_enc(B, y);
    return y;
}

BIJ_HD uint32_t bij_inverse(const BijParams& B, uint32_t q)
{
    uint32_t x = bij_dec(B, q);
    while (x >= B.n) x = bij_dec(B, x);
    return x;
}

}  // namespace ltpc
