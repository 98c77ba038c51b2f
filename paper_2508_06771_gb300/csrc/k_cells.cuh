// k_cells.cuh -- the fused per-cell collision kernel.
//
// One thread-block cluster of C CTAs processes one cell per work item
// (persistent loop, dynamic tickets).  Per cell it performs, on chip:
//   1. pairing order (Table 5, reading of "define partner pairs"): every
//      particle draws a key r_l; the cell's particles are sorted by (r_l, l)
//      with a bucket sort distributed over the cluster's shared memory (a
//      particle alone in its bucket takes its position from the bucket scan);
//   2. step S1 (Table 2), the Takizuka-Abe collision of consecutive entries
//      (CCS4-CCS5 of Table 5), with the optional momentum/energy restoration
//      from the cell's sums after S1 and its state before S1 (taken from the
//      per-cell record that the pass's first kernel forms from the stored
//      moments);
//   3. step S2a for electron-neutral collisions C1/C2 (Table 1) with the
//      null-collision method of Sec. 4.2, staging ionization secondaries
//      (Table 3, CS5) at a deterministic slot;
//   4. the particle-to-cell moments of steps S3a/S3b (Sec. 4.5) of the result.
// Velocities are read once from HBM (gathered through the cell's index list,
// CCS3) and written once.  Latency hiding: the next work item is drawn one
// ticket ahead and copied with cp.async, the cell's parameters are prefetched
// the same way, single-CTA classes gather the velocities with cp.async
// straight into pairing order, and the next cell's id list and velocity
// ranges are brought into L2 while the current cell computes.  Per-cell sums
// are formed per thread and per warp in the working precision (a pair's two
// particles in the two lanes of packed binary32 operations) and combined in
// double.  Cluster CTAs write back the positions they own straight to the
// particles' ids.  Index math is in ltpc_index.h.
#pragma once
#include <cooperative_groups.h>
#include <type_traits>

#include "bijection.cuh"
#include "ltpc_index.h"
#include "ltpc_internal.h"
#include "philox.cuh"

namespace ltpc {
namespace cg = cooperative_groups;

template <int C>
struct Cl {
    static __device__ __forceinline__ unsigned rank()
    {
        if constexpr (C == 1) return 0u;
        else return cg::this_cluster().block_rank();
    }
    static __device__ __forceinline__ void sync()
    {
        if constexpr (C == 1) __syncthreads();
        else cg::this_cluster().sync();
    }
    // Address of `p` (a shared-memory object of this CTA) in CTA `r` of the cluster.
    template <class P>
    static __device__ __forceinline__ P* at(P* p, unsigned r)
    {
        if constexpr (C == 1) return p;
        else return cg::this_cluster().map_shared_rank(p, r);
    }
};

// Elementary functions per working precision.  binary32 uses the SFU
// approximations, one MUFU instruction each (relative errors ~1e-7, far inside
// the 1e-5 moment bar); binary64 uses correctly rounded or library functions
// (1e-12 velocity bar).
template <class T> struct Math;
template <> struct Math<float> {
    static __device__ __forceinline__ float rsqrt(float x) { return rsqrtf(x); }
    static __device__ __forceinline__ float rcp(float x)
    {
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float sqrt(float x)
    {
        float y;
        asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float ln(float x) { return __logf(x); }
    static __device__ __forceinline__ float expm1(float x) { return expm1f(x); }
    // sin and cos of 2 pi u for u in [0, 1], evaluated on [-pi, pi]
    static __device__ __forceinline__ void sincos2pi(float u, float* s, float* c)
    {
        float sx, cx;
        __sincosf(fmaf(6.28318530717958647692f, u, -3.14159265358979323846f), &sx, &cx);
        *s = -sx;
        *c = -cx;
    }
    static __device__ __forceinline__ int ebin(float E)
    {
        // (log10 E + 2) 64/5 clamped to [0, 63] (E = 0, subnormal or NaN: log2 gives
        // -inf or NaN, which fmaxf maps to 0), then its floor without a
        // float-to-integer conversion: t + 2^23 rounded down has floor(t) as its low
        // mantissa bits
        float t = fmaf(__log2f(E), 0.30102999566398120f * 12.8f, 25.6f);
        t = fminf(fmaxf(t, 0.f), 63.f);
        return (int)(__float_as_uint(__fadd_rd(t, 8388608.0f)) & 0x7FFFFFu);
    }
};
template <> struct Math<double> {
    static __device__ __forceinline__ double rsqrt(double x) { return 1.0 / ::sqrt(x); }
    static __device__ __forceinline__ double rcp(double x) { return 1.0 / x; }
    static __device__ __forceinline__ double sqrt(double x) { return ::sqrt(x); }
    static __device__ __forceinline__ double ln(double x) { return ::log(x); }
    static __device__ __forceinline__ double expm1(double x) { return ::expm1(x); }
    static __device__ __forceinline__ void sincos2pi(double u, double* s, double* c) { sincospi(2.0 * u, s, c); }
    static __device__ __forceinline__ int ebin(double E)
    {
        if (!(E > 0.0)) return 0;
        const double t = (log10(E) + 2.0) * 12.8;
        if (t < 0.0) return 0;
        if (t >= 63.0) return 63;
        return (int)t;
    }
};

// Exchange records of the bijection mode's cluster classes: a particle's velocity
// and id in one 16-byte (binary32) or 32-byte (binary64) record.  They move
// between the SMs of a cluster through L2 (.cg: a record another SM wrote is
// never read from a stale line of this SM's L1).
template <class T> struct Xg;
template <> struct Xg<float> {
    static __device__ __forceinline__ void put(void* b, uint32_t i, float x, float y, float z, uint32_t l)
    {
        __stcg(reinterpret_cast<float4*>(b) + i, make_float4(x, y, z, __uint_as_float(l)));
    }
    static __device__ __forceinline__ void get(const void* b, uint32_t i, float& x, float& y, float& z, uint32_t& l)
    {
        const float4 t = __ldcg(reinterpret_cast<const float4*>(b) + i);
        x = t.x; y = t.y; z = t.z;
        l = __float_as_uint(t.w);
    }
};
template <> struct Xg<double> {
    static __device__ __forceinline__ void put(void* b, uint32_t i, double x, double y, double z, uint32_t l)
    {
        double2* p = reinterpret_cast<double2*>(b) + 2 * (size_t)i;
        __stcg(p, make_double2(x, y));
        __stcg(p + 1, make_double2(z, __longlong_as_double((long long)l)));
    }
    static __device__ __forceinline__ void get(const void* b, uint32_t i, double& x, double& y, double& z, uint32_t& l)
    {
        const double2* p = reinterpret_cast<const double2*>(b) + 2 * (size_t)i;
        const double2 t0 = __ldcg(p), t1 = __ldcg(p + 1);
        x = t0.x; y = t0.y; z = t1.x;
        l = (uint32_t)__double_as_longlong(t1.y);
    }
};

// Takizuka-Abe binary collision of an equal-mass pair (a, b): the change
// Delta u of the relative velocity (zero when u = 0); the caller applies
// v_a += Delta u / 2, v_b -= Delta u / 2.  A is the cell coefficient so that
// <delta^2> = A / |u|^3; w holds the pair's three uniforms (Box-Muller radius
// and angle for delta, then the azimuth phi).
template <class T>
__device__ __forceinline__ void ta_delta(T ax, T ay, T az, T bx, T by, T bz, T A, uint4 w, T& dux, T& duy, T& duz)
{
    using M = Math<T>;
    const T ux = ax - bx, uy = ay - by, uz = az - bz;
    const T up2 = ux * ux + uy * uy;
    const T usq = up2 + uz * uz;
    dux = duy = duz = T(0);
    if (usq == T(0)) return;
    const T u = M::sqrt(usq);
    const T iu = M::rcp(u);
    const T var = A * iu * iu * iu;
    T sth, cth, sph, cph;
    M::sincos2pi(unif_angle<T>(w.y), &sth, &cth);
    M::sincos2pi(unif_angle<T>(w.z), &sph, &cph);
    const T delta = M::sqrt(var * (T(-2) * M::ln(unif<T>(w.x)))) * cth;
    // sin(Theta) = 2d/(1+d^2), 1-cos(Theta) = 2d^2/(1+d^2); for |d| > 1 use t = 1/d
    const bool small = fabs(delta) <= T(1);
    const T t = small ? delta : M::rcp(delta);
    const T rr = M::rcp(T(1) + t * t);
    const T sin_t = T(2) * t * rr;
    const T omc_t = small ? T(2) * t * t * rr : T(2) * rr;
    if (up2 > T(0)) {
        const T uperp = M::sqrt(up2);
        const T ip = M::rcp(uperp);
        const T ca = uz * sin_t * cph * ip;
        const T cb = u * sin_t * sph * ip;
        dux = ux * ca - uy * cb - ux * omc_t;
        duy = uy * ca + ux * cb - uy * omc_t;
        duz = -uperp * sin_t * cph - uz * omc_t;
    } else {
        dux = u * sin_t * cph;
        duy = u * sin_t * sph;
        duz = -uz * omc_t;
    }
}

// Two independent pairs at once: pair 0 in the .x lanes, pair 1 in the .y lanes of
// packed binary32 operations, the SFU functions per lane (the steps of ta_delta).
__device__ __forceinline__ void ta_delta2(float2 ax, float2 ay, float2 az, float2 bx, float2 by, float2 bz, float A,
                                          const uint4& w0, const uint4& w1, float2& dux, float2& duy, float2& duz)
{
    using M = Math<float>;
    auto neg = [](float2 v) { return make_float2(-v.x, -v.y); };
    auto mk = [](float a, float b) { return make_float2(a, b); };
    const float2 ux = __fadd2_rn(ax, neg(bx)), uy = __fadd2_rn(ay, neg(by)), uz = __fadd2_rn(az, neg(bz));
    const float2 up2 = __ffma2_rn(uy, uy, __fmul2_rn(ux, ux));
    const float2 usq = __ffma2_rn(uz, uz, up2);
    const float2 u = mk(M::sqrt(usq.x), M::sqrt(usq.y));
    const float2 iu = mk(M::rcp(u.x), M::rcp(u.y));
    const float2 var = __fmul2_rn(__fmul2_rn(__fmul2_rn(mk(A, A), iu), iu), iu);
    float sth0, cth0, sph0, cph0, sth1, cth1, sph1, cph1;
    M::sincos2pi(unif_angle<float>(w0.y), &sth0, &cth0);
    M::sincos2pi(unif_angle<float>(w0.z), &sph0, &cph0);
    M::sincos2pi(unif_angle<float>(w1.y), &sth1, &cth1);
    M::sincos2pi(unif_angle<float>(w1.z), &sph1, &cph1);
    const float2 lg = mk(M::ln(unif<float>(w0.x)), M::ln(unif<float>(w1.x)));
    const float2 vv = __fmul2_rn(var, __fmul2_rn(mk(-2.f, -2.f), lg));
    const float2 delta = __fmul2_rn(mk(M::sqrt(vv.x), M::sqrt(vv.y)), mk(cth0, cth1));
    const bool s0 = fabsf(delta.x) <= 1.f, s1 = fabsf(delta.y) <= 1.f;
    const float2 t = mk(s0 ? delta.x : M::rcp(delta.x), s1 ? delta.y : M::rcp(delta.y));
    const float2 q = __ffma2_rn(t, t, mk(1.f, 1.f));
    const float2 rr = mk(M::rcp(q.x), M::rcp(q.y));
    const float2 t2rr = __fmul2_rn(__fmul2_rn(mk(2.f, 2.f), t), rr);      // sin(Theta)
    const float2 big = __fmul2_rn(mk(2.f, 2.f), rr);
    const float2 smallv = __fmul2_rn(t2rr, t);
    const float2 omc = mk(s0 ? smallv.x : big.x, s1 ? smallv.y : big.y);    // 1 - cos(Theta)
    const float2 uperp = mk(M::sqrt(up2.x), M::sqrt(up2.y));
    const bool p0 = up2.x > 0.f, p1 = up2.y > 0.f;
    const float2 ip = mk(p0 ? M::rcp(uperp.x) : 0.f, p1 ? M::rcp(uperp.y) : 0.f);
    const float2 cph = mk(cph0, cph1), sph = mk(sph0, sph1);
    const float2 ca = __fmul2_rn(__fmul2_rn(__fmul2_rn(uz, t2rr), cph), ip);
    const float2 cb = __fmul2_rn(__fmul2_rn(__fmul2_rn(u, t2rr), sph), ip);
    // general case
    float2 gx = __ffma2_rn(neg(ux), omc, __ffma2_rn(neg(uy), cb, __fmul2_rn(ux, ca)));
    float2 gy = __ffma2_rn(neg(uy), omc, __ffma2_rn(ux, cb, __fmul2_rn(uy, ca)));
    float2 gz = __ffma2_rn(neg(uz), omc, __fmul2_rn(neg(__fmul2_rn(uperp, t2rr)), cph));
    // u_perp = 0
    const float2 us = __fmul2_rn(u, t2rr);
    const float2 hx = __fmul2_rn(us, cph), hy = __fmul2_rn(us, sph), hz = __fmul2_rn(neg(uz), omc);
    const bool z0 = usq.x == 0.f, z1 = usq.y == 0.f;
    dux = mk(z0 ? 0.f : (p0 ? gx.x : hx.x), z1 ? 0.f : (p1 ? gx.y : hx.y));
    duy = mk(z0 ? 0.f : (p0 ? gy.x : hy.x), z1 ? 0.f : (p1 ? gy.y : hy.y));
    duz = mk(z0 ? 0.f : (p0 ? gz.x : hz.x), z1 ? 0.f : (p1 ? gz.y : hz.y));
}

// Isotropic unit vector from two uniforms: cos(theta) = 1 - 2 U_a, phi = 2 pi U_b.
template <class T>
__device__ __forceinline__ void iso_dir(uint32_t wa, uint32_t wb, T& dx, T& dy, T& dz)
{
    const T c = T(1) - T(2) * unif<T>(wa);
    const T s = Math<T>::sqrt(fmax(T(0), T(1) - c * c));
    T sp, cp;
    Math<T>::sincos2pi(unif<T>(wb), &sp, &cp);
    dx = s * cp; dy = s * sp; dz = c;
}

// Non-negative floating-point values ordered through their bit patterns.
template <class T> struct MaxBits;
template <> struct MaxBits<float> {
    using U = unsigned int;
    static __device__ __forceinline__ U to(float x) { return __float_as_uint(x); }
    static __device__ __forceinline__ float from(U u) { return __uint_as_float(u); }
};
template <> struct MaxBits<double> {
    using U = unsigned long long;
    static __device__ __forceinline__ U to(double x) { return (U)__double_as_longlong(x); }
    static __device__ __forceinline__ double from(U u) { return __longlong_as_double((long long)u); }
};

template <class T> struct Vec2;
template <> struct Vec2<float> {
    using type = float2;
    static __device__ __forceinline__ float2 make(float a, float b) { return make_float2(a, b); }
};
template <> struct Vec2<double> {
    using type = double2;
    static __device__ __forceinline__ double2 make(double a, double b) { return make_double2(a, b); }
};

// Exclusive prefix sum of one value per thread over the CTA, and the total.
// One barrier: every warp scans the warps' totals itself.  Callers pass a
// barrier before s_scan is written again (the next call).
// Two values of the working precision processed together: binary32 maps onto
// the packed FADD2/FMUL2/FFMA2 instructions (one issue for both lanes, each
// lane rounded exactly as its scalar form); binary64 stays scalar.
template <class T> struct Pk;
// Accumulators: sum (X) and sum (X^2) of both lanes into s; binary32 keeps one
// partial per lane, binary64 folds both into the first lane (no registers for
// a second lane, which would bring no speed).
template <> struct Pk<float> {
    using V = float2;
    static __device__ __forceinline__ V make(float a, float b) { return make_float2(a, b); }
    static __device__ __forceinline__ V add(V a, V b) { return __fadd2_rn(a, b); }
    static __device__ __forceinline__ V mul(V a, V b) { return __fmul2_rn(a, b); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return __ffma2_rn(a, b, c); }
    static __device__ __forceinline__ void acc(V& s, V x) { s = __fadd2_rn(s, x); }
    static __device__ __forceinline__ void acc_sq(V& s, V x) { s = __ffma2_rn(x, x, s); }
};
template <> struct Pk<double> {
    using V = double2;
    static __device__ __forceinline__ V make(double a, double b) { return make_double2(a, b); }
    static __device__ __forceinline__ V add(V a, V b) { return make_double2(a.x + b.x, a.y + b.y); }
    static __device__ __forceinline__ V mul(V a, V b) { return make_double2(a.x * b.x, a.y * b.y); }
    static __device__ __forceinline__ V fma(V a, V b, V c) { return make_double2(::fma(a.x, b.x, c.x), ::fma(a.y, b.y, c.y)); }
    static __device__ __forceinline__ void acc(V& s, V x) { s.x += x.x; s.x += x.y; }
    static __device__ __forceinline__ void acc_sq(V& s, V x) { s.x = ::fma(x.x, x.x, s.x); s.x = ::fma(x.y, x.y, s.x); }
};

template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_scan, uint32_t* total)
{
    constexpr int NW = NT / 32;
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31u) s_scan[warp] = x;
    __syncthreads();
    const uint32_t wv = lane < (unsigned)NW ? s_scan[lane] : 0u;
    uint32_t z = wv;
#pragma unroll
    for (int o = 1; o < NW; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
        if (lane >= (unsigned)o) z += y;
    }
    *total = __shfl_sync(0xFFFFFFFFu, z, NW - 1);
    return __shfl_sync(0xFFFFFFFFu, z - wv, warp) + x - v;
}

constexpr uint32_t LISTCAP = 512;    // positions handled per round of a masked pass

// Run f(q) for every local position q whose bit is set in mask[0..nw),
// in ascending order of q, spreading the work over all threads in rounds of
// at most LISTCAP positions.  Clears the mask.  CTA-collective.
template <int NT, class F>
__device__ __forceinline__ void for_each_masked(uint32_t* mask, uint32_t nw, uint32_t* list, uint32_t* s_scan, F f)
{
    const unsigned tid = threadIdx.x;
    uint32_t word = tid < nw ? mask[tid] : 0u;
    uint32_t total;
    const uint32_t start = block_excl_scan<NT>((uint32_t)__popc(word), s_scan, &total);
    // round k handles the set bits of global rank [k LISTCAP, (k+1) LISTCAP)
    for (uint32_t base = 0u; base < total; base += LISTCAP) {
        uint32_t off = start, w = word;
        while (w) {
            if (off >= base + LISTCAP) break;
            if (off >= base) list[off - base] = tid * 32u + (uint32_t)(__ffs(w) - 1);
            w &= w - 1u;
            ++off;
        }
        __syncthreads();
        const uint32_t nl = total - base < LISTCAP ? total - base : LISTCAP;
        for (uint32_t i = tid; i < nl; i += NT) f(list[i]);
        if (base + LISTCAP < total) __syncthreads();   // the list is refilled; after the
                                                       // last round the caller's next barrier serves
    }
    if (tid < nw) mask[tid] = 0u;
}

// Sum NQ per-thread partials over the cluster in a fixed order: warp
// butterfly in the working precision (at most 32 x ITEMS values per warp
// partial), then the warps' partials by one warp (in the working precision
// for a single CTA, in double for a cluster) -- lane l takes
// quantity l % NQ and every (32 / NQ)-th warp partial, summed as a tree, and
// the lanes of a quantity are combined by xor shuffles -- and the CTAs in rank
// order in double.  Deterministic for a given block shape.  With C = 1 only
// warp 0 may read `out` afterwards (its lanes wrote it); with C > 1 every thread.
template <int NT, int C, int NQ, class A>
__device__ __forceinline__ void cluster_sum(A (&v)[NQ], A* s_red, double* s_cl, double* out)
{
    static_assert(32 % NQ == 0 && NQ <= NT / 32, "quantities per warp");
    constexpr int NW = NT / 32;
    constexpr int G = 32 / NQ;                       // lanes per quantity
    constexpr int PER = (NW + G - 1) / G;            // warp partials per lane
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    // reduce-scatter butterfly: at offset o (16, 8, ...) a lane keeps one half of its
    // remaining quantities (the upper half if bit o of its lane is set) and adds the
    // partner's copy of that half, so after log2(NQ) levels lane l holds quantity
    // l / G summed over its group of G lanes; the group is then closed by xor
    // shuffles: NQ - 1 + log2(G) shuffles instead of 5 NQ
#pragma unroll
    for (int h = NQ / 2, o = 16; h >= 1; h >>= 1, o >>= 1) {
        const bool up = (lane & (unsigned)o) != 0u;
#pragma unroll
        for (int k = 0; k < h; ++k) {
            const A send = up ? v[k] : v[k + h];
            const A keep = up ? v[k + h] : v[k];
            v[k] = keep + __shfl_xor_sync(0xFFFFFFFFu, send, o);
        }
    }
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) v[0] += __shfl_xor_sync(0xFFFFFFFFu, v[0], o);
    if (lane % (unsigned)G == 0u) s_red[warp * NQ + lane / (unsigned)G] = v[0];
    __syncthreads();
    if (warp == 0) {
        const unsigned k = lane % NQ, g = lane / NQ;
        // a single CTA combines its warps' partials in the working precision (binary64 on
        // the FP64 pipe is the slow part of this serial step), a cluster in double
        using R = typename std::conditional<C == 1, A, double>::type;
        R x[PER];
#pragma unroll
        for (int i = 0; i < PER; ++i) {
            const unsigned w = g + (unsigned)i * G;
            x[i] = w < (unsigned)NW ? (R)s_red[w * NQ + k] : R(0);
        }
#pragma unroll
        for (int h = 1; h < PER; h <<= 1) {
#pragma unroll
            for (int i = 0; i + h < PER; i += 2 * h) x[i] += x[i + h];
        }
        R t = x[0];
#pragma unroll
        for (int o = NQ; o < 32; o <<= 1) t += __shfl_xor_sync(0xFFFFFFFFu, t, o);
        if constexpr (C == 1) {
            // a single CTA: warp 0 holds the totals; its callers read them from
            // warp 0 only, so no further barrier
            if (lane < (unsigned)NQ) out[lane] = 0.0 + (double)t;
            __syncwarp();
        } else {
            if (lane < (unsigned)NQ) s_cl[lane] = t;
        }
    }
    if constexpr (C == 1) return;
    Cl<C>::sync();
    if (threadIdx.x < (unsigned)NQ) {
        double acc = 0.0;
        for (unsigned q = 0; q < (unsigned)C; ++q) acc += *Cl<C>::at(&s_cl[threadIdx.x], q);
        out[threadIdx.x] = acc;
    }
    // s_cl is read remotely until every CTA reaches the next cluster barrier, so the
    // caller alternates two buffers between consecutive calls (no trailing cluster barrier)
    __syncthreads();
}

// Largest value over the cluster (exact in any order); s_cl as in cluster_sum.
template <int NT, int C, class A>
__device__ __forceinline__ A cluster_max(A v, A* s_red, double* s_cl)
{
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        A x = lane < (unsigned)(NT / 32) ? s_red[lane] : A(0);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x = fmax(x, __shfl_xor_sync(0xFFFFFFFFu, x, o));
        if (lane == 0) s_cl[0] = (double)x;
    }
    Cl<C>::sync();
    double m = 0.0;
    for (unsigned q = 0; q < (unsigned)C; ++q) m = fmax(m, *Cl<C>::at(&s_cl[0], q));
    return (A)m;                                     // (alternating buffers, as cluster_sum)
}

__device__ __forceinline__ void flag_error(DevState* ds, uint32_t bit) { atomicOr(&ds->err, bit); }

// Asynchronous global -> shared copy of B bytes (4, 8 or 16; both addresses
// B-aligned).  Completion: cp_async_wait_all() by the issuing thread, then a
// barrier before other threads read the destination.
template <int B>
__device__ __forceinline__ void cp_async(void* smem_dst, const void* gsrc)
{
    static_assert(B == 4 || B == 8 || B == 16, "cp.async size");
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(d), "l"(gsrc), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Hint: bring [p, p + bytes) into L2 (bulk prefetch; the range is widened to
// 16-byte boundaries, which stay inside the 256-byte-aligned array).
__device__ __forceinline__ void prefetch_l2(const void* p, size_t bytes)
{
    const uintptr_t a = reinterpret_cast<uintptr_t>(p) & ~(uintptr_t)15;
    const uintptr_t e = (reinterpret_cast<uintptr_t>(p) + bytes + 15) & ~(uintptr_t)15;
    for (uintptr_t q = a; q < e; q += 0x40000u) {   // chunks below the instruction's size limit
        const uint32_t sz = (uint32_t)(e - q < 0x40000u ? e - q : 0x40000u);
        asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(q), "r"(sz) : "memory");
    }
}

// The null-collision candidate test U < P_null decided from the top 16 bits h
// of the candidate word: the smallest uniform over all words with those bits
// is below P_null exactly when h < H, with H computed here once per cell
// (exact: every quantity is a scaled binary32/binary64 value).
template <class T> __device__ __forceinline__ uint32_t cand_threshold(T pnull);
template <> __device__ __forceinline__ uint32_t cand_threshold<float>(float pnull)
{
    // lo(h) = (256 h + 1) 2^-24 < p  <=>  h < (p 2^24 - 1) / 256, all in binary32:
    // p 2^24 is exact, so is p 2^24 - 1 below 2^24 (and at 2^24 the rounding still
    // gives the same ceiling, 65536), so are the scaling by 1/256 and the ceiling
    const float h = ceilf((pnull * 16777216.0f - 1.0f) * 0.00390625f);
    if (!(h > 0.0f)) return 0u;
    if (h >= 65536.0f) return 65536u;
    return __float_as_uint(h + 8388608.0f) & 0x7FFFFFu;   // integer-valued h < 2^23
}
template <> __device__ __forceinline__ uint32_t cand_threshold<double>(double pnull)
{
    // lo(h) = (65536 h + 1/2) 2^-32 < p  <=>  h < (p 2^32 - 1/2) / 65536
    const double h = ceil((pnull * 4294967296.0 - 0.5) / 65536.0);
    return h <= 0.0 ? 0u : h >= 65536.0 ? 65536u : (uint32_t)h;
}

// Null-collision candidate count of the bijection pairing mode,
// floor(P_null N + U) with U = (w + 1/2) 2^-32 clamped to [0, N].  binary64
// takes the reference's products without contraction; binary32 stays off the
// narrow binary64 pipe (its count can differ from the binary64 one only when
// P_null N + U lies within a few binary32 ulps of an integer).
template <class T> __device__ __forceinline__ uint32_t cand_count(T pnull, uint32_t n, uint32_t w);
template <> __device__ __forceinline__ uint32_t cand_count<double>(double pnull, uint32_t n, uint32_t w)
{
    const double f = floor(__dadd_rn(__dmul_rn(pnull, (double)n), unif<double>(w)));
    return f <= 0.0 ? 0u : (f >= (double)n ? n : (uint32_t)f);
}
template <> __device__ __forceinline__ uint32_t cand_count<float>(float pnull, uint32_t n, uint32_t w)
{
    const float f = floorf(fmaf(pnull, (float)n, unif<float>(w)));
    return f <= 0.0f ? 0u : (f >= (float)n ? n : (uint32_t)f);
}

// Begins of the C ranges of a split (ltpc_index.h), kept in registers so that
// the owner of an item is found by C-1 compares instead of a division.
template <int C>
struct Bounds {
    uint32_t b[C];
    __device__ __forceinline__ void init_split(uint32_t total)
    {
#pragma unroll
        for (int r = 0; r < C; ++r) b[r] = split_begin((uint32_t)r, total, (uint32_t)C);
    }
    __device__ __forceinline__ void init_pos(uint32_t n)
    {
#pragma unroll
        for (int r = 0; r < C; ++r) b[r] = pos_begin((uint32_t)r, n, (uint32_t)C);
    }
    // owner = largest r with b[r] <= t; begin = b[owner]
    __device__ __forceinline__ uint32_t locate(uint32_t t, uint32_t& begin) const
    {
        uint32_t o = 0u, bg = b[0];
#pragma unroll
        for (int r = 1; r < C; ++r) {
            const bool ge = t >= b[r];
            o += ge ? 1u : 0u;
            bg = ge ? b[r] : bg;
        }
        begin = bg;
        return o;
    }
};

// Scalar k of the cell's record in the working precision: 0 = A, 1 = dt,
// 2..4 = mean velocity, 5 = K0, 6 = 1 / N_j (binary32 copies made with the
// record; binary64 as is).
template <class T> __device__ __forceinline__ T cell_scalar(const double* cp, int k);
template <> __device__ __forceinline__ float cell_scalar<float>(const double* cp, int k)
{
    return reinterpret_cast<const float*>(cp + CP_F32)[k];
}
template <> __device__ __forceinline__ double cell_scalar<double>(const double* cp, int k)
{
    return cp[k == 0 ? CP_A : k == 1 ? CP_DT : k < 5 ? CP_C + (k - 2) : k == 5 ? CP_K0 : CP_INVN];
}

// Shared-memory bytes a launch of the cell kernel needs (dynamic part).
template <class T>
__host__ __device__ constexpr size_t cells_dyn_smem(uint32_t capl)
{
    const size_t pair_b = (size_t)capl * (3 * sizeof(T) + 4 + 2) + 16;
    const size_t sort_b = (size_t)capl * 12 + ((size_t)capl + 2) * 4;
    const size_t m = pair_b > sort_b ? pair_b : sort_b;
    return (m + 15) & ~(size_t)15;
}

// Tracing: thread 0 of every CTA adds the SM cycles of each phase.
struct PhaseClock {
    unsigned long long* out;
    long long t;
    __device__ __forceinline__ void start() { if (out && threadIdx.x == 0) t = clock64(); }
    __device__ __forceinline__ void mark(int k)
    {
        if (out && threadIdx.x == 0) {
            const long long now = clock64();
            atomicAdd(out + k, (unsigned long long)(now - t));
            t = now;
        }
    }
};

template <class T, int C, int NT, int ITEMS>
__global__ void __launch_bounds__(NT, (NT <= 256 ? 2 : 1)) k_cells(CellArgs<T> a)
{
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
    static_assert(ITEMS % 2 == 0, "ITEMS must be even");
    constexpr uint32_t CAPL = (uint32_t)NT * ITEMS;
    static_assert(CAPL <= 65536u, "positions are packed in 16 bits");
    static_assert(CAPL / 32 <= NT, "one mask word per thread");
    constexpr int NW = NT / 32;
    constexpr int PER = (CAPL + 2 + NT - 1) / NT;   // bucket counters per thread in the scan

    extern __shared__ __align__(16) unsigned char smem[];
    // pair-phase view
    T* svx = reinterpret_cast<T*>(smem);
    T* svy = svx + CAPL;
    T* svz = svy + CAPL;
    uint32_t* sl = reinterpret_cast<uint32_t*>(svz + CAPL);
    // candidate words: by home index during the sort, by position afterwards;
    // 16 bytes past the sort view's bucket counters, so the sort never overlaps it
    uint16_t* sw = reinterpret_cast<uint16_t*>(reinterpret_cast<unsigned char*>(sl + CAPL) + 16);
    // bijection mode: the cell's six round functions as byte tables, in the space of
    // the candidate words, which only the key sort uses (2 B per position >= 1.5 KB)
    uint8_t (*const s_rt)[256] = reinterpret_cast<uint8_t (*)[256]>(sw);
    static_assert(CAPL * 2 >= 6 * 256, "round-function tables in the candidate-word space");
    // sort-phase view (aliases the pair-phase arrays); ekl holds {key, id} by
    // bucket position, so one 64-bit access moves an entry and one 64-bit
    // compare orders two entries by (key, id)
    uint32_t* stg = reinterpret_cast<uint32_t*>(smem);
    uint2* ekl = reinterpret_cast<uint2*>(stg + CAPL);
    uint32_t* bcnt = stg + 3 * CAPL;

    __shared__ uint32_t s_scan[NW + 1];
    __shared__ T s_redacc[NW * 8];
    __shared__ double s_cl[16];                      // two buffers, alternated between cluster reductions
    __shared__ double s_tot[8];
    __shared__ uint32_t s_hist[4 * NBIN];           // four sub-histograms (less atomic contention)
    __shared__ uint32_t s_cmask[CAPL / 32];         // candidate / work bit masks over local positions
    __shared__ uint32_t s_imask[CAPL / 32];         // ionizing positions
    __shared__ uint32_t s_dmask[CAPL / 32];         // positions of primaries removed by recombination
    __shared__ uint32_t s_ioff[CAPL / 32];          // ionizations before each mask word
    __shared__ uint32_t s_list[LISTCAP];
    __shared__ uint32_t s_misc[4];
    __shared__ T s_par[16];
    __shared__ uint4 s_item[2];
    __shared__ typename MaxBits<T>::U s_vmax;         // largest squared speed (bit pattern)                     // current / next work item {j, N_j, I_j, valid}
    __shared__ __align__(16) double s_cp[NCP];      // the cell's scalars of this pass (CP_* of CellParamArgs)

    const unsigned r = Cl<C>::rank();
    const unsigned tid = threadIdx.x;
    DevState* ds = a.ds;
    // exchange records (bijection mode, clusters): each cluster reuses its own C CAPL
    // records, which stay in L2, when the grid's share fits in the region (one record per
    // particle); otherwise a cell uses the records of its own index-list range
    const bool xg_own = (size_t)gridDim.x * CAPL <= (size_t)a.n_cap;
    const uint32_t xg_first = (uint32_t)(blockIdx.x - r) * CAPL;
    // deep exchange loads (staged or XGB in flight per thread) only where registers allow
    constexpr bool XG_DEEP = NT <= 512;
    constexpr int XGB = XG_DEEP ? 4 : 1;
    const uint32_t list_n = ds->class_n[a.cls];
    const uint32_t step = ds->step;
    const bool do_coul = (a.flags & F_COULOMB) != 0u;
    const bool do_neut = (a.flags & F_NEUTRAL) != 0u;
    const bool do_corr = (a.flags & F_CORRECTION) != 0u;
    const bool do_rec = (a.flags & F_RECOMB) != 0u;

    // Work items are taken one ahead: while a cell is processed, the next
    // ticket is drawn and its item copied into s_item asynchronously.
    if (r == 0 && tid == 0) {
        const uint32_t w = atomicAdd(&ds->ticket[a.cls], 1u);
        const uint4 it = w < list_n ? a.list[w] : make_uint4(0u, 0u, 0u, 0u);
        for (unsigned q = 0; q < (unsigned)C; ++q) *Cl<C>::at(&s_item[0], q) = it;
    }
    Cl<C>::sync();   // every CTA of the cluster is running before any remote access
    PhaseClock pc{a.phase_clk, 0};
    pc.start();
    uint32_t clb = 0u;                                // cluster reductions so far (buffer parity)

    for (uint32_t par = 0u;; par ^= 1u) {
        const uint4 item = s_item[par];
        if (item.w == 0u) break;
        const uint32_t j = item.x;
        const uint32_t n = item.y;
        const uint32_t s = item.z;
        uint32_t wnext = 0u;
        if (r == 0 && tid == 0) wnext = atomicAdd(&ds->ticket[a.cls], 1u);
        if (n == 0u || n > (uint32_t)C * CAPL) {          // uniform over the cluster
            if (r == 0 && tid == 0) {
                if (n != 0u) flag_error(ds, ERR_CELL_TOO_LARGE);
                const uint4 it = wnext < list_n ? a.list[wnext] : make_uint4(0u, 0u, 0u, 0u);
                for (unsigned q = 0; q < (unsigned)C; ++q) *Cl<C>::at(&s_item[par ^ 1u], q) = it;
            }
            Cl<C>::sync();
            continue;
        }
        if (tid == 0) {   // this cell's scalars, consumed after the gather's wait
            const double* cpj = a.cpar + (size_t)j * NCP;
#pragma unroll
            for (int q = 0; q < NCP / 2; ++q) cp_async<16>(&s_cp[2 * q], cpj + 2 * q);
        }
        // Buckets of the pairing-order sort.  A single CTA uses two buckets per
        // particle with 16-bit counters (two per word, in the space of one 32-bit
        // counter per particle), so that most particles are alone in their bucket
        // and take their position straight from the bucket scan; clusters use one
        // bucket per particle with 32-bit counters spread over the CTAs.
        constexpr bool SB = C == 1;
        const uint32_t nb = SB ? 2u * n : n_buckets(n);
        uint16_t* const b16 = reinterpret_cast<uint16_t*>(bcnt);
        const uint32_t hb = split_begin(r, n, C), nh = split_begin(r + 1, n, C) - hb;
        const uint32_t bb = split_begin(r, nb, C), nbl = split_begin(r + 1, nb, C) - bb;
        const uint32_t pb = pos_begin(r, n, C), pe = pos_end(r, n, C);
        const uint32_t nloc = pe > pb ? pe - pb : 0u;
        Bounds<C> PB, BB;            // pairing-position and bucket splits of this cell
        PB.init_pos(n);
        BB.init_split(nb);

        // the cell's bijection words (uniform over the cluster; bij_ab == 0: key sort)
        const uint32_t* bw = reinterpret_cast<const uint32_t*>(a.cpar + (size_t)j * NCP + CP_BIJ);
        const uint32_t bij_ab = __ldg(bw + CPB_AB);
        // this cell's exchange records (bijection mode, clusters)
        const uint32_t xgb = xg_own ? xg_first : s;

        // ---- 1a. zero this CTA's bucket counters (key sort) and histogram.  In the bijection
        // mode this cluster barrier also separates the previous cell's reads of the exchange
        // records from this cell's record stores.
        if (bij_ab == 0u) {
            for (uint32_t i = tid; i <= (SB ? n : nbl); i += NT) bcnt[i] = 0u;   // (SB: n + 1 words)
        }
        for (uint32_t i = tid; i < 4u * NBIN; i += NT) s_hist[i] = 0u;
        for (uint32_t i = tid; i < CAPL / 32u; i += NT) { s_imask[i] = 0u; s_dmask[i] = 0u; }
        if (tid == 0) s_vmax = 0u;
        Cl<C>::sync();

        pc.mark(0);
        // ---- 1b. home slice: particle ids (coalesced), pairing keys, bucket counts
        // Bijection pairing (the cell's record says so; uniform over the cluster):
        // the cell's index list is in ascending id order (storage grouped by cell),
        // so home index hb + k is the particle's id rank and its pairing position
        // is pi(hb + k) -- no keys, no sort.
        uint32_t hl[ITEMS], hp[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {   // all id loads in flight before their first use
            const uint32_t k = tid + (uint32_t)i * NT;
            hl[i] = k < nh ? __ldcs(a.perm + s + hb + k) : 0u;
            hp[i] = 0u;
        }
        uint32_t multi = 0u;           // items whose bucket holds several entries
        auto rt = [&](int i, uint32_t v) -> uint32_t { return s_rt[i][v]; };
        // the bijection's shape (its keys are in the tables), formed where it is used
        auto bij_shape_of = [&]() {
            BijParams B;
            B.n = n; B.a = bij_ab & 0xFFFFu; B.b = bij_ab >> 16; B.mb = __ldg(bw + CPB_MB);
            return B;
        };
        if (bij_ab != 0u) {
            const BijParams B = bij_shape_of();
            if constexpr (C > 1) {
                // the six round functions as byte tables (round i reads its input below b
                // for even i, a for odd i) for the pairing positions of the home particles;
                // the previous cell's readers passed several barriers
                for (uint32_t e = tid; e < 6u * 256u; e += NT) {
                    const uint32_t i = e >> 8, v = e & 255u;
                    const uint32_t m = (i & 1u) ? B.b : B.a, lim = (i & 1u) ? B.a : B.b;
                    if (v < lim) s_rt[i][v] = (uint8_t)bij_round(v, __ldg(bw + CPB_KEY + i), m);
                }
                __syncthreads();
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    const uint32_t k = tid + (uint32_t)i * NT;
                    uint32_t y = 0u;
                    if (k < nh) {
                        y = bij_enc_tab(B, rt, hb + k);
                        while (y >= n) y = bij_enc_tab(B, rt, y);
                    }
                    hp[i] = y;
                }
            } else {                   // (single CTAs: the rounds computed, no tables)
                BijParams K = B;
#pragma unroll
                for (int q = 0; q < 6; ++q) K.key[q] = __ldg(bw + CPB_KEY + q);
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    const uint32_t k = tid + (uint32_t)i * NT;
                    hp[i] = k < nh ? bij_forward(K, hb + k) : 0u;
                }
            }
            if (r == 0 && tid == 0) {   // the next work item, completed by the wait before phase 3
                if (wnext < list_n) cp_async<16>(&s_item[par ^ 1u], a.list + wnext);
                else s_item[par ^ 1u] = make_uint4(0u, 0u, 0u, 0u);
            }
            pc.mark(1); pc.mark(2); pc.mark(3);
        } else {
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t k = tid + (uint32_t)i * NT;
            hp[i] = 0u;
            if (k < nh) {
                const uint32_t l = hl[i];
                const uint4 rw = draw(a.keys, l, step, TAG_PARTICLE);
                const uint32_t b = __umulhi(rw.x, nb);
                uint32_t slot;
                if constexpr (SB) {
                    const uint32_t sh = (b & 1u) << 4;
                    slot = atomicAdd(bcnt + (b >> 1), 1u << sh) >> sh;
                } else {
                    uint32_t b0;
                    const uint32_t ro = BB.locate(b, b0);
                    slot = atomicAdd(Cl<C>::at(bcnt + (b - b0), ro), 1u);
                }
                stg[k] = rw.x;
                sw[k] = (uint16_t)(rw.y >> 16);
                hp[i] = (b << 16) | (slot & 0xFFFFu);
            }
        }
        if (r == 0 && tid == 0) {   // the next work item, completed by the wait before phase 3
            if (wnext < list_n) cp_async<16>(&s_item[par ^ 1u], a.list + wnext);
            else s_item[par ^ 1u] = make_uint4(0u, 0u, 0u, 0u);
        }
        Cl<C>::sync();

        pc.mark(1);
        // ---- 1c. bucket starts: local exclusive scan, then offset by lower CTAs' totals
        if constexpr (SB) {
            // words [0, n]: bucket 2w in the low half, 2w+1 in the high half; word n
            // has no particles, so its low half becomes the end sentinel n
            uint32_t cnt[PER];
            uint32_t sum = 0u;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const uint32_t bi = tid * PER + i;
                cnt[i] = bi <= n ? bcnt[bi] : 0u;
                sum += (cnt[i] & 0xFFFFu) + (cnt[i] >> 16);
            }
            uint32_t tot;
            uint32_t ex = block_excl_scan<NT>(sum, s_scan, &tot);
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const uint32_t bi = tid * PER + i;
                const uint32_t lo = cnt[i] & 0xFFFFu;
                if (bi <= n) bcnt[bi] = ex | ((ex + lo) << 16);
                ex += lo + (cnt[i] >> 16);
            }
        } else {
            uint32_t cnt[PER];
            uint32_t sum = 0u;
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const uint32_t bi = tid * PER + i;
                cnt[i] = bi < nbl ? bcnt[bi] : 0u;
                sum += cnt[i];
            }
            uint32_t tot;
            uint32_t ex = block_excl_scan<NT>(sum, s_scan, &tot);
            uint32_t base = 0u;
            if constexpr (C > 1) {
                if (tid == 0) s_misc[1] = tot;
                Cl<C>::sync();
                for (unsigned q = 0; q < r; ++q) base += *Cl<C>::at(&s_misc[1], q);
            }
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const uint32_t bi = tid * PER + i;
                if (bi < nbl) bcnt[bi] = base + ex;
                ex += cnt[i];
            }
            if (tid == 0) bcnt[nbl] = base + tot;   // start of the next CTA's first bucket
        }
        Cl<C>::sync();

        pc.mark(2);
        // ---- 1d. place (key, id) at bucket start + slot, in the position-owner CTA.
        // SB: a particle alone in its bucket has its final position already.
        if constexpr (SB) {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t k = tid + (uint32_t)i * NT;
                if (k < nh) {
                    const uint32_t b = hp[i] >> 16, slot = hp[i] & 0xFFFFu;
                    const uint32_t bs = b16[b], be = b16[b + 1];
                    if (bs + slot < be && be <= n) {
                        if (be - bs == 1u) {
                            hp[i] = bs | ((uint32_t)sw[k] << 16);
                        } else {
                            ekl[bs + slot] = make_uint2(stg[k], hl[i]);
                            multi |= 1u << i;
                        }
                    } else {
                        flag_error(ds, ERR_INDEX);
                        hp[i] = 0u;
                    }
                }
            }
        } else {
            // clusters: the bucket's start and end are read once here (remote);
            // a particle alone in its bucket is final, the others are placed and
            // keep (start, size) for the ranking, which then reads only entries
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t k = tid + (uint32_t)i * NT;
                if (k < nh) {
                    const uint32_t b = hp[i] >> 16, slot = hp[i] & 0xFFFFu;
                    uint32_t b0;
                    const uint32_t ro = BB.locate(b, b0);
                    const uint32_t* bc = Cl<C>::at(bcnt + (b - b0), ro);   // bc[1]: the next bucket's start
                    const uint32_t bs = bc[0], be = bc[1];
                    if (bs + slot < be && be <= n && be - bs < 65536u) {
                        if (be - bs == 1u) {
                            hp[i] = bs | ((uint32_t)sw[k] << 16);
                        } else {
                            const uint32_t gpos = bs + slot;
                            uint32_t p0;
                            const uint32_t po = PB.locate(gpos, p0);
                            *Cl<C>::at(ekl + (gpos - p0), po) = make_uint2(stg[k], hl[i]);
                            hp[i] = bs | ((be - bs) << 16);
                            multi |= 1u << i;
                        }
                    } else {
                        flag_error(ds, ERR_INDEX);
                        hp[i] = 0u;
                    }
                }
            }
        }
        Cl<C>::sync();

        pc.mark(3);
        // ---- 1e. each particle that shares its bucket ranks itself inside it:
        // its final pairing-order position is the bucket start plus the number of
        // entries of the bucket ordered before (key, id).  With half a particle
        // (single CTAs) or one particle (clusters) per bucket on average, almost
        // every shared bucket holds at most four entries: those are loaded and
        // compared together (independent loads, no divergent walk), and only the
        // rare larger buckets continue serially.
        auto entry = [&](uint32_t t) -> unsigned long long {
            uint32_t t0;
            const uint32_t o = PB.locate(t, t0);
            const uint2 e = *Cl<C>::at(ekl + (t - t0), o);
            return ((unsigned long long)e.x << 32) | e.y;
        };
        if constexpr (SB) {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (multi & (1u << i)) {
                    const uint32_t k = tid + (uint32_t)i * NT;
                    const unsigned long long me = ((unsigned long long)stg[k] << 32) | hl[i];
                    const uint32_t b = hp[i] >> 16;
                    const uint32_t bs = b16[b], be = b16[b + 1];   // checked in 1d: bs < be <= n
                    uint32_t rank = 0u;
#pragma unroll
                    for (uint32_t u = 0; u < 4u; ++u) {
                        if (bs + u < be) rank += entry(bs + u) < me ? 1u : 0u;
                    }
                    for (uint32_t t = bs + 4u; t < be; ++t) rank += entry(t) < me ? 1u : 0u;
                    hp[i] = (bs + rank) | ((uint32_t)sw[k] << 16);
                }
            }
        } else {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                if (multi & (1u << i)) {
                    const uint32_t k = tid + (uint32_t)i * NT;
                    const unsigned long long me = ((unsigned long long)stg[k] << 32) | hl[i];
                    const uint32_t bs = hp[i] & 0xFFFFu, be = bs + (hp[i] >> 16);   // checked in 1d
                    uint32_t rank = 0u;
#pragma unroll
                    for (uint32_t u = 0; u < 4u; ++u) {
                        if (bs + u < be) rank += entry(bs + u) < me ? 1u : 0u;
                    }
                    for (uint32_t t = bs + 4u; t < be; ++t) rank += entry(t) < me ? 1u : 0u;
                    hp[i] = (bs + rank) | ((uint32_t)sw[k] << 16);
                }
            }
        }
        Cl<C>::sync();
        }   // key sort

        pc.mark(4);
        pc.mark(5);
        // ---- 2. gather velocities (coalesced through the id list) into pairing order;
        // single-CTA classes copy them asynchronously, all in flight at once
        if constexpr (C == 1) {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t k = tid + (uint32_t)i * NT;
                if (k < nh) {
                    const uint32_t pos = hp[i] & 0xFFFFu, l = hl[i];
                    cp_async<sizeof(T)>(svx + pos, a.vx + l);
                    cp_async<sizeof(T)>(svy + pos, a.vy + l);
                    cp_async<sizeof(T)>(svz + pos, a.vz + l);
                    sl[pos] = l;
                    if (bij_ab == 0u) sw[pos] = (uint16_t)(hp[i] >> 16);
                    if (a.order_out) a.order_out[s + pos] = l;
                }
            }
            cp_async_wait_all();
        } else if (bij_ab != 0u) {
            // Bijection mode, clusters: every CTA sends its home particles' records
            // (velocity, id) to their pairing positions in the cell's exchange records, one
            // random 16-byte (binary64: 32-byte) store to L2 each; after the cluster barrier
            // below every CTA reads its own positions' records in order.  With 512 threads or
            // fewer (16 warps) the velocities are first staged in this CTA's slots (free until
            // then), all copies in flight at once; 32 warps hide the loads' latency anyway, and
            // their 64 registers leave no room for it.
            const uint32_t xb = xgb;
            if constexpr (XG_DEEP) {
#pragma unroll
                for (int i = 0; i < ITEMS; ++i) {
                    const uint32_t k = tid + (uint32_t)i * NT;
                    if (k < nh) {
                        const uint32_t l = hl[i];
                        cp_async<sizeof(T)>(svx + k, a.vx + l);
                        cp_async<sizeof(T)>(svy + k, a.vy + l);
                        cp_async<sizeof(T)>(svz + k, a.vz + l);
                    }
                }
                cp_async_wait_all();
            }
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t k = tid + (uint32_t)i * NT;
                if (k < nh) {
                    const uint32_t l = hl[i];
                    if constexpr (XG_DEEP) Xg<T>::put(a.xg, xb + hp[i], svx[k], svy[k], svz[k], l);
                    else Xg<T>::put(a.xg, xb + hp[i], a.vx[l], a.vy[l], a.vz[l], l);
                    if (a.order_out) a.order_out[s + hp[i]] = l;
                }
            }
            if (!XG_DEEP && tid == 0) cp_async_wait_all();
        } else {
            // key sort, clusters: the home CTA stores each particle's velocity, id and
            // candidate word into the position owner's shared memory
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t k = tid + (uint32_t)i * NT;
                if (k < nh) {
                    const uint32_t pos = hp[i] & 0xFFFFu, l = hl[i];
                    uint32_t p0;
                    const uint32_t o = PB.locate(pos, p0);
                    const uint32_t lp = pos - p0;
                    const T x = a.vx[l], y = a.vy[l], z = a.vz[l];
                    *Cl<C>::at(svx + lp, o) = x;
                    *Cl<C>::at(svy + lp, o) = y;
                    *Cl<C>::at(svz + lp, o) = z;
                    *Cl<C>::at(sl + lp, o) = l;
                    *Cl<C>::at(sw + lp, o) = (uint16_t)(hp[i] >> 16);
                    if (a.order_out) a.order_out[s + pos] = l;
                }
            }
            if (tid == 0) cp_async_wait_all();
        }
        // pairing positions of the home particles, two per register, for the write-back
        uint32_t hq[ITEMS / 2];
#pragma unroll
        for (int i = 0; i < ITEMS / 2; ++i) hq[i] = (hp[2 * i] & 0xFFFFu) | (hp[2 * i + 1] << 16);
        Cl<C>::sync();
        if constexpr (C > 1) {
            if (bij_ab != 0u) {   // this CTA's pairing positions, in order, from the exchange records
                const uint32_t xb = xgb + pb;
                for (uint32_t q0 = tid; q0 < nloc; q0 += (uint32_t)XGB * NT) {
                    T x[XGB], y[XGB], z[XGB];
                    uint32_t l[XGB];
#pragma unroll
                    for (int u = 0; u < XGB; ++u) {
                        const uint32_t q = q0 + (uint32_t)u * NT;
                        if (q < nloc) Xg<T>::get(a.xg, xb + q, x[u], y[u], z[u], l[u]);
                    }
#pragma unroll
                    for (int u = 0; u < XGB; ++u) {
                        const uint32_t q = q0 + (uint32_t)u * NT;
                        if (q < nloc) { svx[q] = x[u]; svy[q] = y[u]; svz[q] = z[u]; sl[q] = l[u]; }
                    }
                }
                __syncthreads();
            }
        }

        pc.mark(6);
        // The next cell's id list into L2 now, and its first particle id, from
        // which its velocity ranges are prefetched at the end of this cell.
        // Rank 0 only: its s_item[par ^ 1] is complete here (its own copy, waited
        // before the barrier above); the other CTAs of a cluster receive the
        // item only at the end of the iteration.
        uint32_t next_l0 = 0xFFFFFFFFu;
        if (r == 0 && tid == 32u) {
            const uint4 nx = s_item[par ^ 1u];
            if (nx.w != 0u && nx.y != 0u) {
                prefetch_l2(a.perm + nx.z, (size_t)nx.y * 4u);
                next_l0 = a.perm[nx.z];
            }
        }
        // ---- 3. step S1: Takizuka-Abe collisions of pairs (2p, 2p+1), then the
        // optional restoration of the cell's momentum and energy.  The largest
        // squared speed after S1 is tracked for the null-collision bound.
        T vmax2 = T(0);
        // the restoration's pass folded into the moments' (no neutral step: nothing changes
        // the velocities between them, and the largest speed is not needed)
        const bool rest_in_moments = do_coul && n >= 2u && do_corr && !do_neut;
        if (do_coul && n >= 2u) {
            // the cell's scalars in the working precision (A with lnL and dt, and the
            // restoration's state before S1, formed at the start of the pass from the
            // moments the previous pass left; K0 < 0 asks for the sums before S1 to be
            // formed here instead)
            const T A = cell_scalar<T>(s_cp, 0), cx = cell_scalar<T>(s_cp, 2), cy = cell_scalar<T>(s_cp, 3),
                    cz = cell_scalar<T>(s_cp, 4);
            const bool pre_mom = cell_scalar<T>(s_cp, 5) >= T(0);  // uniform over the cluster (same scalars)
            // Pair slot p holds positions 2p and 2p+1, so the pair's two particles sit
            // in the two lanes of one packed value: the update v_a += Du/2, v_b -= Du/2
            // and the sums are packed operations.  The restoration and the moments
            // below walk the same slots, so each thread rereads what it wrote.
            using P = Pk<T>;
            using V2 = typename P::V;
            const V2 C2x = P::make(-cx, -cx), C2y = P::make(-cy, -cy), C2z = P::make(-cz, -cz);
            V2 sx = P::make(T(0), T(0)), sy = sx, sz = sx, ss = sx;      // after S1 (centred)
            V2 bx0 = sx, by0 = sx, bz0 = sx, bs0 = sx;                    // before S1, if needed
            auto psum = [&](V2 X, V2 Y, V2 Z, V2& ax_, V2& ay_, V2& az_, V2& as_) {
                const V2 dx = P::add(X, C2x), dy = P::add(Y, C2y), dz = P::add(Z, C2z);
                P::acc(ax_, dx); P::acc(ay_, dy); P::acc(az_, dz);
                P::acc(as_, P::fma(dz, dz, P::fma(dy, dy, P::mul(dx, dx))));
            };
            const bool pre = do_corr && !pre_mom;
            const uint32_t nslot = (nloc + 1u) / 2u;
            const V2 H = P::make(T(0.5), T(-0.5));
            for (uint32_t p = tid; p < nslot; p += NT) {
                const uint32_t ia = 2u * p, ib = ia + 1u;   // pair slots are even-aligned: one vector access each
                V2 X = *reinterpret_cast<const V2*>(svx + ia);
                V2 Y = *reinterpret_cast<const V2*>(svy + ia);
                V2 Z = *reinterpret_cast<const V2*>(svz + ia);
                if (ib < nloc) {
                    const uint2 L2 = *reinterpret_cast<const uint2*>(sl + ia);
                    if (pre) psum(X, Y, Z, bx0, by0, bz0, bs0);
                    const uint4 w = draw(a.keys, L2.x < L2.y ? L2.x : L2.y, step, TAG_PAIR);
                    T dux, duy, duz;
                    ta_delta<T>(X.x, Y.x, Z.x, X.y, Y.y, Z.y, A, w, dux, duy, duz);
                    X = P::fma(H, P::make(dux, dux), X);
                    Y = P::fma(H, P::make(duy, duy), Y);
                    Z = P::fma(H, P::make(duz, duz), Z);
                    *reinterpret_cast<V2*>(svx + ia) = X;
                    *reinterpret_cast<V2*>(svy + ia) = Y;
                    *reinterpret_cast<V2*>(svz + ia) = Z;
                    if (do_corr) {
                        psum(X, Y, Z, sx, sy, sz, ss);
                    } else {
                        const V2 q2 = P::fma(Z, Z, P::fma(Y, Y, P::mul(X, X)));
                        vmax2 = fmax(vmax2, fmax(q2.x, q2.y));
                    }
                } else {                                      // the odd one out: unchanged
                    const V2 X1 = P::make(X.x, cx), Y1 = P::make(Y.x, cy), Z1 = P::make(Z.x, cz);
                    if (pre) psum(X1, Y1, Z1, bx0, by0, bz0, bs0);
                    if (do_corr) psum(X1, Y1, Z1, sx, sy, sz, ss);
                    else vmax2 = fmax(vmax2, X.x * X.x + Y.x * Y.x + Z.x * Z.x);
                }
            }
            if (do_corr) {
                // sums after S1 (0..3) and, without usable stored moments, before it (4..7)
                T acc[8] = {sx.x + sx.y, sy.x + sy.y, sz.x + sz.y, ss.x + ss.y,
                            bx0.x + bx0.y, by0.x + by0.y, bz0.x + bz0.y, bs0.x + bs0.y};
                if (pre_mom) {
                    T acc4[4] = {acc[0], acc[1], acc[2], acc[3]};
                    cluster_sum<NT, C, 4, T>(acc4, s_redacc, s_cl + 8u * (clb++ & 1u), s_tot);
                } else {
                    cluster_sum<NT, C, 8, T>(acc, s_redacc, s_cl + 8u * (clb++ & 1u), s_tot);
                }
                // x <- V0 + f (x - V1) = f x + (V0 - f V1), with V = c + S1 / n and
                // K = S2 - |S1|^2 / n.  The sums are double; the scalars are formed in
                // the working precision, which they scale (the centred sums keep
                // |S1|^2 / n small against S2, so no cancellation).  Thread 0 does
                // this alone while the CTA waits.
                if (tid == 0) {
                    const T inv_n = cell_scalar<T>(s_cp, 6);
                    T St[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) St[q] = (T)s_tot[q];
                    T K0, V0[3];
                    if (pre_mom) {
                        K0 = cell_scalar<T>(s_cp, 5);
                        V0[0] = cx; V0[1] = cy; V0[2] = cz;
                    } else {
                        K0 = St[7] - (St[4] * St[4] + St[5] * St[5] + St[6] * St[6]) * inv_n;
                        V0[0] = cx + St[4] * inv_n; V0[1] = cy + St[5] * inv_n; V0[2] = cz + St[6] * inv_n;
                    }
                    const T K1 = St[3] - (St[0] * St[0] + St[1] * St[1] + St[2] * St[2]) * inv_n;
                    const T f = (K1 > T(0) && K0 > T(0)) ? Math<T>::sqrt(K0 / K1) : T(1);
                    s_par[4] = f;
                    s_par[5] = V0[0] - f * (cx + St[0] * inv_n);
                    s_par[6] = V0[1] - f * (cy + St[1] * inv_n);
                    s_par[7] = V0[2] - f * (cz + St[2] * inv_n);
                }
                __syncthreads();
                const V2 F = P::make(s_par[4], s_par[4]);
                const V2 OX = P::make(s_par[5], s_par[5]), OY = P::make(s_par[6], s_par[6]),
                         OZ = P::make(s_par[7], s_par[7]);
                // without the neutral step the moments loop (step 5) applies the restoration
                // as it reads the slots: one pass instead of two
                if (!rest_in_moments)
                for (uint32_t p = tid; p < nslot; p += NT) {
                    const uint32_t ia = 2u * p;
                    const V2 X = P::fma(F, *reinterpret_cast<const V2*>(svx + ia), OX);
                    const V2 Y = P::fma(F, *reinterpret_cast<const V2*>(svy + ia), OY);
                    const V2 Z = P::fma(F, *reinterpret_cast<const V2*>(svz + ia), OZ);
                    const V2 q2 = P::fma(Z, Z, P::fma(Y, Y, P::mul(X, X)));
                    if (ia + 1u < nloc) {
                        *reinterpret_cast<V2*>(svx + ia) = X;
                        *reinterpret_cast<V2*>(svy + ia) = Y;
                        *reinterpret_cast<V2*>(svz + ia) = Z;
                        vmax2 = fmax(vmax2, fmax(q2.x, q2.y));
                    } else {
                        svx[ia] = X.x; svy[ia] = Y.x; svz[ia] = Z.x;
                        vmax2 = fmax(vmax2, q2.x);
                    }
                }
            }
            // A single CTA needs no barrier here: the next reads of these positions
            // are by the same threads (same pair slots), or the neutral step follows
            // (its first action is a barrier).
            if (C > 1 && !rest_in_moments) __syncthreads();
        } else if (do_neut) {
            for (uint32_t q = tid; q < nloc; q += NT) {
                const T x = svx[q], y = svy[q], z = svz[q];
                vmax2 = fmax(vmax2, x * x + y * y + z * z);
            }
        }

        pc.mark(7);
        // ---- 4. step S2a: null-collision electron-neutral sampling.  Possible
        // candidates (by the top 16 bits of the candidate word) are compacted
        // through a bit mask so that whole warps redraw and collide them.
        const uint32_t nw = (nloc + 31u) / 32u;
        uint32_t ion_base = 0u;      // secondaries of lower-ranked CTAs of this cell
        const T half_m_over_e = a.c_half_m_over_e;
        if (do_neut) {
            T numax, pnull;
            uint32_t hmin;
            const T dtj = cell_scalar<T>(s_cp, 1);
            auto bound = [&](T md, T& nmx, T& pn, uint32_t& h) {   // null-collision bound of the cell
                nmx = a.c_nsig_tot * Math<T>::sqrt(md);
                // per-particle selection (tables, key pairing): pi_el + pi_ion <=
                // dt v (sigma_el + sigma_ion) n_n <= nu_max dt, so U below that bound
                // (widened past rounding) screens every particle that can collide
                pn = a.xs.per_particle ? fmin(T(1), nmx * dtj * T(1.0001)) : -Math<T>::expm1(-nmx * dtj);
                h = cand_threshold<T>(pn);
            };
            if constexpr (C == 1) {
                // largest squared speed: warp butterfly, then one shared atomicMax on
                // the bit pattern (monotone for non-negative values), one barrier
                T v = vmax2;
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
                if ((tid & 31u) == 0u) atomicMax(&s_vmax, MaxBits<T>::to(v));
                __syncthreads();
                const T md = MaxBits<T>::from(s_vmax);
                if constexpr (sizeof(T) == 4) {
                    bound(md, numax, pnull, hmin);       // every thread, in binary32
                } else {
                    if (tid == 0) bound(md, s_par[11], s_par[12], s_misc[0]);
                    __syncthreads();
                    numax = s_par[11]; pnull = s_par[12]; hmin = s_misc[0];
                }
            } else {
                const T md = cluster_max<NT, C, T>(vmax2, s_redacc, s_cl + 8u * (clb++ & 1u));
                if (tid == 0) bound(md, s_par[11], s_par[12], s_misc[0]);
                __syncthreads();
                numax = s_par[11]; pnull = s_par[12]; hmin = s_misc[0];
            }
            const T nsel = a.c_nsig_el, nsion = a.c_nsig_ion;
            const T e_ion = a.c_e_ion, mr2 = a.c_mratio2;
            // Bijection pairing: the candidates are the particles at pairing positions
            // below n_c = floor(P_null N + U) (cand_count); otherwise each particle's own
            // uniform decides (U < P_null, its 16 top bits screened by hmin first).
            const uint32_t n_cand = bij_ab != 0u ? cand_count<T>(pnull, n, __ldg(bw + CPB_U)) : 0u;
            bool ionized = false;
            auto collide = [&](uint32_t q) {
                const uint32_t l = sl[q];
                const uint4 rw = draw(a.keys, l, step, TAG_PARTICLE);
                const T u1 = unif<T>(rw.y);
                if (bij_ab == 0u && !(u1 < pnull)) return;
                const T x = svx[q], y = svy[q], z = svz[q];
                const T v2 = x * x + y * y + z * z;
                const T v = Math<T>::sqrt(v2);
                const T E = v2 * half_m_over_e;
                bool el, io;
                if (!a.xs.on) {
                    const T nu_el = nsel * v;
                    const T nu_ion = E >= e_ion ? nsion * v : T(0);
                    const T rr = unif<T>(rw.z) * numax;
                    el = rr < nu_el;
                    io = !el && rr < nu_el + nu_ion;
                } else {
                    const T sg_el = xs_el<T>(a.xs, E, a.c_sig_el), sg_ion = xs_ion<T>(a.xs, E, a.c_sig_ion, e_ion);
                    if (a.xs.per_particle) {
                        // Sec. 4.2: pi_c = 1 - exp(-dt v sigma_c n_n), one uniform against
                        // pi_el, pi_el + pi_ion
                        const T pel = -Math<T>::expm1(-dtj * v * sg_el * a.c_nn);
                        const T pio = -Math<T>::expm1(-dtj * v * sg_ion * a.c_nn);
                        el = u1 < pel;
                        io = !el && u1 < pel + pio;
                    } else {
                        const T nu_el = a.c_nn * sg_el * v;
                        const T nu_ion = a.c_nn * sg_ion * v;
                        const T rr = unif<T>(rw.z) * numax;
                        el = rr < nu_el;
                        io = !el && rr < nu_el + nu_ion;
                    }
                }
                if (el) {                                      // C1: elastic, cold heavy target
                    const uint4 sc = draw(a.keys, l, step, TAG_SCATTER);
                    T dx, dy, dz;
                    iso_dir<T>(sc.x, sc.y, dx, dy, dz);
                    const T cchi = (x * dx + y * dy + z * dz) * Math<T>::rcp(v);
                    const T vn = v * Math<T>::sqrt(T(1) - mr2 * (T(1) - cchi));
                    svx[q] = vn * dx; svy[q] = vn * dy; svz[q] = vn * dz;
                } else if (io) {                               // C2: ionization, resolved below
                    atomicOr(&s_imask[q >> 5], 1u << (q & 31u));
                    ionized = true;
                }
            };
            // candidate bit mask over local positions, then block-wide compaction
            for (uint32_t q0 = 0; q0 < nloc; q0 += NT) {
                const uint32_t q = q0 + tid;
                const bool maybe = q < nloc && (bij_ab != 0u ? pb + q < n_cand : (uint32_t)sw[q] < hmin);
                const unsigned m = __ballot_sync(0xFFFFFFFFu, maybe);
                if ((tid & 31u) == 0u && q0 + tid < nloc + 31u) s_cmask[(q0 + tid) >> 5] = m;
            }
            __syncthreads();
            for_each_masked<NT>(s_cmask, nw, s_list, s_scan, collide);
            // ranks of this CTA's ionizations in position order, then across the cluster
            if constexpr (C == 1) {
                if (__syncthreads_or(ionized ? 1 : 0)) {
                    uint32_t tot;
                    const uint32_t wex = block_excl_scan<NT>(tid < nw ? (uint32_t)__popc(s_imask[tid]) : 0u, s_scan, &tot);
                    if (tid < nw) s_ioff[tid] = wex;
                    if (tid == 0) { s_misc[2] = tot; a.ion_count[j] = tot; s_misc[3] = tot; }
                } else if (tid == 0) {
                    s_misc[2] = 0u; a.ion_count[j] = 0u; s_misc[3] = 0u;
                }
                __syncthreads();
            } else {
                __syncthreads();
                uint32_t tot;
                const uint32_t wex = block_excl_scan<NT>(tid < nw ? (uint32_t)__popc(s_imask[tid]) : 0u, s_scan, &tot);
                if (tid < nw) s_ioff[tid] = wex;
                if (tid == 0) s_misc[2] = tot;
                Cl<C>::sync();
                uint32_t all = 0u;
                for (unsigned q = 0; q < (unsigned)C; ++q) {
                    const uint32_t t = *Cl<C>::at(&s_misc[2], q);
                    if (q < r) ion_base += t;
                    all += t;
                }
                if (r == 0 && tid == 0) { a.ion_count[j] = all; s_misc[3] = all; }
                Cl<C>::sync();
            }
        } else {
            if (tid == 0) s_misc[2] = 0u;
            if (r == 0 && tid == 0) {
                a.ion_count[j] = 0u;
                s_misc[3] = 0u;
            }
        }

        pc.mark(8);
        // ---- 5. ionization outcomes (C2), then the moments (S3a/S3b) of the cell
        {
            using M = Math<T>;
            using P = Pk<T>;
            using V2 = typename P::V;
            const T e_ion = a.c_e_ion, two_e_over_m = a.c_two_e_over_m;
            // per-thread sums, two lanes each (positions 2p and 2p+1 of the pair slots):
            // v_x, v_y, v_z, v_x^2, v_y^2, v_z^2, |v|, |v| above the ionization threshold
            // (with tabulated cross sections: sigma_el(E) |v| and sigma_ion(E) |v|)
            V2 q[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) q[k] = P::make(T(0), T(0));
            const bool xs_on = a.xs.on != 0;
            const T sg0 = a.c_sig_el, si0 = a.c_sig_ion;
            uint32_t* hsub = s_hist + ((tid >> 5) & 3u) * NBIN;
            const V2 HM = P::make(half_m_over_e, half_m_over_e);
            auto accum2 = [&](V2 X, V2 Y, V2 Z) {
                const V2 v2 = P::fma(Z, Z, P::fma(Y, Y, P::mul(X, X)));
                const V2 V = P::make(M::sqrt(v2.x), M::sqrt(v2.y));
                const V2 E = P::mul(v2, HM);
                P::acc(q[0], X); P::acc(q[1], Y); P::acc(q[2], Z);
                P::acc_sq(q[3], X); P::acc_sq(q[4], Y); P::acc_sq(q[5], Z);
                if (!xs_on) {
                    P::acc(q[6], V);
                    P::acc(q[7], P::make(E.x >= e_ion ? V.x : T(0), E.y >= e_ion ? V.y : T(0)));
                } else {                                       // tables: sums of sigma(E) |v|
                    P::acc(q[6], P::make(xs_el<T>(a.xs, E.x, sg0) * V.x, xs_el<T>(a.xs, E.y, sg0) * V.y));
                    P::acc(q[7], P::make(xs_ion<T>(a.xs, E.x, si0, e_ion) * V.x, xs_ion<T>(a.xs, E.y, si0, e_ion) * V.y));
                }
                atomicAdd(&hsub[M::ebin(E.x)], 1u);
                atomicAdd(&hsub[M::ebin(E.y)], 1u);
            };
            auto accum = [&](T x, T y, T z) {                  // one particle, into the first lane
                const T v2 = x * x + y * y + z * z;
                const T v = M::sqrt(v2);
                const T E = v2 * half_m_over_e;
                q[0].x += x; q[1].x += y; q[2].x += z;
                q[3].x += x * x; q[4].x += y * y; q[5].x += z * z;
                if (!xs_on) {
                    q[6].x += v;
                    q[7].x += E >= e_ion ? v : T(0);
                } else {
                    q[6].x += xs_el<T>(a.xs, E, sg0) * v;
                    q[7].x += xs_ion<T>(a.xs, E, si0, e_ion) * v;
                }
                atomicAdd(&hsub[M::ebin(E)], 1u);
            };
            if (do_neut && s_misc[2] > 0u) {
                for (uint32_t w = tid; w < nw; w += NT) s_cmask[w] = s_imask[w];
                __syncthreads();
                for_each_masked<NT>(s_cmask, nw, s_list, s_scan, [&](uint32_t q) {
                    const uint32_t l = sl[q];
                    const uint32_t rank = ion_base + s_ioff[q >> 5] + (uint32_t)__popc(s_imask[q >> 5] & ((1u << (q & 31u)) - 1u));
                    const T x = svx[q], y = svy[q], z = svz[q];
                    const T E = (x * x + y * y + z * z) * half_m_over_e;
                    const uint4 sc = draw(a.keys, l, step, TAG_SCATTER);
                    const uint4 sd = draw(a.keys, l, step, TAG_SECONDARY);
                    // E was >= e_ion when the collision was decided; recomputed here it can
                    // round one unit below, so the excess is clamped at zero (a negative
                    // excess would give a NaN speed)
                    const T Ep = fmax(E - e_ion, T(0));
                    const T Es = unif<T>(sc.z) * Ep;
                    const T vp = M::sqrt(two_e_over_m * (Ep - Es)), vs = M::sqrt(two_e_over_m * Es);
                    T dx, dy, dz, ex2, ey2, ez2;
                    iso_dir<T>(sc.x, sc.y, dx, dy, dz);
                    iso_dir<T>(sd.x, sd.y, ex2, ey2, ez2);
                    svx[q] = vp * dx; svy[q] = vp * dy; svz[q] = vp * dz;
                    const T sx = vs * ex2, sy = vs * ey2, sz = vs * ez2;
                    const uint32_t slot = s + rank;
                    a.stage_l[slot] = l;
                    a.stage_vx[slot] = sx; a.stage_vy[slot] = sy; a.stage_vz[slot] = sz;
                    accum(sx, sy, sz);
                });
                __syncthreads();   // the primaries' new velocities before the sums below
            }
            // ---- 5b. recombination C5 (Table 4): RS0, the n_rec primaries of the cell (formed
            // with its record) are its last pairing positions; RS1-RS3, the r-th takes the
            // catalyte n_rec positions before it; RS4, the catalyte takes both kinetic energies
            // and the released one in an isotropic direction (its RECOMB block); RS5, the
            // primary is removed (cell -1, out of the sums below).  Positions may belong to
            // other CTAs of a cluster; rank 0 serves every pair.
            uint32_t n_rec = 0u;
            if (do_rec && n >= 2u) n_rec = reinterpret_cast<const uint32_t*>(s_cp + CP_BIJ)[CPB_NREC];
            if (n_rec > 0u) {                                 // uniform over the cluster
                Cl<C>::sync();                                // every CTA's velocities after C1/C2
                if (r == 0) {
                    const T de = a.c_de_rec;
                    for (uint32_t rr = tid; rr < n_rec; rr += NT) {
                        const uint32_t qp = n - n_rec + rr, qc = n - 2u * n_rec + rr;
                        uint32_t b_p, b_c;
                        const uint32_t op = PB.locate(qp, b_p), oc = PB.locate(qc, b_c);
                        const uint32_t kp = qp - b_p, kc = qc - b_c;
                        const T px = *Cl<C>::at(svx + kp, op), py = *Cl<C>::at(svy + kp, op),
                                pz = *Cl<C>::at(svz + kp, op);
                        const T cx2 = *Cl<C>::at(svx + kc, oc), cy2 = *Cl<C>::at(svy + kc, oc),
                                cz2 = *Cl<C>::at(svz + kc, oc);
                        const uint32_t lp = *Cl<C>::at(sl + kp, op), lc = *Cl<C>::at(sl + kc, oc);
                        const T Ep = (px * px + py * py + pz * pz) * half_m_over_e;
                        const T Ec = (cx2 * cx2 + cy2 * cy2 + cz2 * cz2) * half_m_over_e;
                        const T sp = M::sqrt(two_e_over_m * (Ec + Ep + de));
                        const uint4 wr = draw(a.keys, lc, step, TAG_RECOMB);
                        T dx, dy, dz;
                        iso_dir<T>(wr.x, wr.y, dx, dy, dz);
                        *Cl<C>::at(svx + kc, oc) = sp * dx;
                        *Cl<C>::at(svy + kc, oc) = sp * dy;
                        *Cl<C>::at(svz + kc, oc) = sp * dz;
                        atomicOr(Cl<C>::at(&s_dmask[kp >> 5], op), 1u << (kp & 31u));
                        a.cell[lp] = -1;
                    }
                }
                Cl<C>::sync();
            }
            V2 RF = P::make(T(1), T(1)), RX = P::make(T(0), T(0)), RY = RX, RZ = RX;
            if (rest_in_moments) {
                RF = P::make(s_par[4], s_par[4]);
                RX = P::make(s_par[5], s_par[5]); RY = P::make(s_par[6], s_par[6]); RZ = P::make(s_par[7], s_par[7]);
            }
            for (uint32_t p = tid; 2u * p < nloc; p += NT) {
                const uint32_t ia = 2u * p;
                V2 X = *reinterpret_cast<const V2*>(svx + ia);
                V2 Y = *reinterpret_cast<const V2*>(svy + ia);
                V2 Z = *reinterpret_cast<const V2*>(svz + ia);
                if (rest_in_moments) {                        // the restoration, as in step 3
                    X = P::fma(RF, X, RX); Y = P::fma(RF, Y, RY); Z = P::fma(RF, Z, RZ);
                    if (ia + 1u < nloc) {
                        *reinterpret_cast<V2*>(svx + ia) = X;
                        *reinterpret_cast<V2*>(svy + ia) = Y;
                        *reinterpret_cast<V2*>(svz + ia) = Z;
                    } else {
                        svx[ia] = X.x; svy[ia] = Y.x; svz[ia] = Z.x;
                    }
                }
                if (n_rec == 0u) {
                    if (ia + 1u < nloc) accum2(X, Y, Z);
                    else accum(X.x, Y.x, Z.x);
                } else {                                      // skip the removed primaries
                    const bool live0 = !((s_dmask[ia >> 5] >> (ia & 31u)) & 1u);
                    const bool live1 = ia + 1u < nloc && !((s_dmask[(ia + 1u) >> 5] >> ((ia + 1u) & 31u)) & 1u);
                    if (live0 && live1) {
                        accum2(X, Y, Z);
                    } else {
                        if (live0) accum(X.x, Y.x, Z.x);
                        if (live1) accum(X.y, Y.y, Z.y);
                    }
                }
            }
            T acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = q[k].x + q[k].y;
            cluster_sum<NT, C, 8, T>(acc, s_redacc, s_cl + 8u * (clb++ & 1u), s_tot);
            if (r == 0 && tid < (unsigned)NBIN) {
                uint32_t h = 0u;
                for (unsigned q = 0; q < (unsigned)C; ++q) {
                    const uint32_t* hq = Cl<C>::at(s_hist, q);
                    h += hq[tid] + hq[NBIN + tid] + hq[2 * NBIN + tid] + hq[3 * NBIN + tid];
                }
                a.hist[(size_t)j * NBIN + tid] = h;
            }
            if (r == 0 && tid == 0) {
                a.rec_count[j] = n_rec;
                if (n_rec) atomicOr(&ds->ungroup, 1u);
                double* m = a.mom + (size_t)j * NMOM;
                const double N = (double)(n + s_misc[3] - n_rec);
                m[0] = N;
                m[1] = a.weight * N;
                m[2] = s_tot[0]; m[3] = s_tot[1]; m[4] = s_tot[2];
                m[5] = s_tot[3]; m[6] = s_tot[4]; m[7] = s_tot[5];
                m[8] = a.xs.on ? s_tot[6] : a.sigma_el * s_tot[6];
                m[9] = a.xs.on ? s_tot[7] : a.sigma_ion * s_tot[7];
            }
        }

        pc.mark(9);
        if (r == 0 && tid == 32u && next_l0 != 0xFFFFFFFFu) {   // cell-grouped storage: ids run from next_l0
            const uint4 nx = s_item[par ^ 1u];
            const uint32_t cnt = min(nx.y, a.n_cap - min(next_l0, a.n_cap));
            prefetch_l2(a.vx + next_l0, (size_t)cnt * sizeof(T));
            prefetch_l2(a.vy + next_l0, (size_t)cnt * sizeof(T));
            prefetch_l2(a.vz + next_l0, (size_t)cnt * sizeof(T));
        }
        // ---- 6. write velocities back.  A single CTA goes through its home
        // particles (coalesced global stores; ids and positions read back from
        // shared memory and registers).  A cluster CTA writes the positions it
        // owns straight to their ids: scattered global stores, which the L2
        // merges, cost far less than reading another CTA's shared memory at
        // random positions.
        if constexpr (C == 1) {
#pragma unroll
            for (int i = 0; i < ITEMS; ++i) {
                const uint32_t k = tid + (uint32_t)i * NT;
                if (k < nh) {
                    const uint32_t pos = (hq[i >> 1] >> (16 * (i & 1))) & 0xFFFFu;
                    const uint32_t l = sl[pos];
                    a.vx[l] = svx[pos];
                    a.vy[l] = svy[pos];
                    a.vz[l] = svz[pos];
                }
            }
        } else if (bij_ab != 0u) {
            // bijection mode: each position's record goes back to its home in the exchange
            // region (particles outside the cell's loaded run straight to their ids), and
            // after the cluster barrier every CTA writes its home slice in order
            const uint32_t rs = __ldg(a.run_start + j), rl = min(__ldg(a.run_len + j), n);
            for (uint32_t q = tid; q < nloc; q += NT) {
                const uint32_t l = sl[q], k = l - rs;
                if (k < rl) {
                    Xg<T>::put(a.xg, xgb + k, svx[q], svy[q], svz[q], l);
                } else {
                    a.vx[l] = svx[q];
                    a.vy[l] = svy[q];
                    a.vz[l] = svz[q];
                }
            }
            if (r == 0 && tid == 0) {        // the next item, before the barrier that publishes it
                const uint4 it = s_item[par ^ 1u];
                for (unsigned q = 1; q < (unsigned)C; ++q) *Cl<C>::at(&s_item[par ^ 1u], q) = it;
            }
            // This barrier also ends the cell for the cluster: the remote reads of the moments
            // step are done, and the next cell's record stores come after its first cluster
            // barrier (step 1a), when every CTA has read this cell's records.
            Cl<C>::sync();
            // (16 warps: XGB records per thread in flight before their stores, which the
            // compiler may not move above the next loads)
            const uint32_t he = min(hb + nh, rl), xb = xgb;
            for (uint32_t k0 = hb + tid; k0 < he; k0 += (uint32_t)XGB * NT) {
                T x[XGB], y[XGB], z[XGB];
                uint32_t l[XGB];
#pragma unroll
                for (int u = 0; u < XGB; ++u) {
                    const uint32_t k = k0 + (uint32_t)u * NT;
                    if (k < he) Xg<T>::get(a.xg, xb + k, x[u], y[u], z[u], l[u]);
                }
#pragma unroll
                for (int u = 0; u < XGB; ++u) {
                    const uint32_t k = k0 + (uint32_t)u * NT;
                    if (k < he) {
                        if (l[u] != rs + k) flag_error(ds, ERR_INDEX);
                        a.vx[rs + k] = x[u];
                        a.vy[rs + k] = y[u];
                        a.vz[rs + k] = z[u];
                    }
                }
            }
        } else {
            for (uint32_t q = tid; q < nloc; q += NT) {
                const uint32_t l = sl[q];
                a.vx[l] = svx[q];
                a.vy[l] = svy[q];
                a.vz[l] = svz[q];
            }
        }
        if constexpr (C > 1) {
            if (bij_ab == 0u && r == 0 && tid == 0) {
                const uint4 it = s_item[par ^ 1u];
                for (unsigned q = 1; q < (unsigned)C; ++q) *Cl<C>::at(&s_item[par ^ 1u], q) = it;
            }
        }
        if (C == 1 || bij_ab == 0u) Cl<C>::sync();
        else __syncthreads();
        pc.mark(10);
    }
}

}  // namespace ltpc
