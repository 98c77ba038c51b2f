// k_cells.cuh -- the fused per-cell collision kernel.
//
// One thread-block cluster of C CTAs processes one cell per work item
// (persistent loop, dynamic tickets).  Per cell it performs, on chip:
//   1. pairing order (Table 5, reading of "define partner pairs"): every
//      particle draws a key r_l; the cell's particles are sorted by (r_l, l)
//      with a bucket sort distributed over the cluster's shared memory;
//   2. step S1 (Table 2), the Takizuka-Abe collision of consecutive entries
//      (CCS4-CCS5 of Table 5), with per-cell sums before and after for the
//      optional momentum/energy restoration;
//   3. step S2a for electron-neutral collisions C1/C2 (Table 1) with the
//      null-collision method of Sec. 4.2, staging ionization secondaries
//      (Table 3, CS5) at a deterministic slot;
//   4. the particle-to-cell moments of steps S3a/S3b (Sec. 4.5) of the result.
// Velocities are read once from HBM (gathered through the cell's index list,
// CCS3) and written once.  Index math is in ltpc_index.h.
#pragma once
#include <cooperative_groups.h>

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

template <class T> __device__ __forceinline__ void sincospi_t(T x, T* s, T* c);
template <> __device__ __forceinline__ void sincospi_t<float>(float x, float* s, float* c) { sincospif(x, s, c); }
template <> __device__ __forceinline__ void sincospi_t<double>(double x, double* s, double* c) { sincospi(x, s, c); }

// Takizuka-Abe binary collision of an equal-mass pair (a, b); A is the cell
// coefficient so that <delta^2> = A / |u|^3; w holds the pair's three uniforms.
template <class T>
__device__ __forceinline__ void ta_collide(T& ax, T& ay, T& az, T& bx, T& by, T& bz, T A, uint4 w)
{
    const T ux = ax - bx, uy = ay - by, uz = az - bz;
    const T up2 = ux * ux + uy * uy;
    const T usq = up2 + uz * uz;
    if (usq == T(0)) return;
    const T u = sqrt(usq);
    const T var = A / (usq * u);
    T sth, cth, sph, cph;
    sincospi_t<T>(T(2) * unif<T>(w.y), &sth, &cth);
    sincospi_t<T>(T(2) * unif<T>(w.z), &sph, &cph);
    const T delta = sqrt(var * (T(-2) * log(unif<T>(w.x)))) * cth;
    T sin_t, omc_t;
    if (fabs(delta) <= T(1)) {
        const T d2 = delta * delta;
        const T rr = T(1) / (T(1) + d2);
        sin_t = T(2) * delta * rr;
        omc_t = T(2) * d2 * rr;
    } else {
        const T t = T(1) / delta;
        const T rr = T(1) / (T(1) + t * t);
        sin_t = T(2) * t * rr;
        omc_t = T(2) * rr;
    }
    T dux, duy, duz;
    if (up2 > T(0)) {
        const T uperp = sqrt(up2);
        const T ip = T(1) / uperp;
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
    const T h = T(0.5);
    ax += h * dux; ay += h * duy; az += h * duz;
    bx -= h * dux; by -= h * duy; bz -= h * duz;
}

// Isotropic unit vector from two uniforms: cos(theta) = 1 - 2 U_a, phi = 2 pi U_b.
template <class T>
__device__ __forceinline__ void iso_dir(uint32_t wa, uint32_t wb, T& dx, T& dy, T& dz)
{
    const T c = T(1) - T(2) * unif<T>(wa);
    const T s = sqrt(fmax(T(0), T(1) - c * c));
    T sp, cp;
    sincospi_t<T>(T(2) * unif<T>(wb), &sp, &cp);
    dx = s * cp; dy = s * sp; dz = c;
}

template <class T> __device__ __forceinline__ int energy_bin(T E)
{
    if (!(E > T(0))) return 0;
    const T t = (log10(E) + T(2)) * T(12.8);
    if (t < T(0)) return 0;
    if (t >= T(63)) return 63;
    return (int)t;
}

template <int NT>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_scan, uint32_t* total)
{
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31u) s_scan[warp] = x;
    __syncthreads();
    if (warp == 0) {
        uint32_t wv = lane < NT / 32 ? s_scan[lane] : 0u;
        uint32_t z = wv;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= (unsigned)o) z += y;
        }
        if (lane < NT / 32) s_scan[lane] = z - wv;
        if (lane == NT / 32 - 1) s_scan[NT / 32] = z;
    }
    __syncthreads();
    const uint32_t res = s_scan[warp] + x - v;
    *total = s_scan[NT / 32];
    __syncthreads();
    return res;
}

// Sum NQ per-thread partials over the cluster in a fixed order: warp
// butterfly (accumulator type) -> warps in order (double) -> CTAs in rank order.
template <int NT, int C, int NQ, class A>
__device__ __forceinline__ void cluster_sum(A (&v)[NQ], A* s_red, double* s_cl, double* out)
{
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < NQ; ++k) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xFFFFFFFFu, v[k], o);
    }
    if (lane == 0) {
#pragma unroll
        for (int k = 0; k < NQ; ++k) s_red[warp * NQ + k] = v[k];
    }
    __syncthreads();
    if (threadIdx.x < (unsigned)NQ) {
        double acc = 0.0;
        for (int w = 0; w < NT / 32; ++w) acc += (double)s_red[w * NQ + threadIdx.x];
        s_cl[threadIdx.x] = acc;
    }
    Cl<C>::sync();
    if (threadIdx.x < (unsigned)NQ) {
        double acc = 0.0;
        for (unsigned q = 0; q < (unsigned)C; ++q) acc += *Cl<C>::at(&s_cl[threadIdx.x], q);
        out[threadIdx.x] = acc;
    }
    Cl<C>::sync();
}

template <int NT, int C>
__device__ __forceinline__ double cluster_max_d(double v, double* s_red, double* s_cl)
{
    const unsigned lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, o));
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double m = 0.0;
        for (int w = 0; w < NT / 32; ++w) m = fmax(m, s_red[w]);
        s_cl[0] = m;
    }
    Cl<C>::sync();
    double m = 0.0;
    for (unsigned q = 0; q < (unsigned)C; ++q) m = fmax(m, *Cl<C>::at(&s_cl[0], q));
    Cl<C>::sync();
    return m;
}

__device__ __forceinline__ void flag_error(DevState* ds, uint32_t bit) { atomicOr(&ds->err, bit); }

// Shared-memory bytes a launch of the cell kernel needs (dynamic part).
template <class T>
__host__ __device__ constexpr size_t cells_dyn_smem(uint32_t capl)
{
    const size_t pair_b = (size_t)capl * (3 * sizeof(T) + 4 + 2);
    const size_t sort_b = (size_t)capl * 16 + ((size_t)capl / 4 + 2) * 4;
    const size_t m = pair_b > sort_b ? pair_b : sort_b;
    return (m + 15) & ~(size_t)15;
}

template <class T, int C, int NT, int ITEMS>
__global__ void __launch_bounds__(NT) k_cells(CellArgs<T> a)
{
    static_assert(NT % 32 == 0 && NT <= 1024, "block size");
    static_assert(ITEMS % 2 == 0, "ITEMS must be even");
    constexpr uint32_t CAPL = (uint32_t)NT * ITEMS;
    static_assert(CAPL <= 65536u, "positions are packed in 16 bits");
    constexpr int NW = NT / 32;
    constexpr int PER = (CAPL / 4 + 2 + NT - 1) / NT;   // bucket counters per thread in the scan

    extern __shared__ __align__(16) unsigned char smem[];
    // pair-phase view
    T* svx = reinterpret_cast<T*>(smem);
    T* svy = svx + CAPL;
    T* svz = svy + CAPL;
    uint32_t* sl = reinterpret_cast<uint32_t*>(svz + CAPL);
    uint16_t* sw = reinterpret_cast<uint16_t*>(sl + CAPL);
    // sort-phase view (aliases the pair-phase arrays)
    uint32_t* stg = reinterpret_cast<uint32_t*>(smem);
    uint32_t* ekey = stg + CAPL;
    uint32_t* el = ekey + CAPL;
    uint32_t* epos = el + CAPL;
    uint32_t* bcnt = epos + CAPL;

    __shared__ uint32_t s_scan[NW + 1];
    __shared__ T s_redacc[NW * 8];
    __shared__ double s_redd[NW];
    __shared__ double s_cl[8];
    __shared__ double s_tot[8];
    __shared__ uint32_t s_hist[NBIN];
    __shared__ uint32_t s_misc[4];

    const unsigned r = Cl<C>::rank();
    const unsigned tid = threadIdx.x;
    DevState* ds = a.ds;
    const uint32_t list_n = ds->class_n[a.cls];
    const uint32_t step = ds->step;
    const double dt = ds->dt;
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const bool do_coul = (a.flags & F_COULOMB) != 0u;
    const bool do_neut = (a.flags & F_NEUTRAL) != 0u;
    const bool do_corr = (a.flags & F_CORRECTION) != 0u;

    Cl<C>::sync();   // every CTA of the cluster is running before any remote access

    for (;;) {
        if (r == 0 && tid == 0) {
            const uint32_t w = atomicAdd(&ds->ticket[a.cls], 1u);
            for (unsigned q = 0; q < (unsigned)C; ++q) *Cl<C>::at(&s_misc[0], q) = w;
        }
        Cl<C>::sync();
        const uint32_t witem = s_misc[0];
        if (witem >= list_n) break;
        const uint32_t j = a.list[witem];
        const uint32_t n = a.counts[j];
        const uint32_t s = a.cell_start[j];
        if (n == 0u || n > (uint32_t)C * CAPL) {          // uniform over the cluster
            if (n != 0u && r == 0 && tid == 0) flag_error(ds, ERR_CELL_TOO_LARGE);
            Cl<C>::sync();
            continue;
        }
        const uint32_t nb = n_buckets(n);
        const uint32_t hb = split_begin(r, n, C), nh = split_begin(r + 1, n, C) - hb;
        const uint32_t bb = split_begin(r, nb, C), nbl = split_begin(r + 1, nb, C) - bb;
        const uint32_t pb = pos_begin(r, n, C), pe = pos_end(r, n, C);
        const uint32_t nloc = pe > pb ? pe - pb : 0u;

        // ---- 1a. zero this CTA's bucket counters and histogram
        for (uint32_t i = tid; i <= nbl; i += NT) bcnt[i] = 0u;
        if (tid < (unsigned)NBIN) s_hist[tid] = 0u;
        Cl<C>::sync();

        // ---- 1b. home slice: particle ids (coalesced), pairing keys, bucket counts
        uint32_t hl[ITEMS], hp[ITEMS], hw[ITEMS];
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t k = tid + (uint32_t)i * NT;
            hl[i] = 0u; hp[i] = 0u; hw[i] = 0u;
            if (k < nh) {
                const uint32_t l = a.perm[s + hb + k];
                const uint4 rw = draw(k0, k1, l, step, TAG_PARTICLE);
                const uint32_t b = __umulhi(rw.x, nb);
                const uint32_t ro = split_owner(b, nb, C);
                const uint32_t bi = b - split_begin(ro, nb, C);
                const uint32_t slot = atomicAdd(Cl<C>::at(bcnt + bi, ro), 1u);
                stg[k] = rw.x;
                hl[i] = l;
                hp[i] = (b << 16) | (slot & 0xFFFFu);
                hw[i] = rw.y >> 16;
            }
        }
        Cl<C>::sync();

        // ---- 1c. bucket starts: local exclusive scan, then offset by lower CTAs' totals
        {
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
            if (tid == 0) s_misc[1] = tot;
            Cl<C>::sync();
            uint32_t base = 0u;
            for (unsigned q = 0; q < r; ++q) base += *Cl<C>::at(&s_misc[1], q);
#pragma unroll
            for (int i = 0; i < PER; ++i) {
                const uint32_t bi = tid * PER + i;
                if (bi < nbl) bcnt[bi] = base + ex;
                ex += cnt[i];
            }
            if (tid == 0) bcnt[nbl] = base + tot;   // start of the next CTA's first bucket
        }
        Cl<C>::sync();

        // ---- 1d. place (key, id) at bucket start + slot, in the position-owner CTA
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t k = tid + (uint32_t)i * NT;
            if (k < nh) {
                const uint32_t b = hp[i] >> 16, slot = hp[i] & 0xFFFFu;
                const uint32_t ro = split_owner(b, nb, C);
                const uint32_t gpos = *Cl<C>::at(bcnt + (b - split_begin(ro, nb, C)), ro) + slot;
                if (gpos < n) {
                    const uint32_t po = pos_owner(gpos, n, C);
                    const uint32_t lp = gpos - pos_begin(po, n, C);
                    *Cl<C>::at(ekey + lp, po) = stg[k];
                    *Cl<C>::at(el + lp, po) = hl[i];
                } else {
                    flag_error(ds, ERR_INDEX);
                }
                hp[i] = gpos;
            }
        }
        Cl<C>::sync();

        // ---- 1e. rank inside the bucket -> final pairing-order position
        for (uint32_t q = tid; q < nloc; q += NT) {
            const uint32_t key = ekey[q], l = el[q];
            const uint32_t b = __umulhi(key, nb);
            const uint32_t ro = split_owner(b, nb, C);
            const uint32_t* bc = Cl<C>::at(bcnt + (b - split_begin(ro, nb, C)), ro);
            const uint32_t bs = bc[0], be = bc[1];
            uint32_t rank = 0u;
            if (bs <= be && be <= n) {
                for (uint32_t t = bs; t < be; ++t) {
                    const uint32_t o = pos_owner(t, n, C);
                    const uint32_t lt = t - pos_begin(o, n, C);
                    const uint32_t kk = *Cl<C>::at(ekey + lt, o);
                    const uint32_t ll = *Cl<C>::at(el + lt, o);
                    rank += (kk < key) || (kk == key && ll < l);
                }
            } else {
                flag_error(ds, ERR_INDEX);
            }
            epos[q] = bs + rank;
        }
        Cl<C>::sync();

        // ---- 1f. home slice learns each particle's pairing-order position
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t k = tid + (uint32_t)i * NT;
            if (k < nh) {
                const uint32_t gpos = hp[i] < n ? hp[i] : 0u;
                const uint32_t o = pos_owner(gpos, n, C);
                uint32_t pos = *Cl<C>::at(epos + (gpos - pos_begin(o, n, C)), o);
                if (pos >= n) { flag_error(ds, ERR_INDEX); pos = 0u; }
                hp[i] = pos | (hw[i] << 16);
            }
        }
        Cl<C>::sync();

        // ---- 2. gather velocities (coalesced through the id list) into pairing order
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t k = tid + (uint32_t)i * NT;
            if (k < nh) {
                const uint32_t pos = hp[i] & 0xFFFFu, l = hl[i];
                const uint32_t o = pos_owner(pos, n, C);
                const uint32_t lp = pos - pos_begin(o, n, C);
                const T x = a.vx[l], y = a.vy[l], z = a.vz[l];
                *Cl<C>::at(svx + lp, o) = x;
                *Cl<C>::at(svy + lp, o) = y;
                *Cl<C>::at(svz + lp, o) = z;
                *Cl<C>::at(sl + lp, o) = l;
                *Cl<C>::at(sw + lp, o) = (uint16_t)(hp[i] >> 16);
                if (a.order_out) a.order_out[s + pos] = l;
            }
        }
        Cl<C>::sync();

        const double dtj = dt * a.dt_factor[j];
        // ---- 3. step S1: Takizuka-Abe collisions of pairs (2p, 2p+1)
        if (do_coul && n >= 2u) {
            double lnl = a.lnlam[j];
            if (a.flags & F_LNL_NRL) {
                const double* m = a.mom + (size_t)j * NMOM;
                const double N = m[0];
                lnl = 2.0;
                if (N >= 2.0) {
                    const double mx = m[2] / N, my = m[3] / N, mz = m[4] / N;
                    const double msq = (m[5] + m[6] + m[7]) / N;
                    const double TeV = a.mass * (msq - (mx * mx + my * my + mz * mz)) / 3.0 / (a.mass * a.e_over_m);
                    const double nm3 = a.weight * (double)n * a.inv_vol[j];
                    if (TeV > 0.0 && nm3 > 0.0) {
                        const double lt = log(TeV);
                        const double v = 23.5 - log(sqrt(nm3 * 1e-6) * pow(TeV, -1.25)) -
                                         sqrt(1e-5 + (lt - 2.0) * (lt - 2.0) / 16.0);
                        lnl = v < 2.0 ? 2.0 : v;
                    }
                }
            }
            const T A = (T)(a.coef0 * (double)n * a.inv_vol[j] * lnl * dtj);
            // Centring shift for the restoration sums: the cell's mean velocity at
            // the end of the previous pass (a value no CTA modifies in this pass).
            T cx = T(0), cy = T(0), cz = T(0);
            if (do_corr) {
                const double* m = a.mom + (size_t)j * NMOM;
                if (m[0] > 0.0) { cx = (T)(m[2] / m[0]); cy = (T)(m[3] / m[0]); cz = (T)(m[4] / m[0]); }
            }
            T acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = T(0);
            const uint32_t nslot = (nloc + 1u) / 2u;
            for (uint32_t p = tid; p < nslot; p += NT) {
                const uint32_t ia = 2u * p, ib = ia + 1u;
                T ax = svx[ia], ay = svy[ia], az = svz[ia];
                if (do_corr) {
                    const T dx = ax - cx, dy = ay - cy, dz = az - cz;
                    acc[0] += dx; acc[1] += dy; acc[2] += dz; acc[3] += dx * dx + dy * dy + dz * dz;
                }
                if (ib < nloc) {
                    T bx = svx[ib], by = svy[ib], bz = svz[ib];
                    if (do_corr) {
                        const T dx = bx - cx, dy = by - cy, dz = bz - cz;
                        acc[0] += dx; acc[1] += dy; acc[2] += dz; acc[3] += dx * dx + dy * dy + dz * dz;
                    }
                    const uint32_t la = sl[ia], lb = sl[ib];
                    const uint4 w = draw(k0, k1, la < lb ? la : lb, step, TAG_PAIR);
                    ta_collide<T>(ax, ay, az, bx, by, bz, A, w);
                    svx[ia] = ax; svy[ia] = ay; svz[ia] = az;
                    svx[ib] = bx; svy[ib] = by; svz[ib] = bz;
                    if (do_corr) {
                        const T dx = bx - cx, dy = by - cy, dz = bz - cz;
                        acc[4] += dx; acc[5] += dy; acc[6] += dz; acc[7] += dx * dx + dy * dy + dz * dz;
                    }
                }
                if (do_corr) {
                    const T dx = ax - cx, dy = ay - cy, dz = az - cz;
                    acc[4] += dx; acc[5] += dy; acc[6] += dz; acc[7] += dx * dx + dy * dy + dz * dz;
                }
            }
            if (do_corr) {
                cluster_sum<NT, C, 8, T>(acc, s_redacc, s_cl, s_tot);
                // V = c + S1 / n and K = S2 - |S1|^2 / n, before (0..3) and after (4..7)
                const double nn = (double)n;
                const double K0 = s_tot[3] - (s_tot[0] * s_tot[0] + s_tot[1] * s_tot[1] + s_tot[2] * s_tot[2]) / nn;
                const double K1 = s_tot[7] - (s_tot[4] * s_tot[4] + s_tot[5] * s_tot[5] + s_tot[6] * s_tot[6]) / nn;
                const double f = (K1 > 0.0 && K0 > 0.0) ? sqrt(K0 / K1) : 1.0;
                const T V0x = (T)((double)cx + s_tot[0] / nn), V0y = (T)((double)cy + s_tot[1] / nn),
                        V0z = (T)((double)cz + s_tot[2] / nn);
                const T V1x = (T)((double)cx + s_tot[4] / nn), V1y = (T)((double)cy + s_tot[5] / nn),
                        V1z = (T)((double)cz + s_tot[6] / nn);
                const T ft = (T)f;
                for (uint32_t q = tid; q < nloc; q += NT) {
                    svx[q] = V0x + ft * (svx[q] - V1x);
                    svy[q] = V0y + ft * (svy[q] - V1y);
                    svz[q] = V0z + ft * (svz[q] - V1z);
                }
            }
            __syncthreads();
        }

        // ---- 4. step S2a: null-collision electron-neutral sampling.  Positions are
        // visited in thread-contiguous chunks, so a block scan over threads ranks
        // ionizations in pairing-order position.
        const uint32_t chunk = (nloc + NT - 1u) / NT;
        const uint32_t c0 = tid * chunk < nloc ? tid * chunk : nloc;
        const uint32_t c1 = c0 + chunk < nloc ? c0 + chunk : nloc;
        uint32_t ion_base = 0u;
        if (do_neut) {
            double md = 0.0;   // largest squared speed in the working precision (exact in double)
            for (uint32_t q = tid; q < nloc; q += NT) {
                const T x = svx[q], y = svy[q], z = svz[q];
                md = fmax(md, (double)(x * x + y * y + z * z));
            }
            md = cluster_max_d<NT, C>(md, s_redd, s_cl);
            const double nmx = a.n_neutral * (a.sigma_el + a.sigma_ion) * sqrt(md);
            const T numax = (T)nmx;
            const T pnull = (T)(-expm1(-nmx * dtj));
            const T e_over_m = (T)a.e_over_m, e_ion = (T)a.e_ion;
            const T nsel = (T)(a.n_neutral * a.sigma_el), nsion = (T)(a.n_neutral * a.sigma_ion);
            uint32_t nion = 0u;
            for (uint32_t q = c0; q < c1; ++q) {
                T lo, up;
                unif_hi16_range<T>((uint32_t)sw[q], lo, up);
                uint16_t flag = 0;
                if (lo < pnull) {                      // the candidate test may pass: redraw fully
                    const uint32_t l = sl[q];
                    const uint4 rw = draw(k0, k1, l, step, TAG_PARTICLE);
                    if (unif<T>(rw.y) < pnull) {
                        const T x = svx[q], y = svy[q], z = svz[q];
                        const T v2 = x * x + y * y + z * z;
                        const T v = sqrt(v2);
                        const T E = T(0.5) * v2 / e_over_m;
                        const T nu_el = nsel * v;
                        const T nu_ion = E >= e_ion ? nsion * v : T(0);
                        const T rr = unif<T>(rw.z) * numax;
                        if (rr < nu_el) {                  // C1: elastic, cold heavy target
                            const uint4 sc = draw(k0, k1, l, step, TAG_SCATTER);
                            T dx, dy, dz;
                            iso_dir<T>(sc.x, sc.y, dx, dy, dz);
                            const T cchi = (x * dx + y * dy + z * dz) / v;
                            const T vn = v * sqrt(T(1) - (T)a.mratio2 * (T(1) - cchi));
                            svx[q] = vn * dx; svy[q] = vn * dy; svz[q] = vn * dz;
                        } else if (rr < nu_el + nu_ion) {  // C2: ionization, resolved below
                            flag = 1;
                            ++nion;
                        }
                    }
                }
                sw[q] = flag;
            }
            uint32_t tot;
            const uint32_t ex = block_excl_scan<NT>(nion, s_scan, &tot);
            if (tid == 0) s_misc[2] = tot;
            Cl<C>::sync();
            uint32_t base = 0u, all = 0u;
            for (unsigned q = 0; q < (unsigned)C; ++q) {
                const uint32_t t = *Cl<C>::at(&s_misc[2], q);
                if (q < r) base += t;
                all += t;
            }
            ion_base = base + ex;
            if (r == 0 && tid == 0) a.ion_count[j] = all;
            Cl<C>::sync();
        } else if (r == 0 && tid == 0) {
            a.ion_count[j] = 0u;
        }

        // ---- 5. ionization outcomes, then the moments of the cell after the step
        {
            const T e_over_m = (T)a.e_over_m, e_ion = (T)a.e_ion;
            T acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = T(0);
            auto accum = [&](T x, T y, T z) {
                const T v2 = x * x + y * y + z * z;
                const T v = sqrt(v2);
                const T E = T(0.5) * v2 / e_over_m;
                acc[0] += x; acc[1] += y; acc[2] += z;
                acc[3] += x * x; acc[4] += y * y; acc[5] += z * z;
                acc[6] += v;
                acc[7] += E >= e_ion ? v : T(0);
                atomicAdd(&s_hist[energy_bin<T>(E)], 1u);
            };
            uint32_t nsec = 0u;
            for (uint32_t q = c0; q < c1; ++q) {
                T x = svx[q], y = svy[q], z = svz[q];
                if (do_neut && sw[q] == 1) {
                    const uint32_t l = sl[q];
                    const T E = T(0.5) * (x * x + y * y + z * z) / e_over_m;
                    const uint4 sc = draw(k0, k1, l, step, TAG_SCATTER);
                    const uint4 sd = draw(k0, k1, l, step, TAG_SECONDARY);
                    const T Ep = E - e_ion;
                    const T Es = unif<T>(sc.z) * Ep;
                    const T vp = sqrt(T(2) * (Ep - Es) * e_over_m), vs = sqrt(T(2) * Es * e_over_m);
                    T dx, dy, dz, ex2, ey2, ez2;
                    iso_dir<T>(sc.x, sc.y, dx, dy, dz);
                    iso_dir<T>(sd.x, sd.y, ex2, ey2, ez2);
                    x = vp * dx; y = vp * dy; z = vp * dz;
                    svx[q] = x; svy[q] = y; svz[q] = z;
                    const T sx = vs * ex2, sy = vs * ey2, sz = vs * ez2;
                    const uint32_t slot = s + ion_base + nsec;
                    ++nsec;
                    a.stage_l[slot] = l;
                    a.stage_vx[slot] = sx; a.stage_vy[slot] = sy; a.stage_vz[slot] = sz;
                    accum(sx, sy, sz);
                }
                accum(x, y, z);
            }
            cluster_sum<NT, C, 8, T>(acc, s_redacc, s_cl, s_tot);
            if (r == 0 && tid < (unsigned)NBIN) {
                uint32_t h = 0u;
                for (unsigned q = 0; q < (unsigned)C; ++q) h += *Cl<C>::at(&s_hist[tid], q);
                a.hist[(size_t)j * NBIN + tid] = h;
            }
            if (r == 0 && tid == 0) {
                double* m = a.mom + (size_t)j * NMOM;
                const double N = (double)(n + (do_neut ? a.ion_count[j] : 0u));
                m[0] = N;
                m[1] = a.weight * N;
                m[2] = s_tot[0]; m[3] = s_tot[1]; m[4] = s_tot[2];
                m[5] = s_tot[3]; m[6] = s_tot[4]; m[7] = s_tot[5];
                m[8] = a.sigma_el * s_tot[6];
                m[9] = a.sigma_ion * s_tot[7];
            }
        }

        // ---- 6. write velocities back through the id list (coalesced)
#pragma unroll
        for (int i = 0; i < ITEMS; ++i) {
            const uint32_t k = tid + (uint32_t)i * NT;
            if (k < nh) {
                const uint32_t pos = hp[i] & 0xFFFFu, l = hl[i];
                const uint32_t o = pos_owner(pos, n, C);
                const uint32_t lp = pos - pos_begin(o, n, C);
                a.vx[l] = *Cl<C>::at(svx + lp, o);
                a.vy[l] = *Cl<C>::at(svy + lp, o);
                a.vz[l] = *Cl<C>::at(svz + lp, o);
            }
        }
        Cl<C>::sync();
    }
}

}  // namespace ltpc
