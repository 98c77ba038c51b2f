// k_group.cu -- per-cell grouping of particle ids (Table 5, CCS1-CCS3) and the
// bookkeeping between passes: append of ionization secondaries (Table 3, CS5),
// new cell offsets, and the cluster-class work lists of the cell kernel.
#include <cuda_runtime.h>
#include <stdint.h>

#include "bijection.cuh"
#include "ltpc_internal.h"
#include "ltpc_launch.h"

namespace ltpc {

// CCS1 at load time: N_j by warp-aggregated atomics (counts must be zero).
// The loop runs over whole warps (its bound is rounded up to a multiple of 32
// and the same for every lane), so every lane takes part in each match with
// the full mask; a lane past the end or holding an out-of-range id takes part
// with the sentinel -1 and adds nothing.
static __global__ void k_hist(const int32_t* __restrict__ cell, uint32_t* __restrict__ counts, int32_t M,
                       DevState* ds)
{
    const unsigned long long n = ds->n;
    const unsigned long long n_up = (n + 31ull) & ~31ull;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;   // blockDim is a multiple of 32
    for (unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; l < n_up; l += stride) {
        int32_t c = l < n ? cell[l] : -1;
        if (l < n && (c < 0 || c >= M)) {
            atomicOr(&ds->err, ERR_BAD_CELL);
            c = -1;
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, c);
        const unsigned leader = __ffs(peers) - 1;
        if (c >= 0 && (threadIdx.x & 31u) == leader) atomicAdd(&counts[c], (uint32_t)__popc(peers));
    }
}

// The per-cell scalars of a pass (CellParamArgs), from the cell's count, its
// inputs and the moments left by the previous pass:
//   * the Takizuka-Abe coefficient A = q^4 n_j lnL dt_j / (8 pi eps0^2 mu^2),
//     n_j = w N_j / V_j, with lnL constant or by the NRL electron-electron formula
//     from the cell's temperature and density (clamped below at 2);
//   * for the momentum/energy restoration, the cell's mean velocity V0 and its
//     summed squared peculiar speed K0 = sum |v|^2 - |sum v|^2 / N before the
//     collisions.  The stored moments are sums over exactly the velocities the
//     pass starts from when their count equals N_j; otherwise (an append rolled
//     back by a capacity error), or when the cell drifts faster than its thermal
//     speed (cancellation in the uncentred sums), K0 = -1 asks the pass to form
//     centred sums itself;
//   * in the bijection pairing mode, for a cell of BIJ_MIN_N..BIJ_MAX_N
//     particles, the shape (a, b), the six round keys and the candidate-count
//     word of its pairing bijection (bijection.cuh): words 0-3 of the Philox
//     block (cell, step, PERM, 0), then words 0-2 of the block (cell, step,
//     PERM, 1).
__device__ void cell_params(const CellParamArgs& cp, int32_t j, double dt, uint32_t step)
{
    // One binary64 division per cell (1 / sum of counts of the stored moments);
    // everything else is products, since binary64 runs on a narrow pipe here.
    const double* m = cp.mom + (size_t)j * NMOM;
    const uint32_t n = cp.counts[j];
    double* o = cp.cpar + (size_t)j * NCP;
    const double dtj = dt * cp.dt_factor[j];
    const double N = m[0];
    const double iN = N > 0.0 ? 1.0 / N : 0.0;
    const double mean[3] = {m[2] * iN, m[3] * iN, m[4] * iN};
    const double s2 = m[5] + m[6] + m[7];
    double lnl = cp.lnlam[j];
    if (cp.lnl_nrl) {
        lnl = 2.0;
        if (N >= 2.0) {
            const double TeV = (s2 * iN - (mean[0] * mean[0] + mean[1] * mean[1] + mean[2] * mean[2])) /
                               (3.0 * cp.e_over_m);
            const double nm3 = cp.weight * (double)n * cp.inv_vol[j];
            if (TeV > 0.0 && nm3 > 0.0) {
                // 23.5 - ln(n^1/2 T^-5/4) - (1e-5 + (ln T - 2)^2 / 16)^1/2, n in cm^-3, T in eV
                const double lt = log(TeV);
                const double v = 23.5 - (0.5 * log(nm3 * 1e-6) - 1.25 * lt) -
                                 sqrt(1e-5 + (lt - 2.0) * (lt - 2.0) * 0.0625);
                lnl = v < 2.0 ? 2.0 : v;
            }
        }
    }
    o[CP_A] = cp.coef0 * (double)n * cp.inv_vol[j] * lnl * dtj;
    o[CP_DT] = dtj;
    o[CP_LNL] = lnl;
    for (int q = 0; q < 3; ++q) o[CP_C + q] = mean[q];
    double K0 = -1.0;
    if (n > 0u && N == (double)n) {
        const double drift = m[2] * mean[0] + m[3] * mean[1] + m[4] * mean[2];   // N |mean|^2
        K0 = s2 - drift;
        K0 = K0 > 0.0 ? K0 : 0.0;
        // The stored sums are not centred: when the drift energy exceeds the
        // thermal one, K0 = sum |v|^2 - N |mean|^2 loses digits to cancellation,
        // so the pass forms centred sums itself instead.
        if (drift > K0) K0 = -1.0;
        o[CP_INVN] = iN;
    } else {
        o[CP_INVN] = n > 0u ? 1.0 / (double)n : 0.0;
    }
    o[CP_K0] = K0;
    float* f = reinterpret_cast<float*>(o + CP_F32);
    f[0] = (float)o[CP_A];
    f[1] = (float)dtj;
    for (int q = 0; q < 3; ++q) f[2 + q] = (float)mean[q];
    f[5] = (float)K0;
    f[6] = (float)o[CP_INVN];
    f[7] = 0.0f;
    uint32_t* w = reinterpret_cast<uint32_t*>(o + CP_BIJ);
    for (int q = 0; q < CPB_WORDS; ++q) w[q] = 0u;
    if (cp.k_rec > 0.0 && n >= 2u) {
        // C5 primaries: floor(P_rec N + U), P_rec = 1 - exp(-dt k_rec n^2), at most N / 2 (the
        // products in the reference's order, without contraction)
        const double nj = __dmul_rn(__dmul_rn(cp.weight, (double)n), cp.inv_vol[j]);
        const double prec = -expm1(-__dmul_rn(__dmul_rn(__dmul_rn(dtj, cp.k_rec), nj), nj));
        const uint4 wr = philox4x32_10((uint32_t)j, step, TAG_RECOMB, 0u, cp.keys);
        const double t = floor(__dadd_rn(__dmul_rn(prec, (double)n), fma((double)wr.x, 0x1p-32, 0x1p-33)));
        const uint32_t cap = n / 2u;
        w[CPB_NREC] = t <= 0.0 ? 0u : (t >= (double)cap ? cap : (uint32_t)t);
    }
    if (cp.bijection && n >= BIJ_MIN_N && n <= BIJ_MAX_N) {
        uint32_t a, b, mb;
        bij_shape(n, &a, &b, &mb);
        const uint4 w0 = philox4x32_10((uint32_t)j, step, TAG_PERM, 0u, cp.keys);
        const uint4 w1 = philox4x32_10((uint32_t)j, step, TAG_PERM, 1u, cp.keys);
        w[CPB_AB] = a | (b << 16);
        w[CPB_MB] = mb;
        w[CPB_KEY + 0] = w0.x; w[CPB_KEY + 1] = w0.y; w[CPB_KEY + 2] = w0.z; w[CPB_KEY + 3] = w0.w;
        w[CPB_KEY + 4] = w1.x; w[CPB_KEY + 5] = w1.y;
        w[CPB_U] = w1.z;
    }
}

// CCS3: perm[I_j + rank] = l.  Cell ids outside [0, M) are skipped (the load's
// histogram reports them).  With the cached-grouping option the kernel exits
// at once while the previous grouping still holds.  Each warp takes 128
// consecutive particles (4 per lane, 16-byte loads).  When they all belong to
// one cell -- the usual case for cell-grouped storage -- one cursor atomic
// serves the 128 and the ids are written with 16-byte stores; otherwise one
// atomic per warp and cell.  The first thing the kernel does is form the
// per-cell scalars of the pass (cell_params above), one thread per cell.
static __global__ void __launch_bounds__(256, 8) k_scatter(const int32_t* __restrict__ cell, int32_t M, uint32_t* __restrict__ cursor,
                                 uint32_t* __restrict__ perm, const DevState* __restrict__ ds, CellParamArgs cp,
                                 const uint32_t* __restrict__ run_start, const uint32_t* __restrict__ cell_start,
                                 const uint32_t* __restrict__ aslot)
{
    if (cp.cpar) {                                   // this pass's per-cell scalars, one thread per cell
        const double dt = ds->dt;
        const uint32_t step = ds->step;
        for (int32_t j = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x); j < M; j += (int32_t)(gridDim.x * blockDim.x))
            cell_params(cp, j, dt, step);
    }
    if (ds->grouping_valid) return;                  // cached grouping: perm is current
    const unsigned long long n = ds->n;
    const unsigned long long n_sorted = ds->n_sorted;   // particles below lie in their cell's run
    const unsigned long long n_loaded = ds->n_loaded;   // particles from here on were appended (slot known)
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
    const unsigned long long w0 = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    for (unsigned long long base = w0 * 128ull; base < n; base += nwarps * 128ull) {
        const unsigned long long l0 = base + 4ull * lane;
        int32_t c[4];
        if (l0 + 3 < n) {
            const int4 v = *reinterpret_cast<const int4*>(cell + l0);
            c[0] = v.x; c[1] = v.y; c[2] = v.z; c[3] = v.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) c[u] = l0 + u < n ? cell[l0 + u] : -1;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) c[u] = c[u] < M ? c[u] : -1;
        const int32_t c0 = __shfl_sync(0xFFFFFFFFu, c[0], 0);
        const bool same = c[0] == c0 && c[1] == c0 && c[2] == c0 && c[3] == c0;
        if (__all_sync(0xFFFFFFFFu, same) && c0 >= 0) {           // one cell, 128 particles
            uint32_t b = 0u;
            const uint32_t l = (uint32_t)l0;
            if (base >= n_loaded) {                               // appended: each at its recorded slot
                const uint32_t cs = cell_start[c0];
#pragma unroll
                for (int u = 0; u < 4; ++u) perm[cs + aslot[l + u]] = l + (uint32_t)u;
                continue;
            }
            if (base + 128ull <= n_sorted) {                      // in the cell's run: no atomic
                b = cell_start[c0] + (uint32_t)(base - run_start[c0]) + 4u * lane;
            } else {
                if (lane == 0) b = atomicAdd(&cursor[c0], 128u);
                b = __shfl_sync(0xFFFFFFFFu, b, 0) + 4u * lane;
            }
            if ((b & 3u) == 0u) {
                *reinterpret_cast<uint4*>(perm + b) = make_uint4(l, l + 1u, l + 2u, l + 3u);
            } else {
                perm[b] = l; perm[b + 1] = l + 1u; perm[b + 2] = l + 2u; perm[b + 3] = l + 3u;
            }
            continue;
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {                             // mixed cells
            const unsigned long long l = l0 + u;
            int32_t ca = c[u];
            if (ca >= 0 && l < n_sorted) {                        // in its cell's run
                perm[cell_start[ca] + (uint32_t)(l - run_start[ca])] = (uint32_t)l;
                ca = -1;
            } else if (ca >= 0 && l >= n_loaded) {                // appended: at its recorded slot
                perm[cell_start[ca] + aslot[l]] = (uint32_t)l;
                ca = -1;
            }
            const unsigned peers = __match_any_sync(0xFFFFFFFFu, ca);
            const unsigned leader = __ffs(peers) - 1;
            uint32_t b = 0u;
            if (lane == leader && ca >= 0) b = atomicAdd(&cursor[ca], (uint32_t)__popc(peers));
            b = __shfl_sync(0xFFFFFFFFu, b, leader);
            if (ca >= 0) perm[b + __popc(peers & ((1u << lane) - 1u))] = (uint32_t)l;
        }
    }
}

// Single-CTA bookkeeping between passes (REGROUP_THREADS threads):
//   1. if `append`: exclusive scan of this pass's secondaries per cell into
//      ion_off, capacity check, counts += ion_count, keep the old offsets;
//   2. CCS2: cell_start = exclusive scan of counts, cursor = cell_start + run_len;
//   3. cluster-class work lists (cells in ascending index order per class,
//      each item {cell, N_j, I_j, 1} so that a CTA fetches it with one load);
//   4. reset the work tickets, optionally advance the step number.
static __global__ void __launch_bounds__(REGROUP_THREADS)
k_regroup(int32_t M, uint32_t* __restrict__ counts, uint32_t* __restrict__ cell_start,
          uint32_t* __restrict__ cs_prev, uint32_t* __restrict__ cursor,
          uint32_t* __restrict__ ion_count, uint32_t* __restrict__ ion_off, RegroupLists lists,
          unsigned long long capacity, int append, int advance_step, DevState* ds)
{
    constexpr int NT = REGROUP_THREADS;
    __shared__ uint32_t s_w[NT / 32 + 1];
    __shared__ uint32_t s_cls[MAX_CLASSES][NT / 32 + 1];
    __shared__ unsigned long long s_total;
    __shared__ uint32_t s_max;
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    if (tid == 0) s_max = 0u;
    const uint32_t per = (uint32_t)((M + NT - 1) / NT);
    const uint32_t b0 = min((uint32_t)M, tid * per), b1 = min((uint32_t)M, b0 + per);

    auto block_scan = [&](uint32_t v, uint32_t* tot) -> uint32_t {
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
            if (lane >= (unsigned)o) x += y;
        }
        if (lane == 31u) s_w[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const uint32_t wv = lane < NT / 32 ? s_w[lane] : 0u;
            uint32_t z = wv;
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
                if (lane >= (unsigned)o) z += y;
            }
            if (lane < NT / 32) s_w[lane] = z - wv;
            if (lane == NT / 32 - 1) s_w[NT / 32] = z;
        }
        __syncthreads();
        const uint32_t r = s_w[warp] + x - v;
        *tot = s_w[NT / 32];
        __syncthreads();
        return r;
    };

    // 1. secondaries of the last pass
    uint32_t total_ion = 0u;
    bool appended = false;
    if (append) {
        uint32_t sum = 0u;
        for (uint32_t c = b0; c < b1; ++c) sum += ion_count[c];
        uint32_t tot;
        uint32_t ex = block_scan(sum, &tot);
        if (tid == 0) s_total = (unsigned long long)tot;
        __syncthreads();
        const unsigned long long n0 = ds->n;
        appended = tot > 0u && n0 + tot <= capacity;
        if (tot > 0u && !appended && tid == 0) atomicOr(&ds->err, ERR_CAPACITY);
        for (uint32_t c = b0; c < b1; ++c) {
            ion_off[c] = ex;
            ex += ion_count[c];
            cs_prev[c] = cell_start[c];
            if (appended) counts[c] += ion_count[c];
            ion_count[c] = 0u;
            counts[c] -= lists.rec_count[c];           // primaries removed by recombination
            lists.rec_count[c] = 0u;
        }
        if (tid == 0) { ion_off[M] = tot; cs_prev[M] = cell_start[M]; }
        total_ion = appended ? tot : 0u;
        __syncthreads();
    }

    // 2. CCS2: offsets of the grouping.  After a pass that removed particles the cells are no
    // longer runs of the storage: every particle takes its place from the cursor from now on.
    {
        const bool ungroup = ds->ungroup != 0u;
        uint32_t sum = 0u;
        for (uint32_t c = b0; c < b1; ++c) sum += counts[c];
        uint32_t tot;
        uint32_t ex = block_scan(sum, &tot);
        for (uint32_t c = b0; c < b1; ++c) {
            if (ungroup) lists.run_len[c] = 0u;
            cell_start[c] = ex;
            cursor[c] = ex + lists.run_len[c];   // appended particles follow the cell's run
            ex += counts[c];
        }
        if (tid == 0) cell_start[M] = tot;
    }

    // 3. work lists: class of a cell = first class whose max_n covers it
    {
        uint32_t cnt[MAX_CLASSES];
        for (int k = 0; k < MAX_CLASSES; ++k) cnt[k] = 0u;
        uint32_t mx = 0u;
        for (uint32_t c = b0; c < b1; ++c) {
            const uint32_t n = counts[c];
            mx = max(mx, n);
            if (n == 0u) continue;
            int k = 0;
            while (k < lists.n_classes - 1 && n > lists.max_n[k]) ++k;
            ++cnt[k];
        }
        for (int k = 0; k < lists.n_classes; ++k) {
            uint32_t x = cnt[k];
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
                if (lane >= (unsigned)o) x += y;
            }
            if (lane == 31u) s_cls[k][warp] = x;
            cnt[k] = x - cnt[k];   // exclusive within the warp
        }
        // reduce the largest count
        for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xFFFFFFFFu, mx, o));
        __syncthreads();
        if (warp == 0) {
            for (int k = 0; k < lists.n_classes; ++k) {
                const uint32_t wv = lane < NT / 32 ? s_cls[k][lane] : 0u;
                uint32_t z = wv;
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
                    if (lane >= (unsigned)o) z += y;
                }
                if (lane < NT / 32) s_cls[k][lane] = z - wv;
                if (lane == NT / 32 - 1) s_cls[k][NT / 32] = z;
            }
        }
        if (lane == 0) atomicMax(&s_max, mx);
        __syncthreads();
        uint32_t pos[MAX_CLASSES];
        for (int k = 0; k < lists.n_classes; ++k) pos[k] = s_cls[k][warp] + cnt[k];
        for (uint32_t c = b0; c < b1; ++c) {
            const uint32_t n = counts[c];
            if (n == 0u) continue;
            int k = 0;
            while (k < lists.n_classes - 1 && n > lists.max_n[k]) ++k;
            if (n > lists.max_n[k]) atomicOr(&ds->err, ERR_CELL_TOO_LARGE);
            lists.list[k][pos[k]++] = make_uint4(c, n, cell_start[c], 1u);
        }
        if (tid < (unsigned)MAX_CLASSES) {
            ds->class_n[tid] = tid < (unsigned)lists.n_classes ? s_cls[tid][NT / 32] : 0u;
            ds->ticket[tid] = 0u;
        }
    }
    __syncthreads();
    if (tid == 0) {
        const bool ug = ds->ungroup != 0u;
        if (ug) {
            ds->n_sorted = 0ull;
            ds->n_loaded = ~0ull;
            ds->ungroup = 0u;
        }
        ds->max_count = s_max;
        ds->n_ion = total_ion;
        // after a pass that appended and removed nothing the grouping of the next pass is this one's
        ds->grouping_valid = (lists.cache_grouping && append && total_ion == 0u && !ug) ? 1u : 0u;
        ds->n += total_ion;
        if (advance_step) ds->step += 1u;
    }
}

// Copy the secondaries staged by the last pass to the end of the particle
// arrays: secondary g (in cell order, then pairing-order position of the
// parent) goes to slot n_old + g with the parent's cell and position, and
// records its place in the cell's grouping: the cell's count before this
// append (from the previous offsets) plus its rank among the cell's new ones.
template <class T>
static __global__ void k_append(int32_t M, const uint32_t* __restrict__ ion_off, const uint32_t* __restrict__ cs_prev,
                         const uint32_t* __restrict__ stage_l, const T* __restrict__ svx,
                         const T* __restrict__ svy, const T* __restrict__ svz, T* __restrict__ vx,
                         T* __restrict__ vy, T* __restrict__ vz, int32_t* __restrict__ cell,
                         T* __restrict__ x, uint32_t* __restrict__ aslot, const DevState* __restrict__ ds)
{
    const uint32_t tot = ds->n_ion;
    if (tot == 0u) return;
    const unsigned long long n0 = ds->n - tot;
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < tot; g += gridDim.x * blockDim.x) {
        // last cell j with ion_off[j] <= g
        int32_t lo = 0, hi = M - 1;
        while (lo < hi) {
            const int32_t mid = (lo + hi + 1) >> 1;
            if (ion_off[mid] <= g) lo = mid; else hi = mid - 1;
        }
        const uint32_t src = cs_prev[lo] + (g - ion_off[lo]);
        const unsigned long long dst = n0 + g;
        const uint32_t parent = stage_l[src];
        vx[dst] = svx[src]; vy[dst] = svy[src]; vz[dst] = svz[src];
        cell[dst] = lo;
        aslot[dst] = (cs_prev[lo + 1] - cs_prev[lo]) + (g - ion_off[lo]);
        if (x) x[dst] = x[parent];
    }
}

// Runs of a load (RegroupLists::run_start / run_len).  The load is grouped by
// cell when every cell id is valid and the ids never decrease; then the run of
// cell c starts at the first index holding c and has its N_j particles, and
// the scatter places them without atomics.  Otherwise there are no runs.
static __global__ void k_runs_check(const int32_t* __restrict__ cell, int32_t M, DevState* ds)
{
    const unsigned long long n = ds->n;
    for (unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (unsigned long long)gridDim.x * blockDim.x) {
        const int32_t c = cell[l];
        if (c < 0 || c >= M || (l + 1 < n && cell[l + 1] < c)) {
            atomicOr(&ds->load_unsorted, 1u);
            return;
        }
    }
}

static __global__ void k_runs_set(const int32_t* __restrict__ cell, int32_t M, const uint32_t* __restrict__ counts,
                                  uint32_t* __restrict__ run_start, uint32_t* __restrict__ run_len, DevState* ds,
                                  int require_grouped)
{
    const unsigned long long n = ds->n;
    const bool grouped = ds->load_unsorted == 0u;
    if (require_grouped && !grouped && blockIdx.x == 0 && threadIdx.x == 0) atomicOr(&ds->err, ERR_UNGROUPED);
    const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long c = gt; c < (unsigned long long)M; c += stride) run_len[c] = grouped ? counts[c] : 0u;
    if (grouped) {
        for (unsigned long long l = gt; l < n; l += stride) {
            const int32_t c = cell[l];
            if (l == 0 || cell[l - 1] != c) run_start[c] = (uint32_t)l;
        }
    }
    if (gt == 0) ds->n_sorted = grouped ? n : 0ull;
}

static __global__ void k_reset_cursors(int32_t M, const uint32_t* __restrict__ cell_start,
                                       const uint32_t* __restrict__ run_len, uint32_t* __restrict__ cursor)
{
    for (int32_t c = (int32_t)(blockIdx.x * blockDim.x + threadIdx.x); c < M; c += (int32_t)(gridDim.x * blockDim.x))
        cursor[c] = cell_start[c] + run_len[c];
}

static __global__ void k_set_state(DevState* ds, unsigned long long n, int set_n, uint32_t step, double dt, int set_step)
{
    if (set_n) {
        ds->n = n; ds->n_ion = 0u; ds->grouping_valid = 0u; ds->load_unsorted = 0u; ds->n_sorted = 0ull;
        ds->n_loaded = n;
    }
    if (set_step) { ds->step = step; ds->dt = dt; }
}

// Load-time validation: non-finite velocities.
template <class T>
static __global__ void k_check_finite(const T* __restrict__ vx, const T* __restrict__ vy, const T* __restrict__ vz,
                               DevState* ds)
{
    const unsigned long long n = ds->n;
    for (unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (unsigned long long)gridDim.x * blockDim.x) {
        if (!isfinite(vx[l]) || !isfinite(vy[l]) || !isfinite(vz[l])) {
            atomicOr(&ds->err, ERR_NONFINITE);
            return;
        }
    }
}
cudaError_t launch_hist(const int32_t* cell, uint32_t* counts, int32_t M, DevState* ds, int grid, cudaStream_t s)
{
    k_hist<<<grid, 256, 0, s>>>(cell, counts, M, ds);
    return cudaGetLastError();
}

cudaError_t launch_scatter(const int32_t* cell, int32_t M, uint32_t* cursor, uint32_t* perm, const DevState* ds,
                           int grid, cudaStream_t s, const RegroupLists& runs, const uint32_t* cell_start,
                           const CellParamArgs* cp)
{
    CellParamArgs none = {};
    k_scatter<<<grid, 256, 0, s>>>(cell, M, cursor, perm, ds, cp ? *cp : none, runs.run_start, cell_start,
                                   runs.aslot);
    return cudaGetLastError();
}

cudaError_t launch_regroup(int32_t M, uint32_t* counts, uint32_t* cell_start, uint32_t* cs_prev, uint32_t* cursor,
                           uint32_t* ion_count, uint32_t* ion_off, const RegroupLists& lists,
                           unsigned long long capacity, int append, int advance_step, DevState* ds, cudaStream_t s)
{
    k_regroup<<<1, REGROUP_THREADS, 0, s>>>(M, counts, cell_start, cs_prev, cursor, ion_count, ion_off, lists,
                                            capacity, append, advance_step, ds);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_append(int32_t M, const uint32_t* ion_off, const uint32_t* cs_prev, const uint32_t* stage_l,
                          const T* svx, const T* svy, const T* svz, T* vx, T* vy, T* vz, int32_t* cell, T* x,
                          uint32_t* aslot, const DevState* ds, int grid, cudaStream_t s)
{
    k_append<T><<<grid, 256, 0, s>>>(M, ion_off, cs_prev, stage_l, svx, svy, svz, vx, vy, vz, cell, x, aslot, ds);
    return cudaGetLastError();
}
template cudaError_t launch_append<float>(int32_t, const uint32_t*, const uint32_t*, const uint32_t*, const float*,
                                          const float*, const float*, float*, float*, float*, int32_t*, float*,
                                          uint32_t*, const DevState*, int, cudaStream_t);
template cudaError_t launch_append<double>(int32_t, const uint32_t*, const uint32_t*, const uint32_t*,
                                           const double*, const double*, const double*, double*, double*, double*,
                                           int32_t*, double*, uint32_t*, const DevState*, int, cudaStream_t);

cudaError_t launch_runs(const int32_t* cell, int32_t M, const uint32_t* counts, const RegroupLists& runs, DevState* ds,
                        int grid, cudaStream_t s, int require_grouped)
{
    k_runs_check<<<grid, 256, 0, s>>>(cell, M, ds);
    k_runs_set<<<grid, 256, 0, s>>>(cell, M, counts, runs.run_start, runs.run_len, ds, require_grouped);
    return cudaGetLastError();
}

// Storage compaction: dst[k] = src[perm[k]] for the k < n grouped particles (cells
// ascending, each cell's particles in its grouping order).  Reads follow the id
// list (runs of consecutive ids for cell-grouped storage), writes are coalesced.
template <class T>
static __global__ void __launch_bounds__(256) k_compact_gather(const uint32_t* __restrict__ perm, uint32_t n,
                                                               const T* __restrict__ a0, const T* __restrict__ a1,
                                                               const T* __restrict__ a2, const int32_t* __restrict__ c,
                                                               T* __restrict__ b0, T* __restrict__ b1, T* __restrict__ b2,
                                                               int32_t* __restrict__ d)
{
    for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        const uint32_t l = perm[k];
        b0[k] = a0[l];
        if (b1) b1[k] = a1[l];
        if (b2) b2[k] = a2[l];
        if (d) d[k] = c[l];
    }
}

template <class T>
cudaError_t launch_compact_gather(const uint32_t* perm, uint32_t n, const T* a0, const T* a1, const T* a2,
                                  const int32_t* c, T* b0, T* b1, T* b2, int32_t* d, int grid, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const int g = (int)min((unsigned long long)grid, ((unsigned long long)n + 255ull) / 256ull);
    k_compact_gather<T><<<g, 256, 0, s>>>(perm, n, a0, a1, a2, c, b0, b1, b2, d);
    return cudaGetLastError();
}
template cudaError_t launch_compact_gather<float>(const uint32_t*, uint32_t, const float*, const float*, const float*,
                                                  const int32_t*, float*, float*, float*, int32_t*, int, cudaStream_t);
template cudaError_t launch_compact_gather<double>(const uint32_t*, uint32_t, const double*, const double*,
                                                   const double*, const int32_t*, double*, double*, double*, int32_t*,
                                                   int, cudaStream_t);

cudaError_t launch_reset_cursors(int32_t M, const uint32_t* cell_start, const RegroupLists& runs, uint32_t* cursor,
                                 cudaStream_t s)
{
    k_reset_cursors<<<(M + 255) / 256, 256, 0, s>>>(M, cell_start, runs.run_len, cursor);
    return cudaGetLastError();
}

cudaError_t launch_set_state(DevState* ds, unsigned long long n, int set_n, uint32_t step, double dt, int set_step,
                             cudaStream_t s)
{
    k_set_state<<<1, 1, 0, s>>>(ds, n, set_n, step, dt, set_step);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_check_finite(const T* vx, const T* vy, const T* vz, DevState* ds, int grid, cudaStream_t s)
{
    k_check_finite<T><<<grid, 256, 0, s>>>(vx, vy, vz, ds);
    return cudaGetLastError();
}
template cudaError_t launch_check_finite<float>(const float*, const float*, const float*, DevState*, int,
                                                cudaStream_t);
template cudaError_t launch_check_finite<double>(const double*, const double*, const double*, DevState*, int,
                                                 cudaStream_t);

}  // namespace ltpc
