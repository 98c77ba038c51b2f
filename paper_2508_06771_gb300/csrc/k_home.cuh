// k_home.cuh -- the home-order cell kernel of the bijection pairing mode.
//
// One CTA per cell (persistent loop, dynamic tickets), for cells of
// BIJ_MIN_N..CAPL particles whose index list is in ascending id order (storage
// grouped by cell: the loaded run, then the appended particles at their
// recorded slots).  The particle of id rank k -- its home index -- keeps slot
// k of the cell's velocity arrays in shared memory for the whole pass, so:
//   * the loaded run arrives as three bulk copies (cp.async.bulk, TMA) that
//     complete on an mbarrier while every thread inverts the pairing bijection
//     for its pair slots (position 2p and 2p+1 -> home indices);
//   * step S1 (Takizuka-Abe, CCS4-CCS5 of Table 5) works on the pair slots,
//     reading and writing the two partners' home slots;
//   * the momentum/energy restoration, the null-collision bound and the
//     moments (S3a/S3b, Sec. 4.5) are one sweep of the home slots in 16-byte
//     vectors;
//   * step S2a takes the particles at pairing positions below
//     floor(P_null N + U) as its candidates (Sec. 4.2: P_null N particles),
//     found through a table of the home index at every position, and
//     corrects the sums of the particles it changes;
//   * the result goes back as three bulk stores.
// Only the few particles outside the 16-byte-aligned interior of the run
// (at most W-1 at each end) and the appended ones move with plain loads and
// stores.  Every wait on the mbarrier is bounded: on time-out the kernel sets
// ERR_TIMEOUT, waits once more (also bounded) for its copies and returns.
#pragma once
#include "k_cells.cuh"

namespace ltpc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* m, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(m)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }
// Order this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk copy) accesses of the same memory.
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_expect_tx(uint64_t* m, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* m, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(m)), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bulk copies: both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* m)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(sdst)),
                 "l"(gsrc), "r"(bytes), "r"(smem_u32(m))
                 : "memory");
}
__device__ __forceinline__ void bulk_store(void* gdst, const void* ssrc, uint32_t bytes)
{
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst), "r"(smem_u32(ssrc)),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }

constexpr uint32_t MBAR_SPIN_LIMIT = 1u << 24;   // try_wait rounds before a wait is declared timed out

// Shared-memory bytes of the home kernel's velocity slots.
// (three components, the 16-bit home index of every pairing position, the ids
// of the appended homes)
template <class T>
__host__ __device__ constexpr size_t home_dyn_smem(uint32_t capl)
{
    return (size_t)3 * (capl + 2u * (16u / sizeof(T))) * sizeof(T) + (((size_t)capl + 7u) & ~(size_t)7u) * 2u +
           (size_t)(capl / 3u) * 4u;
}

// Sixteen bytes of one component as W values.
template <class T> struct Vec16;
template <> struct Vec16<float> {
    static constexpr int W = 4;
    static __device__ __forceinline__ void ld(const float* p, float (&v)[4])
    {
        const float4 t = *reinterpret_cast<const float4*>(p);
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
    static __device__ __forceinline__ void st(float* p, const float (&v)[4])
    {
        *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
};
template <> struct Vec16<double> {
    static constexpr int W = 2;
    static __device__ __forceinline__ void ld(const double* p, double (&v)[2])
    {
        const double2 t = *reinterpret_cast<const double2*>(p);
        v[0] = t.x; v[1] = t.y;
    }
    static __device__ __forceinline__ void st(double* p, const double (&v)[2])
    {
        *reinterpret_cast<double2*>(p) = make_double2(v[0], v[1]);
    }
};

template <class T, int NT, int CAPL, bool XS>
__global__ void __launch_bounds__(NT, 1) k_home(CellArgs<T> a)
{
    using VW = Vec16<T>;
    constexpr int W = VW::W;                       // elements per 16 bytes
    constexpr uint32_t PAD = CAPL + 2 * W;         // slots per component (alignment offset + rounding)
    constexpr int PS = (CAPL / 2 + NT - 1) / NT;   // pair slots per thread
    constexpr int NW = NT / 32;
    static_assert(NT % 32 == 0 && NT <= 1024 && NT >= 64, "block size");
    static_assert(CAPL <= 65536 && CAPL % W == 0 && CAPL / 32 <= NT, "capacity");

    extern __shared__ __align__(16) unsigned char smem[];
    T* const sv0 = reinterpret_cast<T*>(smem);     // component c at sv0 + c * PAD; home k at slot k + o
    uint16_t* const sinv = reinterpret_cast<uint16_t*>(sv0 + 3 * PAD);   // home index at each pairing position
    uint32_t* const sid = reinterpret_cast<uint32_t*>(sinv + ((CAPL + 7) & ~7));   // ids of the appended homes
    constexpr uint32_t SIDCAP = CAPL / 3;          // appended homes whose ids the table holds
    __shared__ __align__(8) uint64_t s_bar;        // completion of the bulk loads
    __shared__ uint4 s_item[2];                    // current / next work item {j, N_j, I_j, valid}
    __shared__ __align__(16) uint32_t s_bij[2][12];// bijection words (CPB_*) of the current / next cell
    __shared__ uint32_t s_run[2][2];               // run start and length of the current / next cell
    __shared__ __align__(16) double s_cp[NCP];     // the cell's scalars of this pass
    __shared__ uint32_t s_scan[NW + 1];
    __shared__ T s_redacc[NW * 8];
    __shared__ double s_cl[8];
    __shared__ double s_tot[8];
    __shared__ uint32_t s_hist[4 * NBIN];          // four sub-histograms (less atomic contention)
    __shared__ uint32_t s_imask[CAPL / 32];        // ionizing pairing positions
    __shared__ uint32_t s_ioff[CAPL / 32];         // ionizations before each mask word
    __shared__ T s_par[16];
    __shared__ typename MaxBits<T>::U s_vmax;
    __shared__ __align__(16) uint8_t s_rt[2][6][256];  // round functions of the current / next cell's bijection

    const unsigned tid = threadIdx.x;
    DevState* ds = a.ds;
    const uint32_t list_n = ds->class_n[a.cls];
    const uint32_t step = ds->step;
    const bool do_coul = (a.flags & F_COULOMB) != 0u;
    const bool do_neut = (a.flags & F_NEUTRAL) != 0u;
    const bool do_corr = (a.flags & F_CORRECTION) != 0u;
    T* const gv[3] = {a.vx, a.vy, a.vz};
    // The last warp has the fewest pair slots (slots are dealt round-robin from thread 0), so
    // it runs the copies (DM) and the ticket (TK): waits there delay the least bijection work.
    constexpr unsigned DM = NT - 32u, TK = NT - 31u;
    // a cell's bijection words and run bounds into s_bij / s_run[b] (asynchronous copies of TK)
    auto fetch_cell_words = [&](uint32_t jj, uint32_t b) {
        const double* cpj = a.cpar + (size_t)jj * NCP + CP_BIJ;
#pragma unroll
        for (int q = 0; q < 3; ++q) cp_async<16>(&s_bij[b][4 * q], cpj + 2 * q);
        cp_async<4>(&s_run[b][0], a.run_start + jj);
        cp_async<4>(&s_run[b][1], a.run_len + jj);
    };

    if (tid == DM) {
        mbar_init(&s_bar, 1u);
        fence_mbar_init();
    }
    // a cell's six round functions as byte tables (round i reads R below b for even i, a for
    // odd i), by every thread but the last warp's
    auto fill_round_tables = [&](uint32_t b) {
        const uint32_t ab = s_bij[b][CPB_AB];
        if (ab == 0u || tid >= NT - 32u) return;
        const uint32_t A_ = ab & 0xFFFFu, B_ = ab >> 16;
        for (uint32_t e = tid; e < 6u * 256u; e += NT - 32u) {
            const uint32_t i = e >> 8, r = e & 255u;
            const uint32_t m = (i & 1u) ? B_ : A_, lim = (i & 1u) ? A_ : B_;
            if (r < lim) s_rt[b][i][r] = (uint8_t)bij_round(r, s_bij[b][CPB_KEY + i], m);
        }
    };
    if (tid == TK) {
        const uint32_t w = atomicAdd(&ds->ticket[a.cls], 1u);
        const uint4 it = w < list_n ? a.list[w] : make_uint4(0u, 0u, 0u, 0u);
        s_item[0] = it;
        if (it.w != 0u) fetch_cell_words(it.x, 0u);
        else s_bij[0][CPB_AB] = 0u;
        cp_async_wait_all();
    }
    __syncthreads();
    fill_round_tables(0u);
    __syncthreads();
    PhaseClock pc{a.phase_clk, 0};
    pc.start();
    uint32_t phase = 0u;

    for (uint32_t par = 0u;; par ^= 1u) {
        const uint4 item = s_item[par];
        if (item.w == 0u) break;
        const uint32_t j = item.x, n = item.y, s = item.z;
        const uint32_t* bw = s_bij[par];                            // prefetched with the item
        const uint32_t bij_ab = bw[CPB_AB];
        if (n == 0u || n > (uint32_t)CAPL || bij_ab == 0u) {   // not a cell of this kernel (uniform)
            if (tid == TK) {
                if (n != 0u) flag_error(ds, n > (uint32_t)CAPL ? ERR_CELL_TOO_LARGE : ERR_INDEX);
                const uint32_t wn = atomicAdd(&ds->ticket[a.cls], 1u);
                const uint4 it = wn < list_n ? a.list[wn] : make_uint4(0u, 0u, 0u, 0u);
                s_item[par ^ 1u] = it;
                if (it.w != 0u) fetch_cell_words(it.x, par ^ 1u);
                else s_bij[par ^ 1u][CPB_AB] = 0u;
                cp_async_wait_all();
            }
            __syncthreads();
            fill_round_tables(par ^ 1u);
            __syncthreads();
            continue;
        }
        const uint32_t rs = s_run[par][0];
        const uint32_t rl = min(s_run[par][1], n);                 // loaded run: homes [0, rl)
        const uint32_t o = rs & (uint32_t)(W - 1);                 // slot of home k is k + o
        const uint32_t g0 = (rs + (uint32_t)W - 1u) & ~(uint32_t)(W - 1);       // aligned interior [g0, g1)
        const uint32_t g1e = (rs + rl) & ~(uint32_t)(W - 1);
        const uint32_t g1 = g1e > g0 ? g1e : g0;
        const uint32_t bytes = (g1 - g0) * (uint32_t)sizeof(T);
        const uint32_t nhead = g1 > g0 ? g0 - rs : rl;             // run homes before the interior
        const uint32_t ktail = g1 > g0 ? g1 - rs : rl;             // first run home after it
        const uint32_t nplain = nhead + (rl - ktail) + (n - rl);   // homes moved with plain accesses
        // the plain-access homes in order: [0, nhead), [ktail, rl), [rl, n)
        auto plain_home = [&](uint32_t t) -> uint32_t { return t < nhead ? t : t - nhead + ktail; };
        // id of home k: in the run, or (appended) from the table filled in step 1
        auto id_of = [&](uint32_t k) -> uint32_t {
            return k < rl ? rs + k : (k - rl < SIDCAP ? sid[k - rl] : __ldg(a.perm + s + k));
        };

        // ---- 1. loads.  Thread 0 waits until the previous cell's bulk stores have read the
        // slots (that drain overlaps the bijection work below), then issues the run interior
        // as three bulk copies on the mbarrier, and the record.  Every thread takes one of the
        // few homes outside the interior (ids of appended ones into the table) and holds its
        // velocity in registers until the slots are free; the next ticket is drawn meanwhile.
        if (tid == DM) {
            bulk_wait_read_all();
            fence_proxy_async();
            mbar_expect_tx(&s_bar, 3u * bytes);
            if (bytes) {
#pragma unroll
                for (int c = 0; c < 3; ++c) bulk_load(sv0 + c * PAD + (g0 - rs + o), gv[c] + g0, bytes, &s_bar);
            }
            const double* cpj = a.cpar + (size_t)j * NCP;
#pragma unroll
            for (int q = 0; q < NCP / 2; ++q) cp_async<16>(&s_cp[2 * q], cpj + 2 * q);
            s_vmax = 0u;
        }
        uint32_t pk0 = 0xFFFFFFFFu, pl0 = 0u;          // this thread's first plain home and its id
        T pvx = T(0), pvy = T(0), pvz = T(0);
        if (tid < nplain) {
            pk0 = plain_home(tid);
            pl0 = pk0 < rl ? rs + pk0 : __ldg(a.perm + s + pk0);
            if (pk0 >= rl && pk0 - rl < SIDCAP) sid[pk0 - rl] = pl0;
            pvx = gv[0][pl0]; pvy = gv[1][pl0]; pvz = gv[2][pl0];
        }
        for (uint32_t t = tid + NT; t < nplain; t += NT) {   // more than NT plain homes: ids only here
            const uint32_t k = plain_home(t);
            if (k >= rl && k - rl < SIDCAP) sid[k - rl] = __ldg(a.perm + s + k);
        }
        uint32_t wn = 0u;
        if (tid == TK) wn = atomicAdd(&ds->ticket[a.cls], 1u);
        for (uint32_t i = tid; i < 4u * NBIN; i += NT) s_hist[i] = 0u;
        for (uint32_t i = tid; i < (n + 31u) / 32u; i += NT) s_imask[i] = 0u;
        BijParams B;
        B.n = n; B.a = bij_ab & 0xFFFFu; B.b = bij_ab >> 16; B.mb = bw[CPB_MB];
        pc.mark(0);

        // ---- 2. the pairing bijection, inverted for this thread's pair slots while the copies
        // fly: one pass of the rounds for every position (independent chains), then the rare
        // images at or above n walk on; the home of each position also goes to the table
        const uint8_t(*const rtab)[256] = s_rt[par];       // filled during the previous cell
        auto rt = [&](int i, uint32_t r) -> uint32_t { return rtab[i][r]; };
        uint32_t hx[2 * PS];
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const uint32_t p = tid + (uint32_t)i * NT;
            hx[2 * i] = 2u * p < n ? bij_dec_tab(B, rt, 2u * p) : 0u;
            hx[2 * i + 1] = 2u * p + 1u < n ? bij_dec_tab(B, rt, 2u * p + 1u) : 0u;
        }
#pragma unroll
        for (int i = 0; i < PS; ++i) {
            const uint32_t p = tid + (uint32_t)i * NT;
            if (2u * p < n) {
                uint32_t ka = hx[2 * i], kb = hx[2 * i + 1];
                while (ka >= n) ka = bij_dec_tab(B, rt, ka);
                const bool two = 2u * p + 1u < n;
                if (two) {
                    while (kb >= n) kb = bij_dec_tab(B, rt, kb);
                }
                sinv[2u * p] = (uint16_t)ka;
                if (two) sinv[2u * p + 1u] = (uint16_t)kb;
                if (a.order_out) {                         // inspection: the pairing order of this step
                    a.order_out[s + 2u * p] = id_of(ka);
                    if (two) a.order_out[s + 2u * p + 1u] = id_of(kb);
                }
            }
        }
        if (tid == TK) {                                   // the next work item, completed by the wait below
            if (wn < list_n) cp_async<16>(&s_item[par ^ 1u], a.list + wn);
            else s_item[par ^ 1u] = make_uint4(0u, 0u, 0u, 0u);
        }
        pc.mark(1);

        // ---- 3. wait for the copies (bounded), then every thread sees every slot
        if (tid == DM || tid == TK) cp_async_wait_all();
        if (tid == TK) {                                   // waited before the barrier after S1
            if (s_item[par ^ 1u].w != 0u) fetch_cell_words(s_item[par ^ 1u].x, par ^ 1u);
            else s_bij[par ^ 1u][CPB_AB] = 0u;
        }
        bool done = false;
        for (uint32_t it = 0; it < MBAR_SPIN_LIMIT && !done; ++it) done = mbar_try_wait(&s_bar, phase);
        if (__syncthreads_or(done ? 0 : 1)) {
            if (tid == DM) flag_error(ds, ERR_TIMEOUT);
            for (uint32_t it = 0; it < MBAR_SPIN_LIMIT && !done; ++it) done = mbar_try_wait(&s_bar, phase);
            return;
        }
        phase ^= 1u;
        // the plain homes into their slots (the drain was waited before the bulk copies)
        if (pk0 != 0xFFFFFFFFu) {
            sv0[pk0 + o] = pvx; sv0[PAD + pk0 + o] = pvy; sv0[2 * PAD + pk0 + o] = pvz;
        }
        for (uint32_t t = tid + NT; t < nplain; t += NT) {
            const uint32_t k = plain_home(t);
            const uint32_t l = id_of(k);
#pragma unroll
            for (int c = 0; c < 3; ++c) sv0[c * PAD + k + o] = gv[c][l];
        }
        __syncthreads();
        pc.mark(6);

        T* const svx = sv0 + o;
        T* const svy = sv0 + PAD + o;
        T* const svz = sv0 + 2 * PAD + o;
        const T cx = cell_scalar<T>(s_cp, 2), cy = cell_scalar<T>(s_cp, 3), cz = cell_scalar<T>(s_cp, 4);
        using P = Pk<T>;
        using V2 = typename P::V;

        // ---- 4. step S1 over the pair slots, with the sums the restoration needs
        const bool coul = do_coul && n >= 2u;
        const bool pre_mom = cell_scalar<T>(s_cp, 5) >= T(0);   // K0 < 0: form the sums before S1
        if (coul) {
            const T A = cell_scalar<T>(s_cp, 0);
            const V2 C2x = P::make(-cx, -cx), C2y = P::make(-cy, -cy), C2z = P::make(-cz, -cz);
            V2 sx = P::make(T(0), T(0)), sy = sx, sz = sx, ss = sx;      // after S1 (centred)
            V2 bx0 = sx, by0 = sx, bz0 = sx, bs0 = sx;                    // before S1, if needed
            auto psum = [&](V2 X, V2 Y, V2 Z, V2& ax_, V2& ay_, V2& az_, V2& as_) {
                const V2 dx = P::add(X, C2x), dy = P::add(Y, C2y), dz = P::add(Z, C2z);
                P::acc(ax_, dx); P::acc(ay_, dy); P::acc(az_, dz);
                P::acc(as_, P::fma(dz, dz, P::fma(dy, dy, P::mul(dx, dx))));
            };
            const bool pre = do_corr && !pre_mom;
            const V2 H = P::make(T(0.5), T(-0.5));
            auto slot = [&](int i) {
                const uint32_t p = tid + (uint32_t)i * NT;
                if (2u * p >= n) return;
                // the pair's homes from the table (this thread wrote them in step 2)
                const uint32_t pkv = reinterpret_cast<const uint32_t*>(sinv)[p];
                const uint32_t ka = pkv & 0xFFFFu, kb = pkv >> 16;
                if (2u * p + 1u < n) {
                    const uint32_t la = id_of(ka), lb = id_of(kb);
                    V2 X = P::make(svx[ka], svx[kb]);
                    V2 Y = P::make(svy[ka], svy[kb]);
                    V2 Z = P::make(svz[ka], svz[kb]);
                    if (pre) psum(X, Y, Z, bx0, by0, bz0, bs0);
                    const uint4 w = draw(a.keys, la < lb ? la : lb, step, TAG_PAIR);
                    T dux, duy, duz;
                    ta_delta<T>(X.x, Y.x, Z.x, X.y, Y.y, Z.y, A, w, dux, duy, duz);
                    X = P::fma(H, P::make(dux, dux), X);
                    Y = P::fma(H, P::make(duy, duy), Y);
                    Z = P::fma(H, P::make(duz, duz), Z);
                    svx[ka] = X.x; svy[ka] = Y.x; svz[ka] = Z.x;
                    svx[kb] = X.y; svy[kb] = Y.y; svz[kb] = Z.y;
                    if (do_corr) psum(X, Y, Z, sx, sy, sz, ss);
                } else {                                   // the one left out: unchanged
                    const V2 X1 = P::make(svx[ka], cx), Y1 = P::make(svy[ka], cy), Z1 = P::make(svz[ka], cz);
                    if (pre) psum(X1, Y1, Z1, bx0, by0, bz0, bs0);
                    if (do_corr) psum(X1, Y1, Z1, sx, sy, sz, ss);
                }
            };
            // binary32: two pair slots of a thread at once, in the two lanes of packed
            // operations (the slot pairs i, i+1 are both full pairs except near the end)
            const V2 HP = P::make(T(0.5), T(0.5)), HN = P::make(T(-0.5), T(-0.5));
#pragma unroll
            for (int i = 0; i < PS; i += 2) {
                if constexpr (sizeof(T) == 4) {
                    const uint32_t p1 = tid + (uint32_t)(i + 1) * NT;
                    if (i + 1 < PS && 2u * p1 + 1u < n) {       // two full pairs: packed lanes
                        const uint32_t pk0 = reinterpret_cast<const uint32_t*>(sinv)[tid + (uint32_t)i * NT];
                        const uint32_t pk1 = reinterpret_cast<const uint32_t*>(sinv)[p1];
                        const uint32_t ka0 = pk0 & 0xFFFFu, kb0 = pk0 >> 16;
                        const uint32_t ka1 = pk1 & 0xFFFFu, kb1 = pk1 >> 16;
                        const uint32_t la0 = id_of(ka0), lb0 = id_of(kb0), la1 = id_of(ka1), lb1 = id_of(kb1);
                        V2 AX = P::make(svx[ka0], svx[ka1]), AY = P::make(svy[ka0], svy[ka1]);
                        V2 AZ = P::make(svz[ka0], svz[ka1]);
                        V2 BX = P::make(svx[kb0], svx[kb1]), BY = P::make(svy[kb0], svy[kb1]);
                        V2 BZ = P::make(svz[kb0], svz[kb1]);
                        if (pre) { psum(AX, AY, AZ, bx0, by0, bz0, bs0); psum(BX, BY, BZ, bx0, by0, bz0, bs0); }
                        const uint4 w0 = draw(a.keys, la0 < lb0 ? la0 : lb0, step, TAG_PAIR);
                        const uint4 w1 = draw(a.keys, la1 < lb1 ? la1 : lb1, step, TAG_PAIR);
                        V2 DX, DY, DZ;
                        ta_delta2(AX, AY, AZ, BX, BY, BZ, A, w0, w1, DX, DY, DZ);
                        AX = P::fma(HP, DX, AX); AY = P::fma(HP, DY, AY); AZ = P::fma(HP, DZ, AZ);
                        BX = P::fma(HN, DX, BX); BY = P::fma(HN, DY, BY); BZ = P::fma(HN, DZ, BZ);
                        svx[ka0] = AX.x; svy[ka0] = AY.x; svz[ka0] = AZ.x;
                        svx[ka1] = AX.y; svy[ka1] = AY.y; svz[ka1] = AZ.y;
                        svx[kb0] = BX.x; svy[kb0] = BY.x; svz[kb0] = BZ.x;
                        svx[kb1] = BX.y; svy[kb1] = BY.y; svz[kb1] = BZ.y;
                        if (do_corr) { psum(AX, AY, AZ, sx, sy, sz, ss); psum(BX, BY, BZ, sx, sy, sz, ss); }
                        continue;
                    }
                }
                slot(i);
                if (i + 1 < PS) slot(i + 1);
            }
            if (do_corr) {
                T acc[8] = {sx.x + sx.y, sy.x + sy.y, sz.x + sz.y, ss.x + ss.y,
                            bx0.x + bx0.y, by0.x + by0.y, bz0.x + bz0.y, bs0.x + bs0.y};
                if (pre_mom) {
                    T acc4[4] = {acc[0], acc[1], acc[2], acc[3]};
                    cluster_sum<NT, 1, 4, T>(acc4, s_redacc, s_cl, s_tot);
                } else {
                    cluster_sum<NT, 1, 8, T>(acc, s_redacc, s_cl, s_tot);
                }
                // x <- V0 + f (x - V1) = f x + (V0 - f V1) (as in the cluster kernel)
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
            }
        }
        if (tid == TK) {
            cp_async_wait_all();                           // the next cell's words, for the tables below
            // the next cell's run into L2 now, a whole cell's work before its bulk loads
            const uint4 nx = s_item[par ^ 1u];             // this thread's own copy, waited in step 3
            if (nx.w != 0u && nx.y != 0u) {
                const uint32_t nrs = s_run[par ^ 1u][0], nrl = min(s_run[par ^ 1u][1], nx.y);
                if (nrl) {
#pragma unroll
                    for (int c = 0; c < 3; ++c) prefetch_l2(gv[c] + nrs, (size_t)nrl * sizeof(T));
                }
            }
        }
        __syncthreads();
        pc.mark(7);
        fill_round_tables(par ^ 1u);                       // the next cell's round functions

        // ---- 5. one sweep of the home slots (16-byte vectors): the restoration, the largest
        // squared speed, and the moments of the result (S3a/S3b, Sec. 4.5) with the energy
        // histogram; the neutral step below corrects the sums of the particles it changes
        const bool restore = coul && do_corr;
        const T F = restore ? s_par[4] : T(1);
        const T OX = restore ? s_par[5] : T(0), OY = restore ? s_par[6] : T(0), OZ = restore ? s_par[7] : T(0);
        V2 mq[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) mq[k] = P::make(T(0), T(0));
        uint32_t* hsub = s_hist + ((tid >> 5) & 3u) * NBIN;
        const T half_m_over_e = a.c_half_m_over_e;
        const T e_ion = a.c_e_ion;
        constexpr bool xs_on = XS;                 // tables: the rate sums take sigma(E) |v|
        const T sg0 = a.c_sig_el, si0 = a.c_sig_ion;
        // one particle's contribution, into the first lane, with sign sg (+1 add, -1 remove)
        auto accum = [&](T x, T y, T z, T sg) {
            const T v2 = x * x + y * y + z * z;
            const T v = Math<T>::sqrt(v2);
            const T E = v2 * half_m_over_e;
            mq[0].x += sg * x; mq[1].x += sg * y; mq[2].x += sg * z;
            mq[3].x += sg * (x * x); mq[4].x += sg * (y * y); mq[5].x += sg * (z * z);
            if (!xs_on) {
                mq[6].x += sg * v;
                mq[7].x += E >= e_ion ? sg * v : T(0);
            } else {
                mq[6].x += sg * (xs_el<T>(a.xs, E, sg0) * v);
                mq[7].x += sg * (xs_ion<T>(a.xs, E, si0, e_ion) * v);
            }
            atomicAdd(&hsub[Math<T>::ebin(E)], sg > T(0) ? 1u : 0xFFFFFFFFu);
        };
        T vmax2 = T(0);
        const uint32_t nch = (o + n + (uint32_t)W - 1u) / (uint32_t)W;   // 16-byte chunks of slots
        for (uint32_t c4 = tid; c4 < nch; c4 += NT) {
            const uint32_t q0 = c4 * (uint32_t)W;
            T x[W], y[W], z[W];
            VW::ld(sv0 + q0, x);
            VW::ld(sv0 + PAD + q0, y);
            VW::ld(sv0 + 2 * PAD + q0, z);
            if (restore) {
#pragma unroll
                for (int e = 0; e < W; ++e) { x[e] = fma(F, x[e], OX); y[e] = fma(F, y[e], OY); z[e] = fma(F, z[e], OZ); }
                VW::st(sv0 + q0, x);
                VW::st(sv0 + PAD + q0, y);
                VW::st(sv0 + 2 * PAD + q0, z);
            }
#pragma unroll
            for (int e = 0; e + 1 < W; e += 2) {
                const uint32_t q = q0 + (uint32_t)e;
                const bool in0 = q >= o && q < o + n, in1 = q + 1u >= o && q + 1u < o + n;
                if (in0 && in1) {
                    const V2 X = P::make(x[e], x[e + 1]), Y = P::make(y[e], y[e + 1]), Z = P::make(z[e], z[e + 1]);
                    const V2 v2 = P::fma(Z, Z, P::fma(Y, Y, P::mul(X, X)));
                    vmax2 = fmax(vmax2, fmax(v2.x, v2.y));
                    const V2 V = P::make(Math<T>::sqrt(v2.x), Math<T>::sqrt(v2.y));
                    const V2 E = P::mul(v2, P::make(half_m_over_e, half_m_over_e));
                    P::acc(mq[0], X); P::acc(mq[1], Y); P::acc(mq[2], Z);
                    P::acc_sq(mq[3], X); P::acc_sq(mq[4], Y); P::acc_sq(mq[5], Z);
                    if (!xs_on) {
                        P::acc(mq[6], V);
                        P::acc(mq[7], P::make(E.x >= e_ion ? V.x : T(0), E.y >= e_ion ? V.y : T(0)));
                    } else {
                        P::acc(mq[6], P::make(xs_el<T>(a.xs, E.x, sg0) * V.x, xs_el<T>(a.xs, E.y, sg0) * V.y));
                        P::acc(mq[7], P::make(xs_ion<T>(a.xs, E.x, si0, e_ion) * V.x,
                                              xs_ion<T>(a.xs, E.y, si0, e_ion) * V.y));
                    }
                    atomicAdd(&hsub[Math<T>::ebin(E.x)], 1u);
                    atomicAdd(&hsub[Math<T>::ebin(E.y)], 1u);
                } else {
                    if (in0) {
                        vmax2 = fmax(vmax2, x[e] * x[e] + y[e] * y[e] + z[e] * z[e]);
                        accum(x[e], y[e], z[e], T(1));
                    }
                    if (in1) {
                        vmax2 = fmax(vmax2, x[e + 1] * x[e + 1] + y[e + 1] * y[e + 1] + z[e + 1] * z[e + 1]);
                        accum(x[e + 1], y[e + 1], z[e + 1], T(1));
                    }
                }
            }
        }

        // ---- 6. step S2a: the particles at pairing positions below n_c collide with neutrals
        uint32_t n_ion = 0u;
        if (do_neut) {
            {   // largest squared speed: warp butterfly, one shared atomicMax on the bit pattern
                T v = vmax2;
#pragma unroll
                for (int q = 16; q > 0; q >>= 1) v = fmax(v, __shfl_xor_sync(0xFFFFFFFFu, v, q));
                if ((tid & 31u) == 0u) atomicMax(&s_vmax, MaxBits<T>::to(v));
            }
            __syncthreads();
            const T md = MaxBits<T>::from(s_vmax);
            const T dtj = cell_scalar<T>(s_cp, 1);
            const T numax = a.c_nsig_tot * Math<T>::sqrt(md);
            const T pnull = -Math<T>::expm1(-numax * dtj);
            const uint32_t n_cand = cand_count<T>(pnull, n, bw[CPB_U]);
            const T nsel = a.c_nsig_el, nsion = a.c_nsig_ion, mr2 = a.c_mratio2;
            bool ionized = false;
            for (uint32_t q = tid; q < n_cand; q += NT) {
                const uint32_t k = sinv[q];
                const uint32_t l = id_of(k);
                const uint4 rw = draw(a.keys, l, step, TAG_PARTICLE);
                const T x = svx[k], y = svy[k], z = svz[k];
                const T v2 = x * x + y * y + z * z;
                const T v = Math<T>::sqrt(v2);
                const T E = v2 * half_m_over_e;
                const T nu_el = xs_on ? a.c_nn * xs_el<T>(a.xs, E, sg0) * v : nsel * v;
                const T nu_ion = xs_on ? a.c_nn * xs_ion<T>(a.xs, E, si0, e_ion) * v : E >= e_ion ? nsion * v : T(0);
                const T rr = unif<T>(rw.z) * numax;
                if (rr < nu_el) {                              // C1: elastic, cold heavy target
                    const uint4 sc = draw(a.keys, l, step, TAG_SCATTER);
                    T dx, dy, dz;
                    iso_dir<T>(sc.x, sc.y, dx, dy, dz);
                    const T cchi = (x * dx + y * dy + z * dz) * Math<T>::rcp(v);
                    const T vn = v * Math<T>::sqrt(T(1) - mr2 * (T(1) - cchi));
                    const T nx = vn * dx, ny = vn * dy, nz = vn * dz;
                    svx[k] = nx; svy[k] = ny; svz[k] = nz;
                    accum(x, y, z, T(-1));
                    accum(nx, ny, nz, T(1));
                } else if (rr < nu_el + nu_ion) {              // C2: ionization, resolved below
                    atomicOr(&s_imask[q >> 5], 1u << (q & 31u));
                    ionized = true;
                }
            }
            if (__syncthreads_or(ionized ? 1 : 0)) {
                const uint32_t nw = (n_cand + 31u) / 32u;
                uint32_t tot;
                const uint32_t wex = block_excl_scan<NT>(tid < nw ? (uint32_t)__popc(s_imask[tid]) : 0u, s_scan, &tot);
                if (tid < nw) s_ioff[tid] = wex;
                n_ion = tot;
                __syncthreads();
                const T two_e_over_m = a.c_two_e_over_m;
                for (uint32_t q = tid; q < n_cand; q += NT) {
                    const uint32_t mw = s_imask[q >> 5];
                    if (!(mw & (1u << (q & 31u)))) continue;
                    const uint32_t rank = s_ioff[q >> 5] + (uint32_t)__popc(mw & ((1u << (q & 31u)) - 1u));
                    const uint32_t k = sinv[q];
                    const uint32_t l = id_of(k);
                    const T x = svx[k], y = svy[k], z = svz[k];
                    const T E = (x * x + y * y + z * z) * half_m_over_e;
                    const uint4 sc = draw(a.keys, l, step, TAG_SCATTER);
                    const uint4 sd = draw(a.keys, l, step, TAG_SECONDARY);
                    // E was >= e_ion when the collision was decided; recomputed it can round
                    // one unit below, so the excess is clamped at zero
                    const T Ep = fmax(E - e_ion, T(0));
                    const T Es = unif<T>(sc.z) * Ep;
                    const T vp = Math<T>::sqrt(two_e_over_m * (Ep - Es)), vs = Math<T>::sqrt(two_e_over_m * Es);
                    T dx, dy, dz, ex2, ey2, ez2;
                    iso_dir<T>(sc.x, sc.y, dx, dy, dz);
                    iso_dir<T>(sd.x, sd.y, ex2, ey2, ez2);
                    const T px = vp * dx, py = vp * dy, pz = vp * dz;
                    svx[k] = px; svy[k] = py; svz[k] = pz;
                    const T sx = vs * ex2, sy = vs * ey2, sz = vs * ez2;
                    const uint32_t slot = s + rank;
                    a.stage_l[slot] = l;
                    a.stage_vx[slot] = sx; a.stage_vy[slot] = sy; a.stage_vz[slot] = sz;
                    accum(x, y, z, T(-1));
                    accum(px, py, pz, T(1));
                    accum(sx, sy, sz, T(1));
                }
            }
            if (tid == 0) a.ion_count[j] = n_ion;
        } else if (tid == 0) {
            a.ion_count[j] = 0u;
        }
        pc.mark(8);

        // ---- 7. the cell's sums (their barrier also orders every slot write before the stores)
        {
            T acc[8];
#pragma unroll
            for (int k = 0; k < 8; ++k) acc[k] = mq[k].x + mq[k].y;
            cluster_sum<NT, 1, 8, T>(acc, s_redacc, s_cl, s_tot);   // totals in warp 0
        }
        if (tid < (unsigned)NBIN) {
            a.hist[(size_t)j * NBIN + tid] = s_hist[tid] + s_hist[NBIN + tid] + s_hist[2 * NBIN + tid] +
                                             s_hist[3 * NBIN + tid];
        }
        if (tid == 0) {
            double* m = a.mom + (size_t)j * NMOM;
            const double N = (double)(n + n_ion);
            m[0] = N;
            m[1] = a.weight * N;
            m[2] = s_tot[0]; m[3] = s_tot[1]; m[4] = s_tot[2];
            m[5] = s_tot[3]; m[6] = s_tot[4]; m[7] = s_tot[5];
            m[8] = XS ? s_tot[6] : a.sigma_el * s_tot[6];
            m[9] = XS ? s_tot[7] : a.sigma_ion * s_tot[7];
        }
        pc.mark(9);

        // ---- 8. write-back: the run interior as three bulk stores (their reads of the slots are
        // waited at the next cell's start), the rest with plain stores
        if (tid == DM && bytes) {
            fence_proxy_async();
#pragma unroll
            for (int c = 0; c < 3; ++c) bulk_store(gv[c] + g0, sv0 + c * PAD + (g0 - rs + o), bytes);
            bulk_commit();
        }
        if (pk0 != 0xFFFFFFFFu) {
            gv[0][pl0] = sv0[pk0 + o]; gv[1][pl0] = sv0[PAD + pk0 + o]; gv[2][pl0] = sv0[2 * PAD + pk0 + o];
        }
        for (uint32_t t = tid + NT; t < nplain; t += NT) {
            const uint32_t k = plain_home(t);
            const uint32_t l = id_of(k);
#pragma unroll
            for (int c = 0; c < 3; ++c) gv[c][l] = sv0[c * PAD + k + o];
        }
        __syncthreads();
        pc.mark(10);
    }
    if (tid == DM) bulk_wait_all();
}

}  // namespace ltpc
