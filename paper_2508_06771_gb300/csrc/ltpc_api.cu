// ltpc_api.cu -- host runtime behind the C ABI of include/ltpc.h.
//
// The context carves the two caller-owned device buffers into the particle
// arrays and the work arrays, keeps the cluster-class table of the cell
// kernel, and enqueues one pass (scatter -> cell kernels -> regroup/append)
// per collision step on the caller's stream, optionally as a CUDA graph.
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/ltpc.h"
#include "ltpc_launch.h"

using namespace ltpc;

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr size_t kAlign = 256;

size_t align_up(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

struct Layout {
    size_t state = 0, work = 0;
    // state offsets
    size_t vx, vy, vz, cell, x;
    // work offsets
    size_t perm, counts, cell_start, cs_prev, cursor, ion_count, ion_off, stage_l, stage_vx, stage_vy,
        stage_vz, mom, hist, inv_vol, dt_factor, lnlam, cpar, run_start, run_len, aslot, accel, rec_count, xs, lists, ds,
        xg;
};

bool compute_layout(const ltpc_config* c, Layout* L)
{
    if (!c || c->n_cells <= 0 || c->capacity <= 0 || c->capacity > 0xFFFFFFFFll) return false;
    if (c->precision != LTPC_F32 && c->precision != LTPC_F64) return false;
    const size_t es = c->precision == LTPC_F32 ? 4 : 8;
    const size_t cap = (size_t)c->capacity, M = (size_t)c->n_cells;
    size_t o = 0;
    auto take = [&](size_t bytes) { size_t r = o; o = align_up(o + bytes); return r; };
    L->vx = take(cap * es);
    L->vy = take(cap * es);
    L->vz = take(cap * es);
    L->cell = take(cap * 4);
    L->x = c->has_position ? take(cap * es) : (size_t)-1;
    L->state = o;
    o = 0;
    L->perm = take(cap * 4);
    L->counts = take(M * 4);
    L->cell_start = take((M + 1) * 4);
    L->cs_prev = take((M + 1) * 4);
    L->cursor = take(M * 4);
    L->ion_count = take(M * 4);
    L->ion_off = take((M + 1) * 4);
    L->stage_l = take(cap * 4);
    L->stage_vx = take(cap * es);
    L->stage_vy = take(cap * es);
    L->stage_vz = take(cap * es);
    L->mom = take(M * NMOM * 8);
    L->hist = take(M * NBIN * 4);
    L->inv_vol = take(M * 8);
    L->dt_factor = take(M * 8);
    L->lnlam = take(M * 8);
    L->cpar = take(M * NCP * 8);
    L->run_start = take(M * 4);
    L->run_len = take(M * 4);
    L->aslot = take(cap * 4);
    L->accel = take(M * 8);
    L->rec_count = take(M * 4);
    L->xs = take((size_t)2 * XS_MAX_PIECES * 4 * (8 + 4));   // two tables, binary64 then binary32
    L->lists = take(M * 16 * MAX_CLASSES);
    L->ds = take(sizeof(DevState));
    // bijection mode: the cluster classes' exchange records, one per particle (16 bytes in
    // binary32, 32 in binary64)
    L->xg = c->pairing_mode == LTPC_PAIR_BIJECTION ? take(cap * 4 * es) : (size_t)-1;
    L->work = o;
    return true;
}

}  // namespace

struct ltpc_ctx {
    ltpc_config cfg;
    Layout L;
    cudaStream_t stream;
    cudaStream_t cap_stream = nullptr;   // private stream used only to capture graphs
    int device = 0, sms = 1;
    unsigned char* st = nullptr;   // d_state
    unsigned char* wk = nullptr;   // d_work
    size_t es = 4;
    DevState* ds = nullptr;
    int table = 0;
    RegroupLists lists;
    std::vector<int> kernel_idx;   // per class: index into the precision's kernel list
    std::vector<int> grid;         // per class: CTAs per launch
    const CellKernelEntry* kernels = nullptr;
    int n_kernels = 0;
    double coef0 = 0.0;
    bool correction = false;
    // graph of one fused step
    cudaGraphExec_t gexec = nullptr;
    uint32_t graph_flags = 0;
    int64_t next_step = -1;
    double cur_dt = std::nan("");
    // field and push (ltpc_set_field)
    bool field = false;
    double dx = 0.0;
    int32_t wall = LTPC_WALL_PERIODIC;
    // recombination C5 (ltpc_set_recombination)
    double k_rec = 0.0, de_rec = 0.0;
    // tabulated cross sections and selection (ltpc_set_cross_sections)
    XsArgs xs{};
    bool xs_tables = false;
    double sigma_max = 0.0;
    char cuda_err[256] = {0};

    template <class P> P* w(size_t off) const { return reinterpret_cast<P*>(wk + off); }
    template <class P> P* s(size_t off) const { return reinterpret_cast<P*>(st + off); }
};

namespace {

int fail_cuda(ltpc_ctx* c, cudaError_t e)
{
    if (c) std::snprintf(c->cuda_err, sizeof c->cuda_err, "%s", cudaGetErrorString(e));
    return LTPC_ECUDA;
}

#define CK(expr)                                        \
    do {                                                \
        cudaError_t _e = (expr);                        \
        if (_e != cudaSuccess) return fail_cuda(ctx, _e); \
    } while (0)

int set_table(ltpc_ctx* ctx, int table)
{
    const ClassTable* tabs = nullptr;
    const int nt = class_tables(ctx->cfg.precision, ctx->cfg.pairing_mode, &tabs);
    if (table < 0 || table >= nt) return LTPC_EINVAL;
    const ClassTable& T = tabs[table];
    ctx->table = table;
    ctx->kernel_idx.assign(T.kernel, T.kernel + T.n);
    ctx->grid.assign(T.n, 0);
    ctx->lists.n_classes = T.n;
    ctx->lists.cache_grouping = ctx->cfg.cache_grouping;
    ctx->lists.run_start = ctx->w<uint32_t>(ctx->L.run_start);
    ctx->lists.run_len = ctx->w<uint32_t>(ctx->L.run_len);
    ctx->lists.aslot = ctx->w<uint32_t>(ctx->L.aslot);
    ctx->lists.rec_count = ctx->w<uint32_t>(ctx->L.rec_count);
    for (int k = 0; k < MAX_CLASSES; ++k) {
        ctx->lists.max_n[k] = 0;
        ctx->lists.list[k] = ctx->w<uint4>(ctx->L.lists) + (size_t)k * ctx->cfg.n_cells;
    }
    for (int k = 0; k < T.n; ++k) {
        const CellKernelEntry& e = ctx->kernels[T.kernel[k]];
        ctx->lists.max_n[k] = (uint32_t)(e.shape.cluster * e.shape.threads * e.shape.items);
        int clusters = 0;
        cudaError_t err = e.occupancy(&clusters);
        if (err != cudaSuccess) return fail_cuda(ctx, err);
        if (clusters <= 0) return LTPC_EUNSUPPORTED;
        ctx->grid[k] = clusters * e.shape.cluster;
    }
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
    return LTPC_OK;
}

template <class T>
CellArgs<T> make_args(ltpc_ctx* ctx, uint32_t flags)
{
    CellArgs<T> a;
    const Layout& L = ctx->L;
    a.vx = ctx->s<T>(L.vx); a.vy = ctx->s<T>(L.vy); a.vz = ctx->s<T>(L.vz);
    a.n_cap = (uint32_t)ctx->cfg.capacity;
    a.perm = ctx->w<uint32_t>(L.perm);
    a.counts = ctx->w<uint32_t>(L.counts);
    a.cell_start = ctx->w<uint32_t>(L.cell_start);
    a.cpar = ctx->w<double>(L.cpar);
    a.mom = ctx->w<double>(L.mom);
    a.hist = ctx->w<uint32_t>(L.hist);
    a.ion_count = ctx->w<uint32_t>(L.ion_count);
    a.stage_l = ctx->w<uint32_t>(L.stage_l);
    a.stage_vx = ctx->w<T>(L.stage_vx); a.stage_vy = ctx->w<T>(L.stage_vy); a.stage_vz = ctx->w<T>(L.stage_vz);
    a.ds = ctx->ds;
    a.list = nullptr;
    a.cls = 0;
    a.flags = flags;
    a.seed = ctx->cfg.seed;
    a.keys = philox_keys(ctx->cfg.seed);
    a.coef0 = ctx->coef0;
    a.weight = ctx->cfg.weight;
    a.mass = ctx->cfg.mass;
    a.e_over_m = ctx->cfg.charge / ctx->cfg.mass;
    a.n_neutral = ctx->cfg.n_neutral;
    a.sigma_el = ctx->cfg.sigma_el;
    a.sigma_ion = ctx->cfg.sigma_ion;
    a.e_ion = ctx->cfg.e_ion;
    a.mratio2 = ctx->cfg.mass_neutral > 0 ? 2.0 * ctx->cfg.mass / ctx->cfg.mass_neutral : 0.0;
    a.c_half_m_over_e = (T)(0.5 * ctx->cfg.mass / ctx->cfg.charge);
    a.c_two_e_over_m = (T)(2.0 * ctx->cfg.charge / ctx->cfg.mass);
    a.c_nsig_el = (T)(ctx->cfg.n_neutral * ctx->cfg.sigma_el);
    a.c_nsig_ion = (T)(ctx->cfg.n_neutral * ctx->cfg.sigma_ion);
    a.c_nsig_tot = (T)(ctx->cfg.n_neutral * (ctx->xs_tables ? ctx->sigma_max : ctx->cfg.sigma_el + ctx->cfg.sigma_ion));
    a.c_nn = (T)ctx->cfg.n_neutral;
    a.c_sig_el = (T)ctx->cfg.sigma_el;
    a.c_sig_ion = (T)ctx->cfg.sigma_ion;
    a.xs = ctx->xs;
    a.c_e_ion = (T)ctx->cfg.e_ion;
    a.c_mratio2 = (T)a.mratio2;
    a.cell = ctx->s<int32_t>(L.cell);
    a.rec_count = ctx->w<uint32_t>(L.rec_count);
    a.c_de_rec = (T)ctx->de_rec;
    a.run_start = ctx->w<uint32_t>(L.run_start);
    a.run_len = ctx->w<uint32_t>(L.run_len);
    a.order_out = nullptr;
    a.xg = L.xg != (size_t)-1 ? (void*)ctx->w<unsigned char>(L.xg) : nullptr;
    a.phase_clk = nullptr;
    return a;
}

// Enqueue one pass: scatter (CCS3), the cell kernel per class, then the
// bookkeeping that appends secondaries and regroups for the next pass.
template <class T>
int enqueue_body(ltpc_ctx* ctx, uint32_t flags, bool advance, uint32_t* order_out, cudaStream_t s,
                 cudaEvent_t* ev, unsigned long long* phase_clk);

// With F_PUSH: the collisions (S1, S2a) and their appends, then steps S2b/S2c
// on every particle, CCS1-CCS2 of the new cells, and a pass of moments (S3 of
// the pushed particles in their new cells, which the next pass also starts from).
template <class T>
int enqueue_pass(ltpc_ctx* ctx, uint32_t flags, bool advance, uint32_t* order_out, cudaStream_t s,
                 cudaEvent_t* ev = nullptr, unsigned long long* phase_clk = nullptr)
{
    if (!(flags & F_PUSH) || !ctx->field) return enqueue_body<T>(ctx, flags & ~F_PUSH, advance, order_out, s, ev, phase_clk);
    const Layout& L = ctx->L;
    int rc = enqueue_body<T>(ctx, flags & ~F_PUSH, false, order_out, s, nullptr, phase_clk);
    if (rc) return rc;
    CK(launch_push<T>(ctx->s<T>(L.x), ctx->s<T>(L.vz), ctx->s<int32_t>(L.cell), ctx->w<double>(L.accel),
                      ctx->w<double>(L.cpar), ctx->cfg.n_cells, ctx->dx, ctx->wall == LTPC_WALL_ABSORB ? 1 : 0,
                      ctx->w<uint32_t>(L.run_len), ctx->ds, ctx->sms * 8, s));
    CK(cudaMemsetAsync(ctx->w<uint32_t>(L.counts), 0, (size_t)ctx->cfg.n_cells * 4, s));
    CK(launch_hist_step(ctx->s<int32_t>(L.cell), ctx->w<uint32_t>(L.counts), ctx->cfg.n_cells, ctx->ds, ctx->sms * 8, s));
    CK(launch_regroup(ctx->cfg.n_cells, ctx->w<uint32_t>(L.counts), ctx->w<uint32_t>(L.cell_start),
                      ctx->w<uint32_t>(L.cs_prev), ctx->w<uint32_t>(L.cursor), ctx->w<uint32_t>(L.ion_count),
                      ctx->w<uint32_t>(L.ion_off), ctx->lists, (unsigned long long)ctx->cfg.capacity, 0, 0, ctx->ds,
                      s));
    return enqueue_body<T>(ctx, 0u, advance, nullptr, s, nullptr, nullptr);
}

template <class T>
int enqueue_body(ltpc_ctx* ctx, uint32_t flags, bool advance, uint32_t* order_out, cudaStream_t s,
                 cudaEvent_t* ev, unsigned long long* phase_clk)
{
    const Layout& L = ctx->L;
    const int grid_stream = ctx->sms * 8;
    int ei = 0;
    auto mark = [&]() -> cudaError_t { return ev ? cudaEventRecord(ev[ei++], s) : cudaSuccess; };
    CK(mark());
    CellParamArgs cp = {};
    cp.counts = ctx->w<uint32_t>(L.counts);
    cp.mom = ctx->w<double>(L.mom);
    cp.inv_vol = ctx->w<double>(L.inv_vol);
    cp.dt_factor = ctx->w<double>(L.dt_factor);
    cp.lnlam = ctx->w<double>(L.lnlam);
    cp.cpar = ctx->w<double>(L.cpar);
    cp.coef0 = ctx->coef0;
    cp.weight = ctx->cfg.weight;
    cp.e_over_m = ctx->cfg.charge / ctx->cfg.mass;
    cp.lnl_nrl = ctx->cfg.lnlambda_mode == LTPC_LNL_NRL ? 1 : 0;
    cp.bijection = ctx->cfg.pairing_mode == LTPC_PAIR_BIJECTION ? 1 : 0;
    cp.k_rec = (flags & F_RECOMB) ? ctx->k_rec : 0.0;
    cp.keys = philox_keys(ctx->cfg.seed);
    CK(launch_scatter(ctx->s<int32_t>(L.cell), ctx->cfg.n_cells, ctx->w<uint32_t>(L.cursor), ctx->w<uint32_t>(L.perm), ctx->ds,
                      grid_stream, s, ctx->lists, ctx->w<uint32_t>(L.cell_start), &cp));
    CK(mark());
    CellArgs<T> a = make_args<T>(ctx, flags);
    a.order_out = order_out;
    a.phase_clk = phase_clk;
    for (int k = 0; k < ctx->lists.n_classes; ++k) {
        a.list = ctx->lists.list[k];
        a.cls = (uint32_t)k;
        const CellKernelEntry& e = ctx->kernels[ctx->kernel_idx[k]];
        auto fn = reinterpret_cast<cudaError_t (*)(const CellArgs<T>&, cudaStream_t, int)>(e.launcher);
        CK(fn(a, s, ctx->grid[k]));
        CK(mark());
    }
    CK(launch_regroup(ctx->cfg.n_cells, ctx->w<uint32_t>(L.counts), ctx->w<uint32_t>(L.cell_start),
                      ctx->w<uint32_t>(L.cs_prev), ctx->w<uint32_t>(L.cursor), ctx->w<uint32_t>(L.ion_count),
                      ctx->w<uint32_t>(L.ion_off), ctx->lists, (unsigned long long)ctx->cfg.capacity, 1,
                      advance ? 1 : 0, ctx->ds, s));
    CK(mark());
    CK(launch_append<T>(ctx->cfg.n_cells, ctx->w<uint32_t>(L.ion_off), ctx->w<uint32_t>(L.cs_prev),
                        ctx->w<uint32_t>(L.stage_l), ctx->w<T>(L.stage_vx), ctx->w<T>(L.stage_vy),
                        ctx->w<T>(L.stage_vz), ctx->s<T>(L.vx), ctx->s<T>(L.vy), ctx->s<T>(L.vz),
                        ctx->s<int32_t>(L.cell), ctx->cfg.has_position ? ctx->s<T>(L.x) : nullptr,
                        ctx->w<uint32_t>(L.aslot), ctx->ds, ctx->sms * 2, s));
    CK(mark());
    return LTPC_OK;
}

int enqueue(ltpc_ctx* ctx, uint32_t flags, bool advance, uint32_t* order_out = nullptr, cudaStream_t s = nullptr,
            cudaEvent_t* ev = nullptr, unsigned long long* phase_clk = nullptr)
{
    if (!s) s = ctx->stream;
    return ctx->cfg.precision == LTPC_F32 ? enqueue_pass<float>(ctx, flags, advance, order_out, s, ev, phase_clk)
                                          : enqueue_pass<double>(ctx, flags, advance, order_out, s, ev, phase_clk);
}

int set_state(ltpc_ctx* ctx, int64_t step, double dt)
{
    if (step < 0 || step > 0xFFFFFFFFll || !(std::isfinite(dt))) return LTPC_EINVAL;
    CK(launch_set_state(ctx->ds, 0ull, 0, (uint32_t)step, dt, 1, ctx->stream));
    return LTPC_OK;
}

uint32_t step_flags(const ltpc_ctx* ctx, bool coulomb, bool neutral)
{
    uint32_t f = 0;
    if (coulomb) {
        f |= F_COULOMB;
        if (ctx->correction) f |= F_CORRECTION;
        if (ctx->cfg.lnlambda_mode == LTPC_LNL_NRL) f |= F_LNL_NRL;
    }
    if (neutral && ctx->cfg.n_neutral > 0.0) f |= F_NEUTRAL;
    if (neutral && ctx->k_rec > 0.0) f |= F_RECOMB;
    if (ctx->field) f |= F_PUSH;
    return f;
}

int run_pass(ltpc_ctx* ctx, double dt, int64_t step, uint32_t flags)
{
    int rc = set_state(ctx, step, dt);
    if (rc) return rc;
    rc = enqueue(ctx, flags, true);
    if (rc) return rc;
    ctx->next_step = step + 1;
    ctx->cur_dt = dt;
    return LTPC_OK;
}

int map_err_bits(uint32_t bits)
{
    if (bits & ERR_INDEX) return LTPC_EINTERNAL;
    if (bits & ERR_CAPACITY) return LTPC_ECAPACITY;
    if (bits & ERR_NONFINITE) return LTPC_ENONFINITE;
    if (bits & (ERR_BAD_CELL | ERR_UNGROUPED)) return LTPC_EINVAL;
    if (bits & ERR_CELL_TOO_LARGE) return LTPC_EUNSUPPORTED;
    if (bits & ERR_TIMEOUT) return LTPC_ETIMEOUT;
    return LTPC_OK;
}

int read_errors(ltpc_ctx* ctx)
{
    CK(cudaStreamSynchronize(ctx->stream));
    uint32_t bits = 0;
    CK(cudaMemcpy(&bits, &ctx->ds->err, sizeof bits, cudaMemcpyDeviceToHost));
    if (bits) CK(cudaMemset(&ctx->ds->err, 0, sizeof bits));
    return map_err_bits(bits);
}

}  // namespace

// Class tables: index lists into the compiled shapes of each precision.
namespace ltpc {
static const ClassTable kTabF32[] = {
    {6, {0, 5, 6, 8, 9, 4}},   // one CTA per cell up to 12288 (256/512/1024 threads), clusters of 2 and 4
                               // 1024-thread CTAs up to 49152, then clusters of eight 512-thread CTAs
    {5, {0, 5, 6, 3, 4}},      // one CTA per cell up to 12288, then clusters of 8 (256/512 threads)
    {5, {0, 1, 2, 3, 4}},      // 256-thread CTAs in clusters of 1/2/4/8
    {2, {6, 4}},               // one 1024-thread CTA per cell up to 12288, then clusters of 8
    {5, {0, 5, 7, 3, 4}},      // as table 1 with 512-thread CTAs (24 positions per thread) up to 12288
};
static const ClassTable kTabF64[] = {
    {6, {0, 5, 6, 7, 3, 4}},   // one CTA per cell up to 6144, then clusters of 2/8
    {5, {0, 1, 2, 3, 4}},      // 256-thread CTAs in clusters of 1/2/4/8
};
// Bijection pairing mode: the key-sorted sizes (<= 4096) keep their classes;
// above them the home-order kernel takes what one CTA holds.
static const ClassTable kTabF32Bij[] = {
    {6, {0, 5, 10, 8, 9, 4}},  // home order up to 12288, then clusters of 2 and 4 1024-thread CTAs, 8 x 512
    {5, {0, 5, 10, 3, 4}},     // home order up to 12288, then clusters of 8 (256/512 threads)
    {6, {0, 5, 6, 8, 9, 4}},   // the cluster kernel (one CTA) up to 12288 instead of the home order
    {3, {5, 10, 4}},           // few classes: key sort up to 4096, home order up to 12288, clusters of 8
};
static const ClassTable kTabF64Bij[] = {
    {6, {0, 5, 8, 7, 3, 4}},   // home order up to 6144, then clusters of 2/8
    {6, {0, 5, 6, 7, 3, 4}},   // the cluster kernel up to 6144 instead of the home order
};
int class_tables(int precision, int pairing_mode, const ClassTable** out)
{
    const bool bij = pairing_mode == LTPC_PAIR_BIJECTION;
    if (precision == LTPC_F32) {
        *out = bij ? kTabF32Bij : kTabF32;
        return bij ? (int)(sizeof kTabF32Bij / sizeof kTabF32Bij[0]) : (int)(sizeof kTabF32 / sizeof kTabF32[0]);
    }
    *out = bij ? kTabF64Bij : kTabF64;
    return bij ? (int)(sizeof kTabF64Bij / sizeof kTabF64Bij[0]) : (int)(sizeof kTabF64 / sizeof kTabF64[0]);
}
}  // namespace ltpc

extern "C" {

const char* ltpc_strerror(int code)
{
    switch (code) {
    case LTPC_OK: return "ok";
    case LTPC_EINVAL: return "invalid argument";
    case LTPC_ECAPACITY: return "particle capacity exceeded";
    case LTPC_ECUDA: return "CUDA runtime error";
    case LTPC_ETIMEOUT: return "device wait timed out";
    case LTPC_ENONFINITE: return "non-finite velocity";
    case LTPC_EUNSUPPORTED: return "cell larger than the largest supported class";
    case LTPC_EINTERNAL: return "internal bounds check failed";
    default: return "unknown status";
    }
}

const char* ltpc_last_cuda_error(ltpc_ctx* ctx) { return ctx ? ctx->cuda_err : ""; }

int ltpc_required_bytes(const ltpc_config* cfg, size_t* state_bytes, size_t* work_bytes)
{
    Layout L;
    if (!compute_layout(cfg, &L) || !state_bytes || !work_bytes) return LTPC_EINVAL;
    *state_bytes = L.state;
    *work_bytes = L.work;
    return LTPC_OK;
}

int ltpc_create(ltpc_ctx** out, const ltpc_config* cfg, void* d_state, void* d_work, void* cuda_stream)
{
    if (!out) return LTPC_EINVAL;
    *out = nullptr;
    Layout L;
    if (!compute_layout(cfg, &L) || !d_state || !d_work) return LTPC_EINVAL;
    if (((uintptr_t)d_state | (uintptr_t)d_work) & (kAlign - 1)) return LTPC_EINVAL;
    if (!cfg->inv_volume || !(cfg->mass > 0) || !(cfg->charge > 0) || !(cfg->eps0 > 0) || !(cfg->weight > 0))
        return LTPC_EINVAL;
    if (cfg->lnlambda_mode != LTPC_LNL_CONST && cfg->lnlambda_mode != LTPC_LNL_NRL) return LTPC_EINVAL;
    if (cfg->cache_grouping != 0 && cfg->cache_grouping != 1) return LTPC_EINVAL;
    if (cfg->pairing_mode != LTPC_PAIR_KEY && cfg->pairing_mode != LTPC_PAIR_BIJECTION) return LTPC_EINVAL;
    for (int i = 0; i < 6; ++i)
        if (cfg->reserved[i]) return LTPC_EINVAL;
    ltpc_ctx* ctx = new (std::nothrow) ltpc_ctx();
    if (!ctx) return LTPC_EINVAL;
    ctx->cfg = *cfg;
    ctx->cfg.inv_volume = ctx->cfg.dt_factor = ctx->cfg.lnlambda = nullptr;
    ctx->L = L;
    ctx->stream = (cudaStream_t)cuda_stream;
    ctx->st = (unsigned char*)d_state;
    ctx->wk = (unsigned char*)d_work;
    ctx->es = cfg->precision == LTPC_F32 ? 4 : 8;
    ctx->ds = ctx->w<DevState>(L.ds);
    ctx->correction = cfg->correction < 0 ? cfg->precision == LTPC_F32 : cfg->correction != 0;
    const double mu = 0.5 * cfg->mass, q2 = cfg->charge * cfg->charge;
    ctx->coef0 = q2 * q2 * cfg->weight / (8.0 * kPi * cfg->eps0 * cfg->eps0 * mu * mu);
    int rc = LTPC_OK;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e != cudaSuccess) { fail_cuda(ctx, e); delete ctx; return LTPC_ECUDA; }
    ctx->n_kernels = cfg->precision == LTPC_F32 ? cell_kernels_f32(&ctx->kernels) : cell_kernels_f64(&ctx->kernels);
    const size_t M = (size_t)cfg->n_cells;
    std::vector<double> tmp(M);
    do {
        if ((e = cudaMemsetAsync(ctx->wk, 0, L.work, ctx->stream)) != cudaSuccess) break;
        if ((e = cudaMemcpyAsync(ctx->w<double>(L.inv_vol), cfg->inv_volume, M * 8, cudaMemcpyHostToDevice,
                                 ctx->stream)) != cudaSuccess) break;
        for (size_t j = 0; j < M; ++j) tmp[j] = cfg->dt_factor ? cfg->dt_factor[j] : 1.0;
        if ((e = cudaMemcpyAsync(ctx->w<double>(L.dt_factor), tmp.data(), M * 8, cudaMemcpyHostToDevice,
                                 ctx->stream)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) break;
        for (size_t j = 0; j < M; ++j) tmp[j] = cfg->lnlambda ? cfg->lnlambda[j] : 10.0;
        if ((e = cudaMemcpyAsync(ctx->w<double>(L.lnlam), tmp.data(), M * 8, cudaMemcpyHostToDevice,
                                 ctx->stream)) != cudaSuccess) break;
        if ((e = cudaStreamSynchronize(ctx->stream)) != cudaSuccess) break;
    } while (0);
    if (e != cudaSuccess) { fail_cuda(ctx, e); delete ctx; return LTPC_ECUDA; }
    rc = set_table(ctx, 0);
    if (rc) { delete ctx; return rc; }
    *out = ctx;
    return LTPC_OK;
}

void ltpc_destroy(ltpc_ctx* ctx)
{
    if (!ctx) return;
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
    delete ctx;
}

int ltpc_load_particles(ltpc_ctx* ctx, int64_t n, const int32_t* cell, const void* x, const void* vx,
                        const void* vy, const void* vz, int flags)
{
    if (!ctx || n < 0 || n > ctx->cfg.capacity) return LTPC_EINVAL;
    const bool bin = !cell && ctx->field && ctx->cfg.has_position && x;   // cell = floor(x / dx)
    if (n > 0 && ((!cell && !bin) || !vx || !vy || !vz)) return LTPC_EINVAL;
    if (flags & ~(LTPC_LOAD_SRC_DEVICE | LTPC_LOAD_ASYNC)) return LTPC_EINVAL;
    const bool async = (flags & LTPC_LOAD_ASYNC) != 0;
    const Layout& L = ctx->L;
    cudaStream_t s = ctx->stream;
    const cudaMemcpyKind kind = (flags & LTPC_LOAD_SRC_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    const size_t nb = (size_t)n * ctx->es;
    if (n > 0) {
        CK(cudaMemcpyAsync(ctx->st + L.vx, vx, nb, kind, s));
        CK(cudaMemcpyAsync(ctx->st + L.vy, vy, nb, kind, s));
        CK(cudaMemcpyAsync(ctx->st + L.vz, vz, nb, kind, s));
        if (cell) CK(cudaMemcpyAsync(ctx->st + L.cell, cell, (size_t)n * 4, kind, s));
        if (ctx->cfg.has_position && x) CK(cudaMemcpyAsync(ctx->st + L.x, x, nb, kind, s));
    }
    CK(launch_set_state(ctx->ds, (unsigned long long)n, 1, 0u, 0.0, 0, s));
    if (bin && n > 0) {
        if (ctx->cfg.precision == LTPC_F32)
            CK(launch_bin<float>(ctx->s<float>(L.x), ctx->s<int32_t>(L.cell), ctx->cfg.n_cells, ctx->dx, ctx->ds,
                                 ctx->sms * 4, s));
        else
            CK(launch_bin<double>(ctx->s<double>(L.x), ctx->s<int32_t>(L.cell), ctx->cfg.n_cells, ctx->dx, ctx->ds,
                                  ctx->sms * 4, s));
    }
    CK(cudaMemsetAsync(ctx->w<uint32_t>(L.counts), 0, (size_t)ctx->cfg.n_cells * 4, s));
    CK(cudaMemsetAsync(ctx->w<uint32_t>(L.ion_count), 0, (size_t)ctx->cfg.n_cells * 4, s));
    CK(cudaMemsetAsync(&ctx->ds->err, 0, 4, s));
    CK(launch_hist(ctx->s<int32_t>(L.cell), ctx->w<uint32_t>(L.counts), ctx->cfg.n_cells, ctx->ds, ctx->sms * 8, s));
    if (ctx->cfg.precision == LTPC_F32)
        CK(launch_check_finite<float>(ctx->s<float>(L.vx), ctx->s<float>(L.vy), ctx->s<float>(L.vz), ctx->ds,
                                      ctx->sms * 4, s));
    else
        CK(launch_check_finite<double>(ctx->s<double>(L.vx), ctx->s<double>(L.vy), ctx->s<double>(L.vz), ctx->ds,
                                       ctx->sms * 4, s));
    int rc = async ? LTPC_OK : read_errors(ctx);
    if (rc) return rc;
    CK(launch_runs(ctx->s<int32_t>(L.cell), ctx->cfg.n_cells, ctx->w<uint32_t>(L.counts), ctx->lists, ctx->ds,
                   ctx->sms * 8, s, ctx->cfg.pairing_mode == LTPC_PAIR_BIJECTION ? 1 : 0));
    CK(launch_regroup(ctx->cfg.n_cells, ctx->w<uint32_t>(L.counts), ctx->w<uint32_t>(L.cell_start),
                      ctx->w<uint32_t>(L.cs_prev), ctx->w<uint32_t>(L.cursor), ctx->w<uint32_t>(L.ion_count),
                      ctx->w<uint32_t>(L.ion_off), ctx->lists, (unsigned long long)ctx->cfg.capacity, 0, 0, ctx->ds,
                      s));
    // moments of the loaded state (a pass without collisions)
    rc = enqueue(ctx, 0u, false);
    if (rc) return rc;
    ctx->next_step = -1;
    return async ? LTPC_OK : read_errors(ctx);
}

int ltpc_set_field(ltpc_ctx* ctx, double dx, const double* accel, int32_t boundary)
{
    if (!ctx || !(dx > 0.0) || !std::isfinite(dx) || !accel) return LTPC_EINVAL;
    if (boundary != LTPC_WALL_PERIODIC && boundary != LTPC_WALL_ABSORB) return LTPC_EINVAL;
    if (!ctx->cfg.has_position || ctx->cfg.pairing_mode != LTPC_PAIR_KEY) return LTPC_EINVAL;
    const size_t M = (size_t)ctx->cfg.n_cells;
    for (size_t j = 0; j < M; ++j)
        if (!std::isfinite(accel[j])) return LTPC_EINVAL;
    CK(cudaMemcpyAsync(ctx->w<double>(ctx->L.accel), accel, M * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->field = true;
    ctx->dx = dx;
    ctx->wall = boundary;
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
    return LTPC_OK;
}

int ltpc_set_recombination(ltpc_ctx* ctx, double k_rec, double de_rec)
{
    if (!ctx || !(k_rec >= 0.0) || !std::isfinite(k_rec) || !(de_rec >= 0.0) || !std::isfinite(de_rec))
        return LTPC_EINVAL;
    if (k_rec > 0.0 && ctx->cfg.pairing_mode != LTPC_PAIR_KEY) return LTPC_EINVAL;
    ctx->k_rec = k_rec;
    ctx->de_rec = de_rec;
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
    return LTPC_OK;
}

namespace {

// Host value of one table: the same steps as the device's binary64 evaluator.
double xs_host(const ltpc_xsec& t, double E)
{
    if (!(E > 0.0)) return t.zero_below ? 0.0 : t.coef[0];
    const double u = (std::log(E) - t.lnE0) / t.h;
    if (u < 0.0) return t.zero_below ? 0.0 : t.coef[0];
    const double fi = std::floor(u);
    int32_t i = (int32_t)fi;
    double x;
    if (i >= t.pieces) { i = t.pieces - 1; x = 1.0; }
    else x = u - fi;
    const double* c = t.coef + 4 * (size_t)i;
    return c[0] + x * (c[1] + x * (c[2] + x * c[3]));
}

bool xs_valid(const ltpc_xsec* t)
{
    if (!t) return true;
    if (t->pieces < 1 || t->pieces > XS_MAX_PIECES || (t->zero_below != 0 && t->zero_below != 1) || !t->coef)
        return false;
    if (!std::isfinite(t->lnE0) || !(t->h > 0.0) || !std::isfinite(t->h)) return false;
    for (int i = 0; i < 4 * t->pieces; ++i)
        if (!std::isfinite(t->coef[i])) return false;
    return true;
}

}  // namespace

int ltpc_set_cross_sections(ltpc_ctx* ctx, const ltpc_xsec* el, const ltpc_xsec* ion, double sigma_max,
                            int32_t selection)
{
    if (!ctx || !xs_valid(el) || !xs_valid(ion)) return LTPC_EINVAL;
    if (selection != LTPC_SELECT_NULL && selection != LTPC_SELECT_PER_PARTICLE) return LTPC_EINVAL;
    if (selection == LTPC_SELECT_PER_PARTICLE && ctx->cfg.pairing_mode != LTPC_PAIR_KEY) return LTPC_EINVAL;
    const bool tables = el || ion;
    if (tables && (!(sigma_max > 0.0) || !std::isfinite(sigma_max))) return LTPC_EINVAL;
    // sample both tables (32 points per piece of each, and its knots): no negative
    // value, no sum above sigma_max
    const ltpc_xsec* tabs[2] = {el, ion};
    for (const ltpc_xsec* t : tabs) {
        if (!t) continue;
        for (int i = 0; i <= 32 * t->pieces; ++i) {
            const double E = std::exp(t->lnE0 + t->h * (double)i / 32.0);
            const double se = el ? xs_host(*el, E) : ctx->cfg.sigma_el;
            const double si = ion ? xs_host(*ion, E) : (E >= ctx->cfg.e_ion ? ctx->cfg.sigma_ion : 0.0);
            if (!(se >= 0.0) || !(si >= 0.0) || se + si > sigma_max) return LTPC_EINVAL;
        }
    }
    XsArgs x{};
    x.on = tables || selection == LTPC_SELECT_PER_PARTICLE;
    x.per_particle = selection == LTPC_SELECT_PER_PARTICLE;
    double* dd = ctx->w<double>(ctx->L.xs);
    float* df = reinterpret_cast<float*>(dd + 2 * XS_MAX_PIECES * 4);
    std::vector<double> hd(2 * XS_MAX_PIECES * 4, 0.0);
    std::vector<float> hf(2 * XS_MAX_PIECES * 4, 0.0f);
    for (int k = 0; k < 2; ++k) {
        XsTable& T = k == 0 ? x.el : x.ion;
        const ltpc_xsec* t = tabs[k];
        T.cd = dd + k * XS_MAX_PIECES * 4;
        T.cf = df + k * XS_MAX_PIECES * 4;
        if (!t) continue;
        T.pieces = t->pieces;
        T.zero_below = t->zero_below;
        T.lnE0 = t->lnE0;
        T.h = t->h;
        T.lnE0f = (float)t->lnE0;
        T.inv_hf = (float)(1.0 / t->h);
        for (int i = 0; i < 4 * t->pieces; ++i) {
            hd[k * XS_MAX_PIECES * 4 + i] = t->coef[i];
            hf[k * XS_MAX_PIECES * 4 + i] = (float)t->coef[i];
        }
    }
    CK(cudaMemcpyAsync(dd, hd.data(), hd.size() * 8, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(df, hf.data(), hf.size() * 4, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    ctx->xs = x;
    ctx->xs_tables = tables;
    ctx->sigma_max = tables ? sigma_max : 0.0;
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
    return LTPC_OK;
}

int ltpc_push(ltpc_ctx* ctx, double dt, int64_t step)
{
    if (!ctx || !ctx->field) return LTPC_EINVAL;
    return run_pass(ctx, dt, step, F_PUSH);
}

int ltpc_collide_coulomb(ltpc_ctx* ctx, double dt, int64_t step)
{
    if (!ctx) return LTPC_EINVAL;
    return run_pass(ctx, dt, step, step_flags(ctx, true, false) & ~F_PUSH);
}

int ltpc_collide_neutral(ltpc_ctx* ctx, double dt, int64_t step)
{
    if (!ctx) return LTPC_EINVAL;
    return run_pass(ctx, dt, step, step_flags(ctx, false, true) & ~F_PUSH);
}

int ltpc_step(ltpc_ctx* ctx, double dt, int64_t step)
{
    if (!ctx) return LTPC_EINVAL;
    const uint32_t flags = step_flags(ctx, true, true);
    if (!ctx->cfg.use_graph) return run_pass(ctx, dt, step, flags);
    if (step != ctx->next_step || dt != ctx->cur_dt) {
        int rc = set_state(ctx, step, dt);
        if (rc) return rc;
    }
    if (!ctx->gexec || ctx->graph_flags != flags) {
        if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
        // Capture on the context's private stream (the caller's stream may be the
        // legacy default stream, which cannot be captured); replay on the caller's.
        cudaGraph_t g = nullptr;
        if (!ctx->cap_stream) CK(cudaStreamCreateWithFlags(&ctx->cap_stream, cudaStreamNonBlocking));
        CK(cudaStreamBeginCapture(ctx->cap_stream, cudaStreamCaptureModeThreadLocal));
        int rc = enqueue(ctx, flags, true, nullptr, ctx->cap_stream);
        cudaError_t e = cudaStreamEndCapture(ctx->cap_stream, &g);
        if (rc) { if (g) cudaGraphDestroy(g); return rc; }
        if (e != cudaSuccess) return fail_cuda(ctx, e);
        e = cudaGraphInstantiate(&ctx->gexec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return fail_cuda(ctx, e);
        ctx->graph_flags = flags;
    }
    CK(cudaGraphLaunch(ctx->gexec, ctx->stream));
    ctx->next_step = step + 1;
    ctx->cur_dt = dt;
    return LTPC_OK;
}

int ltpc_profile_step(ltpc_ctx* ctx, double dt, int64_t step, float* ms, int32_t capacity, int32_t* n_out)
{
    if (!ctx || !ms || !n_out) return LTPC_EINVAL;
    const int nk = ctx->lists.n_classes + 3;   // scatter, classes..., regroup, append
    if (capacity < nk) return LTPC_EINVAL;
    cudaEvent_t ev[MAX_CLASSES + 4];
    int made = 0, rc = LTPC_OK;
    for (; made < nk + 1; ++made) {
        cudaError_t e = cudaEventCreate(&ev[made]);
        if (e != cudaSuccess) { rc = fail_cuda(ctx, e); break; }
    }
    if (rc == LTPC_OK) rc = set_state(ctx, step, dt);
    if (rc == LTPC_OK) rc = enqueue(ctx, step_flags(ctx, true, true) & ~F_PUSH, true, nullptr, ctx->stream, ev);
    if (rc == LTPC_OK) {
        cudaError_t e = cudaEventSynchronize(ev[nk]);
        for (int k = 0; k < nk && e == cudaSuccess; ++k) e = cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]);
        if (e != cudaSuccess) rc = fail_cuda(ctx, e);
        ctx->next_step = step + 1;
        ctx->cur_dt = dt;
    }
    for (int k = 0; k < made; ++k) cudaEventDestroy(ev[k]);
    *n_out = nk;
    return rc;
}

int ltpc_profile_phases(ltpc_ctx* ctx, double dt, int64_t step, unsigned long long* d_cycles)
{
    if (!ctx || !d_cycles) return LTPC_EINVAL;
    CK(cudaMemsetAsync(d_cycles, 0, 16 * sizeof(unsigned long long), ctx->stream));
    int rc = set_state(ctx, step, dt);
    if (rc == LTPC_OK) rc = enqueue(ctx, step_flags(ctx, true, true) & ~F_PUSH, true, nullptr, ctx->stream, nullptr, d_cycles);
    ctx->next_step = step + 1;
    ctx->cur_dt = dt;
    return rc;
}

int ltpc_run(ltpc_ctx* ctx, double dt, int64_t step0, int64_t nsteps)
{
    if (!ctx || nsteps < 0) return LTPC_EINVAL;
    for (int64_t k = 0; k < nsteps; ++k) {
        int rc = ltpc_step(ctx, dt, step0 + k);
        if (rc) return rc;
    }
    return LTPC_OK;
}

int ltpc_moments(ltpc_ctx* ctx, double* mom, uint32_t* hist, int dst_is_device)
{
    if (!ctx) return LTPC_EINVAL;
    const size_t M = (size_t)ctx->cfg.n_cells;
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    if (mom) CK(cudaMemcpyAsync(mom, ctx->w<double>(ctx->L.mom), M * NMOM * 8, kind, ctx->stream));
    if (hist) CK(cudaMemcpyAsync(hist, ctx->w<uint32_t>(ctx->L.hist), M * NBIN * 4, kind, ctx->stream));
    if (!dst_is_device) CK(cudaStreamSynchronize(ctx->stream));
    return LTPC_OK;
}

int ltpc_set_moments(ltpc_ctx* ctx, const double* mom, const uint32_t* hist, int src_is_device)
{
    if (!ctx || !mom) return LTPC_EINVAL;
    const size_t M = (size_t)ctx->cfg.n_cells;
    const cudaMemcpyKind kind = src_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CK(cudaMemcpyAsync(ctx->w<double>(ctx->L.mom), mom, M * NMOM * 8, kind, ctx->stream));
    if (hist) CK(cudaMemcpyAsync(ctx->w<uint32_t>(ctx->L.hist), hist, M * NBIN * 4, kind, ctx->stream));
    if (!src_is_device) CK(cudaStreamSynchronize(ctx->stream));
    return LTPC_OK;
}

int ltpc_read_particles(ltpc_ctx* ctx, void* vx, void* vy, void* vz, int32_t* cell, void* x, int64_t* n_out,
                        int dst_is_device)
{
    if (!ctx) return LTPC_EINVAL;
    int rc = read_errors(ctx);
    unsigned long long n = 0;
    CK(cudaMemcpy(&n, &ctx->ds->n, sizeof n, cudaMemcpyDeviceToHost));
    if (n_out) *n_out = (int64_t)n;
    const cudaMemcpyKind kind = dst_is_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    const size_t nb = (size_t)n * ctx->es;
    const Layout& L = ctx->L;
    if (n) {
        if (vx) CK(cudaMemcpyAsync(vx, ctx->st + L.vx, nb, kind, ctx->stream));
        if (vy) CK(cudaMemcpyAsync(vy, ctx->st + L.vy, nb, kind, ctx->stream));
        if (vz) CK(cudaMemcpyAsync(vz, ctx->st + L.vz, nb, kind, ctx->stream));
        if (cell) CK(cudaMemcpyAsync(cell, ctx->st + L.cell, (size_t)n * 4, kind, ctx->stream));
        if (x && ctx->cfg.has_position) CK(cudaMemcpyAsync(x, ctx->st + L.x, nb, kind, ctx->stream));
    }
    CK(cudaStreamSynchronize(ctx->stream));
    return rc;
}

int ltpc_sync(ltpc_ctx* ctx)
{
    if (!ctx) return LTPC_EINVAL;
    return read_errors(ctx);
}

int ltpc_pair_order(ltpc_ctx* ctx, int64_t step, uint32_t* d_order, uint32_t* d_cell_start)
{
    if (!ctx || !d_order) return LTPC_EINVAL;
    const double dt = std::isfinite(ctx->cur_dt) ? ctx->cur_dt : 0.0;
    int rc = set_state(ctx, step, dt);
    if (rc) return rc;
    if (d_cell_start)
        CK(cudaMemcpyAsync(d_cell_start, ctx->w<uint32_t>(ctx->L.cell_start), ((size_t)ctx->cfg.n_cells + 1) * 4,
                           cudaMemcpyDeviceToDevice, ctx->stream));
    rc = enqueue(ctx, 0u, false, d_order);
    ctx->next_step = -1;
    return rc;
}

int ltpc_compact(ltpc_ctx* ctx)
{
    if (!ctx) return LTPC_EINVAL;
    int rc = read_errors(ctx);
    if (rc) return rc;
    const Layout& L = ctx->L;
    const int32_t M = ctx->cfg.n_cells;
    cudaStream_t s = ctx->stream;
    // the grouping of the current particles (CCS3 into perm), then the cursors back
    CK(launch_scatter(ctx->s<int32_t>(L.cell), M, ctx->w<uint32_t>(L.cursor), ctx->w<uint32_t>(L.perm), ctx->ds,
                      ctx->sms * 8, s, ctx->lists, ctx->w<uint32_t>(L.cell_start)));
    CK(launch_reset_cursors(M, ctx->w<uint32_t>(L.cell_start), ctx->lists, ctx->w<uint32_t>(L.cursor), s));
    uint32_t ng = 0;
    CK(cudaMemcpyAsync(&ng, ctx->w<uint32_t>(L.cell_start) + M, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    const uint32_t* perm = ctx->w<uint32_t>(L.perm);
    int32_t* dcell = reinterpret_cast<int32_t*>(ctx->w<uint32_t>(L.stage_l));
    const int grid = ctx->sms * 8;
    auto gather = [&](auto tag) -> int {
        using T = decltype(tag);
        T* b0 = ctx->w<T>(L.stage_vx);
        T* b1 = ctx->w<T>(L.stage_vy);
        T* b2 = ctx->w<T>(L.stage_vz);
        if (ctx->cfg.has_position) {                      // positions first, in place through the stage
            CK(launch_compact_gather<T>(perm, ng, ctx->s<T>(L.x), nullptr, nullptr, nullptr, b0, nullptr, nullptr,
                                        nullptr, grid, s));
            CK(cudaMemcpyAsync(ctx->st + L.x, b0, (size_t)ng * sizeof(T), cudaMemcpyDeviceToDevice, s));
        }
        CK(launch_compact_gather<T>(perm, ng, ctx->s<T>(L.vx), ctx->s<T>(L.vy), ctx->s<T>(L.vz),
                                    ctx->s<int32_t>(L.cell), b0, b1, b2, dcell, grid, s));
        // the compacted particles loaded from the stage: counts, runs, grouping, moments
        return ltpc_load_particles(ctx, (int64_t)ng, dcell, nullptr, b0, b1, b2,
                                   LTPC_LOAD_SRC_DEVICE | LTPC_LOAD_ASYNC);
    };
    return ctx->cfg.precision == LTPC_F32 ? gather(float{}) : gather(double{});
}

int ltpc_grouping(ltpc_ctx* ctx, uint32_t* d_cell_start, uint32_t* d_perm, uint32_t* d_counts)
{
    if (!ctx) return LTPC_EINVAL;
    const size_t M = (size_t)ctx->cfg.n_cells;
    // the grouping of the current particles: redo CCS3 into perm
    CK(launch_scatter(ctx->s<int32_t>(ctx->L.cell), ctx->cfg.n_cells, ctx->w<uint32_t>(ctx->L.cursor), ctx->w<uint32_t>(ctx->L.perm),
                      ctx->ds, ctx->sms * 8, ctx->stream, ctx->lists, ctx->w<uint32_t>(ctx->L.cell_start)));
    // restore the cursors for the next pass
    CK(launch_reset_cursors(ctx->cfg.n_cells, ctx->w<uint32_t>(ctx->L.cell_start), ctx->lists,
                            ctx->w<uint32_t>(ctx->L.cursor), ctx->stream));
    if (d_cell_start)
        CK(cudaMemcpyAsync(d_cell_start, ctx->w<uint32_t>(ctx->L.cell_start), (M + 1) * 4, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    if (d_counts)
        CK(cudaMemcpyAsync(d_counts, ctx->w<uint32_t>(ctx->L.counts), M * 4, cudaMemcpyDeviceToDevice, ctx->stream));
    if (d_perm) {
        unsigned long long n = 0;
        CK(cudaStreamSynchronize(ctx->stream));
        CK(cudaMemcpy(&n, &ctx->ds->n, sizeof n, cudaMemcpyDeviceToHost));
        CK(cudaMemcpyAsync(d_perm, ctx->w<uint32_t>(ctx->L.perm), (size_t)n * 4, cudaMemcpyDeviceToDevice,
                           ctx->stream));
    }
    return LTPC_OK;
}

int ltpc_classes(ltpc_ctx* ctx, int32_t* n_classes, int32_t* cluster, int32_t* threads, int32_t* per_cta,
                 int32_t* max_n)
{
    if (!ctx || !n_classes) return LTPC_EINVAL;
    *n_classes = ctx->lists.n_classes;
    for (int k = 0; k < ctx->lists.n_classes; ++k) {
        const CellShape& sh = ctx->kernels[ctx->kernel_idx[k]].shape;
        if (cluster) cluster[k] = sh.cluster;
        if (threads) threads[k] = sh.threads;
        if (per_cta) per_cta[k] = sh.threads * sh.items;
        if (max_n) max_n[k] = (int32_t)ctx->lists.max_n[k];
    }
    return LTPC_OK;
}

int ltpc_set_class_table(ltpc_ctx* ctx, int32_t table)
{
    if (!ctx) return LTPC_EINVAL;
    int rc = read_errors(ctx);
    if (rc) return rc;
    rc = set_table(ctx, table);
    if (rc) return rc;
    // rebuild the class lists for the current counts
    CK(launch_regroup(ctx->cfg.n_cells, ctx->w<uint32_t>(ctx->L.counts), ctx->w<uint32_t>(ctx->L.cell_start),
                      ctx->w<uint32_t>(ctx->L.cs_prev), ctx->w<uint32_t>(ctx->L.cursor),
                      ctx->w<uint32_t>(ctx->L.ion_count), ctx->w<uint32_t>(ctx->L.ion_off), ctx->lists,
                      (unsigned long long)ctx->cfg.capacity, 0, 0, ctx->ds, ctx->stream));
    return read_errors(ctx);
}

// Views used by the surrogate (k_mlp.cu); not part of the public header.
int ltpc_internal_moments_view(ltpc_ctx* ctx, const double** mom, const uint32_t** hist, const double** inv_vol,
                               int32_t* M, double* weight, double* half_m_over_e, cudaStream_t* stream)
{
    if (!ctx) return LTPC_EINVAL;
    *mom = ctx->w<double>(ctx->L.mom);
    *hist = ctx->w<uint32_t>(ctx->L.hist);
    *inv_vol = ctx->w<double>(ctx->L.inv_vol);
    *M = ctx->cfg.n_cells;
    *weight = ctx->cfg.weight;
    *half_m_over_e = 0.5 * ctx->cfg.mass / ctx->cfg.charge;
    *stream = ctx->stream;
    return LTPC_OK;
}

int ltpc_internal_particles_view(ltpc_ctx* ctx, const void** vx, const void** vy, const void** vz, const int32_t** cell,
                                 const uint32_t** counts, unsigned long long* n, int* precision, uint64_t* seed,
                                 double* sig_el, double* sig_ion, double* e_ion)
{
    if (!ctx) return LTPC_EINVAL;
    int rc = read_errors(ctx);
    if (rc) return rc;
    if (cudaMemcpy(n, &ctx->ds->n, sizeof *n, cudaMemcpyDeviceToHost) != cudaSuccess) return LTPC_ECUDA;
    *vx = ctx->st + ctx->L.vx; *vy = ctx->st + ctx->L.vy; *vz = ctx->st + ctx->L.vz;
    *cell = ctx->s<int32_t>(ctx->L.cell);
    *counts = ctx->w<uint32_t>(ctx->L.counts);
    *precision = ctx->cfg.precision;
    *seed = ctx->cfg.seed;
    *sig_el = ctx->cfg.sigma_el; *sig_ion = ctx->cfg.sigma_ion; *e_ion = ctx->cfg.e_ion;
    return LTPC_OK;
}

int ltpc_internal_xs_view(ltpc_ctx* ctx, XsArgs* xs)
{
    if (!ctx || !xs) return LTPC_EINVAL;
    *xs = ctx->xs;
    return LTPC_OK;
}

int ltpc_autotune(ltpc_ctx* ctx, double dt, int32_t* chosen_table)
{
    (void)dt;
    if (!ctx) return LTPC_EINVAL;
    const ClassTable* tabs = nullptr;
    const int nt = class_tables(ctx->cfg.precision, ctx->cfg.pairing_mode, &tabs);
    // Time a collision-free pass per table: it exercises the same grouping,
    // ordering, staging and reduction work without changing the particles.
    float best = 1e30f;
    int best_t = ctx->table;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    for (int t = 0; t < nt; ++t) {
        int rc = ltpc_set_class_table(ctx, t);
        if (rc) continue;
        rc = enqueue(ctx, 0u, false);
        if (rc) return rc;
        CK(cudaEventRecord(e0, ctx->stream));
        for (int r = 0; r < 3; ++r) {
            rc = enqueue(ctx, 0u, false);
            if (rc) return rc;
        }
        CK(cudaEventRecord(e1, ctx->stream));
        CK(cudaEventSynchronize(e1));
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, e0, e1));
        if (ms < best) { best = ms; best_t = t; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    int rc = ltpc_set_class_table(ctx, best_t);
    if (chosen_table) *chosen_table = best_t;
    return rc;
}

}  // extern "C"
