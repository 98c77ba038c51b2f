/*
 * ltpc.h -- C ABI of the GB300 collision core for collisional-plasma PIC
 * (Almgren-Bell, Al Awar, Geethakrishnan, Gligoric, Biros, "A Portable
 * Multi-GPU Solver for Collisional Plasmas with Coulombic Interactions",
 * arXiv 2508.06771).
 *
 * The library implements, on one GPU, the particle side of one PIC step of
 * Table 2 of the paper:
 *   S1   electron-electron Coulomb collisions, Takizuka-Abe binary model over
 *        a per-cell random pairing (Sec. 4.4, Table 5, CCS1-CCS5);
 *   S2a  electron-neutral elastic (C1) and ionization (C2) collisions with the
 *        null-collision method (Sec. 4.2, Table 3);
 *   S3   per-cell moments (particle-to-cell, Sec. 4.5).
 *
 * Conventions (all entry points):
 *   - Return 0 (LTPC_OK) on success or a negative LTPC_E* code.  No C++
 *     exception or abort crosses the ABI.
 *   - Work is enqueued asynchronously on the CUDA stream given at creation.
 *     Errors detected on the device are sticky and returned by the next
 *     ltpc_sync (or by any call documented as synchronizing).
 *   - The library allocates no device memory: the caller passes two device
 *     buffers sized by ltpc_required_bytes and keeps ownership of them.
 *   - Device arrays are structure-of-arrays, element type given by
 *     ltpc_config.precision (float for LTPC_F32, double for LTPC_F64).
 *   - Particle ids are storage indices 0..n-1.  Random numbers are a pure
 *     function of (seed, particle id or pair id, step, use): Philox4x32-10.
 */
#ifndef LTPC_H
#define LTPC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define LTPC_OK 0
#define LTPC_EINVAL (-1)       /* bad argument or configuration            */
#define LTPC_ECAPACITY (-2)    /* ionization would exceed the capacity     */
#define LTPC_ECUDA (-3)        /* a CUDA runtime call failed               */
#define LTPC_ETIMEOUT (-4)     /* reserved: no entry point waits on the device */
#define LTPC_ENONFINITE (-5)   /* a loaded velocity is NaN or infinite     */
#define LTPC_EUNSUPPORTED (-6) /* a cell is larger than the largest class  */
#define LTPC_EINTERNAL (-7)    /* an internal bounds check failed          */

#define LTPC_F32 0
#define LTPC_F64 1

#define LTPC_LNL_CONST 0       /* Coulomb logarithm per cell from lnlambda[] */
#define LTPC_LNL_NRL 1         /* NRL e-e formula from the cell's moments    */

typedef struct ltpc_ctx ltpc_ctx; /* opaque, host-side, owned by the library */

/* Species, grid and run parameters (SI units; energies in eV).
 * Cell j holds electrons of density n_j = weight * N_j * inv_volume[j] and
 * advances with time step dt_j = dt * dt_factor[j].  Host arrays are copied
 * by ltpc_create and may be freed afterwards. */
typedef struct ltpc_config {
    int32_t precision;          /* LTPC_F32 or LTPC_F64                        */
    int32_t n_cells;            /* M >= 1 (all plasma instances together)      */
    int64_t capacity;           /* N_max: particle slots (Sec. 4.1 buffers)    */
    uint64_t seed;              /* Philox key                                  */
    double mass;                /* electron mass m [kg]                        */
    double charge;              /* elementary charge e [C]                     */
    double eps0;                /* vacuum permittivity [F/m]                   */
    double weight;              /* macro-particle weight w (uniform)           */
    double n_neutral;           /* neutral density n_n [1/m^3]; 0: no S2a      */
    double mass_neutral;        /* neutral mass M [kg]                         */
    double sigma_el;            /* constant elastic cross section [m^2]        */
    double sigma_ion;           /* ionization cross section above threshold    */
    double e_ion;               /* ionization threshold [eV]                   */
    int32_t lnlambda_mode;      /* LTPC_LNL_CONST or LTPC_LNL_NRL              */
    int32_t correction;         /* -1 default (on for F32, off for F64), 0, 1  */
    int32_t has_position;       /* 1: keep a position array x (copied to
                                   secondaries); 0: no positions              */
    int32_t use_graph;          /* 1: ltpc_step/ltpc_run replay a CUDA graph   */
    const double* inv_volume;   /* host [M]: 1/V_j                             */
    const double* dt_factor;    /* host [M] or NULL (all 1)                    */
    const double* lnlambda;     /* host [M] or NULL (all 10); constant mode    */
    int32_t cache_grouping;     /* 1: skip the per-step CCS3 scatter while no
                                   particle was loaded or appended since the
                                   last one (particles never change cells in
                                   this library); 0: group every step          */
    int32_t pairing_mode;       /* LTPC_PAIR_KEY (0) or LTPC_PAIR_BIJECTION    */
    int32_t reserved[6];        /* must be zero                                */
} ltpc_config;

/* Pairing modes (Table 5 pairs consecutive entries of each cell's index list;
 * the order is the library's reading, the same in every class of kernel).
 *   LTPC_PAIR_KEY: every particle draws a key (word 0 of its PARTICLE Philox
 *     block) and a cell's particles are ordered by (key, id); a particle is a
 *     null-collision candidate when word 1 of that block gives U < P_null.
 *   LTPC_PAIR_BIJECTION: cells of 4097..65536 particles put the particle of
 *     id rank r (ascending ids) at pairing position pi(r), pi a keyed
 *     bijection of [0, N_j) drawn per (seed, cell, step) (six mixed-radix
 *     Feistel rounds with cycle walking); the null-collision candidates are
 *     the particles at positions below floor(P_null N_j + U) (the paper's
 *     "P_null N particles", Sec. 4.2).  Smaller cells are paired and sampled
 *     as in LTPC_PAIR_KEY.  This mode needs storage grouped by cell (cell
 *     ids never decreasing at load); a load that is not is rejected with
 *     LTPC_EINVAL.  Particles appended by ionization keep the grouping. */
#define LTPC_PAIR_KEY 0
#define LTPC_PAIR_BIJECTION 1

/* Bytes of the two caller-owned device buffers for `cfg`.
 * state_bytes: particle arrays (vx, vy, vz, cell, optional x) for
 *              cfg->capacity particles.  work_bytes: grouping, staging,
 *              moments and per-cell tables; in LTPC_PAIR_BIJECTION mode also
 *              one exchange record per particle of capacity (16 bytes in
 *              LTPC_F32, 32 in LTPC_F64), through which the CTAs of a cluster
 *              pass a large cell's particles.  Pure host computation. */
int ltpc_required_bytes(const ltpc_config* cfg, size_t* state_bytes, size_t* work_bytes);

/* Create a context on the current CUDA device.  d_state / d_work: device
 * buffers of at least the sizes above, 256-byte aligned, owned by the caller
 * and valid until ltpc_destroy.  cuda_stream: a cudaStream_t (NULL = legacy
 * default stream).  Synchronizing.  Errors: EINVAL (bad config/pointers),
 * ECUDA. */
int ltpc_create(ltpc_ctx** out, const ltpc_config* cfg, void* d_state, void* d_work, void* cuda_stream);

/* Release host-side resources (graphs, the context).  The caller frees the
 * device buffers.  NULL is ignored. */
void ltpc_destroy(ltpc_ctx* ctx);

/* Flags of ltpc_load_particles. */
#define LTPC_LOAD_SRC_DEVICE 1   /* sources are device pointers (else host memory) */
#define LTPC_LOAD_ASYNC 2        /* do not wait on the stream; report device-detected errors later */

/* Load n particles: cell ids (int32, in [0, M); NULL to bin the positions
 * when a field is set, see ltpc_set_field), optional positions x (only
 * if has_position, else ignored), velocities vx, vy, vz in the context's
 * precision.  flags: LTPC_LOAD_SRC_DEVICE selects device sources (host
 * sources should be pinned for full copy bandwidth); LTPC_LOAD_ASYNC makes
 * the call asynchronous.  Builds the per-cell grouping (CCS1-CCS3) and the
 * moments of the loaded state.  Storage ordered by cell (cell ids never
 * decreasing) is recognised: the per-step grouping then places the loaded
 * particles from their cell's run without atomics (results are the same for
 * any order).
 * Synchronizing by default.  Errors: EINVAL (n < 0, n > capacity or unknown
 * flags), ECUDA; ENONFINITE and EINVAL for cell ids out of range are reported
 * by this call, or with LTPC_LOAD_ASYNC by the next ltpc_sync (particles
 * with bad cell ids are then left out of the grouping; host
 * sources must stay unchanged until the stream reaches the copy). */
int ltpc_load_particles(ltpc_ctx* ctx, int64_t n, const int32_t* cell, const void* x,
                        const void* vx, const void* vy, const void* vz, int flags);

/* Walls of ltpc_set_field. */
#define LTPC_WALL_PERIODIC 0     /* a particle leaving [0, L) re-enters at the other end    */
#define LTPC_WALL_ABSORB 1       /* CS7: it is removed (cell id -1, slot kept, no effect)    */

/* Steps S2b/S2c of Table 2 (CS6/CS7 of Table 3): a constant field per cell and
 * the particle push.  Geometry: the n_cells cells are a 1D grid of width dx [m]
 * along z, the domain [0, L), L = n_cells dx, and x is the position along it.
 * accel (host [n_cells], m/s^2) is q E_j / m of each cell (Sec. 4.2 uses a
 * constant grad phi per cell, looked up by the particle's cell).  The push,
 * as S2c writes it, from the pre-push state of particle l in cell j:
 *   x+ = x + dt_j v_z,   v_z+ = v_z + dt_j accel_j,   then cell = floor(x+ / dx),
 * and `boundary` (LTPC_WALL_*) handles the walls.  Once a field is set,
 * ltpc_step and ltpc_run end every step with the push of every particle
 * (secondaries of the step included, from their parent's position), the
 * per-cell grouping of the new cells (CCS1-CCS3 every step) and the moments
 * of the pushed particles (S3 follows S2c), which ltpc_moments then returns;
 * ltpc_collide_coulomb and ltpc_collide_neutral do not push.  A load may then
 * pass cell = NULL with positions: each cell id is floor(x / dx) (positions
 * outside [0, L) are rejected with EINVAL).  Needs has_position and
 * LTPC_PAIR_KEY (a push breaks the grouping of storage by cell that the
 * bijection mode relies on).  Synchronizing.  Errors: EINVAL. */
int ltpc_set_field(ltpc_ctx* ctx, double dx, const double* accel, int32_t boundary);

/* Storage compaction.  Rewrites the particles in the order of the current
 * per-cell grouping: cells ascending, each cell's particles contiguous (for
 * storage grouped by cell, the cell's loaded run and then its appended
 * particles in their append order), removed particles (cell -1) dropped.
 * Particle ids become the new storage indices, so the random streams that
 * later steps draw change with them; the moments are recomputed by a
 * collision-free pass, as after a load.  Between compactions the particles
 * appended by ionization stay outside their cell's run, where every pass
 * reaches them with scattered accesses; compacting every few hundred steps
 * keeps the runs whole.  Reads the grouped count back (one synchronization of
 * the stream), then proceeds asynchronously like a load with LTPC_LOAD_ASYNC.
 * Errors: a pending sticky error, ECUDA. */
int ltpc_compact(ltpc_ctx* ctx);

/* Steps S2b/S2c alone (no collisions) with time step dt (cell j: dt *
 * dt_factor[j]) at step number `step`, then the grouping of the new cells and
 * their moments.  Needs ltpc_set_field.  Asynchronous.  Errors: EINVAL. */
int ltpc_push(ltpc_ctx* ctx, double dt, int64_t step);

/* Recombination C5 of Table 1 (Ar+ + 2e -> Ar_m + e; Sec. 4.3, Table 4
 * RS0-RS5), run in step S2a after C1/C2 by ltpc_step and ltpc_collide_neutral.
 * k_rec [m^6/s]: three-body rate with the ion density taken equal to the
 * electron density, so every electron of cell j recombines with probability
 * P_rec = 1 - exp(-dt_j k_rec n_j^2); de_rec [eV]: energy the catalyte gains
 * besides the primary's kinetic energy.  Each cell takes floor(P_rec N_j + U)
 * primaries (U from the cell's RECOMB Philox block; at most N_j / 2) at the
 * last positions of the step's pairing order; the r-th primary hands its
 * energy to the catalyte n_p positions before it (a unique match inside the
 * cell, in place of the paper's atomic catalyte list) and is removed: its
 * cell id becomes -1 and it takes part in nothing afterwards (slot kept).
 * k_rec = 0 switches C5 off.  Needs LTPC_PAIR_KEY (removals break the
 * grouping of storage by cell that the bijection mode relies on).
 * Errors: EINVAL. */
int ltpc_set_recombination(ltpc_ctx* ctx, double k_rec, double de_rec);

/* ---- tabulated cross sections and per-particle selection (Sec. 4.2) ------
 * The paper evaluates each electron-neutral cross section as a piecewise
 * polynomial fit in place of a table lookup.  One table: interval i of the
 * uniform grid ln E0 + [i, i+1) h (E in eV) holds the cubic
 * c0 + c1 t + c2 t^2 + c3 t^3 [m^2] in t = (ln E - ln E0)/h - i; below E0 the
 * value is 0 (zero_below = 1, as an ionization threshold) or c0 of the first
 * piece (zero_below = 0); above the last knot it is the last piece's value at
 * t = 1.  coef is a host array [pieces][4], copied by the call. */
#define LTPC_XS_MAX_PIECES 256
typedef struct ltpc_xsec {
    int32_t pieces;             /* 1 .. LTPC_XS_MAX_PIECES                      */
    int32_t zero_below;         /* 1: 0 below E0; 0: the first knot's value      */
    double lnE0;                /* ln of the first knot energy (E in eV)        */
    double h;                   /* knot spacing in ln E, > 0                    */
    const double* coef;         /* [pieces][4] host, finite                     */
} ltpc_xsec;

#define LTPC_SELECT_NULL 0          /* null-collision method (Sec. 4.2)          */
#define LTPC_SELECT_PER_PARTICLE 1  /* per-particle collision probabilities      */

/* sigma_el(E) and sigma_ion(E) of C1/C2 from tables (el or ion NULL: that one
 * stays the configuration's constant, resp. step at e_ion), used by the
 * collision decisions of S2a and by the rate sums of the moments (mom 8, 9:
 * sum sigma(E) |v|).  sigma_max [m^2] bounds sigma_el(E) + sigma_ion(E) for
 * every E: the null-collision frequency is nu_max = n_n sigma_max v_max (with
 * both tables NULL it stays n_n (sigma_el + sigma_ion) v_max).  selection:
 * LTPC_SELECT_NULL, or LTPC_SELECT_PER_PARTICLE, where every particle collides
 * with probabilities pi_c = 1 - exp(-dt_j v sigma_c(E) n_n), decided by one
 * uniform U1 of its PARTICLE block against pi_el and pi_el + pi_ion (C1 first,
 * Table 1's order); needs LTPC_PAIR_KEY.  Both tables NULL with
 * LTPC_SELECT_NULL restores the constant cross sections.  The ionization
 * outcome keeps E - e_ion as the energy shared by the two electrons.  binary64
 * evaluates the tables with the natural logarithm, one division and Horner's
 * rule; binary32 with the fast hardware logarithm and binary32 coefficients
 * (relative error near 1e-6).  The call samples each table (32 points per
 * piece and the knots) and rejects a negative value or a sum above sigma_max.
 * Synchronizing.  Errors: EINVAL. */
int ltpc_set_cross_sections(ltpc_ctx* ctx, const ltpc_xsec* el, const ltpc_xsec* ion, double sigma_max,
                            int32_t selection);

/* Step S1 only: Takizuka-Abe Coulomb collisions (Sec. 4.4) with time step
 * dt (cell j uses dt * dt_factor[j]) at step number `step` (0 <= step <
 * 2^32), then the moments.  Asynchronous. */
int ltpc_collide_coulomb(ltpc_ctx* ctx, double dt, int64_t step);

/* Step S2a only: null-collision electron-neutral elastic and ionization
 * collisions (Sec. 4.2); secondaries are appended (the particle count may
 * grow), then the moments.  Asynchronous; ECAPACITY is reported by
 * ltpc_sync when the capacity would be exceeded (the secondaries of that
 * pass are dropped and the primaries keep their post-collision state). */
int ltpc_collide_neutral(ltpc_ctx* ctx, double dt, int64_t step);

/* One full collision step S1 + S2a + S3 (S2a only when n_neutral > 0), fused
 * in one pass per cell.  With use_graph the pass is captured once as a CUDA
 * graph and replayed.  Asynchronous. */
int ltpc_step(ltpc_ctx* ctx, double dt, int64_t step);

/* nsteps consecutive ltpc_step calls for steps step0, step0+1, ... */
int ltpc_run(ltpc_ctx* ctx, double dt, int64_t step0, int64_t nsteps);

/* Tracing: one full step like ltpc_step but launched without a graph, with
 * CUDA events recorded on the context's stream around every kernel of the
 * pass.  ms[k] receives the device time of kernel k in launch order:
 * 0 grouping scatter (CCS3), 1..C cell kernel of each cluster class (see
 * ltpc_classes), C+1 regroup/offsets (CCS2), C+2 append of secondaries.
 * *n_out = C + 3.  `capacity` is the length of ms.  Synchronizing. */
int ltpc_profile_step(ltpc_ctx* ctx, double dt, int64_t step, float* ms, int32_t capacity, int32_t* n_out);

/* Tracing: one full step (no graph) in which thread 0 of every CTA of the
 * cell kernels adds the SM cycles it spent in each phase into d_cycles[16]
 * (device, zeroed by the call): 0 work fetch, 1 pairing keys, 2 bucket
 * offsets, 3 placement, 4 in-bucket rank, 5 position lookup, 6 gather,
 * 7 Coulomb + restoration, 8 neutral sampling, 9 moments, 10 write-back.
 * Asynchronous. */
int ltpc_profile_phases(ltpc_ctx* ctx, double dt, int64_t step, unsigned long long* d_cycles);

/* Per-cell moments of the last pass: mom[10 j + k] (double) with k =
 * 0 N_j, 1 w N_j, 2-4 sum v_x, v_y, v_z, 5-7 sum v_x^2, v_y^2, v_z^2,
 * 8 sum sigma_el |v|, 9 sum sigma_ion(E) |v|; hist[64 j + b] (uint32):
 * counts in 64 log-spaced energy bins on [1e-2, 1e3] eV (end bins clamp).
 * Either pointer may be NULL.  Host destinations synchronize the stream. */
int ltpc_moments(ltpc_ctx* ctx, double* mom, uint32_t* hist, int dst_is_device);

/* Restore the per-cell moments (same layout as ltpc_moments; hist may be
 * NULL), typically from a checkpoint.  A pass takes the cell's state before
 * S1 for the momentum/energy restoration, and the NRL Coulomb logarithm, from
 * the moments the previous pass left (the paper has no such state: it is this
 * library's way of not summing the cell twice).  A checkpoint is therefore
 * (ltpc_read_particles, ltpc_moments, the next step number); resuming with
 * ltpc_load_particles, then ltpc_set_moments, then the same steps and class
 * table, reproduces the uninterrupted run bit for bit.  Call it after the
 * load (which computes moments of its own).  src_is_device: 1 device
 * pointers, 0 host (the call then synchronizes the stream).  Errors: EINVAL
 * (NULL ctx or mom), ECUDA. */
int ltpc_set_moments(ltpc_ctx* ctx, const double* mom, const uint32_t* hist, int src_is_device);

/* Copy the particles out: velocities, cell ids, optional positions (any
 * pointer may be NULL); *n_out receives the particle count.  Synchronizing. */
int ltpc_read_particles(ltpc_ctx* ctx, void* vx, void* vy, void* vz, int32_t* cell, void* x,
                        int64_t* n_out, int dst_is_device);

/* Wait for all work and return (then clear) deferred device errors. */
int ltpc_sync(ltpc_ctx* ctx);

/* Inspection: the pairing order of step `step` for the current grouping
 * (Table 5 pairs entries 2k, 2k+1 of each cell's segment) written to device
 * arrays order[n] and cell_start[M+1] (uint32).  Leaves the particles
 * unchanged.  Asynchronous. */
int ltpc_pair_order(ltpc_ctx* ctx, int64_t step, uint32_t* d_order, uint32_t* d_cell_start);

/* Inspection: the grouping of CCS1-CCS3 (cell_start[M+1], perm[n], counts[M];
 * device pointers, any may be NULL).  perm[cell_start[j] .. cell_start[j+1])
 * holds the ids of cell j: the loaded particles (in index order after a load
 * ordered by cell, otherwise in unspecified order), then the particles
 * appended by ionization in index order.
 * Asynchronous. */
int ltpc_grouping(ltpc_ctx* ctx, uint32_t* d_cell_start, uint32_t* d_perm, uint32_t* d_counts);

/* Cluster classes used for cells of different sizes: class i handles cells
 * with max_n[i-1] < N_j <= max_n[i].  ltpc_classes reports the active ones
 * (cluster size, threads per CTA, positions per CTA, largest cell). */
int ltpc_classes(ltpc_ctx* ctx, int32_t* n_classes, int32_t* cluster, int32_t* threads,
                 int32_t* per_cta, int32_t* max_n);

/* Choose among the compiled class tables by timing collision-free passes
 * (grouping, ordering, staging and moments; the particles are not changed)
 * of each on the loaded particles.  The choice changes
 * only the schedule; the per-cell arithmetic may round differently between
 * tables (reductions follow the CTA shape).  Synchronizing. */
int ltpc_autotune(ltpc_ctx* ctx, double dt, int32_t* chosen_table);
/* Select class table `table` (0 = default) and rebuild the work lists for
 * the current counts.  Synchronizing.  Errors: EINVAL for an unknown table. */
int ltpc_set_class_table(ltpc_ctx* ctx, int32_t table);

/* ---- rate-coefficient surrogate --------------------------------------------
 * A perceptron 66 -> 128 -> 128 -> 2 with GELU that maps a cell's energy
 * distribution to its ionization and elastic rate coefficients
 * k_c = sum sigma_c |v| / N (the C_kc terms of Eq. 1 per electron; Sec. 1
 * motivates resolving the distribution's tail).  Inputs per cell (66): the 64
 * histogram fractions of ltpc_moments, log10 n_e and the mean energy [eV],
 * normalised as (x - mean) / std; outputs: k_ion / scale_0, k_el / scale_1.
 * Weights and activations are bfloat16 with FP32 accumulation (tensor-core
 * MMAs); master weights, biases and Adam moments are FP32.  Parameters are
 * packed as W1 [128][80] (input columns 66..79 zero), b1 [128], W2
 * [128][128], b2 [128], W3 [2][128], b3 [2] (ltpc_mlp_param_count floats).
 * Device arrays X [B][66], T and Y [B][2] are float, row-major.  All calls
 * run on the stream given at creation unless stated; errors as above. */
typedef struct ltpc_mlp ltpc_mlp;
int ltpc_mlp_param_count(void);
/* Bytes of the caller-owned device buffer for batches of up to batch_max rows
 * and up to n_cells_max cells in the context-coupled calls. */
int ltpc_mlp_required_bytes(int32_t batch_max, int32_t n_cells_max, size_t* bytes);
/* Create with deterministic initial weights (uniform +-1/sqrt(fan_in) from
 * Philox with `seed`); d_buf 256-byte aligned.  Synchronizing. */
int ltpc_mlp_create(ltpc_mlp** out, void* d_buf, int32_t batch_max, int32_t n_cells_max, uint64_t seed,
                    void* cuda_stream);
void ltpc_mlp_destroy(ltpc_mlp* mlp);
int ltpc_mlp_set_params(ltpc_mlp* mlp, const float* params, int src_is_device);   /* synchronizing */
int ltpc_mlp_get_params(ltpc_mlp* mlp, float* params, int dst_is_device);         /* synchronizing */
/* Feature means and standard deviations [66] and target scales [2] (host). */
int ltpc_mlp_set_norm(ltpc_mlp* mlp, const float* feat_mean, const float* feat_std, const float* target_scale);
/* Y = network(X) for B <= batch_max rows. */
int ltpc_mlp_forward(ltpc_mlp* mlp, const float* d_X, int32_t B, float* d_Y);
/* Mean-squared-error loss of (X, T) and its gradient w.r.t. every parameter
 * (packed order) into d_grad (may be NULL) and d_loss (may be NULL). */
int ltpc_mlp_gradients(ltpc_mlp* mlp, const float* d_X, const float* d_T, int32_t B, float* d_grad, float* d_loss);
/* One Adam step (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected) on (X, T). */
int ltpc_mlp_train_step(ltpc_mlp* mlp, const float* d_X, const float* d_T, int32_t B, float lr, float* d_loss);
/* Features [M][66] of every cell of `ctx` from its last moments (normalised
 * when `normalize`), and the exact rates [M][2] (k_ion, k_el) if d_T != NULL.
 * Runs on the context's stream. */
int ltpc_mlp_features(ltpc_ctx* ctx, ltpc_mlp* mlp, float* d_X, float* d_T, int normalize);
/* In-loop serving: rates [M][2] (k_ion, k_el in m^3/s) predicted for every
 * cell of `ctx` from its last moments.  Runs on the context's stream. */
int ltpc_mlp_infer(ltpc_ctx* ctx, ltpc_mlp* mlp, float* d_rates);
/* Features [M][66] (normalised) of a random subsample of about per_cell
 * particles of every cell (salt selects the sample) and the direct rate
 * estimate [M][2] of that subsample; the density feature is the whole
 * cell's.  Synchronizing. */
int ltpc_mlp_subsample_features(ltpc_ctx* ctx, ltpc_mlp* mlp, int32_t per_cell, uint32_t salt, float* d_X,
                                float* d_rates_direct);

/* Largest number of cells ltpc_group_cells_noalloc accepts. */
#define LTPC_NOALLOC_MAX_CELLS 131072

/* Grouping of particle ids by cell (counts, start offsets and the index list
 * of ltpc_grouping) for callers that cannot allocate device memory: code
 * inside a program whose memory pool owns the whole device, code whose device
 * budget is already reserved, or a loop that must not pay for an allocation.
 * The paper has no counterpart; it is a service of this library.
 * Inputs: d_cell[n] (device int32 cell ids).  Outputs: d_cell_start[n_cells+1]
 * and d_perm[n] (device uint32): d_perm[d_cell_start[j] ..
 * d_cell_start[j+1]) holds the ids of cell j's particles (order inside a cell
 * unspecified).  The per-cell counters live in a fixed device array of this
 * library (LTPC_NOALLOC_MAX_CELLS + 64 words on every GPU that loads it, kept
 * until exit); no cudaMalloc, cudaFree or allocating library routine is
 * called.  The first call on a device looks up that array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * Every call synchronizes its stream and reads a flag word back.  Every call
 * shares the array and clears what it uses; calls whose work overlaps on the
 * GPU race.  Synchronizes `cuda_stream` (a
 * cudaStream_t, NULL = legacy default stream).  Errors: EINVAL (n < 0,
 * n_cells outside [1, LTPC_NOALLOC_MAX_CELLS], a NULL buffer, or a cell id
 * outside [0, n_cells)), ECUDA. */
int ltpc_group_cells_noalloc(const int32_t* d_cell, int64_t n, int32_t n_cells, uint32_t* d_cell_start,
                             uint32_t* d_perm, void* cuda_stream);

/* Short text for a status code (static storage). */
const char* ltpc_strerror(int code);

/* Last CUDA error text recorded by the context ("" if none). */
const char* ltpc_last_cuda_error(ltpc_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* LTPC_H */
