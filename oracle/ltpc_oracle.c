/*
 * ltpc_oracle.c -- plain, slow, FP64 CPU oracle for the collision hot path of
 * "A Portable Multi-GPU Solver for Collisional Plasmas with Coulombic
 * Interactions" (Almgren-Bell et al., arXiv 2508.06771).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The product path (the CUDA
 * library of the package) never calls it, and the two share no code, header,
 * table or constant generator.  Physical constants and per-cell parameters
 * arrive as arguments from the workload generator.
 *
 * Everything below is sequential FP64 in the order the paper states its steps.
 * It is compiled with -ffp-contract=off so that no fused multiply-add changes
 * the rounding of any expression written here.
 *
 * Pinning status (what each function is checked against in tests/):
 *   orc_philox4x32_10   known-answer vectors of Philox4x32-10 + chi^2 uniformity
 *   orc_group           numpy stable argsort / bincount
 *   orc_pair_order      brute force with an independent Python Philox
 *   orc_ta_pair         rotation invariants, conservation, angle statistics
 *   orc_coulomb         conservation, Maxwellian stationarity, NRL relaxation
 *   orc_neutral         analytic collision counts, energy bookkeeping
 *   orc_moments         numpy bincount sums
 *   orc_nrl_lnlambda    hand-evaluated formulary values
 *   orc_recombine       count law, unique matching, removed count, energy
 *                       bookkeeping
 *   orc_push, orc_bin    closed-form free flight, energy gain identity,
 *                       numpy re-binning and absorbed counts
 *   orc_bij_*, orc_pair_order_mode (bijection mode)
 *                       bijection and inverse on every tested size; chi^2
 *                       uniformity of positions, partners and the left-out
 *                       particle; rate of neighbouring-rank pairs; candidate
 *                       count mean P_null N and uniform selection
 *   orc_xs_eval         within 2 % of the smooth cross sections it tabulates,
 *                       exact at the knots, zero below the threshold
 *   per-particle selection (orc_neutral, selection 1)
 *                       binomial counts against sum pi_c; same mean number of
 *                       real collisions as the null-collision method to first
 *                       order in dt; rate sums against a quadrature
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PI 3.14159265358979323846

/* Random-stream tags: which use a Philox block serves (counter word 2). */
enum { ORC_TAG_PARTICLE = 1, ORC_TAG_PAIR = 2, ORC_TAG_SCATTER = 3, ORC_TAG_SECONDARY = 4, ORC_TAG_PERM = 5,
       ORC_TAG_RECOMB = 6 };

/* Pairing modes (see orc_pair_order_ids).  In the bijection mode, cells of at
 * least ORC_BIJ_MIN_N particles are paired through a keyed bijection of their
 * id ranks; smaller cells keep the key sort. */
enum { ORC_PAIR_KEY = 0, ORC_PAIR_BIJECTION = 1 };
#define ORC_BIJ_MIN_N 4097u

/* Error codes (same numeric meaning as the library's, defined independently). */
enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ECAPACITY = -2 };

/* A cross section as a piecewise cubic in ln E (Sec. 4.2 replaces the
 * table lookup with a piecewise polynomial interpolation): interval i of the
 * uniform grid ln E0 + [i, i+1) h holds c0 + c1 t + c2 t^2 + c3 t^3 with
 * t = (ln E - ln E0)/h - i; below E0 the value is 0 (zero_below) or the
 * first knot's; above the last knot, the last knot's. */
typedef struct {
    int32_t pieces;
    int32_t zero_below;
    double lnE0, h;
    const double *coef;  /* [pieces][4] */
} orc_xs;

typedef struct {
    double mass;         /* electron mass m [kg]                         */
    double charge;       /* elementary charge e [C]                      */
    double eps0;         /* vacuum permittivity [F/m]                    */
    double weight;       /* macro-particle weight w (uniform, Sec. 8)    */
    double n_neutral;    /* neutral density n_n [1/m^3]                  */
    double mass_neutral; /* neutral mass M [kg]                          */
    double sigma_el;     /* constant elastic cross section [m^2]         */
    double sigma_ion;    /* ionization cross section above threshold     */
    double e_ion;        /* ionization threshold [eV]                    */
    uint64_t seed;       /* Philox key                                   */
    int32_t odd_mode;    /* 0: last particle of an odd cell sits out     */
    int32_t correction;  /* 1: restore per-cell momentum+energy after TA */
    int32_t pairing_mode;/* ORC_PAIR_KEY or ORC_PAIR_BIJECTION           */
    int32_t selection;   /* 0 null collision, 1 per-particle probabilities */
    const uint32_t *cell_ids; /* random-stream id of each cell (NULL: its index) */
    const orc_xs *xs_el, *xs_ion; /* tabulated cross sections (NULL: the constant / step ones) */
    double sigma_max;    /* bound on sigma_el + sigma_ion with the tables */
} orc_params;

double orc_xs_eval(const orc_xs *t, double E)
{
    if (!(E > 0.0)) return t->zero_below ? 0.0 : t->coef[0];
    double u = (log(E) - t->lnE0) / t->h;
    if (u < 0.0) return t->zero_below ? 0.0 : t->coef[0];
    double fi = floor(u);
    int32_t i = (int32_t)fi;
    double x;
    if (i >= t->pieces) { i = t->pieces - 1; x = 1.0; }
    else x = u - fi;
    const double *c = t->coef + 4 * (size_t)i;
    return c[0] + x * (c[1] + x * (c[2] + x * c[3]));
}

/* sigma_el(E), sigma_ion(E): the tables when given, else the constant elastic and
 * the step ionization cross sections. */
static double orc_sig_el(const orc_params *p, double E) { return p->xs_el ? orc_xs_eval(p->xs_el, E) : p->sigma_el; }
static double orc_sig_ion(const orc_params *p, double E)
{
    if (p->xs_ion) return orc_xs_eval(p->xs_ion, E);
    return E >= p->e_ion ? p->sigma_ion : 0.0;
}

/* ------------------------------------------------------------------------- *
 * Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, "Parallel random numbers:
 * as easy as 1, 2, 3").  Ten rounds of the Philox S-box on a 4x32-bit counter
 * with a 2x32-bit key; the key is advanced by the Weyl constants between
 * rounds.  The paper's kernels draw uniforms with cupy.random.rand
 * (Sec. 4.2, Sec. 4.4); this build replaces that with counter-based draws.
 * ------------------------------------------------------------------------- */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = (uint64_t)M0 * (uint64_t)c[0];
        uint64_t p1 = (uint64_t)M1 * (uint64_t)c[2];
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c[1] ^ k0;
        uint32_t n2 = hi0 ^ c[3] ^ k1;
        c[0] = n0; c[1] = lo1; c[2] = n2; c[3] = lo0;
    }
    out[0] = c[0]; out[1] = c[1]; out[2] = c[2]; out[3] = c[3];
}

/* One block of four words for stream `tag` of particle (or pair) id `id` at
 * time step `step`: counter = (id lo, step, tag, id hi), key = seed. */
static void orc_draw(uint64_t seed, uint64_t id, uint32_t step, uint32_t tag, uint32_t w[4])
{
    uint32_t ctr[4] = {(uint32_t)id, step, tag, (uint32_t)(id >> 32)};
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    orc_philox4x32_10(ctr, key, w);
}

/* FP64 uniform on (0,1): (w + 1/2) 2^-32, exact in double, never 0 or 1. */
double orc_uniform(uint32_t w) { return ((double)w + 0.5) * (1.0 / 4294967296.0); }

/* ------------------------------------------------------------------------- *
 * Per-cell grouping, Table 5 steps CCS1-CCS3: N_j = |P_j| (CCS1), start
 * offsets I_j by an exclusive prefix sum over N_j (CCS2), and the index array
 * P holding every cell's particles contiguously (CCS3).  The oracle's P is the
 * stable one (ascending particle index inside each cell); the paper's atomic
 * cursor gives the same sets in an arbitrary order.
 * ------------------------------------------------------------------------- */
int orc_group(int64_t n, int32_t M, const int32_t *cell,
              uint32_t *counts, uint64_t *cell_start, uint32_t *perm)
{
    if (n < 0 || M <= 0) return ORC_EINVAL;
    for (int32_t j = 0; j < M; ++j) counts[j] = 0;
    for (int64_t l = 0; l < n; ++l) {
        if (cell[l] == -1) continue;                            /* removed at a wall (CS7) */
        if (cell[l] < 0 || cell[l] >= M) return ORC_EINVAL;
        counts[cell[l]] += 1;                                   /* CCS1 */
    }
    uint64_t acc = 0;
    for (int32_t j = 0; j < M; ++j) { cell_start[j] = acc; acc += counts[j]; }  /* CCS2 */
    cell_start[M] = acc;
    uint64_t *cursor = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)M);
    if (!cursor) return ORC_EINVAL;
    for (int32_t j = 0; j < M; ++j) cursor[j] = cell_start[j];
    for (int64_t l = 0; l < n; ++l)
        if (cell[l] >= 0) perm[cursor[cell[l]]++] = (uint32_t)l;               /* CCS3 */
    free(cursor);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- *
 * In-cell pairing order.  Table 5 pairs consecutive entries of P; the paper's
 * P order comes from atomic increments and is not reproducible.  Reading: each
 * step every particle l draws a key r_l (word 0 of its PARTICLE block) and a
 * cell's particles are ordered by (r_l, l); pairs are entries (0,1), (2,3), ...
 * of that order.  This is the per-step re-randomised partner choice the
 * Takizuka-Abe model needs.
 * ------------------------------------------------------------------------- */
static uint32_t orc_pair_key(uint64_t seed, uint64_t l, uint32_t step)
{
    uint32_t w[4];
    orc_draw(seed, l, step, ORC_TAG_PARTICLE, w);
    return w[0];
}

/* Random-stream id of particle l: ids[l] when the caller keeps a subset of a
 * larger particle set (ids = the particles' indices in that set), else l. */
static uint64_t orc_id(const uint32_t *ids, uint64_t l) { return ids ? (uint64_t)ids[l] : l; }

/* order[cell_start[j] .. cell_start[j+1]) = cell j's particles (storage
 * indices) in pairing order; keys and ties use the particles' ids. */
int orc_pair_order_ids(int64_t n, int32_t M, const int32_t *cell, const uint32_t *ids, uint64_t seed,
                       uint32_t step, uint64_t *cell_start, uint32_t *order);

int orc_pair_order(int64_t n, int32_t M, const int32_t *cell, uint64_t seed, uint32_t step,
                   uint64_t *cell_start, uint32_t *order)
{
    return orc_pair_order_ids(n, M, cell, NULL, seed, step, cell_start, order);
}

typedef struct { uint32_t key; uint32_t id; uint32_t l; } orc_kil;

static int orc_kil_cmp(const void *a, const void *b)
{
    const orc_kil *x = (const orc_kil *)a, *y = (const orc_kil *)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->id != y->id) return x->id < y->id ? -1 : 1;
    return 0;
}

int orc_pair_order_ids(int64_t n, int32_t M, const int32_t *cell, const uint32_t *ids, uint64_t seed,
                       uint32_t step, uint64_t *cell_start, uint32_t *order)
{
    uint32_t *counts = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)M);
    if (!counts) return ORC_EINVAL;
    int rc = orc_group(n, M, cell, counts, cell_start, order);
    free(counts);
    if (rc) return rc;
    orc_kil *tmp = (orc_kil *)malloc(sizeof(orc_kil) * (size_t)(n > 0 ? n : 1));
    if (!tmp) return ORC_EINVAL;
    for (int32_t j = 0; j < M; ++j) {
        uint64_t s = cell_start[j], e = cell_start[j + 1];
        for (uint64_t k = s; k < e; ++k) {
            tmp[k - s].l = order[k];
            tmp[k - s].id = (uint32_t)orc_id(ids, order[k]);
            tmp[k - s].key = orc_pair_key(seed, orc_id(ids, order[k]), step);
        }
        qsort(tmp, (size_t)(e - s), sizeof(orc_kil), orc_kil_cmp);
        for (uint64_t k = s; k < e; ++k) order[k] = tmp[k - s].l;
    }
    free(tmp);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- *
 * Pairing through a keyed bijection (the oracle's second pairing mode).
 * Table 5 only asks that consecutive entries of a cell's index list be
 * paired; any random perfect matching of the cell serves the Takizuka-Abe
 * model.  Reading for cells of n >= ORC_BIJ_MIN_N particles: the cell's
 * particles are ranked by ascending id (r = 0 .. n-1) and the particle of rank
 * r takes pairing position pi(r), where pi is a bijection of [0, n) keyed by
 * (seed, cell, step):
 *   - the domain is written in mixed radix: a = ceil(sqrt(n)), b = ceil(n/a),
 *     x = L b + R with L in [0, a), R in [0, b);
 *   - six Feistel rounds alternate between the two radices: an even round maps
 *     (L, R) with L in [0, a), R in [0, b) to (R, (L + F(R, K_i, a)) mod a) and
 *     an odd round maps (L, R) with L in [0, b), R in [0, a) to
 *     (R, (L + F(R, K_i, b)) mod b), so after six rounds L is in [0, a) again
 *     and the image is L b + R in [0, a b);
 *   - F(R, K, m) = floor(h m / 2^32), h = mix(R xor K), mix(t) = u * M2 mod
 *     2^32 with u = w xor (w >> 16), w = t * M1 mod 2^32 (M1 = 0x9E3779B1,
 *     M2 = 0x85EBCA6B);
 *   - the round keys K_0..K_5 are words 0-3 of the Philox block with counter
 *     (cell, step, PERM, 0) and words 0-1 of the block (cell, step, PERM, 1);
 *     word 2 of the second block is the uniform that rounds the neutral step's
 *     candidate count (orc_neutral_ids);
 *   - images at or above n are mapped again (cycle walking), which restricts
 *     the bijection of [0, a b) to one of [0, n).
 * Pins: bijection and inverse for every tested n, uniformity of positions,
 * partners and the left-out particle, and the rate of pairs of neighbouring
 * ranks (tests/test_oracle_bijection.py).
 * ------------------------------------------------------------------------- */
typedef struct {
    uint32_t n, a, b;
    uint32_t key[6];
    uint32_t u;          /* candidate-count rounding word */
} orc_bij;

static uint32_t orc_bij_mix(uint32_t t)
{
    uint32_t w = t * 0x9E3779B1u;
    uint32_t u = w ^ (w >> 16);
    return u * 0x85EBCA6Bu;
}

static uint32_t orc_bij_f(uint32_t r, uint32_t key, uint32_t m)
{
    return (uint32_t)(((uint64_t)orc_bij_mix(r ^ key) * (uint64_t)m) >> 32);
}

void orc_bij_setup(uint64_t seed, uint64_t cell_id, uint32_t step, uint32_t n, orc_bij *B)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    uint32_t c0[4] = {(uint32_t)cell_id, step, ORC_TAG_PERM, 0u};
    uint32_t c1[4] = {(uint32_t)cell_id, step, ORC_TAG_PERM, 1u};
    uint32_t w0[4], w1[4];
    orc_philox4x32_10(c0, key, w0);
    orc_philox4x32_10(c1, key, w1);
    uint32_t a = 1;
    while ((uint64_t)a * a < n) ++a;              /* ceil(sqrt(n)) */
    B->n = n;
    B->a = a;
    B->b = n > 0 ? (n + a - 1) / a : 1;
    for (int i = 0; i < 4; ++i) B->key[i] = w0[i];
    B->key[4] = w1[0];
    B->key[5] = w1[1];
    B->u = w1[2];
}

/* One pass of the six rounds over [0, a b). */
static uint32_t orc_bij_enc(const orc_bij *B, uint32_t x)
{
    uint32_t L = x / B->b, R = x % B->b;
    for (int i = 0; i < 6; ++i) {
        uint32_t m = (i % 2 == 0) ? B->a : B->b;
        uint32_t t = (L + orc_bij_f(R, B->key[i], m)) % m;
        L = R;
        R = t;
    }
    return L * B->b + R;
}

/* Its inverse: the rounds undone in reverse order. */
static uint32_t orc_bij_dec(const orc_bij *B, uint32_t y)
{
    uint32_t L = y / B->b, R = y % B->b;
    for (int i = 5; i >= 0; --i) {
        uint32_t m = (i % 2 == 0) ? B->a : B->b;
        uint32_t prevR = L;
        uint32_t prevL = (R + m - orc_bij_f(prevR, B->key[i], m)) % m;
        L = prevL;
        R = prevR;
    }
    return L * B->b + R;
}

uint32_t orc_bij_forward(const orc_bij *B, uint32_t r)
{
    uint32_t y = orc_bij_enc(B, r);
    while (y >= B->n) y = orc_bij_enc(B, y);
    return y;
}

uint32_t orc_bij_inverse(const orc_bij *B, uint32_t q)
{
    uint32_t x = orc_bij_dec(B, q);
    while (x >= B->n) x = orc_bij_dec(B, x);
    return x;
}

/* Test access: pi or its inverse for every element of [0, n). */
int orc_bij_table(uint64_t seed, uint64_t cell_id, uint32_t step, uint32_t n, int inverse, uint32_t *out,
                  uint32_t *params_out)
{
    orc_bij B;
    orc_bij_setup(seed, cell_id, step, n, &B);
    for (uint32_t k = 0; k < n; ++k) out[k] = inverse ? orc_bij_inverse(&B, k) : orc_bij_forward(&B, k);
    if (params_out) {
        params_out[0] = B.a; params_out[1] = B.b;
        for (int i = 0; i < 6; ++i) params_out[2 + i] = B.key[i];
        params_out[8] = B.u;
    }
    return ORC_OK;
}

static uint64_t orc_cell_id(const orc_params *p, int32_t j)
{
    return p->cell_ids ? (uint64_t)p->cell_ids[j] : (uint64_t)j;
}

typedef struct { uint32_t id; uint32_t l; } orc_il;

static int orc_il_cmp(const void *a, const void *b)
{
    const orc_il *x = (const orc_il *)a, *y = (const orc_il *)b;
    return x->id < y->id ? -1 : (x->id > y->id ? 1 : 0);
}

/* Pairing order of every cell under the mode in p: the key sort, or for
 * cells of at least ORC_BIJ_MIN_N particles in the bijection mode, the
 * particle of id rank r at position pi(r). */
int orc_pair_order_mode(int64_t n, int32_t M, const int32_t *cell, const uint32_t *ids, const orc_params *p,
                        uint32_t step, uint64_t *cell_start, uint32_t *order)
{
    int rc = orc_pair_order_ids(n, M, cell, ids, p->seed, step, cell_start, order);
    if (rc || p->pairing_mode != ORC_PAIR_BIJECTION) return rc;
    orc_il *tmp = (orc_il *)malloc(sizeof(orc_il) * (size_t)(n > 0 ? n : 1));
    if (!tmp) return ORC_EINVAL;
    for (int32_t j = 0; j < M; ++j) {
        uint64_t s = cell_start[j], cnt = cell_start[j + 1] - cell_start[j];
        if (cnt < ORC_BIJ_MIN_N) continue;
        for (uint64_t k = 0; k < cnt; ++k) {
            tmp[k].l = order[s + k];
            tmp[k].id = (uint32_t)orc_id(ids, order[s + k]);
        }
        qsort(tmp, (size_t)cnt, sizeof(orc_il), orc_il_cmp);       /* ranks by ascending id */
        orc_bij B;
        orc_bij_setup(p->seed, orc_cell_id(p, j), step, (uint32_t)cnt, &B);
        for (uint64_t r = 0; r < cnt; ++r) order[s + orc_bij_forward(&B, (uint32_t)r)] = tmp[r].l;
    }
    free(tmp);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- *
 * Takizuka-Abe binary collision (Takizuka & Abe 1977, the model Sec. 4.4
 * adopts for step S1).  For a pair (a, b) of equal-mass electrons with
 * relative velocity u = v_a - v_b:
 *   delta = tan(Theta/2) is Gaussian with variance <delta^2> = A / |u|^3,
 *   A = q^4 n lnLambda dt / (8 pi eps0^2 mu^2), mu = m/2;
 *   phi is uniform on [0, 2 pi);
 *   u is rotated by Theta about an axis at azimuth phi; both particles take
 *   half of the change with opposite signs (momentum and energy conserved).
 * The three uniforms come from one PAIR block: Box-Muller radius, Box-Muller
 * angle, azimuth.  `A` is the per-cell coefficient.
 * ------------------------------------------------------------------------- */
void orc_ta_pair(double va[3], double vb[3], double A, const uint32_t w[4])
{
    double ux = va[0] - vb[0], uy = va[1] - vb[1], uz = va[2] - vb[2];
    double usq = ux * ux + uy * uy + uz * uz;
    if (usq == 0.0) return;                     /* identical velocities: nothing to rotate */
    double u = sqrt(usq);
    double var = A / (usq * u);                 /* <delta^2> */
    double g = sqrt(-2.0 * log(orc_uniform(w[0]))) * cos(2.0 * ORC_PI * orc_uniform(w[1]));
    double delta = sqrt(var) * g;
    double phi = 2.0 * ORC_PI * orc_uniform(w[2]);

    double sin_t, omc_t;                        /* sin(Theta), 1 - cos(Theta) */
    if (fabs(delta) <= 1.0) {
        double d2 = delta * delta;
        sin_t = 2.0 * delta / (1.0 + d2);
        omc_t = 2.0 * d2 / (1.0 + d2);
    } else {                                    /* same values through t = 1/delta */
        double t = 1.0 / delta, t2 = t * t;
        sin_t = 2.0 * t / (1.0 + t2);
        omc_t = 2.0 / (1.0 + t2);
    }
    double cp = cos(phi), sp = sin(phi);
    double uperp = sqrt(ux * ux + uy * uy);
    double dux, duy, duz;
    if (uperp > 0.0) {
        dux = (ux / uperp) * uz * sin_t * cp - (uy / uperp) * u * sin_t * sp - ux * omc_t;
        duy = (uy / uperp) * uz * sin_t * cp + (ux / uperp) * u * sin_t * sp - uy * omc_t;
        duz = -uperp * sin_t * cp - uz * omc_t;
    } else {                                    /* u along z: rotate about any transverse axis */
        dux = u * sin_t * cp;
        duy = u * sin_t * sp;
        duz = -uz * omc_t;
    }
    va[0] += 0.5 * dux; va[1] += 0.5 * duy; va[2] += 0.5 * duz;
    vb[0] -= 0.5 * dux; vb[1] -= 0.5 * duy; vb[2] -= 0.5 * duz;
}

/* Per-cell Takizuka-Abe coefficient A_j of orc_ta_pair for a cell holding
 * N_j particles: n_j = w N_j / V_j (uniform weights, Sec. 8). */
double orc_ta_coefficient(const orc_params *p, double n_j, double lnlam, double dt)
{
    double mu = 0.5 * p->mass;
    double q2 = p->charge * p->charge;
    return q2 * q2 * n_j * lnlam * dt / (8.0 * ORC_PI * p->eps0 * p->eps0 * mu * mu);
}

/* NRL formulary electron-electron Coulomb logarithm, n in m^-3, T in eV,
 * clamped below at 2.  Used per cell when the logarithm depends on density. */
double orc_nrl_lnlambda(double n_m3, double T_eV)
{
    if (!(n_m3 > 0.0) || !(T_eV > 0.0)) return 2.0;
    double n_cm3 = n_m3 * 1e-6;
    double lt = log(T_eV);
    double v = 23.5 - log(sqrt(n_cm3) * pow(T_eV, -1.25)) - sqrt(1e-5 + (lt - 2.0) * (lt - 2.0) / 16.0);
    return v < 2.0 ? 2.0 : v;
}

/* ------------------------------------------------------------------------- *
 * Step S1 (Table 2), the Coulombic collision step of Table 5: group (CCS1-3),
 * pair consecutive entries of each cell's order, draw the pair's uniforms
 * (CCS4) and update both velocities (CCS5).  An odd cell's last particle sits
 * out (reading of "handled trivially").  With p->correction set, each cell's
 * velocities are then mapped v <- V0 + sqrt(K0/K1) (v - V1), where V0, K0 are
 * the cell's mean velocity and summed squared peculiar speed before the
 * update and V1, K1 after it; this restores both invariants after rounding.
 * Per-cell inputs: inv_vol = 1/V_j, lnlam = Coulomb logarithm, dt = step.
 * ------------------------------------------------------------------------- */
static void orc_cell_mean_k(const uint32_t *idx, uint64_t cnt, const double *vx, const double *vy,
                            const double *vz, double V[3], double *K)
{
    double sx = 0, sy = 0, sz = 0;
    for (uint64_t k = 0; k < cnt; ++k) { sx += vx[idx[k]]; sy += vy[idx[k]]; sz += vz[idx[k]]; }
    V[0] = sx / (double)cnt; V[1] = sy / (double)cnt; V[2] = sz / (double)cnt;
    double s = 0;
    for (uint64_t k = 0; k < cnt; ++k) {
        double dx = vx[idx[k]] - V[0], dy = vy[idx[k]] - V[1], dz = vz[idx[k]] - V[2];
        s += dx * dx + dy * dy + dz * dz;
    }
    *K = s;
}

int orc_coulomb_ids(int64_t n, int32_t M, const int32_t *cell, const uint32_t *ids, double *vx, double *vy,
                    double *vz, const double *inv_vol, const double *lnlam, const double *dt,
                    const orc_params *p, uint32_t step);

int orc_coulomb(int64_t n, int32_t M, const int32_t *cell, double *vx, double *vy, double *vz,
                const double *inv_vol, const double *lnlam, const double *dt,
                const orc_params *p, uint32_t step)
{
    return orc_coulomb_ids(n, M, cell, NULL, vx, vy, vz, inv_vol, lnlam, dt, p, step);
}

int orc_coulomb_ids(int64_t n, int32_t M, const int32_t *cell, const uint32_t *ids, double *vx, double *vy,
                    double *vz, const double *inv_vol, const double *lnlam, const double *dt,
                    const orc_params *p, uint32_t step)
{
    if (n < 0 || M <= 0) return ORC_EINVAL;
    uint64_t *cs = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)M + 1));
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!cs || !order) { free(cs); free(order); return ORC_EINVAL; }
    int rc = orc_pair_order_mode(n, M, cell, ids, p, step, cs, order);
    if (rc) { free(cs); free(order); return rc; }
    for (int32_t j = 0; j < M; ++j) {
        uint64_t s = cs[j], cnt = cs[j + 1] - cs[j];
        if (cnt < 2) continue;
        const uint32_t *o = order + s;
        double V0[3], K0 = 0;
        if (p->correction) orc_cell_mean_k(o, cnt, vx, vy, vz, V0, &K0);
        double A = orc_ta_coefficient(p, p->weight * (double)cnt * inv_vol[j], lnlam[j], dt[j]);
        for (uint64_t k = 0; k + 1 < cnt; k += 2) {            /* CCS4 + CCS5 per pair */
            uint32_t a = o[k], b = o[k + 1];
            uint64_t ia = orc_id(ids, a), ib = orc_id(ids, b);
            uint32_t w[4];
            orc_draw(p->seed, ia < ib ? ia : ib, step, ORC_TAG_PAIR, w);
            double va[3] = {vx[a], vy[a], vz[a]}, vb[3] = {vx[b], vy[b], vz[b]};
            orc_ta_pair(va, vb, A, w);
            vx[a] = va[0]; vy[a] = va[1]; vz[a] = va[2];
            vx[b] = vb[0]; vy[b] = vb[1]; vz[b] = vb[2];
        }
        if (p->correction) {
            double V1[3], K1;
            orc_cell_mean_k(o, cnt, vx, vy, vz, V1, &K1);
            double f = K1 > 0.0 ? sqrt(K0 / K1) : 1.0;
            for (uint64_t k = 0; k < cnt; ++k) {
                uint32_t l = o[k];
                vx[l] = V0[0] + f * (vx[l] - V1[0]);
                vy[l] = V0[1] + f * (vy[l] - V1[1]);
                vz[l] = V0[2] + f * (vz[l] - V1[2]);
            }
        }
    }
    free(cs); free(order);
    return ORC_OK;
}

/* ------------------------------------------------------------------------- *
 * Step S2a for electron-neutral collisions C1 (elastic) and C2 (ionization)
 * with the null-collision method of Sec. 4.2 (Vahedi & Surendra 1995).
 * Per cell j: nu_max = n_n (sigma_el + sigma_ion) v_max with v_max the largest
 * speed in the cell at this point of the step, P_null = 1 - exp(-nu_max dt_j).
 * Particle l (PARTICLE block words 1, 2) is a candidate iff U1 < P_null (in
 * the bijection pairing mode, cells of at least ORC_BIJ_MIN_N particles take
 * their candidates by pairing position instead, see below); a
 * candidate with r = U2 nu_max collides elastically if r < nu_el(v),
 * ionizes if r < nu_el(v) + nu_ion(v), and is otherwise a null collision.
 * Elastic: new direction uniform on the sphere (SCATTER words 0, 1), speed
 * from the energy loss (2m/M)(1 - cos chi) E off a cold neutral.
 * Ionization: E' = E - E_ion shared as U E' (secondary, SCATTER word 2) and
 * (1 - U) E' (primary); primary direction from SCATTER words 0, 1, secondary
 * direction from SECONDARY words 0, 1; the secondary takes the parent's cell
 * and position.  Secondaries are appended (Table 3 CS5) at
 * N_old + offset(cell) + rank of the parent inside the cell, cells in
 * ascending order and parents in the cell's pairing order of this step
 * (orc_pair_order_mode); reading: a deterministic form of the
 * paper's atomic global write index.  Optional outputs: `decision` (0 not a
 * candidate, 1 null, 2 elastic, 3 ionization) and `margin` (distance of the
 * deciding uniform to the nearest decision boundary, relative to 1).
 * ------------------------------------------------------------------------- */
static void orc_iso_dir(uint32_t wa, uint32_t wb, double d[3])
{
    double c = 1.0 - 2.0 * orc_uniform(wa);
    double s = sqrt(fmax(0.0, 1.0 - c * c));
    double ph = 2.0 * ORC_PI * orc_uniform(wb);
    d[0] = s * cos(ph); d[1] = s * sin(ph); d[2] = c;
}

int orc_neutral_ids(int64_t *n_io, int64_t capacity, int32_t M, int32_t *cell, const uint32_t *ids, double *x,
                    double *vx, double *vy, double *vz, const double *dt, const orc_params *p,
                    uint32_t step, int64_t *counts_out, int8_t *decision, double *margin);

int orc_neutral(int64_t *n_io, int64_t capacity, int32_t M, int32_t *cell, double *x,
                double *vx, double *vy, double *vz, const double *dt, const orc_params *p,
                uint32_t step, int64_t *counts_out /* [3]: candidates, elastic, ionization */,
                int8_t *decision, double *margin)
{
    return orc_neutral_ids(n_io, capacity, M, cell, NULL, x, vx, vy, vz, dt, p, step, counts_out, decision, margin);
}

/* With `ids`, random streams use ids[l]; appended secondaries get no id here
 * (ids[n..] is left to the caller). */
int orc_neutral_ids(int64_t *n_io, int64_t capacity, int32_t M, int32_t *cell, const uint32_t *ids, double *x,
                    double *vx, double *vy, double *vz, const double *dt, const orc_params *p,
                    uint32_t step, int64_t *counts_out, int8_t *decision, double *margin)
{
    int64_t n = *n_io;
    if (n < 0 || M <= 0) return ORC_EINVAL;
    double *vmax2 = (double *)calloc((size_t)M, sizeof(double));
    uint32_t *nion = (uint32_t *)calloc((size_t)M, sizeof(uint32_t));
    uint8_t *ionize = (uint8_t *)calloc((size_t)(n > 0 ? n : 1), 1);
    double *sec = (double *)malloc(sizeof(double) * 3 * (size_t)(n > 0 ? n : 1));
    /* bijection mode: candidates chosen by pairing position (see below) */
    const int bij = p->pairing_mode == ORC_PAIR_BIJECTION;
    int8_t *cand = bij ? (int8_t *)calloc((size_t)(n > 0 ? n : 1), 1) : NULL;
    double *cmarg = bij ? (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1)) : NULL;
    uint64_t *bcs = bij ? (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)M + 1)) : NULL;
    uint32_t *bord = bij ? (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1)) : NULL;
    if (!vmax2 || !nion || !ionize || !sec || (bij && (!cand || !cmarg || !bcs || !bord))) {
        free(vmax2); free(nion); free(ionize); free(sec); free(cand); free(cmarg); free(bcs); free(bord);
        return ORC_EINVAL;
    }
    for (int64_t l = 0; l < n; ++l) {
        if (cell[l] < 0) continue;                           /* removed at a wall */
        double v2 = vx[l] * vx[l] + vy[l] * vy[l] + vz[l] * vz[l];
        if (v2 > vmax2[cell[l]]) vmax2[cell[l]] = v2;
    }
    /* nu_max = n_n sigma_max v_max: sigma_max = sigma_el + sigma_ion for the
     * constant / step cross sections, the given bound with tables */
    const double sig_tot = (p->xs_el || p->xs_ion) ? p->sigma_max : p->sigma_el + p->sigma_ion;
    const double e_over_m = p->charge / p->mass;
    const int per_particle = p->selection == 1;
    /* Bijection mode, cells of at least ORC_BIJ_MIN_N particles: the paper
     * selects P_null N particles at random (Sec. 4.2).  Reading: the count is
     * n_c = floor(P_null N + U) with U the cell's candidate-count uniform
     * (orc_bij_setup), so that its mean is P_null N, and the candidates are
     * the particles at pairing positions 0 .. n_c - 1 of this step's order
     * (a uniformly random subset, since the positions are a keyed bijection
     * of the id ranks).  cmarg: distance of P_null N + U to the nearest
     * integer relative to P_null N (for the two particles next to the cut). */
    if (bij && !per_particle) {
        int rc0 = orc_pair_order_mode(n, M, cell, ids, p, step, bcs, bord);
        if (rc0) {
            free(vmax2); free(nion); free(ionize); free(sec); free(cand); free(cmarg); free(bcs); free(bord);
            return rc0;
        }
        for (int64_t l = 0; l < n; ++l) cmarg[l] = 1.0;
        for (int32_t j = 0; j < M; ++j) {
            uint64_t s0 = bcs[j], cnt = bcs[j + 1] - bcs[j];
            if (cnt < ORC_BIJ_MIN_N) continue;
            orc_bij B;
            orc_bij_setup(p->seed, orc_cell_id(p, j), step, (uint32_t)cnt, &B);
            double numax = p->n_neutral * sig_tot * sqrt(vmax2[j]);
            double pnull = -expm1(-numax * dt[j]);
            double t = pnull * (double)cnt + orc_uniform(B.u);
            uint64_t nc = (uint64_t)floor(t);
            if (nc > cnt) nc = cnt;
            double fr = t - floor(t);
            double cm = fmin(fr, 1.0 - fr) / fmax(pnull * (double)cnt, 1.0);
            for (uint64_t q = 0; q < cnt; ++q) cand[bord[s0 + q]] = q < nc ? 1 : -1;
            if (nc > 0) cmarg[bord[s0 + nc - 1]] = cm;
            if (nc < cnt) cmarg[bord[s0 + nc]] = cm;
        }
    }
    int64_t ncand = 0, nel = 0, nio = 0;
    for (int64_t l = 0; l < n; ++l) {
        int32_t j = cell[l];
        if (decision) decision[l] = 0;
        if (j < 0) { if (margin) margin[l] = 1.0; continue; }   /* removed at a wall */
        double numax = p->n_neutral * sig_tot * sqrt(vmax2[j]);
        double pnull = -expm1(-numax * dt[j]);
        uint32_t w[4];
        orc_draw(p->seed, orc_id(ids, (uint64_t)l), step, ORC_TAG_PARTICLE, w);
        double uc = orc_uniform(w[1]);
        int is_cand;
        if (per_particle) {
            /* Sec. 4.2's per-particle selection: pi_c = 1 - exp(-dt v sigma_c(v) n_n) for
             * each collision c, decided by U1 against pi_el, pi_el + pi_ion (reading: one
             * uniform, collisions in the order of Table 1) */
            double v2p = vx[l] * vx[l] + vy[l] * vy[l] + vz[l] * vz[l];
            double vp_ = sqrt(v2p), Ep_ = 0.5 * v2p / e_over_m;
            double pel = -expm1(-dt[j] * vp_ * orc_sig_el(p, Ep_) * p->n_neutral);
            double pio = -expm1(-dt[j] * vp_ * orc_sig_ion(p, Ep_) * p->n_neutral);
            int kind = uc < pel ? 2 : (uc < pel + pio ? 3 : 0);
            if (margin) {
                double mm = fmin(fabs(uc - pel), fabs(uc - pel - pio));
                if (p->xs_ion == NULL && p->sigma_ion > 0.0) mm = fmin(mm, fabs(Ep_ - p->e_ion) / p->e_ion);
                margin[l] = mm;
            }
            if (decision) decision[l] = (int8_t)kind;
            if (kind == 0) continue;
            ++ncand;
            uint32_t s_[4];
            orc_draw(p->seed, orc_id(ids, (uint64_t)l), step, ORC_TAG_SCATTER, s_);
            double d_[3];
            orc_iso_dir(s_[0], s_[1], d_);
            if (kind == 2) {
                ++nel;
                double cchi = (vx[l] * d_[0] + vy[l] * d_[1] + vz[l] * d_[2]) / vp_;
                double f = 1.0 - 2.0 * (p->mass / p->mass_neutral) * (1.0 - cchi);
                double vn = vp_ * sqrt(f);
                vx[l] = vn * d_[0]; vy[l] = vn * d_[1]; vz[l] = vn * d_[2];
            } else {
                ++nio;
                double Ep = fmax(Ep_ - p->e_ion, 0.0);
                double Es = orc_uniform(s_[2]) * Ep;
                double Eprim = Ep - Es;
                double vpr = sqrt(2.0 * Eprim * e_over_m), vs = sqrt(2.0 * Es * e_over_m);
                uint32_t t_[4];
                orc_draw(p->seed, orc_id(ids, (uint64_t)l), step, ORC_TAG_SECONDARY, t_);
                double ds_[3];
                orc_iso_dir(t_[0], t_[1], ds_);
                vx[l] = vpr * d_[0]; vy[l] = vpr * d_[1]; vz[l] = vpr * d_[2];
                sec[3 * l + 0] = vs * ds_[0]; sec[3 * l + 1] = vs * ds_[1]; sec[3 * l + 2] = vs * ds_[2];
                ionize[l] = 1;
                nion[j] += 1;
            }
            continue;
        }
        if (bij && cand[l] != 0) {                 /* cell paired by the bijection */
            is_cand = cand[l] > 0;
            if (margin) margin[l] = cmarg[l];
        } else {
            is_cand = uc < pnull;
            if (margin) margin[l] = fabs(uc - pnull);
        }
        if (!is_cand) continue;
        ++ncand;
        double v2 = vx[l] * vx[l] + vy[l] * vy[l] + vz[l] * vz[l];
        double v = sqrt(v2);
        double E = 0.5 * v2 / e_over_m;                           /* eV */
        double nu_el = p->n_neutral * orc_sig_el(p, E) * v;
        double nu_ion = p->n_neutral * orc_sig_ion(p, E) * v;
        double r = orc_uniform(w[2]) * numax;
        int kind = r < nu_el ? 2 : (r < nu_el + nu_ion ? 3 : 1);
        if (decision) decision[l] = (int8_t)kind;
        if (margin && numax > 0.0) {
            double m1 = fabs(r - nu_el) / numax, m2 = fabs(r - nu_el - nu_ion) / numax;
            double me = (p->xs_ion == NULL && p->sigma_ion > 0.0) ? fabs(E - p->e_ion) / p->e_ion : 1.0;
            double mm = margin[l];
            if (m1 < mm) mm = m1;
            if (m2 < mm) mm = m2;
            if (me < mm) mm = me;
            margin[l] = mm;
        }
        if (kind == 1) continue;
        uint32_t s[4];
        orc_draw(p->seed, orc_id(ids, (uint64_t)l), step, ORC_TAG_SCATTER, s);
        double d[3];
        orc_iso_dir(s[0], s[1], d);
        if (kind == 2) {
            ++nel;
            double cchi = (vx[l] * d[0] + vy[l] * d[1] + vz[l] * d[2]) / v;
            double f = 1.0 - 2.0 * (p->mass / p->mass_neutral) * (1.0 - cchi);
            double vn = v * sqrt(f);
            vx[l] = vn * d[0]; vy[l] = vn * d[1]; vz[l] = vn * d[2];
        } else {
            ++nio;
            double Ep = fmax(E - p->e_ion, 0.0);
            double Es = orc_uniform(s[2]) * Ep;
            double Eprim = Ep - Es;
            double vp = sqrt(2.0 * Eprim * e_over_m), vs = sqrt(2.0 * Es * e_over_m);
            uint32_t t[4];
            orc_draw(p->seed, orc_id(ids, (uint64_t)l), step, ORC_TAG_SECONDARY, t);
            double ds[3];
            orc_iso_dir(t[0], t[1], ds);
            vx[l] = vp * d[0]; vy[l] = vp * d[1]; vz[l] = vp * d[2];
            sec[3 * l + 0] = vs * ds[0]; sec[3 * l + 1] = vs * ds[1]; sec[3 * l + 2] = vs * ds[2];
            ionize[l] = 1;
            nion[j] += 1;
        }
    }
    int rc = ORC_OK;
    if (n + nio > capacity) {
        rc = ORC_ECAPACITY;
    } else {
        /* cells in ascending order; inside a cell, parents in pairing order */
        uint64_t *cs = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)M + 1));
        uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
        if (!cs || !order || orc_pair_order_mode(n, M, cell, ids, p, step, cs, order) != ORC_OK) {
            rc = ORC_EINVAL;
        } else {
            int64_t dst = n;
            for (int64_t k = 0; k < (int64_t)cs[M]; ++k) {   /* live particles (removed ones are not listed) */
                uint32_t l = order[k];
                if (!ionize[l]) continue;
                vx[dst] = sec[3 * l + 0]; vy[dst] = sec[3 * l + 1]; vz[dst] = sec[3 * l + 2];
                cell[dst] = cell[l];
                if (x) x[dst] = x[l];
                ++dst;
            }
            *n_io = n + nio;
        }
        free(cs); free(order);
    }
    if (counts_out) { counts_out[0] = ncand; counts_out[1] = nel; counts_out[2] = nio; }
    free(vmax2); free(nion); free(ionize); free(sec); free(cand); free(cmarg); free(bcs); free(bord);
    return rc;
}

/* ------------------------------------------------------------------------- *
 * Particle-to-cell moments, steps S3a/S3b of Table 2 (Sec. 4.5): plain
 * sequential sums per cell.  mom[10 j + k]:
 *   0 N_j, 1 sum w, 2..4 sum v_x, v_y, v_z, 5..7 sum v_x^2, v_y^2, v_z^2,
 *   8 sum sigma_el |v|, 9 sum sigma_ion(E) |v|   (rate sums C_kc / n_k).
 * hist[64 j + b]: counts over 64 log-spaced energy bins on [1e-2, 1e3] eV,
 * under- and overflow clamped into the end bins.
 * ------------------------------------------------------------------------- */
int orc_energy_bin(double E_eV)
{
    if (!(E_eV > 0.0)) return 0;
    double t = (log10(E_eV) + 2.0) * (64.0 / 5.0);
    if (t < 0.0) return 0;
    if (t >= 63.0) return 63;
    return (int)t;
}

int orc_moments(int64_t n, int32_t M, const int32_t *cell, const double *vx, const double *vy,
                const double *vz, const orc_params *p, double *mom, uint32_t *hist)
{
    if (n < 0 || M <= 0) return ORC_EINVAL;
    memset(mom, 0, sizeof(double) * 10 * (size_t)M);
    if (hist) memset(hist, 0, sizeof(uint32_t) * 64 * (size_t)M);
    const double e_over_m = p->charge / p->mass;
    for (int64_t l = 0; l < n; ++l) {
        int32_t j = cell[l];
        if (j == -1) continue;                               /* removed at a wall */
        if (j < 0 || j >= M) return ORC_EINVAL;
        double *m = mom + 10 * (size_t)j;
        double v2 = vx[l] * vx[l] + vy[l] * vy[l] + vz[l] * vz[l];
        double v = sqrt(v2);
        double E = 0.5 * v2 / e_over_m;
        m[0] += 1.0;
        m[1] += p->weight;
        m[2] += vx[l]; m[3] += vy[l]; m[4] += vz[l];
        m[5] += vx[l] * vx[l]; m[6] += vy[l] * vy[l]; m[7] += vz[l] * vz[l];
        m[8] += orc_sig_el(p, E) * v;
        m[9] += orc_sig_ion(p, E) * v;
        if (hist) hist[64 * (size_t)j + (size_t)orc_energy_bin(E)] += 1;
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------- *
 * Recombination C5 (Table 1: Ar+ + 2e -> Ar_m + e), the kernel of Sec. 4.3 and
 * Table 4 (RS0-RS5), run after C1/C2 in step S2a.  Every cell j with N_j
 * particles at the start of the step (the ones of this step's pairing order):
 *   RS0  the primaries: the paper takes them from CS3's per-particle
 *        probabilities.  Reading: a three-body rate k_rec [m^6/s] with the ion
 *        density equal to the electron density n_j = w N_j / V_j gives every
 *        electron P_rec = 1 - exp(-dt_j k_rec n_j^2); as for the null-collision
 *        candidates, the cell takes n_p = floor(P_rec N_j + U) of them (U from
 *        the Philox block (cell, step, RECOMB, 0), word 0), capped at N_j / 2,
 *        at the last n_p positions of the pairing order (a uniformly random
 *        subset);
 *   RS1  the catalyte list C_j: the cell's other particles; the paper builds it
 *        with an atomic cursor, here it is the pairing order itself;
 *   RS2-RS3  each primary pops a distinct catalyte: the r-th primary (position
 *        N_j - n_p + r) takes the catalyte at position N_j - 2 n_p + r;
 *   RS4  the catalyte takes the primary's kinetic energy, its own and the
 *        released energy dE_rec [eV] (reading: the binding energy left over
 *        when Ar_m forms), in an isotropic direction from words 0-1 of its
 *        RECOMB block;
 *   RS5  the primary is removed (w = 0; here cell = -1, as at an absorbing wall).
 * Pinned by the count law (floor/ceil of P_rec N, mean P_rec N), the unique
 * matching within cells, the removed count and the energy bookkeeping
 * (tests/test_oracle_recombination.py).
 * ------------------------------------------------------------------------- */
int orc_recombine(int64_t n, int32_t M, int32_t *cell, const uint32_t *ids, double *vx, double *vy, double *vz,
                  const double *inv_vol, const double *dt, const orc_params *p, uint32_t step, double k_rec,
                  double de_rec, int64_t *removed)
{
    if (n < 0 || M <= 0) return ORC_EINVAL;
    uint64_t *cs = (uint64_t *)malloc(sizeof(uint64_t) * ((size_t)M + 1));
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n > 0 ? n : 1));
    if (!cs || !order) { free(cs); free(order); return ORC_EINVAL; }
    int rc = orc_pair_order_mode(n, M, cell, ids, p, step, cs, order);
    if (rc) { free(cs); free(order); return rc; }
    const double e_over_m = p->charge / p->mass;
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    int64_t gone = 0;
    for (int32_t j = 0; j < M; ++j) {
        uint64_t s = cs[j], cnt = cs[j + 1] - cs[j];
        if (cnt < 2) continue;
        double nj = p->weight * (double)cnt * inv_vol[j];
        double prec = -expm1(-dt[j] * k_rec * nj * nj);
        uint32_t ctr[4] = {(uint32_t)orc_cell_id(p, j), step, ORC_TAG_RECOMB, 0u}, w[4];
        orc_philox4x32_10(ctr, key, w);
        double t = prec * (double)cnt + orc_uniform(w[0]);
        uint64_t np_ = (uint64_t)floor(t);
        if (np_ > cnt / 2) np_ = cnt / 2;
        for (uint64_t r = 0; r < np_; ++r) {
            uint32_t lp = order[s + cnt - np_ + r], lc = order[s + cnt - 2 * np_ + r];
            double ep = 0.5 * (vx[lp] * vx[lp] + vy[lp] * vy[lp] + vz[lp] * vz[lp]) / e_over_m;
            double ec = 0.5 * (vx[lc] * vx[lc] + vy[lc] * vy[lc] + vz[lc] * vz[lc]) / e_over_m;
            double sp = sqrt(2.0 * (ec + ep + de_rec) * e_over_m);
            uint32_t c[4];
            orc_draw(p->seed, orc_id(ids, lc), step, ORC_TAG_RECOMB, c);
            double d[3];
            orc_iso_dir(c[0], c[1], d);
            vx[lc] = sp * d[0]; vy[lc] = sp * d[1]; vz[lc] = sp * d[2];
            cell[lp] = -1;
            ++gone;
        }
    }
    free(cs); free(order);
    if (removed) *removed = gone;
    return ORC_OK;
}

/* ------------------------------------------------------------------------- *
 * Steps S2b (C2P) and S2c (push) of Table 2, CS6-CS7 of Table 3, on a 1D grid
 * of M cells of width dx along z (the field axis): Sec. 4.2 uses a constant
 * grad phi per cell, looked up by the particle's cell, so the acceleration of
 * particle l is accel[cell_l] (q E / m of its cell, m/s^2).  S2c writes the new
 * state from the old one:
 *   x+ = x + dt_j v_z,   v_z+ = v_z + dt_j accel_j,   j = cell_l (before the push);
 * then the particle is re-binned, cell = floor(x+ / dx) (a1's binning).
 * Boundary (CS7): periodic -- x+ is brought back into [0, L), L = M dx, by
 * adding or subtracting L (the displacement per step is below L) -- or
 * absorbing: a particle with x+ outside [0, L) is removed, which CS7 writes as
 * w = 0 and this oracle as cell = -1 (its velocity and position are kept and it
 * takes part in nothing afterwards).  Removed particles (cell < 0) are skipped.
 * Reading: S2c's Euler update is taken as printed (both from the pre-push
 * values).  Pinned by the closed-form K-step free flight, the energy gain
 * m a dx_l + m a^2 dt^2 / 2 per particle and step (an identity of this update),
 * numpy re-binning counts and absorbed counts (tests/test_oracle_push.py).
 * ------------------------------------------------------------------------- */
enum { ORC_BOUNDARY_PERIODIC = 0, ORC_BOUNDARY_ABSORB = 1 };

int orc_bin(double x, double dx, int32_t M)
{
    double f = floor(x / dx);
    if (!(f >= 0.0)) return 0;
    if (f >= (double)M) return M - 1;
    return (int32_t)f;
}

int orc_push(int64_t n, int32_t M, int32_t *cell, double *x, double *vz, const double *accel,
             const double *dt, double dx, int boundary, int64_t *absorbed)
{
    if (n < 0 || M <= 0 || !(dx > 0.0)) return ORC_EINVAL;
    const double L = dx * (double)M;
    int64_t gone = 0;
    for (int64_t l = 0; l < n; ++l) {
        int32_t j = cell[l];
        if (j < 0) continue;                               /* removed earlier */
        if (j >= M) return ORC_EINVAL;
        double x1 = x[l] + dt[j] * vz[l];
        double v1 = vz[l] + dt[j] * accel[j];
        vz[l] = v1;
        if (boundary == ORC_BOUNDARY_PERIODIC) {
            if (x1 < 0.0) x1 = x1 + L;
            else if (x1 >= L) x1 = x1 - L;
            if (x1 >= L || x1 < 0.0) x1 = 0.0;             /* rounding at the seam */
            x[l] = x1;
            cell[l] = orc_bin(x1, dx, M);
        } else {
            x[l] = x1;
            if (x1 < 0.0 || x1 >= L) { cell[l] = -1; ++gone; }
            else cell[l] = orc_bin(x1, dx, M);
        }
    }
    if (absorbed) *absorbed = gone;
    return ORC_OK;
}

/* One full collision step in the paper's order: S1 Coulomb, S2a electron-
 * neutral, S3 moments of the result.  Either collision can be switched off. */
int orc_step(int64_t *n_io, int64_t capacity, int32_t M, int32_t *cell, double *x,
             double *vx, double *vy, double *vz, const double *inv_vol, const double *lnlam,
             const double *dt, const orc_params *p, uint32_t step, int do_coulomb, int do_neutral,
             double *mom, uint32_t *hist, int64_t *counts_out)
{
    int rc = ORC_OK;
    if (counts_out) { counts_out[0] = counts_out[1] = counts_out[2] = 0; }
    if (do_coulomb) {
        rc = orc_coulomb(*n_io, M, cell, vx, vy, vz, inv_vol, lnlam, dt, p, step);
        if (rc) return rc;
    }
    if (do_neutral) {
        rc = orc_neutral(n_io, capacity, M, cell, x, vx, vy, vz, dt, p, step, counts_out, NULL, NULL);
        if (rc) return rc;
    }
    if (mom) rc = orc_moments(*n_io, M, cell, vx, vy, vz, p, mom, hist);
    return rc;
}
