// ltpc_internal.h -- structures shared by the host runtime and the kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "philox.cuh"
#include "xsec.cuh"

namespace ltpc {

// Device-detected error bits (reported by ltpc_sync as LTPC_E* codes).
enum : uint32_t {
    ERR_CAPACITY = 1u,       // appended secondaries would exceed the capacity
    ERR_TIMEOUT = 2u,        // a bounded device-side wait gave up
    ERR_NONFINITE = 4u,      // a loaded velocity is not finite
    ERR_INDEX = 8u,          // an internal index failed its bounds check (bug guard)
    ERR_CELL_TOO_LARGE = 16u,// a cell exceeds the largest cluster class
    ERR_BAD_CELL = 32u,      // a loaded cell id is outside [0, M)
    ERR_UNGROUPED = 64u,     // the bijection pairing mode was given storage not grouped by cell
};

// What one pass of the cell kernel does.
enum : uint32_t {
    F_COULOMB = 1u,          // step S1: Takizuka-Abe pair collisions
    F_NEUTRAL = 2u,          // step S2a: electron-neutral null-collision sampling
    F_CORRECTION = 4u,       // restore per-cell momentum and energy after S1
    F_LNL_NRL = 8u,          // Coulomb logarithm from the cell's previous moments
    F_PUSH = 16u,            // host only: the pass ends with steps S2b/S2c (a field is set)
    F_RECOMB = 32u,          // recombination C5 after the electron-neutral collisions
};

constexpr int MAX_CLASSES = 8;
constexpr int NMOM = 10;     // moments per cell
constexpr int NBIN = 64;     // energy-histogram bins per cell

// Small device-resident state.  Step number and dt live here so that a
// captured CUDA graph can be replayed for any step.
struct DevState {
    unsigned long long n;             // particles currently stored
    unsigned int err;                 // ERR_* bits, sticky until read
    unsigned int step;                // step number used by the next pass
    double dt;                        // base time step (cell dt = dt * dt_factor[j])
    unsigned int class_n[MAX_CLASSES];// cells in each cluster-class work list
    unsigned int ticket[MAX_CLASSES]; // dynamic work counters, reset every step
    unsigned int n_ion;               // secondaries appended by the last pass
    unsigned int max_count;           // largest cell at the last regrouping
    unsigned int grouping_valid;      // 1: perm still groups the particles (no load, no append since)
    unsigned int load_unsorted;       // 1: the loaded storage is not grouped by cell
    unsigned long long n_sorted;      // particles [0, n_sorted) lie in per-cell runs (cell-grouped load)
    unsigned long long n_loaded;      // particles [n_loaded, n) were appended: each has its slot in its
                                      // cell's grouping (RegroupLists::aslot)
    unsigned int ungroup;             // 1: a pass removed particles; the next regrouping drops the runs
};

// Per-cell scalars of one pass, formed by a grid-wide loop at the start of
// the pass (in the scatter kernel) from the cell's inputs and the moments of
// the previous pass, so that the cell kernel reads them instead of deriving
// them on one thread while its CTA waits.  Twelve doubles per cell.
enum : int {
    CP_A = 0,        // Takizuka-Abe coefficient: <delta^2> = A / |u|^3 (includes lnL and dt of the cell)
    CP_DT = 1,       // dt of the cell
    CP_K0 = 2,       // sum of squared peculiar speeds of the cell (restoration), -1: recompute in the pass
    CP_C = 3,        // 3..5: mean velocity of the cell (restoration target and centring shift)
    CP_INVN = 6,     // 1 / N_j
    CP_LNL = 7,      // Coulomb logarithm used
    CP_F32 = 8,      // 8..11: binary32 copies of A, dt, the mean velocity, K0 and 1 / N_j (seven floats)
    CP_BIJ = 12,     // 12..16: the bijection pairing of the cell as ten 32-bit words (CPB_*), all zero
                     // when the cell is paired by the key sort
    NCP = 18
};
// Words of the bijection record (bijection.cuh).
enum : int {
    CPB_AB = 0,      // a | b << 16 (0: key sort)
    CPB_MB = 1,      // ceil(2^32 / b)
    CPB_KEY = 2,     // 2..7: the six round keys
    CPB_U = 8,       // candidate-count rounding word
    CPB_NREC = 9,    // recombination C5: primaries of the cell this pass (0 when off)
    CPB_WORDS = 10
};
struct CellParamArgs {
    const uint32_t* counts;      // N_j of this pass
    const double* mom;           // moments of the previous pass (or of the load)
    const double* inv_vol;
    const double* dt_factor;
    const double* lnlam;
    double* cpar;                // [M][NCP] out; nullptr: not formed
    double coef0, weight, e_over_m;
    int lnl_nrl;                 // 1: Coulomb logarithm by the NRL e-e formula
    int bijection;               // 1: cells of BIJ_MIN_N..BIJ_MAX_N particles are paired by the bijection
    PhiloxKeys keys;             // round keys of the seed (the bijection's round keys are drawn per cell)
    double k_rec;                // three-body recombination rate [m^6/s] (0: no C5)
};

// Arguments of the cell kernel (one cluster per cell).
template <class T>
struct CellArgs {
    T* vx; T* vy; T* vz;
    uint32_t n_cap;              // length of the particle arrays (capacity)
    const uint32_t* perm;        // particle ids grouped by cell (CCS3 output)
    const uint32_t* counts;      // N_j
    const uint32_t* cell_start;  // I_j
    const double* cpar;          // [M][NCP] per-cell scalars of this pass
    double* mom;                 // [M][NMOM]
    uint32_t* hist;              // [M][NBIN]
    uint32_t* ion_count;         // [M] secondaries staged by this pass
    uint32_t* stage_l;           // parent id of each staged secondary
    T* stage_vx; T* stage_vy; T* stage_vz;
    DevState* ds;
    const uint4* list;           // work items of this class: {cell j, N_j, I_j, 1}
    uint32_t cls;
    uint32_t flags;
    uint64_t seed;
    PhiloxKeys keys;             // round keys of the seed
    double coef0;                // q^4 w / (8 pi eps0^2 mu^2), mu = m/2
    double weight, mass, e_over_m;
    double n_neutral, sigma_el, sigma_ion, e_ion, mratio2;  // mratio2 = 2 m / M
    // the same constants in the working precision (computed on the host)
    T c_half_m_over_e;           // m / (2 e): squared speed -> energy in eV
    T c_two_e_over_m;            // 2 e / m: energy in eV -> squared speed
    T c_nsig_el, c_nsig_ion;     // n_n sigma_el, n_n sigma_ion
    T c_nsig_tot;                // n_n (sigma_el + sigma_ion), rounded once
    T c_e_ion, c_mratio2;
    T c_nn;                      // n_n, for the tabulated cross sections
    T c_sig_el, c_sig_ion;       // the constant cross sections (tables on, one of them absent)
    XsArgs xs;                   // tabulated sigma_el(E), sigma_ion(E); per-particle selection
    int32_t* cell;               // cell id of every particle (C5 marks removed primaries with -1)
    uint32_t* rec_count;         // [M] primaries removed by this pass (C5)
    T c_de_rec;                  // energy released to the catalyte [eV]
    const uint32_t* run_start;   // [M] first index of each cell's loaded run (storage grouped by cell)
    const uint32_t* run_len;     // [M] its length (0: not grouped)
    uint32_t* order_out;         // optional: pairing order written at I_j + position
    void* xg;                    // bijection mode, clusters: one record {v, id} per particle, at
                                 // I_j + position, then I_j + home (Xg<T>); null in the key mode
    unsigned long long* phase_clk; // optional: SM cycles spent per kernel phase (tracing)
};

}  // namespace ltpc
