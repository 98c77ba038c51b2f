// ltpc_launch.h -- launch-side declarations shared by the kernel translation
// units and the host runtime.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "ltpc_internal.h"

namespace ltpc {

constexpr int REGROUP_THREADS = 1024;

struct RegroupLists {
    int32_t n_classes;
    uint32_t max_n[MAX_CLASSES];   // largest cell of each class
    uint4* list[MAX_CLASSES];      // device work lists (M entries each): {cell, N_j, I_j, 1}
    int32_t cache_grouping;        // 1: skip CCS3 while the grouping is unchanged
    // Runs of a cell-grouped load: the loaded particles of cell c occupy
    // [run_start[c], run_start[c] + run_len[c]) (run_len 0 when the load was not
    // grouped by cell).  They take the first run_len[c] places of the cell's
    // grouping in index order; appended particles follow.
    uint32_t* run_start;
    uint32_t* run_len;
    // Slot of every appended particle in its cell's grouping: the cell's
    // count before the append plus the particle's rank among that pass's
    // secondaries of the cell.  The scatter places appended particles there
    // without atomics, after the loaded ones, in ascending index order.
    uint32_t* aslot;
    uint32_t* rec_count;           // [M] primaries removed by the last pass (recombination C5)
};

// One compiled shape of the cell kernel.
struct CellShape {
    int cluster;    // CTAs per cluster
    int threads;    // threads per CTA
    int items;      // positions per thread (positions per CTA = threads * items)
};

// Launch the cell kernel of `shape` over class list `cls`; `grid_ctas` (0 =
// query occupancy) is the number of CTAs, a multiple of the cluster size.
using CellLauncherF = cudaError_t (*)(const CellArgs<float>&, cudaStream_t, int grid_ctas);
using CellLauncherD = cudaError_t (*)(const CellArgs<double>&, cudaStream_t, int grid_ctas);
using CellOccupancyFn = cudaError_t (*)(int* clusters);

struct CellKernelEntry {
    CellShape shape;
    void* launcher;          // CellLauncherF or CellLauncherD
    CellOccupancyFn occupancy;
    size_t smem_bytes;
};

// Compiled shapes per precision (defined in k_cells_f32.cu / k_cells_f64.cu).
int cell_kernels_f32(const CellKernelEntry** out);
int cell_kernels_f64(const CellKernelEntry** out);

// Class tables: which compiled shapes handle which cell sizes.
struct ClassTable {
    int n;
    int kernel[MAX_CLASSES];   // index into the precision's kernel list
};
// Tables of a precision and pairing mode (the home-order kernel serves only
// the bijection mode's tables, and only above its key-sorted sizes).
int class_tables(int precision, int pairing_mode, const ClassTable** out);

// Host-side launchers of the grouping / bookkeeping kernels (k_group.cu).
cudaError_t launch_hist(const int32_t* cell, uint32_t* counts, int32_t M, DevState* ds, int grid, cudaStream_t s);
cudaError_t launch_scatter(const int32_t* cell, int32_t M, uint32_t* cursor, uint32_t* perm, const DevState* ds, int grid,
                           cudaStream_t s, const RegroupLists& runs, const uint32_t* cell_start,
                           const CellParamArgs* cp = nullptr);
cudaError_t launch_runs(const int32_t* cell, int32_t M, const uint32_t* counts, const RegroupLists& runs, DevState* ds,
                        int grid, cudaStream_t s, int require_grouped);
template <class T>
cudaError_t launch_compact_gather(const uint32_t* perm, uint32_t n, const T* a0, const T* a1, const T* a2,
                                  const int32_t* c, T* b0, T* b1, T* b2, int32_t* d, int grid, cudaStream_t s);
cudaError_t launch_reset_cursors(int32_t M, const uint32_t* cell_start, const RegroupLists& runs, uint32_t* cursor,
                                 cudaStream_t s);
cudaError_t launch_regroup(int32_t M, uint32_t* counts, uint32_t* cell_start, uint32_t* cs_prev, uint32_t* cursor,
                           uint32_t* ion_count, uint32_t* ion_off, const RegroupLists& lists,
                           unsigned long long capacity, int append, int advance_step, DevState* ds, cudaStream_t s);
template <class T>
cudaError_t launch_append(int32_t M, const uint32_t* ion_off, const uint32_t* cs_prev, const uint32_t* stage_l,
                          const T* svx, const T* svy, const T* svz, T* vx, T* vy, T* vz, int32_t* cell, T* x,
                          uint32_t* aslot, const DevState* ds, int grid, cudaStream_t s);
cudaError_t launch_set_state(DevState* ds, unsigned long long n, int set_n, uint32_t step, double dt, int set_step,
                             cudaStream_t s);
// Steps S2b/S2c and the per-step grouping after them (k_push.cu).
template <class T>
cudaError_t launch_push(T* x, T* vz, int32_t* cell, const double* accel, const double* cpar, int32_t M, double dx,
                        int absorb, uint32_t* run_len, DevState* ds, int grid, cudaStream_t s);
cudaError_t launch_hist_step(const int32_t* cell, uint32_t* counts, int32_t M, DevState* ds, int grid, cudaStream_t s);
template <class T>
cudaError_t launch_bin(const T* x, int32_t* cell, int32_t M, double dx, DevState* ds, int grid, cudaStream_t s);
template <class T>
cudaError_t launch_check_finite(const T* vx, const T* vy, const T* vz, DevState* ds, int grid, cudaStream_t s);

}  // namespace ltpc
