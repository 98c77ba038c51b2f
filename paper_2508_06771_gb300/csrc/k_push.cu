// k_push.cu -- steps S2b/S2c of Table 2 (CS6/CS7 of Table 3): the particle
// push in a constant field per cell, the re-binning that makes the per-step
// grouping (CCS1-CCS3) necessary, the walls, and the position-to-cell binning
// of a load.
//
// Geometry: M cells of width dx along the field axis z, domain [0, L), L = M dx.
// Sec. 4.2 precomputes grad phi per cell and looks it up by cell id; here the
// caller gives each cell's acceleration a_j = q E_j / m.  S2c as printed:
//   x+ = x + dt_j v_z,  v_z+ = v_z + dt_j a_j   (both from the pre-push state),
// then cell = floor(x+ / dx).  Walls: periodic (x+ brought back into [0, L)),
// or absorbing (CS7 sets w = 0; here the particle's cell becomes -1 and every
// later kernel skips it).  binary64 takes the products and sums without
// contraction, as the reference writes them.
#include <cuda_runtime.h>
#include <stdint.h>

#include "ltpc_internal.h"
#include "ltpc_launch.h"

namespace ltpc {

template <class T> struct PushMath;
template <> struct PushMath<double> {
    static __device__ __forceinline__ double madd(double x, double d, double v) { return __dadd_rn(x, __dmul_rn(d, v)); }
    static __device__ __forceinline__ double div(double x, double y) { return __ddiv_rn(x, y); }
};
template <> struct PushMath<float> {
    static __device__ __forceinline__ float madd(float x, float d, float v) { return fmaf(d, v, x); }
    static __device__ __forceinline__ float div(float x, float y) { return __fdiv_rn(x, y); }
};

template <class T>
__device__ __forceinline__ int32_t bin_of(T x, T dx, int32_t M)
{
    const T f = floor(PushMath<T>::div(x, dx));
    if (!(f >= T(0))) return 0;
    if (f >= (T)M) return M - 1;
    return (int32_t)f;
}

// One thread per particle (grid-stride).  The cell's dt comes from the pass's
// per-cell record (the product dt * dt_factor the collisions use).  After the
// push the storage no longer holds per-cell runs: the first thread clears the
// run bookkeeping so that the next grouping places every particle by cursor.
template <class T>
static __global__ void k_push(T* __restrict__ x, T* __restrict__ vz, int32_t* __restrict__ cell,
                              const double* __restrict__ accel, const double* __restrict__ cpar, int32_t M,
                              T dx, T L, int absorb, uint32_t* __restrict__ run_len, DevState* ds)
{
    const unsigned long long n = ds->n;
    const unsigned long long gt = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long l = gt; l < n; l += stride) {
        const int32_t j = cell[l];
        if (j < 0 || j >= M) continue;                     // removed at a wall
        const T dtj = (T)cpar[(size_t)j * NCP + CP_DT];
        const T v0 = vz[l];
        T x1 = PushMath<T>::madd(x[l], dtj, v0);
        vz[l] = PushMath<T>::madd(v0, dtj, (T)accel[j]);
        if (!absorb) {
            if (x1 < T(0)) x1 = x1 + L;
            else if (x1 >= L) x1 = x1 - L;
            if (x1 >= L || x1 < T(0)) x1 = T(0);           // rounding at the seam
            x[l] = x1;
            cell[l] = bin_of<T>(x1, dx, M);
        } else {
            x[l] = x1;
            cell[l] = (x1 < T(0) || x1 >= L) ? -1 : bin_of<T>(x1, dx, M);
        }
    }
    for (unsigned long long c = gt; c < (unsigned long long)M; c += stride) run_len[c] = 0u;
    if (gt == 0) {
        ds->n_sorted = 0ull;
        ds->n_loaded = n;
        ds->grouping_valid = 0u;
    }
}

// CCS1 of every step after a push: N_j of the live particles (cell -1 = removed,
// skipped silently; any other id outside [0, M) is an internal error).  Whole-warp
// loop with the full match mask, as the load-time histogram.
static __global__ void k_hist_step(const int32_t* __restrict__ cell, uint32_t* __restrict__ counts, int32_t M,
                                   DevState* ds)
{
    const unsigned long long n = ds->n;
    const unsigned long long n_up = (n + 31ull) & ~31ull;
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; l < n_up; l += stride) {
        int32_t c = l < n ? cell[l] : -1;
        if (c >= M || c < -1) {
            atomicOr(&ds->err, ERR_INDEX);
            c = -1;
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, c);
        const unsigned leader = __ffs(peers) - 1;
        if (c >= 0 && (threadIdx.x & 31u) == leader) atomicAdd(&counts[c], (uint32_t)__popc(peers));
    }
}

// a1's binning at load: cell = floor(x / dx) for x in [0, L); a position outside
// the domain or not finite is a bad cell (reported as EINVAL by the load).
template <class T>
static __global__ void k_bin(const T* __restrict__ x, int32_t* __restrict__ cell, int32_t M, T dx, T L, DevState* ds)
{
    const unsigned long long n = ds->n;
    for (unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; l < n;
         l += (unsigned long long)gridDim.x * blockDim.x) {
        const T xl = x[l];
        if (!(xl >= T(0) && xl < L)) {
            cell[l] = -2;                                  // out of range: the histogram reports it
            continue;
        }
        cell[l] = bin_of<T>(xl, dx, M);
    }
}

template <class T>
cudaError_t launch_push(T* x, T* vz, int32_t* cell, const double* accel, const double* cpar, int32_t M, double dx,
                        int absorb, uint32_t* run_len, DevState* ds, int grid, cudaStream_t s)
{
    k_push<T><<<grid, 256, 0, s>>>(x, vz, cell, accel, cpar, M, (T)dx, (T)(dx * (double)M), absorb, run_len, ds);
    return cudaGetLastError();
}
template cudaError_t launch_push<float>(float*, float*, int32_t*, const double*, const double*, int32_t, double, int,
                                        uint32_t*, DevState*, int, cudaStream_t);
template cudaError_t launch_push<double>(double*, double*, int32_t*, const double*, const double*, int32_t, double,
                                         int, uint32_t*, DevState*, int, cudaStream_t);

cudaError_t launch_hist_step(const int32_t* cell, uint32_t* counts, int32_t M, DevState* ds, int grid, cudaStream_t s)
{
    k_hist_step<<<grid, 256, 0, s>>>(cell, counts, M, ds);
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_bin(const T* x, int32_t* cell, int32_t M, double dx, DevState* ds, int grid, cudaStream_t s)
{
    k_bin<T><<<grid, 256, 0, s>>>(x, cell, M, (T)dx, (T)(dx * (double)M), ds);
    return cudaGetLastError();
}
template cudaError_t launch_bin<float>(const float*, int32_t*, int32_t, double, DevState*, int, cudaStream_t);
template cudaError_t launch_bin<double>(const double*, int32_t*, int32_t, double, DevState*, int, cudaStream_t);

}  // namespace ltpc
