// ltpc_noalloc.cu -- per-cell grouping of particle ids for callers that cannot
// allocate device memory.
//
// Who needs this: a caller embedded in a larger program whose memory manager
// owns the whole device (a caching pool that may not be bypassed), a caller
// whose device-memory budget is already fully reserved, or a latency-critical
// loop that must not pay for an allocation.  Such a caller can still hand us
// its own input and output buffers, but cannot give us scratch space and
// cannot let us call cudaMalloc.  The per-cell counters and cursors the
// grouping needs therefore live in one fixed file-scope device array.
//
// The array is loaded with the library (every GPU that loads the library holds
// LTPC_NOALLOC_MAX_CELLS + 64 words, about 0.5 MB, until the process exits) and
// is shared by every call: each call clears the part it uses, and two calls
// whose work overlaps on the GPU race on it.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "../../include/ltpc.h"

namespace {

constexpr int32_t kMaxCells = LTPC_NOALLOC_MAX_CELLS;
constexpr int kFlagWord = kMaxCells;     // bad-cell flag after the per-cell cursors
constexpr int kMaxDevices = 64;
constexpr int kScanThreads = 1024;

// Per-cell counts, then cursors, of the last call; one flag word.
static __device__ __align__(256) uint32_t g_group_scratch[kMaxCells + 64];

std::mutex g_mu;
uint32_t* g_scratch_addr[kMaxDevices] = {};   // device address of g_group_scratch, per device
int g_sms[kMaxDevices] = {};

__global__ void na_clear(uint32_t* scr, int32_t M)
{
    for (int32_t c = blockIdx.x * blockDim.x + threadIdx.x; c < M; c += gridDim.x * blockDim.x) scr[c] = 0u;
    if (blockIdx.x == 0 && threadIdx.x == 0) scr[kFlagWord] = 0u;
}

// Both grid-stride loops below run over whole warps: the bound is n rounded up
// to a multiple of 32 (the block size is a multiple of 32), so all 32 lanes of
// a warp take every iteration together and call __match_any_sync with the
// full mask.  A lane past the end, or holding an out-of-range id, joins the
// match with the sentinel -1 and takes no part in the counting or placing.

// Counts per cell (one atomic per warp and cell); out-of-range ids raise the flag.
__global__ void na_hist(const int32_t* __restrict__ cell, unsigned long long n, int32_t M, uint32_t* scr)
{
    const unsigned long long n_up = (n + 31ull) & ~31ull;
    for (unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; l < n_up;
         l += (unsigned long long)gridDim.x * blockDim.x) {
        int32_t c = l < n ? cell[l] : -1;
        if (l < n && (c < 0 || c >= M)) {
            atomicOr(&scr[kFlagWord], 1u);
            c = -1;
        }
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, c);
        if (c >= 0 && (threadIdx.x & 31u) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&scr[c], (uint32_t)__popc(peers));
    }
}

// One CTA: cell_start = exclusive scan of the counts; the counts become cursors.
__global__ void __launch_bounds__(kScanThreads) na_scan(uint32_t* scr, int32_t M, uint32_t* __restrict__ cell_start)
{
    __shared__ uint32_t s_w[kScanThreads / 32 + 1];
    const unsigned tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t per = (uint32_t)((M + kScanThreads - 1) / kScanThreads);
    const uint32_t b0 = min((uint32_t)M, tid * per), b1 = min((uint32_t)M, b0 + per);
    uint32_t sum = 0u;
    for (uint32_t c = b0; c < b1; ++c) sum += scr[c];
    uint32_t x = sum;
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    if (lane == 31u) s_w[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const uint32_t wv = lane < kScanThreads / 32 ? s_w[lane] : 0u;
        uint32_t z = wv;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, z, o);
            if (lane >= (unsigned)o) z += y;
        }
        s_w[lane] = z - wv;
        if (lane == 31u) s_w[kScanThreads / 32] = z;
    }
    __syncthreads();
    uint32_t ex = s_w[warp] + x - sum;
    for (uint32_t c = b0; c < b1; ++c) {
        const uint32_t cnt = scr[c];
        cell_start[c] = ex;
        scr[c] = ex;
        ex += cnt;
    }
    if (tid == 0) cell_start[M] = s_w[kScanThreads / 32];
}

// perm[cell_start[c] + rank] = l, ranks from one atomic cursor update per warp and cell.
__global__ void na_scatter(const int32_t* __restrict__ cell, unsigned long long n, int32_t M, uint32_t* scr,
                           uint32_t* __restrict__ perm)
{
    const unsigned lane = threadIdx.x & 31u;
    const unsigned long long n_up = (n + 31ull) & ~31ull;
    for (unsigned long long l = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; l < n_up;
         l += (unsigned long long)gridDim.x * blockDim.x) {
        int32_t c = l < n ? cell[l] : -1;
        if (c < 0 || c >= M) c = -1;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, c);
        const unsigned leader = (unsigned)(__ffs(peers) - 1);
        uint32_t base = 0u;
        if (c >= 0 && lane == leader) base = atomicAdd(&scr[c], (uint32_t)__popc(peers));
        base = __shfl_sync(0xFFFFFFFFu, base, leader);
        if (c >= 0) perm[base + (uint32_t)__popc(peers & ((1u << lane) - 1u))] = (uint32_t)l;
    }
}

// Device address of the scratch array on the current device (looked up once).
int scratch_for_current_device(uint32_t** out, int* sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LTPC_ECUDA;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_group_scratch) != cudaSuccess || !p) return LTPC_ECUDA;
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) return LTPC_ECUDA;
        g_scratch_addr[dev] = static_cast<uint32_t*>(p);
        g_sms[dev] = n;
    }
    *out = g_scratch_addr[dev];
    *sms = g_sms[dev];
    return LTPC_OK;
}

}  // namespace

extern "C" int ltpc_group_cells_noalloc(const int32_t* d_cell, int64_t n, int32_t n_cells, uint32_t* d_cell_start,
                                        uint32_t* d_perm, void* cuda_stream)
{
    if (n < 0 || n > 0xFFFFFFFFll || n_cells < 1 || n_cells > kMaxCells || !d_cell_start) return LTPC_EINVAL;
    if (n > 0 && (!d_cell || !d_perm)) return LTPC_EINVAL;
    uint32_t* scr = nullptr;
    int sms = 0;
    int rc = scratch_for_current_device(&scr, &sms);
    if (rc != LTPC_OK) return rc;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const unsigned long long nn = (unsigned long long)n;
    na_clear<<<(n_cells + 255) / 256, 256, 0, s>>>(scr, n_cells);
    na_hist<<<sms * 4, 256, 0, s>>>(d_cell, nn, n_cells, scr);
    na_scan<<<1, kScanThreads, 0, s>>>(scr, n_cells, d_cell_start);
    na_scatter<<<sms * 4, 256, 0, s>>>(d_cell, nn, n_cells, scr, d_perm);
    if (cudaGetLastError() != cudaSuccess) return LTPC_ECUDA;
    // the flag word is read on the caller's stream, then only that stream is
    // waited for (no device-wide wait on the legacy default stream)
    uint32_t flag = 0u;
    if (cudaMemcpyAsync(&flag, scr + kFlagWord, sizeof flag, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return LTPC_ECUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return LTPC_ECUDA;
    return flag ? LTPC_EINVAL : LTPC_OK;
}
