// k_cells_inst.cuh -- launch wrapper for one compiled shape of the cell kernel.
#pragma once
#include "k_cells.cuh"
#include "k_home.cuh"
#include "ltpc_launch.h"

namespace ltpc {

template <class T, int C, int NT, int ITEMS>
struct CellKernel {
    static constexpr uint32_t capl = (uint32_t)NT * ITEMS;
    static size_t smem() { return cells_dyn_smem<T>(capl); }
    static cudaLaunchConfig_t config(cudaLaunchAttribute* attr, int grid, cudaStream_t st)
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3((unsigned)grid, 1, 1);
        cfg.blockDim = dim3(NT, 1, 1);
        cfg.dynamicSmemBytes = smem();
        cfg.stream = st;
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        return cfg;
    }
    // Raise the dynamic shared-memory limit once per process (not a stream
    // operation, so it never runs inside a graph capture after the first call).
    static cudaError_t prepare()
    {
        static cudaError_t once = cudaFuncSetAttribute(k_cells<T, C, NT, ITEMS>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem());
        return once;
    }
    static cudaError_t occupancy(int* clusters)
    {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = config(attr, C, 0);
        return cudaOccupancyMaxActiveClusters(clusters, k_cells<T, C, NT, ITEMS>, &cfg);
    }
    static cudaError_t launch(const CellArgs<T>& a, cudaStream_t st, int grid_ctas)
    {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        if (grid_ctas <= 0) {
            int cl = 0;
            e = occupancy(&cl);
            if (e != cudaSuccess) return e;
            grid_ctas = (cl > 0 ? cl : 1) * C;
        }
        cudaLaunchAttribute attr[1];
        cudaLaunchConfig_t cfg = config(attr, grid_ctas, st);
        return cudaLaunchKernelEx(&cfg, k_cells<T, C, NT, ITEMS>, a);
    }
    static CellKernelEntry entry()
    {
        CellKernelEntry k;
        k.shape = CellShape{C, NT, ITEMS};
        k.launcher = (void*)&launch;
        k.occupancy = &occupancy;
        k.smem_bytes = smem();
        return k;
    }
};

// Launch wrapper of the home-order kernel of the bijection pairing mode
// (one CTA of NT threads per cell of up to CAPL particles).  Two compiled
// forms: constant cross sections, and tabulated ones (chosen per launch).
template <class T, int NT, int CAPL>
struct HomeKernel {
    static size_t smem() { return home_dyn_smem<T>((uint32_t)CAPL); }
    static cudaError_t prepare()
    {
        static cudaError_t once = cudaFuncSetAttribute(k_home<T, NT, CAPL, false>,
                                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem());
        static cudaError_t once_xs = cudaFuncSetAttribute(k_home<T, NT, CAPL, true>,
                                                          cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem());
        return once != cudaSuccess ? once : once_xs;
    }
    static cudaError_t occupancy(int* ctas)
    {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        int a = 0, b = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_home<T, NT, CAPL, false>, NT, smem());
        if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_home<T, NT, CAPL, true>, NT, smem());
        *ctas = a < b ? a : b;
        return e;
    }
    static cudaError_t occupancy_grid(int* ctas)
    {
        int per_sm = 0, dev = 0, sms = 0;
        cudaError_t e = occupancy(&per_sm);
        if (e == cudaSuccess) e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        *ctas = per_sm * sms;
        return e;
    }
    static cudaError_t launch(const CellArgs<T>& a, cudaStream_t st, int grid_ctas)
    {
        cudaError_t e = prepare();
        if (e != cudaSuccess) return e;
        if (grid_ctas <= 0) {
            e = occupancy_grid(&grid_ctas);
            if (e != cudaSuccess) return e;
            if (grid_ctas <= 0) grid_ctas = 1;
        }
        if (a.xs.on)
            k_home<T, NT, CAPL, true><<<grid_ctas, NT, smem(), st>>>(a);
        else
            k_home<T, NT, CAPL, false><<<grid_ctas, NT, smem(), st>>>(a);
        return cudaGetLastError();
    }
    static CellKernelEntry entry()
    {
        CellKernelEntry k;
        k.shape = CellShape{1, NT, CAPL / NT};
        k.launcher = (void*)&launch;
        k.occupancy = &occupancy_grid_per_sm;
        k.smem_bytes = smem();
        return k;
    }
    // clusters (here: CTAs) resident on the whole GPU, as CellKernel::occupancy reports
    static cudaError_t occupancy_grid_per_sm(int* clusters) { return occupancy_grid(clusters); }
};

}  // namespace ltpc
