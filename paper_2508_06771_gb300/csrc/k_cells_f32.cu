// k_cells_f32.cu -- float instantiations of the cell kernel (velocities and the
// collision arithmetic in binary32; the sums of a CTA's warps in binary32, of
// a cluster's CTAs in double).
#include "k_cells_inst.cuh"

namespace ltpc {

static const CellKernelEntry kF32[] = {
    CellKernel<float, 1, 256, 8>::entry(),    // 0: cells <= 2048
    CellKernel<float, 2, 256, 8>::entry(),    // 1: <= 4096
    CellKernel<float, 4, 256, 12>::entry(),   // 2: <= 12288
    CellKernel<float, 8, 256, 16>::entry(),   // 3: <= 32768
    CellKernel<float, 8, 512, 16>::entry(),   // 4: <= 65536
    CellKernel<float, 1, 512, 8>::entry(),    // 5: <= 4096
    CellKernel<float, 1, 1024, 12>::entry(),  // 6: <= 12288, one CTA per cell
    CellKernel<float, 1, 512, 24>::entry(),   // 7: <= 12288, one 512-thread CTA per cell
    CellKernel<float, 2, 1024, 12>::entry(),  // 8: <= 24576, clusters of two 1024-thread CTAs
    CellKernel<float, 4, 1024, 12>::entry(),  // 9: <= 49152, clusters of four 1024-thread CTAs
    HomeKernel<float, 1024, 12288>::entry(),  // 10: bijection cells <= 12288, home order, bulk copies
};

int cell_kernels_f32(const CellKernelEntry** out)
{
    *out = kF32;
    return (int)(sizeof(kF32) / sizeof(kF32[0]));
}

}  // namespace ltpc
