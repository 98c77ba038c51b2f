// k_cells_f64.cu -- double instantiations of the cell kernel (the plain FP64
// form: velocities, collision arithmetic and sums in binary64).
#include "k_cells_inst.cuh"

namespace ltpc {

static const CellKernelEntry kF64[] = {
    CellKernel<double, 1, 256, 8>::entry(),   // 0: cells <= 2048
    CellKernel<double, 2, 256, 8>::entry(),   // 1: <= 4096
    CellKernel<double, 4, 256, 12>::entry(),  // 2: <= 12288
    CellKernel<double, 8, 256, 16>::entry(),  // 3: <= 32768
    CellKernel<double, 8, 512, 12>::entry(),  // 4: <= 49152
    CellKernel<double, 1, 512, 8>::entry(),   // 5: <= 4096
    CellKernel<double, 1, 1024, 6>::entry(),  // 6: <= 6144, one CTA per cell
    CellKernel<double, 2, 1024, 6>::entry(),  // 7: <= 12288
    HomeKernel<double, 1024, 6144>::entry(),  // 8: bijection cells <= 6144, home order, bulk copies
};

int cell_kernels_f64(const CellKernelEntry** out)
{
    *out = kF64;
    return (int)(sizeof(kF64) / sizeof(kF64[0]));
}

}  // namespace ltpc
