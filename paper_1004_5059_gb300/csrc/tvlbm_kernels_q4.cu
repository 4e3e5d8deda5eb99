// Kernel instantiations for the 4-point Gauss-Hermite tensor set (D2Q16).
#include "tvlbm_kernels_impl.cuh"

namespace tvlbm {
const KernelTable* kernel_table_q4() { return Launch<4>::table(); }
}  // namespace tvlbm
