// Kernel instantiations for the 3-point Gauss-Hermite tensor set (D2Q9).
#include "tvlbm_kernels_impl.cuh"

namespace tvlbm {
const KernelTable* kernel_table_q3() { return Launch<3>::table(); }
}  // namespace tvlbm
