// Kernel instantiations for the 6-point Gauss-Hermite tensor set (D2Q36).
#include "tvlbm_kernels_impl.cuh"

namespace tvlbm {
const KernelTable* kernel_table_q6() { return Launch<6>::table(); }
}  // namespace tvlbm
