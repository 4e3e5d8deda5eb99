// Tiled sweep (shared-memory staged source windows).  Declared here; defined below.
#pragma once
#include "tvlbm_kernels.cuh"

namespace tvlbm {

template <int N1>
inline int tiled_supported(int storage) { (void)storage; return 0; }

template <int N1, class C>
inline cudaError_t tiled_sweep(const typename C::T* fin, typename C::T* fout, const KParams& p, cudaStream_t s) {
    (void)fin; (void)fout; (void)p; (void)s;
    return cudaErrorNotSupported;
}

}  // namespace tvlbm
