// Conserved sums that allocate nothing: for callers that cannot call cudaMalloc (code running
// inside another runtime's allocator, a stream-ordered pipeline that owns all device memory, an
// embedded host without an allocator on this path).  Same reduction as tvlbm_conserved_sums, but
// on a packed [Q][ny][nx] population array the caller owns, writing to an output the caller
// owns; the per-block partial sums live in a fixed file-scope device array.
#include <cuda_runtime.h>

#include <mutex>

#include "tvlbm.h"
#include "tvlbm_reduce.cuh"

namespace {

using namespace tvlbm;

// Fixed scratch: kRedBlocks blocks x 5 partial sums.  Every GPU that loads the library keeps
// this array until the process exits.  Each call overwrites all of it, so nothing needs to be
// cleared between calls; calls whose kernels overlap on the GPU race on it.
static __device__ __align__(256) double g_static_partials[kRedBlocks * 5];

// The summation body is the context's (tvlbm_reduce.cuh) on the packed cell source, so the two
// entry points add the same cells in the same order.
template <int N1, class C>
cudaError_t launch_packed(const void* f, int ncell, double rho0, double* partials, double* out5, const KParams& p,
                          cudaStream_t s) {
    reduce_packed_kernel<N1, C><<<kRedBlocks, 256, 0, s>>>((const typename C::T*)f, ncell, rho0, partials, p);
    reduce_final_kernel<<<1, 256, 0, s>>>(partials, out5);
    return cudaGetLastError();
}

template <int N1>
cudaError_t dispatch_storage(int storage, const void* f, int ncell, double rho0, double* partials, double* out5,
                             const KParams& p, cudaStream_t s) {
    switch (storage) {
        case ST_FP64: return launch_packed<N1, CodecF64>(f, ncell, rho0, partials, out5, p, s);
        case ST_FP32: return launch_packed<N1, CodecF32>(f, ncell, rho0, partials, out5, p, s);
        case ST_BF16_DEV: return launch_packed<N1, CodecBF16Dev>(f, ncell, rho0, partials, out5, p, s);
        case ST_FP16_DEV: return launch_packed<N1, CodecF16Dev>(f, ncell, rho0, partials, out5, p, s);
        case ST_FP32_DEV: return launch_packed<N1, CodecF32Dev>(f, ncell, rho0, partials, out5, p, s);
        default: return cudaErrorInvalidValue;
    }
}

// Device address of g_static_partials on the current device.  Outside stream capture it is looked
// up on every call (a device reset reloads the module, and the array may then sit elsewhere) and
// remembered; a call on a capturing stream uses the address the last uncaptured call on this
// device saw, and fails if there was none.
std::mutex g_addr_mutex;
void* g_addr[64];

int static_scratch(cudaStream_t s, void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TVLBM_ECUDA;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) return TVLBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (cs == cudaStreamCaptureStatusNone) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_partials) != cudaSuccess || !ptr) return TVLBM_ECUDA;
        g_addr[dev] = ptr;
    } else if (!g_addr[dev]) {
        return TVLBM_ECUDA;
    }
    *out = g_addr[dev];
    return TVLBM_OK;
}

}  // namespace

extern "C" int tvlbm_conserved_sums_static(const void* populations, int velset, int storage, int nx, int ny,
                                           double rho0, double* out5, void* stream) {
    const int n1 = velset == TVLBM_D2Q9 ? 3 : velset == TVLBM_D2Q16 ? 4 : velset == TVLBM_D2Q36 ? 6 : 0;
    if (!populations || !out5 || !n1 || nx < 1 || ny < 1 || !(rho0 > 0.0)) return TVLBM_EINVAL;
    if (storage < TVLBM_FP64 || storage > TVLBM_FP32_DEV) return TVLBM_EINVAL;
    // 32-bit indexing of the packed array: at most 2^31 - 1 populations
    if ((long long)nx * ny * n1 * n1 > 2147483647LL) return TVLBM_EINVAL;
    double xs[kMaxN1], ws[kMaxN1], cx[kMaxQ], cy[kMaxQ], w[kMaxQ];
    int order = 0;
    if (tvlbm_velocity_set(velset, cx, cy, w, &order) != TVLBM_OK) return TVLBM_EINVAL;
    KParams p = {};
    for (int i = 0; i < n1; ++i) {
        xs[i] = cx[i];                          // l = i + n1 * 0: nodes along x
        ws[i] = 0.0;
        for (int j = 0; j < n1; ++j) ws[i] += w[i + n1 * j];  // marginal weight of node i
        p.xd[i] = xs[i];
        p.wd[i] = ws[i];
    }
    void* scratch = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    const int rc = static_scratch(s, &scratch);
    if (rc) return rc;
    cudaError_t e;
    const int ncell = nx * ny;
    switch (n1) {
        case 3: e = dispatch_storage<3>(storage, populations, ncell, rho0, (double*)scratch, out5, p, s); break;
        case 4: e = dispatch_storage<4>(storage, populations, ncell, rho0, (double*)scratch, out5, p, s); break;
        default: e = dispatch_storage<6>(storage, populations, ncell, rho0, (double*)scratch, out5, p, s); break;
    }
    return e == cudaSuccess ? TVLBM_OK : TVLBM_ECUDA;
}
