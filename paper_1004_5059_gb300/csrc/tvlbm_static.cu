// Conserved sums that allocate nothing: for callers that cannot call cudaMalloc (code running
// inside another runtime's allocator, a stream-ordered pipeline that owns all device memory, an
// embedded host without an allocator on this path).  Same reduction as tvlbm_conserved_sums, but
// on a packed [Q][ny][nx] population array the caller owns, writing to an output the caller
// owns; the per-block partial sums live in a fixed file-scope device array.
#include <cuda_runtime.h>

#include <mutex>

#include "tvlbm.h"
#include "tvlbm_kernels.cuh"

namespace {

using namespace tvlbm;

// Fixed scratch: kRedBlocks blocks x 5 partial sums.  Every GPU that loads the library keeps
// this array until the process exits.  Each call overwrites all of it, so nothing needs to be
// cleared between calls; calls whose kernels overlap on the GPU race on it.
constexpr int kStaticBlocks = kRedBlocks;
static __device__ __align__(256) double g_static_partials[kStaticBlocks * 5];

__device__ __forceinline__ double warp_sum_static(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Pass 1 on a packed array: population l of cell (x, y) at f[(l * ny + y) * nx + x].
template <int N1, class C>
__global__ void __launch_bounds__(256) reduce_packed_kernel(const typename C::T* __restrict__ f, int nx, int ny,
                                                            double rho0, double* __restrict__ partials, KParams p) {
    double acc[5] = {0, 0, 0, 0, 0};
    const int ncell = nx * ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            double r = 0, rx = 0, rxx = 0;
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const double v = (double)C::ld(f + (i + N1 * j) * ncell + c);
                acc[4] += isfinite(v) ? 0.0 : 1.0;
                const double fv = to_f<C, double>(v, p.wd[i] * p.wd[j], rho0);
                r += fv;
                rx += p.xd[i] * fv;
                rxx += p.xd[i] * p.xd[i] * fv;
            }
            acc[0] += r;
            acc[1] += rx;
            acc[2] += p.xd[j] * r;
            acc[3] += 0.5 * (rxx + p.xd[j] * p.xd[j] * r);
        }
    }
    __shared__ double sh[5][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double v = warp_sum_static(acc[k]);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
        partials[blockIdx.x * 5 + threadIdx.x] = t;
    }
}

// Pass 2: one block folds the partials in a fixed order into out5.
__global__ void __launch_bounds__(256) reduce_packed_final_kernel(const double* __restrict__ partials,
                                                                  double* __restrict__ out5) {
    __shared__ double sh[5][8];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < kStaticBlocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += partials[b * 5 + k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double v = warp_sum_static(acc[k]);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
        out5[threadIdx.x] = t;
    }
}

template <int N1, class C>
cudaError_t launch_packed(const void* f, int nx, int ny, double rho0, double* partials, double* out5, const KParams& p,
                          cudaStream_t s) {
    reduce_packed_kernel<N1, C><<<kStaticBlocks, 256, 0, s>>>((const typename C::T*)f, nx, ny, rho0, partials, p);
    reduce_packed_final_kernel<<<1, 256, 0, s>>>(partials, out5);
    return cudaGetLastError();
}

template <int N1>
cudaError_t dispatch_storage(int storage, const void* f, int nx, int ny, double rho0, double* partials, double* out5,
                             const KParams& p, cudaStream_t s) {
    switch (storage) {
        case ST_FP64: return launch_packed<N1, CodecF64>(f, nx, ny, rho0, partials, out5, p, s);
        case ST_FP32: return launch_packed<N1, CodecF32>(f, nx, ny, rho0, partials, out5, p, s);
        case ST_BF16_DEV: return launch_packed<N1, CodecBF16Dev>(f, nx, ny, rho0, partials, out5, p, s);
        case ST_FP16_DEV: return launch_packed<N1, CodecF16Dev>(f, nx, ny, rho0, partials, out5, p, s);
        case ST_FP32_DEV: return launch_packed<N1, CodecF32Dev>(f, nx, ny, rho0, partials, out5, p, s);
        default: return cudaErrorInvalidValue;
    }
}

// Device address of g_static_partials, looked up once per device with that device current.
std::mutex g_addr_mutex;
void* g_addr[64];

int static_scratch(void** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return TVLBM_ECUDA;
    std::lock_guard<std::mutex> lock(g_addr_mutex);
    if (!g_addr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_static_partials) != cudaSuccess || !ptr) return TVLBM_ECUDA;
        g_addr[dev] = ptr;
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
    const int rc = static_scratch(&scratch);
    if (rc) return rc;
    cudaError_t e;
    cudaStream_t s = (cudaStream_t)stream;
    switch (n1) {
        case 3: e = dispatch_storage<3>(storage, populations, nx, ny, rho0, (double*)scratch, out5, p, s); break;
        case 4: e = dispatch_storage<4>(storage, populations, nx, ny, rho0, (double*)scratch, out5, p, s); break;
        default: e = dispatch_storage<6>(storage, populations, nx, ny, rho0, (double*)scratch, out5, p, s); break;
    }
    return e == cudaSuccess ? TVLBM_OK : TVLBM_ECUDA;
}
