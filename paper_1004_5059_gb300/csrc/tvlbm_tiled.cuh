// Tiled sweep: each CTA owns a TX x TY tile of destination cells.  For every velocity l the
// source window the tile gathers from -- (TX + 1) x (TY + 1) cells shifted by (-sh_x - 1,
// -sh_y - 1), widened to a 16-byte aligned start -- is copied global -> shared by one TMA
// tensor load (cp.async.bulk.tensor.3d) that completes on the velocity's own mbarrier.  All Q
// loads are issued up front, so a CTA has its whole input in flight at once; the threads then
// consume the windows in order as they land, lerp in x and y from shared memory, run the
// collision in registers and store the post-collision populations straight to global memory.
#pragma once

#include <cuda.h>  // CUtensorMap (the descriptor type only; the library does not link libcuda)

#include "tvlbm_kernels.cuh"

namespace tvlbm {

// ---- tile shapes ---------------------------------------------------------------------------
template <int N1, class C>
struct TileCfg {
    static constexpr int ES = (int)sizeof(typename C::T);
    static constexpr int A = 16 / ES;            // TMA x coordinates must be 16-byte multiples
    static constexpr int TX = ES == 8 ? 32 : 64; // tile width (one or two warps along x)
    static constexpr int TY = N1 >= 6 ? 8 : 16;  // tile height
    static constexpr int R = N1 >= 6 ? 2 : 4;    // cells per thread, stacked along y
    static constexpr int THREADS = TX * (TY / R);
    static constexpr int BX = TX + A;            // window width: TX + 1 cells after alignment slack
    static constexpr int BY = TY + 1;
    static constexpr int WIN_BYTES = (BX * BY * ES + 127) / 128 * 128;
    static constexpr int Q = N1 * N1;
    static constexpr int SMEM = Q * WIN_BYTES + 8 * Q + 128;  // windows, barriers, alignment slack
};

// ---- PTX wrappers -----------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}
__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
// Wait for phase `parity` of the barrier, giving up after limit_ns of wall time.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if (global_ns() - t0 > limit_ns) return false;
    }
    return true;
}
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x, int y, int z) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(
            smem_addr(dst)),
        "l"(map), "r"(smem_addr(bar)), "r"(x), "r"(y), "r"(z)
        : "memory");
}

template <class C>
__device__ __forceinline__ typename C::R lds(const typename C::T* p) {
    if constexpr (std::is_same<typename C::T, __nv_bfloat16>::value) return __bfloat162float(*p);
    else if constexpr (std::is_same<typename C::T, __half>::value) return __half2float(*p);
    else return *p;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: a TMA load never takes that long

// Store v at (x, y) and, for cells within FILL of a periodic edge, at their frame images.
template <class T>
__device__ __forceinline__ void store_cell(T* f, const KParams& p, long long lbase, int x, int y, bool edge, T v) {
    if (!edge) f[lbase + (long long)(y + HY) * p.pitch + (x + p.hx)] = v;
    else store_with_images(f, p, lbase, x, y, v);
}

template <int N1, class C>
__global__ void __launch_bounds__(TileCfg<N1, C>::THREADS)
    sweep_tiled_kernel(const __grid_constant__ CUtensorMap tmap, typename C::T* __restrict__ fout, const KParams p) {
    using Cfg = TileCfg<N1, C>;
    using T = typename C::T;
    using R = typename C::R;
    constexpr int Q = N1 * N1, TX = Cfg::TX, TY = Cfg::TY, RR = Cfg::R, BX = Cfg::BX, A = Cfg::A;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t* bars = (uint64_t*)(base + Q * Cfg::WIN_BYTES);
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int tid = threadIdx.x;

    if (tid == 0) {
#pragma unroll 1
        for (int l = 0; l < Q; ++l) mbar_init(&bars[l], 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (tid == 0) {
#pragma unroll 1
        for (int l = 0; l < Q; ++l) {
            const int i = l % N1, j = l / N1;
            const int xs = x0 + p.hx - p.sh[i] - 1;
            const int ys = y0 + HY - p.sh[j] - 1;
            mbar_arrive_expect_tx(&bars[l], (uint32_t)(BX * Cfg::BY * Cfg::ES));
            tma_load_3d(base + l * Cfg::WIN_BYTES, &tmap, &bars[l], xs & ~(A - 1), ys, l);
        }
    }

    const int cx = tid % TX, r0 = (tid / TX) * RR;
    R s[Q][RR];
    bool ok = true;
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        const R ay = ka<R>(p, j);
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const int l = i + N1 * j;
            if (ok && !mbar_wait_bounded(&bars[l], 0, kWaitLimitNs)) ok = false;
            const R ax = ka<R>(p, i);
            const int xs = x0 + p.hx - p.sh[i] - 1;
            const int col = cx + (xs & (A - 1));
            const T* w = (const T*)(base + l * Cfg::WIN_BYTES) + r0 * BX + col;
            R a = lds<C>(w + 1), b = lds<C>(w);
            R hprev = fma(ax, b - a, a);
#pragma unroll
            for (int k = 0; k < RR; ++k) {
                a = lds<C>(w + (k + 1) * BX + 1);
                b = lds<C>(w + (k + 1) * BX);
                const R h = fma(ax, b - a, a);
                s[l][k] = fma(ay, hprev - h, h);
                hprev = h;
            }
        }
    }
    if (!ok) {
        // A window never arrived: report it, give the other loads a bounded chance to land
        // (so no copy is still writing this CTA's shared memory), store nothing.
        if (p.status) atomicOr(p.status, 1);
#pragma unroll 1
        for (int l = 0; l < Q; ++l) mbar_wait_bounded(&bars[l], 0, kWaitLimitNs);
        return;
    }
    const int x = x0 + cx;
#pragma unroll
    for (int k = 0; k < RR; ++k) {
        const int y = y0 + r0 + k;
        if (x >= p.nx || y >= p.ny) continue;
        R c[Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) c[l] = s[l][k];
        cell_collide<N1, C::dev, R>(c, p);
        const bool edge = x < FILL || x >= p.nx - FILL || (!p.walls && (y < FILL || y >= p.ny - FILL));
#pragma unroll
        for (int l = 0; l < Q; ++l) store_cell(fout, p, (long long)l * p.plane, x, y, edge, C::enc(c[l]));
    }
}

template <int N1>
inline int tiled_supported(int storage) {
    (void)storage;
    return 1;
}

template <int N1, class C>
inline void tiled_box(int* bx, int* by) {
    *bx = TileCfg<N1, C>::BX;
    *by = TileCfg<N1, C>::BY;
}

template <int N1, class C>
inline cudaError_t tiled_sweep(const CUtensorMap* tmap, typename C::T* fout, const KParams& p, cudaStream_t s) {
    using Cfg = TileCfg<N1, C>;
    static bool attr_set[64] = {};  // per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(sweep_tiled_kernel<N1, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   Cfg::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    const dim3 grid((p.nx + Cfg::TX - 1) / Cfg::TX, (p.ny + Cfg::TY - 1) / Cfg::TY);
    sweep_tiled_kernel<N1, C><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(*tmap, fout, p);
    return cudaGetLastError();
}

}  // namespace tvlbm
