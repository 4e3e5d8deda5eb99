// Tiled sweep: each CTA owns a TX x TY tile of destination cells.  For every velocity l the
// source window the tile gathers from -- (TX + 1) x (TY + 1) cells shifted by (-sh_x - 1,
// -sh_y - 1), widened to a 16-byte aligned start -- is copied global -> shared by one TMA
// tensor load (cp.async.bulk.tensor.3d) completing on the velocity's own mbarrier.  All Q loads
// are issued up front, so the whole tile input is in flight at once.  Each thread then walks R
// consecutive rows of one column: per velocity it keeps the x-interpolated previous row in a
// register, so every cell costs two shared loads and two lerps per velocity; it collides in
// registers and stores straight to global memory (the lanes of a warp are consecutive x, so
// every store instruction writes whole 32-byte sectors).
#pragma once

#include <cuda.h>  // CUtensorMap (the descriptor type only; the library does not link libcuda)

#include "tvlbm_collide.cuh"
#include "tvlbm_kernels.cuh"

namespace tvlbm {

// ---- tile shapes ---------------------------------------------------------------------------
// (TX, TY, RS): tile width, tile height, row segments (threads per column); R = TY / RS rows
// per thread.  FP64 uses half-width tiles.
constexpr int kTileConfigs = 4;
struct TileShape {
    int tx, ty, rs;
};
__host__ __device__ constexpr TileShape tile_shape(int es, int cfg) {
    return es == 8 ? (cfg == 0   ? TileShape{32, 16, 4}
                      : cfg == 1 ? TileShape{32, 8, 4}
                      : cfg == 2 ? TileShape{64, 8, 2}
                                 : TileShape{32, 16, 2})
                   : (cfg == 0   ? TileShape{64, 16, 4}
                      : cfg == 1 ? TileShape{64, 8, 4}
                      : cfg == 2 ? TileShape{128, 8, 2}
                                 : TileShape{32, 16, 4});
}

template <int N1, class C, int CFG>
struct TileCfg {
    static constexpr int ES = (int)sizeof(typename C::T);
    static constexpr int A = 16 / ES;  // TMA x coordinates must be 16-byte multiples
    static constexpr int TX = tile_shape(ES, CFG).tx;
    static constexpr int TY = tile_shape(ES, CFG).ty;
    static constexpr int RS = tile_shape(ES, CFG).rs;
    static constexpr int R = TY / RS;
    static constexpr int THREADS = TX * RS;
    static constexpr int BX = TX + A;  // window width: TX + 1 cells plus alignment slack
    static constexpr int BY = TY + 1;
    static constexpr int WIN_BYTES = (BX * BY * ES + 127) / 128 * 128;
    static constexpr int Q = N1 * N1;
    static constexpr int SMEM = Q * WIN_BYTES + 8 * Q + 128;  // windows, barriers, alignment slack
    static_assert(SMEM <= 227 * 1024, "tile windows exceed shared memory");
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
__device__ __forceinline__ typename C::R lds(const unsigned char* p) {
    using T = typename C::T;
    const T v = *reinterpret_cast<const T*>(p);
    if constexpr (std::is_same<T, __nv_bfloat16>::value) return __bfloat162float(v);
    else if constexpr (std::is_same<T, __half>::value) return __half2float(v);
    else return v;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: a TMA load never takes that long

// Periodic frame images of the value already stored at fluid cell (x, y) of plane lbase.
template <class T>
__device__ __forceinline__ void store_images_of(T* f, const KParams& p, long long lbase, int x, int y) {
    const T v = f[lbase + (long long)(y + HY) * p.pitch + (x + p.hx)];
    const int x0 = x - p.nx * ((x + FILL) / p.nx);
    const int y0 = p.walls ? y : y - p.ny * ((y + FILL) / p.ny);
    const int y1 = p.walls ? y + 1 : p.ny + FILL;
    for (int yy = y0; yy < y1; yy += p.ny)
        for (int xx = x0; xx < p.nx + FILL; xx += p.nx)
            if (xx != x || yy != y) f[lbase + (long long)(yy + HY) * p.pitch + (xx + p.hx)] = v;
}

// Collision of one gathered cell in the codec's arithmetic.
template <int N1, class C>
__device__ __forceinline__ void collide_cell(typename C::R (&s)[N1 * N1], const KParams& p) {
    if constexpr (C::dev) cell_collide_dev<N1>(s, p);
    else cell_collide<N1, false, typename C::R>(s, p);
}

// Store one collided cell: plain stores, then (cells within FILL of a periodic edge) the images.
template <int N1, class C>
__device__ __forceinline__ void store_collided(typename C::T* f, const KParams& p, int x, int y,
                                               const typename C::R (&s)[N1 * N1]) {
    const long long c = (long long)(y + HY) * p.pitch + (x + p.hx);
#pragma unroll
    for (int l = 0; l < N1 * N1; ++l) f[(long long)l * p.plane + c] = C::enc(s[l]);
    const bool edge = x < FILL || x >= p.nx - FILL || (!p.walls && (y < FILL || y >= p.ny - FILL));
    if (edge) {
#pragma unroll 1
        for (int l = 0; l < N1 * N1; ++l) store_images_of(f, p, (long long)l * p.plane, x, y);
    }
}

template <int N1, class C, int CFG>
__global__ void __launch_bounds__(TileCfg<N1, C, CFG>::THREADS)
    sweep_tiled_kernel(const __grid_constant__ CUtensorMap tmap, typename C::T* __restrict__ fout, const KParams p) {
    using Cfg = TileCfg<N1, C, CFG>;
    using R = typename C::R;
    constexpr int Q = N1 * N1, TX = Cfg::TX, TY = Cfg::TY, RR = Cfg::R, BX = Cfg::BX, A = Cfg::A, ES = Cfg::ES;
    constexpr int WIN = Cfg::WIN_BYTES;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 127) & ~(uintptr_t)127);
    uint64_t* bars = (uint64_t*)(base + Q * WIN);
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
            mbar_arrive_expect_tx(&bars[l], (uint32_t)(BX * Cfg::BY * ES));
            tma_load_3d(base + l * WIN, &tmap, &bars[l], xs & ~(A - 1), ys, l);
        }
    }
    bool ok = true;
#pragma unroll 1
    for (int l = 0; l < Q && ok; ++l) ok = mbar_wait_bounded(&bars[l], 0, kWaitLimitNs);
    if (!ok) {
        // A window never arrived: report it, give the other loads a bounded chance to land
        // (so no copy is still writing this CTA's shared memory), store nothing.
        if (p.status) atomicOr(p.status, 1);
#pragma unroll 1
        for (int l = 0; l < Q; ++l) mbar_wait_bounded(&bars[l], 0, kWaitLimitNs);
        return;
    }

    const int cx = tid % TX, r0 = (tid / TX) * RR;
    const int x = x0 + cx;
    // byte offset of column (cx + alignment remainder) within a window row, per x-node
    int off[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) off[i] = (cx + ((x0 + p.hx - p.sh[i] - 1) & (A - 1))) * ES;
    const unsigned char* wrow = base + r0 * BX * ES;
    R hprev[Q];
#pragma unroll
    for (int j = 0; j < N1; ++j)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const unsigned char* q = wrow + (i + N1 * j) * WIN + off[i];
            const R a = lds<C>(q + ES), b = lds<C>(q);
            hprev[i + N1 * j] = fma(ka<R>(p, i), b - a, a);
        }
#pragma unroll 1
    for (int k = 0; k < RR; ++k) {
        wrow += BX * ES;
        R s[Q];
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            const R ay = ka<R>(p, j);
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                const unsigned char* q = wrow + l * WIN + off[i];
                const R a = lds<C>(q + ES), b = lds<C>(q);
                const R h = fma(ka<R>(p, i), b - a, a);
                s[l] = fma(ay, hprev[l] - h, h);
                hprev[l] = h;
            }
        }
        const int y = y0 + r0 + k;
        if (x < p.nx && y < p.ny) {
            collide_cell<N1, C>(s, p);
            store_collided<N1, C>(fout, p, x, y, s);
        }
    }
}

template <int N1>
inline int tiled_supported(int storage) {
    (void)storage;
    return 1;
}

template <int N1, class C>
inline void tiled_box(int cfg, int* bx, int* by) {
    const TileShape t = tile_shape((int)sizeof(typename C::T), cfg);
    *bx = t.tx + 16 / (int)sizeof(typename C::T);
    *by = t.ty + 1;
}

template <int N1, class C, int CFG>
inline cudaError_t tiled_launch(const CUtensorMap* tmap, typename C::T* fout, const KParams& p, cudaStream_t s) {
    using Cfg = TileCfg<N1, C, CFG>;
    static bool attr_set[64] = {};  // per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(sweep_tiled_kernel<N1, C, CFG>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        if (dev >= 0 && dev < 64) attr_set[dev] = true;
    }
    const dim3 grid((p.nx + Cfg::TX - 1) / Cfg::TX, (p.ny + Cfg::TY - 1) / Cfg::TY);
    sweep_tiled_kernel<N1, C, CFG><<<grid, Cfg::THREADS, Cfg::SMEM, s>>>(*tmap, fout, p);
    return cudaGetLastError();
}

template <int N1, class C>
inline cudaError_t tiled_sweep(int cfg, const CUtensorMap* tmap, typename C::T* fout, const KParams& p, cudaStream_t s) {
    switch (cfg) {
        case 0: return tiled_launch<N1, C, 0>(tmap, fout, p, s);
        case 1: return tiled_launch<N1, C, 1>(tmap, fout, p, s);
        case 2: return tiled_launch<N1, C, 2>(tmap, fout, p, s);
        case 3: return tiled_launch<N1, C, 3>(tmap, fout, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tvlbm
