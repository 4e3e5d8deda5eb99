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
// per thread.  Shared memory per CTA = Q input windows.
struct TileShape {
    int tx, ty, rs;
};
__host__ __device__ constexpr TileShape tile_shape_base(int es, int cfg) {
    return es == 8 ? (cfg == 0   ? TileShape{32, 8, 4}
                      : cfg == 1 ? TileShape{32, 4, 2}
                      : cfg == 2 ? TileShape{32, 8, 2}
                                 : TileShape{32, 4, 4})
                   : (cfg == 0   ? TileShape{32, 16, 4}
                      : cfg == 1 ? TileShape{32, 8, 4}
                      : cfg == 2 ? TileShape{64, 8, 4}
                                 : TileShape{64, 16, 4});
}
__host__ __device__ constexpr int tile_smem(int q, int es, TileShape t) {
    return q * (((t.tx + 16 / es) * (t.ty + 1) * es + 127) / 128 * 128) + 8 * q + 128;
}
// A shape whose windows do not fit in shared memory is halved in height.
__host__ __device__ constexpr TileShape tile_shape(int q, int es, int cfg) {
    return tile_smem(q, es, tile_shape_base(es, cfg)) <= 227 * 1024
               ? tile_shape_base(es, cfg)
               : TileShape{tile_shape_base(es, cfg).tx, tile_shape_base(es, cfg).ty / 2,
                           tile_shape_base(es, cfg).rs / 2};
}

template <int N1, class C, int CFG>
struct TileCfg {
    static constexpr int ES = (int)sizeof(typename C::T);
    static constexpr int Q = N1 * N1;
    static constexpr int A = 16 / ES;  // TMA x coordinates must be 16-byte multiples
    static constexpr int TX = tile_shape(Q, ES, CFG).tx;
    static constexpr int TY = tile_shape(Q, ES, CFG).ty;
    static constexpr int RS = tile_shape(Q, ES, CFG).rs;
    static constexpr int R = TY / RS;
    static constexpr int THREADS = TX * RS;
    static constexpr int BX = TX + A;  // window width: TX + 1 cells plus alignment slack
    static constexpr int BY = TY + 1;
    static constexpr int WIN_BYTES = (BX * BY * ES + 127) / 128 * 128;
    static constexpr int SMEM = Q * WIN_BYTES + 8 * Q + 128;  // windows, Q barriers, alignment slack
    // with a per-row reference: the tile rows' entries behind the barriers (16-byte aligned)
    static constexpr int ROWS_OFF = (Q * WIN_BYTES + 8 * Q + 15) / 16 * 16;
    static constexpr int SMEM_ROWS = SMEM + 16 + TY * kRowF * 4;
    static_assert(SMEM_ROWS <= 227 * 1024, "tile windows and row entries exceed shared memory");
    static_assert(SMEM <= 227 * 1024, "tile windows exceed shared memory");
    // resident CTAs per SM to compile for: D2Q36 in 32-bit arithmetic is held to about 168
    // registers a thread (3 CTAs of 128 threads; left alone the compiler takes 253 and 2 fit),
    // and with 16-bit storage, whose windows leave room for a fourth CTA, to 128 (a few words
    // spilled; the 4096 x 512 channel: 118.7 -> 117.8 us per step FP16, 121.0 -> 116.9 BF16).
    // The others compile without a minimum (MINB = 0): even a minimum of 1 lets the compiler
    // take more registers than the occupancy pays for (the batched D2Q16 kernel: 128 instead
    // of 80).
    static constexpr int MINB_D2Q36 = 65536 / (THREADS * (ES == 2 ? 128 : 168));
    static constexpr int MINB = (N1 >= 6 && sizeof(typename C::R) == 4 && MINB_D2Q36 > 1) ? MINB_D2Q36 : 0;
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
// One test of the phase, letting the hardware suspend the thread up to ~1 ms while it is not
// complete (so waiting threads do not spin through issue slots).
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(1000000u)
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

// Shared -> global TMA tensor store of one box (bulk-group completion), its commit, and the waits
// for the group's reads of shared memory / for its writes to complete.
__device__ __forceinline__ void tma_store_3d(const CUtensorMap* map, const void* src, int x, int y, int z) {
    asm volatile("cp.async.bulk.tensor.3d.global.shared::cta.bulk_group [%0, {%2, %3, %4}], [%1];" ::"l"(map),
                 "r"(smem_addr(src)), "r"(x), "r"(y), "r"(z)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_read_all() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// This thread's generic-proxy shared-memory writes, visible to the async proxy (a TMA store).
__device__ __forceinline__ void fence_proxy_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

template <class C>
__device__ __forceinline__ typename C::R lds(const unsigned char* p) {
    using T = typename C::T;
    const T v = *reinterpret_cast<const T*>(p);
    if constexpr (std::is_same<T, __nv_bfloat16>::value) return __bfloat162float(v);
    else if constexpr (std::is_same<T, __half>::value) return __half2float(v);
    else return v;
}
// b - a, b the stored value at p.  For 16-bit storage one mixed-precision subtraction: b is
// widened to FP32 exactly inside the instruction, so the result is that of widening first.
template <class C>
__device__ __forceinline__ typename C::R lds_sub(const unsigned char* p, typename C::R a) {
    using T = typename C::T;
    if constexpr (std::is_same<T, __half>::value) {
        float d;
        asm("sub.rn.f32.f16 %0, %1, %2;" : "=f"(d) : "h"(*reinterpret_cast<const unsigned short*>(p)), "f"(a));
        return d;
    } else if constexpr (std::is_same<T, __nv_bfloat16>::value) {
        float d;
        asm("sub.rn.f32.bf16 %0, %1, %2;" : "=f"(d) : "h"(*reinterpret_cast<const unsigned short*>(p)), "f"(a));
        return d;
    } else {
        return lds<C>(p) - a;
    }
}
// a - b on FP32 pairs (one packed instruction, each lane rounded as the scalar subtraction).
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
    float2 d;
    asm("{\n\t.reg .b64 ra, rb, rd;\n\t"
        "mov.b64 ra, {%2, %3};\n\t"
        "mov.b64 rb, {%4, %5};\n\t"
        "sub.rn.f32x2 rd, ra, rb;\n\t"
        "mov.b64 {%0, %1}, rd;\n\t}"
        : "=f"(d.x), "=f"(d.y)
        : "f"(a.x), "f"(a.y), "f"(b.x), "f"(b.y));
    return d;
}

// Gather one window row for every velocity: h_l = a + alpha_i (b - a), a and b the row's two
// source cells of velocity l (split codecs: a less its rest value), and, unless FIRST, the
// y-interpolation with the previous row's h, s_l = h_l + alpha_j (hprev_l - h_l); hprev <- h.
// In FP32 with an even node count the mirror pairs (i, N1 - 1 - i) of each y-node go through
// packed FP32 instructions, each lane rounded exactly as the scalar form.
template <int N1, class C, int WIN, bool FIRST>
__device__ __forceinline__ void gather_row(const unsigned char* wrow, const int (&off)[N1], const KParams& p,
                                           typename C::R (&hprev)[N1 * N1], typename C::R (&s)[N1 * N1]) {
    using R = typename C::R;
    constexpr int ES = (int)sizeof(typename C::T), H = N1 / 2;
    constexpr bool PACK = std::is_same<R, float>::value && (N1 % 2 == 0);
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        const R ay = ka<R>(p, j);
        if constexpr (PACK) {
#pragma unroll
            for (int i = 0; i < H; ++i) {
                const int m = N1 - 1 - i, l = i + N1 * j, lm = m + N1 * j;
                const unsigned char* qi = wrow + l * WIN + off[i];
                const unsigned char* qm = wrow + lm * WIN + off[m];
                const float ai = lds<C>(qi + ES), am = lds<C>(qm + ES);
                const float2 d2 = make_float2(lds_sub<C>(qi, ai), lds_sub<C>(qm, am));
                const float2 a2 = make_float2(split_rest<C>(p, l, ai), split_rest<C>(p, lm, am));
                const float2 h2 = __ffma2_rn(make_float2(ka<R>(p, i), ka<R>(p, m)), d2, a2);
                if constexpr (!FIRST) {
                    const float2 s2 =
                        __ffma2_rn(make_float2(ay, ay), f2sub(make_float2(hprev[l], hprev[lm]), h2), h2);
                    s[l] = s2.x;
                    s[lm] = s2.y;
                }
                hprev[l] = h2.x;
                hprev[lm] = h2.y;
            }
        } else {
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                const unsigned char* q = wrow + l * WIN + off[i];
                const R a = lds<C>(q + ES);
                const R h = fma(ka<R>(p, i), lds_sub<C>(q, a), split_rest<C>(p, l, a));
                if constexpr (!FIRST) s[l] = fma(ay, hprev[l] - h, h);
                hprev[l] = h;
            }
        }
    }
}


// Collision of one gathered cell (fluid row y) in the codec's arithmetic, relaxation rate of the
// domain; with a per-row deviation reference, against the row's reference (ROWS = false: the
// launch never has one, e.g. a periodic-only form).
// A ROWS launch always has the table (the launch checks it).
// SROW: srow holds the row's reference entries staged in shared memory (else they are read from
// the table in global memory).
template <int N1, class C, bool ROWS, bool SROW = false>
__device__ __forceinline__ void collide_cell(typename C::R (&s)[N1 * N1], const KParams& p, const Geom& g, int y,
                                             const float* srow = nullptr) {
    if constexpr (C::dev) {
        if constexpr (ROWS) {
            if constexpr (SROW) cell_collide_dev<N1, true, true>(s, p, g.omegaf, srow);
            else cell_collide_dev<N1, true>(s, p, g.omegaf, p.rowf + (long long)(y + HY) * kRowF);
        } else {
            cell_collide_dev<N1, false>(s, p, g.omegaf, nullptr);
        }
    }
    else if constexpr (C::split) cell_collide_split<N1>(s, p, g.omegaf);
    else if constexpr (std::is_same<typename C::R, double>::value) cell_collide<N1, false, double>(s, p, g.omegad);
    else cell_collide<N1, false, float>(s, p, g.omegaf);
}

// Store one collided cell.  A cell within FILL of a periodic edge is stored at every position it
// has in the read frame (itself and its periodic images), straight from the registers; the image
// positions are worked out once per cell.
template <int N1, class C>
__device__ __forceinline__ void store_collided(typename C::T* f, const Geom& g, int x, int y,
                                               const typename C::R (&s)[N1 * N1]) {
    using T = typename C::T;
    const bool edge = x < FILL || x >= g.nx - FILL || (!g.walls && (y < FILL || y >= g.ny - FILL));
    if (!edge) {
        T* q = f + ((long long)(y + HY) * g.pitch + (x + g.hx));
#pragma unroll
        for (int l = 0; l < N1 * N1; ++l) {
            stg(q, C::enc(s[l]));
            q += g.plane;
        }
        return;
    }
    const int x0 = x - g.nx * ((x + FILL) / g.nx);
    const int y0 = g.walls ? y : y - g.ny * ((y + FILL) / g.ny);
    const int y1 = g.walls ? y + 1 : g.ny + FILL;
#pragma unroll 1
    for (int yy = y0; yy < y1; yy += g.ny)
#pragma unroll 1
        for (int xx = x0; xx < g.nx + FILL; xx += g.nx) {
            typename C::T* q = f + ((long long)(yy + HY) * g.pitch + (xx + g.hx));
#pragma unroll
            for (int l = 0; l < N1 * N1; ++l) {
                stg(q, C::enc(s[l]));
                q += g.plane;
            }
        }
}

// Store one collided cell at its periodic images only (not at (x, y) itself); true if it has any.
// Used where the cell's own position is written from shared memory by a TMA tensor store.
template <int N1, class C>
__device__ __forceinline__ bool store_images(typename C::T* f, const Geom& g, int x, int y,
                                             const typename C::R (&s)[N1 * N1]) {
    const bool edge = x < FILL || x >= g.nx - FILL || (!g.walls && (y < FILL || y >= g.ny - FILL));
    if (!edge) return false;
    const int x0 = x - g.nx * ((x + FILL) / g.nx);
    const int y0 = g.walls ? y : y - g.ny * ((y + FILL) / g.ny);
    const int y1 = g.walls ? y + 1 : g.ny + FILL;
#pragma unroll 1
    for (int yy = y0; yy < y1; yy += g.ny)
#pragma unroll 1
        for (int xx = x0; xx < g.nx + FILL; xx += g.nx) {
            if (xx == x && yy == y) continue;
            typename C::T* q = f + ((long long)(yy + HY) * g.pitch + (xx + g.hx));
#pragma unroll
            for (int l = 0; l < N1 * N1; ++l) {
                stg(q, C::enc(s[l]));
                q += g.plane;
            }
        }
    return true;
}

// ---- tile sources: where tile t lives --------------------------------------------------------
// One domain: tiles in row-major order over a tiles_x-wide grid; the input descriptor is a
// kernel parameter.
struct SingleSrc {
    CUtensorMap map_in;
    void* fout;
    int tiles_x, ntiles;
    __device__ __forceinline__ void tile(int t, const KParams& p, int tx, int ty, int& x0, int& y0,
                                         const CUtensorMap*& map, void*& out, Geom& g) const {
        x0 = (t % tiles_x) * tx;
        y0 = (t / tiles_x) * ty;
        map = &map_in;
        out = fout;
        g = geom_of(p);
    }
};

// Many domains (see tvlbm_batch.cu): a per-tile domain index, a per-domain table and two
// descriptors per domain in global memory.
struct BatchDomain {
    long long off[2];  // element offsets of the two population buffers from the batch base
    long long plane;
    int nx, ny, pitch, tiles_x, tile_begin, tiles_y;
    float omegaf;
    double omegad;
};
struct BatchSrc {
    const BatchDomain* dom;
    const CUtensorMap* maps;  // [domain][buffer]
    const int* tile_dom;
    unsigned char* base;
    int ntiles, parity, es;
    __device__ __forceinline__ void tile(int t, const KParams& p, int tx, int ty, int& x0, int& y0,
                                         const CUtensorMap*& map, void*& out, Geom& g) const {
        const int d = __ldg(tile_dom + t);
        const BatchDomain& D = dom[d];
        const int local = t - D.tile_begin;
        x0 = (local % D.tiles_x) * tx;
        y0 = (local / D.tiles_x) * ty;
        map = maps + 2 * d + parity;
        out = base + D.off[parity ^ 1] * es;
        g.nx = D.nx;
        g.ny = D.ny;
        g.pitch = D.pitch;
        g.hx = p.hx;
        g.walls = 0;
        g.plane = D.plane;
        g.omegaf = D.omegaf;
        g.omegad = D.omegad;
    }
};

// Gather, collide and store one tile whose Q windows are in shared memory at base.  With sout,
// each cell's own position goes to the shared-memory output tile sout ([Q][TY][TX], the layout a
// TMA tensor store of a TX x TY box reads) and only its periodic images to global memory; the
// return value then says whether this thread stored any image.  With ROWS, srows holds the tile
// rows' reference entries ([TY][kRowF], staged by the caller).
template <int N1, class C, int CFG, bool ROWS>
__device__ __forceinline__ bool tile_compute(const unsigned char* base, int x0, int y0, const Geom& g,
                                             typename C::T* fout, const KParams& p, int tid,
                                             typename C::T* sout = nullptr, const float* srows = nullptr) {
    using Cfg = TileCfg<N1, C, CFG>;
    using R = typename C::R;
    constexpr int Q = N1 * N1, TX = Cfg::TX, RR = Cfg::R, BX = Cfg::BX, A = Cfg::A, ES = Cfg::ES;
    constexpr int WIN = Cfg::WIN_BYTES;
    const int cx = tid % TX, r0 = (tid / TX) * RR;
    const int x = x0 + cx;
    // byte offset of column (cx + alignment remainder) within a window row, per x-node; the tile
    // origin is a multiple of TX (>= A), so the remainder depends on the node only
    int off[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) off[i] = (cx + ((g.hx - p.sh[i] - 1) & (A - 1))) * ES;
    const unsigned char* wrow = base + r0 * BX * ES;
    bool imaged = false;
    R hprev[Q], s[Q];
    gather_row<N1, C, WIN, true>(wrow, off, p, hprev, s);
#pragma unroll 1
    for (int kk = 0; kk < RR; ++kk) {
        wrow += BX * ES;
        gather_row<N1, C, WIN, false>(wrow, off, p, hprev, s);
        const int y = y0 + r0 + kk;
        if (x < g.nx && y < g.ny) {
            collide_cell<N1, C, ROWS, ROWS>(s, p, g, y, srows + (r0 + kk) * kRowF);
            if (sout) {
                typename C::T* q = sout + (r0 + kk) * TX + cx;
#pragma unroll
                for (int l = 0; l < Q; ++l) q[l * (TX * Cfg::TY)] = C::enc(s[l]);
                imaged |= store_images<N1, C>(fout, g, x, y, s);
            } else {
                store_collided<N1, C>(fout, g, x, y, s);
            }
        }
    }
    return imaged;
}

// Tiled sweep: CTA b owns tile b.  It lets the next step's launch be scheduled at once; warp 0
// waits for the previous grid and starts the Q window loads, lane l those of windows l and
// l + 32, then waits for them, lane l watching its own barriers, while the other warps sleep at
// the block barrier.  Each thread walks R rows of one column (x-lerp of the previous row carried in
// registers), collides and stores straight to global memory.  Every wait is bounded; a timeout
// sets the status word and the CTA returns after a bounded drain of its own loads.
// ROWS: the launch has a per-row deviation reference (a separate instantiation, so the common
// launch without one compiles exactly like the dataflow kernel's tile computation).
template <int N1, class C, int CFG, class Src, bool ROWS>
__device__ __forceinline__ void sweep_tiled_body(const Src& src, const KParams& p) {
    using Cfg = TileCfg<N1, C, CFG>;
    using R = typename C::R;
    using T = typename C::T;
    constexpr int Q = N1 * N1, TX = Cfg::TX, TY = Cfg::TY, RR = Cfg::R, BX = Cfg::BX, A = Cfg::A, ES = Cfg::ES;
    constexpr int WIN = Cfg::WIN_BYTES;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // 128-byte aligned base, derived from smem_raw by pointer arithmetic so the compiler keeps
    // the shared address space (window reads compile to shared-memory loads)
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + Q * WIN);
    __shared__ int tile_ok;
    const int tid = threadIdx.x;
    const int t = blockIdx.x;

    pdl_launch_dependents();
    int x0, y0;
    const CUtensorMap* map;
    void* outv;
    Geom g;
    src.tile(t, p, TX, TY, x0, y0, map, outv, g);

    if (tid < 32) {
        // warp 0: lane t sets up and starts windows t and t + 32 (Q <= 64), all lanes at once
        static_assert(Q <= 64, "two windows per lane");
#pragma unroll
        for (int k = 0; k < 2; ++k)
            if (tid + 32 * k < Q) mbar_init(&bars[tid + 32 * k], 1);
        fence_barrier_init();
        pdl_wait();  // the previous step's populations are complete from here on
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int l = tid + 32 * k;
            if (l < Q) {
                const int i = l % N1, j = l / N1;
                mbar_arrive_expect_tx(&bars[l], (uint32_t)(BX * Cfg::BY * ES));
                tma_load_3d(base + l * WIN, map, &bars[l], (x0 + g.hx - p.sh[i] - 1) & ~(A - 1),
                            y0 + HY - p.sh[j] - 1, l);
            }
        }
    }
    float* srows = nullptr;
    if constexpr (ROWS) {
        // the tile rows' reference entries, once the kernels before this one (a reference refresh
        // writes the table) are complete
        pdl_wait();
        srows = reinterpret_cast<float*>(base + Cfg::ROWS_OFF);
        constexpr int V = kRowF / 4;
#pragma unroll 1
        for (int k = tid; k < TY * V; k += Cfg::THREADS) {
            const int r = k / V;
            if (y0 + r < g.ny)
                reinterpret_cast<float4*>(srows)[k] = ld_row4(p.rowf + (long long)(y0 + r + HY) * kRowF + 4 * (k - r * V));
        }
    }
    if (tid < 32) {
        bool ok = true;
#pragma unroll 1
        for (int l = tid; l < Q; l += 32) ok = ok && mbar_wait_bounded(&bars[l], 0, kWaitLimitNs);
        ok = __all_sync(0xffffffffu, ok);
        if (tid == 0) tile_ok = ok ? 1 : 0;
    }
    __syncthreads();
    if (!tile_ok) {
        // A window never arrived: report it, give the loads a bounded chance to land (so no copy
        // still writes this CTA's shared memory), store nothing.
        if (tid == 0) {
            if (p.status) atomicOr(p.status, 1);
#pragma unroll 1
            for (int l = 0; l < Q; ++l) mbar_wait_bounded(&bars[l], 0, kWaitLimitNs);
        }
        return;
    }

    tile_compute<N1, C, CFG, ROWS>(base, x0, y0, g, reinterpret_cast<T*>(outv), p, tid, nullptr, srows);
}

// The kernel, with a minimum of resident CTAs where TileCfg asks for one.
template <int N1, class C, int CFG, class Src, bool ROWS>
__global__ void __launch_bounds__(TileCfg<N1, C, CFG>::THREADS)
    sweep_tiled_kernel(const __grid_constant__ Src src, const KParams p) {
    sweep_tiled_body<N1, C, CFG, Src, ROWS>(src, p);
}
template <int N1, class C, int CFG, class Src, bool ROWS>
__global__ void __launch_bounds__(TileCfg<N1, C, CFG>::THREADS, (TileCfg<N1, C, CFG>::MINB > 0 ? TileCfg<N1, C, CFG>::MINB : 1))
    sweep_tiled_kernel_minb(const __grid_constant__ Src src, const KParams p) {
    sweep_tiled_body<N1, C, CFG, Src, ROWS>(src, p);
}
// (single domains only: the batched kernel's tile lookup needs the registers the minimum takes)
template <int N1, class C, int CFG, class Src, bool ROWS>
constexpr auto tiled_kernel() {
    if constexpr (TileCfg<N1, C, CFG>::MINB > 0 && std::is_same<Src, SingleSrc>::value)
        return sweep_tiled_kernel_minb<N1, C, CFG, Src, ROWS>;
    else
        return sweep_tiled_kernel<N1, C, CFG, Src, ROWS>;
}

template <int N1>
inline int tiled_supported(int storage) {
    (void)storage;
    return 1;
}

template <int N1, class C>
inline void tiled_box(int cfg, int* bx, int* by) {
    const TileShape t = tile_shape(N1 * N1, (int)sizeof(typename C::T), cfg);
    *bx = t.tx + 16 / (int)sizeof(typename C::T);
    *by = t.ty + 1;
}

template <int N1, class C, int CFG, class Src, bool ROWS>
inline cudaError_t tiled_prepare() {
    using Cfg = TileCfg<N1, C, CFG>;
    static bool attr_set[64] = {};  // per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(tiled_kernel<N1, C, CFG, Src, ROWS>(),
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   ROWS ? Cfg::SMEM_ROWS : Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    return cudaSuccess;
}

template <int N1, class C, int CFG, bool ROWS>
inline cudaError_t tiled_launch_rows(const SweepMaps* maps, typename C::T* fout, const KParams& p, cudaStream_t s) {
    using Cfg = TileCfg<N1, C, CFG>;
    const cudaError_t e = tiled_prepare<N1, C, CFG, SingleSrc, ROWS>();
    if (e != cudaSuccess) return e;
    SingleSrc src;
    src.map_in = *(const CUtensorMap*)maps->in;
    src.fout = fout;
    src.tiles_x = (p.nx + Cfg::TX - 1) / Cfg::TX;
    src.ntiles = src.tiles_x * ((p.ny + Cfg::TY - 1) / Cfg::TY);
    return launch_pdl(tiled_kernel<N1, C, CFG, SingleSrc, ROWS>(), dim3(src.ntiles), dim3(Cfg::THREADS),
                      ROWS ? Cfg::SMEM_ROWS : Cfg::SMEM,
                      s, src, p);
}

// Only deviation codecs have a per-row reference.
template <int N1, class C, int CFG>
inline cudaError_t tiled_launch(const SweepMaps* maps, typename C::T* fout, const KParams& p, cudaStream_t s) {
    if constexpr (C::dev) {
        if (p.rowf) return tiled_launch_rows<N1, C, CFG, true>(maps, fout, p, s);
    }
    return tiled_launch_rows<N1, C, CFG, false>(maps, fout, p, s);
}

template <int N1, class C>
inline cudaError_t tiled_sweep(int cfg, const SweepMaps* maps, typename C::T* fout, const KParams& p, cudaStream_t s) {
    switch (cfg) {
        case 0: return tiled_launch<N1, C, 0>(maps, fout, p, s);
        case 1: return tiled_launch<N1, C, 1>(maps, fout, p, s);
        case 2: return tiled_launch<N1, C, 2>(maps, fout, p, s);
        case 3: return tiled_launch<N1, C, 3>(maps, fout, p, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int N1, class C, int CFG>
inline cudaError_t batch_launch(const BatchSrc& src, const KParams& p, cudaStream_t s) {
    using Cfg = TileCfg<N1, C, CFG>;
    const cudaError_t e = tiled_prepare<N1, C, CFG, BatchSrc, false>();
    if (e != cudaSuccess) return e;
    return launch_pdl(tiled_kernel<N1, C, CFG, BatchSrc, false>(), dim3(src.ntiles), dim3(Cfg::THREADS), Cfg::SMEM, s,
                      src, p);
}

template <int N1, class C>
inline cudaError_t batch_sweep(int cfg, const BatchSrc& src, const KParams& p, cudaStream_t s) {
    switch (cfg) {
        case 0: return batch_launch<N1, C, 0>(src, p, s);
        case 1: return batch_launch<N1, C, 1>(src, p, s);
        case 2: return batch_launch<N1, C, 2>(src, p, s);
        case 3: return batch_launch<N1, C, 3>(src, p, s);
        default: return cudaErrorInvalidValue;
    }
}

// ---- multi-step dataflow sweep ----------------------------------------------------------------
// One persistent launch advances n time steps of a periodic domain.  Tasks (step k, tile t) are
// handed out in step-major order from a global counter; a task starts once the 3 x 3 periodic
// neighbourhood of its tile has finished step k - 1 (per-tile counters that every compute warp
// of the task raises with release semantics after its own stores, so a tile has finished step
// k - 1 when its counter reaches k times the warps per task), which covers both the windows it
// reads and the region its own stores overwrite (that region was the neighbours' step k - 1
// input).  The compute warps of a CTA never wait for one another.  A task only waits on
// tasks handed out before it, which are held by running CTAs, so the launch always progresses
// (whether or not all CTAs are resident at once).
// Every wait is bounded: a CTA that gives up raises the abort word and the status bit, and the
// others stop at their next wait.  Requires tiles of at least 4 rows (a source is at most 4 cells
// away, so it lies in a neighbouring tile) and no ragged tiles (a frame image then lies next to a
// tile that neighbours, periodically, the tile that writes it).
__device__ __forceinline__ int ld_relaxed_gpu(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_release_gpu_add(int* p, int v) {
    asm volatile("red.release.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void fence_acquire_gpu() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }
// Generic-proxy global writes (made visible by the acquire) become visible to TMA reads.
__device__ __forceinline__ void fence_proxy_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Task sources of the dataflow kernel.  flow_task(): the step k and tile t of task number `task` and
// the completion counters of t's 3 x 3 periodic neighbourhood; flow_tile(): where tile t is, its
// domain's geometry, the descriptors it loads its step-k windows with and stores its step-k output
// with, and the buffer its periodic images go to.
// One domain (FlowSrc, see tvlbm_kernels.cuh): step k visits tile rows starting at row k (the
// first rows of step k + 1 then depend on the first rows that step k finished).
__device__ __forceinline__ void flow_task(const FlowSrc& src, int task, int& k, int& t, const int* (&nb)[9]) {
    k = task / src.ntiles;
    const int r = task - k * src.ntiles;
    const int tx = r % src.tiles_x, ty = (r / src.tiles_x + k) % src.tiles_y;
    t = ty * src.tiles_x + tx;
#pragma unroll
    for (int d = 0; d < 9; ++d) {
        const int xx = (tx + d % 3 - 1 + src.tiles_x) % src.tiles_x;
        const int yy = (ty + d / 3 - 1 + src.tiles_y) % src.tiles_y;
        nb[d] = src.done + yy * src.tiles_x + xx;
    }
}
__device__ __forceinline__ void flow_tile(const FlowSrc& src, int t, int k, const KParams& p, int TX, int TY, int& x0,
                                          int& y0, Geom& g, const CUtensorMap*& lmap, const CUtensorMap*& smap,
                                          void*& out) {
    x0 = (t % src.tiles_x) * TX;
    y0 = (t / src.tiles_x) * TY;
    g = geom_of(p);
    lmap = &src.map[k & 1];
    smap = &src.smap[(k + 1) & 1];
    out = src.buf[(k + 1) & 1];
}

// Many periodic domains (the batch): the tiles of every domain in one list, tasks in step-major
// order; a tile's neighbourhood wraps within its own domain; per-domain geometry, relaxation and
// descriptors (two per domain for the windows, two for the tile stores) from global tables.
struct BatchFlowSrc {
    const BatchDomain* dom;
    const CUtensorMap* lmaps;  // [domain][buffer], window boxes
    const CUtensorMap* smaps;  // [domain][buffer], tile boxes
    const int* tile_dom;
    unsigned char* base;
    int es, cur;               // element size; the buffer holding every domain's state at launch
    int ntiles, nsteps;
    int* done;
    int* next_task;
    int* abort;
    long long wait_ns;
    int wait_extra;
};
__device__ __forceinline__ void flow_task(const BatchFlowSrc& src, int task, int& k, int& t, const int* (&nb)[9]) {
    k = task / src.ntiles;
    t = task - k * src.ntiles;
    const BatchDomain& D = src.dom[__ldg(src.tile_dom + t)];
    const int local = t - D.tile_begin;
    const int tx = local % D.tiles_x, ty = local / D.tiles_x;
#pragma unroll
    for (int d = 0; d < 9; ++d) {
        const int xx = (tx + d % 3 - 1 + D.tiles_x) % D.tiles_x;
        const int yy = (ty + d / 3 - 1 + D.tiles_y) % D.tiles_y;
        nb[d] = src.done + D.tile_begin + yy * D.tiles_x + xx;
    }
}
__device__ __forceinline__ void flow_tile(const BatchFlowSrc& src, int t, int k, const KParams& p, int TX, int TY,
                                          int& x0, int& y0, Geom& g, const CUtensorMap*& lmap,
                                          const CUtensorMap*& smap, void*& out) {
    const int d = __ldg(src.tile_dom + t);
    const BatchDomain& D = src.dom[d];
    const int local = t - D.tile_begin;
    x0 = (local % D.tiles_x) * TX;
    y0 = (local / D.tiles_x) * TY;
    g.nx = D.nx;
    g.ny = D.ny;
    g.pitch = D.pitch;
    g.hx = p.hx;
    g.walls = 0;
    g.plane = D.plane;
    g.omegaf = D.omegaf;
    g.omegad = D.omegad;
    const int in = (src.cur + k) & 1;
    lmap = src.lmaps + 2 * d + in;
    smap = src.smaps + 2 * d + (in ^ 1);
    out = src.base + D.off[in ^ 1] * src.es;
}

// Layout of the dataflow kernel: the tiled form's compute threads plus one producer warp, and two
// stages of Q windows so that the next task's windows load while the current task is computed.
// Where shared memory also holds a whole output tile ([Q][TY][TX]), the compute threads write the
// collided cells there and a storer warp writes the tile out with TMA tensor stores (TMA_OUT):
// every access to the population buffers then goes through the async proxy but the periodic
// images, so no compute thread waits on a global proxy fence after its stores.
template <int N1, class C, int CFG>
struct FlowCfg {
    using Tile = TileCfg<N1, C, CFG>;
    static constexpr int STAGE_BYTES = Tile::Q * Tile::WIN_BYTES;
    // two stages where they fit (one otherwise: the producer then only overlaps the next
    // task's dependency wait with the current compute)
    static constexpr int STAGES = 2 * STAGE_BYTES + 256 <= 227 * 1024 ? 2 : 1;  // (3 measured slower: fewer CTAs)
    static constexpr int OUT_BYTES = Tile::Q * Tile::TX * Tile::TY * Tile::ES;
    static constexpr bool TMA_OUT = STAGES == 2 && STAGES * STAGE_BYTES + OUT_BYTES + 256 <= 227 * 1024;
    static constexpr int CONSUMERS = Tile::THREADS;          // compute threads (whole warps)
    static constexpr int THREADS = CONSUMERS + 32 + (TMA_OUT ? 32 : 0);  // + the producer (+ storer) warp
    static constexpr uint32_t TX_BYTES = (uint32_t)(Tile::Q * Tile::BX * Tile::BY * Tile::ES);
    // stages, the output tile, barriers + task slots, alignment
    static constexpr int SMEM = STAGES * STAGE_BYTES + (TMA_OUT ? OUT_BYTES : 0) + 128 + 128;
    static_assert(STAGES * 16 + 2 * STAGES * 4 + 16 + 8 <= 128, "barriers and slots exceed their area");
    static_assert(OUT_BYTES % (Tile::Q * 128) == 0 || !TMA_OUT, "output planes must stay 128-byte aligned");
    // resident CTAs per SM to compile for: as many as shared memory holds (228 KB per SM, 1 KB
    // reserved per CTA), but not so many that a thread gets fewer registers than the cell's
    // state needs: 96 for D2Q9/D2Q16 in FP32 (72 measured slower at five CTAs per SM than 96
    // at four), 128 in FP64, 168 for D2Q36 (255 in FP64)
    static constexpr int FIT = (228 * 1024) / (SMEM + 1024);
    static constexpr int REG_FLOOR = N1 >= 6 ? (Tile::ES == 8 ? 255 : 168) : (Tile::ES == 8 ? 128 : 96);
    static constexpr int REG_FIT = 65536 / (THREADS * REG_FLOOR);
    static constexpr int MINB = FIT < 1 ? 1 : (FIT < REG_FIT ? FIT : (REG_FIT < 1 ? 1 : REG_FIT));
    // what a finished task adds to its tile's completion counter: the storer's one release, or
    // one per compute warp
    static constexpr int DONE_PER_TASK = TMA_OUT ? 1 : CONSUMERS / 32;
    static_assert(CONSUMERS % 32 == 0, "compute threads must be whole warps");
    static_assert(SMEM <= 227 * 1024, "dataflow stages exceed shared memory");
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

// Producer (lane 0 of the first extra warp): take a task, wait for its neighbourhood, wait for a
// free stage, publish the task in the stage's slot and start its Q window loads.  A negative slot
// value ends the consumers' loop (-1: no tasks left, -2: a wait gave up).  Consumers (the tiled
// form's threads): wait for a stage, compute the tile, free the stage, and publish the tile's
// completion -- or, with TMA_OUT, hand the tile in shared memory to the storer (lane 0 of the
// second extra warp), which writes it with Q tensor stores, frees the output tile once they have
// read it, and publishes the completion once they are written.  Every wait is bounded; a
// consumer's wait allows for the producer's own ones.
template <int N1, class C, int CFG, class Src>
__global__ void __launch_bounds__(FlowCfg<N1, C, CFG>::THREADS, FlowCfg<N1, C, CFG>::MINB)
    sweep_flow_kernel(const __grid_constant__ Src src, const KParams p) {
    using Cfg = TileCfg<N1, C, CFG>;
    using F = FlowCfg<N1, C, CFG>;
    using T = typename C::T;
    constexpr int Q = N1 * N1, TX = Cfg::TX, TY = Cfg::TY, A = Cfg::A;
    constexpr int WIN = Cfg::WIN_BYTES, NCW = F::CONSUMERS / 32;
    constexpr uint64_t kConsumerLimitNs = 3 * kWaitLimitNs;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    T* out = reinterpret_cast<T*>(base + F::STAGES * F::STAGE_BYTES);  // output tile (TMA_OUT)
    uint64_t* full = reinterpret_cast<uint64_t*>(base + F::STAGES * F::STAGE_BYTES + (F::TMA_OUT ? F::OUT_BYTES : 0));
    uint64_t* empty = full + F::STAGES;
    uint64_t* ofull = empty + F::STAGES;   // output tile written (NCW warp arrivals)
    uint64_t* oempty = ofull + 1;          // output tile read by the stores (storer's arrival)
    volatile int* slot = reinterpret_cast<volatile int*>(oempty + 1);
    volatile int* oslot = slot + 2 * F::STAGES;  // the output tile's (tile, step) or end code
    const int tid = threadIdx.x;
    if (tid == 0) {
#pragma unroll
        for (int st = 0; st < F::STAGES; ++st) {
            mbar_init(&full[st], 1);
            mbar_init(&empty[st], NCW);
        }
        mbar_init(ofull, NCW);
        mbar_init(oempty, 1);
        fence_barrier_init();
    }
    __syncthreads();
    const int total = src.ntiles * src.nsteps;

    if (tid >= F::CONSUMERS + 32) {  // ---- storer warp (TMA_OUT) ----
        if constexpr (F::TMA_OUT) {
            if (tid != F::CONSUMERS + 32) return;
            for (int n = 0;; ++n) {
                if (!mbar_wait_bounded(ofull, n & 1, kConsumerLimitNs)) {
                    atomicExch(src.abort, 1);
                    if (p.status) atomicOr(p.status, 1);
                    return;
                }
                const int t = oslot[0], k = oslot[1];
                if (t < 0) return;  // no tiles left (every store of this thread has completed)
                int x0, y0;
                Geom g;
                const CUtensorMap *lmap, *map;
                void* outp;
                flow_tile(src, t, k, p, TX, TY, x0, y0, g, lmap, map, outp);
#pragma unroll 1
                for (int l = 0; l < Q; ++l) tma_store_3d(map, out + l * (TX * TY), x0 + g.hx, y0 + HY, l);
                bulk_commit();
                bulk_wait_read_all();
                mbar_arrive(oempty);  // the compute threads may write the next tile
                bulk_wait_all();
                fence_proxy_async_global();
                red_release_gpu_add(src.done + t, 1);
            }
        }
        return;
    }

    if (tid >= F::CONSUMERS) {  // ---- producer warp ----
        if (tid != F::CONSUMERS) return;
        // Issue the TMA loads of task `task` (step k, tile t) into stage st and publish it.
        auto issue = [&](int st, int t, int k) {
            int x0, y0;
            Geom g;
            const CUtensorMap *map, *smap;
            void* outp;
            flow_tile(src, t, k, p, TX, TY, x0, y0, g, map, smap, outp);
            slot[st] = t;  // slots: [stage] tile (>= 0) or end code, [STAGES + stage] step
            slot[F::STAGES + st] = k;
            mbar_arrive_expect_tx(&full[st], F::TX_BYTES);
            unsigned char* sb = base + st * F::STAGE_BYTES;
#pragma unroll
            for (int l = 0; l < Q; ++l) {
                const int i = l % N1, j = l / N1;
                tma_load_3d(sb + l * WIN, map, &full[st], (x0 + g.hx - p.sh[i] - 1) & ~(A - 1), y0 + HY - p.sh[j] - 1,
                            l);
            }
        };
        // Wait (bounded) until the 3 x 3 neighbourhoods of nt tasks (their completion counters nb,
        // the counts need) have completed their previous step: 0, or -2 once the wait gives up.
        auto await_nb = [&](const int* const (*nb)[9], const int* need, int nt) -> int {
            const uint64_t t0 = global_ns();
            for (;;) {
                int ready = 0;
                for (int q = 0; q < nt; ++q)
#pragma unroll
                    for (int d = 0; d < 9; ++d) ready += ld_relaxed_gpu(nb[q][d]) >= need[q] ? 1 : 0;
                if (ready == 9 * nt) return 0;
                if (*(volatile int*)src.abort || global_ns() - t0 > (uint64_t)src.wait_ns) return -2;
                __nanosleep(64);
            }
        };
        // Tasks come two at a time (stage 0, then stage 1, in the order they were handed out).
        // Two tasks of the same step do not depend on each other: their neighbourhoods are polled
        // together and one acquire fence covers both (the fence is the larger part of a task's
        // cost for this thread).  Across a step boundary the second may depend on the first, so
        // it is polled only after the first is issued.  With one stage, one task at a time.
        constexpr int PAIR = F::STAGES == 2 ? 2 : 1;
        for (int m = 0;; ++m) {
            const int task0 = atomicAdd(src.next_task, PAIR);
            const bool together = PAIR == 2 && task0 / src.ntiles == (task0 + 1) / src.ntiles;
            int code[2], k[2] = {0, 0}, t[2] = {0, 0}, need[2] = {0, 0};
            const int* nb[2][9];
            int nt = 0;  // tasks of this round that exist
#pragma unroll
            for (int q = 0; q < PAIR; ++q) {
                code[q] = task0 + q < total ? 0 : -1;
                if (!code[q]) {
                    flow_task(src, task0 + q, k[q], t[q], nb[q]);
                    need[q] = k[q] * F::DONE_PER_TASK + src.wait_extra;
                    ++nt;
                }
            }
            bool fenced = false;
            if (together && nt > 0) {
                const int c = await_nb(nb, need, nt);
                if (c) code[0] = code[1] = c;
                else {
                    fence_acquire_gpu();
                    fence_proxy_async_global();
                    fenced = true;
                }
            }
#pragma unroll
            for (int q = 0; q < PAIR; ++q) {
                const int st = q, n = PAIR * m + q;
                const uint32_t par = ((n / F::STAGES) & 1) ^ 1;  // first use of each stage passes at once
                if (!code[q] && !fenced) {
                    code[q] = await_nb(nb + q, need + q, 1);
                    if (!code[q]) {
                        fence_acquire_gpu();
                        fence_proxy_async_global();
                    }
                }
                if (!mbar_wait_bounded(&empty[st], par, kWaitLimitNs)) code[q] = -2;
                if (code[q] == -2) {
                    atomicExch(src.abort, 1);
                    if (p.status) atomicOr(p.status, 1);
                }
                if (code[q]) {
                    slot[st] = code[q];
                    mbar_arrive(&full[st]);  // release: the consumers see the slot
                    return;
                }
                issue(st, t[q], k[q]);
            }
        }
    }

    // ---- compute threads: each warp on its own through the stages ----
    for (int n = 0;; ++n) {
        const int st = n % F::STAGES;
        const uint32_t par = (n / F::STAGES) & 1;
        const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&full[st], par, kConsumerLimitNs));
        if (!ok) {
            if ((tid & 31) == 0) {
                atomicExch(src.abort, 1);
                if (p.status) atomicOr(p.status, 1);
            }
            if constexpr (F::TMA_OUT) {  // end the storer's loop too
                if (tid == 0) oslot[0] = -2;
                if ((tid & 31) == 0) mbar_arrive(ofull);
            }
            return;
        }
        const int code = slot[st];
        if constexpr (F::TMA_OUT) {
            // the output tile must have been read by the previous tile's stores (first use: free)
            const bool free_ok = __all_sync(0xffffffffu, mbar_wait_bounded(oempty, (n & 1) ^ 1, kConsumerLimitNs));
            if (code < 0 || !free_ok) {
                if (!free_ok && (tid & 31) == 0) {
                    atomicExch(src.abort, 1);
                    if (p.status) atomicOr(p.status, 1);
                }
                if (tid == 0) oslot[0] = code < 0 ? code : -2;
                __syncwarp();
                if ((tid & 31) == 0) mbar_arrive(ofull);  // the storer ends once every warp is here
                return;
            }
            const int t = code, k = slot[F::STAGES + st];
            int x0, y0;
            Geom g;
            const CUtensorMap *lmap, *smap;
            void* outp;
            flow_tile(src, t, k, p, TX, TY, x0, y0, g, lmap, smap, outp);
            const bool imaged = tile_compute<N1, C, CFG, false>(base + st * F::STAGE_BYTES, x0, y0, g,
                                                                reinterpret_cast<T*>(outp), p, tid, out);
            fence_proxy_async_shared();          // this thread's output tile writes, visible to the stores
            if (imaged) fence_proxy_async_global();  // its periodic images, visible to later TMA reads
            __syncwarp();
            if ((tid & 31) == 0) {
                mbar_arrive(&empty[st]);  // this warp is done with the stage
                if (tid == 0) {
                    oslot[0] = t;
                    oslot[1] = k;
                }
                mbar_arrive(ofull);
            }
        } else {
            if (code < 0) return;  // no tasks left, or the producer gave up
            const int t = code, k = slot[F::STAGES + st];
            int x0, y0;
            Geom g;
            const CUtensorMap *lmap, *smap;
            void* outp;
            flow_tile(src, t, k, p, TX, TY, x0, y0, g, lmap, smap, outp);
            tile_compute<N1, C, CFG, false>(base + st * F::STAGE_BYTES, x0, y0, g, reinterpret_cast<T*>(outp), p, tid);
            fence_proxy_async_global();  // this thread's stores, visible to the TMA reads of later tasks
            __syncwarp();                // orders the lanes' stores before lane 0's release
            if ((tid & 31) == 0) {
                mbar_arrive(&empty[st]);  // this warp is done with the stage
                red_release_gpu_add(src.done + t, 1);
            }
        }
    }
}

template <int N1, class C, int CFG, class Src>
inline cudaError_t flow_launch(const Src& src, const KParams& p, cudaStream_t s) {
    using F = FlowCfg<N1, C, CFG>;
    static int grid_of[64] = {};  // per device: SMs x resident CTAs
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!grid_of[dev]) {
        cudaError_t e = cudaFuncSetAttribute(sweep_flow_kernel<N1, C, CFG, Src>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, F::SMEM);
        if (e != cudaSuccess) return e;
        int nb = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, sweep_flow_kernel<N1, C, CFG, Src>, F::THREADS, F::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        grid_of[dev] = (nb > 0 ? nb : 1) * sms;
    }
    const long long tasks = (long long)src.ntiles * src.nsteps;
    const int grid = tasks < grid_of[dev] ? (int)tasks : grid_of[dev];
    sweep_flow_kernel<N1, C, CFG, Src><<<grid, F::THREADS, F::SMEM, s>>>(src, p);
    return cudaGetLastError();
}

template <int N1, class C, class Src>
inline cudaError_t flow_sweep(int cfg, const Src& src, const KParams& p, cudaStream_t s) {
    switch (cfg) {
        case 0: return flow_launch<N1, C, 0>(src, p, s);
        case 1: return flow_launch<N1, C, 1>(src, p, s);
        case 2: return flow_launch<N1, C, 2>(src, p, s);
        case 3: return flow_launch<N1, C, 3>(src, p, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace tvlbm
