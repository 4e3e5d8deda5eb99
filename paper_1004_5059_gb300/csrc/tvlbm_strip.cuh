// Strip sweep (TVLBM_FORM_STRIP): the fused collide + area-overlap gather of Sec. "The TVLBM
// model" walked down 128-column strips, with the loads of the rows ahead overlapping the rows
// being computed.
//
// The domain is cut into 128-column strips, and each strip into row ranges, one per CTA (see
// StripSrc), so a CTA owns a run of consecutive destination rows of one strip.  Its four warps
// take the strip's four 32-column quarters (lane = column) and walk the run one row at a time,
// with the x-interpolated previous row of every velocity carried in registers: a destination row
// then needs one new source row per velocity, and a run starts with one extra row for the carry
// (the tiled form pays that extra row once per 4-row thread segment).
//
// Source rows arrive in chunks of CH rows: one TMA tensor load per velocity, a box of BXC x CH
// elements (128 columns, the +1 source column of the interpolation, the 16-byte aligned start),
// into a ring of NS chunk slots completing on the slot's mbarrier.  A chunk is issued NS chunks
// ahead; the CTA meets once per chunk, and there the slot finished last is refilled, so the loads
// of the chunks ahead overlap the collision of the current one.  Each velocity's part of a slot
// starts on a 128-byte boundary (TMA destinations in shared memory).
#pragma once

#include "tvlbm_tiled.cuh"

namespace tvlbm {

template <int N1, class C>
struct StripCfg {
    static constexpr int ES = (int)sizeof(typename C::T);
    static constexpr int Q = N1 * N1;
    static constexpr int A = 16 / ES;                    // TMA x coordinates: 16-byte multiples
    static constexpr int WARPS = 4;
    static constexpr int THREADS = 32 * WARPS;
    static constexpr int SX = 32 * WARPS;                // strip width (columns)
    static constexpr int BXC = strip_box_width(ES);      // box width, elements (SX + A)
    static constexpr int ROW_BYTES = BXC * ES;
    // rows per chunk and chunk slots: as many as fit the CTA's share of shared memory (the CTAs
    // per SM that registers allow -- D2Q36 in 32-bit arithmetic is held to 3, see MINB --
    // sharing about 220 KB)
    static constexpr int CH = strip_chunk_rows(N1, ES);
    static constexpr int NS = strip_slots(N1, ES);
    static constexpr int POP_BYTES = strip_pop_bytes(ES, CH);
    static constexpr int SLOT_BYTES = Q * POP_BYTES;
    static constexpr int SMEM = NS * SLOT_BYTES + NS * 8 + 128;  // ring, barriers, alignment slack
    static_assert(SMEM <= 227 * 1024, "strip ring exceeds shared memory");
    static_assert(BXC >= SX + A, "box narrower than the strip's source columns");
    static_assert(ROW_BYTES % 16 == 0, "TMA box rows must be 16-byte multiples");
    static constexpr int MINB = (N1 >= 6 && sizeof(typename C::R) == 4) ? 65536 / (THREADS * 168) : 0;
};

// Work split.  With at least as many resident CTAs as strips, each strip is cut into P equal row
// ranges (P CTAs per strip, CTA b: strip b / P, part b % P), so the CTAs of neighbouring strips
// walk the same rows at the same time and share the source columns their boxes overlap in L2.
// With more strips than CTAs (P = 0), CTA b walks whole strips b, b + grid, b + 2 grid, ...
struct StripSrc {
    CUtensorMap map_in;  // box strip_box_width(es) x strip_chunk_rows(n1, es) x 1 over the input
    void* fout;
    int nstrips, per_strip;  // strips; CTAs per strip P (0: whole strips, strided)
};

// One run: destination rows [ya, yb) of strip sx; entry t of the run is destination row
// ya - 1 + t (t = 0: the carry row); chunk c holds entries [c CH, c CH + CH).
struct StripRun {
    int sx, ya, yb, c, step;
    __device__ __forceinline__ bool start(const StripSrc& src, int ny) {
        c = 0;
        if (src.per_strip > 0) {
            const int part = (int)blockIdx.x % src.per_strip;
            sx = (int)blockIdx.x / src.per_strip;
            ya = (int)((long long)ny * part / src.per_strip);
            yb = (int)((long long)ny * (part + 1) / src.per_strip);
            step = src.nstrips;  // a single run
        } else {
            sx = (int)blockIdx.x;
            ya = 0;
            yb = ny;
            step = (int)gridDim.x;
        }
        return sx < src.nstrips && ya < yb;
    }
    __device__ __forceinline__ int entries() const { return yb - ya + 1; }
    // to the next chunk; false when the CTA's work is done
    __device__ __forceinline__ bool next(const StripSrc& src, int ny, int ch) {
        if (++c * ch < entries()) return true;
        sx += step;
        if (sx >= src.nstrips) return false;
        ya = 0;
        yb = ny;
        c = 0;
        return true;
    }
};

template <int N1, class C, bool ROWS>
__device__ __forceinline__ void sweep_strip_body(const StripSrc& src, const KParams& p) {
    using Cfg = StripCfg<N1, C>;
    using R = typename C::R;
    using T = typename C::T;
    constexpr int Q = Cfg::Q, NS = Cfg::NS, CH = Cfg::CH, A = Cfg::A, ROWB = Cfg::ROW_BYTES;
    constexpr int POPB = Cfg::POP_BYTES, SLOTB = Cfg::SLOT_BYTES;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((128u - (smem_addr(smem_raw) & 127u)) & 127u);
    uint64_t* bars = reinterpret_cast<uint64_t*>(base + NS * SLOTB);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    pdl_launch_dependents();
    const Geom g = geom_of(p);
    StripRun ld, cc;  // load cursor (NS chunks ahead of the compute) and compute cursor
    if (!ld.start(src, g.ny)) return;  // the whole CTA leaves together
    cc = ld;

    // warp 0 issues the copies: the shifts of the (up to two) velocities each lane loads
    int shx[2] = {0, 0}, shy[2] = {0, 0};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int l = lane + 32 * k;
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            if (l % N1 == i) shx[k] = p.sh[i];
            if (l / N1 == i) shy[k] = p.sh[i];
        }
    }
    if (tid == 0) {
#pragma unroll
        for (int k = 0; k < NS; ++k) mbar_init(&bars[k], 1);
        fence_barrier_init();
    }
    __syncthreads();
    pdl_wait();  // the previous step's populations are complete from here on

    bool ld_more = true;
    auto issue = [&](int slot) {  // warp 0: copy chunk (ld.sx, ld.c) into slot
        const int yk = ld.ya - 1 + ld.c * CH, xs = ld.sx * Cfg::SX + g.hx - 1;
        if (lane == 0) mbar_arrive_expect_tx(&bars[slot], (uint32_t)(Q * CH * ROWB));
        __syncwarp();
        unsigned char* dst = base + slot * SLOTB;
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int l = lane + 32 * k;
            if (l < Q)
                tma_load_3d(dst + l * POPB, &src.map_in, &bars[slot], (xs - shx[k]) & ~(A - 1), yk + HY - shy[k], l);
        }
        ld_more = ld.next(src, g.ny, CH);
    };
    if (warp == 0) {
#pragma unroll 1
        for (int k = 0; k < NS && ld_more; ++k) issue(k);
    }

    // byte offset of this thread's column (+ alignment remainder) within a source row, per
    // x-node; strip origins are multiples of SX (>= A), so the remainder depends on the node only
    const int cx = tid;
    int off[N1];
#pragma unroll
    for (int i = 0; i < N1; ++i) off[i] = (cx + ((g.hx - p.sh[i] - 1) & (A - 1))) * Cfg::ES;

    R hprev[Q], s[Q];
    bool more = true;
    int k = 0;  // chunk index
#pragma unroll 1
    while (more) {
        const int slot = k % NS;
        // each thread orders its reads of the previous chunk's slot before the copy that refills
        // it and waits for this chunk (acquiring it); the CTA then meets
        fence_proxy_async_shared();
        const bool arrived = mbar_wait_bounded(&bars[slot], (uint32_t)((k / NS) & 1), kWaitLimitNs);
        if (!__syncthreads_and(arrived)) {
            // a chunk never arrived: report it and give the copies still in flight a bounded
            // chance to land before the CTA's shared memory is released
            if (tid == 0) {
                if (p.status) atomicOr(p.status, 1);
#pragma unroll 1
                for (int e = 0; e < NS; ++e) mbar_wait_bounded(&bars[(k + e) % NS], (uint32_t)(((k + e) / NS) & 1), kWaitLimitNs);
            }
            __syncthreads();
            return;
        }
        // every thread is done with the previous chunk: refill its slot NS chunks ahead
        if (k > 0 && warp == 0 && ld_more) issue((k - 1) % NS);
        const unsigned char* chunk = base + slot * SLOTB;
        const int left = cc.entries() - cc.c * CH;
        const int rows = left < CH ? left : CH;
        const int x = cc.sx * Cfg::SX + cx;
#pragma unroll 1
        for (int t = 0; t < rows; ++t) {
            const unsigned char* row = chunk + t * ROWB;
            const int e = cc.c * CH + t;  // entry within the run
            if (e == 0) {
                gather_row<N1, C, POPB, true>(row, off, p, hprev, s);
            } else {
                gather_row<N1, C, POPB, false>(row, off, p, hprev, s);
                const int y = cc.ya - 1 + e;
                if (x < g.nx) {
                    collide_cell<N1, C, ROWS>(s, p, g, y);
                    store_collided<N1, C>(reinterpret_cast<T*>(src.fout), g, x, y, s);
                }
            }
        }
        more = cc.next(src, g.ny, CH);
        ++k;
    }
}

template <int N1, class C, bool ROWS>
__global__ void __launch_bounds__(StripCfg<N1, C>::THREADS)
    sweep_strip_kernel(const __grid_constant__ StripSrc src, const KParams p) {
    sweep_strip_body<N1, C, ROWS>(src, p);
}
template <int N1, class C, bool ROWS>
__global__ void __launch_bounds__(StripCfg<N1, C>::THREADS, (StripCfg<N1, C>::MINB > 0 ? StripCfg<N1, C>::MINB : 1))
    sweep_strip_kernel_minb(const __grid_constant__ StripSrc src, const KParams p) {
    sweep_strip_body<N1, C, ROWS>(src, p);
}
template <int N1, class C, bool ROWS>
constexpr auto strip_kernel() {
    if constexpr (StripCfg<N1, C>::MINB > 0)
        return sweep_strip_kernel_minb<N1, C, ROWS>;
    else
        return sweep_strip_kernel<N1, C, ROWS>;
}

// One launch of one time step: about as many CTAs as fit on the device at once, each strip cut
// into at most ny / 8 parts (at least 8 rows a CTA).
template <int N1, class C, bool ROWS>
inline cudaError_t strip_launch_rows(const SweepMaps* maps, typename C::T* fout, const KParams& p, cudaStream_t s) {
    using Cfg = StripCfg<N1, C>;
    static int resident[64] = {};  // CTAs the device holds at once, per device
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!resident[dev]) {
        cudaError_t e = cudaFuncSetAttribute(strip_kernel<N1, C, ROWS>(), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             Cfg::SMEM);
        if (e != cudaSuccess) return e;
        int per_sm = 0, sms = 0;
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, strip_kernel<N1, C, ROWS>(), Cfg::THREADS, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        resident[dev] = (per_sm > 0 ? per_sm : 1) * (sms > 0 ? sms : 1);
    }
    StripSrc src;
    src.map_in = *(const CUtensorMap*)maps->in;
    src.fout = fout;
    src.nstrips = (p.nx + Cfg::SX - 1) / Cfg::SX;
    int per = resident[dev] / src.nstrips;
    if (per > p.ny / 8) per = p.ny / 8;
    src.per_strip = src.nstrips <= resident[dev] ? (per > 1 ? per : 1) : 0;
    const int ctas = src.per_strip > 0 ? src.per_strip * src.nstrips : resident[dev];
    return launch_pdl(strip_kernel<N1, C, ROWS>(), dim3((unsigned)ctas), dim3(Cfg::THREADS), Cfg::SMEM, s, src, p);
}

template <int N1, class C>
inline cudaError_t strip_sweep(const SweepMaps* maps, typename C::T* fout, const KParams& p, cudaStream_t s) {
    if constexpr (C::dev) {
        if (p.rowf) return strip_launch_rows<N1, C, true>(maps, fout, p, s);
    }
    return strip_launch_rows<N1, C, false>(maps, fout, p, s);
}

}  // namespace tvlbm
