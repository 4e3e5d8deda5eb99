// The closure network on Blackwell tensor cores: every matrix product of inference and training
// is one tcgen05 GEMM kernel, D[rows x BN] = A[rows x K] * B[BN x K]^T with BF16 operands in
// K-major layout (TMA 2-D loads, 128-byte swizzle, a STAGES-deep ring of shared-memory stages),
// the FP32 accumulator in TMEM, and an epilogue that reads TMEM row by row (thread = row) and
// fuses bias, GELU, its derivative, the loss, transposed copies and bias gradients.
//
// Forward:  Z1 = X W1^T + b1, H1 = g(Z1);  Z2 = H1 W2^T + b2, H2 = g(Z2);  Y = H2 W3^T + b3.
// Backward (L = mean (Y - Y*)^2):  dY = 2 (Y - Y*) / (rows 12);  dZ2 = (dY W3) o g'(Z2);
//   dZ1 = (dZ2 W2) o g'(Z1);  dW3 = dY^T H2, dW2 = dZ2^T H1, dW1 = dZ1^T X (split over rows,
//   partial sums reduced in a fixed order);  db = column sums (atomics).
// Every operand a later product needs transposed is written transposed by the epilogue that
// produces it, so that all products keep K-major operands.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <new>

#include "tvlbm.h"
#include "tvlbm_closure.h"
#include "tvlbm_host.h"
#include "tvlbm_mlp.h"
#include "tvlbm_tc.cuh"

using namespace tvlbm;
using namespace tvlbm::tc;

namespace {

constexpr int BM = 128, BK = 64;
constexpr int NIN = TVLBM_MLP_IN, NINP = TVLBM_MLP_IN_PAD, NH = TVLBM_MLP_HIDDEN, NOUT = TVLBM_MLP_OUT,
              NOUTP = TVLBM_MLP_OUT_PAD;
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + NH * NIN, OFF_W2 = OFF_B1 + NH, OFF_B2 = OFF_W2 + NH * NH,
              OFF_W3 = OFF_B2 + NH, OFF_B3 = OFF_W3 + NOUT * NH, NPARAM = OFF_B3 + NOUT;
static_assert(NPARAM == TVLBM_MLP_PARAMS, "parameter count");
constexpr int kMaxSplits = 128;

using bf16 = __nv_bfloat16;

// GELU g(z) = z Phi(z), Phi(z) = (1 + erf(z / sqrt 2)) / 2, and g'(z) = Phi(z) + z phi(z).  erf by
// the rational approximation of Abramowitz & Stegun, Handbook of Mathematical Functions, eq.
// 7.1.26 (after Hastings): erf(x) = 1 - (a1 t + ... + a5 t^5) exp(-x^2), t = 1 / (1 + p x), x >= 0,
// |error| <= 1.5e-7, odd in x; the reciprocal and the exponential by the hardware approximations.
// The network stores its activations in BF16 (relative step 2^-8), so the error is invisible.
// E2 = exp(-x^2) = exp(-z^2 / 2) also gives phi(z) = E2 / sqrt(2 pi).
__device__ __forceinline__ float erf_as(float x, float& e2) {
    const float ax = fabsf(x);
    const float t = __fdividef(1.0f, fmaf(0.3275911f, ax, 1.0f));
    const float poly =
        t * fmaf(t, fmaf(t, fmaf(t, fmaf(t, 1.061405429f, -1.453152027f), 1.421413741f), -0.284496736f), 0.254829592f);
    e2 = __expf(-ax * ax);
    return copysignf(fmaf(-poly, e2, 1.0f), x);
}
__device__ __forceinline__ float gelu_f(float z) {
    float e2;
    return 0.5f * z * (1.0f + erf_as(z * 0.70710678118654752f, e2));
}
// Two GELUs in packed FP32 pairs, per lane the operations of gelu_f in its order (a packed
// multiply, add or fused multiply-add rounds each lane as the scalar instruction; the
// reciprocal, the exponential, |x| and the sign stay scalar).  The forward epilogues and
// tvlbm_mlp_activation's g use it.
__device__ __forceinline__ float2 gelu2_f(float2 z) {
    const float2 x = __fmul2_rn(z, make_float2(0.70710678118654752f, 0.70710678118654752f));
    const float2 ax = make_float2(fabsf(x.x), fabsf(x.y));
    const float2 d = __ffma2_rn(make_float2(0.3275911f, 0.3275911f), ax, make_float2(1.0f, 1.0f));
    const float2 t = make_float2(__fdividef(1.0f, d.x), __fdividef(1.0f, d.y));
    float2 q = __ffma2_rn(t, make_float2(1.061405429f, 1.061405429f), make_float2(-1.453152027f, -1.453152027f));
    q = __ffma2_rn(t, q, make_float2(1.421413741f, 1.421413741f));
    q = __ffma2_rn(t, q, make_float2(-0.284496736f, -0.284496736f));
    q = __ffma2_rn(t, q, make_float2(0.254829592f, 0.254829592f));
    const float2 poly = __fmul2_rn(t, q);
    const float2 sq = __fmul2_rn(make_float2(-ax.x, -ax.y), ax);
    const float2 e2 = make_float2(__expf(sq.x), __expf(sq.y));
    const float2 r = __ffma2_rn(make_float2(-poly.x, -poly.y), e2, make_float2(1.0f, 1.0f));
    const float2 er = make_float2(copysignf(r.x, x.x), copysignf(r.y, x.y));
    return __fmul2_rn(__fmul2_rn(make_float2(0.5f, 0.5f), z), __fadd2_rn(make_float2(1.0f, 1.0f), er));
}
__device__ __forceinline__ float gelu_grad_f(float z) {
    float e2;
    const float er = erf_as(z * 0.70710678118654752f, e2);
    return fmaf(z * 0.39894228040143268f, e2, 0.5f * (1.0f + er));
}
__global__ void activation_kernel(const float* __restrict__ z, float* __restrict__ g, float* __restrict__ dg, int n) {
    // pairs of entries, g in the packed form of the forward epilogues (an odd last entry alone)
    for (int i = 2 * (blockIdx.x * blockDim.x + threadIdx.x); i < n; i += 2 * gridDim.x * blockDim.x) {
        if (i + 1 < n) {
            if (g) {
                const float2 r = gelu2_f(make_float2(z[i], z[i + 1]));
                g[i] = r.x;
                g[i + 1] = r.y;
            }
            if (dg) {
                dg[i] = gelu_grad_f(z[i]);
                dg[i + 1] = gelu_grad_f(z[i + 1]);
            }
        } else {
            if (g) g[i] = gelu_f(z[i]);
            if (dg) dg[i] = gelu_grad_f(z[i]);
        }
    }
}
__device__ __forceinline__ float warp_sum_f(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---- epilogues: called by every thread with its row and 16 consecutive accumulator columns ----

// Hidden layer: h = g(z + b) to H[row][col] (and H^T[col][row]); g'(z + b) to G[row][col].
struct EpiHidden {
    const float* bias;
    bf16* H;   // [rows][128] or null
    bf16* HT;  // [128][ldt] or null
    bf16* G;   // [rows][128] or null
    int ldt;
    __device__ void operator()(int row, int c0, const float (&v)[16], int /*lane*/) const {
        alignas(16) bf16 h[16], gg[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float z = v[k] + bias[c0 + k];
            h[k] = __float2bfloat16_rn(gelu_f(z));
            gg[k] = __float2bfloat16_rn(gelu_grad_f(z));
        }
        if (H) {
            uint4* d = reinterpret_cast<uint4*>(H + (size_t)row * NH + c0);
            d[0] = reinterpret_cast<const uint4*>(h)[0];
            d[1] = reinterpret_cast<const uint4*>(h)[1];
        }
        if (G) {
            uint4* d = reinterpret_cast<uint4*>(G + (size_t)row * NH + c0);
            d[0] = reinterpret_cast<const uint4*>(gg)[0];
            d[1] = reinterpret_cast<const uint4*>(gg)[1];
        }
        if (HT) {
#pragma unroll
            for (int k = 0; k < 16; ++k) HT[(size_t)(c0 + k) * ldt + row] = h[k];
        }
    }
};

// Output layer: y = z + b3 to Y (FP32 [rows][16]); with targets, dY = scale (y - y*) to
// dY[row][0..15] (BF16, row length 64) and dY^T[col][row], the loss sum and db3.
struct EpiOut {
    const float* bias;
    float* Y;            // [rows][16] or null
    const float* ystar;  // [rows][16] or null (inference)
    bf16* dY;            // [rows][64]
    bf16* dYT;           // [16][ldt]
    double* loss;
    float* db;  // gradient of b3 (12)
    float scale;
    int ldt;
    __device__ void operator()(int row, int c0, const float (&v)[16], int lane) const {
        float y[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) y[k] = k < NOUT ? v[k] + bias[k] : 0.0f;
        if (Y) {
            float4* d = reinterpret_cast<float4*>(Y + (size_t)row * NOUTP);
#pragma unroll
            for (int q = 0; q < 4; ++q) d[q] = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
        }
        if (!ystar) return;
        (void)c0;
        float sq = 0.0f;
        alignas(16) bf16 g[16];
        float gf[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float d = k < NOUT ? y[k] - ystar[(size_t)row * NOUTP + k] : 0.0f;
            sq = fmaf(d, d, sq);
            gf[k] = scale * d;
            g[k] = __float2bfloat16_rn(gf[k]);
        }
        uint4* d = reinterpret_cast<uint4*>(dY + (size_t)row * NINP);
        d[0] = reinterpret_cast<const uint4*>(g)[0];
        d[1] = reinterpret_cast<const uint4*>(g)[1];
#pragma unroll
        for (int k = 0; k < 16; ++k) dYT[(size_t)k * ldt + row] = g[k];
        const float s = warp_sum_f(sq);
        if (lane == 0) atomicAdd(loss, (double)s);
#pragma unroll
        for (int k = 0; k < NOUT; ++k) {
            const float t = warp_sum_f(gf[k]);
            if (lane == 0) atomicAdd(db + k, t);
        }
    }
};

// Back through a GELU: dz = acc o G to dZ[row][col] (optional) and dZ^T[col][row]; db += dz.
struct EpiBack {
    const bf16* G;  // [rows][128]
    bf16* dZ;       // [rows][128] or null
    bf16* dZT;      // [128][ldt]
    float* db;      // [128]
    int ldt;
    __device__ void operator()(int row, int c0, const float (&v)[16], int lane) const {
        alignas(16) bf16 gb[16], z[16];
        const uint4* gs = reinterpret_cast<const uint4*>(G + (size_t)row * NH + c0);
        reinterpret_cast<uint4*>(gb)[0] = gs[0];
        reinterpret_cast<uint4*>(gb)[1] = gs[1];
        float dz[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            dz[k] = v[k] * __bfloat162float(gb[k]);
            z[k] = __float2bfloat16_rn(dz[k]);
        }
        if (dZ) {
            uint4* d = reinterpret_cast<uint4*>(dZ + (size_t)row * NH + c0);
            d[0] = reinterpret_cast<const uint4*>(z)[0];
            d[1] = reinterpret_cast<const uint4*>(z)[1];
        }
#pragma unroll
        for (int k = 0; k < 16; ++k) dZT[(size_t)(c0 + k) * ldt + row] = z[k];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
            const float t = warp_sum_f(dz[k]);
            if (lane == 0) atomicAdd(db + c0 + k, t);
        }
    }
};

// Split-K partial sums: part[split][row][col] (row < 128, ld = BN).
struct EpiPartial {
    float* part;
    int ld;
    __device__ void operator()(int row, int c0, const float (&v)[16], int /*lane*/) const {
        float* d = part + ((size_t)blockIdx.y * BM + row) * ld + c0;
#pragma unroll
        for (int q = 0; q < 4; ++q)
            reinterpret_cast<float4*>(d)[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
};

// ---- the GEMM kernel ---------------------------------------------------------------------------
template <int BN, int STAGES>
struct GemmCfg {
    static constexpr int A_BYTES = BM * BK * 2;  // 16 KB
    static constexpr int B_BYTES = BN * BK * 2;
    static constexpr int STAGE_BYTES = A_BYTES + B_BYTES;  // multiple of 1024
    static constexpr int SMEM = STAGES * STAGE_BYTES + 1024;
    static constexpr uint32_t TMEM_COLS = BN < 32 ? 32 : BN;
    static_assert(STAGE_BYTES % 1024 == 0, "stages must keep 1024-byte alignment");
    static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "N of a kind::f16 MMA with M = 128");
};

// CTA (blockIdx.x, blockIdx.y): rows [128 x, 128 x + 128), K chunks [y cps, min(kchunks, (y+1) cps)).
// Thread 0 loads stages and issues the MMAs; all 128 threads then drain TMEM through the epilogue
// (warp w owns TMEM lanes, i.e. rows, 32 w .. 32 w + 31).
template <int BN, int STAGES, class Epi>
__global__ void __launch_bounds__(128) gemm_kernel(const __grid_constant__ CUtensorMap ma,
                                                   const __grid_constant__ CUtensorMap mb, int kchunks, int cps, Epi epi,
                                                   int* status) {
    using Cfg = GemmCfg<BN, STAGES>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
    __shared__ uint64_t full[STAGES], empty[STAGES], done;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM;
    const int k0 = blockIdx.y * cps;
    const int nk = min(kchunks, k0 + cps) - k0;  // >= 1 (host grid)

    if (tid == 0) {
#pragma unroll
        for (int s = 0; s < STAGES; ++s) {
            bar_init(&full[s], 1);
            bar_init(&empty[s], 1);
        }
        bar_init(&done, 1);
        bar_init_fence();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, Cfg::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    bool ok = true;
    if (tid == 0) {
        const uint32_t idesc = idesc_bf16_f32(BM, BN);
        auto load = [&](int c) {
            const int s = c % STAGES;
            unsigned char* a = base + s * Cfg::STAGE_BYTES;
            bar_expect_tx(&full[s], (uint32_t)Cfg::STAGE_BYTES);
            tma_load_2d(a, &ma, &full[s], (k0 + c) * BK, m0);
            tma_load_2d(a + Cfg::A_BYTES, &mb, &full[s], (k0 + c) * BK, 0);
        };
        const int pre = nk < STAGES ? nk : STAGES;
        for (int c = 0; c < pre; ++c) load(c);
        int issued = pre;
        for (int c = 0; c < nk; ++c) {
            const int s = c % STAGES;
            const uint32_t par = (uint32_t)((c / STAGES) & 1);
            if (!bar_wait(&full[s], par)) {
                ok = false;
                break;
            }
            tc_fence_after();
            const uint32_t a = saddr(base + s * Cfg::STAGE_BYTES);
            const uint32_t b = a + Cfg::A_BYTES;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(a + kk * 32), sw128_desc(b + kk * 32), idesc, c > 0 || kk > 0);
            mma_commit(&empty[s]);
            if (c + STAGES < nk) {
                if (!bar_wait(&empty[s], par)) {  // the MMAs reading stage s are done
                    ok = false;
                    break;
                }
                load(c + STAGES);
                ++issued;
            }
        }
        mma_commit(&done);
        if (!ok) {
            // let every issued load land before the CTA exits (bounded)
            for (int c = 0; c < issued; ++c) bar_wait(&full[c % STAGES], (uint32_t)((c / STAGES) & 1));
        }
    }
    const bool ready = bar_wait(&done, 0);
    const bool all = __syncthreads_and(ready && ok) != 0;
    tc_fence_after();
    if (all) {
        const int row = m0 + warp * 32 + lane;
        const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
        for (int c0 = 0; c0 < BN; c0 += 16) {
            float v[16];
            __syncwarp();
            tmem_ld16(taddr + (uint32_t)c0, v);
            epi(row, c0, v, lane);
        }
    } else if (tid == 0 && status) {
        atomicOr(status, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, Cfg::TMEM_COLS);
}

// ---- fused inference: the three layers of one 128-row tile in one CTA ---------------------------
// X, W1, W2, W3 arrive by TMA (128-byte swizzle); H1 and H2 never leave shared memory: the
// epilogue threads write them in the same swizzled K-major layout the next MMA reads.  TMEM:
// columns [0, 128) hold layer 1, [128, 256) layer 2, [0, 16) then layer 3.
struct FusedCfg {
    static constexpr int X_OFF = 0, W1_OFF = 16384, W2_OFF = 32768, W3_OFF = 65536, H_OFF = 69632;
    static constexpr int BYTES = H_OFF + 32768;  // 100 KB
    static constexpr int SMEM = BYTES + 1024;
    static constexpr uint32_t TX = 16384 + 16384 + 32768 + 4096;
    static constexpr uint32_t TMEM_COLS = 256;
};

// Row r of a [128][128] BF16 tile stored as two 128-byte-swizzled K-major chunks of 64 columns:
// columns c0 .. c0 + 15 (c0 a multiple of 16) from 16 FP32 values.
__device__ __forceinline__ void store_h_sw128(unsigned char* h, int r, int c0, const float (&v)[16]) {
    const int kc = c0 >> 6, j0 = (c0 & 63) >> 3;  // chunk, first 16-byte unit in the row
#pragma unroll
    for (int half = 0; half < 2; ++half) {
        alignas(16) __nv_bfloat16 b[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) b[q] = __float2bfloat16_rn(v[8 * half + q]);
        const int j = (j0 + half) ^ (r & 7);
        *reinterpret_cast<uint4*>(h + kc * 16384 + r * 128 + j * 16) = *reinterpret_cast<const uint4*>(b);
    }
}

// kFusedGroups warpgroups: warp w reads TMEM lanes 32 (w % 4) .. + 31 (its rows) and takes the
// (w / 4)-th of kFusedGroups column ranges of each hidden layer's epilogue, so every row's 128
// GELUs are split over kFusedGroups threads; the output layer's 16 columns go to the first
// warpgroup.
constexpr int kFusedGroups = 4;
constexpr int kFusedThreads = 128 * kFusedGroups;
static_assert(NH % (16 * kFusedGroups) == 0, "column ranges of whole 16-column loads");
static_assert(NINP == 16 * kFusedGroups, "FEAT: one 16-column input chunk per warpgroup");

// Features 16 G .. 16 G + 15 of cell `cell` (see MlpFeatures); neighbours wrap periodically.
template <int G>
__device__ __forceinline__ void feature_chunk(const MlpFeatures& f, int cell, float (&v)[16]) {
    const int cy = cell / f.nx, cx = cell - cy * f.nx;
    const long long n = (long long)f.nx * f.ny;
    const int xm = cx == 0 ? f.nx - 1 : cx - 1, xp = cx == f.nx - 1 ? 0 : cx + 1;
    const int ym = cy == 0 ? f.ny - 1 : cy - 1, yp = cy == f.ny - 1 ? 0 : cy + 1;
#pragma unroll
    for (int e = 0; e < 16; ++e) {
        constexpr int base = 16 * G;
        const int fi = base + e;  // compile time once unrolled
        if (fi >= NIN) {
            v[e] = 0.0f;
            continue;
        }
        const int k = fi / 6, q = fi % 6;
        const int xx = k % 3 == 0 ? xm : (k % 3 == 1 ? cx : xp), yy = k / 3 == 0 ? ym : (k / 3 == 1 ? cy : yp);
        v[e] = (__ldg(f.m6 + q * n + (long long)yy * f.nx + xx) - f.mu[q]) * f.isg[q];
    }
}

// FEAT: the input tile is built by the CTA's threads from the closure's moments (MlpFeatures)
// instead of loaded by TMA; thread (row r, warpgroup g) makes features 16 g .. 16 g + 15 of row
// r with the closure features kernel's arithmetic, so the inputs are the same BF16 values.
template <bool FEAT>
__global__ void __launch_bounds__(kFusedThreads) mlp_fused_forward_kernel(const __grid_constant__ CUtensorMap mx,
                                                                const __grid_constant__ CUtensorMap mw1,
                                                                const __grid_constant__ CUtensorMap mw2,
                                                                const __grid_constant__ CUtensorMap mw3,
                                                                const float* __restrict__ theta, float* __restrict__ y,
                                                                int* status, const MlpFeatures feat) {
    extern __shared__ unsigned char smem_raw[];
    unsigned char* base = smem_raw + ((1024u - (saddr(smem_raw) & 1023u)) & 1023u);
    __shared__ uint64_t load_bar, mma_bar;
    __shared__ uint32_t tmem_slot;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int m0 = blockIdx.x * BM;
    const float* b1 = theta + OFF_B1;
    const float* b2 = theta + OFF_B2;
    const float* b3 = theta + OFF_B3;
    if (tid == 0) {
        bar_init(&load_bar, 1);
        bar_init(&mma_bar, 1);
        bar_init_fence();
    }
    if (warp == 0) tmem_alloc(&tmem_slot, FusedCfg::TMEM_COLS);
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    unsigned char* xs = base + FusedCfg::X_OFF;
    unsigned char* w1 = base + FusedCfg::W1_OFF;
    unsigned char* w2 = base + FusedCfg::W2_OFF;
    unsigned char* w3 = base + FusedCfg::W3_OFF;
    unsigned char* hs = base + FusedCfg::H_OFF;
    const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16);
    const int r = (warp & 3) * 32 + lane;  // this thread's row of the tile (= its TMEM lane)
    const int cbeg = (warp >> 2) * (NH / kFusedGroups), cend = cbeg + NH / kFusedGroups;  // its column range

    bool ok = true;
    if (tid == 0) {
        bar_expect_tx(&load_bar, FEAT ? FusedCfg::TX - (uint32_t)(BM * NINP * 2) : FusedCfg::TX);
        if (!FEAT) tma_load_2d(xs, &mx, &load_bar, 0, m0);
        tma_load_2d(w1, &mw1, &load_bar, 0, 0);
        tma_load_2d(w2, &mw2, &load_bar, 0, 0);
        tma_load_2d(w2 + 16384, &mw2, &load_bar, BK, 0);
        tma_load_2d(w3, &mw3, &load_bar, 0, 0);
        tma_load_2d(w3 + 2048, &mw3, &load_bar, BK, 0);
    }
    if constexpr (FEAT) {
        // this thread's 16 input columns 16 g .. 16 g + 15 of row r, each builder with its feature
        // indices known at compile time
        const int g = warp >> 2;
        float v[16];
        switch (g) {
            case 0: feature_chunk<0>(feat, m0 + r, v); break;
            case 1: feature_chunk<1>(feat, m0 + r, v); break;
            case 2: feature_chunk<2>(feat, m0 + r, v); break;
            default: feature_chunk<3>(feat, m0 + r, v); break;
        }
        store_h_sw128(xs, r, 16 * g, v);
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> MMA reads
        __syncthreads();
    }
    if (tid == 0) {
        ok = bar_wait(&load_bar, 0);
        if (ok) {
            tc_fence_after();
            const uint32_t idesc = idesc_bf16_f32(BM, NH);
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk)
                mma_bf16(tmem, sw128_desc(saddr(xs) + kk * 32), sw128_desc(saddr(w1) + kk * 32), idesc, kk > 0);
        }
        mma_commit(&mma_bar);
    }
    // layer 1 epilogue: H1 = g(Z1 + b1) into shared memory
    ok = __syncthreads_and((tid != 0 || ok) && bar_wait(&mma_bar, 0)) != 0;
    tc_fence_after();
    if (ok) {
#pragma unroll 1
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            float v[16];
            __syncwarp();
            tmem_ld16(taddr + (uint32_t)c0, v);
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const float2 g = gelu2_f(__fadd2_rn(make_float2(v[k], v[k + 1]), make_float2(b1[c0 + k], b1[c0 + k + 1])));
                v[k] = g.x;
                v[k + 1] = g.y;
            }
            store_h_sw128(hs, r, c0, v);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // generic writes -> MMA reads
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        if (ok) {
            tc_fence_after();
            const uint32_t idesc = idesc_bf16_f32(BM, NH);
#pragma unroll
            for (int kc = 0; kc < 2; ++kc)
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    mma_bf16(tmem + NH, sw128_desc(saddr(hs) + kc * 16384 + kk * 32),
                             sw128_desc(saddr(w2) + kc * 16384 + kk * 32), idesc, kc > 0 || kk > 0);
        }
        mma_commit(&mma_bar);
    }
    // layer 2 epilogue: H2 = g(Z2 + b2) over H1 (the MMA that read H1 has completed)
    ok = __syncthreads_and(ok && bar_wait(&mma_bar, 1)) != 0;
    tc_fence_after();
    if (ok) {
#pragma unroll 1
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
            float v[16];
            __syncwarp();
            tmem_ld16(taddr + (uint32_t)(NH + c0), v);
#pragma unroll
            for (int k = 0; k < 16; k += 2) {
                const float2 g = gelu2_f(__fadd2_rn(make_float2(v[k], v[k + 1]), make_float2(b2[c0 + k], b2[c0 + k + 1])));
                v[k] = g.x;
                v[k + 1] = g.y;
            }
            store_h_sw128(hs, r, c0, v);
        }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    tc_fence_before();
    __syncthreads();
    if (tid == 0) {
        if (ok) {
            tc_fence_after();
            const uint32_t idesc = idesc_bf16_f32(BM, NOUTP);
#pragma unroll
            for (int kc = 0; kc < 2; ++kc)
#pragma unroll
                for (int kk = 0; kk < BK / 16; ++kk)
                    mma_bf16(tmem, sw128_desc(saddr(hs) + kc * 16384 + kk * 32),
                             sw128_desc(saddr(w3) + kc * 2048 + kk * 32), idesc, kc > 0 || kk > 0);
        }
        mma_commit(&mma_bar);
    }
    ok = __syncthreads_and(ok && bar_wait(&mma_bar, 0)) != 0;
    tc_fence_after();
    if (ok && warp < 4) {
        float v[16];
        __syncwarp();
        tmem_ld16(taddr, v);
        float4* d = reinterpret_cast<float4*>(y + (size_t)(m0 + r) * NOUTP);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            float o[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) o[e] = 4 * q + e < NOUT ? v[4 * q + e] + b3[4 * q + e] : 0.0f;
            d[q] = make_float4(o[0], o[1], o[2], o[3]);
        }
    } else if (tid == 0 && status) {
        atomicOr(status, 1);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) tmem_free(tmem, FusedCfg::TMEM_COLS);
}

// ---- small kernels ---------------------------------------------------------------------------

// x [rows][64] -> xt [64][rows]
__global__ void transpose_x_kernel(const bf16* __restrict__ x, bf16* __restrict__ xt, int rows) {
    __shared__ bf16 t[32][33];
    const int r0 = blockIdx.x * 32, c0 = blockIdx.y * 32;
    for (int k = threadIdx.y; k < 32; k += blockDim.y) t[k][threadIdx.x] = x[(size_t)(r0 + k) * NINP + c0 + threadIdx.x];
    __syncthreads();
    for (int k = threadIdx.y; k < 32; k += blockDim.y) xt[(size_t)(c0 + k) * rows + r0 + threadIdx.x] = t[threadIdx.x][k];
}

// grad[dst(r, c)] = sum over splits of part[s][r][c], r < 128, c < cols (fixed order).
__global__ void reduce_partials_kernel(const float* __restrict__ part, int splits, int ld, int cols, float* __restrict__ grad,
                                       int kind) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= BM * cols) return;
    const int r = i / cols, c = i - r * cols;
    float acc = 0.0f;
    for (int s = 0; s < splits; ++s) acc += part[((size_t)s * BM + r) * ld + c];
    if (kind == 0) {  // dW1: [128][64] -> W1[r][c], c < 54
        if (c < NIN) grad[OFF_W1 + r * NIN + c] = acc;
    } else if (kind == 1) {  // dW2
        grad[OFF_W2 + r * NH + c] = acc;
    } else {  // dW3^T: [128 h][16 o] -> W3[o][h], o < 12
        if (c < NOUT) grad[OFF_W3 + c * NH + r] = acc;
    }
}

__global__ void adam_kernel(float* __restrict__ theta, float* __restrict__ m1, float* __restrict__ m2,
                            const float* __restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float a = b1 * m1[i] + (1.0f - b1) * gi;
    const float b = b2 * m2[i] + (1.0f - b2) * gi * gi;
    m1[i] = a;
    m2[i] = b;
    theta[i] -= lr * (a / c1) / (sqrtf(b / c2) + eps);
}

// BF16 copies of the weights in the layouts the products read (zero padding where K or N is padded).
__global__ void cast_weights_kernel(const float* __restrict__ th, bf16* __restrict__ w1p, bf16* __restrict__ w2,
                                    bf16* __restrict__ w2t, bf16* __restrict__ w3p, bf16* __restrict__ w3tp) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < NH * NINP) {  // W1p [128][64]
        const int r = i / NINP, c = i - r * NINP;
        w1p[i] = __float2bfloat16_rn(c < NIN ? th[OFF_W1 + r * NIN + c] : 0.0f);
    }
    if (i < NH * NH) {  // W2 [128][128], W2^T
        const int r = i / NH, c = i - r * NH;
        const bf16 v = __float2bfloat16_rn(th[OFF_W2 + i]);
        w2[i] = v;
        w2t[c * NH + r] = v;
    }
    if (i < NOUTP * NH) {  // W3p [16][128]
        const int o = i / NH, h = i - o * NH;
        w3p[i] = __float2bfloat16_rn(o < NOUT ? th[OFF_W3 + o * NH + h] : 0.0f);
    }
    if (i < NH * NINP) {  // W3^T p [128][64]: [h][o]
        const int h = i / NINP, o = i - h * NINP;
        w3tp[i] = __float2bfloat16_rn(o < NOUT ? th[OFF_W3 + o * NH + h] : 0.0f);
    }
}

}  // namespace

// =============================================================================================
// Host side
// =============================================================================================
struct tvlbm_mlp {
    int device, max_rows;
    cudaStream_t stream;
    unsigned char* mem;
    size_t bytes;
    float *theta, *m1, *m2, *grad, *part;
    double* loss;
    int* status;
    bf16 *w1p, *w2, *w2t, *w3p, *w3tp;
    bf16 *h1, *h1t, *g1, *h2, *h2t, *g2, *dy, *dyt, *dz2, *dz2t, *dz1t, *xt;
    float* ybuf;
    int adam_t;
    unsigned long long uid;
    // descriptors of the last inference call (inputs at cached_x, cached_rows rows)
    const void* cached_x;
    int cached_rows;
    alignas(64) CUtensorMap fwd_maps[4];
    char err[256];
};

namespace {

int mfail(tvlbm_mlp* m, int code, const char* fmt, ...) {
    if (m) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(m->err, sizeof(m->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define MLP_CUDA(m, call, what)                                                                        \
    do {                                                                                               \
        cudaError_t e_ = (call);                                                                       \
        if (e_ != cudaSuccess) return mfail(m, TVLBM_ECUDA, "%s: %s", what, cudaGetErrorString(e_)); \
    } while (0)

// 2-D BF16 tensor map over a row-major [rows][k_total] matrix with row length ld (elements),
// box 64 x box_rows, 128-byte swizzle.
bool bf16_map(CUtensorMap* map, const void* base, int k_total, int rows, int ld, int box_rows) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = host::tensor_map_encoder();
    if (!enc || ((uintptr_t)base & 15) || (ld * 2) % 16) return false;
    cuuint64_t dims[2] = {(cuuint64_t)k_total, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
    cuuint32_t box[2] = {(cuuint32_t)BK, (cuuint32_t)box_rows};
    cuuint32_t es[2] = {1, 1};
    return enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int BN, int STAGES, class Epi>
cudaError_t gemm(const CUtensorMap& ma, const CUtensorMap& mb, int row_tiles, int kchunks, int splits, int cps,
                 const Epi& epi, int* status, cudaStream_t s) {
    using Cfg = GemmCfg<BN, STAGES>;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    if (!attr_set[dev]) {
        const cudaError_t e = cudaFuncSetAttribute(gemm_kernel<BN, STAGES, Epi>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, Cfg::SMEM);
        if (e != cudaSuccess) return e;
        attr_set[dev] = true;
    }
    gemm_kernel<BN, STAGES, Epi><<<dim3(row_tiles, splits), 128, Cfg::SMEM, s>>>(ma, mb, kchunks, cps, epi, status);
    return cudaGetLastError();
}

// Split of kchunks K chunks over at most kMaxSplits CTAs (every split non-empty).
void split_k(int kchunks, int* splits, int* cps) {
    int s = kchunks < kMaxSplits ? kchunks : kMaxSplits;
    *cps = (kchunks + s - 1) / s;
    *splits = (kchunks + *cps - 1) / *cps;
}

int check_rows(tvlbm_mlp* m, int rows) {
    if (rows <= 0 || rows % BM || rows > m->max_rows)
        return mfail(m, TVLBM_EINVAL, "rows %d must be a positive multiple of 128 and at most %d", rows, m->max_rows);
    return TVLBM_OK;
}

int read_status(tvlbm_mlp* m) {
    int st = 0;
    MLP_CUDA(m, cudaMemcpyAsync(&st, m->status, sizeof(int), cudaMemcpyDeviceToHost, m->stream), "status copy");
    MLP_CUDA(m, cudaStreamSynchronize(m->stream), "synchronize");
    if (st) {
        cudaMemsetAsync(m->status, 0, sizeof(int), m->stream);
        cudaStreamSynchronize(m->stream);
        return mfail(m, TVLBM_ETIMEOUT, "a device-side wait of the network kernels timed out");
    }
    return TVLBM_OK;
}

int refresh_weights(tvlbm_mlp* m) {
    cast_weights_kernel<<<(NH * NH + 255) / 256, 256, 0, m->stream>>>(m->theta, m->w1p, m->w2, m->w2t, m->w3p, m->w3tp);
    MLP_CUDA(m, cudaGetLastError(), "cast kernel");
    return TVLBM_OK;
}

}  // namespace

namespace tvlbm {
// Forward pass into y [rows][16] (FP32).  Used by tvlbm_mlp_forward and the closure step.
int mlp_forward_async(tvlbm_mlp* m, const void* x, int rows, float* y) {
    int rc = check_rows(m, rows);
    if (rc) return rc;
    // the weight descriptors never change; the input's are kept for repeated calls on one buffer
    if (m->cached_x != x || m->cached_rows != rows) {
        if (!bf16_map(&m->fwd_maps[0], x, NINP, rows, NINP, BM) ||
            !bf16_map(&m->fwd_maps[1], m->w1p, NINP, NH, NINP, NH) ||
            !bf16_map(&m->fwd_maps[2], m->w2, NH, NH, NH, NH) || !bf16_map(&m->fwd_maps[3], m->w3p, NH, NOUTP, NH, NOUTP)) {
            m->cached_x = nullptr;
            return mfail(m, TVLBM_EINVAL, "TMA descriptor rejected (alignment of x?)");
        }
        m->cached_x = x;
        m->cached_rows = rows;
    }
    const CUtensorMap &mx = m->fwd_maps[0], &mw1 = m->fwd_maps[1], &mw2 = m->fwd_maps[2], &mw3 = m->fwd_maps[3];
    const int tiles = rows / BM;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        MLP_CUDA(m, cudaFuncSetAttribute(mlp_fused_forward_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         FusedCfg::SMEM),
                 "fused forward attribute");
        attr_set[dev] = true;
    }
    MlpFeatures none;
    memset(&none, 0, sizeof(none));
    mlp_fused_forward_kernel<false><<<tiles, kFusedThreads, FusedCfg::SMEM, m->stream>>>(mx, mw1, mw2, mw3, m->theta, y,
                                                                                        m->status, none);
    MLP_CUDA(m, cudaGetLastError(), "fused forward");
    return TVLBM_OK;
}

int mlp_forward_features_async(tvlbm_mlp* m, const MlpFeatures& feat, int rows, float* y) {
    int rc = check_rows(m, rows);
    if (rc) return rc;
    if (!feat.m6 || feat.nx < 1 || feat.ny < 1 || (long long)feat.nx * feat.ny != rows)
        return mfail(m, TVLBM_EINVAL, "feature source does not match the rows");
    // the weight descriptors (the input one is passed along unused)
    CUtensorMap mx, mw1, mw2, mw3;
    memset(&mx, 0, sizeof(mx));
    if (!bf16_map(&mw1, m->w1p, NINP, NH, NINP, NH) || !bf16_map(&mw2, m->w2, NH, NH, NH, NH) ||
        !bf16_map(&mw3, m->w3p, NH, NOUTP, NH, NOUTP))
        return mfail(m, TVLBM_EINVAL, "TMA descriptor rejected");
    const int tiles = rows / BM;
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && !attr_set[dev]) {
        MLP_CUDA(m, cudaFuncSetAttribute(mlp_fused_forward_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         FusedCfg::SMEM),
                 "fused forward attribute");
        attr_set[dev] = true;
    }
    mlp_fused_forward_kernel<true><<<tiles, kFusedThreads, FusedCfg::SMEM, m->stream>>>(mx, mw1, mw2, mw3, m->theta, y,
                                                                                       m->status, feat);
    MLP_CUDA(m, cudaGetLastError(), "fused forward with features");
    return TVLBM_OK;
}
int mlp_max_rows(const tvlbm_mlp* m) { return m->max_rows; }
float* mlp_ybuf(tvlbm_mlp* m) { return m->ybuf; }
int mlp_set_stream(tvlbm_mlp* m, cudaStream_t s) {
    m->stream = s;
    return TVLBM_OK;
}
int mlp_status(tvlbm_mlp* m) { return read_status(m); }
unsigned long long mlp_uid(const tvlbm_mlp* m) { return m->uid; }
cudaStream_t mlp_stream(const tvlbm_mlp* m) { return m->stream; }
}  // namespace tvlbm

extern "C" {

int tvlbm_mlp_create(int max_rows, tvlbm_mlp** out) {
    if (!out) return TVLBM_EINVAL;
    *out = nullptr;
    if (max_rows <= 0 || max_rows % BM || max_rows > (1 << 26)) return TVLBM_EINVAL;
    tvlbm_mlp* m = new (std::nothrow) tvlbm_mlp();
    if (!m) return TVLBM_ENOMEM;
    memset(m, 0, sizeof(*m));
    cudaGetDevice(&m->device);
    m->max_rows = max_rows;
    static std::atomic<unsigned long long> next_uid{1};
    m->uid = next_uid.fetch_add(1);
    const size_t R = (size_t)max_rows;
    int splits = 0, cps = 0;
    split_k(max_rows / BK, &splits, &cps);
    // carve one allocation: FP32 block, then BF16 block (every piece 256-byte aligned)
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off = host::align_up(off + bytes, 256);
        return o;
    };
    const size_t o_theta = take(NPARAM * 4), o_m1 = take(NPARAM * 4), o_m2 = take(NPARAM * 4), o_grad = take(NPARAM * 4);
    const size_t o_part = take((size_t)kMaxSplits * BM * NH * 4), o_loss = take(8), o_status = take(4);
    const size_t o_y = take(R * NOUTP * 4);
    const size_t o_w1p = take(NH * NINP * 2), o_w2 = take(NH * NH * 2), o_w2t = take(NH * NH * 2),
                 o_w3p = take(NOUTP * NH * 2), o_w3tp = take(NH * NINP * 2);
    const size_t o_h1 = take(R * NH * 2), o_h1t = take(R * NH * 2), o_g1 = take(R * NH * 2), o_h2 = take(R * NH * 2),
                 o_h2t = take(R * NH * 2), o_g2 = take(R * NH * 2), o_dy = take(R * NINP * 2),
                 o_dyt = take(R * NOUTP * 2), o_dz2 = take(R * NH * 2), o_dz2t = take(R * NH * 2),
                 o_dz1t = take(R * NH * 2), o_xt = take(R * NINP * 2);
    m->bytes = off;
    if (cudaMalloc((void**)&m->mem, off) != cudaSuccess) {
        delete m;
        return TVLBM_ENOMEM;
    }
    unsigned char* b = m->mem;
    m->theta = (float*)(b + o_theta);
    m->m1 = (float*)(b + o_m1);
    m->m2 = (float*)(b + o_m2);
    m->grad = (float*)(b + o_grad);
    m->part = (float*)(b + o_part);
    m->loss = (double*)(b + o_loss);
    m->status = (int*)(b + o_status);
    m->ybuf = (float*)(b + o_y);
    m->w1p = (bf16*)(b + o_w1p);
    m->w2 = (bf16*)(b + o_w2);
    m->w2t = (bf16*)(b + o_w2t);
    m->w3p = (bf16*)(b + o_w3p);
    m->w3tp = (bf16*)(b + o_w3tp);
    m->h1 = (bf16*)(b + o_h1);
    m->h1t = (bf16*)(b + o_h1t);
    m->g1 = (bf16*)(b + o_g1);
    m->h2 = (bf16*)(b + o_h2);
    m->h2t = (bf16*)(b + o_h2t);
    m->g2 = (bf16*)(b + o_g2);
    m->dy = (bf16*)(b + o_dy);
    m->dyt = (bf16*)(b + o_dyt);
    m->dz2 = (bf16*)(b + o_dz2);
    m->dz2t = (bf16*)(b + o_dz2t);
    m->dz1t = (bf16*)(b + o_dz1t);
    m->xt = (bf16*)(b + o_xt);
    // zero everything once: parameters, moments, and the padded columns of dY (never written)
    if (cudaMemset(m->mem, 0, off) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
        cudaFree(m->mem);
        delete m;
        return TVLBM_ECUDA;
    }
    (void)splits;
    (void)cps;
    *out = m;
    return TVLBM_OK;
}

int tvlbm_mlp_destroy(tvlbm_mlp* m) {
    if (!m) return TVLBM_OK;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    cudaFree(m->mem);
    delete m;
    return TVLBM_OK;
}

int tvlbm_mlp_set_stream(tvlbm_mlp* m, void* stream) {
    if (!m) return TVLBM_EINVAL;
    m->stream = (cudaStream_t)stream;
    return TVLBM_OK;
}

int tvlbm_mlp_set_params(tvlbm_mlp* m, const float* params) {
    if (!m || !params) return TVLBM_EINVAL;
    for (int i = 0; i < NPARAM; ++i)
        if (!isfinite(params[i])) return mfail(m, TVLBM_EINVAL, "parameter %d is not finite", i);
    cudaSetDevice(m->device);
    MLP_CUDA(m, cudaMemcpyAsync(m->theta, params, NPARAM * 4, cudaMemcpyHostToDevice, m->stream), "copy params");
    MLP_CUDA(m, cudaMemsetAsync(m->m1, 0, NPARAM * 4, m->stream), "clear moments");
    MLP_CUDA(m, cudaMemsetAsync(m->m2, 0, NPARAM * 4, m->stream), "clear moments");
    m->adam_t = 0;
    const int rc = refresh_weights(m);
    if (rc) return rc;
    MLP_CUDA(m, cudaStreamSynchronize(m->stream), "synchronize");
    return TVLBM_OK;
}

int tvlbm_mlp_get_params(tvlbm_mlp* m, float* params) {
    if (!m || !params) return TVLBM_EINVAL;
    cudaSetDevice(m->device);
    MLP_CUDA(m, cudaMemcpyAsync(params, m->theta, NPARAM * 4, cudaMemcpyDeviceToHost, m->stream), "copy params");
    MLP_CUDA(m, cudaStreamSynchronize(m->stream), "synchronize");
    return TVLBM_OK;
}

int tvlbm_mlp_forward(tvlbm_mlp* m, const void* x, int rows, float* y) {
    if (!m || !x || !y) return TVLBM_EINVAL;
    cudaSetDevice(m->device);
    return mlp_forward_async(m, x, rows, y);
}

int tvlbm_mlp_loss_grad(tvlbm_mlp* m, const void* x, const float* ystar, int rows, double* loss, float* grad) {
    if (!m || !x || !ystar) return TVLBM_EINVAL;
    int rc = check_rows(m, rows);
    if (rc) return rc;
    cudaSetDevice(m->device);
    cudaStream_t s = m->stream;
    const int tiles = rows / BM;
    CUtensorMap mx, mw1, mh1, mw2, mh2, mw3, mdy, mw3t, mdz2, mw2t, mdz1t, mxt, mdz2t, mh1t, mh2t, mdyt;
    const bool okmaps =
        bf16_map(&mx, x, NINP, rows, NINP, BM) && bf16_map(&mw1, m->w1p, NINP, NH, NINP, NH) &&
        bf16_map(&mh1, m->h1, NH, rows, NH, BM) && bf16_map(&mw2, m->w2, NH, NH, NH, NH) &&
        bf16_map(&mh2, m->h2, NH, rows, NH, BM) && bf16_map(&mw3, m->w3p, NH, NOUTP, NH, NOUTP) &&
        bf16_map(&mdy, m->dy, NINP, rows, NINP, BM) && bf16_map(&mw3t, m->w3tp, NINP, NH, NINP, NH) &&
        bf16_map(&mdz2, m->dz2, NH, rows, NH, BM) && bf16_map(&mw2t, m->w2t, NH, NH, NH, NH) &&
        bf16_map(&mdz1t, m->dz1t, rows, NH, rows, BM) && bf16_map(&mxt, m->xt, rows, NINP, rows, NINP) &&
        bf16_map(&mdz2t, m->dz2t, rows, NH, rows, BM) && bf16_map(&mh1t, m->h1t, rows, NH, rows, NH) &&
        bf16_map(&mh2t, m->h2t, rows, NH, rows, BM) && bf16_map(&mdyt, m->dyt, rows, NOUTP, rows, NOUTP);
    if (!okmaps) return mfail(m, TVLBM_EINVAL, "TMA descriptor rejected (alignment of x?)");
    MLP_CUDA(m, cudaMemsetAsync(m->grad, 0, NPARAM * 4, s), "clear gradient");
    MLP_CUDA(m, cudaMemsetAsync(m->loss, 0, 8, s), "clear loss");
    transpose_x_kernel<<<dim3(rows / 32, NINP / 32), dim3(32, 8), 0, s>>>((const bf16*)x, m->xt, rows);
    MLP_CUDA(m, cudaGetLastError(), "transpose");
    // forward, keeping H, H^T and g'(Z)
    EpiHidden e1{m->theta + OFF_B1, m->h1, m->h1t, m->g1, rows};
    MLP_CUDA(m, (gemm<NH, 2>(mx, mw1, tiles, NINP / BK, 1, NINP / BK, e1, m->status, s)), "layer 1");
    EpiHidden e2{m->theta + OFF_B2, m->h2, m->h2t, m->g2, rows};
    MLP_CUDA(m, (gemm<NH, 2>(mh1, mw2, tiles, NH / BK, 1, NH / BK, e2, m->status, s)), "layer 2");
    EpiOut e3{m->theta + OFF_B3, m->ybuf, ystar, m->dy, m->dyt, m->loss, m->grad + OFF_B3,
              2.0f / ((float)rows * (float)NOUT), rows};
    MLP_CUDA(m, (gemm<NOUTP, 2>(mh2, mw3, tiles, NH / BK, 1, NH / BK, e3, m->status, s)), "layer 3");
    // back through the layers
    EpiBack b2{m->g2, m->dz2, m->dz2t, m->grad + OFF_B2, rows};
    MLP_CUDA(m, (gemm<NH, 2>(mdy, mw3t, tiles, NINP / BK, 1, NINP / BK, b2, m->status, s)), "dH2");
    EpiBack b1{m->g1, nullptr, m->dz1t, m->grad + OFF_B1, rows};
    MLP_CUDA(m, (gemm<NH, 2>(mdz2, mw2t, tiles, NH / BK, 1, NH / BK, b1, m->status, s)), "dH1");
    // weight gradients: K = rows, split over CTAs, partials reduced in a fixed order
    int splits = 0, cps = 0;
    split_k(rows / BK, &splits, &cps);
    EpiPartial p1{m->part, NINP};
    MLP_CUDA(m, (gemm<NINP, 4>(mdz1t, mxt, 1, rows / BK, splits, cps, p1, m->status, s)), "dW1");
    reduce_partials_kernel<<<(BM * NINP + 255) / 256, 256, 0, s>>>(m->part, splits, NINP, NINP, m->grad, 0);
    MLP_CUDA(m, cudaGetLastError(), "reduce dW1");
    EpiPartial p2{m->part, NH};
    MLP_CUDA(m, (gemm<NH, 4>(mdz2t, mh1t, 1, rows / BK, splits, cps, p2, m->status, s)), "dW2");
    reduce_partials_kernel<<<(BM * NH + 255) / 256, 256, 0, s>>>(m->part, splits, NH, NH, m->grad, 1);
    MLP_CUDA(m, cudaGetLastError(), "reduce dW2");
    EpiPartial p3{m->part, NOUTP};
    MLP_CUDA(m, (gemm<NOUTP, 4>(mh2t, mdyt, 1, rows / BK, splits, cps, p3, m->status, s)), "dW3");
    reduce_partials_kernel<<<(BM * NOUTP + 255) / 256, 256, 0, s>>>(m->part, splits, NOUTP, NOUTP, m->grad, 2);
    MLP_CUDA(m, cudaGetLastError(), "reduce dW3");
    if (loss || grad) {
        double l = 0.0;
        if (loss) MLP_CUDA(m, cudaMemcpyAsync(&l, m->loss, 8, cudaMemcpyDeviceToHost, s), "copy loss");
        if (grad) MLP_CUDA(m, cudaMemcpyAsync(grad, m->grad, NPARAM * 4, cudaMemcpyDeviceToHost, s), "copy grad");
        rc = read_status(m);
        if (rc) return rc;
        if (loss) *loss = l / ((double)rows * NOUT);
    }
    return TVLBM_OK;
}

int tvlbm_mlp_adam(tvlbm_mlp* m, float lr, float beta1, float beta2, float eps) {
    if (!m || !(lr >= 0.0f) || !(beta1 >= 0.0f && beta1 < 1.0f) || !(beta2 >= 0.0f && beta2 < 1.0f) || !(eps > 0.0f))
        return mfail(m, TVLBM_EINVAL, "Adam needs lr >= 0, 0 <= beta < 1, eps > 0");
    cudaSetDevice(m->device);
    m->adam_t += 1;
    const float c1 = 1.0f - powf(beta1, (float)m->adam_t), c2 = 1.0f - powf(beta2, (float)m->adam_t);
    adam_kernel<<<(NPARAM + 255) / 256, 256, 0, m->stream>>>(m->theta, m->m1, m->m2, m->grad, NPARAM, lr, beta1, beta2,
                                                             eps, c1, c2);
    MLP_CUDA(m, cudaGetLastError(), "adam kernel");
    return refresh_weights(m);
}

const char* tvlbm_mlp_last_error(const tvlbm_mlp* m) { return m ? m->err : "null network"; }

}  // extern "C"

extern "C" int tvlbm_mlp_activation(const float* z, float* g, float* dg, int n, void* stream) {
    if (!z || n < 0) return TVLBM_EINVAL;
    if (n == 0) return TVLBM_OK;
    const int blocks = (n + 255) / 256 < 1024 ? (n + 255) / 256 : 1024;
    activation_kernel<<<blocks, 256, 0, (cudaStream_t)stream>>>(z, g, dg, n);
    return cudaGetLastError() == cudaSuccess ? TVLBM_OK : TVLBM_ECUDA;
}
