// Learned coarse-grid closure on a context (include/tvlbm_closure.h): per-cell features and the
// network's inputs, projection of a state difference on the non-conserved Hermite basis, block
// averaging from a finer context, and the coarse step whose collision is followed by the
// network's correction  Delta f_l = w_l sum_k o_k psi_k(c_l)  (no mass, momentum or energy).
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "tvlbm.h"
#include "tvlbm_closure.h"
#include "tvlbm_collide.cuh"
#include "tvlbm_ctx.h"
#include "tvlbm_kernels.cuh"
#include "tvlbm_mlp.h"
#include "tvlbm_tiled.cuh"

using namespace tvlbm;

namespace {

constexpr int N1 = 4, Q = 16, NK = TVLBM_MLP_OUT, NF = 6;

struct BasisF {
    float psi[NK][Q];
};
struct BasisD {
    double psi[NK][Q];
};
struct Norm {
    float mu[NF], isg[NF];
};
struct Scale {
    float s[NK];
};

// psi_k(c_l) from the context's nodes: He_a(x_i) He_b(x_j) / sqrt(a! b!), order of the header.
void make_basis(const host::Rule& r, BasisD* bd, BasisF* bf) {
    static const int ab[NK][2] = {{-1, -1}, {1, 1}, {3, 0}, {2, 1}, {1, 2}, {0, 3},
                                  {3, 1}, {2, 2}, {1, 3}, {3, 2}, {2, 3}, {3, 3}};
    auto he = [](int n, double x) {
        double a = 1.0, b = x;
        if (n == 0) return 1.0;
        for (int k = 1; k < n; ++k) {
            const double c = x * b - k * a;
            a = b;
            b = c;
        }
        return b;
    };
    const double fact[4] = {1.0, 1.0, 2.0, 6.0};
    for (int k = 0; k < NK; ++k)
        for (int j = 0; j < N1; ++j)
            for (int i = 0; i < N1; ++i) {
                const double x = r.x[i], y = r.x[j];
                double v;
                if (ab[k][0] < 0) v = 0.5 * (he(2, x) - he(2, y));
                else v = he(ab[k][0], x) * he(ab[k][1], y) / sqrt(fact[ab[k][0]] * fact[ab[k][1]]);
                bd->psi[k][i + N1 * j] = v;
                bf->psi[k][i + N1 * j] = (float)v;
            }
}

// Storage index of population l of fluid cell (x, y).
__device__ __forceinline__ long long cell_index(const KParams& p, int l, int x, int y) {
    return (long long)l * p.plane + (long long)(y + HY) * p.pitch + (x + p.hx);
}

// f_l of cell (x, y) in FP64 (default deviation reference: f = w (rho0 + d)).
template <class C>
__device__ __forceinline__ void load_f(const typename C::T* f, const KParams& p, int x, int y, double (&out)[Q]) {
#pragma unroll
    for (int j = 0; j < N1; ++j)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const int l = i + N1 * j;
            out[l] = to_f<C, double>((double)C::ld(f + cell_index(p, l, x, y)), p.wd[i] * p.wd[j], p.rho0d);
        }
}

// The six moments of one cell from its stored values v[l] (storage space), in arithmetic M:
// m6[q][c] for q = rho, u_x, u_y, T, Pi_xy, Pi_xx - Pi_yy (non-equilibrium parts of the last two).
template <class C, class M>
__device__ __forceinline__ void cell_m6(const typename C::R (&sv)[Q], const KParams& p, float* __restrict__ m6, int x,
                                        int y) {
    M rho = 0, jx = 0, jy = 0, e2 = 0, sxy = 0, sd = 0;
#pragma unroll
    for (int j = 0; j < N1; ++j)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const int l = i + N1 * j;
            const M v = to_f<C, M>((M)sv[l], kw<M>(p, i) * kw<M>(p, j), krho0<M>(p));
            const M cx = kx<M>(p, i), cy = kx<M>(p, j);
            rho += v;
            jx += v * cx;
            jy += v * cy;
            e2 += v * (cx * cx + cy * cy);
            sxy += v * cx * cy;
            sd += v * (cx * cx - cy * cy);
        }
    const M ux = jx / rho, uy = jy / rho;
    const M T = M(0.5) * (e2 / rho - (ux * ux + uy * uy));
    const long long c = (long long)y * p.nx + x, n = (long long)p.nx * p.ny;
    m6[c] = (float)rho;
    m6[n + c] = (float)ux;
    m6[2 * n + c] = (float)uy;
    m6[3 * n + c] = (float)T;
    m6[4 * n + c] = (float)(sxy - rho * ux * uy);
    m6[5 * n + c] = (float)(sd - rho * (ux * ux - uy * uy));
}

// M: the arithmetic (double for the training-side entry points, float on the learned step,
// whose features are rounded to BF16 after normalisation anyway).
template <class C, class M = double>
__global__ void closure_moments_kernel(const typename C::T* __restrict__ f, float* __restrict__ m6, const KParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    typename C::R sv[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) sv[l] = C::ld(f + cell_index(p, l, x, y));
    cell_m6<C, M>(sv, p, m6, x, y);
}

// Row y*nx + x of x_out: the normalised features of the 3 x 3 periodic neighbourhood.
__global__ void closure_features_kernel(const float* __restrict__ m6, int nx, int ny, const Norm nrm,
                                        __nv_bfloat16* __restrict__ xo) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= nx || y >= ny) return;
    const long long n = (long long)nx * ny;
    alignas(16) __nv_bfloat16 row[TVLBM_MLP_IN_PAD];
#pragma unroll
    for (int dy = -1; dy <= 1; ++dy) {
        const int yy = (y + dy + ny) % ny;
#pragma unroll
        for (int dx = -1; dx <= 1; ++dx) {
            const int xx = (x + dx + nx) % nx;
            const int k = (dy + 1) * 3 + (dx + 1);
            const long long c = (long long)yy * nx + xx;
#pragma unroll
            for (int q = 0; q < NF; ++q) row[k * NF + q] = __float2bfloat16_rn((m6[q * n + c] - nrm.mu[q]) * nrm.isg[q]);
        }
    }
#pragma unroll
    for (int k = TVLBM_MLP_IN; k < TVLBM_MLP_IN_PAD; ++k) row[k] = __float2bfloat16_rn(0.0f);
    uint4* d = reinterpret_cast<uint4*>(xo + ((long long)y * nx + x) * TVLBM_MLP_IN_PAD);
#pragma unroll
    for (int q = 0; q < TVLBM_MLP_IN_PAD / 8; ++q) d[q] = reinterpret_cast<const uint4*>(row)[q];
}

template <class C>
__global__ void closure_project_kernel(const typename C::T* __restrict__ fa, const typename C::T* __restrict__ fb,
                                       float* __restrict__ o, const KParams p, const BasisD b, const Scale isc) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    double va[Q], vb[Q];
    load_f<C>(fa, p, x, y, va);
    load_f<C>(fb, p, x, y, vb);
    float* d = o + ((long long)y * p.nx + x) * TVLBM_MLP_OUT_PAD;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l < Q; ++l) acc += (va[l] - vb[l]) * b.psi[k][l];
        d[k] = (float)(acc * (double)isc.s[k]);
    }
#pragma unroll
    for (int k = NK; k < TVLBM_MLP_OUT_PAD; ++k) d[k] = 0.0f;
}

// Non-equilibrium coefficients of a state: n_k = inv_scale_k sum_l (f - f_eq(rho, u, T))_l psi_k(c_l),
// the equilibrium taken at the cell's own moments, all in FP64.
template <class C>
__global__ void closure_noneq_kernel(const typename C::T* __restrict__ f, float* __restrict__ o, const KParams p,
                                     const BasisD b, const Scale isc) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    double v[Q];
    load_f<C>(f, p, x, y, v);
    double rho = 0, jx = 0, jy = 0, e2 = 0;
#pragma unroll
    for (int j = 0; j < N1; ++j)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const double fl = v[i + N1 * j], cx = p.xd[i], cy = p.xd[j];
            rho += fl;
            jx += fl * cx;
            jy += fl * cy;
            e2 += fl * (cx * cx + cy * cy);
        }
    const double ux = jx / rho, uy = jy / rho;
    const double th = 0.5 * (e2 / rho - (ux * ux + uy * uy)) - 1.0;
    double eq[Q];
    cell_equilibrium<N1, false, double>(p, rho, ux, uy, th, eq);
    float* d = o + ((long long)y * p.nx + x) * TVLBM_MLP_OUT_PAD;
#pragma unroll
    for (int k = 0; k < NK; ++k) {
        double acc = 0.0;
#pragma unroll
        for (int l = 0; l < Q; ++l) acc += (v[l] - eq[l]) * b.psi[k][l];
        d[k] = (float)(acc * (double)isc.s[k]);
    }
#pragma unroll
    for (int k = NK; k < TVLBM_MLP_OUT_PAD; ++k) d[k] = 0.0f;
}

// Coarse cell (X, Y) = mean of the m x m fine cells it covers, in FP64, encoded for the coarse
// storage and stored with its periodic images.
template <int NN, class CF, class CC>
__global__ void downsample_kernel(const typename CF::T* __restrict__ ff, const KParams pf, typename CC::T* __restrict__ fc,
                                  const KParams pc, int m) {
    constexpr int QQ = NN * NN;
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y * blockDim.y + threadIdx.y;
    if (X >= pc.nx || Y >= pc.ny) return;
    typename CC::R s[QQ];
    const double inv = 1.0 / ((double)m * m);
#pragma unroll
    for (int j = 0; j < NN; ++j)
#pragma unroll
        for (int i = 0; i < NN; ++i) {
            const int l = i + NN * j;
            const double w = pf.wd[i] * pf.wd[j];
            double acc = 0.0;
            for (int b = 0; b < m; ++b)
                for (int a = 0; a < m; ++a)
                    acc += to_f<CF, double>((double)CF::ld(ff + cell_index(pf, l, X * m + a, Y * m + b)), w, pf.rho0d);
            s[l] = (typename CC::R)from_f<CC, double>(acc * inv, pc.wd[i] * pc.wd[j], pc.rho0d);
        }
    store_collided<NN, CC>(fc, geom_of(pc), X, Y, s);
}

// Streaming alone (the learned step's first half): pull-gather as the plain sweep, stored with
// the frame images, no collision; and the streamed cell's moments into m6 in arithmetic M, from
// the values just stored (so equal to closure_moments_kernel's on the stored state).
template <class C, class M>
__global__ void __launch_bounds__(256) closure_stream_kernel(const typename C::T* __restrict__ fin,
                                                             typename C::T* __restrict__ fout, const KParams p,
                                                             float* __restrict__ m6) {
    using R = typename C::R;
    using T = typename C::T;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    R s[Q];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        const R ay = ka<R>(p, j);
        const int ys = y + HY - p.sh[j];
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const R ax = ka<R>(p, i);
            const int xs = x + p.hx - p.sh[i];
            const T* q = fin + (long long)(i + N1 * j) * p.plane + (long long)ys * p.pitch + xs;
            const R v00 = C::ld(q), v01 = C::ld(q - 1);
            const R v10 = C::ld(q - p.pitch), v11 = C::ld(q - p.pitch - 1);
            const R r0 = fma(ax, v01 - v00, v00);
            const R r1 = fma(ax, v11 - v10, v10);
            s[i + N1 * j] = fma(ay, r1 - r0, r0);
        }
    }
    store_collided<N1, C>(fout, geom_of(p), x, y, s);
    cell_m6<C, M>(s, p, m6, x, y);
}

// The learned collision (second half), in place on the streamed state: every cell becomes
// f_eq(rho, u, T) + w sum_k o_k psi_k with the network's coefficients o_k = scale_k y[c][k]
// (the equilibrium as the BGK collision with dt / tau = 1 computes it, in the storage's
// arithmetic with its conservation corrections).  Each thread reads and writes its own cell
// (and that cell's frame images) only.
template <class C>
__global__ void __launch_bounds__(256) closure_collide_kernel(typename C::T* __restrict__ f, const KParams p,
                                                              const float* __restrict__ yk, const BasisF b,
                                                              const BasisD bd, const Scale sc) {
    using R = typename C::R;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    R s[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) s[l] = C::ld(f + cell_index(p, l, x, y));
    if constexpr (C::dev) cell_collide_dev<N1, false>(s, p, 1.0f, nullptr);
    else cell_collide<N1, false, R>(s, p, R(1));
    // the correction in the storage's arithmetic: a rounded basis table leaves a conserved-moment
    // residue of the order of its rounding, so FP64 storage uses the FP64 table
    const float* yc = yk + ((long long)y * p.nx + x) * TVLBM_MLP_OUT_PAD;
    R o[NK];
#pragma unroll
    for (int k = 0; k < NK; ++k) o[k] = (R)sc.s[k] * (R)yc[k];
#pragma unroll
    for (int l = 0; l < Q; ++l) {
        R d = 0;
#pragma unroll
        for (int k = 0; k < NK; ++k) {
            if constexpr (std::is_same<R, double>::value) d = fma(o[k], bd.psi[k][l], d);
            else d = fmaf(o[k], b.psi[k][l], d);
        }
        // deviation storage holds f / w - rho0: its correction is sum o psi; full f gets w times it
        if constexpr (C::dev) s[l] += d;
        else s[l] += (R)(p.wd[l % N1] * p.wd[l / N1]) * d;
    }
    store_collided<N1, C>(f, geom_of(p), x, y, s);
}

dim3 grid_of(int nx, int ny, dim3 b) { return dim3((nx + b.x - 1) / b.x, (ny + b.y - 1) / b.y); }

void* cur_buf(tvlbm_ctx* c) { return c->mem + c->L.off_f[c->cur]; }
void* other_buf(tvlbm_ctx* c) { return c->mem + c->L.off_f[1 - c->cur]; }

int ctx_fail(tvlbm_ctx* c, int code, const char* msg) {
    if (c) snprintf(c->err, sizeof(c->err), "%s", msg);
    return code;
}

// The closure's requirements on a context.
int closure_ctx_ok(tvlbm_ctx* c) {
    if (!c) return TVLBM_EINVAL;
    if (c->velset != TVLBM_D2Q16) return ctx_fail(c, TVLBM_EINVAL, "the closure is defined for D2Q16");
    if (c->kp.walls) return ctx_fail(c, TVLBM_EINVAL, "the closure needs a periodic domain");
    if (c->storage != TVLBM_FP64 && c->storage != TVLBM_FP32 && c->storage != TVLBM_FP32_DEV)
        return ctx_fail(c, TVLBM_EINVAL, "the closure supports FP64, FP32 and FP32-deviation storage");
    if (c->kp.has_ref) return ctx_fail(c, TVLBM_EINVAL, "the closure needs the default deviation reference");
    return TVLBM_OK;
}

#define CL_CUDA(ctx, call, what)                                      \
    do {                                                              \
        cudaError_t e_ = (call);                                      \
        if (e_ != cudaSuccess) return ctx_fail(ctx, TVLBM_ECUDA, what); \
    } while (0)

cudaError_t launch_moments(tvlbm_ctx* c, float* m6) {
    const dim3 b(32, 8), g = grid_of(c->nx, c->ny, b);
    switch (c->storage) {
        case TVLBM_FP64: closure_moments_kernel<CodecF64><<<g, b, 0, c->stream>>>((const double*)cur_buf(c), m6, c->kp); break;
        case TVLBM_FP32: closure_moments_kernel<CodecF32><<<g, b, 0, c->stream>>>((const float*)cur_buf(c), m6, c->kp); break;
        default: closure_moments_kernel<CodecF32Dev><<<g, b, 0, c->stream>>>((const float*)cur_buf(c), m6, c->kp); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_features(tvlbm_ctx* c, const float* m6, const Norm& nrm, void* x) {
    const dim3 b(32, 8), g = grid_of(c->nx, c->ny, b);
    closure_features_kernel<<<g, b, 0, c->stream>>>(m6, c->nx, c->ny, nrm, (__nv_bfloat16*)x);
    return cudaGetLastError();
}

int make_norm(const float* mu, const float* inv_sigma, Norm* n) {
    if (!mu || !inv_sigma) return TVLBM_EINVAL;
    for (int q = 0; q < NF; ++q) {
        if (!isfinite(mu[q]) || !isfinite(inv_sigma[q])) return TVLBM_EINVAL;
        n->mu[q] = mu[q];
        n->isg[q] = inv_sigma[q];
    }
    return TVLBM_OK;
}

template <class CF>
cudaError_t downsample_from(int coarse_storage, const void* ff, const KParams& pf, void* fc, const KParams& pc, int m,
                            cudaStream_t s) {
    const dim3 b(16, 8), g = grid_of(pc.nx, pc.ny, b);
    switch (coarse_storage) {
        case TVLBM_FP64: downsample_kernel<N1, CF, CodecF64><<<g, b, 0, s>>>((const typename CF::T*)ff, pf, (double*)fc, pc, m); break;
        case TVLBM_FP32: downsample_kernel<N1, CF, CodecF32><<<g, b, 0, s>>>((const typename CF::T*)ff, pf, (float*)fc, pc, m); break;
        default: downsample_kernel<N1, CF, CodecF32Dev><<<g, b, 0, s>>>((const typename CF::T*)ff, pf, (float*)fc, pc, m); break;
    }
    return cudaGetLastError();
}

}  // namespace

extern "C" {

int tvlbm_closure_moments(tvlbm_ctx* c, float* m6) {
    int rc = closure_ctx_ok(c);
    if (rc) return rc;
    if (!m6) return ctx_fail(c, TVLBM_EINVAL, "null output");
    cudaSetDevice(c->device);
    CL_CUDA(c, launch_moments(c, m6), "closure moments kernel");
    return TVLBM_OK;
}

int tvlbm_closure_features(tvlbm_ctx* c, const float* mu, const float* inv_sigma, void* x) {
    int rc = closure_ctx_ok(c);
    if (rc) return rc;
    Norm nrm;
    if (!x || make_norm(mu, inv_sigma, &nrm)) return ctx_fail(c, TVLBM_EINVAL, "null or non-finite argument");
    if ((uintptr_t)x & 15) return ctx_fail(c, TVLBM_EINVAL, "x must be 16-byte aligned");
    cudaSetDevice(c->device);
    float* m6 = (float*)(c->mem + c->L.off_mom);  // 4 doubles per cell of scratch hold 6 floats
    CL_CUDA(c, launch_moments(c, m6), "closure moments kernel");
    CL_CUDA(c, launch_features(c, m6, nrm, x), "closure features kernel");
    return TVLBM_OK;
}

int tvlbm_closure_project(tvlbm_ctx* a, tvlbm_ctx* b, const float* inv_scale, float* o) {
    int rc = closure_ctx_ok(a);
    if (rc) return rc;
    rc = closure_ctx_ok(b);
    if (rc) return rc;
    if (!o || a->nx != b->nx || a->ny != b->ny || a->storage != b->storage || a->device != b->device)
        return ctx_fail(a, TVLBM_EINVAL, "contexts differ in grid, storage or device");
    cudaSetDevice(a->device);
    Scale isc;
    for (int k = 0; k < NK; ++k) {
        isc.s[k] = inv_scale ? inv_scale[k] : 1.0f;
        if (!isfinite(isc.s[k])) return ctx_fail(a, TVLBM_EINVAL, "non-finite inverse scale");
    }
    BasisD bd;
    BasisF bf;
    make_basis(a->rule, &bd, &bf);
    // b's pending work must be complete before a's stream reads it
    if (b->stream != a->stream) CL_CUDA(a, cudaStreamSynchronize(b->stream), "synchronize");
    const dim3 blk(32, 8), g = grid_of(a->nx, a->ny, blk);
    switch (a->storage) {
        case TVLBM_FP64:
            closure_project_kernel<CodecF64><<<g, blk, 0, a->stream>>>((const double*)cur_buf(a), (const double*)cur_buf(b), o, a->kp, bd, isc);
            break;
        case TVLBM_FP32:
            closure_project_kernel<CodecF32><<<g, blk, 0, a->stream>>>((const float*)cur_buf(a), (const float*)cur_buf(b), o, a->kp, bd, isc);
            break;
        default:
            closure_project_kernel<CodecF32Dev><<<g, blk, 0, a->stream>>>((const float*)cur_buf(a), (const float*)cur_buf(b), o, a->kp, bd, isc);
            break;
    }
    CL_CUDA(a, cudaGetLastError(), "closure project kernel");
    return TVLBM_OK;
}

int tvlbm_closure_noneq(tvlbm_ctx* c, const float* inv_scale, float* o) {
    int rc = closure_ctx_ok(c);
    if (rc) return rc;
    if (!o) return ctx_fail(c, TVLBM_EINVAL, "null output");
    Scale isc;
    for (int k = 0; k < NK; ++k) {
        isc.s[k] = inv_scale ? inv_scale[k] : 1.0f;
        if (!isfinite(isc.s[k])) return ctx_fail(c, TVLBM_EINVAL, "non-finite inverse scale");
    }
    cudaSetDevice(c->device);
    BasisD bd;
    BasisF bf;
    make_basis(c->rule, &bd, &bf);
    const dim3 blk(32, 8), g = grid_of(c->nx, c->ny, blk);
    switch (c->storage) {
        case TVLBM_FP64: closure_noneq_kernel<CodecF64><<<g, blk, 0, c->stream>>>((const double*)cur_buf(c), o, c->kp, bd, isc); break;
        case TVLBM_FP32: closure_noneq_kernel<CodecF32><<<g, blk, 0, c->stream>>>((const float*)cur_buf(c), o, c->kp, bd, isc); break;
        default: closure_noneq_kernel<CodecF32Dev><<<g, blk, 0, c->stream>>>((const float*)cur_buf(c), o, c->kp, bd, isc); break;
    }
    CL_CUDA(c, cudaGetLastError(), "closure non-equilibrium kernel");
    return TVLBM_OK;
}

int tvlbm_downsample(tvlbm_ctx* fine, tvlbm_ctx* coarse) {
    if (!fine || !coarse) return TVLBM_EINVAL;
    if (fine->velset != TVLBM_D2Q16 || coarse->velset != TVLBM_D2Q16)
        return ctx_fail(coarse, TVLBM_EINVAL, "downsampling is provided for D2Q16");
    if (fine->kp.walls || coarse->kp.walls) return ctx_fail(coarse, TVLBM_EINVAL, "downsampling needs periodic domains");
    if (fine->kp.has_ref || coarse->kp.has_ref) return ctx_fail(coarse, TVLBM_EINVAL, "default deviation reference only");
    const int m = fine->nx / coarse->nx;
    if (m < 1 || coarse->nx * m != fine->nx || coarse->ny * m != fine->ny)
        return ctx_fail(coarse, TVLBM_EINVAL, "fine grid must be m x the coarse grid in both directions");
    if (fine->device != coarse->device) return ctx_fail(coarse, TVLBM_EINVAL, "contexts on different devices");
    auto ok_storage = [](int s) { return s == TVLBM_FP64 || s == TVLBM_FP32 || s == TVLBM_FP32_DEV; };
    if (!ok_storage(fine->storage) || !ok_storage(coarse->storage))
        return ctx_fail(coarse, TVLBM_EINVAL, "downsampling supports FP64, FP32 and FP32-deviation storage");
    cudaSetDevice(coarse->device);
    if (fine->stream != coarse->stream) CL_CUDA(coarse, cudaStreamSynchronize(fine->stream), "synchronize");
    cudaError_t e;
    switch (fine->storage) {
        case TVLBM_FP64: e = downsample_from<CodecF64>(coarse->storage, cur_buf(fine), fine->kp, cur_buf(coarse), coarse->kp, m, coarse->stream); break;
        case TVLBM_FP32: e = downsample_from<CodecF32>(coarse->storage, cur_buf(fine), fine->kp, cur_buf(coarse), coarse->kp, m, coarse->stream); break;
        default: e = downsample_from<CodecF32Dev>(coarse->storage, cur_buf(fine), fine->kp, cur_buf(coarse), coarse->kp, m, coarse->stream); break;
    }
    CL_CUDA(coarse, e, "downsample kernel");
    return TVLBM_OK;
}

int tvlbm_copy_state(tvlbm_ctx* src, tvlbm_ctx* dst) {
    if (!src || !dst) return TVLBM_EINVAL;
    if (src->nx != dst->nx || src->ny != dst->ny || src->velset != dst->velset || src->storage != dst->storage ||
        src->device != dst->device || src->kp.has_ref != dst->kp.has_ref)
        return ctx_fail(dst, TVLBM_EINVAL, "contexts differ in grid, velocity set, storage, reference or device");
    cudaSetDevice(dst->device);
    if (src->stream != dst->stream) CL_CUDA(dst, cudaStreamSynchronize(src->stream), "synchronize");
    CL_CUDA(dst, cudaMemcpyAsync(cur_buf(dst), cur_buf(src), src->L.buf_bytes, cudaMemcpyDeviceToDevice, dst->stream),
            "copy state");
    return TVLBM_OK;
}

int tvlbm_step_closure(tvlbm_ctx* c, tvlbm_mlp* m, const float* mu, const float* inv_sigma, const float* out_scale,
                       int n) {
    int rc = closure_ctx_ok(c);
    if (rc) return rc;
    Norm nrm;
    if (!m || !out_scale || make_norm(mu, inv_sigma, &nrm) || n < 0)
        return ctx_fail(c, TVLBM_EINVAL, "null or non-finite argument, or negative step count");
    Scale sc;
    for (int k = 0; k < NK; ++k) {
        if (!isfinite(out_scale[k])) return ctx_fail(c, TVLBM_EINVAL, "non-finite output scale");
        sc.s[k] = out_scale[k];
    }
    const long long cells = (long long)c->nx * c->ny;
    if (cells % 128 || cells > mlp_max_rows(m))
        return ctx_fail(c, TVLBM_EINVAL, "nx*ny must be a multiple of 128 and at most the network's max_rows");
    cudaSetDevice(c->device);
    BasisD bd;
    BasisF bf;
    make_basis(c->rule, &bd, &bf);
    mlp_set_stream(m, c->stream);
    const long long ncell = cells;
    // one learned step on stream s: stream, features of the streamed state, network, collision
    auto one_step = [&](cudaStream_t st) -> int {
        float* m6 = (float*)(c->mem + c->L.off_mom);
        float* y = mlp_ybuf(m);
        const dim3 b(32, 4), g = grid_of(c->nx, c->ny, b);  // 128 threads: an even spread of the blocks over the SMs
        // streaming, with the streamed state's moments (FP64 storage: FP64 moments)
        switch (c->storage) {
            case TVLBM_FP64:
                closure_stream_kernel<CodecF64, double><<<g, b, 0, st>>>((const double*)cur_buf(c), (double*)other_buf(c), c->kp, m6);
                break;
            case TVLBM_FP32:
                closure_stream_kernel<CodecF32, float><<<g, b, 0, st>>>((const float*)cur_buf(c), (float*)other_buf(c), c->kp, m6);
                break;
            default:
                closure_stream_kernel<CodecF32Dev, float><<<g, b, 0, st>>>((const float*)cur_buf(c), (float*)other_buf(c), c->kp, m6);
                break;
        }
        CL_CUDA(c, cudaGetLastError(), "closure stream kernel");
        c->cur ^= 1;
        // the network, building its inputs (the 3 x 3 normalised moments) in its own tiles
        MlpFeatures feat;
        feat.m6 = m6;
        feat.nx = c->nx;
        feat.ny = c->ny;
        for (int q = 0; q < NF; ++q) {
            feat.mu[q] = nrm.mu[q];
            feat.isg[q] = nrm.isg[q];
        }
        const int r = mlp_forward_features_async(m, feat, (int)ncell, y);
        if (r) return ctx_fail(c, r, tvlbm_mlp_last_error(m));
        switch (c->storage) {
            case TVLBM_FP64: closure_collide_kernel<CodecF64><<<g, b, 0, st>>>((double*)cur_buf(c), c->kp, y, bf, bd, sc); break;
            case TVLBM_FP32: closure_collide_kernel<CodecF32><<<g, b, 0, st>>>((float*)cur_buf(c), c->kp, y, bf, bd, sc); break;
            default: closure_collide_kernel<CodecF32Dev><<<g, b, 0, st>>>((float*)cur_buf(c), c->kp, y, bf, bd, sc); break;
        }
        CL_CUDA(c, cudaGetLastError(), "closure collide kernel");
        return TVLBM_OK;
    };
    // the graphs replay two steps each; they hold this network and these constants
    float key[24];
    for (int q = 0; q < NF; ++q) {
        key[q] = nrm.mu[q];
        key[NF + q] = nrm.isg[q];
    }
    for (int k = 0; k < NK; ++k) key[2 * NF + k] = sc.s[k];
    if (c->cl_key_net != mlp_uid(m) || memcmp(key, c->cl_key, sizeof(key)) != 0) {
        for (int k = 0; k < 2; ++k)
            if (c->cl_graph[k]) {
                cudaGraphExecDestroy(c->cl_graph[k]);
                c->cl_graph[k] = nullptr;
            }
        c->cl_key_net = mlp_uid(m);
        memcpy(c->cl_key, key, sizeof(key));
    }
    int left = n;
    mlp_set_stream(m, c->stream);
    if (c->graphs && left >= 2) {
        if (!c->cl_graph[c->cur]) {
            rc = one_step(c->stream);  // first launches of every kernel happen outside a capture
            if (rc) return rc;
            --left;
        }
        while (left >= 2) {
            if (!c->cl_graph[c->cur]) {
                const int parity = c->cur;
                cudaGraph_t gr = nullptr;
                CL_CUDA(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
                mlp_set_stream(m, c->capture_stream);
                int r1 = one_step(c->capture_stream);
                if (!r1) r1 = one_step(c->capture_stream);
                mlp_set_stream(m, c->stream);
                const cudaError_t ce = cudaStreamEndCapture(c->capture_stream, &gr);
                c->cur = parity;  // capture does not run the steps
                if (r1) {
                    if (gr) cudaGraphDestroy(gr);
                    return r1;
                }
                CL_CUDA(c, ce, "end capture");
                const cudaError_t ie = cudaGraphInstantiate(&c->cl_graph[parity], gr, 0);
                cudaGraphDestroy(gr);
                if (ie != cudaSuccess) {
                    c->cl_graph[parity] = nullptr;
                    CL_CUDA(c, ie, "graph instantiate");
                }
            }
            CL_CUDA(c, cudaGraphLaunch(c->cl_graph[c->cur], c->stream), "graph launch");
            left -= 2;  // parity unchanged
        }
    }
    for (; left > 0; --left) {
        rc = one_step(c->stream);
        if (rc) return rc;
    }
    return TVLBM_OK;
}

}  // extern "C"
