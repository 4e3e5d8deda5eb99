// The paper's own evolution scheme (Sec. "The TVLBM Evolution scheme", Eq. FVLB) on the unit
// grid: an explicit Euler step f(t + dt) = f + dt (Omega_bar - c . grad f) with the second-order
// stencils over the eight neighbours P1..P8 of P0 (east, north, west, south, north-east,
// north-west, south-west, south-east):
//   d_x f ~ 3/8 (f1 - f3) + 1/16 (f5 - f6 - f7 + f8),  d_y f ~ 3/8 (f2 - f4) + 1/16 (f5 + f6 - f7 - f8),
//   Omega_bar ~ 9/16 Omega(0) + 3/32 (Omega(1..4)) + 1/64 (Omega(5..8)),
// and the collision term of Eq. OMEGAFVLB: BGK plus the Prandtl-number term
// (1 / tau_g) f_eq / (rho T^2) Pi : (c - u)(c - u), applied without its components along the
// collision invariants (an exact Maxwellian has none; a truncated equilibrium leaves a residue).
// Two kernels per step: the collision term of every cell (stored with the periodic frame images
// in a population-sized buffer), then the update, which reads both fields at the 3 x 3 cells.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "tvlbm.h"
#include "tvlbm_ctx.h"
#include "tvlbm_kernels.cuh"
#include "tvlbm_tiled.cuh"

using namespace tvlbm;

namespace {

// Inverse Gram matrix of the collision invariants (1, c_x, c_y, |c|^2) in sum_l w_l g_l h_l, and
// the scheme's constants.
struct FvParams {
    double ginv[4][4];
    double inv_tau, inv_tau_g, dt;
    int prandtl;
};

template <int N1, class C>
__global__ void __launch_bounds__(256) fv_omega_kernel(const typename C::T* __restrict__ f,
                                                       typename C::T* __restrict__ om, const KParams p,
                                                       const FvParams fp) {
    using R = typename C::R;
    constexpr int Q = N1 * N1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    R s[Q];
    R rho = 0, jx = 0, jy = 0, e2 = 0;
#pragma unroll
    for (int j = 0; j < N1; ++j)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const R v = C::ld(f + sidx(p, i + N1 * j, x, y));
            const R cx = kx<R>(p, i), cy = kx<R>(p, j);
            s[i + N1 * j] = v;
            rho += v;
            jx += v * cx;
            jy += v * cy;
            e2 += v * (cx * cx + cy * cy);
        }
    const R ux = jx / rho, uy = jy / rho;
    const R T = R(0.5) * (e2 / rho - (ux * ux + uy * uy));
    R eq[Q];
    cell_equilibrium<N1, false, R>(p, rho, ux, uy, T - R(1), eq);
    R w[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) w[l] = -(s[l] - eq[l]) * (R)fp.inv_tau;
    if (fp.prandtl) {
        R pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const R n = s[i + N1 * j] - eq[i + N1 * j];
                const R dx = kx<R>(p, i) - ux, dy = kx<R>(p, j) - uy;
                pxx += n * dx * dx;
                pxy += n * dx * dy;
                pyy += n * dy * dy;
            }
        const R scale = (R)fp.inv_tau_g / (rho * T * T);
        R raw[Q], m[4] = {0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                const R cx = kx<R>(p, i), cy = kx<R>(p, j);
                const R dx = cx - ux, dy = cy - uy;
                raw[l] = scale * eq[l] * (pxx * dx * dx + R(2) * pxy * dx * dy + pyy * dy * dy);
                m[0] += raw[l];
                m[1] += raw[l] * cx;
                m[2] += raw[l] * cy;
                m[3] += raw[l] * (cx * cx + cy * cy);
            }
        // remove the invariant components: raw -= w sum_k b_k phi_k, G b = m
        R b[4];
#pragma unroll
        for (int a = 0; a < 4; ++a) {
            b[a] = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) b[a] += (R)fp.ginv[a][c] * m[c];
        }
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                const R cx = kx<R>(p, i), cy = kx<R>(p, j);
                const R wl = kw<R>(p, i) * kw<R>(p, j);
                w[l] += raw[l] - wl * (b[0] + b[1] * cx + b[2] * cy + b[3] * (cx * cx + cy * cy));
            }
    }
    store_collided<N1, C>(om, geom_of(p), x, y, w);
}

template <int N1, class C>
__global__ void __launch_bounds__(256) fv_update_kernel(const typename C::T* __restrict__ f,
                                                        const typename C::T* __restrict__ om,
                                                        typename C::T* __restrict__ fout, const KParams p,
                                                        const FvParams fp) {
    using R = typename C::R;
    constexpr int Q = N1 * N1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long pitch = p.pitch;
    R s[Q];
#pragma unroll
    for (int j = 0; j < N1; ++j)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const int l = i + N1 * j;
            const long long c0 = sidx(p, l, x, y);
            const typename C::T* fq = f + c0;
            const typename C::T* oq = om + c0;
            // P1 east, P2 north, P3 west, P4 south, P5 NE, P6 NW, P7 SW, P8 SE (+y is the next row)
            const R f1 = C::ld(fq + 1), f2 = C::ld(fq + pitch), f3 = C::ld(fq - 1), f4 = C::ld(fq - pitch);
            const R f5 = C::ld(fq + pitch + 1), f6 = C::ld(fq + pitch - 1), f7 = C::ld(fq - pitch - 1),
                    f8 = C::ld(fq - pitch + 1);
            const R gx = R(0.375) * (f1 - f3) + R(0.0625) * (f5 - f6 - f7 + f8);
            const R gy = R(0.375) * (f2 - f4) + R(0.0625) * (f5 + f6 - f7 - f8);
            const R obar = R(0.5625) * C::ld(oq) +
                           R(0.09375) * (C::ld(oq + 1) + C::ld(oq + pitch) + C::ld(oq - 1) + C::ld(oq - pitch)) +
                           R(0.015625) * (C::ld(oq + pitch + 1) + C::ld(oq + pitch - 1) + C::ld(oq - pitch - 1) +
                                          C::ld(oq - pitch + 1));
            s[l] = C::ld(fq) + (R)fp.dt * (obar - kx<R>(p, i) * gx - kx<R>(p, j) * gy);
        }
    store_collided<N1, C>(fout, geom_of(p), x, y, s);
}

template <int N1, class C>
cudaError_t launch_fv(const void* f, void* om, void* fout, const KParams& p, const FvParams& fp, cudaStream_t s) {
    using T = typename C::T;
    const dim3 b(32, 8), g((p.nx + 31) / 32, (p.ny + 7) / 8);
    fv_omega_kernel<N1, C><<<g, b, 0, s>>>((const T*)f, (T*)om, p, fp);
    fv_update_kernel<N1, C><<<g, b, 0, s>>>((const T*)f, (const T*)om, (T*)fout, p, fp);
    return cudaGetLastError();
}

template <int N1>
cudaError_t launch_fv_storage(int storage, const void* f, void* om, void* fout, const KParams& p, const FvParams& fp,
                              cudaStream_t s) {
    return storage == TVLBM_FP64 ? launch_fv<N1, CodecF64>(f, om, fout, p, fp, s)
                                 : launch_fv<N1, CodecF32>(f, om, fout, p, fp, s);
}

// Inverse of the 4 x 4 Gram matrix of (1, c_x, c_y, |c|^2) under the set's weights (Gauss-Jordan).
bool gram_inverse(const host::Rule& r, double out[4][4]) {
    double G[4][8];
    memset(G, 0, sizeof(G));
    for (int j = 0; j < r.n; ++j)
        for (int i = 0; i < r.n; ++i) {
            const double w = r.w[i] * r.w[j], cx = r.x[i], cy = r.x[j];
            const double phi[4] = {1.0, cx, cy, cx * cx + cy * cy};
            for (int a = 0; a < 4; ++a)
                for (int b = 0; b < 4; ++b) G[a][b] += w * phi[a] * phi[b];
        }
    for (int a = 0; a < 4; ++a) G[a][4 + a] = 1.0;
    for (int c = 0; c < 4; ++c) {
        int piv = c;
        for (int a = c + 1; a < 4; ++a)
            if (fabs(G[a][c]) > fabs(G[piv][c])) piv = a;
        if (fabs(G[piv][c]) < 1e-14) return false;
        for (int b = 0; b < 8; ++b) {
            const double t = G[c][b];
            G[c][b] = G[piv][b];
            G[piv][b] = t;
        }
        const double d = G[c][c];
        for (int b = 0; b < 8; ++b) G[c][b] /= d;
        for (int a = 0; a < 4; ++a)
            if (a != c) {
                const double m = G[a][c];
                for (int b = 0; b < 8; ++b) G[a][b] -= m * G[c][b];
            }
    }
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) out[a][b] = G[a][4 + b];
    return true;
}

}  // namespace

int fvlb_steps(tvlbm_ctx* c, int n) {
    FvParams fp;
    memset(&fp, 0, sizeof(fp));
    if (!gram_inverse(c->rule, fp.ginv)) {
        snprintf(c->err, sizeof(c->err), "singular invariant Gram matrix");
        return TVLBM_EINVAL;
    }
    fp.inv_tau = 1.0 / c->tau;
    fp.prandtl = isfinite(c->tau_g) ? 1 : 0;
    fp.inv_tau_g = fp.prandtl ? 1.0 / c->tau_g : 0.0;
    fp.dt = c->dt;
    for (int t = 0; t < n; ++t) {
        const void* f = c->mem + c->L.off_f[c->cur];
        void* fout = c->mem + c->L.off_f[1 - c->cur];
        cudaError_t e;
        switch (c->n1) {
            case 3: e = launch_fv_storage<3>(c->storage, f, c->fv_omega, fout, c->kp, fp, c->stream); break;
            case 4: e = launch_fv_storage<4>(c->storage, f, c->fv_omega, fout, c->kp, fp, c->stream); break;
            default: e = launch_fv_storage<6>(c->storage, f, c->fv_omega, fout, c->kp, fp, c->stream); break;
        }
        if (e != cudaSuccess) {
            snprintf(c->err, sizeof(c->err), "finite-volume kernels: %s", cudaGetErrorString(e));
            return TVLBM_ECUDA;
        }
        c->cur ^= 1;
    }
    return TVLBM_OK;
}

extern "C" int tvlbm_set_scheme(tvlbm_ctx* c, int scheme, double tau_g) {
    if (!c) return TVLBM_EINVAL;
    if (scheme == TVLBM_SCHEME_VOLUMETRIC) {
        c->scheme = scheme;
        c->tau_g = INFINITY;
        return TVLBM_OK;
    }
    if (scheme != TVLBM_SCHEME_FVLB) {
        snprintf(c->err, sizeof(c->err), "unknown scheme %d", scheme);
        return TVLBM_EINVAL;
    }
    if (c->kp.walls || (c->storage != TVLBM_FP64 && c->storage != TVLBM_FP32) || isnan(tau_g) || tau_g == 0.0 ||
        !isfinite(c->tau)) {
        snprintf(c->err, sizeof(c->err),
                 "the finite-volume scheme needs a periodic domain, FP64 or FP32 storage, finite tau and tau_g != 0");
        return TVLBM_EINVAL;
    }
    cudaSetDevice(c->device);
    if (!c->fv_omega) {
        void* p = nullptr;
        if (cudaMalloc(&p, c->L.buf_bytes) != cudaSuccess) return TVLBM_ENOMEM;
        if (cudaMemset(p, 0, c->L.buf_bytes) != cudaSuccess) {
            cudaFree(p);
            return TVLBM_ECUDA;
        }
        c->fv_omega = p;
    }
    c->scheme = scheme;
    c->tau_g = tau_g;
    return TVLBM_OK;
}
