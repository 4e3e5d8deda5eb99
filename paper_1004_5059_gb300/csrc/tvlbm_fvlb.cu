// The paper's own evolution scheme (Sec. "The TVLBM Evolution scheme", Eq. FVLB) on the unit
// grid: an explicit Euler step f(t + dt) = f + dt (Omega_bar - c . grad f) with the second-order
// stencils over the eight neighbours P1..P8 of P0 (east, north, west, south, north-east,
// north-west, south-west, south-east):
//   d_x f ~ 3/8 (f1 - f3) + 1/16 (f5 - f6 - f7 + f8),  d_y f ~ 3/8 (f2 - f4) + 1/16 (f5 + f6 - f7 - f8),
//   Omega_bar ~ 9/16 Omega(0) + 3/32 (Omega(1..4)) + 1/64 (Omega(5..8)),
// and the collision term of Eq. OMEGAFVLB: BGK plus the Prandtl-number term
// (1 / tau_g) f_eq / (rho T^2) Pi : (c - u)(c - u), applied without its components along the
// collision invariants (an exact Maxwellian has none; a truncated equilibrium leaves a residue).
// One fused kernel per step (fv_fused_kernel: the collision term of a block of cells in shared
// memory, then the update of its inner cells), or, as the two-kernel form, the collision term of
// every cell (stored with the periodic frame images in a population-sized buffer) and then the
// update, which reads both fields at the 3 x 3 cells.  Both give the same populations.
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
    int pscale;         // relaxation times divided by the local pressure: tau -> tau / p, p = rho T
    int walls;          // channel: wall nodes on the first and last rows
    const double* dy;   // node spacings in y [ny - 1], or null for unit spacing
};

// Wall imposition parameters: wall velocity and temperature per side, the Newton-Raphson mode.
struct WallParams {
    double u[2], T[2];
    int exact, iters;
    double* eq;  // [2][nx][2] wall equilibria (u_eq, T_eq), warm start of the next imposition
};

// Resident CTAs per SM the collision-term kernel is compiled for (as fv_update_minb: each set and
// precision held near its own register need).
template <int N1, class C>
constexpr int fv_omega_minb() {
    return sizeof(typename C::R) == 4 ? (N1 <= 4 ? 4 : 2) : (N1 == 3 ? 3 : (N1 == 4 ? 2 : 1));
}

// Collision term of Eq. OMEGAFVLB at one cell from its populations s: BGK, plus with tau_g the
// Prandtl term less its components along the collision invariants.
template <int N1, class C>
__device__ __forceinline__ void fv_omega_cell(const typename C::R (&s)[N1 * N1], const KParams& p, const FvParams& fp,
                                              typename C::R (&w)[N1 * N1]) {
    using R = typename C::R;
    constexpr int Q = N1 * N1;
    R rho = 0, jx = 0, jy = 0, e2 = 0;
#pragma unroll
    for (int j = 0; j < N1; ++j)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const R v = s[i + N1 * j];
            const R cx = kx<R>(p, i), cy = kx<R>(p, j);
            rho += v;
            jx += v * cx;
            jy += v * cy;
            e2 += v * (cx * cx + cy * cy);
        }
    const R ux = jx / rho, uy = jy / rho;
    const R T = R(0.5) * (e2 / rho - (ux * ux + uy * uy));
    R eq[Q];
    cell_equilibrium<N1, false, R>(p, rho, ux, uy, T - R(1), eq);
    // tau -> tau / p and tau_g -> tau_g / p (constant dynamic viscosity and conductivity)
    const R ps = fp.pscale ? rho * T : R(1);
    const R itau = (R)fp.inv_tau * ps;
#pragma unroll
    for (int l = 0; l < Q; ++l) w[l] = -(s[l] - eq[l]) * itau;
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
        const R scale = (R)fp.inv_tau_g * ps / (rho * T * T);
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
}

template <int N1, class C>
__global__ void __launch_bounds__(256, fv_omega_minb<N1, C>()) fv_omega_kernel(const typename C::T* __restrict__ f,
                                                       typename C::T* __restrict__ om, const KParams p,
                                                       const FvParams fp) {
    using R = typename C::R;
    constexpr int Q = N1 * N1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    R s[Q], w[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) s[l] = C::ld(f + sidx(p, l, x, y));
    fv_omega_cell<N1, C>(s, p, fp, w);
    store_collided<N1, C>(om, geom_of(p), x, y, w);
}

// Resident CTAs per SM the update is compiled for: its time is load latency, so occupancy pays
// (D2Q16 FP32: 4 CTAs of 256 threads at 64 registers, 7.9 against 7.3 G cell updates per second
// at 106 registers and 2 CTAs); each set and precision is held near its own register need.
template <int N1, class C>
constexpr int fv_update_minb() {
    return sizeof(typename C::R) == 4 ? (N1 <= 4 ? 4 : 3) : (N1 <= 3 ? 4 : (N1 == 4 ? 2 : 1));
}

// The update of Eq. FVLB, interior node: population l at the cell from the 3 x 3 neighbourhood of
// populations f(dx, dy) and collision terms o(dx, dy) (dy = +1 the next row; P1 east, P2 north,
// P3 west, P4 south, P5 NE, P6 NW, P7 SW, P8 SE).  ysc: the y spacing factor 2 / (dy_j + dy_j-1)
// of the stencil (1 on the unit grid).
template <class R, class F, class O>
__device__ __forceinline__ R fv_interior(const F& f, const O& o, R ysc, R dt, R cx, R cy) {
    const R f1 = f(1, 0), f2 = f(0, 1), f3 = f(-1, 0), f4 = f(0, -1);
    const R f5 = f(1, 1), f6 = f(-1, 1), f7 = f(-1, -1), f8 = f(1, -1);
    const R gx = R(0.375) * (f1 - f3) + R(0.0625) * (f5 - f6 - f7 + f8);
    const R gy = ysc * (R(0.375) * (f2 - f4) + R(0.0625) * (f5 + f6 - f7 - f8));
    const R obar = R(0.5625) * o(0, 0) + R(0.09375) * (o(1, 0) + o(0, 1) + o(-1, 0) + o(0, -1)) +
                   R(0.015625) * (o(1, 1) + o(-1, 1) + o(-1, -1) + o(1, -1));
    return f(0, 0) + dt * (obar - cx * gx - cy * gy);
}

// What the update of a cell row needs to know about the row: wall node (1 bottom, 2 top, 0
// interior), its fluid-side neighbour row (in), the wall normal's sign, and the y factor (the
// wall spacing dy_w for a wall node, else the interior spacing factor).
template <class R>
struct FvRow {
    int wall, in;
    R sgn, yf;
};
template <class R>
__device__ __forceinline__ FvRow<R> fv_row(const KParams& p, const FvParams& fp, int y) {
    FvRow<R> r;
    r.wall = fp.walls ? (y == 0 ? 1 : (y == p.ny - 1 ? 2 : 0)) : 0;
    r.sgn = r.wall == 1 ? R(1) : R(-1);  // n = +y at the bottom, -y at the top
    r.in = r.wall == 1 ? 1 : -1;
    if (r.wall) r.yf = fp.dy ? (R)(r.wall == 1 ? fp.dy[0] : fp.dy[p.ny - 2]) : R(1);
    else r.yf = fp.dy ? (R)(2.0 / (fp.dy[y] + fp.dy[y - 1])) : R(1);
    return r;
}

// Population l = i + N1 j of the update of Eq. FVLB at a wall node of a channel (Eq. FVLB2), its
// neighbourhood read through ld: ld.f(l, dx, dy) and ld.om(l, dx, dy).  Populations arriving at
// the wall (c . n <= 0) advance with the one-sided stencils into the fluid, the leaving ones keep
// their imposed values.
template <int N1, class C, class Ld>
__device__ __forceinline__ typename C::R fv_wall_one(const Ld& ld, const KParams& p, const FvParams& fp,
                                                     const FvRow<typename C::R>& rw, int i, int j) {
    using R = typename C::R;
    const int l = i + N1 * j;
    const R cy = kx<R>(p, j);
    const R f0 = ld.f(l, 0, 0);
    if (rw.sgn * cy > R(0)) return f0;
    const int in = rw.in;
    const R fE = ld.f(l, 1, 0), fW = ld.f(l, -1, 0), fI = ld.f(l, 0, in), fIE = ld.f(l, 1, in), fIW = ld.f(l, -1, in);
    const R gx = R(0.375) * (fE - fW) + R(0.125) * (fIE - fIW);
    const R gy = rw.sgn * (R(2) / rw.yf) * (R(0.375) * (fI - f0) + R(0.0625) * (fIE + fIW - fE - fW));
    const R obar = R(0.5625) * ld.om(l, 0, 0) + R(0.09375) * (ld.om(l, 1, 0) + ld.om(l, -1, 0)) +
                   R(0.1875) * ld.om(l, 0, in) + R(0.03125) * (ld.om(l, 1, in) + ld.om(l, -1, in));
    return f0 + (R)fp.dt * (obar - kx<R>(p, i) * gx - cy * gy);
}

// Population l of the update at an interior node, its neighbourhood read through ld.
template <int N1, class C, class Ld>
__device__ __forceinline__ typename C::R fv_interior_one(const Ld& ld, const KParams& p, const FvParams& fp,
                                                         const FvRow<typename C::R>& rw, int i, int j) {
    using R = typename C::R;
    const int l = i + N1 * j;
    return fv_interior<R>([&](int dx, int dy) { return ld.f(l, dx, dy); },
                          [&](int dx, int dy) { return ld.om(l, dx, dy); }, rw.yf, (R)fp.dt, kx<R>(p, i),
                          kx<R>(p, j));
}

// Every population of the update at the cell of row y (the wall test taken once per cell, so
// the loads of all velocities can be issued together).
template <int N1, class C, class Ld>
__device__ __forceinline__ void fv_update_cell(const Ld& ld, const KParams& p, const FvParams& fp, int y,
                                               typename C::R (&s)[N1 * N1]) {
    const FvRow<typename C::R> rw = fv_row<typename C::R>(p, fp, y);
    if (rw.wall) {
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int i = 0; i < N1; ++i) s[i + N1 * j] = fv_wall_one<N1, C>(ld, p, fp, rw, i, j);
        return;
    }
#pragma unroll
    for (int j = 0; j < N1; ++j)
#pragma unroll
        for (int i = 0; i < N1; ++i) s[i + N1 * j] = fv_interior_one<N1, C>(ld, p, fp, rw, i, j);
}

// Neighbourhood reads of the two-kernel form: both fields in global memory (framed layout).
template <class C>
struct FvGlobalNbr {
    const typename C::T* fb;  // the cell's element in plane 0 of the populations
    const typename C::T* ob;  // and of the collision term
    long long plane, pitch;
    __device__ __forceinline__ typename C::R f(int l, int dx, int dy) const {
        return C::ld(fb + l * plane + dy * pitch + dx);
    }
    __device__ __forceinline__ typename C::R om(int l, int dx, int dy) const {
        return C::ld(ob + l * plane + dy * pitch + dx);
    }
};

template <int N1, class C>
__global__ void __launch_bounds__(256, fv_update_minb<N1, C>()) fv_update_kernel(const typename C::T* __restrict__ f,
                                                        const typename C::T* __restrict__ om,
                                                        typename C::T* __restrict__ fout, const KParams p,
                                                        const FvParams fp) {
    using R = typename C::R;
    constexpr int Q = N1 * N1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long c0 = sidx(p, 0, x, y);
    const FvGlobalNbr<C> ld{f + c0, om + c0, p.plane, (long long)p.pitch};
    R s[Q];
    fv_update_cell<N1, C>(ld, p, fp, y, s);
    store_collided<N1, C>(fout, geom_of(p), x, y, s);
}

// Fused form: one kernel per step.  A CTA of 32 x BY threads holds a 32 x BY block of cells in
// shared memory, populations and collision terms; its inner 30 x (BY - 2) cells are the CTA's
// output, the outer ring their halo.  Each thread loads its cell (the ring from the periodic
// images or ghost rows of the frame), computes the cell's collision term, and after one block
// barrier the inner cells are updated from their 3 x 3 neighbourhoods in shared memory: the
// collision term never goes through global memory (read Q, write Q values per cell update
// instead of 5 Q), at the cost of recomputing it on the ring (32 BY / (30 (BY - 2)) of the
// cells).  Same arithmetic as the two-kernel form, so the same populations bit for bit.
template <int N1, class C>
constexpr int fv_fused_by() {  // rows of the block: 16 where both fields of 512 cells fit 160 KB
    return 2 * N1 * N1 * 32 * 16 * (int)sizeof(typename C::T) <= 160 * 1024 ? 16 : 8;
}
template <int N1, class C>
constexpr int fv_fused_minb() {  // 2 CTAs (64 registers) for FP32 up to D2Q16, else 1
    return (sizeof(typename C::R) == 4 && N1 <= 4) ? 2 : 1;
}
template <int N1, class C>
constexpr size_t fv_fused_smem() {
    return 2 * (size_t)N1 * N1 * 32 * fv_fused_by<N1, C>() * sizeof(typename C::T);
}

template <class C, int CELLS>
struct FvSharedNbr {
    const typename C::T* fs;  // [Q][CELLS] populations of the block
    const typename C::T* os;  // [Q][CELLS] collision terms of the block
    int c;                    // the cell's index in the block (row-major, 32 per row)
    __device__ __forceinline__ typename C::R f(int l, int dx, int dy) const {
        return (typename C::R)fs[l * CELLS + c + dy * 32 + dx];
    }
    __device__ __forceinline__ typename C::R om(int l, int dx, int dy) const {
        return (typename C::R)os[l * CELLS + c + dy * 32 + dx];
    }
};

template <int N1, class C>
__global__ void __launch_bounds__(32 * fv_fused_by<N1, C>(), fv_fused_minb<N1, C>())
    fv_fused_kernel(const typename C::T* __restrict__ f, typename C::T* __restrict__ fout, const KParams p,
                    const FvParams fp) {
    using R = typename C::R;
    using T = typename C::T;
    static_assert(std::is_same<R, T>::value, "the fused form keeps the stored values in shared memory as read");
    constexpr int Q = N1 * N1, BY = fv_fused_by<N1, C>(), CELLS = 32 * BY;
    extern __shared__ __align__(16) unsigned char fv_smem[];
    T* fs = reinterpret_cast<T*>(fv_smem);
    T* os = fs + Q * CELLS;
    const int tx = threadIdx.x, ty = threadIdx.y, c = ty * 32 + tx;
    const int x = blockIdx.x * 30 + tx - 1, y = blockIdx.y * (BY - 2) + ty - 1;
    // cells up to x = nx and y = ny lie in the frame (periodic images, or the ghost rows beyond a
    // wall, which no wall node's stencil reads); the ring beyond them belongs to no output
    if (x <= p.nx && y <= p.ny) {
        R s[Q], w[Q];
        const T* fb = f + sidx(p, 0, x, y);
#pragma unroll
        for (int l = 0; l < Q; ++l) {
            s[l] = C::ld(fb + l * p.plane);
            fs[l * CELLS + c] = s[l];
        }
        fv_omega_cell<N1, C>(s, p, fp, w);
#pragma unroll
        for (int l = 0; l < Q; ++l) os[l * CELLS + c] = w[l];
    }
    __syncthreads();
    if (tx >= 1 && tx <= 30 && ty >= 1 && ty <= BY - 2 && x < p.nx && y < p.ny) {
        const FvSharedNbr<C, CELLS> ld{fs, os, c};
        R s[Q];
        fv_update_cell<N1, C>(ld, p, fp, y, s);
        store_collided<N1, C>(fout, geom_of(p), x, y, s);
    }
}

// Equilibrium of unit density at velocity (u, 0) and temperature T, FP64.
template <int N1>
__device__ __forceinline__ void wall_feq(const KParams& p, double u, double T, double (&eq)[N1 * N1]) {
    cell_equilibrium<N1, false, double>(p, 1.0, u, 0.0, T - 1.0, eq);
}

// Before a step: the leaving populations of every wall node (c . n > 0, n into the fluid)
// become A f_eq(u_eq, T_eq) with A = sum_{c.n<=0} |c.n| f / sum_{c.n>0} |c.n| f_eq (Eq.
// IMPOSITION); in the exact mode (u_eq, T_eq) follows the Newton-Raphson of App. B so that the
// node's velocity and temperature are the wall's.  One thread per (column, wall); FP64.
template <int N1, class C>
__global__ void fv_impose_kernel(typename C::T* __restrict__ f, const KParams p, const WallParams wp) {
    constexpr int Q = N1 * N1;
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 2 * p.nx) return;
    const int side = t / p.nx, x = t - side * p.nx;
    const int y = side == 0 ? 0 : p.ny - 1;
    const double sgn = side == 0 ? 1.0 : -1.0;
    double v[Q], cn[Q];
    double incoming = 0.0;
#pragma unroll
    for (int j = 0; j < N1; ++j)
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const int l = i + N1 * j;
            v[l] = (double)C::ld(f + sidx(p, l, x, y));
            cn[l] = sgn * p.xd[j];
            if (cn[l] <= 0.0) incoming += -cn[l] * v[l];
        }
    const double uw = wp.u[side], Tw = wp.T[side];
    double* st = wp.eq + (side * p.nx + x) * 2;
    double ue = wp.exact ? st[0] : uw, Te = wp.exact ? st[1] : Tw;
    const int iters = wp.exact ? wp.iters : 0;
    double eq[Q];
    double S = 1.0;
    for (int it = 0;; ++it) {
        wall_feq<N1>(p, ue, Te, eq);
        S = 0.0;
#pragma unroll
        for (int l = 0; l < Q; ++l)
            if (cn[l] > 0.0) S += cn[l] * eq[l];
#pragma unroll
        for (int l = 0; l < Q; ++l)
            if (cn[l] > 0.0) v[l] = incoming / S * eq[l];
        if (it == iters) break;
        double rho = 0.0, mx = 0.0, m2 = 0.0;
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                const double cx = p.xd[i], cy = p.xd[j];
                rho += v[l];
                mx += v[l] * cx;
                m2 += v[l] * (cx * cx + cy * cy);
            }
        const double F1 = rho * uw - mx, F2 = 2.0 * rho * Tw + rho * uw * uw - m2;
        const double h = 1e-6;
        double ep[Q], em[Q];
        double A = 0, B = 0, Cc = 0, D = 0, su = 0, sT = 0, sx = 0, s2 = 0;
        wall_feq<N1>(p, ue + h, Te, ep);
        wall_feq<N1>(p, ue - h, Te, em);
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                if (cn[l] <= 0.0) continue;
                const double cx = p.xd[i], c2 = cx * cx + p.xd[j] * p.xd[j];
                const double du = (ep[l] - em[l]) / (2.0 * h);
                A += cx * du;
                Cc += c2 * du;
                su += cn[l] * du;
                sx += cx * eq[l];
                s2 += c2 * eq[l];
            }
        wall_feq<N1>(p, ue, Te + h, ep);
        wall_feq<N1>(p, ue, Te - h, em);
#pragma unroll
        for (int j = 0; j < N1; ++j)
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                if (cn[l] <= 0.0) continue;
                const double cx = p.xd[i], c2 = cx * cx + p.xd[j] * p.xd[j];
                const double dT = (ep[l] - em[l]) / (2.0 * h);
                B += cx * dT;
                D += c2 * dT;
                sT += cn[l] * dT;
            }
        A -= su * sx / S;
        Cc -= su * s2 / S;
        B -= sT * sx / S;
        D -= sT * s2 / S;
        const double pref = S / ((A * D - B * Cc) * incoming);
        ue += pref * (D * F1 - B * F2);
        Te += pref * (-Cc * F1 + A * F2);
    }
    if (wp.exact) {
        st[0] = ue;
        st[1] = Te;
    }
    const Geom g = geom_of(p);
#pragma unroll
    for (int l = 0; l < Q; ++l)
        if (cn[l] > 0.0) store_with_images(f, g, (long long)l * p.plane, x, y, C::enc((typename C::R)v[l]));
}

template <int N1, class C>
cudaError_t launch_fv(const void* f, void* om, void* fout, const KParams& p, const FvParams& fp, const WallParams& wp,
                      bool split, cudaStream_t s) {
    using T = typename C::T;
    if (fp.walls) fv_impose_kernel<N1, C><<<(2 * p.nx + 127) / 128, 128, 0, s>>>((T*)f, p, wp);
    if (split) {
        const dim3 b(32, 8), g((p.nx + 31) / 32, (p.ny + 7) / 8);
        fv_omega_kernel<N1, C><<<g, b, 0, s>>>((const T*)f, (T*)om, p, fp);
        fv_update_kernel<N1, C><<<g, b, 0, s>>>((const T*)f, (const T*)om, (T*)fout, p, fp);
    } else {
        constexpr int BY = fv_fused_by<N1, C>();
        constexpr size_t smem = fv_fused_smem<N1, C>();
        cudaError_t e = cudaFuncSetAttribute(fv_fused_kernel<N1, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
        const dim3 b(32, BY), g((p.nx + 29) / 30, (p.ny + BY - 3) / (BY - 2));
        fv_fused_kernel<N1, C><<<g, b, smem, s>>>((const T*)f, (T*)fout, p, fp);
    }
    return cudaGetLastError();
}

template <int N1>
cudaError_t launch_fv_storage(int storage, const void* f, void* om, void* fout, const KParams& p, const FvParams& fp,
                              const WallParams& wp, bool split, cudaStream_t s) {
    return storage == TVLBM_FP64 ? launch_fv<N1, CodecF64>(f, om, fout, p, fp, wp, split, s)
                                 : launch_fv<N1, CodecF32>(f, om, fout, p, fp, wp, split, s);
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
    fp.pscale = c->fv_pscale;
    fp.walls = c->kp.walls ? 1 : 0;
    fp.dy = c->fv_dy;
    WallParams wp;
    memset(&wp, 0, sizeof(wp));
    if (fp.walls) {
        if (!c->fv_wall_eq) {
            snprintf(c->err, sizeof(c->err), "channel: call tvlbm_set_fv_walls first");
            return TVLBM_EINVAL;
        }
        wp.u[0] = c->bc.u_lo;
        wp.T[0] = c->bc.T_lo;
        wp.u[1] = c->bc.u_hi;
        wp.T[1] = c->bc.T_hi;
        wp.exact = c->fv_exact;
        wp.iters = c->fv_nr_iters;
        wp.eq = c->fv_wall_eq;
    }
    for (int t = 0; t < n; ++t) {
        void* f = c->mem + c->L.off_f[c->cur];
        void* fout = c->mem + c->L.off_f[1 - c->cur];
        cudaError_t e;
        switch (c->n1) {
            case 3: e = launch_fv_storage<3>(c->storage, f, c->fv_omega, fout, c->kp, fp, wp, c->fv_split != 0, c->stream); break;
            case 4: e = launch_fv_storage<4>(c->storage, f, c->fv_omega, fout, c->kp, fp, wp, c->fv_split != 0, c->stream); break;
            default: e = launch_fv_storage<6>(c->storage, f, c->fv_omega, fout, c->kp, fp, wp, c->fv_split != 0, c->stream); break;
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
    if (c->mesh_mem) {
        snprintf(c->err, sizeof(c->err), "the finite-volume scheme takes its mesh from tvlbm_set_fv_walls");
        return TVLBM_EINVAL;
    }
    if ((c->storage != TVLBM_FP64 && c->storage != TVLBM_FP32) || isnan(tau_g) || tau_g == 0.0 || !isfinite(c->tau)) {
        snprintf(c->err, sizeof(c->err), "the finite-volume scheme needs FP64 or FP32 storage, finite tau and tau_g != 0");
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

extern "C" int tvlbm_set_fv_pressure_scaling(tvlbm_ctx* c, int enable) {
    if (!c) return TVLBM_EINVAL;
    if (c->scheme != TVLBM_SCHEME_FVLB) {
        snprintf(c->err, sizeof(c->err), "pressure scaling applies to the finite-volume scheme");
        return TVLBM_EINVAL;
    }
    c->fv_pscale = enable ? 1 : 0;
    return TVLBM_OK;
}

extern "C" int tvlbm_set_fv_fused(tvlbm_ctx* c, int fused) {
    if (!c) return TVLBM_EINVAL;
    c->fv_split = fused ? 0 : 1;
    return TVLBM_OK;
}

extern "C" int tvlbm_set_fv_walls(tvlbm_ctx* c, int exact, int nr_iters, const double* y_nodes) {
    if (!c) return TVLBM_EINVAL;
    if (!c->kp.walls || c->scheme != TVLBM_SCHEME_FVLB || (exact && nr_iters < 1) || nr_iters > 1000) {
        snprintf(c->err, sizeof(c->err), "needs a channel context in the finite-volume scheme and 1..1000 iterations");
        return TVLBM_EINVAL;
    }
    double* dy_host = nullptr;
    if (y_nodes) {
        dy_host = new double[c->ny - 1];
        for (int j = 0; j + 1 < c->ny; ++j) {
            dy_host[j] = y_nodes[j + 1] - y_nodes[j];
            if (!(dy_host[j] > 0.0) || !isfinite(dy_host[j])) {
                delete[] dy_host;
                snprintf(c->err, sizeof(c->err), "y_nodes must be finite and increasing");
                return TVLBM_EINVAL;
            }
        }
    }
    cudaSetDevice(c->device);
    if (!c->fv_wall_eq && cudaMalloc((void**)&c->fv_wall_eq, sizeof(double) * 4 * c->nx) != cudaSuccess) {
        delete[] dy_host;
        return TVLBM_ENOMEM;
    }
    // warm start of the Newton-Raphson: the walls' own velocity and temperature
    double* eq = new double[4 * c->nx];
    for (int x = 0; x < c->nx; ++x) {
        eq[2 * x] = c->bc.u_lo;
        eq[2 * x + 1] = c->bc.T_lo;
        eq[2 * (c->nx + x)] = c->bc.u_hi;
        eq[2 * (c->nx + x) + 1] = c->bc.T_hi;
    }
    cudaError_t e = cudaMemcpy(c->fv_wall_eq, eq, sizeof(double) * 4 * c->nx, cudaMemcpyHostToDevice);
    delete[] eq;
    if (e == cudaSuccess && dy_host) {
        if (!c->fv_dy) e = cudaMalloc((void**)&c->fv_dy, sizeof(double) * (c->ny - 1));
        if (e == cudaSuccess) e = cudaMemcpy(c->fv_dy, dy_host, sizeof(double) * (c->ny - 1), cudaMemcpyHostToDevice);
    } else if (e == cudaSuccess && c->fv_dy) {
        cudaFree(c->fv_dy);
        c->fv_dy = nullptr;
    }
    delete[] dy_host;
    if (e != cudaSuccess) {
        snprintf(c->err, sizeof(c->err), "CUDA: %s", cudaGetErrorString(e));
        return TVLBM_ECUDA;
    }
    c->fv_exact = exact ? 1 : 0;
    c->fv_nr_iters = exact ? nr_iters : 0;
    return TVLBM_OK;
}
