// Kernel bodies, instantiated per velocity set by tvlbm_kernels_q{3,4,6}.cu.
#pragma once

#include "tvlbm_kernels.cuh"
#include "tvlbm_reduce.cuh"
#include "tvlbm_strip.cuh"
#include "tvlbm_tiled.cuh"

namespace tvlbm {

// =============================================================================================
// Plain sweep: one thread per fluid cell, gathers straight from global memory.
// For velocity l = (i, j) with shift x_i dt = sh_i + a_i (and likewise along y), destination
// (x, y) pulls from the four cells it is overlapped by:
//   s~ = (1-a_y)[(1-a_x) f(x-sh_i, y-sh_j) + a_x f(x-sh_i-1, y-sh_j)]
//      +    a_y [(1-a_x) f(x-sh_i, y-sh_j-1) + a_x f(x-sh_i-1, y-sh_j-1)]
// (the area of the shifted source square inside the destination square).  Periodic images
// and wall ghost rows live in the stored frame, so no index wraps here.
// =============================================================================================
// ROWS: the launch has a per-row deviation reference (chosen at launch, as for the tiled form).
template <int N1, class C, bool ROWS>
__global__ void __launch_bounds__(256) sweep_plain_kernel(const typename C::T* __restrict__ fin,
                                                          typename C::T* __restrict__ fout, const KParams p) {
    using R = typename C::R;
    using T = typename C::T;
    constexpr int Q = N1 * N1;
    pdl_launch_dependents();
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    pdl_wait();  // the previous step's populations are complete from here on
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
            const T* b = fin + (long long)(i + N1 * j) * p.plane + (long long)ys * p.pitch + xs;
            const R v00 = C::ld(b), v01 = C::ld(b - 1);
            const R v10 = C::ld(b - p.pitch), v11 = C::ld(b - p.pitch - 1);
            const R r0 = fma(ax, v01 - v00, split_rest<C>(p, i + N1 * j, v00));
            const R r1 = fma(ax, v11 - v10, split_rest<C>(p, i + N1 * j, v10));
            s[i + N1 * j] = fma(ay, r1 - r0, r0);
        }
    }
    const Geom g = geom_of(p);
    collide_cell<N1, C, ROWS>(s, p, g, y);
    store_collided<N1, C>(fout, g, x, y, s);
}

// =============================================================================================
// Initialisation to the equilibrium of host-given FP64 fields (FP64 arithmetic).
// fields = [rho | ux | uy | T], each [ny][nx].
// =============================================================================================
template <int N1, class C>
__global__ void init_kernel(const double* __restrict__ fields, typename C::T* __restrict__ f, const KParams p) {
    constexpr int Q = N1 * N1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const long long c = (long long)y * p.nx + x, n = (long long)p.nx * p.ny;
    const double rho = fields[c], ux = fields[n + c], uy = fields[2 * n + c], T = fields[3 * n + c];
    double eq[Q];
    if (p.rowd) {
        double pref[Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) pref[l] = ld_row(p.rowd + (long long)(y + HY) * kRowD + l);
        cell_equilibrium<N1, C::dev, double>(p, rho, ux, uy, T - 1.0, eq, pref);
    } else {
        cell_equilibrium<N1, C::dev, double>(p, rho, ux, uy, T - 1.0, eq);
    }
#pragma unroll
    const Geom g = geom_of(p);
#pragma unroll
    for (int l = 0; l < Q; ++l) store_with_images(f, g, (long long)l * p.plane, x, y, C::enc((typename C::R)eq[l]));
}

// =============================================================================================
// Macroscopic fields of the stored state, FP64.  out4 = [rho | ux | uy | T], each [ny][nx].
// =============================================================================================
template <int N1, class C>
__global__ void moments_kernel(const typename C::T* __restrict__ f, double* __restrict__ out4, const KParams p) {
    constexpr int Q = N1 * N1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    double s[Q];
#pragma unroll
    for (int l = 0; l < Q; ++l) s[l] = (double)C::ld(f + sidx(p, l, x, y));
    double rho, ux, uy, th;
    if (p.rowd) {
        double ref4[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) ref4[k] = ld_row(p.rowd + (long long)(y + HY) * kRowD + kMaxQ + k);
        cell_moments<N1, C::dev, double>(s, p, rho, ux, uy, th, ref4);
    } else {
        cell_moments<N1, C::dev, double>(s, p, rho, ux, uy, th);
    }
    const long long c = (long long)y * p.nx + x, n = (long long)p.nx * p.ny;
    out4[c] = rho;
    out4[n + c] = ux;
    out4[2 * n + c] = uy;
    out4[3 * n + c] = 1.0 + th;
}

// =============================================================================================
// Diffuse-reflection walls through ghost rows (Eq. IMPOSITION).
// M_out(x): what the gather would move into the rows beyond the wall for the outgoing
// velocities (c.n > 0, n the wall's outward normal), counting only fluid sources.  Every
// incoming ghost row of column x then holds A(x) f_eq_l(1, u_w, T_w) with
// A = M_out / sum_in |c_y dt| f_eq_l, so a uniform ghost column re-emits exactly M_out.
// Columns of the x-frame are filled too (periodic images).
// A block covers 32 output columns of one wall with one thread per (column, outgoing velocity):
// each sums its velocity's share of M_out (unrolled, so its few loads are in flight together),
// the column's shares are added in a fixed order in shared memory, and the same threads then
// write the incoming velocities' ghost rows (by mirror symmetry there are as many).
// =============================================================================================
template <int N1>
__host__ __device__ constexpr int wall_lanes() { return (N1 / 2) * N1; }  // outgoing (= incoming) velocities per wall

template <int N1, class C>
__global__ void __launch_bounds__(32 * wall_lanes<N1>()) wall_kernel(typename C::T* __restrict__ f, const KParams p) {
    using R = typename C::R;
    constexpr int H = N1 / 2, NL = wall_lanes<N1>();
    __shared__ R part[NL][32];
    __shared__ R amp[32];
    // launched while the previous sweep drains: let the sweep after this kernel be scheduled,
    // then wait until the previous one is complete before reading the populations it wrote
    pdl_launch_dependents();
    pdl_wait();
    const int tx = threadIdx.x, k = threadIdx.y;
    const int side = blockIdx.y;                 // 0: wall at y = -1/2, 1: wall at y = ny - 1/2
    const int xo = blockIdx.x * 32 + tx - FILL;  // output column, in [-FILL, nx + FILL)
    const bool col = xo < p.nx + FILL;
    const int x = ((xo % p.nx) + p.nx) % p.nx;
    const int i = k % N1, jj = k / N1;
    const R rho0 = krho0<R>(p);
    {
        // nodes ascend, so the H lowest y-nodes move towards the wall at y = -1/2
        const int j = side == 0 ? jj : N1 - 1 - jj;
        const int l = i + N1 * j;
        const R ay = ka<R>(p, j), ax = ka<R>(p, i), w = kw<R>(p, i) * kw<R>(p, j);
        R acc = 0;
        if (col) {
#pragma unroll
            for (int d = 1; d <= HY; ++d) {
                const int yd = side == 0 ? -d : p.ny - 1 + d;
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int ys = yd - p.sh[j] - q;
                    if (ys < 0 || ys >= p.ny) continue;  // beyond the wall: no mass
                    const R wy = q ? ay : R(1) - ay;
                    const R ref = rho0 + kPrefRow<R>(p, l, ys);
#pragma unroll
                    for (int pp = 0; pp < 2; ++pp) {
                        const int xs = x - p.sh[i] - pp;
                        const R wx = pp ? ax : R(1) - ax;
                        acc += wx * wy * to_f<C, R>(C::ld(f + sidx(p, l, xs, ys)), w, ref);
                    }
                }
            }
        }
        part[k][tx] = acc;
    }
    __syncthreads();
    if (k == 0) {
        R m = 0;
        for (int kk = 0; kk < NL; ++kk) m += part[kk][tx];
        amp[tx] = m * kinvden<R>(p, side);
    }
    __syncthreads();
    if (!col) return;
    const int j = side == 0 ? N1 - 1 - jj : jj;  // the incoming velocity of this lane
    const int l = i + N1 * j;
    const R w = kw<R>(p, i) * kw<R>(p, j);
    const R fw = amp[tx] * kfeqw<R>(p, side, l);
#pragma unroll
    for (int d = 1; d <= HY; ++d) {
        const int yd = side == 0 ? -d : p.ny - 1 + d;
        f[sidx(p, l, xo, yd)] = C::enc(from_f<C, R>(fw, w, rho0 + kPrefRow<R>(p, l, yd)));
    }
}

// =============================================================================================
// Refresh the periodic frame from the interior (after raw population uploads).
// =============================================================================================
template <class T>
__global__ void halo_kernel(T* __restrict__ f, const KParams p, int Q) {
    const int fx = p.nx + 2 * FILL, fy = p.walls ? p.ny : p.ny + 2 * FILL;
    const long long per = (long long)fx * fy;
    for (long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x; t < per * Q;
         t += (long long)gridDim.x * blockDim.x) {
        const int l = (int)(t / per);
        const long long r = t - (long long)l * per;
        const int yy = (int)(r / fx) - (p.walls ? 0 : FILL);
        const int xx = (int)(r % fx) - FILL;
        if (xx >= 0 && xx < p.nx && yy >= 0 && yy < p.ny) continue;
        const int x = ((xx % p.nx) + p.nx) % p.nx, y = ((yy % p.ny) + p.ny) % p.ny;
        f[sidx(p, l, xx, yy)] = f[sidx(p, l, x, y)];
    }
}

// d_l += delta[r][l] on every stored element (fluid and frame, stored row r) of a
// deviation-coded buffer: one 16-byte vector of a row per thread (the pitch and the plane are
// multiples of 32 elements, so vectors are aligned and never cross a row); grid (pitch / (256 V),
// <= 65535 row blocks striding over the rows, Q).
template <class C>
__global__ void __launch_bounds__(256) reencode_kernel(typename C::T* __restrict__ f, long long plane, int pitch,
                                                       int rows, const float* __restrict__ delta) {
    using T = typename C::T;
    constexpr int V = 16 / (int)sizeof(T);
    const int xv = blockIdx.x * blockDim.x + threadIdx.x, l = blockIdx.z;
    if (xv * V >= pitch) return;
    for (int r = blockIdx.y; r < rows; r += gridDim.y) {
        T* q = f + (long long)l * plane + (long long)r * pitch + (long long)xv * V;
        const float d = __ldg(delta + (long long)r * kMaxQ + l);
        uint4 u = *reinterpret_cast<const uint4*>(q);
        T* e = reinterpret_cast<T*>(&u);
#pragma unroll
        for (int k = 0; k < V; ++k) e[k] = C::enc(lds<C>(reinterpret_cast<const unsigned char*>(e + k)) + d);
        *reinterpret_cast<uint4*>(q) = u;
    }
}

// Decode one velocity plane to FP64 f_l (packed [ny][nx]) / encode FP64 f_l into storage.
template <class C>
__global__ void decode_plane_kernel(const typename C::T* __restrict__ f, int l, int n1, double* __restrict__ out,
                                    const KParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const double w = p.wd[l % n1] * p.wd[l / n1];
    out[(long long)y * p.nx + x] = to_f<C, double>((double)C::ld(f + sidx(p, l, x, y)), w, p.rho0d + kPrefRow<double>(p, l, y));
}
template <class C>
__global__ void encode_plane_kernel(typename C::T* __restrict__ f, int l, int n1, const double* __restrict__ in,
                                    const KParams p) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    const double w = p.wd[l % n1] * p.wd[l / n1];
    f[sidx(p, l, x, y)] =
        C::enc((typename C::R)from_f<C, double>(in[(long long)y * p.nx + x], w, p.rho0d + kPrefRow<double>(p, l, y)));
}

// =============================================================================================
// Per-row deviation reference of a channel.
// =============================================================================================
// Row averages of (u_x, u_y, T) of the stored state, prof = [ux | uy | T][ny]: one block of 256
// threads per fluid row, cell moments in the storage's arithmetic (any profile is an exact
// encoding, so the reference needs no more), sums in FP64 in a fixed order.
template <int N1, class C>
__global__ void __launch_bounds__(256) row_means_kernel(const typename C::T* __restrict__ f, double* __restrict__ prof,
                                                        const KParams p) {
    constexpr int Q = N1 * N1;
    using R = typename C::R;
    __shared__ double sh[3][256];
    const int y = blockIdx.x, t = threadIdx.x;
    const bool rows = p.rowd != nullptr;
    R ref4[4] = {R(0), R(0), R(0), R(0)};
    if (rows)
        for (int k = 0; k < 4; ++k) ref4[k] = (R)ld_row(p.rowd + (long long)(y + HY) * kRowD + kMaxQ + k);
    double acc[3] = {0.0, 0.0, 0.0};
    for (int x = t; x < p.nx; x += blockDim.x) {
        R v[Q];
#pragma unroll
        for (int l = 0; l < Q; ++l) v[l] = C::ld(f + sidx(p, l, x, y));
        R rho, ux, uy, th;
        if (rows) cell_moments<N1, C::dev, R>(v, p, rho, ux, uy, th, ref4);
        else cell_moments<N1, C::dev, R>(v, p, rho, ux, uy, th);
        acc[0] += (double)ux;
        acc[1] += (double)uy;
        acc[2] += 1.0 + (double)th;
    }
#pragma unroll
    for (int k = 0; k < 3; ++k) sh[k][t] = acc[k];
    __syncthreads();
    for (int h = 128; h > 0; h >>= 1) {
        if (t < h)
#pragma unroll
            for (int k = 0; k < 3; ++k) sh[k][t] += sh[k][t + h];
        __syncthreads();
    }
    if (t < 3) prof[(long long)t * p.ny + y] = sh[t][0] / p.nx;
}

// Reference entries of every stored row r (fluid row y = r - HY clamped into the fluid; a row
// whose profile is not a valid state takes the default reference): Pref_l = f_eq_l(rho0, u, T) /
// w_l - rho0, jref, eref in FP64; jref, eref and refD (the float Pref's share of the FP32 constants'
// defects, as for the single reference) in the float table.  One thread per row.
template <int N1>
__global__ void ref_rows_kernel(const double* __restrict__ prof, double* __restrict__ rowd, float* __restrict__ rowf,
                                const KParams p) {
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= p.rows) return;
    const int y = min(max(r - HY, 0), p.ny - 1);
    double ux = prof[y], uy = prof[p.ny + y], T = prof[2 * p.ny + y];
    if (!(T > 0.0) || !isfinite(T) || !isfinite(ux) || !isfinite(uy)) {
        ux = 0.0;
        uy = 0.0;
        T = 1.0;
    }
    double eq[N1 * N1];
    cell_equilibrium<N1, false, double>(p, p.rho0d, ux, uy, T - 1.0, eq);
    double* d = rowd + (long long)r * kRowD;
    float* fr = rowf + (long long)r * kRowF;
    double m = 0.0, mx = 0.0, my = 0.0, me = 0.0;
    for (int j = 0; j < N1; ++j)
        for (int i = 0; i < N1; ++i) {
            const int l = i + N1 * j;
            const double pr = eq[l] / (p.wd[i] * p.wd[j]) - p.rho0d;
            d[l] = pr;
            const double v = (double)(float)pr;
            m += (double)p.wf[i] * p.wf[j] * v;
            mx += (double)p.wxf[i] * p.wf[j] * v;
            my += (double)p.wf[i] * p.wxf[j] * v;
            me += ((double)p.wx2f[i] * p.wf[j] + (double)p.wf[i] * p.wx2f[j]) * v;
        }
    d[kMaxQ] = p.rho0d * ux;
    d[kMaxQ + 1] = p.rho0d * uy;
    d[kMaxQ + 2] = p.rho0d * (2.0 * (T - 1.0) + ux * ux + uy * uy);
    d[kMaxQ + 3] = 0.0;  // an equilibrium of density rho0: no mass beyond rho0
    fr[kRowJ] = (float)d[kMaxQ];
    fr[kRowJ + 1] = (float)d[kMaxQ + 1];
    fr[kRowE] = (float)d[kMaxQ + 2];
    fr[kRowRD] = (float)(-m);
    fr[kRowRD + 1] = (float)(-(mx - (double)fr[kRowJ]));
    fr[kRowRD + 2] = (float)(-(my - (double)fr[kRowJ + 1]));
    fr[kRowRD + 3] = (float)(-(me - (double)fr[kRowE]));
}

// Row averages of the stored populations themselves, per velocity: prof[l][y] = mean over x of
// Pref_l(y) + d_l(x, y), i.e. of f_l / w_l - rho0 (the reference the "mean" kind installs).  One
// block of 128 threads per (fluid row, velocity): 16-byte vector loads of the row, FP32 partial
// sums in a fixed order (any reference is an exact re-encoding, so FP32 means suffice), a
// warp-shuffle and shared-memory tree.
template <int N1, class C>
__global__ void __launch_bounds__(128) row_pop_means_kernel(const typename C::T* __restrict__ f, double* __restrict__ prof,
                                                            const KParams p) {
    using T = typename C::T;
    constexpr int V = 16 / (int)sizeof(T);
    __shared__ float sh[4];
    const int y = blockIdx.x, l = blockIdx.y, t = threadIdx.x;
    const T* row = f + sidx(p, l, 0, y);  // 32-byte aligned (hx columns of frame, pitch a multiple of 32)
    float acc = 0.f;
    const int nv = p.nx / V;
    for (int v = t; v < nv; v += blockDim.x) {
        const uint4 u = __ldg(reinterpret_cast<const uint4*>(row) + v);
        const T* e = reinterpret_cast<const T*>(&u);
#pragma unroll
        for (int k = 0; k < V; ++k) acc += lds<C>(reinterpret_cast<const unsigned char*>(e + k));
    }
    for (int x = nv * V + t; x < p.nx; x += blockDim.x) acc += (float)C::ld(row + x);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((t & 31) == 0) sh[t >> 5] = acc;
    __syncthreads();
    if (t == 0) prof[(long long)l * p.ny + y] = kPrefRow<double>(p, l, y) + (double)((sh[0] + sh[1]) + (sh[2] + sh[3])) / p.nx;
}

// Reference entries of every stored row r from a per-velocity profile prof[l][y] of Pref (fluid
// row y = r - HY clamped into the fluid; a row with a non-finite entry takes the default
// reference): Pref_l, and the reference's moments beyond the rest state rho0 w in FP64 with the
// exact weights, jref = sum w c Pref, eref = sum w |c|^2 Pref, rref = sum w Pref (a general
// reference need not have density rho0); jref, eref and refD in the float table as in
// ref_rows_kernel, refD's mass entry against rref.  One block of 64 threads per row, thread l
// holding velocity l; the sums in a fixed shared-memory order.
template <int N1>
__global__ void __launch_bounds__(64) ref_rows_mean_kernel(const double* __restrict__ prof, double* __restrict__ rowd,
                                                           float* __restrict__ rowf, const KParams p) {
    constexpr int Q = N1 * N1;
    __shared__ double part[8][64];
    __shared__ int bad;
    const int r = blockIdx.x, l = threadIdx.x;
    const int y = min(max(r - HY, 0), p.ny - 1);
    if (l == 0) bad = 0;
    __syncthreads();
    const double v = l < Q ? prof[(long long)l * p.ny + y] : 0.0;
    if (l < Q && !isfinite(v)) atomicOr(&bad, 1);
    __syncthreads();
    const double pr = (l < Q && !bad) ? v : 0.0;
    double* d = rowd + (long long)r * kRowD;
    float* fr = rowf + (long long)r * kRowF;
    if (l < Q) d[l] = pr;
    double c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    if (l < Q) {
        const int i = l % N1, j = l / N1;
        const double w = p.wd[i] * p.wd[j];
        c[0] = w * pr;
        c[1] = w * p.xd[i] * pr;
        c[2] = w * p.xd[j] * pr;
        c[3] = w * (p.xd[i] * p.xd[i] + p.xd[j] * p.xd[j]) * pr;
        const double vf = (double)(float)pr;
        c[4] = (double)p.wf[i] * p.wf[j] * vf;
        c[5] = (double)p.wxf[i] * p.wf[j] * vf;
        c[6] = (double)p.wf[i] * p.wxf[j] * vf;
        c[7] = ((double)p.wx2f[i] * p.wf[j] + (double)p.wf[i] * p.wx2f[j]) * vf;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) part[k][l] = c[k];
    __syncthreads();
    for (int h = 32; h > 0; h >>= 1) {
        if (l < h)
#pragma unroll
            for (int k = 0; k < 8; ++k) part[k][l] += part[k][l + h];
        __syncthreads();
    }
    if (l == 0) {
        const double rr = part[0][0], jx = part[1][0], jy = part[2][0], e = part[3][0];
        d[kMaxQ] = jx;
        d[kMaxQ + 1] = jy;
        d[kMaxQ + 2] = e;
        d[kMaxQ + 3] = rr;
        fr[kRowJ] = (float)jx;
        fr[kRowJ + 1] = (float)jy;
        fr[kRowE] = (float)e;
        fr[kRowRD] = (float)(-(part[4][0] - rr));
        fr[kRowRD + 1] = (float)(-(part[5][0] - (double)fr[kRowJ]));
        fr[kRowRD + 2] = (float)(-(part[6][0] - (double)fr[kRowJ + 1]));
        fr[kRowRD + 3] = (float)(-(part[7][0] - (double)fr[kRowE]));
    }
}

// Gather shift of every fluid row from the FP64 Pref table (the sources of row y lie within FILL
// rows of it): C_l = (1 - omega) S_l - omega Pref_l and the FP32-constant moments of float(S), the
// mass entry with the row reference's rref added.  Ghost rows collide nowhere and get zeros.  One
// block of 64 threads per stored row, thread l holding velocity l; the moments summed in a fixed
// shared-memory order.
template <int N1>
__global__ void __launch_bounds__(64) ref_shift_kernel(const double* __restrict__ rowd, float* __restrict__ rowf,
                                                       const KParams p) {
    constexpr int Q = N1 * N1;
    __shared__ double part[4][64];
    const int r = blockIdx.x, l = threadIdx.x;
    const int y = r - HY;
    float* fr = rowf + (long long)r * kRowF;
    if (y < 0 || y >= p.ny) {
        if (l < kMaxQ) fr[l] = 0.0f;
        if (l < 4) fr[kRowSM + l] = 0.0f;
        return;
    }
    double c[4] = {0, 0, 0, 0};
    if (l < Q) {
        const int i = l % N1, j = l / N1;
        const double om = (double)p.omegaf;
        const double a = p.ad[j];
        const double r0 = rowd[(long long)(y - p.sh[j] + HY) * kRowD + l];
        const double r1 = rowd[(long long)(y - p.sh[j] - 1 + HY) * kRowD + l];
        const double self = rowd[(long long)r * kRowD + l];
        const double S = (1.0 - a) * r0 + a * r1 - self;
        fr[row_slot(N1, l)] = (float)((1.0 - om) * S - om * self);
        const double v = (double)(float)S;
        c[0] = (double)p.wf[i] * p.wf[j] * v;
        c[1] = (double)p.wxf[i] * p.wf[j] * v;
        c[2] = (double)p.wf[i] * p.wxf[j] * v;
        c[3] = ((double)p.wx2f[i] * p.wf[j] + (double)p.wf[i] * p.wx2f[j]) * v;
    } else if (l < kMaxQ) {
        fr[l] = 0.0f;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) part[k][l] = c[k];
    __syncthreads();
    for (int h = 32; h > 0; h >>= 1) {
        if (l < h)
#pragma unroll
            for (int k = 0; k < 4; ++k) part[k][l] += part[k][l + h];
        __syncthreads();
    }
    if (l == 0) {
        // the row reference's own mass beyond rho0 (zero for an equilibrium reference) joins the
        // shift's: the collision's rho - rho0 is their sum plus the gathered deviations' mass
        fr[kRowSM] = (float)(part[0][0] + rowd[(long long)r * kRowD + kMaxQ + 3]);
        fr[kRowSM + 1] = (float)part[1][0];
        fr[kRowSM + 2] = (float)part[2][0];
        fr[kRowSM + 3] = (float)part[3][0];
    }
}

// =============================================================================================
// Host-side launchers for one N1.
// =============================================================================================
template <int N1>
struct Launch {
    static dim3 grid2d(const KParams& p, dim3 b) { return dim3((p.nx + b.x - 1) / b.x, (p.ny + b.y - 1) / b.y); }

    template <class C>
    static cudaError_t sweep_c(int form, int cfg, const void* fin, void* fout, const SweepMaps* maps, const KParams& p,
                               cudaStream_t s) {
        using T = typename C::T;
        if (form == FORM_TILED) return tiled_sweep<N1, C>(cfg, maps, (T*)fout, p, s);
        if (form == FORM_STRIP) return strip_sweep<N1, C>(maps, (T*)fout, p, s);
        const dim3 b(32, 8);
        if constexpr (C::dev) {
            if (p.rowf) return launch_pdl(sweep_plain_kernel<N1, C, true>, grid2d(p, b), b, 0, s, (const T*)fin, (T*)fout, p);
        }
        return launch_pdl(sweep_plain_kernel<N1, C, false>, grid2d(p, b), b, 0, s, (const T*)fin, (T*)fout, p);
    }
    template <class C>
    static cudaError_t init_c(const double* fields, void* f, const KParams& p, cudaStream_t s) {
        const dim3 b(32, 8);
        init_kernel<N1, C><<<grid2d(p, b), b, 0, s>>>(fields, (typename C::T*)f, p);
        return cudaGetLastError();
    }
    template <class C>
    static cudaError_t moments_c(const void* f, double* out4, const KParams& p, cudaStream_t s) {
        const dim3 b(32, 8);
        moments_kernel<N1, C><<<grid2d(p, b), b, 0, s>>>((const typename C::T*)f, out4, p);
        return cudaGetLastError();
    }
    template <class C>
    static cudaError_t reduce_c(const void* f, double* partials, double* out5, const KParams& p, cudaStream_t s) {
        reduce_kernel<N1, C><<<kRedBlocks, 256, 0, s>>>((const typename C::T*)f, partials, p);
        reduce_final_kernel<<<1, 256, 0, s>>>(partials, out5);
        return cudaGetLastError();
    }
    template <class C>
    static cudaError_t wall_c(void* f, const KParams& p, cudaStream_t s) {
        const dim3 grid((p.nx + 2 * FILL + 31) / 32, 2), block(32, wall_lanes<N1>());
        return launch_pdl(wall_kernel<N1, C>, grid, block, 0, s, (typename C::T*)f, p);
    }
    template <class C>
    static cudaError_t halo_c(void* f, const KParams& p, cudaStream_t s) {
        halo_kernel<typename C::T><<<1024, 256, 0, s>>>((typename C::T*)f, p, N1 * N1);
        return cudaGetLastError();
    }
    template <class C>
    static cudaError_t reencode_c(void* f, const float* delta, const KParams& p, cudaStream_t s) {
        if constexpr (!C::dev) return cudaErrorInvalidValue;
        constexpr int V = 16 / (int)sizeof(typename C::T);
        const dim3 grid((p.pitch / V + 255) / 256, p.rows < 65535 ? p.rows : 65535, N1 * N1);
        reencode_kernel<C><<<grid, 256, 0, s>>>((typename C::T*)f, p.plane, p.pitch, p.rows, delta);
        return cudaGetLastError();
    }
    template <class C>
    static cudaError_t decode_c(const void* f, int l, double* out, const KParams& p, cudaStream_t s) {
        const dim3 b(32, 8);
        decode_plane_kernel<C><<<grid2d(p, b), b, 0, s>>>((const typename C::T*)f, l, N1, out, p);
        return cudaGetLastError();
    }
    template <class C>
    static cudaError_t encode_c(void* f, int l, const double* in, const KParams& p, cudaStream_t s) {
        const dim3 b(32, 8);
        encode_plane_kernel<C><<<grid2d(p, b), b, 0, s>>>((typename C::T*)f, l, N1, in, p);
        return cudaGetLastError();
    }

#define TVLBM_DISPATCH(call, args)                              \
    switch (storage) {                                          \
        case ST_FP64: return call<CodecF64> args;               \
        case ST_FP32: return call<CodecF32> args;               \
        case ST_BF16_DEV: return call<CodecBF16Dev> args;       \
        case ST_FP16_DEV: return call<CodecF16Dev> args;        \
        case ST_FP32_DEV: return call<CodecF32Dev> args;        \
        default: return cudaErrorInvalidValue;                  \
    }

    static cudaError_t sweep(int storage, int form, int cfg, const void* fin, void* fout, const SweepMaps* maps,
                             const KParams& p, cudaStream_t s) {
        TVLBM_DISPATCH(sweep_c, (form, cfg, fin, fout, maps, p, s))
    }
    static cudaError_t init(int storage, const double* fields, void* f, const KParams& p, cudaStream_t s) {
        TVLBM_DISPATCH(init_c, (fields, f, p, s))
    }
    static cudaError_t moments(int storage, const void* f, double* out4, const KParams& p, cudaStream_t s) {
        TVLBM_DISPATCH(moments_c, (f, out4, p, s))
    }
    static cudaError_t reduce(int storage, const void* f, double* partials, double* out5, const KParams& p, cudaStream_t s) {
        TVLBM_DISPATCH(reduce_c, (f, partials, out5, p, s))
    }
    static cudaError_t wall(int storage, void* f, const KParams& p, cudaStream_t s) { TVLBM_DISPATCH(wall_c, (f, p, s)) }
    static cudaError_t halo(int storage, void* f, const KParams& p, cudaStream_t s) { TVLBM_DISPATCH(halo_c, (f, p, s)) }
    static cudaError_t decode(int storage, const void* f, int l, double* out, const KParams& p, cudaStream_t s) {
        TVLBM_DISPATCH(decode_c, (f, l, out, p, s))
    }
    static cudaError_t encode(int storage, void* f, int l, const double* in, const KParams& p, cudaStream_t s) {
        TVLBM_DISPATCH(encode_c, (f, l, in, p, s))
    }
    static int tiled_available(int storage) { return tiled_supported<N1>(storage); }
    static void box(int storage, int cfg, int* bx, int* by) {
        switch (storage) {
            case ST_FP64: tiled_box<N1, CodecF64>(cfg, bx, by); break;
            case ST_FP32: tiled_box<N1, CodecF32>(cfg, bx, by); break;
            case ST_BF16_DEV: tiled_box<N1, CodecBF16Dev>(cfg, bx, by); break;
            case ST_FP16_DEV: tiled_box<N1, CodecF16Dev>(cfg, bx, by); break;
            default: tiled_box<N1, CodecF32Dev>(cfg, bx, by); break;
        }
    }
    static void shape(int storage, int cfg, int* tx, int* ty, int* r) {
        const int es = storage == ST_FP64 ? 8 : (storage == ST_BF16_DEV || storage == ST_FP16_DEV) ? 2 : 4;
        const TileShape t = tile_shape(N1 * N1, es, cfg);
        *tx = t.tx;
        *ty = t.ty;
        *r = t.ty / t.rs;
    }
    static cudaError_t reencode(int storage, void* f, const float* delta, const KParams& p, cudaStream_t s) {
        TVLBM_DISPATCH(reencode_c, (f, delta, p, s))
    }
    template <class C>
    static cudaError_t row_means_c(const void* f, double* prof, const KParams& p, cudaStream_t s) {
        row_means_kernel<N1, C><<<p.ny, 256, 0, s>>>((const typename C::T*)f, prof, p);
        return cudaGetLastError();
    }
    static cudaError_t row_means(int storage, const void* f, double* prof, const KParams& p, cudaStream_t s) {
        TVLBM_DISPATCH(row_means_c, (f, prof, p, s))
    }
    template <class C>
    static cudaError_t row_pop_means_c(const void* f, double* prof, const KParams& p, cudaStream_t s) {
        if constexpr (!C::dev) return cudaErrorInvalidValue;
        row_pop_means_kernel<N1, C><<<dim3(p.ny, N1 * N1), 128, 0, s>>>((const typename C::T*)f, prof, p);
        return cudaGetLastError();
    }
    static cudaError_t row_pop_means(int storage, const void* f, double* prof, const KParams& p, cudaStream_t s) {
        TVLBM_DISPATCH(row_pop_means_c, (f, prof, p, s))
    }
    static cudaError_t ref_tables(const double* prof, double* rowd, float* rowf, const KParams& p, cudaStream_t s) {
        const int blocks = (p.rows + 127) / 128;
        ref_rows_kernel<N1><<<blocks, 128, 0, s>>>(prof, rowd, rowf, p);
        ref_shift_kernel<N1><<<p.rows, 64, 0, s>>>(rowd, rowf, p);
        return cudaGetLastError();
    }
    static cudaError_t ref_tables_mean(const double* prof, double* rowd, float* rowf, const KParams& p, cudaStream_t s) {
        ref_rows_mean_kernel<N1><<<p.rows, 64, 0, s>>>(prof, rowd, rowf, p);
        ref_shift_kernel<N1><<<p.rows, 64, 0, s>>>(rowd, rowf, p);
        return cudaGetLastError();
    }
    static cudaError_t flow(int storage, int cfg, const FlowSrc& src, const KParams& p, cudaStream_t s) {
        switch (storage) {
            case ST_FP64: return flow_sweep<N1, CodecF64>(cfg, src, p, s);
            case ST_FP32: return flow_sweep<N1, CodecF32>(cfg, src, p, s);
            case ST_BF16_DEV: return flow_sweep<N1, CodecBF16Dev>(cfg, src, p, s);
            case ST_FP16_DEV: return flow_sweep<N1, CodecF16Dev>(cfg, src, p, s);
            case ST_FP32_DEV: return flow_sweep<N1, CodecF32Dev>(cfg, src, p, s);
            default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t batch_flow(int storage, int cfg, const BatchFlowSrc& src, const KParams& p, cudaStream_t s) {
        switch (storage) {
            case ST_FP64: return flow_sweep<N1, CodecF64>(cfg, src, p, s);
            case ST_FP32: return flow_sweep<N1, CodecF32>(cfg, src, p, s);
            case ST_BF16_DEV: return flow_sweep<N1, CodecBF16Dev>(cfg, src, p, s);
            case ST_FP16_DEV: return flow_sweep<N1, CodecF16Dev>(cfg, src, p, s);
            case ST_FP32_DEV: return flow_sweep<N1, CodecF32Dev>(cfg, src, p, s);
            default: return cudaErrorInvalidValue;
        }
    }
    static cudaError_t batch(int storage, int cfg, const BatchSrc& src, const KParams& p, cudaStream_t s) {
        switch (storage) {
            case ST_FP64: return batch_sweep<N1, CodecF64>(cfg, src, p, s);
            case ST_FP32: return batch_sweep<N1, CodecF32>(cfg, src, p, s);
            case ST_BF16_DEV: return batch_sweep<N1, CodecBF16Dev>(cfg, src, p, s);
            case ST_FP16_DEV: return batch_sweep<N1, CodecF16Dev>(cfg, src, p, s);
            case ST_FP32_DEV: return batch_sweep<N1, CodecF32Dev>(cfg, src, p, s);
            default: return cudaErrorInvalidValue;
        }
    }
#undef TVLBM_DISPATCH

    static const KernelTable* table() {
        static const KernelTable t = {&sweep, &init, &moments, &reduce, &wall, &halo, &decode, &encode, &tiled_available,
                                      &box, &shape, &reencode, &flow, &batch, &batch_flow, &row_means, &ref_tables,
                                      &row_pop_means, &ref_tables_mean};
        return &t;
    }
};

}  // namespace tvlbm
