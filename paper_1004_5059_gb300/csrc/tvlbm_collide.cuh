// Collision for the deviation-storage codecs in FP32: moments -> Hermite equilibrium -> BGK,
// on d_l = f_l / w_l - rho0, using the mirror symmetry of Gauss-Hermite nodes (x_{n-1-i} = -x_i,
// w_{n-1-i} = w_i) and with the relaxation folded into the equilibrium evaluation:
//     d*_ij = (1 - omega) d_ij + omega d_eq_ij,
//     omega d_eq_ij = A_i + B_j + sum_{a=1}^{N-1} X'_ia P_j,N-a          (N + 1 operations),
// where, with X_ia = h_a(u_x) E_ia, P_jk = sum_{1<=b<=k} h_b(u_y) E_jb, SX_i = sum_{a>=1} X_ia:
//     X'_ia = omega rho X_ia,  A_i = omega rho SX_i - omega c_i,
//     B_j  = omega rho P_jN - omega c_j + omega (rho - rho0 - A0),
// and (A0, c_i, c_j) the first-order correction that cancels the defects of the float tables
// (see cell_equilibrium in tvlbm_kernels.cuh for the derivation; the constants here are the
// pre-multiplied products w_i x_i and w_i x_i^2 the moment sums use, and the host evaluates
// the defects for exactly those constants).
// Host-callable so a CPU harness can compare it with the generic path.
#pragma once

#include "tvlbm_kernels.cuh"

namespace tvlbm {

template <int N1>
__host__ __device__ __forceinline__ void cell_collide_dev(float (&s)[N1 * N1], const KParams& p) {
    constexpr int N = N1 - 1, H = N1 / 2;
    constexpr bool ODD = (N1 & 1) != 0;
    // ---- moments: rho = rho0 + sum w d, rho u = sum w c d, sum w |c|^2 d --------------------
    float rr[N1], rx[N1], rxx[N1];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        float r = 0.f, x1 = 0.f, x2 = 0.f;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const int m = N1 - 1 - i;
            const float a = s[i + N1 * j] + s[m + N1 * j];
            const float b = s[i + N1 * j] - s[m + N1 * j];
            r = fmaf(p.wf[i], a, r);
            x1 = fmaf(p.wxf[i], b, x1);
            x2 = fmaf(p.wx2f[i], a, x2);
        }
        if (ODD) r = fmaf(p.wf[H], s[H + N1 * j], r);
        rr[j] = r;
        rx[j] = x1;
        rxx[j] = x2;
    }
    float m0 = 0.f, mx = 0.f, my = 0.f, me = 0.f;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const int m = N1 - 1 - j;
        const float a = rr[j] + rr[m], b = rr[j] - rr[m];
        m0 = fmaf(p.wf[j], a, m0);
        my = fmaf(p.wxf[j], b, my);
        mx = fmaf(p.wf[j], rx[j] + rx[m], mx);
        me = fmaf(p.wx2f[j], a, fmaf(p.wf[j], rxx[j] + rxx[m], me));
    }
    if (ODD) {
        m0 = fmaf(p.wf[H], rr[H], m0);
        mx = fmaf(p.wf[H], rx[H], mx);
        me = fmaf(p.wf[H], rxx[H], me);
    }
    const float rho = p.rho0f + m0;
    const float inv = 1.0f / rho;
    const float ux = mx * inv, uy = my * inv;
    const float th = 0.5f * ((me - 2.0f * m0) * inv - (ux * ux + uy * uy));

    // ---- Hermite coefficients of the Maxwellian, per axis ----------------------------------
    float hx[N + 1], hy[N + 1];
    hx[0] = hy[0] = 1.f;
    hx[1] = ux;
    hy[1] = uy;
#pragma unroll
    for (int n = 1; n < N; ++n) {
        hx[n + 1] = fmaf(ux, hx[n], (float)n * th * hx[n - 1]);
        hy[n + 1] = fmaf(uy, hy[n], (float)n * th * hy[n - 1]);
    }

    // ---- first-order cancellation of the table defects -------------------------------------
    float Dm = 2.f * p.dS[0] * m0, De = 2.f * m0 * (p.dV[0] + p.dS[0]);
    float Dx = rho * ux * (p.dU[1] + p.dS[0]), Dy = rho * uy * (p.dU[1] + p.dS[0]);
#pragma unroll
    for (int a = 2; a <= N; a += 2) {  // dS, dV vanish for odd orders (mirror symmetry)
        Dm = fmaf(rho * p.dS[a], hx[a] + hy[a], Dm);
        De = fmaf(rho * (p.dV[a] + p.dS[a]), hx[a] + hy[a], De);
    }
    if (N >= 2) De = fmaf(rho * p.dS[0], hx[2] + hy[2], De);
#pragma unroll
    for (int a = 3; a <= N; a += 2) {  // dU vanishes for even orders
        Dx = fmaf(rho * p.dU[a], hx[a], Dx);
        Dy = fmaf(rho * p.dU[a], hy[a], Dy);
    }
#pragma unroll
    for (int b = 2; b <= N - 1; b += 2) {
        Dx = fmaf(rho * ux * p.dS[b], hy[b], Dx);
        Dy = fmaf(rho * uy * p.dS[b], hx[b], Dy);
    }
#pragma unroll
    for (int b = 2; b <= N - 2; b += 2) De = fmaf(rho * p.dS[b], fmaf(hx[2], hy[b], hy[2] * hx[b]), De);
    const float G = 0.5f * De - Dm;
    const float om = p.omegaf, orho = om * rho;

    // ---- per-node tables: A_i (x part), B_j (y part), X'_ia, P_jk --------------------------
    float A[N1], B[N1], Xp[N1][N > 1 ? N : 1], P[N1][N + 1];
#pragma unroll
    for (int i = 0; i < (ODD ? H + 1 : H); ++i) {
        const int m = N1 - 1 - i;
        float se = 0.f, so = 0.f, pe = 0.f, po = 0.f;
#pragma unroll
        for (int a = 1; a <= N; ++a) {
            const float xa = hx[a] * p.Ef[i][a];
            const float ya = hy[a] * p.Ef[i][a];
            if (a & 1) { so += xa; po += ya; } else { se += xa; pe += ya; }
            P[i][a] = pe + po;
            P[m][a] = pe - po;
            if (a < N) {
                Xp[i][a] = orho * xa;
                Xp[m][a] = (a & 1) ? -Xp[i][a] : Xp[i][a];
            }
        }
        const float cx2 = 0.5f * G * p.x2f[i];
        const float ci = fmaf(Dx, p.xf[i], cx2), cim = fmaf(-Dx, p.xf[i], cx2);
        const float cj = fmaf(Dy, p.xf[i], cx2), cjm = fmaf(-Dy, p.xf[i], cx2);
        A[i] = fmaf(orho, se + so, -om * ci);
        A[m] = fmaf(orho, se - so, -om * cim);
        B[i] = fmaf(orho, P[i][N], -om * cj);
        B[m] = fmaf(orho, P[m][N], -om * cjm);
    }
    const float wdr = om * (m0 - (Dm - G));
    const float keep = 1.f - om;
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        const float bj = B[j] + wdr;
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            float weq = A[i] + bj;
#pragma unroll
            for (int a = 1; a < N; ++a) weq = fmaf(Xp[i][a], P[j][N - a], weq);
            s[i + N1 * j] = fmaf(keep, s[i + N1 * j], weq);
        }
    }
}

}  // namespace tvlbm
