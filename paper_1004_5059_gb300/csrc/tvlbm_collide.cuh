// Collision for the deviation-storage codecs in FP32: moments -> Hermite equilibrium -> BGK,
// on d_l = f_l / w_l - rho0, using the mirror symmetry of Gauss-Hermite nodes (x_{n-1-i} = -x_i,
// w_{n-1-i} = w_i) and with the relaxation folded into the equilibrium evaluation:
//     d*_ij = (1 - omega) d_ij + omega d_eq_ij,
//     omega d_eq_ij = A_i + B_j + sum_{a=1}^{N-1} X'_ia P_j,N-a          (N + 1 operations),
// where, with X_ia = h_a(u_x) E_ia, P_jk = sum_{1<=b<=k} h_b(u_y) E_jb, SX_i = sum_{a>=1} X_ia
// (the separable Hermite equilibrium of cell_equilibrium, d_eq = (rho - rho0) + rho phi - Pref,
// Pref the deviation of the storage reference, subtracted last when it is not zero):
//     X'_ia = omega rho X_ia,  A_i = omega rho SX_i - omega c_i,
//     B_j  = omega rho P_jN - omega c_j + omega (rho - rho0 - (D_m - G)).
//
// Conservation in FP32.  The float constants (w_i, w_i x_i, w_i x_i^2, E_ia) miss the
// quadrature identities they stand for -- sum w = 1, sum w x^2 = 1, sum w E_a = 0 (a >= 1), ... --
// by ~1e-8.  Uncorrected, every collision then creates mass, momentum and energy in proportion
// to the cell's own values, the same way every step: a drift that accumulates.  With the table
// sums S_a = sum_i w_i E_ia, U_a = sum_i (w x)_i E_ia, V_a = sum_i (w x^2)_i E_ia and their
// defects dS_a = S_a - [a=0], dU_a = U_a - [a=1], dV_a = V_a - [a=0] - [a=2] (evaluated exactly
// by the host from the float constants), the moments of d_eq exceed the measured moments by, to
// first order in the defects,
//     D_m = 2 dS_0 m0 + rho sum_{a>=1} dS_a (h^x_a + h^y_a),
//     D_x = rho u_x (dU_1 + dS_0) + rho sum_{a odd>=3} dU_a h^x_a + rho u_x sum_{b even} dS_b h^y_b,
//     D_e = 2 m0 (dV_0 + dS_0) + rho sum_a (dV_a + dS_a)(h^x_a + h^y_a) + rho dS_0 (h^x_2 + h^y_2)
//           + rho sum_b dS_b (h^x_2 h^y_b + h^y_2 h^x_b)
// (D_y like D_x).  Subtracting c = D_m + D_x x_i + D_y x_j + G (x_i^2 + x_j^2 - 2)/2 with
// G = D_e/2 - D_m, whose moments are (D_m, D_x, D_y, D_e) under exact quadrature, cancels the
// drift up to second order.  A non-default storage reference adds the defect of its own float
// table, refD, computed on the host the same way.
#pragma once

#include "tvlbm_kernels.cuh"

namespace tvlbm {

// A row's reference entries: from global memory (read-only path), or, with SH, from a copy the
// CTA staged in shared memory.
template <bool SH>
__device__ __forceinline__ float4 row_ld4(const float* q) {  // q 16-byte aligned
    if constexpr (SH) return *reinterpret_cast<const float4*>(q);
    else return ld_row4(q);
}

// ROW: row points at the cell row's entries of a per-row reference table (KParams::rowf, or its
// shared-memory copy with ROW_SH); s then holds the plain gather of the stored deviations (the
// row's shift enters through its table).  Without ROW, row is unused.
template <int N1, bool ROW, bool ROW_SH = false>
__device__ __forceinline__ void cell_collide_dev(float (&s)[N1 * N1], const KParams& p, float om, const float* row) {
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
    // the row's entries (16-byte aligned): moments of its gather shift, jref, eref and refD
    // (scalar selects: a pointer into the parameter block would copy it to local memory)
    float4 rsm, rje, rrd;
    if constexpr (ROW) {
        rsm = row_ld4<ROW_SH>(row + kRowSM);
        rje = row_ld4<ROW_SH>(row + kRowJ);
        rrd = row_ld4<ROW_SH>(row + kRowJ + 4);
    } else {
        rsm = make_float4(0.f, 0.f, 0.f, 0.f);
        rje = make_float4(p.jreff[0], p.jreff[1], p.ereff, p.refD[0]);
        rrd = make_float4(p.refD[1], p.refD[2], p.refD[3], 0.f);
    }
    m0 += rsm.x;
    mx += rsm.y;
    my += rsm.z;
    me += rsm.w;
    const float rho = p.rho0f + m0;
    // correctly rounded reciprocal: the approximate hardware one is off by up to an ulp in a
    // direction that repeats from step to step, and the equilibrium velocity it feeds drifted by
    // 1.4e-5 over 1000 steps of the 1024^2 workload (1.4e-6 with this one)
    const float inv = __frcp_rn(rho);
    const float ux = (rje.x + mx) * inv, uy = (rje.y + my) * inv;
    const float th = 0.5f * ((rje.z + me - 2.0f * m0) * inv - (ux * ux + uy * uy));

    // ---- Hermite coefficients of the Maxwellian, per axis ----------------------------------
    // (x, y) side by side in packed FP32 pairs; each lane rounds as the scalar recurrence
    // h_{n+1} = u h_n + (n th) h_{n-1}
    float2 hxy[N + 1];
    hxy[0] = make_float2(1.f, 1.f);
    hxy[1] = make_float2(ux, uy);
#pragma unroll
    for (int n = 1; n < N; ++n) {
        const float nth = (float)n * th;
        hxy[n + 1] = __ffma2_rn(hxy[1], hxy[n], __fmul2_rn(make_float2(nth, nth), hxy[n - 1]));
    }
    float hx[N + 1], hy[N + 1];
#pragma unroll
    for (int n = 0; n <= N; ++n) {
        hx[n] = hxy[n].x;
        hy[n] = hxy[n].y;
    }

    // ---- first-order cancellation of the table defects -------------------------------------
    const float rD0 = rje.w, rD1 = rrd.x, rD2 = rrd.y, rD3 = rrd.z;
    float Dm = fmaf(2.f * p.dS[0], m0, rD0), De = fmaf(2.f * m0, p.dVS[0], rD3);
    float Dx = fmaf(rho * ux, p.dUS, rD1), Dy = fmaf(rho * uy, p.dUS, rD2);
#pragma unroll
    for (int a = 2; a <= N; a += 2) {  // dS, dV vanish for odd orders (mirror symmetry)
        const float hs = rho * (hx[a] + hy[a]);
        Dm = fmaf(p.dS[a], hs, Dm);
        De = fmaf(p.dVS[a], hs, De);  // includes the dS[0] (h_2) term for a = 2
    }
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
    const float orho = om * rho;

    // ---- per-node tables: A_i (x part), B_j (y part), X'_ia, P_jk --------------------------
    // the x and y parts of each node's odd and even sums side by side in packed FP32 pairs
    // (oxy, exy), accumulated by fused multiply-adds
    float A[N1], B[N1], Xp[N1][N > 1 ? N : 1], P[N1][N + 1];
#pragma unroll
    for (int i = 0; i < (ODD ? H + 1 : H); ++i) {
        const int m = N1 - 1 - i;
        float2 exy = make_float2(0.f, 0.f), oxy = make_float2(0.f, 0.f);
#pragma unroll
        for (int a = 1; a <= N; ++a) {
            const float2 e2 = make_float2(p.Ef[i][a], p.Ef[i][a]);
            if (a & 1) oxy = __ffma2_rn(hxy[a], e2, oxy); else exy = __ffma2_rn(hxy[a], e2, exy);
            P[i][a] = exy.y + oxy.y;
            P[m][a] = exy.y - oxy.y;
            if (a < N) {
                Xp[i][a] = orho * (hx[a] * p.Ef[i][a]);
                Xp[m][a] = (a & 1) ? -Xp[i][a] : Xp[i][a];
            }
        }
        const float cx2 = 0.5f * G * p.x2f[i];
        const float ci = fmaf(Dx, p.xf[i], cx2), cim = fmaf(-Dx, p.xf[i], cx2);
        const float cj = fmaf(Dy, p.xf[i], cx2), cjm = fmaf(-Dy, p.xf[i], cx2);
        A[i] = fmaf(orho, exy.x + oxy.x, -om * ci);
        A[m] = fmaf(orho, exy.x - oxy.x, -om * cim);
        B[i] = fmaf(orho, P[i][N], -om * cj);
        B[m] = fmaf(orho, P[m][N], -om * cjm);
    }
    const float wdr = om * (m0 - (Dm - G));
    const float keep = 1.f - om;
    if constexpr (!ODD) {
        // mirror pairs (i, n-1-i) side by side in packed FP32 pairs: half the instructions
        float2 A2[H], X2[H][N > 1 ? N : 1];
#pragma unroll
        for (int i = 0; i < H; ++i) {
            A2[i] = make_float2(A[i], A[N1 - 1 - i]);
#pragma unroll
            for (int a = 1; a < N; ++a) X2[i][a] = make_float2(Xp[i][a], Xp[N1 - 1 - i][a]);
        }
        const float2 keep2 = make_float2(keep, keep);
        float4 rq = make_float4(0.f, 0.f, 0.f, 0.f);  // a row's C entries, two pairs at a time
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            const float bj = B[j] + wdr;
            const float2 bj2 = make_float2(bj, bj);
#pragma unroll
            for (int i = 0; i < H; ++i) {
                const int m = N1 - 1 - i;
                float2 w2 = __fadd2_rn(A2[i], bj2);
#pragma unroll
                for (int a = 1; a < N; ++a) w2 = __ffma2_rn(X2[i][a], make_float2(P[j][N - a], P[j][N - a]), w2);
                float2 s2 = __ffma2_rn(keep2, make_float2(s[i + N1 * j], s[m + N1 * j]), w2);
                if constexpr (ROW) {  // the row's shift kept by the relaxation and its reference's deviation
                    const int pr = j * H + i;  // pair slot (row_slot)
                    if (pr % 2 == 0) rq = row_ld4<ROW_SH>(row + 2 * pr);
                    s2 = __fadd2_rn(s2, pr % 2 == 0 ? make_float2(rq.x, rq.y) : make_float2(rq.z, rq.w));
                }
                s[i + N1 * j] = s2.x;
                s[m + N1 * j] = s2.y;
            }
        }
    } else {
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
    if constexpr (ROW && ODD) {  // the row's gather shift kept by the relaxation and its reference's deviation
#pragma unroll
        for (int l4 = 0; l4 < (N1 * N1 + 3) / 4; ++l4) {
            const float4 c = row_ld4<ROW_SH>(row + 4 * l4);
            const float cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (4 * l4 + k < N1 * N1) s[4 * l4 + k] += cv[k];
        }
    } else if (!ROW && p.has_ref) {  // the reference's own deviation: d_eq -= Pref
#pragma unroll
        for (int l = 0; l < N1 * N1; ++l) s[l] = fmaf(-om, p.Preff[l], s[l]);
    }
}

// Collision for full FP32 populations.  s holds the gathered s_l = f_l - Whi_l, the population
// less the float Whi_l of its rest value w_l (exact while f_l stays within a factor 2 of it), and
// leaves holding f*_l.  The collision takes the state for f'_l = f_l + (w_l - Whi_l): a constant
// offset per velocity, which streaming carries over unchanged (it is uniform in space), so the
// stored f differs from the evolved f' by that fixed offset of ~3e-8 w only and no constant has
// to be subtracted from a freshly rounded sum (which would round the same way in every cell).
// With f_eq(f')_l = w_l (1 + e_l), e_l = (rho - 1) + rho phi_l - c_l, the BGK update of f' is
//     f*_l = Whi_l + [(1 - omega) s_l + w_l omega e_l],
// the deviation collision of cell_collide_dev (rho0 = 1) scaled by the weights: every rounding
// but the final addition of Whi_l is relative to the small bracket, and w_l omega e_l takes the
// exact weight as Whi_l + Wlo_l (no weight-rounding pattern that follows the flow).  With
// omega = 0 the bracket is s_l exactly, so collisionless streaming stays a bit-exact copy.
// Moments of f' are plain sums: rho - 1 = sum s, rho u = sum c s, D rho (T - 1) + rho u^2 =
// sum |c|^2 s - D sum s (its rest part taken at the exact moments 1, 0, D, as the deviation
// collision takes rho0 w).  The FP32 node tables' defects are cancelled to first order as in
// cell_collide_dev (dSx, dUx, dVSx: the defects of the exact weights with the float xf, x2f and
// E tables; the rest part's energy defect under the float x2f enters through dVSx[0], as the
// (rho - rho0) part's does there).
template <int N1>
__device__ __forceinline__ void cell_collide_split(float (&s)[N1 * N1], const KParams& p, float om) {
    constexpr int N = N1 - 1, H = N1 / 2;
    constexpr bool ODD = (N1 & 1) != 0;
    float rr[N1], rx[N1], rxx[N1];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        float r = 0.f, x1 = 0.f, x2 = 0.f;
#pragma unroll
        for (int i = 0; i < H; ++i) {
            const int m = N1 - 1 - i;
            const float a = s[i + N1 * j] + s[m + N1 * j];
            const float b = s[i + N1 * j] - s[m + N1 * j];
            r += a;
            x1 = fmaf(p.xf[i], b, x1);
            x2 = fmaf(p.x2f[i], a, x2);
        }
        if (ODD) r += s[H + N1 * j];
        rr[j] = r;
        rx[j] = x1;
        rxx[j] = x2;
    }
    float m0 = 0.f, mx = 0.f, my = 0.f, me = 0.f;
#pragma unroll
    for (int j = 0; j < H; ++j) {
        const int m = N1 - 1 - j;
        const float a = rr[j] + rr[m];
        m0 += a;
        my = fmaf(p.xf[j], rr[j] - rr[m], my);
        mx += rx[j] + rx[m];
        me = fmaf(p.x2f[j], a, me + (rxx[j] + rxx[m]));
    }
    if (ODD) {
        m0 += rr[H];
        mx += rx[H];
        me += rxx[H];
    }
    const float rho = 1.f + m0;
    const float inv = __frcp_rn(rho);
    const float ux = mx * inv, uy = my * inv;
    const float th = 0.5f * ((me - 2.0f * m0) * inv - (ux * ux + uy * uy));

    float hx[N + 1], hy[N + 1];
    hx[0] = hy[0] = 1.f;
    hx[1] = ux;
    hy[1] = uy;
#pragma unroll
    for (int n = 1; n < N; ++n) {
        hx[n + 1] = fmaf(ux, hx[n], (float)n * th * hx[n - 1]);
        hy[n + 1] = fmaf(uy, hy[n], (float)n * th * hy[n - 1]);
    }

    // first-order cancellation of the float node tables' defects
    float Dm = 2.f * p.dSx[0] * m0, De = 2.f * m0 * p.dVSx[0];
    float Dx = rho * ux * p.dUSx, Dy = rho * uy * p.dUSx;
#pragma unroll
    for (int a = 2; a <= N; a += 2) {
        const float hs = rho * (hx[a] + hy[a]);
        Dm = fmaf(p.dSx[a], hs, Dm);
        De = fmaf(p.dVSx[a], hs, De);
    }
#pragma unroll
    for (int a = 3; a <= N; a += 2) {
        Dx = fmaf(rho * p.dUx[a], hx[a], Dx);
        Dy = fmaf(rho * p.dUx[a], hy[a], Dy);
    }
#pragma unroll
    for (int b = 2; b <= N - 1; b += 2) {
        Dx = fmaf(rho * ux * p.dSx[b], hy[b], Dx);
        Dy = fmaf(rho * uy * p.dSx[b], hx[b], Dy);
    }
#pragma unroll
    for (int b = 2; b <= N - 2; b += 2) De = fmaf(rho * p.dSx[b], fmaf(hx[2], hy[b], hy[2] * hx[b]), De);
    const float G = 0.5f * De - Dm;
    const float orho = om * rho;

    // per-node tables as in cell_collide_dev: omega e_ij = A_i + B_j + sum_a X'_ia P_j,N-a
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
            const int l = i + N1 * j;
            float weq = A[i] + bj;
#pragma unroll
            for (int a = 1; a < N; ++a) weq = fmaf(Xp[i][a], P[j][N - a], weq);
            const float t = fmaf(keep, s[l], fmaf(p.Whi[l], weq, p.Wlo[l] * weq));
            s[l] = p.Whi[l] + t;
        }
    }
}

}  // namespace tvlbm
