// Internal host helpers (see tvlbm_host.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include "tvlbm_host.h"

namespace tvlbm {
namespace host {

namespace {

long double hermite_he(int n, long double x) {
    if (n == 0) return 1.0L;
    long double a = 1.0L, b = x;
    for (int k = 1; k < n; ++k) {
        const long double c = x * b - (long double)k * a;
        a = b;
        b = c;
    }
    return b;
}

}  // namespace

// The driver's cuTensorMapEncodeTiled, looked up once through the runtime (the library does
// not link libcuda).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
    }
    return fn;
}

// =============================================================================================
// Velocity sets: n-point Gauss quadrature for the weight exp(-x^2/2)/sqrt(2 pi).  The nodes
// are the roots of the probabilists' Hermite polynomial He_n (He_{k+1} = x He_k - k He_{k-1}),
// found by bracketing sign changes and polishing with Newton's method (He_n' = n He_{n-1}) in
// long double; the weights are w_i = n! / (n^2 He_{n-1}(x_i)^2).  The paper places its discrete
// velocities on Hermite roots (Sec. "The TVLBM model", Introduction).
// =============================================================================================
bool gauss_hermite_rule(int n, Rule* r) {
    if (n < 1 || n > kMaxN1) return false;
    long double roots[kMaxN1];
    int found = 0;
    const long double lim = sqrtl(4.0L * n + 2.0L) + 1.0L, h = 1e-3L;
    long double xa = -lim, fa = hermite_he(n, xa);
    for (long double xb = -lim + h; xb <= lim + h && found < n; xb += h) {
        const long double fb = hermite_he(n, xb);
        if (fb == 0.0L || (fa < 0.0L) != (fb < 0.0L)) {
            long double lo = xa, hi = xb, flo = fa;
            for (int it = 0; it < 200; ++it) {  // bisection to a tight bracket
                const long double mid = 0.5L * (lo + hi), fm = hermite_he(n, mid);
                if (fm == 0.0L) { lo = hi = mid; break; }
                if ((fm < 0.0L) == (flo < 0.0L)) { lo = mid; flo = fm; } else hi = mid;
            }
            long double x = 0.5L * (lo + hi);
            for (int it = 0; it < 8; ++it) {  // Newton polish
                const long double d = (long double)n * hermite_he(n - 1, x);
                if (d == 0.0L) break;
                x -= hermite_he(n, x) / d;
            }
            roots[found++] = x;
        }
        xa = xb;
        fa = fb;
    }
    if (found != n) return false;
    long double fact = 1.0L;
    for (int k = 2; k <= n; ++k) fact *= k;
    long double w[kMaxN1], sum = 0.0L;
    for (int i = 0; i < n; ++i) {
        const long double h1 = hermite_he(n - 1, roots[i]);
        w[i] = fact / ((long double)n * n * h1 * h1);
    }
    // symmetric rule: enforce exact mirror symmetry (and an exact 0 node for odd n)
    for (int i = 0; i < n / 2; ++i) {
        const long double xs = 0.5L * (roots[n - 1 - i] - roots[i]);
        const long double ws = 0.5L * (w[i] + w[n - 1 - i]);
        roots[i] = -xs;
        roots[n - 1 - i] = xs;
        w[i] = w[n - 1 - i] = ws;
    }
    if (n % 2) roots[n / 2] = 0.0L;
    for (int i = 0; i < n; ++i) sum += w[i];
    r->n = n;
    for (int i = 0; i < n; ++i) {
        r->x[i] = (double)roots[i];
        r->w[i] = (double)(w[i] / sum);
    }
    return true;
}

int nodes_for(int velset) {
    switch (velset) {
        case TVLBM_D2Q9: return 3;
        case TVLBM_D2Q16: return 4;
        case TVLBM_D2Q36: return 6;
        default: return 0;
    }
}

// Shift of one node over one step: s = x dt (dx = 1) = sh + alpha; within 1e-12 of an integer
// it is that integer with alpha = 0 (a space-filling velocity moves exactly).
void shift_of(double x, double dt, int* sh, double* alpha) {
    const double s = x * dt;
    const double r = nearbyint(s);
    if (fabs(s - r) < 1e-12) {
        *sh = (int)r;
        *alpha = 0.0;
    } else {
        const double fl = floor(s);
        *sh = (int)fl;
        *alpha = s - fl;
    }
}

// He_a(x)/a!
double hermite_over_fact(int a, double x) {
    double f = 1.0;
    for (int k = 2; k <= a; ++k) f *= k;
    return (double)hermite_he(a, x) / f;
}

// Separable Hermite equilibrium on the host (FP64), f-space: see cell_equilibrium.
void host_equilibrium(const Rule& r, double rho, double ux, double uy, double T, double* feq) {
    const int n = r.n, N = n - 1;
    double hx[kMaxN1 + 1], hy[kMaxN1 + 1];
    hx[0] = hy[0] = 1.0;
    hx[1] = ux;
    hy[1] = uy;
    for (int k = 1; k < N; ++k) {
        hx[k + 1] = ux * hx[k] + k * (T - 1.0) * hx[k - 1];
        hy[k + 1] = uy * hy[k] + k * (T - 1.0) * hy[k - 1];
    }
    double E[kMaxN1][kMaxN1];  // He_a(x_i) / a!
    for (int i = 0; i < n; ++i)
        for (int a = 0; a <= N; ++a) E[i][a] = hermite_over_fact(a, r.x[i]);
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int a = 0; a <= N; ++a)
                for (int b = 0; a + b <= N; ++b) s += hx[a] * E[i][a] * hy[b] * E[j][b];
            feq[i + n * j] = rho * r.w[i] * r.w[j] * s;
        }
}

size_t elem_size(int storage) {
    switch (storage) {
        case TVLBM_FP64: return 8;
        case TVLBM_FP32: case TVLBM_FP32_DEV: return 4;
        case TVLBM_BF16_DEV: case TVLBM_FP16_DEV: return 2;
        default: return 0;
    }
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

Layout make_layout(int nx, int ny, int Q, int storage) {
    Layout L;
    const size_t es = elem_size(storage);
    // pitch: a multiple of 32 elements holding the fluid and the x frame of hx columns per side
    L.hx = (int)(32 / es);
    L.pitch = (int)align_up((size_t)nx + 2 * L.hx, 32);
    L.rows = ny + 2 * HY;
    L.plane = (long long)L.pitch * L.rows;
    L.buf_bytes = align_up((size_t)Q * L.plane * es, 256);
    L.mom_bytes = align_up((size_t)4 * nx * ny * sizeof(double), 256);
    L.part_bytes = align_up((size_t)kRedBlocks * 5 * sizeof(double), 256);
    L.off_f[0] = 0;
    L.off_f[1] = L.buf_bytes;
    L.off_mom = 2 * L.buf_bytes;
    L.off_part = L.off_mom + L.mom_bytes;
    L.off_sums = L.off_part + L.part_bytes;
    L.off_status = L.off_sums + 128;
    // dataflow counters: task counter, abort word, then one completion counter per tile of at
    // least 32 x 4 cells (the smallest tile of any configuration)
    L.off_flow = L.off_sums + 256;
    L.flow_ints = (size_t)kFlowDone + (size_t)((nx + 31) / 32) * (size_t)((ny + 3) / 4);
    L.total = L.off_flow + align_up(L.flow_ints * sizeof(int), 256);
    return L;
}

const KernelTable* table_for(int n) {
    switch (n) {
        case 3: return kernel_table_q3();
        case 4: return kernel_table_q4();
        case 6: return kernel_table_q6();
        default: return nullptr;
    }
}

int validate(int nx, int ny, int velset, double tau, double dt, const tvlbm_bc* bc, int storage, double rho0,
             char* msg, size_t msglen) {
    const int n = nodes_for(velset);
    if (!n) { snprintf(msg, msglen, "unknown velocity set %d", velset); return TVLBM_EINVAL; }
    if (!elem_size(storage)) { snprintf(msg, msglen, "unknown storage %d", storage); return TVLBM_EINVAL; }
    if (nx < 1 || ny < 1) { snprintf(msg, msglen, "grid %d x %d must be at least 1 x 1", nx, ny); return TVLBM_EINVAL; }
    if ((long long)nx * ny >= (1LL << 31) || nx > (1 << 28) || ny > (1 << 28)) {
        snprintf(msg, msglen, "grid %d x %d too large", nx, ny);
        return TVLBM_EINVAL;
    }
    if (bc && bc->kind != TVLBM_BC_PERIODIC && bc->kind != TVLBM_BC_WALLS) {
        snprintf(msg, msglen, "unknown boundary kind %d", bc->kind);
        return TVLBM_EINVAL;
    }
    const bool walls = bc && bc->kind == TVLBM_BC_WALLS;
    if (walls && ny < 2 * HY + 1) { snprintf(msg, msglen, "walls need ny >= %d", 2 * HY + 1); return TVLBM_EINVAL; }
    if (walls && !(bc->T_lo > 0.0 && bc->T_hi > 0.0 && isfinite(bc->u_lo) && isfinite(bc->u_hi))) {
        snprintf(msg, msglen, "wall temperatures must be > 0 and velocities finite");
        return TVLBM_EINVAL;
    }
    if (!(dt > 0.0) || !isfinite(dt)) { snprintf(msg, msglen, "dt must be > 0"); return TVLBM_EINVAL; }
    // tau = +inf is accepted: no collisions, pure volumetric streaming
    if (!(tau > 0.5 * dt)) { snprintf(msg, msglen, "tau must exceed dt/2"); return TVLBM_EINVAL; }
    if (!(rho0 > 0.0) || !isfinite(rho0)) { snprintf(msg, msglen, "rho0 must be > 0"); return TVLBM_EINVAL; }
    Rule r;
    if (!gauss_hermite_rule(n, &r)) { snprintf(msg, msglen, "quadrature failed"); return TVLBM_EINVAL; }
    for (int i = 0; i < n; ++i) {
        const double s = r.x[i] * dt;
        if (!(s >= -4.0 && s < 4.0)) {
            snprintf(msg, msglen, "shift |c dt| = %g reaches 4 cells; reduce dt", fabs(s));
            return TVLBM_EINVAL;
        }
    }
    return TVLBM_OK;
}

void fill_kparams(KParams& p, const Rule& r, int N, double dt, double tau, double rho0, int nx, int ny,
                  const Layout& L, const tvlbm_bc& bc) {
    memset(&p, 0, sizeof(p));
    for (int i = 0; i < r.n; ++i) {
        int sh;
        double a;
        shift_of(r.x[i], dt, &sh, &a);
        p.sh[i] = sh;
        p.xd[i] = r.x[i];
        p.xf[i] = (float)r.x[i];
        p.x2f[i] = p.xf[i] * p.xf[i];
        p.wd[i] = r.w[i];
        p.wf[i] = (float)r.w[i];
        p.ad[i] = a;
        p.af[i] = (float)a;
        for (int k = 0; k <= N; ++k) {
            p.Ed[i][k] = hermite_over_fact(k, r.x[i]);
            p.Ef[i][k] = (float)p.Ed[i][k];
        }
    }
    // Mirror nodes +-x share one overlap fraction pair alpha(-x) = 1 - alpha(x); keep that exact
    // in float (the member >= 1/2 is rounded, the other is 1 minus it, exact by Sterbenz).
    for (int i = 0; i < r.n; ++i) {
        const int m = r.n - 1 - i;
        if (m == i || p.ad[i] == 0.0 || p.ad[m] == 0.0) continue;
        if (p.ad[i] >= 0.5) p.af[m] = 1.0f - p.af[i];
    }
    // Pre-multiplied FP32 constants of the moment sums and their defects against the
    // quadrature identities (exact products of floats in long double).
    for (int i = 0; i < r.n; ++i) {
        p.wxf[i] = p.wf[i] * p.xf[i];
        p.wx2f[i] = p.wf[i] * p.x2f[i];
    }
    for (int a = 0; a < kMaxN1; ++a) p.dS[a] = p.dU[a] = p.dV[a] = 0.0f;
    for (int a = 0; a <= N; ++a) {
        long double S = 0, U = 0, V = 0;
        for (int i = 0; i < r.n; ++i) {
            const long double e = p.Ef[i][a];
            S += (long double)p.wf[i] * e;
            U += (long double)p.wxf[i] * e;
            V += (long double)p.wx2f[i] * e;
        }
        p.dS[a] = (float)(S - (a == 0 ? 1.0L : 0.0L));
        p.dU[a] = (float)(U - (a == 1 ? 1.0L : 0.0L));
        p.dV[a] = (float)(V - (a == 0 ? 1.0L : 0.0L) - (a == 2 ? 1.0L : 0.0L));
    }
    p.dUS = (float)((long double)p.dU[1] + p.dS[0]);
    for (int a = 0; a < kMaxN1; ++a)
        p.dVS[a] = (float)((long double)p.dV[a] + p.dS[a] + (a == 2 ? (long double)p.dS[0] : 0.0L));
    // Full-f FP32 codec: exact weights as float pairs, and the defects of the float node tables
    // (xf, x2f, E) under the exact weights (long double sums of the FP64 weights times floats).
    for (int l = 0; l < kMaxQ; ++l) p.Whi[l] = p.Wlo[l] = 0.0f;
    for (int j = 0; j < r.n; ++j)
        for (int i = 0; i < r.n; ++i) {
            const double w = r.w[i] * r.w[j];
            const int l = i + r.n * j;
            p.Whi[l] = (float)w;
            p.Wlo[l] = (float)(w - (double)p.Whi[l]);
        }
    for (int a = 0; a < kMaxN1; ++a) p.dSx[a] = p.dUx[a] = p.dVSx[a] = 0.0f;
    for (int a = 0; a <= N; ++a) {
        long double S = 0, U = 0, V = 0;
        for (int i = 0; i < r.n; ++i) {
            const long double w = r.w[i];
            S += w * p.Ef[i][a];
            U += w * p.xf[i] * p.Ef[i][a];
            V += w * p.x2f[i] * p.Ef[i][a];
        }
        const long double dSx = S - (a == 0 ? 1.0L : 0.0L);
        p.dSx[a] = (float)dSx;
        p.dUx[a] = (float)(U - (a == 1 ? 1.0L : 0.0L));
        p.dVSx[a] = (float)(V - (a == 0 ? 1.0L : 0.0L) - (a == 2 ? 1.0L : 0.0L) + dSx);
    }
    for (int a = 0; a <= N; ++a)
        if (a == 2) p.dVSx[a] = (float)((long double)p.dVSx[a] + p.dSx[0]);
    p.dUSx = (float)((long double)p.dUx[1] + p.dSx[0]);
    p.omegad = dt / tau;
    p.omegaf = (float)p.omegad;
    if (p.omegad == 0.0) {
        // collisionless (tau = inf): f* is the gathered f itself, so the full-f FP32 codec splits
        // nothing off and an integer shift stays a bit-exact copy even where a population is
        // beyond a factor 2 of its rest value (where f - Whi rounds)
        for (int l = 0; l < kMaxQ; ++l) p.Whi[l] = p.Wlo[l] = 0.0f;
    }
    p.rho0d = rho0;
    p.rho0f = (float)rho0;
    p.nx = nx;
    p.ny = ny;
    p.pitch = L.pitch;
    p.hx = L.hx;
    p.rows = L.rows;
    p.plane = L.plane;
    p.walls = bc.kind == TVLBM_BC_WALLS;
    if (p.walls) {
        for (int side = 0; side < 2; ++side) {
            const double uw = side ? bc.u_hi : bc.u_lo, Tw = side ? bc.T_hi : bc.T_lo;
            double feq[kMaxQ];
            host_equilibrium(r, 1.0, uw, 0.0, Tw, feq);
            double den = 0.0;
            for (int j = 0; j < r.n; ++j) {
                const bool incoming = side == 0 ? r.x[j] > 0.0 : r.x[j] < 0.0;
                for (int i = 0; i < r.n; ++i) {
                    const int l = i + r.n * j;
                    p.feqwd[side][l] = feq[l];
                    p.feqwf[side][l] = (float)feq[l];
                    if (incoming) den += fabs(r.x[j] * dt) * feq[l];
                }
            }
            p.inv_dend[side] = 1.0 / den;
            p.inv_denf[side] = (float)(1.0 / den);
        }
    }
}

bool encode_tensor_map(CUtensorMap* m, void* base, int storage, const Layout& L, int Q, int bx, int by) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    CUtensorMapDataType dt;
    switch (storage) {
        case TVLBM_FP64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
        case TVLBM_BF16_DEV: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
        case TVLBM_FP16_DEV: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
        default: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    }
    const size_t es = elem_size(storage);
    const cuuint64_t dims[3] = {(cuuint64_t)L.pitch, (cuuint64_t)L.rows, (cuuint64_t)Q};
    const cuuint64_t strides[2] = {(cuuint64_t)L.pitch * es, (cuuint64_t)L.plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    const CUresult r = enc(m, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                           CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

RefEntry reference_entry(const KParams& p, const Rule& r, double rho0, double ux, double uy, double T) {
    const int n = r.n;
    RefEntry e;
    memset(&e, 0, sizeof(e));
    double feq[kMaxQ];
    host_equilibrium(r, rho0, ux, uy, T, feq);
    const bool rest = ux == 0.0 && uy == 0.0 && T == 1.0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const int l = i + n * j;
            const double pr = rest ? 0.0 : feq[l] / (r.w[i] * r.w[j]) - rho0;
            e.Prefd[l] = pr;
            e.Preff[l] = (float)pr;
            if (pr != 0.0) e.nonzero = true;
        }
    e.jrefd[0] = rho0 * ux;
    e.jrefd[1] = rho0 * uy;
    e.erefd = rho0 * (2.0 * (T - 1.0) + ux * ux + uy * uy);
    e.jreff[0] = (float)e.jrefd[0];
    e.jreff[1] = (float)e.jrefd[1];
    e.ereff = (float)e.erefd;
    // the reference table's moments under the FP32 moment constants, exactly, minus their ideal
    long double m = 0, mx = 0, my = 0, me = 0;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            const long double v = e.Preff[i + n * j];
            m += (long double)p.wf[i] * p.wf[j] * v;
            mx += (long double)p.wxf[i] * p.wf[j] * v;
            my += (long double)p.wf[i] * p.wxf[j] * v;
            me += ((long double)p.wx2f[i] * p.wf[j] + (long double)p.wf[i] * p.wx2f[j]) * v;
        }
    e.refD[0] = (float)(-(m - 0.0L));
    e.refD[1] = (float)(-(mx - (long double)e.jreff[0]));
    e.refD[2] = (float)(-(my - (long double)e.jreff[1]));
    e.refD[3] = (float)(-(me - (long double)e.ereff));
    return e;
}

void set_reference_params(KParams& p, const Rule& r, double rho0, double ux, double uy, double T) {
    const RefEntry e = reference_entry(p, r, rho0, ux, uy, T);
    p.has_ref = e.nonzero ? 1 : 0;
    memcpy(p.Prefd, e.Prefd, sizeof(p.Prefd));
    memcpy(p.Preff, e.Preff, sizeof(p.Preff));
    p.jrefd[0] = e.jrefd[0];
    p.jrefd[1] = e.jrefd[1];
    p.erefd = e.erefd;
    p.jreff[0] = e.jreff[0];
    p.jreff[1] = e.jreff[1];
    p.ereff = e.ereff;
    memcpy(p.refD, e.refD, sizeof(p.refD));
    p.rowf = nullptr;
    p.rowd = nullptr;
}

}  // namespace host
}  // namespace tvlbm
