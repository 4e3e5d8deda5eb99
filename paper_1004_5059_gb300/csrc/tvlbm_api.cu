// Host side of the TVLBM library: velocity sets, streaming tables, context lifetime, argument
// validation, memory layout and kernel launches behind the C ABI of include/tvlbm.h.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "tvlbm.h"
#include "tvlbm_kernels.cuh"
#include "tvlbm_tiled.cuh"

using namespace tvlbm;

extern "C" int tvlbm_destroy(tvlbm_ctx* c);

// =============================================================================================
// Velocity sets: n-point Gauss quadrature for the weight exp(-x^2/2)/sqrt(2 pi).  The nodes
// are the roots of the probabilists' Hermite polynomial He_n (He_{k+1} = x He_k - k He_{k-1}),
// found by bracketing sign changes and polishing with Newton's method (He_n' = n He_{n-1}) in
// long double; the weights are w_i = n! / (n^2 He_{n-1}(x_i)^2).  The paper places its discrete
// velocities on Hermite roots (Sec. "The TVLBM model", Introduction).
// =============================================================================================
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

struct Rule {
    int n;
    double x[kMaxN1], w[kMaxN1];
};

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
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            double s = 0.0;
            for (int a = 0; a <= N; ++a)
                for (int b = 0; a + b <= N; ++b)
                    s += hx[a] * hermite_over_fact(a, r.x[i]) * hy[b] * hermite_over_fact(b, r.x[j]);
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

struct Layout {
    int hx, pitch, rows;
    long long plane;
    size_t buf_bytes, mom_bytes, part_bytes, total;
    size_t off_f[2], off_mom, off_part, off_sums, off_status;
};

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
    L.total = L.off_sums + 256;
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

constexpr int kGraphSteps = 32;  // steps per captured graph (even: buffer parity is preserved)

}  // namespace

struct tvlbm_ctx {
    int nx, ny, velset, n1, Q, N, storage, form, graphs;
    double tau, dt, rho0;
    tvlbm_bc bc;
    Rule rule;
    Layout L;
    KParams kp;
    const KernelTable* kt;
    int device;
    unsigned char* mem;
    bool own_mem;
    int cur;
    cudaStream_t stream;
    cudaStream_t capture_stream;
    cudaGraphExec_t graph[2];
    int have_tmap;
    int tile_cfg;                     // tiled-form tile configuration
    alignas(64) CUtensorMap tmap[2];  // TMA descriptors of the two population buffers
    char err[512];
};

namespace {

int fail(tvlbm_ctx* c, int code, const char* fmt, ...) {
    if (c) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(c->err, sizeof(c->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int cuda_fail(tvlbm_ctx* c, cudaError_t e, const char* what) {
    return fail(c, TVLBM_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e), cudaGetErrorString(e));
}

#define TVLBM_CUDA(ctx, call, what)                           \
    do {                                                      \
        cudaError_t e_ = (call);                              \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, what); \
    } while (0)

void* dptr(tvlbm_ctx* c, size_t off) { return c->mem + off; }
void* fcur(tvlbm_ctx* c) { return dptr(c, c->L.off_f[c->cur]); }

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

void fill_params(tvlbm_ctx* c) {
    KParams& p = c->kp;
    memset(&p, 0, sizeof(p));
    const Rule& r = c->rule;
    for (int i = 0; i < r.n; ++i) {
        int sh;
        double a;
        shift_of(r.x[i], c->dt, &sh, &a);
        p.sh[i] = sh;
        p.xd[i] = r.x[i];
        p.xf[i] = (float)r.x[i];
        p.x2f[i] = p.xf[i] * p.xf[i];
        p.wd[i] = r.w[i];
        p.wf[i] = (float)r.w[i];
        p.ad[i] = a;
        p.af[i] = (float)a;
        for (int k = 0; k <= c->N; ++k) {
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
    for (int a = 0; a <= c->N; ++a) {
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
    p.omegad = c->dt / c->tau;
    p.omegaf = (float)p.omegad;
    p.rho0d = c->rho0;
    p.rho0f = (float)c->rho0;
    p.nx = c->nx;
    p.ny = c->ny;
    p.pitch = c->L.pitch;
    p.hx = c->L.hx;
    p.rows = c->L.rows;
    p.plane = c->L.plane;
    p.walls = c->bc.kind == TVLBM_BC_WALLS;
    if (p.walls) {
        for (int side = 0; side < 2; ++side) {
            const double uw = side ? c->bc.u_hi : c->bc.u_lo, Tw = side ? c->bc.T_hi : c->bc.T_lo;
            double feq[kMaxQ];
            host_equilibrium(r, 1.0, uw, 0.0, Tw, feq);
            double den = 0.0;
            for (int j = 0; j < r.n; ++j) {
                const bool incoming = side == 0 ? r.x[j] > 0.0 : r.x[j] < 0.0;
                for (int i = 0; i < r.n; ++i) {
                    const int l = i + r.n * j;
                    p.feqwd[side][l] = feq[l];
                    p.feqwf[side][l] = (float)feq[l];
                    if (incoming) den += fabs(r.x[j] * c->dt) * feq[l];
                }
            }
            p.inv_dend[side] = 1.0 / den;
            p.inv_denf[side] = (float)(1.0 / den);
        }
    }
}

void drop_graphs(tvlbm_ctx* c) {
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
}

// Launch one time step from buffer `from` into buffer 1-from on stream s.
cudaError_t launch_step(tvlbm_ctx* c, int from, cudaStream_t s) {
    void* fin = dptr(c, c->L.off_f[from]);
    void* fout = dptr(c, c->L.off_f[1 - from]);
    if (c->kp.walls) {
        const cudaError_t e = c->kt->wall(c->storage, fin, c->kp, s);
        if (e != cudaSuccess) return e;
    }
    return c->kt->sweep(c->storage, c->form, c->tile_cfg, fin, fout, &c->tmap[from], c->kp, s);
}

// TMA descriptors for the tiled form: a 3-D view [Q][rows][pitch] of each population buffer,
// box = the tile's source window (BX x BY x 1 elements), no swizzle, zero fill out of bounds.
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

bool make_tensor_maps(tvlbm_ctx* c) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || !c->kt->tiled_available(c->storage)) return false;
    int bx = 0, by = 0;
    c->kt->tiled_box(c->storage, c->tile_cfg, &bx, &by);
    CUtensorMapDataType dt;
    switch (c->storage) {
        case TVLBM_FP64: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT64; break;
        case TVLBM_BF16_DEV: dt = CU_TENSOR_MAP_DATA_TYPE_BFLOAT16; break;
        case TVLBM_FP16_DEV: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT16; break;
        default: dt = CU_TENSOR_MAP_DATA_TYPE_FLOAT32; break;
    }
    const size_t es = elem_size(c->storage);
    const cuuint64_t dims[3] = {(cuuint64_t)c->L.pitch, (cuuint64_t)c->L.rows, (cuuint64_t)c->Q};
    const cuuint64_t strides[2] = {(cuuint64_t)c->L.pitch * es, (cuuint64_t)c->L.plane * es};
    const cuuint32_t box[3] = {(cuuint32_t)bx, (cuuint32_t)by, 1};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int b = 0; b < 2; ++b) {
        const CUresult r = enc(&c->tmap[b], dt, 3, dptr(c, c->L.off_f[b]), dims, strides, box, estr,
                               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return false;
    }
    return true;
}

// Read and clear the device status word; a set bit means a bounded device wait gave up.
int check_status(tvlbm_ctx* c) {
    int st = 0;
    int* d = (int*)dptr(c, c->L.off_status);
    TVLBM_CUDA(c, cudaMemcpyAsync(&st, d, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync status");
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "status synchronize");
    if (st) {
        cudaMemsetAsync(d, 0, sizeof(int), c->stream);
        cudaStreamSynchronize(c->stream);
        return fail(c, TVLBM_ETIMEOUT, "a device-side wait for a TMA load timed out (status %d)", st);
    }
    return TVLBM_OK;
}

int build_graph(tvlbm_ctx* c, int parity) {
    cudaGraph_t g = nullptr;
    TVLBM_CUDA(c, cudaStreamBeginCapture(c->capture_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < kGraphSteps && le == cudaSuccess; ++k) le = launch_step(c, (parity + k) & 1, c->capture_stream);
    const cudaError_t ce = cudaStreamEndCapture(c->capture_stream, &g);
    if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_fail(c, le, "kernel launch during capture"); }
    if (ce != cudaSuccess) return cuda_fail(c, ce, "cudaStreamEndCapture");
    const cudaError_t ie = cudaGraphInstantiate(&c->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) { c->graph[parity] = nullptr; return cuda_fail(c, ie, "cudaGraphInstantiate"); }
    return TVLBM_OK;
}

int upload_fields_and_init(tvlbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* T);

int create_common(int nx, int ny, int velset, double tau, double dt, const tvlbm_bc* bc, int storage, double rho0,
                  void* device_memory, size_t bytes, tvlbm_ctx** out) {
    if (!out) return TVLBM_EINVAL;
    *out = nullptr;
    char msg[256];
    int rc = validate(nx, ny, velset, tau, dt, bc, storage, rho0, msg, sizeof(msg));
    if (rc) return rc;
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess || ndev == 0) return TVLBM_ECUDA;
    tvlbm_ctx* c = new (std::nothrow) tvlbm_ctx();
    if (!c) return TVLBM_ENOMEM;
    memset(c, 0, sizeof(*c));
    c->nx = nx;
    c->ny = ny;
    c->velset = velset;
    c->n1 = nodes_for(velset);
    c->Q = c->n1 * c->n1;
    c->N = c->n1 - 1;
    c->storage = storage;
    c->form = FORM_PLAIN;
    c->graphs = 1;
    c->tau = tau;
    c->dt = dt;
    c->rho0 = rho0;
    if (bc) c->bc = *bc; else c->bc.kind = TVLBM_BC_PERIODIC;
    gauss_hermite_rule(c->n1, &c->rule);
    c->L = make_layout(nx, ny, c->Q, storage);
    c->kt = table_for(c->n1);
    fill_params(c);
    cudaGetDevice(&c->device);
    if (device_memory) {
        if (bytes < c->L.total) { delete c; return TVLBM_ENOMEM; }
        if (((uintptr_t)device_memory) & 255) { delete c; return TVLBM_EINVAL; }
        c->mem = (unsigned char*)device_memory;
        c->own_mem = false;
    } else {
        e = cudaMalloc((void**)&c->mem, c->L.total);
        if (e != cudaSuccess) { delete c; return e == cudaErrorMemoryAllocation ? TVLBM_ENOMEM : TVLBM_ECUDA; }
        c->own_mem = true;
    }
    e = cudaStreamCreateWithFlags(&c->capture_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (c->own_mem) cudaFree(c->mem);
        delete c;
        return TVLBM_ECUDA;
    }
    c->stream = nullptr;
    c->kp.status = (int*)dptr(c, c->L.off_status);
    c->tile_cfg = 0;
    c->have_tmap = make_tensor_maps(c) ? 1 : 0;
    if (c->have_tmap) c->form = FORM_TILED;
    // Both buffers (frame included) start as the rest equilibrium f = rho0 w: zero the memory,
    // then initialise through the same path as tvlbm_init_moments.
    e = cudaMemsetAsync(c->mem, 0, c->L.total, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        cudaStreamDestroy(c->capture_stream);
        if (c->own_mem) cudaFree(c->mem);
        delete c;
        return TVLBM_ECUDA;
    }
    {
        // rest equilibrium f = rho0 w everywhere
        const size_t n = (size_t)nx * ny;
        double* h = new (std::nothrow) double[4 * n];
        if (!h) { tvlbm_destroy(c); return TVLBM_ENOMEM; }
        for (size_t k = 0; k < n; ++k) { h[k] = rho0; h[n + k] = 0.0; h[2 * n + k] = 0.0; h[3 * n + k] = 1.0; }
        rc = upload_fields_and_init(c, h, h + n, h + 2 * n, h + 3 * n);
        delete[] h;
        if (rc) { tvlbm_destroy(c); return rc; }
    }
    *out = c;
    return TVLBM_OK;
}

int upload_fields_and_init(tvlbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* T) {
    const size_t n = (size_t)c->nx * c->ny;
    double* d = (double*)dptr(c, c->L.off_mom);
    const double* src[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        TVLBM_CUDA(c, cudaMemcpyAsync(d + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                   "cudaMemcpyAsync fields");
    for (int b = 0; b < 2; ++b) {
        TVLBM_CUDA(c, c->kt->init(c->storage, d, dptr(c, c->L.off_f[b]), c->kp, c->stream), "init kernel");
    }
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "init synchronize");
    return TVLBM_OK;
}

}  // namespace

// =============================================================================================
// C ABI
// =============================================================================================
extern "C" {

int tvlbm_memory_bytes(int nx, int ny, int velset, const tvlbm_bc* bc, int storage, size_t* bytes) {
    if (!bytes) return TVLBM_EINVAL;
    char msg[256];
    const int rc = validate(nx, ny, velset, 1.0, 1.0 / 8.0, bc, storage, 1.0, msg, sizeof(msg));
    if (rc) return rc;
    const int n = nodes_for(velset);
    *bytes = make_layout(nx, ny, n * n, storage).total;
    return TVLBM_OK;
}

int tvlbm_create(int nx, int ny, int velset, double tau, double dt, const tvlbm_bc* bc, int storage, double rho0,
                 tvlbm_ctx** out) {
    return create_common(nx, ny, velset, tau, dt, bc, storage, rho0, nullptr, 0, out);
}

int tvlbm_create_in(int nx, int ny, int velset, double tau, double dt, const tvlbm_bc* bc, int storage, double rho0,
                    void* device_memory, size_t bytes, tvlbm_ctx** out) {
    if (!device_memory) return TVLBM_EINVAL;
    return create_common(nx, ny, velset, tau, dt, bc, storage, rho0, device_memory, bytes, out);
}

int tvlbm_destroy(tvlbm_ctx* c) {
    if (!c) return TVLBM_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);
    drop_graphs(c);
    if (c->capture_stream) cudaStreamDestroy(c->capture_stream);
    if (c->own_mem && c->mem) cudaFree(c->mem);
    delete c;
    return TVLBM_OK;
}

int tvlbm_set_stream(tvlbm_ctx* c, void* stream) {
    if (!c) return TVLBM_EINVAL;
    c->stream = (cudaStream_t)stream;
    return TVLBM_OK;
}

int tvlbm_set_form(tvlbm_ctx* c, int form) {
    if (!c) return TVLBM_EINVAL;
    if (form != FORM_PLAIN && form != FORM_TILED) return fail(c, TVLBM_EINVAL, "unknown form %d", form);
    if (form == FORM_TILED && !c->have_tmap)
        return fail(c, TVLBM_EINVAL, "tiled form not available (no TMA descriptor for this storage/driver)");
    if (form != c->form) drop_graphs(c);
    c->form = form;
    return TVLBM_OK;
}

int tvlbm_set_graphs(tvlbm_ctx* c, int enable) {
    if (!c) return TVLBM_EINVAL;
    c->graphs = enable ? 1 : 0;
    return TVLBM_OK;
}

int tvlbm_tile_count(const tvlbm_ctx* c) { return c ? kTileConfigs : 0; }

int tvlbm_tile_shape(const tvlbm_ctx* c, int config, int* tx, int* ty, int* rows_per_thread) {
    if (!c || config < 0 || config >= kTileConfigs || !tx || !ty || !rows_per_thread) return TVLBM_EINVAL;
    c->kt->tile_shape(c->storage, config, tx, ty, rows_per_thread);
    return TVLBM_OK;
}

int tvlbm_set_tile(tvlbm_ctx* c, int config) {
    if (!c) return TVLBM_EINVAL;
    if (config < 0 || config >= kTileConfigs) return fail(c, TVLBM_EINVAL, "tile configuration %d out of range", config);
    if (config == c->tile_cfg) return TVLBM_OK;
    cudaSetDevice(c->device);
    cudaStreamSynchronize(c->stream);  // launched work keeps its own copy of the descriptors
    const int old = c->tile_cfg;
    c->tile_cfg = config;
    if (!make_tensor_maps(c)) {
        c->tile_cfg = old;
        make_tensor_maps(c);
        return fail(c, TVLBM_EINVAL, "no TMA descriptor for tile configuration %d", config);
    }
    drop_graphs(c);
    return TVLBM_OK;
}

int tvlbm_init_moments(tvlbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* T) {
    if (!c) return TVLBM_EINVAL;
    if (!rho || !ux || !uy || !T) return fail(c, TVLBM_EINVAL, "null field pointer");
    const size_t n = (size_t)c->nx * c->ny;
    for (size_t k = 0; k < n; ++k) {
        if (!(rho[k] > 0.0) || !(T[k] > 0.0) || !isfinite(rho[k]) || !isfinite(T[k]) || !isfinite(ux[k]) ||
            !isfinite(uy[k]))
            return fail(c, TVLBM_EINVAL, "init field invalid at cell %zu (rho, T must be > 0 and finite)", k);
    }
    cudaSetDevice(c->device);
    c->cur = 0;
    return upload_fields_and_init(c, rho, ux, uy, T);
}

int tvlbm_step(tvlbm_ctx* c, int n) {
    if (!c) return TVLBM_EINVAL;
    if (n < 0) return fail(c, TVLBM_EINVAL, "negative step count");
    cudaSetDevice(c->device);
    int left = n;
    if (c->graphs) {
        while (left >= kGraphSteps) {
            if (!c->graph[c->cur]) {
                const int rc = build_graph(c, c->cur);
                if (rc) return rc;
            }
            TVLBM_CUDA(c, cudaGraphLaunch(c->graph[c->cur], c->stream), "cudaGraphLaunch");
            left -= kGraphSteps;  // even count: parity unchanged
        }
    }
    for (; left > 0; --left) {
        TVLBM_CUDA(c, launch_step(c, c->cur, c->stream), "sweep launch");
        c->cur ^= 1;
    }
    return TVLBM_OK;
}

int tvlbm_moments(tvlbm_ctx* c, double* rho, double* ux, double* uy, double* T) {
    if (!c) return TVLBM_EINVAL;
    cudaSetDevice(c->device);
    const size_t n = (size_t)c->nx * c->ny;
    double* d = (double*)dptr(c, c->L.off_mom);
    TVLBM_CUDA(c, c->kt->moments(c->storage, fcur(c), d, c->kp, c->stream), "moments kernel");
    double* dst[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        if (dst[k])
            TVLBM_CUDA(c, cudaMemcpyAsync(dst[k], d + k * n, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                       "cudaMemcpyAsync moments");
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "moments synchronize");
    return check_status(c);
}

int tvlbm_conserved_sums(tvlbm_ctx* c, double out[5]) {
    if (!c || !out) return TVLBM_EINVAL;
    cudaSetDevice(c->device);
    double* part = (double*)dptr(c, c->L.off_part);
    double* sums = (double*)dptr(c, c->L.off_sums);
    TVLBM_CUDA(c, c->kt->reduce(c->storage, fcur(c), part, sums, c->kp, c->stream), "reduction kernels");
    TVLBM_CUDA(c, cudaMemcpyAsync(out, sums, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync sums");
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "sums synchronize");
    return check_status(c);
}

size_t tvlbm_population_bytes(const tvlbm_ctx* c) {
    return c ? (size_t)c->Q * c->nx * c->ny * elem_size(c->storage) : 0;
}

int tvlbm_get_populations(tvlbm_ctx* c, void* host, size_t bytes) {
    if (!c || !host) return TVLBM_EINVAL;
    if (bytes != tvlbm_population_bytes(c)) return fail(c, TVLBM_EINVAL, "expected %zu bytes", tvlbm_population_bytes(c));
    cudaSetDevice(c->device);
    const size_t es = elem_size(c->storage), row = (size_t)c->nx * es;
    const unsigned char* base = (const unsigned char*)fcur(c);
    for (int l = 0; l < c->Q; ++l) {
        const unsigned char* src = base + ((size_t)l * c->L.plane + (size_t)HY * c->L.pitch + c->L.hx) * es;
        TVLBM_CUDA(c, cudaMemcpy2DAsync((unsigned char*)host + (size_t)l * c->ny * row, row, src, (size_t)c->L.pitch * es,
                                        row, c->ny, cudaMemcpyDeviceToHost, c->stream),
                   "cudaMemcpy2DAsync");
    }
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "get_populations synchronize");
    return check_status(c);
}

int tvlbm_set_populations(tvlbm_ctx* c, const void* host, size_t bytes) {
    if (!c || !host) return TVLBM_EINVAL;
    if (bytes != tvlbm_population_bytes(c)) return fail(c, TVLBM_EINVAL, "expected %zu bytes", tvlbm_population_bytes(c));
    cudaSetDevice(c->device);
    const size_t es = elem_size(c->storage), row = (size_t)c->nx * es;
    unsigned char* base = (unsigned char*)fcur(c);
    for (int l = 0; l < c->Q; ++l) {
        unsigned char* dst = base + ((size_t)l * c->L.plane + (size_t)HY * c->L.pitch + c->L.hx) * es;
        TVLBM_CUDA(c, cudaMemcpy2DAsync(dst, (size_t)c->L.pitch * es, (const unsigned char*)host + (size_t)l * c->ny * row,
                                        row, row, c->ny, cudaMemcpyHostToDevice, c->stream),
                   "cudaMemcpy2DAsync");
    }
    TVLBM_CUDA(c, c->kt->halo(c->storage, fcur(c), c->kp, c->stream), "halo kernel");
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "set_populations synchronize");
    return TVLBM_OK;
}

int tvlbm_get_populations_f64(tvlbm_ctx* c, double* host) {
    if (!c || !host) return TVLBM_EINVAL;
    cudaSetDevice(c->device);
    const size_t n = (size_t)c->nx * c->ny;
    double* d = (double*)dptr(c, c->L.off_mom);
    for (int l = 0; l < c->Q; ++l) {
        TVLBM_CUDA(c, c->kt->decode_plane(c->storage, fcur(c), l, d, c->kp, c->stream), "decode kernel");
        TVLBM_CUDA(c, cudaMemcpyAsync(host + (size_t)l * n, d, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
                   "cudaMemcpyAsync");
        TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "decode synchronize");
    }
    return TVLBM_OK;
}

int tvlbm_set_populations_f64(tvlbm_ctx* c, const double* host) {
    if (!c || !host) return TVLBM_EINVAL;
    cudaSetDevice(c->device);
    const size_t n = (size_t)c->nx * c->ny;
    double* d = (double*)dptr(c, c->L.off_mom);
    for (int l = 0; l < c->Q; ++l) {
        TVLBM_CUDA(c, cudaMemcpyAsync(d, host + (size_t)l * n, n * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                   "cudaMemcpyAsync");
        TVLBM_CUDA(c, c->kt->encode_plane(c->storage, fcur(c), l, d, c->kp, c->stream), "encode kernel");
        TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "encode synchronize");
    }
    TVLBM_CUDA(c, c->kt->halo(c->storage, fcur(c), c->kp, c->stream), "halo kernel");
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "set_populations_f64 synchronize");
    return TVLBM_OK;
}

int tvlbm_velocity_set(int velset, double* cx, double* cy, double* w, int* hermite_order) {
    const int n = nodes_for(velset);
    if (!n || !cx || !cy || !w) return TVLBM_EINVAL;
    Rule r;
    if (!gauss_hermite_rule(n, &r)) return TVLBM_EINVAL;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            cx[i + n * j] = r.x[i];
            cy[i + n * j] = r.x[j];
            w[i + n * j] = r.w[i] * r.w[j];
        }
    if (hermite_order) *hermite_order = n - 1;
    return TVLBM_OK;
}

int tvlbm_stream_table(int velset, double dt, int* sx, int* sy, double* ax, double* ay) {
    const int n = nodes_for(velset);
    if (!n || !sx || !sy || !ax || !ay || !(dt > 0.0)) return TVLBM_EINVAL;
    Rule r;
    if (!gauss_hermite_rule(n, &r)) return TVLBM_EINVAL;
    for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
            shift_of(r.x[i], dt, &sx[i + n * j], &ax[i + n * j]);
            shift_of(r.x[j], dt, &sy[i + n * j], &ay[i + n * j]);
        }
    return TVLBM_OK;
}

double tvlbm_bytes_per_cell(const tvlbm_ctx* c) {
    return c ? 2.0 * c->Q * (double)elem_size(c->storage) : 0.0;
}

const char* tvlbm_last_error(const tvlbm_ctx* c) { return c ? c->err : ""; }

const char* tvlbm_strerror(int code) {
    switch (code) {
        case TVLBM_OK: return "ok";
        case TVLBM_EINVAL: return "invalid argument";
        case TVLBM_ENOMEM: return "out of memory";
        case TVLBM_ECUDA: return "CUDA error";
        case TVLBM_ESTATE: return "invalid state";
        case TVLBM_ETIMEOUT: return "device wait timed out";
        case TVLBM_ENONFINITE: return "non-finite populations";
        default: return "unknown status";
    }
}

}  // extern "C"
