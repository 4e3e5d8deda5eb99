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
#include "tvlbm_host.h"
#include "tvlbm_kernels.cuh"
#include "tvlbm_ctx.h"

using namespace tvlbm;
using namespace tvlbm::host;

extern "C" int tvlbm_destroy(tvlbm_ctx* c);

namespace {
constexpr int kGraphSteps = 32;  // steps per captured graph (even: buffer parity is preserved)
}  // namespace



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
    if (c->mesh_mem) return mesh_launch_step(c, fin, fout, s);  // non-uniform y mesh: its own sweep
    if (c->kp.walls) {
        const cudaError_t e = c->kt->wall(c->storage, fin, c->kp, s);
        if (e != cudaSuccess) return e;
    }
    const SweepMaps maps = {c->form == FORM_STRIP ? &c->rmap[from] : &c->tmap[from], nullptr};
    return c->kt->sweep(c->storage, c->form, c->tile_cfg, fin, fout, &maps, c->kp, s);
}

// Tile grid of configuration cfg when the dataflow form can run it: a periodic domain that the
// tiles cover exactly, tiles of at least 4 rows.
bool flow_tiles(const tvlbm_ctx* c, int cfg, int* tiles_x, int* tiles_y) {
    if (!c->have_tmap || c->kp.walls) return false;
    int tx = 0, ty = 0, r = 0;
    c->kt->tile_shape(c->storage, cfg, &tx, &ty, &r);
    if (tx < 32 || ty < 4 || c->nx % tx || c->ny % ty) return false;
    const long long n = (long long)(c->nx / tx) * (c->ny / ty);
    if ((size_t)n + kFlowDone > c->L.flow_ints) return false;
    *tiles_x = c->nx / tx;
    *tiles_y = c->ny / ty;
    return true;
}

// n time steps in dataflow launches (tasks per launch below 2^30, steps per launch at most 2^24,
// so the per-tile counters, warps per task x steps, stay far inside an int).
cudaError_t launch_flow(tvlbm_ctx* c, int n, cudaStream_t s) {
    int tiles_x = 0, tiles_y = 0;
    if (!flow_tiles(c, c->tile_cfg, &tiles_x, &tiles_y)) return cudaErrorInvalidValue;
    const int ntiles = tiles_x * tiles_y;
    const int chunk_max = (1 << 30) / ntiles < (1 << 24) ? (1 << 30) / ntiles : (1 << 24);
    int* ctr = (int*)dptr(c, c->L.off_flow);
    while (n > 0) {
        const int chunk = n < chunk_max ? n : chunk_max;
        FlowSrc src;
        memset(&src, 0, sizeof(src));
        src.map[0] = c->tmap[c->cur];
        src.map[1] = c->tmap[1 - c->cur];
        src.smap[0] = c->smap[c->cur];
        src.smap[1] = c->smap[1 - c->cur];
        src.buf[0] = dptr(c, c->L.off_f[c->cur]);
        src.buf[1] = dptr(c, c->L.off_f[1 - c->cur]);
        src.tiles_x = tiles_x;
        src.tiles_y = tiles_y;
        src.ntiles = ntiles;
        src.nsteps = chunk;
        src.next_task = ctr;
        src.abort = ctr + 1;
        src.done = ctr + kFlowDone;
        src.wait_ns = c->flow_wait_ns;
        src.wait_extra = c->flow_wait_extra;
        cudaError_t e = cudaMemsetAsync(ctr, 0, ((size_t)kFlowDone + ntiles) * sizeof(int), s);
        if (e == cudaSuccess) e = c->kt->flow_sweep(c->storage, c->tile_cfg, src, c->kp, s);
        if (e != cudaSuccess) return e;
        c->cur ^= chunk & 1;
        n -= chunk;
    }
    return cudaSuccess;
}

bool make_tensor_maps(tvlbm_ctx* c) {
    if (!c->kt->tiled_available(c->storage)) return false;
    int bx = 0, by = 0, tx = 0, ty = 0, r = 0;
    c->kt->tiled_box(c->storage, c->tile_cfg, &bx, &by);
    c->kt->tile_shape(c->storage, c->tile_cfg, &tx, &ty, &r);
    for (int b = 0; b < 2; ++b) {
        if (!encode_tensor_map(&c->tmap[b], dptr(c, c->L.off_f[b]), c->storage, c->L, c->Q, bx, by)) return false;
        if (!encode_tensor_map(&c->smap[b], dptr(c, c->L.off_f[b]), c->storage, c->L, c->Q, tx, ty)) return false;
        if (!encode_tensor_map(&c->rmap[b], dptr(c, c->L.off_f[b]), c->storage, c->L, c->Q,
                               strip_box_width((int)elem_size(c->storage)),
                               strip_chunk_rows(c->n1, (int)elem_size(c->storage))))
            return false;
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
    c->scheme = TVLBM_SCHEME_VOLUMETRIC;
    c->tau_g = INFINITY;
    c->rho0 = rho0;
    c->flow_wait_ns = (long long)kWaitLimitNs;
    c->flow_wait_extra = 0;
    if (bc) c->bc = *bc; else c->bc.kind = TVLBM_BC_PERIODIC;
    gauss_hermite_rule(c->n1, &c->rule);
    c->L = make_layout(nx, ny, c->Q, storage);
    c->kt = table_for(c->n1);
    fill_kparams(c->kp, c->rule, c->N, c->dt, c->tau, c->rho0, c->nx, c->ny, c->L, c->bc);
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

// The first cell (lowest index) whose fields are invalid -- rho or T not > 0, or any of the four
// not finite -- into *first (left at its initial all-ones value when every cell is valid).
__global__ void __launch_bounds__(256) validate_fields_kernel(const double* __restrict__ d, long long n,
                                                              unsigned long long* __restrict__ first) {
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n; k += (long long)gridDim.x * blockDim.x) {
        const double rho = d[k], ux = d[n + k], uy = d[2 * n + k], T = d[3 * n + k];
        if (!(rho > 0.0) || !(T > 0.0) || !isfinite(rho) || !isfinite(T) || !isfinite(ux) || !isfinite(uy))
            atomicMin(first, (unsigned long long)k);
    }
}

// Host fields -> device scratch, checked on the device (nothing else is written when a cell is
// invalid), then the initial equilibrium into both population buffers.
int upload_fields_and_init(tvlbm_ctx* c, const double* rho, const double* ux, const double* uy, const double* T) {
    const size_t n = (size_t)c->nx * c->ny;
    double* d = (double*)dptr(c, c->L.off_mom);
    const double* src[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        TVLBM_CUDA(c, cudaMemcpyAsync(d + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice, c->stream),
                   "cudaMemcpyAsync fields");
    unsigned long long* first = (unsigned long long*)dptr(c, c->L.off_part);  // reduction scratch, free here
    TVLBM_CUDA(c, cudaMemsetAsync(first, 0xFF, sizeof(*first), c->stream), "cudaMemsetAsync");
    const long long blocks = ((long long)n + 255) / 256 < 4096 ? ((long long)n + 255) / 256 : 4096;
    validate_fields_kernel<<<(unsigned)blocks, 256, 0, c->stream>>>(d, (long long)n, first);
    TVLBM_CUDA(c, cudaGetLastError(), "field check kernel");
    unsigned long long bad = 0;
    TVLBM_CUDA(c, cudaMemcpyAsync(&bad, first, sizeof(bad), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync check");
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "field check synchronize");
    if (bad != ~0ull)
        return fail(c, TVLBM_EINVAL, "init field invalid at cell %llu (rho, T must be > 0 and finite)", bad);
    for (int b = 0; b < 2; ++b) {
        TVLBM_CUDA(c, c->kt->init(c->storage, d, dptr(c, c->L.off_f[b]), c->kp, c->stream), "init kernel");
    }
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "init synchronize");
    return TVLBM_OK;
}

// ---- per-row deviation reference -----------------------------------------------------------
// Device buffers, allocated on first use: the live tables the kernels read (KParams::rowd /
// rowf), a second pair the next reference is built in, the re-encoding shifts and the profile.
bool ensure_reference_buffers(tvlbm_ctx* c) {
    if (c->ref_mem) return true;
    const size_t rows = (size_t)c->L.rows;
    const size_t bd = align_up(rows * kRowD * sizeof(double), 256), bf = align_up(rows * kRowF * sizeof(float), 256);
    const size_t bdel = align_up(rows * kMaxQ * sizeof(float), 256);
    const size_t bp = align_up((size_t)kMaxQ * c->ny * sizeof(double), 256);  // [3][ny] or [Q][ny] profile
    unsigned char* m = nullptr;
    if (cudaMalloc((void**)&m, 2 * bd + 2 * bf + bdel + bp) != cudaSuccess) return false;
    c->ref_mem = m;
    c->ref_rowd = (double*)m;
    c->ref_new_d = (double*)(m + bd);
    c->ref_rowf = (float*)(m + 2 * bd);
    c->ref_new_f = (float*)(m + 2 * bd + bf);
    c->ref_delta = (float*)(m + 2 * bd + 2 * bf);
    c->ref_prof = (double*)(m + 2 * bd + 2 * bf + bdel);
    return true;
}

// One reference's Pref table: per stored row (rows: [rows][kRowD]) or the same for every row.
struct RefSide {
    const double* rows;
    double c[kMaxQ];
};
RefSide ref_side_of(const KParams& p) {
    RefSide r;
    r.rows = p.rowd;
    for (int l = 0; l < kMaxQ; ++l) r.c[l] = p.Prefd[l];
    return r;
}

// delta[r][l] = Pref_old - Pref_new: the shift that re-expresses a stored deviation.
__global__ void ref_delta_kernel(float* __restrict__ delta, const RefSide from, const RefSide to, int rows, int Q) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= rows * kMaxQ) return;
    const int r = t / kMaxQ, l = t - r * kMaxQ;
    const double o = from.rows ? ld_row(from.rows + (long long)r * kRowD + l) : from.c[l];
    const double n = to.rows ? ld_row(to.rows + (long long)r * kRowD + l) : to.c[l];
    delta[t] = l < Q ? (float)(o - n) : 0.0f;
}

// Re-express the current state from reference `from` to reference `to` (stream-ordered).
cudaError_t reencode_between(tvlbm_ctx* c, const RefSide& from, const RefSide& to) {
    const int n = c->L.rows * kMaxQ;
    ref_delta_kernel<<<(n + 255) / 256, 256, 0, c->stream>>>(c->ref_delta, from, to, c->L.rows, c->Q);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return c->kt->reencode(c->storage, fcur(c), c->ref_delta, c->kp, c->stream);
}

// Switch to the per-row reference of the profile in c->ref_prof (device; mean = false: [3][ny] of
// (ux, uy, T), the rows' equilibria; mean = true: [Q][ny] of Pref itself): build its tables in the
// spare pair, re-encode the state, copy the tables over the live ones (stream-ordered, no host
// synchronisation; the kernel parameters keep the live pointers, so captured graphs stay valid).
// The first switch points the kernel parameters at the live tables.
int install_reference_rows(tvlbm_ctx* c, bool mean) {
    if (mean)
        TVLBM_CUDA(c, c->kt->ref_tables_mean(c->ref_prof, c->ref_new_d, c->ref_new_f, c->kp, c->stream),
                   "reference tables");
    else
        TVLBM_CUDA(c, c->kt->ref_tables(c->ref_prof, c->ref_new_d, c->ref_new_f, c->kp, c->stream), "reference tables");
    RefSide to;
    to.rows = c->ref_new_d;
    for (int l = 0; l < kMaxQ; ++l) to.c[l] = 0.0;
    TVLBM_CUDA(c, reencode_between(c, ref_side_of(c->kp), to), "re-encoding");
    const size_t rows = (size_t)c->L.rows;
    TVLBM_CUDA(c, cudaMemcpyAsync(c->ref_rowd, c->ref_new_d, rows * kRowD * sizeof(double), cudaMemcpyDeviceToDevice,
                                  c->stream), "row tables");
    TVLBM_CUDA(c, cudaMemcpyAsync(c->ref_rowf, c->ref_new_f, rows * kRowF * sizeof(float), cudaMemcpyDeviceToDevice,
                                  c->stream), "row tables");
    if (c->kp.rowf != c->ref_rowf) {
        set_reference_params(c->kp, c->rule, c->rho0, 0.0, 0.0, 1.0);
        c->kp.has_ref = 1;
        c->kp.rowf = c->ref_rowf;
        c->kp.rowd = c->ref_rowd;
        drop_graphs(c);
    }
    return TVLBM_OK;
}

// Reset the per-row reference to the current rows (kind TVLBM_REF_EQUILIBRIUM: the equilibria of
// the row averages of (u_x, u_y, T); TVLBM_REF_MEAN: the row averages of the populations) and
// re-encode.
int refresh_reference_rows(tvlbm_ctx* c) {
    if (!ensure_reference_buffers(c)) return fail(c, TVLBM_ENOMEM, "reference tables");
    const bool mean = c->ref_kind == TVLBM_REF_MEAN;
    if (mean)
        TVLBM_CUDA(c, c->kt->row_pop_means(c->storage, fcur(c), c->ref_prof, c->kp, c->stream), "row means kernel");
    else
        TVLBM_CUDA(c, c->kt->row_means(c->storage, fcur(c), c->ref_prof, c->kp, c->stream), "row means kernel");
    return install_reference_rows(c, mean);
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
    for (int k = 0; k < 2; ++k)
        if (c->cl_graph[k]) cudaGraphExecDestroy(c->cl_graph[k]);
    if (c->fv_omega) cudaFree(c->fv_omega);
    if (c->fv_dy) cudaFree(c->fv_dy);
    if (c->fv_wall_eq) cudaFree(c->fv_wall_eq);
    if (c->mesh_mem) cudaFree(c->mesh_mem);
    if (c->ref_mem) cudaFree(c->ref_mem);
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
    if (form != FORM_PLAIN && form != FORM_TILED && form != FORM_FLOW && form != FORM_STRIP)
        return fail(c, TVLBM_EINVAL, "unknown form %d", form);
    if (form != FORM_PLAIN && !c->have_tmap)
        return fail(c, TVLBM_EINVAL, "tiled forms not available (no TMA descriptor for this storage/driver)");
    if (form != FORM_PLAIN && c->mesh_mem)
        return fail(c, TVLBM_EINVAL, "a non-uniform mesh runs the plain form only");
    int tiles_x = 0, tiles_y = 0;
    if (form == FORM_FLOW && !flow_tiles(c, c->tile_cfg, &tiles_x, &tiles_y))
        return fail(c, TVLBM_EINVAL,
                    "dataflow form needs a periodic domain that tile configuration %d covers exactly", c->tile_cfg);
    if (form != c->form) drop_graphs(c);
    c->form = form;
    return TVLBM_OK;
}

int tvlbm_set_graphs(tvlbm_ctx* c, int enable) {
    if (!c) return TVLBM_EINVAL;
    c->graphs = enable ? 1 : 0;
    return TVLBM_OK;
}


int tvlbm_set_reference(tvlbm_ctx* c, double ux, double uy, double T) {
    if (!c) return TVLBM_EINVAL;
    if (c->storage == TVLBM_FP64 || c->storage == TVLBM_FP32)
        return fail(c, TVLBM_EINVAL, "the reference applies to deviation storage only");
    if (!(T > 0.0) || !isfinite(T) || !isfinite(ux) || !isfinite(uy))
        return fail(c, TVLBM_EINVAL, "reference needs T > 0 and a finite velocity");
    cudaSetDevice(c->device);
    if (!ensure_reference_buffers(c)) return fail(c, TVLBM_ENOMEM, "re-encoding table");
    KParams np = c->kp;
    set_reference_params(np, c->rule, c->rho0, ux, uy, T);
    TVLBM_CUDA(c, reencode_between(c, ref_side_of(c->kp), ref_side_of(np)), "re-encoding");
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "reencode synchronize");
    c->kp = np;
    c->ref_every = 0;
    c->ref_count = 0;
    drop_graphs(c);
    return TVLBM_OK;
}

static int rows_applicable(tvlbm_ctx* c) {
    if (c->mesh_mem) return fail(c, TVLBM_EINVAL, "a non-uniform mesh takes no per-row reference");
    if (c->storage == TVLBM_FP64 || c->storage == TVLBM_FP32)
        return fail(c, TVLBM_EINVAL, "the reference applies to deviation storage only");
    if (!c->kp.walls) return fail(c, TVLBM_EINVAL, "a per-row reference needs a domain with walls");
    return TVLBM_OK;
}

int tvlbm_set_reference_rows(tvlbm_ctx* c, const double* ux, const double* uy, const double* T) {
    if (!c) return TVLBM_EINVAL;
    int rc = rows_applicable(c);
    if (rc) return rc;
    if (!ux || !uy || !T) return fail(c, TVLBM_EINVAL, "null profile");
    for (int y = 0; y < c->ny; ++y)
        if (!(T[y] > 0.0) || !isfinite(T[y]) || !isfinite(ux[y]) || !isfinite(uy[y]))
            return fail(c, TVLBM_EINVAL, "row %d: the reference needs T > 0 and a finite velocity", y);
    cudaSetDevice(c->device);
    if (!ensure_reference_buffers(c)) return fail(c, TVLBM_ENOMEM, "reference tables");
    const double* src[3] = {ux, uy, T};
    for (int k = 0; k < 3; ++k)
        TVLBM_CUDA(c, cudaMemcpyAsync(c->ref_prof + (size_t)k * c->ny, src[k], c->ny * sizeof(double),
                                      cudaMemcpyHostToDevice, c->stream), "profile upload");
    rc = install_reference_rows(c, false);
    if (rc) return rc;
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "reference synchronize");
    return TVLBM_OK;
}

int tvlbm_set_reference_refresh(tvlbm_ctx* c, int every) {
    if (!c) return TVLBM_EINVAL;
    if (every < 0) return fail(c, TVLBM_EINVAL, "negative refresh period");
    if (every == 0) {
        c->ref_every = 0;
        c->ref_count = 0;
        return TVLBM_OK;
    }
    int rc = rows_applicable(c);
    if (rc) return rc;
    cudaSetDevice(c->device);
    if (!c->kp.rowf) {
        rc = refresh_reference_rows(c);
        if (rc) return rc;
    }
    c->ref_every = every;
    c->ref_count = 0;
    return TVLBM_OK;
}

int tvlbm_set_reference_kind(tvlbm_ctx* c, int kind) {
    if (!c) return TVLBM_EINVAL;
    if (kind != TVLBM_REF_EQUILIBRIUM && kind != TVLBM_REF_MEAN) return fail(c, TVLBM_EINVAL, "unknown reference kind %d", kind);
    const int rc = rows_applicable(c);
    if (rc) return rc;
    c->ref_kind = kind;
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
    int tiles_x = 0, tiles_y = 0;
    if (c->form == FORM_FLOW && !flow_tiles(c, config, &tiles_x, &tiles_y))
        return fail(c, TVLBM_EINVAL, "tile configuration %d does not cover the domain exactly (dataflow form)", config);
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
    cudaSetDevice(c->device);
    const int rc = upload_fields_and_init(c, rho, ux, uy, T);  // checks the fields on the device first
    if (rc == TVLBM_OK) c->cur = 0;
    return rc;
}

static int run_steps(tvlbm_ctx* c, int n);

int tvlbm_step(tvlbm_ctx* c, int n) {
    if (!c) return TVLBM_EINVAL;
    if (n < 0) return fail(c, TVLBM_EINVAL, "negative step count");
    cudaSetDevice(c->device);
    if (c->scheme == TVLBM_SCHEME_FVLB) return fvlb_steps(c, n);
    if (c->form == FORM_FLOW) {
        TVLBM_CUDA(c, launch_flow(c, n, c->stream), "dataflow launch");
        return TVLBM_OK;
    }
    if (c->ref_every > 0) {  // per-row reference following the flow: refresh between chunks
        while (n > 0) {
            const int chunk = n < c->ref_every - c->ref_count ? n : c->ref_every - c->ref_count;
            const int rc = run_steps(c, chunk);
            if (rc) return rc;
            n -= chunk;
            c->ref_count += chunk;
            if (c->ref_count >= c->ref_every) {
                const int rr = refresh_reference_rows(c);
                if (rr) return rr;
                c->ref_count = 0;
            }
        }
        return TVLBM_OK;
    }
    return run_steps(c, n);
}

static int run_steps(tvlbm_ctx* c, int n) {
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
    TVLBM_CUDA(c, c->mesh_mem ? mesh_reduce(c, fcur(c), part, sums, c->stream)
                              : c->kt->reduce(c->storage, fcur(c), part, sums, c->kp, c->stream),
               "reduction kernels");
    TVLBM_CUDA(c, cudaMemcpyAsync(out, sums, 5 * sizeof(double), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync sums");
    TVLBM_CUDA(c, cudaStreamSynchronize(c->stream), "sums synchronize");
    const int rc = check_status(c);
    if (rc) return rc;
    if (out[4] > 0.0) return fail(c, TVLBM_ENONFINITE, "%.0f stored populations are not finite", out[4]);
    return TVLBM_OK;
}

int tvlbm_set_flow_wait(tvlbm_ctx* c, double limit_s, int unmet) {
    if (!c) return TVLBM_EINVAL;
    if (!(limit_s >= 1e-6 && limit_s <= 2.0)) return fail(c, TVLBM_EINVAL, "wait limit %g s outside [1e-6, 2]", limit_s);
    if (unmet < 0) return fail(c, TVLBM_EINVAL, "negative unmet count");
    c->flow_wait_ns = (long long)(limit_s * 1e9);
    c->flow_wait_extra = unmet ? (1 << 30) : 0;
    return TVLBM_OK;
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
