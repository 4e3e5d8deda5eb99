// Batched domains: many independent periodic grids of different sizes and relaxation times,
// advanced together.  Tiled form: each time step is one launch of the tiled sweep over a
// work-list of the tiles of every domain (per-tile domain index, per-domain geometry and
// relaxation table, TMA descriptors per domain), and multi-step runs replay captured CUDA
// graphs.  Dataflow form: n time steps of every domain are one persistent launch (the
// single-domain dataflow kernel over the batch's tile list, each tile waiting on its domain's
// 3 x 3 neighbourhood), replayed from a captured graph.  Per-domain operations off the hot path
// (initialisation, moments, sums, population I/O) reuse the single-domain kernels with that
// domain's parameters.
#include <cuda.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <new>
#include <vector>

#include "tvlbm.h"
#include "tvlbm_host.h"
#include "tvlbm_kernels.cuh"
#include "tvlbm_tiled.cuh"

using namespace tvlbm;
using namespace tvlbm::host;

namespace {

constexpr int kBatchGraphSteps = 32;  // steps per captured graph (even: parity preserved)

struct DomainHost {
    int nx, ny;
    double tau;
    Layout L;       // layout of this domain's buffers (offsets relative to off_base)
    size_t off;     // byte offset of this domain's first buffer in the batch block
    KParams kp;     // single-domain parameters (init, moments, sums, I/O)
};

struct BatchLayout {
    size_t tables_off, dom_bytes, maps_off, maps_bytes, tiles_off, tiles_bytes;
    size_t smaps_off, flow_off, flow_bytes;  // tile-store descriptors, dataflow counters
    size_t scratch_off, scratch_bytes, part_off, sums_off, status_off, total;
    int max_tiles;
};

}  // namespace

struct tvlbm_batch {
    int count, velset, n1, Q, N, storage, tile_cfg, graphs, device, cur, ntiles;
    int form;                      // TVLBM_FORM_TILED or TVLBM_FORM_FLOW
    cudaGraphExec_t flow_graph[2]; // dataflow form: one captured launch of flow_graph_n steps, by start parity
    int flow_graph_n;
    double dt, rho0;
    Rule rule;
    std::vector<DomainHost> dom;
    BatchLayout B;
    const KernelTable* kt;
    KParams kp0;  // velocity set and constants shared by all domains
    unsigned char* mem;
    bool own_mem;
    cudaStream_t stream, capture_stream;
    cudaGraphExec_t graph[2];
    char err[512];
};

namespace {

int bfail(tvlbm_batch* b, int code, const char* fmt, ...) {
    if (b) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(b->err, sizeof(b->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

#define BCUDA(b, call, what)                                                                              \
    do {                                                                                                  \
        cudaError_t e_ = (call);                                                                          \
        if (e_ != cudaSuccess) return bfail(b, TVLBM_ECUDA, "%s: %s (%s)", what, cudaGetErrorName(e_),    \
                                            cudaGetErrorString(e_));                                      \
    } while (0)

int tiles_for(const std::vector<DomainHost>& dom, int tx, int ty) {
    long long n = 0;
    for (const DomainHost& d : dom) n += (long long)((d.nx + tx - 1) / tx) * ((d.ny + ty - 1) / ty);
    return n > 2147483647LL ? -1 : (int)n;
}

// Lay out all domains' buffers, then the tables and scratch.
bool make_batch_layout(std::vector<DomainHost>& dom, int Q, int storage, BatchLayout* B, const KernelTable* kt) {
    size_t off = 0;
    long long max_cells = 0;
    for (DomainHost& d : dom) {
        d.L = make_layout(d.nx, d.ny, Q, storage);
        d.off = off;
        off += 2 * d.L.buf_bytes;
        if ((long long)d.nx * d.ny > max_cells) max_cells = (long long)d.nx * d.ny;
    }
    int max_tiles = 0;
    for (int cfg = 0; cfg < kTileConfigs; ++cfg) {
        int tx, ty, r;
        kt->tile_shape(storage, cfg, &tx, &ty, &r);
        const int n = tiles_for(dom, tx, ty);
        if (n < 0) return false;
        if (n > max_tiles) max_tiles = n;
    }
    B->max_tiles = max_tiles;
    B->tables_off = align_up(off, 256);
    B->dom_bytes = align_up(dom.size() * sizeof(BatchDomain), 256);
    B->maps_off = B->tables_off + B->dom_bytes;
    B->maps_bytes = align_up(dom.size() * 2 * sizeof(CUtensorMap), 256);
    B->tiles_off = B->maps_off + B->maps_bytes;
    B->tiles_bytes = align_up((size_t)max_tiles * sizeof(int), 256);
    B->smaps_off = B->tiles_off + B->tiles_bytes;
    B->flow_off = B->smaps_off + B->maps_bytes;
    B->flow_bytes = align_up(((size_t)kFlowDone + max_tiles) * sizeof(int), 256);
    B->scratch_off = B->flow_off + B->flow_bytes;
    B->scratch_bytes = align_up((size_t)max_cells * 4 * sizeof(double), 256);
    B->part_off = B->scratch_off + B->scratch_bytes;
    B->sums_off = B->part_off + align_up((size_t)kRedBlocks * 5 * sizeof(double), 256);
    B->status_off = B->sums_off + 128;
    B->total = B->sums_off + 256;
    return true;
}

int validate_batch(int count, const int* nx, const int* ny, const double* tau, int velset, int storage, double dt,
                   double rho0, char* msg, size_t len) {
    if (count < 1 || !nx || !ny) { snprintf(msg, len, "need at least one domain"); return TVLBM_EINVAL; }
    for (int d = 0; d < count; ++d) {
        const int rc = validate(nx[d], ny[d], velset, tau ? tau[d] : 1.0, dt, nullptr, storage, rho0, msg, len);
        if (rc) return rc;
    }
    return TVLBM_OK;
}

unsigned char* bptr(tvlbm_batch* b, size_t off) { return b->mem + off; }
void* dom_buf(tvlbm_batch* b, int d, int which) { return bptr(b, b->dom[d].off + b->dom[d].L.off_f[which]); }

// Device tables of the current tile configuration: per-domain geometry, descriptors, tile list.
int upload_tables(tvlbm_batch* b) {
    int tx, ty, r, bx, by;
    b->kt->tile_shape(b->storage, b->tile_cfg, &tx, &ty, &r);
    b->kt->tiled_box(b->storage, b->tile_cfg, &bx, &by);
    const size_t es = elem_size(b->storage);
    std::vector<BatchDomain> tab(b->count);
    std::vector<CUtensorMap> maps(2 * b->count), smaps(2 * b->count);
    std::vector<int> tiles;
    tiles.reserve(b->B.max_tiles);
    for (int d = 0; d < b->count; ++d) {
        const DomainHost& D = b->dom[d];
        BatchDomain& T = tab[d];
        memset(&T, 0, sizeof(T));
        T.off[0] = (long long)((D.off + D.L.off_f[0]) / es);
        T.off[1] = (long long)((D.off + D.L.off_f[1]) / es);
        T.plane = D.L.plane;
        T.nx = D.nx;
        T.ny = D.ny;
        T.pitch = D.L.pitch;
        T.tiles_x = (D.nx + tx - 1) / tx;
        T.tiles_y = (D.ny + ty - 1) / ty;
        T.tile_begin = (int)tiles.size();
        T.omegad = b->dt / D.tau;
        T.omegaf = (float)T.omegad;
        const int nt = T.tiles_x * ((D.ny + ty - 1) / ty);
        for (int k = 0; k < nt; ++k) tiles.push_back(d);
        for (int w = 0; w < 2; ++w)
            if (!encode_tensor_map(&maps[2 * d + w], dom_buf(b, d, w), b->storage, D.L, b->Q, bx, by) ||
                !encode_tensor_map(&smaps[2 * d + w], dom_buf(b, d, w), b->storage, D.L, b->Q, tx, ty))
                return bfail(b, TVLBM_ECUDA, "could not encode the TMA descriptors of domain %d", d);
    }
    b->ntiles = (int)tiles.size();
    BCUDA(b, cudaMemcpyAsync(bptr(b, b->B.tables_off), tab.data(), tab.size() * sizeof(BatchDomain),
                             cudaMemcpyHostToDevice, b->stream), "upload domain table");
    BCUDA(b, cudaMemcpyAsync(bptr(b, b->B.maps_off), maps.data(), maps.size() * sizeof(CUtensorMap),
                             cudaMemcpyHostToDevice, b->stream), "upload descriptors");
    BCUDA(b, cudaMemcpyAsync(bptr(b, b->B.smaps_off), smaps.data(), smaps.size() * sizeof(CUtensorMap),
                             cudaMemcpyHostToDevice, b->stream), "upload descriptors");
    BCUDA(b, cudaMemcpyAsync(bptr(b, b->B.tiles_off), tiles.data(), tiles.size() * sizeof(int),
                             cudaMemcpyHostToDevice, b->stream), "upload tile list");
    BCUDA(b, cudaStreamSynchronize(b->stream), "table upload synchronize");
    return TVLBM_OK;
}

void drop_batch_graphs(tvlbm_batch* b) {
    for (int k = 0; k < 2; ++k) {
        if (b->graph[k]) {
            cudaGraphExecDestroy(b->graph[k]);
            b->graph[k] = nullptr;
        }
        if (b->flow_graph[k]) {
            cudaGraphExecDestroy(b->flow_graph[k]);
            b->flow_graph[k] = nullptr;
        }
    }
    b->flow_graph_n = 0;
}

// Whether tile configuration cfg covers every domain exactly with tiles of at least 4 rows (what
// the dataflow form needs: a tile's sources and frame images lie in its 3 x 3 neighbourhood).
bool batch_flow_tiles(const tvlbm_batch* b, int cfg) {
    int tx = 0, ty = 0, r = 0;
    b->kt->tile_shape(b->storage, cfg, &tx, &ty, &r);
    if (tx < 32 || ty < 4) return false;
    for (const DomainHost& D : b->dom)
        if (D.nx % tx || D.ny % ty) return false;
    return true;
}

// n time steps of every domain in dataflow launches from start parity `parity` on stream s (tasks
// per launch below 2^30, steps per launch at most 2^24: the completion counters stay in an int).
cudaError_t launch_batch_flow(tvlbm_batch* b, int n, int parity, cudaStream_t s) {
    const int chunk_max = (1 << 30) / b->ntiles < (1 << 24) ? (1 << 30) / b->ntiles : (1 << 24);
    int* ctr = (int*)bptr(b, b->B.flow_off);
    while (n > 0) {
        const int chunk = n < chunk_max ? n : chunk_max;
        BatchFlowSrc src;
        memset(&src, 0, sizeof(src));
        src.dom = (const BatchDomain*)bptr(b, b->B.tables_off);
        src.lmaps = (const CUtensorMap*)bptr(b, b->B.maps_off);
        src.smaps = (const CUtensorMap*)bptr(b, b->B.smaps_off);
        src.tile_dom = (const int*)bptr(b, b->B.tiles_off);
        src.base = b->mem;
        src.es = (int)elem_size(b->storage);
        src.cur = parity;
        src.ntiles = b->ntiles;
        src.nsteps = chunk;
        src.next_task = ctr;
        src.abort = ctr + 1;
        src.done = ctr + kFlowDone;
        src.wait_ns = (long long)kWaitLimitNs;
        src.wait_extra = 0;
        cudaError_t e = cudaMemsetAsync(ctr, 0, ((size_t)kFlowDone + b->ntiles) * sizeof(int), s);
        if (e == cudaSuccess) e = b->kt->batch_flow(b->storage, b->tile_cfg, src, b->kp0, s);
        if (e != cudaSuccess) return e;
        parity ^= chunk & 1;
        n -= chunk;
    }
    return cudaSuccess;
}

// The dataflow form's n steps from start parity `parity`, captured once as a graph (n fixed by
// the first call; a call with another n launches directly).
int build_flow_graph(tvlbm_batch* b, int n, int parity) {
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    const cudaError_t le = launch_batch_flow(b, n, parity, b->capture_stream);
    const cudaError_t ce = cudaStreamEndCapture(b->capture_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, TVLBM_ECUDA, "launch during capture: %s", cudaGetErrorString(le));
    }
    if (ce != cudaSuccess) return bfail(b, TVLBM_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&b->flow_graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        b->flow_graph[parity] = nullptr;
        return bfail(b, TVLBM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
    }
    return TVLBM_OK;
}

cudaError_t launch_batch_step(tvlbm_batch* b, int parity, cudaStream_t s) {
    BatchSrc src;
    src.dom = (const BatchDomain*)bptr(b, b->B.tables_off);
    src.maps = (const CUtensorMap*)bptr(b, b->B.maps_off);
    src.tile_dom = (const int*)bptr(b, b->B.tiles_off);
    src.base = b->mem;
    src.ntiles = b->ntiles;
    src.parity = parity;
    src.es = (int)elem_size(b->storage);
    return b->kt->batch_sweep(b->storage, b->tile_cfg, src, b->kp0, s);
}

int build_batch_graph(tvlbm_batch* b, int parity) {
    cudaGraph_t g = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->capture_stream, cudaStreamCaptureModeThreadLocal), "cudaStreamBeginCapture");
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < kBatchGraphSteps && le == cudaSuccess; ++k) le = launch_batch_step(b, (parity + k) & 1, b->capture_stream);
    const cudaError_t ce = cudaStreamEndCapture(b->capture_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, TVLBM_ECUDA, "launch during capture: %s", cudaGetErrorString(le));
    }
    if (ce != cudaSuccess) return bfail(b, TVLBM_ECUDA, "cudaStreamEndCapture: %s", cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(&b->graph[parity], g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) {
        b->graph[parity] = nullptr;
        return bfail(b, TVLBM_ECUDA, "cudaGraphInstantiate: %s", cudaGetErrorString(ie));
    }
    return TVLBM_OK;
}

// Per-domain parameters for the single-domain kernels, pointing at the batch's scratch.
KParams domain_params(tvlbm_batch* b, int d) {
    KParams p = b->dom[d].kp;
    p.status = (int*)bptr(b, b->B.status_off);
    return p;
}

int check_batch_status(tvlbm_batch* b) {
    int st = 0;
    int* d = (int*)bptr(b, b->B.status_off);
    BCUDA(b, cudaMemcpyAsync(&st, d, sizeof(int), cudaMemcpyDeviceToHost, b->stream), "status copy");
    BCUDA(b, cudaStreamSynchronize(b->stream), "status synchronize");
    if (st) {
        cudaMemsetAsync(d, 0, sizeof(int), b->stream);
        cudaStreamSynchronize(b->stream);
        return bfail(b, TVLBM_ETIMEOUT, "a device-side wait for a TMA load timed out (status %d)", st);
    }
    return TVLBM_OK;
}

int init_domain(tvlbm_batch* b, int d, const double* rho, const double* ux, const double* uy, const double* T) {
    const DomainHost& D = b->dom[d];
    const size_t n = (size_t)D.nx * D.ny;
    double* f = (double*)bptr(b, b->B.scratch_off);
    const double* src[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        BCUDA(b, cudaMemcpyAsync(f + k * n, src[k], n * sizeof(double), cudaMemcpyHostToDevice, b->stream), "fields copy");
    const KParams p = domain_params(b, d);
    for (int w = 0; w < 2; ++w) BCUDA(b, b->kt->init(b->storage, f, dom_buf(b, d, w), p, b->stream), "init kernel");
    BCUDA(b, cudaStreamSynchronize(b->stream), "init synchronize");
    return TVLBM_OK;
}

int create_batch(int count, const int* nx, const int* ny, const double* tau, int velset, int storage, double dt,
                 double rho0, void* device_memory, size_t bytes, tvlbm_batch** out) {
    if (!out || !tau) return TVLBM_EINVAL;
    *out = nullptr;
    char msg[256];
    int rc = validate_batch(count, nx, ny, tau, velset, storage, dt, rho0, msg, sizeof(msg));
    if (rc) return rc;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) return TVLBM_ECUDA;
    tvlbm_batch* b = new (std::nothrow) tvlbm_batch();
    if (!b) return TVLBM_ENOMEM;
    b->count = count;
    b->velset = velset;
    b->n1 = nodes_for(velset);
    b->Q = b->n1 * b->n1;
    b->N = b->n1 - 1;
    b->storage = storage;
    b->tile_cfg = 0;
    b->graphs = 1;
    b->dt = dt;
    b->rho0 = rho0;
    b->cur = 0;
    b->mem = nullptr;
    b->stream = nullptr;
    b->capture_stream = nullptr;
    b->graph[0] = b->graph[1] = nullptr;
    b->flow_graph[0] = b->flow_graph[1] = nullptr;
    b->flow_graph_n = 0;
    b->form = TVLBM_FORM_TILED;
    b->err[0] = 0;
    gauss_hermite_rule(b->n1, &b->rule);
    b->kt = table_for(b->n1);
    b->dom.resize(count);
    for (int d = 0; d < count; ++d) {
        b->dom[d].nx = nx[d];
        b->dom[d].ny = ny[d];
        b->dom[d].tau = tau[d];
    }
    if (!make_batch_layout(b->dom, b->Q, storage, &b->B, b->kt)) { delete b; return TVLBM_EINVAL; }
    tvlbm_bc periodic;
    memset(&periodic, 0, sizeof(periodic));
    for (int d = 0; d < count; ++d) {
        DomainHost& D = b->dom[d];
        fill_kparams(D.kp, b->rule, b->N, dt, D.tau, rho0, D.nx, D.ny, D.L, periodic);
    }
    b->kp0 = b->dom[0].kp;
    cudaGetDevice(&b->device);
    if (device_memory) {
        if (bytes < b->B.total || ((uintptr_t)device_memory & 255)) { delete b; return bytes < b->B.total ? TVLBM_ENOMEM : TVLBM_EINVAL; }
        b->mem = (unsigned char*)device_memory;
        b->own_mem = false;
    } else {
        const cudaError_t e = cudaMalloc((void**)&b->mem, b->B.total);
        if (e != cudaSuccess) { delete b; return e == cudaErrorMemoryAllocation ? TVLBM_ENOMEM : TVLBM_ECUDA; }
        b->own_mem = true;
    }
    b->kp0.status = (int*)bptr(b, b->B.status_off);
    if (cudaStreamCreateWithFlags(&b->capture_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaMemsetAsync(b->mem, 0, b->B.total, b->stream) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess) {
        tvlbm_batch_destroy(b);
        return TVLBM_ECUDA;
    }
    rc = upload_tables(b);
    if (rc) { tvlbm_batch_destroy(b); return rc; }
    // every domain starts at the rest equilibrium f = rho0 w
    for (int d = 0; d < count && !rc; ++d) {
        const size_t n = (size_t)nx[d] * ny[d];
        std::vector<double> h(4 * n);
        for (size_t k = 0; k < n; ++k) { h[k] = rho0; h[n + k] = 0.0; h[2 * n + k] = 0.0; h[3 * n + k] = 1.0; }
        rc = init_domain(b, d, h.data(), h.data() + n, h.data() + 2 * n, h.data() + 3 * n);
    }
    if (rc) { tvlbm_batch_destroy(b); return rc; }
    *out = b;
    return TVLBM_OK;
}

}  // namespace

extern "C" {

int tvlbm_batch_memory_bytes(int count, const int* nx, const int* ny, int velset, int storage, size_t* bytes) {
    if (!bytes) return TVLBM_EINVAL;
    char msg[256];
    const int rc = validate_batch(count, nx, ny, nullptr, velset, storage, 1.0 / 8.0, 1.0, msg, sizeof(msg));
    if (rc) return rc;
    std::vector<DomainHost> dom(count);
    for (int d = 0; d < count; ++d) {
        dom[d].nx = nx[d];
        dom[d].ny = ny[d];
    }
    BatchLayout B;
    const int n1 = nodes_for(velset);
    if (!make_batch_layout(dom, n1 * n1, storage, &B, table_for(n1))) return TVLBM_EINVAL;
    *bytes = B.total;
    return TVLBM_OK;
}

int tvlbm_batch_create(int count, const int* nx, const int* ny, const double* tau, int velset, int storage, double dt,
                       double rho0, tvlbm_batch** out) {
    return create_batch(count, nx, ny, tau, velset, storage, dt, rho0, nullptr, 0, out);
}

int tvlbm_batch_create_in(int count, const int* nx, const int* ny, const double* tau, int velset, int storage,
                          double dt, double rho0, void* device_memory, size_t bytes, tvlbm_batch** out) {
    if (!device_memory) return TVLBM_EINVAL;
    return create_batch(count, nx, ny, tau, velset, storage, dt, rho0, device_memory, bytes, out);
}

int tvlbm_batch_destroy(tvlbm_batch* b) {
    if (!b) return TVLBM_OK;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    drop_batch_graphs(b);
    if (b->capture_stream) cudaStreamDestroy(b->capture_stream);
    if (b->own_mem && b->mem) cudaFree(b->mem);
    delete b;
    return TVLBM_OK;
}

int tvlbm_batch_set_stream(tvlbm_batch* b, void* stream) {
    if (!b) return TVLBM_EINVAL;
    b->stream = (cudaStream_t)stream;
    return TVLBM_OK;
}

int tvlbm_batch_set_graphs(tvlbm_batch* b, int enable) {
    if (!b) return TVLBM_EINVAL;
    b->graphs = enable ? 1 : 0;
    return TVLBM_OK;
}

int tvlbm_batch_tile_count(const tvlbm_batch* b) { return b ? kTileConfigs : 0; }

int tvlbm_batch_tile_shape(const tvlbm_batch* b, int config, int* tx, int* ty, int* rows_per_thread) {
    if (!b || config < 0 || config >= kTileConfigs || !tx || !ty || !rows_per_thread) return TVLBM_EINVAL;
    b->kt->tile_shape(b->storage, config, tx, ty, rows_per_thread);
    return TVLBM_OK;
}

int tvlbm_batch_set_form(tvlbm_batch* b, int form) {
    if (!b) return TVLBM_EINVAL;
    if (form != TVLBM_FORM_TILED && form != TVLBM_FORM_FLOW) return bfail(b, TVLBM_EINVAL, "unknown batch form %d", form);
    if (form == TVLBM_FORM_FLOW && !batch_flow_tiles(b, b->tile_cfg))
        return bfail(b, TVLBM_EINVAL, "dataflow form needs every domain covered exactly by tile configuration %d",
                     b->tile_cfg);
    if (form != b->form) drop_batch_graphs(b);
    b->form = form;
    return TVLBM_OK;
}

int tvlbm_batch_set_tile(tvlbm_batch* b, int config) {
    if (!b) return TVLBM_EINVAL;
    if (config < 0 || config >= kTileConfigs) return bfail(b, TVLBM_EINVAL, "tile configuration %d out of range", config);
    if (config == b->tile_cfg) return TVLBM_OK;
    if (b->form == TVLBM_FORM_FLOW && !batch_flow_tiles(b, config))
        return bfail(b, TVLBM_EINVAL, "tile configuration %d does not cover every domain exactly (dataflow form)", config);
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    b->tile_cfg = config;
    drop_batch_graphs(b);
    return upload_tables(b);
}

int tvlbm_batch_init_moments(tvlbm_batch* b, int domain, const double* rho, const double* ux, const double* uy,
                             const double* T) {
    if (!b) return TVLBM_EINVAL;
    if (domain < 0 || domain >= b->count) return bfail(b, TVLBM_EINVAL, "domain %d out of range", domain);
    if (!rho || !ux || !uy || !T) return bfail(b, TVLBM_EINVAL, "null field pointer");
    const size_t n = (size_t)b->dom[domain].nx * b->dom[domain].ny;
    for (size_t k = 0; k < n; ++k)
        if (!(rho[k] > 0.0) || !(T[k] > 0.0) || !isfinite(rho[k]) || !isfinite(T[k]) || !isfinite(ux[k]) ||
            !isfinite(uy[k]))
            return bfail(b, TVLBM_EINVAL, "init field of domain %d invalid at cell %zu", domain, k);
    cudaSetDevice(b->device);
    return init_domain(b, domain, rho, ux, uy, T);
}

int tvlbm_batch_step(tvlbm_batch* b, int n) {
    if (!b) return TVLBM_EINVAL;
    if (n < 0) return bfail(b, TVLBM_EINVAL, "negative step count");
    cudaSetDevice(b->device);
    if (b->form == TVLBM_FORM_FLOW) {
        if (n == 0) return TVLBM_OK;
        if (b->graphs && (b->flow_graph_n == 0 || b->flow_graph_n == n)) {
            if (!b->flow_graph[b->cur]) {
                const int rc = build_flow_graph(b, n, b->cur);
                if (rc) return rc;
                b->flow_graph_n = n;
            }
            BCUDA(b, cudaGraphLaunch(b->flow_graph[b->cur], b->stream), "cudaGraphLaunch");
        } else {
            BCUDA(b, launch_batch_flow(b, n, b->cur, b->stream), "batch dataflow launch");
        }
        b->cur ^= n & 1;
        return TVLBM_OK;
    }
    int left = n;
    if (b->graphs) {
        while (left >= kBatchGraphSteps) {
            if (!b->graph[b->cur]) {
                const int rc = build_batch_graph(b, b->cur);
                if (rc) return rc;
            }
            BCUDA(b, cudaGraphLaunch(b->graph[b->cur], b->stream), "cudaGraphLaunch");
            left -= kBatchGraphSteps;
        }
    }
    for (; left > 0; --left) {
        BCUDA(b, launch_batch_step(b, b->cur, b->stream), "batch sweep launch");
        b->cur ^= 1;
    }
    return TVLBM_OK;
}

int tvlbm_batch_moments(tvlbm_batch* b, int domain, double* rho, double* ux, double* uy, double* T) {
    if (!b) return TVLBM_EINVAL;
    if (domain < 0 || domain >= b->count) return bfail(b, TVLBM_EINVAL, "domain %d out of range", domain);
    cudaSetDevice(b->device);
    const size_t n = (size_t)b->dom[domain].nx * b->dom[domain].ny;
    double* s = (double*)bptr(b, b->B.scratch_off);
    BCUDA(b, b->kt->moments(b->storage, dom_buf(b, domain, b->cur), s, domain_params(b, domain), b->stream),
          "moments kernel");
    double* dst[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        if (dst[k]) BCUDA(b, cudaMemcpyAsync(dst[k], s + k * n, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy");
    BCUDA(b, cudaStreamSynchronize(b->stream), "moments synchronize");
    return check_batch_status(b);
}

int tvlbm_batch_conserved_sums(tvlbm_batch* b, int domain, double out[5]) {
    if (!b || !out) return TVLBM_EINVAL;
    if (domain < 0 || domain >= b->count) return bfail(b, TVLBM_EINVAL, "domain %d out of range", domain);
    cudaSetDevice(b->device);
    double* part = (double*)bptr(b, b->B.part_off);
    double* sums = (double*)bptr(b, b->B.sums_off);
    BCUDA(b, b->kt->reduce(b->storage, dom_buf(b, domain, b->cur), part, sums, domain_params(b, domain), b->stream),
          "reduction");
    BCUDA(b, cudaMemcpyAsync(out, sums, 5 * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy sums");
    BCUDA(b, cudaStreamSynchronize(b->stream), "sums synchronize");
    const int rc = check_batch_status(b);
    if (rc) return rc;
    if (out[4] > 0.0) return bfail(b, TVLBM_ENONFINITE, "domain %d: %.0f stored populations are not finite", domain, out[4]);
    return TVLBM_OK;
}

int tvlbm_batch_get_populations_f64(tvlbm_batch* b, int domain, double* host) {
    if (!b || !host) return TVLBM_EINVAL;
    if (domain < 0 || domain >= b->count) return bfail(b, TVLBM_EINVAL, "domain %d out of range", domain);
    cudaSetDevice(b->device);
    const size_t n = (size_t)b->dom[domain].nx * b->dom[domain].ny;
    double* s = (double*)bptr(b, b->B.scratch_off);
    const KParams p = domain_params(b, domain);
    for (int l = 0; l < b->Q; ++l) {
        BCUDA(b, b->kt->decode_plane(b->storage, dom_buf(b, domain, b->cur), l, s, p, b->stream), "decode kernel");
        BCUDA(b, cudaMemcpyAsync(host + (size_t)l * n, s, n * sizeof(double), cudaMemcpyDeviceToHost, b->stream), "copy");
        BCUDA(b, cudaStreamSynchronize(b->stream), "decode synchronize");
    }
    return check_batch_status(b);
}

long long tvlbm_batch_cells(const tvlbm_batch* b) {
    if (!b) return 0;
    long long n = 0;
    for (const DomainHost& d : b->dom) n += (long long)d.nx * d.ny;
    return n;
}

double tvlbm_batch_bytes_per_cell(const tvlbm_batch* b) { return b ? 2.0 * b->Q * (double)elem_size(b->storage) : 0.0; }

const char* tvlbm_batch_last_error(const tvlbm_batch* b) { return b ? b->err : ""; }

}  // extern "C"
