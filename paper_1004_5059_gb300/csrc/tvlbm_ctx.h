// Private: the single-domain context behind the opaque tvlbm_ctx handle of include/tvlbm.h,
// shared by the translation units that launch work on it (tvlbm_api.cu, tvlbm_closure.cu).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include "tvlbm.h"
#include "tvlbm_host.h"
#include "tvlbm_kernels.cuh"

namespace tvlbm {
// Gather tables of a mesh non-uniform in y (tvlbm_set_y_faces, tvlbm_mesh.cu): cell y spans
// [F_y, F_{y+1}], height h_y; x stays uniform.
struct MeshDev {
    int k;             // entries per (y-node, row) of the gather table
    int kb;            // entries per y-node of the wall tables
    const int* src;    // [n1][ny][k] source row of each entry (-1 / ny: beyond the bottom / top wall)
    const double* wd;  // [n1][ny][k] its weight |shifted row interval within the source| / h_y (0 pads)
    const float* wf;
    const int* bsrc;   // [n1][kb] fluid rows whose image crosses the wall that node j moves towards
    const double* bd;  // [n1][kb] the length beyond that wall (0 pads)
    const float* bf;
    const double* h;   // [ny] cell heights
};
}  // namespace tvlbm

struct tvlbm_ctx {
    int nx, ny, velset, n1, Q, N, storage, form, graphs;
    double tau, dt, rho0;
    tvlbm_bc bc;
    tvlbm::host::Rule rule;
    tvlbm::host::Layout L;
    tvlbm::KParams kp;
    const tvlbm::KernelTable* kt;
    int device;
    unsigned char* mem;
    bool own_mem;
    int cur;
    cudaStream_t stream;
    cudaStream_t capture_stream;
    cudaGraphExec_t graph[2];
    int have_tmap;
    int tile_cfg;                     // tiled-form tile configuration
    alignas(64) CUtensorMap tmap[2];  // TMA descriptors: input windows of buffer b
    alignas(64) CUtensorMap smap[2];  //   and one tile of buffer b (the dataflow form's TMA stores)
    alignas(64) CUtensorMap rmap[2];  //   and one source row of buffer b (the warp-strip form)
    int scheme;                       // TVLBM_SCHEME_VOLUMETRIC or TVLBM_SCHEME_FVLB
    double tau_g;                     // Prandtl-term time of the finite-volume scheme (inf: none)
    void* fv_omega;                   // finite-volume scheme: collision-term buffer (own allocation)
    double* fv_dy;                    // finite-volume channel: node spacings in y [ny - 1] (device; null: 1)
    double* fv_wall_eq;               // finite-volume channel: wall equilibria [2][nx][2] (device)
    int fv_exact, fv_nr_iters;        // finite-volume channel: Newton-Raphson imposition, iterations
    int fv_pscale;                    // finite-volume scheme: tau, tau_g divided by the local pressure
    int fv_split;                     // finite-volume scheme: two kernels per step (0: one fused kernel)
    unsigned char* mesh_mem;          // non-uniform y mesh: one device allocation holding the tables
    tvlbm::MeshDev mesh;              //   (null: unit cells)
    unsigned char* ref_mem;           // per-row deviation reference: one device allocation holding
    double* ref_rowd;                 //   the live tables (KParams::rowd / rowf),
    float* ref_rowf;
    double* ref_new_d;                //   the pair the next reference is built in,
    float* ref_new_f;
    float* ref_delta;                 //   the re-encoding shifts [rows][kMaxQ]
    double* ref_prof;                 //   and the profile ([3][ny] (ux, uy, T), or [Q][ny] Pref)
    int ref_every, ref_count;         // refresh period in steps (0: off), steps since the last refresh
    int ref_kind;                     // what a refresh installs: TVLBM_REF_EQUILIBRIUM or TVLBM_REF_MEAN
    long long flow_wait_ns;           // dataflow form: limit of the producer's neighbourhood wait
    int flow_wait_extra;              //   and the unreachable count a failure-path test adds (0)
    cudaGraphExec_t cl_graph[2];      // learned coarse steps: two steps per graph, by start parity
    unsigned long long cl_key_net;    // the network and constants the graphs were captured with
    float cl_key[24];
    char err[512];
};

// Finite-volume scheme (tvlbm_fvlb.cu): n explicit steps of the context's state.
int fvlb_steps(tvlbm_ctx* c, int n);

// Non-uniform y mesh (tvlbm_mesh.cu): one time step from fin into fout (the wall fill, then the
// sweep), and the FP64 conserved sums weighted by the cell heights.
cudaError_t mesh_launch_step(tvlbm_ctx* c, const void* fin, void* fout, cudaStream_t s);
cudaError_t mesh_reduce(tvlbm_ctx* c, const void* f, double* partials, double* out5, cudaStream_t s);
