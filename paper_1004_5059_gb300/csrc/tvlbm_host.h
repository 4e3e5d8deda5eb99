// Internal host helpers shared by the single-domain and batched APIs: velocity sets,
// streaming tables, memory layout, kernel parameters and TMA descriptors.
#pragma once

#include <cuda.h>
#include <cudaTypedefs.h>
#include <stddef.h>

#include "tvlbm.h"
#include "tvlbm_kernels.cuh"

namespace tvlbm {
namespace host {

struct Rule {
    int n;
    double x[kMaxN1], w[kMaxN1];
};

// n-point Gauss-Hermite rule (weight exp(-x^2/2)/sqrt(2 pi)), nodes ascending; false if n is out of range.
bool gauss_hermite_rule(int n, Rule* r);
// Nodes per axis of a velocity set (0 if unknown).
int nodes_for(int velset);
// Shift of one node over one step: x dt = sh + alpha (integer within 1e-12 -> alpha = 0).
void shift_of(double x, double dt, int* sh, double* alpha);
// He_a(x) / a!
double hermite_over_fact(int a, double x);
// Separable Hermite equilibrium f_eq_l(rho, u, T) in FP64 (f-space, l = i + n j).
void host_equilibrium(const Rule& r, double rho, double ux, double uy, double T, double* feq);
// Bytes per stored population (0 if unknown storage).
size_t elem_size(int storage);

struct Layout {
    int hx, pitch, rows;
    long long plane;
    size_t buf_bytes, mom_bytes, part_bytes, total;
    size_t off_f[2], off_mom, off_part, off_sums, off_status;
    size_t off_flow, flow_ints;  // counters of the multi-step dataflow launch
};
size_t align_up(size_t v, size_t a);
Layout make_layout(int nx, int ny, int Q, int storage);

const KernelTable* table_for(int n);

// Argument checks shared by every create call; writes a message on failure.
int validate(int nx, int ny, int velset, double tau, double dt, const tvlbm_bc* bc, int storage, double rho0,
             char* msg, size_t msglen);

// Kernel parameters of one domain (status pointer left null).
void fill_kparams(KParams& p, const Rule& r, int N, double dt, double tau, double rho0, int nx, int ny,
                  const Layout& L, const tvlbm_bc& bc);

// One deviation-storage reference R_l = f_eq_l(rho0, u_ref, T_ref) / w_l: Pref = R - rho0 in FP64
// and float, jref, eref and refD (the float Pref table's share of the FP32 constants' defects,
// see KParams); nonzero unless it is the default reference (0, 0, 1).
struct RefEntry {
    double Prefd[kMaxQ];
    float Preff[kMaxQ];
    double jrefd[2], erefd;
    float jreff[2], ereff, refD[4];
    bool nonzero;
};
RefEntry reference_entry(const KParams& p, const Rule& r, double rho0, double ux, double uy, double T);

// Single deviation-storage reference of the kernel parameters (Pref, jref, eref, refD, has_ref;
// clears the per-row tables); (0, 0, 1) is the default reference.
void set_reference_params(KParams& p, const Rule& r, double rho0, double ux, double uy, double T);

// TMA descriptor of one population buffer: a 3-D view [Q][rows][pitch], box bx x by x 1.
bool encode_tensor_map(CUtensorMap* m, void* base, int storage, const Layout& L, int Q, int bx, int by);
// The driver's cuTensorMapEncodeTiled (null if the driver does not provide it).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder();

}  // namespace host
}  // namespace tvlbm
