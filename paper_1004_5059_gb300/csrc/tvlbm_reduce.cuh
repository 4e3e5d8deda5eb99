// FP64 conserved sums (mass, momentum, energy, and a count of non-finite stored values) in a
// fixed order, so that the result does not depend on scheduling: pass 1 runs a fixed grid of
// kRedBlocks blocks, each summing the cells c = blockIdx.x * blockDim.x + threadIdx.x + k * stride
// in order and then folding its threads with a fixed-shape shuffle tree; pass 2 folds the
// kRedBlocks partials [kRedBlocks][5] = (M, P_x, P_y, E, non-finite count) in one block.
// The moments are those of the velocity set's quadrature (Sec. "The TVLBM model"):
//     M = sum f_l,  P = sum c_l f_l,  E = sum |c_l|^2 f_l / 2,
// taken per row j of the tensor-product set from the node coordinates xd[] (c_l = (x_i, x_j)).
// The cell source is a template parameter, so the context's ghost-framed storage and a packed
// caller-owned array share one summation body (and hence one cell order); a source may weight
// each cell (its size on a non-uniform mesh: the conserved quantities are the size-weighted sums).
#pragma once

#include "tvlbm_kernels.cuh"

namespace tvlbm {

__device__ __forceinline__ double red_warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// A context's storage: ghost-framed planes, deviations read against rho0 + the row's reference.
template <class C>
struct FramedCells {
    const typename C::T* f;
    struct Cell {
        int x, y;
    };
    __device__ long long count(const KParams& p) const { return (long long)p.nx * p.ny; }
    __device__ Cell at(const KParams& p, long long c) const {
        const int y = (int)(c / p.nx);
        return {(int)(c - (long long)y * p.nx), y};
    }
    __device__ double value(const KParams& p, const Cell& k, int l) const { return (double)C::ld(f + sidx(p, l, k.x, k.y)); }
    __device__ double base(const KParams& p, const Cell& k, int l) const { return p.rho0d + kPrefRow<double>(p, l, k.y); }
    __device__ double weight(const KParams&, const Cell&) const { return 1.0; }
};

// A packed caller-owned array: population l of cell c = y * nx + x at f[l * ncell + c], deviations
// read against one rho0.
template <class C>
struct PackedCells {
    const typename C::T* f;
    int ncell;
    double rho0;
    struct Cell {
        int c;
    };
    __device__ long long count(const KParams&) const { return ncell; }
    __device__ Cell at(const KParams&, long long c) const { return {(int)c}; }
    __device__ double value(const KParams&, const Cell& k, int l) const { return (double)C::ld(f + l * ncell + k.c); }
    __device__ double base(const KParams&, const Cell&, int) const { return rho0; }
    __device__ double weight(const KParams&, const Cell&) const { return 1.0; }
};

// Pass 1 body: p supplies the node coordinates xd[] and marginal weights wd[] (w_l = wd_i wd_j).
template <int N1, class C, class Cells>
__device__ __forceinline__ void reduce_cells(const Cells& cells, double* __restrict__ partials, const KParams& p) {
    double acc[5] = {0, 0, 0, 0, 0};
    const long long ncell = cells.count(p);
    for (long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x; c < ncell;
         c += (long long)gridDim.x * blockDim.x) {
        const typename Cells::Cell k = cells.at(p, c);
        const double hw = cells.weight(p, k);  // the cell's size where cells differ (else 1)
#pragma unroll
        for (int j = 0; j < N1; ++j) {
            double r = 0, rx = 0, rxx = 0;
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                const double v = cells.value(p, k, l);
                acc[4] += isfinite(v) ? 0.0 : 1.0;
                const double fv = to_f<C, double>(v, p.wd[i] * p.wd[j], cells.base(p, k, l)) * hw;
                r += fv;
                rx += p.xd[i] * fv;
                rxx += p.xd[i] * p.xd[i] * fv;
            }
            acc[0] += r;
            acc[1] += rx;
            acc[2] += p.xd[j] * r;
            acc[3] += 0.5 * (rxx + p.xd[j] * p.xd[j] * r);
        }
    }
    __shared__ double sh[5][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double v = red_warp_sum(acc[k]);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
        partials[(long long)blockIdx.x * 5 + threadIdx.x] = t;
    }
}

template <int N1, class C>
__global__ void __launch_bounds__(256) reduce_kernel(const typename C::T* __restrict__ f, double* __restrict__ partials,
                                                     const KParams p) {
    reduce_cells<N1, C>(FramedCells<C>{f}, partials, p);
}

template <int N1, class C>
__global__ void __launch_bounds__(256) reduce_packed_kernel(const typename C::T* __restrict__ f, int ncell, double rho0,
                                                            double* __restrict__ partials, const KParams p) {
    reduce_cells<N1, C>(PackedCells<C>{f, ncell, rho0}, partials, p);
}

// Pass 2: one block folds the kRedBlocks partials in a fixed order into out5.
static __global__ void __launch_bounds__(256) reduce_final_kernel(const double* __restrict__ partials,
                                                                  double* __restrict__ out5) {
    __shared__ double sh[5][8];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < kRedBlocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; ++k) acc[k] += partials[(long long)b * 5 + k];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 5; ++k) {
        const double v = red_warp_sum(acc[k]);
        if (lane == 0) sh[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 5) {
        double t = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[threadIdx.x][w];
        out5[threadIdx.x] = t;
    }
}

}  // namespace tvlbm
