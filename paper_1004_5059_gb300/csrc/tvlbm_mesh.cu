// The volumetric (area-overlap) step on a mesh that is non-uniform in y: the grid refinement of
// Sec. "Grid Refinement for simple unidirectional flows" (Eqs. NONUNI1-2, cells crowded towards
// the walls) carried over to the volumetric scheme.  Cell y spans [F_y, F_{y+1}] (height h_y);
// x stays uniform.  A population moves rigidly by s = c dt in one step, so destination row y
// takes, per velocity, sum_r w_r f_r with w_r = |[F_y - s, F_{y+1} - s] within cell r| / h_y (on
// unit cells the uniform scheme's (1 - a, a) pair), and x keeps the uniform (1 - a_x, a_x) pair.
// With walls at F_0 and F_ny the part of the shifted interval beyond a wall is one entry naming
// the ghost row -1 or ny, which holds, per column, A(x) f_eq_l(1, u_w, T_w) for the incoming
// velocities, A = M_out / sum_in |c_y dt| f_eq_l, M_out(x) what the outgoing velocities carry
// beyond the wall (Eq. IMPOSITION: the uniform scheme's ghost-row rule, which is this rule on
// unit cells).  The mass sum_y h_y f_y is conserved; the FP64 sums are weighted by h_y.
// One plain sweep per step (after the wall kernel); the collision is the uniform scheme's.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "tvlbm.h"
#include "tvlbm_ctx.h"
#include "tvlbm_kernels_impl.cuh"

using namespace tvlbm;

namespace {

constexpr int kMaxMeshEntries = 64;  // gather entries per row (cells much thinner than c dt need more)

template <class R>
__device__ __forceinline__ const R* gather_weights(const MeshDev& m) {
    if constexpr (std::is_same<R, double>::value) return m.wd; else return m.wf;
}
template <class R>
__device__ __forceinline__ const R* wall_lengths(const MeshDev& m) {
    if constexpr (std::is_same<R, double>::value) return m.bd; else return m.bf;
}

// One time step of the fluid cells: gather along the mesh tables, collide, store (with the
// periodic images of the frame).  KT > 0: every row's list padded to KT entries (padding: weight
// 0 on the row's first source), unrolled so that all loads of a velocity are in flight together;
// KT = 0: a loop that ends at the first zero weight.  Both add the same terms in the same order.
template <int N1, class C>
constexpr int mesh_sweep_minb() {  // resident CTAs of 256 threads: 3 (85 registers) for FP32 up to D2Q16
    return (sizeof(typename C::R) == 4 && N1 <= 4) ? 3 : 1;
}

template <int N1, class C, int KT>
__global__ void __launch_bounds__(256, mesh_sweep_minb<N1, C>()) mesh_sweep_kernel(const typename C::T* __restrict__ fin,
                                                         typename C::T* __restrict__ fout, const KParams p,
                                                         const MeshDev m) {
    using R = typename C::R;
    using T = typename C::T;
    constexpr int Q = N1 * N1;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    if (x >= p.nx || y >= p.ny) return;
    R s[Q];
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        const long long e0 = ((long long)j * p.ny + y) * m.k;
        const int* src = m.src + e0;
        const R* wt = gather_weights<R>(m) + e0;
        if constexpr (KT > 0) {
            long long ro[KT];  // row offsets of the entries (same for every x-node of this y-node)
            R ws[KT];
#pragma unroll
            for (int k = 0; k < KT; ++k) {
                ro[k] = (long long)(__ldg(src + k) + HY) * p.pitch;
                ws[k] = __ldg(wt + k);
            }
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                const R ax = ka<R>(p, i);
                const T* col = fin + (long long)l * p.plane + (x + p.hx - p.sh[i]);
                R r[KT];
#pragma unroll
                for (int k = 0; k < KT; ++k) {
                    const R v = C::ld(col + ro[k]);
                    r[k] = fma(ax, C::ld(col + ro[k] - 1) - v, split_rest<C>(p, l, v));
                }
                // the first entry, then the others as lerps towards theirs (weights summing to
                // one: a state uniform in space stays exactly uniform)
                R acc = r[0];
#pragma unroll
                for (int k = 1; k < KT; ++k) acc = fma(ws[k], r[k] - r[0], acc);
                s[l] = acc;
            }
        } else {
#pragma unroll
            for (int i = 0; i < N1; ++i) {
                const int l = i + N1 * j;
                const R ax = ka<R>(p, i);
                const T* col = fin + (long long)l * p.plane + (x + p.hx - p.sh[i]);
                const T* b = col + (long long)(__ldg(src) + HY) * p.pitch;
                const R v0 = C::ld(b);
                const R r0 = fma(ax, C::ld(b - 1) - v0, split_rest<C>(p, l, v0));
                R acc = r0;
                for (int k = 1; k < m.k; ++k) {
                    const R wk = __ldg(wt + k);
                    if (wk == R(0)) break;  // the row's list has ended
                    const T* bk = col + (long long)(__ldg(src + k) + HY) * p.pitch;
                    const R vk = C::ld(bk);
                    const R rk = fma(ax, C::ld(bk - 1) - vk, split_rest<C>(p, l, vk));
                    acc = fma(wk, rk - r0, acc);
                }
                s[l] = acc;
            }
        }
    }
    const Geom g = geom_of(p);
    collide_cell<N1, C, false>(s, p, g, y);
    store_collided<N1, C>(fout, g, x, y, s);
}

// Threads per (column, outgoing velocity) of the wall kernel: each sums every CH-th crossing row.
template <int N1>
constexpr int mesh_wall_chunks() {
    return 1024 / (32 * wall_lanes<N1>()) >= 4 ? 4 : (1024 / (32 * wall_lanes<N1>()) >= 2 ? 2 : 1);
}

// The wall fill before a step: per wall and column (frame columns included), M_out(x) from the
// outgoing velocities' rows that cross the wall (after the x part of the gather), then the
// ghost row of every incoming velocity.  Threads (column, outgoing velocity, chunk c) sum the
// crossing rows c, c + CH, ...; the column's shares are added in a fixed order in shared memory.
template <int N1, class C>
__global__ void __launch_bounds__(32 * wall_lanes<N1>() * mesh_wall_chunks<N1>())
    mesh_wall_kernel(typename C::T* __restrict__ f, const KParams p, const MeshDev m) {
    using R = typename C::R;
    using T = typename C::T;
    constexpr int NL = wall_lanes<N1>(), CH = mesh_wall_chunks<N1>();
    __shared__ R part[CH][NL][32];
    __shared__ R amp[32];
    const int tx = threadIdx.x, k = threadIdx.y, c = threadIdx.z;
    const int side = blockIdx.y;                 // 0: wall at F_0, 1: wall at F_ny
    const int xo = blockIdx.x * 32 + tx - FILL;  // output column, in [-FILL, nx + FILL)
    const bool col = xo < p.nx + FILL;
    const int x = ((xo % p.nx) + p.nx) % p.nx;
    const int i = k % N1, jj = k / N1;
    const R rho0 = krho0<R>(p);
    {
        // nodes ascend: the N1 / 2 lowest y-nodes move towards the wall at F_0
        const int j = side == 0 ? jj : N1 - 1 - jj;
        const int l = i + N1 * j;
        const R ax = ka<R>(p, i), w = kw<R>(p, i) * kw<R>(p, j);
        const R ref = rho0 + kPrefRow<R>(p, l, 0);
        R acc = 0;
        if (col) {
            const int* src = m.bsrc + j * m.kb;
            const R* len = wall_lengths<R>(m) + j * m.kb;
            // padded entries (length 0 on row 0) add exact zeros: no data-dependent exit, so the
            // unrolled iterations' loads are in flight together
#pragma unroll 4
            for (int e = c; e < m.kb; e += CH) {
                const R le = __ldg(len + e);
                const T* b = f + sidx(p, l, x - p.sh[i], __ldg(src + e));
                acc += le * ((R(1) - ax) * to_f<C, R>(C::ld(b), w, ref) + ax * to_f<C, R>(C::ld(b - 1), w, ref));
            }
        }
        part[c][k][tx] = acc;
    }
    __syncthreads();
    if (k == 0 && c == 0) {
        R sum = 0;
        for (int kk = 0; kk < NL; ++kk)
            for (int cc = 0; cc < CH; ++cc) sum += part[cc][kk][tx];
        amp[tx] = sum * kinvden<R>(p, side);
    }
    __syncthreads();
    if (!col || c != 0) return;
    const int j = side == 0 ? N1 - 1 - jj : jj;  // the incoming velocity of this lane
    const int l = i + N1 * j;
    const R w = kw<R>(p, i) * kw<R>(p, j);
    const R fw = amp[tx] * kfeqw<R>(p, side, l);
    const int yd = side == 0 ? -1 : p.ny;
    f[sidx(p, l, xo, yd)] = C::enc(from_f<C, R>(fw, w, rho0 + kPrefRow<R>(p, l, yd)));
}

// The context's cells, each weighted by its height.
template <class C>
struct MeshCells : FramedCells<C> {
    const double* h;
    __device__ double weight(const KParams&, const typename FramedCells<C>::Cell& k) const { return __ldg(h + k.y); }
};

template <int N1, class C>
__global__ void __launch_bounds__(256) mesh_reduce_kernel(const typename C::T* __restrict__ f,
                                                          double* __restrict__ partials, const KParams p,
                                                          const double* __restrict__ h) {
    reduce_cells<N1, C>(MeshCells<C>{{f}, h}, partials, p);
}

template <int N1, class C>
cudaError_t step_as(const void* fin, void* fout, const KParams& p, const MeshDev& m, cudaStream_t s) {
    using T = typename C::T;
    if (p.walls) {
        const dim3 block(32, wall_lanes<N1>(), mesh_wall_chunks<N1>()), grid((p.nx + 2 * FILL + 31) / 32, 2);
        mesh_wall_kernel<N1, C><<<grid, block, 0, s>>>((T*)fin, p, m);
    }
    const dim3 block(32, 8), grid((p.nx + 31) / 32, (p.ny + 7) / 8);
    // the table's row length m.k is the longest list; shorter lists are padded to it
    if (m.k <= 2) mesh_sweep_kernel<N1, C, 2><<<grid, block, 0, s>>>((const T*)fin, (T*)fout, p, m);
    else if (m.k == 3) mesh_sweep_kernel<N1, C, 3><<<grid, block, 0, s>>>((const T*)fin, (T*)fout, p, m);
    else if (m.k == 4) mesh_sweep_kernel<N1, C, 4><<<grid, block, 0, s>>>((const T*)fin, (T*)fout, p, m);
    else mesh_sweep_kernel<N1, C, 0><<<grid, block, 0, s>>>((const T*)fin, (T*)fout, p, m);
    return cudaGetLastError();
}

template <int N1, class C>
cudaError_t reduce_as(const void* f, double* partials, double* out5, const KParams& p, const MeshDev& m, cudaStream_t s) {
    mesh_reduce_kernel<N1, C><<<kRedBlocks, 256, 0, s>>>((const typename C::T*)f, partials, p, m.h);
    reduce_final_kernel<<<1, 256, 0, s>>>(partials, out5);
    return cudaGetLastError();
}

template <int N1>
cudaError_t step_n1(int storage, const void* fin, void* fout, const KParams& p, const MeshDev& m, cudaStream_t s) {
    switch (storage) {
        case TVLBM_FP64: return step_as<N1, CodecF64>(fin, fout, p, m, s);
        case TVLBM_FP32: return step_as<N1, CodecF32>(fin, fout, p, m, s);
        case TVLBM_FP32_DEV: return step_as<N1, CodecF32Dev>(fin, fout, p, m, s);
        default: return cudaErrorInvalidValue;
    }
}

template <int N1>
cudaError_t reduce_n1(int storage, const void* f, double* partials, double* out5, const KParams& p, const MeshDev& m,
                      cudaStream_t s) {
    switch (storage) {
        case TVLBM_FP64: return reduce_as<N1, CodecF64>(f, partials, out5, p, m, s);
        case TVLBM_FP32: return reduce_as<N1, CodecF32>(f, partials, out5, p, m, s);
        case TVLBM_FP32_DEV: return reduce_as<N1, CodecF32Dev>(f, partials, out5, p, m, s);
        default: return cudaErrorInvalidValue;
    }
}

// ---- host tables ------------------------------------------------------------------------------

using Entries = std::vector<std::pair<int, double>>;  // (source row, length), in increasing position

void add_entry(Entries& e, int r, double len) {
    for (auto& q : e)
        if (q.first == r) {  // an interval longer than the rest of a periodic mesh meets a row twice
            q.second += len;
            return;
        }
    e.emplace_back(r, len);
}

// The pieces of [lo, hi] in the cells of F: periodic, the mesh repeated with period F_ny - F_0;
// walls, what lies below F_0 or above F_ny as rows -1 / ny.
void interval_entries(const double* F, int ny, double lo, double hi, bool periodic, Entries& e) {
    e.clear();
    if (periodic) {
        const double L = F[ny] - F[0];
        double off = floor((lo - F[0]) / L) * L;
        int r = (int)(std::upper_bound(F, F + ny + 1, lo - off) - F) - 1;
        if (r < 0) r = 0;
        if (r >= ny) {
            r = 0;
            off += L;
        }
        for (int guard = 0; guard < 4 * ny + 8; ++guard) {
            const double a = std::max(lo, F[r] + off), b = std::min(hi, F[r + 1] + off);
            if (b > a) add_entry(e, r, b - a);
            if (F[r + 1] + off >= hi) break;
            if (++r == ny) {
                r = 0;
                off += L;
            }
        }
        return;
    }
    if (lo < F[0]) add_entry(e, -1, std::min(hi, F[0]) - lo);
    int r = (int)(std::upper_bound(F, F + ny + 1, std::max(lo, F[0])) - F) - 1;
    for (r = std::max(r, 0); r < ny && F[r] < hi; ++r) {
        const double a = std::max(lo, F[r]), b = std::min(hi, F[r + 1]);
        if (b > a) add_entry(e, r, b - a);
    }
    if (hi > F[ny]) add_entry(e, ny, hi - std::max(lo, F[ny]));
}

}  // namespace

cudaError_t mesh_launch_step(tvlbm_ctx* c, const void* fin, void* fout, cudaStream_t s) {
    switch (c->n1) {
        case 3: return step_n1<3>(c->storage, fin, fout, c->kp, c->mesh, s);
        case 4: return step_n1<4>(c->storage, fin, fout, c->kp, c->mesh, s);
        default: return step_n1<6>(c->storage, fin, fout, c->kp, c->mesh, s);
    }
}

cudaError_t mesh_reduce(tvlbm_ctx* c, const void* f, double* partials, double* out5, cudaStream_t s) {
    switch (c->n1) {
        case 3: return reduce_n1<3>(c->storage, f, partials, out5, c->kp, c->mesh, s);
        case 4: return reduce_n1<4>(c->storage, f, partials, out5, c->kp, c->mesh, s);
        default: return reduce_n1<6>(c->storage, f, partials, out5, c->kp, c->mesh, s);
    }
}

extern "C" int tvlbm_set_y_faces(tvlbm_ctx* c, const double* faces) {
    if (!c) return TVLBM_EINVAL;
    cudaSetDevice(c->device);
    auto drop = [c]() {
        if (c->mesh_mem) cudaFree(c->mesh_mem);
        c->mesh_mem = nullptr;
        memset(&c->mesh, 0, sizeof(c->mesh));
    };
    if (!faces) {
        cudaStreamSynchronize(c->stream);  // no launch in flight still reads the tables
        drop();
        for (int k = 0; k < 2; ++k)
            if (c->graph[k]) {
                cudaGraphExecDestroy(c->graph[k]);
                c->graph[k] = nullptr;
            }
        return TVLBM_OK;
    }
    auto fail = [c](const char* msg) {
        snprintf(c->err, sizeof(c->err), "%s", msg);
        return TVLBM_EINVAL;
    };
    if (c->scheme != TVLBM_SCHEME_VOLUMETRIC) return fail("a non-uniform mesh applies to the volumetric scheme");
    if (c->storage != TVLBM_FP64 && c->storage != TVLBM_FP32 && c->storage != TVLBM_FP32_DEV)
        return fail("a non-uniform mesh needs FP64, FP32 or FP32-deviation storage");
    if (c->kp.rowf || c->ref_every > 0) return fail("a non-uniform mesh takes no per-row deviation reference");
    const int ny = c->ny, n1 = c->n1;
    for (int k = 0; k <= ny; ++k)
        if (!isfinite(faces[k]) || (k > 0 && !(faces[k] > faces[k - 1]))) return fail("faces must be finite and increasing");
    const bool periodic = !c->kp.walls;
    // gather tables
    std::vector<Entries> rows((size_t)n1 * ny);
    Entries e;
    int K = 2;  // rows padded to at least two entries (the unrolled gather reads two)
    for (int j = 0; j < n1; ++j) {
        const double sft = c->rule.x[j] * c->dt;
        for (int y = 0; y < ny; ++y) {
            interval_entries(faces, ny, faces[y] - sft, faces[y + 1] - sft, periodic, e);
            if (e.empty()) return fail("empty gather row (faces)");
            rows[(size_t)j * ny + y] = e;
            K = std::max(K, (int)e.size());
        }
    }
    // wall tables: rows whose image, moved by c_j dt, crosses the wall node j moves towards
    std::vector<Entries> walls(n1);
    int KB = 1;
    if (!periodic)
        for (int j = 0; j < n1; ++j) {
            const double sft = c->rule.x[j] * c->dt;
            for (int r = 0; r < ny; ++r) {
                const double lo = faces[r] + sft, hi = faces[r + 1] + sft;
                const double len = sft < 0 ? std::min(hi, faces[0]) - lo : (sft > 0 ? hi - std::max(lo, faces[ny]) : 0.0);
                if (len > 0) walls[j].emplace_back(r, len);
            }
            KB = std::max(KB, (int)walls[j].size());
        }
    if (K > kMaxMeshEntries || KB > kMaxMeshEntries)
        return fail("cells too thin for the time step: a row gathers from more than 64 cells");
    const size_t ng = (size_t)n1 * ny * K, nb = (size_t)n1 * KB;
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_src = 0, o_wd = o_src + up(ng * sizeof(int)), o_wf = o_wd + up(ng * sizeof(double));
    const size_t o_bsrc = o_wf + up(ng * sizeof(float)), o_bd = o_bsrc + up(nb * sizeof(int));
    const size_t o_bf = o_bd + up(nb * sizeof(double)), o_h = o_bf + up(nb * sizeof(float));
    const size_t total = o_h + up((size_t)ny * sizeof(double));
    std::vector<unsigned char> host(total, 0);
    int* src = (int*)(host.data() + o_src);
    double* wd = (double*)(host.data() + o_wd);
    float* wf = (float*)(host.data() + o_wf);
    int* bsrc = (int*)(host.data() + o_bsrc);
    double* bd = (double*)(host.data() + o_bd);
    float* bf = (float*)(host.data() + o_bf);
    double* h = (double*)(host.data() + o_h);
    for (int y = 0; y < ny; ++y) h[y] = faces[y + 1] - faces[y];
    for (int j = 0; j < n1; ++j)
        for (int y = 0; y < ny; ++y) {
            const Entries& r = rows[(size_t)j * ny + y];
            const size_t b = ((size_t)j * ny + y) * K;
            for (int k = 0; k < K; ++k) {
                // padding repeats the row's first source with weight 0 (adds an exact zero)
                src[b + k] = k < (int)r.size() ? r[k].first : r[0].first;
                wd[b + k] = k < (int)r.size() ? r[k].second / h[y] : 0.0;
                wf[b + k] = (float)wd[b + k];
            }
        }
    for (int j = 0; j < n1; ++j)
        for (int k = 0; k < KB; ++k) {
            const bool on = k < (int)walls[j].size();
            bsrc[(size_t)j * KB + k] = on ? walls[j][k].first : 0;  // padding: row 0, length 0
            bd[(size_t)j * KB + k] = on ? walls[j][k].second : 0.0;
            bf[(size_t)j * KB + k] = (float)bd[(size_t)j * KB + k];
        }
    unsigned char* mem = nullptr;
    if (cudaMalloc(&mem, total) != cudaSuccess) {
        snprintf(c->err, sizeof(c->err), "mesh tables: device allocation failed");
        return TVLBM_ENOMEM;
    }
    if (cudaMemcpy(mem, host.data(), total, cudaMemcpyHostToDevice) != cudaSuccess) {
        cudaFree(mem);
        snprintf(c->err, sizeof(c->err), "mesh tables: upload failed");
        return TVLBM_ECUDA;
    }
    cudaStreamSynchronize(c->stream);
    drop();
    for (int k = 0; k < 2; ++k)
        if (c->graph[k]) {
            cudaGraphExecDestroy(c->graph[k]);
            c->graph[k] = nullptr;
        }
    c->mesh_mem = mem;
    c->mesh.k = K;
    c->mesh.kb = KB;
    c->mesh.src = (const int*)(mem + o_src);
    c->mesh.wd = (const double*)(mem + o_wd);
    c->mesh.wf = (const float*)(mem + o_wf);
    c->mesh.bsrc = (const int*)(mem + o_bsrc);
    c->mesh.bd = (const double*)(mem + o_bd);
    c->mesh.bf = (const float*)(mem + o_bf);
    c->mesh.h = (const double*)(mem + o_h);
    c->form = FORM_PLAIN;
    return TVLBM_OK;
}
