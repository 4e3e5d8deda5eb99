// Device-side building blocks of the TVLBM sweep: launch parameters, storage codecs, the
// per-cell collision (moments -> Hermite equilibrium -> BGK) and the kernel table that the
// host API dispatches through.  Every kernel is a template on the 1-D node count N1
// (3, 4, 6 -> D2Q9, D2Q16, D2Q36) and on the storage codec.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <type_traits>
#include <utility>

namespace tvlbm {

constexpr int kMaxN1 = 6;
constexpr int kMaxQ = kMaxN1 * kMaxN1;
// Ghost frame around the fluid: hx columns on each side (KParams::hx = 32 bytes worth, so the
// interior starts on a 32-byte sector for every storage type), HY rows above and below; FILL
// of them are ever read (|shift| <= 4 cells).
constexpr int HY = 4;
constexpr int FILL = 4;
constexpr int kRedBlocks = 1024;  // fixed partial count of the FP64 reduction (deterministic)
constexpr int kTileConfigs = 4;  // tile shapes of the tiled form
// Strip form: its TMA box (per velocity) is strip_box_width(es) x strip_chunk_rows(n1, es)
// elements of es bytes -- the 128-column strip, the +1 source column and the 16-byte alignment
// slack, by 2 rows where two 2-row ring slots fit the shared memory a CTA may take (about 220 KB
// over the CTAs per SM that registers allow), else 1 row; the ring has three slots where they
// fit, else two.
constexpr int strip_box_width(int es) { return 128 + 16 / es; }
constexpr int strip_pop_bytes(int es, int ch) { return (ch * strip_box_width(es) * es + 127) / 128 * 128; }
constexpr int strip_smem_budget(int n1) { return (n1 >= 6 ? 220 / 3 : n1 >= 4 ? 220 / 5 : 220 / 8) * 1024; }
constexpr bool strip_fits(int n1, int es, int ch, int slots) {
    return slots * n1 * n1 * strip_pop_bytes(es, ch) + 1024 <= strip_smem_budget(n1);
}
constexpr int strip_chunk_rows(int n1, int es) { return strip_fits(n1, es, 2, 2) ? 2 : 1; }
constexpr int strip_slots(int n1, int es) { return strip_fits(n1, es, strip_chunk_rows(n1, es), 3) ? 3 : 2; }
constexpr int kFlowDone = 16;    // first per-tile counter in the dataflow scratch (64-byte aligned)
constexpr uint64_t kWaitLimitNs = 2000000000ull;  // 2 s: a TMA load never takes that long
// Per-row deviation reference tables (KParams::rowf / rowd): entries per stored row and the
// offsets of the float table's fields.
constexpr int kRowD = kMaxQ + 4;   // doubles per row: Pref_l, jref (2), eref, rref
constexpr int kRowF = kMaxQ + 12;  // floats per row: C_l, S moments (4), jref (2), eref, refD (4)
constexpr int kRowSM = kMaxQ, kRowJ = kMaxQ + 4, kRowE = kMaxQ + 6, kRowRD = kMaxQ + 7;
// Slot of C_l in a float row: for an even node count the mirror pairs (i, n1 - 1 - i) of each
// y-node j side by side, pair j (n1 / 2) + i (the order the FP32 collision relaxes them in);
// for an odd one, l itself.
__host__ __device__ constexpr int row_slot(int n1, int l) {
    return (n1 & 1) ? l
                    : 2 * ((l / n1) * (n1 / 2) + ((l % n1) < n1 / 2 ? l % n1 : n1 - 1 - l % n1)) +
                          ((l % n1) < n1 / 2 ? 0 : 1);
}
static_assert(kMaxQ % 4 == 0 && kRowF % 4 == 0, "row entries are read as float4");

enum Storage { ST_FP64 = 0, ST_FP32 = 1, ST_BF16_DEV = 2, ST_FP16_DEV = 3, ST_FP32_DEV = 4 };
enum Form { FORM_PLAIN = 0, FORM_TILED = 1, FORM_FLOW = 2, FORM_STRIP = 3 };

// Everything a kernel needs, passed by value (lands in the constant bank).
struct KParams {
    // 1-D Gauss-Hermite nodes x_i, weights w_i, overlap fractions alpha_i of the shift x_i dt,
    // integer shifts sh_i = floor(x_i dt), and He_a(x_i)/a! for a <= N.  Same table on both
    // axes (tensor-product set, dx = dy).
    float xf[kMaxN1], wf[kMaxN1], af[kMaxN1];
    double xd[kMaxN1], wd[kMaxN1], ad[kMaxN1];
    float Ef[kMaxN1][kMaxN1];
    double Ed[kMaxN1][kMaxN1];
    float x2f[kMaxN1];   // float(xf * xf)
    float wxf[kMaxN1];   // float(wf * xf): the constants of the FP32 momentum sums
    float wx2f[kMaxN1];  // float(wf * x2f): the constants of the FP32 energy sums
    // Defects of those FP32 constants against the quadrature identities they stand for,
    // evaluated exactly on the host (each ~1e-8, so a float holds it to ~1e-15):
    //   dS[a] = sum_i wf_i E_ia - [a=0],  dU[a] = sum_i wxf_i E_ia - [a=1],
    //   dV[a] = sum_i wx2f_i E_ia - [a=0] - [a=2].
    float dS[kMaxN1], dU[kMaxN1], dV[kMaxN1];
    // combinations of those defects the FP32 collision uses directly: dUS = dU[1] + dS[0],
    // dVS[a] = dV[a] + dS[a] (+ dS[0] for a = 2, the h_2 term of the energy defect)
    float dUS, dVS[kMaxN1];
    // Full-f FP32 codec (cell_collide_split): the FP64 weight w_l = w_i w_j of velocity
    // l = i + n j as a float pair Whi_l + Wlo_l (Whi = float(w_l), Wlo = float(w_l - Whi)), and
    // the defects of the FP32 node tables under the exact weights, whose moment sums are
    // unweighted (constants xf, x2f): dSx[a] = sum_i w_i E_ia - [a=0], dUx[a] = sum_i w_i xf_i E_ia
    // - [a=1], dVSx[a] = sum_i w_i x2f_i E_ia - [a=0] - [a=2] + dSx[a] (+ dSx[0] for a = 2),
    // dUSx = dUx[1] + dSx[0].
    float Whi[kMaxQ], Wlo[kMaxQ];
    float dSx[kMaxN1], dUx[kMaxN1], dUSx, dVSx[kMaxN1];
    int sh[kMaxN1];
    float omegaf, rho0f;
    double omegad, rho0d;
    int nx, ny;      // fluid cells
    int hx;          // frame columns left of the fluid (32 bytes of elements, >= FILL)
    int pitch;       // elements per stored row (>= nx + 2 HX)
    int rows;        // stored rows (ny + 2 HY)
    long long plane; // elements per velocity plane (rows * pitch)
    int walls;       // 0 periodic, 1 diffuse walls at y = -1/2 and y = ny - 1/2
    // Walls: equilibrium f_eq_l(rho=1, u_w, T_w) of each wall (f-space) and the inverse of
    // sum_{incoming} |c_y dt| f_eq_l.
    float feqwf[2][kMaxQ];
    double feqwd[2][kMaxQ];
    float inv_denf[2];
    double inv_dend[2];
    // Deviation storage reference: d_l = f_l / w_l - R_l, R_l = f_eq_l(rho0, u_ref, T_ref) / w_l.
    // Pref_l = R_l - rho0 (zero for the default reference: at rest, T_ref = 1), jref = rho0 u_ref,
    // eref = rho0 (2 (T_ref - 1) + |u_ref|^2), refD = -(moments of the float Pref table under the
    // FP32 moment constants - (0, jref, eref)), the reference's share of the table defects.
    int has_ref;
    float Preff[kMaxQ];
    double Prefd[kMaxQ];
    float jreff[2], ereff, refD[4];
    double jrefd[2], erefd;
    // Per-row reference of a domain with walls (null: the single reference above).  Stored row
    // r = y + HY (ghost rows included) has its own reference R_l(y) = f_eq_l(rho0, u_ref(y),
    // T_ref(y)) / w_l.  Streaming moves d_l + R_l(y_source), so the gathered deviation against
    // R_l(y) is the gather of d plus the shift S_l(y) = (1 - a_j) R_l(y - sh_j) + a_j R_l(y - sh_j - 1)
    // - R_l(y) (exact: R is constant in x).  The FP32 collision takes the moments of S and, after
    // relaxing, adds C_l(y) = (1 - omega) S_l(y) - omega Pref_l(y) (the shift kept by the BGK
    // update and the row reference's own equilibrium deviation).
    //   rowd[r * kRowD + l]: Pref_l; [kMaxQ + 0..1]: jref; [kMaxQ + 2]: eref; [kMaxQ + 3]: rref, the
    //   reference's mass beyond rho0 (0 for an equilibrium of density rho0; a reference taken from
    //   the rows' mean populations has the rows' own density)
    //   rowf[r * kRowF + row_slot(n1, l)]: C_l; [kRowSM + 0..3]: FP32-constant moments (m0, mx,
    //   my, me) of S;
    //   [kRowJ + 0..1]: jref; [kRowE]: eref; [kRowRD + 0..3]: refD of the row's float Pref
    //   (the S mass entry includes rref)
    const float* rowf;
    const double* rowd;
    // Device status word: bit 0 is set by a kernel whose bounded wait gave up.
    int* status;
};

template <class R> __device__ __forceinline__ R kx(const KParams& p, int i) {
    if constexpr (std::is_same<R, double>::value) return p.xd[i]; else return p.xf[i];
}
// Geometry and relaxation of one domain.  A single-domain launch takes it from KParams; the
// batched launch reads it from a per-domain table.
struct Geom {
    int nx, ny, pitch, hx, walls;
    long long plane;
    float omegaf;
    double omegad;
};
__host__ __device__ __forceinline__ Geom geom_of(const KParams& p) {
    Geom g;
    g.nx = p.nx;
    g.ny = p.ny;
    g.pitch = p.pitch;
    g.hx = p.hx;
    g.walls = p.walls;
    g.plane = p.plane;
    g.omegaf = p.omegaf;
    g.omegad = p.omegad;
    return g;
}

template <class R> __device__ __forceinline__ R kx2(const KParams& p, int i) {
    if constexpr (std::is_same<R, double>::value) return p.xd[i] * p.xd[i]; else return p.x2f[i];
}
template <class R> __device__ __forceinline__ R kw(const KParams& p, int i) {
    if constexpr (std::is_same<R, double>::value) return p.wd[i]; else return p.wf[i];
}
template <class R> __device__ __forceinline__ R ka(const KParams& p, int i) {
    if constexpr (std::is_same<R, double>::value) return p.ad[i]; else return p.af[i];
}
template <class R> __device__ __forceinline__ R kE(const KParams& p, int i, int a) {
    if constexpr (std::is_same<R, double>::value) return p.Ed[i][a]; else return p.Ef[i][a];
}
template <class R> __device__ __forceinline__ R komega(const KParams& p) {
    if constexpr (std::is_same<R, double>::value) return p.omegad; else return p.omegaf;
}
template <class R> __device__ __forceinline__ R krho0(const KParams& p) {
    if constexpr (std::is_same<R, double>::value) return p.rho0d; else return p.rho0f;
}
template <class R> __device__ __forceinline__ R kPref(const KParams& p, int l) {
    if constexpr (std::is_same<R, double>::value) return p.Prefd[l]; else return p.Preff[l];
}
// Loads from a per-row reference table that is only read when it exists: the load sits in its
// branch as volatile inline PTX, so it is never issued ahead of the test (a table pointer may be
// null on the same code path).
__device__ __forceinline__ double ld_row(const double* q) {
    double v;
    asm volatile("ld.global.nc.f64 %0, [%1];" : "=d"(v) : "l"(q));
    return v;
}
__device__ __forceinline__ float ld_row(const float* q) {
    float v;
    asm volatile("ld.global.nc.f32 %0, [%1];" : "=f"(v) : "l"(q));
    return v;
}
__device__ __forceinline__ float4 ld_row4(const float* q) {  // q 16-byte aligned
    float4 v;
    asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(q));
    return v;
}

// Pref_l of fluid row y (y may be a ghost row), per-row table or the single reference.
template <class R> __device__ __forceinline__ R kPrefRow(const KParams& p, int l, int y) {
    if (p.rowd) return (R)ld_row(p.rowd + (long long)(y + HY) * kRowD + l);
    if constexpr (std::is_same<R, double>::value) return p.Prefd[l]; else return p.Preff[l];
}
template <class R> __device__ __forceinline__ R kjref(const KParams& p, int k) {
    if constexpr (std::is_same<R, double>::value) return p.jrefd[k]; else return p.jreff[k];
}
template <class R> __device__ __forceinline__ R keref(const KParams& p) {
    if constexpr (std::is_same<R, double>::value) return p.erefd; else return p.ereff;
}
template <class R> __device__ __forceinline__ R kfeqw(const KParams& p, int side, int l) {
    if constexpr (std::is_same<R, double>::value) return p.feqwd[side][l]; else return p.feqwf[side][l];
}
template <class R> __device__ __forceinline__ R kinvden(const KParams& p, int side) {
    if constexpr (std::is_same<R, double>::value) return p.inv_dend[side]; else return p.inv_denf[side];
}

// ---- storage codecs ----------------------------------------------------------------------
// Full codecs store f_l; deviation codecs store d_l = f_l / w_l - R_l (R_l = rho0 for the default
// reference, see KParams).  Sweep arithmetic runs
// in "storage space" (the stored quantity), so the gather and the BGK update are linear in
// what is loaded and stored; moments and equilibrium know which space they are in.
// split: a full FP32 codec whose sweep gathers and collides f_l - Whi_l (exact for a population
// within a factor 2 of its rest value), so that no rounding but the store's is relative to f
// itself (cell_collide_split).
struct CodecF64 {
    using T = double; using R = double; static constexpr bool dev = false, split = false;
    __device__ static R ld(const T* p) { return __ldg(p); }
    __device__ static T enc(R v) { return v; }
};
struct CodecF32 {
    using T = float; using R = float; static constexpr bool dev = false, split = true;
    __device__ static R ld(const T* p) { return __ldg(p); }
    __device__ static T enc(R v) { return v; }
};
struct CodecF32Dev {
    using T = float; using R = float; static constexpr bool dev = true, split = false;
    __device__ static R ld(const T* p) { return __ldg(p); }
    __device__ static T enc(R v) { return v; }
};
struct CodecBF16Dev {
    using T = __nv_bfloat16; using R = float; static constexpr bool dev = true, split = false;
    __device__ static R ld(const T* p) { return __bfloat162float(__ldg(p)); }
    __device__ static T enc(R v) { return __float2bfloat16_rn(v); }
};
struct CodecF16Dev {
    using T = __half; using R = float; static constexpr bool dev = true, split = false;
    __device__ static R ld(const T* p) { return __half2float(__ldg(p)); }
    __device__ static T enc(R v) { return __float2half_rn(v); }
};

// f_l - Whi_l, the population less the float of its rest value (split codecs; exact by
// Sterbenz's lemma for v within a factor 2 of Whi_l).
template <class C>
__device__ __forceinline__ typename C::R split_rest(const KParams& p, int l, typename C::R v) {
    if constexpr (C::split) return v - p.Whi[l]; else return v;
}

// Storage value -> f_l and back, in precision R (used off the hot path: init, moments,
// reductions, walls); ref = R_l, the deviation reference of velocity l.
template <class C, class R>
__device__ __forceinline__ R to_f(R v, R w, R ref) { if constexpr (C::dev) return w * (ref + v); else return v; }
template <class C, class R>
__device__ __forceinline__ R from_f(R f, R w, R ref) { if constexpr (C::dev) return f / w - ref; else return f; }

// ---- moments, equilibrium, BGK on one cell -----------------------------------------------
// s[l], l = i + N1 j, holds the cell's (gathered) populations in storage space.
// Moments (Sec. "The TVLBM model"): rho = sum f, rho u = sum c f, D rho T + rho u^2 = sum |c|^2 f
// with D = 2.  In deviation space f = w (R + d) with R the reference's f_eq / w, whose moments
// are (rho0, rho0 u_ref, rho0 (D T_ref + u_ref^2)) by exact quadrature, so rho = rho0 + sum w d,
// rho u = jref + sum w c d, and T - 1 = ((eref + sum w |c|^2 d - D sum w d)/rho - u^2)/D.
// ref4: the cell row's reference moments (jref_x, jref_y, eref, rref) of a per-row reference, or
// null; rref is the reference's mass beyond rho0 (rho = rho0 + rref + sum w d).
template <int N1, bool DEV, class R>
__device__ __forceinline__ void cell_moments(const R (&s)[N1 * N1], const KParams& p, R& rho, R& ux, R& uy, R& th,
                                             const R* ref4 = nullptr) {
    R m0 = 0, mx = 0, my = 0, me = 0;
#pragma unroll
    for (int j = 0; j < N1; ++j) {
        R r = 0, rx = 0, rxx = 0;
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const R v = DEV ? kw<R>(p, i) * s[i + N1 * j] : s[i + N1 * j];
            const R xi = kx<R>(p, i);
            r += v;
            rx = fma(xi, v, rx);
            rxx = fma(kx2<R>(p, i), v, rxx);
        }
        const R yj = kx<R>(p, j);
        const R wj = DEV ? kw<R>(p, j) : R(1);
        m0 = fma(wj, r, m0);
        mx = fma(wj, rx, mx);
        my = fma(wj * yj, r, my);
        me = fma(wj, fma(kx2<R>(p, j), r, rxx), me);
    }
    if constexpr (DEV) {
        if (ref4) m0 += ref4[3];
        rho = krho0<R>(p) + m0;
        const R inv = R(1) / rho;
        ux = ((ref4 ? ref4[0] : kjref<R>(p, 0)) + mx) * inv;
        uy = ((ref4 ? ref4[1] : kjref<R>(p, 1)) + my) * inv;
        th = R(0.5) * (((ref4 ? ref4[2] : keref<R>(p)) + me - R(2) * m0) * inv - (ux * ux + uy * uy));
    } else {
        rho = m0;
        const R inv = R(1) / rho;
        ux = mx * inv;
        uy = my * inv;
        th = R(0.5) * (me * inv - (ux * ux + uy * uy)) - R(1);
    }
}

// Hermite equilibrium (Sec. "The TVLBM model"; Appendix A) for a tensor-product set, in
// separable form.  The Hermite coefficients of a Maxwellian factorise per axis:
//   f_eq_l = rho w_i w_j sum_{a+b<=N} h_a(u_x) He_a(x_i)/a! * h_b(u_y) He_b(x_j)/b!,
// h_0 = 1, h_1 = u, h_{n+1} = u h_n + n (T-1) h_{n-1}  (the Gaussian moments E[He_n(u+sqrt(T) Z)]).
// With X_ia = h_a(u_x) E_ia (X_i0 = 1), P_jk = sum_{1<=b<=k} h_b(u_y) E_jb:
//   sum_{a+b<=N} X_ia Y_jb = 1 + phi_ij,  phi_ij = sum_{a>=1} X_ia + sum_{a<N} X_ia P_j,N-a.
// Storage-space equilibrium: full f_eq = w rho (1 + phi); deviation d_eq = (rho - rho0) + rho phi - Pref.
// pref: the cell row's Pref table of a per-row reference, or null.
template <int N1, bool DEV, class R>
__device__ __forceinline__ void cell_equilibrium(const KParams& p, R rho, R ux, R uy, R th, R (&eq)[N1 * N1],
                                                 const R* pref = nullptr) {
    constexpr int N = N1 - 1;
    R hx[N + 1], hy[N + 1];
    hx[0] = R(1); hy[0] = R(1);
    hx[1] = ux;   hy[1] = uy;
#pragma unroll
    for (int n = 1; n < N; ++n) {
        hx[n + 1] = fma(ux, hx[n], R(n) * th * hx[n - 1]);
        hy[n + 1] = fma(uy, hy[n], R(n) * th * hy[n - 1]);
    }
    R X[N1][N], SX[N1], P[N1][N + 1];
#pragma unroll
    for (int i = 0; i < N1; ++i) {
        R sx = 0, acc = 0;
#pragma unroll
        for (int a = 1; a <= N; ++a) {
            const R v = hx[a] * kE<R>(p, i, a);
            if (a < N) X[i][a] = v;
            sx += v;
            acc = fma(hy[a], kE<R>(p, i, a), acc);
            P[i][a] = acc;
        }
        SX[i] = sx;
    }
    const R drho = DEV ? rho - krho0<R>(p) : R(0);
#pragma unroll
    for (int j = 0; j < N1; ++j) {
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            R phi = SX[i] + P[j][N];  // a = 0 term: X_i0 = 1
#pragma unroll
            for (int a = 1; a < N; ++a) phi = fma(X[i][a], P[j][N - a], phi);
            if constexpr (DEV) eq[i + N1 * j] = fma(rho, phi, drho) - (pref ? pref[i + N1 * j] : kPref<R>(p, i + N1 * j));
            else eq[i + N1 * j] = (kw<R>(p, i) * kw<R>(p, j) * rho) * (R(1) + phi);
        }
    }
}

// Moments -> equilibrium -> BGK relaxation s* = s + (dt/tau)(s_eq - s), in place.
template <int N1, bool DEV, class R>
__device__ __forceinline__ void cell_collide(R (&s)[N1 * N1], const KParams& p, R om) {
    R rho, ux, uy, th;
    cell_moments<N1, DEV, R>(s, p, rho, ux, uy, th);
    R eq[N1 * N1];
    cell_equilibrium<N1, DEV, R>(p, rho, ux, uy, th, eq);
#pragma unroll
    for (int l = 0; l < N1 * N1; ++l) s[l] = fma(om, eq[l] - s[l], s[l]);
}

// Programmatic dependent launch: a sweep lets the next launch on its stream be scheduled while
// its own tail runs (launch_dependents), and reads its input only after the previous grid's
// writes are complete and visible (wait).  Both are no-ops when launched without the attribute.
__device__ __forceinline__ void pdl_launch_dependents() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch a kernel with programmatic stream serialization (see pdl_wait).
template <class... KArgs, class... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Explicit global-space stores and loads: the population buffers are always global memory, and
// saying so keeps generic accesses (which could alias shared memory) out of the sweeps.
__device__ __forceinline__ void stg(float* p, float v) { asm volatile("st.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory"); }
__device__ __forceinline__ void stg(double* p, double v) { asm volatile("st.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory"); }
__device__ __forceinline__ void stg(__half* p, __half v) {
    asm volatile("st.global.b16 [%0], %1;" ::"l"(p), "h"(__half_as_ushort(v)) : "memory");
}
__device__ __forceinline__ void stg(__nv_bfloat16* p, __nv_bfloat16 v) {
    asm volatile("st.global.b16 [%0], %1;" ::"l"(p), "h"(__bfloat16_as_ushort(v)) : "memory");
}

// Padded storage index of fluid cell (x, y) in velocity plane l (x, y may lie in the frame).
__device__ __forceinline__ long long sidx(const KParams& p, int l, int x, int y) {
    return (long long)l * p.plane + (long long)(y + HY) * p.pitch + (x + p.hx);
}

// Store v at fluid cell (x, y) and at every periodic image of it inside the read frame
// (x in [-FILL, nx+FILL); y likewise when periodic in y).
template <class T>
__device__ __forceinline__ void store_with_images(T* f, const Geom& g, long long lbase, int x, int y, T v) {
    const int x0 = x - g.nx * ((x + FILL) / g.nx);
    if (g.walls) {
        for (int xx = x0; xx < g.nx + FILL; xx += g.nx) stg(f + lbase + (long long)(y + HY) * g.pitch + (xx + g.hx), v);
    } else {
        const int y0 = y - g.ny * ((y + FILL) / g.ny);
        for (int yy = y0; yy < g.ny + FILL; yy += g.ny)
            for (int xx = x0; xx < g.nx + FILL; xx += g.nx) stg(f + lbase + (long long)(yy + HY) * g.pitch + (xx + g.hx), v);
    }
}

// TMA descriptors (CUtensorMap) of a tiled sweep: input windows (out: reserved, may be null).
struct SweepMaps {
    const void* in;
    const void* out;
};

// Work of one multi-step dataflow launch (sweep_flow_kernel): tiles_x x tiles_y tiles, nsteps
// time steps, tasks (step, tile) handed out in step-major order.
struct FlowSrc {
    CUtensorMap map[2];  // input descriptors: [0] the buffer holding the state at launch, [1] the other
    CUtensorMap smap[2]; // output descriptors of the same buffers (box: one tile), for TMA stores
    void* buf[2];        // the same two buffers
    int tiles_x, tiles_y, ntiles, nsteps;
    int* done;       // [ntiles] compute-warp completions in this launch (zeroed before it)
    int* next_task;  // task counter (zeroed before the launch)
    int* abort;      // raised by a CTA whose bounded wait gave up (zeroed before the launch)
    long long wait_ns;  // limit of the producer's wait for a task's neighbourhood (default 2 s)
    int wait_extra;     // added to the completion count that wait needs (0; > 0 only to test the
                        // timeout path: no neighbour reaches it, so the wait gives up)
};

struct BatchSrc;      // tile source of the batched sweep (tvlbm_tiled.cuh)
struct BatchFlowSrc;  // task source of the batched multi-step dataflow launch (tvlbm_tiled.cuh)


// ---- kernel table (one per N1, defined in tvlbm_kernels_q*.cu) ----------------------------
struct KernelTable {
    // maps: TMA descriptors of the tiled form; cfg: its tile configuration (0 .. kTileConfigs-1)
    cudaError_t (*sweep)(int storage, int form, int cfg, const void* fin, void* fout, const SweepMaps* maps,
                         const KParams& p, cudaStream_t s);
    cudaError_t (*init)(int storage, const double* fields, void* f, const KParams& p, cudaStream_t s);
    cudaError_t (*moments)(int storage, const void* f, double* out4, const KParams& p, cudaStream_t s);
    cudaError_t (*reduce)(int storage, const void* f, double* partials, double* out5, const KParams& p, cudaStream_t s);
    cudaError_t (*wall)(int storage, void* f, const KParams& p, cudaStream_t s);
    cudaError_t (*halo)(int storage, void* f, const KParams& p, cudaStream_t s);
    cudaError_t (*decode_plane)(int storage, const void* f, int l, double* out, const KParams& p, cudaStream_t s);
    cudaError_t (*encode_plane)(int storage, void* f, int l, const double* in, const KParams& p, cudaStream_t s);
    int (*tiled_available)(int storage);
    void (*tiled_box)(int storage, int cfg, int* bx, int* by);  // TMA box (elements) of a tile config
    void (*tile_shape)(int storage, int cfg, int* tx, int* ty, int* rows_per_thread);
    // re-express every stored element of buffer f against a new deviation reference:
    // d_l += delta[r * kMaxQ + l] on stored row r (delta: device, [rows][kMaxQ])
    cudaError_t (*reencode)(int storage, void* f, const float* delta, const KParams& p, cudaStream_t s);
    // n time steps of one periodic domain in a single dataflow launch
    cudaError_t (*flow_sweep)(int storage, int cfg, const FlowSrc& src, const KParams& p, cudaStream_t s);
    // one time step of every domain of a batch (one launch over all tiles)
    cudaError_t (*batch_sweep)(int storage, int cfg, const BatchSrc& src, const KParams& p, cudaStream_t s);
    // n time steps of every domain of a batch in one persistent dataflow launch
    cudaError_t (*batch_flow)(int storage, int cfg, const BatchFlowSrc& src, const KParams& p, cudaStream_t s);
    // row averages of (ux, uy, T) of buffer f into prof [3][ny] (device)
    cudaError_t (*row_means)(int storage, const void* f, double* prof, const KParams& p, cudaStream_t s);
    // per-row reference tables (KParams::rowd / rowf layout, p.rows rows) of the profile prof [3][ny]
    cudaError_t (*ref_tables)(const double* prof, double* rowd, float* rowf, const KParams& p, cudaStream_t s);
    // row averages of Pref_l + d_l per velocity of buffer f into prof [Q][ny] (deviation storage)
    cudaError_t (*row_pop_means)(int storage, const void* f, double* prof, const KParams& p, cudaStream_t s);
    // per-row reference tables whose Pref is the profile prof [Q][ny] itself
    cudaError_t (*ref_tables_mean)(const double* prof, double* rowd, float* rowf, const KParams& p, cudaStream_t s);
};

const KernelTable* kernel_table_q3();
const KernelTable* kernel_table_q4();
const KernelTable* kernel_table_q6();

}  // namespace tvlbm
