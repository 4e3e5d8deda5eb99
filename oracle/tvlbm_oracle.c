/*
 * FP64 CPU oracle of the thermal volumetric lattice Boltzmann (TVLBM) time step.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the library path may link, load or call
 * this file; only the tests, the smoke check and the benchmark's CPU-baseline leg
 * use it.  It shares no code, header, table or constant with the CUDA path.
 *
 * It follows the method in the paper's order and notation, written plainly:
 *   - macroscopic moments rho, rho u, rho T            (Sec. "The TVLBM model", moment definitions)
 *   - Hermite equilibrium f_eq = w sum_n a^(n):H^(n)/n! (Sec. "The TVLBM model", Hermite expansion
 *     with the a^(n)_0 and H^(n) tensors in Grad notation), evaluated as full tensor contractions
 *   - BGK relaxation towards f_eq with time tau         (Eq. "eq:lb"), one explicit step of length dt
 *   - volumetric streaming: every population moves by c*dt and is shared among the cells its
 *     shifted cell volume overlaps, with area-overlap weights (the volumetric formulation the
 *     Introduction motivates: conservative, off-lattice velocities)
 *   - diffuse-reflection walls whose re-emitted flux equals the flux hitting the wall
 *     (Eq. "IMPOSITION"), applied through ghost rows.
 *
 * All arithmetic is double precision.  Fields are stored [Q][ny][nx], x fastest.
 * Velocity set and streaming table are passed in by the caller (the oracle's Python side
 * builds them from Gauss-Hermite quadrature).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXQ 64
#define OR_MAXN 6
#define OR_MAXT 64 /* 2^OR_MAXN multi-indices per order */

/* One term of a Grad-notation symmetric tensor component: (T-1)^k (or (-1)^k) times the
 * product of the vector components named in `sing`.  Only pairings whose index pairs are
 * equal survive (each pair contributes a Kronecker delta). */
typedef struct {
    int k;
    int nsing;
    int sing[OR_MAXN];
} or_term;

typedef struct {
    int count;
    int cap;
    or_term *t;
} or_terms;

typedef struct {
    int nx, ny, Q, N, D;
    double tau, dt, omega;
    double cx[OR_MAXQ], cy[OR_MAXQ], w[OR_MAXQ];
    int sx[OR_MAXQ], sy[OR_MAXQ];
    double axw[OR_MAXQ], ayw[OR_MAXQ];
    int walls;
    double u_lo, T_lo, u_hi, T_hi;
    /* Grad expansions of every tensor component (order n, multi-index m in [0, 2^n)). */
    or_terms terms[OR_MAXN + 1][OR_MAXT];
    /* H^(n)_l components for every velocity l */
    double H[OR_MAXQ][OR_MAXN + 1][OR_MAXT];
    double fact[OR_MAXN + 1];
    double *ftilde; /* gathered populations, [Q][ny][nx] */
    double *ghost;  /* wall ghost values, [2][Q][nx] (bottom, top) */
    int nthreads;
} or_ctx;

static void terms_push(or_terms *L, int k, const int *sing, int nsing) {
    if (L->count == L->cap) {
        L->cap = L->cap ? 2 * L->cap : 8;
        L->t = (or_term *)realloc(L->t, (size_t)L->cap * sizeof(or_term));
    }
    or_term *t = &L->t[L->count++];
    t->k = k;
    t->nsing = nsing;
    for (int i = 0; i < nsing; ++i) t->sing[i] = sing[i];
}

/* Enumerate every way of splitting the positions 0..n-1 of the multi-index `idx` into
 * unordered pairs and single positions (Grad's fully symmetric notation, e.g. delta u
 * stands for the 3 distinct placements delta_ij u_k + delta_ik u_j + delta_jk u_i).
 * A pair contributes delta(idx_p, idx_q); pairings containing a vanishing delta are dropped. */
static void enum_pairings(const int *idx, int n, int pos, unsigned used, int k, int *sing, int nsing,
                          or_terms *out) {
    while (pos < n && (used >> pos) & 1u) ++pos;
    if (pos == n) {
        terms_push(out, k, sing, nsing);
        return;
    }
    /* position `pos` stays single */
    sing[nsing] = idx[pos];
    enum_pairings(idx, n, pos + 1, used | (1u << pos), k, sing, nsing + 1, out);
    /* or `pos` is paired with a later free position q carrying the same index */
    for (int q = pos + 1; q < n; ++q) {
        if ((used >> q) & 1u) continue;
        if (idx[q] != idx[pos]) continue; /* delta vanishes */
        enum_pairings(idx, n, pos + 1, used | (1u << pos) | (1u << q), k + 1, sing, nsing, out);
    }
}

/* Symmetric tensor component: sum over terms of coef^k * prod v[sing]. */
static double grad_component(const or_terms *L, double coef, const double v[2]) {
    double s = 0.0;
    for (int i = 0; i < L->count; ++i) {
        const or_term *t = &L->t[i];
        double p = 1.0;
        for (int j = 0; j < t->k; ++j) p *= coef;
        for (int j = 0; j < t->nsing; ++j) p *= v[t->sing[j]];
        s += p;
    }
    return s;
}

/* Hermite tensors H^(n)(c) (Sec. "The TVLBM model"): H^(0)=1, H^(1)=c, H^(2)=c^2-delta,
 * H^(3)=c^3-c delta, H^(4)=c^4-c^2 delta+delta delta, H^(5)=c^5-c^3 delta+delta delta c:
 * the term with k deltas carries the sign (-1)^k. */
static double hermite_component(const or_ctx *C, int n, int m, const double c[2]) {
    return grad_component(&C->terms[n][m], -1.0, c);
}

/* Equilibrium coefficients a^(n)_0 (Sec. "The TVLBM model"): a^(0)=rho, a^(1)=rho u,
 * a^(2)=rho(u^2+(T-1)delta), a^(3)=rho(u^3+(T-1)delta u),
 * a^(4)=rho(u^4+(T-1)delta u^2+(T-1)^2 delta^2), a^(5)=rho(u^5+(T-1)delta u^3+(T-1)^2 delta delta u):
 * the term with k deltas carries (T-1)^k. */
static double a_component(const or_ctx *C, int n, int m, double rho, const double u[2], double T) {
    return rho * grad_component(&C->terms[n][m], T - 1.0, u);
}

static void multi_index(int n, int m, int *idx) {
    for (int p = 0; p < n; ++p) idx[p] = (m >> p) & 1;
}

/* f_eq_l = w_l sum_{n=0}^{N} (1/n!) a^(n)_0 : H^(n)_l, full contraction over all 2^n index tuples. */
static void equilibrium(const or_ctx *C, double rho, double ux, double uy, double T, double *feq) {
    const double u[2] = {ux, uy};
    double a[OR_MAXN + 1][OR_MAXT];
    for (int n = 0; n <= C->N; ++n)
        for (int m = 0; m < (1 << n); ++m) a[n][m] = a_component(C, n, m, rho, u, T);
    for (int l = 0; l < C->Q; ++l) {
        double s = 0.0;
        for (int n = 0; n <= C->N; ++n) {
            double sn = 0.0;
            for (int m = 0; m < (1 << n); ++m) sn += a[n][m] * C->H[l][n][m];
            s += sn / C->fact[n];
        }
        feq[l] = C->w[l] * s;
    }
}

/* Moments (Sec. "The TVLBM model"): rho = sum f, rho u = sum c f, rho T = (1/D) sum |c-u|^2 f. */
static void moments_of(const or_ctx *C, const double *f, size_t stride, double *rho, double *ux, double *uy,
                       double *T) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int l = 0; l < C->Q; ++l) {
        double v = f[(size_t)l * stride];
        r += v;
        jx += C->cx[l] * v;
        jy += C->cy[l] * v;
    }
    double vx = jx / r, vy = jy / r;
    double e = 0.0;
    for (int l = 0; l < C->Q; ++l) {
        double v = f[(size_t)l * stride];
        double dx = C->cx[l] - vx, dy = C->cy[l] - vy;
        e += (dx * dx + dy * dy) * v;
    }
    *rho = r;
    *ux = vx;
    *uy = vy;
    *T = e / (C->D * r);
}

void *oracle_create(int nx, int ny, int Q, int N, const double *cx, const double *cy, const double *w,
                    const int *sx, const int *sy, const double *ax, const double *ay, double tau, double dt,
                    int walls, double u_lo, double T_lo, double u_hi, double T_hi) {
    if (Q > OR_MAXQ || N > OR_MAXN - 1 || nx < 1 || ny < 1) return NULL;
    or_ctx *C = (or_ctx *)calloc(1, sizeof(or_ctx));
    C->nx = nx;
    C->ny = ny;
    C->Q = Q;
    C->N = N;
    C->D = 2;
    C->tau = tau;
    C->dt = dt;
    C->omega = dt / tau;
    C->walls = walls;
    C->u_lo = u_lo;
    C->T_lo = T_lo;
    C->u_hi = u_hi;
    C->T_hi = T_hi;
    C->nthreads = 0;
    for (int l = 0; l < Q; ++l) {
        C->cx[l] = cx[l];
        C->cy[l] = cy[l];
        C->w[l] = w[l];
        C->sx[l] = sx[l];
        C->sy[l] = sy[l];
        C->axw[l] = ax[l];
        C->ayw[l] = ay[l];
    }
    C->fact[0] = 1.0;
    for (int n = 1; n <= OR_MAXN; ++n) C->fact[n] = C->fact[n - 1] * n;
    for (int n = 0; n <= N; ++n) {
        for (int m = 0; m < (1 << n); ++m) {
            int idx[OR_MAXN], sing[OR_MAXN];
            multi_index(n, m, idx);
            enum_pairings(idx, n, 0, 0u, 0, sing, 0, &C->terms[n][m]);
        }
    }
    for (int l = 0; l < Q; ++l) {
        const double c[2] = {cx[l], cy[l]};
        for (int n = 0; n <= N; ++n)
            for (int m = 0; m < (1 << n); ++m) C->H[l][n][m] = hermite_component(C, n, m, c);
    }
    C->ftilde = (double *)malloc(sizeof(double) * (size_t)Q * nx * ny);
    C->ghost = (double *)calloc((size_t)2 * Q * nx, sizeof(double));
    return C;
}

void oracle_destroy(void *p) {
    or_ctx *C = (or_ctx *)p;
    if (!C) return;
    for (int n = 0; n <= OR_MAXN; ++n)
        for (int m = 0; m < OR_MAXT; ++m) free(C->terms[n][m].t);
    free(C->ftilde);
    free(C->ghost);
    free(C);
}

void oracle_set_threads(void *p, int nthreads) { ((or_ctx *)p)->nthreads = nthreads; }

/* Single-cell equilibrium, exported for the tests. */
void oracle_equilibrium(void *p, double rho, double ux, double uy, double T, double *feq) {
    equilibrium((or_ctx *)p, rho, ux, uy, T, feq);
}

/* Equilibrium through the explicit scalar forms of Appendix A (orders 2..5, with u_l = u.c_l,
 * u^2, c_l^2, D), orders 0 and 1 being rho and rho u_l.  Every order is multiplied by rho. */
void oracle_equilibrium_appendix_a(void *p, double rho, double ux, double uy, double T, double *feq) {
    const or_ctx *C = (const or_ctx *)p;
    const double D = C->D, t = T - 1.0, u2 = ux * ux + uy * uy;
    for (int l = 0; l < C->Q; ++l) {
        const double ul = ux * C->cx[l] + uy * C->cy[l];
        const double c2 = C->cx[l] * C->cx[l] + C->cy[l] * C->cy[l];
        double o[6];
        o[0] = 1.0;
        o[1] = ul;
        o[2] = 0.5 * (ul * ul - u2 + t * (c2 - D));
        o[3] = ul / 6.0 * (ul * ul - 3.0 * u2 + 3.0 * t * (c2 - D - 2.0));
        o[4] = (ul * ul * ul * ul - 6.0 * ul * ul * u2 + 3.0 * u2 * u2) / 24.0 +
               t / 4.0 * ((c2 - D - 2.0) * (ul * ul - u2) - 2.0 * ul * ul) +
               t * t / 8.0 * (c2 * c2 - 2.0 * (D + 2.0) * c2 + D * (D + 2.0));
        o[5] = (ul * ul * ul * ul * ul - 10.0 * u2 * ul * ul * ul + 15.0 * u2 * u2 * ul) / 120.0 +
               t / 12.0 * (c2 * ul * ul * ul - (D + 6.0) * ul * ul * ul - 3.0 * c2 * ul * u2 + (3.0 * D + 12.0) * u2 * ul) +
               t * t / 8.0 * (ul * c2 * c2 - (2.0 * D + 8.0) * c2 * ul + (D * D + 6.0 * D + 8.0) * ul);
        double s = 0.0;
        for (int n = 0; n <= C->N && n <= 5; ++n) s += o[n];
        feq[l] = rho * C->w[l] * s;
    }
}

/* f = f_eq(rho, u, T) on every cell. */
void oracle_init(void *p, const double *rho, const double *ux, const double *uy, const double *T, double *f) {
    or_ctx *C = (or_ctx *)p;
    const size_t plane = (size_t)C->nx * C->ny;
#pragma omp parallel for schedule(static) num_threads(C->nthreads > 0 ? C->nthreads : omp_get_max_threads())
    for (long long c = 0; c < (long long)plane; ++c) {
        double feq[OR_MAXQ];
        equilibrium(C, rho[c], ux[c], uy[c], T[c], feq);
        for (int l = 0; l < C->Q; ++l) f[(size_t)l * plane + c] = feq[l];
    }
}

static int wrap(int i, int n) { return ((i % n) + n) % n; }

/* Source value of population l at (x, y) for the gather: periodic in x; periodic in y, or,
 * with walls, the ghost value beyond a wall for populations that enter through it and zero
 * for populations that leave through it (they carry no mass back). */
static double source_value(const or_ctx *C, const double *f, int l, int x, int y) {
    const int nx = C->nx, ny = C->ny;
    x = wrap(x, nx);
    if (!C->walls) return f[((size_t)l * ny + wrap(y, ny)) * nx + x];
    if (y >= 0 && y < ny) return f[((size_t)l * ny + y) * nx + x];
    if (y < 0) return C->cy[l] > 0.0 ? C->ghost[(size_t)l * nx + x] : 0.0;
    return C->cy[l] < 0.0 ? C->ghost[((size_t)C->Q + l) * nx + x] : 0.0;
}

/* Volumetric pull-gather: destination cell (x, y) receives from the source cell whose shifted
 * volume (shift c*dt = (s + alpha) cells per axis, s = floor) covers it: overlap fractions
 * (1-alpha) from the cell s behind and alpha from the cell s+1 behind, per axis, multiplied. */
static double gather(const or_ctx *C, const double *f, int l, int x, int y) {
    const double ax = C->axw[l], ay = C->ayw[l];
    const int bx = x - C->sx[l], by = y - C->sy[l];
    return (1.0 - ay) * ((1.0 - ax) * source_value(C, f, l, bx, by) + ax * source_value(C, f, l, bx - 1, by)) +
           ay * ((1.0 - ax) * source_value(C, f, l, bx, by - 1) + ax * source_value(C, f, l, bx - 1, by - 1));
}

/* Diffuse-reflection wall through ghost rows (Eq. "IMPOSITION"): per wall and column x, the
 * mass that the gather would move out of the fluid into the rows beyond the wall (outgoing
 * populations, c.n > 0 with n the wall's outward normal) is re-emitted by the incoming
 * populations (c.n <= 0) in the shape of the wall equilibrium f_eq(1, u_w, T_w): each incoming
 * ghost row holds A(x) f_eq_l, and a uniform ghost column feeds |c_y| dt of it into the fluid,
 * so A(x) = M_out(x) / sum_in |c_y dt| f_eq_l. */
static void wall_ghosts(or_ctx *C, const double *f) {
    const int nx = C->nx, ny = C->ny, Q = C->Q;
    int depth = 1;
    for (int l = 0; l < Q; ++l) {
        int a = abs(C->sy[l]) + 2;
        if (a > depth) depth = a;
    }
    for (int side = 0; side < 2; ++side) {
        const double uw = side == 0 ? C->u_lo : C->u_hi;
        const double Tw = side == 0 ? C->T_lo : C->T_hi;
        double feqw[OR_MAXQ];
        equilibrium(C, 1.0, uw, 0.0, Tw, feqw);
        double den = 0.0;
        for (int l = 0; l < Q; ++l) {
            const int incoming = side == 0 ? C->cy[l] > 0.0 : C->cy[l] < 0.0;
            if (incoming) den += fabs(C->cy[l] * C->dt) * feqw[l];
        }
        /* ghost values must read as zero while M_out is measured */
        memset(C->ghost + (size_t)side * Q * nx, 0, sizeof(double) * (size_t)Q * nx);
        for (int x = 0; x < nx; ++x) {
            double mout = 0.0;
            for (int l = 0; l < Q; ++l) {
                const int outgoing = side == 0 ? C->cy[l] < 0.0 : C->cy[l] > 0.0;
                if (!outgoing) continue;
                for (int d = 1; d <= depth; ++d) {
                    const int yd = side == 0 ? -d : ny - 1 + d;
                    mout += gather(C, f, l, x, yd);
                }
            }
            const double A = mout / den;
            for (int l = 0; l < Q; ++l) {
                const int incoming = side == 0 ? C->cy[l] > 0.0 : C->cy[l] < 0.0;
                if (incoming) C->ghost[((size_t)side * Q + l) * nx + x] = A * feqw[l];
            }
        }
    }
}

/* One time step from the post-collision state f_in to the post-collision state f_out:
 * stream (volumetric gather), then, per cell, moments, equilibrium and BGK relaxation
 * f* = f - (dt/tau)(f - f_eq)  (Eq. "eq:lb" integrated over one step of length dt). */
static void one_step(or_ctx *C, const double *fin, double *fout) {
    const int nx = C->nx, ny = C->ny, Q = C->Q;
    const size_t plane = (size_t)nx * ny;
    const int nth = C->nthreads > 0 ? C->nthreads : omp_get_max_threads();
    if (C->walls) wall_ghosts(C, fin);
    for (int l = 0; l < Q; ++l) {
#pragma omp parallel for schedule(static) num_threads(nth)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) C->ftilde[(size_t)l * plane + (size_t)y * nx + x] = gather(C, fin, l, x, y);
    }
#pragma omp parallel for schedule(static) num_threads(nth)
    for (long long c = 0; c < (long long)plane; ++c) {
        double rho, ux, uy, T, feq[OR_MAXQ];
        moments_of(C, C->ftilde + c, plane, &rho, &ux, &uy, &T);
        equilibrium(C, rho, ux, uy, T, feq);
        for (int l = 0; l < Q; ++l) {
            const double ft = C->ftilde[(size_t)l * plane + c];
            fout[(size_t)l * plane + c] = ft - C->omega * (ft - feq[l]);
        }
    }
}

/* nsteps steps; f holds the state on entry and on exit, work is a buffer of the same size. */
void oracle_run(void *p, double *f, double *work, int nsteps) {
    or_ctx *C = (or_ctx *)p;
    const size_t n = (size_t)C->Q * C->nx * C->ny;
    double *a = f, *b = work;
    for (int s = 0; s < nsteps; ++s) {
        one_step(C, a, b);
        double *t = a;
        a = b;
        b = t;
    }
    if (a != f) memcpy(f, a, n * sizeof(double));
}

/* Streaming alone (no collision), for the streaming pins. */
void oracle_stream(void *p, const double *fin, double *fout) {
    or_ctx *C = (or_ctx *)p;
    const int nx = C->nx, ny = C->ny;
    if (C->walls) wall_ghosts(C, fin);
    for (int l = 0; l < C->Q; ++l)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) fout[((size_t)l * ny + y) * nx + x] = gather(C, fin, l, x, y);
}

/* Collision alone (moments, equilibrium, BGK) on every cell. */
void oracle_collide(void *p, const double *fin, double *fout) {
    or_ctx *C = (or_ctx *)p;
    const size_t plane = (size_t)C->nx * C->ny;
    for (size_t c = 0; c < plane; ++c) {
        double rho, ux, uy, T, feq[OR_MAXQ];
        moments_of(C, fin + c, plane, &rho, &ux, &uy, &T);
        equilibrium(C, rho, ux, uy, T, feq);
        for (int l = 0; l < C->Q; ++l) {
            const double ft = fin[(size_t)l * plane + c];
            fout[(size_t)l * plane + c] = ft - C->omega * (ft - feq[l]);
        }
    }
}

void oracle_moments(void *p, const double *f, double *rho, double *ux, double *uy, double *T) {
    or_ctx *C = (or_ctx *)p;
    const size_t plane = (size_t)C->nx * C->ny;
    for (size_t c = 0; c < plane; ++c) moments_of(C, f + c, plane, &rho[c], &ux[c], &uy[c], &T[c]);
}

/* Global sums M = sum f, P = sum c f, E = (1/2) sum |c|^2 f over all cells and velocities. */
void oracle_conserved_sums(void *p, const double *f, double *out4) {
    or_ctx *C = (or_ctx *)p;
    const size_t plane = (size_t)C->nx * C->ny;
    double M = 0.0, Px = 0.0, Py = 0.0, E = 0.0;
    for (int l = 0; l < C->Q; ++l) {
        double s = 0.0;
        for (size_t c = 0; c < plane; ++c) s += f[(size_t)l * plane + c];
        M += s;
        Px += C->cx[l] * s;
        Py += C->cy[l] * s;
        E += 0.5 * (C->cx[l] * C->cx[l] + C->cy[l] * C->cy[l]) * s;
    }
    out4[0] = M;
    out4[1] = Px;
    out4[2] = Py;
    out4[3] = E;
}

/* Ghost values of the last wall update, [2][Q][nx] (bottom, top), for the wall pins. */
void oracle_ghosts(void *p, double *out) {
    or_ctx *C = (or_ctx *)p;
    memcpy(out, C->ghost, sizeof(double) * (size_t)2 * C->Q * C->nx);
}
