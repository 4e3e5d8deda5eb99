/*
 * tvlbm.h -- C ABI of the GB300 thermal volumetric lattice Boltzmann (TVLBM) library.
 *
 * The library advances the BGK kinetic equation (Eq. "eq:lb") on a 2-D grid of unit cells
 * with an off-lattice tensor-product Gauss-Hermite velocity set.  One time step is one fused
 * CUDA sweep:
 *   stream   every population moves by c_l dt and is shared among the (up to four) cells its
 *            shifted cell volume overlaps, with area-overlap weights fixed per velocity
 *            (the volumetric formulation of the Introduction: off-lattice velocities without
 *            giving up exact conservation), written as a pull-gather;
 *   moments  rho, u, T (Sec. "The TVLBM model", moment definitions);
 *   equilib. the Hermite expansion f_eq = w sum_n a^(n):H^(n)/n! (Sec. "The TVLBM model";
 *            Appendix A), truncated at the order the velocity set integrates exactly;
 *   relax    f* = f - (dt/tau)(f - f_eq).
 * Walls (optional) are diffuse reflectors: the flux that leaves the fluid through a wall is
 * re-emitted in the shape of the wall equilibrium (Sec. "Boundary Condition: Diffuse
 * Scattering Kernel", Eq. IMPOSITION).
 *
 * Conventions for every call:
 *   - returns TVLBM_OK (0) or a negative TVLBM_E* code; never aborts or exits;
 *     tvlbm_last_error() gives a message for the last failing call on a context;
 *   - host buffers passed in are owned by the caller and only used during the call;
 *   - device memory given to tvlbm_create_in is owned by the caller and must outlive the
 *     context; memory the library allocates itself is freed by tvlbm_destroy;
 *   - grid fields are row-major [ny][nx] (x fastest), FP64; population arrays are
 *     [Q][ny][nx] with velocity index l = i + n*j, where c_l = (x_i, x_j) and x_0 < ... < x_{n-1}
 *     are the n Gauss-Hermite nodes (n = 3, 4, 6 for D2Q9, D2Q16, D2Q36);
 *   - lattice units: cell size dx = dy = 1, sound speed c_s = 1 (reference temperature 1);
 *   - calls on one context are not thread-safe; distinct contexts are independent.
 *   - GPU work is queued on the context's stream (tvlbm_set_stream); calls that return
 *     host data synchronise that stream.
 */
#ifndef TVLBM_H
#define TVLBM_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------------------------- */
#define TVLBM_OK 0
#define TVLBM_EINVAL (-1)     /* invalid argument (size, parameter, null pointer, combination) */
#define TVLBM_ENOMEM (-2)     /* device or host allocation failed, or caller memory too small */
#define TVLBM_ECUDA (-3)      /* a CUDA runtime call failed (including: no GPU present)        */
#define TVLBM_ESTATE (-4)     /* call not valid in the context's current state                 */
#define TVLBM_ETIMEOUT (-5)   /* a bounded device-side wait gave up                            */
#define TVLBM_ENONFINITE (-6) /* non-finite populations detected                               */

/* ---- velocity sets: tensor products of n-point Gauss-Hermite rules ----------------------- */
#define TVLBM_D2Q9 9   /* n = 3, nodes 0, +-sqrt(3); Hermite order N = 2                 */
#define TVLBM_D2Q16 16 /* n = 4, nodes +-sqrt(3 -+ sqrt 6); N = 3                        */
#define TVLBM_D2Q36 36 /* n = 6; N = 5                                                   */

/* ---- population storage ----------------------------------------------------------------- */
#define TVLBM_FP64 0     /* f_l as double; FP64 arithmetic                                   */
#define TVLBM_FP32 1     /* f_l as float;  FP32 arithmetic on f_l - w_l (the unit-density rest
                            population, exact to FP64, split off: only the store rounds
                            relative to f)                                                    */
#define TVLBM_BF16_DEV 2 /* d_l = (f_l - w_l rho0)/w_l as bfloat16 (round to nearest even);
                            FP32 arithmetic                                                   */
#define TVLBM_FP16_DEV 3 /* d_l as IEEE binary16 (round to nearest even); FP32 arithmetic     */
#define TVLBM_FP32_DEV 4 /* d_l as float; FP32 arithmetic                                      */

/* ---- sweep kernel forms ------------------------------------------------------------------ */
#define TVLBM_FORM_PLAIN 0 /* one thread per cell, direct gathers from global memory           */
#define TVLBM_FORM_TILED 1 /* 2-D tiles whose per-velocity source windows are staged in shared
                              memory by TMA; the default                                       */
#define TVLBM_FORM_FLOW 2  /* the tiled sweep of several time steps in one persistent launch: a
                              tile starts a step as soon as its 3 x 3 periodic neighbourhood has
                              finished the previous one (no launch boundary between steps).
                              Periodic domains whose size is a multiple of the tile shape only */
#define TVLBM_FORM_STRIP 3 /* 128-column strips: each CTA walks a run of rows of a strip, one
                              column per thread, carrying the previous row in registers, with a
                              ring of TMA row-chunk copies issued chunks ahead of the compute.
                              Any domain, walls included; independent of the tile configuration */

/* ---- evolution schemes ------------------------------------------------------------------- */
#define TVLBM_SCHEME_VOLUMETRIC 0 /* fused BGK collide + area-overlap pull-gather stream (default)   */
#define TVLBM_SCHEME_FVLB 1       /* the paper's finite-volume update (Sec. "The TVLBM Evolution
                                     scheme", Eq. FVLB): explicit Euler step of length dt with the
                                     second-order 9-point stencils for c . grad f and the weighted
                                     9-point average of the collision term of Eq. OMEGAFVLB         */

/* ---- boundary conditions ----------------------------------------------------------------- */
#define TVLBM_BC_PERIODIC 0
#define TVLBM_BC_WALLS 1 /* periodic in x; diffuse walls on the faces y = -1/2 and y = ny - 1/2 */

typedef struct tvlbm_bc {
    int kind;    /* TVLBM_BC_PERIODIC or TVLBM_BC_WALLS                               */
    double u_lo; /* x-velocity of the wall at y = -1/2 (walls only)                   */
    double T_lo; /* temperature of that wall, > 0                                     */
    double u_hi; /* x-velocity of the wall at y = ny - 1/2                            */
    double T_hi; /* temperature of that wall, > 0                                     */
} tvlbm_bc;

typedef struct tvlbm_ctx tvlbm_ctx;

/* Device bytes a context needs for these arguments (populations, ghost frame, scratch).
 * Host-only; needs no GPU.  bc may be NULL (periodic).  Errors: EINVAL. */
int tvlbm_memory_bytes(int nx, int ny, int velset, const tvlbm_bc *bc, int storage, size_t *bytes);

/* Create a context on the current CUDA device and allocate its device memory.
 *   nx, ny   fluid cells, >= 1 each (walls: ny >= 9);  nx*ny < 2^31
 *   velset   TVLBM_D2Q9 / TVLBM_D2Q16 / TVLBM_D2Q36
 *   tau      BGK relaxation time (Eq. "eq:lb"), tau > dt/2 for a positive viscosity;
 *            +inf gives collisionless streaming
 *   dt       time step; every shift |c dt| must stay below 4 cells
 *   bc       boundary conditions, NULL for periodic
 *   storage  TVLBM_FP64 .. TVLBM_FP32_DEV
 *   rho0     reference density of the deviation storage (also used by FP storage), > 0
 * Populations start at the rest equilibrium f = rho0 w_l.  *out receives the handle.
 * Errors: EINVAL (arguments), ENOMEM, ECUDA (no device or a CUDA failure). */
int tvlbm_create(int nx, int ny, int velset, double tau, double dt, const tvlbm_bc *bc, int storage,
                 double rho0, tvlbm_ctx **out);

/* As tvlbm_create, but the context lives in caller-owned device memory `device_memory` of
 * `bytes` >= tvlbm_memory_bytes(...) bytes, 256-byte aligned; the library allocates no device
 * memory.  Errors: EINVAL, ENOMEM (too small), ECUDA. */
int tvlbm_create_in(int nx, int ny, int velset, double tau, double dt, const tvlbm_bc *bc, int storage,
                    double rho0, void *device_memory, size_t bytes, tvlbm_ctx **out);

/* Free the context (synchronises its stream first).  NULL is accepted. */
int tvlbm_destroy(tvlbm_ctx *ctx);

/* Queue all later GPU work of this context on `stream` (a cudaStream_t; NULL = legacy default).
 * The stream must belong to the context's device. */
int tvlbm_set_stream(tvlbm_ctx *ctx, void *stream);

/* Select the sweep kernel form (TVLBM_FORM_PLAIN / TVLBM_FORM_TILED / TVLBM_FORM_FLOW /
 * TVLBM_FORM_STRIP).  All give the same populations up to floating-point rounding order; the
 * tiled, dataflow and strip forms give identical ones.  Errors: EINVAL (unknown form; a
 * TMA form without a TMA descriptor;
 * the dataflow form on walls or on a domain the current tile configuration does not cover
 * exactly).  With the dataflow form, tvlbm_step(ctx, n) is one launch (captured graphs are not
 * used) and a device-side wait that gives up is reported as ETIMEOUT by the next synchronising
 * call. */
int tvlbm_set_form(tvlbm_ctx *ctx, int form);

/* Select the evolution scheme.  TVLBM_SCHEME_FVLB: f(t + dt) = f + dt (Omega_bar - c . grad f)
 * on the unit grid, Omega_l = -(f_l - f_eq_l) / tau + (1 / tau_g) f_eq_l / (rho T^2)
 * Pi : (c_l - u)(c_l - u) with Pi_ij = sum_l (f_l - f_eq_l)(c_l - u)_i (c_l - u)_j (Eq.
 * OMEGAFVLB; the Prandtl-number term is applied without its components along the collision
 * invariants, which an exact Maxwellian would not have; tau_g = +inf leaves it out).  It
 * shifts the viscosity to T tau tau_g / (tau_g - 2 tau) (the Prandtl number to
 * tau_g / (tau_g - 2 tau)).  The scheme is explicit: it needs |c| dt well below one cell and
 * dt well below tau.  Periodic domains, or channels (walls, see tvlbm_set_fv_walls); FP64 or
 * FP32 storage; allocates one extra population-sized buffer (also for contexts created in
 * caller memory).  Errors: EINVAL (storage, unknown scheme, tau_g = 0 or NaN), ENOMEM. */
int tvlbm_set_scheme(tvlbm_ctx *ctx, int scheme, double tau_g);

/* Finite-volume scheme: enable (1) or disable (0, default) the scaling of both relaxation times
 * with the local pressure, tau -> tau / p and tau_g -> tau_g / p with p = rho T (Sec. "Boundary
 * Conditions: Avoiding temperature and velocity slip", and the grid-refinement section): the
 * dynamic viscosity tau tau_g / (tau_g - 2 tau) and the conductivity c_P tau (c_P = 2) no longer
 * vary with density and temperature, as the closed-form thermal Couette profiles assume.  Call
 * after tvlbm_set_scheme(TVLBM_SCHEME_FVLB).  Errors: EINVAL (not the finite-volume scheme). */
int tvlbm_set_fv_pressure_scaling(tvlbm_ctx *ctx, int enable);

/* Finite-volume scheme: one fused kernel per step (fused = 1, default) or two (fused = 0).  The
 * fused kernel computes the collision term of Eq. OMEGAFVLB for a block of cells in shared memory
 * and updates the block's inner cells from it (Eq. FVLB): Q values read and Q written per cell
 * update.  The two-kernel form stores the collision term of every cell in the buffer
 * tvlbm_set_scheme allocates and reads it back in the update (5 Q values per cell update).  Both
 * run the same arithmetic and give the same populations bit for bit.  May be called at any time;
 * takes effect at the next step.  Errors: EINVAL (null context). */
int tvlbm_set_fv_fused(tvlbm_ctx *ctx, int fused);

/* Finite-volume scheme on a channel (a context created with TVLBM_BC_WALLS): the first and
 * last node rows are wall nodes (walls on the nodes, unlike the volumetric scheme's faces).
 * Populations arriving at a wall node advance with the one-sided stencils of Eq. FVLB2; the
 * leaving ones are set before every step to A f_eq(u_eq, T_eq), A balancing the normal mass
 * flux (Eq. IMPOSITION, |c . n| weights).  exact = 0: (u_eq, T_eq) = the wall's (u, T)
 * (diffuse reflection: velocity slip, temperature jump); exact = 1: (u_eq, T_eq) corrected by
 * nr_iters Newton-Raphson iterations (App. B, warm-started from the previous step per column)
 * so that the wall node's velocity and temperature are the wall's.  y_nodes: host array of the
 * ny node positions (increasing; NULL: unit spacing), e.g. the tanh mesh of Eq. NONUNI2; the
 * x spacing is 1.  Call after tvlbm_set_scheme(TVLBM_SCHEME_FVLB).  Errors: EINVAL (no walls,
 * not the finite-volume scheme, nr_iters < 1 with exact, y_nodes not increasing), ENOMEM. */
int tvlbm_set_fv_walls(tvlbm_ctx *ctx, int exact, int nr_iters, const double *y_nodes);

/* Volumetric scheme on a mesh that is non-uniform in y (the grid refinement of Sec. "Grid
 * Refinement for simple unidirectional flows", Eqs. NONUNI1-2, e.g. cells crowded towards the
 * walls): cell y spans [faces[y], faces[y+1]] (faces: host array of ny + 1 increasing values,
 * copied; x keeps unit cells).  Per velocity, destination row y gathers sum_r w_r f_r with
 * w_r = |[faces[y] - c_y dt, faces[y+1] - c_y dt] within cell r| / h_y, the uniform scheme's area
 * overlap on unequal cells; with walls (a TVLBM_BC_WALLS context, walls at faces[0] and faces[ny])
 * the part beyond a wall is filled with A(x) f_eq(1, u_w, T_w) for the incoming velocities, A
 * re-emitting what the outgoing ones carry beyond it (Eq. IMPOSITION), so mass is conserved.
 * Periodic contexts repeat the mesh with period faces[ny] - faces[0].  The conserved quantities
 * are the sums weighted by the cell heights, which tvlbm_conserved_sums then returns.  Runs the
 * plain form only (sets it; other forms are refused while a mesh is set), FP64, FP32 or
 * FP32-deviation storage with a single reference, the volumetric scheme.  A row may gather from
 * at most 64 cells (cells far thinner than c dt are refused).  faces = NULL returns to unit
 * cells.  Allocates the tables (a few bytes per row and velocity); synchronises.  Errors: EINVAL
 * (faces not finite or not increasing, storage, scheme, a per-row reference, too thin cells),
 * ENOMEM, ECUDA. */
int tvlbm_set_y_faces(tvlbm_ctx *ctx, const double *faces);

/* Enable (1, default) or disable (0) replay of multi-step runs through captured CUDA graphs. */
int tvlbm_set_graphs(tvlbm_ctx *ctx, int enable);

/* Deviation storage only: express the stored populations against the reference equilibrium
 * f_eq(rho0, (ux, uy), T), i.e. store d_l = f_l / w_l - f_eq_l / w_l (default: at rest, T = 1).
 * A reference near the flow's mean state shrinks |d| and with it the half-precision rounding
 * error.  The current state is re-encoded (synchronises).  Errors: EINVAL (full-f storage,
 * T <= 0).  Allocates the context's re-encoding buffer on first use (see
 * tvlbm_set_reference_rows). */
int tvlbm_set_reference(tvlbm_ctx *ctx, double ux, double uy, double T);

/* Deviation storage on a domain with walls: a reference that varies across the channel.  Fluid
 * row y (0 <= y < ny) stores d_l = f_l / w_l - R_l(y), R_l(y) = f_eq_l(rho0, (ux[y], uy[y]), T[y]) / w_l;
 * the ghost rows beyond a wall take the adjacent fluid row's reference.  A wall-driven flow (a
 * Couette channel with a temperature difference) varies mostly across the channel, so a profile
 * that follows it (e.g. linear between the wall values) keeps |d| near the non-equilibrium part
 * and the half-precision rounding error with it.  The time step is unchanged in exact
 * arithmetic: the gather of row y adds S_l(y), the gather of R over the source rows minus R_l(y),
 * and the collision takes the row's reference moments (tables of a few hundred bytes per row,
 * built on the device).  ux, uy, T: host arrays of ny values (copied).  The current state is
 * re-encoded (synchronises); tvlbm_set_reference returns to a single reference.  The first call
 * allocates the context's reference tables and re-encoding buffer with cudaMalloc (about
 * 2 (40 doubles + 48 floats) + 36 floats per stored row and 3 ny doubles; kept until
 * tvlbm_destroy), also for a context created in caller-provided memory.  Errors: EINVAL (full-f storage, periodic domain, null array, T <= 0 or a
 * non-finite value), ENOMEM, ECUDA. */
int tvlbm_set_reference_rows(tvlbm_ctx *ctx, const double *ux, const double *uy, const double *T);

/* Deviation storage on a domain with walls: keep the per-row reference following the flow.
 * Every `every` time steps tvlbm_step resets the reference rows to the current rows (the
 * equilibria of the row averages of (ux, uy, T), or the row averages of the populations, see
 * tvlbm_set_reference_kind) and re-encodes the state: a row-average pass, two small table kernels
 * and one re-encoding pass over the state, queued on the context's stream without a host
 * synchronisation.  With no per-row reference yet, one is taken from the current state at once.
 * A row whose average is not a valid state (T <= 0, not finite) takes the default reference.
 * every = 0 turns refreshing off (the reference stays as it is).  Refreshing only changes the
 * encoding: in exact arithmetic the state is unchanged.  Errors: EINVAL (full-f storage,
 * periodic domain, every < 0), ENOMEM, ECUDA. */
int tvlbm_set_reference_refresh(tvlbm_ctx *ctx, int every);

/* What a refresh of the per-row reference (tvlbm_set_reference_refresh) installs:
 *   TVLBM_REF_EQUILIBRIUM (default)  R_l(y) = f_eq_l(rho0, row average of (ux, uy), row average of T) / w_l;
 *   TVLBM_REF_MEAN                   R_l(y) = the row average of f_l / w_l itself, the full population
 *                                    (non-equilibrium part and the row's density included).
 * With the mean kind, a flow that varies only across the channel (a Couette flow between the
 * walls) is stored as its departures from its own row averages, which stay small between
 * refreshes: the half-precision rounding error shrinks with them (BF16 deviation storage needs
 * it to stay within 1e-3 on such a channel).  Either kind is an exact re-encoding; it takes effect
 * at the next refresh.  Errors: EINVAL (unknown kind, full-f storage, periodic domain). */
#define TVLBM_REF_EQUILIBRIUM 0
#define TVLBM_REF_MEAN 1
int tvlbm_set_reference_kind(tvlbm_ctx *ctx, int kind);

/* Tile configurations of the tiled form (an autotuner picks among them): their number, and
 * the shape of one -- tile width and height in cells and rows each thread walks.
 * tvlbm_set_tile selects one (synchronises the stream; default 0).  Errors: EINVAL (out of
 * range; with the dataflow form, a configuration that does not cover the domain exactly). */
int tvlbm_tile_count(const tvlbm_ctx *ctx);
int tvlbm_tile_shape(const tvlbm_ctx *ctx, int config, int *tx, int *ty, int *rows_per_thread);
int tvlbm_set_tile(tvlbm_ctx *ctx, int config);

/* Initialise every cell to the equilibrium f_eq(rho, u, T) (Sec. "The TVLBM model"),
 * computed in FP64 and rounded to the storage format.  Host FP64 fields [ny][nx];
 * requires rho > 0 and T > 0 everywhere (EINVAL otherwise, nothing written).
 * Synchronises the stream. */
int tvlbm_init_moments(tvlbm_ctx *ctx, const double *rho, const double *ux, const double *uy, const double *T);

/* Advance n >= 0 time steps (asynchronous on the context's stream).  Each step: (walls) fill
 * the ghost rows from the flux leaving the fluid (Eq. IMPOSITION), then one fused sweep
 * stream -> moments -> equilibrium -> BGK -> store.  Errors: EINVAL (n < 0), ECUDA. */
int tvlbm_step(tvlbm_ctx *ctx, int n);

/* Macroscopic fields of the current state (Sec. "The TVLBM model": rho = sum f,
 * rho u = sum c f, rho T = (1/D) sum |c - u|^2 f, D = 2), computed in FP64 on the GPU from
 * the stored populations.  Any output pointer may be NULL.  Host arrays [ny][nx].
 * Synchronises the stream. */
int tvlbm_moments(tvlbm_ctx *ctx, double *rho, double *ux, double *uy, double *T);

/* Global sums over all fluid cells and velocities, accumulated in FP64 on the GPU by a
 * deterministic two-pass reduction (the conserved quantities of the Abstract and Sec. "The
 * TVLBM model"):
 *   out[0] = M  = sum f,  out[1] = P_x = sum c_x f,  out[2] = P_y = sum c_y f,
 *   out[3] = E  = (1/2) sum |c|^2 f,  out[4] = number of non-finite stored populations.
 * Synchronises the stream.  Returns TVLBM_ENONFINITE, with out filled, when out[4] > 0 (a
 * device wait that gave up since the last synchronising call is reported first, as
 * TVLBM_ETIMEOUT). */
int tvlbm_conserved_sums(tvlbm_ctx *ctx, double out[5]);

/* Failure-path hook of the dataflow form (TVLBM_FORM_FLOW), for tests: limit_s is the limit of
 * the wait of a launch's producer for a task's 3 x 3 neighbourhood (default 2 s; accepted
 * 1e-6 .. 2 s); unmet != 0 makes that wait require a completion count no tile reaches.  A wait
 * that gives up raises the launch's abort word and the device status; the other CTAs stop at
 * their next wait, every CTA drains the loads it started, and the launch ends early with the
 * populations partly advanced.  tvlbm_step still returns TVLBM_OK (it does not synchronise); the
 * next synchronising call returns TVLBM_ETIMEOUT and clears the status.  Restore the state with
 * tvlbm_set_populations (or tvlbm_init_moments).  Errors: EINVAL. */
int tvlbm_set_flow_wait(tvlbm_ctx *ctx, double limit_s, int unmet);

/* Conserved sums that allocate nothing, for callers that cannot call cudaMalloc or any other
 * allocator on this path (code running inside another framework's memory pool or a
 * stream-ordered pipeline that owns all device memory).  The paper has no counterpart: this
 * is an interface variant of tvlbm_conserved_sums, the same FP64 two-pass reduction.
 *   populations  device pointer, packed [Q][ny][nx] in the storage format (the layout
 *                tvlbm_get_populations returns), caller-owned
 *   velset, storage, nx, ny, rho0   describe that array (rho0: the reference density of
 *                deviation storage, read as d = f/w - rho0, the default reference; an array
 *                saved under tvlbm_set_reference or a per-row reference is not in that form)
 *   out5         device pointer to 5 doubles, caller-owned: M, P_x, P_y, E, #non-finite
 *   stream       cudaStream_t the two kernels are queued on (asynchronous; NULL = default)
 * The per-block partial sums live in a fixed device array of 1024 x 5 doubles (40 KiB) that
 * every GPU which loads the library holds until the process exits.  A call on a stream that
 * is not capturing looks up that array's address (cudaGetSymbolAddress, with the device
 * current) every time, so a device reset that reloads the library's module is followed; a call
 * on a capturing stream uses the address the last such call on this device saw, so make one
 * call before any stream capture (else ECUDA).  Each call overwrites the whole array, so
 * nothing needs clearing; calls that overlap on the GPU race on it.  No cudaMalloc, cudaFree
 * or allocating library call, so a call can be captured in a CUDA graph.
 * Errors: EINVAL (null pointer, unknown set or storage, Q*nx*ny > 2^31 - 1 populations),
 * ECUDA (including a first call under stream capture). */
int tvlbm_conserved_sums_static(const void *populations, int velset, int storage, int nx, int ny, double rho0,
                                double *out5, void *stream);

/* Checkpoint: copy the raw stored populations (storage format, [Q][ny][nx], no ghost frame)
 * to / from host memory of exactly tvlbm_population_bytes(ctx) bytes.  set_populations also
 * refreshes the periodic ghost frame.  Both synchronise the stream.  Errors: EINVAL (size). */
size_t tvlbm_population_bytes(const tvlbm_ctx *ctx);
int tvlbm_get_populations(tvlbm_ctx *ctx, void *host, size_t bytes);
int tvlbm_set_populations(tvlbm_ctx *ctx, const void *host, size_t bytes);

/* Populations decoded to f_l in FP64, [Q][ny][nx] (deviation storage: f = w (rho0 + d)). */
int tvlbm_get_populations_f64(tvlbm_ctx *ctx, double *host);
/* Encode FP64 populations f_l [Q][ny][nx] into the storage format (round to nearest even). */
int tvlbm_set_populations_f64(tvlbm_ctx *ctx, const double *host);

/* The library's velocity set (host-only; no GPU): Q nodes c_l = (cx[l], cy[l]) and weights
 * w[l], ordered l = i + n j; *hermite_order receives N.  Arrays hold >= 36 entries.
 * Errors: EINVAL (unknown set). */
int tvlbm_velocity_set(int velset, double *cx, double *cy, double *w, int *hermite_order);

/* Per-velocity streaming table (host-only): shift of c_l dt in cells along x and y as
 * integer part (floor) and overlap fraction alpha in [0, 1); a shift within 1e-12 of an
 * integer counts as that integer with alpha = 0.  Arrays hold >= 36 entries. */
int tvlbm_stream_table(int velset, double dt, int *sx, int *sy, double *ax, double *ay);

/* Algorithmic bytes moved by one sweep per fluid cell: Q * (read + write) * bytes per stored
 * population (halo re-reads and ghost-frame copies not counted). */
double tvlbm_bytes_per_cell(const tvlbm_ctx *ctx);

/* ---- batched domains ------------------------------------------------------------------------
 * Many independent periodic domains of different sizes and relaxation times (one velocity set,
 * storage and dt), advanced together: each time step one launch of the tiled sweep over the
 * tiles of every domain (multi-step runs replay captured CUDA graphs), or many time steps in one
 * persistent dataflow launch (tvlbm_batch_set_form).
 * Domain d is nx[d] x ny[d] cells with relaxation time tau[d]; everything else follows the
 * single-domain calls above (layouts, errors, ownership, stream semantics). */
typedef struct tvlbm_batch tvlbm_batch;

/* Device bytes of a batch (host-only).  Errors: EINVAL. */
int tvlbm_batch_memory_bytes(int count, const int *nx, const int *ny, int velset, int storage, size_t *bytes);
/* Create a batch on the current device (library-owned memory, or caller-owned device memory of
 * >= tvlbm_batch_memory_bytes bytes, 256-byte aligned).  All domains start at rest.
 * Errors: EINVAL, ENOMEM, ECUDA. */
int tvlbm_batch_create(int count, const int *nx, const int *ny, const double *tau, int velset, int storage, double dt,
                       double rho0, tvlbm_batch **out);
int tvlbm_batch_create_in(int count, const int *nx, const int *ny, const double *tau, int velset, int storage,
                          double dt, double rho0, void *device_memory, size_t bytes, tvlbm_batch **out);
int tvlbm_batch_destroy(tvlbm_batch *b);
int tvlbm_batch_set_stream(tvlbm_batch *b, void *stream);
int tvlbm_batch_set_graphs(tvlbm_batch *b, int enable);
/* Batch form: TVLBM_FORM_TILED (default; one launch per time step over every domain's tiles,
 * 32-step captured graphs) or TVLBM_FORM_FLOW (tvlbm_batch_step(b, n) advances every domain n
 * steps in ONE persistent launch of the dataflow sweep over the batch's tile list: a tile starts
 * step k once the 3 x 3 periodic neighbourhood of tiles of its own domain has finished step
 * k - 1; the launch is captured as a CUDA graph on the first call and replayed for calls with the
 * same n; its device waits are bounded as in the single-domain form).  The populations are the
 * same, bit for bit.  Errors: EINVAL (unknown form; the dataflow form with a tile configuration
 * that does not cover every domain exactly). */
int tvlbm_batch_set_form(tvlbm_batch *b, int form);
/* Tile configurations of the batched sweep (as tvlbm_tile_*); set_tile rebuilds the tile list. */
int tvlbm_batch_tile_count(const tvlbm_batch *b);
int tvlbm_batch_tile_shape(const tvlbm_batch *b, int config, int *tx, int *ty, int *rows_per_thread);
int tvlbm_batch_set_tile(tvlbm_batch *b, int config);
/* Initialise domain d to the equilibrium of host FP64 fields [ny[d]][nx[d]] (synchronises). */
int tvlbm_batch_init_moments(tvlbm_batch *b, int domain, const double *rho, const double *ux, const double *uy,
                             const double *T);
/* Advance every domain n time steps (asynchronous). */
int tvlbm_batch_step(tvlbm_batch *b, int n);
/* Diagnostics and populations of domain d, as tvlbm_moments / tvlbm_conserved_sums (including
 * its TVLBM_ENONFINITE) / tvlbm_get_populations_f64 (synchronise). */
int tvlbm_batch_moments(tvlbm_batch *b, int domain, double *rho, double *ux, double *uy, double *T);
int tvlbm_batch_conserved_sums(tvlbm_batch *b, int domain, double out[5]);
int tvlbm_batch_get_populations_f64(tvlbm_batch *b, int domain, double *host);
/* Total fluid cells of all domains; algorithmic bytes per cell update (as tvlbm_bytes_per_cell). */
long long tvlbm_batch_cells(const tvlbm_batch *b);
double tvlbm_batch_bytes_per_cell(const tvlbm_batch *b);
const char *tvlbm_batch_last_error(const tvlbm_batch *b);

/* Message of the last failing call on ctx (never NULL; "" if none). */
const char *tvlbm_last_error(const tvlbm_ctx *ctx);

/* Static description of a status code. */
const char *tvlbm_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* TVLBM_H */
