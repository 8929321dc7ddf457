/*
 * dg.h -- C ABI of libdg, a GB300 (sm_103a) implementation of the explicit split-form DGSEM
 * hot path of "Towards Exascale CFD Simulations Using the Discontinuous Galerkin Solver FLEXI"
 * (arXiv 2306.12891): the right-hand side of the compressible Euler / Navier-Stokes-Fourier
 * equations on curved hexahedra with Legendre-Gauss-Lobatto nodes (Sec. 2), its explicit
 * low-storage Runge-Kutta stage update (Sec. 2, Eq. (1)), and the DG/FV subcell blend with the
 * modified Persson indicator (Sec. 4.1, Eqs. (6)-(7)).
 *
 * Conventions
 *  - n = N+1; node index = i + n*(j + n*k), i along xi.
 *  - Solution arrays U, Ut: FP64, layout [n_elems][5][n][n][n] with the conservative variables
 *    (rho, rho u, rho v, rho w, E). Unless a name ends in _host, every array argument is a
 *    DEVICE pointer owned by the caller (e.g. a torch tensor) and must stay valid until the
 *    work queued on the context's stream has finished.
 *  - All solver calls are asynchronous on the context's CUDA stream, except those documented as
 *    synchronising. No call throws; a non-zero dg_status is returned and dg_last_error() gives
 *    text. A context is not thread-safe: one host thread at a time.
 *  - The library owns its geometry (metrics, Jacobian, face normals), its work buffers and the
 *    LSERK register; dg_free() releases them.
 */
#ifndef DG_H
#define DG_H
#ifdef __cplusplus
extern "C" {
#endif

typedef struct dg_ctx dg_ctx; /* opaque, library-owned */

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = -1,          /* bad argument: null pointer, size, enum value, N out of range */
  DG_ERR_MESH = -2,         /* inconsistent face table (index out of range, face slot unused or reused) */
  DG_ERR_JACOBIAN = -3,     /* J <= 0 or not finite at some node */
  DG_ERR_CUDA = -4,         /* a CUDA runtime call failed (text in dg_last_error) */
  DG_ERR_NONPHYSICAL = -5,  /* rho <= 0, p <= 0 or a non-finite value met by a kernel */
  DG_ERR_UNSUPPORTED = -6,  /* valid request the library does not implement */
  DG_ERR_OOM = -7           /* device allocation failed */
} dg_status;

enum { DG_EULER = 0, DG_NAVIER_STOKES = 1 };
/* split-form two-point volume fluxes (Sec. 2: "split-form DG formulation"; Sec. 4.1) */
enum { DG_VFLUX_KG = 0, DG_VFLUX_PIROZZOLI = 1, DG_VFLUX_EC = 2, DG_VFLUX_CENTRAL = 3 };
/* surface Riemann fluxes */
enum { DG_SFLUX_LLF = 0, DG_SFLUX_ROE = 1, DG_SFLUX_EC = 2 };
/* DG_FP64: all arithmetic FP64. DG_FP32_BULK: volume/surface/lifting arithmetic in FP32 with FP32
 * accumulation; LSERK state, metrics, Jacobian scaling and reductions stay FP64. U, Ut stay FP64. */
enum { DG_FP64 = 0, DG_FP32_BULK = 1 };
/* boundary kinds (faceR of a face with elemR = -1) */
enum { DG_BC_WALL_MODEL = 0 };
/* Legendre-Gauss-Lobatto nodes (Sec. 2), the only node set */
enum { DG_NODES_LGL = 0 };

/* Unstructured hexahedral mesh; elements are the unit of work (Sec. 2). Host memory, read by
 * dg_init only (copied). Periodic connections are ordinary faces. */
typedef struct {
  int n_elems;
  int n_geo;          /* geometry degree; must equal N (isoparametric, nodes = LGL nodes) */
  const double *xyz;  /* [n_elems][3][n_geo+1]^3 physical coordinates of the nodes */
  int n_faces;
  const int *face;    /* [n_faces][5]: elemL, faceL, elemR, faceR, orient.
                         local faces 0:xi-, 1:xi+, 2:eta-, 3:eta+, 4:zeta-, 5:zeta+;
                         face point (p,q) = the two tangential node indices in increasing
                         dimension order; orient maps L's (p,q) to R's:
                         (a,b) = bit2 ? (q,p) : (p,q); a = N-a if bit0; b = N-b if bit1.
                         A boundary face has elemR = -1, faceR = its DG_BC_* kind, orient 0. */
} dg_mesh;

typedef struct {
  int equations;      /* DG_EULER | DG_NAVIER_STOKES */
  int volume_flux;    /* DG_VFLUX_* */
  int surface_flux;   /* DG_SFLUX_* */
  int precision;      /* DG_FP64 | DG_FP32_BULK */
  double gamma, R, mu, Pr; /* ideal gas, constant viscosity, Prandtl number */
  int shock_capturing;     /* 1: DG/FV subcell blend (Sec. 4.1, Eq. (6)) */
  double alpha_min;        /* alpha < alpha_min -> pure DG (Sec. 4.2: 0.01) */
  double alpha_max;        /* alpha clipped to alpha_max (Sec. 4.2: 0.7) */
  double sharpness;        /* s of the indicator sigmoid (Sec. 4.1, Eq. (7)) */
  double alpha_fixed;      /* >= 0: use this blending coefficient on every element; < 0: indicator */
  double p_ref;            /* DG_FP32_BULK only (ignored in DG_FP64): reference pressure removed from the
                              pressure term of the momentum flux. Exact: its contribution is p_ref times the
                              discrete metric identity, zero. Set it near the mean pressure (e.g. p0 of a
                              low-Mach flow) so FP32 forms p - p_ref from O(1) numbers; 0 disables it. */
  /* Wall-modelled walls (Sec. 3): faces with elemR = -1 and faceR = DG_BC_WALL_MODEL. The advective
   * flux is the Riemann flux against the mirror state (no penetration), the BR1 face value uses the
   * same mirror state, and the viscous flux through the wall is the wall shear stress
   * tau_w = rho u_tau^2 against the tangential velocity at the exchange node (wm_index nodes from the
   * wall along the element's wall-normal line, 1 <= wm_index <= N): u_tau from Spalding's law of the
   * wall (Sec. 3, Eq. (2)), the input velocity mapped by the van Driest transform (Eq. (5), freestream
   * speed wm_uinf and Mach number wm_mainf) when wm_van_driest != 0; adiabatic wall at rest. */
  int wm_index;
  double wm_uinf, wm_mainf;
  int wm_van_driest;
} dg_params;

/* Build a solver for `mesh` at polynomial degree N (1..7) with `nodes` = DG_NODES_LGL.
 * Copies the mesh to the device, computes curl-form metrics, Jacobian and face normals on the
 * GPU, and checks them. `cuda_stream` (cudaStream_t, may be NULL = legacy default stream) is the
 * stream every later call is queued on. Synchronising. On success *out owns all device memory. */
dg_status dg_init(const dg_mesh *mesh, int N, int nodes, const dg_params *params, void *cuda_stream,
                  dg_ctx **out);

/* Ut = L(U): the DGSEM time derivative at time t (Sec. 2; Sec. 4.1, Eq. (6) when shock capturing
 * is on). U and Ut are device arrays [n_elems][5][n]^3 and must not overlap. */
dg_status dg_rhs(dg_ctx *ctx, const double *U, double *Ut, double t);

/* One LSERK(5,4) step (Carpenter-Kennedy 2N-storage, five stages, Sec. 2 "explicit Runge-Kutta"):
 * U <- U(t + dt), in place. The register g is library-owned. */
dg_status dg_lserk_step(dg_ctx *ctx, double *U, double dt, double t);

/* n_steps LSERK steps of size dt starting at time t. By default (dg_use_graphs) the launch sequence
 * of one step is captured into a CUDA graph on the first call for a given (U, dt) and replayed
 * for the remaining steps on a library stream ordered after and before the context stream by
 * events (asynchronous as before; the first step runs directly). Kernel timing disables it. */
dg_status dg_lserk_steps(dg_ctx *ctx, double *U, double dt, double t, int n_steps);

/* The same step on a HOST array U_host: copies it to a library-owned device buffer, steps, and
 * returns the result in U_host; synchronising. Page-locked U_host (16-byte aligned, a whole number of
 * 16-byte words) is read by a copy kernel over the host link, and the last stage's volume kernel
 * writes the new state straight into it; other host memory goes through the copy engines both ways.
 * The bits equal dg_lserk_step's. DG_ERR_ARG for a null array or a non-finite dt. */
dg_status dg_lserk_step_host(dg_ctx *ctx, double *U_host, double dt, double t);

/* alpha[e] = blending coefficient of element e (Sec. 4.1, Eq. (7): modified Persson indicator on
 * rho*p, clipped to [alpha_min, alpha_max] (Sec. 4.2), extended to face neighbours by 1/2).
 * alpha: device array [n_elems]. */
dg_status dg_indicator(dg_ctx *ctx, const double *U, double *alpha);

/* Integral diagnostics over the mesh with LGL quadrature (synchronising; host out[8]):
 * out[0..4] = sum J w Ut_v; out[5] = sum J w v.Ut (v = entropy variables);
 * out[6] = sum J w rho|u|^2/2; out[7] = sum J w d/dt(rho|u|^2/2). */
dg_status dg_invariants(dg_ctx *ctx, const double *U, const double *Ut, double out[8]);

/* The same eight integrals as dg_invariants, for callers that cannot allocate device memory where
 * they need them: a host framework whose caching allocator already holds nearly all of the device
 * memory (a cudaMalloc there fails, or forces the pool to give memory back), or real-time and
 * embedded callers whose rules forbid any allocation after start-up. (The paper has no
 * counterpart; this is a service of the library.)
 *  - Needs no context and allocates nothing: every input and output belongs to the caller.
 *    U, Ut: device [n_elems][5][N+1]^3; J: device Jacobian [n_elems][N+1]^3 (e.g. from
 *    dg_get_metrics); out8: device double[8], written asynchronously on `cuda_stream`
 *    (no synchronisation; read it after the stream has reached this work).
 *  - Partial sums live in one fixed device array of 2048 x 8 doubles (128 KiB) inside the library,
 *    which every GPU that loads the library keeps until exit. At most 33,554,432 nodes
 *    (n_elems * (N+1)^3) fit; larger problems return DG_ERR_UNSUPPORTED before any launch.
 *    Bad arguments return DG_ERR_ARG, launch failures DG_ERR_CUDA.
 *  - The first call on each device looks up the array's device address (with that device
 *    current); make that first call before any stream capture.
 *  - All calls share the array and it keeps the last call's partial sums; calls whose kernels
 *    overlap on the GPU (different streams, several host threads) race on it -- serialise them. */
dg_status dg_invariants_noalloc(int N, int n_elems, double gamma, const double *U, const double *Ut,
                                const double *J, double *out8, void *cuda_stream);

/* ---- Discrete adjoint (vector-Jacobian products). The paper's solver (Sec. 2) is an explicit
 * method of lines U' = L(U); these calls give the exact transposed derivatives of the discrete
 * operator this library applies, for gradient-based use (optimisation, sensitivities, training).
 * Supported: FP64 (DG_FP64), no shock capturing, volume flux DG_VFLUX_KG or DG_VFLUX_PIROZZOLI, any
 * surface flux, Euler or Navier-Stokes. Anything else returns DG_ERR_UNSUPPORTED before any
 * launch. The Roe and LLF fluxes contain |.| and max: where an argument is exactly zero (or two are
 * equal) the one-sided derivative of the branch the forward kernel takes is used.
 * Work buffers are library-owned; the state buffers of the LSERK adjoints are allocated on first
 * use (DG_ERR_OOM if that fails) and kept until dg_free. For Navier-Stokes every product is taken at
 * the viscous stress that the forward lifting forms at the same state: the calls below that
 * recompute stage states keep that record beside each (6 doubles per node), and dg_rhs_vjp runs the
 * face and lifting kernels at U first. All arrays are device arrays
 * [n_elems][5][n]^3 on the context stream; asynchronous unless stated. ---- */

/* (Meshes with wall faces are not supported by the adjoint: DG_ERR_UNSUPPORTED.) */

/* Ubar = (dL/dU)(U)^T lambda. Ubar must overlap neither U nor lambda. */
dg_status dg_rhs_vjp(dg_ctx *ctx, const double *U, const double *lambda, double *Ubar, double t);

/* Reverse of one LSERK(5,4) step from state U (unchanged): on entry Ubar is the cotangent of the
 * state after the step, on exit that of U. The step's four inner stage states are recomputed
 * (library-owned, 4 state buffers); the stages are then run backwards:
 * gbar = B_5 Ubar; for s = 5..1: Ubar += dt (dL/dU)(U^(s-1))^T gbar; gbar = A_s gbar + B_(s-1) Ubar. */
dg_status dg_lserk_step_vjp(dg_ctx *ctx, const double *U, double *Ubar, double dt, double t);

/* Reverse of n_steps LSERK steps from U0 (unchanged) with two-level checkpointing: a forward sweep
 * stores the state every `interval` steps (ceil(n_steps/interval) buffers); each segment is then
 * recomputed once from its checkpoint and reversed step by step. On entry Ubar is the cotangent of
 * U(n_steps), on exit that of U0. Memory: when 5 + ceil(n_steps/interval) + 5*interval state buffers
 * fit with 10% of the device memory to spare, the recomputation keeps every stage state of the
 * segment; otherwise it keeps the step start states (5 + ceil(n_steps/interval) + interval - 1
 * buffers) and each step's stages are recomputed before it is reversed. Both give identical bits.
 * Not synchronising (cudaMemGetInfo aside). */
dg_status dg_lserk_steps_vjp(dg_ctx *ctx, const double *U0, double *Ubar, double dt, double t, int n_steps,
                             int interval);

/* Budget in bytes for the buffers of dg_lserk_steps_vjp and dg_lserk_steps_record (decides whether a
 * segment's stage states, or a recording's, are kept; for Navier-Stokes each kept state also keeps
 * the lifting's viscous stress record of it, 6/5 of a state); 0 restores the default (free device
 * memory less 10% of the total). Buffers already allocated are kept. */
dg_status dg_adjoint_memory_limit(dg_ctx *ctx, double bytes);

/* The forward run recorded for a later reverse sweep (what an autograd framework does): advances U
 * by n_steps LSERK steps like dg_lserk_steps and keeps, in library buffers, every stage state (with
 * its viscous stress record for Navier-Stokes) when they fit in the adjoint's memory budget
 * (dg_adjoint_memory_limit), else the state every `interval` steps. *tape identifies the recording; a new recording invalidates the
 * previous one. */
dg_status dg_lserk_steps_record(dg_ctx *ctx, double *U, double dt, double t, int n_steps, int interval,
                                long long *tape);

/* Reverse of a recorded run: Ubar (cotangent of the final state) -> cotangent of the initial state.
 * With every stage state recorded this is 5 n_steps vector-Jacobian products and no recomputation;
 * from checkpoints, each segment is recomputed once (as dg_lserk_steps_vjp). DG_ERR_ARG if the tape
 * has been recorded over. */
dg_status dg_lserk_steps_vjp_recorded(dg_ctx *ctx, long long tape, double *Ubar);

/* *tape = the id of the recording that dg_lserk_steps_vjp_recorded accepts now, or 0 when there is
 * none (never recorded, or a recording that failed part way). Host-only query; no GPU work. A caller
 * that may have recorded over its tape checks this before the reverse sweep instead of treating an
 * error of the sweep as a stale tape. */
dg_status dg_tape_current(const dg_ctx *ctx, long long *tape);

/* grad = d/dU of the kinetic-energy integral sum J w rho|u|^2/2 (out[6] of dg_invariants). */
dg_status dg_kinetic_energy_grad(dg_ctx *ctx, const double *U, double *grad);

/* *dt = cfl * min over nodes of 2J / ((2N+1) sum_d (|u.Ja^d| + c|Ja^d|)) (synchronising). */
dg_status dg_max_dt(dg_ctx *ctx, const double *U, double cfl, double *dt);

/* DG_OK, or DG_ERR_NONPHYSICAL if any kernel since the last call met rho <= 0, p <= 0 or a
 * non-finite state, or DG_ERR_CUDA if a kernel gave up waiting for a bulk copy (bounded waits;
 * clears the flags; synchronising). */
dg_status dg_check(dg_ctx *ctx);

/* Copy the device metrics to caller device arrays Ja [n_elems][3 d][3 c][n]^3 and J [n_elems][n]^3. */
dg_status dg_get_metrics(dg_ctx *ctx, double *Ja, double *J);

/* The FP32-bulk volume operator without the blend (N = 3, 5, 7 and 16-byte aligned U, Ut, g):
 * 3 (default; N = 7, other N take mode 2): a persistent kernel whose line threads form each
 * two-point flux once for both of its nodes (pair symmetry) while separate warps apply the FP64
 * epilogue to the previous element; inputs arrive by TMA bulk copies one element ahead.
 * 2: the same pipeline with one thread per node; 1: mode 2 without warp specialisation; 0: the
 * plain node-per-thread kernel. Modes 1-3 also run the FP32 lifting as a TMA-fed persistent kernel
 * (same arithmetic, same bits as mode 0's). Modes 0-2 give identical bits; mode 3 sums in another
 * order, so it agrees with them to FP32 rounding. No effect in FP64. DG_ERR_ARG for other values. */
dg_status dg_use_tma(dg_ctx *ctx, int mode);

/* 1 (default): multi-step calls replay a CUDA graph of one step; 0: every kernel is launched. Both
 * run the same kernels and give identical bits. */
dg_status dg_use_graphs(dg_ctx *ctx, int enable);

/* Kernel timing on the context stream: when enabled, CUDA events bracket every launch and
 * per-kernel totals accumulate (ms, launches). Names: "face", "lift", "volume", "indicator",
 * "spread", "other", "adj_face", "adj_visc", "adj_volume". dg_timing_get fills up to `cap` entries and returns the count. */
dg_status dg_timing_enable(dg_ctx *ctx, int enable);
int dg_timing_get(dg_ctx *ctx, const char **names, double *ms, long long *launches, int cap);
/* total kernel launches issued by this context */
long long dg_launch_count(const dg_ctx *ctx);

void dg_free(dg_ctx *ctx);
const char *dg_last_error(const dg_ctx *ctx);
const char *dg_status_string(int status);

/* Host-only (no GPU needed): the LGL nodes xi[n], weights w[n] and derivative matrix D[n*n]
 * (D[i*n+j] = l_j'(xi_i)) this library builds its kernels' tables from. */
dg_status dg_basis(int N, double *xi, double *w, double *D);

/* Measure the GPU's FMA throughput: kind 0 = FP64, 1 = FP32. Runs a bounded FMA-chain kernel on
 * `cuda_stream` (synchronising) and returns FLOP/s in *flops. */
dg_status dg_probe_fma(int kind, void *cuda_stream, double *flops);

/* The wall model alone, for n wall points (device arrays; asynchronous on cuda_stream):
 * utau[i] = friction velocity for tangential speed U[i] at wall distance h[i] and kinematic viscosity
 * nu[i] -- the root of u+ y+(u+) = h U / nu for Spalding's y+(u+) (Sec. 3, Eq. (2)), by Newton from
 * min(sqrt(h U / nu), 60), at most 100 iterations -- with U first mapped by the van Driest transform
 * (Eq. (5)) when van_driest != 0. iters (nullable) receives the Newton iterations per point. */
dg_status dg_wall_model(int n, const double *U, const double *h, const double *nu, double uinf, double mainf,
                        double gamma, double Pr, int van_driest, double *utau, int *iters, void *cuda_stream);

/* Self-check of the library's integer-pipe float<->double conversions (used by the FP32-bulk
 * epilogue) against the GPU's own conversions on `count` counter-generated bit patterns per
 * direction, special values included. mismatches[0]: float->double, mismatches[1]: double->float
 * (round to nearest even); by design float subnormals and doubles below 2^-126 in magnitude
 * convert to zero and are not counted. Synchronising. */
dg_status dg_check_conversions(void *cuda_stream, long long count, long long mismatches[2]);

#ifdef __cplusplus
}
#endif
#endif
