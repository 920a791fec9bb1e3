/*
 * hweno.h - C ABI of the B300 (sm_103a) HWENO-GR solver for the 2D compressible
 * Navier-Stokes equations.
 *
 * Method: the fifth-order finite-volume HWENO scheme with gradient reconstruction
 * of Guo, Fan and Zhao (arXiv 2608.10569).  Unknowns per cell are the cell average
 * and the two scaled first moments of the four conserved variables (Sec. 3.1); the
 * spatial operator is the semi-discrete system Eq. (3.2) with the PP local
 * Lax-Friedrichs flux Eq. (3.3), characteristic unified-stencil HWENO traces
 * (Eq. (3.4), Appendix A.2), the PP limiter on the conservative face states, and
 * viscous gradients from weak-derivative moments reconstructed by the same scalar
 * HWENO routine (Eqs. (3.6)-(3.9)).  Time stepping is SSP-RK3 with modified
 * moments (Eq. (2.12) and its 2D analogue) under the time-step and restart rules of
 * Sec. 5; boundary ghost cells follow Remark 4.1.  The paper's comparison scheme,
 * HWENO-DR, is selected per handle (hweno_config.scheme): its viscous gradients are the
 * derivatives of the characteristic candidates, combined with the nonlinear weights of
 * the convective reconstruction (Eq. (3.5)); everything else is shared.
 *
 * Conventions shared by every entry point
 *   - Every function returns int: HWENO_OK (0) or a negative HWENO_ERR_* code; the
 *     message of the last failure on a handle is hweno_last_error(h).
 *   - State layout ("q"): contiguous double array [3][4][ny][nx]: index
 *     ((m*4 + v)*ny + j)*nx + i, moment m in {0: cell average, 1: scaled
 *     xi-moment, 2: scaled eta-moment}, conserved variable v in
 *     {rho, rho*u, rho*v, E}; i runs along x, j along y.
 *   - on_device = 1: the pointer is CUDA device memory of the handle's device
 *     (for example a torch tensor's data_ptr); 0: host memory (pinned or
 *     pageable).  The caller owns every buffer it passes; the library never
 *     keeps a caller pointer after the call returns.
 *   - The library owns all its device memory, allocated in hweno_init and
 *     released in hweno_destroy; no other call allocates.
 *   - All device work runs on the stream given to hweno_init.  Calls that take
 *     host buffers or return host values synchronise that stream before they
 *     return; hweno_step/hweno_advance synchronise once per time step (to read
 *     the admissibility flag and the time step).
 *   - A handle is not thread-safe; use one handle per host thread.
 */
#ifndef HWENO_H
#define HWENO_H

#ifdef __cplusplus
extern "C" {
#endif

#define HWENO_OK 0
#define HWENO_ERR_ARG (-1)          /* invalid argument or configuration */
#define HWENO_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define HWENO_ERR_INADMISSIBLE (-3) /* a stage stayed inadmissible after max_halvings */
#define HWENO_ERR_NONFINITE (-4)    /* NaN/Inf in the residual or the state */
#define HWENO_ERR_TIMEOUT (-5)      /* a bounded device wait gave up */
#define HWENO_ERR_STATE (-6)        /* call order: e.g. stepping before set_state */

/* boundary conditions, Remark 4.1 (per side: xlo, xhi, ylo, yhi) */
#define HWENO_BC_PERIODIC 0  /* both sides of the direction must be periodic */
#define HWENO_BC_NOSLIP 1    /* stationary adiabatic no-slip wall: both momenta odd */
#define HWENO_BC_SYMMETRY 2  /* reflective parity: normal momentum odd */
#define HWENO_BC_SLIP 3      /* stationary slip wall: same parity as symmetry */
#define HWENO_BC_INFLOW 4    /* prescribed state in the ghost cells (averages from
                                hweno_config.inflow, moments 0) */
#define HWENO_BC_OUTFLOW 5   /* ghost cells copy the adjacent interior cell (average and
                                moments) */
/* Corner ghost cells: a y-face inflow fills its ghost rows across the padded width;
 * otherwise the y-face rule maps the row into the interior and the x-face rule then
 * applies to that row (mirror parities multiply; an x-face inflow state takes the
 * y mirror's parity).  Every entry point takes inflow and outflow faces; in the
 * adjoint an outflow ghost's adjoint returns to the edge cell and an inflow ghost's is
 * dropped (the prescribed state is a constant). */

/* arithmetic of the spatial operator */
#define HWENO_FP64 0  /* everything in FP64 */
#define HWENO_MIXED 1 /* reconstruction, weights and fluxes in FP32; the stored state,
                         the RK update, the positivity limiter's checks and theta
                         solve, and all reductions in FP64.  A step or residual whose
                         state has, in some cell, an internal energy below 1e-4 of the
                         total (kinetic share |m|^2 / (2 rho E) above 1 - 1e-4) runs the
                         FP64 operator instead: FP32 fluxes of E move such an internal
                         energy by more than 6e-4 of itself per stage (hweno_diag
                         counts these steps).  Handles only: the mixed cases of a
                         batch always run in FP32. */

/* viscous gradients */
#define HWENO_SCHEME_GR 0 /* weak-derivative moments through the scalar HWENO (Eqs. (3.6)-(3.9)) */
#define HWENO_SCHEME_DR 1 /* differentiated characteristic candidates with the convective
                             weights (Eq. (3.5)); fourth order; HWENO_FP64 only */

/* source terms added to the spatial operator (dU/dt = R(U) + S(t)) */
#define HWENO_SOURCE_NONE 0
#define HWENO_SOURCE_MMS52 1 /* Example 5.2's manufactured source: S = U_t + F_x + G_y of
                                its manufactured fields, for any domain, gamma, Pr and Re;
                                cell average and scaled moments by 4x4 Gauss quadrature,
                                at the handle's time (hweno_set_time) in hweno_residual and
                                at t^n, t^n + dt, t^n + dt/2 in the stages of a step */

typedef struct hweno_handle hweno_handle;

/* Problem statement (Sec. 3.1, Sec. 5).  Uniform cells dx = (x1-x0)/nx,
 * dy = (y1-y0)/ny.  Re is the Reynolds number (the inverse dimensionless
 * viscosity), Pr the Prandtl number, gamma the ratio of specific heats. */
typedef struct {
    int nx, ny;               /* cells; >= 4 each (a wall mirrors 4 ghost layers) */
    double x0, x1, y0, y1;    /* domain */
    double gamma, Pr, Re;     /* gas and flow parameters */
    int bc[4];                /* HWENO_BC_* for xlo, xhi, ylo, yhi */
    double cfl;               /* CFL number of dt = CFL h / alpha* (Sec. 5: 0.6) */
    double b_visc;            /* viscous step factor of dt <= b Re h^2 (Sec. 5: 0.001) */
    double eps_pp;            /* positivity-limiter epsilon (Sec. 5: 1e-12) */
    double eps_weno;          /* epsilon of the nonlinear weights (Appendix A: 1e-8) */
    int max_halvings;         /* restarts with dt/2 before HWENO_ERR_INADMISSIBLE (the
                                 paper sets no limit; default 60, dt down to 2^-60 of the
                                 rule's: Sedov 2D's first step needs 37) */
    int precision;            /* HWENO_FP64 or HWENO_MIXED */
    int scheme;               /* HWENO_SCHEME_GR or HWENO_SCHEME_DR (handles, and FP64
                                 batches whose cases all take DR; the adjoint and
                                 hweno_residual_noalloc take GR) */
    int source;               /* HWENO_SOURCE_NONE or HWENO_SOURCE_MMS52 (handles and
                                 batches, at each case's time; not the adjoint or
                                 hweno_residual_noalloc) */
    double inflow[4][2][4];   /* per face (xlo, xhi, ylo, yhi) with HWENO_BC_INFLOW: the
                                 conserved state (rho, rho u, rho v, E) of a ghost cell whose
                                 centre lies inside [0] or outside [1] the face's band;
                                 rho > 0 and p > 0 required; ignored on other faces */
    double band[4][2];        /* per inflow face: centre c and half width w >= 0 of the band
                                 |s - c| < w, s the ghost cell centre's coordinate along the
                                 face (y on x-faces, x on y-faces; w = 0: state [1] alone) */
    int linear_grad;          /* 1: the linear weights in the gradient reconstruction
                                 (Eq. (3.9)) only, the ablation of Remark 3.1; HWENO_SCHEME_GR
                                 handles, batches (the same for every case),
                                 hweno_residual_noalloc and the adjoint; 0 otherwise */
    int pad_;                 /* unused, 0 */
} hweno_config;

/* Diagnostics of the run so far (Sec. 5: PP-limiter percentage; Remark 3.1:
 * global maximum of the LF coefficient). */
typedef struct {
    double t;                 /* time reached */
    double dt_last;           /* last accepted time step */
    double alpha_star;        /* face max of max(|u|+c,|v|+c) at the last step's first stage */
    double beta_max;          /* max LF coefficient over the last step's stages */
    double pp_active;         /* limiter activations (cell-stages) since set_state */
    double cell_stages;       /* cell-stages evaluated since set_state (accepted steps) */
    double min_rho, min_p;    /* over cell averages of the current state */
    double totals[4];         /* domain integrals of rho, rho u, rho v, E (FP64,
                                 fixed-order deterministic sum) */
    long long steps;          /* accepted steps since set_state */
    long long rejected;       /* rejected (halved) step attempts since set_state */
    long long fp64_steps;     /* HWENO_MIXED handles: accepted steps since set_state that
                                 ran the FP64 operator because the state's largest kinetic
                                 share |m|^2 / (2 rho E) exceeded 1 - 1e-4 (internal
                                 energy below 1e-4 of the total, which FP32 fluxes of E
                                 cannot resolve); 0 for HWENO_FP64 handles */
    double max_kinetic_share; /* HWENO_MIXED handles: that share over the cells of the
                                 state after set_state or the last accepted step (1 for
                                 an inadmissible cell); 0 for HWENO_FP64 handles */
} hweno_diag;

/* Fill *cfg with the paper's defaults (Sec. 5, Appendix A): periodic boxes on
 * [0,1]^2, gamma 1.4, Pr 0.72, Re 1000, CFL 0.6, b 0.001, eps_PP 1e-12,
 * eps_WENO 1e-8, 60 halvings, FP64.  nx, ny are set to 0 and must be given. */
int hweno_config_default(hweno_config* cfg);

/* Create a solver on the current CUDA device.  stream: a cudaStream_t passed as
 * void* (NULL = the legacy default stream).  Allocates all device memory
 * (about 2.6 KB per padded cell in FP64).  Errors: HWENO_ERR_ARG for an invalid
 * configuration, HWENO_ERR_CUDA if allocation fails.  *out is NULL on error. */
int hweno_init(const hweno_config* cfg, void* stream, hweno_handle** out);

/* Release the handle and its device memory (waits for the stream). */
void hweno_destroy(hweno_handle* h);

/* Static text of the last error on h (or of the last failed hweno_init when
 * h is NULL).  Never NULL. */
const char* hweno_last_error(const hweno_handle* h);

/* Load the state q [3][4][ny][nx] (layout above) and set t.  Resets the
 * diagnostics counters.  Does not check admissibility. */
int hweno_set_state(hweno_handle* h, const double* q, int on_device);
int hweno_set_time(hweno_handle* h, double t);

/* Copy the current state out to q [3][4][ny][nx]. */
int hweno_get_state(hweno_handle* h, double* q, int on_device);

/* One evaluation of the spatial operator at the current state (Eq. (3.2)):
 * ghost fill, characteristic HWENO traces and modified moments, PP limiter,
 * weak-derivative moments, gradient HWENO, PP-LLF face fluxes, volume fluxes.
 *   rhs  [3][4][ny][nx]: d/dt of the average, xi-moment and eta-moment
 *   vhat [2][4][ny][nx]: the modified moments (xi, eta) of Eq. (3.4), or NULL
 * Updates alpha_star/beta_max in the diagnostics; does not advance time.
 * Errors: HWENO_ERR_STATE before set_state; HWENO_ERR_NONFINITE if any output is
 * not finite (outputs are still written). */
int hweno_residual(hweno_handle* h, double* rhs, double* vhat, int on_device);

/* One SSP-RK3 step with modified moments (Eq. (2.12), 2D analogue).
 *   dt > 0: trial step; dt <= 0: dt = min(CFL h / alpha*, b Re h^2) (Sec. 5).
 * A stage whose cell averages are not all of positive density and pressure
 * rejects the step and repeats it from t^n with dt/2 (Sec. 5), at most
 * max_halvings times.  *dt_used, *rejections may be NULL.
 * Errors: HWENO_ERR_INADMISSIBLE (state left at t^n), HWENO_ERR_NONFINITE. */
int hweno_step(hweno_handle* h, double dt, double* dt_used, int* rejections);

/* Step with the rule of Sec. 5 until t_end (the last step is shortened to land
 * on t_end) or max_steps steps.  *t_reached, *steps may be NULL. */
int hweno_advance(hweno_handle* h, double t_end, int max_steps, double* t_reached, int* steps);

/* Diagnostics (min_rho, min_p and totals are computed on demand). */
int hweno_get_diag(hweno_handle* h, hweno_diag* d);

/* Intermediate fields of the last hweno_residual call, for parity checks
 * against an independent implementation, copied to out as [n][ny][nx]:
 *   which 0: limited face traces, n = 48 (point k*4 + conserved variable v;
 *            points 0-2 left, 3-5 right, 6-8 bottom, 9-11 top face, Gauss order)
 *         1: unlimited volume values, n = 36 (point (3G+H)*4 + v)
 *         2: weak-derivative moments, n = 18 (6*w + {x0, x_xi, x_eta, y0, y_xi, y_eta},
 *            w in {u, v, e})
 *         3: reconstructed gradients, n = 126 (point*6 + {u_x,u_y,v_x,v_y,e_x,e_y},
 *            points 0-11 face, 12-20 volume)
 *         4: limiter factors theta_rho, theta_p, n = 2
 * Errors: HWENO_ERR_ARG for an unknown 'which'; HWENO_ERR_STATE before a residual. */
int hweno_debug_fields(hweno_handle* h, int which, double* out, int on_device);

/* Kernel timing of the residual's dominant kernel: enable = 1 records CUDA events
 * around every launch of each kernel of the spatial operator; hweno_profile_read
 * returns, for kernel index k (0 ghost, 1 conservative reconstruction, 2 face
 * moments, 3 weak moments, 4 gradient reconstruction (k_dr under HWENO_SCHEME_DR),
 * 5 face fluxes, 6 assembly, 7 RK update, 8 source term), the launches and the summed
 * device milliseconds since enabling.
 * Reading synchronises the stream. */
int hweno_profile(hweno_handle* h, int enable);
int hweno_profile_read(hweno_handle* h, int kernel, long long* launches, double* total_ms);

/* Peak arithmetic throughput of the device, measured with chains of dependent-free
 * FMAs (8 independent chains per thread, 8 blocks of 256 threads per SM, best of 3
 * launches on the handle's stream): which 0 = FP64 FMA, 1 = FP32 FMA; *tflops in
 * TFLOP/s counting an FMA as 2 flops.  The roofline denominator of the FP64 and
 * mixed residual, whose kernels are bound by these pipes, not by HBM.  Takes about
 * 0.1-0.3 s; synchronises the stream. */
int hweno_measure_peak(hweno_handle* h, int which, double* tflops);

/* Number of this library's kernel launches issued on the handle since set_state
 * (the count bench tools report as gpu_launches). */
long long hweno_launch_count(const hweno_handle* h);

/* ---- Discrete adjoint (FP64) -----------------------------------------------------
 * Hand-written vector-Jacobian products of the SSP-RK3 step of Eq. (2.12) (2D
 * analogue) with the spatial operator of Eq. (3.2): the characteristic HWENO with its
 * nonlinear weights and the derivatives of the eigenvectors with respect to the cell
 * average, the weak-derivative gradient reconstruction, the PP-LLF fluxes (the
 * Lax-Friedrichs coefficient is differentiated through the state that attains it),
 * the ghost cells, and the modified moments that re-enter every stage.  The time step
 * is frozen (a given dt), as a checkpointed rollout records it.  The positivity limiter
 * is differentiated on the branch it took: its density factor through the point of
 * minimum density, its pressure factor through the smallest root of the pressure
 * quadratic (implicit-function theorem), and eps = min(eps_PP, rho_bar, p_bar) through
 * the term that set it.  The paper has no adjoint; the derivatives are those of its
 * discrete scheme. */

/* Allocate the adjoint buffers (about 6.3 KB per padded cell); FP64 HWENO-GR handles
 * without a source term only (HWENO_ERR_ARG otherwise). */
int hweno_adjoint_init(hweno_handle* h);

/* xbar = (dR/dx)^T rbar + (dM/dx)^T mbar and *mubar = d<rbar, R>/dmu + d<mbar, M>/dmu
 * at the state x, for the residual R [3][4][ny][nx] and the modified moments M
 * [2][4][ny][nx] of hweno_residual; rbar or mbar may be NULL (zero).  Replaces the
 * handle's state with x. */
int hweno_adjoint_residual(hweno_handle* h, const double* x, const double* rbar, const double* mbar, double* xbar,
                           double* mubar, int on_device);

/* Storage for hweno_adjoint_segment and recording: the three stage states of up to
 * max_steps steps and, with keep_intermediates, the forward intermediates the reverse
 * reads (about 4.3 KB per padded cell and stage), so that the reverse recomputes nothing.  When those do
 * not fit in 80 % of the free device memory only the states are kept and every stage is
 * re-evaluated during the reverse.  Returns 1 if intermediates are kept, 0 if not.
 * Storage of at least max_steps steps that is already reserved serves again, unchanged
 * (recorded steps included), when it keeps intermediates, when none are asked for, or
 * when an earlier request for them was refused for lack of memory. */
int hweno_adjoint_reserve(hweno_handle* h, int max_steps, int keep_intermediates);

/* Recording for the adjoint.  With on != 0 (after hweno_adjoint_reserve), each step
 * hweno_step or hweno_advance accepts from now on is recorded into the next slot of the
 * reserved storage: its stage states, its intermediates if they are kept, and its step
 * size; more steps than reserved fail with HWENO_ERR_STATE.  on = 0 stops recording and
 * keeps what was recorded.  The recording costs one state copy per step. */
int hweno_adjoint_record(hweno_handle* h, int on);

/* The adjoint through the recorded steps, last to first, with their step sizes held
 * fixed: lam_start = (d q^{end} / d q^{first})^T lam_end, *mubar (may be NULL) = the
 * mu = 1/Re derivative of <lam_end, q^{end}>.  Buffers [3][4][ny][nx], host or device per
 * on_device.  Errors: HWENO_ERR_STATE with nothing recorded.  Ends recording; the
 * handle's state is unchanged. */
int hweno_adjoint_replay(hweno_handle* h, const double* lam_end, double* lam_start, double* mubar, int on_device);

/* The adjoint through a checkpoint segment: recompute the nsteps steps from q_start with
 * the step sizes dts[0..nsteps-1] (host array), keeping their stage states (and
 * intermediates), then the reverse sweep of hweno_adjoint_replay over them.  Errors:
 * HWENO_ERR_STATE without enough reserved storage, HWENO_ERR_INADMISSIBLE if a stage is
 * inadmissible at the given steps.  Replaces any
 * recording and leaves the handle without a state (call hweno_set_state before stepping
 * again). */
int hweno_adjoint_segment(hweno_handle* h, const double* q_start, int nsteps, const double* dts,
                          const double* lam_end, double* lam_start, double* mubar, int on_device);

/* lam = (d q^{n+1} / d q^n)^T lam_next for the step q^n -> q^{n+1} taken with dt, and
 * *mubar = (d q^{n+1} / d mu)^T lam_next with mu = 1/Re (the viscosity).  q: the state
 * q^n, lam_next and lam: adjoint states, all [3][4][ny][nx]; on_device as elsewhere.
 * The step's stage states are recomputed from q^n.  Replaces the handle's state with
 * q^n.  Errors: HWENO_ERR_STATE before hweno_adjoint_init, HWENO_ERR_INADMISSIBLE if a
 * stage of the forward step is inadmissible. */
int hweno_adjoint_step(hweno_handle* h, const double* q, double dt, const double* lam_next, double* lam,
                       double* mubar, int on_device);

/* ---- Batched ensembles ---------------------------------------------------------
 * Many independent problems (own grid, physics, boundaries; one common precision)
 * advanced together.  Each kernel of the spatial operator runs as one launch for all
 * cases: persistent blocks (a multiple of the SM count) walk a work list of
 * (case, tile) items; one SSP-RK3 step of the whole ensemble is a CUDA graph, captured
 * at init and replayed per step.  Each case keeps its own time step (the rule of
 * Sec. 5) and its own restarts: after a replay the flags of all cases are read back
 * (one synchronisation per step) and only the rejected cases are replayed with half
 * their step.  The method is the one of hweno_step; the paper solves one problem at a
 * time and has no counterpart of the batching itself. */
typedef struct hweno_batch hweno_batch;

/* Create ncases solvers (cfgs[0..ncases-1], as for hweno_init, all with the same
 * precision, scheme, linear_grad and max_halvings; HWENO_SCHEME_DR in
 * HWENO_FP64 only) sharing one stream; NULL stream: the batch creates its own
 * non-blocking stream (graph capture needs one).  Allocates everything.  Errors as
 * hweno_init; HWENO_ERR_ARG for cases that differ in precision, scheme, linear_grad or
 * max_halvings. */
int hweno_batch_init(const hweno_config* cfgs, int ncases, void* stream, hweno_batch** out);
void hweno_batch_destroy(hweno_batch* b);
const char* hweno_batch_last_error(const hweno_batch* b);

/* The solver of case k, for hweno_set_state / hweno_get_state / hweno_get_diag (and,
 * if wanted, hweno_step on that case alone).  Owned by the batch. */
int hweno_batch_case(hweno_batch* b, int k, hweno_handle** h);

/* nsteps SSP-RK3 steps of every case, each with its own dt = min(CFL h/alpha*, b Re h^2).
 * *rejections (may be NULL): restarted case-steps.  Errors: HWENO_ERR_STATE if a case
 * has no state, HWENO_ERR_INADMISSIBLE after max_halvings restarts of a case. */
int hweno_batch_step(hweno_batch* b, int nsteps, int* rejections);

/* Autotuner: times every batched kernel of the spatial operator for the block shapes
 * 32x4, 16x8, 64x2 and 128x1 on the current states (their tile lists differ), keeps
 * the fastest per kernel and re-captures the step graph.  chosen (6 ints, may be
 * NULL): the index of the kept shape for cons, face moments, weak moments, gradients,
 * fluxes and assembly/RK; -1 for the three gradient kinds of an HWENO-DR batch, whose
 * derivative kernel keeps its 32x2 block, and for the fluxes of a mixed batch, whose
 * flux tile kernels keep their 32x7 tiles (a mixed batch's assembly/RK index is timed
 * on its stage update), and for its three gradient kinds when it runs them in the
 * TMA-staged pass over 32x8 tiles (at most 64 cases, as a handle does).  Does not change
 * the states. */
int hweno_batch_autotune(hweno_batch* b, int* chosen);

/* Kernel launches issued by the batch (graph replays count their nodes). */
long long hweno_batch_launch_count(const hweno_batch* b);

/* The spatial operator of hweno_residual for callers that cannot allocate device
 * memory while they run: programs whose device memory belongs to another allocator
 * under a fixed budget (a framework's caching pool, a reserved arena), where an extra
 * cudaMalloc can fail or fragment that budget, and latency-bound loops that cannot
 * take cudaMalloc's implicit device-wide synchronisation.  The paper has no
 * counterpart: this is a deployment variant of the same evaluation.
 *
 * No handle: cfg describes the problem as for hweno_init (HWENO_SCHEME_GR, no source).
 * q [3][4][ny][nx] (the
 * state layout above), rhs [3][4][ny][nx] and vhat [2][4][ny][nx] (or NULL) are
 * caller-owned DEVICE buffers on the current device.  All intermediate fields live
 * in one library-static device array of about 9.9 MB that every GPU loading the
 * library holds until the process exits; the grid must satisfy
 * (ny + 8) * round_up(nx + 8, 16) <= 4096 padded cells (for example 56 x 56 or
 * 120 x 24), larger grids return HWENO_ERR_ARG with the sizes in the message.
 * The call enqueues its work on `stream` (a cudaStream_t as void*, NULL = legacy
 * default stream) and returns without waiting; it calls no cudaMalloc, cudaFree or
 * other allocating routine.  The first call on each device looks up the array's
 * device address (cudaGetSymbolAddress, with that device current); make that first
 * call before any stream capture.  Every call on a device shares the one array and
 * it keeps the previous call's contents: calls whose work overlaps on the GPU (two
 * streams, or host threads without ordering) race and corrupt each other's
 * results, so order them on one stream.  It does not report non-finite results.
 * Errors (HWENO_ERR_ARG, HWENO_ERR_CUDA) are read with hweno_last_error(NULL). */
int hweno_residual_noalloc(const hweno_config* cfg, const double* q, double* rhs, double* vhat,
                           void* stream);

#ifdef __cplusplus
}
#endif
#endif /* HWENO_H */
