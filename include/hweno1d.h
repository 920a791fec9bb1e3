/*
 * hweno1d.h - C ABI of the B300 (sm_103a) one-dimensional HWENO-GR / HWENO-DR solver
 * for the 1D compressible Navier-Stokes equations.
 *
 * Method: Sec. 2 of Guo, Fan and Zhao (arXiv 2608.10569).  Unknowns per cell are the
 * cell average and the scaled first moment of (rho, rho u, E); the spatial operator is
 * the semi-discrete system Eq. (2.2) (four-point Lobatto volume rule) with the PP local
 * Lax-Friedrichs flux Eq. (2.3), characteristic unified-stencil HWENO values and
 * modified moments (Eq. (2.4), Appendix A.1), the PP limiter on the four Lobatto values,
 * and viscous gradients from weak-derivative moments (HWENO-GR, Eqs. (2.6)-(2.9)) or
 * from the differentiated candidates (HWENO-DR, Eq. (2.5)).  Time stepping is SSP-RK3
 * with modified moments (Eq. (2.12)) under the time-step and restart rules of Sec. 5;
 * ghost cells follow Remark 4.1.
 *
 * Design: the problems are small (tens to thousands of cells), so one thread block
 * advances one problem through its whole time loop on the device (residuals, the step
 * rule, stage updates, admissibility tests and restarts), and many problems run as the
 * blocks of one launch.
 *
 * Conventions
 *   - State layout ("q"): contiguous double array [2][3][n]: index (m*3 + v)*n + i,
 *     m 0 the cell average and 1 the scaled first moment, v in {rho, rho*u, E}.
 *   - q, rhs and vhat are DEVICE pointers; the caller owns them.  Each call allocates a
 *     device workspace, enqueues its work on `stream` (a cudaStream_t as void*, NULL =
 *     legacy default stream), waits for it, and frees the workspace.
 *   - Every function returns HWENO_OK (0) or a negative HWENO_ERR_* code of hweno.h;
 *     the message of the last failure is hweno1d_last_error().
 */
#ifndef HWENO1D_H
#define HWENO1D_H

#ifdef __cplusplus
extern "C" {
#endif

#define HWENO1D_BC_PERIODIC 0   /* both sides periodic */
#define HWENO1D_BC_REFLECTIVE 1 /* stationary wall: m odd, rho and E even */
#define HWENO1D_BC_INFLOW 2     /* the prescribed state (inflow[side]), zero moments */
#define HWENO1D_BC_OUTFLOW 3    /* the adjacent interior cell's average and moment */

#define HWENO1D_SOURCE_NONE 0
#define HWENO1D_SOURCE_MMS51 1 /* Example 5.1's manufactured source S = U_t + F_x */

#define HWENO1D_MAX_CELLS 8192

typedef struct {
    int n;                  /* cells, 4 .. HWENO1D_MAX_CELLS */
    int bc[2];              /* HWENO1D_BC_* of the left and right ends */
    int scheme;             /* 0 HWENO-GR, 1 HWENO-DR */
    double x0, x1;          /* domain; dx = (x1 - x0)/n */
    double gamma, Pr, Re;
    double cfl;             /* dt = min(CFL dx / alpha*, b Re dx^2) (Sec. 5) */
    double b_visc;
    double eps_pp;          /* positivity-limiter epsilon */
    double eps_weno;        /* epsilon of the nonlinear weights */
    int max_halvings;       /* restarts with dt/2 before HWENO_ERR_INADMISSIBLE (the paper
                               sets no limit; default 60) */
    int source;             /* HWENO1D_SOURCE_* */
    double inflow[2][3];    /* conserved states of inflow ends (left, right) */
} hweno1d_config;

/* Paper defaults: gamma 1.4, Pr 0.72, Re 1000, CFL 0.6, b 0.001, eps_PP 1e-12,
 * eps_WENO 1e-8, 60 halvings, periodic ends on [0, 1]; n is left 0. */
int hweno1d_config_default(hweno1d_config* c);

/* Advance nprob independent problems from t0 to t_end (at most max_steps steps each)
 * under the step rule of Sec. 5, one thread block per problem.  q[k] is problem k's
 * state (device, [2][3][n_k]), updated in place.  out (host, 5*nprob doubles, may be
 * NULL): per problem the time reached, the steps taken, the restarts, the status (0,
 * HWENO_ERR_INADMISSIBLE when a stage stays inadmissible after max_halvings restarts,
 * HWENO_ERR_NONFINITE when a residual is not finite; the state is then the last
 * accepted one) and the limiter activations (interior cells the PP limiter acted on,
 * summed over the three stage evaluations of every accepted step: Table 5.3's count).
 * Errors: HWENO_ERR_ARG for an invalid configuration, HWENO_ERR_CUDA. */
int hweno1d_advance(const hweno1d_config* cfgs, int nprob, double* const* q, double t0, double t_end,
                    int max_steps, double* out, void* stream);

/* One SSP-RK3 step of one problem from time t: dt > 0 a trial step, dt <= 0 the rule
 * of Sec. 5.  out (host, 4 doubles, may be NULL): the step taken, the restarts, the
 * status and the limiter activations, as in hweno1d_advance. */
int hweno1d_step(const hweno1d_config* cfg, double* q, double t, double dt, double* out, void* stream);

/* One evaluation of the spatial operator at time t (the source's time): rhs [2][3][n]
 * (d/dt of the average and the moment) and, if not NULL, vhat [3][n] (the modified
 * moments of Eq. (2.4)); device buffers. */
int hweno1d_residual(const hweno1d_config* cfg, const double* q, double t, double* rhs, double* vhat,
                     void* stream);

const char* hweno1d_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* HWENO1D_H */
