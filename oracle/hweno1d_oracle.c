/*
 * FP64 CPU ORACLE of the ONE-DIMENSIONAL HWENO-GR and HWENO-DR schemes for the 1D
 * compressible Navier-Stokes equations (Sec. 2 of Guo, Fan, Zhao: "An efficient and
 * robust fifth-order HWENO scheme with gradient reconstruction for compressible
 * Navier-Stokes equations").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or load this
 * file; only the test-suite uses it.  It is deliberately plain and slow: one cell at a
 * time, every step in the order the paper gives it, small linear systems solved by
 * Gaussian elimination, polynomials as coefficient arrays with exact monomial integrals.
 *
 * Passages followed:
 *   model, flux split f = f^a - f^d, tau, q ......... Eq. (2.1) and the definitions after it
 *   moment balances, 4-point Lobatto volume rule ..... Eq. (2.2) and the points after Eq. (2.3)
 *   PP Lax-Friedrichs flux, wave-speed bound ......... Eq. (2.3)
 *   characteristic reconstruction .................... Sec. 2.1 (left eigenvectors of f^a's Jacobian)
 *   nonlinear combination, modified moment ........... Eq. (2.4)
 *   candidates p0, p1, p2 and their weights ......... Appendix A.1
 *   PP limiter ....................................... Sec. 2.1 (the four Lobatto points)
 *   HWENO-DR gradients ............................... Eq. (2.5)
 *   HWENO-GR interface averages, weak moments,
 *     gradient reconstruction ........................ Eqs. (2.6)-(2.9)
 *   SSP-RK3 with modified moments .................... Eq. (2.12)
 *   time step, restart ............................... Sec. 5
 *   ghost cells ...................................... Remark 4.1
 *   manufactured source .............................. Example 5.1
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   smoothness indicator  classical integral form in the scaled coordinate:
 *                         beta(p) = sum_{l=1..4} int_{-1/2}^{1/2} (d^l p / dxi^l)^2 dxi
 *   characteristic state  eigenvectors at the cell's own average, for all stencil data
 *   limiter               eps = min(eps_PP, rho_bar, p(u_bar)); density factor, then the
 *                         pressure root of the quadratic; all four Lobatto values rescaled
 *   GR inputs             interface averages and the Lobatto cell mean w_bar from the
 *                         limited point values
 *   DR chain rule         with the limited point values (the derivatives are those of
 *                         the unlimited reconstruction)
 *   LF coefficient        per interface, max over both traces of max(|u| + c, PP bound)
 *   ghost cells           reflective: m odd, rho and E even, the moment with the opposite
 *                         parity; inflow: the prescribed state, zero moments; outflow:
 *                         the adjacent interior cell's average and moment
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define OR1_G 4 /* ghost layers: the residual of cell i depends on cells i-4..i+4 */

enum { OR1_BC_PERIODIC = 0, OR1_BC_REFLECTIVE = 1, OR1_BC_INFLOW = 2, OR1_BC_OUTFLOW = 3 };

typedef struct {
    int n;                  /* cells */
    int bc[2];              /* left, right */
    int pad0_;
    double x0, x1;
    double gamma, Pr, Re;
    double cfl, b_visc, eps_pp, eps_weno;
    int max_halvings;
    int linear_weights;     /* 1: omega_m = gamma_m (exactness pins only) */
    int limiter;            /* 1: PP limiter active */
    int scheme;             /* 0 HWENO-GR, 1 HWENO-DR */
    int source;             /* 1: Example 5.1's manufactured source */
    int pad1_;
    double time;            /* time of a residual evaluation (the source's t) */
    double inflow[2][3];    /* conserved states of inflow ghost cells (left, right) */
} or1_cfg;

/* linear weights of Appendix A.1 */
static const double OR1_GAMMA[3] = {199.0 / 200.0, 1.0 / 400.0, 1.0 / 400.0};

/* four-point Lobatto rule on the scaled cell: nodes -1/2, -sqrt(5)/10, sqrt(5)/10, 1/2,
 * weights 1/12, 5/12, 5/12, 1/12 (Sec. 2.1) */
static double or1_lnode(int g) {
    double a = sqrt(5.0) / 10.0;
    return g == 0 ? -0.5 : (g == 1 ? -a : (g == 2 ? a : 0.5));
}
static double or1_lweight(int g) { return (g == 0 || g == 3) ? 1.0 / 12.0 : 5.0 / 12.0; }

/* ------------------------------------------------------------------ */
/* polynomials in the scaled coordinate: c[0] + c[1] xi + ... + c[4] xi^4 */

/* int_{a}^{b} xi^k dxi */
static double or1_mono_int(int k, double a, double b) {
    return (pow(b, k + 1) - pow(a, k + 1)) / (k + 1);
}

static double or1_poly(const double c[5], double xi) {
    double s = 0.0, x = 1.0;
    for (int k = 0; k < 5; k++) { s += c[k] * x; x *= xi; }
    return s;
}

static void or1_deriv(const double c[5], double d[5]) {
    for (int k = 0; k < 4; k++) d[k] = (k + 1) * c[k + 1];
    d[4] = 0.0;
}

/* int_{-1/2}^{1/2} p(xi) xi dxi */
static double or1_moment(const double c[5]) {
    double s = 0.0;
    for (int k = 0; k < 5; k++) s += c[k] * or1_mono_int(k + 1, -0.5, 0.5);
    return s;
}

/* constants of the reconstruction, computed once per process from their definitions:
 * the inverse of p0's condition matrix, and the quadratic form of the smoothness
 * indicator, beta(p) = sum over l = 1..4 of int (p^(l))^2 = c^T Q c with
 * Q[a][b] = sum_l (a)_l (b)_l int xi^(a-l) xi^(b-l) ((k)_l the falling factorial) */
static double OR1_P0INV[5][5], OR1_BETA_Q[5][5];
static int or1_tables_ready = 0;

static void or1_solve(int n, double A[5][5], double r[5], double x[5]);

static void or1_tables(void) {
    if (or1_tables_ready) return;
    const int cell[5] = {-1, 0, 1, -1, 1};
    double A[5][5];
    for (int row = 0; row < 5; row++) {
        double a = cell[row] - 0.5, b = cell[row] + 0.5;
        for (int k = 0; k < 5; k++) {
            if (row < 3) A[row][k] = or1_mono_int(k, a, b);  /* average over cell j */
            else /* first moment over cell j: int xi^k (xi - j) */
                A[row][k] = or1_mono_int(k + 1, a, b) - cell[row] * or1_mono_int(k, a, b);
        }
    }
    for (int col = 0; col < 5; col++) {
        double M[5][5], e[5] = {0, 0, 0, 0, 0}, x[5];
        memcpy(M, A, sizeof(M));
        e[col] = 1.0;
        or1_solve(5, M, e, x);
        for (int k = 0; k < 5; k++) OR1_P0INV[k][col] = x[k];
    }
    for (int a = 0; a < 5; a++)
        for (int b = 0; b < 5; b++) {
            double s = 0.0;
            for (int l = 1; l <= 4; l++) {
                if (a < l || b < l) continue;
                double fa = 1.0, fb = 1.0;
                for (int t = 0; t < l; t++) { fa *= a - t; fb *= b - t; }
                s += fa * fb * or1_mono_int(a - l + b - l, -0.5, 0.5);
            }
            OR1_BETA_Q[a][b] = s;
        }
    or1_tables_ready = 1;
}

/* classical smoothness indicator: sum over l = 1..4 of int (p^(l))^2 on the cell */
static double or1_beta(const double c[5]) {
    double s = 0.0;
    for (int a = 0; a < 5; a++)
        for (int b = 0; b < 5; b++) s += c[a] * OR1_BETA_Q[a][b] * c[b];
    return s;
}

/* solve the n x n system A x = r by Gaussian elimination with partial pivoting */
static void or1_solve(int n, double A[5][5], double r[5], double x[5]) {
    for (int c = 0; c < n; c++) {
        int p = c;
        for (int k = c + 1; k < n; k++)
            if (fabs(A[k][c]) > fabs(A[p][c])) p = k;
        if (p != c) {
            for (int k = 0; k < n; k++) { double t = A[c][k]; A[c][k] = A[p][k]; A[p][k] = t; }
            double t = r[c]; r[c] = r[p]; r[p] = t;
        }
        for (int k = c + 1; k < n; k++) {
            double f = A[k][c] / A[c][c];
            for (int m = c; m < n; m++) A[k][m] -= f * A[c][m];
            r[k] -= f * r[c];
        }
    }
    for (int c = n - 1; c >= 0; c--) {
        double s = r[c];
        for (int k = c + 1; k < n; k++) s -= A[c][k] * x[k];
        x[c] = s / A[c][c];
    }
}

/* ------------------------------------------------------------------ */
/* scalar HWENO with unified stencils (Appendix A.1).
 * d5 = (a_{i-1}, a_i, a_{i+1}, b_{i-1}, b_{i+1}): the zeroth moments of the three cells
 * and the first moments of the two neighbours, in the centre cell's scaled coordinate */
typedef struct {
    double c0[5];          /* quartic p0 */
    double c1[5], c2[5];   /* linear p1 on {i-1, i}, p2 on {i, i+1} */
    double beta[3], omega[3];
} or1_hweno;

static void or1_hweno_build(const double d5[5], double eps, int linear, or1_hweno* h) {
    /* p0: averages over cells j = -1, 0, 1 and first moments over j = -1, 1 */
    or1_tables();
    for (int k = 0; k < 5; k++) {
        double s = 0.0;
        for (int m = 0; m < 5; m++) s += OR1_P0INV[k][m] * d5[m];
        h->c0[k] = s;
    }
    /* linear candidates through two averages: the average of a + s xi over cell j is a + s j */
    memset(h->c1, 0, sizeof(h->c1));
    memset(h->c2, 0, sizeof(h->c2));
    h->c1[1] = d5[1] - d5[0];
    h->c1[0] = d5[1];
    h->c2[1] = d5[2] - d5[1];
    h->c2[0] = d5[1];
    h->beta[0] = or1_beta(h->c0);
    h->beta[1] = or1_beta(h->c1);
    h->beta[2] = or1_beta(h->c2);
    if (linear) {
        for (int m = 0; m < 3; m++) h->omega[m] = OR1_GAMMA[m];
        return;
    }
    double ts = 0.5 * (fabs(h->beta[0] - h->beta[1]) + fabs(h->beta[0] - h->beta[2]));
    double tau = ts * ts;
    double w[3], ws = 0.0;
    for (int m = 0; m < 3; m++) {
        w[m] = OR1_GAMMA[m] * (1.0 + tau / (h->beta[m] + eps));
        ws += w[m];
    }
    for (int m = 0; m < 3; m++) h->omega[m] = w[m] / ws;
}

/* the combination of Eq. (2.4) applied to values v0, v1, v2 of p0, p1, p2 (point values,
 * derivatives or moments alike) */
static double or1_combine(const or1_hweno* h, double v0, double v1, double v2) {
    double inner = v0 / OR1_GAMMA[0] - OR1_GAMMA[1] / OR1_GAMMA[0] * v1 - OR1_GAMMA[2] / OR1_GAMMA[0] * v2;
    return h->omega[0] * inner + h->omega[1] * v1 + h->omega[2] * v2;
}

static double or1_eval(const or1_hweno* h, double xi) {
    return or1_combine(h, or1_poly(h->c0, xi), or1_poly(h->c1, xi), or1_poly(h->c2, xi));
}

/* Eq. (2.5): the candidates' derivatives (scaled units) with the same weights */
static double or1_eval_d(const or1_hweno* h, double xi) {
    double d0[5], d1[5], d2[5];
    or1_deriv(h->c0, d0);
    or1_deriv(h->c1, d1);
    or1_deriv(h->c2, d2);
    return or1_combine(h, or1_poly(d0, xi), or1_poly(d1, xi), or1_poly(d2, xi));
}

static double or1_eval_moment(const or1_hweno* h) {
    return or1_combine(h, or1_moment(h->c0), or1_moment(h->c1), or1_moment(h->c2));
}

/* ------------------------------------------------------------------ */
/* gas (Sec. 2.1): u = (rho, m, E) */
static double or1_pressure(const double u[3], double g) {
    return (g - 1.0) * (u[2] - 0.5 * u[1] * u[1] / u[0]);
}

/* eigenvectors of the Jacobian of f^a at u: columns of R are the fields u - c, u, u + c */
static void or1_eigen(const double ub[3], double g, double L[3][3], double R[3][3]) {
    double rho = ub[0], u = ub[1] / rho;
    double p = or1_pressure(ub, g);
    double c = sqrt(g * p / rho);
    double H = (ub[2] + p) / rho;
    R[0][0] = 1.0;         R[0][1] = 1.0;           R[0][2] = 1.0;
    R[1][0] = u - c;       R[1][1] = u;             R[1][2] = u + c;
    R[2][0] = H - u * c;   R[2][1] = 0.5 * u * u;   R[2][2] = H + u * c;
    /* L = R^{-1} by the adjugate */
    double det = R[0][0] * (R[1][1] * R[2][2] - R[1][2] * R[2][1])
               - R[0][1] * (R[1][0] * R[2][2] - R[1][2] * R[2][0])
               + R[0][2] * (R[1][0] * R[2][1] - R[1][1] * R[2][0]);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            int r0 = (b + 1) % 3, r1 = (b + 2) % 3, c0 = (a + 1) % 3, c1 = (a + 2) % 3;
            L[a][b] = (R[r0][c0] * R[r1][c1] - R[r0][c1] * R[r1][c0]) / det;
        }
}

/* ------------------------------------------------------------------ */
/* ghost cells (Remark 4.1); q layout [6][n]: plane 3 m + v, m 0 average, 1 moment */
static void or1_fetch(const or1_cfg* c, const double* q, int i, double out[6]) {
    int n = c->n;
    if (i >= 0 && i < n) {
        for (int k = 0; k < 6; k++) out[k] = q[k * n + i];
        return;
    }
    int side = i < 0 ? 0 : 1;
    int bc = c->bc[side];
    if (bc == OR1_BC_PERIODIC) {
        int s = ((i % n) + n) % n;
        for (int k = 0; k < 6; k++) out[k] = q[k * n + s];
    } else if (bc == OR1_BC_REFLECTIVE) {
        int s = side == 0 ? -1 - i : 2 * n - 1 - i;
        const double par[3] = {1.0, -1.0, 1.0};
        for (int v = 0; v < 3; v++) {
            out[v] = par[v] * q[v * n + s];
            out[3 + v] = -par[v] * q[(3 + v) * n + s];
        }
    } else if (bc == OR1_BC_INFLOW) {
        for (int v = 0; v < 3; v++) { out[v] = c->inflow[side][v]; out[3 + v] = 0.0; }
    } else { /* outflow: the adjacent interior cell */
        int s = side == 0 ? 0 : n - 1;
        for (int k = 0; k < 6; k++) out[k] = q[k * n + s];
    }
}

/* ------------------------------------------------------------------ */
/* Example 5.1: manufactured fields rho = 2 + a sin(2 pi x), u = 1 + a cos(2 pi x),
 * e = 1 + a sin(2 pi x), a = 0.2 exp(-t), and the source S = U_t + F_x */
static void or1_mms_source(const or1_cfg* c, double x, double t, double S[3]) {
    const double tp = 6.283185307179586476925286766559;
    double a = 0.2 * exp(-t), sn = sin(tp * x), cs = cos(tp * x);
    double rho = 2.0 + a * sn, rho_t = -a * sn, rho_x = a * tp * cs;
    double u = 1.0 + a * cs, u_t = -a * cs, u_x = -a * tp * sn, u_xx = -a * tp * tp * cs;
    double e = 1.0 + a * sn, e_t = -a * sn, e_x = a * tp * cs, e_xx = -a * tp * tp * sn;
    double g = c->gamma, Re = c->Re, Pr = c->Pr;
    double m = rho * u, m_t = rho_t * u + rho * u_t, m_x = rho_x * u + rho * u_x;
    double E = rho * (e + 0.5 * u * u);
    double E_t = rho_t * (e + 0.5 * u * u) + rho * (e_t + u * u_t);
    double E_x = rho_x * (e + 0.5 * u * u) + rho * (e_x + u * u_x);
    double p = (g - 1.0) * rho * e, p_x = (g - 1.0) * (rho_x * e + rho * e_x);
    double tau = 4.0 / 3.0 * u_x / Re, tau_x = 4.0 / 3.0 * u_xx / Re;
    double q_x = -g * e_xx / (Pr * Re);
    S[0] = rho_t + m_x;
    S[1] = m_t + m_x * u + m * u_x + p_x - tau_x;
    S[2] = E_t + (E_x + p_x) * u + (E + p) * u_x - (u_x * tau + u * tau_x - q_x);
}

/* cell average and scaled first moment of S by 4-point Gauss-Legendre */
static void or1_mms_moments(const or1_cfg* c, int i, double t, double out[6]) {
    double dx = (c->x1 - c->x0) / c->n, xc = c->x0 + (i + 0.5) * dx;
    double ri = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), ro = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
    double wi = (18.0 + sqrt(30.0)) / 36.0, wo = (18.0 - sqrt(30.0)) / 36.0;
    double nd[4] = {-0.5 * ro, -0.5 * ri, 0.5 * ri, 0.5 * ro}, wt[4] = {0.5 * wo, 0.5 * wi, 0.5 * wi, 0.5 * wo};
    for (int k = 0; k < 6; k++) out[k] = 0.0;
    for (int a = 0; a < 4; a++) {
        double S[3];
        or1_mms_source(c, xc + nd[a] * dx, t, S);
        for (int v = 0; v < 3; v++) {
            out[v] += wt[a] * S[v];
            out[3 + v] += wt[a] * nd[a] * S[v];
        }
    }
}

/* ------------------------------------------------------------------ */
/* padded working line */
typedef struct {
    const or1_cfg* c;
    int nb;            /* padded length */
    double* Q;         /* [nb][6] */
    double* pts;       /* [nb][4][3] point values at the Lobatto points (limited after the limiter) */
    double* dpts;      /* [nb][4][3] HWENO-DR: conservative x-derivatives there */
    double* mom;       /* [nb][3] modified moments */
    double* theta;     /* [nb][2] */
    int* active;
    double* rw;        /* [nb][4] weak moments: 2 w + (r0, r1), w in {u, e} */
    double* grad;      /* [nb][4][2] (u_x, e_x) at the Lobatto points */
    double* flux;      /* [nb][3] numerical flux at the interface right of the cell */
    double* bf;        /* [nb] its LF coefficient */
} or1_work;

#define I1(W, i) ((size_t)((i) + OR1_G))

/* Sec. 2.1 and Eq. (2.4): characteristic reconstruction of one cell at the Lobatto
 * points, its modified moment and, for HWENO-DR, the derivatives of Eq. (2.5) */
static void or1_cons_cell(or1_work* W, int i) {
    const or1_cfg* c = W->c;
    size_t id = I1(W, i);
    const double* ub = W->Q + 6 * id;
    const double* ql = W->Q + 6 * I1(W, i - 1);
    const double* qr = W->Q + 6 * I1(W, i + 1);
    double L[3][3], R[3][3];
    or1_eigen(ub, c->gamma, L, R);
    double dx = (c->x1 - c->x0) / c->n;
    double chp[4][3], chd[4][3], chm[3];
    for (int k = 0; k < 3; k++) {
        double d5[5] = {0, 0, 0, 0, 0};
        for (int v = 0; v < 3; v++) {
            d5[0] += L[k][v] * ql[v];
            d5[1] += L[k][v] * ub[v];
            d5[2] += L[k][v] * qr[v];
            d5[3] += L[k][v] * ql[3 + v];
            d5[4] += L[k][v] * qr[3 + v];
        }
        or1_hweno h;
        or1_hweno_build(d5, c->eps_weno, c->linear_weights, &h);
        for (int g = 0; g < 4; g++) {
            chp[g][k] = or1_eval(&h, or1_lnode(g));
            chd[g][k] = or1_eval_d(&h, or1_lnode(g)) / dx;
        }
        chm[k] = or1_eval_moment(&h);
    }
    for (int v = 0; v < 3; v++) {
        for (int g = 0; g < 4; g++) {
            double s = 0.0, sd = 0.0;
            for (int k = 0; k < 3; k++) { s += R[v][k] * chp[g][k]; sd += R[v][k] * chd[g][k]; }
            W->pts[12 * id + 3 * g + v] = s;
            W->dpts[12 * id + 3 * g + v] = sd;
        }
        double s = 0.0;
        for (int k = 0; k < 3; k++) s += R[v][k] * chm[k];
        W->mom[3 * id + v] = s;
    }
}

/* smallest t in [0, 1] with p(ub + t (uq - ub)) = eps, for p(uq) < eps <= p(ub):
 * (E + t dE)(rho + t drho) - (m + t dm)^2 / 2 - eps/(g-1) (rho + t drho) = 0 */
static double or1_theta_root(const double ub[3], const double uq[3], double eps, double g) {
    double dr = uq[0] - ub[0], dm = uq[1] - ub[1], dE = uq[2] - ub[2];
    double k = eps / (g - 1.0);
    double A = dE * dr - 0.5 * dm * dm;
    double B = ub[2] * dr + dE * ub[0] - ub[1] * dm - k * dr;
    double C = ub[2] * ub[0] - 0.5 * ub[1] * ub[1] - k * ub[0];
    double t;
    if (fabs(A) < 1e-300) t = -C / B;
    else {
        double disc = B * B - 4.0 * A * C;
        if (disc < 0.0) disc = 0.0;
        double sq = sqrt(disc);
        double t1 = (-B - sq) / (2.0 * A), t2 = (-B + sq) / (2.0 * A);
        t = 2.0;
        if (t1 >= 0.0 && t1 <= 1.0) t = t1;
        if (t2 >= 0.0 && t2 <= 1.0 && t2 < t) t = t2;
        if (t > 1.0) t = 1.0;
    }
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
}

/* PP limiter (Sec. 2.1): the four Lobatto values rescaled about the cell average */
static void or1_limit_cell(or1_work* W, int i) {
    const or1_cfg* c = W->c;
    size_t id = I1(W, i);
    const double* ub = W->Q + 6 * id;
    double* pts = W->pts + 12 * id;
    double g = c->gamma;
    double pb = or1_pressure(ub, g);
    W->theta[2 * id] = 1.0;
    W->theta[2 * id + 1] = 1.0;
    W->active[id] = 0;
    if (!(ub[0] > 0.0) || !(pb > 0.0) || !c->limiter) return;
    double eps = c->eps_pp;
    if (ub[0] < eps) eps = ub[0];
    if (pb < eps) eps = pb;
    double rmin = ub[0];
    for (int k = 0; k < 4; k++) if (pts[3 * k] < rmin) rmin = pts[3 * k];
    double th_r = 1.0;
    if (rmin < eps) th_r = (ub[0] - eps) / (ub[0] - rmin);
    double th_p = 1.0, tmp[4][3];
    for (int k = 0; k < 4; k++) {
        tmp[k][0] = ub[0] + th_r * (pts[3 * k] - ub[0]);
        tmp[k][1] = pts[3 * k + 1];
        tmp[k][2] = pts[3 * k + 2];
        if (or1_pressure(tmp[k], g) < eps) {
            double t = or1_theta_root(ub, tmp[k], eps, g);
            if (t < th_p) th_p = t;
        }
    }
    for (int k = 0; k < 4; k++)
        for (int v = 0; v < 3; v++) pts[3 * k + v] = ub[v] + th_p * (tmp[k][v] - ub[v]);
    W->theta[2 * id] = th_r;
    W->theta[2 * id + 1] = th_p;
    W->active[id] = th_r < 1.0 || th_p < 1.0;
}

/* dissipative variables u, e of a conservative state */
static void or1_dissip(const double s[3], double w[2]) {
    w[0] = s[1] / s[0];
    w[1] = s[2] / s[0] - 0.5 * w[0] * w[0];
}

/* Eqs. (2.6) and (2.8): interface averages and the weak moments of w_x, w in {u, e} */
static void or1_weak_cell(or1_work* W, int i) {
    const or1_cfg* c = W->c;
    double dx = (c->x1 - c->x0) / c->n;
    size_t id = I1(W, i);
    const double* pc = W->pts + 12 * id;
    const double* pl = W->pts + 12 * I1(W, i - 1);
    const double* pr = W->pts + 12 * I1(W, i + 1);
    double wl[2], wr[2], a[2], b[2], wm[2], wbar[2] = {0.0, 0.0};
    /* left interface: the right trace of cell i-1 and the left trace of cell i */
    or1_dissip(pl + 9, a);
    or1_dissip(pc, b);
    for (int n = 0; n < 2; n++) wl[n] = 0.5 * (a[n] + b[n]);
    or1_dissip(pc + 9, a);
    or1_dissip(pr, b);
    for (int n = 0; n < 2; n++) wr[n] = 0.5 * (a[n] + b[n]);
    for (int g = 0; g < 4; g++) {
        or1_dissip(pc + 3 * g, wm);
        for (int n = 0; n < 2; n++) wbar[n] += or1_lweight(g) * wm[n];
    }
    for (int n = 0; n < 2; n++) {
        W->rw[4 * id + 2 * n] = (wr[n] - wl[n]) / dx;
        W->rw[4 * id + 2 * n + 1] = (0.5 * (wr[n] + wl[n]) - wbar[n]) / dx;
    }
}

/* Eq. (2.9): HWENO-GR gradients at the Lobatto points from the weak moments */
static void or1_grad_cell(or1_work* W, int i) {
    const or1_cfg* c = W->c;
    size_t id = I1(W, i), il = I1(W, i - 1), ir = I1(W, i + 1);
    for (int n = 0; n < 2; n++) {
        double d5[5] = {W->rw[4 * il + 2 * n], W->rw[4 * id + 2 * n], W->rw[4 * ir + 2 * n],
                        W->rw[4 * il + 2 * n + 1], W->rw[4 * ir + 2 * n + 1]};
        or1_hweno h;
        or1_hweno_build(d5, c->eps_weno, c->linear_weights, &h);
        for (int g = 0; g < 4; g++) W->grad[8 * id + 2 * g + n] = or1_eval(&h, or1_lnode(g));
    }
}

/* Eq. (2.5) then the chain rule: HWENO-DR gradients of (u, e) at the Lobatto points */
static void or1_dr_cell(or1_work* W, int i) {
    size_t id = I1(W, i);
    for (int g = 0; g < 4; g++) {
        const double* s = W->pts + 12 * id + 3 * g;
        const double* d = W->dpts + 12 * id + 3 * g;
        double u = s[1] / s[0], en = s[2] / s[0];
        double ux = (d[1] - u * d[0]) / s[0];
        double enx = (d[2] - en * d[0]) / s[0];
        W->grad[8 * id + 2 * g] = ux;
        W->grad[8 * id + 2 * g + 1] = enx - u * ux;
    }
}

/* physical flux f = f^a - f^d of Eq. (2.1), with tau = 4/3 u_x / Re, q = -g e_x/(Pr Re) */
static void or1_phys_flux(const or1_cfg* c, const double s[3], const double gr[2], double f[3]) {
    double g = c->gamma;
    double rho = s[0], u = s[1] / rho, p = or1_pressure(s, g);
    double tau = 4.0 / 3.0 * gr[0] / c->Re, q = -g * gr[1] / (c->Pr * c->Re);
    f[0] = rho * u;
    f[1] = rho * u * u + p - tau;
    f[2] = (s[2] + p) * u - (tau * u - q);
}

/* max(|u| + c, the PP wave-speed bound of Eq. (2.3)) */
static double or1_wave_bound(const or1_cfg* c, const double s[3], const double gr[2]) {
    double g = c->gamma;
    double rho = s[0], u = s[1] / rho, p = or1_pressure(s, g);
    double e = p / ((g - 1.0) * rho);
    double tau = 4.0 / 3.0 * gr[0] / c->Re, q = -g * gr[1] / (c->Pr * c->Re);
    double pp = fabs(u) + (sqrt(rho * rho * q * q + 2.0 * rho * rho * e * (tau - p) * (tau - p)) + rho * fabs(q))
                          / (2.0 * rho * rho * e);
    double ac = fabs(u) + sqrt(g * p / rho);
    return ac > pp ? ac : pp;
}

/* Eq. (2.3) at the interface right of cell i */
static void or1_face_flux(or1_work* W, int i) {
    const or1_cfg* c = W->c;
    size_t il = I1(W, i), ir = I1(W, i + 1);
    const double* sl = W->pts + 12 * il + 9;  /* right trace of cell i */
    const double* sr = W->pts + 12 * ir;      /* left trace of cell i+1 */
    const double* gl = W->grad + 8 * il + 6;
    const double* gr = W->grad + 8 * ir;
    double bl = or1_wave_bound(c, sl, gl), br = or1_wave_bound(c, sr, gr);
    double beta = bl > br ? bl : br;
    double fl[3], fr[3];
    or1_phys_flux(c, sl, gl, fl);
    or1_phys_flux(c, sr, gr, fr);
    for (int v = 0; v < 3; v++) W->flux[3 * il + v] = 0.5 * (fl[v] + fr[v] - beta * (sr[v] - sl[v]));
    W->bf[il] = beta;
}

/* ------------------------------------------------------------------ */
#define OR1_NDIAG 8

/* Eq. (2.2) on every cell: rhs [6][n] (average, moment), vhat [3][n]; diag: alpha*,
 * beta_max, limiter activations, nonfinite entries; dumps (may be NULL): pts [12][n],
 * grad [8][n], theta [2][n] */
int or1_residual(const or1_cfg* c, const double* q, double* rhs, double* vhat, double* diag, double* dump_pts,
                 double* dump_grad, double* dump_theta) {
    int n = c->n, nb = n + 2 * OR1_G;
    or1_work W;
    memset(&W, 0, sizeof(W));
    W.c = c;
    W.nb = nb;
    W.Q = calloc(6 * (size_t)nb, sizeof(double));
    W.pts = calloc(12 * (size_t)nb, sizeof(double));
    W.dpts = calloc(12 * (size_t)nb, sizeof(double));
    W.mom = calloc(3 * (size_t)nb, sizeof(double));
    W.theta = calloc(2 * (size_t)nb, sizeof(double));
    W.active = calloc((size_t)nb, sizeof(int));
    W.rw = calloc(4 * (size_t)nb, sizeof(double));
    W.grad = calloc(8 * (size_t)nb, sizeof(double));
    W.flux = calloc(3 * (size_t)nb, sizeof(double));
    W.bf = calloc((size_t)nb, sizeof(double));
    int rc = 0;
    if (!W.Q || !W.pts || !W.dpts || !W.mom || !W.theta || !W.active || !W.rw || !W.grad || !W.flux || !W.bf) {
        rc = -1;
        goto done;
    }
    double dx = (c->x1 - c->x0) / n;
    for (int i = -OR1_G; i < n + OR1_G; i++) or1_fetch(c, q, i, W.Q + 6 * I1(&W, i));
    for (int i = -3; i < n + 3; i++) { or1_cons_cell(&W, i); or1_limit_cell(&W, i); }
    if (c->scheme == 1) {
        for (int i = -1; i < n + 1; i++) or1_dr_cell(&W, i);
    } else {
        for (int i = -2; i < n + 2; i++) or1_weak_cell(&W, i);
        for (int i = -1; i < n + 1; i++) or1_grad_cell(&W, i);
    }
    for (int i = -1; i < n; i++) or1_face_flux(&W, i);
    double nonfinite = 0.0, amax = 0.0, bmax = 0.0, act = 0.0;
    for (int i = 0; i < n; i++) {
        size_t id = I1(&W, i);
        const double* fR = W.flux + 3 * id;
        const double* fL = W.flux + 3 * I1(&W, i - 1);
        double vol[3] = {0.0, 0.0, 0.0};
        for (int g = 0; g < 4; g++) {
            double f[3];
            or1_phys_flux(c, W.pts + 12 * id + 3 * g, W.grad + 8 * id + 2 * g, f);
            for (int v = 0; v < 3; v++) vol[v] += or1_lweight(g) * f[v];
        }
        double r[6];
        for (int v = 0; v < 3; v++) {
            r[v] = -(fR[v] - fL[v]) / dx;
            r[3 + v] = -(fL[v] + fR[v]) / (2.0 * dx) + vol[v] / dx;
        }
        if (c->source == 1) {
            double sm[6];
            or1_mms_moments(c, i, c->time, sm);
            for (int k = 0; k < 6; k++) r[k] += sm[k];
        }
        for (int k = 0; k < 6; k++) {
            if (rhs) rhs[k * n + i] = r[k];
            if (!isfinite(r[k])) nonfinite += 1.0;
        }
        if (vhat)
            for (int v = 0; v < 3; v++) vhat[v * n + i] = W.mom[3 * id + v];
        if (dump_pts) for (int k = 0; k < 12; k++) dump_pts[k * n + i] = W.pts[12 * id + k];
        if (dump_grad) for (int k = 0; k < 8; k++) dump_grad[k * n + i] = W.grad[8 * id + k];
        if (dump_theta) { dump_theta[i] = W.theta[2 * id]; dump_theta[n + i] = W.theta[2 * id + 1]; }
        act += W.active[id];
    }
    for (int i = -1; i <= n; i++) {
        size_t id = I1(&W, i);
        for (int g = 0; g < 4; g += 3) {
            if ((i == -1 && g == 0) || (i == n && g == 3)) continue;
            const double* s = W.pts + 12 * id + 3 * g;
            double a = fabs(s[1] / s[0]) + sqrt(c->gamma * or1_pressure(s, c->gamma) / s[0]);
            if (!(a <= amax)) amax = a;
        }
    }
    for (int i = -1; i < n; i++) if (W.bf[I1(&W, i)] > bmax) bmax = W.bf[I1(&W, i)];
    if (diag) {
        for (int k = 0; k < OR1_NDIAG; k++) diag[k] = 0.0;
        diag[0] = amax;
        diag[1] = bmax;
        diag[2] = act;
        diag[3] = nonfinite;
    }
done:
    free(W.Q); free(W.pts); free(W.dpts); free(W.mom); free(W.theta); free(W.active);
    free(W.rw); free(W.grad); free(W.flux); free(W.bf);
    return rc;
}

static int or1_admissible(const or1_cfg* c, const double* q) {
    int n = c->n;
    for (int i = 0; i < n; i++) {
        double u[3] = {q[i], q[n + i], q[2 * n + i]};
        if (!(u[0] > 0.0) || !(or1_pressure(u, c->gamma) > 0.0)) return 0;
    }
    return 1;
}

/* one SSP-RK3 step with modified moments (Eq. (2.12)) under the rule of Sec. 5;
 * stats: dt, rejections, alpha*, beta_max, limiter activations, status */
int or1_step(const or1_cfg* c, double* q, double t, double t_end, double dt_fixed, double* stats) {
    int n = c->n;
    size_t sz = 6 * (size_t)n * sizeof(double);
    double *r0 = malloc(sz), *m0 = malloc(sz / 2), *r = malloc(sz), *m = malloc(sz / 2);
    double *q1 = malloc(sz), *q2 = malloc(sz), *q3 = malloc(sz);
    double diag[OR1_NDIAG];
    int status = 0;
    for (int k = 0; k < 6; k++) stats[k] = 0.0;
    or1_cfg cs = *c;
    cs.time = t;
    or1_residual(&cs, q, r0, m0, diag, NULL, NULL, NULL);
    double bmax = diag[1], act = diag[2];
    stats[2] = diag[0];
    double h = (c->x1 - c->x0) / n, dt;
    if (dt_fixed > 0.0) dt = dt_fixed;
    else {
        dt = c->cfl * h / diag[0];
        double dv = c->b_visc * c->Re * h * h;
        if (dv < dt) dt = dv;
    }
    if (t + dt > t_end) dt = t_end - t;
    int rej = 0;
    for (;;) {
        double sb = bmax, sa = act;
        for (int i = 0; i < n; i++)
            for (int v = 0; v < 3; v++) {
                q1[v * n + i] = q[v * n + i] + dt * r0[v * n + i];
                q1[(3 + v) * n + i] = m0[v * n + i] + dt * r0[(3 + v) * n + i];
            }
        int ok = or1_admissible(c, q1);
        if (ok) {
            cs.time = t + dt;
            or1_residual(&cs, q1, r, m, diag, NULL, NULL, NULL);
            if (diag[1] > sb) sb = diag[1];
            sa += diag[2];
            for (int i = 0; i < n; i++)
                for (int v = 0; v < 3; v++) {
                    q2[v * n + i] = 0.75 * q[v * n + i] + 0.25 * (q1[v * n + i] + dt * r[v * n + i]);
                    q2[(3 + v) * n + i] = 0.75 * m0[v * n + i] + 0.25 * (m[v * n + i] + dt * r[(3 + v) * n + i]);
                }
            ok = or1_admissible(c, q2);
        }
        if (ok) {
            cs.time = t + 0.5 * dt;
            or1_residual(&cs, q2, r, m, diag, NULL, NULL, NULL);
            if (diag[1] > sb) sb = diag[1];
            sa += diag[2];
            for (int i = 0; i < n; i++)
                for (int v = 0; v < 3; v++) {
                    q3[v * n + i] = q[v * n + i] / 3.0 + 2.0 / 3.0 * (q2[v * n + i] + dt * r[v * n + i]);
                    q3[(3 + v) * n + i] = m0[v * n + i] / 3.0 + 2.0 / 3.0 * (m[v * n + i] + dt * r[(3 + v) * n + i]);
                }
            ok = or1_admissible(c, q3);
        }
        if (ok) {
            memcpy(q, q3, sz);
            stats[3] = sb;
            stats[4] = sa;
            break;
        }
        if (rej >= c->max_halvings) { status = -3; break; }
        rej++;
        dt *= 0.5;
    }
    stats[0] = dt;
    stats[1] = rej;
    stats[5] = status;
    free(r0); free(m0); free(r); free(m); free(q1); free(q2); free(q3);
    return status;
}

/* steps until t_end; stats: dt of the last step, -, -, -, limiter activations, status,
 * t reached, steps, rejections */
int or1_advance(const or1_cfg* c, double* q, double t0, double t_end, int max_steps, double* stats) {
    double t = t0, st[6] = {0.0, 0.0, 0.0, 0.0, 0.0, 0.0}, act = 0.0;
    int steps = 0, rej = 0, status = 0;
    while (t < t_end && steps < max_steps) {
        status = or1_step(c, q, t, t_end, 0.0, st);
        if (status) break;
        t += st[0];
        rej += (int)st[1];
        act += st[4];
        steps++;
        if (t_end - t <= 1e-14 * (fabs(t_end) > 1.0 ? fabs(t_end) : 1.0)) t = t_end;
    }
    for (int k = 0; k < 10; k++) stats[k] = 0.0;
    stats[0] = st[0];
    stats[4] = act;
    stats[5] = status;
    stats[6] = t;
    stats[7] = steps;
    stats[8] = rej;
    return status;
}

/* one scalar reconstruction (unit pins): d5 -> values and DR derivatives (scaled
 * units) at the 4 Lobatto points, the modified moment, beta[3], omega[3], c0[5] */
int or1_hweno_scalar(const double* d5, double eps, int linear, double* pts4, double* dpts4, double* mom,
                     double* beta3, double* omega3, double* c0) {
    or1_hweno h;
    or1_hweno_build(d5, eps, linear, &h);
    for (int g = 0; g < 4; g++) {
        pts4[g] = or1_eval(&h, or1_lnode(g));
        dpts4[g] = or1_eval_d(&h, or1_lnode(g));
    }
    *mom = or1_eval_moment(&h);
    for (int m = 0; m < 3; m++) { beta3[m] = h.beta[m]; omega3[m] = h.omega[m]; }
    for (int k = 0; k < 5; k++) c0[k] = h.c0[k];
    return 0;
}

/* Example 5.1's source at a point (unit pins) */
int or1_mms_source_export(const or1_cfg* c, double x, double t, double* S) {
    or1_mms_source(c, x, t, S);
    return 0;
}
