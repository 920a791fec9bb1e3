/*
 * FP64 CPU ORACLE of the HWENO-GR spatial residual and SSP-RK3 step for the
 * 2D compressible Navier-Stokes equations (Guo, Fan, Zhao: "An efficient and
 * robust fifth-order HWENO scheme with gradient reconstruction for compressible
 * Navier-Stokes equations").
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may call, link or
 * load this file; only the test-suite, the smoke check and the CPU-baseline leg
 * of the benchmark use it.  It is deliberately plain and slow: one cell at a
 * time, every step in the order the paper gives it, no blocking or fusion,
 * constants from the exact-rational generator in gen_tables.py.
 *
 * Passages followed:
 *   model and fluxes ...................... Sec. 3.1, Eq. (3.1) and the flux definitions
 *   moment balances ....................... Eq. (3.2) (semi-discrete system)
 *   PP Lax-Friedrichs flux ................ Eq. (3.3)
 *   Gauss points .......................... Sec. 3.1 (three-point rule, weights 5/18, 4/9, 5/18)
 *   characteristic reconstruction ......... Sec. 3.1 (projection with left eigenvectors)
 *   nonlinear combination, moments ........ Eq. (3.4)
 *   PP limiter ............................ Sec. 3.1 (checked at face and volume points,
 *                                           only face values modified), Sec. 5 (eps_PP)
 *   face moments, weak-derivative moments . Eqs. (3.6)-(3.8)
 *   gradient reconstruction ............... Eq. (3.9), Remark 3.1
 *   HWENO-DR comparison gradients ......... Eq. (3.5) (differentiated candidates, the
 *                                           convective weights reused)
 *   HWENO candidates, weights ............. Appendix A.2, Eqs. (A.4)-(A.6)
 *   SSP-RK3 with modified moments ......... Eq. (2.12) and its 2D analogue (Sec. 3.1)
 *   time step, restart .................... Sec. 5 (CFL, b*Re*h^2, halving), Sec. 4
 *   ghost cells ........................... Remark 4.1
 *   manufactured source ................... Example 5.2 (fields, S = U_t + F_x + G_y)
 *
 * Readings where the paper is silent (also listed in the design notes):
 *   smoothness indicator  classical integral form in scaled coordinates (gen_tables.py)
 *   least squares         unit weights; exact rows as the appendix states
 *   characteristic state  eigenvectors at the cell's own average; x-system gives x-face
 *                         traces and the xi-moment, y-system the y-face traces and the
 *                         eta-moment; volume values are the mean of the two systems
 *   limiter               eps = min(eps_PP, rho_bar, p(u_bar)); density scaling first,
 *                         then the pressure root of the quadratic in t
 *   gradient inputs       face averages from limited traces, cell mean from the
 *                         unlimited volume values
 *   DR gradients          each system differentiates at its own face points; volume
 *                         points take the mean of the two systems' conservative
 *                         derivatives (as for the volume values); u, v, e follow by the
 *                         chain rule with the state the scheme holds at the point (the
 *                         limited face traces, the volume values), while the derivatives
 *                         stay those of the unlimited reconstruction
 *   LF coefficient        per face, max over 3 points x 2 sides of max(|u_n|+c, PP bound)
 *   ghost moments         mirror: normal moment takes -parity, tangential +parity
 *   inflow / outflow      inflow: the prescribed state with zero moments; outflow: the
 *                         adjacent interior cell's average and moments; corners as the x
 *                         pass then the y pass over the full padded width (a y-face
 *                         inflow fills its whole ghost row)
 *   parity unpinned:      the smoothness-indicator normalisation and the characteristic
 *                         state are not fixed by the paper; the pins hold for any choice.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include "oracle_tables.h"

#define OR_G 4 /* ghost layers: residual of cell i depends on states i-4..i+4 */

enum { OR_BC_PERIODIC = 0, OR_BC_NOSLIP = 1, OR_BC_SYMMETRY = 2, OR_BC_SLIP = 3, OR_BC_INFLOW = 4,
       OR_BC_OUTFLOW = 5 };

typedef struct {
    int nx, ny;
    double x0, x1, y0, y1;
    double gamma, Pr, Re;
    int bc[4]; /* xlo, xhi, ylo, yhi */
    double cfl, b_visc, eps_pp, eps_weno;
    int max_halvings;
    int linear_weights; /* 1: omega_m = gamma_m (used only by exactness pins) */
    int limiter;        /* 1: PP limiter active */
    int scheme;         /* viscous gradients: 0 HWENO-GR (Sec. 3.2), 1 HWENO-DR (Eq. (3.5)) */
    int source;         /* 1: Example 5.2's manufactured source added to every residual */
    int pad2_;
    double time;        /* time of a residual evaluation (the source's t) */
    /* inflow faces (Remark 4.1): per side xlo, xhi, ylo, yhi the conserved state A inside
     * the band |t - band[s][0]| < band[s][1] of the face coordinate t (y on x-faces, x on
     * y-faces; the ghost cell's centre) and B elsewhere */
    double inflow[4][2][4];
    double band[4][2];
    int linear_grad;    /* 1: linear weights in the gradient reconstruction only (ablation) */
    int pad3_;
} or_cfg;

/* linear weights of Appendix A.2 */
static const double OR_GAMMA[5] = {0.99, 0.0025, 0.0025, 0.0025, 0.0025};

static double or_gnode(int g) { return (g - 1) * sqrt(15.0) / 10.0; }
static double or_gweight(int g) { return g == 1 ? 4.0 / 9.0 : 5.0 / 18.0; }

/* 12 face points of a cell: 0-2 left x-face, 3-5 right x-face, 6-8 bottom
 * y-face, 9-11 top y-face (Gauss index along the face); 9 volume points
 * v = 3*G + H at (xi_G, eta_H). */
static void or_face_point(int k, double* xi, double* eta) {
    int side = k / 3, g = k % 3;
    if (side == 0) { *xi = -0.5; *eta = or_gnode(g); }
    else if (side == 1) { *xi = 0.5; *eta = or_gnode(g); }
    else if (side == 2) { *xi = or_gnode(g); *eta = -0.5; }
    else { *xi = or_gnode(g); *eta = 0.5; }
}
static void or_vol_point(int v, double* xi, double* eta) {
    *xi = or_gnode(v / 3);
    *eta = or_gnode(v % 3);
}

/* ------------------------------------------------------------------ */
/* ideal gas (Sec. 3.1)                                                 */
static double or_pressure(const double u[4], double g) {
    return (g - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]);
}

/* ------------------------------------------------------------------ */
/* ghost cells (Remark 4.1) as an index map on the unpadded state      */
/* q layout: [12][ny][nx], plane = 4*moment + var, moment 0=avg 1=xi 2=eta */
static void or_parity(int bc, int normal_dir, double s[4]) {
    s[0] = 1.0; s[1] = 1.0; s[2] = 1.0; s[3] = 1.0;
    if (bc == OR_BC_NOSLIP) { s[1] = -1.0; s[2] = -1.0; }
    else { /* symmetry / slip: normal velocity odd */
        if (normal_dir == 0) s[1] = -1.0; else s[2] = -1.0;
    }
}

/* the prescribed inflow state of side s for a ghost cell whose face coordinate is t */
static void or_inflow_state(const or_cfg* c, int s, double t, double out[12]) {
    int in = fabs(t - c->band[s][0]) < c->band[s][1];
    for (int v = 0; v < 4; v++) {
        out[v] = c->inflow[s][in ? 0 : 1][v];
        out[4 + v] = 0.0;
        out[8 + v] = 0.0;
    }
}

static void or_fetch(const or_cfg* c, const double* q, int i, int j, double out[12]) {
    int nx = c->nx, ny = c->ny;
    double sa[4] = {1, 1, 1, 1}, sx[4] = {1, 1, 1, 1}, sy[4] = {1, 1, 1, 1};
    int ii = i, jj = j;
    double dx = (c->x1 - c->x0) / nx, dy = (c->y1 - c->y0) / ny;
    /* a y-face inflow fills its whole ghost row, corners included */
    if (jj < 0 || jj >= ny) {
        int s = jj < 0 ? 2 : 3;
        if (c->bc[s] == OR_BC_INFLOW) {
            or_inflow_state(c, s, c->x0 + (i + 0.5) * dx, out);
            return;
        }
    }
    /* the row the y rule maps j to, with its parities */
    if (jj < 0 || jj >= ny) {
        int bc = jj < 0 ? c->bc[2] : c->bc[3];
        if (bc == OR_BC_PERIODIC) {
            jj = ((jj % ny) + ny) % ny;
        } else if (bc == OR_BC_OUTFLOW) {
            jj = jj < 0 ? 0 : ny - 1;
        } else {
            double s[4];
            or_parity(bc, 1, s);
            jj = jj < 0 ? -1 - jj : 2 * ny - 1 - jj;
            for (int v = 0; v < 4; v++) { sa[v] *= s[v]; sx[v] *= s[v]; sy[v] *= -s[v]; }
        }
    }
    if (ii < 0 || ii >= nx) {
        int bc = ii < 0 ? c->bc[0] : c->bc[1];
        if (bc == OR_BC_INFLOW) {
            double st[12];
            or_inflow_state(c, ii < 0 ? 0 : 1, c->y0 + (jj + 0.5) * dy, st);
            for (int v = 0; v < 4; v++) {
                out[v] = sa[v] * st[v];
                out[4 + v] = 0.0;
                out[8 + v] = 0.0;
            }
            return;
        }
        if (bc == OR_BC_PERIODIC) {
            ii = ((ii % nx) + nx) % nx;
        } else if (bc == OR_BC_OUTFLOW) {
            ii = ii < 0 ? 0 : nx - 1;
        } else {
            double s[4];
            or_parity(bc, 0, s);
            ii = ii < 0 ? -1 - ii : 2 * nx - 1 - ii;
            for (int v = 0; v < 4; v++) { sa[v] *= s[v]; sx[v] *= -s[v]; sy[v] *= s[v]; }
        }
    }
    size_t n = (size_t)nx * ny, at = (size_t)jj * nx + ii;
    for (int v = 0; v < 4; v++) {
        out[v] = sa[v] * q[(size_t)v * n + at];
        out[4 + v] = sx[v] * q[(size_t)(4 + v) * n + at];
        out[8 + v] = sy[v] * q[(size_t)(8 + v) * n + at];
    }
}

/* ------------------------------------------------------------------ */
/* eigenvectors of the Euler flux Jacobian in direction (nx_, ny_) in  */
/* {(1,0),(0,1)}; columns of R: u-c, u, shear, u+c                      */
static void or_eigen(const double ub[4], double g, int dir, double L[4][4], double R[4][4]) {
    double rho = ub[0];
    double u = ub[1] / rho, v = ub[2] / rho;
    double p = or_pressure(ub, g);
    double c = sqrt(g * p / rho);
    double H = (ub[3] + p) / rho;
    double q2 = u * u + v * v;
    double b1 = (g - 1.0) / (c * c), b2 = 0.5 * b1 * q2;
    /* normal / tangential velocity and the index of each momentum */
    double un = dir == 0 ? u : v, ut = dir == 0 ? v : u;
    int in = dir == 0 ? 1 : 2, it = dir == 0 ? 2 : 1;
    memset(L, 0, sizeof(double) * 16);
    memset(R, 0, sizeof(double) * 16);
    /* right eigenvectors */
    R[0][0] = 1.0; R[in][0] = un - c; R[it][0] = ut; R[3][0] = H - un * c;
    R[0][1] = 1.0; R[in][1] = un;     R[it][1] = ut; R[3][1] = 0.5 * q2;
    R[0][2] = 0.0; R[in][2] = 0.0;    R[it][2] = 1.0; R[3][2] = ut;
    R[0][3] = 1.0; R[in][3] = un + c; R[it][3] = ut; R[3][3] = H + un * c;
    /* left eigenvectors (rows), L = R^{-1} */
    L[0][0] = 0.5 * (b2 + un / c); L[0][in] = 0.5 * (-b1 * un - 1.0 / c); L[0][it] = -0.5 * b1 * ut; L[0][3] = 0.5 * b1;
    L[1][0] = 1.0 - b2;            L[1][in] = b1 * un;                    L[1][it] = b1 * ut;         L[1][3] = -b1;
    L[2][0] = -ut;                 L[2][in] = 0.0;                        L[2][it] = 1.0;             L[2][3] = 0.0;
    L[3][0] = 0.5 * (b2 - un / c); L[3][in] = 0.5 * (-b1 * un + 1.0 / c); L[3][it] = -0.5 * b1 * ut; L[3][3] = 0.5 * b1;
}

/* ------------------------------------------------------------------ */
/* scalar unified-stencil HWENO (Appendix A.2)                          */
typedef struct {
    double c0[15];      /* quartic p0 */
    double cl[4][15];   /* linear p1..p4, embedded in the monomial basis */
    double omega[5];
    double beta[5];
} or_hweno;

static double or_poly(const double c[15], double xi, double eta) {
    double xp[5] = {1.0, xi, xi * xi, xi * xi * xi, xi * xi * xi * xi};
    double yp[5] = {1.0, eta, eta * eta, eta * eta * eta, eta * eta * eta * eta};
    double s = 0.0;
    for (int k = 0; k < 15; k++) s += c[k] * xp[OR_MONO_P[k]] * yp[OR_MONO_Q[k]];
    return s;
}

/* cell offsets of labels 1..9 (row-major from (i-1,j-1)) */
static void or_label_off(int k, int* a, int* b) {
    *a = (k - 1) % 3 - 1;
    *b = (k - 1) / 3 - 1;
}

/* linear candidate through the averages of three stencil cells: the average of
 * c0 + c1 xi + c2 eta over cell (a,b) is c0 + c1 a + c2 b; solved by Cramer. */
static void or_linear_candidate(const double d17[17], const int lab[3], double cl[15]) {
    double A[3][3], r[3];
    for (int t = 0; t < 3; t++) {
        int a, b;
        or_label_off(lab[t], &a, &b);
        A[t][0] = 1.0; A[t][1] = a; A[t][2] = b;
        r[t] = d17[lab[t] - 1];
    }
    double det = A[0][0] * (A[1][1] * A[2][2] - A[1][2] * A[2][1])
               - A[0][1] * (A[1][0] * A[2][2] - A[1][2] * A[2][0])
               + A[0][2] * (A[1][0] * A[2][1] - A[1][1] * A[2][0]);
    double x[3];
    for (int col = 0; col < 3; col++) {
        double M[3][3];
        memcpy(M, A, sizeof(M));
        for (int t = 0; t < 3; t++) M[t][col] = r[t];
        x[col] = (M[0][0] * (M[1][1] * M[2][2] - M[1][2] * M[2][1])
                - M[0][1] * (M[1][0] * M[2][2] - M[1][2] * M[2][0])
                + M[0][2] * (M[1][0] * M[2][1] - M[1][1] * M[2][0])) / det;
    }
    memset(cl, 0, sizeof(double) * 15);
    cl[0] = x[0]; cl[1] = x[1]; cl[2] = x[2];
}

static double or_beta(const double c[15]) {
    double s = 0.0;
    for (int a = 0; a < 15; a++)
        for (int b = 0; b < 15; b++) s += c[a] * OR_BETA_B[a][b] * c[b];
    return s;
}

static void or_hweno_build(const double d17[17], double eps, int linear, or_hweno* h) {
    static const int S[4][3] = {{2, 4, 5}, {2, 5, 6}, {4, 5, 8}, {5, 6, 8}};
    for (int k = 0; k < 15; k++) {
        double s = 0.0;
        for (int n = 0; n < 17; n++) s += OR_P0MAP[k][n] * d17[n];
        h->c0[k] = s;
    }
    for (int m = 0; m < 4; m++) or_linear_candidate(d17, S[m], h->cl[m]);
    h->beta[0] = or_beta(h->c0);
    for (int m = 0; m < 4; m++) h->beta[m + 1] = or_beta(h->cl[m]);
    if (linear) {
        for (int m = 0; m < 5; m++) h->omega[m] = OR_GAMMA[m];
        return;
    }
    double tsum = 0.0;
    for (int s = 1; s <= 4; s++) tsum += fabs(h->beta[0] - h->beta[s]);
    double tau = (0.25 * tsum) * (0.25 * tsum);
    double wt[5], wsum = 0.0;
    for (int m = 0; m < 5; m++) {
        wt[m] = OR_GAMMA[m] * (1.0 + tau / (h->beta[m] + eps));
        wsum += wt[m];
    }
    for (int m = 0; m < 5; m++) h->omega[m] = wt[m] / wsum;
}

/* Eq. (3.4): u = w0 (p0/g0 - sum gm/g0 pm) + sum wm pm, for the point value */
static double or_hweno_eval(const or_hweno* h, double xi, double eta) {
    double p0 = or_poly(h->c0, xi, eta);
    double inner = p0 / OR_GAMMA[0], outer = 0.0;
    for (int m = 0; m < 4; m++) {
        double pm = or_poly(h->cl[m], xi, eta);
        inner -= OR_GAMMA[m + 1] / OR_GAMMA[0] * pm;
        outer += h->omega[m + 1] * pm;
    }
    return h->omega[0] * inner + outer;
}

/* same combination applied to the centre-cell moments of the candidates */
static double or_hweno_moment(const or_hweno* h, const double mom[15]) {
    double m0 = 0.0;
    for (int k = 0; k < 15; k++) m0 += h->c0[k] * mom[k];
    double inner = m0 / OR_GAMMA[0], outer = 0.0;
    for (int m = 0; m < 4; m++) {
        double pm = 0.0;
        for (int k = 0; k < 15; k++) pm += h->cl[m][k] * mom[k];
        inner -= OR_GAMMA[m + 1] / OR_GAMMA[0] * pm;
        outer += h->omega[m + 1] * pm;
    }
    return h->omega[0] * inner + outer;
}

/* derivative of a quartic in the scaled coordinate xi (axis 0) or eta (axis 1),
 * monomial by monomial: d/dxi xi^p eta^q = p xi^(p-1) eta^q */
static double or_poly_d(const double c[15], int axis, double xi, double eta) {
    double s = 0.0;
    for (int k = 0; k < 15; k++) {
        int p = OR_MONO_P[k], q = OR_MONO_Q[k];
        int e = axis == 0 ? p : q;
        if (e == 0) continue;
        if (axis == 0) p -= 1; else q -= 1;
        double t = e;
        for (int a = 0; a < p; a++) t *= xi;
        for (int b = 0; b < q; b++) t *= eta;
        s += c[k] * t;
    }
    return s;
}

/* HWENO-DR (Eq. (3.5)): the candidates' derivatives in the combination of Eq. (3.4),
 * with the nonlinear weights of the value reconstruction (constant over the cell):
 * w0 (p0'/g0 - sum gm/g0 pm') + sum wm pm', derivative in scaled units */
static double or_hweno_eval_d(const or_hweno* h, int axis, double xi, double eta) {
    double d0 = or_poly_d(h->c0, axis, xi, eta);
    double inner = d0 / OR_GAMMA[0], outer = 0.0;
    for (int m = 0; m < 4; m++) {
        double dm = or_poly_d(h->cl[m], axis, xi, eta);
        inner -= OR_GAMMA[m + 1] / OR_GAMMA[0] * dm;
        outer += h->omega[m + 1] * dm;
    }
    return h->omega[0] * inner + outer;
}

/* gradients (u_x, u_y, v_x, v_y, e_x, e_y) of the dissipative variables from a
 * conservative state s and its physical derivatives sx, sy, by the chain rule of
 * u = m/rho, v = n/rho, e = E/rho - (u^2 + v^2)/2 */
static void or_dissip_grad(const double s[4], const double sx[4], const double sy[4], double g[6]) {
    double rho = s[0], u = s[1] / rho, v = s[2] / rho, en = s[3] / rho;
    for (int l = 0; l < 2; l++) {
        const double* D = l == 0 ? sx : sy;
        double ud = (D[1] - u * D[0]) / rho;
        double vd = (D[2] - v * D[0]) / rho;
        double end = (D[3] - en * D[0]) / rho;
        g[0 + l] = ud;
        g[2 + l] = vd;
        g[4 + l] = end - (u * ud + v * vd);
    }
}

/* ------------------------------------------------------------------ */
/* padded working grid                                                  */
typedef struct {
    const or_cfg* c;
    int bx, by;        /* padded extents */
    double* Q;         /* [bx*by][12] padded state */
    double* face;      /* [bx*by][12][4] limited face traces */
    double* vol;       /* [bx*by][9][4] unlimited volume values */
    double* mom;       /* [bx*by][8] modified moments (xi: 0-3, eta: 4-7) */
    double* theta;     /* [bx*by][2] */
    int* active;       /* [bx*by] limiter activation */
    int* bad;          /* [bx*by] inadmissible cell average met */
    double* rm;        /* [bx*by][18] weak-derivative moments, 6*w + {x0,xxi,xeta,y0,yxi,yeta} */
    double* grad;      /* [bx*by][21][6] (u_x,u_y,v_x,v_y,e_x,e_y) at 12 face + 9 volume points */
    double* dcons;     /* HWENO-DR: [bx*by][21][2][4] conservative x/y derivatives there */
    double* fx;        /* [bx*by][3][4] flux at the x-face on the right of the cell */
    double* fy;        /* [bx*by][3][4] flux at the y-face on top of the cell */
    double* bfx;       /* [bx*by] LF coefficient of that x-face */
    double* bfy;
} or_work;

#define IDX(W, i, j) ((size_t)((j) + OR_G) * (W)->bx + (size_t)((i) + OR_G))

/* 17 conservative data (4 vars each) of the stencil around padded cell (i,j) */
static void or_gather17(const or_work* W, int i, int j, double d[17][4]) {
    static const int exact_xi[2] = {4, 6}, exact_eta[2] = {2, 8};
    static const int ls_xi[2] = {2, 8}, ls_eta[2] = {4, 6};
    for (int k = 1; k <= 9; k++) {
        int a, b;
        or_label_off(k, &a, &b);
        const double* s = W->Q + 12 * IDX(W, i + a, j + b);
        for (int v = 0; v < 4; v++) d[k - 1][v] = s[v];
    }
    for (int t = 0; t < 2; t++) {
        int a, b;
        or_label_off(exact_xi[t], &a, &b);
        for (int v = 0; v < 4; v++) d[9 + t][v] = W->Q[12 * IDX(W, i + a, j + b) + 4 + v];
        or_label_off(exact_eta[t], &a, &b);
        for (int v = 0; v < 4; v++) d[11 + t][v] = W->Q[12 * IDX(W, i + a, j + b) + 8 + v];
        or_label_off(ls_xi[t], &a, &b);
        for (int v = 0; v < 4; v++) d[13 + t][v] = W->Q[12 * IDX(W, i + a, j + b) + 4 + v];
        or_label_off(ls_eta[t], &a, &b);
        for (int v = 0; v < 4; v++) d[15 + t][v] = W->Q[12 * IDX(W, i + a, j + b) + 8 + v];
    }
}

/* conservative characteristic reconstruction of one cell (Sec. 3.1, Eq. (3.4)) */
static void or_cons_cell(or_work* W, int i, int j) {
    const or_cfg* c = W->c;
    size_t id = IDX(W, i, j);
    double d[17][4];
    or_gather17(W, i, j, d);
    const double* ub = W->Q + 12 * id;
    double* face = W->face + 48 * id;
    double* vol = W->vol + 36 * id;
    double volx[9][4], voly[9][4];
    /* HWENO-DR: conservative x- and y-derivatives at this system's face points and
     * at the volume points (summed over the two systems) */
    const int dr = c->scheme == 1;
    const double hx = (c->x1 - c->x0) / c->nx, hy = (c->y1 - c->y0) / c->ny;
    double dface[12][2][4], dvol[9][2][4];
    memset(dvol, 0, sizeof(dvol));
    for (int dir = 0; dir < 2; dir++) {
        double L[4][4], R[4][4];
        or_eigen(ub, c->gamma, dir, L, R);
        double chf[6][4], chv[9][4], chm[4];
        double dchf[6][2][4], dchv[9][2][4];
        for (int k = 0; k < 4; k++) {
            double d17[17];
            for (int n = 0; n < 17; n++) {
                double s = 0.0;
                for (int v = 0; v < 4; v++) s += L[k][v] * d[n][v];
                d17[n] = s;
            }
            or_hweno h;
            or_hweno_build(d17, c->eps_weno, c->linear_weights, &h);
            for (int f = 0; f < 6; f++) {
                double xi, eta;
                or_face_point(6 * dir + f, &xi, &eta);
                chf[f][k] = or_hweno_eval(&h, xi, eta);
            }
            for (int v = 0; v < 9; v++) {
                double xi, eta;
                or_vol_point(v, &xi, &eta);
                chv[v][k] = or_hweno_eval(&h, xi, eta);
            }
            chm[k] = or_hweno_moment(&h, dir == 0 ? OR_MOM_XI : OR_MOM_ETA);
            if (dr)
                for (int l = 0; l < 2; l++) {
                    double hl = l == 0 ? hx : hy;
                    for (int f = 0; f < 6; f++) {
                        double xi, eta;
                        or_face_point(6 * dir + f, &xi, &eta);
                        dchf[f][l][k] = or_hweno_eval_d(&h, l, xi, eta) / hl;
                    }
                    for (int v = 0; v < 9; v++) {
                        double xi, eta;
                        or_vol_point(v, &xi, &eta);
                        dchv[v][l][k] = or_hweno_eval_d(&h, l, xi, eta) / hl;
                    }
                }
        }
        if (dr)
            for (int v = 0; v < 4; v++)
                for (int l = 0; l < 2; l++) {
                    for (int f = 0; f < 6; f++) {
                        double s = 0.0;
                        for (int k = 0; k < 4; k++) s += R[v][k] * dchf[f][l][k];
                        dface[6 * dir + f][l][v] = s;
                    }
                    for (int p = 0; p < 9; p++) {
                        double s = 0.0;
                        for (int k = 0; k < 4; k++) s += R[v][k] * dchv[p][l][k];
                        dvol[p][l][v] += 0.5 * s;
                    }
                }
        /* transform back to conservative variables */
        for (int v = 0; v < 4; v++) {
            for (int f = 0; f < 6; f++) {
                double s = 0.0;
                for (int k = 0; k < 4; k++) s += R[v][k] * chf[f][k];
                face[4 * (6 * dir + f) + v] = s;
            }
            for (int p = 0; p < 9; p++) {
                double s = 0.0;
                for (int k = 0; k < 4; k++) s += R[v][k] * chv[p][k];
                if (dir == 0) volx[p][v] = s; else voly[p][v] = s;
            }
            double s = 0.0;
            for (int k = 0; k < 4; k++) s += R[v][k] * chm[k];
            W->mom[8 * id + 4 * dir + v] = s;
        }
    }
    for (int p = 0; p < 9; p++)
        for (int v = 0; v < 4; v++) vol[4 * p + v] = 0.5 * (volx[p][v] + voly[p][v]);
    if (dr) {
        /* the derivatives of the unlimited reconstruction: the limiter leaves them alone */
        double* dc = W->dcons + 168 * id;
        for (int k = 0; k < 12; k++)
            for (int l = 0; l < 2; l++)
                for (int v = 0; v < 4; v++) dc[8 * k + 4 * l + v] = dface[k][l][v];
        for (int p = 0; p < 9; p++)
            for (int l = 0; l < 2; l++)
                for (int v = 0; v < 4; v++) dc[8 * (12 + p) + 4 * l + v] = dvol[p][l][v];
    }
}

/* smallest t in [0,1] with p(ub + t (uq - ub)) = eps, p(uq) < eps <= p(ub).
 * (E + t dE)(rho + t drho) - |m + t dm|^2 / 2 - eps/(g-1) (rho + t drho) = 0 */
static double or_theta_root(const double ub[4], const double uq[4], double eps, double g) {
    double d[4];
    for (int v = 0; v < 4; v++) d[v] = uq[v] - ub[v];
    double e1 = eps / (g - 1.0);
    double a = d[3] * d[0] - 0.5 * (d[1] * d[1] + d[2] * d[2]);
    double b = ub[3] * d[0] + ub[0] * d[3] - (ub[1] * d[1] + ub[2] * d[2]) - e1 * d[0];
    double cc = ub[3] * ub[0] - 0.5 * (ub[1] * ub[1] + ub[2] * ub[2]) - e1 * ub[0];
    double t;
    if (fabs(a) < 1e-300) {
        t = -cc / b;
    } else {
        double disc = b * b - 4.0 * a * cc;
        if (disc < 0.0) disc = 0.0;
        double sq = sqrt(disc);
        double qq = -0.5 * (b + (b >= 0.0 ? sq : -sq));
        double r1 = qq / a, r2 = (qq != 0.0) ? cc / qq : r1;
        double lo = r1 < r2 ? r1 : r2, hi = r1 < r2 ? r2 : r1;
        t = (lo >= 0.0 && lo <= 1.0) ? lo : hi;
    }
    if (t < 0.0) t = 0.0;
    if (t > 1.0) t = 1.0;
    return t;
}

/* PP limiter (Sec. 3.1 after Eq. (3.4); Sec. 5 for eps_PP) */
static void or_limit_cell(or_work* W, int i, int j) {
    const or_cfg* c = W->c;
    size_t id = IDX(W, i, j);
    const double* ub = W->Q + 12 * id;
    double* face = W->face + 48 * id;
    const double* vol = W->vol + 36 * id;
    double g = c->gamma;
    double pb = or_pressure(ub, g);
    W->theta[2 * id] = 1.0;
    W->theta[2 * id + 1] = 1.0;
    W->active[id] = 0;
    W->bad[id] = 0;
    if (!(ub[0] > 0.0) || !(pb > 0.0)) { W->bad[id] = 1; return; }
    if (!c->limiter) return;
    double eps = c->eps_pp;
    if (ub[0] < eps) eps = ub[0];
    if (pb < eps) eps = pb;
    /* density */
    double rmin = ub[0];
    for (int k = 0; k < 12; k++) if (face[4 * k] < rmin) rmin = face[4 * k];
    for (int k = 0; k < 9; k++) if (vol[4 * k] < rmin) rmin = vol[4 * k];
    double th_r = 1.0;
    if (rmin < eps) th_r = (ub[0] - eps) / (ub[0] - rmin);
    /* pressure, with the density already rescaled */
    double th_p = 1.0;
    double pts[21][4];
    for (int k = 0; k < 21; k++) {
        const double* s = k < 12 ? face + 4 * k : vol + 4 * (k - 12);
        pts[k][0] = ub[0] + th_r * (s[0] - ub[0]);
        for (int v = 1; v < 4; v++) pts[k][v] = s[v];
        if (or_pressure(pts[k], g) < eps) {
            double t = or_theta_root(ub, pts[k], eps, g);
            if (t < th_p) th_p = t;
        }
    }
    for (int k = 0; k < 12; k++)
        for (int v = 0; v < 4; v++) face[4 * k + v] = ub[v] + th_p * (pts[k][v] - ub[v]);
    W->theta[2 * id] = th_r;
    W->theta[2 * id + 1] = th_p;
    W->active[id] = (th_r < 1.0 || th_p < 1.0);
}

/* dissipative variables u, v, e of a conservative state */
static void or_dissip(const double s[4], double w[3]) {
    w[0] = s[1] / s[0];
    w[1] = s[2] / s[0];
    w[2] = s[3] / s[0] - 0.5 * (w[0] * w[0] + w[1] * w[1]);
}

/* weak-derivative moments of one cell, Eqs. (3.6)-(3.8) */
static void or_rmom_cell(or_work* W, int i, int j, double dx, double dy) {
    size_t id = IDX(W, i, j);
    const double* fc = W->face + 48 * id;
    const double* fl = W->face + 48 * IDX(W, i - 1, j);
    const double* fr = W->face + 48 * IDX(W, i + 1, j);
    const double* fb = W->face + 48 * IDX(W, i, j - 1);
    const double* ft = W->face + 48 * IDX(W, i, j + 1);
    const double* vol = W->vol + 36 * id;
    /* cell mean of w from the volume values */
    double wbar[3] = {0, 0, 0};
    for (int G = 0; G < 3; G++)
        for (int H = 0; H < 3; H++) {
            double w[3];
            or_dissip(vol + 4 * (3 * G + H), w);
            for (int n = 0; n < 3; n++) wbar[n] += or_gweight(G) * or_gweight(H) * w[n];
        }
    /* face moments W^{x,0}, W^{x,1} on the left/right faces, W^{y,0}, W^{y,1} bottom/top */
    double Wx0[2][3] = {{0}}, Wx1[2][3] = {{0}}, Wy0[2][3] = {{0}}, Wy1[2][3] = {{0}};
    for (int g = 0; g < 3; g++) {
        double wa[3], wb[3];
        double wg = or_gweight(g), xg = or_gnode(g);
        /* left face: minus side = right trace of cell i-1, plus side = left trace of cell i */
        or_dissip(fl + 4 * (3 + g), wa); or_dissip(fc + 4 * (0 + g), wb);
        for (int n = 0; n < 3; n++) { double h = 0.5 * (wa[n] + wb[n]); Wx0[0][n] += wg * h; Wx1[0][n] += wg * h * xg; }
        or_dissip(fc + 4 * (3 + g), wa); or_dissip(fr + 4 * (0 + g), wb);
        for (int n = 0; n < 3; n++) { double h = 0.5 * (wa[n] + wb[n]); Wx0[1][n] += wg * h; Wx1[1][n] += wg * h * xg; }
        or_dissip(fb + 4 * (9 + g), wa); or_dissip(fc + 4 * (6 + g), wb);
        for (int n = 0; n < 3; n++) { double h = 0.5 * (wa[n] + wb[n]); Wy0[0][n] += wg * h; Wy1[0][n] += wg * h * xg; }
        or_dissip(fc + 4 * (9 + g), wa); or_dissip(ft + 4 * (6 + g), wb);
        for (int n = 0; n < 3; n++) { double h = 0.5 * (wa[n] + wb[n]); Wy0[1][n] += wg * h; Wy1[1][n] += wg * h * xg; }
    }
    double* r = W->rm + 18 * id;
    for (int n = 0; n < 3; n++) {
        r[6 * n + 0] = (Wx0[1][n] - Wx0[0][n]) / dx;
        r[6 * n + 1] = (0.5 * (Wx0[1][n] + Wx0[0][n]) - wbar[n]) / dx;
        r[6 * n + 2] = (Wx1[1][n] - Wx1[0][n]) / dx;
        r[6 * n + 3] = (Wy0[1][n] - Wy0[0][n]) / dy;
        r[6 * n + 4] = (Wy1[1][n] - Wy1[0][n]) / dy;
        r[6 * n + 5] = (0.5 * (Wy0[1][n] + Wy0[0][n]) - wbar[n]) / dy;
    }
}

/* gradient reconstruction of one cell (Eq. (3.9)): scalar HWENO, componentwise */
static void or_grad_cell(or_work* W, int i, int j) {
    const or_cfg* c = W->c;
    size_t id = IDX(W, i, j);
    static const int exact_xi[2] = {4, 6}, exact_eta[2] = {2, 8};
    static const int ls_xi[2] = {2, 8}, ls_eta[2] = {4, 6};
    for (int n = 0; n < 3; n++)
        for (int l = 0; l < 2; l++) {
            int o = 6 * n + 3 * l; /* r^{l,0}, r^{l,xi}, r^{l,eta} */
            double d17[17];
            for (int k = 1; k <= 9; k++) {
                int a, b;
                or_label_off(k, &a, &b);
                d17[k - 1] = W->rm[18 * IDX(W, i + a, j + b) + o];
            }
            for (int t = 0; t < 2; t++) {
                int a, b;
                or_label_off(exact_xi[t], &a, &b);
                d17[9 + t] = W->rm[18 * IDX(W, i + a, j + b) + o + 1];
                or_label_off(exact_eta[t], &a, &b);
                d17[11 + t] = W->rm[18 * IDX(W, i + a, j + b) + o + 2];
                or_label_off(ls_xi[t], &a, &b);
                d17[13 + t] = W->rm[18 * IDX(W, i + a, j + b) + o + 1];
                or_label_off(ls_eta[t], &a, &b);
                d17[15 + t] = W->rm[18 * IDX(W, i + a, j + b) + o + 2];
            }
            or_hweno h;
            or_hweno_build(d17, c->eps_weno, c->linear_weights || c->linear_grad, &h);
            for (int k = 0; k < 21; k++) {
                double xi, eta;
                if (k < 12) or_face_point(k, &xi, &eta); else or_vol_point(k - 12, &xi, &eta);
                W->grad[126 * id + 6 * k + 2 * n + l] = or_hweno_eval(&h, xi, eta);
            }
        }
}

/* HWENO-DR gradients of one cell (Eq. (3.5)): the chain rule at each point, with the
 * limited face traces and the volume values the fluxes use */
static void or_dr_grad_cell(or_work* W, int i, int j) {
    size_t id = IDX(W, i, j);
    const double* dc = W->dcons + 168 * id;
    double* gr = W->grad + 126 * id;
    for (int k = 0; k < 12; k++) or_dissip_grad(W->face + 48 * id + 4 * k, dc + 8 * k, dc + 8 * k + 4, gr + 6 * k);
    for (int p = 0; p < 9; p++)
        or_dissip_grad(W->vol + 36 * id + 4 * p, dc + 8 * (12 + p), dc + 8 * (12 + p) + 4, gr + 6 * (12 + p));
}

/* physical fluxes f (dir 0) and g (dir 1) of Sec. 3.1 */
static void or_phys_flux(const or_cfg* c, int dir, const double s[4], const double gr[6], double f[4]) {
    double g = c->gamma, Re = c->Re, Pr = c->Pr;
    double rho = s[0], u = s[1] / rho, v = s[2] / rho;
    double p = or_pressure(s, g);
    double ux = gr[0], uy = gr[1], vx = gr[2], vy = gr[3], ex = gr[4], ey = gr[5];
    double txx = 4.0 * ux / 3.0 - 2.0 * vy / 3.0;
    double txy = uy + vx;
    double tyy = 4.0 * vy / 3.0 - 2.0 * ux / 3.0;
    if (dir == 0) {
        f[0] = rho * u;
        f[1] = rho * u * u + p - txx / Re;
        f[2] = rho * u * v - txy / Re;
        f[3] = (s[3] + p) * u - (txx * u + txy * v + g * ex / Pr) / Re;
    } else {
        f[0] = rho * v;
        f[1] = rho * u * v - txy / Re;
        f[2] = rho * v * v + p - tyy / Re;
        f[3] = (s[3] + p) * v - (txy * u + tyy * v + g * ey / Pr) / Re;
    }
}

/* max(|u_n| + c, PP wave-speed bound of Eq. (3.3)) */
static double or_wave_bound(const or_cfg* c, int dir, const double s[4], const double gr[6]) {
    double g = c->gamma, Re = c->Re, Pr = c->Pr;
    double rho = s[0], u = s[1] / rho, v = s[2] / rho;
    double p = or_pressure(s, g);
    double e = p / ((g - 1.0) * rho);
    double cs = sqrt(g * p / rho);
    double ux = gr[0], uy = gr[1], vx = gr[2], vy = gr[3];
    double txx = 4.0 * ux / 3.0 - 2.0 * vy / 3.0;
    double txy = uy + vx;
    double tyy = 4.0 * vy / 3.0 - 2.0 * ux / 3.0;
    double un, q, s1, s2;
    if (dir == 0) { un = u; q = g * gr[4] / (Pr * Re); s1 = txx / Re - p; s2 = txy / Re; }
    else { un = v; q = g * gr[5] / (Pr * Re); s1 = txy / Re; s2 = tyy / Re - p; }
    double pp = fabs(un) + (sqrt(rho * rho * q * q + 2.0 * rho * rho * e * (s1 * s1 + s2 * s2)) + rho * fabs(q))
                           / (2.0 * rho * rho * e);
    double ac = fabs(un) + cs;
    return ac > pp ? ac : pp;
}

/* PP local Lax-Friedrichs flux at the x-face right of cell (i,j) (dir 0) or
 * the y-face on top of it (dir 1), Eq. (3.3) */
static void or_face_flux(or_work* W, int dir, int i, int j) {
    const or_cfg* c = W->c;
    size_t il = IDX(W, i, j), ir = dir == 0 ? IDX(W, i + 1, j) : IDX(W, i, j + 1);
    int kl = dir == 0 ? 3 : 9, kr = dir == 0 ? 0 : 6;
    double beta = 0.0;
    for (int g = 0; g < 3; g++) {
        double bl = or_wave_bound(c, dir, W->face + 48 * il + 4 * (kl + g), W->grad + 126 * il + 6 * (kl + g));
        double br = or_wave_bound(c, dir, W->face + 48 * ir + 4 * (kr + g), W->grad + 126 * ir + 6 * (kr + g));
        if (bl > beta) beta = bl;
        if (br > beta) beta = br;
    }
    double* out = (dir == 0 ? W->fx : W->fy) + 12 * il;
    for (int g = 0; g < 3; g++) {
        const double* sl = W->face + 48 * il + 4 * (kl + g);
        const double* sr = W->face + 48 * ir + 4 * (kr + g);
        double fl[4], fr[4];
        or_phys_flux(c, dir, sl, W->grad + 126 * il + 6 * (kl + g), fl);
        or_phys_flux(c, dir, sr, W->grad + 126 * ir + 6 * (kr + g), fr);
        for (int v = 0; v < 4; v++) out[4 * g + v] = 0.5 * (fl[v] + fr[v] - beta * (sr[v] - sl[v]));
    }
    if (dir == 0) W->bfx[il] = beta; else W->bfy[il] = beta;
}

/* Eq. (3.2): the three moment balances of one interior cell */
static void or_assemble_cell(or_work* W, int i, int j, double dx, double dy, double r[12]) {
    const or_cfg* c = W->c;
    size_t id = IDX(W, i, j);
    const double* fR = W->fx + 12 * id;
    const double* fL = W->fx + 12 * IDX(W, i - 1, j);
    const double* gT = W->fy + 12 * id;
    const double* gB = W->fy + 12 * IDX(W, i, j - 1);
    for (int v = 0; v < 4; v++) {
        double a = 0.0, b = 0.0;
        for (int g = 0; g < 3; g++) {
            a += or_gweight(g) * (fR[4 * g + v] - fL[4 * g + v]);
            b += or_gweight(g) * (gT[4 * g + v] - gB[4 * g + v]);
        }
        r[v] = -a / dx - b / dy;
        /* xi-moment */
        double s1 = 0.0, s2 = 0.0, s3 = 0.0;
        for (int g = 0; g < 3; g++) {
            s1 += or_gweight(g) * (fL[4 * g + v] + fR[4 * g + v]);
            s2 += or_gweight(g) * or_gnode(g) * (gT[4 * g + v] - gB[4 * g + v]);
        }
        for (int G = 0; G < 3; G++)
            for (int H = 0; H < 3; H++) {
                int p = 3 * G + H;
                double f[4];
                or_phys_flux(c, 0, W->vol + 36 * id + 4 * p, W->grad + 126 * id + 6 * (12 + p), f);
                s3 += or_gweight(G) * or_gweight(H) * f[v];
            }
        r[4 + v] = -s1 / (2.0 * dx) - s2 / dy + s3 / dx;
        /* eta-moment */
        s1 = 0.0; s2 = 0.0; s3 = 0.0;
        for (int g = 0; g < 3; g++) {
            s1 += or_gweight(g) * or_gnode(g) * (fR[4 * g + v] - fL[4 * g + v]);
            s2 += or_gweight(g) * (gB[4 * g + v] + gT[4 * g + v]);
        }
        for (int G = 0; G < 3; G++)
            for (int H = 0; H < 3; H++) {
                int p = 3 * G + H;
                double f[4];
                or_phys_flux(c, 1, W->vol + 36 * id + 4 * p, W->grad + 126 * id + 6 * (12 + p), f);
                s3 += or_gweight(G) * or_gweight(H) * f[v];
            }
        r[8 + v] = -s1 / dx - s2 / (2.0 * dy) + s3 / dy;
    }
}

/* ------------------------------------------------------------------ */
/* Example 5.2: manufactured solution and its source term              */
/* one manufactured field  base + 0.1 e^{-t} (sin(2 pi (a1 x + b1 y)) + cos(2 pi (a2 x + b2 y)))
 * with its t-, first and second space derivatives; w = 0 rho, 1 u, 2 v, 3 e */
typedef struct { double f, ft, fx, fy, fxx, fxy, fyy; } or_mfield;

static void or_mms_field(int w, double x, double y, double t, or_mfield* F) {
    static const double base[4] = {2.0, 1.0, 2.0, 2.0};
    static const double ab[4][4] = {{2, -1, -1, 2}, {-1, 1, 1, 1}, {1, 1, 1, -1}, {1, -1, 1, 1}};
    const double tp = 6.283185307179586476925286766559;
    double a1 = ab[w][0], b1 = ab[w][1], a2 = ab[w][2], b2 = ab[w][3];
    double amp = 0.1 * exp(-t);
    double p1 = tp * (a1 * x + b1 * y), p2 = tp * (a2 * x + b2 * y);
    double s1 = sin(p1), c1 = cos(p1), s2 = sin(p2), c2 = cos(p2);
    F->f = base[w] + amp * (s1 + c2);
    F->ft = -amp * (s1 + c2);
    F->fx = amp * tp * (a1 * c1 - a2 * s2);
    F->fy = amp * tp * (b1 * c1 - b2 * s2);
    F->fxx = -amp * tp * tp * (a1 * a1 * s1 + a2 * a2 * c2);
    F->fxy = -amp * tp * tp * (a1 * b1 * s1 + a2 * b2 * c2);
    F->fyy = -amp * tp * tp * (b1 * b1 * s1 + b2 * b2 * c2);
}

/* S = U_t + F_x + G_y at (x, y, t) for the manufactured fields: the equations of
 * Example 5.2 (the fluxes of Sec. 3.1), differentiated by the product and chain rules */
static void or_mms_source(const or_cfg* c, double x, double y, double t, double S[4]) {
    or_mfield R, U, V, Q;
    or_mms_field(0, x, y, t, &R);
    or_mms_field(1, x, y, t, &U);
    or_mms_field(2, x, y, t, &V);
    or_mms_field(3, x, y, t, &Q);
    double g = c->gamma, Re = c->Re, Pr = c->Pr;
    double rho = R.f, u = U.f, v = V.f, e = Q.f;
    /* momenta m = rho u, n = rho v */
    double m = rho * u, m_t = R.ft * u + rho * U.ft, m_x = R.fx * u + rho * U.fx, m_y = R.fy * u + rho * U.fy;
    double n = rho * v, n_t = R.ft * v + rho * V.ft, n_x = R.fx * v + rho * V.fx, n_y = R.fy * v + rho * V.fy;
    /* total energy E = rho (e + k), k = (u^2 + v^2)/2; pressure p = (g - 1) rho e */
    double k = 0.5 * (u * u + v * v);
    double k_t = u * U.ft + v * V.ft, k_x = u * U.fx + v * V.fx, k_y = u * U.fy + v * V.fy;
    double E = rho * (e + k);
    double E_t = R.ft * (e + k) + rho * (Q.ft + k_t);
    double E_x = R.fx * (e + k) + rho * (Q.fx + k_x);
    double E_y = R.fy * (e + k) + rho * (Q.fy + k_y);
    double p = (g - 1.0) * rho * e;
    double p_x = (g - 1.0) * (R.fx * e + rho * Q.fx), p_y = (g - 1.0) * (R.fy * e + rho * Q.fy);
    /* viscous stresses and their derivatives */
    double txx = (4.0 * U.fx - 2.0 * V.fy) / 3.0, txy = U.fy + V.fx, tyy = (4.0 * V.fy - 2.0 * U.fx) / 3.0;
    double txx_x = (4.0 * U.fxx - 2.0 * V.fxy) / 3.0, tyy_y = (4.0 * V.fyy - 2.0 * U.fxy) / 3.0;
    double txy_x = U.fxy + V.fxx, txy_y = U.fyy + V.fxy;
    /* x- and y-derivatives of the viscous energy fluxes txx u + txy v + g/Pr e_x and
     * txy u + tyy v + g/Pr e_y */
    double hx_x = txx_x * u + txx * U.fx + txy_x * v + txy * V.fx + g / Pr * Q.fxx;
    double hy_y = txy_y * u + txy * U.fy + tyy_y * v + tyy * V.fy + g / Pr * Q.fyy;
    S[0] = R.ft + m_x + n_y;
    S[1] = m_t + (m_x * u + m * U.fx) + p_x + (m_y * v + m * V.fy) - (txx_x + txy_y) / Re;
    S[2] = n_t + (n_x * u + n * U.fx) + (n_y * v + n * V.fy) + p_y - (txy_x + tyy_y) / Re;
    S[3] = E_t + (E_x + p_x) * u + (E + p) * U.fx + (E_y + p_y) * v + (E + p) * V.fy - (hx_x + hy_y) / Re;
}

/* cell average and scaled first moments of S over cell (i, j) at time t: 4-point
 * Gauss-Legendre per direction (nodes +-sqrt(3/7 -+ 2/7 sqrt(6/5)), weights
 * (18 +- sqrt(30))/36 on [-1, 1], halved onto the scaled cell [-1/2, 1/2]) */
static void or_mms_moments(const or_cfg* c, int i, int j, double t, double out[12]) {
    double dx = (c->x1 - c->x0) / c->nx, dy = (c->y1 - c->y0) / c->ny;
    double xc = c->x0 + (i + 0.5) * dx, yc = c->y0 + (j + 0.5) * dy;
    double ri = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), ro = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
    double wi = (18.0 + sqrt(30.0)) / 36.0, wo = (18.0 - sqrt(30.0)) / 36.0;
    double nd[4] = {-0.5 * ro, -0.5 * ri, 0.5 * ri, 0.5 * ro}, wt[4] = {0.5 * wo, 0.5 * wi, 0.5 * wi, 0.5 * wo};
    for (int k = 0; k < 12; k++) out[k] = 0.0;
    for (int a = 0; a < 4; a++)
        for (int b = 0; b < 4; b++) {
            double S[4];
            or_mms_source(c, xc + nd[a] * dx, yc + nd[b] * dy, t, S);
            double w = wt[a] * wt[b];
            for (int v = 0; v < 4; v++) {
                out[v] += w * S[v];
                out[4 + v] += w * nd[a] * S[v];
                out[8 + v] += w * nd[b] * S[v];
            }
        }
}

static int or_work_alloc(or_work* W, const or_cfg* c, int bx, int by) {
    memset(W, 0, sizeof(*W));
    W->c = c;
    W->bx = bx;
    W->by = by;
    size_t n = (size_t)bx * by;
    W->Q = calloc(12 * n, sizeof(double));
    W->face = calloc(48 * n, sizeof(double));
    W->vol = calloc(36 * n, sizeof(double));
    W->mom = calloc(8 * n, sizeof(double));
    W->theta = calloc(2 * n, sizeof(double));
    W->active = calloc(n, sizeof(int));
    W->bad = calloc(n, sizeof(int));
    W->rm = calloc(18 * n, sizeof(double));
    W->grad = calloc(126 * n, sizeof(double));
    W->dcons = c->scheme == 1 ? calloc(168 * n, sizeof(double)) : NULL;
    W->fx = calloc(12 * n, sizeof(double));
    W->fy = calloc(12 * n, sizeof(double));
    W->bfx = calloc(n, sizeof(double));
    W->bfy = calloc(n, sizeof(double));
    return (W->Q && W->face && W->vol && W->mom && W->theta && W->active && W->bad && W->rm &&
            W->grad && (W->dcons || c->scheme != 1) && W->fx && W->fy && W->bfx && W->bfy) ? 0 : -1;
}

static void or_work_free(or_work* W) {
    free(W->Q); free(W->face); free(W->vol); free(W->mom); free(W->theta); free(W->active);
    free(W->bad); free(W->rm); free(W->grad); free(W->dcons); free(W->fx); free(W->fy); free(W->bfx); free(W->bfy);
}

/* diagnostics written by or_residual: [0] alpha*, [1] beta_max, [2] limiter
 * activations (interior cells), [3] inadmissible cell averages met, [4] nonfinite
 * residual entries */
#define OR_NDIAG 8

/* The spatial operator on the region [ox, ox+wx) x [oy, oy+wy) of interior cells
 * (the padded work grid holds that region plus OR_G ghost layers, filled from the
 * global state through or_fetch).  rhs/vhat are written for the region only,
 * layout [12][wy][wx] and [8][wy][wx]. */
static int or_region(const or_cfg* c, const double* q, int ox, int oy, int wx, int wy,
                     double* rhs, double* vhat, double* diag, double* dump_face, double* dump_vol,
                     double* dump_rm, double* dump_grad, double* dump_theta) {
    or_work W;
    int bx = wx + 2 * OR_G, by = wy + 2 * OR_G;
    if (or_work_alloc(&W, c, bx, by)) { or_work_free(&W); return -1; }
    double dx = (c->x1 - c->x0) / c->nx, dy = (c->y1 - c->y0) / c->ny;
    for (int j = -OR_G; j < wy + OR_G; j++)
        for (int i = -OR_G; i < wx + OR_G; i++) or_fetch(c, q, ox + i, oy + j, W.Q + 12 * IDX(&W, i, j));
    /* conservative reconstruction + limiter on the region grown by 3 */
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = -3; j < wy + 3; j++)
        for (int i = -3; i < wx + 3; i++) { or_cons_cell(&W, i, j); or_limit_cell(&W, i, j); }
    if (c->scheme == 1) { /* HWENO-DR: the derivatives came with the traces */
#pragma omp parallel for schedule(dynamic, 1)
        for (int j = -1; j < wy + 1; j++)
            for (int i = -1; i < wx + 1; i++) or_dr_grad_cell(&W, i, j);
    } else {
#pragma omp parallel for schedule(dynamic, 1)
        for (int j = -2; j < wy + 2; j++)
            for (int i = -2; i < wx + 2; i++) or_rmom_cell(&W, i, j, dx, dy);
#pragma omp parallel for schedule(dynamic, 1)
        for (int j = -1; j < wy + 1; j++)
            for (int i = -1; i < wx + 1; i++) or_grad_cell(&W, i, j);
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = 0; j < wy; j++)
        for (int i = -1; i < wx; i++) or_face_flux(&W, 0, i, j);
#pragma omp parallel for schedule(dynamic, 1)
    for (int j = -1; j < wy; j++)
        for (int i = 0; i < wx; i++) or_face_flux(&W, 1, i, j);
    size_t n = (size_t)wx * wy;
    double nonfinite = 0.0;
    for (int j = 0; j < wy; j++)
        for (int i = 0; i < wx; i++) {
            double r[12];
            or_assemble_cell(&W, i, j, dx, dy, r);
            if (c->source == 1) { /* Example 5.2: dU/dt = R(U) + S */
                double sm[12];
                or_mms_moments(c, ox + i, oy + j, c->time, sm);
                for (int k = 0; k < 12; k++) r[k] += sm[k];
            }
            size_t at = (size_t)j * wx + i;
            for (int k = 0; k < 12; k++) {
                if (rhs) rhs[k * n + at] = r[k];
                if (!isfinite(r[k])) nonfinite += 1.0;
            }
            size_t id = IDX(&W, i, j);
            if (vhat)
                for (int k = 0; k < 8; k++) vhat[k * n + at] = W.mom[8 * id + k];
            if (dump_face) for (int k = 0; k < 48; k++) dump_face[k * n + at] = W.face[48 * id + k];
            if (dump_vol) for (int k = 0; k < 36; k++) dump_vol[k * n + at] = W.vol[36 * id + k];
            if (dump_rm) for (int k = 0; k < 18; k++) dump_rm[k * n + at] = W.rm[18 * id + k];
            if (dump_grad) for (int k = 0; k < 126; k++) dump_grad[k * n + at] = W.grad[126 * id + k];
            if (dump_theta) { dump_theta[at] = W.theta[2 * id]; dump_theta[n + at] = W.theta[2 * id + 1]; }
        }
    if (diag) {
        double amax = 0.0, bmax = 0.0, act = 0.0, bad = 0.0;
        for (int j = 0; j < wy; j++)
            for (int i = 0; i < wx; i++) {
                size_t id = IDX(&W, i, j);
                act += W.active[id];
                bad += W.bad[id];
            }
        /* alpha*: face-point states of the faces of the region's cells */
        for (int j = -1; j <= wy; j++)
            for (int i = -1; i <= wx; i++) {
                int inx = (j >= 0 && j < wy), iny = (i >= 0 && i < wx);
                size_t id = IDX(&W, i, j);
                for (int k = 0; k < 12; k++) {
                    int side = k / 3;
                    /* points on a face of an interior cell */
                    int use = 0;
                    if (inx && side == 1 && i >= -1 && i < wx) use = 1;
                    if (inx && side == 0 && i >= 0 && i <= wx) use = 1;
                    if (iny && side == 3 && j >= -1 && j < wy) use = 1;
                    if (iny && side == 2 && j >= 0 && j <= wy) use = 1;
                    if (!use) continue;
                    const double* s = W.face + 48 * id + 4 * k;
                    double p = or_pressure(s, c->gamma);
                    double cs = sqrt(c->gamma * p / s[0]);
                    double a1 = fabs(s[1] / s[0]) + cs, a2 = fabs(s[2] / s[0]) + cs;
                    double a = a1 > a2 ? a1 : a2;
                    if (!(a <= amax)) amax = a;
                }
            }
        for (int j = 0; j < wy; j++)
            for (int i = -1; i < wx; i++) { double b = W.bfx[IDX(&W, i, j)]; if (b > bmax) bmax = b; }
        for (int j = -1; j < wy; j++)
            for (int i = 0; i < wx; i++) { double b = W.bfy[IDX(&W, i, j)]; if (b > bmax) bmax = b; }
        for (int k = 0; k < OR_NDIAG; k++) diag[k] = 0.0;
        diag[0] = amax;
        diag[1] = bmax;
        diag[2] = act;
        diag[3] = bad;
        diag[4] = nonfinite;
    }
    or_work_free(&W);
    return 0;
}

/* ================================================================== */
/* exported API (ctypes)                                                */

/* residual of the whole grid: q [12][ny][nx] -> rhs [12][ny][nx], vhat [8][ny][nx] */
int or_residual(const or_cfg* c, const double* q, double* rhs, double* vhat, double* diag,
                double* dump_face, double* dump_vol, double* dump_rm, double* dump_grad,
                double* dump_theta) {
    return or_region(c, q, 0, 0, c->nx, c->ny, rhs, vhat, diag, dump_face, dump_vol, dump_rm,
                     dump_grad, dump_theta);
}

/* residual of selected cells only (sampled checks of full-size grids):
 * rhs [ncell][12], vhat [ncell][8] */
int or_residual_cells(const or_cfg* c, const double* q, int ncell, const int* ci, const int* cj,
                      double* rhs, double* vhat) {
    int err = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(| : err)
    for (int k = 0; k < ncell; k++) {
        double r[12], m[8];
        or_cfg cc = *c;
        err |= or_region(&cc, q, ci[k], cj[k], 1, 1, r, m, NULL, NULL, NULL, NULL, NULL, NULL);
        for (int t = 0; t < 12; t++) rhs[12 * k + t] = r[t];
        for (int t = 0; t < 8; t++) vhat[8 * k + t] = m[t];
    }
    return err;
}

/* admissibility of the cell averages after a stage (Sec. 5): 1 if every cell
 * has positive density and pressure */
static int or_admissible(const or_cfg* c, const double* q) {
    size_t n = (size_t)c->nx * c->ny;
    for (size_t k = 0; k < n; k++) {
        double u[4] = {q[k], q[n + k], q[2 * n + k], q[3 * n + k]};
        if (!(u[0] > 0.0) || !(or_pressure(u, c->gamma) > 0.0)) return 0;
        for (int t = 0; t < 12; t++) if (!isfinite(q[t * n + k])) return 0;
    }
    return 1;
}

/* one SSP-RK3 step with modified moments (Eq. (2.12), 2D analogue) and the
 * restart rule of Sec. 5.  q [12][ny][nx] is updated in place.  dt_fixed > 0
 * forces the trial step; otherwise dt = min(CFL h / alpha*, b Re h^2, t_end - t).
 * stats: [0] dt used, [1] rejections, [2] alpha*, [3] beta_max (stage max),
 * [4] limiter activations (sum over the 3 stages), [5] status (0 ok, -3 inadmissible,
 * -4 nonfinite). */
int or_step(const or_cfg* c, double* q, double t, double t_end, double dt_fixed, double* stats) {
    size_t n = (size_t)c->nx * c->ny;
    double *r0 = malloc(12 * n * sizeof(double)), *m0 = malloc(8 * n * sizeof(double));
    double *r = malloc(12 * n * sizeof(double)), *m = malloc(8 * n * sizeof(double));
    double *q1 = malloc(12 * n * sizeof(double)), *q2 = malloc(12 * n * sizeof(double));
    double *q3 = malloc(12 * n * sizeof(double));
    double diag[OR_NDIAG];
    int status = 0;
    for (int k = 0; k < 6; k++) stats[k] = 0.0;
    /* stage times of the SSP-RK3 step (a source term's t): t, t + dt, t + dt/2 */
    or_cfg cs = *c;
    cs.time = t;
    or_residual(&cs, q, r0, m0, diag, NULL, NULL, NULL, NULL, NULL);
    double bmax = diag[1], act = diag[2];
    stats[2] = diag[0];
    double h = (c->x1 - c->x0) / c->nx;
    double hy = (c->y1 - c->y0) / c->ny;
    if (hy < h) h = hy;
    double dt;
    if (dt_fixed > 0.0) dt = dt_fixed;
    else {
        dt = c->cfl * h / diag[0];
        double dv = c->b_visc * c->Re * h * h;
        if (dv < dt) dt = dv;
    }
    if (t + dt > t_end) dt = t_end - t;
    int rej = 0;
    for (;;) {
        int ok = 1;
        double sb = bmax, sa = act;
        /* stage 1 */
        for (size_t k = 0; k < n; k++)
            for (int v = 0; v < 4; v++) {
                q1[v * n + k] = q[v * n + k] + dt * r0[v * n + k];
                q1[(4 + v) * n + k] = m0[v * n + k] + dt * r0[(4 + v) * n + k];
                q1[(8 + v) * n + k] = m0[(4 + v) * n + k] + dt * r0[(8 + v) * n + k];
            }
        ok = or_admissible(c, q1);
        if (ok) {
            cs.time = t + dt;
            or_residual(&cs, q1, r, m, diag, NULL, NULL, NULL, NULL, NULL);
            if (diag[1] > sb) sb = diag[1];
            sa += diag[2];
            for (size_t k = 0; k < n; k++)
                for (int v = 0; v < 4; v++) {
                    q2[v * n + k] = 0.75 * q[v * n + k] + 0.25 * (q1[v * n + k] + dt * r[v * n + k]);
                    q2[(4 + v) * n + k] = 0.75 * m0[v * n + k] + 0.25 * (m[v * n + k] + dt * r[(4 + v) * n + k]);
                    q2[(8 + v) * n + k] = 0.75 * m0[(4 + v) * n + k] + 0.25 * (m[(4 + v) * n + k] + dt * r[(8 + v) * n + k]);
                }
            ok = or_admissible(c, q2);
        }
        if (ok) {
            cs.time = t + 0.5 * dt;
            or_residual(&cs, q2, r, m, diag, NULL, NULL, NULL, NULL, NULL);
            if (diag[1] > sb) sb = diag[1];
            sa += diag[2];
            for (size_t k = 0; k < n; k++)
                for (int v = 0; v < 4; v++) {
                    q3[v * n + k] = q[v * n + k] / 3.0 + 2.0 / 3.0 * (q2[v * n + k] + dt * r[v * n + k]);
                    q3[(4 + v) * n + k] = m0[v * n + k] / 3.0 + 2.0 / 3.0 * (m[v * n + k] + dt * r[(4 + v) * n + k]);
                    q3[(8 + v) * n + k] = m0[(4 + v) * n + k] / 3.0 + 2.0 / 3.0 * (m[(4 + v) * n + k] + dt * r[(8 + v) * n + k]);
                }
            ok = or_admissible(c, q3);
        }
        if (ok) {
            memcpy(q, q3, 12 * n * sizeof(double));
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

/* advance to t_end (or max_steps): stats as or_step plus [6] t reached,
 * [7] steps taken, [8] total rejections, [9] total limiter activations */
int or_advance(const or_cfg* c, double* q, double t0, double t_end, int max_steps, double* stats) {
    double t = t0, st[6];
    int steps = 0, status = 0;
    double rej = 0.0, act = 0.0;
    for (int k = 0; k < 10; k++) stats[k] = 0.0;
    while (t < t_end && steps < max_steps) {
        status = or_step(c, q, t, t_end, 0.0, st);
        if (status) break;
        t += st[0];
        steps++;
        rej += st[1];
        act += st[4];
        for (int k = 0; k < 6; k++) stats[k] = st[k];
        if (t_end - t <= 1e-14 * (t_end > 1.0 ? t_end : 1.0)) t = t_end;
    }
    stats[5] = status;
    stats[6] = t;
    stats[7] = steps;
    stats[8] = rej;
    stats[9] = act;
    return status;
}

/* ghost-filled copy of the state: out [12][ny+8][nx+8] */
int or_fill_ghosts(const or_cfg* c, const double* q, double* out) {
    int bx = c->nx + 2 * OR_G, by = c->ny + 2 * OR_G;
    size_t n = (size_t)bx * by;
    for (int j = -OR_G; j < c->ny + OR_G; j++)
        for (int i = -OR_G; i < c->nx + OR_G; i++) {
            double s[12];
            or_fetch(c, q, i, j, s);
            for (int k = 0; k < 12; k++) out[k * n + (size_t)(j + OR_G) * bx + (i + OR_G)] = s[k];
        }
    return 0;
}

/* single scalar reconstruction (unit pins): d17 -> values at the 12 face and 9
 * volume points, the two centre moments, and beta[5], omega[5] */
int or_hweno_scalar(const double* d17, double eps, int linear, double* pts21, double* mom2,
                    double* beta5, double* omega5, double* c0) {
    or_hweno h;
    or_hweno_build(d17, eps, linear, &h);
    for (int k = 0; k < 21; k++) {
        double xi, eta;
        if (k < 12) or_face_point(k, &xi, &eta); else or_vol_point(k - 12, &xi, &eta);
        pts21[k] = or_hweno_eval(&h, xi, eta);
    }
    mom2[0] = or_hweno_moment(&h, OR_MOM_XI);
    mom2[1] = or_hweno_moment(&h, OR_MOM_ETA);
    for (int m = 0; m < 5; m++) { beta5[m] = h.beta[m]; omega5[m] = h.omega[m]; }
    for (int k = 0; k < 15; k++) c0[k] = h.c0[k];
    return 0;
}

/* the HWENO-DR derivatives of one scalar reconstruction (unit pins): d17 ->
 * d/dxi and d/deta (scaled units) at the 12 face and 9 volume points */
int or_hweno_scalar_dr(const double* d17, double eps, int linear, double* dxi21, double* deta21) {
    or_hweno h;
    or_hweno_build(d17, eps, linear, &h);
    for (int k = 0; k < 21; k++) {
        double xi, eta;
        if (k < 12) or_face_point(k, &xi, &eta); else or_vol_point(k - 12, &xi, &eta);
        dxi21[k] = or_hweno_eval_d(&h, 0, xi, eta);
        deta21[k] = or_hweno_eval_d(&h, 1, xi, eta);
    }
    return 0;
}

/* Example 5.2's source at a point (unit pins): S[4] */
int or_mms_source_export(const or_cfg* c, double x, double y, double t, double* S) {
    or_mms_source(c, x, y, t, S);
    return 0;
}

/* limiter on one cell for the root pin: returns theta_p computed by the
 * quadratic route for the point uq (4) about ub (4) */
double or_theta_root_export(const double* ub, const double* uq, double eps, double g) {
    return or_theta_root(ub, uq, eps, g);
}

/* PP wave-speed bound of Eq. (3.3) at one face-point state s (conserved) with the
 * gradients gr = (u_x, u_y, v_x, v_y, e_x, e_y), for the positivity pin */
double or_wave_bound_export(const or_cfg* c, int dir, const double* s, const double* gr) {
    return or_wave_bound(c, dir, s, gr);
}

/* eigenvector pair for pins */
int or_eigen_export(const double* ub, double g, int dir, double* L, double* R) {
    double l[4][4], r[4][4];
    or_eigen(ub, g, dir, l, r);
    memcpy(L, l, sizeof(l));
    memcpy(R, r, sizeof(r));
    return 0;
}
