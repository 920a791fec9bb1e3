/*
 * FORWARD-MODE (DUAL-NUMBER) BUILD OF THE FP64 CPU ORACLE.  TEST INFRASTRUCTURE ONLY:
 * like hweno_oracle.c, nothing in the product path may call, link or load it.
 *
 * It recompiles hweno_oracle.c unchanged, with its floating-point type replaced by a
 * dual number (value, tangent).  Every statement of the oracle then also carries the
 * derivative along a chosen direction, so one evaluation gives F(q) and the exact
 * Jacobian-vector product J v = dF/dq v (plus the derivative with respect to
 * mu = 1/Re) with no difference quotient: the discrete tangent of the residual of
 * Eq. (3.2) and of the SSP-RK3 step of Eq. (2.12), to rounding.  The value parts are
 * the oracle's own results bit for bit (the same operations in the same order).
 *
 * Derivative rules at the non-smooth points the oracle passes through: |x| and the
 * comparisons act on the value part, d|x| = sign(x) dx with sign(0) = 0, and
 * d sqrt(x) = dx / (2 sqrt(x)); d sin = cos dx, d cos = -sin dx, d exp = exp dx (the
 * manufactured source, which depends on mu).  The step size of a step is an input (dt_fixed), so
 * it carries no tangent: the tangent is the one of the map q -> q^{n+1} at fixed dt.
 */
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <math.h>
#include <stdlib.h>
#include <string.h>

struct or_dual {
    double v, d;
    or_dual() = default;
    constexpr or_dual(double x) : v(x), d(0.0) {}
    constexpr or_dual(double x, double dx) : v(x), d(dx) {}
};

static inline or_dual operator+(const or_dual& a, const or_dual& b) { return or_dual(a.v + b.v, a.d + b.d); }
static inline or_dual operator-(const or_dual& a, const or_dual& b) { return or_dual(a.v - b.v, a.d - b.d); }
static inline or_dual operator-(const or_dual& a) { return or_dual(-a.v, -a.d); }
static inline or_dual operator*(const or_dual& a, const or_dual& b) {
    return or_dual(a.v * b.v, a.d * b.v + a.v * b.d);
}
static inline or_dual operator/(const or_dual& a, const or_dual& b) {
    const double q = a.v / b.v;
    return or_dual(q, (a.d - q * b.d) / b.v);
}
static inline or_dual& operator+=(or_dual& a, const or_dual& b) { return a = a + b; }
static inline or_dual& operator-=(or_dual& a, const or_dual& b) { return a = a - b; }
static inline or_dual& operator*=(or_dual& a, const or_dual& b) { return a = a * b; }
static inline or_dual& operator/=(or_dual& a, const or_dual& b) { return a = a / b; }
static inline bool operator<(const or_dual& a, const or_dual& b) { return a.v < b.v; }
static inline bool operator<=(const or_dual& a, const or_dual& b) { return a.v <= b.v; }
static inline bool operator>(const or_dual& a, const or_dual& b) { return a.v > b.v; }
static inline bool operator>=(const or_dual& a, const or_dual& b) { return a.v >= b.v; }
static inline bool operator==(const or_dual& a, const or_dual& b) { return a.v == b.v; }
static inline bool operator!=(const or_dual& a, const or_dual& b) { return a.v != b.v; }
static inline or_dual sqrt(const or_dual& a) {
    const double s = std::sqrt(a.v);
    return or_dual(s, a.d / (2.0 * s));
}
static inline or_dual fabs(const or_dual& a) {
    const double sg = a.v > 0.0 ? 1.0 : (a.v < 0.0 ? -1.0 : 0.0);
    return or_dual(std::fabs(a.v), sg * a.d);
}
static inline bool isfinite(const or_dual& a) { return std::isfinite(a.v) && std::isfinite(a.d); }
static inline or_dual sin(const or_dual& a) { return or_dual(std::sin(a.v), std::cos(a.v) * a.d); }
static inline or_dual cos(const or_dual& a) { return or_dual(std::cos(a.v), -std::sin(a.v) * a.d); }
static inline or_dual exp(const or_dual& a) {
    const double e = std::exp(a.v);
    return or_dual(e, e * a.d);
}

/* the oracle, with every double a dual number */
#define double or_dual
#include "hweno_oracle.c"
#undef double

/* the plain configuration record of the ctypes front-end (same layout as the C build) */
typedef struct {
    int nx, ny;
    double x0, x1, y0, y1;
    double gamma, Pr, Re;
    int bc[4];
    double cfl, b_visc, eps_pp, eps_weno;
    int max_halvings, linear_weights, limiter, scheme;
    int source, pad2_;
    double time;
    double inflow[4][2][4];
    double band[4][2];
    int linear_grad, pad3_;
} or_cfg_plain;

/* the dual configuration: mu = 1/Re moves with tangent dmu, so dRe = -Re^2 dmu */
static void or_cfg_dual(const or_cfg_plain* a, double dmu, or_cfg* b) {
    b->nx = a->nx;
    b->ny = a->ny;
    b->x0 = a->x0; b->x1 = a->x1; b->y0 = a->y0; b->y1 = a->y1;
    b->gamma = a->gamma;
    b->Pr = a->Pr;
    b->Re = or_dual(a->Re, -a->Re * a->Re * dmu);
    for (int k = 0; k < 4; k++) b->bc[k] = a->bc[k];
    b->cfl = a->cfl; b->b_visc = a->b_visc; b->eps_pp = a->eps_pp; b->eps_weno = a->eps_weno;
    b->max_halvings = a->max_halvings;
    b->linear_weights = a->linear_weights;
    b->limiter = a->limiter;
    b->scheme = a->scheme;
    b->source = a->source;
    b->pad2_ = 0;
    b->time = a->time;
    for (int s = 0; s < 4; s++) {
        for (int k = 0; k < 2; k++)
            for (int v = 0; v < 4; v++) b->inflow[s][k][v] = a->inflow[s][k][v];
        b->band[s][0] = a->band[s][0];
        b->band[s][1] = a->band[s][1];
    }
    b->linear_grad = a->linear_grad;
    b->pad3_ = 0;
}

extern "C" {

/* residual and its tangent: q, qdot [12][ny][nx]; rhs, rhs_dot [12][ny][nx];
 * vhat, vhat_dot [8][ny][nx] (either pair may be NULL); dmu the tangent of mu */
int or_jvp_residual(const or_cfg_plain* cp, const double* q, const double* qdot, double dmu, double* rhs,
                    double* rhs_dot, double* vhat, double* vhat_dot) {
    or_cfg c;
    or_cfg_dual(cp, dmu, &c);
    const size_t n = (size_t)cp->nx * cp->ny;
    or_dual* Q = (or_dual*)malloc(12 * n * sizeof(or_dual));
    or_dual* R = (or_dual*)malloc(12 * n * sizeof(or_dual));
    or_dual* V = (or_dual*)malloc(8 * n * sizeof(or_dual));
    if (!Q || !R || !V) { free(Q); free(R); free(V); return -1; }
    for (size_t k = 0; k < 12 * n; k++) Q[k] = or_dual(q[k], qdot ? qdot[k] : 0.0);
    int rc = or_residual(&c, Q, R, V, NULL, NULL, NULL, NULL, NULL, NULL);
    for (size_t k = 0; k < 12 * n; k++) {
        if (rhs) rhs[k] = R[k].v;
        if (rhs_dot) rhs_dot[k] = R[k].d;
    }
    for (size_t k = 0; k < 8 * n; k++) {
        if (vhat) vhat[k] = V[k].v;
        if (vhat_dot) vhat_dot[k] = V[k].d;
    }
    free(Q); free(R); free(V);
    return rc;
}

/* one SSP-RK3 step of size dt with its tangent, in place on (q, qdot); stats as
 * or_step (value parts) */
int or_jvp_step(const or_cfg_plain* cp, double* q, double* qdot, double dmu, double dt, double* stats) {
    or_cfg c;
    or_cfg_dual(cp, dmu, &c);
    const size_t n = (size_t)cp->nx * cp->ny;
    or_dual* Q = (or_dual*)malloc(12 * n * sizeof(or_dual));
    if (!Q) return -1;
    for (size_t k = 0; k < 12 * n; k++) Q[k] = or_dual(q[k], qdot[k]);
    or_dual st[6];
    int rc = or_step(&c, Q, or_dual(0.0), or_dual(1e300), or_dual(dt), st);
    for (size_t k = 0; k < 12 * n; k++) {
        q[k] = Q[k].v;
        qdot[k] = Q[k].d;
    }
    if (stats)
        for (int k = 0; k < 6; k++) stats[k] = st[k].v;
    free(Q);
    return rc;
}

}  /* extern "C" */
