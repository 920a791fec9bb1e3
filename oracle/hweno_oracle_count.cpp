/*
 * OPERATION-COUNTING BUILD OF THE FP64 CPU ORACLE.  TEST AND MEASUREMENT
 * INFRASTRUCTURE ONLY: like hweno_oracle.c, nothing in the product path may call, link
 * or load it.  It gives the algorithmic floating-point work of the method, per interior
 * cell and RK stage, independently of the CUDA kernels whose speed it is set against.
 *
 * It recompiles hweno_oracle.c unchanged, with its floating-point type replaced by a
 * counting number: a value and the identity of the computation that produced it.  Values
 * that depend on the solution state carry a nonzero identity (the state's values get
 * fresh ones); literals, the tables of exact constants and the configuration carry none.
 * An operation is counted once per distinct computation:
 *   - operations on state-free values only (powers of the Gauss nodes, 1/gamma_0, 1/dx)
 *     are compile-time constants and free;
 *   - a product or quotient with a state-free 0 or +-1, or a sum with a state-free 0, is
 *     free (straight-line code never performs it), and a product with a state-free 0 is
 *     itself a state-free 0;
 *   - the same operation on the same operands (commuted operands included) is counted
 *     only the first time: the oracle's plain form recomputes values (the physical flux
 *     of a volume point per conserved variable, the primitive variables of a face trace
 *     in both neighbouring cells, the reconstruction of a ghost cell whose state is a
 *     periodic copy), and a program that keeps a value it already has does not pay
 *     for it again.
 * Additions and subtractions, multiplications, divisions, square roots, and the
 * transcendental functions of the manufactured source are counted separately; |x|,
 * negation and comparisons are not floating-point work.  The oracle's own algebra is kept
 * otherwise: each candidate polynomial evaluated at each point and combined as Eq. (3.4)
 * prints, the data projected before reconstruction (Sec. 3.1), the PP limiter's checks
 * at all 21 points (Sec. 3.1).  On a periodic grid every ghost cell holds a copy of an
 * interior cell's state, so the counts of one spatial operator divided by the number of
 * cells are the work per cell, with no halo.
 */
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <unordered_map>

enum { OC_ADD = 0, OC_MUL, OC_DIV, OC_SQRT, OC_TRANS, OC_N };
static long long g_oc[OC_N];
static uint64_t g_oc_next = 1;  // next identity of a state-dependent value

struct or_cnt {
    double v;
    uint64_t id;  // 0: state-free
    or_cnt() = default;
    constexpr or_cnt(double x) : v(x), id(0) {}
    constexpr or_cnt(double x, uint64_t i) : v(x), id(i) {}
};

// a computation: the operation and its two operands, each the identity of a
// state-dependent value or the bit pattern of a state-free one (flagged in kinds)
struct oc_key {
    uint64_t op, a, b;
    bool operator==(const oc_key& o) const { return op == o.op && a == o.a && b == o.b; }
};
struct oc_hash {
    size_t operator()(const oc_key& k) const {
        uint64_t h = k.op * 0x9e3779b97f4a7c15ull;
        h ^= k.a + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        h ^= k.b + 0x9e3779b97f4a7c15ull + (h << 6) + (h >> 2);
        return (size_t)h;
    }
};
static std::unordered_map<oc_key, uint64_t, oc_hash> g_oc_seen;

enum { OP_ADD = 1, OP_SUB, OP_MUL, OP_DIV, OP_SQRT, OP_NEG, OP_ABS, OP_SIN, OP_COS, OP_EXP };

static inline uint64_t oc_operand(const or_cnt& a) {
    if (a.id) return a.id;
    uint64_t b;
    memcpy(&b, &a.v, sizeof(b));
    return b;
}

static inline bool oc_const_is(const or_cnt& a, double x) { return !a.id && a.v == x; }
static inline void oc_reset() {
    memset(g_oc, 0, sizeof(g_oc));
    g_oc_seen.clear();
    g_oc_next = 1;
}

// the result of a state-dependent computation: its identity, counted the first time
static inline or_cnt oc_result(int kind, int op, const or_cnt& a, const or_cnt& b, bool commutes, double r) {
    uint64_t x = oc_operand(a), y = oc_operand(b);
    uint64_t cx = a.id ? 0u : 1u, cy = b.id ? 0u : 1u;  // state-free operand flags
    if (commutes && (cx > cy || (cx == cy && x > y))) {
        uint64_t t = x; x = y; y = t;
        t = cx; cx = cy; cy = t;
    }
    const oc_key k{(uint64_t)op | (cx << 8) | (cy << 9), x, y};
    auto it = g_oc_seen.find(k);
    if (it != g_oc_seen.end()) return or_cnt(r, it->second);
    const uint64_t id = g_oc_next++;
    g_oc_seen.emplace(k, id);
    if (kind >= 0) g_oc[kind]++;
    return or_cnt(r, id);
}

static inline or_cnt operator+(const or_cnt& a, const or_cnt& b) {
    const double r = a.v + b.v;
    if (!a.id && !b.id) return or_cnt(r);
    if (oc_const_is(a, 0.0)) return b;
    if (oc_const_is(b, 0.0)) return a;
    return oc_result(OC_ADD, OP_ADD, a, b, true, r);
}
static inline or_cnt operator-(const or_cnt& a) {
    if (!a.id) return or_cnt(-a.v);
    return oc_result(-1, OP_NEG, a, or_cnt(0.0), false, -a.v);
}
static inline or_cnt operator-(const or_cnt& a, const or_cnt& b) {
    const double r = a.v - b.v;
    if (!a.id && !b.id) return or_cnt(r);
    if (oc_const_is(b, 0.0)) return a;
    if (oc_const_is(a, 0.0)) return -b;
    return oc_result(OC_ADD, OP_SUB, a, b, false, r);
}
static inline or_cnt operator*(const or_cnt& a, const or_cnt& b) {
    const double r = a.v * b.v;
    if (oc_const_is(a, 0.0) || oc_const_is(b, 0.0)) return or_cnt(r);
    if (!a.id && !b.id) return or_cnt(r);
    if (oc_const_is(a, 1.0)) return b;
    if (oc_const_is(b, 1.0)) return a;
    if (oc_const_is(a, -1.0)) return -b;
    if (oc_const_is(b, -1.0)) return -a;
    return oc_result(OC_MUL, OP_MUL, a, b, true, r);
}
static inline or_cnt operator/(const or_cnt& a, const or_cnt& b) {
    const double r = a.v / b.v;
    if (oc_const_is(a, 0.0)) return or_cnt(r);
    if (!a.id && !b.id) return or_cnt(r);
    if (oc_const_is(b, 1.0)) return a;
    if (oc_const_is(b, -1.0)) return -a;
    return oc_result(OC_DIV, OP_DIV, a, b, false, r);
}
static inline or_cnt& operator+=(or_cnt& a, const or_cnt& b) { return a = a + b; }
static inline or_cnt& operator-=(or_cnt& a, const or_cnt& b) { return a = a - b; }
static inline or_cnt& operator*=(or_cnt& a, const or_cnt& b) { return a = a * b; }
static inline or_cnt& operator/=(or_cnt& a, const or_cnt& b) { return a = a / b; }
static inline bool operator<(const or_cnt& a, const or_cnt& b) { return a.v < b.v; }
static inline bool operator<=(const or_cnt& a, const or_cnt& b) { return a.v <= b.v; }
static inline bool operator>(const or_cnt& a, const or_cnt& b) { return a.v > b.v; }
static inline bool operator>=(const or_cnt& a, const or_cnt& b) { return a.v >= b.v; }
static inline bool operator==(const or_cnt& a, const or_cnt& b) { return a.v == b.v; }
static inline bool operator!=(const or_cnt& a, const or_cnt& b) { return a.v != b.v; }
static inline or_cnt oc_unary(int kind, int op, const or_cnt& a, double r) {
    if (!a.id) return or_cnt(r);
    return oc_result(kind, op, a, or_cnt(0.0), false, r);
}
static inline or_cnt sqrt(const or_cnt& a) { return oc_unary(OC_SQRT, OP_SQRT, a, std::sqrt(a.v)); }
static inline or_cnt fabs(const or_cnt& a) { return oc_unary(-1, OP_ABS, a, std::fabs(a.v)); }
static inline bool isfinite(const or_cnt& a) { return std::isfinite(a.v); }
static inline or_cnt sin(const or_cnt& a) { return oc_unary(OC_TRANS, OP_SIN, a, std::sin(a.v)); }
static inline or_cnt cos(const or_cnt& a) { return oc_unary(OC_TRANS, OP_COS, a, std::cos(a.v)); }
static inline or_cnt exp(const or_cnt& a) { return oc_unary(OC_TRANS, OP_EXP, a, std::exp(a.v)); }

/* the oracle, with every double a counting number */
#define double or_cnt
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

static void oc_cfg(const or_cfg_plain* a, or_cfg* b) {
    b->nx = a->nx;
    b->ny = a->ny;
    b->x0 = a->x0; b->x1 = a->x1; b->y0 = a->y0; b->y1 = a->y1;
    b->gamma = a->gamma;
    b->Pr = a->Pr;
    b->Re = a->Re;
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

static or_cnt* oc_state(const double* q, size_t n) {
    or_cnt* Q = (or_cnt*)malloc(n * sizeof(or_cnt));
    if (Q)
        for (size_t k = 0; k < n; k++) Q[k] = or_cnt(q[k], g_oc_next++);
    return Q;
}

static void oc_take(long long* out) {
    for (int k = 0; k < OC_N; k++) {
        out[k] += g_oc[k];
        g_oc[k] = 0;
    }
}

extern "C" {

/* phases of one spatial operator, in the order of the oracle's residual:
 * out[OC_N * p + k], p = 0 traces (or_cons_cell), 1 limiter (or_limit_cell),
 * 2 weak-derivative moments (or_rmom_cell), 3 gradients (or_grad_cell, or HWENO-DR's
 * or_dr_grad_cell), 4 face fluxes (or_face_flux, both directions), 5 moment balances
 * (or_assemble_cell; with the source, its moments), 6 alpha* (the time step's face
 * maximum over the interior cells' faces).  A computation met again in a later phase is
 * counted where it first occurred. */
int or_count_phases(const or_cfg_plain* cp, const double* q, long long* out) {
    or_cfg c;
    oc_cfg(cp, &c);
    oc_reset();
    const int wx = cp->nx, wy = cp->ny;
    or_cnt* Q = oc_state(q, 12 * (size_t)wx * wy);
    if (!Q) return -1;
    or_work W;
    const int bx = wx + 2 * OR_G, by = wy + 2 * OR_G;
    if (or_work_alloc(&W, &c, bx, by)) { or_work_free(&W); free(Q); return -1; }
    for (int k = 0; k < 7 * OC_N; k++) out[k] = 0;
    const or_cnt dx = (c.x1 - c.x0) / c.nx, dy = (c.y1 - c.y0) / c.ny;
    for (int j = -OR_G; j < wy + OR_G; j++)
        for (int i = -OR_G; i < wx + OR_G; i++) or_fetch(&c, Q, i, j, W.Q + 12 * IDX(&W, i, j));
    oc_take(out + 6 * OC_N);  /* the ghost fill: copies (and sign changes) only */
    for (int k = 0; k < OC_N; k++) out[6 * OC_N + k] = 0;
    for (int j = -3; j < wy + 3; j++)
        for (int i = -3; i < wx + 3; i++) {
            or_cons_cell(&W, i, j);
            oc_take(out + 0 * OC_N);
            or_limit_cell(&W, i, j);
            oc_take(out + 1 * OC_N);
        }
    if (c.scheme == 1) {
        for (int j = -1; j < wy + 1; j++)
            for (int i = -1; i < wx + 1; i++) or_dr_grad_cell(&W, i, j);
        oc_take(out + 3 * OC_N);
    } else {
        for (int j = -2; j < wy + 2; j++)
            for (int i = -2; i < wx + 2; i++) or_rmom_cell(&W, i, j, dx, dy);
        oc_take(out + 2 * OC_N);
        for (int j = -1; j < wy + 1; j++)
            for (int i = -1; i < wx + 1; i++) or_grad_cell(&W, i, j);
        oc_take(out + 3 * OC_N);
    }
    for (int j = 0; j < wy; j++)
        for (int i = -1; i < wx; i++) or_face_flux(&W, 0, i, j);
    for (int j = -1; j < wy; j++)
        for (int i = 0; i < wx; i++) or_face_flux(&W, 1, i, j);
    oc_take(out + 4 * OC_N);
    for (int j = 0; j < wy; j++)
        for (int i = 0; i < wx; i++) {
            or_cnt r[12];
            or_assemble_cell(&W, i, j, dx, dy, r);
            if (c.source == 1) {
                or_cnt sm[12];
                or_mms_moments(&c, i, j, c.time, sm);
                for (int k = 0; k < 12; k++) r[k] += sm[k];
            }
        }
    oc_take(out + 5 * OC_N);
    or_work_free(&W);
    free(Q);
    /* alpha*: the whole residual with and without its diagnostics */
    long long with[OC_N], without[OC_N];
    for (int pass = 0; pass < 2; pass++) {
        oc_reset();
        or_cnt* Q2 = oc_state(q, 12 * (size_t)wx * wy);
        or_cnt* R = (or_cnt*)malloc(12 * (size_t)wx * wy * sizeof(or_cnt));
        or_cnt* V = (or_cnt*)malloc(8 * (size_t)wx * wy * sizeof(or_cnt));
        if (!Q2 || !R || !V) { free(Q2); free(R); free(V); return -1; }
        or_cnt diag[OR_NDIAG];
        or_residual(&c, Q2, R, V, pass == 0 ? diag : NULL, NULL, NULL, NULL, NULL, NULL);
        long long* o = pass == 0 ? with : without;
        for (int k = 0; k < OC_N; k++) o[k] = g_oc[k];
        free(Q2); free(R); free(V);
    }
    for (int k = 0; k < OC_N; k++) out[6 * OC_N + k] = with[k] - without[k];
    oc_reset();
    return 0;
}

/* counts of whole calls: what = 0 the residual with its diagnostics (alpha*, beta_max),
 * 1 the residual without them, 2 one SSP-RK3 step of size dt (three residuals with
 * diagnostics, stage updates, admissibility checks) */
int or_count_call(const or_cfg_plain* cp, const double* q, int what, double dt, long long* out) {
    or_cfg c;
    oc_cfg(cp, &c);
    oc_reset();
    const size_t n = (size_t)cp->nx * cp->ny;
    or_cnt* Q = oc_state(q, 12 * n);
    or_cnt* R = (or_cnt*)malloc(12 * n * sizeof(or_cnt));
    or_cnt* V = (or_cnt*)malloc(8 * n * sizeof(or_cnt));
    if (!Q || !R || !V) { free(Q); free(R); free(V); return -1; }
    for (int k = 0; k < OC_N; k++) out[k] = 0;
    int rc = 0;
    or_cnt diag[OR_NDIAG], st[6];
    if (what == 0) rc = or_residual(&c, Q, R, V, diag, NULL, NULL, NULL, NULL, NULL);
    else if (what == 1) rc = or_residual(&c, Q, R, V, NULL, NULL, NULL, NULL, NULL, NULL);
    else rc = or_step(&c, Q, or_cnt(0.0), or_cnt(1e300), or_cnt(dt), st);
    oc_take(out);
    free(Q); free(R); free(V);
    oc_reset();
    return rc;
}

/* counts of one theta root of the limiter (ub, uq state-dependent; eps, gamma not) */
double or_count_theta_root(const double* ub, const double* uq, double eps, double g, long long* out) {
    oc_reset();
    or_cnt a[4], b[4];
    for (int k = 0; k < 4; k++) { a[k] = or_cnt(ub[k], g_oc_next++); b[k] = or_cnt(uq[k], g_oc_next++); }
    for (int k = 0; k < OC_N; k++) out[k] = 0;
    const or_cnt t = or_theta_root(a, b, or_cnt(eps), or_cnt(g));
    oc_take(out);
    oc_reset();
    return t.v;
}

/* counts of one scalar reconstruction from 17 state-dependent data and its evaluation
 * at npts points (xi, eta): out[0..OC_N) the build (p0, candidates, indicators,
 * weights), out[OC_N..2 OC_N) the evaluations */
int or_count_hweno(const double* d17, double eps, int linear, int npts, const double* xi, const double* eta,
                   long long* out) {
    oc_reset();
    or_cnt d[17];
    for (int k = 0; k < 17; k++) d[k] = or_cnt(d17[k], g_oc_next++);
    for (int k = 0; k < 2 * OC_N; k++) out[k] = 0;
    or_hweno h;
    or_hweno_build(d, or_cnt(eps), linear, &h);
    oc_take(out);
    for (int p = 0; p < npts; p++) (void)or_hweno_eval(&h, or_cnt(xi[p]), or_cnt(eta[p]));
    oc_take(out + OC_N);
    oc_reset();
    return 0;
}

}  /* extern "C" */
