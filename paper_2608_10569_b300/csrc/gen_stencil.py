"""Generate hweno_stencil.h: straight-line device code for the stencil-fixed parts of
the unified-stencil HWENO reconstruction (Appendix A.2, Eqs. (A.4)-(A.6)).

The constants are derived here in float64 with numpy:
  * the 17 moment conditions of the quartic p0 on the 3x3 stencil are assembled from
    closed-form float integrals of each monomial over the stencil cells;
  * the 13 exact conditions and 4 least-squares conditions (unit weights) give the
    KKT system, solved with numpy.linalg.solve plus iterative refinement;
  * the smoothness indicator is the integral over the cell, in scaled coordinates,
    of the squares of all derivatives of orders 1..4 (a quadratic form).
Entries below 1e-13 in magnitude are exact zeros of the underlying rational map and
are dropped, so the emitted code multiplies only by the non-zero entries.

Layouts used by the kernels (and fixed here):
  monomials  k -> xi^p eta^q, ordered by total degree then decreasing p:
             1, xi, eta, xi^2, xi eta, eta^2, xi^3, ..., eta^4
  data       d[0..8] cell averages of the 3x3 block, row-major from (i-1, j-1);
             d[9], d[10]  xi-moments of (i-1, j), (i+1, j)      (exact)
             d[11], d[12] eta-moments of (i, j-1), (i, j+1)     (exact)
             d[13], d[14] xi-moments of (i, j-1), (i, j+1)      (least squares)
             d[15], d[16] eta-moments of (i-1, j), (i+1, j)     (least squares)

Run: python gen_stencil.py  (writes hweno_stencil.h beside this file)
"""
import os

import numpy as np

MONO = [(p, d - p) for d in range(5) for p in range(d, -1, -1)]


def _ipow(k, lo, hi):
    """integral of t^k over [lo, hi] in closed form (float)"""
    return (hi ** (k + 1) - lo ** (k + 1)) / (k + 1)


def functionals():
    """17 x 15 matrix: data functional applied to each monomial (closed-form integrals
    over cells [a-1/2, a+1/2] x [b-1/2, b+1/2] of the unit-spaced stencil)"""
    off = [(a, b) for b in (-1, 0, 1) for a in (-1, 0, 1)]

    def avg(a, b):
        return [_ipow(p, a - 0.5, a + 0.5) * _ipow(q, b - 0.5, b + 0.5) for p, q in MONO]

    def xi_m(a, b):
        return [(_ipow(p + 1, a - 0.5, a + 0.5) - a * _ipow(p, a - 0.5, a + 0.5)) *
                _ipow(q, b - 0.5, b + 0.5) for p, q in MONO]

    def eta_m(a, b):
        return [_ipow(p, a - 0.5, a + 0.5) *
                (_ipow(q + 1, b - 0.5, b + 0.5) - b * _ipow(q, b - 0.5, b + 0.5)) for p, q in MONO]

    rows = [avg(a, b) for (a, b) in off]
    rows += [xi_m(-1, 0), xi_m(1, 0), eta_m(0, -1), eta_m(0, 1)]
    rows += [xi_m(0, -1), xi_m(0, 1), eta_m(-1, 0), eta_m(1, 0)]
    return np.array(rows)


def p0_map():
    A = functionals()
    E, L = A[:13], A[13:]
    K = np.zeros((28, 28))
    K[:15, :15] = L.T @ L
    K[:15, 15:] = E.T
    K[15:, :15] = E
    rhs = np.zeros((28, 17))
    rhs[:15, 13:] = L.T
    rhs[15:, :13] = np.eye(13)
    X = np.linalg.solve(K, rhs)
    # two rounds of iterative refinement with the residual formed in extended precision
    for _ in range(2):
        r = rhs.astype(np.longdouble) - K.astype(np.longdouble) @ X.astype(np.longdouble)
        X = X + np.linalg.solve(K, r.astype(np.float64))
    M = X[:15]
    M[np.abs(M) < 1e-13] = 0.0
    return M


def beta_form():
    """B[i][j] = sum over 1 <= a+b <= 4 of the cell integral of d^(a,b) m_i * d^(a,b) m_j"""
    def deriv(p, q, a, b):
        if a > p or b > q:
            return None
        c = 1.0
        for t in range(a):
            c *= p - t
        for t in range(b):
            c *= q - t
        return c, p - a, q - b

    B = np.zeros((15, 15))
    for a in range(5):
        for b in range(5 - a):
            if a + b == 0:
                continue
            for i, (pi, qi) in enumerate(MONO):
                di = deriv(pi, qi, a, b)
                if di is None:
                    continue
                for j, (pj, qj) in enumerate(MONO):
                    dj = deriv(pj, qj, a, b)
                    if dj is None:
                        continue
                    B[i, j] += di[0] * dj[0] * _ipow(di[1] + dj[1], -0.5, 0.5) * _ipow(di[2] + dj[2], -0.5, 0.5)
    B[np.abs(B) < 1e-13] = 0.0
    return B


def _lit(x):
    return "T(%r)" % float(x)


def emit():
    M = p0_map()
    B = beta_form()
    out = []
    out.append("// Generated by gen_stencil.py (float64 numpy derivation); do not edit.\n")
    out.append("// Unified-stencil HWENO constants of Appendix A.2 as straight-line code.\n")
    out.append("#pragma once\n\n")
    out.append("// p0 coefficients (15 monomials) from the 17 stencil data: constrained least squares\n")
    out.append("template <class T> __device__ __forceinline__ void hw_p0_coeffs(const T* d, T* c) {\n")
    for k in range(15):
        terms = [(M[k, n], n) for n in range(17) if M[k, n] != 0.0]
        expr = " + ".join("%s * d[%d]" % (_lit(v), n) for v, n in terms)
        out.append("  c[%d] = %s;\n" % (k, expr))
    out.append("}\n\n")
    out.append("// smoothness indicator of a quartic: c^T B c over the non-constant monomials\n")
    out.append("template <class T> __device__ __forceinline__ T hw_beta_quartic(const T* c) {\n")
    out.append("  T s = T(0);\n")
    for i in range(1, 15):
        terms = []
        if B[i, i] != 0.0:
            terms.append("%s * c[%d]" % (_lit(B[i, i]), i))
        for j in range(i + 1, 15):
            if B[i, j] != 0.0:
                terms.append("%s * c[%d]" % (_lit(2.0 * B[i, j]), j))
        if terms:
            out.append("  s += c[%d] * (%s);\n" % (i, " + ".join(terms)))
    out.append("  return s;\n}\n\n")
    # moments over the centre cell of each monomial times xi or eta
    mx = [_ipow(p + 1, -0.5, 0.5) * _ipow(q, -0.5, 0.5) for p, q in MONO]
    my = [_ipow(p, -0.5, 0.5) * _ipow(q + 1, -0.5, 0.5) for p, q in MONO]
    out.append("// scaled first moments over the centre cell: avg(p xi), avg(p eta)\n")
    for name, m in (("hw_moment_xi", mx), ("hw_moment_eta", my)):
        out.append("template <class T> __device__ __forceinline__ T %s(const T* c) {\n" % name)
        terms = ["%s * c[%d]" % (_lit(v), k) for k, v in enumerate(m) if abs(v) > 1e-15]
        out.append("  return %s;\n}\n" % " + ".join(terms))
    # transposes for the discrete adjoint
    out.append("\n// adjoint of hw_p0_coeffs: dbar[n] += sum_k M[k][n] cbar[k]\n")
    out.append("template <class T> __device__ __forceinline__ void hw_p0_coeffs_T(const T* cbar, T* dbar) {\n")
    for n in range(17):
        terms = [(M[k, n], k) for k in range(15) if M[k, n] != 0.0]
        if terms:
            out.append("  dbar[%d] += %s;\n" % (n, " + ".join("%s * cbar[%d]" % (_lit(v), k) for v, k in terms)))
    out.append("}\n\n// gradient of the smoothness indicator: g = 2 B c\n")
    out.append("template <class T> __device__ __forceinline__ void hw_beta_quartic_grad(const T* c, T* g) {\n")
    out.append("  g[0] = T(0);\n")
    for i in range(1, 15):
        terms = ["%s * c[%d]" % (_lit(2.0 * B[i, j]), j) for j in range(1, 15) if B[i, j] != 0.0]
        out.append("  g[%d] = %s;\n" % (i, " + ".join(terms) if terms else "T(0)"))
    out.append("}\n")
    for name, m in (("hw_moment_xi_T", mx), ("hw_moment_eta_T", my)):
        out.append("template <class T> __device__ __forceinline__ void %s(T mbar, T* cbar) {\n" % name)
        for k, v in enumerate(m):
            if abs(v) > 1e-15:
                out.append("  cbar[%d] += %s * mbar;\n" % (k, _lit(v)))
        out.append("}\n")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hweno_stencil.h")
    with open(path, "w") as f:
        f.write("".join(out))
    return path


if __name__ == "__main__":
    print("wrote", emit())
