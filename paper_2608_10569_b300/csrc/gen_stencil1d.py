"""Generate hweno1d_stencil.h: straight-line device code for the stencil-fixed parts of
the one-dimensional unified-stencil HWENO reconstruction (Appendix A.1).

The constants are exact rationals derived here with sympy and emitted as doubles:
  * the quartic p0 = sum_k c_k xi^k satisfies five conditions on the three-cell
    stencil (scaled coordinate, unit cells centred at -1, 0, 1): the averages over the
    three cells and the first moments int p0 (xi - j) over cells j = -1 and 1; the
    5 x 5 system is inverted exactly, so c = M d;
  * the smoothness indicator of a quartic is the integral over the centre cell of the
    squares of its derivatives of orders 1..4, a quadratic form c^T B c;
  * the modified moment of a quartic is int xi p0 over the centre cell.

Layouts used by the kernels (and fixed here):
  monomials  k -> xi^k, k = 0..4
  data       d[0], d[1], d[2]: averages of cells i-1, i, i+1;
             d[3], d[4]: first moments of cells i-1, i+1

Run: python gen_stencil1d.py  (writes hweno1d_stencil.h beside this file)
"""
import os

import sympy as sp

XI = sp.Symbol("xi")
HALF = sp.Rational(1, 2)


def conditions():
    """5 x 5 matrix: data functional (row) applied to monomial xi^k (column)"""
    rows = []
    for j in (-1, 0, 1):
        rows.append([sp.integrate(XI ** k, (XI, j - HALF, j + HALF)) for k in range(5)])
    for j in (-1, 1):
        rows.append([sp.integrate(XI ** k * (XI - j), (XI, j - HALF, j + HALF)) for k in range(5)])
    return sp.Matrix(rows)


def beta_form():
    B = sp.zeros(5, 5)
    for a in range(5):
        for b in range(5):
            B[a, b] = sum(sp.integrate(sp.diff(XI ** a, XI, l) * sp.diff(XI ** b, XI, l), (XI, -HALF, HALF))
                          for l in range(1, 5))
    return B


def lit(x):
    return "T(%r)" % float(x)


def emit():
    M = conditions().inv()
    B = beta_form()
    mom = [sp.integrate(XI ** (k + 1), (XI, -HALF, HALF)) for k in range(5)]
    out = ["// Generated by gen_stencil1d.py (exact rationals via sympy); do not edit.",
           "// One-dimensional unified-stencil HWENO constants of Appendix A.1 as straight-line code.",
           "#pragma once", "",
           "// p0 coefficients (xi^0..xi^4) from the five stencil data",
           "template <class T> __host__ __device__ __forceinline__ void hw1_p0_coeffs(const T* d, T* c) {"]
    for k in range(5):
        terms = [f"{lit(M[k, m])} * d[{m}]" for m in range(5) if M[k, m] != 0]
        out.append(f"  c[{k}] = " + " + ".join(terms) + ";")
    out += ["}", "",
            "// smoothness indicator of a quartic: sum over orders 1..4 of the cell integral of the",
            "// squared derivative (a quadratic form in its coefficients)",
            "template <class T> __host__ __device__ __forceinline__ T hw1_beta_quartic(const T* c) {",
            "  T s = T(0);"]
    for a in range(5):
        for b in range(a, 5):
            v = B[a, b] * (1 if a == b else 2)
            if v != 0:
                out.append(f"  s += {lit(v)} * c[{a}] * c[{b}];")
    out += ["  return s;", "}", "",
            "// modified moment int xi p(xi) over the centre cell of a quartic",
            "template <class T> __host__ __device__ __forceinline__ T hw1_moment(const T* c) {",
            "  return " + " + ".join(f"{lit(mom[k])} * c[{k}]" for k in range(5) if mom[k] != 0) + ";",
            "}", ""]
    return "\n".join(out)


if __name__ == "__main__":
    here = os.path.dirname(os.path.abspath(__file__))
    with open(os.path.join(here, "hweno1d_stencil.h"), "w") as f:
        f.write(emit())
