"""Exact-rational constant tables for the FP64 CPU oracle (test infrastructure).

This script derives, in exact rational arithmetic (``fractions.Fraction``), the
stencil-dependent constants of the two-dimensional unified-stencil HWENO
reconstruction (Appendix A.2, Eqs. (A.4)-(A.6)) and writes them to
``oracle_tables.h`` as correctly rounded double literals.  Only the oracle uses
the header.

Conventions (all in the scaled coordinates of the centre cell,
xi = (x - x_i)/dx, eta = (y - y_j)/dy; the 3x3 stencil cell with offset (a, b)
covers [a-1/2, a+1/2] x [b-1/2, b+1/2]):

* Cell labels I1..I9 run row-major from (i-1, j-1): I2=(i, j-1), I4=(i-1, j),
  I5=(i, j), I6=(i+1, j), I8=(i, j+1)  (the labelling figure of Appendix A.2 is
  missing from the paper; the result is invariant under the row flip because
  the sub-stencils S1..S4 form a symmetric set with equal linear weights).
* The quartic p0 has the 15 monomials xi^p eta^q, p+q <= 4, ordered by total
  degree, then by decreasing p.
* The 17 input data of one scalar reconstruction are ordered
  [a1..a9, xi-mom(I4), xi-mom(I6), eta-mom(I2), eta-mom(I8),
   xi-mom(I2), xi-mom(I8), eta-mom(I4), eta-mom(I6)].
  The first 13 conditions are imposed exactly and the last 4 in the
  least-squares sense (Appendix A.2: "the nine zeroth-order conditions, the
  xi-conditions for k=4,6 and the eta-conditions for k=2,8 are imposed exactly;
  the remaining first-order moment conditions are included in a least-squares
  sense").  The least-squares rows carry unit weights.
* Smoothness indicator of a polynomial p (the paper cites an external formula
  without printing it; this oracle uses the classical integral indicator in the
  scaled coordinates): beta(p) = sum over multi-indices 1 <= a+b <= 4 of
  the integral over the unit cell of (d^a/dxi^a d^b/deta^b p)^2, i.e. the
  quadratic form c^T B c on the monomial coefficients c.

Run ``python oracle/gen_tables.py`` to regenerate ``oracle/oracle_tables.h``.
"""
from fractions import Fraction as F
import os

MONOS = [(p, d - p) for d in range(5) for p in range(d, -1, -1)]  # 15 (p, q)
assert len(MONOS) == 15

# stencil offsets of I1..I9, row-major from (i-1, j-1)
OFFS = [(a, b) for b in (-1, 0, 1) for a in (-1, 0, 1)]
LABEL = {k + 1: OFFS[k] for k in range(9)}
assert LABEL[2] == (0, -1) and LABEL[4] == (-1, 0) and LABEL[5] == (0, 0)
assert LABEL[6] == (1, 0) and LABEL[8] == (0, 1)


def int_pow(k, lo, hi):
    """Exact integral of t^k over [lo, hi]."""
    return (F(hi) ** (k + 1) - F(lo) ** (k + 1)) / (k + 1)


def cell_avg_row(a, b):
    """Average over cell (a,b) of each monomial (the cell has unit area)."""
    return [int_pow(p, F(2 * a - 1, 2), F(2 * a + 1, 2)) *
            int_pow(q, F(2 * b - 1, 2), F(2 * b + 1, 2)) for p, q in MONOS]


def _int_shifted(p, c):
    """Integral over [c-1/2, c+1/2] of t^p (t - c)."""
    lo, hi = F(2 * c - 1, 2), F(2 * c + 1, 2)
    return int_pow(p + 1, lo, hi) - c * int_pow(p, lo, hi)


def cell_xi_mom_row(a, b):
    """Average over cell (a,b) of monomial * (xi - a): the cell's own scaled xi-moment."""
    return [_int_shifted(p, a) * int_pow(q, F(2 * b - 1, 2), F(2 * b + 1, 2)) for p, q in MONOS]


def cell_eta_mom_row(a, b):
    return [int_pow(p, F(2 * a - 1, 2), F(2 * a + 1, 2)) * _int_shifted(q, b) for p, q in MONOS]


def data_rows():
    """The 17 linear functionals (rows) in the documented data order."""
    rows = [cell_avg_row(*LABEL[k]) for k in range(1, 10)]
    rows += [cell_xi_mom_row(*LABEL[4]), cell_xi_mom_row(*LABEL[6]),
             cell_eta_mom_row(*LABEL[2]), cell_eta_mom_row(*LABEL[8])]
    rows += [cell_xi_mom_row(*LABEL[2]), cell_xi_mom_row(*LABEL[8]),
             cell_eta_mom_row(*LABEL[4]), cell_eta_mom_row(*LABEL[6])]
    return rows


def solve_exact(A, B):
    """Gauss-Jordan elimination over the rationals: returns A^{-1} B (A square)."""
    n = len(A)
    M = [list(A[i]) + list(B[i]) for i in range(n)]
    for col in range(n):
        piv = next(r for r in range(col, n) if M[r][col] != 0)
        M[col], M[piv] = M[piv], M[col]
        pv = M[col][col]
        M[col] = [x / pv for x in M[col]]
        for r in range(n):
            if r != col and M[r][col] != 0:
                f = M[r][col]
                M[r] = [x - f * y for x, y in zip(M[r], M[col])]
    return [row[n:] for row in M]


def p0_map():
    """15x17 rational matrix Mp with c = Mp d for the equality-constrained LS problem.

    minimise ||A c - d_ls||^2 subject to E c = d_eq, through the KKT system
      [A^T A  E^T] [c]   [A^T d_ls]
      [E      0  ] [l] = [d_eq    ].
    """
    rows = data_rows()
    E, A = rows[:13], rows[13:]
    n, me, ml = 15, 13, 4
    AtA = [[sum(A[r][i] * A[r][j] for r in range(ml)) for j in range(n)] for i in range(n)]
    K = [AtA[i] + [E[r][i] for r in range(me)] for i in range(n)]
    K += [E[r] + [F(0)] * me for r in range(me)]
    # right-hand side as a linear map of the 17 data: columns = data
    RHS = [[F(0)] * 17 for _ in range(n + me)]
    for i in range(n):
        for r in range(ml):
            RHS[i][13 + r] = A[r][i]
    for r in range(me):
        RHS[n + r][r] = F(1)
    sol = solve_exact(K, RHS)
    return [sol[i] for i in range(n)]


def dmono(p, q, a, b):
    """d^a/dxi^a d^b/deta^b of xi^p eta^q -> (coef, p', q') or None."""
    if a > p or b > q:
        return None
    c = 1
    for t in range(a):
        c *= (p - t)
    for t in range(b):
        c *= (q - t)
    return (c, p - a, q - b)


def beta_matrix():
    """B[i][j] = sum_{1<=a+b<=4} int_unit d^(a,b) m_i * d^(a,b) m_j."""
    h = F(1, 2)
    B = [[F(0)] * 15 for _ in range(15)]
    for a in range(5):
        for b in range(5 - a):
            if a + b == 0:
                continue
            for i, (pi, qi) in enumerate(MONOS):
                di = dmono(pi, qi, a, b)
                if di is None:
                    continue
                for j, (pj, qj) in enumerate(MONOS):
                    dj = dmono(pj, qj, a, b)
                    if dj is None:
                        continue
                    B[i][j] += (di[0] * dj[0] * int_pow(di[1] + dj[1], -h, h) *
                                int_pow(di[2] + dj[2], -h, h))
    return B


def centre_moment_rows():
    """Scaled first moments over the centre cell: int m xi, int m eta."""
    return cell_xi_mom_row(0, 0), cell_eta_mom_row(0, 0)


def fmt(x):
    return repr(float(x))


def main():
    Mp = p0_map()
    rows = data_rows()
    # sanity: exact rows satisfied identically (E Mp = [I 0])
    for r in range(13):
        for col in range(17):
            v = sum(rows[r][i] * Mp[i][col] for i in range(15))
            assert v == (1 if col == r else 0)
    B = beta_matrix()
    mx, my = centre_moment_rows()
    out = []
    out.append("/* Generated by oracle/gen_tables.py from exact rational arithmetic.\n"
               " * Oracle-only constants (test infrastructure); see that script for the\n"
               " * monomial order, the data order and the stencil labels. */\n")
    out.append("#ifndef HWENO_ORACLE_TABLES_H\n#define HWENO_ORACLE_TABLES_H\n\n")
    out.append("static const int OR_MONO_P[15] = {%s};\n" % ", ".join(str(p) for p, q in MONOS))
    out.append("static const int OR_MONO_Q[15] = {%s};\n\n" % ", ".join(str(q) for p, q in MONOS))
    out.append("/* p0 coefficients = OR_P0MAP * data17 (equality-constrained least squares) */\n")
    out.append("static const double OR_P0MAP[15][17] = {\n")
    for i in range(15):
        out.append("  {" + ", ".join(fmt(x) for x in Mp[i]) + "},\n")
    out.append("};\n\n/* smoothness indicator quadratic form on the 15 monomial coefficients */\n")
    out.append("static const double OR_BETA_B[15][15] = {\n")
    for i in range(15):
        out.append("  {" + ", ".join(fmt(x) for x in B[i]) + "},\n")
    out.append("};\n\n/* centre-cell scaled moments of each monomial: avg(m*xi), avg(m*eta) */\n")
    out.append("static const double OR_MOM_XI[15] = {" + ", ".join(fmt(x) for x in mx) + "};\n")
    out.append("static const double OR_MOM_ETA[15] = {" + ", ".join(fmt(x) for x in my) + "};\n\n")
    out.append("#endif\n")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_tables.h")
    with open(path, "w") as f:
        f.write("".join(out))
    print("wrote", path)


if __name__ == "__main__":
    main()
