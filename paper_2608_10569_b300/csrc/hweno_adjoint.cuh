// Discrete adjoint (vector-Jacobian products) of the FP64 spatial operator.
//
// For a state x, the forward evaluation gives the residual R(x) (Eq. (3.2)) and the
// modified moments M(x) (Eq. (3.4)).  Given seeds Rbar (12 planes) and Mbar (8 planes)
// the kernels below compute xbar = (dR/dx)^T Rbar + (dM/dx)^T Mbar and the derivative
// with respect to mu = 1/Re, by reverse passes through the kernels of the forward
// operator, last to first:
//   assembly (volume part) -> face fluxes -> gradient HWENO -> weak/face moments ->
//   characteristic HWENO with its eigenvectors -> ghost cells.
// Each reverse kernel recomputes its own cell's forward arithmetic from the stored
// forward intermediates, then applies the transposed chain rule.  Where a forward
// output feeds several cells (stencils), the reverse kernel writes one contribution
// per stencil slot and a gather kernel sums them in a fixed order (deterministic, no
// atomics).  Branches are differentiated on the side the forward took: |x| by sign(x),
// max() by its argument (the Lax-Friedrichs coefficient goes to the state that set it).
// The positivity limiter is differentiated on the branch the forward took: through its
// density factor, the argmin point of its minimum density, the argmin point of its
// smallest pressure root (implicit-function theorem on the pressure quadratic) and the
// term that set eps.
#pragma once
#include "hweno_ops.cuh"

namespace hw {

__device__ __forceinline__ double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

// adjoint planes of one operator evaluation (padded layout like the forward planes)
struct Adj {
  double* R;      // 12 seeds: residual adjoint (interior)
  double* M;      // 8 seeds: modified-moment adjoint (interior)
  double* face;   // 48: adjoint of the limited face primitives (rho, u, v, e) per point
  double* vol;    // 36: adjoint of the volume primitives
  double* gr;     // 126: adjoint of the gradients at the 21 points
  double* rm;     // 18: adjoint of the weak-derivative moments
  double* cg;     // 102: per-cell contributions of k_grad's reverse to its 17 stencil data x 6
  double* cc;     // 68: per-cell contributions of k_cons's reverse to its 17 stencil data x 4
  double* q;      // 12: adjoint of the padded state (ghost layers included)
  double* mu;     // 1 double: d/d(1/Re), accumulated
};

// ---------------------------------------------------------------------------
// adjoints of the pointwise helpers

// cons -> prim (rho, u, v, e) VJP: given wbar at U, accumulate Ubar; takes the primitive
// values W = (rho, u, v, e) of U
__device__ __forceinline__ void prim_T_w(const double* W, const double* wb, double* Ub) {
  const double rr = 1.0 / W[0];
  const double u = W[1], v = W[2], e = W[3];
  Ub[1] += (wb[1] - wb[3] * u) * rr;
  Ub[2] += (wb[2] - wb[3] * v) * rr;
  Ub[3] += wb[3] * rr;
  Ub[0] += wb[0] + rr * (-wb[1] * u - wb[2] * v + wb[3] * (-e + 0.5 * (u * u + v * v)));
}

// prim (rho, u, v, e) -> cons:  given Ubar, accumulate wbar
__device__ __forceinline__ void cons_T(const double* w, const double* Ub, double* wb) {
  const double rho = w[0], u = w[1], v = w[2], e = w[3];
  wb[0] += Ub[0] + Ub[1] * u + Ub[2] * v + Ub[3] * (e + 0.5 * (u * u + v * v));
  wb[1] += Ub[1] * rho + Ub[3] * rho * u;
  wb[2] += Ub[2] * rho + Ub[3] * rho * v;
  wb[3] += Ub[3] * rho;
}

// physical flux (phys_flux) adjoint: given fbar, accumulate wbar, sbar and mu-bar
__device__ __forceinline__ void phys_flux_T(int dir, const double* w, const double* s, double gamma, double rPr,
                                            double rRe, const double* fb, double* wb, double* sb, double& mub) {
  const double rho = w[0], u = w[1], v = w[2], e = w[3];
  const double p = (gamma - 1.0) * rho * e;
  const double E = rho * (e + 0.5 * (u * u + v * v));
  const double txx = 4.0 / 3.0 * s[0] - 2.0 / 3.0 * s[3];
  const double txy = s[1] + s[2];
  const double tyy = 4.0 / 3.0 * s[3] - 2.0 / 3.0 * s[0];
  double rb = 0, ub = 0, vb = 0, eb = 0, pb, Eb, txxb = 0, txyb = 0, tyyb = 0;
  if (dir == 0) {
    const double m = rho * u;
    const double mb = fb[0] + fb[1] * u + fb[2] * v;
    ub += fb[1] * m + fb[3] * (E + p) - fb[3] * txx * rRe;
    vb += fb[2] * m - fb[3] * txy * rRe;
    pb = fb[1] + fb[3] * u;
    Eb = fb[3] * u;
    txxb = -fb[1] * rRe - fb[3] * u * rRe;
    txyb = -fb[2] * rRe - fb[3] * v * rRe;
    sb[4] += -fb[3] * gamma * rPr * rRe;
    mub += -fb[1] * txx - fb[2] * txy - fb[3] * (txx * u + txy * v + gamma * s[4] * rPr);
    rb += mb * u;
    ub += mb * rho;
  } else {
    const double n = rho * v;
    const double nb = fb[0] + fb[1] * u + fb[2] * v;
    ub += fb[1] * n - fb[3] * txy * rRe;
    vb += fb[2] * n + fb[3] * (E + p) - fb[3] * tyy * rRe;
    pb = fb[2] + fb[3] * v;
    Eb = fb[3] * v;
    txyb = -fb[1] * rRe - fb[3] * u * rRe;
    tyyb = -fb[2] * rRe - fb[3] * v * rRe;
    sb[5] += -fb[3] * gamma * rPr * rRe;
    mub += -fb[1] * txy - fb[2] * tyy - fb[3] * (txy * u + tyy * v + gamma * s[5] * rPr);
    rb += nb * v;
    vb += nb * rho;
  }
  rb += pb * (gamma - 1.0) * e;
  eb += pb * (gamma - 1.0) * rho;
  rb += Eb * (e + 0.5 * (u * u + v * v));
  eb += Eb * rho;
  ub += Eb * rho * u;
  vb += Eb * rho * v;
  sb[0] += 4.0 / 3.0 * txxb - 2.0 / 3.0 * tyyb;
  sb[3] += -2.0 / 3.0 * txxb + 4.0 / 3.0 * tyyb;
  sb[1] += txyb;
  sb[2] += txyb;
  wb[0] += rb;
  wb[1] += ub;
  wb[2] += vb;
  wb[3] += eb;
}

// wave_bound adjoint on the branch the forward took: given bbar, accumulate
__device__ __forceinline__ void wave_bound_T(int dir, const double* w, const double* s, double gamma, double rPr,
                                             double rRe, double bb, double* wb, double* sb, double& mub) {
  const double rho = w[0], e = w[3];
  const double p = (gamma - 1.0) * rho * e;
  const double cs = sqrt(gamma * (gamma - 1.0) * e);
  const double txx = 4.0 / 3.0 * s[0] - 2.0 / 3.0 * s[3];
  const double txy = s[1] + s[2];
  const double tyy = 4.0 / 3.0 * s[3] - 2.0 / 3.0 * s[0];
  const double un = dir == 0 ? w[1] : w[2];
  double q, s1, s2;
  if (dir == 0) { q = gamma * s[4] * rPr * rRe; s1 = txx * rRe - p; s2 = txy * rRe; }
  else { q = gamma * s[5] * rPr * rRe; s1 = txy * rRe; s2 = tyy * rRe - p; }
  const double r2e = rho * rho * e;
  const double S = s1 * s1 + s2 * s2;
  const double X = rho * rho * q * q + 2.0 * r2e * S;
  const double sq = sqrt(X);
  const double A = sq + rho * fabs(q), Bd = 2.0 * r2e;
  const double pp = fabs(un) + A / Bd;
  const double ac = fabs(un) + cs;
  const double unb = bb * sgn(un);
  if (dir == 0) wb[1] += unb; else wb[2] += unb;
  if (ac >= pp) {  // fmax(ac, pp) returned ac
    wb[3] += bb * gamma * (gamma - 1.0) / (2.0 * cs);
    return;
  }
  const double Ab = bb / Bd, Bdb = -bb * A / (Bd * Bd);
  const double Xb = X > 0.0 ? Ab / (2.0 * sq) : 0.0;
  double rb = Ab * fabs(q) + Xb * 2.0 * rho * q * q;
  double qb = Ab * rho * sgn(q) + Xb * 2.0 * rho * rho * q;
  double r2eb = Xb * 2.0 * S + Bdb * 2.0;
  const double Sb = Xb * 2.0 * r2e;
  rb += r2eb * 2.0 * rho * e;
  double eb = r2eb * rho * rho;
  const double s1b = Sb * 2.0 * s1, s2b = Sb * 2.0 * s2;
  double pb = 0, txxb = 0, txyb = 0, tyyb = 0;
  if (dir == 0) {
    txxb += s1b * rRe; mub += s1b * txx; pb -= s1b;
    txyb += s2b * rRe; mub += s2b * txy;
    sb[4] += qb * gamma * rPr * rRe; mub += qb * gamma * s[4] * rPr;
  } else {
    txyb += s1b * rRe; mub += s1b * txy;
    tyyb += s2b * rRe; mub += s2b * tyy; pb -= s2b;
    sb[5] += qb * gamma * rPr * rRe; mub += qb * gamma * s[5] * rPr;
  }
  rb += pb * (gamma - 1.0) * e;
  eb += pb * (gamma - 1.0) * rho;
  sb[0] += 4.0 / 3.0 * txxb - 2.0 / 3.0 * tyyb;
  sb[3] += -2.0 / 3.0 * txxb + 4.0 / 3.0 * tyyb;
  sb[1] += txyb;
  sb[2] += txyb;
  wb[0] += rb;
  wb[3] += eb;
}

// ---------------------------------------------------------------------------
// adjoints of the point evaluations (linear maps of the 15 coefficients)
__device__ __forceinline__ void line3_T(const double* ob, double* ab) {
  const double g = GN, g2 = g * g;
  const double evb = ob[0] + ob[2], odb = ob[2] - ob[0];
  ab[0] += evb + ob[1];
  ab[2] += evb * g2;
  ab[4] += evb * g2 * g2;
  ab[1] += odb * g;
  ab[3] += odb * g * g2;
}
__device__ __forceinline__ void collapse_x_T(double h, const double* Eb, const double* Ob, double* cb) {
  const double h2 = h * h;
  cb[0] += Eb[0]; cb[3] += Eb[0] * h2; cb[10] += Eb[0] * h2 * h2;
  cb[1] += Ob[0] * h; cb[6] += Ob[0] * h * h2;
  cb[2] += Eb[1]; cb[7] += Eb[1] * h2;
  cb[4] += Ob[1] * h; cb[11] += Ob[1] * h * h2;
  cb[5] += Eb[2]; cb[12] += Eb[2] * h2;
  cb[8] += Ob[2] * h;
  cb[9] += Eb[3];
  cb[13] += Ob[3] * h;
  cb[14] += Eb[4];
}
__device__ __forceinline__ void collapse_y_T(double h, const double* Eb, const double* Ob, double* cb) {
  const double h2 = h * h;
  cb[0] += Eb[0]; cb[5] += Eb[0] * h2; cb[14] += Eb[0] * h2 * h2;
  cb[2] += Ob[0] * h; cb[9] += Ob[0] * h * h2;
  cb[1] += Eb[1]; cb[8] += Eb[1] * h2;
  cb[4] += Ob[1] * h; cb[13] += Ob[1] * h * h2;
  cb[3] += Eb[2]; cb[12] += Eb[2] * h2;
  cb[7] += Ob[2] * h;
  cb[6] += Eb[3];
  cb[11] += Ob[3] * h;
  cb[10] += Eb[4];
}
// pair of lines (minus, plus) back to even/odd parts
__device__ __forceinline__ void pm_T(const double* am, const double* ap, double* Eb, double* Ob) {
#pragma unroll
  for (int q = 0; q < 4; q++) {
    Eb[q] = am[q] + ap[q];
    Ob[q] = ap[q] - am[q];
  }
  Eb[4] = am[4] + ap[4];
}
__device__ __forceinline__ void eval_xfaces_T(const double* ob, double* cb) {
  double am[5] = {0, 0, 0, 0, 0}, ap[5] = {0, 0, 0, 0, 0}, Eb[5], Ob[4];
  line3_T(ob, am);
  line3_T(ob + 3, ap);
  pm_T(am, ap, Eb, Ob);
  collapse_x_T(0.5, Eb, Ob, cb);
}
__device__ __forceinline__ void eval_yfaces_T(const double* ob, double* cb) {
  double am[5] = {0, 0, 0, 0, 0}, ap[5] = {0, 0, 0, 0, 0}, Eb[5], Ob[4];
  line3_T(ob, am);
  line3_T(ob + 3, ap);
  pm_T(am, ap, Eb, Ob);
  collapse_y_T(0.5, Eb, Ob, cb);
}
__device__ __forceinline__ void eval_vol_T(const double* ob, double* cb) {
  double am[5] = {0, 0, 0, 0, 0}, ac[5] = {0, 0, 0, 0, 0}, ap[5] = {0, 0, 0, 0, 0}, Eb[5], Ob[4];
  line3_T(ob, am);
  line3_T(ob + 3, ac);
  line3_T(ob + 6, ap);
  cb[0] += ac[0]; cb[2] += ac[1]; cb[5] += ac[2]; cb[9] += ac[3]; cb[14] += ac[4];
  pm_T(am, ap, Eb, Ob);
  collapse_x_T(GN, Eb, Ob, cb);
}

// ---------------------------------------------------------------------------
// adjoint of hweno_combine_coeffs<double> (the product form of the weights).  Takes the
// forward's beta_0 and reciprocal rs = 1/S' (as the forward recorded them) and the
// gradient gr = d beta_0 / d c0; recomputes the rest of the weights from (c0, s, ctr);
// given Cbar accumulates c0b, sb, ctrb.
__device__ __forceinline__ void hweno_combine_T(const double* c0, const double* s, double ctr, double eps,
                                                double b0, double rs, const double* gr, const double* Cb,
                                                double* c0b, double* sb, double& ctrb) {
  const double dxm = s[0], dxp = s[1], dym = s[2], dyp = s[3];
  const double b[5] = {b0, dxm * dxm + dym * dym, dxp * dxp + dym * dym, dxm * dxm + dyp * dyp, dxp * dxp + dyp * dyp};
  double e[5];
  for (int m = 1; m < 5; m++) e[m] = b0 - b[m];
  const double ts = 0.25 * (fabs(e[1]) + fabs(e[2]) + fabs(e[3]) + fabs(e[4]));
  const double tau = ts * ts;
  double D[5];
  for (int m = 0; m < 5; m++) D[m] = b[m] + eps;
  const double D12 = D[1] * D[2], D34 = D[3] * D[4];
  const double R[5] = {0.0, D[2] * D34, D[1] * D34, D12 * D[4], D12 * D[3]};
  const double Q0 = D12 * D34, P = D[0] * Q0;
  const double SR = (R[1] + R[2]) + (R[3] + R[4]);
  const double a0 = (P + tau * Q0) * rs;
  const double g = GAML * tau * rs;
  double a[5];
  for (int m = 1; m < 5; m++) a[m] = g * R[m] * e[m];
  const double A1 = a[1] + a[3], A2 = a[2] + a[4], A3 = a[1] + a[2], A4 = a[3] + a[4];
  // reverse of C = a0 c0 (+ (1 - a0) ctr at k = 0) + slope terms
  double a0b = 0.0;
  for (int k = 0; k < 15; k++) {
    c0b[k] += a0 * Cb[k];
    a0b += Cb[k] * c0[k];
  }
  a0b -= Cb[0] * ctr;
  ctrb += (1.0 - a0) * Cb[0];
  const double A1b = Cb[1] * dxm, A2b = Cb[1] * dxp, A3b = Cb[2] * dym, A4b = Cb[2] * dyp;
  double sbl[4] = {Cb[1] * A1, Cb[1] * A2, Cb[2] * A3, Cb[2] * A4};
  double ab[5] = {0.0, A1b + A3b, A2b + A3b, A1b + A4b, A2b + A4b};
  // weights
  double gb = 0.0, Rb[5] = {0, 0, 0, 0, 0}, eb[5] = {0, 0, 0, 0, 0};
  for (int m = 1; m < 5; m++) {
    gb += ab[m] * R[m] * e[m];
    Rb[m] += ab[m] * g * e[m];
    eb[m] += ab[m] * g * R[m];
  }
  double taub = gb * GAML * rs, rsb = gb * GAML * tau;
  double Pb = a0b * rs, Q0b = a0b * tau * rs;
  taub += a0b * Q0 * rs;
  rsb += a0b * (P + tau * Q0);
  const double Spb = -rsb * rs * rs;
  Pb += Spb;
  taub += Spb * (GAM0 * Q0 + GAML * D[0] * SR);
  Q0b += Spb * tau * GAM0;
  double Db[5] = {0, 0, 0, 0, 0};
  Db[0] += Spb * tau * GAML * SR;
  const double SRb = Spb * tau * GAML * D[0];
  for (int m = 1; m < 5; m++) Rb[m] += SRb;
  Db[0] += Pb * Q0;
  Q0b += Pb * D[0];
  double D12b = Q0b * D34, D34b = Q0b * D12;
  Db[2] += Rb[1] * D34; D34b += Rb[1] * D[2];
  Db[1] += Rb[2] * D34; D34b += Rb[2] * D[1];
  D12b += Rb[3] * D[4]; Db[4] += Rb[3] * D12;
  D12b += Rb[4] * D[3]; Db[3] += Rb[4] * D12;
  Db[1] += D12b * D[2]; Db[2] += D12b * D[1];
  Db[3] += D34b * D[4]; Db[4] += D34b * D[3];
  double bb[5];
  for (int m = 0; m < 5; m++) bb[m] = Db[m];
  const double tsb = 2.0 * ts * taub;
  for (int m = 1; m < 5; m++) {
    eb[m] += 0.25 * tsb * sgn(e[m]);
    bb[0] += eb[m];
    bb[m] -= eb[m];
  }
  const double sxmb = bb[1] + bb[3], sxpb = bb[2] + bb[4], symb = bb[1] + bb[2], sypb = bb[3] + bb[4];
  sb[0] += sbl[0] + 2.0 * dxm * sxmb;
  sb[1] += sbl[1] + 2.0 * dxp * sxpb;
  sb[2] += sbl[2] + 2.0 * dym * symb;
  sb[3] += sbl[3] + 2.0 * dyp * sypb;
  for (int k = 0; k < 15; k++) c0b[k] += bb[0] * gr[k];
}

// ---------------------------------------------------------------------------
// characteristic maps: adjoints with respect to the vector and to the state parameters
struct CharBar {
  double u, v, c, H, hq2, hb1, hb2, hrc;
};

// The state-parameter parts of the map adjoints are bilinear in (vector, adjoint): each
// call adds to a few sums, and char_sums_finish turns the sums of one direction into
// CharBar once.
struct CharSums {
  // to_char: sum Bh x0, Bh xn, Ah x0, Ah x3, Ah xn, Ah xt, yb2 x0  (Ah = A/2 adjoint, Bh = B/2)
  double B0, Bn, A0, A3, An, At, Y20;
  // from_char: sum x3b (y0 + y3), x3b dd, xnb dd, x3b y1, xnb x0, x3b y2, xtb x0
  double H, X3d, Xnd, X31, Xn0, X32, Xt0;
};

template <int DIR>
__device__ __forceinline__ void to_char_T(const CharState<double>& s, const double* x, const double* yb, double* xb,
                                          CharSums& m) {
  const double un = DIR == 0 ? s.u : s.v, ut = DIR == 0 ? s.v : s.u;
  const double xn = DIR == 0 ? x[1] : x[2], xt = DIR == 0 ? x[2] : x[1];
  const double Ahb = yb[0] - 2.0 * yb[1] + yb[3];
  const double Bhb = yb[0] - yb[3];
  const double bh = Bhb * s.hrc, ah = Ahb * s.hb1;
  xb[0] += (yb[1] - yb[2] * ut) + bh * un + Ahb * s.hb2;
  xb[DIR == 0 ? 1 : 2] += -bh - ah * un;
  xb[DIR == 0 ? 2 : 1] += yb[2] - ah * ut;
  xb[3] += ah;
  m.B0 += Bhb * x[0];
  m.Bn += Bhb * xn;
  m.A0 += Ahb * x[0];
  m.A3 += Ahb * x[3];
  m.An += Ahb * xn;
  m.At += Ahb * xt;
  m.Y20 += yb[2] * x[0];
}

template <int DIR>
__device__ __forceinline__ void from_char_T(const CharState<double>& s, const double* y, const double* xbar,
                                            double* yb, CharSums& m) {
  const double un = DIR == 0 ? s.u : s.v, ut = DIR == 0 ? s.v : s.u;
  const double x0 = y[0] + y[1] + y[3];
  const double dd = y[3] - y[0];
  const double x3b = xbar[3], xnb = xbar[DIR == 0 ? 1 : 2], xtb = xbar[DIR == 0 ? 2 : 1];
  // x0 = y0 + y1 + y3, xn = un x0 + c dd, xt = ut x0 + y2,
  // x3 = H (y0 + y3) + un c dd + hq2 y1 + ut y2
  const double ddb = s.c * (x3b * un + xnb);
  const double x0b = xbar[0] + xtb * ut + xnb * un;
  const double hb = x3b * s.H;
  yb[0] += hb - ddb + x0b;
  yb[3] += hb + ddb + x0b;
  yb[1] += x3b * s.hq2 + x0b;
  yb[2] += x3b * ut + xtb;
  m.H += x3b * (y[0] + y[3]);
  m.X3d += x3b * dd;
  m.Xnd += xnb * dd;
  m.X31 += x3b * y[1];
  m.Xn0 += xnb * x0;
  m.X32 += x3b * y[2];
  m.Xt0 += xtb * x0;
}

template <int DIR>
__device__ __forceinline__ void char_sums_finish(const CharState<double>& s, const CharSums& m, CharBar& sb) {
  const double un = DIR == 0 ? s.u : s.v, ut = DIR == 0 ? s.v : s.u;
  sb.hrc += un * m.B0 - m.Bn;
  sb.hb2 += m.A0;
  sb.hb1 += m.A3 - un * m.An - ut * m.At;
  sb.H += m.H;
  sb.c += un * m.X3d + m.Xnd;
  sb.hq2 += m.X31;
  const double unb = s.hrc * m.B0 - s.hb1 * m.An + s.c * m.X3d + m.Xn0;
  const double utb = -m.Y20 - s.hb1 * m.At + m.X32 + m.Xt0;
  if (DIR == 0) { sb.u += unb; sb.v += utb; }
  else { sb.v += unb; sb.u += utb; }
}

// adjoint of pp_limit in a cell where it acted (thr < 1 or thp < 1).  ub: the cell
// average; fu, vu: the unlimited face and volume values (conserved); thr, thp: the
// forward's factors.  Given Fb, the adjoint of the limited face values, writes fb, the
// adjoint of the unlimited face values, and accumulates vb (volume values) and ubb
// (average).  Ties go to the first point, as in the forward's strict comparisons.
__device__ void pp_limit_T(const double* ub, const double (*fu)[4], const double (*vu)[4], double gamma,
                           double eps_pp, double thr, double thp, const double (*Fb)[4], double (*fb)[4],
                           double (*vb)[4], double* ubb) {
  const double gm1 = gamma - 1.0;
  const double pb = pressure(ub, gamma);
  // eps = min(eps_pp, rho_bar, p_bar) and the term that set it
  double eps = eps_pp;
  int esrc = 0;
  if (ub[0] < eps) { eps = ub[0]; esrc = 1; }
  if (pb < eps) { eps = pb; esrc = 2; }
  // the face map: f~0 = ub0 + thp thr (f0 - ub0), f~v = ubv + thp (fv - ubv)
  const double A = thp * thr;
  double thpb = 0.0, thrb = 0.0, epsb = 0.0;
  for (int k = 0; k < 12; k++) {
    const double d0 = fu[k][0] - ub[0];
    fb[k][0] = A * Fb[k][0];
    ubb[0] += (1.0 - A) * Fb[k][0];
    thpb += thr * d0 * Fb[k][0];
    thrb += thp * d0 * Fb[k][0];
    for (int v = 1; v < 4; v++) {
      fb[k][v] = thp * Fb[k][v];
      ubb[v] += (1.0 - thp) * Fb[k][v];
      thpb += (fu[k][v] - ub[v]) * Fb[k][v];
    }
  }
  // pressure factor: the smallest root t* over the points below eps, with the density
  // already rescaled; P(t) = U3 U0 - |U12|^2/2 - e1 U0 at U = ub + t (w - ub)
  if (thp < 1.0) {
    int ks = -1;
    double tmin = 1.0;
    for (int k = 0; k < 21; k++) {
      const double* sp = k < 12 ? fu[k] : vu[k - 12];
      const double wv[4] = {ub[0] + thr * (sp[0] - ub[0]), sp[1], sp[2], sp[3]};
      const double lhs = gm1 * (wv[3] * wv[0] - 0.5 * (wv[1] * wv[1] + wv[2] * wv[2]));
      if (lhs < eps * wv[0]) {
        const double t = theta_root(ub, wv, eps, gamma);
        if (t < tmin) { tmin = t; ks = k; }
      }
    }
    if (ks >= 0 && tmin > 0.0 && tmin < 1.0) {
      const double* sp = ks < 12 ? fu[ks] : vu[ks - 12];
      const double wv[4] = {ub[0] + thr * (sp[0] - ub[0]), sp[1], sp[2], sp[3]};
      const double e1 = eps / gm1;
      double U[4], dP[4], dPdt = 0.0;
      for (int v = 0; v < 4; v++) U[v] = ub[v] + tmin * (wv[v] - ub[v]);
      dP[0] = U[3] - e1;
      dP[1] = -U[1];
      dP[2] = -U[2];
      dP[3] = U[0];
      for (int v = 0; v < 4; v++) dPdt += dP[v] * (wv[v] - ub[v]);
      const double G = -thpb / dPdt;
      double wb[4];
      for (int v = 0; v < 4; v++) {
        ubb[v] += G * (1.0 - tmin) * dP[v];
        wb[v] = G * tmin * dP[v];
      }
      epsb += -G * U[0] / gm1;
      // w0 = ub0 + thr (s0 - ub0)
      ubb[0] += (1.0 - thr) * wb[0];
      thrb += (sp[0] - ub[0]) * wb[0];
      double* sb = ks < 12 ? fb[ks] : vb[ks - 12];
      sb[0] += thr * wb[0];
      for (int v = 1; v < 4; v++) sb[v] += wb[v];
    }
  }
  // density factor thr = (ub0 - eps) / (ub0 - rmin) at the point of minimum density
  if (thr < 1.0) {
    int km = -1;
    double rmin = ub[0];
    for (int k = 0; k < 12; k++)
      if (fu[k][0] < rmin) { rmin = fu[k][0]; km = k; }
    for (int k = 0; k < 9; k++)
      if (vu[k][0] < rmin) { rmin = vu[k][0]; km = 12 + k; }
    if (km >= 0) {
      const double D = ub[0] - rmin;
      ubb[0] += thrb * (eps - rmin) / (D * D);
      epsb += -thrb / D;
      const double rb = thrb * (ub[0] - eps) / (D * D);
      if (km < 12) fb[km][0] += rb;
      else vb[km - 12][0] += rb;
    }
  }
  // eps = min(eps_pp, rho_bar, p_bar)
  if (esrc == 1) {
    ubb[0] += epsb;
  } else if (esrc == 2) {
    const double u = ub[1] / ub[0], v = ub[2] / ub[0];
    ubb[0] += epsb * gm1 * 0.5 * (u * u + v * v);
    ubb[1] -= epsb * gm1 * u;
    ubb[2] -= epsb * gm1 * v;
    ubb[3] += epsb * gm1;
  }
}

// adjoint of char_state: accumulate ubar
__device__ __forceinline__ void char_state_T(const double* ub, double gamma, const CharBar& sb, double* ubb) {
  const double rr = 1.0 / ub[0];
  const double u = ub[1] * rr, v = ub[2] * rr;
  const double hq2 = 0.5 * (u * u + v * v);
  const double p = (gamma - 1.0) * (ub[3] - ub[0] * hq2);
  const double c2 = gamma * p * rr;
  const double c = sqrt(c2);
  const double hb1 = 0.5 * (gamma - 1.0) / c2;
  double cb = sb.c + sb.hrc * (-0.5 / (c * c));
  const double hb1b = sb.hb1 + sb.hb2 * hq2;
  double hq2b = sb.hq2 + sb.hb2 * hb1;
  double c2b = hb1b * (-0.5 * (gamma - 1.0) / (c2 * c2)) + cb / (2.0 * c);
  double Eb = sb.H * rr;
  double pb = sb.H * rr + c2b * gamma * rr;
  double rrb = sb.H * (ub[3] + p) + c2b * gamma * p;
  Eb += pb * (gamma - 1.0);
  double rhob = -pb * (gamma - 1.0) * hq2;
  hq2b += -pb * (gamma - 1.0) * ub[0];
  const double uu = sb.u + hq2b * u, vv = sb.v + hq2b * v;
  ubb[1] += uu * rr;
  ubb[2] += vv * rr;
  rrb += uu * ub[1] + vv * ub[2];
  rhob += -rrb * rr * rr;
  ubb[0] += rhob;
  ubb[3] += Eb;
}

// ---------------------------------------------------------------------------
// reverse kernels (regions as the forward kernels; see hweno_ops.cuh)

// volume part of the assembly (interior cells): the volume fluxes' adjoints
__global__ void __launch_bounds__(128) ka_assemble(Grid g, Work w, Adj a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  double mub = 0.0;
  if (i < g.nx && j < g.ny) {
    const long long c = cidx(g, i, j);
    const double rdx = g.rdx, rdy = g.rdy, rPr = g.rPr, rRe = g.rRe;
    double Rb1[4], Rb2[4];
    for (int v = 0; v < 4; v++) {
      Rb1[v] = a.R[(long long)(4 + v) * g.ps + c];
      Rb2[v] = a.R[(long long)(8 + v) * g.ps + c];
    }
    for (int G = 0; G < 3; G++)
      for (int H = 0; H < 3; H++) {
        const int k = 3 * G + H;
        double st[4], gs[6], wb[4] = {0, 0, 0, 0}, sb[6] = {0, 0, 0, 0, 0, 0}, fb[4], hb[4];
        for (int v = 0; v < 4; v++) st[v] = w.vol[(long long)(4 * k + v) * g.ps + c];
        for (int n = 0; n < 6; n++) gs[n] = w.gr[(long long)(6 * (12 + k) + n) * g.ps + c];
        const double wgt = gweight<double>(G) * gweight<double>(H);
        for (int v = 0; v < 4; v++) {
          fb[v] = wgt * Rb1[v] * rdx;
          hb[v] = wgt * Rb2[v] * rdy;
        }
        phys_flux_T(0, st, gs, g.gamma, rPr, rRe, fb, wb, sb, mub);
        phys_flux_T(1, st, gs, g.gamma, rPr, rRe, hb, wb, sb, mub);
        for (int v = 0; v < 4; v++) a.vol[(long long)(4 * k + v) * g.ps + c] = wb[v];
        for (int n = 0; n < 6; n++) a.gr[(long long)(6 * (12 + k) + n) * g.ps + c] = sb[n];
      }
  }
  mub = warp_sum_d(mub);
  if (lane_id() == 0 && mub != 0.0) atomicAdd(a.mu, mub);
}

// face fluxes: seeds of the face Gauss sums from the two adjacent cells' residual
// adjoints, then the PP-LLF flux and its coefficient beta
__global__ void __launch_bounds__(128) ka_flux(Grid g, Work w, Adj a) {
  const int dir = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x - (dir == 0 ? 1 : 0);
  const int j = blockIdx.y * blockDim.y + threadIdx.y - (dir == 0 ? 0 : 1);
  double mub = 0.0;
  if (i < g.nx && j < g.ny) {
    const long long cl = cidx(g, i, j);
    const long long cr = dir == 0 ? cidx(g, i + 1, j) : cidx(g, i, j + 1);
    const bool inL = i >= 0 && j >= 0;
    const bool inR = dir == 0 ? (i + 1 < g.nx) : (j + 1 < g.ny);
    const double r = dir == 0 ? g.rdx : g.rdy;
    // S0/S1 seeds: x-face: r0 (-r, +r), r1 (-r/2 both), r2 via S1 (-r, +r);
    //              y-face: r0 (-r, +r), r2 (-r/2 both), r1 via S1 (-r, +r)
    const int kh = dir == 0 ? 1 : 2, ks = dir == 0 ? 2 : 1;
    double S0b[4], S1b[4];
    for (int v = 0; v < 4; v++) {
      double s0 = 0.0, s1 = 0.0;
      if (inL) {
        s0 += -r * a.R[(long long)v * g.ps + cl] - 0.5 * r * a.R[(long long)(4 * kh + v) * g.ps + cl];
        s1 += -r * a.R[(long long)(4 * ks + v) * g.ps + cl];
      }
      if (inR) {
        s0 += r * a.R[(long long)v * g.ps + cr] - 0.5 * r * a.R[(long long)(4 * kh + v) * g.ps + cr];
        s1 += r * a.R[(long long)(4 * ks + v) * g.ps + cr];
      }
      S0b[v] = s0;
      S1b[v] = s1;
    }
    const int kl = dir == 0 ? 3 : 9, kr = dir == 0 ? 0 : 6;
    const double gam = g.gamma, rPr = g.rPr, rRe = g.rRe;
    double st[2][3][4], gs[2][3][6];
    for (int gp = 0; gp < 3; gp++)
      for (int s = 0; s < 2; s++) {
        const long long cc = s == 0 ? cl : cr;
        const int k = (s == 0 ? kl : kr) + gp;
        for (int v = 0; v < 4; v++) st[s][gp][v] = w.face[(long long)(4 * k + v) * g.ps + cc];
        for (int n = 0; n < 6; n++) gs[s][gp][n] = w.gr[(long long)(6 * k + n) * g.ps + cc];
      }
    double beta = 0.0;
    int as = 0, ag = 0;
    for (int gp = 0; gp < 3; gp++)
      for (int s = 0; s < 2; s++) {
        const double bnd = wave_bound<double>(dir, st[s][gp], gs[s][gp], gam, rPr, rRe);
        if (bnd > beta) { beta = bnd; as = s; ag = gp; }
      }
    double wb[2][3][4], sb[2][3][6];
    for (int s = 0; s < 2; s++)
      for (int gp = 0; gp < 3; gp++) {
        for (int v = 0; v < 4; v++) wb[s][gp][v] = 0.0;
        for (int n = 0; n < 6; n++) sb[s][gp][n] = 0.0;
      }
    double betab = 0.0;
    for (int gp = 0; gp < 3; gp++) {
      const double wg = gweight<double>(gp), wt = gweight<double>(gp) * gnode<double>(gp);
      double fhb[4], fb[4], Ub[4];
      for (int v = 0; v < 4; v++) fhb[v] = wg * S0b[v] + (gp != 1 ? wt * S1b[v] : 0.0);
      double U[2][4];
      for (int s = 0; s < 2; s++) {
        const double* p = st[s][gp];
        U[s][0] = p[0];
        U[s][1] = p[0] * p[1];
        U[s][2] = p[0] * p[2];
        U[s][3] = p[0] * (p[3] + 0.5 * (p[1] * p[1] + p[2] * p[2]));
      }
      for (int v = 0; v < 4; v++) betab += -0.5 * fhb[v] * (U[1][v] - U[0][v]);
      for (int s = 0; s < 2; s++) {
        for (int v = 0; v < 4; v++) {
          fb[v] = 0.5 * fhb[v];
          Ub[v] = (s == 0 ? 0.5 : -0.5) * beta * fhb[v];
        }
        phys_flux_T(dir, st[s][gp], gs[s][gp], gam, rPr, rRe, fb, wb[s][gp], sb[s][gp], mub);
        cons_T(st[s][gp], Ub, wb[s][gp]);
      }
    }
    wave_bound_T(dir, st[as][ag], gs[as][ag], gam, rPr, rRe, betab, wb[as][ag], sb[as][ag], mub);
    for (int gp = 0; gp < 3; gp++)
      for (int s = 0; s < 2; s++) {
        const long long cc = s == 0 ? cl : cr;
        const int k = (s == 0 ? kl : kr) + gp;
        for (int v = 0; v < 4; v++) a.face[(long long)(4 * k + v) * g.ps + cc] = wb[s][gp][v];
        for (int n = 0; n < 6; n++) a.gr[(long long)(6 * k + n) * g.ps + cc] = sb[s][gp][n];
      }
  }
  mub = warp_sum_d(mub);
  if (lane_id() == 0 && mub != 0.0) atomicAdd(a.mu, mub);
}

// gradient HWENO (cells of the interior grown by 1): per field, the adjoint of the
// combination, written as contributions to the 17 stencil data.  LIN: the linear
// weights of Remark 3.1's ablation, whose combination is p0 itself (C = P0 d), so the
// adjoint is P0^T applied to the coefficients' adjoint
template <bool LIN = false>
__global__ void __launch_bounds__(128) ka_grad(Grid g, Work w, Adj a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 1;
  const int j = blockIdx.y * blockDim.y + threadIdx.y - 1;
  if (i >= g.nx + 1 || j >= g.ny + 1) return;
  const long long c = cidx(g, i, j);
  for (int comp = 0; comp < 6; comp++) {
    const int n = comp >> 1, l = comp & 1;
    const double* A = w.rm + (long long)(6 * n + 3 * l) * g.ps;
    // the 5-point stencil of the averages for the slopes; p0 coefficients and weight
    // factors as the forward wrote them
    double d[17];
    d[1] = A[cidx(g, i, j - 1)];
    d[3] = A[cidx(g, i - 1, j)];
    d[4] = A[c];
    d[5] = A[cidx(g, i + 1, j)];
    d[7] = A[cidx(g, i, j + 1)];
    double ob[21];
    for (int k = 0; k < 21; k++) ob[k] = a.gr[(long long)(6 * k + comp) * g.ps + c];
    double Cb[15] = {0};
    eval_xfaces_T(ob, Cb);
    eval_yfaces_T(ob + 6, Cb);
    eval_vol_T(ob + 12, Cb);
    double c0b[15] = {0}, sb[4] = {0, 0, 0, 0}, ctrb = 0.0;
    if constexpr (LIN) {
      for (int k = 0; k < 15; k++) c0b[k] = Cb[k];
    } else {
      const double* y = w.yrec + (long long)(YREC_GR + 17 * comp) * g.ps + c;
      double c0[15];
      for (int k = 0; k < 15; k++) c0[k] = y[(long long)k * g.ps];
      const double b0 = y[(long long)15 * g.ps], rs = y[(long long)16 * g.ps];
      const double s[4] = {d[4] - d[3], d[5] - d[4], d[4] - d[1], d[7] - d[4]};
      double gr[15];
      hw_beta_quartic_grad<double>(c0, gr);
      hweno_combine_T(c0, s, d[4], g.eps_weno, b0, rs, gr, Cb, c0b, sb, ctrb);
    }
    double db[17] = {0};
    hw_p0_coeffs_T<double>(c0b, db);
    db[4] += ctrb + sb[0] - sb[1] + sb[2] - sb[3];
    db[3] -= sb[0];
    db[5] += sb[1];
    db[1] -= sb[2];
    db[7] += sb[3];
    for (int k = 0; k < 17; k++) a.cg[(long long)(17 * comp + k) * g.ps + c] = db[k];
  }
}

// gather of stencil contributions (17 slots of the 3x3 stencil of hweno_stencil.h) into
// the adjoint of one (average, xi-moment, eta-moment) triple of planes.  src: the
// contribution planes of the field, dst: [avg, xi, eta] planes, region of producing
// cells [lo, hi) in both directions (offsets from the interior), consumer region
// grown by one.
__device__ __forceinline__ double gather_avg(const Grid& g, const double* src, int i, int j, int lo, int hix, int hiy) {
  double s = 0.0;
  for (int b = -1; b <= 1; b++)
    for (int aa = -1; aa <= 1; aa++) {
      // producer k = (i - aa, j - b) sees this cell at offset (aa, b)
      const int ki = i - aa, kj = j - b;
      if (ki < lo || kj < lo || ki >= hix || kj >= hiy) continue;
      s += src[(long long)((b + 1) * 3 + (aa + 1)) * g.ps + cidx(g, ki, kj)];
    }
  return s;
}
__device__ __forceinline__ double gather_one(const Grid& g, const double* src, int slot, int ki, int kj, int lo,
                                             int hix, int hiy) {
  if (ki < lo || kj < lo || ki >= hix || kj >= hiy) return 0.0;
  return src[(long long)slot * g.ps + cidx(g, ki, kj)];
}
// xi-moments are read by producers (i+1, j) slot 9, (i-1, j) slot 10, (i, j+1) slot 13,
// (i, j-1) slot 14; eta-moments by (i, j+1) slot 11, (i, j-1) slot 12, (i+1, j) slot 15,
// (i-1, j) slot 16
__device__ __forceinline__ void gather_triple(const Grid& g, const double* src, int i, int j, int lo, int hix,
                                              int hiy, double& avg, double& xi, double& eta) {
  avg = gather_avg(g, src, i, j, lo, hix, hiy);
  xi = gather_one(g, src, 9, i + 1, j, lo, hix, hiy) + gather_one(g, src, 10, i - 1, j, lo, hix, hiy) +
       gather_one(g, src, 13, i, j + 1, lo, hix, hiy) + gather_one(g, src, 14, i, j - 1, lo, hix, hiy);
  eta = gather_one(g, src, 11, i, j + 1, lo, hix, hiy) + gather_one(g, src, 12, i, j - 1, lo, hix, hiy) +
        gather_one(g, src, 15, i + 1, j, lo, hix, hiy) + gather_one(g, src, 16, i - 1, j, lo, hix, hiy);
}

// weak-moment adjoints of cells in the interior grown by 2, from ka_grad's contributions
__global__ void ka_gather_rm(Grid g, Adj a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 2;
  const int j = blockIdx.y * blockDim.y + threadIdx.y - 2;
  if (i >= g.nx + 2 || j >= g.ny + 2) return;
  const long long c = cidx(g, i, j);
  for (int comp = 0; comp < 6; comp++) {
    const int n = comp >> 1, l = comp & 1;
    double av, xi, eta;
    gather_triple(g, a.cg + (long long)17 * comp * g.ps, i, j, -1, g.nx + 1, g.ny + 1, av, xi, eta);
    double* r = a.rm + (long long)(6 * n + 3 * l) * g.ps + c;
    r[0] = av;
    r[g.ps] = xi;
    r[2 * g.ps] = eta;
  }
}

// face moments and weak moments: face-centric adjoint of W from the weak-moment
// adjoints of the two adjacent cells, then onto the face points' u, v, e
__global__ void ka_face_moments(Grid g, Adj a) {
  const int dir = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x - (dir == 0 ? 3 : 2);
  const int j = blockIdx.y * blockDim.y + threadIdx.y - (dir == 0 ? 2 : 3);
  if (i >= g.nx + 2 || j >= g.ny + 2) return;
  const long long cl = cidx(g, i, j);
  const long long cr = dir == 0 ? cidx(g, i + 1, j) : cidx(g, i, j + 1);
  // weak moments exist for cells of the interior grown by 2
  const bool inL = i >= -2 && j >= -2;
  const bool inR = dir == 0 ? (i + 1 < g.nx + 2) : (j + 1 < g.ny + 2);
  const double r = dir == 0 ? g.rdx : g.rdy;
  // x: r0 = (W0+ - W0-) r, r_xi = (W0+ + W0-)/2 r - wbar r, r_eta = (W1+ - W1-) r
  // y: r0 = (W0+ - W0-) r, r_xi = (W1+ - W1-) r, r_eta = (W0+ + W0-)/2 r - wbar r
  const int o0 = dir == 0 ? 0 : 3, oh = dir == 0 ? 1 : 5, o1 = dir == 0 ? 2 : 4;
  const int kl = dir == 0 ? 3 : 9, kr = dir == 0 ? 0 : 6;
  for (int n = 0; n < 3; n++) {
    double W0b = 0.0, W1b = 0.0;
    if (inL) {
      const double* rb = a.rm + (long long)(6 * n) * g.ps + cl;
      W0b += r * rb[(long long)o0 * g.ps] + 0.5 * r * rb[(long long)oh * g.ps];
      W1b += r * rb[(long long)o1 * g.ps];
    }
    if (inR) {
      const double* rb = a.rm + (long long)(6 * n) * g.ps + cr;
      W0b += -r * rb[(long long)o0 * g.ps] + 0.5 * r * rb[(long long)oh * g.ps];
      W1b += -r * rb[(long long)o1 * g.ps];
    }
    for (int gp = 0; gp < 3; gp++) {
      const double hb = 0.5 * gweight<double>(gp) * (W0b + gnode<double>(gp) * W1b);
      a.face[(long long)(4 * (kl + gp) + 1 + n) * g.ps + cl] += hb;
      a.face[(long long)(4 * (kr + gp) + 1 + n) * g.ps + cr] += hb;
    }
  }
}

// characteristic HWENO and primitives (cells of the interior grown by 3): contributions
// to the 17 stencil data of the four conserved variables
__global__ void __launch_bounds__(128) ka_cons(Grid g, const double* __restrict__ q, Work w, Adj a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x - 3;
  const int j = blockIdx.y * blockDim.y + threadIdx.y - 3;
  if (i < g.nx + 3 && j < g.ny + 3) {
    const long long c = cidx(g, i, j);
    // p0 coefficients as the forward wrote them; the slopes from the 5-point stencil
    double ub[4], cc[4][15], sl[4][4], ctr[4];
    for (int v = 0; v < 4; v++) {
      const double* Q = q + (long long)v * g.ps;
      const double dc = Q[c], dw = Q[cidx(g, i - 1, j)], de = Q[cidx(g, i + 1, j)];
      const double ds = Q[cidx(g, i, j - 1)], dn = Q[cidx(g, i, j + 1)];
      ub[v] = dc;
      for (int k = 0; k < 15; k++) cc[v][k] = w.yrec[(long long)(YREC_CC + 15 * v + k) * g.ps + c];
      sl[v][0] = dc - dw;
      sl[v][1] = de - dc;
      sl[v][2] = dc - ds;
      sl[v][3] = dn - dc;
      ctr[v] = dc;
    }
    CharState<double> cs;
    char_state<double>(ub, g.gamma, cs);
    const double eps = g.eps_weno;
    // adjoints of the conserved point values, from the stored primitive point values
    // (the face values are the limited ones)
    double fb[12][4], vb[9][4];
    for (int k = 0; k < 12; k++) {
      double wbp[4], wp[4];
      for (int v = 0; v < 4; v++) {
        wbp[v] = a.face[(long long)(4 * k + v) * g.ps + c];
        wp[v] = w.face[(long long)(4 * k + v) * g.ps + c];
        fb[k][v] = 0.0;
      }
      prim_T_w(wp, wbp, fb[k]);
    }
    // cell mean of u, v, e from the volume values feeds both weak moments
    const bool in2 = i >= -2 && j >= -2 && i < g.nx + 2 && j < g.ny + 2;
    double wbarb[3] = {0.0, 0.0, 0.0};
    if (in2)
      for (int n = 0; n < 3; n++)
        wbarb[n] = -a.rm[(long long)(6 * n + 1) * g.ps + c] * g.rdx - a.rm[(long long)(6 * n + 5) * g.ps + c] * g.rdy;
    for (int G = 0; G < 3; G++)
      for (int H = 0; H < 3; H++) {
        const int k = 3 * G + H;
        double wbp[4];
        for (int v = 0; v < 4; v++) {
          wbp[v] = a.vol[(long long)(4 * k + v) * g.ps + c];
          vb[k][v] = 0.0;
        }
        const double wgt = gweight<double>(G) * gweight<double>(H);
        for (int n = 0; n < 3; n++) wbp[1 + n] += wgt * wbarb[n];
        double wp[4];
        for (int v = 0; v < 4; v++) wp[v] = w.vol[(long long)(4 * k + v) * g.ps + c];
        prim_T_w(wp, wbp, vb[k]);
      }
    // where the limiter acted: from the limited to the unlimited face values, whose
    // conserved form is R y of the recorded characteristic values (as the forward
    // formed them); the volume values are unlimited
    double ubl[4] = {0, 0, 0, 0};
    const double thr = w.theta[c], thp = w.theta[g.ps + c];
    if (thr < 1.0 || thp < 1.0) {
      double fu[12][4], vu[9][4], Fb[12][4];
      for (int dir = 0; dir < 2; dir++)
        for (int k = 0; k < 6; k++) {
          double y[4];
          for (int f = 0; f < 4; f++) y[f] = w.yrec[(long long)(72 * dir + 18 * f + k) * g.ps + c];
          if (dir == 0) from_char<double, 0>(cs, y, fu[k]); else from_char<double, 1>(cs, y, fu[6 + k]);
        }
      for (int k = 0; k < 9; k++) {
        const double r = w.vol[(long long)(4 * k) * g.ps + c], u = w.vol[(long long)(4 * k + 1) * g.ps + c];
        const double v = w.vol[(long long)(4 * k + 2) * g.ps + c], e = w.vol[(long long)(4 * k + 3) * g.ps + c];
        vu[k][0] = r;
        vu[k][1] = r * u;
        vu[k][2] = r * v;
        vu[k][3] = r * (e + 0.5 * (u * u + v * v));
      }
      for (int k = 0; k < 12; k++)
        for (int v = 0; v < 4; v++) Fb[k][v] = fb[k][v];
      pp_limit_T(ub, fu, vu, g.gamma, g.eps_pp, thr, thp, Fb, fb, vb, ubl);
    }
    const bool interior = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
    double mb[2][4];
    for (int v = 0; v < 4; v++) {
      mb[0][v] = interior ? a.M[(long long)v * g.ps + c] : 0.0;
      mb[1][v] = interior ? a.M[(long long)(4 + v) * g.ps + c] : 0.0;
    }
    // reverse of the two directional reconstructions
    double ccb[4][15], slb[4][4], ctrb[4] = {0, 0, 0, 0}, ubb[4] = {0, 0, 0, 0};
    for (int v = 0; v < 4; v++) {
      for (int k = 0; k < 15; k++) ccb[v][k] = 0.0;
      for (int k = 0; k < 4; k++) slb[v][k] = 0.0;
    }
    CharBar sb = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int dir = 0; dir < 2; dir++) {
      // projections (forward)
      double pc[15][4], ps[4][4], pz[4];
      for (int k = 0; k < 15; k++) {
        const double x[4] = {cc[0][k], cc[1][k], cc[2][k], cc[3][k]};
        if (dir == 0) to_char<double, 0>(cs, x, pc[k]); else to_char<double, 1>(cs, x, pc[k]);
      }
      for (int k = 0; k < 4; k++) {
        const double x[4] = {sl[0][k], sl[1][k], sl[2][k], sl[3][k]};
        if (dir == 0) to_char<double, 0>(cs, x, ps[k]); else to_char<double, 1>(cs, x, ps[k]);
      }
      if (dir == 0) to_char<double, 0>(cs, ctr, pz); else to_char<double, 1>(cs, ctr, pz);
      // this direction's characteristic point values and weight factors per field, as
      // the forward wrote them
      const double* yr = w.yrec + (long long)(72 * dir) * g.ps + c;
      double chf[4][6], chv[4][9], chm[4], wrec[4][2];
      for (int f = 0; f < 4; f++) {
        const double* y = yr + (long long)(18 * f) * g.ps;
        for (int k = 0; k < 6; k++) chf[f][k] = y[k * g.ps];
        for (int k = 0; k < 9; k++) chv[f][k] = y[(6 + k) * g.ps];
        chm[f] = y[15 * g.ps];
        wrec[f][0] = y[16 * g.ps];
        wrec[f][1] = y[17 * g.ps];
      }
      // back-projection adjoints -> char value adjoints
      CharSums ms = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
      double chfb[4][6], chvb[4][9], chmb[4] = {0, 0, 0, 0};
      for (int f = 0; f < 4; f++) {
        for (int k = 0; k < 6; k++) chfb[f][k] = 0.0;
        for (int k = 0; k < 9; k++) chvb[f][k] = 0.0;
      }
      for (int k = 0; k < 6; k++) {
        const double y[4] = {chf[0][k], chf[1][k], chf[2][k], chf[3][k]};
        double yb[4] = {0, 0, 0, 0};
        if (dir == 0) from_char_T<0>(cs, y, fb[k], yb, ms); else from_char_T<1>(cs, y, fb[6 + k], yb, ms);
        for (int f = 0; f < 4; f++) chfb[f][k] = yb[f];
      }
      for (int k = 0; k < 9; k++) {
        const double y[4] = {chv[0][k], chv[1][k], chv[2][k], chv[3][k]};
        const double xb[4] = {0.5 * vb[k][0], 0.5 * vb[k][1], 0.5 * vb[k][2], 0.5 * vb[k][3]};
        double yb[4] = {0, 0, 0, 0};
        if (dir == 0) from_char_T<0>(cs, y, xb, yb, ms); else from_char_T<1>(cs, y, xb, yb, ms);
        for (int f = 0; f < 4; f++) chvb[f][k] = yb[f];
      }
      {
        double yb[4] = {0, 0, 0, 0};
        if (dir == 0) from_char_T<0>(cs, chm, mb[0], yb, ms); else from_char_T<1>(cs, chm, mb[1], yb, ms);
        for (int f = 0; f < 4; f++) chmb[f] = yb[f];
      }
      // per field: point evaluations and the combination
      double pcb[15][4], psb[4][4], pzb[4];
      for (int f = 0; f < 4; f++) {
        double Cb[15] = {0};
        if (dir == 0) eval_xfaces_T(chfb[f], Cb); else eval_yfaces_T(chfb[f], Cb);
        eval_vol_T(chvb[f], Cb);
        if (dir == 0) hw_moment_xi_T<double>(chmb[f], Cb); else hw_moment_eta_T<double>(chmb[f], Cb);
        double c0[15], s[4], c0b[15] = {0}, sbb[4] = {0, 0, 0, 0}, zb = 0.0;
        for (int k = 0; k < 15; k++) c0[k] = pc[k][f];
        for (int k = 0; k < 4; k++) s[k] = ps[k][f];
        double gr[15];
        hw_beta_quartic_grad<double>(c0, gr);
        hweno_combine_T(c0, s, pz[f], eps, wrec[f][0], wrec[f][1], gr, Cb, c0b, sbb, zb);
        for (int k = 0; k < 15; k++) pcb[k][f] = c0b[k];
        for (int k = 0; k < 4; k++) psb[k][f] = sbb[k];
        pzb[f] = zb;
      }
      // projection adjoints -> conserved coefficient adjoints and state parameters
      for (int k = 0; k < 15; k++) {
        const double x[4] = {cc[0][k], cc[1][k], cc[2][k], cc[3][k]};
        double xb[4] = {0, 0, 0, 0};
        if (dir == 0) to_char_T<0>(cs, x, pcb[k], xb, ms); else to_char_T<1>(cs, x, pcb[k], xb, ms);
        for (int v = 0; v < 4; v++) ccb[v][k] += xb[v];
      }
      for (int k = 0; k < 4; k++) {
        const double x[4] = {sl[0][k], sl[1][k], sl[2][k], sl[3][k]};
        double xb[4] = {0, 0, 0, 0};
        if (dir == 0) to_char_T<0>(cs, x, psb[k], xb, ms); else to_char_T<1>(cs, x, psb[k], xb, ms);
        for (int v = 0; v < 4; v++) slb[v][k] += xb[v];
      }
      {
        double xb[4] = {0, 0, 0, 0};
        if (dir == 0) to_char_T<0>(cs, ctr, pzb, xb, ms); else to_char_T<1>(cs, ctr, pzb, xb, ms);
        for (int v = 0; v < 4; v++) ctrb[v] += xb[v];
      }
      if (dir == 0) char_sums_finish<0>(cs, ms, sb); else char_sums_finish<1>(cs, ms, sb);
    }
    char_state_T(ub, g.gamma, sb, ubb);
    for (int v = 0; v < 4; v++) {
      double db[17] = {0};
      hw_p0_coeffs_T<double>(ccb[v], db);
      db[4] += ctrb[v] + ubb[v] + ubl[v] + slb[v][0] - slb[v][1] + slb[v][2] - slb[v][3];
      db[3] -= slb[v][0];
      db[5] += slb[v][1];
      db[1] -= slb[v][2];
      db[7] += slb[v][3];
      for (int k = 0; k < 17; k++) a.cc[(long long)(17 * v + k) * g.ps + c] = db[k];
    }
  }
}

// state adjoint of every padded cell from ka_cons's contributions
__global__ void ka_gather_q(Grid g, Adj a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x - NG;
  const int j = blockIdx.y * blockDim.y + threadIdx.y - NG;
  if (i >= g.nx + NG || j >= g.ny + NG) return;
  const long long c = cidx(g, i, j);
  for (int v = 0; v < 4; v++) {
    double av, xi, eta;
    gather_triple(g, a.cc + (long long)17 * v * g.ps, i, j, -3, g.nx + 3, g.ny + 3, av, xi, eta);
    a.q[(long long)v * g.ps + c] = av;
    a.q[(long long)(4 + v) * g.ps + c] = xi;
    a.q[(long long)(8 + v) * g.ps + c] = eta;
  }
}

// adjoint of the ghost fill: every ghost adjoint goes back to its source cell with the
// ghost's sign (y pass first: it ran last in the forward); an outflow ghost's goes to the
// adjacent interior cell with sign 1, an inflow ghost's is dropped (its value is the
// prescribed state, independent of the solution).  Atomic adds: on grids with fewer
// than 8 cells a periodic source feeds ghosts on both sides, and an outflow edge cell
// feeds all four ghost layers.
__global__ void ka_ghost_y(Grid g, Adj a) {
  const int W = g.nx + 2 * NG;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8 * W) return;
  const int r = t / W, i = t % W - NG;
  const int side = r / 4, k = r % 4;
  const int j = side == 0 ? -1 - k : g.ny + k;
  const int bc = g.bc[2 + side];
  if (bc == HWENO_BC_INFLOW) return;
  const long long d = cidx(g, i, j), s = cidx(g, i, ghost_src(bc, j, g.ny));
  const bool mir = is_mirror(bc);
  for (int m = 0; m < 3; m++)
    for (int v = 0; v < 4; v++) {
      const double sg = mir ? bc_sign(bc, 1, v) * (m == 2 ? -1.0 : 1.0) : 1.0;
      atomicAdd(&a.q[(4 * m + v) * g.ps + s], sg * a.q[(4 * m + v) * g.ps + d]);
    }
}
__global__ void ka_ghost_x(Grid g, Adj a) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 8 * g.ny) return;
  const int j = t / 8, cix = t % 8;
  const int side = cix / 4, k = cix % 4;
  const int i = side == 0 ? -1 - k : g.nx + k;
  const int bc = g.bc[side];
  if (bc == HWENO_BC_INFLOW) return;
  const long long d = cidx(g, i, j), s = cidx(g, ghost_src(bc, i, g.nx), j);
  const bool mir = is_mirror(bc);
  for (int m = 0; m < 3; m++)
    for (int v = 0; v < 4; v++) {
      const double sg = mir ? bc_sign(bc, 0, v) * (m == 1 ? -1.0 : 1.0) : 1.0;
      atomicAdd(&a.q[(4 * m + v) * g.ps + s], sg * a.q[(4 * m + v) * g.ps + d]);
    }
}

// seeds of one stage's operator VJP and the RK combination of the adjoints:
//   mode 0: R = scale_r * lam, M = scale_m * lam_mom (+ extra_m * base_mom if given)
__global__ void ka_seed(Grid g, const double* __restrict__ lam, double sr, double sm,
                        const double* __restrict__ bmom, double sb, Adj a) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const long long c = cidx(g, i, j);
  for (int k = 0; k < 12; k++) a.R[(long long)k * g.ps + c] = sr * lam[(long long)k * g.ps + c];
  for (int k = 0; k < 8; k++) {
    double m = sm * lam[(long long)(4 + k) * g.ps + c];
    if (bmom) m += sb * bmom[(long long)(4 + k) * g.ps + c];
    a.M[(long long)k * g.ps + c] = m;
  }
}

// out = xbar (interior of a.q) + [ca * lam_avg + cb * bavg; 0]  (interior cells)
__global__ void ka_finish(Grid g, const Adj a, const double* __restrict__ lam, double ca,
                          const double* __restrict__ bvec, double cb, double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const long long c = cidx(g, i, j);
  for (int k = 0; k < 12; k++) {
    double x = a.q[(long long)k * g.ps + c];
    if (k < 4) {
      x += ca * lam[(long long)k * g.ps + c];
      if (bvec) x += cb * bvec[(long long)k * g.ps + c];
    }
    out[(long long)k * g.ps + c] = x;
  }
}

// bvec = alpha * bvec + beta * v  over the 12 planes (interior); alpha = 0 overwrites
// without reading bvec, whose old contents (a previous sweep's, possibly non-finite)
// must not reach the result as 0 * inf or 0 * NaN
__global__ void ka_axpby(Grid g, double* __restrict__ bvec, double alpha, const double* __restrict__ v, double beta) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  const int j = blockIdx.y * blockDim.y + threadIdx.y;
  if (i >= g.nx || j >= g.ny) return;
  const long long c = cidx(g, i, j);
  for (int k = 0; k < 12; k++) {
    const double b = alpha == 0.0 ? 0.0 : alpha * bvec[(long long)k * g.ps + c];
    bvec[(long long)k * g.ps + c] = b + beta * v[(long long)k * g.ps + c];
  }
}

}  // namespace hw
