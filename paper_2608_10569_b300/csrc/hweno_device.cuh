// Device arithmetic of the HWENO-GR spatial operator (templated on the compute
// type T: double for the FP64 path, float for the mixed path).
//
// Paper: Guo, Fan, Zhao, "An efficient and robust fifth-order HWENO scheme with
// gradient reconstruction for compressible Navier-Stokes equations".
//   scalar reconstruction ..... Appendix A.2, Eqs. (A.4)-(A.6)
//   nonlinear combination ..... Eq. (3.4) / Eq. (3.9)
//   Gauss points .............. Sec. 3.1 (offsets 0, +-sqrt(15)/10; weights 4/9, 5/18)
//   characteristic fields ..... Sec. 3.1 (left eigenvectors of the Euler Jacobian)
//   PP limiter ................ Sec. 3.1 and Sec. 5 (eps_PP)
//   fluxes, LF coefficient .... Sec. 3.1 flux definitions, Eq. (3.3)
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include "hweno_stencil.h"

namespace hw {

// three-point Gauss rule on the scaled cell [-1/2, 1/2]
constexpr double GN = 0.3872983346207416885;   // sqrt(15)/10

// precision-preserving math for the templated bodies: the float forms are the FP32
// instructions, the double forms the FP64 ones (no promotion of FP32 work to FP64)
__device__ __forceinline__ float tsqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tfabs(float x) { return fabsf(x); }
__device__ __forceinline__ double tfabs(double x) { return fabs(x); }
__device__ __forceinline__ float tfmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tfmax(double a, double b) { return fmax(a, b); }
// a / b: IEEE division in FP64; in FP32 the reciprocal-multiply form (at most 2 ulp, for
// divisors between 2^-126 and 2^126, which the mixed path's weights, densities and sound
// speeds are)
__device__ __forceinline__ float tdiv(float a, float b) { return __fdividef(a, b); }
__device__ __forceinline__ double tdiv(double a, double b) { return a / b; }
constexpr double GW_OUT = 5.0 / 18.0;
constexpr double GW_MID = 4.0 / 9.0;
// linear weights of Appendix A.2
constexpr double GAM0 = 0.99;
constexpr double GAML = 0.0025;

template <class T>
__device__ __forceinline__ T gweight(int g) { return g == 1 ? T(GW_MID) : T(GW_OUT); }
template <class T>
__device__ __forceinline__ T gnode(int g) { return T(g - 1) * T(GN); }

// ---------------------------------------------------------------------------
// scalar unified-stencil HWENO (Appendix A.2).
// c0: the quartic's 15 coefficients; s = (dxm, dxp, dym, dyp): the one-sided
// differences of the averages (centre minus left, right minus centre, centre minus
// bottom, top minus centre); ctr: the centre average in the same representation as
// c0 (zero when the data are offsets from it).  The four linear candidates share the
// centre average and take their slopes from S1={2,4,5}: (dxm, dym), S2={2,5,6}:
// (dxp, dym), S3={4,5,8}: (dxm, dyp), S4={5,6,8}: (dxp, dyp).  Writes the
// coefficients C of the nonlinear combination w0 (p0/g0 - sum gm/g0 pm) + sum wm pm
// of Eq. (3.4) with the weights of Eq. (A.6).
// REC (FP64 only): also return beta_0 and the reciprocal 1/S' in rec[0], rec[1] for a
// reverse sweep.
template <class T, bool REC = false>
__device__ __forceinline__ void hweno_combine_coeffs(const T* c0, const T* s, T ctr, T eps, T* C,
                                                     T* rec = nullptr) {
  const T dxm = s[0], dxp = s[1], dym = s[2], dyp = s[3];
  const T sxm = dxm * dxm, sxp = dxp * dxp, sym = dym * dym, syp = dyp * dyp;
  const T b0 = hw_beta_quartic<T>(c0);
  const T b1 = sxm + sym, b2 = sxp + sym, b3 = sxm + syp, b4 = sxp + syp;
  const T e1 = b0 - b1, e2 = b0 - b2, e3 = b0 - b3, e4 = b0 - b4;
  const T ts = T(0.25) * (tfabs(e1) + tfabs(e2) + tfabs(e3) + tfabs(e4));
  const T tau = ts * ts;
  // omega_m = gamma_m (1 + tau/D_m) / S with D_m = beta_m + eps.  The combination
  // coefficients of Eq. (3.4) are a0 = omega0/gamma0 and a_m = omega_m - a0 gamma_m.
  T a0, a[4];
  if constexpr (sizeof(T) == 8) {
    // FP64: one reciprocal.  With P = prod D_k, Q_m = P/D_m and R_m = P/(D_0 D_m):
    //   omega_m ~ gamma_m (P + tau Q_m),  a0 = (P + tau Q_0)/S',
    //   a_m = gamma_m tau (Q_m - Q_0)/S' = gamma_m tau R_m (beta_0 - beta_m)/S',
    //   S' = sum_m gamma_m (P + tau Q_m) = P + tau (gamma0 Q_0 + gammaL D_0 sum R_m).
    // D_m >= eps = 1e-8, so P >= 1e-40 stays a normal double.
    const T D0 = b0 + eps, D1 = b1 + eps, D2 = b2 + eps, D3 = b3 + eps, D4 = b4 + eps;
    const T D12 = D1 * D2, D34 = D3 * D4;
    const T R1 = D2 * D34, R2 = D1 * D34, R3 = D12 * D4, R4 = D12 * D3;
    const T Q0 = D12 * D34;
    const T P = D0 * Q0;
    const T Sp = P + tau * (T(GAM0) * Q0 + T(GAML) * D0 * ((R1 + R2) + (R3 + R4)));
    const T rs = T(1) / Sp;
    if constexpr (REC) {
      rec[0] = b0;
      rec[1] = rs;
    }
    a0 = (P + tau * Q0) * rs;
    const T g = T(GAML) * tau * rs;
    a[0] = g * R1 * e1;
    a[1] = g * R2 * e2;
    a[2] = g * R3 * e3;
    a[3] = g * R4 * e4;
  } else {
    // FP32: the products above leave the float range for smooth data (eps^5 = 1e-40),
    // so divide once per candidate: t_m = tau/D_m, a0 = (1 + t0)/S,
    // a_m = gamma_m (t_m - t0)/S with S = gamma0 (1 + t0) + gammaL sum (1 + t_m).
    const T t0 = tdiv(tau, b0 + eps), t1 = tdiv(tau, b1 + eps), t2 = tdiv(tau, b2 + eps);
    const T t3 = tdiv(tau, b3 + eps), t4 = tdiv(tau, b4 + eps);
    const T wsum = T(GAM0) * (T(1) + t0) + T(GAML) * ((T(4) + t1) + (t2 + t3) + t4);
    const T rs = tdiv(T(1), wsum);
    a0 = (T(1) + t0) * rs;
    const T gl = T(GAML) * rs;
    a[0] = gl * (t1 - t0);
    a[1] = gl * (t2 - t0);
    a[2] = gl * (t3 - t0);
    a[3] = gl * (t4 - t0);
  }
#pragma unroll
  for (int k = 0; k < 15; k++) C[k] = a0 * c0[k];
  // the linear candidates' constant terms are the centre average; their weights sum
  // to 1 - a0
  C[0] += (T(1) - a0) * ctr;
  C[1] += (a[0] + a[2]) * dxm + (a[1] + a[3]) * dxp;
  C[2] += (a[0] + a[1]) * dym + (a[2] + a[3]) * dyp;
}

// scalar reconstruction from the 17 data in the order of hweno_stencil.h
template <class T>
__device__ __forceinline__ void hweno_combine(const T* d, T eps, T* C) {
  T c0[15];
  hw_p0_coeffs<T>(d, c0);
  const T s[4] = {d[4] - d[3], d[5] - d[4], d[4] - d[1], d[7] - d[4]};
  hweno_combine_coeffs<T>(c0, s, d[4], eps, C);
}

// ---------------------------------------------------------------------------
// point evaluation of a quartic with monomial order
// 1, x, y, x^2, xy, y^2, x^3, x^2y, xy^2, y^3, x^4, x^3y, x^2y^2, xy^3, y^4
// collapse along x at x = +-h: even part E_q and odd part O_q of sum_p c_pq x^p
template <class T>
__device__ __forceinline__ void collapse_x(const T* c, T h, T* E, T* O) {
  const T h2 = h * h;
  E[0] = c[0] + h2 * (c[3] + h2 * c[10]);
  O[0] = h * (c[1] + h2 * c[6]);
  E[1] = c[2] + h2 * c[7];
  O[1] = h * (c[4] + h2 * c[11]);
  E[2] = c[5] + h2 * c[12];
  O[2] = h * c[8];
  E[3] = c[9];
  O[3] = h * c[13];
  E[4] = c[14];
}
template <class T>
__device__ __forceinline__ void collapse_y(const T* c, T h, T* E, T* O) {
  const T h2 = h * h;
  E[0] = c[0] + h2 * (c[5] + h2 * c[14]);
  O[0] = h * (c[2] + h2 * c[9]);
  E[1] = c[1] + h2 * c[8];
  O[1] = h * (c[4] + h2 * c[13]);
  E[2] = c[3] + h2 * c[12];
  O[2] = h * c[7];
  E[3] = c[6];
  O[3] = h * c[11];
  E[4] = c[10];
}
// 1D quartic a0..a4 at t = -g, 0, +g
template <class T>
__device__ __forceinline__ void line3(const T* a, T* out) {
  const T g = T(GN), g2 = g * g;
  const T ev = a[0] + g2 * (a[2] + g2 * a[4]);
  const T od = g * (a[1] + g2 * a[3]);
  out[0] = ev - od;
  out[1] = a[0];
  out[2] = ev + od;
}
// values at the x-faces: [left (xi=-1/2) eta_G, right (xi=+1/2) eta_G]
template <class T>
__device__ __forceinline__ void eval_xfaces(const T* c, T* out) {
  T E[5], O[4], a[5];
  collapse_x<T>(c, T(0.5), E, O);
#pragma unroll
  for (int q = 0; q < 4; q++) a[q] = E[q] - O[q];
  a[4] = E[4];
  line3<T>(a, out);
#pragma unroll
  for (int q = 0; q < 4; q++) a[q] = E[q] + O[q];
  line3<T>(a, out + 3);
}
// values at the y-faces: [bottom (eta=-1/2) xi_G, top (eta=+1/2) xi_G]
template <class T>
__device__ __forceinline__ void eval_yfaces(const T* c, T* out) {
  T E[5], O[4], a[5];
  collapse_y<T>(c, T(0.5), E, O);
#pragma unroll
  for (int q = 0; q < 4; q++) a[q] = E[q] - O[q];
  a[4] = E[4];
  line3<T>(a, out);
#pragma unroll
  for (int q = 0; q < 4; q++) a[q] = E[q] + O[q];
  line3<T>(a, out + 3);
}
// values at the 9 volume points, index 3G + H at (xi_G, eta_H)
template <class T>
__device__ __forceinline__ void eval_vol(const T* c, T* out) {
  T E[5], O[4], a[5], v[3];
  collapse_x<T>(c, T(GN), E, O);
#pragma unroll
  for (int q = 0; q < 4; q++) a[q] = E[q] - O[q];
  a[4] = E[4];
  line3<T>(a, v);
  out[0] = v[0]; out[1] = v[1]; out[2] = v[2];
  // xi = 0: the coefficients with p = 0
  a[0] = c[0]; a[1] = c[2]; a[2] = c[5]; a[3] = c[9]; a[4] = c[14];
  line3<T>(a, v);
  out[3] = v[0]; out[4] = v[1]; out[5] = v[2];
#pragma unroll
  for (int q = 0; q < 4; q++) a[q] = E[q] + O[q];
  a[4] = E[4];
  line3<T>(a, v);
  out[6] = v[0]; out[7] = v[1]; out[8] = v[2];
}

// physical partial derivatives of a quartic in the scaled coordinates, as quartics in
// the same monomial order (the five quartic slots zero): with f = (r, 2r, 3r, 4r) and
// r = 1/dx (resp. 1/dy), d/dx xi^p eta^q = p r xi^(p-1) eta^q
template <class T>
__device__ __forceinline__ void poly_dx(const T* c, const T* f, T* d) {
  d[0] = f[0] * c[1]; d[1] = f[1] * c[3]; d[2] = f[0] * c[4];
  d[3] = f[2] * c[6]; d[4] = f[1] * c[7]; d[5] = f[0] * c[8];
  d[6] = f[3] * c[10]; d[7] = f[2] * c[11]; d[8] = f[1] * c[12]; d[9] = f[0] * c[13];
  d[10] = d[11] = d[12] = d[13] = d[14] = T(0);
}
template <class T>
__device__ __forceinline__ void poly_dy(const T* c, const T* f, T* d) {
  d[0] = f[0] * c[2]; d[1] = f[0] * c[4]; d[2] = f[1] * c[5];
  d[3] = f[0] * c[7]; d[4] = f[1] * c[8]; d[5] = f[2] * c[9];
  d[6] = f[0] * c[11]; d[7] = f[1] * c[12]; d[8] = f[2] * c[13]; d[9] = f[3] * c[14];
  d[10] = d[11] = d[12] = d[13] = d[14] = T(0);
}

// ---------------------------------------------------------------------------
// local characteristic fields of the Euler flux Jacobian at a state (Sec. 3.1).
// Right eigenvectors in direction n (normal velocity un, tangential ut), columns in
// the order u_n - c, u_n (entropy), shear, u_n + c:
//   r1 = (1, un - c, ut, H - un c), r2 = (1, un, ut, q^2/2), r3 = (0, 0, 1, ut),
//   r4 = (1, un + c, ut, H + un c)        (components ordered rho, m_n, m_t, E)
// and L = R^{-1}.  Both maps are applied in factored form: with
//   A = b2 x0 + b1 (x3 - un x_n - ut x_t),  B = (un x0 - x_n)/c,  b1 = (g-1)/c^2,
//   b2 = b1 q^2/2:   y0 = (A + B)/2, y1 = x0 - A, y2 = x_t - ut x0, y3 = (A - B)/2,
// and back  x0 = y0 + y1 + y3, x_n = un x0 + c (y3 - y0), x_t = ut x0 + y2,
//           x3 = H (y0 + y3) + un c (y3 - y0) + q^2/2 y1 + ut y2.
template <class T>
struct CharState {
  T u, v, c, H, hq2;      // velocity, sound speed, total enthalpy, q^2/2
  T hb1, hb2, hrc;        // b1/2, b2/2, 1/(2c)
};

template <class T>
__device__ __forceinline__ void char_state(const T* ub, T gamma, CharState<T>& s) {
  const T rr = tdiv(T(1), ub[0]);
  s.u = ub[1] * rr;
  s.v = ub[2] * rr;
  s.hq2 = T(0.5) * (s.u * s.u + s.v * s.v);
  const T p = (gamma - T(1)) * (ub[3] - ub[0] * s.hq2);
  const T c2 = gamma * p * rr;
  s.c = tsqrt(c2);
  s.H = (ub[3] + p) * rr;
  const T b1 = tdiv(gamma - T(1), c2);
  s.hb1 = T(0.5) * b1;
  s.hb2 = s.hb1 * s.hq2;
  s.hrc = tdiv(T(0.5), s.c);
}

// x (rho, m, n, E) -> characteristic y for direction DIR (0: x, 1: y)
template <class T, int DIR>
__device__ __forceinline__ void to_char(const CharState<T>& s, const T* x, T* y) {
  const T un = DIR == 0 ? s.u : s.v, ut = DIR == 0 ? s.v : s.u;
  const T xn = DIR == 0 ? x[1] : x[2], xt = DIR == 0 ? x[2] : x[1];
  const T Ah = s.hb2 * x[0] + s.hb1 * (x[3] - un * xn - ut * xt);  // A/2
  const T Bh = s.hrc * (un * x[0] - xn);                             // B/2
  y[0] = Ah + Bh;
  y[1] = x[0] - T(2) * Ah;
  y[2] = xt - ut * x[0];
  y[3] = Ah - Bh;
}

template <class T, int DIR>
__device__ __forceinline__ void from_char(const CharState<T>& s, const T* y, T* x) {
  const T un = DIR == 0 ? s.u : s.v, ut = DIR == 0 ? s.v : s.u;
  const T x0 = y[0] + y[1] + y[3];
  const T dd = y[3] - y[0];
  const T xn = un * x0 + s.c * dd;
  const T xt = ut * x0 + y[2];
  x[0] = x0;
  x[DIR == 0 ? 1 : 2] = xn;
  x[DIR == 0 ? 2 : 1] = xt;
  x[3] = s.H * (y[0] + y[3]) + (un * s.c) * dd + s.hq2 * y[1] + ut * y[2];
}

// ---------------------------------------------------------------------------
// ideal gas helpers (Sec. 3.1)
__device__ __forceinline__ double pressure(const double* u, double gamma) {
  return (gamma - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]);
}

// smallest t in [0,1] with p(ub + t (uq - ub)) = eps, written as the quadratic
// (E + t dE)(rho + t drho) - |m + t dm|^2/2 - eps/(gamma-1) (rho + t drho) = 0
__device__ __forceinline__ double theta_root(const double* ub, const double* uq, double eps,
                                              double gamma) {
  const double d0 = uq[0] - ub[0], d1 = uq[1] - ub[1], d2 = uq[2] - ub[2], d3 = uq[3] - ub[3];
  const double e1 = eps / (gamma - 1.0);
  const double a = d3 * d0 - 0.5 * (d1 * d1 + d2 * d2);
  const double b = ub[3] * d0 + ub[0] * d3 - (ub[1] * d1 + ub[2] * d2) - e1 * d0;
  const double cc = ub[3] * ub[0] - 0.5 * (ub[1] * ub[1] + ub[2] * ub[2]) - e1 * ub[0];
  double t;
  if (fabs(a) < 1e-300) {
    t = -cc / b;
  } else {
    double disc = b * b - 4.0 * a * cc;
    disc = disc < 0.0 ? 0.0 : disc;
    const double sq = sqrt(disc);
    const double qq = -0.5 * (b + (b >= 0.0 ? sq : -sq));
    const double r1 = qq / a;
    const double r2 = qq != 0.0 ? cc / qq : r1;
    const double lo = fmin(r1, r2), hi = fmax(r1, r2);
    t = (lo >= 0.0 && lo <= 1.0) ? lo : hi;
  }
  return fmin(fmax(t, 0.0), 1.0);
}

// Positivity-preserving limiter of one cell (Sec. 3.1, Sec. 5), always in FP64:
// density scaling about the average over all 21 points, then the pressure root;
// only the 12 face states are rescaled.  Returns 1 when it changed anything.
__device__ __forceinline__ int pp_limit(const double* ub, double (*face)[4], const double (*vol)[4],
                                        double gamma, double eps_pp, double* th_out) {
  const double pb = pressure(ub, gamma);
  th_out[0] = 1.0;
  th_out[1] = 1.0;
  double eps = fmin(eps_pp, fmin(ub[0], pb));
  double rmin = ub[0];
#pragma unroll
  for (int k = 0; k < 12; k++) rmin = fmin(rmin, face[k][0]);
#pragma unroll
  for (int k = 0; k < 9; k++) rmin = fmin(rmin, vol[k][0]);
  const double thr = rmin < eps ? (ub[0] - eps) / (ub[0] - rmin) : 1.0;
  // pressure check with the density rescaled; p < eps  <=>  (g-1)(E rho - |m|^2/2) < eps rho
  double thp = 1.0;
  const double gm1 = gamma - 1.0;
#pragma unroll 1
  for (int k = 0; k < 21; k++) {
    const double* s = k < 12 ? face[k] : vol[k - 12];
    double w[4] = {ub[0] + thr * (s[0] - ub[0]), s[1], s[2], s[3]};
    const double lhs = gm1 * (w[3] * w[0] - 0.5 * (w[1] * w[1] + w[2] * w[2]));
    if (lhs < eps * w[0]) thp = fmin(thp, theta_root(ub, w, eps, gamma));
  }
  if (thr < 1.0 || thp < 1.0) {
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double r = ub[0] + thr * (face[k][0] - ub[0]);
      face[k][0] = ub[0] + thp * (r - ub[0]);
#pragma unroll
      for (int v = 1; v < 4; v++) face[k][v] = ub[v] + thp * (face[k][v] - ub[v]);
    }
  }
  th_out[0] = thr;
  th_out[1] = thp;
  return (thr < 1.0 || thp < 1.0) ? 1 : 0;
}

// ---------------------------------------------------------------------------
// physical flux in direction dir from primitive state (rho, u, v, e) and
// gradients s = (u_x, u_y, v_x, v_y, e_x, e_y); also returns the conserved state.
struct Phys {
  double gamma, Pr, Re;
};

template <class T>
__device__ __forceinline__ void phys_flux(int dir, const T* w, const T* s, T gamma, T rPr, T rRe,
                                          T* f) {
  const T rho = w[0], u = w[1], v = w[2], e = w[3];
  const T p = (gamma - T(1)) * rho * e;
  const T E = rho * (e + T(0.5) * (u * u + v * v));
  const T txx = T(4.0 / 3.0) * s[0] - T(2.0 / 3.0) * s[3];
  const T txy = s[1] + s[2];
  const T tyy = T(4.0 / 3.0) * s[3] - T(2.0 / 3.0) * s[0];
  if (dir == 0) {
    const T m = rho * u;
    f[0] = m;
    f[1] = m * u + p - txx * rRe;
    f[2] = m * v - txy * rRe;
    f[3] = (E + p) * u - (txx * u + txy * v + gamma * s[4] * rPr) * rRe;
  } else {
    const T n = rho * v;
    f[0] = n;
    f[1] = n * u - txy * rRe;
    f[2] = n * v + p - tyy * rRe;
    f[3] = (E + p) * v - (txy * u + tyy * v + gamma * s[5] * rPr) * rRe;
  }
}

// max(|u_n| + c, PP wave-speed bound of Eq. (3.3))
template <class T>
__device__ __forceinline__ T wave_bound(int dir, const T* w, const T* s, T gamma, T rPr, T rRe) {
  const T rho = w[0], e = w[3];
  const T p = (gamma - T(1)) * rho * e;
  const T cs = tsqrt(gamma * (gamma - T(1)) * e);
  const T txx = T(4.0 / 3.0) * s[0] - T(2.0 / 3.0) * s[3];
  const T txy = s[1] + s[2];
  const T tyy = T(4.0 / 3.0) * s[3] - T(2.0 / 3.0) * s[0];
  T un, q, s1, s2;
  if (dir == 0) {
    un = w[1]; q = gamma * s[4] * rPr * rRe; s1 = txx * rRe - p; s2 = txy * rRe;
  } else {
    un = w[2]; q = gamma * s[5] * rPr * rRe; s1 = txy * rRe; s2 = tyy * rRe - p;
  }
  const T r2e = rho * rho * e;
  const T pp = tfabs(un) + tdiv(tsqrt(rho * rho * q * q + T(2) * r2e * (s1 * s1 + s2 * s2)) + rho * tfabs(q),
                                T(2) * r2e);
  return tfmax(tfabs(un) + cs, pp);
}

}  // namespace hw
