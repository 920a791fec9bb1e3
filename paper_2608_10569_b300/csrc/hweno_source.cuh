// Example 5.2's manufactured source term on the GPU: S = U_t + F_x + G_y of the
// manufactured fields (the equations of Sec. 3.1), integrated over each interior cell
// into its average and scaled first moments and added to the residual, so that the
// semi-discrete system becomes dU/dt = R(U) + S(t).
//
// Fields: rho = 2 + a (sin th1 + cos th2), u = 1 + a (sin(-th4) + cos th3),
//         v = 2 + a (sin th3 + cos th4),   e = 2 + a (sin th4 + cos th3),
// with a = 0.1 exp(-t), th1 = 2 pi (2x - y), th2 = 2 pi (-x + 2y), th3 = 2 pi (x + y),
// th4 = 2 pi (x - y); p = (gamma - 1) rho e, E = rho (e + (u^2 + v^2)/2).
#pragma once
#include "hweno_kernels.cuh"

namespace hw {

// 4-point Gauss-Legendre rule on the scaled cell [-1/2, 1/2] (nodes and weights from
// their closed forms, evaluated on the host)
struct Quad4 {
  double nd[4], wt[4];
};

// 4-point Gauss-Legendre on [-1/2, 1/2]: nodes sqrt(3/7 -+ 2/7 sqrt(6/5)) / 2, weights
// (18 +- sqrt(30)) / 72
inline Quad4 make_quad4() {
  const double ri = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), ro = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
  const double wi = (18.0 + sqrt(30.0)) / 72.0, wo = (18.0 - sqrt(30.0)) / 72.0;
  return Quad4{{-0.5 * ro, -0.5 * ri, 0.5 * ri, 0.5 * ro}, {wo, wi, wi, wo}};
}

// one field base + a (sin(2 pi (a1 x + b1 y)) + cos(2 pi (a2 x + b2 y))), given the sine
// and cosine of both angles: its value and t-, first and second space derivatives
struct MField {
  double f, ft, fx, fy, fxx, fxy, fyy;
};

__device__ __forceinline__ MField mms_field(double base, double amp, double a1, double b1, double s1, double c1,
                                            double a2, double b2, double s2, double c2) {
  constexpr double TP = 6.283185307179586476925286766559;
  const double w = s1 + c2;
  const double k1 = amp * TP, k2 = amp * TP * TP;
  MField F;
  F.f = base + amp * w;
  F.ft = -amp * w;
  F.fx = k1 * (a1 * c1 - a2 * s2);
  F.fy = k1 * (b1 * c1 - b2 * s2);
  F.fxx = -k2 * (a1 * a1 * s1 + a2 * a2 * c2);
  F.fxy = -k2 * (a1 * b1 * s1 + a2 * b2 * c2);
  F.fyy = -k2 * (b1 * b1 * s1 + b2 * b2 * c2);
  return F;
}

// S at (x, y) for the amplitude amp = 0.1 exp(-t)
__device__ __forceinline__ void mms_source(const Grid& g, double x, double y, double amp, double* S) {
  constexpr double TP = 6.283185307179586476925286766559;
  double s1, c1, s2, c2, s3, c3, s4, c4;
  sincos(TP * (2.0 * x - y), &s1, &c1);
  sincos(TP * (2.0 * y - x), &s2, &c2);
  sincos(TP * (x + y), &s3, &c3);
  sincos(TP * (x - y), &s4, &c4);
  const MField R = mms_field(2.0, amp, 2.0, -1.0, s1, c1, -1.0, 2.0, s2, c2);
  const MField U = mms_field(1.0, amp, -1.0, 1.0, -s4, c4, 1.0, 1.0, s3, c3);
  const MField V = mms_field(2.0, amp, 1.0, 1.0, s3, c3, 1.0, -1.0, s4, c4);
  const MField Q = mms_field(2.0, amp, 1.0, -1.0, s4, c4, 1.0, 1.0, s3, c3);
  const double gm = g.gamma, rRe = g.rRe, gPr = g.gamma * g.rPr;
  const double rho = R.f, u = U.f, v = V.f, e = Q.f;
  // momenta, kinetic energy, total energy and pressure with their derivatives
  const double m = rho * u, mt = R.ft * u + rho * U.ft, mx = R.fx * u + rho * U.fx, my = R.fy * u + rho * U.fy;
  const double n = rho * v, nt = R.ft * v + rho * V.ft, nx = R.fx * v + rho * V.fx, ny = R.fy * v + rho * V.fy;
  const double k = 0.5 * (u * u + v * v);
  const double kt = u * U.ft + v * V.ft, kx = u * U.fx + v * V.fx, ky = u * U.fy + v * V.fy;
  const double E = rho * (e + k);
  const double Et = R.ft * (e + k) + rho * (Q.ft + kt);
  const double Ex = R.fx * (e + k) + rho * (Q.fx + kx);
  const double Ey = R.fy * (e + k) + rho * (Q.fy + ky);
  const double p = (gm - 1.0) * rho * e;
  const double px = (gm - 1.0) * (R.fx * e + rho * Q.fx), py = (gm - 1.0) * (R.fy * e + rho * Q.fy);
  // viscous stresses, their divergence, and the divergence of the viscous energy flux
  const double txx = (4.0 * U.fx - 2.0 * V.fy) * (1.0 / 3.0), tyy = (4.0 * V.fy - 2.0 * U.fx) * (1.0 / 3.0);
  const double txy = U.fy + V.fx;
  const double txx_x = (4.0 * U.fxx - 2.0 * V.fxy) * (1.0 / 3.0), tyy_y = (4.0 * V.fyy - 2.0 * U.fxy) * (1.0 / 3.0);
  const double txy_x = U.fxy + V.fxx, txy_y = U.fyy + V.fxy;
  const double hdiv = txx_x * u + txx * U.fx + txy_x * v + txy * V.fx + gPr * Q.fxx + txy_y * u + txy * U.fy +
                      tyy_y * v + tyy * V.fy + gPr * Q.fyy;
  S[0] = R.ft + mx + ny;
  S[1] = mt + mx * u + m * U.fx + px + my * v + m * V.fy - (txx_x + txy_y) * rRe;
  S[2] = nt + nx * u + n * U.fx + ny * v + n * V.fy + py - (txy_x + tyy_y) * rRe;
  S[3] = Et + (Ex + px) * u + (E + p) * U.fx + (Ey + py) * v + (E + p) * V.fy - hdiv * rRe;
}

// adds the source's cell average and scaled first moments at t = t0 + cst * dt (dt the
// device-side step of the current attempt) to rhs, on the interior cells
__device__ __forceinline__ void source_body(const Grid& g, const Quad4& qd, double t0, double cst,
                                            const Diag* __restrict__ diag, double* __restrict__ rhs, int gx,
                                            int gy) {
  const int i = gx, j = gy;
  if (i >= g.nx || j >= g.ny) return;
  const double t = t0 + cst * diag->dt;
  const double amp = 0.1 * exp(-t);
  const double xc = g.x0 + (i + 0.5) * g.dx, yc = g.y0 + (j + 0.5) * g.dy;
  double acc[12];
#pragma unroll
  for (int k = 0; k < 12; k++) acc[k] = 0.0;
#pragma unroll 1
  for (int a = 0; a < 4; a++)
#pragma unroll
    for (int b = 0; b < 4; b++) {
      double S[4];
      mms_source(g, xc + qd.nd[a] * g.dx, yc + qd.nd[b] * g.dy, amp, S);
      const double w = qd.wt[a] * qd.wt[b];
#pragma unroll
      for (int v = 0; v < 4; v++) {
        acc[v] += w * S[v];
        acc[4 + v] += w * qd.nd[a] * S[v];
        acc[8 + v] += w * qd.nd[b] * S[v];
      }
    }
  const long long c = cidx(g, i, j);
#pragma unroll
  for (int k = 0; k < 12; k++) rhs[(long long)k * g.ps + c] += acc[k];
}

}  // namespace hw
