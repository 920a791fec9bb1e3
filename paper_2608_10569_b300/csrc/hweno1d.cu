// B300 (sm_103a) one-dimensional HWENO-GR / HWENO-DR solver (Sec. 2 of Guo, Fan, Zhao,
// arXiv 2608.10569) and the C ABI declared in include/hweno1d.h.
//
// The per-cell functions are __host__ __device__: they hold no thread-level state.
// One thread block owns one problem: its threads stride over the cells in each phase
// of the spatial operator (ghost fill, characteristic reconstruction and limiter,
// gradients, interface fluxes, moment balances), with __syncthreads between phases;
// block reductions give alpha*, beta and the admissibility flags, and thread 0 takes
// the time-step, restart and termination decisions, which shared memory broadcasts.
// Every loop is bounded (cells, max_steps, max_halvings); nothing waits on another
// block.
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <vector>

#include "hweno.h"
#include "hweno1d.h"
#include "hweno1d_stencil.h"

namespace hw1 {

constexpr int G = 4;         // ghost cells per end
constexpr int THREADS = 256;
constexpr double GAM0 = 199.0 / 200.0, GAML = 1.0 / 400.0;  // linear weights (Appendix A.1)
constexpr double SQ5_10 = 0.22360679774997896964;            // sqrt(5)/10: interior Lobatto nodes
constexpr double TWO_PI = 6.283185307179586476925286766559;

struct Prob {
  int n, bc0, bc1, scheme, max_halvings, source;
  double x0, dx, rdx, gamma, rPr, rRe, cfl, visc_cap, eps_pp, eps_weno;
  double inflow[2][3];
  double* q;    // [6][n] state (device)
  double* w;    // workspace (device), laid out by layout()
};

// workspace of one problem: padded planes of P = n + 2G cells (state 6, Lobatto values
// 12, their derivatives 12, modified moments 3, weak moments 4, gradients 8, fluxes 3,
// LF coefficients 1), then planes of n cells (residuals 6 + 6, modified moments 3 + 3,
// stage states 6 + 6 + 6)
constexpr int PADDED_PLANES = 6 + 12 + 12 + 3 + 4 + 8 + 3 + 1;
constexpr int CELL_PLANES = 6 + 6 + 3 + 3 + 6 + 6 + 6;
__host__ __device__ inline long long workspace_doubles(int n) {
  return (long long)(n + 2 * G) * PADDED_PLANES + (long long)n * CELL_PLANES;
}

struct Ptrs {
  double *Q, *pts, *dpts, *mom, *rw, *grad, *flux, *bf;  // padded, [k][P]
  double *r0, *r, *m0, *m, *q1, *q2, *q3;                // [k][n]
};

__host__ __device__ __forceinline__ Ptrs layout(const Prob& p) {
  const long long P = p.n + 2 * G;
  double* a = p.w;
  Ptrs s;
  s.Q = a; a += 6 * P;
  s.pts = a; a += 12 * P;
  s.dpts = a; a += 12 * P;
  s.mom = a; a += 3 * P;
  s.rw = a; a += 4 * P;
  s.grad = a; a += 8 * P;
  s.flux = a; a += 3 * P;
  s.bf = a; a += P;
  s.r0 = a; a += 6 * (long long)p.n;
  s.r = a; a += 6 * (long long)p.n;
  s.m0 = a; a += 3 * (long long)p.n;
  s.m = a; a += 3 * (long long)p.n;
  s.q1 = a; a += 6 * (long long)p.n;
  s.q2 = a; a += 6 * (long long)p.n;
  s.q3 = a;
  return s;
}

__host__ __device__ __forceinline__ double lnode(int g) { return g == 0 ? -0.5 : (g == 1 ? -SQ5_10 : (g == 2 ? SQ5_10 : 0.5)); }
__host__ __device__ __forceinline__ double lweight(int g) { return (g == 0 || g == 3) ? 1.0 / 12.0 : 5.0 / 12.0; }

__host__ __device__ __forceinline__ double pressure(const double* u, double g) {
  return (g - 1.0) * (u[2] - 0.5 * u[1] * u[1] / u[0]);
}

// ---------------------------------------------------------------------------
// ghost fill of the padded state (Remark 4.1); k = padded index, cell i = k - G
__host__ __device__ void fetch(const Prob& p, const double* q, int i, double* out) {
  const int n = p.n;
  if (i >= 0 && i < n) {
#pragma unroll
    for (int k = 0; k < 6; k++) out[k] = q[k * n + i];
    return;
  }
  const int side = i < 0 ? 0 : 1;
  const int bc = side == 0 ? p.bc0 : p.bc1;
  if (bc == HWENO1D_BC_PERIODIC) {
    const int s = ((i % n) + n) % n;
    for (int k = 0; k < 6; k++) out[k] = q[k * n + s];
  } else if (bc == HWENO1D_BC_REFLECTIVE) {
    const int s = side == 0 ? -1 - i : 2 * n - 1 - i;
    const double par[3] = {1.0, -1.0, 1.0};
    for (int v = 0; v < 3; v++) {
      out[v] = par[v] * q[v * n + s];
      out[3 + v] = -par[v] * q[(3 + v) * n + s];
    }
  } else if (bc == HWENO1D_BC_INFLOW) {
    for (int v = 0; v < 3; v++) {
      out[v] = p.inflow[side][v];
      out[3 + v] = 0.0;
    }
  } else {
    const int s = side == 0 ? 0 : n - 1;
    for (int k = 0; k < 6; k++) out[k] = q[k * n + s];
  }
}

// ---------------------------------------------------------------------------
// scalar HWENO (Appendix A.1) as the coefficients of the combined polynomial: the
// weights are constant over the cell, so Eq. (2.4)'s combination of the candidates is
// one quartic C; its values, derivatives (Eq. (2.5)) and moment follow from C
__host__ __device__ void hweno1(const double* d, double eps, double* C) {
  double c0[5];
  hw1_p0_coeffs<double>(d, c0);
  const double sm = d[1] - d[0], sp = d[2] - d[1];
  const double b0 = hw1_beta_quartic<double>(c0), b1 = sm * sm, b2 = sp * sp;
  const double ts = 0.5 * (fabs(b0 - b1) + fabs(b0 - b2));
  const double tau = ts * ts;
  const double w0 = GAM0 * (1.0 + tau / (b0 + eps));
  const double w1 = GAML * (1.0 + tau / (b1 + eps));
  const double w2 = GAML * (1.0 + tau / (b2 + eps));
  const double rs = 1.0 / (w0 + w1 + w2);
  const double a0 = w0 * rs / GAM0;
  const double a1 = w1 * rs - a0 * GAML, a2 = w2 * rs - a0 * GAML;
#pragma unroll
  for (int k = 0; k < 5; k++) C[k] = a0 * c0[k];
  C[0] += (a1 + a2) * d[1];
  C[1] += a1 * sm + a2 * sp;
}

__host__ __device__ __forceinline__ double poly5(const double* C, double x) {
  return C[0] + x * (C[1] + x * (C[2] + x * (C[3] + x * C[4])));
}
__host__ __device__ __forceinline__ double dpoly5(const double* C, double x) {
  return C[1] + x * (2.0 * C[2] + x * (3.0 * C[3] + x * 4.0 * C[4]));
}

// eigenvectors of the Jacobian of f^a at u (fields u - c, u, u + c) and their inverse
__host__ __device__ void eigen(const double* ub, double g, double L[3][3], double R[3][3]) {
  const double rho = ub[0], u = ub[1] / rho;
  const double p = pressure(ub, g);
  const double c = sqrt(g * p / rho);
  const double H = (ub[2] + p) / rho;
  R[0][0] = 1.0; R[0][1] = 1.0; R[0][2] = 1.0;
  R[1][0] = u - c; R[1][1] = u; R[1][2] = u + c;
  R[2][0] = H - u * c; R[2][1] = 0.5 * u * u; R[2][2] = H + u * c;
  const double b1 = (g - 1.0) / (c * c), b2 = 0.5 * b1 * u * u, rc = 1.0 / c;
  L[0][0] = 0.5 * (b2 + u * rc); L[0][1] = -0.5 * (b1 * u + rc); L[0][2] = 0.5 * b1;
  L[1][0] = 1.0 - b2;            L[1][1] = b1 * u;               L[1][2] = -b1;
  L[2][0] = 0.5 * (b2 - u * rc); L[2][1] = -0.5 * (b1 * u - rc); L[2][2] = 0.5 * b1;
}

// characteristic reconstruction of padded cell k (Sec. 2.1, Eq. (2.4)): the Lobatto
// values, their x-derivatives (Eq. (2.5)) and the modified moment, then the limiter
__host__ __device__ int cons_cell(const Prob& p, const Ptrs& s, int k) {
  const long long P = p.n + 2 * G;
  double ub[3], ql[6], qr[6];
  for (int v = 0; v < 3; v++) ub[v] = s.Q[v * P + k];
  for (int m = 0; m < 6; m++) {
    ql[m] = s.Q[m * P + k - 1];
    qr[m] = s.Q[m * P + k + 1];
  }
  double L[3][3], R[3][3];
  eigen(ub, p.gamma, L, R);
  double cp[4][3], cd[4][3], cm[3];
  for (int f = 0; f < 3; f++) {
    double d[5] = {0, 0, 0, 0, 0};
    for (int v = 0; v < 3; v++) {
      d[0] += L[f][v] * ql[v];
      d[1] += L[f][v] * ub[v];
      d[2] += L[f][v] * qr[v];
      d[3] += L[f][v] * ql[3 + v];
      d[4] += L[f][v] * qr[3 + v];
    }
    double C[5];
    hweno1(d, p.eps_weno, C);
    for (int g = 0; g < 4; g++) {
      cp[g][f] = poly5(C, lnode(g));
      cd[g][f] = dpoly5(C, lnode(g)) * p.rdx;
    }
    cm[f] = hw1_moment<double>(C);
  }
  double pts[4][3];
  for (int v = 0; v < 3; v++) {
    for (int g = 0; g < 4; g++) {
      double a = 0.0, b = 0.0;
      for (int f = 0; f < 3; f++) {
        a += R[v][f] * cp[g][f];
        b += R[v][f] * cd[g][f];
      }
      pts[g][v] = a;
      s.dpts[(3 * g + v) * P + k] = b;
    }
    double a = 0.0;
    for (int f = 0; f < 3; f++) a += R[v][f] * cm[f];
    s.mom[v * P + k] = a;
  }
  // PP limiter (Sec. 2.1): all four Lobatto values rescaled about the cell average;
  // active when either factor is below 1
  int active = 0;
  const double pb = pressure(ub, p.gamma);
  if (ub[0] > 0.0 && pb > 0.0) {
    double eps = fmin(p.eps_pp, fmin(ub[0], pb));
    double rmin = ub[0];
    for (int g = 0; g < 4; g++) rmin = fmin(rmin, pts[g][0]);
    const double thr = rmin < eps ? (ub[0] - eps) / (ub[0] - rmin) : 1.0;
    double thp = 1.0;
    for (int g = 0; g < 4; g++) {
      pts[g][0] = ub[0] + thr * (pts[g][0] - ub[0]);
      if (pressure(pts[g], p.gamma) < eps) {
        // smallest t in [0, 1] with p(ub + t (u - ub)) = eps
        const double dr = pts[g][0] - ub[0], dm = pts[g][1] - ub[1], dE = pts[g][2] - ub[2];
        const double kk = eps / (p.gamma - 1.0);
        const double A = dE * dr - 0.5 * dm * dm;
        const double B = ub[2] * dr + dE * ub[0] - ub[1] * dm - kk * dr;
        const double Cq = ub[2] * ub[0] - 0.5 * ub[1] * ub[1] - kk * ub[0];
        double t;
        if (fabs(A) < 1e-300) {
          t = -Cq / B;
        } else {
          const double sq = sqrt(fmax(B * B - 4.0 * A * Cq, 0.0));
          const double t1 = (-B - sq) / (2.0 * A), t2 = (-B + sq) / (2.0 * A);
          t = 2.0;
          if (t1 >= 0.0 && t1 <= 1.0) t = t1;
          if (t2 >= 0.0 && t2 <= 1.0 && t2 < t) t = t2;
        }
        thp = fmin(thp, fmin(fmax(t, 0.0), 1.0));
      }
    }
    for (int g = 0; g < 4; g++)
      for (int v = 0; v < 3; v++) pts[g][v] = ub[v] + thp * (pts[g][v] - ub[v]);
    active = thr < 1.0 || thp < 1.0;
  }
  for (int g = 0; g < 4; g++)
    for (int v = 0; v < 3; v++) s.pts[(3 * g + v) * P + k] = pts[g][v];
  return active;
}

__host__ __device__ __forceinline__ void dissip(const double* st, double* w) {
  w[0] = st[1] / st[0];
  w[1] = st[2] / st[0] - 0.5 * w[0] * w[0];
}

__host__ __device__ __forceinline__ void point(const Ptrs& s, long long P, int k, int g, double* st) {
  for (int v = 0; v < 3; v++) st[v] = s.pts[(3 * g + v) * P + k];
}

// Eqs. (2.6), (2.8): interface averages and weak moments of u_x, e_x in padded cell k
__host__ __device__ void weak_cell(const Prob& p, const Ptrs& s, int k) {
  const long long P = p.n + 2 * G;
  double a[3], b[3], wa[2], wb[2], wl[2], wr[2], wbar[2] = {0.0, 0.0};
  point(s, P, k - 1, 3, a); point(s, P, k, 0, b);
  dissip(a, wa); dissip(b, wb);
  for (int n = 0; n < 2; n++) wl[n] = 0.5 * (wa[n] + wb[n]);
  point(s, P, k, 3, a); point(s, P, k + 1, 0, b);
  dissip(a, wa); dissip(b, wb);
  for (int n = 0; n < 2; n++) wr[n] = 0.5 * (wa[n] + wb[n]);
  for (int g = 0; g < 4; g++) {
    point(s, P, k, g, a);
    dissip(a, wa);
    for (int n = 0; n < 2; n++) wbar[n] += lweight(g) * wa[n];
  }
  for (int n = 0; n < 2; n++) {
    s.rw[(2 * n) * P + k] = (wr[n] - wl[n]) * p.rdx;
    s.rw[(2 * n + 1) * P + k] = (0.5 * (wr[n] + wl[n]) - wbar[n]) * p.rdx;
  }
}

// Eq. (2.9): GR gradients at the Lobatto points of padded cell k
__host__ __device__ void grad_cell(const Prob& p, const Ptrs& s, int k) {
  const long long P = p.n + 2 * G;
  for (int n = 0; n < 2; n++) {
    const double* A = s.rw + (2 * n) * P;
    const double* B = s.rw + (2 * n + 1) * P;
    const double d[5] = {A[k - 1], A[k], A[k + 1], B[k - 1], B[k + 1]};
    double C[5];
    hweno1(d, p.eps_weno, C);
    for (int g = 0; g < 4; g++) s.grad[(2 * g + n) * P + k] = poly5(C, lnode(g));
  }
}

// Eq. (2.5) then the chain rule with the limited values: DR gradients of cell k
__host__ __device__ void dr_cell(const Prob& p, const Ptrs& s, int k) {
  const long long P = p.n + 2 * G;
  for (int g = 0; g < 4; g++) {
    double st[3];
    point(s, P, k, g, st);
    const double rr = 1.0 / st[0];
    const double u = st[1] * rr, en = st[2] * rr;
    const double d0 = s.dpts[(3 * g) * P + k], d1 = s.dpts[(3 * g + 1) * P + k], d2 = s.dpts[(3 * g + 2) * P + k];
    const double ux = (d1 - u * d0) * rr;
    s.grad[(2 * g) * P + k] = ux;
    s.grad[(2 * g + 1) * P + k] = (d2 - en * d0) * rr - u * ux;
  }
}

// f = f^a - f^d of Eq. (2.1), tau = 4/3 u_x / Re, q = -g e_x / (Pr Re)
__host__ __device__ __forceinline__ void phys_flux(const Prob& p, const double* st, double ux, double ex, double* f) {
  const double rho = st[0], u = st[1] / rho, pr = pressure(st, p.gamma);
  const double tau = (4.0 / 3.0) * ux * p.rRe, qh = -p.gamma * ex * p.rPr * p.rRe;
  f[0] = rho * u;
  f[1] = rho * u * u + pr - tau;
  f[2] = (st[2] + pr) * u - (tau * u - qh);
}

// max(|u| + c, the PP wave-speed bound of Eq. (2.3))
__host__ __device__ __forceinline__ double wave_bound(const Prob& p, const double* st, double ux, double ex) {
  const double rho = st[0], u = st[1] / rho, pr = pressure(st, p.gamma);
  const double e = pr / ((p.gamma - 1.0) * rho);
  const double tau = (4.0 / 3.0) * ux * p.rRe, qh = -p.gamma * ex * p.rPr * p.rRe;
  const double pp = fabs(u) + (sqrt(rho * rho * qh * qh + 2.0 * rho * rho * e * (tau - pr) * (tau - pr)) + rho * fabs(qh)) /
                                  (2.0 * rho * rho * e);
  return fmax(fabs(u) + sqrt(p.gamma * pr / rho), pp);
}

// Example 5.1's source at (x, t), and its cell average and scaled moment (4-point Gauss)
__host__ __device__ void mms_source(const Prob& p, double x, double t, double* S) {
  const double a = 0.2 * exp(-t);
  double sn, cs;
  sincos(TWO_PI * x, &sn, &cs);
  const double rho = 2.0 + a * sn, rho_t = -a * sn, rho_x = a * TWO_PI * cs;
  const double u = 1.0 + a * cs, u_t = -a * cs, u_x = -a * TWO_PI * sn, u_xx = -a * TWO_PI * TWO_PI * cs;
  const double e = 1.0 + a * sn, e_t = -a * sn, e_x = a * TWO_PI * cs, e_xx = -a * TWO_PI * TWO_PI * sn;
  const double g = p.gamma;
  const double m_t = rho_t * u + rho * u_t, m_x = rho_x * u + rho * u_x, m = rho * u;
  const double k = 0.5 * u * u;
  const double E = rho * (e + k), E_t = rho_t * (e + k) + rho * (e_t + u * u_t), E_x = rho_x * (e + k) + rho * (e_x + u * u_x);
  const double pr = (g - 1.0) * rho * e, p_x = (g - 1.0) * (rho_x * e + rho * e_x);
  const double tau = (4.0 / 3.0) * u_x * p.rRe, tau_x = (4.0 / 3.0) * u_xx * p.rRe;
  const double q_x = -g * e_xx * p.rPr * p.rRe;
  S[0] = rho_t + m_x;
  S[1] = m_t + m_x * u + m * u_x + p_x - tau_x;
  S[2] = E_t + (E_x + p_x) * u + (E + pr) * u_x - (u_x * tau + u * tau_x - q_x);
}

// ---------------------------------------------------------------------------
// block reductions
__device__ double block_max(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = sh[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); k++) m = fmax(m, sh[k]);
    sh[0] = m;
  }
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

// block sum of small non-negative integers held as doubles (exact)
__device__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = sh[0];
    for (int k = 1; k < (int)(blockDim.x >> 5); k++) m += sh[k];
    sh[0] = m;
  }
  __syncthreads();
  const double r = sh[0];
  __syncthreads();
  return r;
}

// one evaluation of Eq. (2.2) at state q (averages and moments, [6][n]) and time t:
// rhs [6][n], mom [3][n]; returns alpha*, beta and the interior cells the limiter acted
// on through the block; *bad is set when an output is not finite
__device__ void residual(const Prob& p, const Ptrs& s, const double* q, double t, double* rhs, double* mom,
                         double* sh, double* alpha, double* beta, double* act, int* bad) {
  const int n = p.n;
  const long long P = n + 2 * G;
  for (int k = threadIdx.x; k < P; k += blockDim.x) {
    double v[6];
    fetch(p, q, k - G, v);
    for (int m = 0; m < 6; m++) s.Q[m * P + k] = v[m];
  }
  __syncthreads();
  double act_local = 0.0;
  for (int k = threadIdx.x; k < n + 6; k += blockDim.x) {  // cells -3 .. n+2
    const int a = cons_cell(p, s, k + 1);
    if (k >= 3 && k < n + 3) act_local += a;
  }
  __syncthreads();
  if (p.scheme == 1) {
    for (int k = threadIdx.x; k < n + 2; k += blockDim.x) dr_cell(p, s, k + 3);  // cells -1 .. n
  } else {
    for (int k = threadIdx.x; k < n + 4; k += blockDim.x) weak_cell(p, s, k + 2);  // cells -2 .. n+1
    __syncthreads();
    for (int k = threadIdx.x; k < n + 2; k += blockDim.x) grad_cell(p, s, k + 3);  // cells -1 .. n
  }
  __syncthreads();
  double amax = 0.0, bmax = 0.0;
  for (int k = threadIdx.x; k < n + 1; k += blockDim.x) {  // interfaces right of cells -1 .. n-1
    const int kl = k + 3, kr = k + 4;
    double sl[3], sr[3];
    point(s, P, kl, 3, sl);
    point(s, P, kr, 0, sr);
    const double uxl = s.grad[6 * P + kl], exl = s.grad[7 * P + kl];
    const double uxr = s.grad[0 * P + kr], exr = s.grad[1 * P + kr];
    const double b = fmax(wave_bound(p, sl, uxl, exl), wave_bound(p, sr, uxr, exr));
    double fl[3], fr[3];
    phys_flux(p, sl, uxl, exl, fl);
    phys_flux(p, sr, uxr, exr, fr);
    for (int v = 0; v < 3; v++) s.flux[v * P + kl] = 0.5 * (fl[v] + fr[v] - b * (sr[v] - sl[v]));
    bmax = fmax(bmax, b);
    // alpha*: the traces on the interfaces of interior cells
    if (k >= 1) amax = fmax(amax, fabs(sl[1] / sl[0]) + sqrt(p.gamma * pressure(sl, p.gamma) / sl[0]));
    if (k <= n - 1) amax = fmax(amax, fabs(sr[1] / sr[0]) + sqrt(p.gamma * pressure(sr, p.gamma) / sr[0]));
  }
  __syncthreads();
  int nonfinite = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int k = i + G;
    double vol[3] = {0.0, 0.0, 0.0};
    for (int g = 0; g < 4; g++) {
      double st[3], f[3];
      point(s, P, k, g, st);
      phys_flux(p, st, s.grad[(2 * g) * P + k], s.grad[(2 * g + 1) * P + k], f);
      for (int v = 0; v < 3; v++) vol[v] += lweight(g) * f[v];
    }
    double r[6];
    for (int v = 0; v < 3; v++) {
      const double fR = s.flux[v * P + k], fL = s.flux[v * P + k - 1];
      r[v] = -(fR - fL) * p.rdx;
      r[3 + v] = -(fL + fR) * (0.5 * p.rdx) + vol[v] * p.rdx;
    }
    if (p.source == HWENO1D_SOURCE_MMS51) {
      const double ri = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), ro = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
      const double wi = (18.0 + sqrt(30.0)) / 72.0, wo = (18.0 - sqrt(30.0)) / 72.0;
      const double nd[4] = {-0.5 * ro, -0.5 * ri, 0.5 * ri, 0.5 * ro}, wt[4] = {wo, wi, wi, wo};
      const double xc = p.x0 + (i + 0.5) * p.dx;
      for (int a = 0; a < 4; a++) {
        double S[3];
        mms_source(p, xc + nd[a] * p.dx, t, S);
        for (int v = 0; v < 3; v++) {
          r[v] += wt[a] * S[v];
          r[3 + v] += wt[a] * nd[a] * S[v];
        }
      }
    }
    for (int m = 0; m < 6; m++) {
      rhs[m * n + i] = r[m];
      if (!isfinite(r[m])) nonfinite = 1;
    }
    for (int v = 0; v < 3; v++) mom[v * n + i] = s.mom[v * P + k];
  }
  *alpha = block_max(amax, sh);
  *beta = block_max(bmax, sh);
  *act = block_sum(act_local, sh);
  *bad = __syncthreads_or(nonfinite);
}

// the averages of a stage are admissible: positive density and pressure everywhere
__device__ int admissible(const Prob& p, const double* q) {
  int bad = 0;
  for (int i = threadIdx.x; i < p.n; i += blockDim.x) {
    const double u[3] = {q[i], q[p.n + i], q[2 * p.n + i]};
    if (!(u[0] > 0.0) || !(pressure(u, p.gamma) > 0.0)) bad = 1;
  }
  return !__syncthreads_or(bad);
}

// out = a * [base_avg; base_mom] + b * ([cur_avg; cur_mom] + dt * r) on the interior
__device__ void stage(const Prob& p, double a, const double* base, const double* bmom, double b, const double* cur,
                      const double* cmom, double dt, const double* r, double* out) {
  const int n = p.n;
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    for (int v = 0; v < 3; v++) {
      out[v * n + i] = a * base[v * n + i] + b * (cur[v * n + i] + dt * r[v * n + i]);
      out[(3 + v) * n + i] = a * bmom[v * n + i] + b * (cmom[v * n + i] + dt * r[(3 + v) * n + i]);
    }
  __syncthreads();
}

// mode 0: advance to t_end (max_steps); mode 1: one step (dt_in > 0 forced); mode 2:
// one residual (rhs into r0, modified moments into m0).  out per problem (OUT doubles):
// the time reached (mode 0) or the step taken (mode 1), steps, rejections, status, and
// the limiter activations (interior cells the limiter acted on, summed over the three
// stage evaluations of the accepted steps; mode 2: of the one evaluation).
constexpr int OUT = 5;
__global__ void __launch_bounds__(THREADS) k_solve(const Prob* probs, int mode, double t0, double t_end,
                                                    int max_steps, double dt_in, double* out) {
  const Prob& p = probs[blockIdx.x];
  const Ptrs s = layout(p);
  __shared__ double sh[THREADS / 32];
  __shared__ double s_dt;
  double t = t0, dt_last = 0.0, alpha, beta, act, pp_total = 0.0;
  int steps = 0, rej_total = 0, status = 0, bad;
  double* o = out + (long long)OUT * blockIdx.x;
  if (mode == 2) {
    residual(p, s, p.q, t0, s.r0, s.m0, sh, &alpha, &beta, &act, &bad);
    if (threadIdx.x == 0) {
      o[0] = t0;
      o[3] = bad ? HWENO_ERR_NONFINITE : 0;
      o[4] = act;
    }
    return;
  }
  const int n = p.n;
  for (int it = 0; it < (mode == 1 ? 1 : max_steps); it++) {
    if (mode == 0 && !(t < t_end)) break;
    residual(p, s, p.q, t, s.r0, s.m0, sh, &alpha, &beta, &act, &bad);
    if (bad) { status = HWENO_ERR_NONFINITE; break; }
    const double act0 = act;
    if (threadIdx.x == 0) {
      double dt = dt_in > 0.0 ? dt_in : fmin(p.cfl * p.dx / alpha, p.visc_cap);
      if (mode == 0 && t + dt > t_end) dt = t_end - t;
      s_dt = dt;
    }
    __syncthreads();
    double dt = s_dt;
    int rej = 0, ok = 0;
    double sa = act0;
    for (int h = 0; h <= p.max_halvings; h++) {
      sa = act0;  // the activations of an attempt count only when it is accepted
      // stage 1: [u; vhat]^n + dt F
      for (int i = threadIdx.x; i < n; i += blockDim.x)
        for (int v = 0; v < 3; v++) {
          s.q1[v * n + i] = p.q[v * n + i] + dt * s.r0[v * n + i];
          s.q1[(3 + v) * n + i] = s.m0[v * n + i] + dt * s.r0[(3 + v) * n + i];
        }
      __syncthreads();
      ok = admissible(p, s.q1);
      if (ok) {
        residual(p, s, s.q1, t + dt, s.r, s.m, sh, &alpha, &beta, &act, &bad);
        sa += act;
        ok = !bad;
      }
      if (ok) {
        stage(p, 0.75, p.q, s.m0, 0.25, s.q1, s.m, dt, s.r, s.q2);
        ok = admissible(p, s.q2);
      }
      if (ok) {
        residual(p, s, s.q2, t + 0.5 * dt, s.r, s.m, sh, &alpha, &beta, &act, &bad);
        sa += act;
        ok = !bad;
      }
      if (ok) {
        stage(p, 1.0 / 3.0, p.q, s.m0, 2.0 / 3.0, s.q2, s.m, dt, s.r, s.q3);
        ok = admissible(p, s.q3);
      }
      if (ok) break;
      rej++;
      dt *= 0.5;
    }
    if (!ok) { status = HWENO_ERR_INADMISSIBLE; break; }  // restarts count for accepted steps only
    for (int i = threadIdx.x; i < 6 * n; i += blockDim.x) p.q[i] = s.q3[i];
    __syncthreads();
    t += dt;
    dt_last = dt;
    steps++;
    rej_total += rej;
    pp_total += sa;
    if (mode == 0 && t_end - t <= 1e-14 * fmax(1.0, fabs(t_end))) t = t_end;
  }
  if (threadIdx.x == 0) {
    o[0] = mode == 0 ? t : dt_last;
    o[1] = steps;
    o[2] = rej_total;
    o[3] = status;
    o[4] = pp_total;
  }
}

}  // namespace hw1

// ---------------------------------------------------------------------------
// C ABI
static char g_err1[512] = "no error";

static int fail1(int rc, const char* msg) {
  snprintf(g_err1, sizeof(g_err1), "%s", msg);
  return rc;
}

static int check_cfg(const hweno1d_config& c) {
  if (c.n < 4 || c.n > HWENO1D_MAX_CELLS) return fail1(HWENO_ERR_ARG, "n must be in 4 .. HWENO1D_MAX_CELLS");
  for (int k = 0; k < 2; k++)
    if (c.bc[k] < HWENO1D_BC_PERIODIC || c.bc[k] > HWENO1D_BC_OUTFLOW) return fail1(HWENO_ERR_ARG, "unknown boundary");
  if ((c.bc[0] == HWENO1D_BC_PERIODIC) != (c.bc[1] == HWENO1D_BC_PERIODIC))
    return fail1(HWENO_ERR_ARG, "periodic ends must be set on both sides");
  if (c.scheme != HWENO_SCHEME_GR && c.scheme != HWENO_SCHEME_DR) return fail1(HWENO_ERR_ARG, "unknown scheme");
  if (c.source != HWENO1D_SOURCE_NONE && c.source != HWENO1D_SOURCE_MMS51)
    return fail1(HWENO_ERR_ARG, "unknown source term");
  if (!(c.x1 > c.x0) || !(c.gamma > 1.0) || !(c.Pr > 0.0) || !(c.Re > 0.0))
    return fail1(HWENO_ERR_ARG, "need x1 > x0, gamma > 1, Pr > 0, Re > 0");
  if (!(c.cfl > 0.0) || !(c.b_visc > 0.0) || !(c.eps_pp > 0.0) || !(c.eps_weno > 0.0) || c.max_halvings < 0)
    return fail1(HWENO_ERR_ARG, "cfl, b_visc, eps_pp, eps_weno must be > 0");
  return HWENO_OK;
}

static hw1::Prob make_prob(const hweno1d_config& c, double* q, double* w) {
  hw1::Prob p;
  p.n = c.n;
  p.bc0 = c.bc[0];
  p.bc1 = c.bc[1];
  p.scheme = c.scheme;
  p.max_halvings = c.max_halvings;
  p.source = c.source;
  p.x0 = c.x0;
  p.dx = (c.x1 - c.x0) / c.n;
  p.rdx = 1.0 / p.dx;
  p.gamma = c.gamma;
  p.rPr = 1.0 / c.Pr;
  p.rRe = 1.0 / c.Re;
  p.cfl = c.cfl;
  p.visc_cap = c.b_visc * c.Re * p.dx * p.dx;
  p.eps_pp = c.eps_pp;
  p.eps_weno = c.eps_weno;
  for (int s = 0; s < 2; s++)
    for (int v = 0; v < 3; v++) p.inflow[s][v] = c.inflow[s][v];
  p.q = q;
  p.w = w;
  return p;
}

// runs mode on nprob problems; out_host OUT*nprob doubles
static int run(const hweno1d_config* cfgs, int nprob, double* const* q, int mode, double t0, double t_end,
               int max_steps, double dt_in, double* out_host, double* rhs, double* vhat, void* stream) {
  if (!cfgs || nprob < 1 || !q) return fail1(HWENO_ERR_ARG, "NULL argument or no problem");
  long long total = 0;
  for (int k = 0; k < nprob; k++) {
    int rc = check_cfg(cfgs[k]);
    if (rc) return rc;
    if (!q[k]) return fail1(HWENO_ERR_ARG, "NULL state");
    total += hw1::workspace_doubles(cfgs[k].n);
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* work = nullptr;
  hw1::Prob* dprob = nullptr;
  double* dout = nullptr;
  cudaError_t e = cudaMalloc(&work, (size_t)total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&dprob, nprob * sizeof(hw1::Prob));
  if (e == cudaSuccess) e = cudaMalloc(&dout, hw1::OUT * nprob * sizeof(double));
  std::vector<hw1::Prob> hp(nprob);
  long long off = 0;
  for (int k = 0; k < nprob; k++) {
    hp[k] = make_prob(cfgs[k], q[k], work + off);
    off += hw1::workspace_doubles(cfgs[k].n);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(dout, 0, hw1::OUT * nprob * sizeof(double), st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(dprob, hp.data(), nprob * sizeof(hw1::Prob), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    hw1::k_solve<<<nprob, hw1::THREADS, 0, st>>>(dprob, mode, t0, t_end, max_steps, dt_in, dout);
    e = cudaGetLastError();
  }
  // the residual of mode 2 sits in the first problem's workspace (r0, m0)
  if (e == cudaSuccess && mode == 2) {
    const int n = cfgs[0].n;
    const long long P = n + 2 * hw1::G;
    const double* r0 = work + P * hw1::PADDED_PLANES;
    const double* m0 = r0 + 12LL * n;
    e = cudaMemcpyAsync(rhs, r0, 6 * (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess && vhat)
      e = cudaMemcpyAsync(vhat, m0, 3 * (size_t)n * sizeof(double), cudaMemcpyDeviceToDevice, st);
  }
  std::vector<double> ho(hw1::OUT * nprob, 0.0);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ho.data(), dout, hw1::OUT * nprob * sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(work);
  cudaFree(dprob);
  cudaFree(dout);
  if (e != cudaSuccess) return fail1(HWENO_ERR_CUDA, cudaGetErrorString(e));
  if (out_host) memcpy(out_host, ho.data(), ho.size() * sizeof(double));
  return HWENO_OK;
}

extern "C" {

int hweno1d_config_default(hweno1d_config* c) {
  if (!c) return HWENO_ERR_ARG;
  memset(c, 0, sizeof(*c));
  c->x0 = 0.0; c->x1 = 1.0;
  c->gamma = 1.4; c->Pr = 0.72; c->Re = 1000.0;
  c->cfl = 0.6; c->b_visc = 1e-3; c->eps_pp = 1e-12; c->eps_weno = 1e-8;
  c->max_halvings = 60;
  return HWENO_OK;
}

int hweno1d_advance(const hweno1d_config* cfgs, int nprob, double* const* q, double t0, double t_end,
                    int max_steps, double* out, void* stream) {
  if (max_steps < 0) return fail1(HWENO_ERR_ARG, "max_steps must be >= 0");
  return run(cfgs, nprob, q, 0, t0, t_end, max_steps, 0.0, out, nullptr, nullptr, stream);
}

int hweno1d_step(const hweno1d_config* cfg, double* q, double t, double dt, double* out, void* stream) {
  double o[hw1::OUT];
  int rc = run(cfg, 1, &q, 1, t, INFINITY, 1, dt, o, nullptr, nullptr, stream);
  if (rc) return rc;
  if (out) {
    out[0] = o[0];
    out[1] = o[2];
    out[2] = o[3];
    out[3] = o[4];
  }
  return HWENO_OK;
}

int hweno1d_residual(const hweno1d_config* cfg, const double* q, double t, double* rhs, double* vhat,
                     void* stream) {
  if (!rhs) return fail1(HWENO_ERR_ARG, "rhs is NULL");
  double* qq = const_cast<double*>(q);
  double o[hw1::OUT];
  int rc = run(cfg, 1, &qq, 2, t, t, 0, 0.0, o, rhs, vhat, stream);
  if (rc) return rc;
  if (o[3] != 0.0) return fail1(HWENO_ERR_NONFINITE, "non-finite residual");
  return HWENO_OK;
}

const char* hweno1d_last_error(void) { return g_err1; }

}  // extern "C"
