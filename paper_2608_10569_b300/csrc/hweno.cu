// B300 (sm_103a) HWENO-GR solver: kernels of the spatial operator, the SSP-RK3
// stage update, reductions, and the C ABI declared in include/hweno.h.
//
// Paper: Guo, Fan, Zhao, "An efficient and robust fifth-order HWENO scheme with
// gradient reconstruction for compressible Navier-Stokes equations" (arXiv 2608.10569).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "hweno.h"
#include "hweno_kernels.cuh"
#include "hweno_mixed.cuh"

namespace hw {

constexpr int BX = 32, BY = 4;

// ---------------------------------------------------------------------------
// conservative characteristic reconstruction, modified moments and PP limiter of
// every cell of the interior grown by 3 (Sec. 3.1, Eq. (3.4), Appendix A.2)
template <class T>
__global__ void __launch_bounds__(BX * BY) k_cons(Grid g, const double* __restrict__ q, Work w,
                                                  double* __restrict__ mom, Diag* diag) {
  const int i = blockIdx.x * BX + threadIdx.x - 3;
  const int j = blockIdx.y * BY + threadIdx.y - 3;
  unsigned long long pp = 0;
  unsigned int flags = 0;
  if (i < g.nx + 3 && j < g.ny + 3) {
    constexpr bool OFF = sizeof(T) == 4;  // FP32: reconstruct offsets from the average
    const long long c = cidx(g, i, j);
    double ub[4];
    T cc[4][15], sl[4][4], ctr[4];
#pragma unroll
    for (int v = 0; v < 4; v++) {
      double d[17];
      gather17<OFF>(g, q, v, i, j, d);
      ub[v] = q[(long long)v * g.ps + c];
      T dt[17];
#pragma unroll
      for (int k = 0; k < 17; k++) dt[k] = (T)d[k];
      hw_p0_coeffs<T>(dt, cc[v]);
      sl[v][0] = (T)(d[4] - d[3]);
      sl[v][1] = (T)(d[5] - d[4]);
      sl[v][2] = (T)(d[4] - d[1]);
      sl[v][3] = (T)(d[7] - d[4]);
      ctr[v] = OFF ? T(0) : (T)ub[v];
    }
    const T ut[4] = {(T)ub[0], (T)ub[1], (T)ub[2], (T)ub[3]};
    const T eps = (T)g.eps_weno;
    double face[12][4], vol[9][4], volx[9][4], mx[4], my[4];
    CharState<T> cs;
    char_state<T>(ut, (T)g.gamma, cs);
    recon_dir<T, 0, double>(cc, sl, ctr, cs, eps, face, volx, mx);
    recon_dir<T, 1, double>(cc, sl, ctr, cs, eps, face + 6, vol, my);
#pragma unroll
    for (int v = 0; v < 4; v++) {
#pragma unroll
      for (int k = 0; k < 12; k++)
        if (OFF) face[k][v] += ub[v];
#pragma unroll
      for (int k = 0; k < 9; k++) {
        vol[k][v] = 0.5 * (volx[k][v] + vol[k][v]);
        if (OFF) vol[k][v] += ub[v];
      }
    }
    double th[2] = {1.0, 1.0};
    const double pb = pressure(ub, g.gamma);
    const bool interior = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
    if (!(ub[0] > 0.0) || !(pb > 0.0)) {
      flags |= FLAG_BADAVG;
    } else if (pp_limit(ub, face, vol, g.gamma, g.eps_pp, th) && interior) {
      pp = 1;
    }
    // primitive (rho, u, v, e) at the 12 limited face points and the 9 volume points
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double rr = 1.0 / face[k][0];
      const double u = face[k][1] * rr, v = face[k][2] * rr;
      const double e = face[k][3] * rr - 0.5 * (u * u + v * v);
      w.face[(long long)(4 * k + 0) * g.ps + c] = face[k][0];
      w.face[(long long)(4 * k + 1) * g.ps + c] = u;
      w.face[(long long)(4 * k + 2) * g.ps + c] = v;
      w.face[(long long)(4 * k + 3) * g.ps + c] = e;
    }
    double wb[3] = {0.0, 0.0, 0.0};
#pragma unroll
    for (int G = 0; G < 3; G++)
#pragma unroll
      for (int H = 0; H < 3; H++) {
        const int k = 3 * G + H;
        const double rr = 1.0 / vol[k][0];
        const double u = vol[k][1] * rr, v = vol[k][2] * rr;
        const double e = vol[k][3] * rr - 0.5 * (u * u + v * v);
        w.vol[(long long)(4 * k + 0) * g.ps + c] = vol[k][0];
        w.vol[(long long)(4 * k + 1) * g.ps + c] = u;
        w.vol[(long long)(4 * k + 2) * g.ps + c] = v;
        w.vol[(long long)(4 * k + 3) * g.ps + c] = e;
        const double wgt = gweight<double>(G) * gweight<double>(H);
        wb[0] += wgt * u;
        wb[1] += wgt * v;
        wb[2] += wgt * e;
      }
#pragma unroll
    for (int n = 0; n < 3; n++) w.wbar[(long long)n * g.ps + c] = wb[n];
    w.theta[c] = th[0];
    w.theta[g.ps + c] = th[1];
    if (interior) {
#pragma unroll
      for (int v = 0; v < 4; v++) {
        mom[(long long)v * g.ps + c] = mx[v];
        mom[(long long)(4 + v) * g.ps + c] = my[v];
      }
    }
  }
  // block reduction of the activation count and flags: one atomic per warp
  pp = warp_sum_u64(pp);
  flags = __reduce_or_sync(0xffffffffu, flags);
  if ((threadIdx.x & 31) == 0) {
    if (pp) atomicAdd(&diag->pp_count, pp);
    if (flags) atomicOr(&diag->flags, flags);
  }
}

// face moments W^{x,0}, W^{x,1} (blockIdx.z = 0) of the x-faces right of cells
// i in [-3, nx+2), j in [-2, ny+2), and W^{y,0}, W^{y,1} (z = 1) of the y-faces
// above cells i in [-2, nx+2), j in [-3, ny+2)  (Eq. (3.6) with the interface
// average of the two traces)
__global__ void k_face_moments(Grid g, Work w) {
  const int dir = blockIdx.z;
  const int i = blockIdx.x * BX + threadIdx.x - (dir == 0 ? 3 : 2);
  const int j = blockIdx.y * BY + threadIdx.y - (dir == 0 ? 2 : 3);
  if (i >= g.nx + 2 || j >= g.ny + 2) return;
  const long long cl = cidx(g, i, j);
  const long long cr = dir == 0 ? cidx(g, i + 1, j) : cidx(g, i, j + 1);
  const int kl = dir == 0 ? 3 : 9, kr = dir == 0 ? 0 : 6;
  double W0[3] = {0.0, 0.0, 0.0}, W1[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int gp = 0; gp < 3; gp++) {
    const double wg = gweight<double>(gp), xg = gnode<double>(gp);
#pragma unroll
    for (int n = 0; n < 3; n++) {
      const double a = w.face[(long long)(4 * (kl + gp) + 1 + n) * g.ps + cl];
      const double b = w.face[(long long)(4 * (kr + gp) + 1 + n) * g.ps + cr];
      const double h = 0.5 * (a + b);
      W0[n] += wg * h;
      W1[n] += wg * h * xg;
    }
  }
  double* out = dir == 0 ? w.wx : w.wy;
#pragma unroll
  for (int n = 0; n < 3; n++) {
    out[(long long)n * g.ps + cl] = W0[n];
    out[(long long)(3 + n) * g.ps + cl] = W1[n];
  }
}

// weak-derivative moments (Eqs. (3.7)-(3.8)) of cells in the interior grown by 2
__global__ void k_weak_moments(Grid g, Work w) {
  const int i = blockIdx.x * BX + threadIdx.x - 2;
  const int j = blockIdx.y * BY + threadIdx.y - 2;
  if (i >= g.nx + 2 || j >= g.ny + 2) return;
  const long long c = cidx(g, i, j), cl = cidx(g, i - 1, j), cb = cidx(g, i, j - 1);
  const double rdx = 1.0 / g.dx, rdy = 1.0 / g.dy;
#pragma unroll
  for (int n = 0; n < 3; n++) {
    const double xr0 = w.wx[(long long)n * g.ps + c], xl0 = w.wx[(long long)n * g.ps + cl];
    const double xr1 = w.wx[(long long)(3 + n) * g.ps + c], xl1 = w.wx[(long long)(3 + n) * g.ps + cl];
    const double yt0 = w.wy[(long long)n * g.ps + c], yb0 = w.wy[(long long)n * g.ps + cb];
    const double yt1 = w.wy[(long long)(3 + n) * g.ps + c], yb1 = w.wy[(long long)(3 + n) * g.ps + cb];
    const double wb = w.wbar[(long long)n * g.ps + c];
    double* r = w.rm + (long long)(6 * n) * g.ps + c;
    r[0] = (xr0 - xl0) * rdx;
    r[g.ps] = (0.5 * (xr0 + xl0) - wb) * rdx;
    r[2 * g.ps] = (xr1 - xl1) * rdx;
    r[3 * g.ps] = (yt0 - yb0) * rdy;
    r[4 * g.ps] = (yt1 - yb1) * rdy;
    r[5 * g.ps] = (0.5 * (yt0 + yb0) - wb) * rdy;
  }
}

// gradient reconstruction (Eq. (3.9)): the scalar HWENO of Appendix A.2 applied to
// the weak-derivative moments of each of u, v, e in each direction, on cells of the
// interior grown by 1; values at the 12 face and 9 volume points
template <class T>
__global__ void __launch_bounds__(BX * BY) k_grad(Grid g, Work w) {
  const int i = blockIdx.x * BX + threadIdx.x - 1;
  const int j = blockIdx.y * BY + threadIdx.y - 1;
  if (i >= g.nx + 1 || j >= g.ny + 1) return;
  const long long c = cidx(g, i, j);
  const T eps = (T)g.eps_weno;
#pragma unroll 1
  for (int comp = 0; comp < 6; comp++) {
    const int n = comp >> 1, l = comp & 1;
    const double* A = w.rm + (long long)(6 * n + 3 * l) * g.ps;
    const double* X = A + g.ps;
    const double* Y = A + 2 * g.ps;
    constexpr bool OFF = sizeof(T) == 4;  // FP32: reconstruct offsets from the centre value
    const double cen = OFF ? A[c] : 0.0;
    T d[17];
#pragma unroll
    for (int b = -1; b <= 1; b++)
#pragma unroll
      for (int a = -1; a <= 1; a++) d[(b + 1) * 3 + (a + 1)] = (T)(A[cidx(g, i + a, j + b)] - cen);
    if (OFF) d[4] = T(0);
    d[9] = (T)X[cidx(g, i - 1, j)];
    d[10] = (T)X[cidx(g, i + 1, j)];
    d[11] = (T)Y[cidx(g, i, j - 1)];
    d[12] = (T)Y[cidx(g, i, j + 1)];
    d[13] = (T)X[cidx(g, i, j - 1)];
    d[14] = (T)X[cidx(g, i, j + 1)];
    d[15] = (T)Y[cidx(g, i - 1, j)];
    d[16] = (T)Y[cidx(g, i + 1, j)];
    T C[15];
    hweno_combine<T>(d, eps, C);
    T vx[6], vy[6], vv[9];
    eval_xfaces<T>(C, vx);
    eval_yfaces<T>(C, vy);
    eval_vol<T>(C, vv);
    double* out = w.gr + (long long)comp * g.ps + c;
    // FP64: the values themselves; FP32: offsets, restored in FP64
#pragma unroll
    for (int k = 0; k < 6; k++) out[(long long)(6 * k) * g.ps] = OFF ? cen + (double)vx[k] : (double)vx[k];
#pragma unroll
    for (int k = 0; k < 6; k++) out[(long long)(6 * (6 + k)) * g.ps] = OFF ? cen + (double)vy[k] : (double)vy[k];
#pragma unroll
    for (int k = 0; k < 9; k++) out[(long long)(6 * (12 + k)) * g.ps] = OFF ? cen + (double)vv[k] : (double)vv[k];
  }
}

// PP local Lax-Friedrichs fluxes (Eq. (3.3)) of the interior faces: x-faces right
// of cells i in [-1, nx), j in [0, ny) (blockIdx.z = 0); y-faces above cells
// i in [0, nx), j in [-1, ny) (z = 1).  Also the face maxima alpha* and beta.
template <class T>
__global__ void __launch_bounds__(BX * BY) k_flux(Grid g, Work w, Diag* diag) {
  const int dir = blockIdx.z;
  const int i = blockIdx.x * BX + threadIdx.x - (dir == 0 ? 1 : 0);
  const int j = blockIdx.y * BY + threadIdx.y - (dir == 0 ? 0 : 1);
  double amax = 0.0, bmax = 0.0;
  if (i < g.nx && j < g.ny) {
    const long long cl = cidx(g, i, j);
    const long long cr = dir == 0 ? cidx(g, i + 1, j) : cidx(g, i, j + 1);
    const int kl = dir == 0 ? 3 : 9, kr = dir == 0 ? 0 : 6;
    const T gam = (T)g.gamma, rPr = (T)(1.0 / g.Pr), rRe = (T)(1.0 / g.Re);
    T st[2][3][4], gs[2][3][6];
#pragma unroll
    for (int gp = 0; gp < 3; gp++)
#pragma unroll
      for (int s = 0; s < 2; s++) {
        const long long cc = s == 0 ? cl : cr;
        const int k = (s == 0 ? kl : kr) + gp;
#pragma unroll
        for (int v = 0; v < 4; v++) st[s][gp][v] = (T)w.face[(long long)(4 * k + v) * g.ps + cc];
#pragma unroll
        for (int n = 0; n < 6; n++) gs[s][gp][n] = (T)w.gr[(long long)(6 * k + n) * g.ps + cc];
      }
    T beta = T(0);
#pragma unroll
    for (int gp = 0; gp < 3; gp++)
#pragma unroll
      for (int s = 0; s < 2; s++) {
        beta = fmax(beta, wave_bound<T>(dir, st[s][gp], gs[s][gp], gam, rPr, rRe));
        const T cs = sqrt(gam * (gam - T(1)) * st[s][gp][3]);
        amax = fmax(amax, (double)fmax(fabs(st[s][gp][1]) + cs, fabs(st[s][gp][2]) + cs));
      }
    bmax = (double)beta;
    // the moment balances use each face's fluxes only through the Gauss sums
    // S0 = sum_g w_g fhat_g and S1 = sum_g w_g t_g fhat_g (t_g: the transverse Gauss
    // offset): both cells read the same stored sums, so the telescoping is exact
    T S0[4] = {T(0), T(0), T(0), T(0)}, S1[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll
    for (int gp = 0; gp < 3; gp++) {
      T fl[4], fr[4], ul[4], ur[4];
      phys_flux<T>(dir, st[0][gp], gs[0][gp], gam, rPr, rRe, fl);
      phys_flux<T>(dir, st[1][gp], gs[1][gp], gam, rPr, rRe, fr);
#pragma unroll
      for (int s = 0; s < 2; s++) {
        T* u = s == 0 ? ul : ur;
        const T* p = st[s][gp];
        u[0] = p[0];
        u[1] = p[0] * p[1];
        u[2] = p[0] * p[2];
        u[3] = p[0] * (p[3] + T(0.5) * (p[1] * p[1] + p[2] * p[2]));
      }
      const T wg = gweight<T>(gp), wt = gweight<T>(gp) * gnode<T>(gp);
#pragma unroll
      for (int v = 0; v < 4; v++) {
        const T fh = T(0.5) * (fl[v] + fr[v] - beta * (ur[v] - ul[v]));
        S0[v] += wg * fh;
        if (gp != 1) S1[v] += wt * fh;
      }
    }
    double* out = (dir == 0 ? w.fx : w.fy) + cl;
#pragma unroll
    for (int v = 0; v < 4; v++) {
      out[(long long)v * g.ps] = (double)S0[v];
      out[(long long)(4 + v) * g.ps] = (double)S1[v];
    }
  }
  amax = warp_max(amax);
  bmax = warp_max(bmax);
  if ((threadIdx.x & 31) == 0) {
    atomic_max_pos(&diag->alpha_bits, amax);
    atomic_max_pos(&diag->beta_bits, bmax);
  }
}

// moment balances Eq. (3.2) of the interior cells
template <class T>
__global__ void __launch_bounds__(BX * BY) k_assemble(Grid g, Work w, double* __restrict__ rhs,
                                                      Diag* diag) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  unsigned int bad = 0;
  if (i < g.nx && j < g.ny) {
    const long long c = cidx(g, i, j), cl = cidx(g, i - 1, j), cb = cidx(g, i, j - 1);
    const T gam = (T)g.gamma, rPr = (T)(1.0 / g.Pr), rRe = (T)(1.0 / g.Re);
    // volume quadrature of f and g at the tensor Gauss points
    double vf[4] = {0, 0, 0, 0}, vg[4] = {0, 0, 0, 0};
#pragma unroll 1
    for (int G = 0; G < 3; G++)
#pragma unroll
      for (int H = 0; H < 3; H++) {
        const int k = 3 * G + H;
        T st[4], gs[6], f[4], h[4];
#pragma unroll
        for (int v = 0; v < 4; v++) st[v] = (T)w.vol[(long long)(4 * k + v) * g.ps + c];
#pragma unroll
        for (int n = 0; n < 6; n++) gs[n] = (T)w.gr[(long long)(6 * (12 + k) + n) * g.ps + c];
        phys_flux<T>(0, st, gs, gam, rPr, rRe, f);
        phys_flux<T>(1, st, gs, gam, rPr, rRe, h);
        const double wgt = gweight<double>(G) * gweight<double>(H);
#pragma unroll
        for (int v = 0; v < 4; v++) {
          vf[v] += wgt * (double)f[v];
          vg[v] += wgt * (double)h[v];
        }
      }
    const double rdx = 1.0 / g.dx, rdy = 1.0 / g.dy;
#pragma unroll
    for (int v = 0; v < 4; v++) {
      // face Gauss sums: S0 = sum w_g fhat_g, S1 = sum w_g t_g fhat_g (see k_flux)
      const double fR0 = w.fx[(long long)v * g.ps + c], fL0 = w.fx[(long long)v * g.ps + cl];
      const double fR1 = w.fx[(long long)(4 + v) * g.ps + c], fL1 = w.fx[(long long)(4 + v) * g.ps + cl];
      const double gT0 = w.fy[(long long)v * g.ps + c], gB0 = w.fy[(long long)v * g.ps + cb];
      const double gT1 = w.fy[(long long)(4 + v) * g.ps + c], gB1 = w.fy[(long long)(4 + v) * g.ps + cb];
      const double r0 = -(fR0 - fL0) * rdx - (gT0 - gB0) * rdy;
      const double r1 = -(fL0 + fR0) * (0.5 * rdx) - (gT1 - gB1) * rdy + vf[v] * rdx;
      const double r2 = -(fR1 - fL1) * rdx - (gB0 + gT0) * (0.5 * rdy) + vg[v] * rdy;
      rhs[(long long)v * g.ps + c] = r0;
      rhs[(long long)(4 + v) * g.ps + c] = r1;
      rhs[(long long)(8 + v) * g.ps + c] = r2;
      if (!isfinite(r0) || !isfinite(r1) || !isfinite(r2)) bad = FLAG_NONFINITE;
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&diag->flags, bad);
}

// SSP-RK3 stage with modified moments (Eq. (2.10), 2D analogue) on interior cells:
//   stage 1: out = [u^n; vhat^n] + dt F,                        base = [u^n; vhat^n]
//   stage 2: out = 3/4 base + 1/4 ([u^(1); vhat^(1)] + dt F)
//   stage 3: out = 1/3 base + 2/3 ([u^(2); vhat^(2)] + dt F)
// plus the admissibility test of the output averages (Sec. 5).
__global__ void k_rk(Grid g, int stage, const double* __restrict__ qin, const double* __restrict__ mom,
                     const double* __restrict__ rhs, double* __restrict__ base, double* __restrict__ qout,
                     Diag* diag) {
  const int i = blockIdx.x * BX + threadIdx.x;
  const int j = blockIdx.y * BY + threadIdx.y;
  unsigned int bad = 0;
  if (i < g.nx && j < g.ny) {
    const long long c = cidx(g, i, j);
    const double dt = diag->dt;
    double out[12];
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const double cur = k < 4 ? qin[(long long)k * g.ps + c] : mom[(long long)(k - 4) * g.ps + c];
      const double f = rhs[(long long)k * g.ps + c];
      if (stage == 1) {
        base[(long long)k * g.ps + c] = cur;
        out[k] = cur + dt * f;
      } else if (stage == 2) {
        out[k] = 0.75 * base[(long long)k * g.ps + c] + 0.25 * (cur + dt * f);
      } else {
        out[k] = base[(long long)k * g.ps + c] * (1.0 / 3.0) + (2.0 / 3.0) * (cur + dt * f);
      }
      qout[(long long)k * g.ps + c] = out[k];
      if (!isfinite(out[k])) bad = FLAG_INADMISSIBLE;
    }
    // p > 0 <=> rho E - |m|^2 / 2 > 0 once rho > 0
    const double rp = out[3] * out[0] - 0.5 * (out[1] * out[1] + out[2] * out[2]);
    if (!(out[0] > 0.0) || !(rp > 0.0)) bad = FLAG_INADMISSIBLE;
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if ((threadIdx.x & 31) == 0 && bad) atomicOr(&diag->flags, bad);
}

// time step of Sec. 5: dt = min(CFL h / alpha*, b Re h^2), or a forced trial
// value, capped by the remaining time
__global__ void k_dt(Diag* diag, double cfl, double h, double visc_cap, double forced, double cap) {
  const double a = __longlong_as_double((long long)diag->alpha_bits);
  double dt = forced > 0.0 ? forced : fmin(cfl * h / a, visc_cap);
  if (dt > cap) dt = cap;
  diag->dt = dt;
}

__global__ void k_scale_dt(Diag* diag, double f) { diag->dt *= f; }

// scatter a contiguous [n][ny][nx] array into padded planes, and back
__global__ void k_scatter(Grid g, int n, const double* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * N;
       t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / N, r = t % N;
    const int j = (int)(r / g.nx), i = (int)(r % g.nx);
    dst[p * g.ps + cidx(g, i, j)] = src[t];
  }
}
__global__ void k_gather(Grid g, int n, const double* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * N;
       t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / N, r = t % N;
    const int j = (int)(r / g.nx), i = (int)(r % g.nx);
    dst[t] = src[p * g.ps + cidx(g, i, j)];
  }
}
// primitive (rho, u, v, e) point sets back to conserved variables, gathered
__global__ void k_gather_cons(Grid g, int npts, const double* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < npts * N;
       t += (long long)gridDim.x * blockDim.x) {
    const long long k = t / N, r = t % N;
    const int j = (int)(r / g.nx), i = (int)(r % g.nx);
    const long long c = cidx(g, i, j);
    const double rho = src[(4 * k + 0) * g.ps + c], u = src[(4 * k + 1) * g.ps + c];
    const double v = src[(4 * k + 2) * g.ps + c], e = src[(4 * k + 3) * g.ps + c];
    dst[(4 * k + 0) * N + r] = rho;
    dst[(4 * k + 1) * N + r] = rho * u;
    dst[(4 * k + 2) * N + r] = rho * v;
    dst[(4 * k + 3) * N + r] = rho * (e + 0.5 * (u * u + v * v));
  }
}

// deterministic reductions of the state: per-row partials in a fixed order, then
// one block adds the rows in order.  part: [ny][6] = (sum rho, rho u, rho v, E,
// min rho, min p)
__global__ void k_state_rows(Grid g, const double* __restrict__ q, double* part) {
  const int j = blockIdx.x;
  if (threadIdx.x != 0 || j >= g.ny) return;
  double s[4] = {0, 0, 0, 0}, mr = INFINITY, mp = INFINITY;
  for (int i = 0; i < g.nx; i++) {
    const long long c = cidx(g, i, j);
    double u[4];
    for (int v = 0; v < 4; v++) { u[v] = q[(long long)v * g.ps + c]; s[v] += u[v]; }
    mr = fmin(mr, u[0]);
    mp = fmin(mp, (g.gamma - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]));
  }
  for (int v = 0; v < 4; v++) part[6 * j + v] = s[v];
  part[6 * j + 4] = mr;
  part[6 * j + 5] = mp;
}
__global__ void k_state_final(Grid g, const double* part, double* out) {
  if (threadIdx.x != 0) return;
  double s[4] = {0, 0, 0, 0}, mr = INFINITY, mp = INFINITY;
  for (int j = 0; j < g.ny; j++) {
    for (int v = 0; v < 4; v++) s[v] += part[6 * j + v];
    mr = fmin(mr, part[6 * j + 4]);
    mp = fmin(mp, part[6 * j + 5]);
  }
  for (int v = 0; v < 4; v++) out[v] = s[v] * g.dx * g.dy;
  out[4] = mr;
  out[5] = mp;
}

// FMA-chain throughput probe: 8 independent chains per thread, x <- x*a + b
// (a < 1 so every chain converges to b/(1-a) and stays finite).  The store is
// taken only if the impossible value -1 appears, so the work cannot be removed.
template <class T>
__global__ void k_fma_peak(T* sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 1
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int r = 0; r < 16; r++)
#pragma unroll
      for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) s += x[k];
  if (s == (T)-1) sink[0] = s;
}

}  // namespace hw

// ===========================================================================
// host side

using namespace hw;

namespace {

enum { K_GHOST = 0, K_CONS, K_FACEMOM, K_WEAK, K_GRAD, K_FLUX, K_ASSEMBLE, K_RK, K_NKIND };

struct EventPair {
  cudaEvent_t a, b;
  int kind;
};

}  // namespace

struct hweno_handle {
  hweno_config cfg;
  cudaStream_t st;
  Grid g;
  double* pool = nullptr;
  double *Q, *QS, *BASE, *RHS0, *RHS, *MOM0, *MOM, *STAGE, *PART;
  Work w;
  Diag* d_diag = nullptr;
  Diag* h_diag = nullptr;  // pinned
  double* h_red = nullptr; // pinned [6]
  double* d_red = nullptr;
  bool have_state = false, have_residual = false;
  double t = 0.0;
  // counters
  double pp_total = 0.0, cell_stages = 0.0;
  long long steps = 0, rejected = 0, launches = 0;
  double alpha = 0.0, beta = 0.0, dt_last = 0.0;
  // profiling
  bool prof = false;
  std::vector<EventPair> ev;
  long long prof_n[K_NKIND];
  double prof_ms[K_NKIND];
  char err[512];
};

static char g_init_err[512] = "no error";

static int fail(hweno_handle* h, int code, const char* msg) {
  if (h) snprintf(h->err, sizeof(h->err), "%s", msg);
  else snprintf(g_init_err, sizeof(g_init_err), "%s", msg);
  return code;
}

static int cuda_fail(hweno_handle* h, cudaError_t e, const char* where) {
  char buf[400];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return fail(h, HWENO_ERR_CUDA, buf);
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

// launch bookkeeping: optional CUDA events around each kernel of the operator
struct Prof {
  hweno_handle* h;
  int kind;
  cudaEvent_t a{}, b{};
  Prof(hweno_handle* h_, int k) : h(h_), kind(k) {
    h->launches++;
    if (h->prof) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, h->st);
    }
  }
  ~Prof() {
    if (h->prof) {
      cudaEventRecord(b, h->st);
      h->ev.push_back({a, b, kind});
    }
  }
};

static dim3 grid2(int wx, int wy, int z = 1) {
  return dim3((unsigned)((wx + BX - 1) / BX), (unsigned)((wy + BY - 1) / BY), (unsigned)z);
}

// ghost fill of a 12-plane state set
static void launch_ghost(hweno_handle* h, double* q) {
  const Grid& g = h->g;
  {
    Prof p(h, K_GHOST);
    const int n = 8 * g.ny;
    k_ghost_x<<<(n + 127) / 128, 128, 0, h->st>>>(g, q);
  }
  {
    Prof p(h, K_GHOST);
    const int n = 8 * (g.nx + 2 * NG);
    k_ghost_y<<<(n + 127) / 128, 128, 0, h->st>>>(g, q);
  }
}

// one spatial-operator evaluation of state q (12 planes): rhs (12 planes) and the
// modified moments mom (8 planes)
static int residual_eval(hweno_handle* h, double* q, double* rhs, double* mom) {
  const Grid& g = h->g;
  launch_ghost(h, q);
  if (h->cfg.precision == HWENO_MIXED) {
    {
      Prof p(h, K_GHOST);
      k_split<<<4 * 148, 256, 0, h->st>>>(g, q, mixed_planes(h->w, g.ps).hilo);
    }
    {
      Prof p(h, K_CONS);
      k_cons_mixed<<<grid2(g.nx + 6, g.ny + 6), dim3(BX, BY), 0, h->st>>>(g, q, h->w, mom, h->d_diag);
    }
    {
      Prof p(h, K_FACEMOM);
      k_face_moments_mixed<<<grid2(g.nx + 5, g.ny + 5, 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
    }
    {
      Prof p(h, K_WEAK);
      k_weak_moments_mixed<<<grid2(g.nx + 4, g.ny + 4), dim3(BX, BY), 0, h->st>>>(g, h->w);
    }
    {
      Prof p(h, K_GRAD);
      k_grad_mixed<<<grid2(g.nx + 2, g.ny + 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
    }
    {
      Prof p(h, K_FLUX);
      k_flux_mixed<<<grid2(g.nx + 1, g.ny + 1, 2), dim3(BX, BY), 0, h->st>>>(g, h->w, h->d_diag);
    }
    {
      Prof p(h, K_ASSEMBLE);
      k_assemble_mixed<<<grid2(g.nx, g.ny), dim3(BX, BY), 0, h->st>>>(g, h->w, rhs, h->d_diag);
    }
  } else {
    {
      Prof p(h, K_CONS);
      k_cons<double><<<grid2(g.nx + 6, g.ny + 6), dim3(BX, BY), 0, h->st>>>(g, q, h->w, mom, h->d_diag);
    }
    {
      Prof p(h, K_FACEMOM);
      k_face_moments<<<grid2(g.nx + 5, g.ny + 5, 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
    }
    {
      Prof p(h, K_WEAK);
      k_weak_moments<<<grid2(g.nx + 4, g.ny + 4), dim3(BX, BY), 0, h->st>>>(g, h->w);
    }
    {
      Prof p(h, K_GRAD);
      k_grad<double><<<grid2(g.nx + 2, g.ny + 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
    }
    {
      Prof p(h, K_FLUX);
      k_flux<double><<<grid2(g.nx + 1, g.ny + 1, 2), dim3(BX, BY), 0, h->st>>>(g, h->w, h->d_diag);
    }
    {
      Prof p(h, K_ASSEMBLE);
      k_assemble<double><<<grid2(g.nx, g.ny), dim3(BX, BY), 0, h->st>>>(g, h->w, rhs, h->d_diag);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "spatial operator launch");
  return HWENO_OK;
}

static int launch_rk(hweno_handle* h, int stage, const double* qin, const double* mom,
                     const double* rhs, double* qout) {
  Prof p(h, K_RK);
  k_rk<<<grid2(h->g.nx, h->g.ny), dim3(BX, BY), 0, h->st>>>(h->g, stage, qin, mom, rhs, h->BASE, qout,
                                                            h->d_diag);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "rk launch");
  return HWENO_OK;
}

static double h_min(const hweno_handle* h) {
  const double dx = h->g.dx, dy = h->g.dy;
  return dx < dy ? dx : dy;
}

static int valid_bc(int b) { return b >= HWENO_BC_PERIODIC && b <= HWENO_BC_SLIP; }

extern "C" {

int hweno_config_default(hweno_config* c) {
  if (!c) return HWENO_ERR_ARG;
  memset(c, 0, sizeof(*c));
  c->x0 = 0.0; c->x1 = 1.0; c->y0 = 0.0; c->y1 = 1.0;
  c->gamma = 1.4; c->Pr = 0.72; c->Re = 1000.0;
  for (int k = 0; k < 4; k++) c->bc[k] = HWENO_BC_PERIODIC;
  c->cfl = 0.6; c->b_visc = 1e-3; c->eps_pp = 1e-12; c->eps_weno = 1e-8;
  c->max_halvings = 20;
  c->precision = HWENO_FP64;
  return HWENO_OK;
}

const char* hweno_last_error(const hweno_handle* h) { return h ? h->err : g_init_err; }

long long hweno_launch_count(const hweno_handle* h) { return h ? h->launches : 0; }

int hweno_init(const hweno_config* cfg, void* stream, hweno_handle** out) {
  hweno_handle* h = nullptr;
  if (!out) return fail(nullptr, HWENO_ERR_ARG, "hweno_init: out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, HWENO_ERR_ARG, "hweno_init: cfg is NULL");
  const hweno_config& c = *cfg;
  if (c.nx < 4 || c.ny < 4) return fail(nullptr, HWENO_ERR_ARG, "nx and ny must be >= 4");
  if ((long long)c.nx * c.ny > (1LL << 31)) return fail(nullptr, HWENO_ERR_ARG, "grid too large");
  if (!(c.x1 > c.x0) || !(c.y1 > c.y0)) return fail(nullptr, HWENO_ERR_ARG, "empty domain");
  if (!(c.gamma > 1.0) || !(c.Pr > 0.0) || !(c.Re > 0.0)) return fail(nullptr, HWENO_ERR_ARG, "need gamma > 1, Pr > 0, Re > 0");
  for (int k = 0; k < 4; k++)
    if (!valid_bc(c.bc[k])) return fail(nullptr, HWENO_ERR_ARG, "unknown boundary condition");
  if ((c.bc[0] == HWENO_BC_PERIODIC) != (c.bc[1] == HWENO_BC_PERIODIC) ||
      (c.bc[2] == HWENO_BC_PERIODIC) != (c.bc[3] == HWENO_BC_PERIODIC))
    return fail(nullptr, HWENO_ERR_ARG, "periodic boundaries must be set on both sides");
  if (!(c.cfl > 0.0) || !(c.b_visc > 0.0) || !(c.eps_pp > 0.0) || !(c.eps_weno > 0.0) || c.max_halvings < 0)
    return fail(nullptr, HWENO_ERR_ARG, "cfl, b_visc, eps_pp, eps_weno must be > 0");
  if (c.precision != HWENO_FP64 && c.precision != HWENO_MIXED)
    return fail(nullptr, HWENO_ERR_ARG, "precision must be HWENO_FP64 or HWENO_MIXED");
  if (c.scheme != 0 || c.reserved != 0) return fail(nullptr, HWENO_ERR_ARG, "scheme must be 0 (HWENO-GR)");

  h = new (std::nothrow) hweno_handle();
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "host allocation failed");
  h->cfg = c;
  h->st = (cudaStream_t)stream;
  snprintf(h->err, sizeof(h->err), "no error");
  for (int k = 0; k < K_NKIND; k++) { h->prof_n[k] = 0; h->prof_ms[k] = 0.0; }
  Grid& g = h->g;
  g.nx = c.nx;
  g.ny = c.ny;
  g.pitch = ((c.nx + 2 * NG + 15) / 16) * 16;
  g.ps = (long long)(c.ny + 2 * NG) * g.pitch;
  g.dx = (c.x1 - c.x0) / c.nx;
  g.dy = (c.y1 - c.y0) / c.ny;
  g.gamma = c.gamma; g.Pr = c.Pr; g.Re = c.Re;
  g.eps_pp = c.eps_pp; g.eps_weno = c.eps_weno;
  for (int k = 0; k < 4; k++) g.bc[k] = c.bc[k];

  const long long N = (long long)c.nx * c.ny;
  // planes: Q 12, QS 12, BASE 12, RHS0 12, RHS 12, MOM0 8, MOM 8, face 48, vol 36,
  // wbar 3, wx 6, wy 6, rm 18, gr 126, fx 12, fy 12, theta 2
  const long long nplanes = 12 * 5 + 16 + 48 + 36 + 3 + 12 + 18 + 126 + 24 + 2;
  const long long total = nplanes * g.ps + 4 * N + 6LL * c.ny + 16;
  cudaError_t e = cudaMalloc(&h->pool, (size_t)total * sizeof(double));
  if (e != cudaSuccess) {
    snprintf(g_init_err, sizeof(g_init_err), "device allocation of %.2f GB failed: %s",
             total * 8.0 / 1e9, cudaGetErrorString(e));
    delete h;
    return HWENO_ERR_CUDA;
  }
  double* p = h->pool;
  auto take = [&](long long n) { double* r = p; p += n * g.ps; return r; };
  h->Q = take(12); h->QS = take(12); h->BASE = take(12); h->RHS0 = take(12); h->RHS = take(12);
  h->MOM0 = take(8); h->MOM = take(8);
  h->w.face = take(48); h->w.vol = take(36); h->w.wbar = take(3); h->w.wx = take(6); h->w.wy = take(6);
  h->w.rm = take(18); h->w.gr = take(126); h->w.fx = take(12); h->w.fy = take(12); h->w.theta = take(2);
  h->STAGE = p; p += 4 * N;
  h->PART = p; p += 6LL * c.ny;
  h->d_red = p;
  e = cudaMemsetAsync(h->pool, 0, (size_t)total * sizeof(double), h->st);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_diag, sizeof(Diag));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_diag, 0, sizeof(Diag), h->st);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_diag, sizeof(Diag));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_red, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    snprintf(g_init_err, sizeof(g_init_err), "init: %s", cudaGetErrorString(e));
    hweno_destroy(h);
    return HWENO_ERR_CUDA;
  }
  *out = h;
  return HWENO_OK;
}

void hweno_destroy(hweno_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  for (auto& ep : h->ev) { cudaEventDestroy(ep.a); cudaEventDestroy(ep.b); }
  if (h->pool) cudaFree(h->pool);
  if (h->d_diag) cudaFree(h->d_diag);
  if (h->h_diag) cudaFreeHost(h->h_diag);
  if (h->h_red) cudaFreeHost(h->h_red);
  delete h;
}

}  // extern "C"

static long long origin(const Grid& g) { return (long long)NG * g.pitch + NG; }

// contiguous [n][ny][nx] (host or device) <-> n padded planes
static int copy_planes_in(hweno_handle* h, const double* src, int n, double* dst, int on_device) {
  const Grid& g = h->g;
  const size_t row = (size_t)g.nx * sizeof(double);
  for (int k = 0; k < n; k++) {
    const double* s = src + (long long)k * g.nx * g.ny;
    double* d = dst + (long long)k * g.ps + origin(g);
    CK(cudaMemcpy2DAsync(d, (size_t)g.pitch * sizeof(double), s, row, row, (size_t)g.ny,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st),
       "copy into the solver");
  }
  return HWENO_OK;
}

static int copy_planes_out(hweno_handle* h, const double* src, int n, double* dst, int on_device) {
  const Grid& g = h->g;
  const size_t row = (size_t)g.nx * sizeof(double);
  for (int k = 0; k < n; k++) {
    const double* s = src + (long long)k * g.ps + origin(g);
    double* d = dst + (long long)k * g.nx * g.ny;
    CK(cudaMemcpy2DAsync(d, row, s, (size_t)g.pitch * sizeof(double), row, (size_t)g.ny,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st),
       "copy out of the solver");
  }
  return HWENO_OK;
}

static int reset_diag(hweno_handle* h) {
  CK(cudaMemsetAsync(h->d_diag, 0, sizeof(Diag), h->st), "diag reset");
  return HWENO_OK;
}

static int read_diag(hweno_handle* h) {
  CK(cudaMemcpyAsync(h->h_diag, h->d_diag, sizeof(Diag), cudaMemcpyDeviceToHost, h->st), "diag read");
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  return HWENO_OK;
}

static double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
}

extern "C" {

int hweno_set_state(hweno_handle* h, const double* q, int on_device) {
  if (!h || !q) return fail(h, HWENO_ERR_ARG, "hweno_set_state: NULL argument");
  int rc = copy_planes_in(h, q, 12, h->Q, on_device);
  if (rc) return rc;
  h->have_state = true;
  h->have_residual = false;
  h->pp_total = 0.0;
  h->cell_stages = 0.0;
  h->steps = 0;
  h->rejected = 0;
  h->launches = 0;
  h->t = 0.0;
  if (!on_device) CK(cudaStreamSynchronize(h->st), "stream synchronize");
  return HWENO_OK;
}

int hweno_set_time(hweno_handle* h, double t) {
  if (!h) return HWENO_ERR_ARG;
  h->t = t;
  return HWENO_OK;
}

int hweno_get_state(hweno_handle* h, double* q, int on_device) {
  if (!h || !q) return fail(h, HWENO_ERR_ARG, "hweno_get_state: NULL argument");
  if (!h->have_state) return fail(h, HWENO_ERR_STATE, "hweno_get_state before hweno_set_state");
  int rc = copy_planes_out(h, h->Q, 12, q, on_device);
  if (rc) return rc;
  if (!on_device) CK(cudaStreamSynchronize(h->st), "stream synchronize");
  return HWENO_OK;
}

int hweno_residual(hweno_handle* h, double* rhs, double* vhat, int on_device) {
  if (!h) return HWENO_ERR_ARG;
  if (!h->have_state) return fail(h, HWENO_ERR_STATE, "hweno_residual before hweno_set_state");
  int rc = reset_diag(h);
  if (!rc) rc = residual_eval(h, h->Q, h->RHS, h->MOM);
  if (rc) return rc;
  h->have_residual = true;
  if (rhs && (rc = copy_planes_out(h, h->RHS, 12, rhs, on_device))) return rc;
  if (vhat && (rc = copy_planes_out(h, h->MOM, 8, vhat, on_device))) return rc;
  if ((rc = read_diag(h))) return rc;
  h->alpha = bits_to_double(h->h_diag->alpha_bits);
  h->beta = bits_to_double(h->h_diag->beta_bits);
  if (h->h_diag->flags & FLAG_NONFINITE) return fail(h, HWENO_ERR_NONFINITE, "non-finite residual");
  return HWENO_OK;
}

// one SSP-RK3 step from h->Q; on success the new state is in h->Q
static int do_step(hweno_handle* h, double dt_forced, double t_cap, double* dt_used, int* rejections) {
  const Grid& g = h->g;
  int rc = reset_diag(h);
  if (!rc) rc = residual_eval(h, h->Q, h->RHS0, h->MOM0);
  if (rc) return rc;
  {
    Prof p(h, K_RK);
    k_dt<<<1, 1, 0, h->st>>>(h->d_diag, h->cfg.cfl, h_min(h), h->cfg.b_visc * h->cfg.Re * h_min(h) * h_min(h),
                             dt_forced, t_cap);
  }
  if ((rc = read_diag(h))) return rc;
  const Diag first = *h->h_diag;
  if (first.flags & FLAG_NONFINITE) return fail(h, HWENO_ERR_NONFINITE, "non-finite residual at t^n");
  double dt = first.dt;
  if (!(dt > 0.0) || !isfinite(dt)) return fail(h, HWENO_ERR_NONFINITE, "time step is not positive and finite");
  int rej = 0;
  for (;;) {
    // stage flags and counters of this attempt; keep dt and the stage-1 maxima
    CK(cudaMemsetAsync(&h->d_diag->pp_count, 0, sizeof(unsigned long long), h->st), "diag");
    CK(cudaMemsetAsync(&h->d_diag->flags, 0, sizeof(unsigned int), h->st), "diag");
    if ((rc = launch_rk(h, 1, h->Q, h->MOM0, h->RHS0, h->QS))) return rc;
    if ((rc = residual_eval(h, h->QS, h->RHS, h->MOM))) return rc;
    if ((rc = launch_rk(h, 2, h->QS, h->MOM, h->RHS, h->QS))) return rc;
    if ((rc = residual_eval(h, h->QS, h->RHS, h->MOM))) return rc;
    if ((rc = launch_rk(h, 3, h->QS, h->MOM, h->RHS, h->QS))) return rc;
    if ((rc = read_diag(h))) return rc;
    const Diag& d = *h->h_diag;
    if (!(d.flags & (FLAG_INADMISSIBLE | FLAG_NONFINITE))) {
      double* tmp = h->Q;
      h->Q = h->QS;
      h->QS = tmp;
      h->alpha = bits_to_double(first.alpha_bits);
      const double b2 = bits_to_double(d.beta_bits), b1 = bits_to_double(first.beta_bits);
      h->beta = b1 > b2 ? b1 : b2;
      h->pp_total += (double)first.pp_count + (double)d.pp_count;
      h->cell_stages += 3.0 * g.nx * (double)g.ny;
      h->dt_last = dt;
      h->steps++;
      h->rejected += rej;
      if (dt_used) *dt_used = dt;
      if (rejections) *rejections = rej;
      return HWENO_OK;
    }
    if (rej >= h->cfg.max_halvings) {
      h->rejected += rej;
      if (rejections) *rejections = rej;
      return fail(h, HWENO_ERR_INADMISSIBLE, "stage inadmissible after max_halvings restarts");
    }
    rej++;
    dt *= 0.5;
    k_scale_dt<<<1, 1, 0, h->st>>>(h->d_diag, 0.5);
    h->launches++;
  }
}

int hweno_step(hweno_handle* h, double dt, double* dt_used, int* rejections) {
  if (!h) return HWENO_ERR_ARG;
  if (!h->have_state) return fail(h, HWENO_ERR_STATE, "hweno_step before hweno_set_state");
  double used = 0.0;
  int rc = do_step(h, dt > 0.0 ? dt : 0.0, INFINITY, &used, rejections);
  if (rc) return rc;
  h->t += used;
  h->have_residual = false;
  if (dt_used) *dt_used = used;
  return HWENO_OK;
}

int hweno_advance(hweno_handle* h, double t_end, int max_steps, double* t_reached, int* steps) {
  if (!h) return HWENO_ERR_ARG;
  if (!h->have_state) return fail(h, HWENO_ERR_STATE, "hweno_advance before hweno_set_state");
  int n = 0, rc = HWENO_OK;
  while (h->t < t_end && n < max_steps) {
    double used = 0.0;
    rc = do_step(h, 0.0, t_end - h->t, &used, nullptr);
    if (rc) break;
    h->t += used;
    n++;
    const double scale = fabs(t_end) > 1.0 ? fabs(t_end) : 1.0;
    if (t_end - h->t <= 1e-14 * scale) h->t = t_end;
  }
  h->have_residual = false;
  if (t_reached) *t_reached = h->t;
  if (steps) *steps = n;
  return rc;
}

int hweno_get_diag(hweno_handle* h, hweno_diag* d) {
  if (!h || !d) return HWENO_ERR_ARG;
  memset(d, 0, sizeof(*d));
  d->t = h->t;
  d->dt_last = h->dt_last;
  d->alpha_star = h->alpha;
  d->beta_max = h->beta;
  d->pp_active = h->pp_total;
  d->cell_stages = h->cell_stages;
  d->steps = h->steps;
  d->rejected = h->rejected;
  if (h->have_state) {
    k_state_rows<<<h->g.ny, 32, 0, h->st>>>(h->g, h->Q, h->PART);
    k_state_final<<<1, 32, 0, h->st>>>(h->g, h->PART, h->d_red);
    h->launches += 2;
    CK(cudaMemcpyAsync(h->h_red, h->d_red, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->st), "diag");
    CK(cudaStreamSynchronize(h->st), "stream synchronize");
    for (int v = 0; v < 4; v++) d->totals[v] = h->h_red[v];
    d->min_rho = h->h_red[4];
    d->min_p = h->h_red[5];
  }
  return HWENO_OK;
}

int hweno_debug_fields(hweno_handle* h, int which, double* out, int on_device) {
  if (!h || !out) return fail(h, HWENO_ERR_ARG, "hweno_debug_fields: NULL argument");
  if (which < 0 || which > 4) return fail(h, HWENO_ERR_ARG, "hweno_debug_fields: unknown field set");
  if (!h->have_residual) return fail(h, HWENO_ERR_STATE, "hweno_debug_fields before hweno_residual");
  const Grid& g = h->g;
  const long long N = (long long)g.nx * g.ny;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (h->cfg.precision == HWENO_MIXED && which <= 3) {
    // FP32 intermediates of the mixed path, widened to FP64
    const WorkF f = mixed_planes(h->w, g.ps);
    if (which <= 1) {
      const int npts = which == 0 ? 12 : 9;
      const float* src = which == 0 ? f.face : f.vol;
      for (int k = 0; k < npts; k++) {
        k_gather_cons_f<<<256, 256, 0, h->st>>>(g, src + (long long)4 * k * g.ps, h->STAGE);
        h->launches++;
        CK(cudaMemcpyAsync(out + 4 * k * N, h->STAGE, 4 * N * sizeof(double), kind, h->st), "debug copy");
      }
    } else {
      const int n = which == 2 ? 18 : 126;
      const float* src = which == 2 ? f.rm : f.gr;
      for (int k = 0; k < n; k += 4) {
        const int m = n - k < 4 ? n - k : 4;
        k_gather_f<<<256, 256, 0, h->st>>>(g, m, src + (long long)k * g.ps, h->STAGE);
        h->launches++;
        CK(cudaMemcpyAsync(out + (long long)k * N, h->STAGE, m * N * sizeof(double), kind, h->st), "debug copy");
      }
    }
  } else if (which <= 1) {
    const int npts = which == 0 ? 12 : 9;
    const double* src = which == 0 ? h->w.face : h->w.vol;
    for (int k = 0; k < npts; k++) {
      k_gather_cons<<<256, 256, 0, h->st>>>(g, 1, src + (long long)4 * k * g.ps, h->STAGE);
      h->launches++;
      CK(cudaMemcpyAsync(out + 4 * k * N, h->STAGE, 4 * N * sizeof(double), kind, h->st), "debug copy");
    }
  } else {
    const int n = which == 2 ? 18 : (which == 3 ? 126 : 2);
    const double* src = which == 2 ? h->w.rm : (which == 3 ? h->w.gr : h->w.theta);
    int rc = copy_planes_out(h, src, n, out, on_device);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  return HWENO_OK;
}

int hweno_profile(hweno_handle* h, int enable) {
  if (!h) return HWENO_ERR_ARG;
  h->prof = enable != 0;
  return HWENO_OK;
}

int hweno_profile_read(hweno_handle* h, int kernel, long long* launches, double* total_ms) {
  if (!h || kernel < 0 || kernel >= K_NKIND) return fail(h, HWENO_ERR_ARG, "hweno_profile_read: bad kernel");
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  for (auto& ep : h->ev) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ep.a, ep.b);
    h->prof_n[ep.kind]++;
    h->prof_ms[ep.kind] += ms;
    cudaEventDestroy(ep.a);
    cudaEventDestroy(ep.b);
  }
  h->ev.clear();
  if (launches) *launches = h->prof_n[kernel];
  if (total_ms) *total_ms = h->prof_ms[kernel];
  return HWENO_OK;
}

int hweno_measure_peak(hweno_handle* h, int which, double* tflops) {
  if (!h || !tflops || (which != 0 && which != 1)) return fail(h, HWENO_ERR_ARG, "hweno_measure_peak: bad argument");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev), "device");
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  const int threads = 256, blocks = sms * 8;
  const int iters = which == 0 ? 2048 : 65536;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a), "event");
  CK(cudaEventCreate(&b), "event");
  double best = 0.0;
  for (int rep = 0; rep < 3; rep++) {
    CK(cudaEventRecord(a, h->st), "event");
    if (which == 0) k_fma_peak<double><<<blocks, threads, 0, h->st>>>(h->STAGE, iters, 0.999999, 1e-6);
    else k_fma_peak<float><<<blocks, threads, 0, h->st>>>((float*)h->STAGE, iters, 0.999999f, 1e-6f);
    h->launches++;
    CK(cudaEventRecord(b, h->st), "event");
    CK(cudaEventSynchronize(b), "event");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b), "event");
    const double flops = 2.0 * 8.0 * 16.0 * (double)iters * threads * (double)blocks;
    const double tf = flops / (ms * 1e-3) / 1e12;
    if (tf > best) best = tf;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *tflops = best;
  return HWENO_OK;
}

}  // extern "C"

// ===========================================================================
// Residual evaluation that allocates nothing: inputs and outputs are the caller's
// device buffers, and every intermediate plane lives in one library-static device
// array.  For callers that may not allocate device memory once they are running:
// programs whose device memory is owned by another allocator under a fixed budget
// (a framework's caching pool, a reserved arena), where a cudaMalloc can fail or
// fragment that budget, and latency-bound loops, where cudaMalloc's implicit
// device-wide synchronisation is not acceptable.

#include <mutex>

namespace {
// 12 state + 12 residual + 8 modified-moment planes, then the Work planes
constexpr long long NOALLOC_PLANES = 12 + 12 + 8 + 48 + 36 + 3 + 6 + 6 + 18 + 126 + 12 + 12 + 2;
// padded cells per plane: (ny + 8) * round_up(nx + 8, 16) may not exceed this
// (for example grids up to 56 x 56, or 120 x 24)
constexpr long long NOALLOC_MAX_PLANE = 4096;
constexpr long long NOALLOC_DOUBLES = NOALLOC_PLANES * NOALLOC_MAX_PLANE + 16;  // + Diag
constexpr int NOALLOC_MAX_DEVICES = 64;
double* g_noalloc_addr[NOALLOC_MAX_DEVICES];  // device address of the array, per device
std::mutex g_noalloc_mu;
}  // namespace

// about 9.9 MB on every device that loads the library, held until the process exits
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// host code cannot use g_noalloc_scratch as a device pointer: look its address up
// once per device, with that device current
static int noalloc_scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "hweno_residual_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return fail(nullptr, HWENO_ERR_ARG, "hweno_residual_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(nullptr, e, "hweno_residual_noalloc: cudaGetSymbolAddress");
    g_noalloc_addr[dev] = (double*)p;
  }
  *out = g_noalloc_addr[dev];
  return HWENO_OK;
}

static int noalloc_check_config(const hweno_config& c) {
  if (c.nx < 4 || c.ny < 4) return fail(nullptr, HWENO_ERR_ARG, "nx and ny must be >= 4");
  if (!(c.x1 > c.x0) || !(c.y1 > c.y0)) return fail(nullptr, HWENO_ERR_ARG, "empty domain");
  if (!(c.gamma > 1.0) || !(c.Pr > 0.0) || !(c.Re > 0.0))
    return fail(nullptr, HWENO_ERR_ARG, "need gamma > 1, Pr > 0, Re > 0");
  for (int k = 0; k < 4; k++)
    if (!valid_bc(c.bc[k])) return fail(nullptr, HWENO_ERR_ARG, "unknown boundary condition");
  if ((c.bc[0] == HWENO_BC_PERIODIC) != (c.bc[1] == HWENO_BC_PERIODIC) ||
      (c.bc[2] == HWENO_BC_PERIODIC) != (c.bc[3] == HWENO_BC_PERIODIC))
    return fail(nullptr, HWENO_ERR_ARG, "periodic boundaries must be set on both sides");
  if (!(c.eps_pp > 0.0) || !(c.eps_weno > 0.0)) return fail(nullptr, HWENO_ERR_ARG, "eps_pp, eps_weno must be > 0");
  if (c.precision != HWENO_FP64 && c.precision != HWENO_MIXED)
    return fail(nullptr, HWENO_ERR_ARG, "precision must be HWENO_FP64 or HWENO_MIXED");
  if (c.scheme != 0 || c.reserved != 0) return fail(nullptr, HWENO_ERR_ARG, "scheme must be 0 (HWENO-GR)");
  return HWENO_OK;
}

extern "C" int hweno_residual_noalloc(const hweno_config* cfg, const double* q, double* rhs, double* vhat,
                                      void* stream) {
  if (!cfg || !q || !rhs) return fail(nullptr, HWENO_ERR_ARG, "hweno_residual_noalloc: NULL argument");
  int rc = noalloc_check_config(*cfg);
  if (rc) return rc;
  const hweno_config& c = *cfg;
  Grid g;
  g.nx = c.nx;
  g.ny = c.ny;
  g.pitch = ((c.nx + 2 * NG + 15) / 16) * 16;
  g.ps = (long long)(c.ny + 2 * NG) * g.pitch;
  if (g.ps > NOALLOC_MAX_PLANE) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "hweno_residual_noalloc: grid %d x %d needs %lld padded cells per plane, the static "
             "scratch holds %lld ((ny + 8) * round_up(nx + 8, 16) must be <= %lld)",
             c.nx, c.ny, g.ps, NOALLOC_MAX_PLANE, NOALLOC_MAX_PLANE);
    return fail(nullptr, HWENO_ERR_ARG, buf);
  }
  g.dx = (c.x1 - c.x0) / c.nx;
  g.dy = (c.y1 - c.y0) / c.ny;
  g.gamma = c.gamma; g.Pr = c.Pr; g.Re = c.Re;
  g.eps_pp = c.eps_pp; g.eps_weno = c.eps_weno;
  for (int k = 0; k < 4; k++) g.bc[k] = c.bc[k];

  double* base = nullptr;
  if ((rc = noalloc_scratch_address(&base))) return rc;
  // the same spatial operator as hweno_residual, on a stack handle whose planes all
  // point into the static array (no profiling, so the handle allocates nothing)
  hweno_handle tmp;
  tmp.cfg = c;
  tmp.st = (cudaStream_t)stream;
  tmp.g = g;
  double* p = base;
  auto take = [&](long long n) { double* r = p; p += n * g.ps; return r; };
  double* Q = take(12);
  double* R = take(12);
  double* M = take(8);
  tmp.w.face = take(48); tmp.w.vol = take(36); tmp.w.wbar = take(3); tmp.w.wx = take(6); tmp.w.wy = take(6);
  tmp.w.rm = take(18); tmp.w.gr = take(126); tmp.w.fx = take(12); tmp.w.fy = take(12); tmp.w.theta = take(2);
  tmp.d_diag = reinterpret_cast<Diag*>(p);
  tmp.prof = false;
  // the reductions accumulate into the Diag words: they start from zero on every call;
  // every other plane is written before it is read within the call
  cudaError_t e = cudaMemsetAsync(tmp.d_diag, 0, sizeof(Diag), tmp.st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "hweno_residual_noalloc: clearing the reductions");
  k_scatter<<<256, 256, 0, tmp.st>>>(g, 12, q, Q);
  rc = residual_eval(&tmp, Q, R, M);
  if (rc) return fail(nullptr, rc, tmp.err);
  k_gather<<<256, 256, 0, tmp.st>>>(g, 12, R, rhs);
  if (vhat) k_gather<<<256, 256, 0, tmp.st>>>(g, 8, M, vhat);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "hweno_residual_noalloc: launch");
  return HWENO_OK;
}
