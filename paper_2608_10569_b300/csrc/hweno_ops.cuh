// Per-cell bodies of the spatial-operator kernels and the SSP-RK3 stage, as device
// functions of the position (gx, gy[, gz]) in the launch region of each kernel.  The
// single-grid kernels (hweno.cu) call them with gx = blockIdx.x*blockDim.x +
// threadIdx.x; the batched kernels map persistent blocks over a (case, tile) list.
// Each kernel's launch region and its offset to cell indices (i, j):
//   cons          (nx+6) x (ny+6)        i = gx - 3, j = gy - 3
//   face moments  (nx+5) x (ny+5) x 2    z = 0: i = gx - 3, j = gy - 2; z = 1: i = gx - 2, j = gy - 3
//   weak moments  (nx+4) x (ny+4)        i = gx - 2, j = gy - 2
//   grad, dr      (nx+2) x (ny+2)        i = gx - 1, j = gy - 1
//   flux          (nx+1) x (ny+1) x 2    z = 0: i = gx - 1, j = gy; z = 1: i = gx, j = gy - 1
//   assemble, rk  nx x ny                i = gx, j = gy
#pragma once
#include "hweno_kernels.cuh"

namespace hw {

// lane of the calling thread in its warp, for any block shape
__device__ __forceinline__ int lane_id() { return (threadIdx.x + threadIdx.y * blockDim.x) & 31; }


// ---------------------------------------------------------------------------
// conservative characteristic reconstruction, modified moments and PP limiter of
// every cell of the interior grown by 3 (Sec. 3.1, Eq. (3.4), Appendix A.2)
// FP64: per-thread scratch of cons_body in dynamic shared memory, [96][128] doubles:
// the p0 coefficients (60) and the x-system's volume values (36), so that they do not
// occupy registers while the other reconstruction steps run (launch with
// CONS_SMEM_BYTES of dynamic shared memory, blocks of 128 threads)
constexpr int CONS_SMEM_BYTES = 96 * 128 * 8;

// REC (FP64 only): also write the reconstruction data a reverse sweep reads (Work::yrec)
// DR (FP64 only): also write the combination coefficients HWENO-DR differentiates
// (Work::dr) for the cells of the interior grown by 1
template <class T, bool REC = false, bool DR = false>
__device__ __forceinline__ void cons_body(const Grid& g, const double* __restrict__ q, const Work& w,
                                          double* __restrict__ mom, Diag* diag, int gx, int gy) {
  const int i = gx - 3;
  const int j = gy - 3;
  unsigned long long pp = 0;
  unsigned int flags = 0;
  if (i < g.nx + 3 && j < g.ny + 3) {
    constexpr bool OFF = sizeof(T) == 4;  // FP32: reconstruct offsets from the average
    const long long c = cidx(g, i, j);
    extern __shared__ double cons_smem[];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    double* ccs = cons_smem + tid;             // [60][128]: p0 coefficients
    double* park = cons_smem + 60 * 128 + tid;  // [36][128]: x-system volume values
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
      if constexpr (REC) {
#pragma unroll
        for (int k = 0; k < 15; k++) w.yrec[(long long)(YREC_CC + 15 * v + k) * g.ps + c] = cc[v][k];
      }
      if constexpr (!OFF) {
#pragma unroll
        for (int k = 0; k < 15; k++) ccs[(15 * v + k) * 128] = cc[v][k];
      }
      sl[v][0] = (T)(d[4] - d[3]);
      sl[v][1] = (T)(d[5] - d[4]);
      sl[v][2] = (T)(d[4] - d[1]);
      sl[v][3] = (T)(d[7] - d[4]);
      ctr[v] = OFF ? T(0) : (T)ub[v];
    }
    // a compiler barrier: the reconstructions below load the coefficients from the
    // shared slot instead of keeping the stored registers alive
    if constexpr (!OFF) asm volatile("" ::: "memory");
    const T ut[4] = {(T)ub[0], (T)ub[1], (T)ub[2], (T)ub[3]};
    const T eps = (T)g.eps_weno;
    double face[12][4], vol[9][4], volx[9][4], mx[4], my[4];
    CharState<T> cs;
    char_state<T>(ut, (T)g.gamma, cs);
    const bool interior = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
    // FP64: the coefficients are read from the shared slot, and the x-system's volume
    // values wait there while the y-system is reconstructed (fewer live registers)
    const CoefRegs<T> ccr{cc};
    const CoefShared<double> ccsh{ccs};
    double* dw = nullptr;
    if constexpr (DR) {
      if (i >= -1 && i <= g.nx && j >= -1 && j <= g.ny) dw = w.dr + c;
    }
    if constexpr (OFF) recon_dir<T, 0, double, REC>(ccr, sl, ctr, cs, eps, face, volx, mx, nullptr, g.ps);
    else
      recon_dir<T, 0, double, REC>(ccsh, sl, ctr, cs, eps, face, volx, mx, REC ? w.yrec + c : nullptr, g.ps,
                                   DR ? dw : nullptr);
    if (interior) {
#pragma unroll
      for (int v = 0; v < 4; v++) mom[(long long)v * g.ps + c] = mx[v];
    }
    if constexpr (!OFF) {
#pragma unroll
      for (int k = 0; k < 9; k++)
#pragma unroll
        for (int v = 0; v < 4; v++) park[(4 * k + v) * 128] = volx[k][v];
      asm volatile("" ::: "memory");
    }
    if constexpr (OFF) recon_dir<T, 1, double, REC>(ccr, sl, ctr, cs, eps, face + 6, vol, my, nullptr, g.ps);
    else
      recon_dir<T, 1, double, REC>(ccsh, sl, ctr, cs, eps, face + 6, vol, my,
                                   REC ? w.yrec + 72 * g.ps + c : nullptr, g.ps,
                                   DR && dw ? dw + 60 * g.ps : nullptr);
#pragma unroll
    for (int v = 0; v < 4; v++) {
#pragma unroll
      for (int k = 0; k < 12; k++)
        if (OFF) face[k][v] += ub[v];
#pragma unroll
      for (int k = 0; k < 9; k++) {
        const double vx = OFF ? volx[k][v] : park[(4 * k + v) * 128];
        vol[k][v] = 0.5 * (vx + vol[k][v]);
        if (OFF) vol[k][v] += ub[v];
      }
    }
    double th[2] = {1.0, 1.0};
    const double pb = pressure(ub, g.gamma);
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
      for (int v = 0; v < 4; v++) mom[(long long)(4 + v) * g.ps + c] = my[v];
    }
  }
  // block reduction of the activation count and flags: one atomic per warp
  pp = warp_sum_u64(pp);
  flags = __reduce_or_sync(0xffffffffu, flags);
  if (lane_id() == 0) {
    if (pp) atomicAdd(&diag->pp_count, pp);
    if (flags) atomicOr(&diag->flags, flags);
  }
}

// face moments W^{x,0}, W^{x,1} (blockIdx.z = 0) of the x-faces right of cells
// i in [-3, nx+2), j in [-2, ny+2), and W^{y,0}, W^{y,1} (z = 1) of the y-faces
// above cells i in [-2, nx+2), j in [-3, ny+2)  (Eq. (3.6) with the interface
// average of the two traces)
__device__ __forceinline__ void face_moments_body(const Grid& g, const Work& w, int gx, int gy, int gz) {
  const int dir = gz;
  const int i = gx - (dir == 0 ? 3 : 2);
  const int j = gy - (dir == 0 ? 2 : 3);
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
__device__ __forceinline__ void weak_moments_body(const Grid& g, const Work& w, int gx, int gy) {
  const int i = gx - 2;
  const int j = gy - 2;
  if (i >= g.nx + 2 || j >= g.ny + 2) return;
  const long long c = cidx(g, i, j), cl = cidx(g, i - 1, j), cb = cidx(g, i, j - 1);
  const double rdx = g.rdx, rdy = g.rdy;
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
// REC (FP64 only): also write each component's p0 coefficients and weight factors
// (Work::yrec)
// LIN: the linear weights (omega_m = gamma_m), which make the combination p0 itself:
// the ablation of Remark 3.1
template <class T, bool REC = false, bool LIN = false>
__device__ __forceinline__ void grad_body(const Grid& g, const Work& w, int gx, int gy) {
  const int i = gx - 1;
  const int j = gy - 1;
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
    if constexpr (LIN) {
      hw_p0_coeffs<T>(d, C);
    } else if constexpr (REC) {
      T c0[15], wr[2];
      hw_p0_coeffs<T>(d, c0);
      const T s[4] = {d[4] - d[3], d[5] - d[4], d[4] - d[1], d[7] - d[4]};
      hweno_combine_coeffs<T, true>(c0, s, d[4], eps, C, wr);
      double* y = w.yrec + (long long)(YREC_GR + 17 * comp) * g.ps + c;
#pragma unroll
      for (int k = 0; k < 15; k++) y[(long long)k * g.ps] = c0[k];
      y[(long long)15 * g.ps] = wr[0];
      y[(long long)16 * g.ps] = wr[1];
    } else {
      hweno_combine<T>(d, eps, C);
    }
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

// ---------------------------------------------------------------------------
// HWENO-DR viscous gradients (Eq. (3.5)) of cells of the interior grown by 1.  The
// nonlinear weights are constant over the cell, so the combination of the candidates'
// derivatives is the derivative of the combined polynomial that cons_body stored per
// characteristic field and direction (Work::dr).  The back-transform to conserved
// variables is linear, so it is applied to the coefficients: P_d = R_d C_d, one
// conservative quartic per variable and direction.  Each direction's polynomials give
// the xi/eta derivatives at its own face points; the volume points use the mean of the
// two directions' polynomials, as the volume values do.  The chain rule of u = m/rho,
// v = n/rho, e = E/rho - (u^2+v^2)/2 takes the state the fluxes use at the point (the
// limited face traces, the volume values; primitive in Work::face and Work::vol) and
// gives the gradients at the 21 points in the layout k_grad writes (Work::gr).
// Per-thread scratch in dynamic shared memory, [120][DR_THREADS] doubles: this
// direction's polynomials and the running mean (blocks of DR_THREADS threads).
constexpr int DR_THREADS = 64;
constexpr int DR_SMEM_BYTES = 120 * DR_THREADS * 8;

// (u_x, u_y, v_x, v_y, e_x, e_y) from the primitive state w = (rho, u, v, e) and the
// conserved variables' derivatives Ux, Uy
__device__ __forceinline__ void dissip_grad(const double* w, const double* Ux, const double* Uy, double* gr) {
  const double rr = 1.0 / w[0];
  const double u = w[1], v = w[2], en = w[3] + 0.5 * (u * u + v * v);
  const double ux = (Ux[1] - u * Ux[0]) * rr, vx = (Ux[2] - v * Ux[0]) * rr;
  const double uy = (Uy[1] - u * Uy[0]) * rr, vy = (Uy[2] - v * Uy[0]) * rr;
  gr[0] = ux;
  gr[1] = uy;
  gr[2] = vx;
  gr[3] = vy;
  gr[4] = (Ux[3] - en * Ux[0]) * rr - (u * ux + v * vx);
  gr[5] = (Uy[3] - en * Uy[0]) * rr - (u * uy + v * vy);
}

// the gradients at NP points k0 .. k0+NP-1 from the conserved variables' derivatives
// dx, dy there and the primitive state of the point sets at prim (point k0 - kp first)
template <int NP>
__device__ __forceinline__ void dr_store(const Grid& g, const Work& w, long long c, const double (*dx)[NP],
                                         const double (*dy)[NP], int k0, const double* prim, int kp) {
#pragma unroll
  for (int p = 0; p < NP; p++) {
    const int kk = k0 - kp + p;
    const double st[4] = {prim[(long long)(4 * kk) * g.ps + c], prim[(long long)(4 * kk + 1) * g.ps + c],
                          prim[(long long)(4 * kk + 2) * g.ps + c], prim[(long long)(4 * kk + 3) * g.ps + c]};
    const double Ux[4] = {dx[0][p], dx[1][p], dx[2][p], dx[3][p]};
    const double Uy[4] = {dy[0][p], dy[1][p], dy[2][p], dy[3][p]};
    double gr[6];
    dissip_grad(st, Ux, Uy, gr);
#pragma unroll
    for (int n = 0; n < 6; n++) w.gr[(long long)(6 * (k0 + p) + n) * g.ps + c] = gr[n];
  }
}

// direction DIR: its conservative polynomials into P, half of them into the mean Pv,
// then the gradients at its six face points (both faces from one collapse per
// derivative polynomial)
template <int DIR>
__device__ __forceinline__ void dr_direction(const Grid& g, const Work& w, long long c, const CharState<double>& cs,
                                             const double* fx, const double* fy, double* P, double* Pv) {
  const double* C = w.dr + (long long)(60 * DIR) * g.ps + c;
#pragma unroll
  for (int k = 0; k < 15; k++) {
    const double y[4] = {C[(long long)k * g.ps], C[(long long)(15 + k) * g.ps], C[(long long)(30 + k) * g.ps],
                         C[(long long)(45 + k) * g.ps]};
    double x[4];
    from_char<double, DIR>(cs, y, x);
#pragma unroll
    for (int v = 0; v < 4; v++) {
      P[(15 * v + k) * DR_THREADS] = x[v];
      double* m = Pv + (15 * v + k) * DR_THREADS;
      *m = DIR == 0 ? 0.5 * x[v] : *m + 0.5 * x[v];
    }
  }
  // a compiler barrier: the evaluations below reload the coefficients from the slot
  asm volatile("" ::: "memory");
  double dx[4][6], dy[4][6];
#pragma unroll
  for (int v = 0; v < 4; v++) {
    double cv[15], d[15];
#pragma unroll
    for (int k = 0; k < 15; k++) cv[k] = P[(15 * v + k) * DR_THREADS];
    poly_dx<double>(cv, fx, d);
    if (DIR == 0) eval_xfaces<double>(d, dx[v]); else eval_yfaces<double>(d, dx[v]);
    poly_dy<double>(cv, fy, d);
    if (DIR == 0) eval_xfaces<double>(d, dy[v]); else eval_yfaces<double>(d, dy[v]);
    // one variable's coefficients live at a time: the next variable's loads wait here
    asm volatile("" ::: "memory");
  }
  dr_store<6>(g, w, c, dx, dy, 6 * DIR, w.face, 0);
  asm volatile("" ::: "memory");
}

// the volume points from the mean of the two directions' polynomials
__device__ __forceinline__ void dr_volume(const Grid& g, const Work& w, long long c, const double* fx,
                                          const double* fy, const double* Pv) {
  double dx[4][9], dy[4][9];
#pragma unroll
  for (int v = 0; v < 4; v++) {
    double cv[15], d[15];
#pragma unroll
    for (int k = 0; k < 15; k++) cv[k] = Pv[(15 * v + k) * DR_THREADS];
    poly_dx<double>(cv, fx, d);
    eval_vol<double>(d, dx[v]);
    poly_dy<double>(cv, fy, d);
    eval_vol<double>(d, dy[v]);
    asm volatile("" ::: "memory");
  }
  dr_store<9>(g, w, c, dx, dy, 12, w.vol, 12);
}

__device__ __forceinline__ void dr_body(const Grid& g, const double* __restrict__ q, const Work& w, int gx,
                                        int gy) {
  const int i = gx - 1;
  const int j = gy - 1;
  if (i >= g.nx + 1 || j >= g.ny + 1) return;
  extern __shared__ double dr_smem[];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  double* P = dr_smem + tid;
  double* Pv = dr_smem + 60 * DR_THREADS + tid;
  const long long c = cidx(g, i, j);
  const double ub[4] = {q[c], q[g.ps + c], q[2 * g.ps + c], q[3 * g.ps + c]};
  CharState<double> cs;
  char_state<double>(ub, g.gamma, cs);
  // the derivative factors p/dx, p/dy of the monomials' exponents p = 1..4
  const double fx[4] = {g.rdx, 2.0 * g.rdx, 3.0 * g.rdx, 4.0 * g.rdx};
  const double fy[4] = {g.rdy, 2.0 * g.rdy, 3.0 * g.rdy, 4.0 * g.rdy};
  dr_direction<0>(g, w, c, cs, fx, fy, P, Pv);
  dr_direction<1>(g, w, c, cs, fx, fy, P, Pv);
  dr_volume(g, w, c, fx, fy, Pv);
}

// PP local Lax-Friedrichs fluxes (Eq. (3.3)) of the interior faces: x-faces right
// of cells i in [-1, nx), j in [0, ny) (blockIdx.z = 0); y-faces above cells
// i in [0, nx), j in [-1, ny) (z = 1).  Also the face maxima alpha* and beta.
template <class T>
__device__ __forceinline__ void flux_body(const Grid& g, const Work& w, Diag* diag, int gx, int gy, int gz) {
  const int dir = gz;
  const int i = gx - (dir == 0 ? 1 : 0);
  const int j = gy - (dir == 0 ? 0 : 1);
  double amax = 0.0, bmax = 0.0;
  if (i < g.nx && j < g.ny) {
    const long long cl = cidx(g, i, j);
    const long long cr = dir == 0 ? cidx(g, i + 1, j) : cidx(g, i, j + 1);
    const int kl = dir == 0 ? 3 : 9, kr = dir == 0 ? 0 : 6;
    const T gam = (T)g.gamma, rPr = (T)g.rPr, rRe = (T)g.rRe;
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
        beta = tfmax(beta, wave_bound<T>(dir, st[s][gp], gs[s][gp], gam, rPr, rRe));
        const T cs = tsqrt(gam * (gam - T(1)) * st[s][gp][3]);
        amax = fmax(amax, (double)tfmax(tfabs(st[s][gp][1]) + cs, tfabs(st[s][gp][2]) + cs));
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
  if (lane_id() == 0) {
    atomic_max_pos(&diag->alpha_bits, amax);
    atomic_max_pos(&diag->beta_bits, bmax);
  }
}

// moment balances Eq. (3.2) of the interior cells
template <class T>
__device__ __forceinline__ void assemble_body(const Grid& g, const Work& w, double* __restrict__ rhs,
                                              Diag* diag, int gx, int gy) {
  const int i = gx;
  const int j = gy;
  unsigned int bad = 0;
  if (i < g.nx && j < g.ny) {
    const long long c = cidx(g, i, j), cl = cidx(g, i - 1, j), cb = cidx(g, i, j - 1);
    const T gam = (T)g.gamma, rPr = (T)g.rPr, rRe = (T)g.rRe;
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
    const double rdx = g.rdx, rdy = g.rdy;
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
      if (!finite_d(r0) || !finite_d(r1) || !finite_d(r2)) bad = FLAG_NONFINITE;
    }
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (lane_id() == 0 && bad) atomicOr(&diag->flags, bad);
}

// SSP-RK3 stage with modified moments (Eq. (2.12), 2D analogue) on interior cells:
//   stage 1: out = [u^n; vhat^n] + dt F,                        base = [u^n; vhat^n]
//   stage 2: out = 3/4 base + 1/4 ([u^(1); vhat^(1)] + dt F)
//   stage 3: out = 1/3 base + 2/3 ([u^(2); vhat^(2)] + dt F)
// plus the admissibility test of the output averages (Sec. 5).
// The SSP-RK3 stage update of one cell from its 12 residual values f (Eq. (2.12) in
// its 2D form): writes qout, and the base at stage 1; returns FLAG_INADMISSIBLE when the
// new cell average is not admissible or not finite.
// KEF (mixed handles): at stage 3, also the kinetic share |m|^2 / (2 rho E) of the new
// state in kef, the measure that routes a mixed handle's next step

// the admissibility of the new cell average out[0..4) and, KEF at stage 3, its kinetic
// share: p > 0 <=> rho E - |m|^2 / 2 > 0 once rho > 0; the share decides between FP32
// and FP64 at a margin of 1e-4, which an FP32 ratio of the FP64 energies resolves
template <bool KEF>
__device__ __forceinline__ unsigned int rk_admissible(int stage, const double* out, double& kef) {
  const double rp = out[3] * out[0] - 0.5 * (out[1] * out[1] + out[2] * out[2]);
  const bool ok = out[0] > 0.0 && rp > 0.0;
  if constexpr (KEF) {
    if (stage == 3) kef = ok ? 1.0 - (double)tdiv((float)rp, (float)(out[3] * out[0])) : 1.0;
  }
  return ok ? 0u : FLAG_INADMISSIBLE;
}

template <bool KEF = false>
__device__ __forceinline__ unsigned int rk_cell(const Grid& g, int stage, long long c, double dt,
                                                const double* __restrict__ qin, const double* __restrict__ mom,
                                                const double* f, double* __restrict__ base,
                                                double* __restrict__ qout, double& kef) {
  unsigned int bad = 0;
  double out[12];
#pragma unroll
  for (int k = 0; k < 12; k++) {
    const double cur = k < 4 ? qin[(long long)k * g.ps + c] : mom[(long long)(k - 4) * g.ps + c];
    if (stage == 1) {
      base[(long long)k * g.ps + c] = cur;
      out[k] = cur + dt * f[k];
    } else if (stage == 2) {
      out[k] = 0.75 * base[(long long)k * g.ps + c] + 0.25 * (cur + dt * f[k]);
    } else {
      out[k] = base[(long long)k * g.ps + c] * (1.0 / 3.0) + (2.0 / 3.0) * (cur + dt * f[k]);
    }
    qout[(long long)k * g.ps + c] = out[k];
    if (!finite_d(out[k])) bad = FLAG_INADMISSIBLE;
  }
  return bad | rk_admissible<KEF>(stage, out, kef);
}

// the mixed path's base of the moments (float values): 8 float planes in the room of the
// base group's double planes 4-7
__host__ __device__ inline float* mixed_moment_base(double* base, long long ps) { return (float*)(base + 4 * ps); }

// The mixed path's stage update of one cell: the averages as rk_cell does, from their
// FP64 balances f0; the moments in FP32, from their FP32 balances fm.  The moments that
// enter a stage are the modified moments of the FP32 reconstruction (Eq. (2.11)), FP32
// values held in FP64 planes, and their balances carry FP32 rounding of the flux
// scale, far above an FP32 rounding of the moments themselves; so the update runs in
// single precision (explicit fused multiply-adds, the same in every kernel) and the
// FP64 planes receive the FP32 result exactly (widen_f, narrow_exact: integer
// operations, since B300's FP64 pipe also carries the conversions).  Also writes the
// hi/lo split of the new state (the 12 hi planes and the averages' 4 lo planes at hilo:
// the moments are float values, and no kernel reads their lo planes), so that the next
// evaluation needs no separate split pass.
template <bool KEF = false>
__device__ __forceinline__ unsigned int rk_cell_mixed(const Grid& g, int stage, long long c, double dt,
                                                      const double* __restrict__ qin,
                                                      const double* __restrict__ mom, const double* f0,
                                                      const float* fm, double* __restrict__ base,
                                                      double* __restrict__ qout, float* __restrict__ hilo,
                                                      double& kef) {
  unsigned int bad = 0;
  double out[4];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const double cur = qin[(long long)k * g.ps + c];
    const double t = fma(dt, f0[k], cur);  // explicit roundings, the same in every kernel
    if (stage == 1) {
      base[(long long)k * g.ps + c] = cur;
      out[k] = t;
    } else if (stage == 2) {
      out[k] = fma(0.75, base[(long long)k * g.ps + c], dmul_rn(0.25, t));
    } else {
      out[k] = fma(1.0 / 3.0, base[(long long)k * g.ps + c], dmul_rn(2.0 / 3.0, t));
    }
    qout[(long long)k * g.ps + c] = out[k];
    float hi, lo;
    split_hilo(out[k], hi, lo);
    hilo[(long long)k * g.ps + c] = hi;
    hilo[(long long)(12 + k) * g.ps + c] = lo;
    if (!finite_d(out[k])) bad = FLAG_INADMISSIBLE;
  }
  const float dtf = (float)dt;
  float* basef = mixed_moment_base(base, g.ps);
#pragma unroll
  for (int k = 4; k < 12; k++) {
    const float cur = narrow_exact(mom[(long long)(k - 4) * g.ps + c]);
    const float t = fmaf(dtf, fm[k - 4], cur);
    float* b = basef + (long long)(k - 4) * g.ps + c;
    float o;
    if (stage == 1) {
      *b = cur;
      o = t;
    } else if (stage == 2) {
      o = fmaf(0.75f, *b, 0.25f * t);
    } else {
      o = fmaf(1.0f / 3.0f, *b, (2.0f / 3.0f) * t);
    }
    qout[(long long)k * g.ps + c] = widen_f(o);
    hilo[(long long)k * g.ps + c] = o;  // a float value: no lo part
    if (!finite_f(o)) bad = FLAG_INADMISSIBLE;
  }
  return bad | rk_admissible<KEF>(stage, out, kef);
}

// the warp's flags and (KEF, stage 3) kinetic shares into the step's reductions
template <bool KEF>
__device__ __forceinline__ void rk_reduce(int stage, unsigned int bad, double kef, Diag* diag) {
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (lane_id() == 0 && bad) atomicOr(&diag->flags, bad);
  if constexpr (KEF) {
    if (stage == 3) {
      kef = warp_max(fmax(kef, 0.0));
      if (lane_id() == 0) atomic_max_pos(&diag->kefrac_bits, kef);
    }
  }
}

// the stage update of cell (gx, gy) from the residual planes rhs; SPLIT: the mixed path's
// (rk_cell_mixed, the moments' balances narrowed from their FP64 planes exactly)
template <bool SPLIT = false, bool KEF = false>
__device__ __forceinline__ void rk_body(const Grid& g, int stage, const double* __restrict__ qin,
                                        const double* __restrict__ mom, const double* __restrict__ rhs,
                                        double* __restrict__ base, double* __restrict__ qout, Diag* diag,
                                        int gx, int gy, float* __restrict__ hilo = nullptr) {
  const int i = gx;
  const int j = gy;
  unsigned int bad = 0;
  double kef = 0.0;
  if (i < g.nx && j < g.ny) {
    const long long c = cidx(g, i, j);
    if constexpr (SPLIT) {
      double f0[4];
      float fm[8];
#pragma unroll
      for (int k = 0; k < 4; k++) f0[k] = rhs[(long long)k * g.ps + c];
#pragma unroll
      for (int k = 0; k < 8; k++) fm[k] = narrow_exact(rhs[(long long)(4 + k) * g.ps + c]);
      bad = rk_cell_mixed<KEF>(g, stage, c, diag->dt, qin, mom, f0, fm, base, qout, hilo, kef);
    } else {
      double f[12];
#pragma unroll
      for (int k = 0; k < 12; k++) f[k] = rhs[(long long)k * g.ps + c];
      bad = rk_cell<KEF>(g, stage, c, diag->dt, qin, mom, f, base, qout, kef);
    }
  }
  rk_reduce<KEF>(stage, bad, kef, diag);
}

}  // namespace hw
