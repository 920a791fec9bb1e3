// Mixed-precision spatial operator: reconstruction, weights, gradients, fluxes and the
// moment balances in FP32; the stored state, the positivity limiter's checks and theta
// solve where they can bind, the face-flux differences of the average balances (exact
// conservation) and the RK update in FP64.
//
// FP32 intermediates share the handle's scratch planes: a float plane k of a group
// starts at (float*)group + k * ps, so a group of n double planes holds 2n float
// planes.  The state is kept split into float planes hi (the double truncated to 24
// significant bits) and lo (the remainder), stored after the 48 float face planes in the
// face group's unused half; the RK update writes the split with the state, a separate
// pass splits a state set from outside.  Offsets from a cell's own average,
// (hi_k - hi_c) + (lo_k - lo_c), are then exact to FP32 rounding of the offset itself
// rather than of the average.
#pragma once
#include "hweno_ops.cuh"

namespace hw {

struct WorkF {
  float* face;   // 48: point k x (rho, u, v, e), limited
  float* vol;    // 36: point k x (rho, u, v, e)
  float* wbar;   // 3
  float* wx;     // 6
  float* wy;     // 6
  float* rm;     // 18
  float* gr;     // 126: 6 components at the 12 face points, then at the 9 volume points
  float* hilo;   // 24: hi of the 12 state planes, then lo (kept for the 4 average planes only)
  // the volume integrals of Eq. (3.2), per interior cell, from the gradient pass: vs, 14
  // sums of the gradient components over the 3x3 volume points (vol_visc_sums); iv, 8
  // quadrature sums of the inviscid fluxes (x then y, per conserved variable).  Float planes 126-147 of the
  // gradient group, which holds 252.
  float* vs;
  float* iv;
};

// FP32 face sums of the mixed path: S0 (planes 0-3) and S1 (4-7) of each conserved
// variable, in the face-flux group's double planes 8-11, which it does not use otherwise
__host__ __device__ inline float* mixed_face_sums(double* f, long long ps) { return (float*)(f + 8 * ps); }
__host__ __device__ inline const float* mixed_face_sums(const double* f, long long ps) {
  return (const float*)(f + 8 * ps);
}

__host__ __device__ inline WorkF mixed_planes(const Work& w, long long ps) {
  WorkF f;
  f.face = (float*)w.face;
  f.hilo = (float*)w.face + 48 * ps;
  f.vol = (float*)w.vol;
  f.wbar = (float*)w.wbar;
  f.wx = (float*)w.wx;
  f.wy = (float*)w.wy;
  f.rm = (float*)w.rm;
  f.gr = (float*)w.gr;
  f.vs = f.gr + 126 * ps;
  f.iv = f.vs + 14 * ps;
  return f;
}

__global__ void k_split(Grid g, const double* __restrict__ q, float* __restrict__ hilo) {
  const long long n = 12 * g.ps;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n;
       t += (long long)gridDim.x * blockDim.x) {
    float hi, lo;
    split_hilo(q[t], hi, lo);
    hilo[t] = hi;
    if (t < 4 * g.ps) hilo[n + t] = lo;  // the averages' lo planes (no kernel reads the moments')
  }
}

__device__ __forceinline__ void to_prim(const double* s, float* w) {
  const double rr = 1.0 / s[0];
  const double u = s[1] * rr, v = s[2] * rr;
  w[0] = (float)s[0];
  w[1] = (float)u;
  w[2] = (float)v;
  w[3] = (float)(s[3] * rr - 0.5 * (u * u + v * v));
}

__device__ __forceinline__ void to_prim_f(const float* s, float* w) {
  const float rr = tdiv(1.0f, s[0]);
  w[0] = s[0];
  w[1] = s[1] * rr;
  w[2] = s[2] * rr;
  w[3] = s[3] * rr - 0.5f * (w[1] * w[1] + w[2] * w[2]);
}

// FP32 admissibility filter: true only if the FP64 limiter check would certainly pass
// (rho and the internal energy clear of zero by a margin far above FP32 rounding) and
// the internal energy is at least 1 % of E, so that FP32 primitives keep about 6
// significant digits of e.  Otherwise the cell takes the FP64 route.
__device__ __forceinline__ bool clearly_fine(const float* s, float rho_ref) {
  const float ke = 0.5f * (s[1] * s[1] + s[2] * s[2]);
  const float ie = s[3] * s[0] - ke;  // rho * (rho e)
  return s[0] > 1e-4f * rho_ref && ie > 1e-2f * (fabsf(s[3] * s[0]) + ke);
}

__device__ __forceinline__ void cons_mixed_body(const Grid& g, const double* __restrict__ q, const Work& w,
                                                double* __restrict__ mom, Diag* diag, int gx, int gy) {
  const int i = gx - 3;
  const int j = gy - 3;
  unsigned long long pp = 0;
  unsigned int flags = 0;
  const WorkF f = mixed_planes(w, g.ps);
  if (i < g.nx + 3 && j < g.ny + 3) {
    const long long c = cidx(g, i, j);
    const long long n12 = 12 * g.ps;
    // the p0 coefficients (60) and the x-system's volume values (36) wait in this
    // thread's slot of shared memory, [96][128] floats (blocks of 128 threads), so that
    // they do not occupy registers while the reconstructions run
    __shared__ float mixed_smem[96 * 128];
    const int tid = threadIdx.y * blockDim.x + threadIdx.x;
    float* ccs = mixed_smem + tid;
    float* park = mixed_smem + 60 * 128 + tid;
    float cc[4][15], sl[4][4], hc[4], lc[4];
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const float* H = f.hilo + (long long)v * g.ps;
      const float* L = H + n12;
      const float* X = f.hilo + (long long)(4 + v) * g.ps;
      const float* Y = f.hilo + (long long)(8 + v) * g.ps;
      hc[v] = H[c];
      lc[v] = L[c];
      float d[17];
#pragma unroll
      for (int b = -1; b <= 1; b++)
#pragma unroll
        for (int a = -1; a <= 1; a++) {
          const long long k = cidx(g, i + a, j + b);
          d[(b + 1) * 3 + (a + 1)] = (H[k] - hc[v]) + (L[k] - lc[v]);
        }
      d[4] = 0.0f;
      d[9] = X[cidx(g, i - 1, j)];
      d[10] = X[cidx(g, i + 1, j)];
      d[11] = Y[cidx(g, i, j - 1)];
      d[12] = Y[cidx(g, i, j + 1)];
      d[13] = X[cidx(g, i, j - 1)];
      d[14] = X[cidx(g, i, j + 1)];
      d[15] = Y[cidx(g, i - 1, j)];
      d[16] = Y[cidx(g, i + 1, j)];
      hw_p0_coeffs<float>(d, cc[v]);
#pragma unroll
      for (int k = 0; k < 15; k++) ccs[(15 * v + k) * 128] = cc[v][k];
      sl[v][0] = -d[3];
      sl[v][1] = d[5];
      sl[v][2] = -d[1];
      sl[v][3] = d[7];
    }
    const float ubf[4] = {hc[0] + lc[0], hc[1] + lc[1], hc[2] + lc[2], hc[3] + lc[3]};
    const float zero[4] = {0.f, 0.f, 0.f, 0.f};
    float face[12][4], vol[9][4], volx[9][4], mx[4], my[4];
    CharState<float> cs;
    char_state<float>(ubf, g.gammaf, cs);
    asm volatile("" ::: "memory");  // the reconstructions load the coefficients from shared memory
    const CoefShared<float> ccsh{ccs};
    recon_dir<float, 0>(ccsh, sl, zero, cs, g.eps_wenof, face, volx, mx);
#pragma unroll
    for (int k = 0; k < 9; k++)
#pragma unroll
      for (int v = 0; v < 4; v++) park[(4 * k + v) * 128] = volx[k][v];
    asm volatile("" ::: "memory");
    recon_dir<float, 1>(ccsh, sl, zero, cs, g.eps_wenof, face + 6, vol, my);
#pragma unroll
    for (int k = 0; k < 9; k++)
#pragma unroll
      for (int v = 0; v < 4; v++) vol[k][v] = 0.5f * (park[(4 * k + v) * 128] + vol[k][v]);
    // face[][] and vol[][] hold offsets from the cell average
    bool fine = true;
#pragma unroll
    for (int k = 0; k < 21; k++) {
      float s[4];
#pragma unroll
      for (int v = 0; v < 4; v++) s[v] = (k < 12 ? face[k][v] : vol[k - 12][v]) + ubf[v];
      fine = fine && clearly_fine(s, ubf[0]);
    }
    const bool interior = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
    double th[2] = {1.0, 1.0};
    float wb[3] = {0.f, 0.f, 0.f};
    if (fine) {
#pragma unroll
      for (int k = 0; k < 12; k++) {
        float s[4], p[4];
#pragma unroll
        for (int v = 0; v < 4; v++) s[v] = face[k][v] + ubf[v];
        to_prim_f(s, p);
#pragma unroll
        for (int v = 0; v < 4; v++) f.face[(long long)(4 * k + v) * g.ps + c] = p[v];
      }
#pragma unroll
      for (int G = 0; G < 3; G++)
#pragma unroll
        for (int Hh = 0; Hh < 3; Hh++) {
          const int k = 3 * G + Hh;
          float s[4], p[4];
#pragma unroll
          for (int v = 0; v < 4; v++) s[v] = vol[k][v] + ubf[v];
          to_prim_f(s, p);
#pragma unroll
          for (int v = 0; v < 4; v++) f.vol[(long long)(4 * k + v) * g.ps + c] = p[v];
          const float wgt = gweight<float>(G) * gweight<float>(Hh);
          wb[0] += wgt * p[1];
          wb[1] += wgt * p[2];
          wb[2] += wgt * p[3];
        }
    } else {
      // FP64 route: the limiter of Sec. 3.1 on ub + offset, exactly as in the FP64 path
      double ub[4], fd[12][4], vd[9][4];
#pragma unroll
      for (int v = 0; v < 4; v++) ub[v] = q[(long long)v * g.ps + c];
#pragma unroll
      for (int v = 0; v < 4; v++) {
#pragma unroll
        for (int k = 0; k < 12; k++) fd[k][v] = ub[v] + (double)face[k][v];
#pragma unroll
        for (int k = 0; k < 9; k++) vd[k][v] = ub[v] + (double)vol[k][v];
      }
      const double pb = pressure(ub, g.gamma);
      if (!(ub[0] > 0.0) || !(pb > 0.0)) flags |= FLAG_BADAVG;
      else if (pp_limit(ub, fd, vd, g.gamma, g.eps_pp, th) && interior) pp = 1;
#pragma unroll
      for (int k = 0; k < 12; k++) {
        float p[4];
        to_prim(fd[k], p);
#pragma unroll
        for (int v = 0; v < 4; v++) f.face[(long long)(4 * k + v) * g.ps + c] = p[v];
      }
#pragma unroll
      for (int G = 0; G < 3; G++)
#pragma unroll
        for (int Hh = 0; Hh < 3; Hh++) {
          const int k = 3 * G + Hh;
          float p[4];
          to_prim(vd[k], p);
#pragma unroll
          for (int v = 0; v < 4; v++) f.vol[(long long)(4 * k + v) * g.ps + c] = p[v];
          const float wgt = gweight<float>(G) * gweight<float>(Hh);
          wb[0] += wgt * p[1];
          wb[1] += wgt * p[2];
          wb[2] += wgt * p[3];
        }
    }
#pragma unroll
    for (int n = 0; n < 3; n++) f.wbar[(long long)n * g.ps + c] = wb[n];
    w.theta[c] = th[0];
    w.theta[g.ps + c] = th[1];
    if (interior) {
      // the conversion instruction: this kernel leaves the FP64 pipe nearly idle, and the
      // 8 conversions cost it less than widen_f's integer form (measured, 8 % of the kernel)
#pragma unroll
      for (int v = 0; v < 4; v++) {
        mom[(long long)v * g.ps + c] = (double)mx[v];
        mom[(long long)(4 + v) * g.ps + c] = (double)my[v];
      }
    }
  }
  pp = warp_sum_u64(pp);
  flags = __reduce_or_sync(0xffffffffu, flags);
  if (lane_id() == 0) {
    if (pp) atomicAdd(&diag->pp_count, pp);
    if (flags) atomicOr(&diag->flags, flags);
  }
}

// Eq. (3.6) in FP32 on the float traces
__device__ __forceinline__ void face_moments_mixed_body(const Grid& g, const Work& w, int gx, int gy, int gz) {
  const int dir = gz;
  const int i = gx - (dir == 0 ? 3 : 2);
  const int j = gy - (dir == 0 ? 2 : 3);
  if (i >= g.nx + 2 || j >= g.ny + 2) return;
  const WorkF f = mixed_planes(w, g.ps);
  const long long cl = cidx(g, i, j);
  const long long cr = dir == 0 ? cidx(g, i + 1, j) : cidx(g, i, j + 1);
  const int kl = dir == 0 ? 3 : 9, kr = dir == 0 ? 0 : 6;
  float W0[3] = {0.f, 0.f, 0.f}, W1[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int gp = 0; gp < 3; gp++) {
    const float wg = gweight<float>(gp), xg = gnode<float>(gp);
#pragma unroll
    for (int n = 0; n < 3; n++) {
      const float a = f.face[(long long)(4 * (kl + gp) + 1 + n) * g.ps + cl];
      const float b = f.face[(long long)(4 * (kr + gp) + 1 + n) * g.ps + cr];
      const float h = 0.5f * (a + b);
      W0[n] += wg * h;
      W1[n] += wg * h * xg;
    }
  }
  float* out = dir == 0 ? f.wx : f.wy;
#pragma unroll
  for (int n = 0; n < 3; n++) {
    out[(long long)n * g.ps + cl] = W0[n];
    out[(long long)(3 + n) * g.ps + cl] = W1[n];
  }
}

// Eqs. (3.7)-(3.8) in FP32
__device__ __forceinline__ void weak_moments_mixed_body(const Grid& g, const Work& w, int gx, int gy) {
  const int i = gx - 2;
  const int j = gy - 2;
  if (i >= g.nx + 2 || j >= g.ny + 2) return;
  const WorkF f = mixed_planes(w, g.ps);
  const long long c = cidx(g, i, j), cl = cidx(g, i - 1, j), cb = cidx(g, i, j - 1);
  const float rdx = g.rdxf, rdy = g.rdyf;
#pragma unroll
  for (int n = 0; n < 3; n++) {
    const float xr0 = f.wx[(long long)n * g.ps + c], xl0 = f.wx[(long long)n * g.ps + cl];
    const float xr1 = f.wx[(long long)(3 + n) * g.ps + c], xl1 = f.wx[(long long)(3 + n) * g.ps + cl];
    const float yt0 = f.wy[(long long)n * g.ps + c], yb0 = f.wy[(long long)n * g.ps + cb];
    const float yt1 = f.wy[(long long)(3 + n) * g.ps + c], yb1 = f.wy[(long long)(3 + n) * g.ps + cb];
    const float wb = f.wbar[(long long)n * g.ps + c];
    float* r = f.rm + (long long)(6 * n) * g.ps + c;
    r[0] = (xr0 - xl0) * rdx;
    r[g.ps] = (0.5f * (xr0 + xl0) - wb) * rdx;
    r[2 * g.ps] = (xr1 - xl1) * rdx;
    r[3 * g.ps] = (yt0 - yb0) * rdy;
    r[4 * g.ps] = (yt1 - yb1) * rdy;
    r[5 * g.ps] = (0.5f * (yt0 + yb0) - wb) * rdy;
  }
}

// The viscous part of Eq. (3.2)'s volume integrals.  The viscous fluxes are linear in
// the six gradient components s = (u_x, u_y, v_x, v_y, e_x, e_y), with coefficients 1, u,
// v (and gamma / Pr for e) over Re, so their 3x3-point quadrature sums need only, per
// component, S = sum_k w_k s_k and, for the velocity gradients, Su = sum_k w_k u_k s_k
// and Sv = sum_k w_k v_k s_k: 14 sums, accumulated as each component is reconstructed, in
// place of the 54 volume-point gradients (balance_mixed combines them with the inviscid
// sums, formed here too from the volume values).
// one volume point's inviscid fluxes (the terms of phys_flux without gradients) from its
// primitive values p = (rho, u, v, e), weighted by wgt into iv (x fluxes, then y fluxes)
// (explicit roundings, the same in every kernel)
__device__ __forceinline__ void inviscid_acc(const float* p, float wgt, float gam, float* iv) {
  const float rho = p[0], u = p[1], v = p[2], e = p[3];
  const float pr = mul_rn(mul_rn(gam - 1.0f, rho), e);
  const float E = mul_rn(rho, fmaf(0.5f, fmaf(u, u, mul_rn(v, v)), e));
  const float m = mul_rn(rho, u), n = mul_rn(rho, v), H = add_rn(E, pr);
  iv[0] = fmaf(wgt, m, iv[0]);
  iv[1] = fmaf(wgt, fmaf(m, u, pr), iv[1]);
  iv[2] = fmaf(wgt, mul_rn(m, v), iv[2]);
  iv[3] = fmaf(wgt, mul_rn(H, u), iv[3]);
  iv[4] = fmaf(wgt, n, iv[4]);
  iv[5] = fmaf(wgt, mul_rn(n, u), iv[5]);
  iv[6] = fmaf(wgt, fmaf(n, v, pr), iv[6]);
  iv[7] = fmaf(wgt, mul_rn(H, v), iv[7]);
}

// vol_weights: w_k u_k and w_k v_k of cell c's volume points (k = 3 G + H, w_k the
// product of the Gauss weights), and the inviscid part of the volume integrals from the
// same points' primitive values into f.iv
__device__ __forceinline__ void vol_weights(const Grid& g, const WorkF& f, long long c, float* wu, float* wv) {
  float iv[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
  for (int k = 0; k < 9; k++) {
    const float wk = gweight<float>(k / 3) * gweight<float>(k % 3);
    float p[4];
#pragma unroll
    for (int v = 0; v < 4; v++) p[v] = f.vol[(long long)(4 * k + v) * g.ps + c];
    wu[k] = mul_rn(wk, p[1]);
    wv[k] = mul_rn(wk, p[2]);
    inviscid_acc(p, wk, g.gammaf, iv);
  }
#pragma unroll
  for (int k = 0; k < 8; k++) f.iv[(long long)k * g.ps + c] = iv[k];
}
// component comp's sums from its volume-point values cen + vv[k], into f.vs: S at plane
// comp, Su at 6 + comp and Sv at 10 + comp (comp < 4)
__device__ __forceinline__ void vol_visc_sums(const Grid& g, const WorkF& f, long long c, int comp, float cen,
                                              const float* vv, const float* wu, const float* wv) {
  float S = 0.f, Su = 0.f, Sv = 0.f;
#pragma unroll
  for (int k = 0; k < 9; k++) {
    const float sk = add_rn(cen, vv[k]);
    S = fmaf(gweight<float>(k / 3) * gweight<float>(k % 3), sk, S);
    Su = fmaf(wu[k], sk, Su);
    Sv = fmaf(wv[k], sk, Sv);
  }
  f.vs[(long long)comp * g.ps + c] = S;
  if (comp < 4) {
    f.vs[(long long)(6 + comp) * g.ps + c] = Su;
    f.vs[(long long)(10 + comp) * g.ps + c] = Sv;
  }
}

// Eq. (3.9) in FP32 on offsets from the centre value; LIN: the linear weights, whose
// combination is p0 itself (the ablation of Remark 3.1).  Interior cells also get the
// volume sums (vol_visc_sums); VOLG: also the gradients at the 9 volume points (the
// debug export's full field; the operator needs only their sums)
template <bool LIN = false, bool VOLG = false>
__device__ __forceinline__ void grad_mixed_body(const Grid& g, const Work& w, int gx, int gy) {
  const int i = gx - 1;
  const int j = gy - 1;
  if (i >= g.nx + 1 || j >= g.ny + 1) return;
  const WorkF f = mixed_planes(w, g.ps);
  const long long c = cidx(g, i, j);
  const float eps = g.eps_wenof;
  const bool interior = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
  float wu[9], wv[9];
  if (interior) vol_weights(g, f, c, wu, wv);
#pragma unroll 1
  for (int comp = 0; comp < 6; comp++) {
    const int n = comp >> 1, l = comp & 1;
    const float* A = f.rm + (long long)(6 * n + 3 * l) * g.ps;
    const float* X = A + g.ps;
    const float* Y = A + 2 * g.ps;
    const float cen = A[c];
    float d[17];
#pragma unroll
    for (int b = -1; b <= 1; b++)
#pragma unroll
      for (int a = -1; a <= 1; a++) d[(b + 1) * 3 + (a + 1)] = A[cidx(g, i + a, j + b)] - cen;
    d[4] = 0.0f;
    d[9] = X[cidx(g, i - 1, j)];
    d[10] = X[cidx(g, i + 1, j)];
    d[11] = Y[cidx(g, i, j - 1)];
    d[12] = Y[cidx(g, i, j + 1)];
    d[13] = X[cidx(g, i, j - 1)];
    d[14] = X[cidx(g, i, j + 1)];
    d[15] = Y[cidx(g, i - 1, j)];
    d[16] = Y[cidx(g, i + 1, j)];
    float C[15];
    if constexpr (LIN)
      hw_p0_coeffs<float>(d, C);
    else
      hweno_combine<float>(d, eps, C);
    float vx[6], vy[6], vv[9];
    eval_xfaces<float>(C, vx);
    eval_yfaces<float>(C, vy);
    eval_vol<float>(C, vv);
    float* out = f.gr + (long long)comp * g.ps + c;
#pragma unroll
    for (int k = 0; k < 6; k++) out[(long long)(6 * k) * g.ps] = cen + vx[k];
#pragma unroll
    for (int k = 0; k < 6; k++) out[(long long)(6 * (6 + k)) * g.ps] = cen + vy[k];
    if constexpr (VOLG) {
#pragma unroll
      for (int k = 0; k < 9; k++) out[(long long)(6 * (12 + k)) * g.ps] = cen + vv[k];
    }
    if (interior) vol_visc_sums(g, f, c, comp, cen, vv, wu, wv);
  }
}

// Eq. (3.3) in FP32 at one face (dir 0: the x-face between cells cl and cr = cl + 1 in
// x; dir 1: the y-face): the weighted sums S0[v] = sum_g w_g fhat_g and S1[v] = sum_g
// w_g s_g fhat_g of the PP-LLF fluxes at its three Gauss points (s_g the tangential
// node); returns the Lax-Friedrichs coefficient beta and raises amax to the face's
// largest max(|u| + c, |v| + c)
__device__ __forceinline__ float face_sums_mixed(const Grid& g, const WorkF& f, int dir, long long cl, long long cr,
                                                 float* S0, float* S1, float& amax) {
  const int kl = dir == 0 ? 3 : 9, kr = dir == 0 ? 0 : 6;
  const float gam = g.gammaf, rPr = g.rPrf, rRe = g.rRef;
  float st[2][3][4], gs[2][3][6];
#pragma unroll
  for (int gp = 0; gp < 3; gp++)
#pragma unroll
    for (int s = 0; s < 2; s++) {
      const long long cc = s == 0 ? cl : cr;
      const int k = (s == 0 ? kl : kr) + gp;
#pragma unroll
      for (int v = 0; v < 4; v++) st[s][gp][v] = f.face[(long long)(4 * k + v) * g.ps + cc];
#pragma unroll
      for (int n = 0; n < 6; n++) gs[s][gp][n] = f.gr[(long long)(6 * k + n) * g.ps + cc];
    }
  float beta = 0.f;
#pragma unroll
  for (int gp = 0; gp < 3; gp++)
#pragma unroll
    for (int s = 0; s < 2; s++) {
      beta = fmaxf(beta, wave_bound<float>(dir, st[s][gp], gs[s][gp], gam, rPr, rRe));
      const float cs = sqrtf(gam * (gam - 1.f) * st[s][gp][3]);
      amax = fmaxf(amax, fmaxf(fabsf(st[s][gp][1]) + cs, fabsf(st[s][gp][2]) + cs));
    }
#pragma unroll
  for (int v = 0; v < 4; v++) S0[v] = S1[v] = 0.f;
#pragma unroll
  for (int gp = 0; gp < 3; gp++) {
    float fl[4], fr[4], ul[4], ur[4];
    phys_flux<float>(dir, st[0][gp], gs[0][gp], gam, rPr, rRe, fl);
    phys_flux<float>(dir, st[1][gp], gs[1][gp], gam, rPr, rRe, fr);
#pragma unroll
    for (int s = 0; s < 2; s++) {
      float* u = s == 0 ? ul : ur;
      const float* p = st[s][gp];
      u[0] = p[0];
      u[1] = p[0] * p[1];
      u[2] = p[0] * p[2];
      u[3] = p[0] * (p[3] + 0.5f * (p[1] * p[1] + p[2] * p[2]));
    }
    const float wg = gweight<float>(gp), wt = gweight<float>(gp) * gnode<float>(gp);
#pragma unroll
    for (int v = 0; v < 4; v++) {
      const float fh = 0.5f * (fl[v] + fr[v] - beta * (ur[v] - ul[v]));
      S0[v] += wg * fh;
      if (gp != 1) S1[v] += wt * fh;
    }
  }
  return beta;
}

// One face's sums written to the face-flux planes (S0 in FP64 planes 0-3 and again, with
// S1, as FP32 planes in 8-11), and assemble_mixed_body below: the per-face and per-cell
// form of what the flux tile kernels compute in shared memory.  No GPU kernel launches
// them; the host checks run them as the reference the tiles must equal.
__device__ __forceinline__ void flux_mixed_body(const Grid& g, const Work& w, Diag* diag, int gx, int gy, int gz) {
  const int dir = gz;
  const int i = gx - (dir == 0 ? 1 : 0);
  const int j = gy - (dir == 0 ? 0 : 1);
  float amax = 0.f, bmax = 0.f;
  const WorkF f = mixed_planes(w, g.ps);
  if (i < g.nx && j < g.ny) {
    const long long cl = cidx(g, i, j);
    const long long cr = dir == 0 ? cidx(g, i + 1, j) : cidx(g, i, j + 1);
    float S0[4], S1[4];
    bmax = face_sums_mixed(g, f, dir, cl, cr, S0, S1, amax);
    // S0 in FP64 planes 0-3: the average balances difference it in FP64, so their sum
    // over a periodic grid telescopes to FP64 rounding; S0 and S1 again as FP32 planes
    // (in double planes 8-11) for the moment balances, which run in FP32
    double* out = (dir == 0 ? w.fx : w.fy) + cl;
    float* outf = mixed_face_sums(dir == 0 ? w.fx : w.fy, g.ps) + cl;
#pragma unroll
    for (int v = 0; v < 4; v++) {
      out[(long long)v * g.ps] = widen_f(S0[v]);
      outf[(long long)v * g.ps] = S0[v];
      outf[(long long)(4 + v) * g.ps] = S1[v];
    }
  }
  amax = warp_max(amax);
  bmax = warp_max(bmax);
  if (lane_id() == 0) {
    atomic_max_pos(&diag->alpha_bits, (double)amax);
    atomic_max_pos(&diag->beta_bits, (double)bmax);
  }
}

// Eq. (3.2) for one cell: the volume integrals in FP32 from the sums that the trace pass
// (inviscid, f.iv) and the gradient pass (viscous, f.vs) leave, and the three balances from the face sums (S0 in [0, 4), S1 in [4, 8)) of its right
// (sR) and left (sL) x-faces and top (tT) and bottom (tB) y-faces: the average balances
// r0 in FP64 from the same S0 widened to FP64 (dR, dL, dT, dB: exact, so a periodic sum
// telescopes to FP64 rounding), the moment balances rm (x moments, then y moments) in
// FP32 like the volume fluxes they combine with.  Returns FLAG_NONFINITE for a
// non-finite balance.
__device__ __forceinline__ unsigned int balance_mixed(const Grid& g, const WorkF& f, long long c, const float* sR,
                                                      const float* sL, const float* tT, const float* tB,
                                                      const double* dR, const double* dL, const double* dT,
                                                      const double* dB, double* r0, float* rm) {
  unsigned int bad = 0;
  // the volume integrals: the inviscid sums minus the viscous ones over Re, those from the
  // gradient sums of vol_visc_sums (the stresses' and heat flux's linear combinations)
  float S[6], Su[4], Sv[4], vf[4], vg[4];
#pragma unroll
  for (int k = 0; k < 6; k++) S[k] = f.vs[(long long)k * g.ps + c];
#pragma unroll
  for (int k = 0; k < 4; k++) {
    Su[k] = f.vs[(long long)(6 + k) * g.ps + c];
    Sv[k] = f.vs[(long long)(10 + k) * g.ps + c];
  }
  // (explicit roundings, the same in every kernel)
  const float rRe = g.rRef, gk = mul_rn(g.gammaf, g.rPrf);
  const float c43 = 4.0f / 3.0f, c23 = -2.0f / 3.0f;
  const float txx = fmaf(c43, S[0], mul_rn(c23, S[3]));
  const float txy = add_rn(S[1], S[2]);
  const float tyy = fmaf(c43, S[3], mul_rn(c23, S[0]));
  const float ex = fmaf(gk, S[4], add_rn(fmaf(c43, Su[0], mul_rn(c23, Su[3])), add_rn(Sv[1], Sv[2])));
  const float ey = fmaf(gk, S[5], add_rn(add_rn(Su[1], Su[2]), fmaf(c43, Sv[3], mul_rn(c23, Sv[0]))));
#pragma unroll
  for (int v = 0; v < 4; v++) {
    vf[v] = f.iv[(long long)v * g.ps + c];
    vg[v] = f.iv[(long long)(4 + v) * g.ps + c];
  }
  vf[1] = fmaf(-txx, rRe, vf[1]);
  vf[2] = fmaf(-txy, rRe, vf[2]);
  vf[3] = fmaf(-ex, rRe, vf[3]);
  vg[1] = fmaf(-txy, rRe, vg[1]);
  vg[2] = fmaf(-tyy, rRe, vg[2]);
  vg[3] = fmaf(-ey, rRe, vg[3]);
  const double rdx = g.rdx, rdy = g.rdy;
  const float rdxf = g.rdxf, rdyf = g.rdyf, hx = 0.5f * rdxf, hy = 0.5f * rdyf;
#pragma unroll
  for (int v = 0; v < 4; v++) {
    r0[v] = -dadd_rn(dmul_rn(dadd_rn(dR[v], -dL[v]), rdx), dmul_rn(dadd_rn(dT[v], -dB[v]), rdy));
    rm[v] = fmaf(vf[v], rdxf, -add_rn(mul_rn(add_rn(sL[v], sR[v]), hx), mul_rn(add_rn(tT[4 + v], -tB[4 + v]), rdyf)));
    rm[4 + v] = fmaf(vg[v], rdyf,
                     -add_rn(mul_rn(add_rn(sR[4 + v], -sL[4 + v]), rdxf), mul_rn(add_rn(tB[v], tT[v]), hy)));
    if (!finite_d(r0[v]) || !finite_f(rm[v]) || !finite_f(rm[4 + v])) bad = FLAG_NONFINITE;
  }
  return bad;
}

// the residual planes of cell c: the FP64 average balances, the FP32 moment balances
// widened exactly
__device__ __forceinline__ void store_residual_mixed(const Grid& g, long long c, const double* r0, const float* rm,
                                                     double* __restrict__ rhs) {
#pragma unroll
  for (int k = 0; k < 4; k++) rhs[(long long)k * g.ps + c] = r0[k];
#pragma unroll
  for (int k = 0; k < 8; k++) rhs[(long long)(4 + k) * g.ps + c] = widen_f(rm[k]);
}

__device__ __forceinline__ void assemble_mixed_body(const Grid& g, const Work& w, double* __restrict__ rhs,
                                                    Diag* diag, int gx, int gy) {
  const int i = gx;
  const int j = gy;
  unsigned int bad = 0;
  const WorkF f = mixed_planes(w, g.ps);
  if (i < g.nx && j < g.ny) {
    const long long c = cidx(g, i, j), cl = cidx(g, i - 1, j), cb = cidx(g, i, j - 1);
    const float* fxf = mixed_face_sums(w.fx, g.ps);
    const float* fyf = mixed_face_sums(w.fy, g.ps);
    float sR[8], sL[8], tT[8], tB[8];
    double dR[4], dL[4], dT[4], dB[4];
#pragma unroll
    for (int k = 0; k < 8; k++) {
      sR[k] = fxf[(long long)k * g.ps + c];
      sL[k] = fxf[(long long)k * g.ps + cl];
      tT[k] = fyf[(long long)k * g.ps + c];
      tB[k] = fyf[(long long)k * g.ps + cb];
    }
#pragma unroll
    for (int v = 0; v < 4; v++) {  // the FP64 planes of S0 (flux_mixed_body's widening)
      dR[v] = w.fx[(long long)v * g.ps + c];
      dL[v] = w.fx[(long long)v * g.ps + cl];
      dT[v] = w.fy[(long long)v * g.ps + c];
      dB[v] = w.fy[(long long)v * g.ps + cb];
    }
    double r0[4];
    float rm[8];
    bad = balance_mixed(g, f, c, sR, sL, tT, tB, dR, dL, dT, dB, r0, rm);
    store_residual_mixed(g, c, r0, rm, rhs);
  }
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (lane_id() == 0 && bad) atomicOr(&diag->flags, bad);
}

// Stages 2 and 3 of a mixed step, after the gradients: the face flux sums of a tile of
// FR_TX x FR_TY cells in shared memory (a face on the tile's edge is also computed by the
// neighbouring tile, with the same operations on the same data, so both cells of a face
// difference the same value and conservation is kept), then the balances and the stage
// update of the tile's cells.  The residual and the face sums never go to HBM.  The
// operations are those of flux_mixed_body, assemble_mixed_body and rk_body in their
// order (the host build, which fuses no multiply-add, finds the results equal bit for
// bit; on the GPU each kernel's fusions may differ, within FP32 rounding).  Stage 1's
// update cannot be fused this way: its step size needs alpha* over every face first, and
// its residual is kept for restarts (k_flux_asm_mixed writes it).
constexpr int FR_TX = 32, FR_TY = 7, FR_THREADS = 256;
// resident blocks per SM that the tile kernels' register budget is set for (3: 80
// registers, no spills)
#ifndef HWENO_FR_MIN_BLOCKS
#define HWENO_FR_MIN_BLOCKS 3
#endif
static_assert((FR_TX + 1) * FR_TY <= FR_THREADS && FR_TX * (FR_TY + 1) <= FR_THREADS, "one face per thread");

// the tile's face sums: x-face right of cell (i0 - 1 + a, j0 + b) at sx[k][b][a], y-face
// above cell (i0 + a, j0 - 1 + b) at sy[k][b][a], k = S0 (0-3), S1 (4-7); S0 again widened
// to FP64 in dx, dy (once per face rather than once per cell)
struct FluxTile {
  float sx[8][FR_TY][FR_TX + 1];
  float sy[8][FR_TY + 1][FR_TX];
  double dx[4][FR_TY][FR_TX + 1];
  double dy[4][FR_TY + 1][FR_TX];
};

// thread t's x-face and y-face of the tile at (i0, j0)
__device__ __forceinline__ void flux_tile_faces(const Grid& g, const WorkF& f, int i0, int j0, int t, FluxTile& ft,
                                                float& amax, float& bmax) {
  if (t < (FR_TX + 1) * FR_TY) {
    const int a = t % (FR_TX + 1), b = t / (FR_TX + 1);
    const int i = i0 - 1 + a, j = j0 + b;
    if (i < g.nx && j < g.ny) {
      float S[8];
      bmax = fmaxf(bmax, face_sums_mixed(g, f, 0, cidx(g, i, j), cidx(g, i + 1, j), S, S + 4, amax));
#pragma unroll
      for (int k = 0; k < 8; k++) ft.sx[k][b][a] = S[k];
#pragma unroll
      for (int k = 0; k < 4; k++) ft.dx[k][b][a] = widen_f(S[k]);
    }
  }
  if (t < FR_TX * (FR_TY + 1)) {
    const int a = t % FR_TX, b = t / FR_TX;
    const int i = i0 + a, j = j0 - 1 + b;
    if (i < g.nx && j < g.ny) {
      float S[8];
      bmax = fmaxf(bmax, face_sums_mixed(g, f, 1, cidx(g, i, j), cidx(g, i, j + 1), S, S + 4, amax));
#pragma unroll
      for (int k = 0; k < 8; k++) ft.sy[k][b][a] = S[k];
#pragma unroll
      for (int k = 0; k < 4; k++) ft.dy[k][b][a] = widen_f(S[k]);
    }
  }
}

// thread t's cell of the tile: its balances from the tile's face sums into r (false for
// a thread without a cell); *bad gets FLAG_NONFINITE for a non-finite balance
__device__ __forceinline__ bool flux_tile_balance(const Grid& g, const WorkF& f, int i0, int j0, int t,
                                                  const FluxTile& ft, long long& c, double* r0, float* rm,
                                                  unsigned int* bad) {
  if (t >= FR_TX * FR_TY) return false;
  const int a = t % FR_TX, b = t / FR_TX;
  const int i = i0 + a, j = j0 + b;
  if (i >= g.nx || j >= g.ny) return false;
  float sR[8], sL[8], tT[8], tB[8];
  double dR[4], dL[4], dT[4], dB[4];
#pragma unroll
  for (int k = 0; k < 8; k++) {
    sR[k] = ft.sx[k][b][a + 1];
    sL[k] = ft.sx[k][b][a];
    tT[k] = ft.sy[k][b + 1][a];
    tB[k] = ft.sy[k][b][a];
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    dR[k] = ft.dx[k][b][a + 1];
    dL[k] = ft.dx[k][b][a];
    dT[k] = ft.dy[k][b + 1][a];
    dB[k] = ft.dy[k][b][a];
  }
  c = cidx(g, i, j);
  *bad |= balance_mixed(g, f, c, sR, sL, tT, tB, dR, dL, dT, dB, r0, rm);
  return true;
}

// thread t's cell of the tile: its balances from the tile's face sums and its stage
// update; returns the flags, and (KEF) the kinetic share at stage 3 in kef
template <bool KEF>
__device__ __forceinline__ unsigned int flux_tile_cell(const Grid& g, const WorkF& f, int i0, int j0, int t,
                                                       const FluxTile& ft, int stage, double dt,
                                                       const double* __restrict__ qin, const double* __restrict__ mom,
                                                       double* __restrict__ base, double* __restrict__ qout,
                                                       float* __restrict__ hilo, double& kef) {
  long long c = 0;
  double r0[4];
  float rm[8];
  unsigned int bad = 0;
  if (!flux_tile_balance(g, f, i0, j0, t, ft, c, r0, rm, &bad)) return 0;
  bad |= rk_cell_mixed<KEF>(g, stage, c, dt, qin, mom, r0, rm, base, qout, hilo, kef);
  return bad;
}

// the tile's alpha* and beta_max contributions into the reductions
__device__ __forceinline__ void flux_tile_reduce(float amax, float bmax, Diag* diag) {
  amax = warp_max(amax);
  bmax = warp_max(bmax);
  if (lane_id() == 0) {
    atomic_max_pos(&diag->alpha_bits, (double)amax);
    atomic_max_pos(&diag->beta_bits, (double)bmax);
  }
}

// Eqs. (3.3) and (3.2) of the mixed path, for a residual that is kept (stage 1 of a
// step, whose step size needs alpha* over every face first and whose residual serves
// the restarts; hweno_residual): the tile's face sums in shared memory, then the
// balances of its cells into rhs.  The arithmetic is that of k_flux_rk_mixed's first
// part.
__global__ void __launch_bounds__(FR_THREADS, HWENO_FR_MIN_BLOCKS) k_flux_asm_mixed(Grid g, Work w, double* __restrict__ rhs, Diag* diag) {
  __shared__ FluxTile ft;
  const WorkF f = mixed_planes(w, g.ps);
  const int i0 = blockIdx.x * FR_TX, j0 = blockIdx.y * FR_TY, t = threadIdx.x;
  float amax = 0.f, bmax = 0.f;
  flux_tile_faces(g, f, i0, j0, t, ft, amax, bmax);
  flux_tile_reduce(amax, bmax, diag);
  __syncthreads();
  long long c = 0;
  double r0[4];
  float rm[8];
  unsigned int bad = 0;
  if (flux_tile_balance(g, f, i0, j0, t, ft, c, r0, rm, &bad)) store_residual_mixed(g, c, r0, rm, rhs);
  bad = __reduce_or_sync(0xffffffffu, bad);
  if (lane_id() == 0 && bad) atomicOr(&diag->flags, bad);
}

__global__ void __launch_bounds__(FR_THREADS, HWENO_FR_MIN_BLOCKS) k_flux_rk_mixed(Grid g, Work w, int stage, const double* __restrict__ qin,
                                                               const double* __restrict__ mom, double* __restrict__ base,
                                                               double* __restrict__ qout, Diag* diag,
                                                               float* __restrict__ hilo) {
  __shared__ FluxTile ft;
  const WorkF f = mixed_planes(w, g.ps);
  const int i0 = blockIdx.x * FR_TX, j0 = blockIdx.y * FR_TY, t = threadIdx.x;
  float amax = 0.f, bmax = 0.f;
  flux_tile_faces(g, f, i0, j0, t, ft, amax, bmax);
  flux_tile_reduce(amax, bmax, diag);
  __syncthreads();
  double kef = 0.0;
  const unsigned int bad = flux_tile_cell<true>(g, f, i0, j0, t, ft, stage, diag->dt, qin, mom, base, qout, hilo,
                                                kef);
  rk_reduce<true>(stage, bad, kef, diag);
}

// float planes back to a contiguous double array (debug output of the mixed path)
__global__ void k_gather_f(Grid g, int n, const float* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * N;
       t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / N, r = t % N;
    const int jj = (int)(r / g.nx), ii = (int)(r % g.nx);
    dst[t] = (double)src[p * g.ps + cidx(g, ii, jj)];
  }
}
__global__ void k_gather_cons_f(Grid g, const float* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)g.nx * g.ny;
  for (long long r = blockIdx.x * (long long)blockDim.x + threadIdx.x; r < N;
       r += (long long)gridDim.x * blockDim.x) {
    const int jj = (int)(r / g.nx), ii = (int)(r % g.nx);
    const long long c = cidx(g, ii, jj);
    const double rho = src[c], u = src[g.ps + c], v = src[2 * g.ps + c], e = src[3 * g.ps + c];
    dst[r] = rho;
    dst[N + r] = rho * u;
    dst[2 * N + r] = rho * v;
    dst[3 * N + r] = rho * (e + 0.5 * (u * u + v * v));
  }
}

// single-grid kernels of the mixed path
// 3 blocks of 128 per SM (168 registers): with the coefficients in shared memory the
// extra resident warps hide more latency than the few remaining spills cost
__global__ void __launch_bounds__(128, 3) k_cons_mixed(Grid g, const double* __restrict__ q, Work w,
                                                    double* __restrict__ mom, Diag* diag) {
  cons_mixed_body(g, q, w, mom, diag, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}
__global__ void k_face_moments_mixed(Grid g, Work w) {
  face_moments_mixed_body(g, w, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y,
                          blockIdx.z);
}
__global__ void k_weak_moments_mixed(Grid g, Work w) {
  weak_moments_mixed_body(g, w, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}
template <bool LIN = false, bool VOLG = false>
__global__ void __launch_bounds__(128) k_grad_mixed(Grid g, Work w) {
  grad_mixed_body<LIN, VOLG>(g, w, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}

}  // namespace hw
