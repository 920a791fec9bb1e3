// Kernels of the HWENO-GR spatial operator and the SSP-RK3 stage update.
//
// Data layout in HBM (all planes FP64, structure of arrays):
//   padded plane: (ny + 8) rows x pitch doubles, pitch = nx + 8 rounded up to a
//   multiple of 16 (128-byte rows); cell (i, j), i in [-4, nx+4), j in [-4, ny+4),
//   sits at (j + 4) * pitch + (i + 4).  A "plane set" of n planes is n consecutive
//   planes of plane_stride doubles.
//
// One spatial-operator evaluation runs these kernels in order (regions in cells):
//   ghost_x / ghost_y   fill the 4 ghost layers of the 12 state planes (Remark 4.1)
//   k_cons              characteristic HWENO traces + limiter on the interior grown by 3
//   k_face_moments      face moments W^{x,0}, W^{x,1}, W^{y,0}, W^{y,1} (Eq. (3.6))
//   k_weak_moments      weak-derivative moments r (Eqs. (3.7)-(3.8)) on interior + 2
//   k_grad              gradient HWENO (Eq. (3.9)) on interior + 1
//   (HWENO-DR instead: k_cons_dr also stores the characteristic combinations, and
//    k_dr differentiates them on interior + 1 in place of the three kernels above)
//   k_flux              PP-LLF face fluxes (Eq. (3.3)) of the interior faces
//   k_assemble          moment balances Eq. (3.2) on the interior
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "hweno_device.cuh"

namespace hw {

constexpr int NG = 4;  // ghost layers

struct Grid {
  int nx, ny, pitch;
  long long ps;  // plane stride in doubles
  double dx, dy;
  double gamma, Pr, Re;
  double eps_pp, eps_weno;
  int bc[4];
  double rdx, rdy, rPr, rRe;  // 1/dx, 1/dy, 1/Pr, 1/Re (correctly rounded, on the host)
  double x0, y0;              // domain origin (coordinates of a source term)
};

// x is neither infinite nor NaN: an exponent-field test in the integer pipe
__device__ __forceinline__ bool finite_d(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}
__device__ __forceinline__ bool finite_f(float x) { return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u; }

// hi/lo split of the 12 ghost-filled state planes (whole padded planes), with integer
// operations only: hi keeps the sign, the exponent and the leading 23 mantissa bits of
// x (truncation), lo is the float nearest below the exact remainder x - hi (the trailing
// 29 mantissa bits, normalised).  Zero gives (0, 0); magnitudes below 2^-74 or beyond
// the float range take hi = fl(x), lo = 0.
__device__ __forceinline__ void split_hilo(double x, float& hi, float& lo) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7ff);
  const int fe = E - 1023 + 127;
  if (E == 0) {  // zero (or a double denormal, below any float): signed zero
    hi = __int_as_float((int)sign);
    lo = 0.0f;
    return;
  }
  // the remainder's float exponent field is fe - 52 + top >= fe - 52: keep it >= 1
  if (fe < 53 || fe > 254) {  // |x| < 2^-74, beyond the float range, inf or nan
    hi = (float)x;
    lo = 0.0f;
    return;
  }
  const unsigned long long m = b & 0xfffffffffffffull;
  hi = __int_as_float((int)(sign | ((unsigned int)fe << 23) | (unsigned int)(m >> 29)));
  const unsigned int r = (unsigned int)(m & 0x1fffffffull);  // remainder: r * 2^(E - 1075)
  if (r == 0u) {
    lo = 0.0f;
    return;
  }
  const int top = 31 - __clz((int)r);          // highest set bit, 0..28
  const int le = fe - 52 + top;                 // float exponent field of the remainder
  const unsigned int mant = top >= 23 ? (r >> (top - 23)) : (r << (23 - top));
  lo = __int_as_float((int)(sign | ((unsigned int)le << 23) | (mant & 0x7fffffu)));
}

__device__ __forceinline__ long long cidx(const Grid& g, int i, int j) {
  return (long long)(j + NG) * g.pitch + (i + NG);
}

constexpr int YREC_CC = 144, YREC_GR = 204, YREC_PLANES = 306;

// scratch planes of one spatial-operator evaluation
struct Work {
  double* face;   // 48 planes: point k (0..11) x (rho, u, v, e), limited
  double* vol;    // 36 planes: point k (0..8) x (rho, u, v, e), unlimited
  double* wbar;   // 3 planes: cell means of u, v, e (Eq. (3.8))
  double* wx;     // 6 planes at the x-face right of a cell: W^{x,0}(u,v,e), W^{x,1}(u,v,e)
  double* wy;     // 6 planes at the y-face above a cell
  double* rm;     // 18 planes: 6*w + (x0, x_xi, x_eta, y0, y_xi, y_eta)
  double* gr;     // 126 planes: point k (0..20) x (u_x, u_y, v_x, v_y, e_x, e_y)
  double* fx;     // x-face right of a cell: planes 0-3 S0 = sum_g w_g fhat_g, 4-7
                  // S1 = sum_g w_g eta_g fhat_g, per conserved variable (12 allocated)
  double* fy;     // y-face above a cell: the same with xi_g
  double* theta;  // 2 planes: limiter factors
  // YREC_PLANES planes, only while a step is recorded for the adjoint (else null):
  //   72 d + 18 f + slot  per direction d and field f of the characteristic
  //       reconstruction: slots 0-5 the face values, 6-14 the volume values, 15 the
  //       moment (characteristic variables), 16 beta_0 and 17 1/S' of the weights;
  //   YREC_CC + 15 v + k  the p0 coefficients of conserved variable v;
  //   YREC_GR + 17 m + k  gradient component m: k < 15 its p0 coefficients, 15 beta_0,
  //       16 1/S'
  double* yrec = nullptr;
  // 120 planes, HWENO-DR only (else null): 60 d + 15 f + k, coefficient k of the
  // nonlinear combination of characteristic field f of direction d's reconstruction
  // (absolute values), for cells of the interior grown by 1
  double* dr = nullptr;
};

// device-side reductions and flags of one evaluation / step
struct Diag {
  unsigned long long alpha_bits;  // max of non-negative doubles via their bit patterns
  unsigned long long beta_bits;
  unsigned long long pp_count;    // limiter activations (interior cells)
  unsigned int flags;             // bit 0: stage output inadmissible, bit 1: nonfinite rhs,
                                  // bit 2: inadmissible cell average met by the limiter
  unsigned int pad;
  double dt;                      // time step of the current step
};

enum { FLAG_INADMISSIBLE = 1u, FLAG_NONFINITE = 2u, FLAG_BADAVG = 4u };

__device__ __forceinline__ void atomic_max_pos(unsigned long long* a, double v) {
  // ordering of non-negative IEEE doubles equals the ordering of their bit patterns;
  // NaN patterns sort above +inf and therefore surface in the maximum
  atomicMax(a, (unsigned long long)__double_as_longlong(v));
}

template <class T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------------------
// ghost cells (Remark 4.1).  x pass over the interior rows, then y pass over the
// full padded width, so corners take the product of the two parities.
// Mirror across a face with parity s per variable: ghost average = s * average,
// moment normal to the face = -s * moment, tangential moment = s * moment.
__device__ __forceinline__ double bc_sign(int bc, int normal_dir, int v) {
  if (v == 0 || v == 3) return 1.0;
  if (bc == 1) return -1.0;                 // no-slip: both momenta odd
  return (v == 1 + normal_dir) ? -1.0 : 1.0;  // symmetry/slip: normal momentum odd
}

// planes [p0, p1) of the state (plane 4 m + v: moment m of variable v), or of its
// hi/lo split (24 float planes: plane p holds state plane p mod 12)
template <class E>
__device__ __forceinline__ void ghost_x_body(const Grid& g, E* q, int t, int p0 = 0, int p1 = 12) {
  // t over 8 ghost columns x ny rows
  if (t >= 8 * g.ny) return;
  const int j = t / 8, c = t % 8;
  const int side = c / 4, k = c % 4;  // side 0: i = -1-k, side 1: i = nx+k
  const int i = side == 0 ? -1 - k : g.nx + k;
  const int bc = g.bc[side];
  int src;
  if (bc == 0) src = side == 0 ? ((i % g.nx) + g.nx) % g.nx : i % g.nx;
  else src = side == 0 ? -1 - i : 2 * g.nx - 1 - i;
  const long long d = cidx(g, i, j), s = cidx(g, src, j);
  for (int p = p0; p < p1; p++) {
    const int m = (p % 12) >> 2, v = p & 3;
    E sg = E(1);
    if (bc != 0) sg = E(bc_sign(bc, 0, v) * (m == 1 ? -1.0 : 1.0));
    q[p * g.ps + d] = sg * q[p * g.ps + s];
  }
}

template <class E>
__device__ __forceinline__ void ghost_y_body(const Grid& g, E* q, int t, int p0 = 0, int p1 = 12) {
  // t over 8 ghost rows x padded width
  const int W = g.nx + 2 * NG;
  if (t >= 8 * W) return;
  const int r = t / W, i = t % W - NG;
  const int side = r / 4, k = r % 4;
  const int j = side == 0 ? -1 - k : g.ny + k;
  const int bc = g.bc[2 + side];
  int src;
  if (bc == 0) src = side == 0 ? ((j % g.ny) + g.ny) % g.ny : j % g.ny;
  else src = side == 0 ? -1 - j : 2 * g.ny - 1 - j;
  const long long d = cidx(g, i, j), s = cidx(g, i, src);
  for (int p = p0; p < p1; p++) {
    const int m = (p % 12) >> 2, v = p & 3;
    E sg = E(1);
    if (bc != 0) sg = E(bc_sign(bc, 1, v) * (m == 2 ? -1.0 : 1.0));
    q[p * g.ps + d] = sg * q[p * g.ps + s];
  }
}

// one plane per blockIdx.y: 12 x the threads of a cell-wise loop over the planes;
// with hilo, blockIdx.y = 12..35 fills the 24 planes of the state's hi/lo split too
__global__ void k_ghost_x(Grid g, double* q, float* hilo) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
  if (p < 12) ghost_x_body(g, q, t, p, p + 1);
  else ghost_x_body(g, hilo, t, p - 12, p - 11);
}
__global__ void k_ghost_y(Grid g, double* q, float* hilo) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
  if (p < 12) ghost_y_body(g, q, t, p, p + 1);
  else ghost_y_body(g, hilo, t, p - 12, p - 11);
}

// ---------------------------------------------------------------------------
// gather the 17 data of one conserved variable (plane offset v) around (i, j) in the
// order of hweno_stencil.h; with OFF the averages are taken relative to the centre
// average (so d[4] == 0), which keeps the FP32 reconstruction accurate
template <bool OFF>
__device__ __forceinline__ void gather17(const Grid& g, const double* q, int v, int i, int j,
                                         double* d) {
  const double* A = q + (long long)v * g.ps;
  const double* X = q + (long long)(4 + v) * g.ps;
  const double* Y = q + (long long)(8 + v) * g.ps;
  const double c = OFF ? A[cidx(g, i, j)] : 0.0;
#pragma unroll
  for (int b = -1; b <= 1; b++)
#pragma unroll
    for (int a = -1; a <= 1; a++) d[(b + 1) * 3 + (a + 1)] = A[cidx(g, i + a, j + b)] - c;
  if (OFF) d[4] = 0.0;
  d[9] = X[cidx(g, i - 1, j)];
  d[10] = X[cidx(g, i + 1, j)];
  d[11] = Y[cidx(g, i, j - 1)];
  d[12] = Y[cidx(g, i, j + 1)];
  d[13] = X[cidx(g, i, j - 1)];
  d[14] = X[cidx(g, i, j + 1)];
  d[15] = Y[cidx(g, i - 1, j)];
  d[16] = Y[cidx(g, i + 1, j)];
}

// characteristic reconstruction of one direction: per field, project the conserved
// p0 coefficients, slopes and centre average (p0 is linear in the data, so these are
// the coefficients of the projected data), form the nonlinear combination, evaluate
// it at this direction's 6 face points, the 9 volume points and the moment, and
// transform back.  cc, sl, ctr hold absolute values (FP64) or offsets from the centre
// average (FP32, ctr = 0); the outputs are in the same representation (moments are
// unaffected by the offset).
// the p0 coefficients of the 4 conserved variables, cc(v, k): held in registers, or in
// this thread's slot of a shared-memory array [60][128] (blocks of 128 threads)
template <class T>
struct CoefRegs {
  const T (*c)[15];
  __device__ __forceinline__ T operator()(int v, int k) const { return c[v][k]; }
};
template <class T>
struct CoefShared {
  const T* p;  // &smem[0][thread]
  __device__ __forceinline__ T operator()(int v, int k) const { return p[(15 * v + k) * 128]; }
};

// REC (FP64): also store this direction's characteristic point values and weight
// factors of every field at yr[(18 f + slot) * yps] (the Work::yrec layout).
// dw (HWENO-DR, FP64): also store each field's combination coefficients at
// dw[(15 f + k) * yps] (the Work::dr layout).
template <class T, int DIR, class O, bool REC = false, class CC>
__device__ __forceinline__ void recon_dir(const CC& cc, const T (*sl)[4], const T* ctr,
                                          const CharState<T>& cs, T eps, O (*face)[4], O (*vol)[4],
                                          O* mom, double* yr = nullptr, long long yps = 0,
                                          double* dw = nullptr) {
  T chf[4][6], chv[4][9], chm[4];
  T pc[15][4], ps[4][4], pz[4];
#pragma unroll
  for (int k = 0; k < 15; k++) {
    const T x[4] = {cc(0, k), cc(1, k), cc(2, k), cc(3, k)};
    to_char<T, DIR>(cs, x, pc[k]);
  }
#pragma unroll
  for (int k = 0; k < 4; k++) {
    const T x[4] = {sl[0][k], sl[1][k], sl[2][k], sl[3][k]};
    to_char<T, DIR>(cs, x, ps[k]);
  }
  to_char<T, DIR>(cs, ctr, pz);
#pragma unroll
  for (int f = 0; f < 4; f++) {
    T c0[15], s[4], C[15];
#pragma unroll
    for (int k = 0; k < 15; k++) c0[k] = pc[k][f];
#pragma unroll
    for (int k = 0; k < 4; k++) s[k] = ps[k][f];
    T wr[2];
    hweno_combine_coeffs<T, REC>(c0, s, pz[f], eps, C, wr);
    if (dw) {
#pragma unroll
      for (int k = 0; k < 15; k++) dw[(long long)(15 * f + k) * yps] = (double)C[k];
    }
    if (DIR == 0) eval_xfaces<T>(C, chf[f]); else eval_yfaces<T>(C, chf[f]);
    eval_vol<T>(C, chv[f]);
    chm[f] = DIR == 0 ? hw_moment_xi<T>(C) : hw_moment_eta<T>(C);
    if constexpr (REC) {
      double* y = yr + (long long)(18 * f) * yps;
#pragma unroll
      for (int k = 0; k < 6; k++) y[k * yps] = chf[f][k];
#pragma unroll
      for (int k = 0; k < 9; k++) y[(6 + k) * yps] = chv[f][k];
      y[15 * yps] = chm[f];
      y[16 * yps] = wr[0];
      y[17 * yps] = wr[1];
    }
  }
#pragma unroll
  for (int k = 0; k < 6; k++) {
    const T y[4] = {chf[0][k], chf[1][k], chf[2][k], chf[3][k]};
    T x[4];
    from_char<T, DIR>(cs, y, x);
#pragma unroll
    for (int v = 0; v < 4; v++) face[k][v] = (O)x[v];
  }
#pragma unroll
  for (int k = 0; k < 9; k++) {
    const T y[4] = {chv[0][k], chv[1][k], chv[2][k], chv[3][k]};
    T x[4];
    from_char<T, DIR>(cs, y, x);
#pragma unroll
    for (int v = 0; v < 4; v++) vol[k][v] = (O)x[v];
  }
  {
    T x[4];
    from_char<T, DIR>(cs, chm, x);
#pragma unroll
    for (int v = 0; v < 4; v++) mom[v] = (O)x[v];
  }
}

}  // namespace hw
