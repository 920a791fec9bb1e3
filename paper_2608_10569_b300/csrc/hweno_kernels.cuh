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
#include "hweno_state.cuh"

namespace hw {

// x is neither infinite nor NaN: an exponent-field test in the integer pipe
__device__ __forceinline__ bool finite_d(double x) {
  return ((unsigned)__double2hiint(x) & 0x7ff00000u) != 0x7ff00000u;
}
__device__ __forceinline__ bool finite_f(float x) { return (__float_as_uint(x) & 0x7f800000u) != 0x7f800000u; }

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
  unsigned long long kefrac_bits; // mixed handles: max over cells of the kinetic share
                                  // |m|^2 / (2 rho E) of the stage-3 state, as the bits of a
                                  // double in [0, 1] (1 where that state is inadmissible)
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

// one plane per blockIdx.y: 12 x the threads of a cell-wise loop over the planes;
// with hilo, blockIdx.y = 12..27 fills the 16 planes of the state's hi/lo split that are
// kept (the 12 hi planes and the averages' 4 lo planes; the moments' lo parts are 0)
constexpr int HILO_KEPT = 16;
// both ghost passes in one launch (ghost_xy_body): threads 0 .. 8 ny - 1 the x ghosts,
// the next 8 (nx + 8) the y ghosts
__global__ void k_ghost(Grid g, const __grid_constant__ Open o, double* q, float* hilo) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x, p = blockIdx.y;
  if (p < 12) ghost_xy_body(g, &o, q, t, p, p + 1);
  else ghost_xy_body(g, &o, hilo, t, p - 12, p - 11);
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
