// The 2D spatial operator of the CUDA path, run on the host (test infrastructure): the
// kernels' own bodies (hweno_state.cuh, hweno_ops.cuh, hweno_mixed.cuh,
// hweno_source.cuh), each called over the index range of its launch, in the operator's
// order.  Every plane set is an allocation of its own, so that an access past one shows
// under AddressSanitizer; a NaN fill (NaN as a double and as either float half) makes a
// read of a value that no earlier kernel wrote reach the output.
#pragma once
#include "shim.h"
#include <algorithm>
#include <vector>
#include "hweno_mixed.cuh"
#include "hweno_source.cuh"
#include "hweno_tma.cuh"

namespace hw {
double cons_smem[CONS_SMEM_BYTES / sizeof(double)];
double dr_smem[DR_SMEM_BYTES / sizeof(double)];
}  // namespace hw

namespace host2d {
using namespace hw;

inline double nan_fill() {
  const unsigned long long b = 0x7FF800007FC00000ull;  // high half 0x7FF80000, low 0x7FC00000
  double f;
  memcpy(&f, &b, sizeof(f));
  return f;
}

// the scratch planes of one evaluation, one allocation per plane set
struct Scratch {
  std::vector<double> face, vol, wbar, wx, wy, rm, gr, fx, fy, theta, dr;
  Work w;
  Scratch(const Grid& g, int scheme, double fill) {
    auto planes = [&](int k) { return std::vector<double>((size_t)k * g.ps, fill); };
    face = planes(48); vol = planes(36); wbar = planes(3); wx = planes(6); wy = planes(6);
    rm = planes(18); gr = planes(126); fx = planes(12); fy = planes(12); theta = planes(2);
    dr = planes(scheme == HWENO_SCHEME_DR ? 120 : 0);
    w.face = face.data(); w.vol = vol.data(); w.wbar = wbar.data(); w.wx = wx.data(); w.wy = wy.data();
    w.rm = rm.data(); w.gr = gr.data(); w.fx = fx.data(); w.fy = fy.data(); w.theta = theta.data();
    w.yrec = nullptr;
    w.dr = scheme == HWENO_SCHEME_DR ? dr.data() : nullptr;
  }
};

// k_grad_tma_mixed on the host: per tile, the two boxes the tensor copies bring into
// shared memory (copied here from the float planes, zero outside them, as the copies
// fill), then the weak moments of the grown tile and the gradients of the tile's cells
inline void grad_tma_emulated(const hweno_config& c, const Grid& g, const Work& w) {
  const WorkF f = mixed_planes(w, g.ps);
  const long long rows = g.ny + 2 * NG;
  std::vector<float> sm(GT_TR_FLOATS + GT_WB_FLOATS + GT_R_FLOATS);
  const int ntx = (g.nx + 2 + GT_X - 1) / GT_X, nty = (g.ny + 2 + GT_Y - 1) / GT_Y;
  for (int by = 0; by < nty; by++)
    for (int bx = 0; bx < ntx; bx++) {
      const int a = -1 + GT_X * bx, b = -1 + GT_Y * by;
      const long long x0 = GT_X * bx, y0 = b - 2 + NG;
      memset(sm.data(), 0xFF, sm.size() * sizeof(float));  // shared memory starts undefined: NaN
      auto fetch = [&](const float* plane, long long y, long long x) {
        return (x < g.pitch && y < rows) ? plane[y * g.pitch + x] : 0.0f;
      };
      for (int k = 0; k < 12; k++)
        for (int n = 0; n < 3; n++)
          for (int y = 0; y < GB_Y; y++)
            for (int x = 0; x < GB_X; x++)
              sm[((k * 3 + n) * GB_Y + y) * GB_X + x] = fetch(f.face + (long long)(4 * k + 1 + n) * g.ps, y0 + y, x0 + x);
      for (int n = 0; n < 3; n++)
        for (int y = 0; y < GB_Y; y++)
          for (int x = 0; x < GB_X; x++)
            sm[GT_TR_FLOATS + (n * GB_Y + y) * GB_X + x] = fetch(f.wbar + (long long)n * g.ps, y0 + y, x0 + x);
      GradTile tt{sm.data(), sm.data() + GT_TR_FLOATS, sm.data() + GT_TR_FLOATS + GT_WB_FLOATS};
      for (int k = 0; k < GR_X * GR_Y; k++) gradtile_weak_cell(g, tt, k % GR_X, k / GR_X);
      for (int t = 0; t < GT_THREADS; t++) {
        const int tx = t % GT_X, ty = t / GT_X, i = a + tx, j = b + ty;
        // the kernel forms the volume weights (and the inviscid sums) while its copies fly
        float wu[9], wv[9];
        if (i >= 0 && i < g.nx && j >= 0 && j < g.ny) vol_weights(g, f, cidx(g, i, j), wu, wv);
        if (i < g.nx + 1 && j < g.ny + 1) {
          if (c.linear_grad) gradtile_grad_cell<true>(g, w, tt, tx, ty, i, j, wu, wv);
          else gradtile_grad_cell<false>(g, w, tt, tx, ty, i, j, wu, wv);
        }
      }
    }
}

// the mixed path up to the gradients at state q (ghost cells already filled): the split
// of the ghost-filled state (k_split), traces, face and weak moments, gradients (tma: as
// k_grad_tma_mixed forms the last three)
inline void mixed_front(const hweno_config& c, const Grid& g, Scratch& s, double* q, double* mom, Diag* diag,
                        bool tma = false) {
  const int nx = g.nx, ny = g.ny;
  Work& w = s.w;
  float* hilo = mixed_planes(w, g.ps).hilo;
  const long long np = 12 * g.ps;
  for (long long k = 0; k < np; k++) {  // as k_split: the moments' lo planes stay unwritten
    float hi, lo;
    split_hilo(q[k], hi, lo);
    hilo[k] = hi;
    if (k < 4 * g.ps) hilo[np + k] = lo;
  }
  for (int gy = 0; gy < ny + 6; gy++)
    for (int gx = 0; gx < nx + 6; gx++) cons_mixed_body(g, q, w, mom, diag, gx, gy);
  if (tma) {
    grad_tma_emulated(c, g, w);
    return;
  }
  for (int gz = 0; gz < 2; gz++)
    for (int gy = 0; gy < ny + 5; gy++)
      for (int gx = 0; gx < nx + 5; gx++) face_moments_mixed_body(g, w, gx, gy, gz);
  for (int gy = 0; gy < ny + 4; gy++)
    for (int gx = 0; gx < nx + 4; gx++) weak_moments_mixed_body(g, w, gx, gy);
  for (int gy = 0; gy < ny + 2; gy++)
    for (int gx = 0; gx < nx + 2; gx++) {
      if (c.linear_grad) grad_mixed_body<true>(g, w, gx, gy);
      else grad_mixed_body(g, w, gx, gy);
    }
}

// stage 2 or 3 of a mixed step as k_flux_rk_mixed runs it: the front at q (ghosts filled
// here), then per tile the face sums of every thread of the block, then every thread's
// cell (the barrier between the two phases)
inline void fused_stage(const hweno_config& c, const Grid& g, const Open& o, Scratch& s, double* q, double* mom,
                        double* base, double* qout, int stage, Diag* diag, bool tma) {
  for (int k = 0; k < 8 * g.ny + 8 * (g.nx + 2 * NG); k++) ghost_xy_body(g, &o, q, k);  // k_ghost
  mixed_front(c, g, s, q, mom, diag, tma);
  const WorkF f = mixed_planes(s.w, g.ps);
  std::vector<float> hilo_out(24 * (size_t)g.ps);
  static FluxTile ft;
  for (int j0 = 0; j0 < g.ny; j0 += FR_TY)
    for (int i0 = 0; i0 < g.nx; i0 += FR_TX) {
      float amax = 0.f, bmax = 0.f;
      memset(&ft, 0xFF, sizeof(ft));  // shared memory starts undefined: NaN
      for (int t = 0; t < FR_THREADS; t++) flux_tile_faces(g, f, i0, j0, t, ft, amax, bmax);
      for (int t = 0; t < FR_THREADS; t++) {
        double kef = 0.0;
        diag->flags |= flux_tile_cell<true>(g, f, i0, j0, t, ft, stage, diag->dt, q, mom, base, qout, hilo_out.data(),
                                            kef);
      }
    }
}

// the mixed path's fluxes and balances as k_flux_asm_mixed runs them: per tile, every
// thread's faces, then every thread's cell, into rhs
inline void flux_asm_tiles(const Grid& g, Scratch& s, double* rhs, Diag* diag) {
  const WorkF f = mixed_planes(s.w, g.ps);
  static FluxTile ft;
  for (int j0 = 0; j0 < g.ny; j0 += FR_TY)
    for (int i0 = 0; i0 < g.nx; i0 += FR_TX) {
      float amax = 0.f, bmax = 0.f;
      memset(&ft, 0xFF, sizeof(ft));  // shared memory starts undefined: NaN
      for (int t = 0; t < FR_THREADS; t++) flux_tile_faces(g, f, i0, j0, t, ft, amax, bmax);
      double a = amax, b = bmax;
      diag->alpha_bits = std::max(diag->alpha_bits, (unsigned long long)__double_as_longlong(a));
      diag->beta_bits = std::max(diag->beta_bits, (unsigned long long)__double_as_longlong(b));
      for (int t = 0; t < FR_THREADS; t++) {
        long long c = 0;
        double r0[4];
        float rm[8];
        unsigned int bad = 0;
        if (flux_tile_balance(g, f, i0, j0, t, ft, c, r0, rm, &bad)) store_residual_mixed(g, c, r0, rm, rhs);
        diag->flags |= bad;
      }
    }
}

// one evaluation at state q (12 padded planes, ghosts filled here): rhs (12) and the
// modified moments mom (8); the source term, when configured, at time t; tiles: the mixed
// path's fluxes and balances as its tile kernel runs them
inline void residual(const hweno_config& c, const Grid& g, const Open& o, const Quad4& quad, Scratch& s,
                     double* q, double* rhs, double* mom, Diag* diag, double t, bool mixed, bool tma = false,
                     bool tiles = false) {
  const int nx = g.nx, ny = g.ny;
  Work& w = s.w;
  for (int k = 0; k < 8 * ny + 8 * (nx + 2 * NG); k++) ghost_xy_body(g, &o, q, k);  // k_ghost
  if (mixed && tiles) {
    mixed_front(c, g, s, q, mom, diag, tma);
    flux_asm_tiles(g, s, rhs, diag);
  } else if (mixed) {
    mixed_front(c, g, s, q, mom, diag, tma);
    for (int gz = 0; gz < 2; gz++)
      for (int gy = 0; gy < ny + 1; gy++)
        for (int gx = 0; gx < nx + 1; gx++) flux_mixed_body(g, w, diag, gx, gy, gz);
    for (int gy = 0; gy < ny; gy++)
      for (int gx = 0; gx < nx; gx++) assemble_mixed_body(g, w, rhs, diag, gx, gy);
  } else {
    const bool drs = c.scheme == HWENO_SCHEME_DR;
    for (int gy = 0; gy < ny + 6; gy++)
      for (int gx = 0; gx < nx + 6; gx++) {
        if (drs) cons_body<double, false, true>(g, q, w, mom, diag, gx, gy);
        else cons_body<double>(g, q, w, mom, diag, gx, gy);
      }
    if (drs) {
      for (int gy = 0; gy < ny + 2; gy++)
        for (int gx = 0; gx < nx + 2; gx++) dr_body(g, q, w, gx, gy);
    } else {
      for (int gz = 0; gz < 2; gz++)
        for (int gy = 0; gy < ny + 5; gy++)
          for (int gx = 0; gx < nx + 5; gx++) face_moments_body(g, w, gx, gy, gz);
      for (int gy = 0; gy < ny + 4; gy++)
        for (int gx = 0; gx < nx + 4; gx++) weak_moments_body(g, w, gx, gy);
      for (int gy = 0; gy < ny + 2; gy++)
        for (int gx = 0; gx < nx + 2; gx++) {
          if (c.linear_grad) grad_body<double, false, true>(g, w, gx, gy);
          else grad_body<double>(g, w, gx, gy);
        }
    }
    for (int gz = 0; gz < 2; gz++)
      for (int gy = 0; gy < ny + 1; gy++)
        for (int gx = 0; gx < nx + 1; gx++) flux_body<double>(g, w, diag, gx, gy, gz);
    for (int gy = 0; gy < ny; gy++)
      for (int gx = 0; gx < nx; gx++) assemble_body<double>(g, w, rhs, diag, gx, gy);
  }
  if (c.source == HWENO_SOURCE_MMS52)
    for (int gy = 0; gy < ny; gy++)
      for (int gx = 0; gx < nx; gx++) source_body(g, quad, t, 0.0, diag, rhs, gx, gy);
}

// the configuration record of the harnesses' input files: 11 ints (nx, ny, bc[4], scheme,
// source, linear_grad, nan_fill, mixed: 0 FP64, 1 mixed, 2 mixed with stages 2 and 3 fused, 3 that and the
// TMA-staged gradients), 50 doubles (x0, x1, y0, y1, gamma, Pr, Re,
// eps_pp, eps_weno, t, inflow[4][2][4], band[4][2])
struct Input {
  hweno_config c;
  bool nan_fill, mixed, fused;  // fused: the mixed path with stages 2 and 3 fused
  bool tma;                     // the mixed path's gradients as k_grad_tma_mixed forms them
  double t;
};
inline bool read_input(FILE* f, Input& in) {
  int hi[11];
  double hd[50];
  if (fread(hi, sizeof(int), 11, f) != 11 || fread(hd, sizeof(double), 50, f) != 50) return false;
  hweno_config& c = in.c;
  memset(&c, 0, sizeof(c));
  c.nx = hi[0];
  c.ny = hi[1];
  for (int k = 0; k < 4; k++) c.bc[k] = hi[2 + k];
  c.scheme = hi[6];
  c.source = hi[7];
  c.linear_grad = hi[8];
  in.nan_fill = hi[9] != 0;
  in.mixed = hi[10] != 0;
  in.fused = hi[10] >= 2;
  in.tma = hi[10] == 3;
  c.x0 = hd[0]; c.x1 = hd[1]; c.y0 = hd[2]; c.y1 = hd[3];
  c.gamma = hd[4]; c.Pr = hd[5]; c.Re = hd[6]; c.eps_pp = hd[7]; c.eps_weno = hd[8];
  in.t = hd[9];
  memcpy(c.inflow, hd + 10, sizeof(c.inflow));
  memcpy(c.band, hd + 42, sizeof(c.band));
  return true;
}

}  // namespace host2d
