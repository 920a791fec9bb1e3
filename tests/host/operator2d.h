// The 2D spatial operator of the CUDA path, run on the host (test infrastructure): the
// kernels' own bodies (hweno_state.cuh, hweno_ops.cuh, hweno_mixed.cuh,
// hweno_source.cuh), each called over the index range of its launch, in the operator's
// order.  Every plane set is an allocation of its own, so that an access past one shows
// under AddressSanitizer; a NaN fill (NaN as a double and as either float half) makes a
// read of a value that no earlier kernel wrote reach the output.
#pragma once
#include "shim.h"
#include <vector>
#include "hweno_mixed.cuh"
#include "hweno_source.cuh"

namespace hw {
double cons_smem[CONS_SMEM_BYTES / sizeof(double)];
double dr_smem[DR_SMEM_BYTES / sizeof(double)];
}  // namespace hw

namespace host2d {
using namespace hw;

inline double nan_fill() {
  const unsigned long long b = 0x7FC000007FC00000ull;
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

// one evaluation at state q (12 padded planes, ghosts filled here): rhs (12) and the
// modified moments mom (8); the source term, when configured, at time t
inline void residual(const hweno_config& c, const Grid& g, const Open& o, const Quad4& quad, Scratch& s,
                     double* q, double* rhs, double* mom, Diag* diag, double t, bool mixed) {
  const int nx = g.nx, ny = g.ny;
  Work& w = s.w;
  for (int k = 0; k < 8 * ny; k++) ghost_x_body(g, &o, q, k);
  for (int k = 0; k < 8 * (nx + 2 * NG); k++) ghost_y_body(g, &o, q, k);
  if (mixed) {
    // the split of the ghost-filled state (k_split), then the FP32 bodies
    float* hilo = mixed_planes(w, g.ps).hilo;
    const long long np = 12 * g.ps;
    for (long long k = 0; k < np; k++) split_hilo(q[k], hilo[k], hilo[np + k]);
    for (int gy = 0; gy < ny + 6; gy++)
      for (int gx = 0; gx < nx + 6; gx++) cons_mixed_body(g, q, w, mom, diag, gx, gy);
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
// source, linear_grad, nan_fill, mixed), 50 doubles (x0, x1, y0, y1, gamma, Pr, Re,
// eps_pp, eps_weno, t, inflow[4][2][4], band[4][2])
struct Input {
  hweno_config c;
  bool nan_fill, mixed;
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
  c.x0 = hd[0]; c.x1 = hd[1]; c.y0 = hd[2]; c.y1 = hd[3];
  c.gamma = hd[4]; c.Pr = hd[5]; c.Re = hd[6]; c.eps_pp = hd[7]; c.eps_weno = hd[8];
  in.t = hd[9];
  memcpy(c.inflow, hd + 10, sizeof(c.inflow));
  memcpy(c.band, hd + 42, sizeof(c.band));
  return true;
}

}  // namespace host2d
