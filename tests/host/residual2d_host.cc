// Runs one evaluation of the 2D spatial operator with the CUDA path's own code compiled
// for the host (hweno_state.cuh, hweno_ops.cuh, hweno_mixed.cuh, hweno_source.cuh): the
// grid from make_grid, the ghost passes, then each kernel's body over the index range
// of its launch, in the order of the operator: traces and limiter, face and weak
// moments, the gradient reconstruction (or the HWENO-DR derivatives), face fluxes,
// balances and the manufactured source; FP64, or the mixed path (the hi/lo split of the
// ghost-filled state, then its FP32 bodies).  Every plane set is an allocation of its
// own, so that an access past one shows under AddressSanitizer; with a NaN fill (NaN as
// a double and as either float half), a read of a scratch value that no earlier kernel
// wrote reaches the output.
//
// Input: 11 ints (nx, ny, bc[4], scheme, source, linear_grad, nan_fill, mixed), 50 doubles
// (x0, x1, y0, y1, gamma, Pr, Re, eps_pp, eps_weno, t, inflow[4][2][4], band[4][2]), then
// q[12][ny][nx].  Output (doubles): rhs[12][ny][nx], vhat[8][ny][nx], theta[2][ny][nx],
// then alpha*, beta_max, limiter activations, flags.
#include "shim.h"
#include <cstdio>
#include <vector>
#include "hweno_mixed.cuh"
#include "hweno_source.cuh"

namespace hw {
double cons_smem[CONS_SMEM_BYTES / sizeof(double)];
double dr_smem[DR_SMEM_BYTES / sizeof(double)];
}  // namespace hw

using namespace hw;

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  int hi[11];
  double hd[50];
  if (fread(hi, sizeof(int), 11, f) != 11 || fread(hd, sizeof(double), 50, f) != 50) return 2;
  hweno_config c;
  memset(&c, 0, sizeof(c));
  c.nx = hi[0];
  c.ny = hi[1];
  for (int k = 0; k < 4; k++) c.bc[k] = hi[2 + k];
  c.scheme = hi[6];
  c.source = hi[7];
  c.linear_grad = hi[8];
  const bool nan_fill = hi[9] != 0;
  const bool mixed = hi[10] != 0;
  c.x0 = hd[0]; c.x1 = hd[1]; c.y0 = hd[2]; c.y1 = hd[3];
  c.gamma = hd[4]; c.Pr = hd[5]; c.Re = hd[6]; c.eps_pp = hd[7]; c.eps_weno = hd[8];
  const double t = hd[9];
  memcpy(c.inflow, hd + 10, sizeof(c.inflow));
  memcpy(c.band, hd + 42, sizeof(c.band));
  const Grid g = make_grid(c);
  const Open o = make_open(c);
  const Quad4 quad = make_quad4();
  const int nx = g.nx, ny = g.ny;
  const size_t n = (size_t)nx * ny;
  std::vector<double> in(12 * n);
  if (fread(in.data(), sizeof(double), in.size(), f) != in.size()) return 3;
  fclose(f);

  double fill = 0.0;
  if (nan_fill) {
    const unsigned long long b = 0x7FC000007FC00000ull;
    memcpy(&fill, &b, sizeof(fill));
  }
  auto planes = [&](int k) { return std::vector<double>((size_t)k * g.ps, fill); };
  std::vector<double> q = planes(12), rhs = planes(12), mom = planes(8);
  std::vector<double> face = planes(48), vol = planes(36), wbar = planes(3), wx = planes(6), wy = planes(6);
  std::vector<double> rm = planes(18), gr = planes(126), fx = planes(12), fy = planes(12), theta = planes(2);
  std::vector<double> dr = planes(c.scheme == HWENO_SCHEME_DR ? 120 : 0);
  Work w;
  w.face = face.data(); w.vol = vol.data(); w.wbar = wbar.data(); w.wx = wx.data(); w.wy = wy.data();
  w.rm = rm.data(); w.gr = gr.data(); w.fx = fx.data(); w.fy = fy.data(); w.theta = theta.data();
  w.yrec = nullptr;
  w.dr = c.scheme == HWENO_SCHEME_DR ? dr.data() : nullptr;
  Diag diag;
  memset(&diag, 0, sizeof(diag));
  for (int p = 0; p < 12; p++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) q[p * g.ps + cidx(g, i, j)] = in[p * n + (size_t)j * nx + i];

  for (int k = 0; k < 8 * ny; k++) ghost_x_body(g, &o, q.data(), k);
  for (int k = 0; k < 8 * (nx + 2 * NG); k++) ghost_y_body(g, &o, q.data(), k);
  if (mixed) {
    // the split of the ghost-filled state (k_split), then the FP32 bodies
    float* hilo = mixed_planes(w, g.ps).hilo;
    const long long np = 12 * g.ps;
    for (long long k = 0; k < np; k++) split_hilo(q[k], hilo[k], hilo[np + k]);
    for (int gy = 0; gy < ny + 6; gy++)
      for (int gx = 0; gx < nx + 6; gx++) cons_mixed_body(g, q.data(), w, mom.data(), &diag, gx, gy);
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
        for (int gx = 0; gx < nx + 1; gx++) flux_mixed_body(g, w, &diag, gx, gy, gz);
    for (int gy = 0; gy < ny; gy++)
      for (int gx = 0; gx < nx; gx++) assemble_mixed_body(g, w, rhs.data(), &diag, gx, gy);
  }
  if (!mixed) {
    const bool drs = c.scheme == HWENO_SCHEME_DR;
    for (int gy = 0; gy < ny + 6; gy++)
      for (int gx = 0; gx < nx + 6; gx++) {
        if (drs) cons_body<double, false, true>(g, q.data(), w, mom.data(), &diag, gx, gy);
        else cons_body<double>(g, q.data(), w, mom.data(), &diag, gx, gy);
      }
    if (drs) {
      for (int gy = 0; gy < ny + 2; gy++)
        for (int gx = 0; gx < nx + 2; gx++) dr_body(g, q.data(), w, gx, gy);
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
        for (int gx = 0; gx < nx + 1; gx++) flux_body<double>(g, w, &diag, gx, gy, gz);
    for (int gy = 0; gy < ny; gy++)
      for (int gx = 0; gx < nx; gx++) assemble_body<double>(g, w, rhs.data(), &diag, gx, gy);
  }
  if (c.source == HWENO_SOURCE_MMS52)
    for (int gy = 0; gy < ny; gy++)
      for (int gx = 0; gx < nx; gx++) source_body(g, quad, t, 0.0, &diag, rhs.data(), gx, gy);

  FILE* out = fopen(argv[2], "wb");
  if (!out) return 4;
  auto put = [&](const std::vector<double>& a, int k) {
    for (int p = 0; p < k; p++)
      for (int j = 0; j < ny; j++) fwrite(&a[p * g.ps + cidx(g, 0, j)], sizeof(double), nx, out);
  };
  put(rhs, 12);
  put(mom, 8);
  put(theta, 2);
  double alpha, beta;
  memcpy(&alpha, &diag.alpha_bits, sizeof(alpha));
  memcpy(&beta, &diag.beta_bits, sizeof(beta));
  const double tail[4] = {alpha, beta, (double)diag.pp_count, (double)diag.flags};
  fwrite(tail, sizeof(double), 4, out);
  fclose(out);
  return 0;
}
