// The reverse sweep of the 2D spatial operator (Eq. (3.2) with the PP limiter and the
// modified moments of Eq. (3.4)) with the CUDA path's own code compiled for the host:
// the recording forward (the bodies of k_cons_rec, k_face_moments, k_weak_moments,
// k_grad_rec, k_flux and k_assemble), then the nine reverse kernels of one sweep
// (ka_assemble ... ka_ghost_x), each called once per index of its launch, in the
// sweep's order.  Every plane that the sweep does not clear starts as NaN, so a reverse
// kernel that read a value no earlier kernel wrote would spoil the result.  Input: the
// configuration record of operator2d.h, then q[12][ny][nx], rbar[12][ny][nx] and
// mbar[8][ny][nx].  Output (doubles): xbar[12][ny][nx], mubar (the derivative with
// respect to 1/Re), then the forward's rhs[12][ny][nx].
#include <cstdio>
#include "operator2d.h"
#include "hweno_adjoint.cuh"

using namespace host2d;

namespace {

// blockIdx over [0, nx) x [0, ny) x [0, nz) with one thread per block
template <class F>
void launch(int nx, int ny, int nz, F&& body) {
  blockDim = {1, 1, 1};
  threadIdx = {0, 0, 0};
  gridDim = {(unsigned)nx, (unsigned)ny, (unsigned)nz};
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        blockIdx = {(unsigned)x, (unsigned)y, (unsigned)z};
        body();
      }
}

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  Input in;
  if (!read_input(f, in)) return 2;
  const hweno_config& c = in.c;
  if (c.scheme != HWENO_SCHEME_GR || c.source || in.mixed) return 2;  // the adjoint's scope
  const Grid g = make_grid(c);
  const Open o = make_open(c);
  const int nx = g.nx, ny = g.ny;
  const size_t n = (size_t)nx * ny;
  std::vector<double> src(12 * n), rb(12 * n), mb(8 * n);
  if (fread(src.data(), sizeof(double), src.size(), f) != src.size()) return 3;
  if (fread(rb.data(), sizeof(double), rb.size(), f) != rb.size()) return 3;
  if (fread(mb.data(), sizeof(double), mb.size(), f) != mb.size()) return 3;
  fclose(f);
  const double fill = nan_fill();
  auto planes = [&](int k, double v) { return std::vector<double>((size_t)k * g.ps, v); };
  auto interior_in = [&](std::vector<double>& dst, const std::vector<double>& s, int k) {
    for (int p = 0; p < k; p++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) dst[p * g.ps + cidx(g, i, j)] = s[p * n + (size_t)j * nx + i];
  };
  auto interior_out = [&](const std::vector<double>& s, int k, FILE* out) {
    for (int p = 0; p < k; p++)
      for (int j = 0; j < ny; j++) fwrite(&s[p * g.ps + cidx(g, 0, j)], sizeof(double), nx, out);
  };

  // the recording forward at q (its ghost cells filled in place, as launch_ghost does)
  std::vector<double> q = planes(12, fill), rhs = planes(12, fill), mom = planes(8, fill);
  std::vector<double> yrec = planes(YREC_PLANES, fill);
  interior_in(q, src, 12);
  Scratch s(g, c.scheme, fill);
  Work& w = s.w;
  w.yrec = yrec.data();
  Diag diag;
  memset(&diag, 0, sizeof(diag));
  for (int k = 0; k < 8 * ny + 8 * (nx + 2 * NG); k++) ghost_xy_body(g, &o, q.data(), k);
  for (int gy = 0; gy < ny + 6; gy++)
    for (int gx = 0; gx < nx + 6; gx++) cons_body<double, true>(g, q.data(), w, mom.data(), &diag, gx, gy);
  for (int gz = 0; gz < 2; gz++)
    for (int gy = 0; gy < ny + 5; gy++)
      for (int gx = 0; gx < nx + 5; gx++) face_moments_body(g, w, gx, gy, gz);
  for (int gy = 0; gy < ny + 4; gy++)
    for (int gx = 0; gx < nx + 4; gx++) weak_moments_body(g, w, gx, gy);
  for (int gy = 0; gy < ny + 2; gy++)
    for (int gx = 0; gx < nx + 2; gx++) {
      if (c.linear_grad) grad_body<double, true, true>(g, w, gx, gy);
      else grad_body<double, true>(g, w, gx, gy);
    }
  for (int gz = 0; gz < 2; gz++)
    for (int gy = 0; gy < ny + 1; gy++)
      for (int gx = 0; gx < nx + 1; gx++) flux_body<double>(g, w, &diag, gx, gy, gz);
  for (int gy = 0; gy < ny; gy++)
    for (int gx = 0; gx < nx; gx++) assemble_body<double>(g, w, rhs.data(), &diag, gx, gy);

  // the sweep: seeds in the interior of zeroed planes; face, vol and gr cleared as the
  // sweep clears them; everything else as NaN
  std::vector<double> R = planes(12, 0.0), M = planes(8, 0.0), face = planes(48, 0.0), vol = planes(36, 0.0),
                      gr = planes(126, 0.0), rm = planes(18, fill), cg = planes(102, fill), cc = planes(68, fill),
                      qb = planes(12, fill), mu(2, 0.0);
  interior_in(R, rb, 12);
  interior_in(M, mb, 8);
  Adj a;
  a.R = R.data(); a.M = M.data(); a.face = face.data(); a.vol = vol.data(); a.gr = gr.data();
  a.rm = rm.data(); a.cg = cg.data(); a.cc = cc.data(); a.q = qb.data(); a.mu = mu.data();
  launch(nx, ny, 1, [&] { ka_assemble(g, w, a); });
  launch(nx + 1, ny + 1, 2, [&] { ka_flux(g, w, a); });
  launch(nx + 2, ny + 2, 1, [&] {
    if (c.linear_grad) ka_grad<true>(g, w, a);
    else ka_grad(g, w, a);
  });
  launch(nx + 4, ny + 4, 1, [&] { ka_gather_rm(g, a); });
  launch(nx + 5, ny + 5, 2, [&] { ka_face_moments(g, a); });
  launch(nx + 6, ny + 6, 1, [&] { ka_cons(g, q.data(), w, a); });
  launch(nx + 8, ny + 8, 1, [&] { ka_gather_q(g, a); });
  launch(8 * (nx + 2 * NG), 1, 1, [&] { ka_ghost_y(g, a); });
  launch(8 * ny, 1, 1, [&] { ka_ghost_x(g, a); });

  FILE* out = fopen(argv[2], "wb");
  if (!out) return 4;
  interior_out(qb, 12, out);
  fwrite(&mu[0], sizeof(double), 1, out);
  interior_out(rhs, 12, out);
  fclose(out);
  return diag.flags != 0 ? 5 : 0;
}
