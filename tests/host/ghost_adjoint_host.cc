// Runs the adjoint of the 2D ghost fill (ka_ghost_y, then ka_ghost_x: the adjoint
// kernels themselves, compiled for the host, one call per thread index) on a padded
// adjoint field, next to the forward ghost passes with the inflow states set to zero
// (the ghost fill is then linear in the state).  Input: 6 ints (nx, ny, bc[4]), 12 doubles
// (x0, x1, y0, y1, band[4][2]), then q[12][ny][nx] and lambda[12][ny+8][nx+8].  Output
// (doubles): the ghost-filled q [12][ny+8][nx+8], then the adjoint's interior
// [12][ny][nx].
#include "shim.h"
#include <cstdio>
#include <vector>
#include "hweno_adjoint.cuh"

using namespace hw;

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  int hi[6];
  double hd[12];
  if (fread(hi, sizeof(int), 6, f) != 6 || fread(hd, sizeof(double), 12, f) != 12) return 2;
  hweno_config c;
  memset(&c, 0, sizeof(c));
  c.nx = hi[0];
  c.ny = hi[1];
  for (int k = 0; k < 4; k++) c.bc[k] = hi[2 + k];
  c.x0 = hd[0]; c.x1 = hd[1]; c.y0 = hd[2]; c.y1 = hd[3];
  c.gamma = 1.4; c.Pr = 0.72; c.Re = 100.0;
  memcpy(c.band, hd + 4, sizeof(c.band));
  const Grid g = make_grid(c);
  const Open o = make_open(c);  // zero states: the linear part of the ghost fill
  const int nx = g.nx, ny = g.ny, W = nx + 2 * NG, H = ny + 2 * NG;
  const size_t n = (size_t)nx * ny;
  std::vector<double> in(12 * n), lam_in(12 * (size_t)W * H);
  if (fread(in.data(), sizeof(double), in.size(), f) != in.size()) return 3;
  if (fread(lam_in.data(), sizeof(double), lam_in.size(), f) != lam_in.size()) return 3;
  fclose(f);
  std::vector<double> q(12 * g.ps, 0.0), lam(12 * g.ps, 0.0);
  for (int p = 0; p < 12; p++) {
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) q[p * g.ps + cidx(g, i, j)] = in[p * n + (size_t)j * nx + i];
    for (int j = -NG; j < ny + NG; j++)
      for (int i = -NG; i < nx + NG; i++)
        lam[p * g.ps + cidx(g, i, j)] = lam_in[(size_t)p * W * H + (size_t)(j + NG) * W + (i + NG)];
  }
  for (int k = 0; k < 8 * ny; k++) ghost_x_body(g, &o, q.data(), k);
  for (int k = 0; k < 8 * W; k++) ghost_y_body(g, &o, q.data(), k);
  Adj a;
  memset(&a, 0, sizeof(a));
  a.q = lam.data();
  for (unsigned t = 0; t < (unsigned)(8 * W); t++) {
    blockIdx.x = t;
    ka_ghost_y(g, a);
  }
  for (unsigned t = 0; t < (unsigned)(8 * ny); t++) {
    blockIdx.x = t;
    ka_ghost_x(g, a);
  }
  FILE* out = fopen(argv[2], "wb");
  if (!out) return 4;
  for (int p = 0; p < 12; p++)
    for (int j = -NG; j < ny + NG; j++) fwrite(&q[p * g.ps + cidx(g, -NG, j)], sizeof(double), W, out);
  for (int p = 0; p < 12; p++)
    for (int j = 0; j < ny; j++) fwrite(&lam[p * g.ps + cidx(g, 0, j)], sizeof(double), nx, out);
  fclose(out);
  return 0;
}
