// Runs the 2D ghost-cell rules of hweno_state.cuh (the device code, compiled for the
// host) over a whole state: the one-launch form ghost_xy_body over every thread index, on
// the 12 FP64 planes and on the 24 float planes of their hi/lo split (split from the
// interior, ghosts filled by the same passes).  Input: 6 ints (nx, ny, bc[4]), 44
// doubles (x0, x1, y0, y1, inflow[4][2][4], band[4][2]), then q[12][ny][nx].  Output:
// the padded planes [12][ny+8][nx+8] as doubles, then [24][ny+8][nx+8] as floats.
#include "shim.h"
#include <cstdio>
#include <vector>
#include "hweno_state.cuh"

using namespace hw;

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  int hdr[6];
  double dh[44];
  if (fread(hdr, sizeof(int), 6, f) != 6 || fread(dh, sizeof(double), 44, f) != 44) return 2;
  Grid g;
  memset(&g, 0, sizeof(g));
  g.nx = hdr[0];
  g.ny = hdr[1];
  for (int k = 0; k < 4; k++) g.bc[k] = hdr[2 + k];
  g.pitch = ((g.nx + 2 * NG + 15) / 16) * 16;
  g.ps = (long long)(g.ny + 2 * NG) * g.pitch;
  g.x0 = dh[0];
  g.y0 = dh[2];
  g.dx = (dh[1] - dh[0]) / g.nx;
  g.dy = (dh[3] - dh[2]) / g.ny;
  Open o;
  memcpy(o.state, dh + 4, sizeof(o.state));
  memcpy(o.band, dh + 36, sizeof(o.band));
  const size_t n = (size_t)g.nx * g.ny;
  std::vector<double> in(12 * n);
  if (fread(in.data(), sizeof(double), in.size(), f) != in.size()) return 3;
  fclose(f);
  // unset cells hold NaN, so a ghost the passes miss shows
  std::vector<double> q(12 * g.ps, NAN);
  std::vector<float> hilo(24 * g.ps, NAN);
  for (int p = 0; p < 12; p++)
    for (int j = 0; j < g.ny; j++)
      for (int i = 0; i < g.nx; i++) {
        const double x = in[p * n + (size_t)j * g.nx + i];
        q[p * g.ps + cidx(g, i, j)] = x;
        split_hilo(x, hilo[p * g.ps + cidx(g, i, j)], hilo[(12 + p) * g.ps + cidx(g, i, j)]);
      }
  // the kernels' one-launch form: x ghosts and y ghosts by thread index, a corner formed
  // from the x rule in place of reading the x pass's cell (the threads run in reverse
  // order here, so no y thread can see an x ghost its x thread wrote first)
  for (int t = 8 * g.ny + 8 * (g.nx + 2 * NG) - 1; t >= 0; t--) {
    ghost_xy_body(g, &o, q.data(), t);
    ghost_xy_body(g, &o, hilo.data(), t, 0, 24);
  }
  FILE* w = fopen(argv[2], "wb");
  if (!w) return 4;
  for (int p = 0; p < 12; p++)
    for (int j = -NG; j < g.ny + NG; j++)
      fwrite(&q[p * g.ps + cidx(g, -NG, j)], sizeof(double), g.nx + 2 * NG, w);
  for (int p = 0; p < 24; p++)
    for (int j = -NG; j < g.ny + NG; j++)
      fwrite(&hilo[p * g.ps + cidx(g, -NG, j)], sizeof(float), g.nx + 2 * NG, w);
  fclose(w);
  return 0;
}
