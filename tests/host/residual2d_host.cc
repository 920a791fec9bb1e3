// One evaluation of the 2D spatial operator with the CUDA path's own code compiled for
// the host (operator2d.h): FP64 or the mixed path.  Input: the configuration record of
// operator2d.h, then q[12][ny][nx].  Output (doubles): rhs[12][ny][nx], vhat[8][ny][nx],
// theta[2][ny][nx], then alpha*, beta_max, limiter activations, flags.
#include <cstdio>
#include "operator2d.h"

using namespace host2d;

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  Input in;
  if (!read_input(f, in)) return 2;
  const hweno_config& c = in.c;
  const Grid g = make_grid(c);
  const Open o = make_open(c);
  const Quad4 quad = make_quad4();
  const int nx = g.nx, ny = g.ny;
  const size_t n = (size_t)nx * ny;
  std::vector<double> src(12 * n);
  if (fread(src.data(), sizeof(double), src.size(), f) != src.size()) return 3;
  fclose(f);
  const double fill = in.nan_fill ? nan_fill() : 0.0;
  std::vector<double> q(12 * g.ps, fill), rhs(12 * g.ps, fill), mom(8 * g.ps, fill);
  Scratch s(g, c.scheme, fill);
  Diag diag;
  memset(&diag, 0, sizeof(diag));
  for (int p = 0; p < 12; p++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) q[p * g.ps + cidx(g, i, j)] = src[p * n + (size_t)j * nx + i];
  residual(c, g, o, quad, s, q.data(), rhs.data(), mom.data(), &diag, in.t, in.mixed);

  FILE* out = fopen(argv[2], "wb");
  if (!out) return 4;
  auto put = [&](const std::vector<double>& a, int k) {
    for (int p = 0; p < k; p++)
      for (int j = 0; j < ny; j++) fwrite(&a[p * g.ps + cidx(g, 0, j)], sizeof(double), nx, out);
  };
  put(rhs, 12);
  put(mom, 8);
  put(s.theta, 2);
  double alpha, beta;
  memcpy(&alpha, &diag.alpha_bits, sizeof(alpha));
  memcpy(&beta, &diag.beta_bits, sizeof(beta));
  const double tail[4] = {alpha, beta, (double)diag.pp_count, (double)diag.flags};
  fwrite(tail, sizeof(double), 4, out);
  fclose(out);
  return 0;
}
