// One evaluation of the 2D spatial operator with the CUDA path's own code compiled for
// the host (operator2d.h): FP64 or the mixed path (its separate kernels; with the record's
// mixed mode 2 or 3 the flux tiles, and with 3 the TMA-staged gradients too).  Input: the
// configuration record of operator2d.h, then q[12][ny][nx].  Output (doubles):
// rhs[12][ny][nx], vhat[8][ny][nx],
// theta[2][ny][nx], then alpha*, beta_max, limiter activations, flags, then the
// intermediate fields as hweno_debug_fields exports them (FP64 path): the 12 face and 9
// volume points as (rho, rho u, rho v, E), the 18 weak moments and the 126 gradients.
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
  residual(c, g, o, quad, s, q.data(), rhs.data(), mom.data(), &diag, in.t, in.mixed, in.tma, in.fused);

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
  // points stored as (rho, u, v, e), exported as the conservative variables
  auto put_cons = [&](const std::vector<double>& a, int npts) {
    std::vector<double> row(nx);
    for (int k = 0; k < npts; k++)
      for (int v = 0; v < 4; v++)
        for (int j = 0; j < ny; j++) {
          for (int i = 0; i < nx; i++) {
            const long long c = cidx(g, i, j);
            const double rho = a[(4 * k) * g.ps + c], u = a[(4 * k + 1) * g.ps + c];
            const double w = a[(4 * k + 2) * g.ps + c], e = a[(4 * k + 3) * g.ps + c];
            row[i] = v == 0 ? rho : v == 1 ? rho * u : v == 2 ? rho * w : rho * (e + 0.5 * (u * u + w * w));
          }
          fwrite(row.data(), sizeof(double), nx, out);
        }
  };
  put_cons(s.face, 12);
  put_cons(s.vol, 9);
  put(s.rm, 18);
  put(s.gr, 126);
  fclose(out);
  return 0;
}
