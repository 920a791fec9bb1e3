// The adjoint of the gradient reconstruction with the linear weights (ka_grad<true>, the
// reverse kernel itself, called once per thread index) against its forward
// (grad_body<double, false, true>), both compiled for the host: with the linear weights
// the map from the 17 stencil data of each field to its 21 gradient values is linear, so
// for any weak moments rm and any adjoint seeds lambda, sum lambda . F(rm) equals the sum
// over cells and fields of the reverse's 17 contributions times the stencil data they
// belong to.  Input: 2 ints (nx, ny), a seed.  Output: the two sums and their scale.
#include "shim.h"
#include <cstdio>
#include <random>
#include <vector>
#include "hweno_adjoint.cuh"

using namespace hw;

int main(int argc, char** argv) {
  if (argc != 4) return 1;
  hweno_config c;
  memset(&c, 0, sizeof(c));
  c.nx = atoi(argv[1]);
  c.ny = atoi(argv[2]);
  c.x1 = 1.0; c.y1 = 1.0; c.gamma = 1.4; c.Pr = 0.72; c.Re = 100.0; c.eps_weno = 1e-8;
  const Grid g = make_grid(c);
  std::mt19937_64 rng(atoi(argv[3]));
  std::normal_distribution<double> nd(0.0, 1.0);
  std::vector<double> rm(18 * g.ps), gr(126 * g.ps, 0.0), grb(126 * g.ps), cg(102 * g.ps, 0.0);
  for (auto& x : rm) x = nd(rng);
  for (auto& x : grb) x = nd(rng);
  Work w;
  memset(&w, 0, sizeof(w));
  w.rm = rm.data();
  w.gr = gr.data();
  Adj a;
  memset(&a, 0, sizeof(a));
  a.gr = grb.data();
  a.cg = cg.data();
  for (int gy = 0; gy < g.ny + 2; gy++)
    for (int gx = 0; gx < g.nx + 2; gx++) grad_body<double, false, true>(g, w, gx, gy);
  for (unsigned by = 0; by < (unsigned)(g.ny + 2); by++)
    for (unsigned bx = 0; bx < (unsigned)(g.nx + 2); bx++) {
      blockIdx.x = bx;
      blockIdx.y = by;
      ka_grad<true>(g, w, a);
    }
  double lhs = 0.0, rhs = 0.0, scale = 0.0;
  for (int j = -1; j <= g.ny; j++)
    for (int i = -1; i <= g.nx; i++) {
      const long long cc = cidx(g, i, j);
      for (int comp = 0; comp < 6; comp++) {
        for (int k = 0; k < 21; k++) {
          const long long p = (long long)(6 * k + comp) * g.ps + cc;
          lhs += grb[p] * gr[p];
          scale += fabs(grb[p] * gr[p]);
        }
        // the stencil data of grad_body, in its order
        const int n = comp >> 1, l = comp & 1;
        const double* A = rm.data() + (long long)(6 * n + 3 * l) * g.ps;
        const double* X = A + g.ps;
        const double* Y = A + 2 * g.ps;
        double d[17];
        for (int b = -1; b <= 1; b++)
          for (int aa = -1; aa <= 1; aa++) d[(b + 1) * 3 + (aa + 1)] = A[cidx(g, i + aa, j + b)];
        d[9] = X[cidx(g, i - 1, j)];
        d[10] = X[cidx(g, i + 1, j)];
        d[11] = Y[cidx(g, i, j - 1)];
        d[12] = Y[cidx(g, i, j + 1)];
        d[13] = X[cidx(g, i, j - 1)];
        d[14] = X[cidx(g, i, j + 1)];
        d[15] = Y[cidx(g, i - 1, j)];
        d[16] = Y[cidx(g, i + 1, j)];
        for (int k = 0; k < 17; k++) rhs += cg[(long long)(17 * comp + k) * g.ps + cc] * d[k];
      }
    }
  printf("%.17g %.17g %.17g\n", lhs, rhs, scale);
  return 0;
}
