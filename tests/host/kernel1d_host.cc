// Runs the 1D solver's kernel k_solve (its own source, extracted by test_host1d.py up to
// the launch-based part of the C ABI) as one host thread per problem.  Input: 7 ints
// (n, bc[2], scheme, source, max_halvings, mode), 19 doubles (x0, x1, gamma, Pr, Re, cfl,
// b_visc, eps_pp, eps_weno, inflow[2][3], t0, t_end, max_steps, dt), then q[6][n].
// mode 2 one residual, 1 one step (forced dt if > 0), 0 advance.
#include "shim.h"
#include <cstdio>
#include <vector>
#include "kernel1d_extracted.inc"

int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "rb");
  int hdr[7];
  double dh[19];
  if (fread(hdr, sizeof(int), 7, f) != 7 || fread(dh, sizeof(double), 19, f) != 19) return 2;
  hweno1d_config c;
  memset(&c, 0, sizeof(c));
  c.n = hdr[0]; c.bc[0] = hdr[1]; c.bc[1] = hdr[2]; c.scheme = hdr[3]; c.source = hdr[4]; c.max_halvings = hdr[5];
  const int mode = hdr[6];
  c.x0 = dh[0]; c.x1 = dh[1]; c.gamma = dh[2]; c.Pr = dh[3]; c.Re = dh[4]; c.cfl = dh[5]; c.b_visc = dh[6];
  c.eps_pp = dh[7]; c.eps_weno = dh[8];
  for (int k = 0; k < 6; k++) c.inflow[k / 3][k % 3] = dh[9 + k];
  const double t0 = dh[15], t_end = dh[16], dt_in = dh[18];
  const int max_steps = (int)dh[17];
  if (check_cfg(c)) return 4;
  const int n = c.n;
  std::vector<double> q(6 * n), work(hw1::workspace_doubles(n)), out(hw1::OUT, 0.0);
  if (fread(q.data(), sizeof(double), 6 * n, f) != (size_t)(6 * n)) return 3;
  fclose(f);
  hw1::Prob p = make_prob(c, q.data(), work.data());
  hw1::k_solve(&p, mode, t0, t_end, max_steps, dt_in, out.data());
  FILE* o = fopen(argv[2], "wb");
  if (mode == 2) {
    const long long P = n + 2 * hw1::G;
    const double* r0 = work.data() + P * hw1::PADDED_PLANES;
    fwrite(r0, sizeof(double), 6 * n, o);
    fwrite(r0 + 12LL * n, sizeof(double), 3 * n, o);
  } else {
    fwrite(q.data(), sizeof(double), 6 * n, o);
  }
  fwrite(out.data(), sizeof(double), hw1::OUT, o);
  fclose(o);
  return 0;
}
