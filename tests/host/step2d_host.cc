// SSP-RK3 steps of the 2D operator with the CUDA path's own bodies compiled for the host
// (operator2d.h and rk_body), in the order of a handle's step: the stage-1 evaluation and
// the step rule (dt = min(CFL h / alpha*, b Re h^2), or a forced dt), then per attempt
// the three stage updates with their evaluations, then the flags; an attempt whose stage
// output is inadmissible or not finite is repeated with dt / 2, at most max_halvings
// times.  FP64, or the mixed path (each evaluation splits its ghost-filled state: the
// split a handle's stage update writes, ghost-filled, is the same), or the mixed path
// with stages 2 and 3 as its fused kernel runs them.  Input: the
// configuration record of operator2d.h, then an int nsteps,
// doubles cfl, b_visc, dt_forced, an int max_halvings, and q[12][ny][nx].  Output
// (doubles): q[12][ny][nx] after the steps taken, the status (0, or -3 when a step stays
// inadmissible, -4 when a residual at t^n is not finite), then per step taken (and the
// failed one) its dt and restarts.
#include <cstdio>
#include <utility>
#include "operator2d.h"

using namespace host2d;

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  Input in;
  if (!read_input(f, in)) return 2;
  int nsteps, max_halvings;
  double cfl, b_visc, dt_forced;
  if (fread(&nsteps, sizeof(int), 1, f) != 1 || fread(&cfl, sizeof(double), 1, f) != 1 ||
      fread(&b_visc, sizeof(double), 1, f) != 1 || fread(&dt_forced, sizeof(double), 1, f) != 1 ||
      fread(&max_halvings, sizeof(int), 1, f) != 1)
    return 2;
  const hweno_config& c = in.c;
  const Grid g = make_grid(c);
  const Open o = make_open(c);
  const Quad4 quad = make_quad4();
  const int nx = g.nx, ny = g.ny;
  const size_t n = (size_t)nx * ny;
  std::vector<double> src(12 * n);
  if (fread(src.data(), sizeof(double), src.size(), f) != src.size()) return 3;
  fclose(f);
  auto planes = [&](int k) { return std::vector<double>((size_t)k * g.ps, 0.0); };
  std::vector<double> Q = planes(12), QS = planes(12), Q1 = planes(12), Q2 = planes(12), BASE = planes(12);
  std::vector<double> RHS0 = planes(12), RHS = planes(12), MOM0 = planes(8), MOM = planes(8);
  Scratch s(g, c.scheme, 0.0);
  for (int p = 0; p < 12; p++)
    for (int j = 0; j < ny; j++)
      for (int i = 0; i < nx; i++) Q[p * g.ps + cidx(g, i, j)] = src[p * n + (size_t)j * nx + i];
  const double hmin = g.dx < g.dy ? g.dx : g.dy;
  // the mixed path's stage update is k_rk_split's (its split output is the split the next
  // evaluation forms again from the ghost-filled state)
  std::vector<float> hilo_out(24 * (size_t)g.ps);
  auto stage = [&](int k, const double* qin, const double* mom, const double* rhs, double* qout, Diag* d) {
    for (int gy = 0; gy < ny; gy++)
      for (int gx = 0; gx < nx; gx++) {
        if (in.mixed) rk_body<true>(g, k, qin, mom, rhs, BASE.data(), qout, d, gx, gy, hilo_out.data());
        else rk_body<false>(g, k, qin, mom, rhs, BASE.data(), qout, d, gx, gy);
      }
  };
  std::vector<double> log;
  int status = 0;
  double t = in.t;
  for (int step = 0; step < nsteps && !status; step++) {
    Diag d[2];  // the attempt's counters and flags, and the stage-1 ones
    memset(d, 0, sizeof(d));
    residual(c, g, o, quad, s, Q.data(), RHS0.data(), MOM0.data(), &d[0], t, in.mixed, in.tma, in.fused);
    double alpha;
    memcpy(&alpha, &d[0].alpha_bits, sizeof(alpha));
    d[0].dt = dt_forced > 0.0 ? dt_forced : fmin(cfl * hmin / alpha, b_visc * c.Re * hmin * hmin);
    d[1] = d[0];
    for (int rej = 0;; rej++) {
      d[0].pp_count = 0;
      d[0].flags = 0;
      const double dt = d[0].dt;
      stage(1, Q.data(), MOM0.data(), RHS0.data(), Q1.data(), &d[0]);
      if (in.fused) {  // stages 2 and 3 as the mixed path's fused kernel runs them
        fused_stage(c, g, o, s, Q1.data(), MOM.data(), BASE.data(), Q2.data(), 2, &d[0], in.tma);
        fused_stage(c, g, o, s, Q2.data(), MOM.data(), BASE.data(), QS.data(), 3, &d[0], in.tma);
      } else {
        residual(c, g, o, quad, s, Q1.data(), RHS.data(), MOM.data(), &d[0], t + dt, in.mixed);
        stage(2, Q1.data(), MOM.data(), RHS.data(), Q2.data(), &d[0]);
        residual(c, g, o, quad, s, Q2.data(), RHS.data(), MOM.data(), &d[0], t + 0.5 * dt, in.mixed);
        stage(3, Q2.data(), MOM.data(), RHS.data(), QS.data(), &d[0]);
      }
      if (d[1].flags & FLAG_NONFINITE) {
        status = -4;
        break;
      }
      if (!(d[0].flags & (FLAG_INADMISSIBLE | FLAG_NONFINITE))) {
        std::swap(Q, QS);
        t += dt;
        log.push_back(dt);
        log.push_back(rej);
        break;
      }
      if (rej >= max_halvings) {
        status = -3;
        log.push_back(0.0);
        log.push_back(rej);
        break;
      }
      d[0].dt *= 0.5;
    }
  }
  FILE* out = fopen(argv[2], "wb");
  if (!out) return 4;
  for (int p = 0; p < 12; p++)
    for (int j = 0; j < ny; j++) fwrite(&Q[p * g.ps + cidx(g, 0, j)], sizeof(double), nx, out);
  const double st = status;
  fwrite(&st, sizeof(double), 1, out);
  fwrite(log.data(), sizeof(double), log.size(), out);
  fclose(out);
  return 0;
}
