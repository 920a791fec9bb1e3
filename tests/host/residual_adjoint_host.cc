// The discrete adjoint of the 2D spatial operator (Eq. (3.2) with the PP limiter and the
// modified moments of Eq. (3.4)) and of one SSP-RK3 step (Eq. (2.12) in its 2D form) at a
// fixed dt, with the CUDA path's own code compiled for the host.  The recording forward
// runs the bodies of k_cons_rec, k_face_moments, k_weak_moments, k_grad_rec, k_flux and
// k_assemble (and of k_rk for the step's stages); a sweep runs the nine reverse kernels
// (ka_assemble ... ka_ghost_x), and the step's reverse the seeds, sweeps and combinations
// of hweno_adjoint_step in its order, each kernel called once per index of its launch.
// Every plane that the sequence does not clear or seed starts as NaN, so a kernel that
// read a value no earlier kernel wrote would spoil the result.
//
// Input: the configuration record of operator2d.h, an int mode and a double dt, then
// q[12][ny][nx] and
//   mode 0 (residual): rbar[12][ny][nx], mbar[8][ny][nx];
//   mode 1 (step):     lam_next[12][ny][nx].
// Output (doubles): mode 0: xbar[12][ny][nx], mubar (the derivative with respect to
// 1/Re), the forward's rhs[12][ny][nx]; mode 1: lam[12][ny][nx], mubar, the step's
// q_next[12][ny][nx].
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

struct Run {
  const hweno_config& c;
  const Grid g;
  const Open o;
  Scratch s;
  std::vector<double> yrec;
  Diag diag;
  Run(const hweno_config& cfg, double fill)
      : c(cfg), g(make_grid(cfg)), o(make_open(cfg)), s(g, cfg.scheme, fill),
        yrec((size_t)YREC_PLANES * g.ps, fill) {
    s.w.yrec = yrec.data();
    memset(&diag, 0, sizeof(diag));
  }

  // the recording forward at q, whose ghost cells it fills in place (as launch_ghost does)
  void forward(double* q, double* rhs, double* mom) {
    const int nx = g.nx, ny = g.ny;
    Work& w = s.w;
    for (int k = 0; k < 8 * ny + 8 * (nx + 2 * NG); k++) ghost_xy_body(g, &o, q, k);
    for (int gy = 0; gy < ny + 6; gy++)
      for (int gx = 0; gx < nx + 6; gx++) cons_body<double, true>(g, q, w, mom, &diag, gx, gy);
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
      for (int gx = 0; gx < nx; gx++) assemble_body<double>(g, w, rhs, &diag, gx, gy);
  }

  // one sweep (adjoint_operator): face, vol and gr cleared, then the nine kernels
  void sweep(const double* q, Adj& a) {
    const int nx = g.nx, ny = g.ny;
    const Work& w = s.w;
    std::fill(a.face, a.face + 48 * g.ps, 0.0);
    std::fill(a.vol, a.vol + 36 * g.ps, 0.0);
    std::fill(a.gr, a.gr + 126 * g.ps, 0.0);
    launch(nx, ny, 1, [&] { ka_assemble(g, w, a); });
    launch(nx + 1, ny + 1, 2, [&] { ka_flux(g, w, a); });
    launch(nx + 2, ny + 2, 1, [&] {
      if (c.linear_grad) ka_grad<true>(g, w, a);
      else ka_grad(g, w, a);
    });
    launch(nx + 4, ny + 4, 1, [&] { ka_gather_rm(g, a); });
    launch(nx + 5, ny + 5, 2, [&] { ka_face_moments(g, a); });
    launch(nx + 6, ny + 6, 1, [&] { ka_cons(g, q, w, a); });
    launch(nx + 8, ny + 8, 1, [&] { ka_gather_q(g, a); });
    launch(8 * (nx + 2 * NG), 1, 1, [&] { ka_ghost_y(g, a); });
    launch(8 * ny, 1, 1, [&] { ka_ghost_x(g, a); });
  }
};

}  // namespace

int main(int argc, char** argv) {
  if (argc != 3) return 1;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 1;
  Input in;
  if (!read_input(f, in)) return 2;
  int mode = 0;
  double dt = 0.0;
  if (fread(&mode, sizeof(int), 1, f) != 1 || fread(&dt, sizeof(double), 1, f) != 1) return 2;
  const hweno_config& c = in.c;
  if (c.scheme != HWENO_SCHEME_GR || c.source || in.mixed || mode < 0 || mode > 1) return 2;  // the adjoint's scope
  const double fill = nan_fill();
  Run r(c, fill);
  const Grid& g = r.g;
  const int nx = g.nx, ny = g.ny;
  const size_t n = (size_t)nx * ny;
  auto planes = [&](int k, double v) { return std::vector<double>((size_t)k * g.ps, v); };
  auto read_interior = [&](std::vector<double>& dst, int k) {
    std::vector<double> s(k * n);
    if (fread(s.data(), sizeof(double), s.size(), f) != s.size()) return false;
    for (int p = 0; p < k; p++)
      for (int j = 0; j < ny; j++)
        for (int i = 0; i < nx; i++) dst[p * g.ps + cidx(g, i, j)] = s[p * n + (size_t)j * nx + i];
    return true;
  };
  std::vector<double> q = planes(12, fill), rhs = planes(12, fill), mom = planes(8, fill);
  if (!read_interior(q, 12)) return 3;

  // the adjoint's planes: the seeds' planes zero outside the interior (as the pool starts),
  // the rest NaN until the sequence writes them
  std::vector<double> R = planes(12, 0.0), M = planes(8, 0.0), face = planes(48, fill), vol = planes(36, fill),
                      gr = planes(126, fill), rm = planes(18, fill), cg = planes(102, fill), cc = planes(68, fill),
                      qb = planes(12, fill), mu(2, 0.0);
  Adj a;
  a.R = R.data(); a.M = M.data(); a.face = face.data(); a.vol = vol.data(); a.gr = gr.data();
  a.rm = rm.data(); a.cg = cg.data(); a.cc = cc.data(); a.q = qb.data(); a.mu = mu.data();
  std::vector<double> out1(12 * n), out2;

  if (mode == 0) {
    if (!read_interior(R, 12) || !read_interior(M, 8)) return 3;
    fclose(f);
    r.forward(q.data(), rhs.data(), mom.data());
    r.sweep(q.data(), a);
    out1.assign(qb.begin(), qb.end());
    out2.assign(rhs.begin(), rhs.end());
  } else {
    // hweno_adjoint_step: forward stage states q1 and q2 at the forced dt, then per stage
    // in reverse: the base adjoint, the operator re-evaluated at the stage's input, the
    // seeds, a sweep and the combination
    std::vector<double> lam = planes(12, fill), bb = planes(12, fill), tmp = planes(12, fill);
    if (!read_interior(lam, 12)) return 3;
    fclose(f);
    std::vector<double> base = planes(12, fill), rhs0 = planes(12, fill), mom0 = planes(8, fill);
    std::vector<double> q1 = planes(12, fill), q2 = planes(12, fill), q3 = planes(12, fill);
    Diag& d = r.diag;
    auto stage = [&](int k, const double* qin, const double* mm, const double* rh, double* qout) {
      for (int gy = 0; gy < ny; gy++)
        for (int gx = 0; gx < nx; gx++) rk_body<false>(g, k, qin, mm, rh, base.data(), qout, &d, gx, gy);
    };
    r.forward(q.data(), rhs0.data(), mom0.data());
    d.dt = dt;
    stage(1, q.data(), mom0.data(), rhs0.data(), q1.data());
    r.forward(q1.data(), rhs.data(), mom.data());
    stage(2, q1.data(), mom.data(), rhs.data(), q2.data());
    r.forward(q2.data(), rhs.data(), mom.data());
    stage(3, q2.data(), mom.data(), rhs.data(), q3.data());
    if (d.flags & (FLAG_INADMISSIBLE | FLAG_NONFINITE)) return 5;
    const double* st[3] = {q.data(), q1.data(), q2.data()};
    const double sr[3] = {dt, 0.25 * dt, (2.0 / 3.0) * dt}, sm[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int k = 2; k >= 0; k--) {
      if (k == 2) launch(nx, ny, 1, [&] { ka_axpby(g, bb.data(), 0.0, lam.data(), 1.0 / 3.0); });
      if (k == 1) launch(nx, ny, 1, [&] { ka_axpby(g, bb.data(), 1.0, lam.data(), 0.75); });
      r.forward(const_cast<double*>(st[k]), rhs.data(), mom.data());
      launch(nx, ny, 1, [&] { ka_seed(g, lam.data(), sr[k], sm[k], k == 0 ? bb.data() : nullptr, 1.0, a); });
      r.sweep(st[k], a);
      launch(nx, ny, 1, [&] { ka_finish(g, a, lam.data(), sm[k], k == 0 ? bb.data() : nullptr, 1.0, tmp.data()); });
      std::swap(lam, tmp);
    }
    out1.assign(lam.begin(), lam.end());
    out2.assign(q3.begin(), q3.end());
  }
  if (r.diag.flags & FLAG_NONFINITE) return 5;

  FILE* out = fopen(argv[2], "wb");
  if (!out) return 4;
  for (int p = 0; p < 12; p++)
    for (int j = 0; j < ny; j++) fwrite(&out1[p * g.ps + cidx(g, 0, j)], sizeof(double), nx, out);
  fwrite(&mu[0], sizeof(double), 1, out);
  for (int p = 0; p < 12; p++)
    for (int j = 0; j < ny; j++) fwrite(&out2[p * g.ps + cidx(g, 0, j)], sizeof(double), nx, out);
  fclose(out);
  return 0;
}
