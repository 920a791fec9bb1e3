// Host check of the 1D solver: the product's per-cell __host__ __device__ functions,
// driven sequentially in the kernel's phase order, for the CPU test suite (test
// infrastructure: it compiles the kernel source for the host; the oracle is compared in
// Python).  Usage: host1d <input> <output>; the formats are those of test_host1d.py.
#include "hweno1d.cu"
#include <cstdio>
#include <cstdlib>
#include <vector>
using namespace hw1;

static void residual_host(const Prob& p, const Ptrs& s, const double* q, double t, double* rhs, double* mom,
                          double* alpha, double* beta) {
  const int n = p.n;
  const long long P = n + 2 * G;
  for (int k = 0; k < P; k++) {
    double v[6];
    fetch(p, q, k - G, v);
    for (int m = 0; m < 6; m++) s.Q[m * P + k] = v[m];
  }
  for (int k = 0; k < n + 6; k++) cons_cell(p, s, k + 1);
  if (p.scheme == 1) {
    for (int k = 0; k < n + 2; k++) dr_cell(p, s, k + 3);
  } else {
    for (int k = 0; k < n + 4; k++) weak_cell(p, s, k + 2);
    for (int k = 0; k < n + 2; k++) grad_cell(p, s, k + 3);
  }
  double amax = 0.0, bmax = 0.0;
  for (int k = 0; k < n + 1; k++) {
    const int kl = k + 3, kr = k + 4;
    double sl[3], sr[3];
    point(s, P, kl, 3, sl);
    point(s, P, kr, 0, sr);
    const double uxl = s.grad[6 * P + kl], exl = s.grad[7 * P + kl];
    const double uxr = s.grad[0 * P + kr], exr = s.grad[1 * P + kr];
    const double b = fmax(wave_bound(p, sl, uxl, exl), wave_bound(p, sr, uxr, exr));
    double fl[3], fr[3];
    phys_flux(p, sl, uxl, exl, fl);
    phys_flux(p, sr, uxr, exr, fr);
    for (int v = 0; v < 3; v++) s.flux[v * P + kl] = 0.5 * (fl[v] + fr[v] - b * (sr[v] - sl[v]));
    bmax = fmax(bmax, b);
    if (k >= 1) amax = fmax(amax, fabs(sl[1] / sl[0]) + sqrt(p.gamma * pressure(sl, p.gamma) / sl[0]));
    if (k <= n - 1) amax = fmax(amax, fabs(sr[1] / sr[0]) + sqrt(p.gamma * pressure(sr, p.gamma) / sr[0]));
  }
  for (int i = 0; i < n; i++) {
    const int k = i + G;
    double vol[3] = {0, 0, 0};
    for (int g = 0; g < 4; g++) {
      double st[3], f[3];
      point(s, P, k, g, st);
      phys_flux(p, st, s.grad[(2 * g) * P + k], s.grad[(2 * g + 1) * P + k], f);
      for (int v = 0; v < 3; v++) vol[v] += lweight(g) * f[v];
    }
    double r[6];
    for (int v = 0; v < 3; v++) {
      const double fR = s.flux[v * P + k], fL = s.flux[v * P + k - 1];
      r[v] = -(fR - fL) * p.rdx;
      r[3 + v] = -(fL + fR) * (0.5 * p.rdx) + vol[v] * p.rdx;
    }
    if (p.source == HWENO1D_SOURCE_MMS51) {
      const double ri = sqrt(3.0 / 7.0 - 2.0 / 7.0 * sqrt(6.0 / 5.0)), ro = sqrt(3.0 / 7.0 + 2.0 / 7.0 * sqrt(6.0 / 5.0));
      const double wi = (18.0 + sqrt(30.0)) / 72.0, wo = (18.0 - sqrt(30.0)) / 72.0;
      const double nd[4] = {-0.5 * ro, -0.5 * ri, 0.5 * ri, 0.5 * ro}, wt[4] = {wo, wi, wi, wo};
      const double xc = p.x0 + (i + 0.5) * p.dx;
      for (int a = 0; a < 4; a++) {
        double S[3];
        mms_source(p, xc + nd[a] * p.dx, t, S);
        for (int v = 0; v < 3; v++) { r[v] += wt[a] * S[v]; r[3 + v] += wt[a] * nd[a] * S[v]; }
      }
    }
    for (int m = 0; m < 6; m++) rhs[m * n + i] = r[m];
    for (int v = 0; v < 3; v++) mom[v * n + i] = s.mom[v * P + k];
  }
  *alpha = amax;
  *beta = bmax;
}

static bool admissible_host(const Prob& p, const double* q) {
  for (int i = 0; i < p.n; i++) {
    const double u[3] = {q[i], q[p.n + i], q[2 * p.n + i]};
    if (!(u[0] > 0.0) || !(pressure(u, p.gamma) > 0.0)) return false;
  }
  return true;
}

int main(int argc, char** argv) {
  FILE* f = fopen(argv[1], "rb");
  int hdr[7];
  double dh[19];
  if (fread(hdr, sizeof(int), 7, f) != 7 || fread(dh, sizeof(double), 19, f) != 19) return 2;
  hweno1d_config c;
  hweno1d_config_default(&c);
  c.n = hdr[0]; c.bc[0] = hdr[1]; c.bc[1] = hdr[2]; c.scheme = hdr[3]; c.source = hdr[4]; c.max_halvings = hdr[5];
  const int mode = hdr[6];
  c.x0 = dh[0]; c.x1 = dh[1]; c.gamma = dh[2]; c.Pr = dh[3]; c.Re = dh[4]; c.cfl = dh[5]; c.b_visc = dh[6];
  c.eps_pp = dh[7]; c.eps_weno = dh[8];
  for (int k = 0; k < 6; k++) c.inflow[k / 3][k % 3] = dh[9 + k];
  const double t0 = dh[15], t_end = dh[16];
  const int max_steps = (int)dh[17];
  const int n = c.n;
  std::vector<double> q(6 * n), work(workspace_doubles(n));
  if (fread(q.data(), sizeof(double), 6 * n, f) != (size_t)(6 * n)) return 3;
  fclose(f);
  Prob p = make_prob(c, q.data(), work.data());
  Ptrs s = layout(p);
  FILE* o = fopen(argv[2], "wb");
  double alpha, beta;
  if (mode == 0) {
    residual_host(p, s, q.data(), t0, s.r0, s.m0, &alpha, &beta);
    fwrite(s.r0, sizeof(double), 6 * n, o);
    fwrite(s.m0, sizeof(double), 3 * n, o);
    double d[2] = {alpha, beta};
    fwrite(d, sizeof(double), 2, o);
  } else {
    double t = t0;
    int steps = 0, status = 0, rej_total = 0;
    while (t < t_end && steps < max_steps) {
      residual_host(p, s, p.q, t, s.r0, s.m0, &alpha, &beta);
      double dt = fmin(p.cfl * p.dx / alpha, p.visc_cap);
      if (t + dt > t_end) dt = t_end - t;
      int rej = 0;
      bool ok = false;
      for (int h = 0; h <= p.max_halvings; h++) {
        for (int i = 0; i < n; i++)
          for (int v = 0; v < 3; v++) {
            s.q1[v * n + i] = p.q[v * n + i] + dt * s.r0[v * n + i];
            s.q1[(3 + v) * n + i] = s.m0[v * n + i] + dt * s.r0[(3 + v) * n + i];
          }
        ok = admissible_host(p, s.q1);
        if (ok) {
          residual_host(p, s, s.q1, t + dt, s.r, s.m, &alpha, &beta);
          for (int i = 0; i < n; i++)
            for (int v = 0; v < 3; v++) {
              s.q2[v * n + i] = 0.75 * p.q[v * n + i] + 0.25 * (s.q1[v * n + i] + dt * s.r[v * n + i]);
              s.q2[(3 + v) * n + i] = 0.75 * s.m0[v * n + i] + 0.25 * (s.m[v * n + i] + dt * s.r[(3 + v) * n + i]);
            }
          ok = admissible_host(p, s.q2);
        }
        if (ok) {
          residual_host(p, s, s.q2, t + 0.5 * dt, s.r, s.m, &alpha, &beta);
          for (int i = 0; i < n; i++)
            for (int v = 0; v < 3; v++) {
              s.q3[v * n + i] = p.q[v * n + i] / 3.0 + 2.0 / 3.0 * (s.q2[v * n + i] + dt * s.r[v * n + i]);
              s.q3[(3 + v) * n + i] = s.m0[v * n + i] / 3.0 + 2.0 / 3.0 * (s.m[v * n + i] + dt * s.r[(3 + v) * n + i]);
            }
          ok = admissible_host(p, s.q3);
        }
        if (ok) break;
        rej++;
        dt *= 0.5;
      }
      if (!ok) { status = -3; break; }
      for (int i = 0; i < 6 * n; i++) p.q[i] = s.q3[i];
      t += dt;
      steps++;
      rej_total += rej;
      if (t_end - t <= 1e-14 * fmax(1.0, fabs(t_end))) t = t_end;
    }
    fwrite(p.q, sizeof(double), 6 * n, o);
    double d[4] = {t, (double)steps, (double)rej_total, (double)status};
    fwrite(d, sizeof(double), 4, o);
  }
  fclose(o);
  return 0;
}
