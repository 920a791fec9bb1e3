// The state's layout in HBM and its ghost cells (Remark 4.1), as functions that compile
// for the device and, through a qualifier shim, for the host, so that the ghost rules
// can be run on the CPU against an independent implementation.
//
//   padded plane: (ny + 8) rows x pitch doubles, pitch = nx + 8 rounded up to a
//   multiple of 16 (128-byte rows); cell (i, j), i in [-4, nx+4), j in [-4, ny+4),
//   sits at (j + 4) * pitch + (i + 4).  Plane 4 m + v holds moment m (average,
//   xi-moment, eta-moment) of conserved variable v (rho, rho u, rho v, E).
#pragma once
#include <math.h>
#include <string.h>

#include "hweno.h"

namespace hw {

constexpr int NG = 4;  // ghost layers

struct Grid {
  int nx, ny, pitch;
  long long ps;  // plane stride in doubles
  double dx, dy;
  double gamma, Pr, Re;
  double eps_pp, eps_weno;
  int bc[4];
  double rdx, rdy, rPr, rRe;  // 1/dx, 1/dy, 1/Pr, 1/Re (correctly rounded, on the host)
  double x0, y0;              // domain origin (coordinates of a source term and of inflow bands)
  // the mixed path's single-precision copies (rounded on the host: a per-thread conversion
  // would occupy the FP64 pipe)
  float gammaf, rPrf, rRef, rdxf, rdyf, eps_wenof;
};

// prescribed states of HWENO_BC_INFLOW faces (Remark 4.1): per face (xlo, xhi, ylo,
// yhi), the conserved state inside [0] and outside [1] the band |s - centre| < half
// width, s the ghost cell centre's coordinate along the face
struct Open {
  double state[4][2][4];
  double band[4][2];
};

// the grid of a configuration: padded pitch and plane stride, spacings and their
// reciprocals (correctly rounded on the host), gas constants, faces and origin
inline Grid make_grid(const hweno_config& c) {
  Grid g;
  g.nx = c.nx;
  g.ny = c.ny;
  g.pitch = ((c.nx + 2 * NG + 15) / 16) * 16;
  g.ps = (long long)(c.ny + 2 * NG) * g.pitch;
  g.dx = (c.x1 - c.x0) / c.nx;
  g.dy = (c.y1 - c.y0) / c.ny;
  g.gamma = c.gamma; g.Pr = c.Pr; g.Re = c.Re;
  g.eps_pp = c.eps_pp; g.eps_weno = c.eps_weno;
  for (int k = 0; k < 4; k++) g.bc[k] = c.bc[k];
  g.rdx = 1.0 / g.dx; g.rdy = 1.0 / g.dy; g.rPr = 1.0 / g.Pr; g.rRe = 1.0 / g.Re;
  g.x0 = c.x0; g.y0 = c.y0;
  g.gammaf = (float)g.gamma; g.rPrf = (float)g.rPr; g.rRef = (float)g.rRe;
  g.rdxf = (float)g.rdx; g.rdyf = (float)g.rdy; g.eps_wenof = (float)g.eps_weno;
  return g;
}

// the prescribed states of a configuration's inflow faces
inline Open make_open(const hweno_config& c) {
  Open o;
  memcpy(o.state, c.inflow, sizeof(o.state));
  memcpy(o.band, c.band, sizeof(o.band));
  return o;
}

__host__ __device__ __forceinline__ long long cidx(const Grid& g, int i, int j) {
  return (long long)(j + NG) * g.pitch + (i + NG);
}

// x0 + (k + 1/2) d with both operations rounded as written (never contracted), so
// that a band test sees the same coordinate wherever it is computed
__host__ __device__ __forceinline__ double centre(double x0, int k, double d) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(x0, __dmul_rn(k + 0.5, d));
#else
  return x0 + (k + 0.5) * d;
#endif
}

// bit casts and a leading-zero count: the device intrinsics, or their host forms
__host__ __device__ __forceinline__ unsigned long long bits_of(double x) {
#ifdef __CUDA_ARCH__
  return (unsigned long long)__double_as_longlong(x);
#else
  unsigned long long b;
  memcpy(&b, &x, sizeof(b));
  return b;
#endif
}
__host__ __device__ __forceinline__ float float_of(unsigned int b) {
#ifdef __CUDA_ARCH__
  return __int_as_float((int)b);
#else
  float f;
  memcpy(&f, &b, sizeof(f));
  return f;
#endif
}
__host__ __device__ __forceinline__ double double_of(unsigned long long b) {
#ifdef __CUDA_ARCH__
  return __longlong_as_double((long long)b);
#else
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
#endif
}
__host__ __device__ __forceinline__ unsigned int bits_of_f(float x) {
#ifdef __CUDA_ARCH__
  return (unsigned int)__float_as_int(x);
#else
  unsigned int b;
  memcpy(&b, &x, sizeof(b));
  return b;
#endif
}

// single roundings that the compiler may not fuse into multiply-adds: an expression
// written with these (and fmaf / fma) rounds the same way in every kernel that inlines it
__host__ __device__ __forceinline__ float add_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ float mul_rn(float a, float b) {
#ifdef __CUDA_ARCH__
  return __fmul_rn(a, b);
#else
  return a * b;
#endif
}
__host__ __device__ __forceinline__ double dadd_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dadd_rn(a, b);
#else
  return a + b;
#endif
}
__host__ __device__ __forceinline__ double dmul_rn(double a, double b) {
#ifdef __CUDA_ARCH__
  return __dmul_rn(a, b);
#else
  return a * b;
#endif
}

__host__ __device__ __forceinline__ int clz32(unsigned int r) {  // r != 0
#ifdef __CUDA_ARCH__
  return __clz((int)r);
#else
  return __builtin_clz(r);
#endif
}

// Conversions between float values and their FP64 planes in integer operations only:
// on B300 the FP64 pipe also carries float/double conversions, and a conversion left in
// a rarely taken branch is often evaluated for every value and selected afterwards.

// x widened to double: the same value, exactly, for every float (subnormal ones
// normalised; infinities and NaN, whose payload is kept, to their doubles)
__host__ __device__ __forceinline__ double widen_f(float x) {
  const unsigned int b = bits_of_f(x);
  const unsigned int e = (b >> 23) & 0xffu, m = b & 0x7fffffu;
  const unsigned long long s = (unsigned long long)(b & 0x80000000u) << 32;
  if (e == 0u) {
    if (m == 0u) return double_of(s);
    const int sh = clz32(m) - 8;  // brings the leading bit to position 23
    return double_of(s | ((unsigned long long)(897 - sh) << 52) | ((unsigned long long)((m << sh) & 0x7fffffu) << 29));
  }
  const unsigned long long ed = e == 0xffu ? 0x7ffull : (unsigned long long)(e + 896u);
  return double_of(s | (ed << 52) | ((unsigned long long)m << 29));
}

// x truncated to a float: its sign, exponent and leading 23 mantissa bits in the normal
// float range, the truncated subnormal below it (zero below 2^-149), infinity beyond
// it; NaN stays NaN.  Exact for a double that holds a float value.
__host__ __device__ __forceinline__ float narrow_trunc(double x) {
  const unsigned long long b = bits_of(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7ff);
  const unsigned long long m = b & 0xfffffffffffffull;
  const int fe = E - 896;
  if (fe >= 1 && fe <= 254) return float_of(sign | ((unsigned int)fe << 23) | (unsigned int)(m >> 29));
  if (E == 0x7ff) {  // infinity; NaN keeps its leading payload bits (a quiet bit if none is left)
    const unsigned int pl = (unsigned int)(m >> 29);
    return float_of(sign | 0x7f800000u | (m == 0ull ? 0u : (pl != 0u ? pl : 0x400000u)));
  }
  if (fe > 254) return float_of(sign | 0x7f800000u);
  const int sh = 30 - fe;  // the subnormal's integer mantissa is (2^52 + m) >> sh
  return float_of(sign | (sh < 64 ? (unsigned int)((m | (1ull << 52)) >> sh) : 0u));
}

// a double that holds a float value, narrowed to that float (exactly)
__host__ __device__ __forceinline__ float narrow_exact(double x) { return narrow_trunc(x); }

// hi/lo split of a state value, with integer operations only: hi keeps the sign, the
// exponent and the leading 23 mantissa bits of x (truncation), lo is the float nearest
// below the exact remainder x - hi (the trailing 29 mantissa bits, normalised).  Zero
// gives (0, 0); magnitudes below 2^-74 or beyond the float range take hi =
// narrow_trunc(x), lo = 0.
__host__ __device__ __forceinline__ void split_hilo(double x, float& hi, float& lo) {
  const unsigned long long b = bits_of(x);
  const unsigned int sign = (unsigned int)(b >> 32) & 0x80000000u;
  const int E = (int)((b >> 52) & 0x7ff);
  const int fe = E - 1023 + 127;
  if (E == 0) {  // zero (or a double denormal, below any float): signed zero
    hi = float_of(sign);
    lo = 0.0f;
    return;
  }
  // the remainder's float exponent field is fe - 52 + top >= fe - 52: keep it >= 1
  if (fe < 53 || fe > 254) {  // |x| < 2^-74, beyond the float range, inf or nan
    hi = narrow_trunc(x);
    lo = 0.0f;
    return;
  }
  const unsigned long long m = b & 0xfffffffffffffull;
  hi = float_of(sign | ((unsigned int)fe << 23) | (unsigned int)(m >> 29));
  const unsigned int r = (unsigned int)(m & 0x1fffffffull);  // remainder: r * 2^(E - 1075)
  if (r == 0u) {
    lo = 0.0f;
    return;
  }
  const int top = 31 - clz32(r);  // highest set bit, 0..28
  const int le = fe - 52 + top;   // float exponent field of the remainder
  const unsigned int mant = top >= 23 ? (r >> (top - 23)) : (r << (23 - top));
  lo = float_of(sign | ((unsigned int)le << 23) | (mant & 0x7fffffu));
}

// ---------------------------------------------------------------------------
// ghost cells (Remark 4.1).  x pass over the interior rows, then y pass over the
// full padded width from interior rows, so that a corner takes the y rule applied to
// the x rule's column: the product of two mirror parities, a y-face inflow state
// across its whole ghost row, an x-face inflow state (with the y mirror's parity) at
// the row the y rule maps to.
// Mirror across a face with parity s per variable: ghost average = s * average,
// moment normal to the face = -s * moment, tangential moment = s * moment.  Outflow
// copies the adjacent interior cell (average and moments); inflow holds the face's
// prescribed state with zero moments.
__host__ __device__ __forceinline__ double bc_sign(int bc, int normal_dir, int v) {
  if (v == 0 || v == 3) return 1.0;
  if (bc == HWENO_BC_NOSLIP) return -1.0;     // no-slip: both momenta odd
  return (v == 1 + normal_dir) ? -1.0 : 1.0;  // symmetry/slip: normal momentum odd
}

// the source index of ghost index k (k < 0 or k >= n) along a direction of n cells
__host__ __device__ __forceinline__ int ghost_src(int bc, int k, int n) {
  if (bc == HWENO_BC_PERIODIC) return k < 0 ? ((k % n) + n) % n : k % n;
  if (bc == HWENO_BC_OUTFLOW) return k < 0 ? 0 : n - 1;
  return k < 0 ? -1 - k : 2 * n - 1 - k;  // mirror
}

__host__ __device__ __forceinline__ bool is_mirror(int bc) {
  return bc == HWENO_BC_NOSLIP || bc == HWENO_BC_SYMMETRY || bc == HWENO_BC_SLIP;
}

// value of inflow plane p: the FP64 state itself, or on the float planes of the
// hi/lo split (planes 0..11 hi, 12..23 lo) the part that split_hilo gives
__host__ __device__ __forceinline__ double open_value(double x, int, const double*) { return x; }
__host__ __device__ __forceinline__ float open_value(double x, int p, const float*) {
  float hi, lo;
  split_hilo(x, hi, lo);
  return p < 12 ? hi : lo;
}

// the inflow state of face f for a ghost cell centred at s along the face
__host__ __device__ __forceinline__ const double* inflow_state(const Open& o, int f, double s) {
  return o.state[f][fabs(s - o.band[f][0]) < o.band[f][1] ? 0 : 1];
}

// planes [p0, p1) of the state (plane 4 m + v: moment m of variable v), or of its
// hi/lo split (24 float planes, of which the mixed path keeps 16: plane p holds state
// plane p mod 12).  o may be NULL
// where no face is an inflow face.
template <class E>
__host__ __device__ __forceinline__ void ghost_x_body(const Grid& g, const Open* o, E* q, int t, int p0 = 0,
                                                      int p1 = 12) {
  // t over 8 ghost columns x ny rows
  if (t >= 8 * g.ny) return;
  const int j = t / 8, c = t % 8;
  const int side = c / 4, k = c % 4;  // side 0: i = -1-k, side 1: i = nx+k
  const int i = side == 0 ? -1 - k : g.nx + k;
  const int bc = g.bc[side];
  const long long d = cidx(g, i, j);
  if (bc == HWENO_BC_INFLOW) {
    if (!o) return;
    const double* st = inflow_state(*o, side, centre(g.y0, j, g.dy));
    for (int p = p0; p < p1; p++) q[p * g.ps + d] = (p % 12) < 4 ? E(open_value(st[p & 3], p, q)) : E(0);
    return;
  }
  const long long s = cidx(g, ghost_src(bc, i, g.nx), j);
  const bool mir = is_mirror(bc);
  for (int p = p0; p < p1; p++) {
    const int m = (p % 12) >> 2, v = p & 3;
    E sg = E(1);
    if (mir) sg = E(bc_sign(bc, 0, v) * (m == 1 ? -1.0 : 1.0));
    q[p * g.ps + d] = sg * q[p * g.ps + s];
  }
}

template <class E>
__host__ __device__ __forceinline__ void ghost_y_body(const Grid& g, const Open* o, E* q, int t, int p0 = 0,
                                                      int p1 = 12) {
  // t over 8 ghost rows x padded width
  const int W = g.nx + 2 * NG;
  if (t >= 8 * W) return;
  const int r = t / W, i = t % W - NG;
  const int side = r / 4, k = r % 4;
  const int j = side == 0 ? -1 - k : g.ny + k;
  const int bc = g.bc[2 + side];
  const long long d = cidx(g, i, j);
  if (bc == HWENO_BC_INFLOW) {
    if (!o) return;
    const double* st = inflow_state(*o, 2 + side, centre(g.x0, i, g.dx));
    for (int p = p0; p < p1; p++) q[p * g.ps + d] = (p % 12) < 4 ? E(open_value(st[p & 3], p, q)) : E(0);
    return;
  }
  const long long s = cidx(g, i, ghost_src(bc, j, g.ny));
  const bool mir = is_mirror(bc);
  for (int p = p0; p < p1; p++) {
    const int m = (p % 12) >> 2, v = p & 3;
    E sg = E(1);
    if (mir) sg = E(bc_sign(bc, 1, v) * (m == 2 ? -1.0 : 1.0));
    q[p * g.ps + d] = sg * q[p * g.ps + s];
  }
}

// Both passes in one launch: thread t < 8 ny fills an x ghost as ghost_x_body does; the
// others fill the y ghosts as ghost_y_body does, except that a corner's source cell,
// an x ghost that the x pass writes in the same launch, is formed here by the x rule
// instead of read (the same operations on the same interior value, so the result equals
// the two passes' bit for bit).  The two parts write disjoint cells and read interior
// cells only.
template <class E>
__host__ __device__ __forceinline__ void ghost_xy_body(const Grid& g, const Open* o, E* q, int t, int p0 = 0,
                                                       int p1 = 12) {
  if (t < 8 * g.ny) {
    ghost_x_body(g, o, q, t, p0, p1);
    return;
  }
  t -= 8 * g.ny;
  const int W = g.nx + 2 * NG;
  if (t >= 8 * W) return;
  const int r = t / W, i = t % W - NG;
  const int side = r / 4, k = r % 4;
  const int j = side == 0 ? -1 - k : g.ny + k;
  const int bc = g.bc[2 + side];
  if (bc == HWENO_BC_INFLOW || (i >= 0 && i < g.nx)) {
    ghost_y_body(g, o, q, t, p0, p1);
    return;
  }
  // a corner: the y rule applied to the x rule's value at the source row js
  const long long d = cidx(g, i, j);
  const int js = ghost_src(bc, j, g.ny);
  const int xside = i < 0 ? 0 : 1, bcx = g.bc[xside];
  const bool mir = is_mirror(bc), mirx = is_mirror(bcx);
  const double* st = nullptr;
  if (bcx == HWENO_BC_INFLOW) {
    if (!o) return;
    st = inflow_state(*o, xside, centre(g.y0, js, g.dy));
  }
  const long long sx = bcx == HWENO_BC_INFLOW ? 0 : cidx(g, ghost_src(bcx, i, g.nx), js);
  for (int p = p0; p < p1; p++) {
    const int m = (p % 12) >> 2, v = p & 3;
    E src;
    if (st) {
      src = (p % 12) < 4 ? E(open_value(st[p & 3], p, q)) : E(0);
    } else {
      E sgx = E(1);
      if (mirx) sgx = E(bc_sign(bcx, 0, v) * (m == 1 ? -1.0 : 1.0));
      src = sgx * q[p * g.ps + sx];
    }
    E sg = E(1);
    if (mir) sg = E(bc_sign(bc, 1, v) * (m == 2 ? -1.0 : 1.0));
    q[p * g.ps + d] = sg * src;
  }
}

}  // namespace hw
