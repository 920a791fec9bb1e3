// Generated by gen_stencil1d.py (exact rationals via sympy); do not edit.
// One-dimensional unified-stencil HWENO constants of Appendix A.1 as straight-line code.
#pragma once

// p0 coefficients (xi^0..xi^4) from the five stencil data
template <class T> __host__ __device__ __forceinline__ void hw1_p0_coeffs(const T* d, T* c) {
  c[0] = T(-0.11197916666666667) * d[0] + T(1.2239583333333333) * d[1] + T(-0.11197916666666667) * d[2] + T(-0.421875) * d[3] + T(0.421875) * d[4];
  c[1] = T(-0.8289473684210527) * d[0] + T(0.8289473684210527) * d[2] + T(-3.9473684210526314) * d[3] + T(-3.9473684210526314) * d[4];
  c[2] = T(1.4375) * d[0] + T(-2.875) * d[1] + T(1.4375) * d[2] + T(5.625) * d[3] + T(-5.625) * d[4];
  c[3] = T(0.2631578947368421) * d[0] + T(-0.2631578947368421) * d[2] + T(3.1578947368421053) * d[3] + T(3.1578947368421053) * d[4];
  c[4] = T(-0.625) * d[0] + T(1.25) * d[1] + T(-0.625) * d[2] + T(-3.75) * d[3] + T(3.75) * d[4];
}

// smoothness indicator of a quartic: sum over orders 1..4 of the cell integral of the
// squared derivative (a quadratic form in its coefficients)
template <class T> __host__ __device__ __forceinline__ T hw1_beta_quartic(const T* c) {
  T s = T(0);
  s += T(1.0) * c[1] * c[1];
  s += T(0.5) * c[1] * c[3];
  s += T(4.333333333333333) * c[2] * c[2];
  s += T(4.2) * c[2] * c[4];
  s += T(39.1125) * c[3] * c[3];
  s += T(625.8357142857143) * c[4] * c[4];
  return s;
}

// modified moment int xi p(xi) over the centre cell of a quartic
template <class T> __host__ __device__ __forceinline__ T hw1_moment(const T* c) {
  return T(0.08333333333333333) * c[1] + T(0.0125) * c[3];
}
