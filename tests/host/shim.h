// CUDA qualifiers, intrinsics and block primitives for running device code on the host
// (test infrastructure): one thread block of a kernel becomes a single host thread,
// shared memory is ordinary memory, barriers are no-ops, and a warp is one lane.  A
// shuffle returns zero, the contribution of the absent partner lanes: the neutral
// element of the sums and of the maxima of non-negative values (wave speeds) that the
// kernels reduce.  Warp votes and __syncthreads_or return the lane's own value, and the
// atomics are plain read-modify-writes.  With blockDim = 1 every block-strided loop of a
// kernel visits all its indices in order, so the kernel's own control flow and
// arithmetic run unchanged.
#pragma once
#include <cmath>
#include <cstring>

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __shared__
#define __grid_constant__
#define __launch_bounds__(...)

struct Dim3Shim {
  unsigned x, y, z;
};
static Dim3Shim threadIdx = {0, 0, 0}, blockIdx = {0, 0, 0}, blockDim = {1, 1, 1}, gridDim = {1, 1, 1};

static inline void __syncthreads() {}
static inline int __syncthreads_or(int v) { return v != 0; }
template <class T>
static inline T __shfl_xor_sync(unsigned, T, int) { return T(0); }
static inline unsigned __reduce_or_sync(unsigned, unsigned v) { return v; }
template <class T>
static inline T atomicAdd(T* a, T v) { const T o = *a; *a = o + v; return o; }
template <class T>
static inline T atomicOr(T* a, T v) { const T o = *a; *a = o | v; return o; }
template <class T>
static inline T atomicMax(T* a, T v) { const T o = *a; *a = o > v ? o : v; return o; }
static inline long long __double_as_longlong(double x) { long long b; memcpy(&b, &x, 8); return b; }
static inline int __double2hiint(double x) { return (int)(__double_as_longlong(x) >> 32); }
static inline double __longlong_as_double(long long b) { double x; memcpy(&x, &b, 8); return x; }
static inline unsigned __float_as_uint(float x) { unsigned b; memcpy(&b, &x, 4); return b; }
static inline float __int_as_float(int b) { float x; memcpy(&x, &b, 4); return x; }
static inline float __fdividef(float a, float b) { return a / b; }

using std::isfinite;
