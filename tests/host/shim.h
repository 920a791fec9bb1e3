// CUDA qualifiers and block primitives for running device code on the host (test
// infrastructure): one thread block of a kernel becomes a single host thread, barriers
// are no-ops, a warp shuffle returns the lane's own value (a one-lane warp), and
// __syncthreads_or returns its argument.  With blockDim.x = 1 every block-strided loop
// of a kernel visits all its indices in order, so the kernel's own control flow and
// arithmetic run unchanged.
#pragma once
#include <cmath>
#include <cstring>

#define __global__
#define __device__
#define __host__
#define __forceinline__ inline
#define __shared__ static
#define __launch_bounds__(...)

struct Dim3Shim {
  unsigned x, y, z;
};
static Dim3Shim threadIdx = {0, 0, 0}, blockIdx = {0, 0, 0}, blockDim = {1, 1, 1};

static inline void __syncthreads() {}
static inline int __syncthreads_or(int v) { return v != 0; }
static inline double __shfl_xor_sync(unsigned, double v, int) { return v; }

using std::isfinite;
