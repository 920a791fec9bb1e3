// The mixed path's viscous gradients in one pass over a tile staged by the Tensor Memory
// Accelerator: face moments (Eq. (3.6)), weak-derivative moments (Eqs. (3.7)-(3.8)) and
// the gradient reconstruction (Eq. (3.9)), which the separate kernels
// k_face_moments_mixed, k_weak_moments_mixed and k_grad_mixed run through HBM.
//
// A block owns GT_X x GT_Y cells of the gradient region (the interior grown by 1).  One
// thread issues two tensor copies into shared memory: the FP32 traces (u, v, e) at the
// 12 face points of the tile and a 2-cell halo around it (a 4D box: x, y, variable,
// point, over the face group's float planes) and the cell means w-bar over the same
// box.  Every thread waits on the copies' mbarrier (a bounded wait: past its limit the
// block sets FLAG_TIMEOUT and returns).  The weak moments of the tile grown by 1 are
// then formed in shared memory from the face moments of each cell's four faces, and
// each thread reconstructs the six gradient components of its cell from them.  The
// operations of each quantity are those of the separate kernels in their order (the
// host build finds the gradients equal bit for bit; on the GPU the kernels' multiply-add
// fusions may differ, within FP32 rounding).
#pragma once
#ifdef __CUDACC__
#include <cuda.h>
#endif

#include "hweno_mixed.cuh"

namespace hw {

constexpr int GT_X = 32, GT_Y = 8, GT_THREADS = GT_X * GT_Y;
// the staged box: 40 columns from the padded column 32 * blockIdx.x (cells a - 3 .. a + 36
// for the tile origin a = -1 + 32 blockIdx.x, the start kept on a 16-byte boundary), and
// 12 rows from the tile's row b - 2
constexpr int GB_X = 40, GB_Y = GT_Y + 4;
constexpr int GR_X = GT_X + 2, GR_Y = GT_Y + 2;  // weak moments: the tile grown by 1
constexpr int GT_TR_FLOATS = 12 * 3 * GB_Y * GB_X;  // [point][u, v, e][row][column]
constexpr int GT_WB_FLOATS = 3 * GB_Y * GB_X;        // [u, v, e][row][column]
constexpr int GT_R_FLOATS = 18 * GR_Y * GR_X;        // [6 n + slot][row][column]
// dynamic shared memory: the three arrays from a 128-byte boundary of the block's region
// (whose base the launch guarantees only to 16 bytes), then the mbarrier
constexpr int GT_DATA_BYTES = 4 * (GT_TR_FLOATS + GT_WB_FLOATS + GT_R_FLOATS);
constexpr int GT_SMEM_BYTES = 128 + GT_DATA_BYTES + 16;
constexpr unsigned GT_TX_BYTES = 4u * (GT_TR_FLOATS + GT_WB_FLOATS);
static_assert((4 * GT_TR_FLOATS) % 128 == 0 && (4 * (GT_TR_FLOATS + GT_WB_FLOATS)) % 128 == 0,
              "each staged array starts on a 128-byte boundary");
static_assert(GR_X * GR_Y <= 2 * GT_THREADS, "two weak-moment cells per thread at most");

enum { FLAG_TIMEOUT = 8u };

// the tile's staged data: local column x = i - (a - 3), row y = j - (b - 2)
struct GradTile {
  const float* tr;  // [12][3][GB_Y][GB_X]
  const float* wb;  // [3][GB_Y][GB_X]
  float* r;         // [18][GR_Y][GR_X]
  __device__ __forceinline__ float trace(int k, int n, int y, int x) const {
    return tr[((k * 3 + n) * GB_Y + y) * GB_X + x];
  }
};

// the weak moments of cell (rx, ry) of the grown tile (cell (a - 1 + rx, b - 1 + ry)): the
// face moments of its four faces (Eq. (3.6)), then Eqs. (3.7)-(3.8), with the operations
// of face_moments_mixed_body and weak_moments_mixed_body
__device__ __forceinline__ void gradtile_weak_cell(const Grid& g, const GradTile& tt, int rx, int ry) {
  const int x = rx + 2, y = ry + 1;  // the cell's staged column and row
  // face moments of the x-face right of staged cell (xl, y) and of the y-face above (x, yb)
  auto wface = [&](int dir, int xl, int yl, float* W0, float* W1) {
    const int kl = dir == 0 ? 3 : 9, kr = dir == 0 ? 0 : 6;
    const int xr = dir == 0 ? xl + 1 : xl, yr = dir == 0 ? yl : yl + 1;
#pragma unroll
    for (int n = 0; n < 3; n++) W0[n] = W1[n] = 0.f;
#pragma unroll
    for (int gp = 0; gp < 3; gp++) {
      const float wg = gweight<float>(gp), xg = gnode<float>(gp);
#pragma unroll
      for (int n = 0; n < 3; n++) {
        const float av = tt.trace(kl + gp, n, yl, xl);
        const float bv = tt.trace(kr + gp, n, yr, xr);
        const float h = 0.5f * (av + bv);
        W0[n] += wg * h;
        W1[n] += wg * h * xg;
      }
    }
  };
  float xr0[3], xr1[3], xl0[3], xl1[3], yt0[3], yt1[3], yb0[3], yb1[3];
  wface(0, x, y, xr0, xr1);
  wface(0, x - 1, y, xl0, xl1);
  wface(1, x, y, yt0, yt1);
  wface(1, x, y - 1, yb0, yb1);
  const float rdx = g.rdxf, rdy = g.rdyf;
  const int plane = GR_Y * GR_X, at = ry * GR_X + rx;
#pragma unroll
  for (int n = 0; n < 3; n++) {
    const float wb = tt.wb[(n * GB_Y + y) * GB_X + x];
    float* r = tt.r + (6 * n) * plane + at;
    r[0] = (xr0[n] - xl0[n]) * rdx;
    r[plane] = (0.5f * (xr0[n] + xl0[n]) - wb) * rdx;
    r[2 * plane] = (xr1[n] - xl1[n]) * rdx;
    r[3 * plane] = (yt0[n] - yb0[n]) * rdy;
    r[4 * plane] = (yt1[n] - yb1[n]) * rdy;
    r[5 * plane] = (0.5f * (yt0[n] + yb0[n]) - wb) * rdy;
  }
}

// the six gradient components of tile cell (tx, ty), cell (i, j), from the staged weak
// moments, with the operations of grad_mixed_body (its volume sums for interior cells,
// from the weights wu, wv that vol_weights formed; VOLG: also the volume-point
// gradients); LIN: the linear weights (Remark 3.1)
template <bool LIN, bool VOLG = false>
__device__ __forceinline__ void gradtile_grad_cell(const Grid& g, const Work& w, const GradTile& tt, int tx,
                                                            int ty, int i, int j, const float* wu, const float* wv) {
  const WorkF f = mixed_planes(w, g.ps);
  const long long c = cidx(g, i, j);
  const float eps = g.eps_wenof;
  const bool interior = i >= 0 && i < g.nx && j >= 0 && j < g.ny;
  const int plane = GR_Y * GR_X;
  const int rx = tx + 1, ry = ty + 1;
#pragma unroll 1
  for (int comp = 0; comp < 6; comp++) {
    const int n = comp >> 1, l = comp & 1;
    const float* A = tt.r + (6 * n + 3 * l) * plane;
    const float* X = A + plane;
    const float* Y = A + 2 * plane;
    auto at = [&](int a, int b) { return (ry + b) * GR_X + (rx + a); };
    const float cen = A[at(0, 0)];
    float d[17];
#pragma unroll
    for (int b = -1; b <= 1; b++)
#pragma unroll
      for (int a = -1; a <= 1; a++) d[(b + 1) * 3 + (a + 1)] = A[at(a, b)] - cen;
    d[4] = 0.0f;
    d[9] = X[at(-1, 0)];
    d[10] = X[at(1, 0)];
    d[11] = Y[at(0, -1)];
    d[12] = Y[at(0, 1)];
    d[13] = X[at(0, -1)];
    d[14] = X[at(0, 1)];
    d[15] = Y[at(-1, 0)];
    d[16] = Y[at(1, 0)];
    float C[15];
    if constexpr (LIN)
      hw_p0_coeffs<float>(d, C);
    else
      hweno_combine<float>(d, eps, C);
    float vx[6], vy[6], vv[9];
    eval_xfaces<float>(C, vx);
    eval_yfaces<float>(C, vy);
    eval_vol<float>(C, vv);
    float* out = f.gr + (long long)comp * g.ps + c;
#pragma unroll
    for (int k = 0; k < 6; k++) out[(long long)(6 * k) * g.ps] = cen + vx[k];
#pragma unroll
    for (int k = 0; k < 6; k++) out[(long long)(6 * (6 + k)) * g.ps] = cen + vy[k];
    if constexpr (VOLG) {
#pragma unroll
      for (int k = 0; k < 9; k++) out[(long long)(6 * (12 + k)) * g.ps] = cen + vv[k];
    }
    if (interior) vol_visc_sums(g, f, c, comp, cen, vv, wu, wv);
  }
}

#ifdef __CUDACC__
// ---------------------------------------------------------------------------
// Tensor Memory Accelerator and mbarrier primitives (PTX ISA: cp.async.bulk.tensor,
// mbarrier).  One CTA is its own cluster here, so shared::cluster addresses are this
// CTA's shared memory.
__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
// one bounded attempt: true once the phase with this parity has completed
__device__ __forceinline__ bool mbar_try(unsigned bar, unsigned parity) {
  unsigned done;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(done)
      : "r"(bar), "r"(parity)
      : "memory");
  return done != 0;
}
// wait for the phase with at most `limit` attempts (each try_wait may itself suspend the
// thread for a while); false if it did not complete
__device__ __forceinline__ bool mbar_wait_bounded(unsigned bar, unsigned parity, long long limit) {
  for (long long k = 0; k < limit; k++)
    if (mbar_try(bar, parity)) return true;
  return false;
}
__device__ __forceinline__ void tma_load_4d(unsigned dst, const CUtensorMap* map, int x, int y, int z, int w,
                                            unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
      "[%6];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(w), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void tma_load_3d(unsigned dst, const CUtensorMap* map, int x, int y, int z, unsigned bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

// attempts of the bounded waits: far longer than any copy of a ~75 KB box takes
constexpr long long GT_WAIT_LIMIT = 1ll << 22;

// One tile of the gradient pass, tile (bx, by) of the gradient region: origin cell
// (a, b) = (-1 + GT_X bx, -1 + GT_Y by).  Thread 0 issues the two tensor copies on the
// block's mbarrier at b_addr (parity: the phase this use completes); while they fly every
// thread forms its cell's volume weights and inviscid sums (global loads); then each
// waits (bounded), the block forms the weak moments of the grown tile and each thread
// its cell's gradients.  Returns false when a wait gave up (FLAG_TIMEOUT set in diag):
// the block must stop.  The caller separates two uses of the shared tile by a barrier.
template <bool LIN>
__device__ __forceinline__ bool grad_tma_tile(const Grid& g, const Work& w, const CUtensorMap* tr_map,
                                              const CUtensorMap* wb_map, int bx, int by, float* gt_smem,
                                              unsigned b_addr, unsigned parity, Diag* diag) {
  const int t = threadIdx.x;
  const int a = -1 + GT_X * bx, b = -1 + GT_Y * by;  // tile origin (cell)
  if (t == 0) {
    mbar_expect_tx(b_addr, GT_TX_BYTES);
    // padded column 32 bx is cell a - 3; padded row b - 2 + NG; variables 1..3 (u, v, e)
    // of every point; the w-bar planes over the same columns and rows
    tma_load_4d(smem_addr(gt_smem), tr_map, GT_X * bx, b - 2 + NG, 1, 0, b_addr);
    tma_load_3d(smem_addr(gt_smem + GT_TR_FLOATS), wb_map, GT_X * bx, b - 2 + NG, 0, b_addr);
  }
  // while the copies are in flight: this thread's cell's volume values (global loads),
  // their weights for the viscous volume sums and the inviscid sums
  const int tx = t % GT_X, ty = t / GT_X;
  const int i = a + tx, j = b + ty;
  float wu[9], wv[9];
  if (i >= 0 && i < g.nx && j >= 0 && j < g.ny) vol_weights(g, mixed_planes(w, g.ps), cidx(g, i, j), wu, wv);
  if (!mbar_wait_bounded(b_addr, parity, GT_WAIT_LIMIT)) {
    if (t == 0) {
      atomicOr(&diag->flags, FLAG_TIMEOUT);
      mbar_wait_bounded(b_addr, parity, GT_WAIT_LIMIT);  // the copies may still land: give them time
    }
    return false;
  }
  GradTile tt{gt_smem, gt_smem + GT_TR_FLOATS, gt_smem + GT_TR_FLOATS + GT_WB_FLOATS};
  for (int k = t; k < GR_X * GR_Y; k += GT_THREADS) gradtile_weak_cell(g, tt, k % GR_X, k / GR_X);
  __syncthreads();
  if (i < g.nx + 1 && j < g.ny + 1) gradtile_grad_cell<LIN>(g, w, tt, tx, ty, i, j, wu, wv);
  return true;
}

// the block's staged tile (from a 128-byte boundary of the dynamic shared memory, whose
// base the launch guarantees only to 16 bytes) and its mbarrier after it, initialised by
// thread 0 (one arrival per phase)
__device__ __forceinline__ float* grad_tma_smem(unsigned char* raw, unsigned* b_addr) {
  float* gt_smem = (float*)(((unsigned long long)raw + 127) & ~127ull);
  *b_addr = smem_addr((unsigned char*)gt_smem + GT_DATA_BYTES);
  if (threadIdx.x == 0) mbar_init(*b_addr, 1);
  __syncthreads();
  return gt_smem;
}

template <bool LIN = false>
__global__ void __launch_bounds__(GT_THREADS) k_grad_tma_mixed(Grid g, Work w, const __grid_constant__ CUtensorMap tr_map,
                                                               const __grid_constant__ CUtensorMap wb_map, Diag* diag) {
  extern __shared__ __align__(16) unsigned char gt_raw[];
  unsigned b_addr;
  float* gt_smem = grad_tma_smem(gt_raw, &b_addr);
  grad_tma_tile<LIN>(g, w, &tr_map, &wb_map, (int)blockIdx.x, (int)blockIdx.y, gt_smem, b_addr, 0u, diag);
}
#endif

}  // namespace hw
