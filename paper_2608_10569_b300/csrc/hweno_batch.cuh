// Batched kernels: one launch of each spatial-operator kernel advances every case of an
// ensemble of independent problems with their own grids.  Blocks are persistent: a grid
// sized to the SMs loops over a work list of (case, tile) items, where a case's tiles
// cover that kernel's launch region.  The per-cell work is the single-grid bodies.
#pragma once
#include "hweno_mixed.cuh"
#include "hweno_source.cuh"
#include "hweno_tma.cuh"

namespace hw {

// device description of one case of a batch
struct CaseDev {
  Grid g;
  Work w;
  double *Q, *QS, *BASE, *RHS0, *RHS, *MOM0, *MOM;
  Diag* diag;
  double cfl, hmin, visc_cap;  // time-step rule of Sec. 5
  double dt_scale;             // 1, or 2^-k after k restarts of this step
  int active;                  // 0: the case does no work in this launch
  int split_ok;                // mixed: the kept split planes hold the split of Q (the last
                               // accepted stage update wrote them), so stage 1 needs no split pass
  Open open;                   // prescribed states of the case's inflow faces
  Quad4 quad;                  // the source term's Gauss rule
  double t;                    // the case's time at the start of the step
  int source;                  // HWENO_SOURCE_* of the case
  int pad2;
};

// work list of one kernel: case c owns items [start[c], start[c+1]); its tiles are
// tx[c] x ty[c] per z-slice of the launch region
struct TileList {
  const int* start;
  const int* tx;
  const int* ty;
};

__device__ __forceinline__ int find_case(const int* start, int ncase, int t) {
  int lo = 0, hi = ncase - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (start[mid] <= t) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// position of this thread in case c's launch region for work item t
__device__ __forceinline__ void tile_pos(const TileList& L, int c, int t, int& gx, int& gy, int& gz) {
  int l = t - L.start[c];
  const int per = L.tx[c] * L.ty[c];
  gz = l / per;
  l -= gz * per;
  const int by = l / L.tx[c], bx = l - by * L.tx[c];
  gx = bx * blockDim.x + threadIdx.x;
  gy = by * blockDim.y + threadIdx.y;
}

// the batch's work lists, one per kind of launch region
enum { BR_CONS = 0, BR_FACE, BR_WEAK, BR_GRAD, BR_FLUX, BR_INT, BR_GHOST, BR_SPLIT, BR_FR, BR_FRA, BR_GT, BR_N };

// launch-region extents (x, y, z) of list kind k for a grid: those of the single-grid
// kernel the kind stands for
inline void batch_region(int k, const Grid& g, int& wx, int& wy, int& wz) {
  wz = 1;
  switch (k) {
    case BR_CONS: wx = g.nx + 6; wy = g.ny + 6; break;
    case BR_FACE: wx = g.nx + 5; wy = g.ny + 5; wz = 2; break;
    case BR_WEAK: wx = g.nx + 4; wy = g.ny + 4; break;
    case BR_GRAD: case BR_GT: wx = g.nx + 2; wy = g.ny + 2; break;
    case BR_FLUX: wx = g.nx + 1; wy = g.ny + 1; wz = 2; break;
    case BR_INT: case BR_FR: case BR_FRA: wx = g.nx; wy = g.ny; break;
    case BR_GHOST: wx = 8 * g.ny + 8 * (g.nx + 2 * NG); wy = 1; break;
    default: wx = (int)(12 * g.ps); wy = 1; break;  // BR_SPLIT
  }
}

// the work list of kind k over n cases with bx x by tiles, as TileList reads it:
// out[c] the first item of case c and out[n] the total, out[n + 1 + c] and
// out[2n + 1 + c] the case's tiles across and down (3n + 1 ints); grid_of(c) gives
// case c's grid.  Returns the total.
template <class GridOf>
inline int batch_layout(int k, int n, GridOf grid_of, int bx, int by, int* out) {
  int total = 0;
  for (int c = 0; c < n; c++) {
    int wx, wy, wz;
    batch_region(k, grid_of(c), wx, wy, wz);
    const int tx = (wx + bx - 1) / bx, ty = (wy + by - 1) / by;
    out[c] = total;
    out[n + 1 + c] = tx;
    out[2 * n + 1 + c] = ty;
    total += tx * ty * wz;
  }
  out[n] = total;
  return total;
}

#define HW_BATCH_LOOP(L, ncase)                                   \
  const int total_ = (L).start[ncase];                             \
  for (int t_ = blockIdx.x; t_ < total_; t_ += gridDim.x) {        \
    const int c_ = find_case((L).start, ncase, t_);                \
    const CaseDev& cd = cases[c_];                                 \
    if (!cd.active) continue;                                      \
    const Grid cg = cd.g; /* local copies: the bodies' stores to */ \
    const Work cw = cd.w; /* the planes cannot alias them */       \
    int gx, gy, gz;                                                \
    tile_pos(L, c_, t_, gx, gy, gz);                               \
    (void)gz;

#define HW_BATCH_END }

// which = 0: stage 1 (state Q, residual into RHS0/MOM0); 1: stages 2, 3 (QS -> RHS/MOM).
// DR (FP64): also store the characteristic combinations HWENO-DR differentiates
template <int MIXED, bool DR = false>
__global__ void __launch_bounds__(128, MIXED ? 3 : 1) kb_cons(const CaseDev* __restrict__ cases, TileList L, int ncase, int which) {
  HW_BATCH_LOOP(L, ncase)
  const double* q = which == 0 ? cd.Q : cd.QS;
  double* mom = which == 0 ? cd.MOM0 : cd.MOM;
  if (MIXED) cons_mixed_body(cg, q, cw, mom, cd.diag, gx, gy);
  else if (DR) cons_body<double, false, true>(cg, q, cw, mom, cd.diag, gx, gy);
  else cons_body<double>(cg, q, cw, mom, cd.diag, gx, gy);
  HW_BATCH_END
}

// HWENO-DR gradients (Eq. (3.5)) in place of the face moments, weak moments and gradient
// reconstruction: blocks of DR_THREADS threads with DR_SMEM_BYTES of shared memory
__global__ void __launch_bounds__(DR_THREADS) kb_dr(const CaseDev* __restrict__ cases, TileList L, int ncase,
                                                    int which) {
  HW_BATCH_LOOP(L, ncase)
  dr_body(cg, which == 0 ? cd.Q : cd.QS, cw, gx, gy);
  HW_BATCH_END
}

template <int MIXED>
__global__ void kb_face_moments(const CaseDev* __restrict__ cases, TileList L, int ncase) {
  HW_BATCH_LOOP(L, ncase)
  if (MIXED) face_moments_mixed_body(cg, cw, gx, gy, gz);
  else face_moments_body(cg, cw, gx, gy, gz);
  HW_BATCH_END
}

template <int MIXED>
__global__ void kb_weak_moments(const CaseDev* __restrict__ cases, TileList L, int ncase) {
  HW_BATCH_LOOP(L, ncase)
  if (MIXED) weak_moments_mixed_body(cg, cw, gx, gy);
  else weak_moments_body(cg, cw, gx, gy);
  HW_BATCH_END
}

// LIN: the linear weights in the gradient reconstruction (Remark 3.1's ablation)
template <int MIXED, bool LIN = false>
__global__ void __launch_bounds__(128) kb_grad(const CaseDev* __restrict__ cases, TileList L, int ncase) {
  HW_BATCH_LOOP(L, ncase)
  if (MIXED) grad_mixed_body<LIN>(cg, cw, gx, gy);
  else grad_body<double, false, LIN>(cg, cw, gx, gy);
  HW_BATCH_END
}

// the FP64 face fluxes and balances (a mixed batch runs them in the flux tile kernels below)
__global__ void __launch_bounds__(128) kb_flux(const CaseDev* __restrict__ cases, TileList L, int ncase) {
  HW_BATCH_LOOP(L, ncase)
  flux_body<double>(cg, cw, cd.diag, gx, gy, gz);
  HW_BATCH_END
}

__global__ void __launch_bounds__(128) kb_assemble(const CaseDev* __restrict__ cases, TileList L, int ncase,
                                                   int which) {
  HW_BATCH_LOOP(L, ncase)
  double* rhs = which == 0 ? cd.RHS0 : cd.RHS;
  assemble_body<double>(cg, cw, rhs, cd.diag, gx, gy);
  HW_BATCH_END
}

// Example 5.2's manufactured source of the cases that have it, added to the residual at
// the stage time t + cst * dt (dt of the current attempt, read on the device)
__global__ void __launch_bounds__(128) kb_source(const CaseDev* __restrict__ cases, TileList L, int ncase,
                                                 int which, double cst) {
  HW_BATCH_LOOP(L, ncase)
  if (cd.source == HWENO_SOURCE_MMS52)
    source_body(cg, cd.quad, cd.t, cst, cd.diag, which == 0 ? cd.RHS0 : cd.RHS, gx, gy);
  HW_BATCH_END
}

// MIXED: also the hi/lo split of the new state (the next stage's evaluation then needs
// no split pass)
template <int MIXED>
__global__ void __launch_bounds__(128) kb_rk(const CaseDev* __restrict__ cases, TileList L, int ncase, int stage) {
  HW_BATCH_LOOP(L, ncase)
  float* hilo = MIXED ? mixed_planes(cw, cg.ps).hilo : nullptr;
  if (stage == 1) rk_body<MIXED != 0>(cg, 1, cd.Q, cd.MOM0, cd.RHS0, cd.BASE, cd.QS, cd.diag, gx, gy, hilo);
  else rk_body<MIXED != 0>(cg, stage, cd.QS, cd.MOM, cd.RHS, cd.BASE, cd.QS, cd.diag, gx, gy, hilo);
  HW_BATCH_END
}

// stages 2 and 3 of a mixed batch, after the gradients: k_flux_rk_mixed's tile (the
// face sums of FR_TX x FR_TY cells in shared memory, then the balances and the in-place
// stage update of QS) over a work list of (case, tile) items, the same arithmetic as a
// single handle's stage
__global__ void __launch_bounds__(FR_THREADS, HWENO_FR_MIN_BLOCKS) kb_flux_rk_mixed(const CaseDev* __restrict__ cases, TileList L,
                                                                int ncase, int stage) {
  __shared__ FluxTile ft;
  const int total = L.start[ncase];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int c = find_case(L.start, ncase, item);
    const CaseDev& cd = cases[c];
    if (!cd.active) continue;  // the same for every thread of the block
    const Grid cg = cd.g;
    const Work cw = cd.w;
    const int l = item - L.start[c];
    const int by = l / L.tx[c], bx = l - by * L.tx[c];
    const int i0 = bx * FR_TX, j0 = by * FR_TY;
    const WorkF f = mixed_planes(cw, cg.ps);
    float amax = 0.f, bmax = 0.f;
    flux_tile_faces(cg, f, i0, j0, threadIdx.x, ft, amax, bmax);
    flux_tile_reduce(amax, bmax, cd.diag);
    __syncthreads();
    double kef = 0.0;
    const unsigned int bad = flux_tile_cell<false>(cg, f, i0, j0, threadIdx.x, ft, stage, cd.diag->dt, cd.QS,
                                                   cd.MOM, cd.BASE, cd.QS, mixed_planes(cw, cg.ps).hilo, kef);
    rk_reduce<false>(stage, bad, kef, cd.diag);
    __syncthreads();  // the next item writes the tile again
  }
}

// the fluxes and balances of a mixed batch's kept residual (stage 1: RHS0; a stage with
// a source term: RHS), k_flux_asm_mixed's tile over the same work list
__global__ void __launch_bounds__(FR_THREADS, HWENO_FR_MIN_BLOCKS) kb_flux_asm_mixed(const CaseDev* __restrict__ cases, TileList L,
                                                                 int ncase, int which) {
  __shared__ FluxTile ft;
  const int total = L.start[ncase];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int c = find_case(L.start, ncase, item);
    const CaseDev& cd = cases[c];
    if (!cd.active) continue;  // the same for every thread of the block
    const Grid cg = cd.g;
    const Work cw = cd.w;
    const int l = item - L.start[c];
    const int by = l / L.tx[c], bx = l - by * L.tx[c];
    const int i0 = bx * FR_TX, j0 = by * FR_TY;
    const WorkF f = mixed_planes(cw, cg.ps);
    float amax = 0.f, bmax = 0.f;
    flux_tile_faces(cg, f, i0, j0, threadIdx.x, ft, amax, bmax);
    flux_tile_reduce(amax, bmax, cd.diag);
    __syncthreads();
    long long cc = 0;
    double r0[4];
    float rm[8];
    unsigned int bad = 0;
    if (flux_tile_balance(cg, f, i0, j0, threadIdx.x, ft, cc, r0, rm, &bad))
      store_residual_mixed(cg, cc, r0, rm, which == 0 ? cd.RHS0 : cd.RHS);
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (lane_id() == 0 && bad) atomicOr(&cd.diag->flags, bad);
    __syncthreads();  // the next item writes the tile again
  }
}

// ghost fill, both passes in one launch (ghost_xy_body): 1D items, gx = element index (the
// 8 ny x ghosts, then the 8 (nx + 8) y ghosts); with split (or for a case whose split is
// current), also the kept planes of the state's hi/lo split
__global__ void kb_ghost(const CaseDev* __restrict__ cases, TileList L, int ncase, int which, int split) {
  HW_BATCH_LOOP(L, ncase)
  double* q = which == 0 ? cd.Q : cd.QS;
  ghost_xy_body(cg, &cd.open, q, gx);
  if (split || cd.split_ok) ghost_xy_body(cg, &cd.open, mixed_planes(cw, cg.ps).hilo, gx, 0, HILO_KEPT);
  HW_BATCH_END
}

// hi/lo split of the mixed path: 1D items over the 12 whole padded planes (none for a
// case whose split is current)
__global__ void kb_split(const CaseDev* __restrict__ cases, TileList L, int ncase, int which) {
  HW_BATCH_LOOP(L, ncase)
  const double* q = which == 0 ? cd.Q : cd.QS;
  const long long n = 12 * cg.ps;
  if (gx < n && !cd.split_ok) {
    float* hilo = mixed_planes(cw, cg.ps).hilo;
    float hi, lo;
    split_hilo(q[gx], hi, lo);
    hilo[gx] = hi;
    if (gx < 4 * cg.ps) hilo[n + gx] = lo;  // the averages' lo planes
  }
  HW_BATCH_END
}

// per-case reductions: reset before a step, time step after the stage-1 residual
__global__ void kb_reset(const CaseDev* __restrict__ cases, int ncase) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncase || !cases[c].active) return;
  Diag* d = cases[c].diag;
  d->alpha_bits = 0ull;
  d->beta_bits = 0ull;
  d->pp_count = 0ull;
  d->flags = 0u;
}

__global__ void kb_dt(const CaseDev* __restrict__ cases, int ncase) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncase || !cases[c].active) return;
  const CaseDev& cd = cases[c];
  const double a = __longlong_as_double((long long)cd.diag->alpha_bits);
  cd.diag->dt = fmin(cd.cfl * cd.hmin / a, cd.visc_cap) * cd.dt_scale;
}

#ifdef __CUDACC__
// the tensor maps of a mixed batch's cases (traces and cell means, as a handle builds them
// for its own TMA-staged gradient pass), passed to kb_grad_tma_mixed as one kernel
// parameter: at most BT_MAX_CASES cases (a larger batch runs the separate kernels)
constexpr int BT_MAX_CASES = 64;
struct BatchTraceMaps {
  CUtensorMap tr[BT_MAX_CASES];
  CUtensorMap wb[BT_MAX_CASES];
};

// the gradient pass of a mixed batch: k_grad_tma_mixed's tiles (GT_X x GT_Y cells of each
// case's gradient region, copied into shared memory by the Tensor Memory Accelerator)
// over a work list of (case, tile) items; the block's mbarrier completes one phase per
// tile it processes
template <bool LIN>
__global__ void __launch_bounds__(GT_THREADS) kb_grad_tma_mixed(const CaseDev* __restrict__ cases, TileList L,
                                                                int ncase,
                                                                const __grid_constant__ BatchTraceMaps maps) {
  extern __shared__ __align__(16) unsigned char gt_raw[];
  unsigned b_addr;
  float* gt_smem = grad_tma_smem(gt_raw, &b_addr);
  unsigned parity = 0;
  const int total = L.start[ncase];
  for (int item = blockIdx.x; item < total; item += gridDim.x) {
    const int c = find_case(L.start, ncase, item);
    const CaseDev& cd = cases[c];
    if (!cd.active) continue;  // the same for every thread of the block
    const Grid cg = cd.g;
    const Work cw = cd.w;
    const int l = item - L.start[c];
    const int by = l / L.tx[c], bx = l - by * L.tx[c];
    if (!grad_tma_tile<LIN>(cg, cw, &maps.tr[c], &maps.wb[c], bx, by, gt_smem, b_addr, parity, cd.diag)) return;
    parity ^= 1u;
    __syncthreads();  // the next tile overwrites the staged data and the weak moments
  }
}
#endif

}  // namespace hw
