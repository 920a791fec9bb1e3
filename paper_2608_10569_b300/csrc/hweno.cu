// B300 (sm_103a) HWENO-GR solver: kernels of the spatial operator, the SSP-RK3
// stage update, reductions, and the C ABI declared in include/hweno.h.
//
// Paper: Guo, Fan, Zhao, "An efficient and robust fifth-order HWENO scheme with
// gradient reconstruction for compressible Navier-Stokes equations" (arXiv 2608.10569).
#include <cuda_runtime.h>
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <atomic>
#include <new>
#include <vector>

#include "hweno.h"
#include "hweno_ops.cuh"
#include "hweno_mixed.cuh"
#include "hweno_batch.cuh"
#include "hweno_adjoint.cuh"
#include "hweno_source.cuh"
#include "hweno_tma.cuh"

namespace hw {

constexpr int BX = 32, BY = 4;

// single-grid kernels: one thread per position of the launch region
template <class T>
__global__ void __launch_bounds__(BX * BY) k_cons(Grid g, const double* __restrict__ q, Work w,
                                                  double* __restrict__ mom, Diag* diag) {
  cons_body<T>(g, q, w, mom, diag, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}
// the FP64 traces of a step recorded for the adjoint (Work::yrec set)
__global__ void __launch_bounds__(BX * BY) k_cons_rec(Grid g, const double* __restrict__ q, Work w,
                                                      double* __restrict__ mom, Diag* diag) {
  cons_body<double, true>(g, q, w, mom, diag, blockIdx.x * blockDim.x + threadIdx.x,
                          blockIdx.y * blockDim.y + threadIdx.y);
}
// HWENO-DR: the FP64 traces also store the characteristic combinations (Work::dr)
__global__ void __launch_bounds__(BX * BY) k_cons_dr(Grid g, const double* __restrict__ q, Work w,
                                                     double* __restrict__ mom, Diag* diag) {
  cons_body<double, false, true>(g, q, w, mom, diag, blockIdx.x * blockDim.x + threadIdx.x,
                                 blockIdx.y * blockDim.y + threadIdx.y);
}
// HWENO-DR gradients from those combinations, in place of the gradient reconstruction
__global__ void __launch_bounds__(DR_THREADS) k_dr(Grid g, const double* __restrict__ q, Work w) {
  dr_body(g, q, w, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}
// Example 5.2's manufactured source, added to the residual at t0 + cst * dt
__global__ void __launch_bounds__(BX * BY) k_source(Grid g, Quad4 qd, double t0, double cst, const Diag* diag,
                                                    double* __restrict__ rhs) {
  source_body(g, qd, t0, cst, diag, rhs, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}
template <bool LIN = false>
__global__ void __launch_bounds__(BX * BY) k_grad_rec(Grid g, Work w) {
  grad_body<double, true, LIN>(g, w, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}
__global__ void k_face_moments(Grid g, Work w) {
  face_moments_body(g, w, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y, blockIdx.z);
}
__global__ void k_weak_moments(Grid g, Work w) {
  weak_moments_body(g, w, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}
template <class T, bool LIN = false>
__global__ void __launch_bounds__(BX * BY) k_grad(Grid g, Work w) {
  grad_body<T, false, LIN>(g, w, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}
template <class T>
__global__ void __launch_bounds__(BX * BY) k_flux(Grid g, Work w, Diag* diag) {
  flux_body<T>(g, w, diag, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y, blockIdx.z);
}
template <class T>
__global__ void __launch_bounds__(BX * BY) k_assemble(Grid g, Work w, double* __restrict__ rhs, Diag* diag) {
  assemble_body<T>(g, w, rhs, diag, blockIdx.x * blockDim.x + threadIdx.x, blockIdx.y * blockDim.y + threadIdx.y);
}
__global__ void k_rk(Grid g, int stage, const double* __restrict__ qin, const double* __restrict__ mom,
                     const double* __restrict__ rhs, double* __restrict__ base, double* __restrict__ qout,
                     Diag* diag) {
  rk_body(g, stage, qin, mom, rhs, base, qout, diag, blockIdx.x * blockDim.x + threadIdx.x,
          blockIdx.y * blockDim.y + threadIdx.y);
}
// the mixed path's stage update: also the hi/lo split of the new state and its largest
// kinetic share
__global__ void k_rk_split(Grid g, int stage, const double* __restrict__ qin, const double* __restrict__ mom,
                           const double* __restrict__ rhs, double* __restrict__ base, double* __restrict__ qout,
                           Diag* diag, float* __restrict__ hilo) {
  rk_body<true, true>(g, stage, qin, mom, rhs, base, qout, diag, blockIdx.x * blockDim.x + threadIdx.x,
                      blockIdx.y * blockDim.y + threadIdx.y, hilo);
}
// a mixed handle's stage update on the FP64 route: the largest kinetic share, no split
__global__ void k_rk_kef(Grid g, int stage, const double* __restrict__ qin, const double* __restrict__ mom,
                         const double* __restrict__ rhs, double* __restrict__ base, double* __restrict__ qout,
                         Diag* diag) {
  rk_body<false, true>(g, stage, qin, mom, rhs, base, qout, diag, blockIdx.x * blockDim.x + threadIdx.x,
                       blockIdx.y * blockDim.y + threadIdx.y);
}
// the largest kinetic share |m|^2 / (2 rho E) over the cells of q (1 where a cell is
// inadmissible), into diag->kefrac_bits
__global__ void k_kinetic_share(Grid g, const double* __restrict__ q, Diag* diag) {
  const long long N = (long long)g.nx * g.ny;
  double kef = 0.0;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < N; t += (long long)gridDim.x * blockDim.x) {
    const long long c = cidx(g, (int)(t % g.nx), (int)(t / g.nx));
    const double r = q[c], m = q[g.ps + c], n = q[2 * g.ps + c], E = q[3 * g.ps + c];
    const double rp = E * r - 0.5 * (m * m + n * n);
    kef = fmax(kef, (r > 0.0 && rp > 0.0) ? 1.0 - rp / (E * r) : 1.0);
  }
  kef = warp_max(kef);
  if (lane_id() == 0) atomic_max_pos(&diag->kefrac_bits, kef);
}

// time step of Sec. 5: dt = min(CFL h / alpha*, b Re h^2), or a forced trial
// value, capped by the remaining time
__global__ void k_dt(Diag* diag, double cfl, double h, double visc_cap, double forced, double cap) {
  const double a = __longlong_as_double((long long)diag->alpha_bits);
  double dt = forced > 0.0 ? forced : fmin(cfl * h / a, visc_cap);
  if (dt > cap) dt = cap;
  diag->dt = dt;
}

__global__ void k_scale_dt(Diag* diag, double f) { diag->dt *= f; }

// keep the stage-1 maxima, flags and dt of a step in the second slot, so that one
// read at the end of the step's attempt brings both back
__global__ void k_stash(Diag* diag) { diag[1] = diag[0]; }

// scatter a contiguous [n][ny][nx] array into padded planes, and back
__global__ void k_scatter(Grid g, int n, const double* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * N;
       t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / N, r = t % N;
    const int j = (int)(r / g.nx), i = (int)(r % g.nx);
    dst[p * g.ps + cidx(g, i, j)] = src[t];
  }
}
__global__ void k_gather(Grid g, int n, const double* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < n * N;
       t += (long long)gridDim.x * blockDim.x) {
    const long long p = t / N, r = t % N;
    const int j = (int)(r / g.nx), i = (int)(r % g.nx);
    dst[t] = src[p * g.ps + cidx(g, i, j)];
  }
}
// primitive (rho, u, v, e) point sets back to conserved variables, gathered
__global__ void k_gather_cons(Grid g, int npts, const double* __restrict__ src, double* __restrict__ dst) {
  const long long N = (long long)g.nx * g.ny;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < npts * N;
       t += (long long)gridDim.x * blockDim.x) {
    const long long k = t / N, r = t % N;
    const int j = (int)(r / g.nx), i = (int)(r % g.nx);
    const long long c = cidx(g, i, j);
    const double rho = src[(4 * k + 0) * g.ps + c], u = src[(4 * k + 1) * g.ps + c];
    const double v = src[(4 * k + 2) * g.ps + c], e = src[(4 * k + 3) * g.ps + c];
    dst[(4 * k + 0) * N + r] = rho;
    dst[(4 * k + 1) * N + r] = rho * u;
    dst[(4 * k + 2) * N + r] = rho * v;
    dst[(4 * k + 3) * N + r] = rho * (e + 0.5 * (u * u + v * v));
  }
}

// deterministic reductions of the state: per-row partials in a fixed order, then
// one block adds the rows in order.  part: [ny][6] = (sum rho, rho u, rho v, E,
// min rho, min p)
__global__ void k_state_rows(Grid g, const double* __restrict__ q, double* part) {
  const int j = blockIdx.x;
  if (threadIdx.x != 0 || j >= g.ny) return;
  double s[4] = {0, 0, 0, 0}, mr = INFINITY, mp = INFINITY;
  for (int i = 0; i < g.nx; i++) {
    const long long c = cidx(g, i, j);
    double u[4];
    for (int v = 0; v < 4; v++) { u[v] = q[(long long)v * g.ps + c]; s[v] += u[v]; }
    mr = fmin(mr, u[0]);
    mp = fmin(mp, (g.gamma - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]));
  }
  for (int v = 0; v < 4; v++) part[6 * j + v] = s[v];
  part[6 * j + 4] = mr;
  part[6 * j + 5] = mp;
}
__global__ void k_state_final(Grid g, const double* part, double* out) {
  if (threadIdx.x != 0) return;
  double s[4] = {0, 0, 0, 0}, mr = INFINITY, mp = INFINITY;
  for (int j = 0; j < g.ny; j++) {
    for (int v = 0; v < 4; v++) s[v] += part[6 * j + v];
    mr = fmin(mr, part[6 * j + 4]);
    mp = fmin(mp, part[6 * j + 5]);
  }
  for (int v = 0; v < 4; v++) out[v] = s[v] * g.dx * g.dy;
  out[4] = mr;
  out[5] = mp;
}

// FMA-chain throughput probe: 8 independent chains per thread, x <- x*a + b
// (a < 1 so every chain converges to b/(1-a) and stays finite).  The store is
// taken only if the impossible value -1 appears, so the work cannot be removed.
template <class T>
__global__ void k_fma_peak(T* sink, int iters, T a, T b) {
  T x[8];
#pragma unroll
  for (int k = 0; k < 8; k++) x[k] = (T)(threadIdx.x + k) * (T)1e-3;
#pragma unroll 1
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int r = 0; r < 16; r++)
#pragma unroll
      for (int k = 0; k < 8; k++) x[k] = fma(x[k], a, b);
  }
  T s = 0;
#pragma unroll
  for (int k = 0; k < 8; k++) s += x[k];
  if (s == (T)-1) sink[0] = s;
}

}  // namespace hw

// ===========================================================================
// host side

using namespace hw;

namespace {

enum { K_GHOST = 0, K_CONS, K_FACEMOM, K_WEAK, K_GRAD, K_FLUX, K_ASSEMBLE, K_RK, K_SOURCE, K_NKIND };

struct EventPair {
  cudaEvent_t a, b;
  int kind;
};

}  // namespace

struct hweno_handle {
  hweno_config cfg;
  cudaStream_t st;
  Grid g;
  double* pool = nullptr;
  double *Q, *QS, *BASE, *RHS0, *RHS, *MOM0, *MOM, *STAGE, *PART;
  Work w;
  Diag* d_diag = nullptr;
  Diag* h_diag = nullptr;  // pinned
  double* h_red = nullptr; // pinned [6]
  double* d_red = nullptr;
  bool have_state = false, have_residual = false;
  const double* split_of = nullptr;  // mixed path: the state whose hi/lo split is current
  // mixed path: the largest kinetic share |m|^2 / (2 rho E) over the cells of the state
  // (measured at set_state and by every accepted step), and whether the current step
  // or residual runs the FP64 operator because that share exceeds MIXED_MAX_KINETIC_SHARE
  double ke_share = 0.0;
  bool route64 = false;
  long long steps64 = 0;
  double t = 0.0;
  // counters
  double pp_total = 0.0, cell_stages = 0.0;
  long long steps = 0, rejected = 0, launches = 0;
  double alpha = 0.0, beta = 0.0, dt_last = 0.0;
  // adjoint buffers (hweno_adjoint_init)
  double* apool = nullptr;
  Adj adj{};
  double *AST1 = nullptr, *ALAM = nullptr, *ABB = nullptr, *ATMP = nullptr;
  double* AYREC = nullptr;  // reconstruction record of a stage re-evaluated for the reverse
  // segment storage (hweno_adjoint_reserve): 3 stage states per step, and optionally the
  // forward intermediates of every stage
  double* spool = nullptr;
  int seg_max = 0;
  int seg_keep = 0;
  bool seg_keep_refused = false;  // intermediates were asked for and did not fit
  bool recording = false;        // do_step records each accepted step into the next slot
  int rec_count = 0;             // recorded steps
  std::vector<double> rec_dts;   // their step sizes
  // profiling
  bool prof = false;
  std::vector<EventPair> ev;
  // mixed path: tensor maps of the FP32 traces and cell means for the TMA-staged
  // gradient kernel (tma false: the separate face-moment, weak-moment and gradient kernels)
  CUtensorMap tr_map, wb_map;
  bool tma = false;
  Quad4 quad{};  // the source term's 4-point Gauss rule
  Open open{};   // prescribed states of the inflow faces
  long long prof_n[K_NKIND];
  double prof_ms[K_NKIND];
  char err[512];
};

// The mixed path's precision bound.  Its FP32 face fluxes of the total energy carry
// rounding of about 2^-24 of that flux; a stage then moves the internal energy by about
// 2^-24 x (kinetic / internal energy) x the CFL-sized factor dt |u| / h.  Where the
// internal energy falls below 1e-4 of the total (the kinetic share above 1 - 1e-4) that
// is 6e-4 of the internal energy per stage, and the Mach-1500 colliding streams
// (internal share 7.5e-7) would lose positivity within a few steps.  A mixed handle
// therefore runs the FP64 operator for a step or residual whose state exceeds this share
// anywhere, and returns to FP32 once the state is back under it.
constexpr double MIXED_MAX_KINETIC_SHARE = 1.0 - 1e-4;

static char g_init_err[512] = "no error";

static int fail(hweno_handle* h, int code, const char* msg) {
  if (h) snprintf(h->err, sizeof(h->err), "%s", msg);
  else snprintf(g_init_err, sizeof(g_init_err), "%s", msg);
  return code;
}

static int cuda_fail(hweno_handle* h, cudaError_t e, const char* where) {
  char buf[400];
  snprintf(buf, sizeof(buf), "%s: %s", where, cudaGetErrorString(e));
  return fail(h, HWENO_ERR_CUDA, buf);
}

#define CK(call, where)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, where); \
  } while (0)

// launch bookkeeping: optional CUDA events around each kernel of the operator
struct Prof {
  hweno_handle* h;
  int kind;
  cudaEvent_t a{}, b{};
  Prof(hweno_handle* h_, int k) : h(h_), kind(k) {
    h->launches++;
    if (h->prof) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
      cudaEventRecord(a, h->st);
    }
  }
  ~Prof() {
    if (h->prof) {
      cudaEventRecord(b, h->st);
      h->ev.push_back({a, b, kind});
    }
  }
};

static dim3 grid2(int wx, int wy, int z = 1) {
  return dim3((unsigned)((wx + BX - 1) / BX), (unsigned)((wy + BY - 1) / BY), (unsigned)z);
}

// ghost fill of a 12-plane state set
// ghost fill of q's 12 planes and, with hilo, of the kept planes of its hi/lo split
// (HILO_KEPT: the 12 hi planes and the averages' 4 lo planes)
static void launch_ghost(hweno_handle* h, double* q, float* hilo = nullptr) {
  const Grid& g = h->g;
  const int planes = hilo ? 12 + HILO_KEPT : 12;
  Prof p(h, K_GHOST);
  const int n = 8 * g.ny + 8 * (g.nx + 2 * NG);
  k_ghost<<<dim3((n + 127) / 128, planes), 128, 0, h->st>>>(g, h->open, q, hilo);
}

// the FP64 cell-trace kernels take CONS_SMEM_BYTES of dynamic shared memory (above the
// 48 KB default): allowed once per device
static cudaError_t cons_smem_allow() {
  static std::atomic<unsigned int> done{0};  // bit per device; callers may be on several threads
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 32 && (done.load() >> dev) & 1u) return cudaSuccess;
  e = cudaFuncSetAttribute(k_cons<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONS_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cons_rec, cudaFuncAttributeMaxDynamicSharedMemorySize, CONS_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_cons<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONS_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_cons_dr, cudaFuncAttributeMaxDynamicSharedMemorySize, CONS_SMEM_BYTES);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dr, cudaFuncAttributeMaxDynamicSharedMemorySize, DR_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_cons<0, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, CONS_SMEM_BYTES);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(kb_dr, cudaFuncAttributeMaxDynamicSharedMemorySize, DR_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grad_tma_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_grad_tma_mixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_grad_tma_mixed<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM_BYTES);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(kb_grad_tma_mixed<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, GT_SMEM_BYTES);
  if (e == cudaSuccess && dev < 32) done.fetch_or(1u << dev);
  return e;
}

// one spatial-operator evaluation of state q (12 planes): rhs (12 planes) and the
// modified moments mom (8 planes); a source term is taken at t + cst * dt (t the
// handle's time, dt the device-side step of the current attempt)
// cuTensorMapEncodeTiled, from the driver through the runtime (no link to the driver
// library); null where the driver does not provide it
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
static EncodeTiledFn encode_tiled() {
  static std::atomic<EncodeTiledFn> fn{nullptr};
  static std::atomic<bool> tried{false};
  if (!tried.load()) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess && p)
      fn.store((EncodeTiledFn)p);
    tried.store(true);
  }
  return fn.load();
}

// tensor maps of the mixed path's FP32 face traces (x: pitch, y: padded rows, variable,
// point; the face group's float plane 4 k + v) and cell means (x, y, variable) for the
// boxes k_grad_tma_mixed copies; false if they cannot be made
static bool encode_trace_maps(const Grid& g, const Work& w, CUtensorMap* tr, CUtensorMap* wb) {
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return false;
  const WorkF f = mixed_planes(w, g.ps);
  const cuuint64_t row = (cuuint64_t)g.pitch * sizeof(float), plane = (cuuint64_t)g.ps * sizeof(float);
  const cuuint64_t dt[4] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 2 * NG), 4, 12};
  const cuuint64_t st[3] = {row, plane, 4 * plane};
  const cuuint32_t bt[4] = {GB_X, GB_Y, 3, 12};
  const cuuint32_t one[4] = {1, 1, 1, 1};
  if (enc(tr, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, f.face, dt, st, bt, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
          CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
          CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
    return false;
  const cuuint64_t dw[3] = {(cuuint64_t)g.pitch, (cuuint64_t)(g.ny + 2 * NG), 3};
  const cuuint64_t sw[2] = {row, plane};
  const cuuint32_t bw[3] = {GB_X, GB_Y, 3};
  return enc(wb, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, f.wbar, dw, sw, bw, one, CU_TENSOR_MAP_INTERLEAVE_NONE,
             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// the mixed path's face moments, weak-derivative moments and gradients in separate
// kernels through HBM, from the traces in the handle's planes; volg: also the gradients
// at the volume points (the debug export; the operator needs only their sums)
static void mixed_grad_separate(hweno_handle* h, bool volg) {
  const Grid& g = h->g;
  {
    Prof p(h, K_FACEMOM);
    k_face_moments_mixed<<<grid2(g.nx + 5, g.ny + 5, 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
  }
  {
    Prof p(h, K_WEAK);
    k_weak_moments_mixed<<<grid2(g.nx + 4, g.ny + 4), dim3(BX, BY), 0, h->st>>>(g, h->w);
  }
  Prof p(h, K_GRAD);
  const dim3 grid = grid2(g.nx + 2, g.ny + 2), blk(BX, BY);
  if (h->cfg.linear_grad) {
    if (volg) k_grad_mixed<true, true><<<grid, blk, 0, h->st>>>(g, h->w);
    else k_grad_mixed<true><<<grid, blk, 0, h->st>>>(g, h->w);
  } else {
    if (volg) k_grad_mixed<false, true><<<grid, blk, 0, h->st>>>(g, h->w);
    else k_grad_mixed<false><<<grid, blk, 0, h->st>>>(g, h->w);
  }
}

// the mixed path's operator up to the gradients: ghost cells (and the FP32 split of a
// state set from outside), traces and limiter, then face moments, weak-derivative
// moments and gradients (one TMA-staged kernel where the handle has the tensor maps)
static void mixed_front(hweno_handle* h, double* q, double* mom) {
  const Grid& g = h->g;
  float* hilo = mixed_planes(h->w, g.ps).hilo;
  if (h->split_of == q) {
    // the stage update that wrote q also wrote the interior of its split
    launch_ghost(h, q, hilo);
  } else {
    launch_ghost(h, q);
    Prof p(h, K_GHOST);
    k_split<<<4 * 148, 256, 0, h->st>>>(g, q, hilo);
    h->split_of = q;
  }
  {
    Prof p(h, K_CONS);
    k_cons_mixed<<<grid2(g.nx + 6, g.ny + 6), dim3(BX, BY), 0, h->st>>>(g, q, h->w, mom, h->d_diag);
  }
  if (h->tma) {
    Prof p(h, K_GRAD);
    const dim3 grid((unsigned)((g.nx + 2 + GT_X - 1) / GT_X), (unsigned)((g.ny + 2 + GT_Y - 1) / GT_Y));
    if (h->cfg.linear_grad)
      k_grad_tma_mixed<true><<<grid, GT_THREADS, GT_SMEM_BYTES, h->st>>>(g, h->w, h->tr_map, h->wb_map, h->d_diag);
    else
      k_grad_tma_mixed<false><<<grid, GT_THREADS, GT_SMEM_BYTES, h->st>>>(g, h->w, h->tr_map, h->wb_map, h->d_diag);
    return;
  }
  mixed_grad_separate(h, false);
}

static int residual_eval(hweno_handle* h, double* q, double* rhs, double* mom, double cst = 0.0) {
  const Grid& g = h->g;
  if (h->cfg.precision == HWENO_MIXED && !h->route64) {
    mixed_front(h, q, mom);
    {
      Prof p(h, K_FLUX);
      const dim3 grid((unsigned)((g.nx + FR_TX - 1) / FR_TX), (unsigned)((g.ny + FR_TY - 1) / FR_TY));
      k_flux_asm_mixed<<<grid, FR_THREADS, 0, h->st>>>(g, h->w, rhs, h->d_diag);
    }
  } else if (h->cfg.scheme == HWENO_SCHEME_DR) {
    launch_ghost(h, q);
    {
      Prof p(h, K_CONS);
      k_cons_dr<<<grid2(g.nx + 6, g.ny + 6), dim3(BX, BY), CONS_SMEM_BYTES, h->st>>>(g, q, h->w, mom, h->d_diag);
    }
    {
      Prof p(h, K_GRAD);
      const dim3 blk(32, DR_THREADS / 32);
      k_dr<<<dim3((g.nx + 2 + 31) / 32, (g.ny + 2 + blk.y - 1) / blk.y), blk, DR_SMEM_BYTES, h->st>>>(g, q, h->w);
    }
    {
      Prof p(h, K_FLUX);
      k_flux<double><<<grid2(g.nx + 1, g.ny + 1, 2), dim3(BX, BY), 0, h->st>>>(g, h->w, h->d_diag);
    }
    {
      Prof p(h, K_ASSEMBLE);
      k_assemble<double><<<grid2(g.nx, g.ny), dim3(BX, BY), 0, h->st>>>(g, h->w, rhs, h->d_diag);
    }
  } else {
    launch_ghost(h, q);
    {
      Prof p(h, K_CONS);
      if (h->w.yrec)
        k_cons_rec<<<grid2(g.nx + 6, g.ny + 6), dim3(BX, BY), CONS_SMEM_BYTES, h->st>>>(g, q, h->w, mom,
                                                                                     h->d_diag);
      else
        k_cons<double><<<grid2(g.nx + 6, g.ny + 6), dim3(BX, BY), CONS_SMEM_BYTES, h->st>>>(g, q, h->w, mom,
                                                                                         h->d_diag);
    }
    {
      Prof p(h, K_FACEMOM);
      k_face_moments<<<grid2(g.nx + 5, g.ny + 5, 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
    }
    {
      Prof p(h, K_WEAK);
      k_weak_moments<<<grid2(g.nx + 4, g.ny + 4), dim3(BX, BY), 0, h->st>>>(g, h->w);
    }
    {
      Prof p(h, K_GRAD);
      if (h->w.yrec)
        if (h->cfg.linear_grad) k_grad_rec<true><<<grid2(g.nx + 2, g.ny + 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
        else k_grad_rec<<<grid2(g.nx + 2, g.ny + 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
      else if (h->cfg.linear_grad)
        k_grad<double, true><<<grid2(g.nx + 2, g.ny + 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
      else
        k_grad<double><<<grid2(g.nx + 2, g.ny + 2), dim3(BX, BY), 0, h->st>>>(g, h->w);
    }
    {
      Prof p(h, K_FLUX);
      k_flux<double><<<grid2(g.nx + 1, g.ny + 1, 2), dim3(BX, BY), 0, h->st>>>(g, h->w, h->d_diag);
    }
    {
      Prof p(h, K_ASSEMBLE);
      k_assemble<double><<<grid2(g.nx, g.ny), dim3(BX, BY), 0, h->st>>>(g, h->w, rhs, h->d_diag);
    }
  }
  if (h->cfg.source == HWENO_SOURCE_MMS52) {
    Prof p(h, K_SOURCE);
    k_source<<<grid2(g.nx, g.ny), dim3(BX, BY), 0, h->st>>>(g, h->quad, h->t, cst, h->d_diag, rhs);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "spatial operator launch");
  return HWENO_OK;
}

static int launch_rk(hweno_handle* h, int stage, const double* qin, const double* mom,
                     const double* rhs, double* qout);

// stage 2 or 3 of a step: the operator on the stage state q and the stage update into
// qout.  On the mixed path (without a source term) the face fluxes, the balances and the
// update run as one tile kernel, k_flux_rk_mixed, with the separate kernels' operations
// in their order; otherwise the residual goes through HBM.
static int stage_eval_rk(hweno_handle* h, double* q, int stage, double* qout, double cst) {
  const Grid& g = h->g;
  if (h->cfg.precision == HWENO_MIXED && !h->route64 && h->cfg.source == HWENO_SOURCE_NONE) {
    mixed_front(h, q, h->MOM);
    {
      Prof p(h, K_FLUX);
      const dim3 grid((unsigned)((g.nx + FR_TX - 1) / FR_TX), (unsigned)((g.ny + FR_TY - 1) / FR_TY));
      k_flux_rk_mixed<<<grid, FR_THREADS, 0, h->st>>>(g, h->w, stage, q, h->MOM, h->BASE, qout, h->d_diag,
                                                      mixed_planes(h->w, g.ps).hilo);
    }
    h->split_of = qout;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(h, e, "fused stage launch");
    return HWENO_OK;
  }
  int rc = residual_eval(h, q, h->RHS, h->MOM, cst);
  if (!rc) rc = launch_rk(h, stage, q, h->MOM, h->RHS, qout);
  return rc;
}

static int launch_rk(hweno_handle* h, int stage, const double* qin, const double* mom,
                     const double* rhs, double* qout) {
  Prof p(h, K_RK);
  if (h->cfg.precision == HWENO_MIXED && !h->route64) {
    k_rk_split<<<grid2(h->g.nx, h->g.ny), dim3(BX, BY), 0, h->st>>>(h->g, stage, qin, mom, rhs, h->BASE, qout,
                                                                  h->d_diag, mixed_planes(h->w, h->g.ps).hilo);
    h->split_of = qout;
  } else if (h->cfg.precision == HWENO_MIXED) {
    k_rk_kef<<<grid2(h->g.nx, h->g.ny), dim3(BX, BY), 0, h->st>>>(h->g, stage, qin, mom, rhs, h->BASE, qout,
                                                                h->d_diag);
  } else {
    k_rk<<<grid2(h->g.nx, h->g.ny), dim3(BX, BY), 0, h->st>>>(h->g, stage, qin, mom, rhs, h->BASE, qout,
                                                              h->d_diag);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "rk launch");
  return HWENO_OK;
}

static double h_min(const hweno_handle* h) {
  const double dx = h->g.dx, dy = h->g.dy;
  return dx < dy ? dx : dy;
}

static int valid_bc(int b) { return b >= HWENO_BC_PERIODIC && b <= HWENO_BC_OUTFLOW; }

// the prescribed states of the inflow faces: finite, with rho > 0 and p > 0, and
// bands of finite centre and half width >= 0
static int check_inflow(const hweno_config& c) {
  for (int k = 0; k < 4; k++) {
    if (c.bc[k] != HWENO_BC_INFLOW) continue;
    if (!isfinite(c.band[k][0]) || !isfinite(c.band[k][1]) || !(c.band[k][1] >= 0.0))
      return fail(nullptr, HWENO_ERR_ARG, "an inflow band needs a finite centre and a half width >= 0");
    for (int a = 0; a < 2; a++) {
      const double* u = c.inflow[k][a];
      bool ok = true;
      for (int v = 0; v < 4; v++) ok = ok && isfinite(u[v]);
      const double p = ok && u[0] > 0.0 ? (c.gamma - 1.0) * (u[3] - 0.5 * (u[1] * u[1] + u[2] * u[2]) / u[0]) : -1.0;
      if (!(u[0] > 0.0) || !(p > 0.0))
        return fail(nullptr, HWENO_ERR_ARG, "an inflow state needs finite values with rho > 0 and p > 0");
    }
  }
  return HWENO_OK;
}


extern "C" {

int hweno_config_default(hweno_config* c) {
  if (!c) return HWENO_ERR_ARG;
  memset(c, 0, sizeof(*c));
  c->x0 = 0.0; c->x1 = 1.0; c->y0 = 0.0; c->y1 = 1.0;
  c->gamma = 1.4; c->Pr = 0.72; c->Re = 1000.0;
  for (int k = 0; k < 4; k++) c->bc[k] = HWENO_BC_PERIODIC;
  c->cfl = 0.6; c->b_visc = 1e-3; c->eps_pp = 1e-12; c->eps_weno = 1e-8;
  c->max_halvings = 60;
  c->precision = HWENO_FP64;
  return HWENO_OK;
}

const char* hweno_last_error(const hweno_handle* h) { return h ? h->err : g_init_err; }

long long hweno_launch_count(const hweno_handle* h) { return h ? h->launches : 0; }

int hweno_init(const hweno_config* cfg, void* stream, hweno_handle** out) {
  hweno_handle* h = nullptr;
  if (!out) return fail(nullptr, HWENO_ERR_ARG, "hweno_init: out is NULL");
  *out = nullptr;
  if (!cfg) return fail(nullptr, HWENO_ERR_ARG, "hweno_init: cfg is NULL");
  const hweno_config& c = *cfg;
  if (c.nx < 4 || c.ny < 4) return fail(nullptr, HWENO_ERR_ARG, "nx and ny must be >= 4");
  if ((long long)c.nx * c.ny > (1LL << 31)) return fail(nullptr, HWENO_ERR_ARG, "grid too large");
  if (!(c.x1 > c.x0) || !(c.y1 > c.y0)) return fail(nullptr, HWENO_ERR_ARG, "empty domain");
  if (!(c.gamma > 1.0) || !(c.Pr > 0.0) || !(c.Re > 0.0)) return fail(nullptr, HWENO_ERR_ARG, "need gamma > 1, Pr > 0, Re > 0");
  for (int k = 0; k < 4; k++)
    if (!valid_bc(c.bc[k])) return fail(nullptr, HWENO_ERR_ARG, "unknown boundary condition");
  if ((c.bc[0] == HWENO_BC_PERIODIC) != (c.bc[1] == HWENO_BC_PERIODIC) ||
      (c.bc[2] == HWENO_BC_PERIODIC) != (c.bc[3] == HWENO_BC_PERIODIC))
    return fail(nullptr, HWENO_ERR_ARG, "periodic boundaries must be set on both sides");
  if (!(c.cfl > 0.0) || !(c.b_visc > 0.0) || !(c.eps_pp > 0.0) || !(c.eps_weno > 0.0) || c.max_halvings < 0)
    return fail(nullptr, HWENO_ERR_ARG, "cfl, b_visc, eps_pp, eps_weno must be > 0");
  if (c.precision != HWENO_FP64 && c.precision != HWENO_MIXED)
    return fail(nullptr, HWENO_ERR_ARG, "precision must be HWENO_FP64 or HWENO_MIXED");
  if (c.scheme != HWENO_SCHEME_GR && c.scheme != HWENO_SCHEME_DR)
    return fail(nullptr, HWENO_ERR_ARG, "scheme must be HWENO_SCHEME_GR or HWENO_SCHEME_DR");
  if (c.scheme == HWENO_SCHEME_DR && c.precision != HWENO_FP64)
    return fail(nullptr, HWENO_ERR_ARG, "HWENO_SCHEME_DR runs in HWENO_FP64");
  if (c.source != HWENO_SOURCE_NONE && c.source != HWENO_SOURCE_MMS52)
    return fail(nullptr, HWENO_ERR_ARG, "source must be HWENO_SOURCE_NONE or HWENO_SOURCE_MMS52");
  if (check_inflow(c)) return HWENO_ERR_ARG;
  if (c.linear_grad != 0 && c.linear_grad != 1) return fail(nullptr, HWENO_ERR_ARG, "linear_grad must be 0 or 1");
  if (c.linear_grad && c.scheme != HWENO_SCHEME_GR)
    return fail(nullptr, HWENO_ERR_ARG, "linear_grad ablates the gradient reconstruction of HWENO_SCHEME_GR");

  h = new (std::nothrow) hweno_handle();
  if (!h) return fail(nullptr, HWENO_ERR_ARG, "host allocation failed");
  h->cfg = c;
  h->st = (cudaStream_t)stream;
  snprintf(h->err, sizeof(h->err), "no error");
  for (int k = 0; k < K_NKIND; k++) { h->prof_n[k] = 0; h->prof_ms[k] = 0.0; }
  h->g = make_grid(c);
  const Grid& g = h->g;
  h->open = make_open(c);
  h->quad = make_quad4();

  const long long N = (long long)c.nx * c.ny;
  // planes: Q 12, QS 12, BASE 12, RHS0 12, RHS 12, MOM0 8, MOM 8, face 48, vol 36,
  // wbar 3, wx 6, wy 6, rm 18, gr 126, fx 12, fy 12, theta 2; HWENO-DR: dr 120
  const long long ndr = c.scheme == HWENO_SCHEME_DR ? 120 : 0;
  const long long nplanes = 12 * 5 + 16 + 48 + 36 + 3 + 12 + 18 + 126 + 24 + 2 + ndr;
  const long long total = nplanes * g.ps + 4 * N + 6LL * c.ny + 16;
  cudaError_t e = cons_smem_allow();
  if (e == cudaSuccess) e = cudaMalloc(&h->pool, (size_t)total * sizeof(double));
  if (e != cudaSuccess) {
    snprintf(g_init_err, sizeof(g_init_err), "device allocation of %.2f GB failed: %s",
             total * 8.0 / 1e9, cudaGetErrorString(e));
    delete h;
    return HWENO_ERR_CUDA;
  }
  double* p = h->pool;
  auto take = [&](long long n) { double* r = p; p += n * g.ps; return r; };
  h->Q = take(12); h->QS = take(12); h->BASE = take(12); h->RHS0 = take(12); h->RHS = take(12);
  h->MOM0 = take(8); h->MOM = take(8);
  h->w.face = take(48); h->w.vol = take(36); h->w.wbar = take(3); h->w.wx = take(6); h->w.wy = take(6);
  h->w.rm = take(18); h->w.gr = take(126); h->w.fx = take(12); h->w.fy = take(12); h->w.theta = take(2);
  if (ndr) h->w.dr = take(ndr);
  if (c.precision == HWENO_MIXED) h->tma = encode_trace_maps(g, h->w, &h->tr_map, &h->wb_map);
  h->STAGE = p; p += 4 * N;
  h->PART = p; p += 6LL * c.ny;
  h->d_red = p;
  e = cudaMemsetAsync(h->pool, 0, (size_t)total * sizeof(double), h->st);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_diag, 2 * sizeof(Diag));
  if (e == cudaSuccess) e = cudaMemsetAsync(h->d_diag, 0, 2 * sizeof(Diag), h->st);
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_diag, 2 * sizeof(Diag));
  if (e == cudaSuccess) e = cudaMallocHost(&h->h_red, 8 * sizeof(double));
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->st);
  if (e != cudaSuccess) {
    snprintf(g_init_err, sizeof(g_init_err), "init: %s", cudaGetErrorString(e));
    hweno_destroy(h);
    return HWENO_ERR_CUDA;
  }
  *out = h;
  return HWENO_OK;
}

void hweno_destroy(hweno_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  for (auto& ep : h->ev) { cudaEventDestroy(ep.a); cudaEventDestroy(ep.b); }
  if (h->pool) cudaFree(h->pool);
  if (h->apool) cudaFree(h->apool);
  if (h->spool) cudaFree(h->spool);
  if (h->d_diag) cudaFree(h->d_diag);
  if (h->h_diag) cudaFreeHost(h->h_diag);
  if (h->h_red) cudaFreeHost(h->h_red);
  delete h;
}

}  // extern "C"

static long long origin(const Grid& g) { return (long long)NG * g.pitch + NG; }

// contiguous [n][ny][nx] (host or device) <-> n padded planes
static int copy_planes_in(hweno_handle* h, const double* src, int n, double* dst, int on_device) {
  const Grid& g = h->g;
  const size_t row = (size_t)g.nx * sizeof(double);
  for (int k = 0; k < n; k++) {
    const double* s = src + (long long)k * g.nx * g.ny;
    double* d = dst + (long long)k * g.ps + origin(g);
    CK(cudaMemcpy2DAsync(d, (size_t)g.pitch * sizeof(double), s, row, row, (size_t)g.ny,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, h->st),
       "copy into the solver");
  }
  return HWENO_OK;
}

static int copy_planes_out(hweno_handle* h, const double* src, int n, double* dst, int on_device) {
  const Grid& g = h->g;
  const size_t row = (size_t)g.nx * sizeof(double);
  for (int k = 0; k < n; k++) {
    const double* s = src + (long long)k * g.ps + origin(g);
    double* d = dst + (long long)k * g.nx * g.ny;
    CK(cudaMemcpy2DAsync(d, row, s, (size_t)g.pitch * sizeof(double), row, (size_t)g.ny,
                         on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, h->st),
       "copy out of the solver");
  }
  return HWENO_OK;
}

static int reset_diag(hweno_handle* h) {
  CK(cudaMemsetAsync(h->d_diag, 0, sizeof(Diag), h->st), "diag reset");
  return HWENO_OK;
}

static int read_diag(hweno_handle* h) {
  CK(cudaMemcpyAsync(h->h_diag, h->d_diag, 2 * sizeof(Diag), cudaMemcpyDeviceToHost, h->st), "diag read");
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  return HWENO_OK;
}

static double bits_to_double(unsigned long long b) {
  double d;
  memcpy(&d, &b, sizeof(d));
  return d;
}

extern "C" {

int hweno_set_state(hweno_handle* h, const double* q, int on_device) {
  if (!h || !q) return fail(h, HWENO_ERR_ARG, "hweno_set_state: NULL argument");
  h->split_of = nullptr;
  int rc = copy_planes_in(h, q, 12, h->Q, on_device);
  if (rc) return rc;
  h->have_state = true;
  h->have_residual = false;
  h->pp_total = 0.0;
  h->cell_stages = 0.0;
  h->steps = 0;
  h->rejected = 0;
  h->launches = 0;
  h->steps64 = 0;
  h->t = 0.0;
  if (h->cfg.precision == HWENO_MIXED) {
    // the precision route of the first step or residual: one reduction and one read
    CK(cudaMemsetAsync(&h->d_diag->kefrac_bits, 0, sizeof(unsigned long long), h->st), "diag");
    k_kinetic_share<<<2 * 148, 256, 0, h->st>>>(h->g, h->Q, h->d_diag);
    h->launches++;
    CK(cudaGetLastError(), "kinetic share launch");
    if ((rc = read_diag(h))) return rc;
    h->ke_share = bits_to_double(h->h_diag->kefrac_bits);
  }
  if (!on_device) CK(cudaStreamSynchronize(h->st), "stream synchronize");
  return HWENO_OK;
}

// the precision route of a mixed handle's next step or residual (see
// MIXED_MAX_KINETIC_SHARE); the FP64 operator overwrites the planes of the FP32 split
static void choose_route(hweno_handle* h) {
  h->route64 = h->cfg.precision == HWENO_MIXED && !(h->ke_share <= MIXED_MAX_KINETIC_SHARE);
  if (h->route64) h->split_of = nullptr;
}

int hweno_set_time(hweno_handle* h, double t) {
  if (!h) return HWENO_ERR_ARG;
  h->t = t;
  return HWENO_OK;
}

int hweno_get_state(hweno_handle* h, double* q, int on_device) {
  if (!h || !q) return fail(h, HWENO_ERR_ARG, "hweno_get_state: NULL argument");
  if (!h->have_state) return fail(h, HWENO_ERR_STATE, "hweno_get_state before hweno_set_state");
  int rc = copy_planes_out(h, h->Q, 12, q, on_device);
  if (rc) return rc;
  if (!on_device) CK(cudaStreamSynchronize(h->st), "stream synchronize");
  return HWENO_OK;
}

int hweno_residual(hweno_handle* h, double* rhs, double* vhat, int on_device) {
  if (!h) return HWENO_ERR_ARG;
  if (!h->have_state) return fail(h, HWENO_ERR_STATE, "hweno_residual before hweno_set_state");
  choose_route(h);
  int rc = reset_diag(h);
  if (!rc) rc = residual_eval(h, h->Q, h->RHS, h->MOM);
  if (rc) return rc;
  h->have_residual = true;
  if (rhs && (rc = copy_planes_out(h, h->RHS, 12, rhs, on_device))) return rc;
  if (vhat && (rc = copy_planes_out(h, h->MOM, 8, vhat, on_device))) return rc;
  if ((rc = read_diag(h))) return rc;
  h->alpha = bits_to_double(h->h_diag->alpha_bits);
  h->beta = bits_to_double(h->h_diag->beta_bits);
  if (h->h_diag->flags & FLAG_TIMEOUT) return fail(h, HWENO_ERR_TIMEOUT, "a tensor copy's wait gave up");
  if (h->h_diag->flags & FLAG_NONFINITE) return fail(h, HWENO_ERR_NONFINITE, "non-finite residual");
  return HWENO_OK;
}

// one SSP-RK3 step from h->Q; on success the new state is in h->Q
// planes of the forward intermediates the reverse kernels read
// planes of the forward intermediates the reverse kernels read, kept per stage: the
// limited face and volume point values, the limiter factors, the weak moments, the
// gradients and the characteristic reconstruction data; the other scratch is shared
static const long long SEG_WORK_PLANES = 48 + 36 + 2 + 18 + 126 + YREC_PLANES;

static Work seg_work(hweno_handle* h, int n, int stage) {
  const long long ps = h->g.ps;
  double* p = h->spool + (long long)h->seg_max * 36 * ps + ((long long)n * 3 + stage) * SEG_WORK_PLANES * ps;
  Work w = h->w;  // the shared planes are the same in every scratch set
  w.face = p; p += 48 * ps;
  w.vol = p; p += 36 * ps;
  w.theta = p; p += 2 * ps;
  w.rm = p; p += 18 * ps;
  w.gr = p; p += 126 * ps;
  w.yrec = p;
  return w;
}

static double* seg_state(hweno_handle* h, int n, int k) {  // k = 0: q^n, 1: q1, 2: q2
  return h->spool + ((long long)n * 3 + k) * 12 * h->g.ps;
}


// restores the handle's scratch set on every exit of a scope that points it elsewhere
struct WorkGuard {
  hweno_handle* h;
  Work w;
  explicit WorkGuard(hweno_handle* hh) : h(hh), w(hh->w) {}
  ~WorkGuard() { h->w = w; }
};

static int do_step(hweno_handle* h, double dt_forced, double t_cap, double* dt_used, int* rejections) {
  const Grid& g = h->g;
  // recording for the adjoint: stage states (and intermediates) go to the next slot
  const int rec = h->recording ? h->rec_count : -1;
  if (rec >= h->seg_max && h->recording)
    return fail(h, HWENO_ERR_STATE, "recording more steps than hweno_adjoint_reserve allowed");
  const bool keep = rec >= 0 && h->seg_keep;
  WorkGuard wg(h);
  choose_route(h);
  double* q1 = rec >= 0 ? seg_state(h, rec, 1) : h->QS;
  double* q2 = rec >= 0 ? seg_state(h, rec, 2) : h->QS;
  if (keep) h->w = seg_work(h, rec, 0);
  int rc = reset_diag(h);
  if (!rc) rc = residual_eval(h, h->Q, h->RHS0, h->MOM0);
  if (rc) return rc;
  if (rec >= 0)  // q^n with its ghost cells, as the reverse reads it
    CK(cudaMemcpyAsync(seg_state(h, rec, 0), h->Q, (size_t)12 * g.ps * sizeof(double), cudaMemcpyDeviceToDevice,
                       h->st), "record copy");
  {
    Prof p(h, K_RK);
    k_dt<<<1, 1, 0, h->st>>>(h->d_diag, h->cfg.cfl, h_min(h), h->cfg.b_visc * h->cfg.Re * h_min(h) * h_min(h),
                             dt_forced, t_cap);
    k_stash<<<1, 1, 0, h->st>>>(h->d_diag);
    h->launches++;
  }
  // no host round trip until the attempt's stages are queued: the stages read dt on
  // the device, and the stage-1 flags wait in the second slot
  int rej = 0;
  for (;;) {
    // stage flags and counters of this attempt; keep dt and the stage-1 maxima
    CK(cudaMemsetAsync(&h->d_diag->pp_count, 0, sizeof(unsigned long long), h->st), "diag");
    CK(cudaMemsetAsync(&h->d_diag->flags, 0, sizeof(unsigned int), h->st), "diag");
    CK(cudaMemsetAsync(&h->d_diag->kefrac_bits, 0, sizeof(unsigned long long), h->st), "diag");
    if ((rc = launch_rk(h, 1, h->Q, h->MOM0, h->RHS0, q1))) return rc;
    if (keep) h->w = seg_work(h, rec, 1);
    // stage times of SSP-RK3 (a source term's t): t^n, t^n + dt, t^n + dt/2
    if ((rc = stage_eval_rk(h, q1, 2, q2, 1.0))) return rc;
    if (keep) h->w = seg_work(h, rec, 2);
    if ((rc = stage_eval_rk(h, q2, 3, h->QS, 0.5))) return rc;
    if ((rc = read_diag(h))) return rc;
    const Diag first = h->h_diag[1];
    const Diag& d = h->h_diag[0];
    if ((first.flags | d.flags) & FLAG_TIMEOUT) return fail(h, HWENO_ERR_TIMEOUT, "a tensor copy's wait gave up");
    if (first.flags & FLAG_NONFINITE) return fail(h, HWENO_ERR_NONFINITE, "non-finite residual at t^n");
    const double dt = d.dt;
    if (!(dt > 0.0) || !isfinite(dt)) return fail(h, HWENO_ERR_NONFINITE, "time step is not positive and finite");
    if (!(d.flags & (FLAG_INADMISSIBLE | FLAG_NONFINITE))) {
      double* tmp = h->Q;
      h->Q = h->QS;
      h->QS = tmp;
      h->alpha = bits_to_double(first.alpha_bits);
      const double b2 = bits_to_double(d.beta_bits), b1 = bits_to_double(first.beta_bits);
      h->beta = b1 > b2 ? b1 : b2;
      h->pp_total += (double)first.pp_count + (double)d.pp_count;
      h->cell_stages += 3.0 * g.nx * (double)g.ny;
      h->dt_last = dt;
      h->steps++;
      h->rejected += rej;
      if (h->cfg.precision == HWENO_MIXED) {
        h->ke_share = bits_to_double(d.kefrac_bits);
        if (h->route64) h->steps64++;
      }
      if (rec >= 0) {
        h->rec_dts.push_back(dt);
        h->rec_count++;
      }
      if (dt_used) *dt_used = dt;
      if (rejections) *rejections = rej;
      return HWENO_OK;
    }
    if (rej >= h->cfg.max_halvings) {
      h->rejected += rej;
      if (rejections) *rejections = rej;
      return fail(h, HWENO_ERR_INADMISSIBLE, "stage inadmissible after max_halvings restarts");
    }
    rej++;
    k_scale_dt<<<1, 1, 0, h->st>>>(h->d_diag, 0.5);
    h->launches++;
  }
}

int hweno_step(hweno_handle* h, double dt, double* dt_used, int* rejections) {
  if (!h) return HWENO_ERR_ARG;
  if (!h->have_state) return fail(h, HWENO_ERR_STATE, "hweno_step before hweno_set_state");
  double used = 0.0;
  int rc = do_step(h, dt > 0.0 ? dt : 0.0, INFINITY, &used, rejections);
  if (rc) return rc;
  h->t += used;
  h->have_residual = false;
  if (dt_used) *dt_used = used;
  return HWENO_OK;
}

int hweno_advance(hweno_handle* h, double t_end, int max_steps, double* t_reached, int* steps) {
  if (!h) return HWENO_ERR_ARG;
  if (!h->have_state) return fail(h, HWENO_ERR_STATE, "hweno_advance before hweno_set_state");
  int n = 0, rc = HWENO_OK;
  while (h->t < t_end && n < max_steps) {
    double used = 0.0;
    rc = do_step(h, 0.0, t_end - h->t, &used, nullptr);
    if (rc) break;
    h->t += used;
    n++;
    const double scale = fabs(t_end) > 1.0 ? fabs(t_end) : 1.0;
    if (t_end - h->t <= 1e-14 * scale) h->t = t_end;
  }
  h->have_residual = false;
  if (t_reached) *t_reached = h->t;
  if (steps) *steps = n;
  return rc;
}

int hweno_get_diag(hweno_handle* h, hweno_diag* d) {
  if (!h || !d) return HWENO_ERR_ARG;
  memset(d, 0, sizeof(*d));
  d->t = h->t;
  d->dt_last = h->dt_last;
  d->alpha_star = h->alpha;
  d->beta_max = h->beta;
  d->pp_active = h->pp_total;
  d->cell_stages = h->cell_stages;
  d->steps = h->steps;
  d->rejected = h->rejected;
  d->fp64_steps = h->steps64;
  d->max_kinetic_share = h->cfg.precision == HWENO_MIXED ? h->ke_share : 0.0;
  if (h->have_state) {
    k_state_rows<<<h->g.ny, 32, 0, h->st>>>(h->g, h->Q, h->PART);
    k_state_final<<<1, 32, 0, h->st>>>(h->g, h->PART, h->d_red);
    h->launches += 2;
    CK(cudaMemcpyAsync(h->h_red, h->d_red, 6 * sizeof(double), cudaMemcpyDeviceToHost, h->st), "diag");
    CK(cudaStreamSynchronize(h->st), "stream synchronize");
    for (int v = 0; v < 4; v++) d->totals[v] = h->h_red[v];
    d->min_rho = h->h_red[4];
    d->min_p = h->h_red[5];
  }
  return HWENO_OK;
}

int hweno_debug_fields(hweno_handle* h, int which, double* out, int on_device) {
  if (!h || !out) return fail(h, HWENO_ERR_ARG, "hweno_debug_fields: NULL argument");
  if (which < 0 || which > 4) return fail(h, HWENO_ERR_ARG, "hweno_debug_fields: unknown field set");
  if (!h->have_residual) return fail(h, HWENO_ERR_STATE, "hweno_debug_fields before hweno_residual");
  const Grid& g = h->g;
  const long long N = (long long)g.nx * g.ny;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (h->cfg.precision == HWENO_MIXED && !h->route64 && which <= 3) {
    // FP32 intermediates of the mixed path, widened to FP64; the weak moments and the
    // full gradient field from the separate kernels (the TMA-staged pass keeps the weak
    // moments in shared memory, and the operator's passes write no volume-point
    // gradients), on the traces of the last evaluation: the same values
    const WorkF f = mixed_planes(h->w, g.ps);
    if (which >= 2) mixed_grad_separate(h, true);
    if (which <= 1) {
      const int npts = which == 0 ? 12 : 9;
      const float* src = which == 0 ? f.face : f.vol;
      for (int k = 0; k < npts; k++) {
        k_gather_cons_f<<<256, 256, 0, h->st>>>(g, src + (long long)4 * k * g.ps, h->STAGE);
        h->launches++;
        CK(cudaMemcpyAsync(out + 4 * k * N, h->STAGE, 4 * N * sizeof(double), kind, h->st), "debug copy");
      }
    } else {
      const int n = which == 2 ? 18 : 126;
      const float* src = which == 2 ? f.rm : f.gr;
      for (int k = 0; k < n; k += 4) {
        const int m = n - k < 4 ? n - k : 4;
        k_gather_f<<<256, 256, 0, h->st>>>(g, m, src + (long long)k * g.ps, h->STAGE);
        h->launches++;
        CK(cudaMemcpyAsync(out + (long long)k * N, h->STAGE, m * N * sizeof(double), kind, h->st), "debug copy");
      }
    }
  } else if (which <= 1) {
    const int npts = which == 0 ? 12 : 9;
    const double* src = which == 0 ? h->w.face : h->w.vol;
    for (int k = 0; k < npts; k++) {
      k_gather_cons<<<256, 256, 0, h->st>>>(g, 1, src + (long long)4 * k * g.ps, h->STAGE);
      h->launches++;
      CK(cudaMemcpyAsync(out + 4 * k * N, h->STAGE, 4 * N * sizeof(double), kind, h->st), "debug copy");
    }
  } else {
    const int n = which == 2 ? 18 : (which == 3 ? 126 : 2);
    const double* src = which == 2 ? h->w.rm : (which == 3 ? h->w.gr : h->w.theta);
    int rc = copy_planes_out(h, src, n, out, on_device);
    if (rc) return rc;
  }
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  return HWENO_OK;
}

int hweno_profile(hweno_handle* h, int enable) {
  if (!h) return HWENO_ERR_ARG;
  h->prof = enable != 0;
  return HWENO_OK;
}

int hweno_profile_read(hweno_handle* h, int kernel, long long* launches, double* total_ms) {
  if (!h || kernel < 0 || kernel >= K_NKIND) return fail(h, HWENO_ERR_ARG, "hweno_profile_read: bad kernel");
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  for (auto& ep : h->ev) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ep.a, ep.b);
    h->prof_n[ep.kind]++;
    h->prof_ms[ep.kind] += ms;
    cudaEventDestroy(ep.a);
    cudaEventDestroy(ep.b);
  }
  h->ev.clear();
  if (launches) *launches = h->prof_n[kernel];
  if (total_ms) *total_ms = h->prof_ms[kernel];
  return HWENO_OK;
}

int hweno_measure_peak(hweno_handle* h, int which, double* tflops) {
  if (!h || !tflops || (which != 0 && which != 1)) return fail(h, HWENO_ERR_ARG, "hweno_measure_peak: bad argument");
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev), "device");
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "device attribute");
  const int threads = 256, blocks = sms * 8;
  const int iters = which == 0 ? 2048 : 65536;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a), "event");
  CK(cudaEventCreate(&b), "event");
  double best = 0.0;
  for (int rep = 0; rep < 3; rep++) {
    CK(cudaEventRecord(a, h->st), "event");
    if (which == 0) k_fma_peak<double><<<blocks, threads, 0, h->st>>>(h->STAGE, iters, 0.999999, 1e-6);
    else k_fma_peak<float><<<blocks, threads, 0, h->st>>>((float*)h->STAGE, iters, 0.999999f, 1e-6f);
    h->launches++;
    CK(cudaEventRecord(b, h->st), "event");
    CK(cudaEventSynchronize(b), "event");
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, a, b), "event");
    const double flops = 2.0 * 8.0 * 16.0 * (double)iters * threads * (double)blocks;
    const double tf = flops / (ms * 1e-3) / 1e12;
    if (tf > best) best = tf;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  *tflops = best;
  return HWENO_OK;
}

}  // extern "C"

// ===========================================================================
// Discrete adjoint of one SSP-RK3 step (FP64 path)

// (dR/dx)^T R + (dM/dx)^T M at the state x whose forward intermediates are in h->w
static int adjoint_operator(hweno_handle* h, const double* x) {
  const Grid& g = h->g;
  Adj& a = h->adj;
  if (!h->w.yrec) return fail(h, HWENO_ERR_STATE, "adjoint sweep without the forward's reconstruction record");
  const size_t P = (size_t)g.ps * sizeof(double);
  CK(cudaMemsetAsync(a.face, 0, 48 * P, h->st), "adjoint clear");
  CK(cudaMemsetAsync(a.vol, 0, 36 * P, h->st), "adjoint clear");
  CK(cudaMemsetAsync(a.gr, 0, 126 * P, h->st), "adjoint clear");
  const dim3 blk(BX, BY);
  ka_assemble<<<grid2(g.nx, g.ny), blk, 0, h->st>>>(g, h->w, a);
  ka_flux<<<grid2(g.nx + 1, g.ny + 1, 2), blk, 0, h->st>>>(g, h->w, a);
  if (h->cfg.linear_grad) ka_grad<true><<<grid2(g.nx + 2, g.ny + 2), blk, 0, h->st>>>(g, h->w, a);
  else ka_grad<<<grid2(g.nx + 2, g.ny + 2), blk, 0, h->st>>>(g, h->w, a);
  ka_gather_rm<<<grid2(g.nx + 4, g.ny + 4), blk, 0, h->st>>>(g, a);
  ka_face_moments<<<grid2(g.nx + 5, g.ny + 5, 2), blk, 0, h->st>>>(g, a);
  ka_cons<<<grid2(g.nx + 6, g.ny + 6), blk, 0, h->st>>>(g, x, h->w, a);
  ka_gather_q<<<grid2(g.nx + 8, g.ny + 8), blk, 0, h->st>>>(g, a);
  ka_ghost_y<<<(8 * (g.nx + 2 * NG) + 127) / 128, 128, 0, h->st>>>(g, a);
  ka_ghost_x<<<(8 * g.ny + 127) / 128, 128, 0, h->st>>>(g, a);
  h->launches += 9;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(h, e, "adjoint launch");
  return HWENO_OK;
}

extern "C" {

int hweno_adjoint_init(hweno_handle* h) {
  if (!h) return HWENO_ERR_ARG;
  if (h->cfg.precision != HWENO_FP64) return fail(h, HWENO_ERR_ARG, "the adjoint is implemented for HWENO_FP64");
  if (h->cfg.scheme != HWENO_SCHEME_GR || h->cfg.source != HWENO_SOURCE_NONE)
    return fail(h, HWENO_ERR_ARG, "the adjoint is implemented for HWENO_SCHEME_GR without a source term");
  if (h->apool) return HWENO_OK;
  const Grid& g = h->g;
  // R 12, M 8, face 48, vol 36, gr 126, rm 18, cg 102, cc 68, q 12, stage-1 state 12,
  // lambda 12, base adjoint 12, temporary 12, reconstruction record
  const long long nplanes = 12 + 8 + 48 + 36 + 126 + 18 + 102 + 68 + 12 + 12 * 4 + YREC_PLANES;
  const long long total = nplanes * g.ps + 8;
  CK(cudaMalloc(&h->apool, (size_t)total * sizeof(double)), "adjoint allocation");
  CK(cudaMemsetAsync(h->apool, 0, (size_t)total * sizeof(double), h->st), "adjoint clear");
  double* p = h->apool;
  auto take = [&](long long n) { double* r = p; p += n * g.ps; return r; };
  Adj& a = h->adj;
  a.R = take(12); a.M = take(8); a.face = take(48); a.vol = take(36); a.gr = take(126); a.rm = take(18);
  a.cg = take(102); a.cc = take(68); a.q = take(12);
  h->AST1 = take(12); h->ALAM = take(12); h->ABB = take(12); h->ATMP = take(12);
  h->AYREC = take(YREC_PLANES);
  a.mu = p;
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  return HWENO_OK;
}

extern "C" int hweno_adjoint_reserve(hweno_handle* h, int max_steps, int keep_intermediates) {
  if (!h || max_steps < 1) return fail(h, HWENO_ERR_ARG, "hweno_adjoint_reserve: bad argument");
  if (!h->apool) return fail(h, HWENO_ERR_STATE, "hweno_adjoint_reserve before hweno_adjoint_init");
  // storage that is large enough serves again, and so does storage whose request for
  // intermediates was already refused for lack of memory: reallocating it would drop
  // what has been recorded
  if (h->spool && h->seg_max >= max_steps && (h->seg_keep || !keep_intermediates || h->seg_keep_refused))
    return h->seg_keep ? 1 : HWENO_OK;
  if (h->spool) {
    CK(cudaStreamSynchronize(h->st), "stream synchronize");
    cudaFree(h->spool);
    h->spool = nullptr;
  }
  const long long ps = h->g.ps;
  long long planes = (long long)max_steps * 36;
  int keep = keep_intermediates ? 1 : 0;
  if (keep) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    const long long with = planes + (long long)max_steps * 3 * SEG_WORK_PLANES;
    if ((double)with * ps * sizeof(double) > 0.8 * (double)fr) keep = 0;  // fall back to recomputation
    else planes = with;
  }
  CK(cudaMalloc(&h->spool, (size_t)planes * ps * sizeof(double)), "adjoint segment allocation");
  h->rec_count = 0;
  h->rec_dts.clear();
  h->seg_max = max_steps;
  h->seg_keep = keep;
  h->seg_keep_refused = keep_intermediates && !keep;
  return keep ? 1 : HWENO_OK;
}

// the reverse sweep over the recorded steps rec_count-1 .. 0: lam (in h->ALAM) becomes
// the adjoint at the first recorded state; mu-bar accumulates in a.mu
static int adjoint_reverse(hweno_handle* h) {
  const Grid& g = h->g;
  Adj& a = h->adj;
  const bool keep = h->seg_keep != 0;
  WorkGuard wg(h);
  h->w.yrec = h->AYREC;  // for stages re-evaluated here
  int rc = HWENO_OK;
  const dim3 gi = grid2(g.nx, g.ny), blk(BX, BY);
  for (int n = h->rec_count - 1; n >= 0 && !rc; n--) {
    const double dt = h->rec_dts[n];
    double* st[3] = {seg_state(h, n, 0), seg_state(h, n, 1), seg_state(h, n, 2)};
    // stage 3 at q2, stage 2 at q1, stage 1 at q^n (the Shu-Osher weights of each stage)
    const double sr[3] = {dt, 0.25 * dt, (2.0 / 3.0) * dt}, sm[3] = {1.0, 0.25, 2.0 / 3.0};
    for (int stage = 2; stage >= 0 && !rc; stage--) {
      if (stage == 2) ka_axpby<<<gi, blk, 0, h->st>>>(g, h->ABB, 0.0, h->ALAM, 1.0 / 3.0);
      if (stage == 1) ka_axpby<<<gi, blk, 0, h->st>>>(g, h->ABB, 1.0, h->ALAM, 0.75);
      if (keep) h->w = seg_work(h, n, stage);
      else if ((rc = residual_eval(h, st[stage], h->RHS, h->MOM))) break;
      ka_seed<<<gi, blk, 0, h->st>>>(g, h->ALAM, sr[stage], sm[stage], stage == 0 ? h->ABB : nullptr, 1.0, a);
      if ((rc = adjoint_operator(h, st[stage]))) break;
      ka_finish<<<gi, blk, 0, h->st>>>(g, a, h->ALAM, sm[stage], stage == 0 ? h->ABB : nullptr, 1.0, h->ATMP);
      h->launches += 3;
      std::swap(h->ALAM, h->ATMP);
    }
  }
  if (rc) return rc;
  CK(cudaGetLastError(), "adjoint launch");
  return HWENO_OK;
}

// lam_start and mu-bar from h->ALAM and a.mu after a reverse sweep
static int adjoint_finish(hweno_handle* h, double* lam_start, double* mubar, int on_device) {
  int rc;
  if ((rc = copy_planes_out(h, h->ALAM, 12, lam_start, on_device))) return rc;
  double hm[2];
  CK(cudaMemcpyAsync(h->h_red, h->adj.mu, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st), "adjoint read");
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  memcpy(hm, h->h_red, sizeof(hm));
  if (mubar) *mubar = hm[0];
  return HWENO_OK;
}

extern "C" int hweno_adjoint_record(hweno_handle* h, int on) {
  if (!h) return HWENO_ERR_ARG;
  if (on && !h->spool) return fail(h, HWENO_ERR_STATE, "hweno_adjoint_record before hweno_adjoint_reserve");
  h->recording = on != 0;
  if (on) {
    h->rec_count = 0;
    h->rec_dts.clear();
  }
  return HWENO_OK;
}

extern "C" int hweno_adjoint_replay(hweno_handle* h, const double* lam_end, double* lam_start, double* mubar,
                                    int on_device) {
  if (!h || !lam_end || !lam_start) return fail(h, HWENO_ERR_ARG, "hweno_adjoint_replay: bad argument");
  if (!h->spool || h->rec_count < 1) return fail(h, HWENO_ERR_STATE, "hweno_adjoint_replay: no recorded steps");
  h->recording = false;
  int rc;
  if ((rc = copy_planes_in(h, lam_end, 12, h->ALAM, on_device))) return rc;
  CK(cudaMemsetAsync(h->adj.mu, 0, 2 * sizeof(double), h->st), "adjoint clear");
  if ((rc = adjoint_reverse(h))) return rc;
  return adjoint_finish(h, lam_start, mubar, on_device);
}

extern "C" int hweno_adjoint_segment(hweno_handle* h, const double* q_start, int nsteps, const double* dts,
                                     const double* lam_end, double* lam_start, double* mubar, int on_device) {
  if (!h || !q_start || !dts || !lam_end || !lam_start || nsteps < 1)
    return fail(h, HWENO_ERR_ARG, "hweno_adjoint_segment: bad argument");
  if (!h->spool || nsteps > h->seg_max)
    return fail(h, HWENO_ERR_STATE, "hweno_adjoint_segment: reserve storage for this many steps first");
  const bool keep = h->seg_keep != 0;
  h->recording = false;
  int rc;
  if ((rc = copy_planes_in(h, q_start, 12, seg_state(h, 0, 0), on_device))) return rc;
  if ((rc = copy_planes_in(h, lam_end, 12, h->ALAM, on_device))) return rc;
  if ((rc = reset_diag(h))) return rc;
  // forward recomputation of the segment with the given step sizes, keeping the stage
  // states (and intermediates)
  {
    WorkGuard wg(h);
    for (int n = 0; n < nsteps && !rc; n++) {
      double* q0 = seg_state(h, n, 0);
      double* q1 = seg_state(h, n, 1);
      double* q2 = seg_state(h, n, 2);
      double* out = n + 1 < nsteps ? seg_state(h, n + 1, 0) : h->QS;
      if (keep) h->w = seg_work(h, n, 0);
      if ((rc = residual_eval(h, q0, h->RHS0, h->MOM0))) break;
      k_dt<<<1, 1, 0, h->st>>>(h->d_diag, h->cfg.cfl, h_min(h), 1.0, dts[n], INFINITY);
      if ((rc = launch_rk(h, 1, q0, h->MOM0, h->RHS0, q1))) break;
      if (keep) h->w = seg_work(h, n, 1);
      if ((rc = residual_eval(h, q1, h->RHS, h->MOM))) break;
      if ((rc = launch_rk(h, 2, q1, h->MOM, h->RHS, q2))) break;
      if (keep) h->w = seg_work(h, n, 2);
      if ((rc = residual_eval(h, q2, h->RHS, h->MOM))) break;
      if ((rc = launch_rk(h, 3, q2, h->MOM, h->RHS, out))) break;
    }
  }
  if (rc) return rc;
  if ((rc = read_diag(h))) return rc;
  if (h->h_diag->flags & (FLAG_INADMISSIBLE | FLAG_NONFINITE))
    return fail(h, HWENO_ERR_INADMISSIBLE, "hweno_adjoint_segment: a forward stage is inadmissible at the given steps");
  h->rec_count = nsteps;
  h->rec_dts.assign(dts, dts + nsteps);
  CK(cudaMemsetAsync(h->adj.mu, 0, 2 * sizeof(double), h->st), "adjoint clear");
  if ((rc = adjoint_reverse(h))) return rc;
  h->rec_count = 0;
  h->have_state = false;  // the handle's state buffers hold segment data now
  return adjoint_finish(h, lam_start, mubar, on_device);
}

int hweno_adjoint_residual(hweno_handle* h, const double* x, const double* rbar, const double* mbar, double* xbar,
                           double* mubar, int on_device) {
  if (!h || !x || !xbar) return fail(h, HWENO_ERR_ARG, "hweno_adjoint_residual: bad argument");
  if (!h->apool) return fail(h, HWENO_ERR_STATE, "hweno_adjoint_residual before hweno_adjoint_init");
  const Grid& g = h->g;
  Adj& a = h->adj;
  WorkGuard wg(h);
  h->w.yrec = h->AYREC;
  int rc;
  h->split_of = nullptr;
  if ((rc = copy_planes_in(h, x, 12, h->Q, on_device))) return rc;
  h->have_state = true;
  const size_t P = (size_t)g.ps * sizeof(double);
  CK(cudaMemsetAsync(a.R, 0, 12 * P, h->st), "adjoint clear");
  CK(cudaMemsetAsync(a.M, 0, 8 * P, h->st), "adjoint clear");
  if (rbar && (rc = copy_planes_in(h, rbar, 12, a.R, on_device))) return rc;
  if (mbar && (rc = copy_planes_in(h, mbar, 8, a.M, on_device))) return rc;
  CK(cudaMemsetAsync(a.mu, 0, 2 * sizeof(double), h->st), "adjoint clear");
  if ((rc = reset_diag(h))) return rc;
  if ((rc = residual_eval(h, h->Q, h->RHS, h->MOM))) return rc;
  h->have_residual = true;
  if ((rc = adjoint_operator(h, h->Q))) return rc;
  if ((rc = copy_planes_out(h, a.q, 12, xbar, on_device))) return rc;
  double hm[2];
  CK(cudaMemcpyAsync(h->h_red, a.mu, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st), "adjoint read");
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  memcpy(hm, h->h_red, sizeof(hm));
  if (mubar) *mubar = hm[0];
  return HWENO_OK;
}

int hweno_adjoint_step(hweno_handle* h, const double* q, double dt, const double* lam_next, double* lam,
                       double* mubar, int on_device) {
  if (!h || !q || !lam_next || !lam || !(dt > 0.0)) return fail(h, HWENO_ERR_ARG, "hweno_adjoint_step: bad argument");
  if (!h->apool) return fail(h, HWENO_ERR_STATE, "hweno_adjoint_step before hweno_adjoint_init");
  const Grid& g = h->g;
  Adj& a = h->adj;
  WorkGuard wg(h);
  h->w.yrec = h->AYREC;
  int rc;
  h->split_of = nullptr;
  if ((rc = copy_planes_in(h, q, 12, h->Q, on_device))) return rc;
  if ((rc = copy_planes_in(h, lam_next, 12, h->ALAM, on_device))) return rc;
  h->have_state = true;
  h->have_residual = false;
  // forward stage states q1 (kept in AST1) and q2 (in QS), dt forced
  if ((rc = reset_diag(h))) return rc;
  if ((rc = residual_eval(h, h->Q, h->RHS0, h->MOM0))) return rc;
  k_dt<<<1, 1, 0, h->st>>>(h->d_diag, h->cfg.cfl, h_min(h), 1.0, dt, INFINITY);
  if ((rc = launch_rk(h, 1, h->Q, h->MOM0, h->RHS0, h->QS))) return rc;
  CK(cudaMemcpyAsync(h->AST1, h->QS, 12 * (size_t)g.ps * sizeof(double), cudaMemcpyDeviceToDevice, h->st), "stage copy");
  if ((rc = residual_eval(h, h->QS, h->RHS, h->MOM))) return rc;
  if ((rc = launch_rk(h, 2, h->QS, h->MOM, h->RHS, h->QS))) return rc;
  if ((rc = read_diag(h))) return rc;
  if (h->h_diag->flags & (FLAG_INADMISSIBLE | FLAG_NONFINITE)) return fail(h, HWENO_ERR_INADMISSIBLE, "hweno_adjoint_step: the forward step is inadmissible at this dt");
  CK(cudaMemsetAsync(a.mu, 0, 2 * sizeof(double), h->st), "adjoint clear");
  const dim3 gi = grid2(g.nx, g.ny), blk(BX, BY);
  // stage 3: q3 = B/3 + 2/3 G(q2):  Bbar = lam/3, G's seed 2/3 lam
  ka_axpby<<<gi, blk, 0, h->st>>>(g, h->ABB, 0.0, h->ALAM, 1.0 / 3.0);
  if ((rc = residual_eval(h, h->QS, h->RHS, h->MOM))) return rc;
  ka_seed<<<gi, blk, 0, h->st>>>(g, h->ALAM, dt * (2.0 / 3.0), 2.0 / 3.0, nullptr, 0.0, a);
  if ((rc = adjoint_operator(h, h->QS))) return rc;
  ka_finish<<<gi, blk, 0, h->st>>>(g, a, h->ALAM, 2.0 / 3.0, nullptr, 0.0, h->ATMP);
  std::swap(h->ALAM, h->ATMP);  // lam = q2bar
  // stage 2: q2 = 3/4 B + 1/4 G(q1)
  ka_axpby<<<gi, blk, 0, h->st>>>(g, h->ABB, 1.0, h->ALAM, 0.75);
  if ((rc = residual_eval(h, h->AST1, h->RHS, h->MOM))) return rc;
  ka_seed<<<gi, blk, 0, h->st>>>(g, h->ALAM, dt * 0.25, 0.25, nullptr, 0.0, a);
  if ((rc = adjoint_operator(h, h->AST1))) return rc;
  ka_finish<<<gi, blk, 0, h->st>>>(g, a, h->ALAM, 0.25, nullptr, 0.0, h->ATMP);
  std::swap(h->ALAM, h->ATMP);  // lam = q1bar
  // stage 1: q1 = G(q), B = [q_avg; M(q)]
  if ((rc = residual_eval(h, h->Q, h->RHS, h->MOM))) return rc;
  ka_seed<<<gi, blk, 0, h->st>>>(g, h->ALAM, dt, 1.0, h->ABB, 1.0, a);
  if ((rc = adjoint_operator(h, h->Q))) return rc;
  ka_finish<<<gi, blk, 0, h->st>>>(g, a, h->ALAM, 1.0, h->ABB, 1.0, h->ATMP);
  h->launches += 9;
  if ((rc = copy_planes_out(h, h->ATMP, 12, lam, on_device))) return rc;
  double hm[2];
  CK(cudaMemcpyAsync(h->h_red, a.mu, 2 * sizeof(double), cudaMemcpyDeviceToHost, h->st), "adjoint read");
  CK(cudaStreamSynchronize(h->st), "stream synchronize");
  memcpy(hm, h->h_red, sizeof(hm));
  if (mubar) *mubar = hm[0];
  return HWENO_OK;
}

}  // extern "C"

// ===========================================================================
// Batched ensembles: many independent problems advanced together, one launch of each
// kernel for all cases, one CUDA graph per SSP-RK3 step of the whole ensemble.

namespace {

struct BatchList {
  int bx = 32, by = 4;  // block shape of the kernels that use this list
  int total = 0;        // work items
  int grid = 0;         // persistent blocks
  int* d = nullptr;     // device: start[n+1], tx[n], ty[n]
  TileList tl() const { return TileList{d, d + (n + 1), d + (2 * n + 1)}; }
  int n = 0;
};
}  // namespace

struct hweno_batch {
  int n = 0;
  int mixed = 0;
  int dr = 0;   // HWENO-DR: kb_dr on the BR_GRAD list in place of the three gradient kernels
  int lin = 0;     // the linear-gradient ablation: the LIN instantiations of kb_grad
  int source = 0;  // some case has a source term: kb_source after each stage's balances
  // mixed: the cases' tensor maps for kb_grad_tma_mixed (tma: every case has them and the
  // batch holds at most BT_MAX_CASES cases; else the separate gradient kernels)
  bool tma = false;
  BatchTraceMaps* maps = nullptr;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  std::vector<hweno_handle*> h;
  CaseDev* d_cases = nullptr;
  CaseDev* h_cases = nullptr;  // pinned mirror
  Diag* d_diag = nullptr;
  Diag* h_diag = nullptr;      // pinned
  BatchList L[BR_N];
  cudaGraphExec_t exec = nullptr;
  long long launches = 0;
  int graph_launches = 0;  // kernels in the captured step graph
  int sms = 148;
  char err[512];
};

static int bfail(hweno_batch* b, int code, const char* msg) {
  if (b) snprintf(b->err, sizeof(b->err), "%s", msg);
  snprintf(g_init_err, sizeof(g_init_err), "%s", msg);
  return code;
}

#define BCK(call, where)                                                        \
  do {                                                                          \
    cudaError_t e_ = (call);                                                    \
    if (e_ != cudaSuccess) {                                                    \
      char m_[400];                                                             \
      snprintf(m_, sizeof(m_), "%s: %s", where, cudaGetErrorString(e_));        \
      return bfail(b, HWENO_ERR_CUDA, m_);                                      \
    }                                                                           \
  } while (0)

static int build_list(hweno_batch* b, int k, int bx, int by) {
  BatchList& L = b->L[k];
  std::vector<int> host(3 * b->n + 1);
  const int total = batch_layout(k, b->n, [&](int c) -> const Grid& { return b->h[c]->g; }, bx, by, host.data());
  L.n = b->n;
  L.bx = bx;
  L.by = by;
  L.total = total;
  if (!L.d) BCK(cudaMalloc(&L.d, host.size() * sizeof(int)), "batch work list");
  BCK(cudaMemcpyAsync(L.d, host.data(), host.size() * sizeof(int), cudaMemcpyHostToDevice, b->st), "batch list");
  BCK(cudaStreamSynchronize(b->st), "batch list");
  return HWENO_OK;
}

// persistent grid: blocks resident on all SMs at once, never more than the items
template <class K>
static int persistent_grid(hweno_batch* b, K kernel, int items, size_t smem = 0, int threads = 128) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  const int g = b->sms * per_sm;
  return items < g ? (items > 0 ? items : 1) : g;
}

// enqueue one SSP-RK3 step of every active case (no host synchronisation: capturable)
static void batch_enqueue_step(hweno_batch* b) {
  const int n = b->n;
  const dim3 blk1(128, 1);
  auto dims = [&](int k) { return dim3(b->L[k].bx, b->L[k].by); };
  auto grid = [&](int k) { return b->L[k].grid; };
  kb_reset<<<(n + 127) / 128, 128, 0, b->st>>>(b->d_cases, n);
  b->launches++;
  for (int stage = 1; stage <= 3; stage++) {
    const int which = stage == 1 ? 0 : 1;
    // mixed: stages 2 and 3 read the split their stage update wrote, and so does stage 1
    // of a case whose last accepted step wrote it (split_ok); the other cases' stage 1
    // splits its state (a case repeated after a rejected attempt, or set from outside)
    const int split = b->mixed && stage > 1;
    kb_ghost<<<grid(BR_GHOST), blk1, 0, b->st>>>(b->d_cases, b->L[BR_GHOST].tl(), n, which, split);
    b->launches++;
    if (b->mixed) {
      if (stage == 1) {
        kb_split<<<grid(BR_SPLIT), blk1, 0, b->st>>>(b->d_cases, b->L[BR_SPLIT].tl(), n, which);
        b->launches++;
      }
      kb_cons<1><<<grid(BR_CONS), dims(BR_CONS), 0, b->st>>>(b->d_cases, b->L[BR_CONS].tl(), n, which);
      b->launches++;
      if (b->tma) {
        // face moments, weak moments and gradients in one TMA-staged pass, as a handle does
        if (b->lin)
          kb_grad_tma_mixed<true><<<grid(BR_GT), GT_THREADS, GT_SMEM_BYTES, b->st>>>(b->d_cases, b->L[BR_GT].tl(), n,
                                                                                     *b->maps);
        else
          kb_grad_tma_mixed<false><<<grid(BR_GT), GT_THREADS, GT_SMEM_BYTES, b->st>>>(b->d_cases, b->L[BR_GT].tl(),
                                                                                      n, *b->maps);
        b->launches++;
      } else {
        kb_face_moments<1><<<grid(BR_FACE), dims(BR_FACE), 0, b->st>>>(b->d_cases, b->L[BR_FACE].tl(), n);
        kb_weak_moments<1><<<grid(BR_WEAK), dims(BR_WEAK), 0, b->st>>>(b->d_cases, b->L[BR_WEAK].tl(), n);
        if (b->lin) kb_grad<1, true><<<grid(BR_GRAD), dims(BR_GRAD), 0, b->st>>>(b->d_cases, b->L[BR_GRAD].tl(), n);
        else kb_grad<1><<<grid(BR_GRAD), dims(BR_GRAD), 0, b->st>>>(b->d_cases, b->L[BR_GRAD].tl(), n);
        b->launches += 3;
      }
      if (stage > 1 && !b->source) {
        // stages 2 and 3: fluxes, balances and the stage update in one tile kernel
        kb_flux_rk_mixed<<<grid(BR_FR), FR_THREADS, 0, b->st>>>(b->d_cases, b->L[BR_FR].tl(), n, stage);
        b->launches++;
        continue;
      }
      // a kept residual: fluxes and balances in one tile kernel
      kb_flux_asm_mixed<<<grid(BR_FRA), FR_THREADS, 0, b->st>>>(b->d_cases, b->L[BR_FRA].tl(), n, which);
      b->launches++;
    } else if (b->dr) {
      kb_cons<0, true><<<grid(BR_CONS), dims(BR_CONS), CONS_SMEM_BYTES, b->st>>>(b->d_cases, b->L[BR_CONS].tl(),
                                                                                 n, which);
      kb_dr<<<grid(BR_GRAD), dims(BR_GRAD), DR_SMEM_BYTES, b->st>>>(b->d_cases, b->L[BR_GRAD].tl(), n, which);
      kb_flux<<<grid(BR_FLUX), dims(BR_FLUX), 0, b->st>>>(b->d_cases, b->L[BR_FLUX].tl(), n);
      kb_assemble<<<grid(BR_INT), dims(BR_INT), 0, b->st>>>(b->d_cases, b->L[BR_INT].tl(), n, which);
      b->launches += 4;
    } else {
      kb_cons<0><<<grid(BR_CONS), dims(BR_CONS), CONS_SMEM_BYTES, b->st>>>(b->d_cases, b->L[BR_CONS].tl(), n,
                                                                           which);
      kb_face_moments<0><<<grid(BR_FACE), dims(BR_FACE), 0, b->st>>>(b->d_cases, b->L[BR_FACE].tl(), n);
      kb_weak_moments<0><<<grid(BR_WEAK), dims(BR_WEAK), 0, b->st>>>(b->d_cases, b->L[BR_WEAK].tl(), n);
      if (b->lin) kb_grad<0, true><<<grid(BR_GRAD), dims(BR_GRAD), 0, b->st>>>(b->d_cases, b->L[BR_GRAD].tl(), n);
      else kb_grad<0><<<grid(BR_GRAD), dims(BR_GRAD), 0, b->st>>>(b->d_cases, b->L[BR_GRAD].tl(), n);
      kb_flux<<<grid(BR_FLUX), dims(BR_FLUX), 0, b->st>>>(b->d_cases, b->L[BR_FLUX].tl(), n);
      kb_assemble<<<grid(BR_INT), dims(BR_INT), 0, b->st>>>(b->d_cases, b->L[BR_INT].tl(), n, which);
      b->launches += 6;
    }
    if (b->source) {
      // stage times of SSP-RK3: t^n, t^n + dt, t^n + dt/2 (stage 1's is t^n, before dt)
      const double cst = stage == 1 ? 0.0 : (stage == 2 ? 1.0 : 0.5);
      kb_source<<<grid(BR_INT), dims(BR_INT), 0, b->st>>>(b->d_cases, b->L[BR_INT].tl(), n, which, cst);
      b->launches++;
    }
    if (stage == 1) {
      kb_dt<<<(n + 127) / 128, 128, 0, b->st>>>(b->d_cases, n);
      b->launches++;
    }
    if (b->mixed) kb_rk<1><<<grid(BR_INT), dims(BR_INT), 0, b->st>>>(b->d_cases, b->L[BR_INT].tl(), n, stage);
    else kb_rk<0><<<grid(BR_INT), dims(BR_INT), 0, b->st>>>(b->d_cases, b->L[BR_INT].tl(), n, stage);
    b->launches++;
  }
}

static int batch_grids(hweno_batch* b) {
  b->L[BR_GHOST].grid = persistent_grid(b, kb_ghost, b->L[BR_GHOST].total);
  b->L[BR_SPLIT].grid = persistent_grid(b, kb_split, b->L[BR_SPLIT].total);
  if (b->mixed) {
    b->L[BR_CONS].grid = persistent_grid(b, kb_cons<1>, b->L[BR_CONS].total);
    b->L[BR_FACE].grid = persistent_grid(b, kb_face_moments<1>, b->L[BR_FACE].total);
    b->L[BR_WEAK].grid = persistent_grid(b, kb_weak_moments<1>, b->L[BR_WEAK].total);
    b->L[BR_GRAD].grid = b->lin ? persistent_grid(b, kb_grad<1, true>, b->L[BR_GRAD].total)
                                : persistent_grid(b, kb_grad<1>, b->L[BR_GRAD].total);
    if (b->tma)
      b->L[BR_GT].grid = b->lin ? persistent_grid(b, kb_grad_tma_mixed<true>, b->L[BR_GT].total, GT_SMEM_BYTES,
                                                  GT_THREADS)
                                : persistent_grid(b, kb_grad_tma_mixed<false>, b->L[BR_GT].total, GT_SMEM_BYTES,
                                                  GT_THREADS);
    b->L[BR_INT].grid = persistent_grid(b, kb_rk<1>, b->L[BR_INT].total);  // BR_FLUX: unused
    b->L[BR_FR].grid = persistent_grid(b, kb_flux_rk_mixed, b->L[BR_FR].total, 0, FR_THREADS);
    b->L[BR_FRA].grid = persistent_grid(b, kb_flux_asm_mixed, b->L[BR_FRA].total, 0, FR_THREADS);
  } else if (b->dr) {
    b->L[BR_CONS].grid = persistent_grid(b, kb_cons<0, true>, b->L[BR_CONS].total, CONS_SMEM_BYTES);
    b->L[BR_GRAD].grid = persistent_grid(b, kb_dr, b->L[BR_GRAD].total, DR_SMEM_BYTES, DR_THREADS);
    b->L[BR_FLUX].grid = persistent_grid(b, kb_flux, b->L[BR_FLUX].total);
    b->L[BR_INT].grid = persistent_grid(b, kb_assemble, b->L[BR_INT].total);
  } else {
    b->L[BR_CONS].grid = persistent_grid(b, kb_cons<0>, b->L[BR_CONS].total, CONS_SMEM_BYTES);
    b->L[BR_FACE].grid = persistent_grid(b, kb_face_moments<0>, b->L[BR_FACE].total);
    b->L[BR_WEAK].grid = persistent_grid(b, kb_weak_moments<0>, b->L[BR_WEAK].total);
    b->L[BR_GRAD].grid = b->lin ? persistent_grid(b, kb_grad<0, true>, b->L[BR_GRAD].total)
                                : persistent_grid(b, kb_grad<0>, b->L[BR_GRAD].total);
    b->L[BR_FLUX].grid = persistent_grid(b, kb_flux, b->L[BR_FLUX].total);
    b->L[BR_INT].grid = persistent_grid(b, kb_assemble, b->L[BR_INT].total);
  }
  return HWENO_OK;
}

static int batch_capture(hweno_batch* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  cudaGraph_t graph = nullptr;
  BCK(cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal), "graph capture begin");
  const long long l0 = b->launches;
  batch_enqueue_step(b);
  b->graph_launches = (int)(b->launches - l0);
  b->launches = l0;  // captured launches run (and are counted) at each replay
  BCK(cudaStreamEndCapture(b->st, &graph), "graph capture end");
  cudaError_t e = cudaGraphInstantiate(&b->exec, graph, 0);
  cudaGraphDestroy(graph);
  BCK(e, "graph instantiate");
  return HWENO_OK;
}

static int batch_upload(hweno_batch* b) {
  BCK(cudaMemcpyAsync(b->d_cases, b->h_cases, b->n * sizeof(CaseDev), cudaMemcpyHostToDevice, b->st),
      "batch case upload");
  return HWENO_OK;
}

static void batch_refresh_case(hweno_batch* b, int c) {
  hweno_handle* h = b->h[c];
  CaseDev& cd = b->h_cases[c];
  cd.g = h->g;
  cd.w = h->w;
  cd.open = h->open;
  cd.quad = h->quad;
  cd.t = h->t;
  cd.source = h->cfg.source;
  cd.Q = h->Q; cd.QS = h->QS; cd.BASE = h->BASE; cd.RHS0 = h->RHS0; cd.RHS = h->RHS;
  cd.MOM0 = h->MOM0; cd.MOM = h->MOM;
  cd.diag = b->d_diag + c;
  cd.cfl = h->cfg.cfl;
  cd.hmin = h_min(h);
  cd.visc_cap = h->cfg.b_visc * h->cfg.Re * cd.hmin * cd.hmin;
  cd.dt_scale = 1.0;
  cd.active = 1;
  cd.split_ok = b->mixed && h->split_of == h->Q ? 1 : 0;
}

extern "C" {

int hweno_batch_init(const hweno_config* cfgs, int ncases, void* stream, hweno_batch** out) {
  if (!out) return fail(nullptr, HWENO_ERR_ARG, "hweno_batch_init: out is NULL");
  *out = nullptr;
  if (!cfgs || ncases < 1) return fail(nullptr, HWENO_ERR_ARG, "hweno_batch_init: need at least one case");
  for (int c = 1; c < ncases; c++)
    if (cfgs[c].precision != cfgs[0].precision)
      return fail(nullptr, HWENO_ERR_ARG, "hweno_batch_init: all cases must use the same precision");
  for (int c = 0; c < ncases; c++) {
    if (cfgs[c].scheme != cfgs[0].scheme)
      return fail(nullptr, HWENO_ERR_ARG, "hweno_batch_init: all cases must use the same scheme");
    if (cfgs[c].scheme == HWENO_SCHEME_DR && cfgs[c].precision != HWENO_FP64)
      return fail(nullptr, HWENO_ERR_ARG, "hweno_batch_init: HWENO_SCHEME_DR runs in HWENO_FP64");
  }
  for (int c = 0; c < ncases; c++)
    if (check_inflow(cfgs[c])) return HWENO_ERR_ARG;
  for (int c = 0; c < ncases; c++)
    if (cfgs[c].linear_grad != cfgs[0].linear_grad)
      return fail(nullptr, HWENO_ERR_ARG, "hweno_batch_init: all cases must use the same linear_grad");
  // hweno_batch_step counts restart rounds for all cases together
  for (int c = 0; c < ncases; c++)
    if (cfgs[c].max_halvings != cfgs[0].max_halvings)
      return fail(nullptr, HWENO_ERR_ARG, "hweno_batch_init: all cases must use the same max_halvings");
  hweno_batch* b = new (std::nothrow) hweno_batch();
  if (!b) return fail(nullptr, HWENO_ERR_ARG, "host allocation failed");
  snprintf(b->err, sizeof(b->err), "no error");
  b->n = ncases;
  b->mixed = cfgs[0].precision == HWENO_MIXED;
  b->dr = cfgs[0].scheme == HWENO_SCHEME_DR;
  b->lin = cfgs[0].linear_grad != 0;
  for (int c = 0; c < ncases; c++)
    if (cfgs[c].source != HWENO_SOURCE_NONE) b->source = 1;
  b->st = (cudaStream_t)stream;
  if (!b->st) {  // graphs cannot be captured on the legacy default stream
    if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete b;
      return fail(nullptr, HWENO_ERR_CUDA, "hweno_batch_init: stream creation failed");
    }
    b->own_stream = true;
  }
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  int rc = HWENO_OK;
  for (int c = 0; c < ncases && !rc; c++) {
    hweno_handle* h = nullptr;
    rc = hweno_init(&cfgs[c], b->st, &h);
    if (!rc) b->h.push_back(h);
  }
  if (!rc) {
    cudaError_t e = cudaMalloc(&b->d_cases, ncases * sizeof(CaseDev));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_cases, ncases * sizeof(CaseDev));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_diag, ncases * sizeof(Diag));
    if (e == cudaSuccess) e = cudaMallocHost(&b->h_diag, ncases * sizeof(Diag));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_diag, 0, ncases * sizeof(Diag), b->st);
    if (e != cudaSuccess) rc = bfail(b, HWENO_ERR_CUDA, "hweno_batch_init: allocation failed");
  }
  if (!rc && b->mixed && ncases <= BT_MAX_CASES) {
    b->tma = true;
    for (int c = 0; c < ncases; c++) b->tma = b->tma && b->h[c]->tma;
    if (b->tma) {
      b->maps = new (std::nothrow) BatchTraceMaps();
      if (!b->maps) {
        b->tma = false;
      } else {
        for (int c = 0; c < ncases; c++) {
          b->maps->tr[c] = b->h[c]->tr_map;
          b->maps->wb[c] = b->h[c]->wb_map;
        }
      }
    }
  }
  for (int k = 0; k < BR_N && !rc; k++) {
    if (b->dr && k == BR_GRAD) rc = build_list(b, k, 32, DR_THREADS / 32);  // kb_dr's block
    else if (k == BR_FR || k == BR_FRA) rc = build_list(b, k, FR_TX, FR_TY);  // the mixed tile kernels
    else if (k == BR_GT) rc = build_list(b, k, GT_X, GT_Y);                   // kb_grad_tma_mixed's tiles
    else rc = build_list(b, k, k <= BR_INT ? 32 : 128, k <= BR_INT ? 4 : 1);
  }
  if (!rc) rc = batch_grids(b);
  if (!rc) {
    for (int c = 0; c < ncases; c++) batch_refresh_case(b, c);
    rc = batch_upload(b);
  }
  if (!rc) rc = batch_capture(b);
  if (rc) {
    hweno_batch_destroy(b);
    return rc;
  }
  *out = b;
  return HWENO_OK;
}

void hweno_batch_destroy(hweno_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto* h : b->h) hweno_destroy(h);
  for (int k = 0; k < BR_N; k++)
    if (b->L[k].d) cudaFree(b->L[k].d);
  if (b->d_cases) cudaFree(b->d_cases);
  if (b->h_cases) cudaFreeHost(b->h_cases);
  if (b->d_diag) cudaFree(b->d_diag);
  if (b->h_diag) cudaFreeHost(b->h_diag);
  if (b->own_stream) cudaStreamDestroy(b->st);
  delete b->maps;
  delete b;
}

const char* hweno_batch_last_error(const hweno_batch* b) { return b ? b->err : g_init_err; }

int hweno_batch_case(hweno_batch* b, int k, hweno_handle** h) {
  if (!b || !h || k < 0 || k >= b->n) return bfail(b, HWENO_ERR_ARG, "hweno_batch_case: bad index");
  *h = b->h[k];
  return HWENO_OK;
}

long long hweno_batch_launch_count(const hweno_batch* b) { return b ? b->launches : 0; }

// one replay of the step graph for the active cases, then the flags
static int batch_attempt(hweno_batch* b) {
  int rc = batch_upload(b);
  if (rc) return rc;
  BCK(cudaGraphLaunch(b->exec, b->st), "graph launch");
  b->launches += b->graph_launches;
  BCK(cudaMemcpyAsync(b->h_diag, b->d_diag, b->n * sizeof(Diag), cudaMemcpyDeviceToHost, b->st), "diag read");
  BCK(cudaStreamSynchronize(b->st), "stream synchronize");
  return HWENO_OK;
}

int hweno_batch_step(hweno_batch* b, int nsteps, int* rejections) {
  if (!b || nsteps < 0) return bfail(b, HWENO_ERR_ARG, "hweno_batch_step: bad argument");
  for (int c = 0; c < b->n; c++)
    if (!b->h[c]->have_state) return bfail(b, HWENO_ERR_STATE, "hweno_batch_step: a case has no state");
  int rej_total = 0;
  std::vector<int> pending(b->n);
  for (int s = 0; s < nsteps; s++) {
    for (int c = 0; c < b->n; c++) {
      batch_refresh_case(b, c);
      pending[c] = 1;
    }
    for (int round = 0;; round++) {
      int rc = batch_attempt(b);
      if (rc) return rc;
      int left = 0;
      for (int c = 0; c < b->n; c++)
        if (pending[c] && (b->h_diag[c].flags & FLAG_TIMEOUT))
          return bfail(b, HWENO_ERR_TIMEOUT, "hweno_batch_step: a tensor copy's wait gave up");
      for (int c = 0; c < b->n; c++) {
        if (!pending[c]) continue;
        const Diag& d = b->h_diag[c];
        hweno_handle* h = b->h[c];
        if (!(d.flags & (FLAG_INADMISSIBLE | FLAG_NONFINITE))) {
          double* tmp = h->Q;
          h->Q = h->QS;
          h->QS = tmp;
          // the accepted stage-3 update wrote the split of its output, the new Q
          h->split_of = b->mixed ? h->Q : nullptr;
          h->t += d.dt;
          h->dt_last = d.dt;
          h->steps++;
          h->rejected += round;
          h->pp_total += (double)d.pp_count;
          h->cell_stages += 3.0 * h->g.nx * (double)h->g.ny;
          h->alpha = bits_to_double(d.alpha_bits);
          h->beta = bits_to_double(d.beta_bits);
          h->have_residual = false;
          pending[c] = 0;
          b->h_cases[c].active = 0;
        } else {
          left++;
          b->h_cases[c].dt_scale *= 0.5;
          b->h_cases[c].active = 1;
          b->h_cases[c].split_ok = 0;  // the attempt's stage updates overwrote the split
          h->split_of = nullptr;
        }
      }
      if (!left) break;
      rej_total += left;
      if (round + 1 > b->h[0]->cfg.max_halvings) {
        if (rejections) *rejections = rej_total;
        return bfail(b, HWENO_ERR_INADMISSIBLE, "hweno_batch_step: a case stayed inadmissible after max_halvings restarts");
      }
    }
  }
  if (rejections) *rejections = rej_total;
  return HWENO_OK;
}

// Time each batched kernel of the spatial operator for the candidate block shapes on the
// current states (one step is computed and discarded, so the states do not change), keep
// the fastest shape per kernel, and re-capture the step graph.
int hweno_batch_autotune(hweno_batch* b, int* chosen) {
  if (!b) return bfail(b, HWENO_ERR_ARG, "hweno_batch_autotune: NULL batch");
  for (int c = 0; c < b->n; c++)
    if (!b->h[c]->have_state) return bfail(b, HWENO_ERR_STATE, "hweno_batch_autotune: a case has no state");
  static const int shapes[4][2] = {{32, 4}, {16, 8}, {64, 2}, {128, 1}};
  for (int c = 0; c < b->n; c++) batch_refresh_case(b, c);
  int rc = batch_upload(b);
  if (rc) return rc;
  batch_enqueue_step(b);  // fills every scratch plane; QS is overwritten next step anyway
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0), "event");
  BCK(cudaEventCreate(&e1), "event");
  const int n = b->n;
  for (int k = BR_CONS; k <= BR_INT; k++) {
    // HWENO-DR: kb_dr keeps its DR_THREADS block on the BR_GRAD list; the face- and
    // weak-moment lists are unused
    if (b->dr && (k == BR_FACE || k == BR_WEAK || k == BR_GRAD)) {
      if (chosen) chosen[k] = -1;
      continue;
    }
    // mixed: the face fluxes run in the flux tile kernels, whose tiles are fixed, and with
    // the tensor maps the gradient kinds in kb_grad_tma_mixed's fixed tiles
    if ((b->mixed && k == BR_FLUX) || (b->tma && (k == BR_FACE || k == BR_WEAK || k == BR_GRAD))) {
      if (chosen) chosen[k] = -1;
      continue;
    }
    float best = 1e30f;
    int bi = 0;
    for (int si = 0; si < 4; si++) {
      if ((rc = build_list(b, k, shapes[si][0], shapes[si][1]))) return rc;
      batch_grids(b);
      const dim3 blk(shapes[si][0], shapes[si][1]);
      const int gr = b->L[k].grid;
      const TileList tl = b->L[k].tl();
      float ms_sum = 0.f;
      for (int rep = 0; rep < 3; rep++) {
        BCK(cudaEventRecord(e0, b->st), "event");
        switch (k) {
          case BR_CONS:
            if (b->mixed) kb_cons<1><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n, 1);
            else if (b->dr) kb_cons<0, true><<<gr, blk, CONS_SMEM_BYTES, b->st>>>(b->d_cases, tl, n, 1);
            else kb_cons<0><<<gr, blk, CONS_SMEM_BYTES, b->st>>>(b->d_cases, tl, n, 1);
            break;
          case BR_FACE:
            if (b->mixed) kb_face_moments<1><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n);
            else kb_face_moments<0><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n);
            break;
          case BR_WEAK:
            if (b->mixed) kb_weak_moments<1><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n);
            else kb_weak_moments<0><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n);
            break;
          case BR_GRAD:
            if (b->mixed && b->lin) kb_grad<1, true><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n);
            else if (b->mixed) kb_grad<1><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n);
            else if (b->lin) kb_grad<0, true><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n);
            else kb_grad<0><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n);
            break;
          case BR_FLUX:
            kb_flux<<<gr, blk, 0, b->st>>>(b->d_cases, tl, n);
            break;
          default:
            // mixed: the list's kernel is the stage update (on the scratch stage state)
            if (b->mixed) kb_rk<1><<<gr, blk, 0, b->st>>>(b->d_cases, tl, n, 2);
            else kb_assemble<<<gr, blk, 0, b->st>>>(b->d_cases, tl, n, 1);
            break;
        }
        b->launches++;
        BCK(cudaEventRecord(e1, b->st), "event");
        BCK(cudaEventSynchronize(e1), "event");
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) ms_sum += ms;  // the first launch warms the caches
      }
      if (ms_sum < best) {
        best = ms_sum;
        bi = si;
      }
    }
    if ((rc = build_list(b, k, shapes[bi][0], shapes[bi][1]))) return rc;
    if (chosen) chosen[k] = bi;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // the discarded step and the timed stage updates overwrote the split planes
  for (int c = 0; c < b->n; c++) b->h[c]->split_of = nullptr;
  batch_grids(b);
  BCK(cudaStreamSynchronize(b->st), "stream synchronize");
  return batch_capture(b);
}

}  // extern "C"

// ===========================================================================
// Residual evaluation that allocates nothing: inputs and outputs are the caller's
// device buffers, and every intermediate plane lives in one library-static device
// array.  For callers that may not allocate device memory once they are running:
// programs whose device memory is owned by another allocator under a fixed budget
// (a framework's caching pool, a reserved arena), where a cudaMalloc can fail or
// fragment that budget, and latency-bound loops, where cudaMalloc's implicit
// device-wide synchronisation is not acceptable.

#include <mutex>

namespace {
// 12 state + 12 residual + 8 modified-moment planes, then the Work planes
constexpr long long NOALLOC_PLANES = 12 + 12 + 8 + 48 + 36 + 3 + 6 + 6 + 18 + 126 + 12 + 12 + 2;
// padded cells per plane: (ny + 8) * round_up(nx + 8, 16) may not exceed this
// (for example grids up to 56 x 56, or 120 x 24)
constexpr long long NOALLOC_MAX_PLANE = 4096;
constexpr long long NOALLOC_DOUBLES = NOALLOC_PLANES * NOALLOC_MAX_PLANE + 16;  // + Diag
static_assert(sizeof(Diag) <= 16 * sizeof(double), "the reductions' words fit the array's tail");
constexpr int NOALLOC_MAX_DEVICES = 64;
double* g_noalloc_addr[NOALLOC_MAX_DEVICES];  // device address of the array, per device
std::mutex g_noalloc_mu;
}  // namespace

// about 9.9 MB on every device that loads the library, held until the process exits
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_DOUBLES];

// host code cannot use g_noalloc_scratch as a device pointer: look its address up
// once per device, with that device current
static int noalloc_scratch_address(double** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "hweno_residual_noalloc: cudaGetDevice");
  if (dev < 0 || dev >= NOALLOC_MAX_DEVICES)
    return fail(nullptr, HWENO_ERR_ARG, "hweno_residual_noalloc: device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return cuda_fail(nullptr, e, "hweno_residual_noalloc: cudaGetSymbolAddress");
    g_noalloc_addr[dev] = (double*)p;
  }
  *out = g_noalloc_addr[dev];
  return HWENO_OK;
}

static int noalloc_check_config(const hweno_config& c) {
  if (c.nx < 4 || c.ny < 4) return fail(nullptr, HWENO_ERR_ARG, "nx and ny must be >= 4");
  if (!(c.x1 > c.x0) || !(c.y1 > c.y0)) return fail(nullptr, HWENO_ERR_ARG, "empty domain");
  if (!(c.gamma > 1.0) || !(c.Pr > 0.0) || !(c.Re > 0.0))
    return fail(nullptr, HWENO_ERR_ARG, "need gamma > 1, Pr > 0, Re > 0");
  for (int k = 0; k < 4; k++)
    if (!valid_bc(c.bc[k])) return fail(nullptr, HWENO_ERR_ARG, "unknown boundary condition");
  if ((c.bc[0] == HWENO_BC_PERIODIC) != (c.bc[1] == HWENO_BC_PERIODIC) ||
      (c.bc[2] == HWENO_BC_PERIODIC) != (c.bc[3] == HWENO_BC_PERIODIC))
    return fail(nullptr, HWENO_ERR_ARG, "periodic boundaries must be set on both sides");
  if (!(c.eps_pp > 0.0) || !(c.eps_weno > 0.0)) return fail(nullptr, HWENO_ERR_ARG, "eps_pp, eps_weno must be > 0");
  if (c.precision != HWENO_FP64 && c.precision != HWENO_MIXED)
    return fail(nullptr, HWENO_ERR_ARG, "precision must be HWENO_FP64 or HWENO_MIXED");
  if (c.scheme != HWENO_SCHEME_GR || c.source != HWENO_SOURCE_NONE)
    return fail(nullptr, HWENO_ERR_ARG, "hweno_residual_noalloc runs HWENO_SCHEME_GR without a source term");
  if (c.linear_grad != 0 && c.linear_grad != 1) return fail(nullptr, HWENO_ERR_ARG, "linear_grad must be 0 or 1");
  return check_inflow(c);
}

extern "C" int hweno_residual_noalloc(const hweno_config* cfg, const double* q, double* rhs, double* vhat,
                                      void* stream) {
  if (!cfg || !q || !rhs) return fail(nullptr, HWENO_ERR_ARG, "hweno_residual_noalloc: NULL argument");
  int rc = noalloc_check_config(*cfg);
  if (rc) return rc;
  const hweno_config& c = *cfg;
  const Grid g = make_grid(c);
  if (g.ps > NOALLOC_MAX_PLANE) {
    char buf[256];
    snprintf(buf, sizeof(buf),
             "hweno_residual_noalloc: grid %d x %d needs %lld padded cells per plane, the static "
             "scratch holds %lld ((ny + 8) * round_up(nx + 8, 16) must be <= %lld)",
             c.nx, c.ny, g.ps, NOALLOC_MAX_PLANE, NOALLOC_MAX_PLANE);
    return fail(nullptr, HWENO_ERR_ARG, buf);
  }

  double* base = nullptr;
  if ((rc = noalloc_scratch_address(&base))) return rc;
  // the same spatial operator as hweno_residual, on a stack handle whose planes all
  // point into the static array (no profiling, so the handle allocates nothing)
  hweno_handle tmp;
  tmp.cfg = c;
  tmp.st = (cudaStream_t)stream;
  tmp.g = g;
  tmp.open = make_open(c);
  double* p = base;
  auto take = [&](long long n) { double* r = p; p += n * g.ps; return r; };
  double* Q = take(12);
  double* R = take(12);
  double* M = take(8);
  tmp.w.face = take(48); tmp.w.vol = take(36); tmp.w.wbar = take(3); tmp.w.wx = take(6); tmp.w.wy = take(6);
  tmp.w.rm = take(18); tmp.w.gr = take(126); tmp.w.fx = take(12); tmp.w.fy = take(12); tmp.w.theta = take(2);
  tmp.d_diag = reinterpret_cast<Diag*>(p);
  tmp.prof = false;
  // the reductions accumulate into the Diag words: they start from zero on every call;
  // every other plane is written before it is read within the call
  cudaError_t e = cons_smem_allow();
  if (e == cudaSuccess) e = cudaMemsetAsync(tmp.d_diag, 0, sizeof(Diag), tmp.st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "hweno_residual_noalloc: clearing the reductions");
  k_scatter<<<256, 256, 0, tmp.st>>>(g, 12, q, Q);
  rc = residual_eval(&tmp, Q, R, M);
  if (rc) return fail(nullptr, rc, tmp.err);
  k_gather<<<256, 256, 0, tmp.st>>>(g, 12, R, rhs);
  if (vhat) k_gather<<<256, 256, 0, tmp.st>>>(g, 8, M, vhat);
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "hweno_residual_noalloc: launch");
  return HWENO_OK;
}
