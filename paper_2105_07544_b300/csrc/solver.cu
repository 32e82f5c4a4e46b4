// Host orchestration of the gmresb3 solver and its C ABI (include/gmresb3.h).
//
// A handle owns the matrix (FP64 values, their FP32 round-to-nearest copy, one int32 index set)
// and, per solver kind, a workspace: the Krylov basis V (ld x (m+1), column-major, ld a multiple
// of the 128-row tile), the work vector w, the small FP64 cycle state (H, Givens, g, scales),
// per-CTA partial sums and the polynomial buffers.  One restart cycle (m Arnoldi steps, the
// least-squares solve, x = x + p(A) V y and the FP64 residual of the next cycle) is captured
// once as a CUDA graph and replayed; the host reads one small status record per cycle.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstring>
#include <functional>
#include <memory>
#include <mutex>
#include <new>
#include <type_traits>
#include <vector>

#include "../../include/gmresb3.h"
#include "kernels.cuh"
#include "cluster_cycle.cuh"
#include "poly_host.h"
#include "bjacobi_host.h"
#include "handle_view.h"
#include <thread>

using namespace gmresb3;
typedef __nv_bfloat16 bf16;

namespace {

// ------------------------------------------------------------------------------------------------
// Error plumbing
// ------------------------------------------------------------------------------------------------
struct CudaFail {
  int code;
};
#define CK(call)                                                                   \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) throw CudaFail{e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM \
                                                                           : GMRES_ERR_CUDA}; \
  } while (0)

template <typename T> T* dalloc(size_t count) {
  void* p = nullptr;
  CK(cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
  return (T*)p;
}

// ------------------------------------------------------------------------------------------------
// Launch configuration
// ------------------------------------------------------------------------------------------------
struct Launch {
  int grid = 0;
  int stages = 1;   // sweep stages, or basis stages of an SpMV kernel
  int sc = 0;       // CSR stages of an SpMV kernel
  size_t smem = 0;
};

int g_num_sms(int dev) {
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  return v > 0 ? v : 1;
}

// Default target bytes per sweep stage and the cap on 128-row tiles grouped into one stage
// (on the 150^3 Laplacian: 16 KB 368.8 ms, 24 KB 365.1 ms, 32 KB 367.9 ms, 48 KB 398.4 ms per
// GMRES-IR solve).
constexpr size_t kStageTarget = 24 * 1024;
constexpr size_t kMaxTilesPerStage = 16;
constexpr size_t kSmemPerSm = 228 * 1024;    // shared memory of one SM (227 KB usable per CTA)
constexpr size_t kSmemReserve = 1024;        // per-CTA reservation of the runtime

// Let a kernel take the per-CTA maximum of dynamic shared memory (less its static part).
template <typename K> void allow_max_dynamic_smem(K kernel) {
  int dev = 0, optin = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  CK(cudaFuncGetAttributes(&fa, kernel));
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          optin - (int)fa.sharedSizeBytes));
}

// Pick stages and grid for a pipelined kernel.  ctas_per_sm = 0: prefer >= 2 stages within
// ~56 KB per CTA (4 CTAs per SM), then ~70 KB (3 per SM, with room for static shared memory),
// then ~112 KB, then whatever fits in one CTA per SM.  (Measured on the CGS2 sweeps at 150^3:
// three CTAs with two stages beat two CTAs with three or four stages by 5-15 %; fewer, deeper
// CTAs left some SMs finishing well after the rest.)
// ctas_per_sm = c > 0: size the stages for c resident CTAs per SM (fewer if they do not fit).
template <typename K>
Launch plan_pipelined(K kernel, size_t stage_bytes, size_t fixed, int ntiles, int sms,
                      int ctas_per_sm = 0) {
  static const size_t auto_budgets[] = {56 * 1024, 70 * 1024, 112 * 1024, 220 * 1024};
  size_t tuned[4];
  const size_t* budgets = auto_budgets;
  int nb = 4;
  if (ctas_per_sm > 0) {
    nb = 0;
    for (int c = std::min(ctas_per_sm, 4); c >= 1; --c)
      tuned[nb++] = std::min<size_t>(220 * 1024, kSmemPerSm / c - kSmemReserve);
    budgets = tuned;
  }
  Launch L;
  int st = 0;
  for (int i = 0; i < nb; ++i) {
    const size_t b = budgets[i];
    if (b <= fixed) continue;
    int s = (int)std::min<size_t>(kMaxStages, (b - fixed) / stage_bytes);
    if (s >= 2 || (i == nb - 1 && s >= 1)) {
      st = s;
      break;
    }
  }
  if (st < 1) throw CudaFail{GMRES_ERR_UNSUPPORTED};
  L.stages = st;
  L.smem = fixed + (size_t)st * stage_bytes;
  // Allow the per-CTA maximum, not this launch's size: a captured cycle holds launches of one
  // kernel with different sizes, and a graph node is checked against the kernel's attribute as
  // it stands when the node runs (a profiler's replay does), not as it stood at capture.
  int dev = 0, optin = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  CK(cudaFuncGetAttributes(&fa, kernel));
  if (L.smem + fa.sharedSizeBytes > (size_t)optin) throw CudaFail{GMRES_ERR_UNSUPPORTED};
  CK(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          optin - (int)fa.sharedSizeBytes));
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, L.smem));
  per_sm = std::max(1, std::min(per_sm, 8));
  L.grid = std::max(1, std::min(ntiles, sms * per_sm));
  return L;
}

// SpMV lanes per row from the mean nonzeros per row w: a row per thread up to w = 12 (its eight
// unrolled loads cover stencil rows), else the power of two L <= 32 with about five nonzeros per
// lane.
int auto_lanes(long n, long nnz) {
  const double w = n > 0 ? (double)nnz / (double)n : 0.0;
  if (w <= 12.0) return 1;
  int L = 2;
  while (L < 32 && 2.0 * L * 5.0 <= w) L *= 2;
  return L;
}

// Grid of a row-per-thread (lanes = 1) or lanes-per-row kernel (no shared memory): full
// occupancy (or ctas_per_sm CTAs per SM when that is lower), at most one row per lane group.
template <typename K> int plan_rows(K kernel, long n, int lanes, int sms, int ctas_per_sm = 0) {
  int per_sm = 0;
  CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
  per_sm = std::max(1, std::min(per_sm, 8));
  if (ctas_per_sm > 0) per_sm = std::min(per_sm, ctas_per_sm);
  const long need = (n * std::max(1, lanes) + kThreads - 1) / kThreads;
  return (int)std::max<long>(1, std::min<long>(need, (long)sms * per_sm));
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// Handle
// ------------------------------------------------------------------------------------------------
struct DevMatrix {
  int n = 0;
  long nnz = 0;
  int ntiles = 0;
  long ld = 0;             // padded vector length (ntiles * kTile)
  int* rowptr = nullptr;   // ld + 8 entries
  int* col = nullptr;      // nnz + 16
  double* v64 = nullptr;   // nnz + 16
  float* v32 = nullptr;    // nnz + 16
  int lanes = 1;            // SpMV lanes per row (from nonzeros per row, or the tuning)
  long blk_nnz[2] = {0, 0}; // most nonzeros in one block of 256 / 512 consecutive rows
  int* sptr = nullptr;      // sliced FP32 copy (SELL-32), or null
  int* scol = nullptr;
  float* sval = nullptr;
  Csr<double> csr64() const { return Csr<double>{n, lanes, rowptr, col, v64}; }
  Csr<float> csr32() const {
    Csr<float> c{n, lanes, rowptr, col, v32};
    c.sptr = sptr;
    c.scol = scol;
    c.sval = sval;
    return c;
  }
};

enum Kind { KIND_IR_F32 = 0, KIND_IR_BF16 = 1, KIND_F64 = 2, KIND_IR_F16 = 3, KIND_COUNT = 4 };

struct Workspace {
  Kind kind;
  int m = 0;               // allocated restart length
  long ld = 0;             // padded vector length
  long vts = 0;            // tile stride of the tile-blocked basis: (m + 1) * kTile
  void* V = nullptr;       // basis, [tile][column][kTile rows]
  void* w = nullptr;
  void* B[4] = {nullptr, nullptr, nullptr, nullptr};   // poly buffers B0, B1, B2 and Y
  void* Z = nullptr;       // cycle-end V y before p(A)
  double* x = nullptr;     // solution (internal copy)
  double* b = nullptr;     // right-hand side (internal copy)
  double* small = nullptr; // H, R, cs, sn, g, h1, h2, s, c
  double* part = nullptr;
  double* part2 = nullptr;
  unsigned* gcnt = nullptr;
  CycleState* st = nullptr;
  CycleState* st_host = nullptr;   // pinned mirror
  int maxgrid = 0;
  Krylov K{};
  cudaGraphExec_t graph = nullptr;
  int graph_m = -1;
  int graph_poly = -1;
  int graph_tuning = -1;
  int graph_mode = -1;
  int graph_launches = 0;
  ~Workspace() {
    if (graph) cudaGraphExecDestroy(graph);
    cudaFree(V);
    cudaFree(w);
    for (auto p : B) cudaFree(p);
    cudaFree(Z);
    cudaFree(x);
    cudaFree(b);
    cudaFree(small);
    cudaFree(part);
    cudaFree(part2);
    cudaFree(gcnt);
    cudaFree(st);
    if (st_host) cudaFreeHost(st_host);
  }
};

struct gmres_ctx {
  int dev = 0;
  int sms = 1;
  cudaStream_t stream = nullptr;       // private stream (graph capture and replay)
  cudaStream_t user_stream = nullptr;  // caller's stream, ordered with the private one by events
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  DevMatrix A;
  int m = 0;
  gmres_precisions_t prec{};
  gmres_params_t params{};
  gmres_tuning_t tuning{};                   // launch shapes (all 0 = the built-in heuristics)
  int tuning_gen = 0;                        // bumped by every change; graphs are keyed on it
  struct BlockJacobi {
    int k = 0;                 // block size (0 = no block Jacobi)
    int nblocks = 0;
    int* idx = nullptr;        // RCM order (or identity), n entries: block b = idx[b k .. b k + k)
    float* inv32 = nullptr;    // block inverses, [block][column][row] (k = 1: 1 / a_ii, natural order)
    double* inv64 = nullptr;
    std::vector<int32_t> perm;
    void release() {
      cudaFree(idx);
      cudaFree(inv32);
      cudaFree(inv64);
      *this = BlockJacobi{};
    }
  } bj;
  std::vector<std::complex<double>> roots;   // Leja-ordered roots of pi(t); empty = no poly
  std::vector<PolyStepDesc> sched;
  std::unique_ptr<Workspace> ws[KIND_COUNT];
  int64_t launches = 0;
  int expire_wait = 0;                       // test hook (gmres_test_expire_wait)
  std::vector<cudaEvent_t> prof_ev;         // profiling: an event pair per timed launch group
  ~gmres_ctx() {
    for (auto& w : ws) w.reset();
    bj.release();
    cudaFree(A.rowptr);
    cudaFree(A.col);
    cudaFree(A.v64);
    cudaFree(A.v32);
    cudaFree(A.sptr);
    cudaFree(A.scol);
    cudaFree(A.sval);
    if (ev_in) cudaEventDestroy(ev_in);
    if (ev_out) cudaEventDestroy(ev_out);
    for (auto e : prof_ev)
      if (e) cudaEventDestroy(e);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

size_t elem_size(Kind k) {
  return k == KIND_F64 ? 8 : ((k == KIND_IR_BF16 || k == KIND_IR_F16) ? 2 : 4);
}
size_t acc_size(Kind k) { return k == KIND_F64 ? 8 : 4; }

Workspace& get_ws(gmres_ctx& h, Kind kind, int m) {
  auto& slot = h.ws[kind];
  if (slot && slot->m >= m) return *slot;
  slot.reset();
  auto W = std::make_unique<Workspace>();
  W->kind = kind;
  W->m = m;
  W->ld = h.A.ld;
  W->vts = (long)(m + 1) * kTile;
  const size_t ld = (size_t)W->ld;
  const size_t sv = elem_size(kind), sa = acc_size(kind);
  CK(cudaMalloc(&W->V, ld * (m + 1) * sv));
  CK(cudaMemsetAsync(W->V, 0, ld * (m + 1) * sv, h.stream));
  CK(cudaMalloc(&W->w, ld * sa));
  CK(cudaMemsetAsync(W->w, 0, ld * sa, h.stream));
  for (auto& p : W->B) {
    CK(cudaMalloc(&p, ld * sa));
    CK(cudaMemsetAsync(p, 0, ld * sa, h.stream));
  }
  CK(cudaMalloc(&W->Z, ld * sa));
  CK(cudaMemsetAsync(W->Z, 0, ld * sa, h.stream));
  W->x = dalloc<double>(ld);
  CK(cudaMemsetAsync(W->x, 0, ld * 8, h.stream));
  W->b = dalloc<double>(ld);
  CK(cudaMemsetAsync(W->b, 0, ld * 8, h.stream));
  const size_t m1 = m + 1;
  const size_t nsmall = 2 * m1 * m + 2 * m + 7 * m1 + 8;
  W->small = dalloc<double>(nsmall);
  CK(cudaMemsetAsync(W->small, 0, nsmall * 8, h.stream));
  W->maxgrid = std::max(h.sms * 16, 64);
  W->part = dalloc<double>((size_t)W->maxgrid * kPartLd);
  CK(cudaMemsetAsync(W->part, 0, (size_t)W->maxgrid * kPartLd * 8, h.stream));
  const int gs2 = (W->maxgrid + kGroup - 1) / kGroup;
  W->part2 = dalloc<double>((size_t)gs2 * kPartLd);
  CK(cudaMemsetAsync(W->part2, 0, (size_t)gs2 * kPartLd * 8, h.stream));
  W->gcnt = dalloc<unsigned>((size_t)3 * gs2);
  CK(cudaMemsetAsync(W->gcnt, 0, (size_t)3 * gs2 * sizeof(unsigned), h.stream));
  W->st = dalloc<CycleState>(1);
  CK(cudaMemsetAsync(W->st, 0, sizeof(CycleState), h.stream));
  CK(cudaMallocHost(&W->st_host, sizeof(CycleState)));
  std::memset(W->st_host, 0, sizeof(CycleState));
  double* p = W->small;
  Krylov& K = W->K;
  K.H = p; p += m1 * m;
  K.R = p; p += m1 * m;
  K.cs = p; p += m;
  K.sn = p; p += m;
  K.g = p; p += m1;
  K.h1 = p; p += m1;
  K.h2 = p; p += m1;
  K.s = p; p += m1;
  K.c = p; p += m1;
  K.ca = p; p += m1;
  K.cb = p; p += m1;
  K.part = W->part;
  K.gs = W->maxgrid;   // partial-sum slots are column-major with this stride
  K.part2 = W->part2;
  K.gs2 = gs2;
  K.gcnt = W->gcnt;
  K.st = W->st;
  K.m = m;
  slot = std::move(W);
  return *slot;
}

// ------------------------------------------------------------------------------------------------
// Typed engine: launches of one solver kind
// ------------------------------------------------------------------------------------------------
// Optional per-class event timing (profiling mode, no graphs).
// Per-class device time of a profiled cycle.  Each timed launch group is bracketed by an event
// pair from a pool; the pairs are read only when the pool is full or the cycle has ended, so
// the kernels run back to back as in a graph (no host synchronisation between them).
constexpr int kProfPairs = 1024;
struct Prof {
  std::vector<cudaEvent_t>& ev;   // 2 kProfPairs events, created on first use
  cudaStream_t s;
  double t[8] = {0};
  int n = 0;
  int cls[kProfPairs];
  Prof(std::vector<cudaEvent_t>& pool, cudaStream_t st) : ev(pool), s(st) {
    while (ev.size() < 2 * (size_t)kProfPairs) {
      cudaEvent_t e;
      CK(cudaEventCreate(&e));
      ev.push_back(e);
    }
  }
  template <class F> void time(int c, F fn) {
    if (n == kProfPairs) flush();
    CK(cudaEventRecord(ev[2 * n], s));
    fn();
    CK(cudaEventRecord(ev[2 * n + 1], s));
    cls[n++] = c;
  }
  void flush() {
    if (n == 0) return;
    CK(cudaEventSynchronize(ev[2 * n - 1]));
    for (int i = 0; i < n; ++i) {
      float ms = 0.f;
      CK(cudaEventElapsedTime(&ms, ev[2 * i], ev[2 * i + 1]));
      t[cls[i]] += ms * 1e-3;
    }
    n = 0;
  }
};

// TA/TV/TW/ACC: matrix values, basis storage, w, accumulation.  PA/PACC: matrix values and
// vectors of the polynomial preconditioner (the FP64 solver may apply it in FP32: variant (a) of Section III-D).
template <typename TA, typename TV, typename TW, typename ACC, typename PA = TA,
          typename PACC = ACC>
struct Engine {
  typedef TV TVt;
  typedef ACC ACCt;
  gmres_ctx& h;
  Workspace& W;
  Prof* prof = nullptr;
  int launches = 0;
  bool fp32_outer = false;   // single-precision GMRES (FP32 residual)
  bool dc = h.params.orth == 1;   // DCGS2 (delayed second pass) instead of CGS2

  template <class F> void timed(int cls, F fn) {
    if (prof) prof->time(cls, fn);
    else fn();
  }

  Csr<TA> csr() const;
  Csr<PA> pcsr() const;

  void note(int n = 1) { launches += n; }

  // Traversal direction of the kernels that stream the basis or the matrix (the SpMVs, the
  // polynomial steps, the sweeps).  Each such launch runs against the previous one, so that it
  // starts on the tiles and rows its predecessor read last, which are still in the 126 MB L2.
  // The toggle restarts with every cycle, so a captured cycle and a directly launched one run
  // the same directions.
  int rev = 0;
  int flip() { return rev ^= 1; }

  // ---- inner SpMV of step j fused with the first projection: w = s_j A z_j, h1, ||w|| ----
  template <typename TX> void spmv_proj(VRef<TX> x, int j) {
    auto kern = k_spmv_proj<TA, TX, TV, TW, ACC>;
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0));
    per_sm = std::max(1, std::min(per_sm, 8));
    if (h.tuning.spmv_ctas_per_sm > 0) per_sm = std::min(per_sm, h.tuning.spmv_ctas_per_sm);
    const long need = ((long)h.A.n + kFusedRows * kWarps - 1) / (kFusedRows * kWarps);
    const int grid = (int)std::max<long>(1, std::min<long>({need, (long)h.sms * per_sm, (long)W.maxgrid}));
    kern<<<grid, kThreads, 0, h.stream>>>(csr(), x, (const TV*)W.V, W.vts, (TW*)W.w, W.K, j,
                                          flip());
    CK(cudaGetLastError());
    note();
  }

  // ---- FP64 solver: inner SpMV alone (w = s_j A z_j), then the projection sweep ----
  template <typename TX> void spmv_w(VRef<TX> x, int j) {
    auto kern = k_spmv_w<TA, TX, TW, ACC>;
    const int grid = std::min(plan_rows(kern, h.A.n, h.A.lanes, h.sms, h.tuning.spmv_ctas_per_sm), W.maxgrid);
    kern<<<grid, kThreads, 0, h.stream>>>(csr(), x, (TW*)W.w, W.K, j, flip());
    CK(cudaGetLastError());
    note();
  }
  void sweep_proj(int j) { sweep<SWEEP_PROJ>(j, nullptr, nullptr, (ACC*)nullptr); }

  // SpMV and first projection of step j: one fused kernel in FP32 arithmetic; the FP64 solver
  // (FP64-ALU bound) keeps them apart.
  static constexpr bool kFused = sizeof(ACC) == 4;
  template <typename TX> void spmv_and_proj(VRef<TX> x, int j) {
    if constexpr (kFused) {
      timed(GMRES_T_SPMV, [&] { spmv_proj<TX>(x, j); });
    } else {
      timed(GMRES_T_SPMV, [&] { spmv_w<TX>(x, j); });
      timed(GMRES_T_CGS_PROJ, [&] { sweep_proj(j); });
    }
  }

  // ---- DCGS2 (one reduction per step) ----
  // x = s_j A z with the one reduction of step j (spmv = 0: the cycle-end reduction only)
  template <typename TX> void dc_reduce(VRef<TX> x, int j, int spmv) {
    auto kern = k_dc_reduce<TA, TX, TV, TW, ACC>;
    int per_sm = 0;
    CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, 0));
    per_sm = std::max(1, std::min(per_sm, 8));
    if (h.tuning.spmv_ctas_per_sm > 0) per_sm = std::min(per_sm, h.tuning.spmv_ctas_per_sm);
    const long need = ((long)h.A.n + kFusedRows * kWarps - 1) / (kFusedRows * kWarps);
    const int grid = (int)std::max<long>(1, std::min<long>({need, (long)h.sms * per_sm, (long)W.maxgrid}));
    kern<<<grid, kThreads, 0, h.stream>>>(csr(), x, (const TV*)W.V, W.vts, (TW*)W.w, W.K, j, spmv,
                                          flip());
    CK(cudaGetLastError());
    note();
  }
  void dc_update(int j) {
    sweep<SWEEP_DC_UPDATE>(j, (TV*)W.V + (size_t)(j + 1) * kTile, nullptr, (ACC*)nullptr);
  }
  void dc_finish(int m) {
    timed(GMRES_T_CGS_PROJ, [&] {
      dc_reduce<TV>(VRef<TV>{(const TV*)W.V + (size_t)m * kTile, W.vts}, m, 0);
    });
  }

  void sweep_pass2(int j) { sweep<SWEEP_PASS2>(j, nullptr, nullptr, (ACC*)nullptr); }
  void sweep_update(int j) {
    sweep<SWEEP_UPDATE>(j, (TV*)W.V + (size_t)(j + 1) * kTile, nullptr, (ACC*)nullptr);
  }
  void sweep_solution(double* x64, ACC* z) { sweep<SWEEP_SOLUTION>(W.m, nullptr, x64, z); }

  template <int MODE> void sweep(int j, TV* vout, double* x64, ACC* z) {
    auto kern = k_sweep<MODE, TV, TW, ACC, ACC>;
    // the solution sweep reads st->k columns (<= m): size it for m
    const int ncols = (MODE == SWEEP_SOLUTION) ? W.m : j + 1;
    const size_t sw = (MODE == SWEEP_SOLUTION) ? 0 : sizeof(TW);   // PROJ/PASS2/UPDATE read w
    const size_t tile = (size_t)ncols * kTile * sizeof(TV) + align16((size_t)kTile * sw);
    // tiles per stage: ~16 KB per stage (or the tuned target) keeps enough bytes in flight at
    // small ncols
    const size_t target =
        h.tuning.sweep_stage_kb > 0 ? (size_t)h.tuning.sweep_stage_kb * 1024 : kStageTarget;
    const int rb = (int)std::max<size_t>(1, std::min<size_t>(kMaxTilesPerStage,
                                                             (target + tile - 1) / tile));
    const size_t fixed = sweep_smem_bytes(ncols, 0, sizeof(TV), sizeof(TW), sizeof(ACC),
                                          MODE == SWEEP_PASS2 ? rb : 0);
    const int ngroups = (h.A.ntiles + rb - 1) / rb;
    Launch L = plan_pipelined(kern, (size_t)rb * tile, fixed, ngroups, h.sms,
                              h.tuning.sweep_ctas_per_sm);
    L.grid = std::min(L.grid, W.maxgrid);
    kern<<<L.grid, kThreads, L.smem, h.stream>>>(h.A.n, (const TV*)W.V, W.vts, (const TW*)W.w, W.K,
                                                  j, L.stages, rb, vout, x64, z, flip());
    CK(cudaGetLastError());
    note();
  }

  void solve_small() {
    // R's columns staged in shared memory: (m + 1) m doubles for the workspace's m (the
    // attribute admits the per-CTA maximum, as for the sweeps)
    const size_t smem = (size_t)(W.K.m + 1) * W.K.m * sizeof(double);
    allow_max_dynamic_smem(k_solve);
    k_solve<<<1, kThreads, smem, h.stream>>>(W.K);
    CK(cudaGetLastError());
    note();
  }

  void residual(int first) {
    float* rs = is_half_v<TV> ? (float*)W.w : nullptr;   // FP16 basis: r staged in FP32
    if (fp32_outer) {   // single-precision GMRES: FP32 values and arithmetic
      auto kern = k_residual<TV, float>;
      const int grid = std::min(plan_rows(kern, h.A.n, h.A.lanes, h.sms), W.maxgrid);
      kern<<<grid, kThreads, 0, h.stream>>>(h.A.csr32(), W.x, W.b, (TV*)W.V, W.vts, W.K, first,
                                            rs);
    } else {
      auto kern = k_residual<TV>;
      const int grid = std::min(plan_rows(kern, h.A.n, h.A.lanes, h.sms), W.maxgrid);
      kern<<<grid, kThreads, 0, h.stream>>>(h.A.csr64(), W.x, W.b, (TV*)W.V, W.vts, W.K, first,
                                            rs);
    }
    CK(cudaGetLastError());
    note();
    if constexpr (is_half_v<TV>) {
      const int grid = std::min(h.sms * 4, W.maxgrid);
      k_v0_half<<<grid, kThreads, 0, h.stream>>>(h.A.n, rs, (__half*)W.V, W.vts, W.K);
      CK(cudaGetLastError());
      note();
    }
  }

  void bnorm() {
    const int grid = std::min(W.maxgrid, h.sms * 4);
    k_bnorm<<<grid, kThreads, 0, h.stream>>>(W.b, h.A.n, W.K);
    CK(cudaGetLastError());
    note();
  }

  template <typename TX, typename TP>
  void poly_step_launch(VRef<TX> x, VRef<TP> P, PACC* Pn, PACC* Y, const PolyCoef& c, int gate) {
    auto kern = k_poly_step<PA, TX, TP, PACC>;
    const int grid = plan_rows(kern, h.A.n, h.A.lanes, h.sms, h.tuning.spmv_ctas_per_sm);
    kern<<<grid, kThreads, 0, h.stream>>>(pcsr(), x, P, Pn, Y, PolyCoefT<PACC>::of(c), W.st, gate,
                                          flip());
    CK(cudaGetLastError());
    note();
  }

  // Apply the right preconditioner (block Jacobi or the polynomial) to `in`, result in Y = B[3].
  template <typename TIN> void precond_apply(VRef<TIN> in, int gate) {
    if (h.bj.k > 0) bj_apply<TIN>(in, gate);
    else poly_apply<TIN>(in, gate);
  }

  // Block Jacobi (Section III-D) in the polynomial's precision PACC (FP32 inverses inside
  // GMRES-IR and in the FP64 solver's FP32 variant, FP64 otherwise).
  template <typename TIN> void bj_apply(VRef<TIN> in, int gate) {
    PACC* Y = (PACC*)W.B[3];
    const PACC* inv = (const PACC*)(sizeof(PACC) == 4 ? (const void*)h.bj.inv32
                                                       : (const void*)h.bj.inv64);
    if (h.bj.k == 1) {
      k_diag_scale<TIN, PACC, PACC><<<h.sms * 4, kThreads, 0, h.stream>>>(in, Y, inv, h.A.n, W.st,
                                                                         gate);
    } else {
      const int grid = (h.bj.nblocks + kWarps - 1) / kWarps;
      k_bjacobi<TIN, PACC, PACC><<<grid, kThreads, 0, h.stream>>>(
          in, Y, h.bj.idx, inv, h.bj.k, h.A.n, h.bj.nblocks, W.st, gate);
    }
    CK(cudaGetLastError());
    note();
  }

  // Apply p(A) to `in` (type TIN) with the result in Y = B[3].
  template <typename TIN> void poly_apply(VRef<TIN> in, int gate) {
    PACC* buf[4] = {nullptr, (PACC*)W.B[0], (PACC*)W.B[1], (PACC*)W.B[2]};
    auto ref = [](PACC* p) { return VRef<PACC>{p, kTile}; };
    PACC* Y = (PACC*)W.B[3];
    for (const auto& d : h.sched) {
      PolyCoef c;
      c.cp_p = d.cp_p;
      c.cp_x = d.cp_x;
      c.cp_t = d.cp_t;
      c.cy_y = d.cy_y;
      c.cy_p = d.cy_p;
      c.cy_x = d.cy_x;
      c.cy_t = d.cy_t;
      c.cy_n = d.cy_n;
      c.write_p = d.pn != PB_NONE;
      c.write_y = d.write_y;
      c.read_y = d.read_y;
      PACC* Pn = d.pn == PB_NONE ? nullptr : buf[d.pn];
      if (d.x == PB_IN && d.p == PB_IN)
        poly_step_launch<TIN, TIN>(in, in, Pn, Y, c, gate);
      else if (d.x == PB_IN)
        poly_step_launch<TIN, PACC>(in, ref(buf[d.p]), Pn, Y, c, gate);
      else if (d.p == PB_IN)
        poly_step_launch<PACC, TIN>(ref(buf[d.x]), in, Pn, Y, c, gate);
      else
        poly_step_launch<PACC, PACC>(ref(buf[d.x]), ref(buf[d.p]), Pn, Y, c, gate);
    }
  }

  // One Arnoldi step j (0-based) of the inner cycle.
  void step(int j, bool poly) {
    const VRef<TV> vj{(const TV*)W.V + (size_t)j * kTile, W.vts};
    if (dc) {   // z = U_j (or p(A) U_j): SpMV with the one reduction, then the update
      if (poly) {
        timed(GMRES_T_PRECOND, [&] { precond_apply<TV>(vj, 1); });
        timed(GMRES_T_SPMV, [&] { dc_reduce<PACC>(VRef<PACC>{(const PACC*)W.B[3], kTile}, j, 1); });
      } else {
        timed(GMRES_T_SPMV, [&] { dc_reduce<TV>(vj, j, 1); });
      }
      timed(GMRES_T_CGS_UPDATE, [&] { dc_update(j); });
      return;
    }
    if (poly) {
      timed(GMRES_T_PRECOND, [&] { precond_apply<TV>(vj, 1); });
      spmv_and_proj<PACC>(VRef<PACC>{(const PACC*)W.B[3], kTile}, j);
    } else {
      spmv_and_proj<TV>(vj, j);
    }
    timed(GMRES_T_CGS_PASS2, [&] { sweep_pass2(j); });
    timed(GMRES_T_CGS_UPDATE, [&] { sweep_update(j); });
  }

  // Cycle end: y = R^{-1} g, x += p(A) V y, FP64 residual of the next cycle.
  void cycle_end(bool poly) {
    timed(GMRES_T_SOLUTION, [&] {
      solve_small();
      if (poly) {
        sweep_solution(nullptr, (ACC*)W.Z);
        precond_apply<ACC>(VRef<ACC>{(const ACC*)W.Z, kTile}, 2);
        const int grid = h.sms * 4;
        k_axpy_x<PACC><<<grid, 256, 0, h.stream>>>(W.x, (const PACC*)W.B[3], h.A.n, W.st);
        CK(cudaGetLastError());
        note();
      } else {
        sweep_solution(W.x, nullptr);
      }
    });
    timed(GMRES_T_RESIDUAL, [&] { residual(0); });
  }

  void cycle(int m, bool poly) {
    rev = 0;
    for (int j = 0; j < m; ++j) step(j, poly);
    if (dc) dc_finish(m);
    cycle_end(poly);
  }
};

template <typename T> Csr<T> csr_of(const DevMatrix& A);
template <> Csr<float> csr_of<float>(const DevMatrix& A) { return A.csr32(); }
template <> Csr<double> csr_of<double>(const DevMatrix& A) { return A.csr64(); }

template <typename TA, typename TV, typename TW, typename ACC, typename PA, typename PACC>
Csr<TA> Engine<TA, TV, TW, ACC, PA, PACC>::csr() const {
  return csr_of<TA>(h.A);
}
template <typename TA, typename TV, typename TW, typename ACC, typename PA, typename PACC>
Csr<PA> Engine<TA, TV, TW, ACC, PA, PACC>::pcsr() const {
  return csr_of<PA>(h.A);
}

typedef Engine<float, float, float, float> EngIR32;
typedef Engine<float, bf16, float, float> EngIR16;
typedef Engine<float, __half, float, float> EngIRh;   // FP16 basis (stored scaled)
typedef Engine<double, double, double, double> Eng64;
typedef Engine<double, double, double, double, float, float> Eng64P32;   // FP32 polynomial

// ------------------------------------------------------------------------------------------------
// Solve driver
// ------------------------------------------------------------------------------------------------
// The private stream is non-blocking: it does not synchronise with the legacy default stream by
// itself.  Every entry point that reads caller data first orders the private stream after the
// caller's stream (NULL = the legacy default stream) and orders the caller's stream after its
// own work before it returns.
void order_after_caller(gmres_ctx& h) {
  CK(cudaEventRecord(h.ev_in, h.user_stream));
  CK(cudaStreamWaitEvent(h.stream, h.ev_in, 0));
}

void order_caller_after(gmres_ctx& h) {
  CK(cudaEventRecord(h.ev_out, h.stream));
  CK(cudaStreamWaitEvent(h.user_stream, h.ev_out, 0));
}

void copy_in(gmres_ctx& h, double* dst, const double* src, size_t n) {
  CK(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, h.stream));
}

void read_state(gmres_ctx& h, Workspace& W) {
  CK(cudaMemcpyAsync(W.st_host, W.st, sizeof(CycleState), cudaMemcpyDeviceToHost, h.stream));
  CK(cudaStreamSynchronize(h.stream));
}

enum SolveMode { MODE_IR = 0, MODE_FP64 = 1, MODE_FP32 = 2 };

// Small systems: one restart cycle per launch of k_cycle_cluster on one thread-block cluster.
struct ClusterPlan {
  int nctas = 0;   // 0: the system does not qualify (the per-step kernels run)
  int rpt = 1;     // rows per thread (256 or 512 rows per CTA)
  int nnzcap = 0;  // staged nonzeros per CTA
  size_t smem = 0;
};

template <typename TA, typename TV, typename ACC, int RPT>
bool cluster_plan_try(gmres_ctx& h, const Workspace& W, ClusterPlan& out) {
  using L = ClusterSmem<TA, TV, ACC, RPT>;
  const long nctas = ((long)h.A.n + L::RS - 1) / L::RS;
  if (h.A.n < 1 || nctas > kClusterMax) return false;
  const long nnzcap = std::max<long>(4, (h.A.blk_nnz[RPT - 1] + 3) / 4 * 4);
  if (nnzcap > (1L << 20)) return false;
  const size_t smem = L::bytes(W.m, (int)nnzcap);
  auto kern = k_cycle_cluster<TA, TV, ACC, RPT>;
  int dev = 0, optin = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  cudaFuncAttributes fa{};
  CK(cudaFuncGetAttributes(&fa, kern));
  if (smem + fa.sharedSizeBytes > (size_t)optin) return false;
  // the per-CTA maximum, so that a launch of another size (another handle) stays valid
  CK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                          optin - (int)fa.sharedSizeBytes));
  if (nctas > 8) CK(cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1));
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)nctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)nctas);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  int clusters = 0;
  if (cudaOccupancyMaxActiveClusters(&clusters, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (clusters < 1) return false;
  out.nctas = (int)nctas;
  out.rpt = RPT;
  out.nnzcap = (int)nnzcap;
  out.smem = smem;
  return true;
}

// The plan for engine E: FP64 GMRES (FP64 basis) or GMRES-IR with an FP32 or BF16 basis, CGS2,
// no preconditioner, not profiling, cluster_cycle = 0.
template <typename E>
ClusterPlan cluster_plan(gmres_ctx& h, const Workspace& W, int mode, bool poly) {
  ClusterPlan p;
  const gmres_params_t& P = h.params;
  if (h.tuning.cluster_cycle != 0 || poly || P.orth != 0 || P.profiling || mode == MODE_FP32)
    return p;
  if constexpr (std::is_same<E, Eng64>::value) {
    if (!cluster_plan_try<double, double, double, 1>(h, W, p))
      cluster_plan_try<double, double, double, 2>(h, W, p);
  } else if constexpr (std::is_same<E, EngIR32>::value) {
    if (!cluster_plan_try<float, float, float, 1>(h, W, p))
      cluster_plan_try<float, float, float, 2>(h, W, p);
  } else if constexpr (std::is_same<E, EngIR16>::value) {
    if (!cluster_plan_try<float, bf16, float, 1>(h, W, p))
      cluster_plan_try<float, bf16, float, 2>(h, W, p);
  }
  return p;
}

template <typename TA, typename TV, typename ACC, int RPT>
void cluster_launch_t(gmres_ctx& h, Workspace& W, const ClusterPlan& p) {
  cudaLaunchConfig_t cfg{};
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = (unsigned)p.nctas;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.gridDim = dim3((unsigned)p.nctas);
  cfg.blockDim = dim3(kClusterThreads);
  cfg.dynamicSmemBytes = p.smem;
  cfg.stream = h.stream;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const ClusterShape cs{h.A.n, p.nctas, W.m, p.nnzcap, W.vts};
  CK(cudaLaunchKernelEx(&cfg, k_cycle_cluster<TA, TV, ACC, RPT>, csr_of<TA>(h.A), h.A.csr64(),
                        (const double*)W.b, W.x, (TV*)W.V, W.K, cs));
}

template <typename E> void cluster_launch(gmres_ctx& h, Workspace& W, const ClusterPlan& p) {
  if constexpr (std::is_same<E, Eng64>::value) {
    if (p.rpt == 1) cluster_launch_t<double, double, double, 1>(h, W, p);
    else cluster_launch_t<double, double, double, 2>(h, W, p);
  } else if constexpr (std::is_same<E, EngIR32>::value) {
    if (p.rpt == 1) cluster_launch_t<float, float, float, 1>(h, W, p);
    else cluster_launch_t<float, float, float, 2>(h, W, p);
  } else if constexpr (std::is_same<E, EngIR16>::value) {
    if (p.rpt == 1) cluster_launch_t<float, bf16, float, 1>(h, W, p);
    else cluster_launch_t<float, bf16, float, 2>(h, W, p);
  }
}

// Solve modes: GMRES-IR (Algorithm 2), FP64 GMRES (Algorithm 1), and single-precision GMRES
// (Algorithm 1 in FP32 throughout: FP32 b, residual and update; the first phase of GMRES-FD).

template <typename E>
int run_solve(gmres_ctx& h, Workspace& W, const double* b, double* x, double tol,
              gmres_stats_t* stats, int mode) {
  const bool fp64 = mode == MODE_FP64;
  const bool gmres_stop = mode != MODE_IR;   // implicit test at tol ||b||, loss-of-accuracy
  auto t0 = std::chrono::steady_clock::now();
  const gmres_params_t& P = h.params;
  const int m = P.m > 0 ? P.m : h.m;
  const bool poly = !h.sched.empty() || h.bj.k > 0;   // right-preconditioned
  if (P.orth == 1 && is_half_v<typename E::TVt>) throw CudaFail{GMRES_ERR_UNSUPPORTED};
  E eng{h, W};
  eng.fp32_outer = mode == MODE_FP32;
  double tk[8] = {0};
  const size_t n = (size_t)h.A.n;

  order_after_caller(h);
  copy_in(h, W.b, b, n);
  copy_in(h, W.x, x, n);
  if (mode == MODE_FP32) {
    // single precision throughout: b and the initial guess are rounded to FP32
    k_round_f32<<<h.sms * 4, 256, 0, h.stream>>>(W.b, (long)n);
    k_round_f32<<<h.sms * 4, 256, 0, h.stream>>>(W.x, (long)n);
    CK(cudaGetLastError());
    eng.note(2);
  }

  CycleState init{};
  init.jmax = m;
  init.implicit_fp64 = gmres_stop ? 1 : 0;
  init.fp32_outer = mode == MODE_FP32 ? 1 : 0;
  init.tol = tol;
  init.inner_tol = gmres_stop ? 0.0 : P.inner_tol;
  init.uround = fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
  init.expire_wait = h.expire_wait;
  h.expire_wait = 0;   // the hook arms one solve
  CK(cudaMemcpyAsync(W.st, &init, sizeof(CycleState), cudaMemcpyHostToDevice, h.stream));
  eng.bnorm();
  eng.residual(1);
  read_state(h, W);

  gmres_stats_t S{};
  if (stats) {
    S.res_history = stats->res_history;
    S.res_history_cap = stats->res_history_cap;
  }
  auto hist = [&](double v) {
    if (S.res_history && S.res_history_len < S.res_history_cap) S.res_history[S.res_history_len] = v;
    S.res_history_len++;
  };
  CycleState* hs = W.st_host;
  const double bnorm = hs->bnorm;
  int status = GMRES_NOT_CONVERGED;
  if (!(bnorm > 0.0) || !std::isfinite(bnorm)) {
    // b = 0: x = 0 solves exactly; NaN/Inf in b: report
    if (bnorm == 0.0) {
      CK(cudaMemsetAsync(W.x, 0, n * 8, h.stream));
      status = GMRES_OK;
      S.rel_res_explicit = 0.0;
    } else {
      status = GMRES_NAN;
      S.rel_res_explicit = NAN;
    }
    hist(S.rel_res_explicit);
  } else {
    hist(hs->rel_res);
    double best = hs->rel_res;
    int stall = 0;
    if (hs->converged) status = GMRES_OK;
    else if (hs->nan) status = GMRES_NAN;
    const bool use_graph = P.use_graphs && !P.profiling;
    const ClusterPlan cp = cluster_plan<E>(h, W, mode, poly);
    while (status == GMRES_NOT_CONVERGED) {
      const int64_t left = P.maxiter - S.iters;
      if (left <= 0) break;
      if (P.time_limit_s > 0) {
        const double el =
            std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
        if (el > P.time_limit_s) break;
      }
      const int jm = (int)std::min<int64_t>(m, left);
      if (jm != hs->jmax) {
        // shorter last cycle: the step kernels beyond jmax return at once
        CK(cudaMemcpyAsync(&W.st->jmax, &jm, sizeof(int), cudaMemcpyHostToDevice, h.stream));
        hs->jmax = jm;
      }
      if (cp.nctas > 0) {
        cluster_launch<E>(h, W, cp);
        eng.note();
      } else if (use_graph) {
        if (!W.graph || W.graph_m != m || W.graph_poly != (int)poly ||
            W.graph_tuning != h.tuning_gen || W.graph_mode != mode + 8 * P.orth) {
          if (W.graph) {
            cudaGraphExecDestroy(W.graph);
            W.graph = nullptr;
          }
          cudaGraph_t g;
          CK(cudaStreamBeginCapture(h.stream, cudaStreamCaptureModeThreadLocal));
          E cap{h, W};
          cap.fp32_outer = eng.fp32_outer;
          try {
            cap.cycle(m, poly);
          } catch (...) {
            cudaStreamEndCapture(h.stream, &g);
            if (g) cudaGraphDestroy(g);
            throw;
          }
          CK(cudaStreamEndCapture(h.stream, &g));
          cudaError_t e = cudaGraphInstantiate(&W.graph, g, 0);
          cudaGraphDestroy(g);
          CK(e);
          W.graph_m = m;
          W.graph_poly = (int)poly;
          W.graph_tuning = h.tuning_gen;
          W.graph_mode = mode + 8 * P.orth;
          W.graph_launches = cap.launches;
        }
        CK(cudaGraphLaunch(W.graph, h.stream));
        eng.launches += W.graph_launches;
      } else if (P.profiling) {
        Prof pr(h.prof_ev, h.stream);
        eng.prof = &pr;
        eng.cycle(m, poly);
        eng.prof = nullptr;
        pr.flush();
        for (int i = 0; i < 8; ++i) tk[i] += pr.t[i];
      } else {
        eng.cycle(m, poly);
      }
      read_state(h, W);
      S.iters += hs->last_k;
      S.cycles += 1;
      hist(hs->rel_res);
      S.rel_res_implicit = gmres_stop ? hs->last_implicit / bnorm
                                : hs->last_implicit / std::max(hs->gamma, 1e-300);
      if (hs->err) {   // a bulk-copy wait ran out; the cycle's results are not used
        status = GMRES_TIMEOUT;
        break;
      }
      if (hs->nan) {
        status = GMRES_NAN;
        break;
      }
      if (hs->converged) {
        status = GMRES_OK;
        break;
      }
      if (gmres_stop && hs->loa > P.max_loss_of_accuracy) {
        status = GMRES_LOSS_OF_ACCURACY;
        break;
      }
      if (!gmres_stop && P.stagnation_cycles > 0) {
        if (hs->rel_res < 0.9 * best) {
          best = hs->rel_res;
          stall = 0;
        } else if (++stall >= P.stagnation_cycles) {
          status = GMRES_STAGNATION;
          break;
        }
      }
      if (hs->last_k <= 0) break;  // no progress possible
    }
    S.rel_res_explicit = hs->rel_res;
    S.loss_of_accuracy = hs->loa;
    S.breakdowns = hs->breakdowns;
  }
  CK(cudaMemcpyAsync(x, W.x, n * sizeof(double), cudaMemcpyDefault, h.stream));
  order_caller_after(h);
  CK(cudaStreamSynchronize(h.stream));
  S.status = status;
  S.kernel_launches = eng.launches;
  for (int i = 0; i < 8; ++i) S.t_kernel[i] = tk[i];
  S.solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = S;
  return status;
}

}  // namespace

// ------------------------------------------------------------------------------------------------
// Setup helpers
// ------------------------------------------------------------------------------------------------
namespace {

int validate_csr_host(int64_t n, int64_t nnz, const int32_t* rp, const int32_t* ci, const double* v) {
  if (rp[0] != 0 || rp[n] != nnz) return GMRES_ERR_INVALID_ARG;
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return GMRES_ERR_INVALID_ARG;
  for (int64_t p = 0; p < nnz; ++p) {
    if (ci[p] < 0 || ci[p] >= n) return GMRES_ERR_INVALID_ARG;
    if (!std::isfinite(v[p])) return GMRES_ERR_INVALID_ARG;
  }
  return GMRES_OK;
}

void upload_matrix(gmres_ctx& h, const gmres_csr_t* A) {
  DevMatrix& M = h.A;
  M.n = (int)A->n;
  M.nnz = A->nnz;
  M.ntiles = (int)((A->n + kTile - 1) / kTile);
  M.ld = (long)M.ntiles * kTile;
  // host staging with padding: rowptr entries past n repeat nnz; col/val padded with zeros
  std::vector<int32_t> rp((size_t)M.ld + 8, (int32_t)A->nnz);
  std::vector<int32_t> ci((size_t)A->nnz + 16, 0);
  std::vector<double> va((size_t)A->nnz + 16, 0.0);
  const size_t n1 = (size_t)A->n + 1;
  order_after_caller(h);
  CK(cudaMemcpyAsync(rp.data(), A->rowptr, n1 * 4, cudaMemcpyDefault, h.stream));
  if (A->nnz > 0) {
    CK(cudaMemcpyAsync(ci.data(), A->colidx, (size_t)A->nnz * 4, cudaMemcpyDefault, h.stream));
    CK(cudaMemcpyAsync(va.data(), A->val, (size_t)A->nnz * 8, cudaMemcpyDefault, h.stream));
  }
  CK(cudaStreamSynchronize(h.stream));
  for (size_t i = n1; i < rp.size(); ++i) rp[i] = (int32_t)A->nnz;
  const int v = validate_csr_host(A->n, A->nnz, rp.data(), ci.data(), va.data());
  if (v != GMRES_OK) throw CudaFail{v};
  M.lanes = auto_lanes(M.n, M.nnz);
  for (int q = 0; q < 2; ++q) {   // row blocks of the cluster cycle (256 or 512 rows per CTA)
    const long rs = 256L << q;
    for (long r0 = 0; r0 < M.n; r0 += rs)
      M.blk_nnz[q] = std::max<long>(M.blk_nnz[q], (long)rp[(size_t)std::min<long>(r0 + rs, M.n)] - rp[(size_t)r0]);
  }
  M.rowptr = dalloc<int>(rp.size());
  M.col = dalloc<int>(ci.size());
  M.v64 = dalloc<double>(va.size());
  M.v32 = dalloc<float>(va.size());
  // Uploads on the private stream: a plain cudaMemcpy from pageable memory may return before its
  // DMA lands, and the non-blocking private stream would not wait for it (the cast below reads v64).
  CK(cudaMemcpyAsync(M.rowptr, rp.data(), rp.size() * 4, cudaMemcpyHostToDevice, h.stream));
  CK(cudaMemcpyAsync(M.col, ci.data(), ci.size() * 4, cudaMemcpyHostToDevice, h.stream));
  CK(cudaMemcpyAsync(M.v64, va.data(), va.size() * 8, cudaMemcpyHostToDevice, h.stream));
  k_cast_f64_f32<<<h.sms * 4, 256, 0, h.stream>>>(M.v64, M.v32, (long)va.size());
  CK(cudaGetLastError());
  // SELL-32 copy of the FP32 matrix for the row-per-thread SpMV kernels, when padding the slices
  // to their longest row adds at most a quarter to the nonzeros
  {
    const long nsl = (M.n + 31) / 32;
    std::vector<int32_t> sp((size_t)nsl + 2, 0);
    long tot = 0;
    for (long s = 0; s < nsl; ++s) {
      int w = 0;
      for (long r = 32 * s; r < std::min<long>(32 * s + 32, M.n); ++r) w = std::max(w, rp[r + 1] - rp[r]);
      sp[(size_t)s] = (int32_t)std::min<long>(tot, INT32_MAX);
      tot += 32L * w;
    }
    sp[(size_t)nsl] = sp[(size_t)nsl + 1] = (int32_t)std::min<long>(tot, INT32_MAX);
    if (M.n > 0 && tot <= (long)(1.25 * (double)M.nnz) + 32 && tot < INT32_MAX - 64) {
      M.sptr = dalloc<int>(sp.size());
      M.scol = dalloc<int>((size_t)tot + 16);
      M.sval = dalloc<float>((size_t)tot + 16);
      CK(cudaMemcpyAsync(M.sptr, sp.data(), sp.size() * 4, cudaMemcpyHostToDevice, h.stream));
      k_build_sell<<<h.sms * 4, 256, 0, h.stream>>>(M.n, nsl * 32, M.rowptr, M.col, M.v32, M.sptr,
                                                     M.scol, M.sval);
      CK(cudaGetLastError());
    }
  }
  CK(cudaStreamSynchronize(h.stream));
}

// Arnoldi from r0 (device, copied into W.b) for k steps; returns steps taken.
template <typename E>
int run_arnoldi(gmres_ctx& h, Workspace& W, const double* r0, int k, bool fp64, bool poly) {
  if (h.params.orth == 1 && is_half_v<typename E::TVt>) throw CudaFail{GMRES_ERR_UNSUPPORTED};
  const size_t n = (size_t)h.A.n;
  CK(cudaMemcpyAsync(W.b, r0, n * 8, cudaMemcpyDefault, h.stream));
  CK(cudaMemsetAsync(W.x, 0, n * 8, h.stream));
  CycleState init{};
  init.jmax = k;
  init.implicit_fp64 = 1;
  init.tol = 0.0;
  init.uround = fp64 ? std::ldexp(1.0, -53) : std::ldexp(1.0, -24);
  CK(cudaMemcpyAsync(W.st, &init, sizeof(CycleState), cudaMemcpyHostToDevice, h.stream));
  E eng{h, W};
  eng.bnorm();
  eng.residual(1);
  for (int j = 0; j < k; ++j) eng.step(j, poly);
  if (eng.dc) eng.dc_finish(k);
  read_state(h, W);
  if (W.st_host->err) throw CudaFail{GMRES_TIMEOUT};
  return W.st_host->k;
}

void build_poly(gmres_ctx& h, int d, const double* start) {
  const int k = d + 1;
  Workspace& W = get_ws(h, KIND_F64, std::max(h.m, k));
  const size_t n = (size_t)h.A.n;
  std::vector<double> ones;
  const double* src = start;
  if (!src) {
    ones.assign(n, 1.0);
    src = ones.data();
  }
  const int steps = run_arnoldi<Eng64>(h, W, src, k, true, false);
  if (steps < 2) return;   // degree 0: no preconditioner
  const int m1 = W.m + 1;
  std::vector<double> H((size_t)m1 * W.m);
  CK(cudaMemcpyAsync(H.data(), W.K.H, H.size() * 8, cudaMemcpyDeviceToHost, h.stream));
  CK(cudaStreamSynchronize(h.stream));
  std::vector<std::complex<double>> theta;
  if (!harmonic_ritz(steps, H.data(), m1, theta)) throw CudaFail{GMRES_ERR_INVALID_ARG};
  h.roots = leja_order(theta);
  h.sched = poly_schedule(h.roots);
}

}  // namespace

namespace {
int run_guarded(const std::function<void()>& fn) {
  try {
    fn();
    return GMRES_OK;
  } catch (const CudaFail& f) {
    cudaGetLastError();
    return f.code;
  } catch (const std::bad_alloc&) {
    return GMRES_ERR_OOM;
  } catch (...) {
    return GMRES_ERR_CUDA;
  }
}

bool prec_ok(const gmres_precisions_t& p) {
  if (p.matrix != GMRES_F32 || p.inner != GMRES_F32) return false;
  if (p.basis != GMRES_F32 && p.basis != GMRES_BF16 && p.basis != GMRES_F16) return false;
  if (p.precond != GMRES_F32 && p.precond != GMRES_F64) return false;
  return true;
}
}  // namespace

// ------------------------------------------------------------------------------------------------
// C ABI
// ------------------------------------------------------------------------------------------------
extern "C" {

void gmres_default_params(gmres_params_t* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->m = 0;
  p->maxiter = 200000;
  p->time_limit_s = 0.0;
  p->inner_tol = 0.0;
  p->use_graphs = 1;
  p->profiling = 0;
  p->stagnation_cycles = 0;
  p->max_loss_of_accuracy = 20;
  p->orth = 0;
}

const char* gmres_status_string(int s) {
  switch (s) {
    case GMRES_OK: return "converged";
    case GMRES_ERR_INVALID_ARG: return "invalid argument";
    case GMRES_ERR_OOM: return "out of device memory";
    case GMRES_ERR_CUDA: return "CUDA error";
    case GMRES_ERR_UNSUPPORTED: return "unsupported configuration";
    case GMRES_NOT_CONVERGED: return "not converged";
    case GMRES_NAN: return "NaN or Inf encountered";
    case GMRES_LOSS_OF_ACCURACY: return "loss of accuracy (implicit and explicit residuals differ)";
    case GMRES_STAGNATION: return "stagnation";
    case GMRES_TIMEOUT: return "timeout";
    default: return "unknown status";
  }
}

int gmres_create(const gmres_csr_t* A, int m, int poly_degree, gmres_precisions_t prec,
                 const double* poly_start, gmres_handle_t* out) {
  if (!out) return GMRES_ERR_INVALID_ARG;
  *out = nullptr;
  if (!A || !A->rowptr || A->n < 1 || A->nnz < 0 || A->n >= (1ll << 31) - 4096 ||
      A->nnz >= (1ll << 31) - 64 || (A->nnz > 0 && (!A->colidx || !A->val)))
    return GMRES_ERR_INVALID_ARG;
  if (m < 1 || m > kMaxCols - 1) return GMRES_ERR_INVALID_ARG;
  if (poly_degree < 0 || poly_degree > kMaxCols - 2) return GMRES_ERR_INVALID_ARG;
  if (!prec_ok(prec)) return GMRES_ERR_UNSUPPORTED;
  gmres_ctx* h = new (std::nothrow) gmres_ctx();
  if (!h) return GMRES_ERR_OOM;
  const int rc = run_guarded([&] {
    CK(cudaGetDevice(&h->dev));
    h->sms = g_num_sms(h->dev);
    CK(cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking));
    CK(cudaEventCreateWithFlags(&h->ev_in, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&h->ev_out, cudaEventDisableTiming));
    h->m = m;
    h->prec = prec;
    gmres_default_params(&h->params);
    upload_matrix(*h, A);
    if (poly_degree > 0) build_poly(*h, poly_degree, poly_start);
    CK(cudaStreamSynchronize(h->stream));
  });
  if (rc != GMRES_OK) {
    delete h;
    return rc;
  }
  *out = h;
  return GMRES_OK;
}

int gmres_destroy(gmres_handle_t h) {
  if (!h) return GMRES_OK;
  cudaStreamSynchronize(h->stream);
  delete h;
  return GMRES_OK;
}

int gmres_set_stream(gmres_handle_t h, void* s) {
  if (!h) return GMRES_ERR_INVALID_ARG;
  h->user_stream = (cudaStream_t)s;
  return GMRES_OK;
}

int gmres_set_tuning(gmres_handle_t h, const gmres_tuning_t* t) {
  if (!h || !t) return GMRES_ERR_INVALID_ARG;
  const int L = t->spmv_lanes_per_row;
  if (t->sweep_stage_kb < 0 || t->sweep_stage_kb > 128 || t->sweep_ctas_per_sm < 0 ||
      t->sweep_ctas_per_sm > 4 || t->spmv_ctas_per_sm < 0 || t->spmv_ctas_per_sm > 8 || L < 0 ||
      L > 32 || (L & (L - 1)) != 0 || (t->cluster_cycle != 0 && t->cluster_cycle != -1))
    return GMRES_ERR_INVALID_ARG;
  h->tuning = *t;
  h->A.lanes = L > 0 ? L : auto_lanes(h->A.n, h->A.nnz);
  h->tuning_gen += 1;
  return GMRES_OK;
}

int gmres_get_tuning(gmres_handle_t h, gmres_tuning_t* t) {
  if (!h || !t) return GMRES_ERR_INVALID_ARG;
  *t = h->tuning;
  return GMRES_OK;
}

int gmres_set_params(gmres_handle_t h, const gmres_params_t* p) {
  if (!h || !p) return GMRES_ERR_INVALID_ARG;
  if (p->m < 0 || p->m > h->m || p->maxiter < 0 || p->time_limit_s < 0 || p->inner_tol < 0 ||
      p->inner_tol >= 1.0 || p->stagnation_cycles < 0 || p->max_loss_of_accuracy < 0 ||
      (p->orth != 0 && p->orth != 1))
    return GMRES_ERR_INVALID_ARG;
  h->params = *p;
  return GMRES_OK;
}

static int solve_common(gmres_handle_t h, const double* b, double* x, double tol,
                        gmres_stats_t* stats, bool fp64) {
  if (!h || !b || !x || !(tol >= 0.0)) return GMRES_ERR_INVALID_ARG;
  int status = GMRES_OK;
  const int rc = run_guarded([&] {
    if (fp64) {
      Workspace& W = get_ws(*h, KIND_F64, h->m);
      if (h->prec.precond == GMRES_F32 && (!h->sched.empty() || h->bj.k > 0))
        status = run_solve<Eng64P32>(*h, W, b, x, tol, stats, MODE_FP64);
      else
        status = run_solve<Eng64>(*h, W, b, x, tol, stats, MODE_FP64);
    } else if (h->prec.basis == GMRES_BF16) {
      Workspace& W = get_ws(*h, KIND_IR_BF16, h->m);
      status = run_solve<EngIR16>(*h, W, b, x, tol, stats, MODE_IR);
    } else if (h->prec.basis == GMRES_F16) {
      Workspace& W = get_ws(*h, KIND_IR_F16, h->m);
      status = run_solve<EngIRh>(*h, W, b, x, tol, stats, MODE_IR);
    } else {
      Workspace& W = get_ws(*h, KIND_IR_F32, h->m);
      status = run_solve<EngIR32>(*h, W, b, x, tol, stats, MODE_IR);
    }
  });
  if (rc != GMRES_OK) {
    if (stats) stats->status = rc;
    return rc;
  }
  return status;
}

int gmres_ir_solve(gmres_handle_t h, const double* b, double* x, double tol, gmres_stats_t* stats) {
  return solve_common(h, b, x, tol, stats, false);
}

int gmres_solve_fp64(gmres_handle_t h, const double* b, double* x, double tol,
                     gmres_stats_t* stats) {
  return solve_common(h, b, x, tol, stats, true);
}

int gmres_solve_fp32(gmres_handle_t h, const double* b, double* x, double tol,
                     gmres_stats_t* stats) {
  if (!h || !b || !x || !(tol >= 0.0)) return GMRES_ERR_INVALID_ARG;
  if (h->prec.basis != GMRES_F32) return GMRES_ERR_UNSUPPORTED;
  int status = GMRES_OK;
  const int rc = run_guarded([&] {
    Workspace& W = get_ws(*h, KIND_IR_F32, h->m);
    status = run_solve<EngIR32>(*h, W, b, x, tol, stats, MODE_FP32);
  });
  if (rc != GMRES_OK) {
    if (stats) stats->status = rc;
    return rc;
  }
  return status;
}

int gmres_fd_solve(gmres_handle_t h, const double* b, double* x, double tol, int64_t switch_iters,
                   gmres_stats_t* stats, int64_t* fp32_iters) {
  if (!h || !b || !x || !(tol >= 0.0) || switch_iters < 0) return GMRES_ERR_INVALID_ARG;
  if (h->prec.basis != GMRES_F32) return GMRES_ERR_UNSUPPORTED;
  const gmres_params_t saved = h->params;
  gmres_stats_t s1{}, s2{};
  if (stats) {
    s1.res_history = stats->res_history;
    s1.res_history_cap = stats->res_history_cap;
  }
  int status = GMRES_OK;
  const auto t0 = std::chrono::steady_clock::now();
  const int rc = run_guarded([&] {
    int64_t done = 0;
    if (switch_iters > 0) {
      // the FP32 phase runs to the switch point: its loss-of-accuracy events (FP32 implicit
      // residuals below tol) only restart it
      h->params.maxiter = std::min<int64_t>(switch_iters, saved.maxiter);
      h->params.max_loss_of_accuracy = 1 << 30;
      Workspace& W = get_ws(*h, KIND_IR_F32, h->m);
      status = run_solve<EngIR32>(*h, W, b, x, tol, &s1, MODE_FP32);
      done = s1.iters;
    }
    {  // FP64 GMRES from the FP32 iterate (it stops at once if that already meets tol in FP64)
      h->params.maxiter = std::max<int64_t>(0, saved.maxiter - done);
      h->params.max_loss_of_accuracy = saved.max_loss_of_accuracy;
      if (stats && s1.res_history) {   // the FP64 phase appends to the same history
        const int64_t used = std::min(s1.res_history_len, s1.res_history_cap);
        s2.res_history = s1.res_history + used;
        s2.res_history_cap = s1.res_history_cap - used;
      }
      Workspace& W = get_ws(*h, KIND_F64, h->m);
      status = run_solve<Eng64>(*h, W, b, x, tol, &s2, MODE_FP64);
    }
  });
  h->params = saved;
  if (fp32_iters) *fp32_iters = s1.iters;
  if (stats) {
    gmres_stats_t S = s2;
    S.iters = s1.iters + s2.iters;
    S.cycles = s1.cycles + s2.cycles;
    S.breakdowns = s1.breakdowns + s2.breakdowns;
    S.loss_of_accuracy = s1.loss_of_accuracy + s2.loss_of_accuracy;
    S.kernel_launches = s1.kernel_launches + s2.kernel_launches;
    S.res_history = stats->res_history;
    S.res_history_cap = stats->res_history_cap;
    S.res_history_len = s1.res_history_len + s2.res_history_len;
    for (int i = 0; i < 8; ++i) S.t_kernel[i] = s1.t_kernel[i] + s2.t_kernel[i];
    S.solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    S.status = rc != GMRES_OK ? rc : status;
    *stats = S;
  }
  return rc != GMRES_OK ? rc : status;
}

int gmres_autotune(gmres_handle_t h, const double* b, int cycles, gmres_tuning_t* best,
                   double* best_s_per_iter, double* default_s_per_iter) {
  if (!h || !b || cycles < 1 || cycles > 100) return GMRES_ERR_INVALID_ARG;
  const gmres_params_t saved_params = h->params;
  const gmres_tuning_t saved_tuning = h->tuning;
  double t_best = 0.0, t_default = 0.0;
  gmres_tuning_t chosen{};
  const int rc = run_guarded([&] {
    const bool bf16 = h->prec.basis == GMRES_BF16, f16 = h->prec.basis == GMRES_F16;
    Workspace& W = get_ws(*h, bf16 ? KIND_IR_BF16 : (f16 ? KIND_IR_F16 : KIND_IR_F32), h->m);
    const int m = h->params.m > 0 ? h->params.m : h->m;
    std::vector<double> x((size_t)h->A.n);
    auto run = [&](int64_t iters) {
      std::fill(x.begin(), x.end(), 0.0);
      h->params.maxiter = iters;
      gmres_stats_t st{};
      if (bf16) run_solve<EngIR16>(*h, W, b, x.data(), 0.0, &st, MODE_IR);
      else if (f16) run_solve<EngIRh>(*h, W, b, x.data(), 0.0, &st, MODE_IR);
      else run_solve<EngIR32>(*h, W, b, x.data(), 0.0, &st, MODE_IR);
      return st;
    };
    h->params.time_limit_s = 0.0;
    h->params.inner_tol = 0.0;
    h->params.use_graphs = 1;
    h->params.profiling = 0;
    h->params.stagnation_cycles = 0;
    static const int stage_kb[] = {0, 16, 32};
    static const int sweep_ctas[] = {0, 1, 2, 3};
    static const int spmv_ctas[] = {0, 4};
    bool have = false;
    auto try_shape = [&](const gmres_tuning_t& cand) {
      h->tuning = cand;
      h->tuning.cluster_cycle = -1;                          // the shapes are the step kernels'
      h->A.lanes = cand.spmv_lanes_per_row > 0 ? cand.spmv_lanes_per_row
                                               : auto_lanes(h->A.n, h->A.nnz);
      h->tuning_gen += 1;                                    // a fresh graph per candidate
      run(m);                                                // capture + warm-up
      const auto t0 = std::chrono::steady_clock::now();
      const gmres_stats_t st = run((int64_t)m * cycles);
      const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      const double cost = el / (double)std::max<int64_t>(1, st.iters);
      if (!have || cost < t_best) {
        have = true;
        t_best = cost;
        chosen = cand;
      }
      return cost;
    };
    for (int a : stage_kb)
      for (int c : sweep_ctas)
        for (int s : spmv_ctas) {
          const double cost = try_shape(gmres_tuning_t{a, c, s, 0});
          if (a == 0 && c == 0 && s == 0) t_default = cost;
        }
    // then the SpMV lanes per row around the automatic choice, with the best shapes so far
    const int La = auto_lanes(h->A.n, h->A.nnz);
    const gmres_tuning_t base = chosen;
    for (int L = std::max(1, La / 4); L <= std::min(32, La * 4); L *= 2) {
      if (L == La) continue;
      gmres_tuning_t cand = base;
      cand.spmv_lanes_per_row = L;
      try_shape(cand);
    }
  });
  h->params = saved_params;
  h->tuning_gen += 1;   // a fresh graph for the shapes kept
  if (rc != GMRES_OK) {
    h->tuning = saved_tuning;
    h->A.lanes = saved_tuning.spmv_lanes_per_row > 0 ? saved_tuning.spmv_lanes_per_row
                                                     : auto_lanes(h->A.n, h->A.nnz);
    return rc;
  }
  chosen.cluster_cycle = saved_tuning.cluster_cycle;
  h->tuning = chosen;
  h->A.lanes = chosen.spmv_lanes_per_row > 0 ? chosen.spmv_lanes_per_row
                                             : auto_lanes(h->A.n, h->A.nnz);
  if (best) *best = chosen;
  if (best_s_per_iter) *best_s_per_iter = t_best;
  if (default_s_per_iter) *default_s_per_iter = t_default;
  return GMRES_OK;
}

int gmres_spmv(gmres_handle_t h, gmres_prec_t prec, const void* x, void* y) {
  if (!h || !x || !y || (prec != GMRES_F64 && prec != GMRES_F32)) return GMRES_ERR_INVALID_ARG;
  return run_guarded([&] {
    order_after_caller(*h);
    if (prec == GMRES_F64) {
      auto kern = k_spmv<double, double, double>;
      kern<<<plan_rows(kern, h->A.n, h->A.lanes, h->sms), kThreads, 0, h->stream>>>(
          h->A.csr64(), VRef<double>{(const double*)x, kTile}, (double*)y);
    } else {
      auto kern = k_spmv<float, float, float>;
      kern<<<plan_rows(kern, h->A.n, h->A.lanes, h->sms), kThreads, 0, h->stream>>>(
          h->A.csr32(), VRef<float>{(const float*)x, kTile}, (float*)y);
    }
    CK(cudaGetLastError());
    CK(cudaStreamSynchronize(h->stream));
  });
}

int gmres_precond_apply(gmres_handle_t h, gmres_prec_t prec, const void* v, void* z) {
  if (!h || !v || !z || (prec != GMRES_F64 && prec != GMRES_F32)) return GMRES_ERR_INVALID_ARG;
  return run_guarded([&] {
    const size_t n = (size_t)h->A.n;
    const size_t es = prec == GMRES_F64 ? 8 : 4;
    order_after_caller(*h);
    if (h->sched.empty() && h->bj.k == 0) {
      CK(cudaMemcpyAsync(z, v, n * es, cudaMemcpyDefault, h->stream));
      CK(cudaStreamSynchronize(h->stream));
      return;
    }
    if (prec == GMRES_F64) {
      Workspace& W = get_ws(*h, KIND_F64, h->m);
      Eng64 e{*h, W};
      e.precond_apply<double>(VRef<double>{(const double*)v, kTile}, 0);
      CK(cudaMemcpyAsync(z, W.B[3], n * es, cudaMemcpyDeviceToDevice, h->stream));
    } else {
      Workspace& W = get_ws(*h, KIND_IR_F32, h->m);
      EngIR32 e{*h, W};
      e.precond_apply<float>(VRef<float>{(const float*)v, kTile}, 0);
      CK(cudaMemcpyAsync(z, W.B[3], n * es, cudaMemcpyDeviceToDevice, h->stream));
    }
    CK(cudaStreamSynchronize(h->stream));
  });
}

int gmres_set_block_jacobi(gmres_handle_t h, int block_size, int reorder) {
  if (!h || block_size < 0 || block_size > 64) return GMRES_ERR_INVALID_ARG;
  if (!h->sched.empty()) return GMRES_ERR_INVALID_ARG;   // one preconditioner per handle
  return run_guarded([&] {
    h->bj.release();
    h->tuning_gen += 1;   // the cycle graphs are rebuilt with (or without) the preconditioner
    if (block_size == 0) return;
    const int n = h->A.n;
    const size_t nnz = (size_t)h->A.nnz;
    std::vector<int32_t> rp((size_t)n + 1), ci(nnz);
    std::vector<double> va(nnz);
    CK(cudaMemcpyAsync(rp.data(), h->A.rowptr, rp.size() * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(ci.data(), h->A.col, nnz * 4, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaMemcpyAsync(va.data(), h->A.v64, nnz * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    std::vector<int32_t> perm;
    if (reorder) {
      perm = rcm_order(n, rp.data(), ci.data());
    } else {
      perm.resize(n);
      for (int i = 0; i < n; ++i) perm[i] = i;
    }
    std::vector<double> inv;
    if (block_size == 1) {   // diagonal scaling, natural order
      inv.assign(n, 0.0);
      for (int i = 0; i < n; ++i) {
        double d = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; ++p)
          if (ci[p] == i) d += va[p];
        if (d == 0.0 || !std::isfinite(d)) throw CudaFail{GMRES_ERR_INVALID_ARG};
        inv[i] = 1.0 / d;
      }
    } else {
      const int threads = (int)std::max(1u, std::thread::hardware_concurrency());
      if (!block_inverses(n, rp.data(), ci.data(), va.data(), perm, block_size, inv, threads))
        throw CudaFail{GMRES_ERR_INVALID_ARG};   // a singular diagonal block
    }
    std::vector<float> inv32(inv.size());
    for (size_t i = 0; i < inv.size(); ++i) inv32[i] = (float)inv[i];
    auto& B = h->bj;
    B.idx = dalloc<int>(n);
    B.inv64 = dalloc<double>(inv.size());
    B.inv32 = dalloc<float>(inv.size());
    CK(cudaMemcpyAsync(B.idx, perm.data(), (size_t)n * 4, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(B.inv64, inv.data(), inv.size() * 8, cudaMemcpyHostToDevice, h->stream));
    CK(cudaMemcpyAsync(B.inv32, inv32.data(), inv32.size() * 4, cudaMemcpyHostToDevice, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    B.k = block_size;
    B.nblocks = (n + block_size - 1) / block_size;
    B.perm = std::move(perm);
  });
}

int gmres_block_jacobi_perm(gmres_handle_t h, int32_t* perm, int64_t cap) {
  if (!h || !perm) return GMRES_ERR_INVALID_ARG;
  if (h->bj.k == 0 || cap < (int64_t)h->bj.perm.size()) return GMRES_ERR_INVALID_ARG;
  std::copy(h->bj.perm.begin(), h->bj.perm.end(), perm);
  return GMRES_OK;
}

int gmres_poly_roots(gmres_handle_t h, double* re, double* im, int cap, int* count) {
  if (!h || !count) return GMRES_ERR_INVALID_ARG;
  *count = (int)h->roots.size();
  if ((int)h->roots.size() > cap || (!h->roots.empty() && (!re || !im)))
    return h->roots.empty() ? GMRES_OK : GMRES_ERR_INVALID_ARG;
  for (size_t i = 0; i < h->roots.size(); ++i) {
    re[i] = h->roots[i].real();
    im[i] = h->roots[i].imag();
  }
  return GMRES_OK;
}

int gmres_arnoldi(gmres_handle_t h, gmres_prec_t inner, int k, const double* r0, double* H,
                  double* V, int* steps) {
  if (!h || !r0 || !H || !steps || k < 1 || k > h->m ||
      (inner != GMRES_F64 && inner != GMRES_F32))
    return GMRES_ERR_INVALID_ARG;
  return run_guarded([&] {
    const bool poly = !h->sched.empty() || h->bj.k > 0;
    Workspace* Wp;
    int st;
    order_after_caller(*h);
    if (inner == GMRES_F64) {
      Wp = &get_ws(*h, KIND_F64, h->m);
      if (poly && h->prec.precond == GMRES_F32)
        st = run_arnoldi<Eng64P32>(*h, *Wp, r0, k, true, poly);
      else
        st = run_arnoldi<Eng64>(*h, *Wp, r0, k, true, poly);
    } else if (h->prec.basis == GMRES_BF16) {
      Wp = &get_ws(*h, KIND_IR_BF16, h->m);
      st = run_arnoldi<EngIR16>(*h, *Wp, r0, k, false, poly);
    } else if (h->prec.basis == GMRES_F16) {
      Wp = &get_ws(*h, KIND_IR_F16, h->m);
      st = run_arnoldi<EngIRh>(*h, *Wp, r0, k, false, poly);
    } else {
      Wp = &get_ws(*h, KIND_IR_F32, h->m);
      st = run_arnoldi<EngIR32>(*h, *Wp, r0, k, false, poly);
    }
    Workspace& W = *Wp;
    *steps = st;
    const int m1 = W.m + 1;
    std::vector<double> Hf((size_t)m1 * W.m);
    CK(cudaMemcpyAsync(Hf.data(), W.K.H, Hf.size() * 8, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    for (int j = 0; j < k; ++j)
      for (int i = 0; i <= k; ++i) H[(size_t)j * (k + 1) + i] = (j < st) ? Hf[(size_t)j * m1 + i] : 0.0;
    if (V) {
      const int ncols = std::min(st + 1, k + 1);
      dim3 grid(std::max(1, std::min(h->sms * 2, (h->A.n + 255) / 256)), ncols);
      if (W.kind == KIND_F64)
        k_basis_export<double><<<grid, 256, 0, h->stream>>>((const double*)W.V, W.vts, W.K.s, ncols,
                                                            h->A.n, V);
      else if (W.kind == KIND_IR_F16)
        k_basis_export<__half><<<grid, 256, 0, h->stream>>>((const __half*)W.V, W.vts, W.K.s,
                                                            ncols, h->A.n, V);
      else if (W.kind == KIND_IR_BF16)
        k_basis_export<bf16><<<grid, 256, 0, h->stream>>>((const bf16*)W.V, W.vts, W.K.s, ncols,
                                                          h->A.n, V);
      else
        k_basis_export<float><<<grid, 256, 0, h->stream>>>((const float*)W.V, W.vts, W.K.s, ncols,
                                                           h->A.n, V);
      CK(cudaGetLastError());
      CK(cudaStreamSynchronize(h->stream));
    }
  });
}

int gmres_test_expire_wait(gmres_handle_t h, int armed) {
  if (!h || (armed != 0 && armed != 1)) return GMRES_ERR_INVALID_ARG;
  h->expire_wait = armed;
  return GMRES_OK;
}

int gmres_hessenberg_eigvals(int k, const double* H, double* re, double* im) {
  if (k < 1 || !H || !re || !im) return GMRES_ERR_INVALID_ARG;
  std::vector<std::complex<double>> ev;
  if (!hessenberg_eigvals(k, H, k, ev)) return GMRES_ERR_INVALID_ARG;
  for (int i = 0; i < k; ++i) {
    re[i] = ev[i].real();
    im[i] = ev[i].imag();
  }
  return GMRES_OK;
}

}  // extern "C"

gmresb3::HandleView gmresb3::handle_view(gmres_handle_t h) {
  return HandleView{h->A.n, h->A.nnz, h->A.rowptr, h->A.col, h->A.v64, h->dev, h->sms,
                    (void*)h->user_stream};
}

// ------------------------------------------------------------------------------------------------
// Polynomial application without device allocation (gmres_precond_apply_noalloc)
//
// Some callers must not allocate device memory while they run: code inside a memory-pool or
// arena that owns every byte of the GPU, real-time loops where cudaMalloc's implicit
// synchronisation is not allowed, or plugins whose host forbids allocation after start-up.  For
// them this entry point applies p(A) with its work vectors in a fixed array that is part of the
// library's device image.  That array exists on every GPU that loads the library, until the
// process exits.
// ------------------------------------------------------------------------------------------------
namespace {

constexpr int64_t kNoAllocMaxN = int64_t(1) << 19;            // largest n accepted
constexpr size_t kNoAllocHeader = 256;                        // unused, keeps the layout
constexpr size_t kNoAllocBytes = kNoAllocHeader + 3 * (size_t)kNoAllocMaxN * sizeof(double);

// 256 unused bytes | work vector B0 | B1 | B2  (12 MiB + 256 bytes)
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_noalloc_mu;
void* g_noalloc_addr[256] = {};

// Device address of the scratch array on the current device.  Host code only holds a stand-in
// for the symbol, so the address is looked up once per device with cudaGetSymbolAddress.
int noalloc_scratch_address(void** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return GMRES_ERR_CUDA;
  }
  if (dev < 0 || dev >= 256) return GMRES_ERR_UNSUPPORTED;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return GMRES_ERR_CUDA;
    }
    g_noalloc_addr[dev] = p;
  }
  *out = g_noalloc_addr[dev];
  return GMRES_OK;
}

template <typename TA, typename ACC>
void noalloc_poly_apply(gmres_ctx& h, const Csr<TA>& A, const ACC* v, ACC* z, unsigned char* base) {
  const size_t vec_bytes = ((size_t)h.A.n * sizeof(ACC) + 255) & ~size_t(255);
  ACC* buf[4] = {nullptr, (ACC*)(base + kNoAllocHeader), (ACC*)(base + kNoAllocHeader + vec_bytes),
                 (ACC*)(base + kNoAllocHeader + 2 * vec_bytes)};
  auto kern = k_poly_step<TA, ACC, ACC, ACC>;
  const int grid = plan_rows(kern, h.A.n, h.A.lanes, h.sms, h.tuning.spmv_ctas_per_sm);
  int rev = 0;   // consecutive steps walk the rows in opposite directions (L2 reuse)
  for (const auto& d : h.sched) {
    PolyCoef c;
    c.cp_p = d.cp_p;
    c.cp_x = d.cp_x;
    c.cp_t = d.cp_t;
    c.cy_y = d.cy_y;
    c.cy_p = d.cy_p;
    c.cy_x = d.cy_x;
    c.cy_t = d.cy_t;
    c.cy_n = d.cy_n;
    c.write_p = d.pn != PB_NONE;
    c.write_y = d.write_y;
    c.read_y = d.read_y;
    const ACC* x = d.x == PB_IN ? v : buf[d.x];
    const ACC* P = d.p == PB_IN ? v : buf[d.p];
    ACC* Pn = d.pn == PB_NONE ? nullptr : buf[d.pn];
    kern<<<grid, kThreads, 0, h.stream>>>(A, VRef<ACC>{x, kTile}, VRef<ACC>{P, kTile}, Pn, z,
                                           PolyCoefT<ACC>::of(c), nullptr, 0, rev ^= 1);
    CK(cudaGetLastError());
  }
}

}  // namespace

extern "C" int gmres_precond_apply_noalloc(gmres_handle_t h, gmres_prec_t prec, const void* v,
                                           void* z) {
  if (!h || !v || !z || (prec != GMRES_F64 && prec != GMRES_F32)) return GMRES_ERR_INVALID_ARG;
  if ((int64_t)h->A.n > kNoAllocMaxN) return GMRES_ERR_INVALID_ARG;   // beyond the fixed scratch
  {  // z is written while later rows of v are still read: the two must not overlap
    const uintptr_t bytes = (uintptr_t)h->A.n * (prec == GMRES_F64 ? 8 : 4);
    const uintptr_t a = (uintptr_t)v, c = (uintptr_t)z;
    if (a < c + bytes && c < a + bytes) return GMRES_ERR_INVALID_ARG;
  }
  if (h->bj.k > 0) return GMRES_ERR_UNSUPPORTED;   // the polynomial only
  int prev = -1;
  if (cudaGetDevice(&prev) != cudaSuccess) {
    cudaGetLastError();
    return GMRES_ERR_CUDA;
  }
  if (prev != h->dev && cudaSetDevice(h->dev) != cudaSuccess) {
    cudaGetLastError();
    return GMRES_ERR_CUDA;
  }
  unsigned char* base = nullptr;
  int rc = noalloc_scratch_address((void**)&base);
  if (rc == GMRES_OK) {
    rc = run_guarded([&] {
      const size_t n = (size_t)h->A.n;
      const size_t es = prec == GMRES_F64 ? 8 : 4;
      order_after_caller(*h);
      if (h->sched.empty()) {
        CK(cudaMemcpyAsync(z, v, n * es, cudaMemcpyDeviceToDevice, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        return;
      }
      if (prec == GMRES_F64)
        noalloc_poly_apply<double, double>(*h, h->A.csr64(), (const double*)v, (double*)z, base);
      else
        noalloc_poly_apply<float, float>(*h, h->A.csr32(), (const float*)v, (float*)z, base);
      CK(cudaStreamSynchronize(h->stream));
    });
  }
  if (prev != h->dev) cudaSetDevice(prev);
  return rc;
}
