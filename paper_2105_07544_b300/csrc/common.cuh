// Shared device helpers of the gmresb3 kernels: element types, reductions and the bulk-copy
// (TMA engine) / mbarrier primitives in inline PTX for sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gmresb3 {

// Rows per tile of every streaming kernel and threads per CTA.  Vectors and basis columns are
// padded to a multiple of kTile rows.
constexpr int kTile = 128;
constexpr int kTileShift = 7;
static_assert((1 << kTileShift) == kTile, "kTile must be 2^kTileShift");
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
// Basis columns a sweep can hold (restart length m <= 127).  Column i belongs to warp
// i % kWarps; lane l of every warp owns the tile rows 4l..4l+3.
constexpr int kMaxCols = 128;
// Slots per CTA in the partial-sum array: kMaxCols column sums, four norms, then a second block
// of kMaxCols column sums starting at kSlotB (the two-vector projection of the DCGS2 variant).
constexpr int kSlotB = kMaxCols + 4;
constexpr int kPartLd = kSlotB + kMaxCols;
// Bulk-copy waits give up after this many nanoseconds of %globaltimer (error flag, no hang).
constexpr unsigned long long kWaitLimitNs = 200000000ull;

// ---- element conversions ---------------------------------------------------------------------
__device__ __forceinline__ float cvt_f32(float v) { return v; }
__device__ __forceinline__ float cvt_f32(double v) { return (float)v; }
__device__ __forceinline__ float cvt_f32(__nv_bfloat16 v) { return __bfloat162float(v); }
__device__ __forceinline__ float cvt_f32(__half v) { return __half2float(v); }

template <typename A> struct Conv;
template <> struct Conv<float> {
  __device__ __forceinline__ static float from(float v) { return v; }
  __device__ __forceinline__ static float from(double v) { return (float)v; }
  __device__ __forceinline__ static float from(__nv_bfloat16 v) { return __bfloat162float(v); }
  __device__ __forceinline__ static float from(__half v) { return __half2float(v); }
};
template <> struct Conv<double> {
  __device__ __forceinline__ static double from(float v) { return (double)v; }
  __device__ __forceinline__ static double from(double v) { return v; }
  __device__ __forceinline__ static double from(__nv_bfloat16 v) {
    return (double)__bfloat162float(v);
  }
  __device__ __forceinline__ static double from(__half v) { return (double)__half2float(v); }
};
template <> struct Conv<__nv_bfloat16> {
  __device__ __forceinline__ static __nv_bfloat16 from(float v) { return __float2bfloat16_rn(v); }
  __device__ __forceinline__ static __nv_bfloat16 from(double v) {
    return __float2bfloat16_rn((float)v);
  }
};
// FP16 (round to nearest even): the basis is stored scaled into FP16's range (see k_sweep UPDATE
// and k_v0_half), never raw.
template <> struct Conv<__half> {
  __device__ __forceinline__ static __half from(float v) { return __float2half_rn(v); }
  __device__ __forceinline__ static __half from(double v) { return __float2half_rn((float)v); }
};

template <typename A, typename T> __device__ __forceinline__ A cv(T v) { return Conv<A>::from(v); }

// ---- warp / block reductions (fixed order: results do not depend on timing) ------------------
template <typename T> __device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T> __device__ __forceinline__ T block_sum(T v, T* red /* kWarps */) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  T s = 0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) s += red[i];
  return s;
}

// ---- mbarrier + bulk async copy (cp.async.bulk, executed by the TMA unit) --------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

// Copy `bytes` (a multiple of 16) from global `src` (16-byte aligned) to shared `dst` (16-byte
// aligned); completion is counted on `bar` as transaction bytes.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// The same copy with an L2 eviction-priority policy (from createpolicy) for the source lines.
__device__ __forceinline__ void bulk_g2s_hint(void* dst, const void* src, uint32_t bytes,
                                              uint64_t* bar, uint64_t policy) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
      " [%0], [%1], %2, [%3], %4;" ::"r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(policy)
      : "memory");
}

// L2 eviction priorities.  A kernel that streams more than the L2 holds loads what it reads once
// and what the next kernel will not start on as evict-first, so that those lines are replaced
// before the ones the next kernel reads first (the basis tiles at the end of its traversal).
__device__ __forceinline__ uint64_t l2_evict_first_policy() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Read-only load with an L2 policy, issued only if `pred` (else `dflt`), for the matrix arrays
// (padded, but the predicate keeps a load off an entry the row does not own).
__device__ __forceinline__ int ld_hint_if(bool pred, const int* a, int dflt, uint64_t policy) {
  int v = dflt;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
      "@q ld.global.nc.L2::cache_hint.b32 %0, [%1], %3;\n\t}"
      : "+r"(v) : "l"(a), "r"((unsigned)pred), "l"(policy));
  return v;
}
__device__ __forceinline__ float ld_hint_if(bool pred, const float* a, float dflt,
                                            uint64_t policy) {
  float v = dflt;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
      "@q ld.global.nc.L2::cache_hint.f32 %0, [%1], %3;\n\t}"
      : "+f"(v) : "l"(a), "r"((unsigned)pred), "l"(policy));
  return v;
}
__device__ __forceinline__ double ld_hint_if(bool pred, const double* a, double dflt,
                                             uint64_t policy) {
  double v = dflt;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\t"
      "@q ld.global.nc.L2::cache_hint.f64 %0, [%1], %3;\n\t}"
      : "+d"(v) : "l"(a), "r"((unsigned)pred), "l"(policy));
  return v;
}

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wait for the phase of `bar` with parity `parity`.  Bounded by kWaitLimitNs: returns false if
// the phase did not complete in time (the caller flags an error and skips the tile's work).
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  const uint32_t a = smem_u32(bar);
  unsigned long long t0 = 0;
  for (uint32_t it = 0;; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((it & 255u) == 0u) {
      const unsigned long long t = globaltimer();
      if (it == 0) t0 = t;
      else if (t - t0 > kWaitLimitNs) return false;
    }
  }
}

// After a wait on use `first` of a ring of nstages barriers ran out: wait (bounded) for the uses
// first .. min(first + nstages, total) - 1, whose copies were issued and not yet consumed, so no
// bulk copy is still writing this CTA's shared memory when it exits.  Use u lives on barrier
// u % nstages with phase parity (u / nstages) & 1.  Returns false if one of them did not land.
__device__ __forceinline__ bool drain_stages(uint64_t* bar, int nstages, int first, int total) {
  bool all = true;
  const int hi = min(first + nstages, total);
  for (int u = first; u < hi; ++u) all &= mbar_wait(&bar[u % nstages], (uint32_t)((u / nstages) & 1));
  return all;
}

__device__ __forceinline__ void mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// Last-CTA-done detection: every CTA has written its partials; the CTA that increments the
// counter last returns true and sees all of them.  The counter is reset by that CTA.
__device__ __forceinline__ bool arrive_last(unsigned* counter, int* flag_smem) {
  // The CTA barrier orders every thread's partials before thread 0's gpu-scope fence, which
  // (cumulatively) releases them with the arrival; the other threads do not wait for their own
  // outstanding stores (a basis column, w) here.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    *flag_smem = (prev == gridDim.x - 1) ? 1 : 0;
  }
  __syncthreads();
  const bool last = *flag_smem != 0;
  if (last) __threadfence();
  return last;
}

}  // namespace gmresb3
