// Device kernels of the gmresb3 solver.
//
// One GMRES(m) inner iteration (Algorithm 1 with the two classical Gram-Schmidt passes of
// Section III-A) is one CSR SpMV fused with the first projection and two streaming sweeps over
// the Krylov basis V:
//
//   k_spmv_proj         : w = s_j A z_j (CSR SpMV: two rows per lane, or a lane group per row for
//                         long rows), the first projection h1 = V_j^T w and ||w||
//   k_sweep<PASS2>      : w' = w - V_j (s h1) on the fly and the second projection h2 = V_j^T w'
//   k_sweep<UPDATE>     : w'' = w' - V_j (s h2) with w' recomputed, v_{j+1} = w'' (stored
//                         unscaled), ||w''||, and (last CTA) the Hessenberg column, its Givens
//                         rotation and stop tests
//
// so V_j is streamed three times per iteration, the minimum for CGS2 without changing the
// algorithm.  Basis columns are stored unscaled with a per-column FP64 scale s_i
// (v_i = s_i V[:, i]); the scale is folded into the projection coefficients.
//
// The basis is tile-blocked ([128-row tile][column][row]), so the columns a sweep needs from one
// tile are one contiguous block: each pipeline stage is one cp.async.bulk copy (the TMA engine)
// of up to 64 KB plus the tile of w, completing on a per-stage mbarrier several tiles ahead of
// the compute.  Grids are persistent (a multiple of the SM count); cross-CTA sums are written as
// per-CTA partials and reduced in a fixed order by the last CTA to finish, so every result is
// deterministic.
#pragma once

#include "common.cuh"

namespace gmresb3 {

// ------------------------------------------------------------------------------------------------
// Device state of a restart cycle (one per workspace)
// ------------------------------------------------------------------------------------------------
struct CycleState {
  int stop;           // 1: the cycle has ended; later step kernels return at once
  int reason;         // 1 implicit tolerance met, 2 lucky breakdown, 3 NaN/Inf, 4 step limit
  int k;              // Arnoldi steps completed in the current cycle
  int last_k;         // steps of the cycle that just ended (saved by the residual kernel)
  int last_reason;    // reason of the cycle that just ended
  int converged;      // explicit residual <= tol
  int nan;            // NaN/Inf seen in a norm
  int err;            // a bulk-copy wait timed out
  int jmax;           // steps per cycle (the restart length m of this solve)
  int implicit_fp64;  // 1: implicit stop at tol ||b|| (FP64 GMRES); 0: inner_tol gamma (IR)
  int loa;            // loss-of-accuracy events (implicit met tol, explicit did not)
  int breakdowns;     // lucky breakdowns
  int fp32_outer;     // 1: single-precision GMRES (FP32 residual and update; GMRES-FD phase 1)
  unsigned cnt[8];    // last-CTA counters, one per kernel kind
  double bnorm, tol, inner_tol, uround;
  double gamma;       // norm of the stored first basis vector of this cycle
  double rel_res;     // explicit ||b - A x|| / ||b||
  double implicit;    // |g_{k+1}| after the latest step
  double last_implicit;
  double az2;         // ||A z_j||^2 of the current step
  int expire_wait;    // test hook: 1 = CTA 0 of step 0's PASS2 sweep leaves its first pipeline
                      // stage unfilled, so that bounded wait runs out (err = 1)
  double hp2;         // DCGS2: squared norm of the provisional Hessenberg column of the last step
};

enum { CNT_A = 0, CNT_B = 1, CNT_C = 2, CNT_R = 3, CNT_U = 4, CNT_MISC = 5 };

// Small dense state of one cycle (FP64, device).  H and R are (m+1) x m column-major.
struct Krylov {
  double* H;     // raw Hessenberg H-bar
  double* R;     // Givens-rotated copy (upper triangular part used by the solve)
  double* cs;    // rotations
  double* sn;
  double* g;     // rotated right-hand side gamma e1
  double* h1;    // first-pass projection coefficients (scaled: true v_i^T w)
  double* h2;    // second-pass coefficients
  double* s;     // column scales: v_i = s_i V[:, i]
  double* c;     // solution coefficients s_i y_i
  double* ca;    // DCGS2 update: coefficients of the delayed second pass of column j
  double* cb;    // DCGS2 update: coefficients of the next candidate
  double* part;  // per-CTA partial sums, column-major: slot q of CTA b at part[q * gs + b]
  CycleState* st;
  int m;         // allocated restart length (H has m+1 rows)
  int gs;        // stride of a partial-sum slot (>= the largest grid)
  double* part2; // per-group sums of the partials (groups of kGroup CTAs), column-major, stride gs2
  int gs2;
  unsigned* gcnt;// per-group arrival counters, [3 sweep kinds][gs2]
};

template <typename TA> struct Csr {
  int n;
  int lanes;                        // lanes per row of the SpMV kernels: <= 1 a row per thread,
                                    // 2..32 (a power of two) a group of lanes per row
  const int* __restrict__ rowptr;   // padded: entries up to (ntiles*kTile + 8) exist (= nnz)
  const int* __restrict__ col;      // padded by >= 16 entries
  const TA* __restrict__ val;       // padded by >= 16 entries
  // Optional sliced copy (SELL-32) for the fused SpMV + projection kernels, whose warps take 64
  // consecutive rows (two slices): slice s holds rows 32 s ..
  // 32 s + 31 column-major, entry k of row 32 s + l at sptr[s] + 32 k + l (column -1, value 0
  // past the row's end), width (sptr[s + 1] - sptr[s]) / 32; sptr has nslices + 2 entries.
  // The same entries in the same order as the CSR rows, so sums are bit for bit the same; a
  // warp's loads of entry k are one contiguous 128-byte segment instead of a strided gather.
  const int* __restrict__ sptr = nullptr;
  const int* __restrict__ scol = nullptr;
  const TA* __restrict__ sval = nullptr;
};

// A vector of n elements in tile-blocked storage: element r lives at
// p[(r / kTile) * ts + r % kTile].  A plain contiguous vector is the case ts = kTile; column i of
// the tile-blocked Krylov basis (restart length m) is p = V + i * kTile, ts = (m + 1) * kTile, so
// that the first c columns of one 128-row tile are a single contiguous block of c * kTile values.
template <typename T> struct VRef {
  const T* p;
  long ts;
  __device__ __forceinline__ T operator[](long r) const {
    return p[(r >> kTileShift) * ts + (r & (kTile - 1))];
  }
};

// ------------------------------------------------------------------------------------------------
// Shared-memory layout of the pipelined kernels (host and device agree on it)
// ------------------------------------------------------------------------------------------------
constexpr int kMaxStages = 8;

__host__ __device__ constexpr size_t align16(size_t b) { return (b + 15) & ~size_t(15); }

// Sweep stage: basis tile (ncols columns) | w tile
__host__ __device__ constexpr size_t sweep_stage_bytes(int ncols, int sv, int sw) {
  return (size_t)ncols * kTile * sv + align16((size_t)kTile * sw);
}
// Stages | coefficients (two sets) | w' of a stage's tiles (PASS2: rbw = tiles per stage, else 0)
// | barriers
__host__ __device__ constexpr size_t sweep_smem_bytes(int ncols, int nstages, int sv, int sw,
                                                       int sacc, int rbw) {
  return (size_t)nstages * sweep_stage_bytes(ncols, sv, sw) + align16((size_t)2 * kMaxCols * sacc) +
         align16((size_t)rbw * kTile * sacc) + kMaxStages * 8 + 16;
}

// ------------------------------------------------------------------------------------------------
// Building blocks
// ------------------------------------------------------------------------------------------------

// Four consecutive elements starting at p (16-byte aligned for float/double, 8 for bf16).
__device__ __forceinline__ void load4(const float* p, float (&o)[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
__device__ __forceinline__ void load4(const __nv_bfloat16* p, float (&o)[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const __nv_bfloat162 a = *reinterpret_cast<const __nv_bfloat162*>(&v.x);
  const __nv_bfloat162 b = *reinterpret_cast<const __nv_bfloat162*>(&v.y);
  const float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
  o[0] = fa.x; o[1] = fa.y; o[2] = fb.x; o[3] = fb.y;
}
__device__ __forceinline__ void load4(const __half* p, float (&o)[4]) {
  const uint2 v = *reinterpret_cast<const uint2*>(p);
  const __half2 a = *reinterpret_cast<const __half2*>(&v.x);
  const __half2 b = *reinterpret_cast<const __half2*>(&v.y);
  const float2 fa = __half22float2(a), fb = __half22float2(b);
  o[0] = fa.x; o[1] = fa.y; o[2] = fb.x; o[3] = fb.y;
}
__device__ __forceinline__ void load4(const double* p, double (&o)[4]) {
  const double2 a = reinterpret_cast<const double2*>(p)[0];
  const double2 b = reinterpret_cast<const double2*>(p)[1];
  o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

template <typename TV>
__device__ __forceinline__ void load4(const TV* p, double (&o)[4]) {
  float f[4];
  load4(p, f);
  o[0] = f[0]; o[1] = f[1]; o[2] = f[2]; o[3] = f[3];
}
__device__ __forceinline__ void load4(const double* p, float (&o)[4]) {
  double d[4];
  load4(p, d);
  o[0] = (float)d[0]; o[1] = (float)d[1]; o[2] = (float)d[2]; o[3] = (float)d[3];
}

// Columns per warp of the projection: column i belongs to warp i % kWarps, slot i / kWarps.
constexpr int kColsPerWarp = kMaxCols / kWarps;

__device__ __forceinline__ void store4(float* p, const float (&v)[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}
__device__ __forceinline__ void store4(double* p, const double (&v)[4]) {
  reinterpret_cast<double2*>(p)[0] = make_double2(v[0], v[1]);
  reinterpret_cast<double2*>(p)[1] = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void store4(__nv_bfloat16* p, const float (&v)[4]) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v[0], v[1]);
  const __nv_bfloat162 b = __floats2bfloat162_rn(v[2], v[3]);
  uint2 u;
  u.x = *reinterpret_cast<const uint32_t*>(&a);
  u.y = *reinterpret_cast<const uint32_t*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}

__device__ __forceinline__ void store4(__half* p, const float (&v)[4]) {
  const __half2 a = __floats2half2_rn(v[0], v[1]);
  const __half2 b = __floats2half2_rn(v[2], v[3]);
  uint2 u;
  u.x = *reinterpret_cast<const uint32_t*>(&a);
  u.y = *reinterpret_cast<const uint32_t*>(&b);
  *reinterpret_cast<uint2*>(p) = u;
}

template <typename TV> constexpr bool is_half_v = false;
template <> constexpr bool is_half_v<__half> = true;

// Projection of one staged tile: acc[c] += sum over this lane's rows 4l..4l+3 of T[i][r] wr[r]
// for the columns i = warp + c kWarps < ncols.  The lane sums stay in registers across tiles and
// are reduced over the warp once, in store_proj_partials.
template <typename ACC, typename TV>
__device__ __forceinline__ void project_tile(const TV* __restrict__ T, const ACC (&wr)[4],
                                             int ncols, ACC (&acc)[kColsPerWarp]) {
  const int wid = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c) {
    const int i = wid + c * kWarps;
    if (i >= ncols) break;   // a real branch: slots past ncols issue nothing
    ACC v[4];
    load4(T + (size_t)i * kTile + 4 * l, v);
    acc[c] += v[0] * wr[0];
    acc[c] += v[1] * wr[1];
    acc[c] += v[2] * wr[2];
    acc[c] += v[3] * wr[3];
  }
}

// Update of one row r of a staged tile by the thread that owns it: u = sum_i T[i][r] coef[i] over
// the ncols columns, in four interleaved partial sums (columns i = 4p + q go to sum q) added as
// (s0 + s1) + (s2 + s3).  No other thread takes part, so a tile's update needs no CTA barrier.
template <typename ACC, typename TV>
__device__ __forceinline__ ACC row_update(const TV* __restrict__ T, const ACC* __restrict__ coef,
                                          int ncols, int r) {
  ACC s0 = 0, s1 = 0, s2 = 0, s3 = 0;
  int i = 0;
  for (; i + 4 <= ncols; i += 4) {
    s0 += cv<ACC>(T[(size_t)i * kTile + r]) * coef[i];
    s1 += cv<ACC>(T[(size_t)(i + 1) * kTile + r]) * coef[i + 1];
    s2 += cv<ACC>(T[(size_t)(i + 2) * kTile + r]) * coef[i + 2];
    s3 += cv<ACC>(T[(size_t)(i + 3) * kTile + r]) * coef[i + 3];
  }
  if (i < ncols) s0 += cv<ACC>(T[(size_t)i * kTile + r]) * coef[i];
  if (i + 1 < ncols) s1 += cv<ACC>(T[(size_t)(i + 1) * kTile + r]) * coef[i + 1];
  if (i + 2 < ncols) s2 += cv<ACC>(T[(size_t)(i + 2) * kTile + r]) * coef[i + 2];
  return (s0 + s1) + (s2 + s3);
}

// Both CGS updates of row r from one pass over the staged tile: sum1 = sum_i T[i][r] c1[i] and
// sum2 = sum_i T[i][r] c2[i], each in the four interleaved partial sums of row_update (so sum1 is
// bit for bit the sum PASS2 subtracted).
template <typename ACC, typename TV>
__device__ __forceinline__ void row_update2(const TV* __restrict__ T, const ACC* __restrict__ c1,
                                            const ACC* __restrict__ c2, int ncols, int r,
                                            ACC& sum1, ACC& sum2) {
  ACC a0 = 0, a1 = 0, a2 = 0, a3 = 0, b0 = 0, b1 = 0, b2 = 0, b3 = 0;
  int i = 0;
  for (; i + 4 <= ncols; i += 4) {
    const ACC v0 = cv<ACC>(T[(size_t)i * kTile + r]), v1 = cv<ACC>(T[(size_t)(i + 1) * kTile + r]);
    const ACC v2 = cv<ACC>(T[(size_t)(i + 2) * kTile + r]), v3 = cv<ACC>(T[(size_t)(i + 3) * kTile + r]);
    a0 += v0 * c1[i];
    a1 += v1 * c1[i + 1];
    a2 += v2 * c1[i + 2];
    a3 += v3 * c1[i + 3];
    b0 += v0 * c2[i];
    b1 += v1 * c2[i + 1];
    b2 += v2 * c2[i + 2];
    b3 += v3 * c2[i + 3];
  }
  if (i < ncols) {
    const ACC v = cv<ACC>(T[(size_t)i * kTile + r]);
    a0 += v * c1[i];
    b0 += v * c2[i];
  }
  if (i + 1 < ncols) {
    const ACC v = cv<ACC>(T[(size_t)(i + 1) * kTile + r]);
    a1 += v * c1[i + 1];
    b1 += v * c2[i + 1];
  }
  if (i + 2 < ncols) {
    const ACC v = cv<ACC>(T[(size_t)(i + 2) * kTile + r]);
    a2 += v * c1[i + 2];
    b2 += v * c2[i + 2];
  }
  sum1 = (a0 + a1) + (a2 + a3);
  sum2 = (b0 + b1) + (b2 + b3);
}

// Reduce the lane sums of every column over its warp and write them as this CTA's partials
// (slot i of CTA b at part[i * gs + b]).
template <typename ACC>
__device__ __forceinline__ void store_proj_partials(double* part, int gs, int ncols,
                                                    ACC (&acc)[kColsPerWarp]) {
  const int wid = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c) {
    const int i = wid + c * kWarps;
    if (i >= ncols) break;
    const ACC v = warp_sum(acc[c]);
    if (l == 0) part[(size_t)i * gs + blockIdx.x] = (double)v;
  }
}

// Sum of one partial slot over the G CTAs, by a whole warp: lanes read consecutive CTAs
// (coalesced) with sixteen independent loads in flight per lane (one L2 round trip for up to 512
// CTAs); a fixed order (deterministic).
__device__ __forceinline__ double warp_slot_sum(const double* __restrict__ p, int G) {
  const int l = threadIdx.x & 31;
  double s = 0.0;
  for (int b0 = 0; b0 < G; b0 += 512) {
    double a[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int b = b0 + 32 * k + l;
      a[k] = b < G ? __ldcg(p + b) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] += a[k + 8];
    s += ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  }
  return warp_sum(s);
}

// In the last CTA: out[i] = scale[i] * sum_b part[i][b] for i < ncols, FP64, fixed order.
// Warp w owns columns w, w + kWarps, ...; it sums two of them at a time, so every lane keeps
// sixteen coalesced loads in flight and the serial tail of a sweep is a few L2 round trips.
__device__ __forceinline__ void reduce_cols(const double* part, int gs, int G, int ncols,
                                            const double* scale, double* out) {
  const int wid = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int i0 = wid; i0 < ncols; i0 += 2 * kWarps) {
    const int i1 = i0 + kWarps;
    const bool two = i1 < ncols;
    const double* p0 = part + (size_t)i0 * gs;
    const double* p1 = part + (size_t)(two ? i1 : i0) * gs;
    double s0 = 0.0, s1 = 0.0;
    for (int b0 = 0; b0 < G; b0 += 256) {
      double a[8], c[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) {
        const int b = b0 + 32 * k + l;
        a[k] = b < G ? __ldcg(p0 + b) : 0.0;
        c[k] = (two && b < G) ? __ldcg(p1 + b) : 0.0;
      }
      s0 += ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
      s1 += ((c[0] + c[1]) + (c[2] + c[3])) + ((c[4] + c[5]) + (c[6] + c[7]));
    }
    s0 = warp_sum(s0);
    s1 = warp_sum(s1);
    if (l == 0) {
      out[i0] = scale ? scale[i0] * s0 : s0;
      if (two) out[i1] = scale ? scale[i1] * s1 : s1;
    }
  }
}

// Called by warp 0 of the last CTA; the result is valid in all its lanes.
__device__ __forceinline__ double reduce_slot(const double* part, int gs, int G, int slot) {
  return warp_slot_sum(part + (size_t)slot * gs, G);
}

// Two-level cross-CTA sums.  FP64 runs at a small fraction of the FP32 rate on this GPU, so one
// CTA summing every CTA's partials of every column is bound by its SM's FP64 pipe.  Instead the
// last CTA of each group of kGroup consecutive CTAs sums its group (a few hundred FP64 adds), and
// the last group sums the group totals (one coalesced load per lane and slot).  The grouping is
// by CTA index, so the order of every sum is fixed (deterministic).
constexpr int kGroup = 16;

// slot of the q-th reduced quantity: the ncols columns, then consecutive slots from extra_slot
// (one norm for CGS2, a second block of columns for DCGS2)
__device__ __forceinline__ int red_slot(int q, int ncols, int extra_slot) {
  return q < ncols ? q : extra_slot + (q - ncols);
}

// Group leader: part2[slot(q)][grp] = sum over the group's rows b0..b0+gsize-1 of part[slot(q)][b]
// for q < nslots.  Half-warps take one slot each (gsize <= 16 rows, one load per lane).
__device__ __forceinline__ void group_sums(const double* __restrict__ part, int gs, int b0,
                                           int gsize, int nslots, int ncols, int extra_slot,
                                           double* __restrict__ part2, int gs2, int grp) {
  const int t = threadIdx.x, wid = t >> 5, hf = (t >> 4) & 1, hl = t & 15;
  // the loop bound is per warp, so both halves of a warp always shuffle together
  for (int qb = 2 * wid; qb < nslots; qb += 2 * kWarps) {
    const int q = qb + hf;
    const bool in = q < nslots && hl < gsize;
    const int slot = red_slot(q < nslots ? q : qb, ncols, extra_slot);
    double v = in ? __ldcg(part + (size_t)slot * gs + b0 + hl) : 0.0;
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (hl == 0 && q < nslots) part2[(size_t)slot * gs2 + grp] = v;
  }
}

// Last group: out[q] = scale[q] * sum over the ngrp groups of part2[slot(q)][g] (q < ncols), the
// sums of the slots after them to extra[q - ncols].  Warp w takes slots w, w + kWarps, ...; every
// load of a round (up to 96 groups) is issued before any sum.
__device__ __forceinline__ void final_sums(const double* __restrict__ part2, int gs2, int ngrp,
                                           int nslots, int ncols, int extra_slot,
                                           const double* __restrict__ scale,
                                           double* __restrict__ out, double* __restrict__ extra) {
  const int wid = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int q0 = wid; q0 < nslots; q0 += 4 * kWarps) {
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    double sc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + u * kWarps;
      sc[u] = (q < nslots && q < ncols && scale) ? scale[q] : 1.0;
    }
    for (int gb = 0; gb < ngrp; gb += 96) {
      double v[4][3];
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int q = q0 + u * kWarps;
        const bool in = q < nslots;
        const int slot = in ? red_slot(q, ncols, extra_slot) : 0;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          const int g = gb + l + 32 * k;
          v[u][k] = (in && g < ngrp) ? __ldcg(part2 + (size_t)slot * gs2 + g) : 0.0;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) acc[u] += (v[u][0] + v[u][1]) + v[u][2];
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int q = q0 + u * kWarps;
      const double sum = warp_sum(acc[u]);
      if (l == 0 && q < nslots) {
        if (q < ncols) out[q] = sc[u] * sum;
        else extra[q - ncols] = sum;
      }
    }
  }
}

// Rotations 0..j-1 applied to the column h = col[0..j] by one warp: with x_0 = h_0, rotation i
// maps (x_i, h_{i+1}) to (c_i x_i + s_i h_{i+1}, -s_i x_i + c_i h_{i+1}); the first becomes
// col[i], the second is x_{i+1}.  The recurrence x_{i+1} = a_i x_i + b_i (a_i = -s_i,
// b_i = c_i h_{i+1}) is a first-order linear recurrence, evaluated as a warp scan of the affine
// maps (A, B): each lane composes its block of up to four consecutive rotations, a Hillis-Steele
// scan combines the lanes (five levels, one dependent FP64 operation each), and each lane then
// replays its block from its starting x.  The dependent FP64 chain is about 2 ceil(j / 32) + 7
// operations instead of j, which matters where each dependent FP64 operation costs hundreds of
// cycles.  Returns x_j (the entry the new rotation eliminates) in every lane.
__device__ __forceinline__ double givens_apply_warp(double* col, const double* rc,
                                                   const double* rsn, int j) {
  const int lane = threadIdx.x & 31;
  const double x0 = col[0];
  if (j == 0) return x0;
  const int ne = (j + 31) >> 5;            // rotations per lane, 1..4
  const int i0 = lane * ne;
  double av[4], bv[4], cv_[4], sv[4], hv[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + q;
    const bool in = q < ne && i < j;
    cv_[q] = in ? rc[i] : 1.0;
    sv[q] = in ? rsn[i] : 0.0;
    hv[q] = in ? col[i + 1] : 0.0;
    av[q] = -sv[q];
    bv[q] = cv_[q] * hv[q];
  }
  __syncwarp();                             // every lane has read col before any lane writes it
  // this lane's block as one affine map x -> A x + B (identity for lanes past the end)
  double A = 1.0, B = 0.0;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    if (q < ne && i0 + q < j) {
      B = fma(av[q], B, bv[q]);
      A = av[q] * A;
    }
  }
  // inclusive scan over the lanes: (A, B) <- (A, B) o (A', B') of the lane `off` below
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const double Ap = __shfl_up_sync(0xffffffffu, A, off);
    const double Bp = __shfl_up_sync(0xffffffffu, B, off);
    if (lane >= off) {
      B = fma(A, Bp, B);
      A = A * Ap;
    }
  }
  // exclusive prefix: the map from x_0 to the x at the start of this lane's block
  double Ae = __shfl_up_sync(0xffffffffu, A, 1);
  double Be = __shfl_up_sync(0xffffffffu, B, 1);
  if (lane == 0) {
    Ae = 1.0;
    Be = 0.0;
  }
  double x = fma(Ae, x0, Be);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + q;
    if (q < ne && i < j) {
      col[i] = fma(cv_[q], x, sv[q] * hv[q]);
      x = fma(av[q], x, bv[q]);
    }
  }
  // x_j sits with the lane of rotation j - 1
  const int last = (j - 1) / ne;
  const double xj = __shfl_sync(0xffffffffu, x, last);
  __syncwarp();
  return xj;
}

// r = sqrt(a^2 + b^2) for a Givens rotation: the plain formula (one fused multiply-add and a
// square root) wherever no intermediate can over- or underflow, else hypot.
__device__ __forceinline__ double givens_radius(double a, double b) {
  const double big = fmax(fabs(a), fabs(b));
  return (big < 1e150 && big > 1e-150) ? sqrt(fma(a, a, b * b)) : hypot(a, b);
}

// Last-arrival detection with an explicit participant count.
__device__ __forceinline__ bool arrive_last_of(unsigned* counter, unsigned count, int* flag_smem) {
  // The CTA barrier orders every thread's partials before thread 0's gpu-scope fence, which
  // (cumulatively) releases them with the arrival; the other threads do not wait for their own
  // outstanding stores (a basis column, w) here.
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned prev = atomicAdd(counter, 1u);
    *flag_smem = (prev == count - 1) ? 1 : 0;
  }
  __syncthreads();
  const bool last = *flag_smem != 0;
  if (last) __threadfence();
  return last;
}

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

// ------------------------------------------------------------------------------------------------
// CSR SpMV, one row per thread, grid-stride over rows with a per-row epilogue.
//
// Stencil-like rows are short (5-7 nonzeros), so a thread loads its row's column indices and
// values directly (seven independent loads in flight, predicated) and gathers x from L2; the
// kernels carry no shared memory and run at full occupancy, which hides the gather latency.
// Microbenchmarks on B300: 4.5 TB/s for this shape on the 150^3 Laplacian against 1.2 TB/s for a
// shared-memory-staged tile pipeline; on the 2500^2 five-point stencil 5.2 TB/s against
// 2.4-3.7 TB/s for a warp-cooperative CSR slice staged in shared memory; seven-wide loads
// instead of eight free registers (the polynomial step went from 0.72 to 0.77 of HBM).  Rows
// longer than 7 finish in a plain loop.
// ------------------------------------------------------------------------------------------------
constexpr int kRowUnroll = 7;

template <typename TA, typename TX, typename ACC>
__device__ __forceinline__ ACC row_dot(const Csr<TA>& A, const VRef<TX>& x, int row) {
  const int a = __ldg(A.rowptr + row), b = __ldg(A.rowptr + row + 1);
  int c[kRowUnroll];
  ACC v[kRowUnroll];
#pragma unroll
  for (int k = 0; k < kRowUnroll; ++k) {
    const bool in = a + k < b;
    c[k] = in ? __ldg(A.col + a + k) : -1;
    v[k] = in ? cv<ACC>(A.val[a + k]) : ACC(0);
  }
  ACC s = 0;
#pragma unroll
  for (int k = 0; k < kRowUnroll; ++k)
    if (c[k] >= 0) s += v[k] * cv<ACC>(x[c[k]]);
  for (int p = a + kRowUnroll; p < b; ++p) s += cv<ACC>(A.val[p]) * cv<ACC>(x[__ldg(A.col + p)]);
  return s;
}

// CSR SpMV with L lanes per row (L = 2..32), for rows with many nonzeros: the lanes of a group
// take every L-th nonzero of the row (consecutive lanes, consecutive entries: coalesced col/val
// loads), then add their partial sums by a butterfly over the group (a fixed order); the group's
// first lane runs the epilogue.  The groups of a warp walk their rows together, so every lane
// reaches the shuffles.
template <typename TA, typename TX, typename ACC, typename Epi, int L>
__device__ __forceinline__ void spmv_rows_vec(const Csr<TA>& A, const VRef<TX>& x, Epi& epi,
                                              int rev) {
  constexpr int G = 32 / L;   // rows per warp and pass
  const int lane = threadIdx.x & 31, li = lane & (L - 1);
  const long warp = (blockIdx.x * (long)blockDim.x + threadIdx.x) >> 5;
  const long nwarps = ((long)gridDim.x * blockDim.x) >> 5;
  for (long base = warp * G; base < A.n; base += nwarps * G) {   // warp-uniform
    const bool valid = base + lane / L < A.n;
    const long r = rev ? A.n - 1 - (base + lane / L) : base + lane / L;
    ACC s = 0;
    if (valid) {
      const int a = __ldg(A.rowptr + r), b = __ldg(A.rowptr + r + 1);
#pragma unroll 4
      for (int p = a + li; p < b; p += L) s += cv<ACC>(A.val[p]) * cv<ACC>(x[__ldg(A.col + p)]);
    }
#pragma unroll
    for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (valid && li == 0) {
      epi.prefetch((int)r);
      epi.apply((int)r, s);
    }
  }
}

// ROWS = rows per thread and iteration (1 or 2); the default takes one for FP64 accumulation.
// A.lanes > 1 selects the lanes-per-row form above.  rev = 1 walks the rows from the last one
// (row q of the walk is row n - 1 - q), so that a launch starts on the rows, matrix entries and
// vector entries its predecessor touched last and left in L2; every row's result is the same.
template <typename TA, typename TX, typename ACC, typename Epi, int ROWS = (sizeof(ACC) == 8 ? 1 : 2)>
__device__ __forceinline__ void spmv_rows(const Csr<TA>& A, const VRef<TX>& x, Epi& epi,
                                          int rev = 0) {
  if (A.lanes > 1) {
    switch (A.lanes) {
      case 2: spmv_rows_vec<TA, TX, ACC, Epi, 2>(A, x, epi, rev); return;
      case 4: spmv_rows_vec<TA, TX, ACC, Epi, 4>(A, x, epi, rev); return;
      case 8: spmv_rows_vec<TA, TX, ACC, Epi, 8>(A, x, epi, rev); return;
      case 16: spmv_rows_vec<TA, TX, ACC, Epi, 16>(A, x, epi, rev); return;
      default: spmv_rows_vec<TA, TX, ACC, Epi, 32>(A, x, epi, rev); return;
    }
  }
  if constexpr (ROWS == 1) {
    // one row per thread and iteration (for FP64, two would double the live FP64 registers and
    // cost the occupancy that hides the gather latency of the SpMV)
    const long stride = (long)gridDim.x * blockDim.x;
    for (long q = blockIdx.x * (long)blockDim.x + threadIdx.x; q < A.n; q += stride) {
      const long r = rev ? A.n - 1 - q : q;
      epi.prefetch((int)r);
      epi.apply((int)r, row_dot<TA, TX, ACC>(A, x, (int)r));
    }
  } else {
    // two rows per thread and iteration (r and r + half the stride), their loads interleaved, so
    // each thread keeps twice as many independent loads in flight
    const long stride = 2L * gridDim.x * blockDim.x;
    const long half = (long)gridDim.x * blockDim.x;
    for (long q0 = blockIdx.x * (long)blockDim.x + threadIdx.x; q0 < A.n; q0 += stride) {
      const bool has1 = q0 + half < A.n;
      const long r0 = rev ? A.n - 1 - q0 : q0;
      const long r1 = rev ? A.n - 1 - (q0 + half) : q0 + half;   // used only if has1
      const int a0 = __ldg(A.rowptr + r0), b0 = __ldg(A.rowptr + r0 + 1);
      const int a1 = has1 ? __ldg(A.rowptr + r1) : 0, b1 = has1 ? __ldg(A.rowptr + r1 + 1) : 0;
      epi.prefetch((int)r0);
      int c0[kRowUnroll], c1[kRowUnroll];
      ACC v0[kRowUnroll], v1[kRowUnroll];
#pragma unroll
      for (int k = 0; k < kRowUnroll; ++k) {
        const bool i0 = a0 + k < b0, i1 = a1 + k < b1;
        c0[k] = i0 ? __ldg(A.col + a0 + k) : -1;
        c1[k] = i1 ? __ldg(A.col + a1 + k) : -1;
        v0[k] = i0 ? cv<ACC>(A.val[a0 + k]) : ACC(0);
        v1[k] = i1 ? cv<ACC>(A.val[a1 + k]) : ACC(0);
      }
      ACC s0 = 0, s1 = 0;
#pragma unroll
      for (int k = 0; k < kRowUnroll; ++k) {
        if (c0[k] >= 0) s0 += v0[k] * cv<ACC>(x[c0[k]]);
        if (c1[k] >= 0) s1 += v1[k] * cv<ACC>(x[c1[k]]);
      }
      for (int p = a0 + kRowUnroll; p < b0; ++p) s0 += cv<ACC>(A.val[p]) * cv<ACC>(x[__ldg(A.col + p)]);
      for (int p = a1 + kRowUnroll; p < b1; ++p) s1 += cv<ACC>(A.val[p]) * cv<ACC>(x[__ldg(A.col + p)]);
      epi.apply((int)r0, s0);
      if (has1) {
        epi.prefetch((int)r1);
        epi.apply((int)r1, s1);
      }
    }
  }
}

// Inner SpMV of step j alone, w = s_j A z_j, for the FP64 solver: its first projection runs as
// k_sweep<PROJ>.  (Fused with the projection, the FP64 kernel needs twice the registers and the
// reduce-scatter's FP64 adds on B300's slow FP64 pipe; measured slower on the FP64 solver.)
template <typename TA, typename TX, typename TW, typename ACC>
__global__ void __launch_bounds__(kThreads, sizeof(ACC) == 4 ? 5 : 1)
    k_spmv_w(Csr<TA> A, VRef<TX> x, TW* __restrict__ w, Krylov K, int j, int rev) {
  const CycleState* st = K.st;
  if (st->stop || st->err) return;
  struct Epi {
    TW* w;
    ACC scale;
    __device__ void prefetch(int) {}
    __device__ void apply(int row, ACC ax) { w[row] = cv<TW>(ax * scale); }
  } epi{w, (ACC)K.s[j]};
  spmv_rows<TA, TX, ACC>(A, x, epi, rev);
}

// ------------------------------------------------------------------------------------------------
// Inner SpMV of step j fused with the first CGS projection:
//   w = s_j A z_j,   h1 = s_i V_j^T w (i = 0..j),   ||w||^2
// The kernel keeps the SpMV's shape (no shared-memory pipeline, full occupancy to hide the gather
// latency).  Each warp takes 64 consecutive rows (two 32-row slices of one 128-row tile): lane l
// computes rows b + l and b + 32 + l, writes w, and then reads the same rows of the basis columns
// straight from the tile-blocked basis (one coalesced 128-byte load per column and slice).  Sixteen
// columns at a time, the per-lane products are summed over the warp by a reduce-scatter (16
// shuffles for 16 columns), so each lane keeps one running column sum per 16 columns.  Per CTA the
// warps' sums are added in a fixed order and the usual two-level cross-CTA sum gives h1 and ||w||.
// Compared with a separate projection sweep this saves reading w back, one launch and its
// pipeline fill and tail, and runs the SpMV's latency-bound gathers under the basis stream.
// ------------------------------------------------------------------------------------------------
constexpr int kFusedRows = 64;                    // rows of one warp iteration
constexpr int kFusedBatches = kMaxCols / 16;      // 16-column batches of the projection

// Sum over the warp of 16 per-lane values, scattered: lanes l and l ^ 1 receive the total of
// p[(l >> 1) & 15].  Halving exchanges over lane bits 4, 3, 2, 1 (8 + 4 + 2 + 1 shuffles) and a
// last pairwise sum; every sum is taken in a fixed order.
template <typename T> __device__ __forceinline__ T reduce_scatter16(T (&p)[16]) {
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int h = 8; h >= 1; h >>= 1) {
    const bool up = (l & (2 * h)) != 0;   // this lane keeps the upper h of the current 2h values
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const T send = up ? p[k] : p[k + h];
      const T keep = up ? p[k + h] : p[k];
      p[k] = keep + __shfl_xor_sync(0xffffffffu, send, 2 * h);
    }
  }
  return p[0] + __shfl_xor_sync(0xffffffffu, p[0], 1);
}

// A x for the warp's 64 rows b .. b + 63: lane l returns rows b + l (o0) and b + 32 + l (o1).
// L = 1: each lane its two rows, loads interleaved (the sums of spmv_rows).  L > 1: L lanes per
// row over 2 L sub-passes (the sums of spmv_rows_vec), the group leaders' results handed to the
// row's lane through wbuf (64 values of this warp).  Rows >= n give 0.
// Bytes at the end of a sweep's traversal kept at normal L2 priority (the 126 MB L2 less the
// vectors the next kernel also touches).
constexpr size_t kL2KeepBytes = (size_t)64 << 20;

template <typename TA, typename TX, typename ACC, int L>
__device__ __forceinline__ void fused_rows(const Csr<TA>& A, const VRef<TX>& x, long b, ACC& o0,
                                           ACC& o1, ACC* __restrict__ wbuf) {
  const int lane = threadIdx.x & 31;
  if constexpr (L == 1) {
    const long r0 = b + lane, r1 = b + 32 + lane;
    const bool h0 = r0 < A.n, h1 = r1 < A.n;
    // the matrix is read once per launch: evict-first in L2 (the policy is made here, not kept
    // in a register across the caller's loop)
    const uint64_t pol = l2_evict_first_policy();
    if (A.sptr) {
      // the two 32-row slices b / 32 and b / 32 + 1 (b is a multiple of 64)
      const long s0 = b >> 5;
      const int p0 = __ldg(A.sptr + s0), p1 = __ldg(A.sptr + s0 + 1), p2 = __ldg(A.sptr + s0 + 2);
      const int w0 = (p1 - p0) >> 5, w1 = (p2 - p1) >> 5;
      const int q0 = p0 + lane, q1 = p1 + lane;
      int c0[kRowUnroll], c1[kRowUnroll];
      ACC v0[kRowUnroll], v1[kRowUnroll];
#pragma unroll
      for (int k = 0; k < kRowUnroll; ++k) {
        const bool i0 = k < w0, i1 = k < w1;
        c0[k] = ld_hint_if(i0, A.scol + q0 + 32 * k, -1, pol);
        c1[k] = ld_hint_if(i1, A.scol + q1 + 32 * k, -1, pol);
        v0[k] = cv<ACC>(ld_hint_if(i0, A.sval + q0 + 32 * k, TA(0), pol));
        v1[k] = cv<ACC>(ld_hint_if(i1, A.sval + q1 + 32 * k, TA(0), pol));
      }
      ACC s0s = 0, s1s = 0;
#pragma unroll
      for (int k = 0; k < kRowUnroll; ++k) {
        if (c0[k] >= 0) s0s += v0[k] * cv<ACC>(x[c0[k]]);
        if (c1[k] >= 0) s1s += v1[k] * cv<ACC>(x[c1[k]]);
      }
      for (int k = kRowUnroll; k < w0; ++k) {
        const int c = __ldg(A.scol + q0 + 32 * k);
        if (c >= 0) s0s += cv<ACC>(A.sval[q0 + 32 * k]) * cv<ACC>(x[c]);
      }
      for (int k = kRowUnroll; k < w1; ++k) {
        const int c = __ldg(A.scol + q1 + 32 * k);
        if (c >= 0) s1s += cv<ACC>(A.sval[q1 + 32 * k]) * cv<ACC>(x[c]);
      }
      o0 = s0s;
      o1 = s1s;
      return;
    }
    const int a0 = ld_hint_if(h0, A.rowptr + r0, 0, pol), e0 = ld_hint_if(h0, A.rowptr + r0 + 1, 0, pol);
    const int a1 = ld_hint_if(h1, A.rowptr + r1, 0, pol), e1 = ld_hint_if(h1, A.rowptr + r1 + 1, 0, pol);
    int c0[kRowUnroll], c1[kRowUnroll];
    ACC v0[kRowUnroll], v1[kRowUnroll];
#pragma unroll
    for (int k = 0; k < kRowUnroll; ++k) {
      const bool i0 = a0 + k < e0, i1 = a1 + k < e1;
      c0[k] = ld_hint_if(i0, A.col + a0 + k, -1, pol);
      c1[k] = ld_hint_if(i1, A.col + a1 + k, -1, pol);
      v0[k] = cv<ACC>(ld_hint_if(i0, A.val + a0 + k, TA(0), pol));
      v1[k] = cv<ACC>(ld_hint_if(i1, A.val + a1 + k, TA(0), pol));
    }
    ACC s0 = 0, s1 = 0;
#pragma unroll
    for (int k = 0; k < kRowUnroll; ++k) {
      if (c0[k] >= 0) s0 += v0[k] * cv<ACC>(x[c0[k]]);
      if (c1[k] >= 0) s1 += v1[k] * cv<ACC>(x[c1[k]]);
    }
    for (int p = a0 + kRowUnroll; p < e0; ++p) s0 += cv<ACC>(A.val[p]) * cv<ACC>(x[__ldg(A.col + p)]);
    for (int p = a1 + kRowUnroll; p < e1; ++p) s1 += cv<ACC>(A.val[p]) * cv<ACC>(x[__ldg(A.col + p)]);
    o0 = s0;
    o1 = s1;
  } else {
    constexpr int G = 32 / L;   // rows per sub-pass
    const int li = lane & (L - 1);
#pragma unroll 1
    for (int sp = 0; sp < 2 * L; ++sp) {
      const long r = b + sp * G + lane / L;
      ACC s = 0;
      if (r < A.n) {
        const int a = __ldg(A.rowptr + r), e = __ldg(A.rowptr + r + 1);
#pragma unroll 4
        for (int p = a + li; p < e; p += L) s += cv<ACC>(A.val[p]) * cv<ACC>(x[__ldg(A.col + p)]);
      }
#pragma unroll
      for (int o = L / 2; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (li == 0) wbuf[sp * G + lane / L] = s;
    }
    __syncwarp();
    o0 = wbuf[lane];
    o1 = wbuf[32 + lane];
    __syncwarp();
  }
}

// Cross-CTA sums of the first projection: this CTA's partials are in part (slots 0..ncols-1 the
// columns, slot kMaxCols the norm); the last group's last CTA writes h1 = s_i * sum and az2.
__device__ __forceinline__ void proj_cross_cta(Krylov& K, int ncols, int* flag) {
  CycleState* st = K.st;
  const int G = gridDim.x;
  const int nslots = ncols + 1;
  const int grp = blockIdx.x / kGroup, ngrp = (G + kGroup - 1) / kGroup;
  const int b0 = grp * kGroup, gsize = min(kGroup, G - b0);
  unsigned* gc = K.gcnt + (size_t)CNT_A * K.gs2 + grp;
  if (!arrive_last_of(gc, (unsigned)gsize, flag)) return;
  group_sums(K.part, K.gs, b0, gsize, nslots, ncols, kMaxCols, K.part2, K.gs2, grp);
  if (threadIdx.x == 0) *gc = 0;
  if (!arrive_last_of(&st->cnt[CNT_A], (unsigned)ngrp, flag)) return;
  final_sums(K.part2, K.gs2, ngrp, nslots, ncols, kMaxCols, K.s, K.h1, &st->az2);
  if (threadIdx.x == 0) st->cnt[CNT_A] = 0;
}

// Shared memory of k_spmv_proj (declared once in the kernel, whatever the lanes per row).
template <typename ACC> struct SpmvProjSmem {
  ACC wbuf[kWarps][kFusedRows];   // L > 1: row sums handed to their lanes
  ACC red[kWarps][kMaxCols];      // per-warp column sums
  ACC redn[kWarps];
  int flag;
};

template <typename TA, typename TX, typename TV, typename TW, typename ACC, int L>
__device__ __forceinline__ void spmv_proj_impl(const Csr<TA>& A, const VRef<TX>& x,
                                               const TV* __restrict__ V, long vts,
                                               TW* __restrict__ w, Krylov& K, int j, int rev,
                                               SpmvProjSmem<ACC>& sm) {
  auto& wbuf = sm.wbuf;
  auto& red = sm.red;
  auto& redn = sm.redn;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int ncols = j + 1;
  const int nb = (ncols + 15) >> 4;
  const ACC scale = (ACC)K.s[j];
  ACC acc[kFusedBatches];
#pragma unroll
  for (int q = 0; q < kFusedBatches; ++q) acc[q] = 0;
  ACC nrm2 = 0;
  const long nch = (A.n + kFusedRows - 1) / kFusedRows;
  for (long ch = (long)blockIdx.x * kWarps + wid; ch < nch; ch += (long)gridDim.x * kWarps) {
    const long b = (rev ? nch - 1 - ch : ch) * kFusedRows;
    ACC s0, s1;
    fused_rows<TA, TX, ACC, L>(A, x, b, s0, s1, wbuf[wid]);
    const long r0 = b + lane, r1 = b + 32 + lane;
    const bool h0 = r0 < A.n, h1 = r1 < A.n;
    const TW q0 = cv<TW>(s0 * scale), q1 = cv<TW>(s1 * scale);
    if (h0) w[r0] = q0;
    if (h1) w[r1] = q1;
    const ACC w0 = h0 ? cv<ACC>(q0) : ACC(0), w1 = h1 ? cv<ACC>(q1) : ACC(0);
    nrm2 += w0 * w0 + w1 * w1;
    // the 64 rows lie in one tile (b is a multiple of 64); padded rows of V are zero
    const TV* Vt = V + (size_t)(b >> kTileShift) * vts + (b & (kTile - 1)) + lane;
#pragma unroll
    for (int q = 0; q < kFusedBatches; ++q) {
      if (q >= nb) break;
      ACC p[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int c = 16 * q + k;
        ACC va = 0, vb = 0;
        if (c < ncols) {
          va = cv<ACC>(Vt[(size_t)c * kTile]);
          vb = cv<ACC>(Vt[(size_t)c * kTile + 32]);
        }
        p[k] = va * w0 + vb * w1;
      }
      acc[q] += reduce_scatter16(p);
    }
  }
  // per-warp column sums (even lanes hold column 16 q + lane / 2), then the CTA's, fixed order
#pragma unroll
  for (int q = 0; q < kFusedBatches; ++q) {
    const int c = 16 * q + (lane >> 1);
    if (q < nb && (lane & 1) == 0 && c < ncols) red[wid][c] = acc[q];
  }
  nrm2 = warp_sum(nrm2);
  if (lane == 0) redn[wid] = nrm2;
  __syncthreads();
  for (int c = t; c < ncols; c += kThreads) {
    ACC sum = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) sum += red[q][c];
    K.part[(size_t)c * K.gs + blockIdx.x] = (double)sum;
  }
  if (t == 0) {
    ACC sum = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) sum += redn[q];
    K.part[(size_t)kMaxCols * K.gs + blockIdx.x] = (double)sum;
  }
  proj_cross_cta(K, ncols, &sm.flag);
}

template <typename TA, typename TX, typename TV, typename TW, typename ACC>
__global__ void __launch_bounds__(kThreads, sizeof(ACC) == 4 ? 4 : 2)
    k_spmv_proj(Csr<TA> A, VRef<TX> x, const TV* __restrict__ V, long vts, TW* __restrict__ w,
                Krylov K, int j, int rev) {
  const CycleState* st = K.st;
  if (st->stop || st->err) return;
  __shared__ SpmvProjSmem<ACC> sm;
  switch (A.lanes) {
    case 2: spmv_proj_impl<TA, TX, TV, TW, ACC, 2>(A, x, V, vts, w, K, j, rev, sm); return;
    case 4: spmv_proj_impl<TA, TX, TV, TW, ACC, 4>(A, x, V, vts, w, K, j, rev, sm); return;
    case 8: spmv_proj_impl<TA, TX, TV, TW, ACC, 8>(A, x, V, vts, w, K, j, rev, sm); return;
    case 16: spmv_proj_impl<TA, TX, TV, TW, ACC, 16>(A, x, V, vts, w, K, j, rev, sm); return;
    case 32: spmv_proj_impl<TA, TX, TV, TW, ACC, 32>(A, x, V, vts, w, K, j, rev, sm); return;
    default: spmv_proj_impl<TA, TX, TV, TW, ACC, 1>(A, x, V, vts, w, K, j, rev, sm); return;
  }
}

// ------------------------------------------------------------------------------------------------
// DCGS2: classical Gram-Schmidt with the second pass delayed by one step (Bielich, Langou, Thomas,
// Swirydowicz, Yamazaki, Boman 2022).  A different algorithm from the CGS2 of Section III-A: the
// same Arnoldi factorisation in exact arithmetic, with one global reduction per step.  Basis
// columns are stored unscaled: V[:, i] with scale s_i (v_i = s_i V[:, i]) for the final columns
// i < j, and in column j the candidate U_j (u_j = s_j U_j, one projection done, not normalised).
// Step j is two kernels:
//   k_dc_reduce : x = s_j A z (z = U_j, or p(A) U_j), and the one reduction
//                 a_i = V_i^T U_j, b_i = V_i^T x  (i = 0..j; i = j gives U_j^T U_j and U_j^T x);
//                 the last CTA then finishes column j-1 of H (delayed pass), its Givens rotation
//                 and the stop tests, and forms the next provisional column and the update's
//                 coefficients (dc_small)
//   k_sweep<DC_UPDATE> : V[:, j] = U_j - sum_i V_i ca_i, then
//                 U_{j+1} = x - sum_i V_i cb_i - V[:, j] cb_j  (no reduction, no tail)
// After the last step one more k_dc_reduce without the SpMV finishes column m-1.
// ------------------------------------------------------------------------------------------------

// Reduce-scatter of 8 per-lane values: lanes l with equal l >> 2 receive the total of p[(l >> 2) & 7]
// (halving exchanges over lane bits 4, 3, 2, then sums over bits 1 and 0; fixed order).
template <typename T> __device__ __forceinline__ T reduce_scatter8(T (&p)[8]) {
  const int l = threadIdx.x & 31;
#pragma unroll
  for (int h = 4; h >= 1; h >>= 1) {
    const bool up = (l & (4 * h)) != 0;
#pragma unroll
    for (int k = 0; k < h; ++k) {
      const T send = up ? p[k] : p[k + h];
      const T keep = up ? p[k + h] : p[k];
      p[k] = keep + __shfl_xor_sync(0xffffffffu, send, 4 * h);
    }
  }
  T v = p[0] + __shfl_xor_sync(0xffffffffu, p[0], 2);
  return v + __shfl_xor_sync(0xffffffffu, v, 1);
}

template <typename ACC> struct DcSmem {
  ACC wbuf[kWarps][kFusedRows];   // L > 1: row sums handed to their lanes
  ACC red1[kWarps][kMaxCols];     // per-warp sums of V_i^T U_j
  ACC red2[kWarps][kMaxCols];     // per-warp sums of V_i^T x
  double sv[kMaxCols];            // dc_small: s_i = s_i' kappa a_i
  double zv[kMaxCols];            //           z_i = s_i' b_i
  double tv[kMaxCols + 1];        //           t = Hbar s
  double red[kWarps];
  int flag;
};

// Sum over the CTA of one value per thread (FP64, fixed order); valid in every thread.
__device__ __forceinline__ double cta_sum(double v, double* red) {
  return block_sum(v, red);
}

// Last CTA of step j (all threads): a_i, alpha' in K.h1[0..j], b_i, beta' in K.h2[0..j] (raw sums of
// the stored vectors); K.s[i] = scale of final column i (i < j), K.s[j] = kappa, the candidate's
// scale.  spmv = 0: the cycle-end call (no x; finish column j - 1 only).
template <typename ACC>
__device__ __forceinline__ void dc_small(Krylov& K, int j, int spmv, DcSmem<ACC>& sm) {
  CycleState* st = K.st;
  const int t = threadIdx.x, lane = t & 31;
  const int m1 = K.m + 1;
  const double kap = K.s[j];
  for (int i = t; i < j; i += kThreads) {
    sm.sv[i] = K.s[i] * kap * K.h1[i];
    sm.zv[i] = spmv ? K.s[i] * K.h2[i] : 0.0;
  }
  const double alpha = kap * kap * K.h1[j];
  const double beta = spmv ? kap * K.h2[j] : 0.0;
  __syncthreads();
  double ps = 0.0, pz = 0.0;
  for (int i = t; i < j; i += kThreads) {
    ps += sm.sv[i] * sm.sv[i];
    pz += sm.sv[i] * sm.zv[i];
  }
  const double ss = cta_sum(ps, sm.red);
  const double sz = cta_sum(pz, sm.red);
  double nu = 1.0;
  if (j >= 1) {
    // column jc = j - 1 final: provisional coefficients plus the delayed second pass
    const int jc = j - 1;
    const double nu2 = alpha - ss;
    nu = sqrt(fmax(nu2, 0.0));
    double* Hc = K.H + (size_t)jc * m1;
    for (int i = t; i < j; i += kThreads) Hc[i] += sm.sv[i];
    if (t == 0) Hc[j] = nu;
    __syncthreads();
    if (t < 32) {   // warp 0: rotations of column jc, new rotation, g, stop tests (as in CGS2)
      double* col = sm.tv;   // staging (free until t is formed below)
      double* Rc = K.R + (size_t)jc * m1;
      for (int i = lane; i <= j; i += 32) col[i] = Hc[i];
      __syncwarp();
      const double xr = givens_apply_warp(col, K.cs, K.sn, jc);
      if (lane == 0) {
        const double gj = K.g[jc];
        const double r = givens_radius(xr, nu);
        double c = 1.0, sgn = 0.0;
        if (r != 0.0) {
          const double ir = 1.0 / r;
          c = xr * ir;
          sgn = nu * ir;
        }
        K.cs[jc] = c;
        K.sn[jc] = sgn;
        col[jc] = r;
        col[j] = 0.0;
        K.g[j] = -sgn * gj;
        K.g[jc] = c * gj;
        const double imp = fabs(sgn * gj);
        st->implicit = imp;
        st->k = j;
        int reason = 0;
        if (!finite_d(nu) || !finite_d(imp) || !finite_d(r) || !finite_d(alpha)) {
          reason = 3;
          st->nan = 1;
        } else if (!(nu > 10.0 * st->uround * sqrt(st->hp2 + nu * nu))) {
          reason = 2;   // lucky breakdown (u_j in the span of the basis)
          st->breakdowns += 1;
        } else {
          const double thr = st->implicit_fp64 ? st->tol * st->bnorm : st->inner_tol * st->gamma;
          if (imp <= thr) reason = 1;
          else if (j >= st->jmax || !spmv) reason = 4;
        }
        if (reason) {
          st->reason = reason;
          st->stop = 1;
        }
      }
      __syncwarp();
      for (int i = lane; i <= j; i += 32) Rc[i] = col[i];
    }
  }
  __syncthreads();
  if (st->stop || !spmv) return;
  // v_j = (u_j - Q s) / nu: stored column j gets scale kappa / nu
  const double sig = (j >= 1) ? kap / nu : kap;
  // t = Hbar_j s (Hbar_j = H[0..j, 0..j-1], final); c = [z, (beta - s^T z) / nu]
  for (int i = t; i <= j; i += kThreads) {
    double acc = 0.0;
    for (int k = (i > 0 ? i - 1 : 0); k < j; ++k) acc += K.H[(size_t)k * m1 + i] * sm.sv[k];
    sm.tv[i] = acc;
  }
  __syncthreads();
  const double cj = (beta - sz) / nu;
  double ph = 0.0;
  double* Hn = K.H + (size_t)j * m1;   // provisional column j = [Q, v_j]^T A v_j
  for (int i = t; i <= j; i += kThreads) {
    const double ci = i < j ? sm.zv[i] : cj;
    const double hn = (ci - sm.tv[i]) / nu;
    Hn[i] = hn;
    ph += hn * hn;
    if (i < j) {
      K.ca[i] = K.s[i] * K.s[i] * K.h1[i];    // sigma_i s_i / kappa
      K.cb[i] = K.s[i] * sm.zv[i];            // sigma_i z_i
    }
  }
  const double hp2 = cta_sum(ph, sm.red);
  if (t == 0) {
    K.cb[j] = sig * cj;
    K.s[j] = sig;
    K.s[j + 1] = 1.0 / nu;                    // scale of the next candidate
    st->hp2 = hp2;
  }
}

template <typename TA, typename TX, typename TV, typename TW, typename ACC, int L>
__device__ __forceinline__ void dc_reduce_impl(const Csr<TA>& A, const VRef<TX>& x,
                                               const TV* __restrict__ V, long vts,
                                               TW* __restrict__ xout, Krylov& K, int j, int spmv,
                                               int rev, DcSmem<ACC>& sm) {
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int ncols = j + 1;
  const int nb = (ncols + 7) >> 3;
  for (int c = lane; c < kMaxCols; c += 32) {
    sm.red1[wid][c] = 0;
    sm.red2[wid][c] = 0;
  }
  __syncwarp();
  const ACC scale = (ACC)K.s[j];
  const long nch = (A.n + kFusedRows - 1) / kFusedRows;
  for (long ch = (long)blockIdx.x * kWarps + wid; ch < nch; ch += (long)gridDim.x * kWarps) {
    const long b = (rev ? nch - 1 - ch : ch) * kFusedRows;
    ACC x0 = 0, x1 = 0;
    if (spmv) {
      ACC s0, s1;
      fused_rows<TA, TX, ACC, L>(A, x, b, s0, s1, sm.wbuf[wid]);
      const long r0 = b + lane, r1 = b + 32 + lane;
      const bool h0 = r0 < A.n, h1 = r1 < A.n;
      const TW q0 = cv<TW>(s0 * scale), q1 = cv<TW>(s1 * scale);
      if (h0) xout[r0] = q0;
      if (h1) xout[r1] = q1;
      x0 = h0 ? cv<ACC>(q0) : ACC(0);
      x1 = h1 ? cv<ACC>(q1) : ACC(0);
    }
    // the 64 rows lie in one tile (b is a multiple of 64, b + 63 < n); padded rows of V are zero
    const TV* Vt = V + (size_t)(b >> kTileShift) * vts + (b & (kTile - 1)) + lane;
    const ACC u0 = cv<ACC>(Vt[(size_t)j * kTile]), u1 = cv<ACC>(Vt[(size_t)j * kTile + 32]);
    // sixteen columns' rows are loaded at once (32 loads in flight per lane), then reduced as two
    // halves of eight against U_j and against x
    for (int q2 = 0; q2 < nb; q2 += 2) {
      ACC va[16], vb[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const int c = 8 * q2 + k;
        va[k] = 0;
        vb[k] = 0;
        if (c < ncols) {
          va[k] = cv<ACC>(Vt[(size_t)c * kTile]);
          vb[k] = cv<ACC>(Vt[(size_t)c * kTile + 32]);
        }
      }
#pragma unroll
      for (int hh = 0; hh < 2; ++hh) {
        const int q = q2 + hh;
        if (q >= nb) break;
        ACC p[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) p[k] = va[8 * hh + k] * u0 + vb[8 * hh + k] * u1;
        const ACC ta = reduce_scatter8(p);
        if ((lane & 3) == 0) sm.red1[wid][8 * q + (lane >> 2)] += ta;
        if (spmv) {
#pragma unroll
          for (int k = 0; k < 8; ++k) p[k] = va[8 * hh + k] * x0 + vb[8 * hh + k] * x1;
          const ACC tb = reduce_scatter8(p);
          if ((lane & 3) == 0) sm.red2[wid][8 * q + (lane >> 2)] += tb;
        }
      }
    }
  }
  __syncthreads();
  for (int c = t; c < ncols; c += kThreads) {
    ACC s1 = 0, s2 = 0;
#pragma unroll
    for (int q = 0; q < kWarps; ++q) {
      s1 += sm.red1[q][c];
      s2 += sm.red2[q][c];
    }
    K.part[(size_t)c * K.gs + blockIdx.x] = (double)s1;
    K.part[(size_t)(kSlotB + c) * K.gs + blockIdx.x] = (double)s2;
  }
  // two-level cross-CTA sums: raw a (and alpha') to K.h1, raw b (and beta') to K.h2
  CycleState* st = K.st;
  const int G = gridDim.x;
  const int nslots = spmv ? 2 * ncols : ncols;
  const int grp = blockIdx.x / kGroup, ngrp = (G + kGroup - 1) / kGroup;
  const int b0 = grp * kGroup, gsize = min(kGroup, G - b0);
  unsigned* gc = K.gcnt + (size_t)CNT_A * K.gs2 + grp;
  if (!arrive_last_of(gc, (unsigned)gsize, &sm.flag)) return;
  group_sums(K.part, K.gs, b0, gsize, nslots, ncols, kSlotB, K.part2, K.gs2, grp);
  if (t == 0) *gc = 0;
  if (!arrive_last_of(&st->cnt[CNT_A], (unsigned)ngrp, &sm.flag)) return;
  final_sums(K.part2, K.gs2, ngrp, nslots, ncols, kSlotB, nullptr, K.h1, K.h2);
  if (t == 0) st->cnt[CNT_A] = 0;
  __syncthreads();
  dc_small<ACC>(K, j, spmv, sm);
}

template <typename TA, typename TX, typename TV, typename TW, typename ACC>
__global__ void __launch_bounds__(kThreads, sizeof(ACC) == 4 ? 4 : 2)
    k_dc_reduce(Csr<TA> A, VRef<TX> x, const TV* __restrict__ V, long vts, TW* __restrict__ xout,
                Krylov K, int j, int spmv, int rev) {
  const CycleState* st = K.st;
  if (st->stop || st->err) return;
  __shared__ DcSmem<ACC> sm;
  switch (spmv ? A.lanes : 1) {
    case 2: dc_reduce_impl<TA, TX, TV, TW, ACC, 2>(A, x, V, vts, xout, K, j, spmv, rev, sm); return;
    case 4: dc_reduce_impl<TA, TX, TV, TW, ACC, 4>(A, x, V, vts, xout, K, j, spmv, rev, sm); return;
    case 8: dc_reduce_impl<TA, TX, TV, TW, ACC, 8>(A, x, V, vts, xout, K, j, spmv, rev, sm); return;
    case 16: dc_reduce_impl<TA, TX, TV, TW, ACC, 16>(A, x, V, vts, xout, K, j, spmv, rev, sm); return;
    case 32: dc_reduce_impl<TA, TX, TV, TW, ACC, 32>(A, x, V, vts, xout, K, j, spmv, rev, sm); return;
    default: dc_reduce_impl<TA, TX, TV, TW, ACC, 1>(A, x, V, vts, xout, K, j, spmv, rev, sm); return;
  }
}

// ------------------------------------------------------------------------------------------------
// Basis sweeps (kernels B and C, and the cycle-end solution update)
// ------------------------------------------------------------------------------------------------
enum SweepMode {
  SWEEP_PASS2 = 0, SWEEP_UPDATE = 1, SWEEP_SOLUTION = 2, SWEEP_PROJ = 3,
  SWEEP_DC_UPDATE = 4   // DCGS2 update of step j (vout = column j + 1; column j rewritten)
};

// UPDATE subtracts the two CGS passes one after the other, w' = w - V (s h1), w'' = w' - V (s h2),
// from one read of V: w' is bit for bit the vector PASS2 projected, as in the unfused algorithm.
// The FP64 solver (bound by B300's FP64 units, not by memory) subtracts V s (h1 + h2) at once,
// which halves its FP64 work in this sweep and differs only at FP64 rounding level.
template <typename ACC> constexpr bool kTwoPassUpdate = sizeof(ACC) == 4;

// A stage holds rb consecutive 128-row tiles (rb chosen by the host so that a stage carries
// ~16 KB even for the first steps of a cycle, when a tile's basis block is only a few columns):
// per tile the basis block (ncols columns, one contiguous copy) and, except for SOLUTION, the
// tile of w.
template <int MODE, typename TV, typename TW, typename ACC, typename TZ>
__global__ void __launch_bounds__(kThreads, 3)
    k_sweep(int n, const TV* __restrict__ V, long vts, const TW* __restrict__ w, Krylov K, int j,
            int nstages, int rb, TV* __restrict__ vout, double* __restrict__ x64,
            TZ* __restrict__ zout, int rev) {
  CycleState* st = K.st;
  // PROJ (FP64 solver only)/PASS2/UPDATE belong to step j of the cycle; SOLUTION runs once per
  // cycle
  if ((MODE != SWEEP_SOLUTION && st->stop) || st->err) return;
  const int ncols = (MODE == SWEEP_SOLUTION) ? st->k : j + 1;
  if (ncols <= 0) {
    return;
  }
  extern __shared__ __align__(128) unsigned char smem[];
  const bool has_w = (MODE != SWEEP_SOLUTION);
  const size_t vt_bytes = (size_t)ncols * kTile * sizeof(TV);
  const size_t wt_bytes = has_w ? align16((size_t)kTile * sizeof(TW)) : 0;
  const size_t sub_bytes = vt_bytes + wt_bytes;          // one tile inside a stage
  const size_t stage_bytes = (size_t)rb * sub_bytes;
  unsigned char* stages = smem;
  ACC* coef = (ACC*)(smem + (size_t)nstages * stage_bytes);
  ACC* coef2 = coef + kMaxCols;                          // UPDATE: coefficients of the 2nd pass
  ACC* wst = (ACC*)((unsigned char*)coef + align16((size_t)2 * kMaxCols * sizeof(ACC)));   // PASS2: w'
  const int rbw = (MODE == SWEEP_PASS2) ? rb : 0;
  uint64_t* bar = (uint64_t*)((unsigned char*)wst + align16((size_t)rbw * kTile * sizeof(ACC)));
  __shared__ ACC red[kWarps];
  __shared__ int flag;

  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  for (int i = t; i < ncols && MODE != SWEEP_PROJ; i += kThreads) {
    if (MODE == SWEEP_DC_UPDATE) {
      if (i < j) {
        coef[i] = (ACC)K.ca[i];
        coef2[i] = (ACC)K.cb[i];
      }
    } else if (MODE == SWEEP_PASS2) {
      coef[i] = (ACC)(K.s[i] * K.h1[i]);
    } else if (MODE == SWEEP_UPDATE) {
      if constexpr (kTwoPassUpdate<ACC>) {
        coef[i] = (ACC)(K.s[i] * K.h1[i]);
        coef2[i] = (ACC)(K.s[i] * K.h2[i]);
      } else {
        coef[i] = (ACC)(K.s[i] * (K.h1[i] + K.h2[i]));
      }
    } else {
      coef[i] = (ACC)K.c[i];
    }
  }
  const ACC cbj = (MODE == SWEEP_DC_UPDATE) ? (ACC)K.cb[j] : ACC(0);
  // FP16 basis: the new column is stored times sig = sqrt(n / ||w||^2), so its entries are O(1)
  // whatever ||w|| is (||w''|| <= ||w||); the lazy scale absorbs sig.  Other types store w''.
  double sig = 1.0;
  if constexpr (is_half_v<TV> && MODE == SWEEP_UPDATE) {
    const double az2 = st->az2;
    if (az2 > 0.0 && isfinite(az2)) sig = sqrt((double)n / az2);
  }
  if (t == 0) {
    for (int s = 0; s < nstages; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();

  const int ntiles = (n + kTile - 1) / kTile;
  const int ngroups = (ntiles + rb - 1) / rb;
  const int G = gridDim.x;
  const int my_groups = blockIdx.x < ngroups ? (ngroups - 1 - blockIdx.x) / G + 1 : 0;
  auto tiles_in = [&](int grp) { return min(rb, ntiles - grp * rb); };
  // CTA b takes groups b, b + G, ... counted from the first group or (rev) from the last one
  auto group_of = [&](int it) { const int g = blockIdx.x + it * G; return rev ? ngroups - 1 - g : g; };
  // test hook: the first stage of CTA 0 in step 0's PASS2 sweep is never filled
  const bool expire = MODE == SWEEP_PASS2 && j == 0 && blockIdx.x == 0 && st->expire_wait;
  // the last kL2KeepBytes of the traversal are loaded at normal priority, the rest evict-first
  const long keep_groups = (long)(kL2KeepBytes / ((size_t)rb * sub_bytes)) + 1;
  const uint64_t pol = l2_evict_first_policy();
  auto issue = [&](int it) {   // warp 0: lane q copies tile q of the group
    const int s = it % nstages;
    const int grp = group_of(it);
    const int nt = tiles_in(grp);
    const bool keep = blockIdx.x + (long)it * G >= ngroups - keep_groups;
    if (expire && it == 0) return;
    unsigned char* stp = stages + (size_t)s * stage_bytes;
    // No proxy fence here: the stage was only read (generic loads, ordered by the CTA barrier)
    // since its last fill.
    if (lane == 0)
      mbar_arrive_expect_tx(&bar[s], (uint32_t)nt * (uint32_t)(vt_bytes + (has_w ? kTile * sizeof(TW) : 0)));
    __syncwarp();
    if (lane < nt) {
      const long tile = (long)grp * rb + lane;
      unsigned char* dst = stp + (size_t)lane * sub_bytes;
      if (keep) {
        bulk_g2s(dst, V + (size_t)tile * vts, (uint32_t)vt_bytes, &bar[s]);
        if (has_w) bulk_g2s(dst + vt_bytes, w + tile * kTile, kTile * sizeof(TW), &bar[s]);
      } else {
        bulk_g2s_hint(dst, V + (size_t)tile * vts, (uint32_t)vt_bytes, &bar[s], pol);
        if (has_w)
          bulk_g2s_hint(dst + vt_bytes, w + tile * kTile, kTile * sizeof(TW), &bar[s], pol);
      }
    }
  };
  if (wid == 0) {
    const int pro = min(nstages, my_groups);
    for (int it = 0; it < pro; ++it) issue(it);
  }

  ACC acc[kColsPerWarp];
#pragma unroll
  for (int c = 0; c < kColsPerWarp; ++c) acc[c] = 0;
  ACC nrm2 = 0;
  int failed_it = -1;
  for (int it = 0; it < my_groups; ++it) {
    const int s = it % nstages;
    const uint32_t par = (uint32_t)((it / nstages) & 1);
    const int grp = group_of(it);
    const int nt = tiles_in(grp);
    const bool ok = mbar_wait(&bar[s], par);
    if (!__syncthreads_and(ok)) {
      failed_it = it;
      break;
    }
    if (MODE == SWEEP_PROJ) {
      // first CGS pass: h1 partials against w, and ||w||^2 (for the breakdown test)
      for (int q = 0; q < nt; ++q) {
        unsigned char* sub = stages + (size_t)s * stage_bytes + (size_t)q * sub_bytes;
        ACC wr[4];
        load4((const TW*)(sub + vt_bytes) + 4 * lane, wr);
        if (wid == 0) nrm2 += wr[0] * wr[0] + wr[1] * wr[1] + wr[2] * wr[2] + wr[3] * wr[3];
        project_tile<ACC, TV>((const TV*)sub, wr, ncols, acc);
      }
      __syncthreads();     // the stage is free
      if (wid == 0 && it + nstages < my_groups) issue(it + nstages);
      continue;
    }
    // Row-owner update: threads 0..127 take the even tiles of the stage, 128..255 the odd
    // ones, one row each; every row's sum over the columns stays in its thread.
    const int r = t & (kTile - 1);
    for (int q = t >> 7; q < nt; q += 2) {
      const long tile = (long)grp * rb + q;
      const long row = tile * kTile + r;
      unsigned char* sub = stages + (size_t)s * stage_bytes + (size_t)q * sub_bytes;
      const TV* v_s = (const TV*)sub;
      double xold = 0.0;
      if (MODE == SWEEP_SOLUTION && x64) xold = x64[row];   // padded, in bounds
      if (MODE == SWEEP_DC_UPDATE) {
        // column j: V_j = U_j - sum_{i<j} V_i ca_i; column j + 1: U_{j+1} = x - sum V_i cb_i - V_j cb_j
        ACC sa = 0, sb = 0;
        if (j > 0) row_update2<ACC, TV>(v_s, coef, coef2, j, r, sa, sb);
        const ACC uj = cv<ACC>(v_s[(size_t)j * kTile + r]);
        const TV vq = cv<TV>(uj - sa);
        if (j > 0) vout[(size_t)tile * vts + r - kTile] = vq;
        const ACC xv = cv<ACC>(((const TW*)(sub + vt_bytes))[r]);
        vout[(size_t)tile * vts + r] = cv<TV>((xv - sb) - cv<ACC>(vq) * cbj);
      } else if (MODE == SWEEP_PASS2) {
        const ACC sum = row_update<ACC, TV>(v_s, coef, ncols, r);
        wst[q * kTile + r] = cv<ACC>(((const TW*)(sub + vt_bytes))[r]) - sum;   // w' = w - V (s h1)
      } else if (MODE == SWEEP_UPDATE) {
        // v_{j+1} = w'' stored unscaled; padded rows stay zero
        const ACC wv = cv<ACC>(((const TW*)(sub + vt_bytes))[r]);
        ACC w2;
        if constexpr (kTwoPassUpdate<ACC>) {
          ACC sum1, sum2;
          row_update2<ACC, TV>(v_s, coef, coef2, ncols, r, sum1, sum2);
          w2 = (wv - sum1) - sum2;                    // w' = w - V (s h1), w'' = w' - V (s h2)
        } else {
          w2 = wv - row_update<ACC, TV>(v_s, coef, ncols, r);
        }
        const TV qv = is_half_v<TV> ? cv<TV>(w2 * (ACC)sig) : cv<TV>(w2);
        vout[(size_t)tile * vts + r] = qv;
        const ACC qa = cv<ACC>(qv);
        nrm2 += qa * qa;
      } else {
        const ACC sum = row_update<ACC, TV>(v_s, coef, ncols, r);
        if (x64) {
          // x += V (s y); padded rows add zero.  Single-precision GMRES keeps x in FP32.
          x64[row] = st->fp32_outer ? (double)((float)xold + (float)sum) : xold + (double)sum;
        } else {
          zout[row] = cv<TZ>(sum);
        }
      }
    }
    if (MODE == SWEEP_PASS2) {
      __syncthreads();   // w' of every tile of the stage
      for (int q = 0; q < nt; ++q) {
        ACC wr[4];
        load4(wst + (size_t)q * kTile + 4 * lane, wr);
        project_tile<ACC, TV>((const TV*)(stages + (size_t)s * stage_bytes + (size_t)q * sub_bytes),
                              wr, ncols, acc);   // h2 partials against w'
      }
    }
    __syncthreads();     // the stage is free
    if (wid == 0 && it + nstages < my_groups) issue(it + nstages);
  }
  if (failed_it >= 0 && t == 0) {
    // A wait ran out.  The copies of groups failed_it .. failed_it + nstages - 1 were issued and
    // may still be landing in this CTA's shared memory: wait for each (bounded) before the
    // barriers are invalidated, then flag the cycle (the host reports GMRES_TIMEOUT and every
    // later kernel of the cycle returns at once).  The CTA still takes part in the cross-CTA
    // sums below (with meaningless partials), so the arrival counters stay consistent.
    drain_stages(bar, nstages, failed_it, my_groups);
    atomicExch(&st->err, 1);
  }
  __syncthreads();
  if (t == 0)
    for (int s = 0; s < nstages; ++s) mbar_inval(&bar[s]);

  if (MODE == SWEEP_SOLUTION || MODE == SWEEP_DC_UPDATE) return;
  if (MODE == SWEEP_PASS2 || MODE == SWEEP_PROJ) store_proj_partials(K.part, K.gs, ncols, acc);
  if (MODE != SWEEP_PASS2) {
    const ACC nb = block_sum(nrm2, red);
    const int slot = MODE == SWEEP_PROJ ? kMaxCols : kMaxCols + 1;
    if (t == 0) K.part[(size_t)slot * K.gs + blockIdx.x] = (double)nb;
  }
  if (MODE == SWEEP_PROJ) {
    proj_cross_cta(K, ncols, &flag);
    return;
  }
  const int cnt_id = (MODE == SWEEP_PASS2) ? CNT_B : CNT_C;
  if (MODE == SWEEP_PASS2) {
    // two-level sum: group leaders, then the last group
    const int nslots = ncols;
    const int grp = blockIdx.x / kGroup, ngrp = (G + kGroup - 1) / kGroup;
    const int b0 = grp * kGroup, gsize = min(kGroup, G - b0);
    unsigned* gc = K.gcnt + (size_t)cnt_id * K.gs2 + grp;
    if (!arrive_last_of(gc, (unsigned)gsize, &flag)) return;
    group_sums(K.part, K.gs, b0, gsize, nslots, ncols, kMaxCols, K.part2, K.gs2, grp);
    if (t == 0) *gc = 0;
    if (!arrive_last_of(&st->cnt[cnt_id], (unsigned)ngrp, &flag)) return;
    final_sums(K.part2, K.gs2, ngrp, nslots, ncols, kMaxCols, K.s, K.h2, &st->az2);
    if (t == 0) st->cnt[cnt_id] = 0;
    return;
  }
  if (!arrive_last(&st->cnt[cnt_id], &flag)) return;
  // ---- SWEEP_UPDATE, last CTA: Hessenberg column j, Givens rotation, stop tests ----
  // Warp 0 stages the column and the earlier rotations in shared memory with independent loads,
  // lane 0 runs the rotation chain there, and the warp writes the rotated column back.
  if constexpr (MODE == SWEEP_UPDATE) {
    __shared__ double col[kMaxCols + 2], rc[kMaxCols], rs[kMaxCols];
    if (t >= 32) return;
    // everything the rotation needs is requested before the norm's sum, so the loads overlap
    const int m1 = K.m + 1;
    double* Hc = K.H + (size_t)j * m1;
    double* Rc = K.R + (size_t)j * m1;
    for (int i = lane; i <= j; i += 32) col[i] = K.h1[i] + K.h2[i];
    for (int i = lane; i < j; i += 32) {
      rc[i] = K.cs[i];
      rs[i] = K.sn[i];
    }
    const double gj = K.g[j];
    const double uround = st->uround, az2 = st->az2, tol = st->tol, bnorm = st->bnorm;
    const double inner_tol = st->inner_tol, gamma = st->gamma;
    const int implicit_fp64 = st->implicit_fp64, jmax = st->jmax;
    const double nrm2_tot = reduce_slot(K.part, K.gs, G, kMaxCols + 1);
    const double qn = sqrt(nrm2_tot);   // norm of the stored column (sig times ||w''||)
    const double hn = qn / sig;
    __syncwarp();
    for (int i = lane; i <= j; i += 32) Hc[i] = col[i];
    __syncwarp();
    // the earlier rotations, applied by the warp as a scan (a short dependent FP64 chain)
    const double x = givens_apply_warp(col, rc, rs, j);
    if (lane == 0) {
      Hc[j + 1] = hn;
      const double a = x, bb = hn;
      const double r = givens_radius(a, bb);
      double c = 1.0, sgn = 0.0;
      if (r != 0.0) {
        const double ir = 1.0 / r;
        c = a * ir;
        sgn = bb * ir;
      }
      K.cs[j] = c;
      K.sn[j] = sgn;
      col[j] = r;
      col[j + 1] = 0.0;
      K.g[j + 1] = -sgn * gj;
      K.g[j] = c * gj;
      const double imp = fabs(sgn * gj);
      st->implicit = imp;
      st->k = j + 1;
      K.s[j + 1] = 1.0 / qn;
      int reason = 0;
      if (!finite_d(hn) || !finite_d(imp) || !finite_d(r)) {
        reason = 3;
        st->nan = 1;
      } else if (hn <= 10.0 * uround * sqrt(az2)) {
        reason = 2;
        st->breakdowns += 1;
      } else {
        const double thr = implicit_fp64 ? tol * bnorm : inner_tol * gamma;
        if (imp <= thr) reason = 1;
        else if (j + 1 >= jmax) reason = 4;
      }
      if (reason) {
        st->reason = reason;
        st->stop = 1;
      }
      st->cnt[cnt_id] = 0;
    }
    __syncwarp();
    for (int i = lane; i <= j + 1; i += 32) Rc[i] = col[i];
  }
}

// ------------------------------------------------------------------------------------------------
// Cycle end: back substitution R y = g (one warp), c_i = s_i y_i
// ------------------------------------------------------------------------------------------------
// The CTA first stages the k columns of R (k (m+1) doubles, dynamic shared memory sized for the
// workspace's m) in one coalesced pass, so the warp's serial chain reads no global memory.
static __global__ void __launch_bounds__(kThreads) k_solve(Krylov K) {
  extern __shared__ double Rs[];   // column i of R at Rs[i (m+1) ..]
  CycleState* st = K.st;
  const int k = st->k;
  const int l = threadIdx.x;
  const int m1 = K.m + 1;
  __shared__ double gsh[kMaxCols + 1];
  for (long e = l; e < (long)k * m1; e += blockDim.x) Rs[e] = K.R[e];
  for (int i = l; i < k; i += blockDim.x) gsh[i] = K.g[i];
  __syncthreads();
  if (l >= 32) return;
  // column-oriented: y_i = g_i / R_ii, then g_r -= R_ri y_i for r < i
  for (int i = k - 1; i >= 0; --i) {
    const double yi = gsh[i] / Rs[(size_t)i * m1 + i];
    __syncwarp();
    for (int r = l; r < i; r += 32) gsh[r] -= Rs[(size_t)i * m1 + r] * yi;
    if (l == 0) K.c[i] = K.s[i] * yi;
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------------
// Residual: r = b - A x in FP64; V[:,0] = TV(r); ||r||, ||TV(r)||; last CTA sets up the cycle
// ------------------------------------------------------------------------------------------------
// TR: arithmetic of the residual (double; float for single-precision GMRES, whose b and x hold
// FP32 values).
// FP16 basis: r is staged in FP32 (rs) and scaled into FP16 by k_v0_half once ||r|| is known.
template <typename TV, typename TR = double> struct EpiResidual {
  const double* __restrict__ b;
  TV* __restrict__ v0;   // basis column 0 (tile-blocked, tile stride vts)
  float* __restrict__ rs;
  long vts;
  TR bval;
  double r2, q2;
  __device__ void prefetch(int row) { bval = (TR)b[row]; }
  __device__ void apply(int row, TR ax) {
    const double r = (double)(TR)(bval - ax);
    r2 += r * r;
    if constexpr (is_half_v<TV>) {
      rs[row] = (float)r;
    } else {
      const TV q = cv<TV>(r);
      v0[(size_t)(row >> kTileShift) * vts + (row & (kTile - 1))] = q;
      const double qd = cv<double>(q);
      q2 += qd * qd;
    }
  }
};

template <typename TV, typename TR = double>
__global__ void __launch_bounds__(kThreads)
    k_residual(Csr<TR> A, const double* __restrict__ x, const double* __restrict__ b,
               TV* __restrict__ v0, long vts, Krylov K, int first, float* __restrict__ rs) {
  CycleState* st = K.st;
  EpiResidual<TV, TR> epi{b, v0, rs, vts, TR(0), 0.0, 0.0};
  spmv_rows<TR, double, TR>(A, VRef<double>{x, kTile}, epi);
  __shared__ double red[kWarps];
  __shared__ int flag;
  const double r2 = block_sum(epi.r2, red);
  const double q2 = block_sum(epi.q2, red);
  if (threadIdx.x == 0) {
    K.part[(size_t)(kMaxCols + 2) * K.gs + blockIdx.x] = r2;
    K.part[(size_t)(kMaxCols + 3) * K.gs + blockIdx.x] = q2;
  }
  if (!arrive_last(&st->cnt[CNT_R], &flag)) return;
  double r2t = 0.0, q2t = 0.0;
  if (threadIdx.x < 32) {
    r2t = reduce_slot(K.part, K.gs, gridDim.x, kMaxCols + 2);
    q2t = reduce_slot(K.part, K.gs, gridDim.x, kMaxCols + 3);
  }
  if (threadIdx.x == 0) {
    const double rel = sqrt(r2t) / st->bnorm;
    // FP16 basis: ||r|| for now; k_v0_half replaces it with the stored vector's norm
    const double gam = is_half_v<TV> ? sqrt(r2t) : sqrt(q2t);
    // bookkeeping of the cycle that just ended
    if (!first) {
      st->last_k = st->k;
      st->last_reason = st->reason;
      st->last_implicit = st->implicit;
      if (st->implicit_fp64 && st->reason == 1 && !(rel <= st->tol)) st->loa += 1;
    }
    st->rel_res = rel;
    st->gamma = gam;
    st->converged = (rel <= st->tol) ? 1 : 0;
    if (!finite_d(rel) || !finite_d(gam)) st->nan = 1;
    K.s[0] = 1.0 / gam;
    K.g[0] = gam;
    st->k = 0;
    st->reason = 0;
    st->implicit = gam;
    st->stop = (st->converged || st->nan || gam == 0.0) ? 1 : 0;
    st->cnt[CNT_R] = 0;
  }
}

// FP16 basis, cycle start: V0 = fp16(c r) with c = sqrt(n) / ||r|| (entries O(1)), and the
// cycle's scalars from the stored vector: s_0 = 1 / ||V0||, gamma = g_0 = ||V0|| / c, so the inner
// problem's right-hand side is V0 / c exactly.
static __global__ void __launch_bounds__(kThreads)
    k_v0_half(int n, const float* __restrict__ rs, __half* __restrict__ v0, long vts, Krylov K) {
  CycleState* st = K.st;
  if (st->stop) return;
  const double gr = st->gamma;
  const double c = (gr > 0.0 && isfinite(gr)) ? sqrt((double)n) / gr : 1.0;
  double q2 = 0.0;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x) {
    const __half q = __float2half_rn((float)(c * (double)rs[r]));
    v0[(size_t)(r >> kTileShift) * vts + (r & (kTile - 1))] = q;
    const double qd = (double)__half2float(q);
    q2 += qd * qd;
  }
  __shared__ double red[kWarps];
  __shared__ int flag;
  const double q2b = block_sum(q2, red);
  if (threadIdx.x == 0) K.part[(size_t)(kMaxCols + 3) * K.gs + blockIdx.x] = q2b;
  if (!arrive_last(&st->cnt[CNT_U], &flag)) return;
  double q2t = 0.0;
  if (threadIdx.x < 32) q2t = reduce_slot(K.part, K.gs, gridDim.x, kMaxCols + 3);
  if (threadIdx.x == 0) {
    const double sq = sqrt(q2t);
    const double gam = sq / c;
    K.s[0] = 1.0 / sq;
    K.g[0] = gam;
    st->gamma = gam;
    st->implicit = gam;
    if (!finite_d(gam) || !(sq > 0.0)) {
      st->nan = finite_d(gam) ? st->nan : 1;
      st->stop = 1;
    }
    st->cnt[CNT_U] = 0;
  }
}

// ------------------------------------------------------------------------------------------------
// Polynomial preconditioner step: t = A x;  Pn = cp_p P + cp_x x + cp_t t;
// Y = cy_y Y + cy_p P + cy_x x + cy_t t + cy_n Pn.  (One SpMV of p(A) = sum_k pi_{k-1}(A)/theta_k.)
// ------------------------------------------------------------------------------------------------
struct PolyCoef {
  double cp_p, cp_x, cp_t;
  double cy_y, cy_p, cy_x, cy_t, cy_n;
  int write_p, write_y, read_y;
};

// The coefficients in the step's arithmetic precision, rounded once on the host, so that the
// kernel's multiply-adds take them straight from the parameter bank.
template <typename ACC> struct PolyCoefT {
  ACC cp_p, cp_x, cp_t;
  ACC cy_y, cy_p, cy_x, cy_t, cy_n;
  int write_p, write_y, read_y;
  static PolyCoefT of(const PolyCoef& c) {
    return {(ACC)c.cp_p, (ACC)c.cp_x, (ACC)c.cp_t, (ACC)c.cy_y, (ACC)c.cy_p, (ACC)c.cy_x,
            (ACC)c.cy_t, (ACC)c.cy_n, c.write_p, c.write_y, c.read_y};
  }
};

template <typename ACC, typename TX, typename TP> struct EpiPoly {
  VRef<TX> x;
  VRef<TP> P;
  ACC* Pn;
  ACC* Y;
  PolyCoefT<ACC> c;
  ACC xr, pr, yr;
  __device__ void prefetch(int row) {
    xr = cv<ACC>(x[row]);
    pr = cv<ACC>(P[row]);
    yr = c.read_y ? Y[row] : ACC(0);
  }
  __device__ void apply(int row, ACC t) {
    const ACC pn = c.cp_p * pr + c.cp_x * xr + c.cp_t * t;
    if (c.write_p) Pn[row] = pn;
    if (c.write_y) Y[row] = c.cy_y * yr + c.cy_p * pr + c.cy_x * xr + c.cy_t * t + c.cy_n * pn;
  }
};

// gate: 0 always run; 1 skip when the cycle has stopped (steps inside the cycle); 2 skip when
// the finished cycle took no step (the cycle-end application to V y).
template <typename TA, typename TX, typename TP, typename ACC>
__global__ void __launch_bounds__(kThreads)
    k_poly_step(Csr<TA> A, VRef<TX> x, VRef<TP> P, ACC* Pn, ACC* Y, PolyCoefT<ACC> c,
                const CycleState* st, int gate, int rev) {
  if (gate != 0 && st->err) return;
  if (gate == 1 && st->stop) return;
  if (gate == 2 && st->k <= 0) return;
  EpiPoly<ACC, TX, TP> epi{x, P, Pn, Y, c, ACC(0), ACC(0), ACC(0)};
  // two rows per thread in every precision (measured faster for this epilogue in FP64 too)
  spmv_rows<TA, TX, ACC, EpiPoly<ACC, TX, TP>, 2>(A, x, epi, rev);
}

// ------------------------------------------------------------------------------------------------
// Block Jacobi preconditioner (Section III-D): z[I_b] = B_b^{-1} x[I_b] for the index sets
// I_b = idx[b k .. b k + k) of the RCM order.  One warp per block (k <= 64): lanes hold the block's
// x entries (rows l and l + 32), the inverse is read column by column (column-major, coalesced
// over the lanes) and each lane writes its rows of z.  The gate is that of k_poly_step.
// ------------------------------------------------------------------------------------------------
template <typename TX, typename TZ, typename TM>
__global__ void __launch_bounds__(kThreads)
    k_bjacobi(VRef<TX> x, TZ* __restrict__ z, const int* __restrict__ idx,
              const TM* __restrict__ inv, int k, int n, int nblocks, const CycleState* st,
              int gate) {
  if (gate != 0 && st->err) return;
  if (gate == 1 && st->stop) return;
  if (gate == 2 && st->k <= 0) return;
  const int lane = threadIdx.x & 31;
  const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (b >= nblocks) return;
  const long base = (long)b * k;
  const int kb = min(k, (int)(n - base));
  const int r0 = lane < kb ? idx[base + lane] : 0;
  const int r1 = lane + 32 < kb ? idx[base + lane + 32] : 0;
  const TM x0 = lane < kb ? cv<TM>(x[r0]) : TM(0);
  const TM x1 = lane + 32 < kb ? cv<TM>(x[r1]) : TM(0);
  const TM* M = inv + base * k;
  TM y0 = 0, y1 = 0;
  for (int c = 0; c < kb; ++c) {
    const TM xc = __shfl_sync(0xffffffffu, c < 32 ? x0 : x1, c & 31);
    const TM* mc = M + (size_t)c * k;
    if (lane < kb) y0 += mc[lane] * xc;
    if (lane + 32 < kb) y1 += mc[lane + 32] * xc;
  }
  if (lane < kb) z[r0] = cv<TZ>(y0);
  if (lane + 32 < kb) z[r1] = cv<TZ>(y1);
}

// Block size 1: z = x / diag(A), elementwise (dinv = 1 / a_ii).
template <typename TX, typename TZ, typename TM>
__global__ void __launch_bounds__(kThreads)
    k_diag_scale(VRef<TX> x, TZ* __restrict__ z, const TM* __restrict__ dinv, int n,
                 const CycleState* st, int gate) {
  if (gate != 0 && st->err) return;
  if (gate == 1 && st->stop) return;
  if (gate == 2 && st->k <= 0) return;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x)
    z[r] = cv<TZ>(dinv[r] * cv<TM>(x[r]));
}

// y = A x (plain, for the building-block entry point)
template <typename TA, typename TX, typename ACC>
__global__ void __launch_bounds__(kThreads) k_spmv(Csr<TA> A, VRef<TX> x, ACC* __restrict__ y) {
  struct Epi {
    ACC* y;
    __device__ void prefetch(int) {}
    __device__ void apply(int row, ACC ax) { y[row] = ax; }
  } epi{y};
  spmv_rows<TA, TX, ACC>(A, x, epi);
}

// ------------------------------------------------------------------------------------------------
// Small element-wise kernels (setup and cycle end)
// ------------------------------------------------------------------------------------------------
// Sliced copy (SELL-32) of the FP32 matrix, one thread per row of the padded slices: entry k of
// row r goes to sptr[r / 32] + 32 k + r % 32; entries past the row's end get column -1, value 0.
static __global__ void k_build_sell(int n, long nrows_pad, const int* __restrict__ rowptr,
                                    const int* __restrict__ col, const float* __restrict__ val,
                                    const int* __restrict__ sptr, int* __restrict__ scol,
                                    float* __restrict__ sval) {
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < nrows_pad;
       r += (long)gridDim.x * blockDim.x) {
    const int p = sptr[r >> 5], w = (sptr[(r >> 5) + 1] - p) >> 5;
    const int a = r < n ? rowptr[r] : 0, len = r < n ? rowptr[r + 1] - a : 0;
    for (int k = 0; k < w; ++k) {
      const long idx = (long)p + 32L * k + (r & 31);
      scol[idx] = k < len ? col[a + k] : -1;
      sval[idx] = k < len ? val[a + k] : 0.0f;
    }
  }
}

static __global__ void k_cast_f64_f32(const double* __restrict__ a, float* __restrict__ b, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];   // round to nearest even
}

template <typename TZ>
__global__ void k_axpy_x(double* __restrict__ x, const TZ* __restrict__ z, int n,
                         const CycleState* st) {
  if (st && st->k <= 0) return;
  const bool f32 = st && st->fp32_outer;   // single-precision GMRES keeps x in FP32
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    x[i] = f32 ? (double)((float)x[i] + cv<float>(z[i])) : x[i] + cv<double>(z[i]);
}

template <typename TV>
__global__ void k_basis_export(const TV* __restrict__ V, long vts, const double* __restrict__ s,
                               int ncols, int n, double* __restrict__ out) {
  const int i = blockIdx.y;
  if (i >= ncols) return;
  const double sc = s[i];
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < n; r += (long)gridDim.x * blockDim.x)
    out[(size_t)i * n + r] =
        sc * cv<double>(V[(size_t)(r >> kTileShift) * vts + (size_t)i * kTile + (r & (kTile - 1))]);
}

// ||a||_2 in FP64 into st->bnorm (per-CTA partials, last CTA reduces in fixed order)
static __global__ void __launch_bounds__(kThreads) k_bnorm(const double* __restrict__ a, int n, Krylov K) {
  double s = 0.0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    s += a[i] * a[i];
  __shared__ double red[kWarps];
  __shared__ int flag;
  s = block_sum(s, red);
  if (threadIdx.x == 0) K.part[(size_t)(kMaxCols + 2) * K.gs + blockIdx.x] = s;
  if (!arrive_last(&K.st->cnt[CNT_MISC], &flag)) return;
  if (threadIdx.x < 32) {
    const double t = reduce_slot(K.part, K.gs, gridDim.x, kMaxCols + 2);
    if (threadIdx.x == 0) {
      K.st->bnorm = sqrt(t);
      K.st->cnt[CNT_MISC] = 0;
    }
  }
}

// a[i] = (double)(float)a[i]: the right-hand side of single-precision GMRES.
static __global__ void k_round_f32(double* __restrict__ a, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    a[i] = (double)(float)a[i];
}

static __global__ void k_copy_f64(const double* __restrict__ a, double* __restrict__ b, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x)
    b[i] = a[i];
}

}  // namespace gmresb3
