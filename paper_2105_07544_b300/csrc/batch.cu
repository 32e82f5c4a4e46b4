// Batched block GMRES-IR: many independent sparse systems, p = 8 right-hand sides each.
//
// The method is the paper's GMRES-IR (Algorithm 2) applied to a block of right-hand sides: an
// FP64 residual R = B - A X and update X += U, and an inner block GMRES(m) cycle in FP32 whose
// Krylov basis is stored in BF16.  The inner cycle is Algorithm 1 with blocks of p vectors: block
// classical Gram-Schmidt run twice (Section III-A's CGS2, where V^T W is now a dense product),
// each new block orthonormalised by a Cholesky QR, and the block least-squares problem solved by
// Householder reflectors updated step by step (one per column of the band Hessenberg matrix).
//
// B300 layout: the systems form one block-diagonal matrix whose blocks are padded to 128-row
// tiles, so one row-per-thread SpMM serves all systems; the basis is tile-blocked
// ([tile][block][128 rows][8]) so a tile's first j blocks are one contiguous bulk copy; the
// products V^T W and V C run on the tensor cores (mma.sync m16n8k16, BF16 in, FP32 accumulate,
// N = 8 = the number of right-hand sides), W and the coefficients split into BF16 high and low
// parts so that the products keep about 16 bits; per-system sums are per-chunk partials reduced
// by one CTA per system in a fixed order.  Orthonormalisation is lazy: the stored block U_k and
// an 8 x 8 transform T_k with Q_k = U_k T_k.  One block cycle of all systems is one CUDA graph.
#include <cuda_runtime.h>
#include <cuda_bf16.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <functional>
#include <memory>
#include <new>
#include <vector>

#include "../../include/gmresb3.h"
#include "kernels.cuh"

using namespace gmresb3;
typedef __nv_bfloat16 bf16;

namespace gmresb3 {
namespace batch {

constexpr int kP = 8;                        // right-hand sides per system
constexpr int kBlk = kTile * kP;             // elements of one (tile, block) of the basis
constexpr int kMaxSteps = 32;                // block steps per cycle
constexpr int kChunkTiles = 16;              // default tiles per chunk of a sweep
constexpr int kSweepSmemKb = 64;             // default sweep pipeline budget (three CTAs per SM)
constexpr int kSweepStages = 3;              // default cap on sweep pipeline stages
constexpr int kMaxMt = 3;                    // 16-column M-tiles per warp (48 blocks)
constexpr int kMaxBlocks = kMaxSteps + 1;
// SysState.breakdowns is set to this when a sweep's bounded wait for a bulk copy ran out.
constexpr int kTimeoutMark = 1 << 20;

// Per-system state (device).
struct SysState {
  int k;           // block steps completed in this cycle
  int stop;        // this system's cycle has ended (step limit or breakdown)
  int done;        // converged: every column's relative residual <= tol
  int breakdowns;
  int cycles;      // cycles run
  int iters;       // block steps run
  int first;       // 1 until the first residual has set bnorm
  int pc0, pc1;    // chunk range of this cycle (coarse or fine list, chosen by kb_compact)
  int pad;
  double bn[kP];   // ||b_c||
  double rel[kP];  // explicit relative residuals
  float D[kP];     // column norms of R (scaling of the first block)
  float imp[kP];   // implicit residual norms of the inner problem
};

struct SysDesc {
  int row0;        // first global (padded) row
  int n;           // rows
  int t0, t1;      // tile range
  int c0, c1;      // chunk range in the coarse list
  int f0, f1;      // chunk range in the fine list (after the coarse list in the same array)
};

struct Chunk {
  int sys, t0, t1;
};

// Pointers of the per-system small arrays (all offsets by system inside the kernels).
struct Small {
  float* T;        // [sys][kMaxBlocks][64]   transform of block i (Q_i = U_i T_i)
  float* H1;       // [sys][kMaxBlocks][64]   first-pass coefficients
  float* R;        // [sys][(m+1)8 x m8] column-major, triangularised block Hessenberg
  float* rc;       // [sys][m8][8]            reflector of column c: v_1 .. v_8 (v_0 = 1)
  float* rs;       // [sys][m8][8]            reflector of column c: tau in entry 0
  float* g;        // [sys][(m+1)8][8]        transformed right-hand side
  float* Z;        // [sys][kMaxBlocks][64]   solution coefficients T_i Y_i
  bf16* Chi;       // [sys][kMaxBlocks][64]   update coefficients (high part)
  bf16* Clo;       // [sys][kMaxBlocks][64]   update coefficients (low part)
  float* part;     // [chunk][kMaxBlocks*64]  per-chunk partial sums
  double* tpart;   // [tile][16]              per-tile partial sums (residual)
  float* tgram;    // [tile][64]              per-tile Gram partials (first block)
  SysState* st;
  const SysDesc* sd;
  int m;
};

// ------------------------------------------------------------------------------------------------
// Tensor-core helpers (legacy mma.sync path)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void ldsm_x4(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t (&r)[4], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(smem_u32(p)));
}
__device__ __forceinline__ void ldsm_x2_t(uint32_t (&r)[2], const void* p) {
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];"
               : "=r"(r[0]), "=r"(r[1])
               : "r"(smem_u32(p)));
}
// D = A (16x16 bf16) * B (16x8 bf16) + D (fp32)
__device__ __forceinline__ void mma_bf16(float (&d)[4], const uint32_t (&a)[4],
                                         const uint32_t (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

__device__ __forceinline__ void split_bf16(float v, bf16& hi, bf16& lo) {
  hi = __float2bfloat16_rn(v);
  lo = __float2bfloat16_rn(v - __bfloat162float(hi));
}

// Column sums of v[0..N) over the 32 lanes of a warp by a transposing butterfly: at each of the
// first log2(N) levels a lane trades half of its columns with its partner and adds the other
// half, so the warp does N - 1 + (5 - log2 N) additions per lane instead of 5 N.  Afterwards lane
// l holds in v[0] the total of column l / (32 / N) (N <= 32), or in v[0], v[1] the totals of
// columns 2l, 2l + 1 (N = 64).  Fixed order: the result does not depend on timing.
template <int C, int M, typename T, int N>
__device__ __forceinline__ void col_sums_level(T (&v)[N], int lane) {
  if constexpr (M >= 1) {
    if constexpr (C > 1) {   // trade the upper or lower half of the C columns held
      constexpr int half = C / 2;
      const bool up = (lane & M) != 0;
#pragma unroll
      for (int q = 0; q < half; ++q) {
        const T send = up ? v[q] : v[q + half];
        const T keep = up ? v[q + half] : v[q];
        v[q] = keep + __shfl_xor_sync(0xffffffffu, send, M);
      }
      col_sums_level<half, M / 2>(v, lane);
    } else {
      v[0] += __shfl_xor_sync(0xffffffffu, v[0], M);
      col_sums_level<1, M / 2>(v, lane);
    }
  }
}
template <int N, typename T> __device__ __forceinline__ void warp_col_sums(T (&v)[N]) {
  static_assert(N >= 1 && N <= 64 && (N & (N - 1)) == 0, "power of two up to 64");
  col_sums_level<N, 16>(v, threadIdx.x & 31);
}

// ------------------------------------------------------------------------------------------------
// Residual: R = B - A X (FP64), R stored in FP32 into W, per-tile partial sums of R^2 and B^2
// ------------------------------------------------------------------------------------------------
// Kernels over rows take the active tile list of the cycle (the tiles of the systems not yet
// converged, built by kb_compact) and stride over it with a persistent grid of 128-thread CTAs,
// so that late cycles with few systems left do not launch and retire a CTA per idle tile.
struct Active {
  const int* tiles;    // [ntiles]  active tiles, system order
  const int* chunks;   // [nchunks] active sweep chunks, system order
  const int* cnt;      // [0] active tiles, [1] active chunks
};

__device__ __forceinline__ void residual_tile(const Csr<double>& A, const double* __restrict__ X,
                                              const double* __restrict__ B, float* __restrict__ W,
                                              int tile, bool first, Small S) {
  const int t = threadIdx.x;
  const long row = (long)tile * kTile + t;
  double r[kP], bb[kP];
  float rf[kP];   // R rounded to FP32 (stored into W, and squared for the norms)
#pragma unroll
  for (int c = 0; c < kP; ++c) {
    r[c] = bb[c] = 0.0;
    rf[c] = 0.f;
  }
  if (row < A.n) {
    const int a = A.rowptr[row], e = A.rowptr[row + 1];
    const double2* br = reinterpret_cast<const double2*>(B + row * kP);
#pragma unroll
    for (int q = 0; q < kP / 2; ++q) {
      const double2 bv = br[q];
      bb[2 * q] = bv.x;
      bb[2 * q + 1] = bv.y;
    }
    double ax[kP];
#pragma unroll
    for (int c = 0; c < kP; ++c) ax[c] = 0.0;
#pragma unroll 4
    for (int p = a; p < e; ++p) {
      const double v = A.val[p];
      const double2* xr = reinterpret_cast<const double2*>(X + (long)A.col[p] * kP);
#pragma unroll
      for (int q = 0; q < kP / 2; ++q) {
        const double2 xv = xr[q];
        ax[2 * q] += v * xv.x;
        ax[2 * q + 1] += v * xv.y;
      }
    }
#pragma unroll
    for (int c = 0; c < kP; ++c) {
      r[c] = bb[c] - ax[c];
      rf[c] = (float)r[c];
    }
    float4* wr = reinterpret_cast<float4*>(W + row * kP);
    wr[0] = make_float4(rf[0], rf[1], rf[2], rf[3]);
    wr[1] = make_float4(rf[4], rf[5], rf[6], rf[7]);
  }
  // Per-tile sums of R^2 (and of B^2 on the first residual, the only one that uses them).  They
  // feed only the convergence test and the column scaling, so FP32 squares of the FP32-rounded
  // entries suffice (relative error ~1e-7) and keep B300's slow FP64 pipe for A X; a tile with an
  // entry outside [2^-60, 2^60] (other than zero), where FP32 squares could underflow or a sum
  // overflow, takes the FP64 squares instead (the same choice in the whole CTA).
  __shared__ double red[kTile / 32][2 * kP];
  const int w = t >> 5, l = t & 31;
  auto safe32 = [](float v) {
    const float a = fabsf(v);
    return a == 0.f || (a >= 0x1p-60f && a <= 0x1p60f);
  };
  float bf[kP];
#pragma unroll
  for (int c = 0; c < kP; ++c) bf[c] = first ? (float)bb[c] : 0.f;
  bool ok = true;
#pragma unroll
  for (int c = 0; c < kP; ++c) ok = ok && safe32(rf[c]) && safe32(bf[c]);
  const bool fast = __syncthreads_and(ok) != 0;
  if (fast) {
    float v[kP];
#pragma unroll
    for (int c = 0; c < kP; ++c) v[c] = rf[c] * rf[c];
    warp_col_sums(v);
    if ((l & 3) == 0) red[w][l >> 2] = (double)v[0];
    if (first) {
#pragma unroll
      for (int c = 0; c < kP; ++c) v[c] = bf[c] * bf[c];
      warp_col_sums(v);
      if ((l & 3) == 0) red[w][kP + (l >> 2)] = (double)v[0];
    }
  } else {
    double v[kP];
#pragma unroll
    for (int c = 0; c < kP; ++c) v[c] = r[c] * r[c];
    warp_col_sums(v);
    if ((l & 3) == 0) red[w][l >> 2] = v[0];
    if (first) {
#pragma unroll
      for (int c = 0; c < kP; ++c) v[c] = bb[c] * bb[c];
      warp_col_sums(v);
      if ((l & 3) == 0) red[w][kP + (l >> 2)] = v[0];
    }
  }
  __syncthreads();
  if (t < (first ? 2 * kP : kP)) {
    double s = 0.0;
    for (int q = 0; q < kTile / 32; ++q) s += red[q][t];
    S.tpart[(size_t)tile * 16 + t] = s;   // [tile][R^2 of 8 columns, B^2 of 8 columns]
  }
  __syncthreads();   // red is reused by the next tile
}

__global__ void __launch_bounds__(kTile)
    kb_residual(Csr<double> A, const double* __restrict__ X, const double* __restrict__ B,
                float* __restrict__ W, const int* __restrict__ tile_sys, Active act, Small S) {
  const int ntl = act.cnt[0];
  for (int i = blockIdx.x; i < ntl; i += gridDim.x) {
    const int tile = act.tiles[i];
    const SysState* st = S.st + tile_sys[tile];
    if (st->done) continue;   // uniform over the CTA
    residual_tile(A, X, B, W, tile, st->first != 0, S);
  }
}

// Active work lists of the next block cycle: the tiles and sweep chunks of the systems not yet
// converged, in system order.  One CTA per system: its offsets are the tile and chunk counts of
// the active systems before it; the last CTA writes the totals.
__global__ void __launch_bounds__(128)
    kb_compact(Small S, int nsys, int fine_below, int* __restrict__ tiles,
               int* __restrict__ chunks, int* __restrict__ cnt) {
  const int s = blockIdx.x, t = threadIdx.x, lane = t & 31, w = t >> 5;
  // tiles before s, coarse chunks before s, fine chunks before s, and the three totals
  int v[6] = {0, 0, 0, 0, 0, 0};
  for (int q = t; q < nsys; q += 128) {
    if (S.st[q].done) continue;
    const SysDesc d = S.sd[q];
    const int nt = d.t1 - d.t0, nc = d.c1 - d.c0, nf = d.f1 - d.f0;
    v[3] += nt;
    v[4] += nc;
    v[5] += nf;
    if (q < s) {
      v[0] += nt;
      v[1] += nc;
      v[2] += nf;
    }
  }
  __shared__ int red[4][6];
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    const int r = warp_sum(v[j]);
    if (lane == 0) red[w][j] = r;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < 6; ++j) v[j] = red[0][j] + red[1][j] + red[2][j] + red[3][j];
  // few tiles left: the fine list gives the sweeps more work items than the coarse one
  const bool fine = v[3] < fine_below;
  if (!S.st[s].done) {
    const SysDesc d = S.sd[s];
    const int a = fine ? d.f0 : d.c0, e = fine ? d.f1 : d.c1, off = fine ? v[2] : v[1];
    for (int i = t; i < d.t1 - d.t0; i += 128) tiles[v[0] + i] = d.t0 + i;
    for (int i = t; i < e - a; i += 128) chunks[off + i] = a + i;
    if (t == 0) {
      S.st[s].pc0 = a;
      S.st[s].pc1 = e;
    }
  }
  if (s == nsys - 1 && t == 0) {
    cnt[0] = v[3];
    cnt[1] = fine ? v[5] : v[4];
  }
}

// One CTA of 256 threads per system: explicit relative residuals, convergence, column scales of
// the next cycle.  Thread (p, slot) sums the p-th sixteenth of the system's tiles (in tile
// order), the sixteen part sums are added in order.
__global__ void __launch_bounds__(256) kb_sys_residual(Small S, double tol) {
  const int sys = blockIdx.x;
  SysState* st = S.st + sys;
  if (st->done) return;
  const SysDesc d = S.sd[sys];
  const int t = threadIdx.x, slot = t & 15, p = t >> 4;
  const int nslot = st->first ? 16 : kP;   // B^2 slots exist on the first residual only
  __shared__ double part[16][16];
  __shared__ double tot[16];
  const int nt = d.t1 - d.t0, per = (nt + 15) / 16;
  const int ta = d.t0 + min(nt, p * per), tb = d.t0 + min(nt, (p + 1) * per);
  double acc = 0.0;
  if (slot < nslot) {
#pragma unroll 4
    for (int tile = ta; tile < tb; ++tile) acc += S.tpart[(size_t)tile * 16 + slot];
  }
  part[p][slot] = acc;
  __syncthreads();
  if (t < 16) {
    double v = part[0][t];
    for (int q = 1; q < 16; ++q) v += part[q][t];
    tot[t] = v;
  }
  __syncthreads();
  if (t < kP) {
    const double s = tot[t];
    if (st->first) st->bn[t] = sqrt(tot[t + kP]);
    const double bn = st->bn[t] > 0.0 ? st->bn[t] : 1.0;
    st->rel[t] = sqrt(s) / bn;
    st->D[t] = (float)sqrt(s);
  }
  __syncthreads();
  if (t == 0) {
    bool all = true;
    for (int c = 0; c < kP; ++c) {
      const double v = st->rel[c];
      if (!(v <= tol)) all = false;
    }
    st->first = 0;
    st->done = all ? 1 : 0;
    st->k = 0;
    st->stop = all ? 1 : 0;
  }
}

// First block: U_0 = bf16(R D^{-1}) into basis block 0, per-tile Gram partials of U_0.
__device__ __forceinline__ void start_tile(const float* __restrict__ W, bf16* __restrict__ U,
                                           long uts, int n, int tile, const SysState* st, Small S) {
  const int t = threadIdx.x;
  const long row = (long)tile * kTile + t;
  float u[kP];
#pragma unroll
  for (int c = 0; c < kP; ++c) {
    const float dc = st->D[c];
    const float v = (row < n && dc > 0.f) ? W[row * kP + c] / dc : 0.f;
    u[c] = __bfloat162float(__float2bfloat16_rn(v));
  }
  bf16* dst = U + (size_t)tile * uts + (size_t)t * kP;
#pragma unroll
  for (int c = 0; c < kP; ++c) dst[c] = __float2bfloat16_rn(u[c]);
  __shared__ float red[kTile / 32][64];
  const int w = t >> 5, l = t & 31;
  float v[64];
#pragma unroll
  for (int ij = 0; ij < 64; ++ij) v[ij] = u[ij >> 3] * u[ij & 7];
  warp_col_sums(v);
  red[w][2 * l] = v[0];
  red[w][2 * l + 1] = v[1];
  __syncthreads();
  if (t < 64) {
    float s = 0.f;
    for (int q = 0; q < kTile / 32; ++q) s += red[q][t];
    S.tgram[(size_t)tile * 64 + t] = s;
  }
  __syncthreads();   // red is reused by the next tile
}

__global__ void __launch_bounds__(kTile)
    kb_start(const float* __restrict__ W, bf16* __restrict__ U, long uts, int n,
             const int* __restrict__ tile_sys, Active act, Small S) {
  const int ntl = act.cnt[0];
  for (int i = blockIdx.x; i < ntl; i += gridDim.x) {
    const int tile = act.tiles[i];
    const SysState* st = S.st + tile_sys[tile];
    if (st->done) continue;   // uniform over the CTA
    start_tile(W, U, uts, n, tile, st, S);
  }
}

// Reciprocal square root of a Cholesky pivot d > 0 in FP64.
__device__ __forceinline__ double rsqrt_pivot(double d) { return rsqrt(d); }

// Shifted Cholesky QR of an 8 x 8 Gram matrix G (double, row-major, shared memory) by lanes 0..7
// of one warp: G = L L^T, T = L^{-T} (row-major float) and Rt = L^T (row-major float).
// Right-looking, in registers: lane i holds row i of G; at pivot j lane j's updated diagonal and
// then the new column L[., j] are broadcast by shuffles, and every lane i > j removes L[i][j]
// L[c][j] from its entries j < c <= i.  Each entry sees the same subtractions in the same order
// as the row-by-row (Cholesky-Banachiewicz) form, so L is the same; only the dependent chain is
// shorter (no shared-memory round trip per term).  One FP64 reciprocal square root per pivot
// gives both l_jj = d_j / sqrt(d_j) and the scaling of column j, so no division sits on the
// chain.  On breakdown the diagonal is shifted once by 11 (n p + p (p + 1)) u |G|_max 8 (shifted
// Cholesky QR) and the factorisation retried.  Returns the success flag in lanes 0..7 (the same
// in each); T and Rt are written only on success.  Ls: 64 doubles of shared scratch.  Called by
// lanes 0..7 only.
__device__ bool cholqr_warp(const double* __restrict__ Gs, double* __restrict__ Ls, long nrows,
                            float* __restrict__ T, float* __restrict__ Rt, double uround) {
  const int i = threadIdx.x & 7;
  bool ok = false;
  double shift = 0.0;
  double l[8], rinv[8];
  for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
    if (attempt == 1) {
      double nrm = 0.0;
      for (int e = 0; e < 64; ++e) nrm = fmax(nrm, fabs(Gs[e]));
      shift = 11.0 * ((double)nrows * kP + kP * (kP + 1)) * uround * nrm * 8.0;
    }
#pragma unroll
    for (int c = 0; c < 8; ++c) l[c] = (c == i) ? Gs[i * 8 + c] + shift : Gs[i * 8 + c];
    ok = true;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const double d = __shfl_sync(0xffu, l[j], j);   // pivot: lane j's updated diagonal
      if (!(d > 0.0)) {                                // the same value in every lane
        ok = false;
        break;
      }
      const double r = rsqrt_pivot(d);
      rinv[j] = r;
      const double lij = (i == j) ? d * r : l[j] * r;  // meaningful for i >= j
      l[j] = lij;
#pragma unroll
      for (int c = j + 1; c < 8; ++c) {
        const double lcj = __shfl_sync(0xffu, lij, c);   // L[c][j] from lane c > j
        if (c <= i) l[c] -= lij * lcj;
      }
    }
  }
  if (!ok) return false;
#pragma unroll
  for (int c = 0; c < 8; ++c) Ls[i * 8 + c] = (c <= i) ? l[c] : 0.0;
  __syncwarp(0xffu);
  // column i of L^{-1}: forward substitution L x = e_i, column by column (x_c is removed from
  // every later row as soon as it is known: the same subtractions, in the same order, as the
  // row-by-row form, with the rows' updates independent of one another)
  double x[8], sv[8];
#pragma unroll
  for (int r = 0; r < 8; ++r) sv[r] = (r == i) ? 1.0 : 0.0;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    x[c] = sv[c] * rinv[c];
#pragma unroll
    for (int r = c + 1; r < 8; ++r) sv[r] -= Ls[r * 8 + c] * x[c];
  }
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    T[i * 8 + r] = (float)x[r];                          // T = (L^{-1})^T: row i is column i of L^{-1}
    Rt[r * 8 + i] = (r <= i) ? (float)l[r] : 0.f;        // Rt = L^T: column i is row i of L
  }
  return true;
}

// One CTA of 512 threads per system: thread (p, e) sums Gram entry e over the p-th eighth of the
// system's tiles (in tile order), the eight part sums are added in order, then warp 0 factors
// the first block (Cholesky QR); B0 = L0^T D is the inner right-hand side.
__global__ void __launch_bounds__(512) kb_sys_start_n(Small S, int nsys) {
  const int sys = blockIdx.x;
  if (sys >= nsys) return;
  SysState* st = S.st + sys;
  if (st->done) return;
  const SysDesc d = S.sd[sys];
  const int t = threadIdx.x, e = t & 63, p = t >> 6;
  const int m = S.m;
  const int ld = (m + 1) * kP;   // rows of R and g
  float* g = S.g + (size_t)sys * ld * kP;
  for (int i = t; i < ld * kP; i += 512) g[i] = 0.f;
  __shared__ double Gp[8][64];
  __shared__ double Gs[64], Ls[64];
  __shared__ float Rt[64];
  __shared__ int s_ok;
  const int nt = d.t1 - d.t0, per = (nt + 7) / 8;
  const int ta = d.t0 + min(nt, p * per), tb = d.t0 + min(nt, (p + 1) * per);
  // compensated (Kahan) FP32 sum of the part's tile partials: FP64-like accuracy for a sum of
  // FP32 terms without warp-wide FP64 adds, which on this part occupy the FP64 pipe for tens of
  // cycles each
  float sum = 0.f, comp = 0.f;
#pragma unroll 8
  for (int tile = ta; tile < tb; ++tile) {
    const float yv = S.tgram[(size_t)tile * 64 + e] - comp;
    const float tv = sum + yv;
    comp = (tv - sum) - yv;
    sum = tv;
  }
  Gp[p][e] = (double)sum - (double)comp;
  __syncthreads();
  if (t < 64) {
    double v = Gp[0][t];
    for (int q = 1; q < 8; ++q) v += Gp[q][t];
    Gs[t] = v;
  }
  __syncthreads();
  if (t < 8) {
    float* T0 = S.T + (size_t)sys * kMaxBlocks * 64;
    const bool ok = cholqr_warp(Gs, Ls, d.n, T0, Rt, ldexp(1.0, -24));
    if (t == 0) s_ok = ok ? 1 : 0;
  }
  __syncthreads();
  if (!s_ok) {
    if (t == 0) {
      st->stop = 1;
      st->breakdowns += 1;
    }
    return;
  }
  // g(0:8, c) = (L^T D)(:, c)
  if (t < 64) g[(size_t)(t >> 3) * kP + (t & 7)] = Rt[t] * st->D[t & 7];
  if (t == 0) {
    st->k = 0;
    st->stop = 0;
  }
}

// ------------------------------------------------------------------------------------------------
// SpMM of step k: W = (A U_k) T_k
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void spmm_row(const Csr<float>& A, const bf16* __restrict__ U, long uts,
                                         int k, float* __restrict__ W, long row, int sys, Small S) {
  const int a = A.rowptr[row], e = A.rowptr[row + 1];
  float y[kP];
#pragma unroll
  for (int c = 0; c < kP; ++c) y[c] = 0.f;
#pragma unroll 4
  for (int p = a; p < e; ++p) {
    const int col = A.col[p];
    const float v = A.val[p];
    const uint4 raw = *reinterpret_cast<const uint4*>(
        U + (size_t)(col >> kTileShift) * uts + (size_t)k * kBlk + (size_t)(col & (kTile - 1)) * kP);
    const bf16* ub = reinterpret_cast<const bf16*>(&raw);
#pragma unroll
    for (int c = 0; c < kP; ++c) y[c] += v * __bfloat162float(ub[c]);
  }
  const float* T = S.T + ((size_t)sys * kMaxBlocks + k) * 64;
  float o[kP];
#pragma unroll
  for (int c = 0; c < kP; ++c) o[c] = 0.f;
#pragma unroll
  for (int i = 0; i < kP; ++i) {
    const float4 t0 = __ldg(reinterpret_cast<const float4*>(T + i * 8));
    const float4 t1 = __ldg(reinterpret_cast<const float4*>(T + i * 8 + 4));
    o[0] += y[i] * t0.x; o[1] += y[i] * t0.y; o[2] += y[i] * t0.z; o[3] += y[i] * t0.w;
    o[4] += y[i] * t1.x; o[5] += y[i] * t1.y; o[6] += y[i] * t1.z; o[7] += y[i] * t1.w;
  }
  float4* wr = reinterpret_cast<float4*>(W + row * kP);
  wr[0] = make_float4(o[0], o[1], o[2], o[3]);
  wr[1] = make_float4(o[4], o[5], o[6], o[7]);
}

__global__ void __launch_bounds__(kTile)
    kb_spmm(Csr<float> A, const bf16* __restrict__ U, long uts, int k, float* __restrict__ W,
            const int* __restrict__ tile_sys, Active act, Small S) {
  const int ntl = act.cnt[0];
  for (int i = blockIdx.x; i < ntl; i += gridDim.x) {
    const int tile = act.tiles[i];
    const int sys = tile_sys[tile];
    const SysState* st = S.st + sys;
    if (st->stop || st->done) continue;
    const long row = (long)tile * kTile + threadIdx.x;
    if (row < A.n) spmm_row(A, U, uts, k, W, row, sys, S);
  }
}

// ------------------------------------------------------------------------------------------------
// Block sweeps over chunks of tiles (tensor cores)
//   PROJ  : P += U_{0..k}^T W
//   PASS2 : W' = W - U C1 ; P += U^T W'
//   UPDATE: W'' = W - U C12 ; U_{k+1} = bf16(W'') ; G += U_{k+1}^T U_{k+1}
//   XUPDATE (cycle end): X += U_{0..m-1} Z  (Z = T Y per block; FP64 X)
// ------------------------------------------------------------------------------------------------
enum { BS_PROJ = 0, BS_PASS2 = 1, BS_UPDATE = 2, BS_XUPDATE = 3 };
static_assert(kMaxSteps * 64 <= 2 * kBlk, "XUPDATE stages Z's middle part in the W staging");

__host__ __device__ constexpr size_t bs_stage_bytes(int nblk) {
  return (size_t)nblk * kBlk * 2 + (size_t)kBlk * 4;   // U blocks (bf16) + W tile (fp32)
}
__host__ __device__ constexpr size_t bs_fixed_bytes() {
  // W hi/lo (bf16), C hi/lo (kMaxBlocks blocks), zero block, Gram/partial staging, bars
  return (size_t)2 * kBlk * 2 + (size_t)2 * kMaxBlocks * 64 * 2 + (size_t)kBlk * 2 +
         (size_t)kWarps * 64 * 4 + kMaxStages * 8 + 64;
}

template <int MODE>
__global__ void __launch_bounds__(kThreads, 2)
    kb_sweep(const bf16* __restrict__ U, bf16* __restrict__ Uw, long uts, int k,
             const float* __restrict__ W, const Chunk* __restrict__ chunks, Active act,
             Small S, int nstages, int rev, double* __restrict__ X) {
  extern __shared__ __align__(128) unsigned char smem[];
  const int nblk = k + 1;                       // basis blocks 0..k
  const size_t stage_bytes = bs_stage_bytes(nblk);
  unsigned char* stages = smem;
  bf16* w_hi = (bf16*)(smem + (size_t)nstages * stage_bytes);
  bf16* w_lo = w_hi + kBlk;
  bf16* c_hi = w_lo + kBlk;
  bf16* c_lo = c_hi + kMaxBlocks * 64;
  bf16* zblk = c_lo + kMaxBlocks * 64;          // a zero block (odd block counts)
  float* gst = (float*)(zblk + kBlk);           // [kWarps][64] Gram staging
  uint64_t* bar = (uint64_t*)(gst + kWarps * 64);
  __shared__ int s_skip;

  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int g8 = lane >> 2, t4 = lane & 3;
  for (int i = t; i < kBlk; i += kThreads) zblk[i] = __float2bfloat16_rn(0.f);
  if (t == 0) {
    for (int s = 0; s < nstages; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  const int nmt = (nblk + 1) / 2;               // 16-column M-tiles of the projection
  int phase_base = 0;                           // uses of each stage so far (for parity)

  const int nact = act.cnt[1];
  const uint64_t pol = l2_evict_first_policy();
  // The cycle's chunks are walked from the first or (rev) from the last one, against the previous
  // sweep, so that a sweep starts on the tiles its predecessor left in L2; the last
  // kL2KeepBytes of the walk are loaded at normal priority, the rest evict-first.  The partial
  // sums are stored by chunk, so their order, and every result, is the same either way.
  for (int ai = blockIdx.x; ai < nact; ai += gridDim.x) {
    const int ci = act.chunks[rev ? nact - 1 - ai : ai];
    const Chunk ch = chunks[ci];
    __syncthreads();   // everyone is done with the previous chunk's s_skip and coefficients
    if (MODE == BS_XUPDATE) {
      // the cycle has ended (stop is set); systems that took no block step add nothing
      const SysState& sst = S.st[ch.sys];
      if (t == 0) s_skip = (sst.done || sst.k <= 0) ? 1 : 0;
      // Z of the blocks the cycle built, split exactly into three bf16 parts (high, middle in
      // the W staging, which this mode does not use, and low: 3 x 8 bits hold an FP32 value, so
      // U Z is the FP32 product up to the order of the sums, whatever cancellation Z carries);
      // the blocks beyond (not built in this cycle: their basis tiles are loaded but must not
      // contribute) are zero
      const int kk = sst.k;
      const size_t off = (size_t)ch.sys * kMaxBlocks * 64;
      bf16* c_md = w_hi;   // nblk * 64 <= kMaxSteps * 64 = 2 kBlk entries
      for (int i = t; i < nblk * 64; i += kThreads) {
        const float z = (i >> 6) < kk ? S.Z[off + i] : 0.f;
        c_hi[i] = __float2bfloat16_rn(z);
        const float r1 = z - __bfloat162float(c_hi[i]);
        c_md[i] = __float2bfloat16_rn(r1);
        c_lo[i] = __float2bfloat16_rn(r1 - __bfloat162float(c_md[i]));
      }
    } else if (t == 0) {
      s_skip = (S.st[ch.sys].stop || S.st[ch.sys].done) ? 1 : 0;
    }
    if (MODE != BS_PROJ && MODE != BS_XUPDATE) {
      // coefficient blocks of this system, bf16 high/low, [block][8 basis][8 rhs]
      const size_t off = (size_t)ch.sys * kMaxBlocks * 64;
      for (int i = t; i < nblk * 64; i += kThreads) {
        c_hi[i] = S.Chi[off + i];
        c_lo[i] = S.Clo[off + i];
      }
    }
    __syncthreads();
    if (s_skip) continue;
    const int ntl = ch.t1 - ch.t0;
    const bool keep = (size_t)(nact - ai) * ntl * stage_bytes <= kL2KeepBytes;
    auto issue = [&](int it) {   // warp 0
      const int s = (phase_base + it) % nstages;
      unsigned char* stp = stages + (size_t)s * stage_bytes;
      const long tile = ch.t0 + it;
      if (lane == 0) {
        const size_t wbytes = (MODE == BS_XUPDATE) ? 0 : (size_t)kBlk * 4;   // XUPDATE: no W
        mbar_arrive_expect_tx(&bar[s], (uint32_t)((size_t)nblk * kBlk * 2 + wbytes));
        if (MODE == BS_XUPDATE) {
          bulk_g2s_hint(stp, U + (size_t)tile * uts, (uint32_t)((size_t)nblk * kBlk * 2), &bar[s],
                        pol);
        } else if (keep) {
          bulk_g2s(stp, U + (size_t)tile * uts, (uint32_t)((size_t)nblk * kBlk * 2), &bar[s]);
          bulk_g2s(stp + (size_t)nblk * kBlk * 2, W + tile * kBlk, (uint32_t)(kBlk * 4), &bar[s]);
        } else {
          bulk_g2s_hint(stp, U + (size_t)tile * uts, (uint32_t)((size_t)nblk * kBlk * 2), &bar[s],
                        pol);
          bulk_g2s_hint(stp + (size_t)nblk * kBlk * 2, W + tile * kBlk, (uint32_t)(kBlk * 4),
                        &bar[s], pol);
        }
      }
    };
    if (wid == 0)
      for (int it = 0; it < min(nstages, ntl); ++it) issue(it);

    float acc[kMaxMt][4];
#pragma unroll
    for (int q = 0; q < kMaxMt; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[q][e] = 0.f;
    float gacc[2] = {0.f, 0.f};
    int failed_it = -1;
    for (int it = 0; it < ntl; ++it) {
      const int use = phase_base + it;
      const int s = use % nstages;
      const uint32_t par = (uint32_t)((use / nstages) & 1);
      const long tile = ch.t0 + it;
      unsigned char* stp = stages + (size_t)s * stage_bytes;
      const bf16* Ut = (const bf16*)stp;                       // [blk][128][8]
      const float* Wt = (const float*)(stp + (size_t)nblk * kBlk * 2);   // [128][8]
      const bool ok = mbar_wait(&bar[s], par);
      if (!__syncthreads_and(ok)) {
        failed_it = it;
        break;
      }
      const int r0 = wid * 16;                                 // this warp's 16 rows
      if (MODE == BS_PROJ) {
        for (int i = t; i < kBlk; i += kThreads) split_bf16(Wt[i], w_hi[i], w_lo[i]);
      } else {
        // D = U (rows r0..r0+15) * C  (K = 16 basis columns per step)
        float dacc[4] = {0.f, 0.f, 0.f, 0.f};
        for (int ks = 0; ks < nmt; ++ks) {
          const int b0 = 2 * ks, b1 = 2 * ks + 1;
          const bf16* B0 = Ut + (size_t)b0 * kBlk;
          const bf16* B1 = (b1 < nblk) ? Ut + (size_t)b1 * kBlk : zblk;
          const int mi = lane >> 3, ri = lane & 7;
          const bf16* src = (mi & 2 ? B1 : B0) + (size_t)(r0 + (mi & 1) * 8 + ri) * kP;
          uint32_t a[4];
          ldsm_x4(a, src);
          // B = C rows 16ks..16ks+15 (basis), 8 columns; rows beyond the blocks are zero
          const int bi = lane & 15;
          const bf16* csrc_hi = (16 * ks + bi < nblk * 8) ? c_hi + (size_t)(16 * ks + bi) * 8 : zblk;
          const bf16* csrc_lo = (16 * ks + bi < nblk * 8) ? c_lo + (size_t)(16 * ks + bi) * 8 : zblk;
          uint32_t bh[2], bl[2];
          ldsm_x2_t(bh, csrc_hi);
          ldsm_x2_t(bl, csrc_lo);
          mma_bf16(dacc, a, bh);
          if (MODE == BS_XUPDATE) {   // middle part of Z (staged in w_hi)
            const bf16* csrc_md = (16 * ks + bi < nblk * 8) ? w_hi + (size_t)(16 * ks + bi) * 8 : zblk;
            uint32_t bm[2];
            ldsm_x2_t(bm, csrc_md);
            mma_bf16(dacc, a, bm);
          }
          mma_bf16(dacc, a, bl);
        }
        if (MODE == BS_XUPDATE) {
          // X += D in FP64 on this warp's fragment: rows r0+g8 (+8), columns 2 t4 (+1); padded
          // rows of the tile are written too (their basis rows are zero, so they stay zero)
          double2* x0 = reinterpret_cast<double2*>(X + ((size_t)tile * kTile + r0 + g8) * kP + 2 * t4);
          double2* x1 = x0 + 8 * kP / 2;
          double2 a0 = *x0, a1 = *x1;
          a0.x += (double)dacc[0];
          a0.y += (double)dacc[1];
          a1.x += (double)dacc[2];
          a1.y += (double)dacc[3];
          *x0 = a0;
          *x1 = a1;
          __syncthreads();   // stage free
          if (wid == 0 && it + nstages < ntl) issue(it + nstages);
          continue;
        }
        // W' = W - D on this warp's fragment: rows r0+g8 (+8), columns 2 t4 (+1)
        const float2 w0 = *reinterpret_cast<const float2*>(Wt + (size_t)(r0 + g8) * kP + 2 * t4);
        const float2 w1 =
            *reinterpret_cast<const float2*>(Wt + (size_t)(r0 + g8 + 8) * kP + 2 * t4);
        const float v00 = w0.x - dacc[0], v01 = w0.y - dacc[1];
        const float v10 = w1.x - dacc[2], v11 = w1.y - dacc[3];
        const size_t i0 = (size_t)(r0 + g8) * kP + 2 * t4, i1 = i0 + 8 * kP;
        if (MODE == BS_PASS2) {
          split_bf16(v00, w_hi[i0], w_lo[i0]);
          split_bf16(v01, w_hi[i0 + 1], w_lo[i0 + 1]);
          split_bf16(v10, w_hi[i1], w_lo[i1]);
          split_bf16(v11, w_hi[i1 + 1], w_lo[i1 + 1]);
        } else {
          // U_{k+1} = bf16(W''): into smem (Gram) and into basis block k+1 in global memory
          w_hi[i0] = __float2bfloat16_rn(v00);
          w_hi[i0 + 1] = __float2bfloat16_rn(v01);
          w_hi[i1] = __float2bfloat16_rn(v10);
          w_hi[i1 + 1] = __float2bfloat16_rn(v11);
          __syncwarp();
          // store this warp's 16 rows of the new block (16 rows x 16 bytes)
          const int rr = lane >> 1, hh = lane & 1;
          const uint2 val = *reinterpret_cast<const uint2*>(w_hi + (size_t)(r0 + rr) * kP + 4 * hh);
          *reinterpret_cast<uint2*>(Uw + (size_t)tile * uts + (size_t)(k + 1) * kBlk +
                                    (size_t)(r0 + rr) * kP + 4 * hh) = val;
          // Gram: G += Wb^T Wb over these 16 rows: A = Wb^T (8 x 16, zero-padded to 16 rows)
          uint32_t a[4], b[2];
          {
            const int mi = lane >> 3, ri = lane & 7;
            // matrices: (cols 0-7 of rows r0..r0+7)^T, zero, (rows r0+8..15)^T, zero
            const bf16* src = (mi & 1) ? zblk : w_hi + (size_t)(r0 + (mi >> 1) * 8 + ri) * kP;
            ldsm_x4_t(a, src);
            const bf16* bsrc = w_hi + (size_t)(r0 + (lane & 15)) * kP;
            ldsm_x2_t(b, bsrc);
          }
          float gd[4] = {0.f, 0.f, 0.f, 0.f};
          mma_bf16(gd, a, b);
          gacc[0] += gd[0];   // G[g8][2 t4], G[g8][2 t4 + 1]
          gacc[1] += gd[1];
        }
      }
      if (MODE != BS_UPDATE) {
        __syncthreads();   // w_hi / w_lo complete
        // P += U^T W: M-tiles mt = wid + 8 q (16 basis columns), K = 128 rows in 8 steps
#pragma unroll
        for (int q = 0; q < kMaxMt; ++q) {
          const int mt = wid + q * kWarps;
          if (mt >= nmt) break;
          const int b0 = 2 * mt, b1 = 2 * mt + 1;
          const bf16* B0 = Ut + (size_t)b0 * kBlk;
          const bf16* B1 = (b1 < nblk) ? Ut + (size_t)b1 * kBlk : zblk;
          for (int kk = 0; kk < kTile / 16; ++kk) {
            const int mi = lane >> 3, ri = lane & 7;
            // matrices: (B0 rows 16kk..+7)^T, (B1 rows 16kk..+7)^T, (B0 rows +8..)^T, (B1 ..)^T
            const bf16* src = ((mi & 1) ? B1 : B0) + (size_t)(16 * kk + (mi >> 1) * 8 + ri) * kP;
            uint32_t a[4];
            ldsm_x4_t(a, src);
            uint32_t bh[2], bl[2];
            ldsm_x2_t(bh, w_hi + (size_t)(16 * kk + (lane & 15)) * kP);
            ldsm_x2_t(bl, w_lo + (size_t)(16 * kk + (lane & 15)) * kP);
            mma_bf16(acc[q], a, bh);
            mma_bf16(acc[q], a, bl);
          }
        }
      }
      __syncthreads();   // stage and w_hi/w_lo free
      if (wid == 0 && it + nstages < ntl) issue(it + nstages);
    }
    if (failed_it >= 0) {
      // A wait ran out: wait (bounded) for the copies this chunk issued and has not consumed, so
      // none is still writing shared memory when the barriers are invalidated; flag the system
      // (the host stops the solve with GMRES_TIMEOUT).
      if (t == 0) {
        drain_stages(bar, nstages, phase_base + failed_it, phase_base + ntl);
        atomicExch(&S.st[ch.sys].breakdowns, kTimeoutMark);
      }
      break;
    }
    phase_base += ntl;
    if (MODE == BS_XUPDATE) continue;
    // ---- chunk partials ----
    float* part = S.part + (size_t)ci * kMaxBlocks * 64;
    if (MODE != BS_UPDATE) {
#pragma unroll
      for (int q = 0; q < kMaxMt; ++q) {
        const int mt = wid + q * kWarps;
        if (mt >= nmt) break;
        // rows of P: basis column 16 mt + g8 (+8), columns 2 t4 (+1)
        const int i0 = 16 * mt + g8, i1 = i0 + 8;
        if (i0 < nblk * 8) {
          part[(size_t)i0 * 8 + 2 * t4] = acc[q][0];
          part[(size_t)i0 * 8 + 2 * t4 + 1] = acc[q][1];
        }
        if (i1 < nblk * 8) {
          part[(size_t)i1 * 8 + 2 * t4] = acc[q][2];
          part[(size_t)i1 * 8 + 2 * t4 + 1] = acc[q][3];
        }
      }
    } else {
      gst[wid * 64 + g8 * 8 + 2 * t4] = gacc[0];
      gst[wid * 64 + g8 * 8 + 2 * t4 + 1] = gacc[1];
      __syncthreads();
      if (t < 64) {
        float sum = 0.f;
        for (int q = 0; q < kWarps; ++q) sum += gst[q * 64 + t];
        part[t] = sum;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  if (t == 0)
    for (int s = 0; s < nstages; ++s) mbar_inval(&bar[s]);
}

// ------------------------------------------------------------------------------------------------
// Per-system small steps (one CTA of 64 threads per system)
// ------------------------------------------------------------------------------------------------
// PROJ / PASS2 reduction: H_i = T_i^T sum_c P_i; coefficients of the next update.  One CTA of
// 1024 threads per system: first the chunk sums of all (block, entry) pairs, each split over up
// to 16 threads when there are few pairs (the late cycles' fine chunk lists have about a hundred
// chunks per system), then sixteen basis blocks at a time, one thread per (block, entry), for
// the two 8 x 8 products.
template <int MODE>
__global__ void __launch_bounds__(1024) kb_sys_coef(Small S, int k) {
  const int sys = blockIdx.x;
  SysState* st = S.st + sys;
  if (st->stop || st->done) return;
  const int nblk = k + 1;
  const int m = S.m;
  const int ld = (m + 1) * kP;
  const int t = threadIdx.x, sub = t >> 6, e = t & 63, a = e >> 3, b = e & 7;
  __shared__ float Pall[kMaxBlocks * 64];   // chunk sums, [block][entry]
  __shared__ float Pp[1024];                // part sums
  __shared__ float Hs[16][64], Ts[16][64];
  {
    // Sums over the cycle's chunks of every (block, entry): with few outputs, each output's
    // chunk range is split into P contiguous parts (P threads), added in part order.
    const int O = nblk * 64;
    const int P = max(1, min(16, 1024 / O));
    const int c0 = st->pc0, nc = st->pc1 - c0;
    if (P == 1) {
      for (int o = t; o < O; o += 1024) {
        float p = 0.f;
#pragma unroll 8
        for (int c = c0; c < c0 + nc; ++c) p += S.part[(size_t)c * kMaxBlocks * 64 + o];
        Pall[o] = p;
      }
    } else {
      const int per = (nc + P - 1) / P;
      if (t < P * O) {
        const int o = t % O, q = t / O;
        const int ca = c0 + min(nc, q * per), cb = c0 + min(nc, (q + 1) * per);
        float p = 0.f;
#pragma unroll 8
        for (int c = ca; c < cb; ++c) p += S.part[(size_t)c * kMaxBlocks * 64 + o];
        Pp[q * O + o] = p;
      }
      __syncthreads();
      if (t < O) {
        float p = Pp[t];
        for (int q = 1; q < P; ++q) p += Pp[q * O + t];
        Pall[t] = p;
      }
    }
  }
  __syncthreads();
  for (int i0 = 0; i0 < nblk; i0 += 16) {
    const int i = i0 + sub;
    const bool in = i < nblk;
    if (in) Ts[sub][e] = S.T[((size_t)sys * kMaxBlocks + i) * 64 + e];
    __syncthreads();
    float h = 0.f;
    if (in) {
      const float* Ps = Pall + i * 64;
      for (int r = 0; r < 8; ++r) h += Ts[sub][r * 8 + a] * Ps[r * 8 + b];   // T^T P
      float* H1 = S.H1 + ((size_t)sys * kMaxBlocks + i) * 64;
      if (MODE == BS_PASS2) {
        h += H1[e];
        // raw block H_{i,k} into column block k of the (to be triangularised) Hessenberg matrix
        float* R = S.R + (size_t)sys * ld * (m * kP);
        R[(size_t)(k * kP + b) * ld + i * kP + a] = h;
      } else {
        H1[e] = h;
      }
      Hs[sub][e] = h;
    }
    __syncthreads();
    if (in) {
      float c = 0.f;
      for (int r = 0; r < 8; ++r) c += Ts[sub][a * 8 + r] * Hs[sub][r * 8 + b];   // T H
      bf16 hi, lo;
      split_bf16(c, hi, lo);
      const size_t off = ((size_t)sys * kMaxBlocks + i) * 64 + e;
      S.Chi[off] = hi;
      S.Clo[off] = lo;
    }
    __syncthreads();
  }
}

// Householder reflector H = I - tau v v^T (v_0 = 1) taking a nine-entry window x (rows c .. c+8
// of column c of the block Hessenberg matrix, the rows its eight subdiagonal entries and the
// diagonal occupy) to (beta, 0, ..., 0): beta = -sign(x_0) ||x||, tau = (beta - x_0) / beta,
// v_i = x_i / (x_0 - beta) (the convention of LAPACK's larfg).  The norm is taken on x divided by
// its largest entry, so that no square overflows or underflows.  x_1 .. x_8 all zero: H = I.
__device__ __forceinline__ void householder9(float (&x)[9], float (&v)[8], float& tau) {
  float amax = 0.f;
#pragma unroll
  for (int i = 1; i < 9; ++i) amax = fmaxf(amax, fabsf(x[i]));
  tau = 0.f;
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = 0.f;
  if (amax == 0.f) return;
  amax = fmaxf(amax, fabsf(x[0]));
  const float inv = 1.f / amax;
  float q[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const float y = x[i] * inv;
    q[i] = y * y;
  }
  const float ss = (((q[0] + q[1]) + (q[2] + q[3])) + ((q[4] + q[5]) + (q[6] + q[7]))) + q[8];
  const float mu = amax * sqrtf(ss);
  const float beta = x[0] >= 0.f ? -mu : mu;
  tau = (beta - x[0]) / beta;
  const float sc = 1.f / (x[0] - beta);   // |x_0 - beta| >= ||x|| > 0
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = x[i + 1] * sc;
  x[0] = beta;
#pragma unroll
  for (int i = 1; i < 9; ++i) x[i] = 0.f;
}

// y <- (I - tau v v^T) y on a nine-entry window (v_0 = 1): one dot product (summed as a pairwise
// tree) and one update, so the dependent chain per reflector is a few operations long.
__device__ __forceinline__ void apply_householder9(float (&y)[9], const float (&v)[8], float tau) {
  float p[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) p[i] = v[i] * y[i + 1];
  const float d = y[0] + (((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7])));
  const float td = tau * d;
  y[0] -= td;
#pragma unroll
  for (int i = 0; i < 8; ++i) y[i + 1] = fmaf(-td, v[i], y[i + 1]);
}

// UPDATE reduction: Cholesky QR of the new block, Hessenberg subdiagonal block, and its
// elimination.  One CTA of 256 threads per system.  Column c of the band (eight subdiagonals) is
// triangularised by one Householder reflector on rows c .. c+8, stored as v_1..v_8 (rc) and tau
// (rs).  The reflectors of the earlier columns never reach the subdiagonal block (they touch rows
// < 8k + 8), so warp 1 applies them to the new columns while warp 0 factors the Gram matrix; then
// warp 0 eliminates the new columns' subdiagonals with every row a reflector can touch (block
// rows k and k+1) held in registers.
__global__ void __launch_bounds__(256) kb_sys_update(Small S, int k) {
  const int sys = blockIdx.x;
  SysState* st = S.st + sys;
  if (st->stop || st->done) return;
  const SysDesc d = S.sd[sys];
  const int m = S.m;
  const int ld = (m + 1) * kP;
  float* R = S.R + (size_t)sys * ld * (m * kP);
  float* g = S.g + (size_t)sys * ld * kP;
  float* rc = S.rc + (size_t)sys * (m * kP) * 8;
  float* rs = S.rs + (size_t)sys * (m * kP) * 8;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int nrow = (k + 2) * kP;       // rows touched by this step (block rows 0 .. k+1)
  const int nprev = k * kP;            // columns whose reflectors are applied to the new ones
  __shared__ float colS[kP][(kMaxSteps + 1) * kP];
  __shared__ float rcS[kMaxSteps * kP * 8], rsS[kMaxSteps * kP * 8];
  __shared__ float gS[(kMaxSteps + 1) * kP * kP];
  __shared__ double Gp[4][64];
  __shared__ double Gs[64], Ls[64];
  __shared__ float RtS[64];
  __shared__ int s_ok;
  {   // Gram of the new block: entry e summed over the p-th quarter of the system's chunks
    const int e = t & 63, p = t >> 6;
    const int c0 = st->pc0, nc = st->pc1 - c0, per = (nc + 3) / 4;
    const int ca = c0 + min(nc, p * per), cb = c0 + min(nc, (p + 1) * per);
    double acc = 0.0;
#pragma unroll 8
    for (int c = ca; c < cb; ++c) acc += S.part[(size_t)c * kMaxBlocks * 64 + e];
    Gp[p][e] = acc;
  }
  // (unrolled so that each thread has several independent loads in flight per loop)
#pragma unroll 4
  for (int i = t; i < nprev * 8; i += 256) {
    rcS[i] = rc[i];
    rsS[i] = rs[i];
  }
#pragma unroll 4
  for (int i = t; i < nrow * kP; i += 256) gS[i] = g[i];
  // the new columns' rows 0 .. 8k+7 (the subdiagonal block rows come from the factorisation)
#pragma unroll 4
  for (int i = t; i < kP * nrow; i += 256) {
    const int q = i / nrow, r = i % nrow;
    colS[q][r] = r < nprev + kP ? R[(size_t)(k * kP + q) * ld + r] : 0.f;
  }
  __syncthreads();
  if (t < 64) Gs[t] = ((Gp[0][t] + Gp[1][t]) + Gp[2][t]) + Gp[3][t];
  __syncthreads();
  if (wid == 0) {
    if (lane < 8) {
      float* Tn = S.T + ((size_t)sys * kMaxBlocks + k + 1) * 64;
      const bool ok = cholqr_warp(Gs, Ls, d.n, Tn, RtS, ldexp(1.0, -24));
      if (lane == 0) s_ok = ok ? 1 : 0;
    }
  } else if (wid == 1 && lane < kP && nprev > 0) {
    // earlier columns' reflectors on new column `lane`: column c's reflector touches rows
    // c .. c+8 and row c no later column touches, so the lane carries the window of rows
    // c .. c+8 in registers, retires row c and takes in row c+9 per column
    float* col = colS[lane];
    float wv[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) wv[r] = col[r];
    for (int c = 0; c < nprev; ++c) {
      float v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = rcS[c * 8 + q];
      apply_householder9(wv, v, rsS[c * 8]);
      col[c] = wv[0];
#pragma unroll
      for (int r = 0; r < 8; ++r) wv[r] = wv[r + 1];
      wv[8] = col[c + 9];   // row c + 9 <= nprev + 8 < nrow
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) col[nprev + r] = wv[r];   // row nprev + 8 is not touched
  }
  __syncthreads();
  // subdiagonal block (k+1, k) = L^T (upper triangular), or zero on breakdown
  if (t < 64) colS[t & 7][(k + 1) * kP + (t >> 3)] = s_ok ? RtS[t] : 0.f;
  __syncthreads();
  if (wid == 0 && lane < 2 * kP) {
    // New columns one by one: a reflector on rows c .. c+8 eliminates rows c+1 .. c+8, c = 8k + qc.
    // Lanes 0..7 own new column `lane`, lanes 8..15 right-hand-side column lane - 8 of g.  The
    // reflector of column c touches rows c .. c+8 and row c no later one does: every lane carries
    // that window in registers, retires row c and takes in row c+9 (of 8k .. 8k+15) per column.
    const bool colLane = lane < kP;
    float* base = colLane ? &colS[lane][nprev] : &gS[(size_t)nprev * kP + (lane - kP)];
    const int stride = colLane ? 1 : kP;
    float w[9];
#pragma unroll
    for (int r = 0; r < 9; ++r) w[r] = base[r * stride];
    for (int qc = 0; qc < kP; ++qc) {
      // lane qc forms its column's reflector on its own window; v and tau are broadcast and the
      // later columns and every right-hand side apply it
      float v[8], tau = 0.f;
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = 0.f;
      if (lane == qc) {
        householder9(w, v, tau);
        float4* vc = reinterpret_cast<float4*>(rc + (size_t)(nprev + qc) * 8);
        vc[0] = make_float4(v[0], v[1], v[2], v[3]);
        vc[1] = make_float4(v[4], v[5], v[6], v[7]);
        rs[(size_t)(nprev + qc) * 8] = tau;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) v[q] = __shfl_sync(0xffffu, v[q], qc);
      tau = __shfl_sync(0xffffu, tau, qc);
      if (lane > qc) apply_householder9(w, v, tau);   // later new columns and every rhs
      base[qc * stride] = w[0];
#pragma unroll
      for (int r = 0; r < 8; ++r) w[r] = w[r + 1];
      if (qc + 9 < 2 * kP) w[8] = base[(qc + 9) * stride];
    }
#pragma unroll
    for (int r = 0; r < 8; ++r) base[(kP + r) * stride] = w[r];   // rows 8k+8 .. 8k+15
    if (!colLane) {   // implicit residual: rows 8(k+1) .. 8(k+2)-1 of g
      float s2 = 0.f;
#pragma unroll
      for (int r = 0; r < 8; ++r) s2 += w[r] * w[r];
      st->imp[lane - kP] = sqrtf(s2);
    }
  }
  __syncthreads();
  // write back the transformed columns and g
  for (int i = t; i < kP * nrow; i += 256) {
    const int q = i / nrow, r = i % nrow;
    R[(size_t)(k * kP + q) * ld + r] = colS[q][r];
  }
  for (int i = t; i < nrow * kP; i += 256) g[i] = gS[i];
  if (t == 0) {
    st->k = k + 1;
    st->iters += 1;
    if (!s_ok) {
      st->breakdowns += 1;
      st->stop = 1;
    } else if (k + 1 >= m) {
      st->stop = 1;
    }
  }
}

// Cycle end: Y = R^{-1} g (8 columns), Z_i = T_i Y_i.  One CTA of 256 threads per system; block
// back substitution over the 8 x 8 blocks of the triangularised (upper triangular) R.  The diagonal
// blocks are staged in shared memory; for block I, lanes 0..7 of warp 0 solve the diagonal block
// (lane c: right-hand side c) while every thread t < 8I has its row of R's block column I in
// flight, then thread t removes the solved block from row t of the right-hand sides.
__global__ void __launch_bounds__(256) kb_sys_solve(Small S) {
  const int sys = blockIdx.x;
  SysState* st = S.st + sys;
  if (st->done) return;
  const int kk = st->k;
  const int m = S.m;
  const int ld = (m + 1) * kP;
  const float* R = S.R + (size_t)sys * ld * (m * kP);
  const float* g = S.g + (size_t)sys * ld * kP;
  const int t = threadIdx.x;
  __shared__ float rhs[kMaxSteps * kP][kP];   // g, reduced as blocks are solved
  __shared__ float y[kMaxSteps * kP][kP];
  __shared__ float dg[kMaxSteps][kP][kP];     // diagonal blocks: dg[I][a][b] = R(8I + a, 8I + b)
  const int nn = kk * kP;
  for (int i = t; i < nn * kP; i += 256) rhs[i / kP][i % kP] = g[i];
  for (int i = t; i < kk * 64; i += 256) {
    const int I = i >> 6, a = (i >> 3) & 7, b = i & 7;
    dg[I][a][b] = R[(size_t)(I * kP + b) * ld + I * kP + a];
  }
  __syncthreads();
  for (int I = kk - 1; I >= 0; --I) {
    const int r0 = I * kP;
    float rv[kP];   // R(t, 8I + q): row t of block column I (t < 8I)
    if (t < r0) {
#pragma unroll
      for (int q = 0; q < kP; ++q) rv[q] = R[(size_t)(r0 + q) * ld + t];
    }
    if (t < kP) {
      for (int i = kP - 1; i >= 0; --i) {
        float sv = rhs[r0 + i][t];
        for (int j = i + 1; j < kP; ++j) sv -= dg[I][i][j] * y[r0 + j][t];
        const float rii = dg[I][i][i];
        y[r0 + i][t] = rii != 0.f ? sv / rii : 0.f;
      }
    }
    __syncthreads();
    if (t < r0) {
#pragma unroll
      for (int c = 0; c < kP; ++c) {
        float sv = rhs[t][c];
#pragma unroll
        for (int q = 0; q < kP; ++q) sv -= rv[q] * y[r0 + q][c];
        rhs[t][c] = sv;
      }
    }
    __syncthreads();
  }
  // Z_b = T_b Y_b: thread per (block, row a, column c)
  for (int e = t; e < kk * 64; e += 256) {
    const int b = e >> 6, a = (e >> 3) & 7, c = e & 7;
    const float* T = S.T + ((size_t)sys * kMaxBlocks + b) * 64;
    float sv = 0.f;
#pragma unroll
    for (int r = 0; r < 8; ++r) sv += T[a * 8 + r] * y[b * kP + r][c];
    S.Z[((size_t)sys * kMaxBlocks + b) * 64 + a * 8 + c] = sv;
  }
  if (t == 0) st->cycles += 1;
}

}  // namespace batch
}  // namespace gmresb3

// ------------------------------------------------------------------------------------------------
// Host side
// ------------------------------------------------------------------------------------------------
namespace {

using namespace gmresb3::batch;

struct BFail {
  int code;
};
#define BCK(call)                                                                         \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess)                                                                \
      throw BFail{e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA};      \
  } while (0)

template <typename T> T* balloc(size_t count) {
  void* p = nullptr;
  BCK(cudaMalloc(&p, std::max<size_t>(count, 1) * sizeof(T)));
  BCK(cudaMemset(p, 0, std::max<size_t>(count, 1) * sizeof(T)));
  return (T*)p;
}

// column-major per-system blocks <-> padded row-major [row][8]
__global__ void kb_pack(const double* __restrict__ src, double* __restrict__ dst, int N,
                        const int* __restrict__ tile_sys, const SysDesc* __restrict__ sd,
                        const long* __restrict__ soff) {
  const long row = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (row >= N) return;
  const int sys = tile_sys[row >> kTileShift];
  const SysDesc d = sd[sys];
  const long r = row - d.row0;
#pragma unroll
  for (int c = 0; c < kP; ++c) dst[row * kP + c] = (r < d.n) ? src[soff[sys] + (long)c * d.n + r] : 0.0;
}

__global__ void kb_unpack(const double* __restrict__ src, double* __restrict__ dst, int N,
                          const int* __restrict__ tile_sys, const SysDesc* __restrict__ sd,
                          const long* __restrict__ soff) {
  const long row = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (row >= N) return;
  const int sys = tile_sys[row >> kTileShift];
  const SysDesc d = sd[sys];
  const long r = row - d.row0;
  if (r >= d.n) return;
#pragma unroll
  for (int c = 0; c < kP; ++c) dst[soff[sys] + (long)c * d.n + r] = src[row * kP + c];
}

}  // namespace

struct gmres_batch_ctx {
  int dev = 0, sms = 1, nsys = 0, m = 0;
  int N = 0, ntiles = 0, nchunks = 0;
  long total_n = 0;                  // sum of n_s (unpadded)
  cudaStream_t stream = nullptr, user_stream = nullptr;
  cudaEvent_t ev = nullptr;
  int* rowptr = nullptr;
  int* col = nullptr;
  double* v64 = nullptr;
  float* v32 = nullptr;
  int* tile_sys = nullptr;
  SysDesc* sd = nullptr;
  Chunk* chunks = nullptr;
  long* soff = nullptr;
  std::vector<SysDesc> hsd;
  bf16* U = nullptr;
  long uts = 0;
  float* W = nullptr;
  double* X = nullptr;
  double* B = nullptr;
  double* stage = nullptr;           // caller layout staging (device)
  Small S{};
  SysState* st_host = nullptr;
  cudaGraphExec_t graph = nullptr;
  int graph_launches = 0;
  int profiling = 0;
  gmres_batch_tuning_t tuning{};     // launch shapes (0 = default)
  size_t chunk_cap = 0;              // chunks the chunk list and partial sums are allocated for
  int* act_tiles = nullptr;          // active work lists of the current cycle (kb_compact)
  int* act_chunks = nullptr;
  int* act_cnt = nullptr;
  int grid_spmm = 0;                 // persistent grids of the kernels over active tiles
  int grid_start = 0;
  int grid_res = 0;
  cudaEvent_t pev[2] = {nullptr, nullptr};
  ~gmres_batch_ctx() {
    for (auto e : pev)
      if (e) cudaEventDestroy(e);
    if (graph) cudaGraphExecDestroy(graph);
    void* ptrs[] = {rowptr, col, v64, v32, tile_sys, sd, chunks, soff, U, W, X, B, stage,
                    act_tiles, act_chunks, act_cnt,
                    S.T, S.H1, S.R, S.rc, S.rs, S.g, S.Z, S.Chi, S.Clo, S.part, S.tpart,
                    S.tgram, S.st};
    for (void* p : ptrs) cudaFree(p);
    if (st_host) cudaFreeHost(st_host);
    if (ev) cudaEventDestroy(ev);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

int brun(const std::function<void()>& fn) {
  try {
    fn();
    return GMRES_OK;
  } catch (const BFail& f) {
    cudaGetLastError();
    return f.code;
  } catch (const std::bad_alloc&) {
    return GMRES_ERR_OOM;
  } catch (...) {
    return GMRES_ERR_CUDA;
  }
}

struct BLaunch {
  int grid, stages;
  size_t smem;
};

int eff_chunk_tiles(const gmres_batch_ctx& b) {
  return b.tuning.chunk_tiles ? b.tuning.chunk_tiles : kChunkTiles;
}
// Chunks of the late cycles (few systems left): half the size, at least four tiles.
int fine_chunk_tiles(const gmres_batch_ctx& b) { return std::max(4, eff_chunk_tiles(b) / 2); }

// Split every system's tile range into chunks of the tuned size (one sweep work item each),
// record each system's chunk range, and upload both; the chunk list and the per-chunk partial
// sums grow when a smaller chunk size needs more chunks.  Drops the captured cycle graph.  New
// buffers are allocated before the old ones are released and the host ranges are committed last,
// so a failed allocation leaves the batch as it was.
void build_chunks(gmres_batch_ctx& b) {
  const int ct = eff_chunk_tiles(b), cf = fine_chunk_tiles(b);
  std::vector<Chunk> chs;
  std::vector<SysDesc> sd = b.hsd;
  for (int s = 0; s < b.nsys; ++s) {
    SysDesc& d = sd[s];
    d.c0 = (int)chs.size();
    for (int t = d.t0; t < d.t1; t += ct) chs.push_back(Chunk{s, t, std::min(t + ct, d.t1)});
    d.c1 = (int)chs.size();
  }
  for (int s = 0; s < b.nsys; ++s) {
    SysDesc& d = sd[s];
    d.f0 = (int)chs.size();
    for (int t = d.t0; t < d.t1; t += cf) chs.push_back(Chunk{s, t, std::min(t + cf, d.t1)});
    d.f1 = (int)chs.size();
  }
  BCK(cudaStreamSynchronize(b.stream));   // no queued work still reads the old lists
  if (chs.size() > b.chunk_cap) {
    Chunk* nc = nullptr;
    float* np = nullptr;
    int* na = nullptr;
    try {
      nc = balloc<Chunk>(chs.size());
      np = balloc<float>(chs.size() * kMaxBlocks * 64);
      na = balloc<int>(chs.size());
    } catch (...) {
      cudaFree(nc);
      cudaFree(np);
      cudaFree(na);
      throw;
    }
    cudaFree(b.chunks);
    cudaFree(b.S.part);
    cudaFree(b.act_chunks);
    b.chunks = nc;
    b.S.part = np;
    b.act_chunks = na;
    b.chunk_cap = chs.size();
    // balloc clears on the legacy default stream: order the private stream after it
    BCK(cudaEventRecord(b.ev, 0));
    BCK(cudaStreamWaitEvent(b.stream, b.ev, 0));
  }
  BCK(cudaMemcpyAsync(b.chunks, chs.data(), chs.size() * sizeof(Chunk), cudaMemcpyHostToDevice, b.stream));
  BCK(cudaMemcpyAsync(b.sd, sd.data(), b.nsys * sizeof(SysDesc), cudaMemcpyHostToDevice, b.stream));
  BCK(cudaStreamSynchronize(b.stream));   // the host vectors go out of scope
  b.hsd = sd;
  b.nchunks = (int)chs.size();
  if (b.graph) {
    cudaGraphExecDestroy(b.graph);
    b.graph = nullptr;
  }
}

template <int MODE> BLaunch plan_sweep(const gmres_batch_ctx& b, int nblk) {
  auto kern = kb_sweep<MODE>;
  const size_t stage = bs_stage_bytes(nblk);
  const size_t fixed = bs_fixed_bytes();
  const size_t budget = (size_t)(b.tuning.sweep_smem_kb ? b.tuning.sweep_smem_kb : kSweepSmemKb) * 1024;
  const size_t cap = (size_t)(b.tuning.sweep_max_stages ? b.tuning.sweep_max_stages : kSweepStages);
  int st = (int)std::min<size_t>(cap, std::max<size_t>(2, (budget - std::min(fixed, budget)) / stage));
  while (st > 1 && fixed + st * stage > 220 * 1024) --st;
  BLaunch L{0, st, fixed + st * stage};
  // The per-CTA maximum, not this launch's size: one captured cycle holds sweeps of different
  // sizes, and a graph node is checked against the attribute as it stands when the node runs.
  int optin = 0;
  BCK(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, b.dev));
  cudaFuncAttributes fa{};
  BCK(cudaFuncGetAttributes(&fa, kern));
  if (L.smem + fa.sharedSizeBytes > (size_t)optin) throw BFail{GMRES_ERR_UNSUPPORTED};
  BCK(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           optin - (int)fa.sharedSizeBytes));
  int per_sm = 0;
  BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kThreads, L.smem));
  per_sm = std::max(1, per_sm);
  L.grid = std::max(1, std::min(b.nchunks, b.sms * per_sm));
  return L;
}

Active active(const gmres_batch_ctx& b) { return Active{b.act_tiles, b.act_chunks, b.act_cnt}; }

// Active tile and chunk lists from the systems' converged flags (before every cycle).
// The fine chunk list is taken once the active tiles would give the sweeps fewer coarse chunks
// than two CTAs per SM.
void launch_compact(const gmres_batch_ctx& b, cudaStream_t s) {
  const int fine_below = 2 * b.sms * eff_chunk_tiles(b);
  kb_compact<<<b.nsys, 128, 0, s>>>(b.S, b.nsys, fine_below, b.act_tiles, b.act_chunks, b.act_cnt);
}

// Launch the kernels of one block cycle (+ residual of the next one).
// One block cycle of all systems.  With tk (profiling), each kernel class is bracketed by CUDA
// events on the batch's stream and its time added to tk[class]; cl counts launches per class.
int launch_cycle(gmres_batch_ctx& b, double tol, double* tk = nullptr, int64_t* cl = nullptr) {
  int n = 0;
  cudaStream_t s = b.stream;
  auto timed = [&](int cls, int nl, auto fn) {
    if (!tk) {
      fn();
    } else {
      BCK(cudaEventRecord(b.pev[0], s));
      fn();
      BCK(cudaEventRecord(b.pev[1], s));
      BCK(cudaEventSynchronize(b.pev[1]));
      float ms = 0.f;
      BCK(cudaEventElapsedTime(&ms, b.pev[0], b.pev[1]));
      tk[cls] += ms * 1e-3;
      cl[cls] += nl;
    }
    n += nl;
  };
  const Active act = active(b);
  timed(GMRES_BT_CYCLE, 2, [&] {
    kb_start<<<b.grid_start, kTile, 0, s>>>(b.W, b.U, b.uts, b.N, b.tile_sys, act, b.S);
    kb_sys_start_n<<<b.nsys, 512, 0, s>>>(b.S, b.nsys);
  });
  const Csr<float> A32{b.N, 0, b.rowptr, b.col, b.v32};
  // The three sweeps of a block step walk their chunks in alternating directions (the SpMM
  // forward, then backward, forward, backward), each starting where its predecessor ended.
  for (int k = 0; k < b.m; ++k) {
    timed(GMRES_BT_SPMM, 1, [&] {
      kb_spmm<<<b.grid_spmm, kTile, 0, s>>>(A32, b.U, b.uts, k, b.W, b.tile_sys, act, b.S);
    });
    BLaunch L0 = plan_sweep<BS_PROJ>(b, k + 1);
    timed(GMRES_BT_SWEEP, 1, [&] {
      kb_sweep<BS_PROJ><<<L0.grid, kThreads, L0.smem, s>>>(b.U, b.U, b.uts, k, b.W, b.chunks,
                                                           act, b.S, L0.stages, 1, nullptr);
    });
    timed(GMRES_BT_SMALL, 1, [&] { kb_sys_coef<BS_PROJ><<<b.nsys, 1024, 0, s>>>(b.S, k); });
    BLaunch L1 = plan_sweep<BS_PASS2>(b, k + 1);
    timed(GMRES_BT_SWEEP, 1, [&] {
      kb_sweep<BS_PASS2><<<L1.grid, kThreads, L1.smem, s>>>(b.U, b.U, b.uts, k, b.W, b.chunks,
                                                            act, b.S, L1.stages, 0, nullptr);
    });
    timed(GMRES_BT_SMALL, 1, [&] { kb_sys_coef<BS_PASS2><<<b.nsys, 1024, 0, s>>>(b.S, k); });
    BLaunch L2 = plan_sweep<BS_UPDATE>(b, k + 1);
    timed(GMRES_BT_SWEEP, 1, [&] {
      kb_sweep<BS_UPDATE><<<L2.grid, kThreads, L2.smem, s>>>(b.U, b.U, b.uts, k, b.W, b.chunks,
                                                             act, b.S, L2.stages, 1, nullptr);
    });
    timed(GMRES_BT_SMALL, 1, [&] { kb_sys_update<<<b.nsys, 256, 0, s>>>(b.S, k); });
  }
  BLaunch LX = plan_sweep<BS_XUPDATE>(b, b.m);
  timed(GMRES_BT_CYCLE, 5, [&] {
    kb_sys_solve<<<b.nsys, 256, 0, s>>>(b.S);
    // X += U Z over the cycle's chunks: the tensor-core sweep over the m basis blocks
    kb_sweep<BS_XUPDATE><<<LX.grid, kThreads, LX.smem, s>>>(b.U, b.U, b.uts, b.m - 1, b.W, b.chunks,
                                                            act, b.S, LX.stages, 0, b.X);
    const Csr<double> A64{b.N, 0, b.rowptr, b.col, b.v64};
    kb_residual<<<b.grid_res, kTile, 0, s>>>(A64, b.X, b.B, b.W, b.tile_sys, act, b.S);
    kb_sys_residual<<<b.nsys, 256, 0, s>>>(b.S, tol);
    launch_compact(b, s);
  });
  BCK(cudaGetLastError());
  return n;
}

}  // namespace

extern "C" {

int gmres_batch_create(int nsys, const gmres_csr_t* A, int nrhs, int m, gmres_precisions_t prec,
                       gmres_batch_t* out) {
  if (!out) return GMRES_ERR_INVALID_ARG;
  *out = nullptr;
  if (nsys < 1 || !A || nrhs != kP || m < 1 || m > kMaxSteps) return GMRES_ERR_INVALID_ARG;
  if (prec.matrix != GMRES_F32 || prec.inner != GMRES_F32 || prec.basis != GMRES_BF16 ||
      prec.precond != GMRES_F32)
    return GMRES_ERR_UNSUPPORTED;
  gmres_batch_ctx* b = new (std::nothrow) gmres_batch_ctx();
  if (!b) return GMRES_ERR_OOM;
  const int rc = brun([&] {
    BCK(cudaGetDevice(&b->dev));
    cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, b->dev);
    BCK(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    BCK(cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming));
    BCK(cudaEventCreate(&b->pev[0]));
    BCK(cudaEventCreate(&b->pev[1]));
    // Uploads and clears below run on the legacy default stream (plain cudaMemcpy / cudaMemset,
    // which may return before the device is done); the non-blocking private stream does not
    // synchronise with it by itself, so it waits on an event recorded there before using them.
    auto join_legacy = [&] {
      BCK(cudaEventRecord(b->ev, 0));
      BCK(cudaStreamWaitEvent(b->stream, b->ev, 0));
    };
    b->nsys = nsys;
    b->m = m;
    // block-diagonal assembly on the host, each system padded to whole tiles
    std::vector<int> rp(1, 0), ci;
    std::vector<double> va;
    std::vector<int> tsys;
    std::vector<long> soff(nsys);
    long roff = 0, nsum = 0;
    for (int s = 0; s < nsys; ++s) {
      const gmres_csr_t& a = A[s];
      if (a.n < 1 || a.nnz < 0 || !a.rowptr || (a.nnz > 0 && (!a.colidx || !a.val)))
        throw BFail{GMRES_ERR_INVALID_ARG};
      std::vector<int32_t> r(a.n + 1), c(a.nnz);
      std::vector<double> v(a.nnz);
      BCK(cudaMemcpy(r.data(), a.rowptr, (a.n + 1) * 4, cudaMemcpyDefault));
      if (a.nnz) {
        BCK(cudaMemcpy(c.data(), a.colidx, a.nnz * 4, cudaMemcpyDefault));
        BCK(cudaMemcpy(v.data(), a.val, a.nnz * 8, cudaMemcpyDefault));
      }
      if (r[0] != 0 || r[a.n] != a.nnz) throw BFail{GMRES_ERR_INVALID_ARG};
      SysDesc d{};
      d.row0 = (int)roff;
      d.n = (int)a.n;
      d.t0 = (int)(roff / kTile);
      const long npad = (a.n + kTile - 1) / kTile * kTile;
      d.t1 = d.t0 + (int)(npad / kTile);
      for (long i = 0; i < a.n; ++i) {
        if (r[i + 1] < r[i]) throw BFail{GMRES_ERR_INVALID_ARG};
        for (int p = r[i]; p < r[i + 1]; ++p) {
          if (c[p] < 0 || c[p] >= a.n || !std::isfinite(v[p])) throw BFail{GMRES_ERR_INVALID_ARG};
          ci.push_back((int)(c[p] + roff));
          va.push_back(v[p]);
        }
        rp.push_back((int)ci.size());
      }
      for (long i = a.n; i < npad; ++i) rp.push_back((int)ci.size());   // empty padding rows
      for (int t = d.t0; t < d.t1; ++t) tsys.push_back(s);
      b->hsd.push_back(d);
      soff[s] = nsum * kP;
      nsum += a.n;
      roff += npad;
    }
    if (roff >= (1ll << 31) - 1024 || ci.size() >= (size_t)(1ll << 31) - 64) throw BFail{GMRES_ERR_INVALID_ARG};
    b->N = (int)roff;
    b->ntiles = (int)(roff / kTile);
    b->total_n = nsum;
    rp.resize(rp.size() + 8, (int)ci.size());
    ci.resize(ci.size() + 16, 0);
    va.resize(va.size() + 16, 0.0);
    b->rowptr = balloc<int>(rp.size());
    b->col = balloc<int>(ci.size());
    b->v64 = balloc<double>(va.size());
    b->v32 = balloc<float>(va.size());
    BCK(cudaMemcpy(b->rowptr, rp.data(), rp.size() * 4, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->col, ci.data(), ci.size() * 4, cudaMemcpyHostToDevice));
    BCK(cudaMemcpy(b->v64, va.data(), va.size() * 8, cudaMemcpyHostToDevice));
    join_legacy();   // the cast reads v64
    k_cast_f64_f32<<<b->sms * 4, 256, 0, b->stream>>>(b->v64, b->v32, (long)va.size());
    BCK(cudaGetLastError());
    b->tile_sys = balloc<int>(tsys.size());
    BCK(cudaMemcpy(b->tile_sys, tsys.data(), tsys.size() * 4, cudaMemcpyHostToDevice));
    b->sd = balloc<SysDesc>(nsys);
    b->act_tiles = balloc<int>(b->ntiles);
    b->act_cnt = balloc<int>(4);
    {   // persistent grids: every resident 128-thread CTA, at most one per tile
      auto grid_of = [&](auto kern) {
        int per_sm = 0;
        BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTile, 0));
        return std::max(1, std::min(b->ntiles, b->sms * std::max(1, per_sm)));
      };
      b->grid_spmm = grid_of(kb_spmm);
      b->grid_start = grid_of(kb_start);
      b->grid_res = grid_of(kb_residual);
    }
    b->soff = balloc<long>(nsys);
    BCK(cudaMemcpy(b->soff, soff.data(), nsys * sizeof(long), cudaMemcpyHostToDevice));
    b->uts = (long)(m + 1) * kBlk;
    b->U = balloc<bf16>((size_t)b->ntiles * b->uts);
    b->W = balloc<float>((size_t)b->N * kP);
    b->X = balloc<double>((size_t)b->N * kP);
    b->B = balloc<double>((size_t)b->N * kP);
    b->stage = balloc<double>((size_t)nsum * kP);
    const size_t ld = (size_t)(m + 1) * kP;
    Small& S = b->S;
    S.T = balloc<float>((size_t)nsys * kMaxBlocks * 64);
    S.H1 = balloc<float>((size_t)nsys * kMaxBlocks * 64);
    S.R = balloc<float>((size_t)nsys * ld * m * kP);
    S.rc = balloc<float>((size_t)nsys * m * kP * 8);
    S.rs = balloc<float>((size_t)nsys * m * kP * 8);
    S.g = balloc<float>((size_t)nsys * ld * kP);
    S.Z = balloc<float>((size_t)nsys * kMaxBlocks * 64);
    S.Chi = balloc<bf16>((size_t)nsys * kMaxBlocks * 64);
    S.Clo = balloc<bf16>((size_t)nsys * kMaxBlocks * 64);
    S.tpart = balloc<double>((size_t)b->ntiles * 16);
    S.tgram = balloc<float>((size_t)b->ntiles * 64);
    S.st = balloc<SysState>(nsys);
    S.sd = b->sd;
    S.m = m;
    BCK(cudaMallocHost(&b->st_host, nsys * sizeof(SysState)));
    join_legacy();
    build_chunks(*b);   // chunk list, system chunk ranges and partial sums (default shapes)
  });
  if (rc != GMRES_OK) {
    delete b;
    return rc;
  }
  *out = b;
  return GMRES_OK;
}

int gmres_batch_destroy(gmres_batch_t b) {
  if (!b) return GMRES_OK;
  cudaStreamSynchronize(b->stream);
  delete b;
  return GMRES_OK;
}

int gmres_batch_set_profiling(gmres_batch_t b, int on) {
  if (!b) return GMRES_ERR_INVALID_ARG;
  b->profiling = on ? 1 : 0;
  return GMRES_OK;
}

int gmres_batch_set_tuning(gmres_batch_t b, const gmres_batch_tuning_t* t) {
  if (!b || !t) return GMRES_ERR_INVALID_ARG;
  const gmres_batch_tuning_t v = *t;
  if (v.chunk_tiles != 0 && (v.chunk_tiles < 4 || v.chunk_tiles > 64)) return GMRES_ERR_INVALID_ARG;
  if (v.sweep_smem_kb != 0 && (v.sweep_smem_kb < 64 || v.sweep_smem_kb > 220)) return GMRES_ERR_INVALID_ARG;
  if (v.sweep_max_stages != 0 && (v.sweep_max_stages < 2 || v.sweep_max_stages > kMaxStages))
    return GMRES_ERR_INVALID_ARG;
  if (v.reserved != 0) return GMRES_ERR_INVALID_ARG;
  const gmres_batch_tuning_t old = b->tuning;
  b->tuning = v;
  const int rc = brun([&] {
    if (eff_chunk_tiles(*b) != (old.chunk_tiles ? old.chunk_tiles : kChunkTiles)) {
      build_chunks(*b);
    } else if (b->graph) {   // the sweep launch shapes are baked into the captured graph
      BCK(cudaStreamSynchronize(b->stream));
      cudaGraphExecDestroy(b->graph);
      b->graph = nullptr;
    }
  });
  if (rc != GMRES_OK) b->tuning = old;
  return rc;
}

int gmres_batch_get_tuning(gmres_batch_t b, gmres_batch_tuning_t* t) {
  if (!b || !t) return GMRES_ERR_INVALID_ARG;
  *t = b->tuning;
  return GMRES_OK;
}

int gmres_batch_set_stream(gmres_batch_t b, void* s) {
  if (!b) return GMRES_ERR_INVALID_ARG;
  b->user_stream = (cudaStream_t)s;
  return GMRES_OK;
}

int gmres_batch_ir_solve(gmres_batch_t b, const double* Bin, double* Xio, double tol,
                         int max_cycles, gmres_batch_stats_t* stats) {
  if (!b || !Bin || !Xio || !(tol >= 0.0) || max_cycles < 0) return GMRES_ERR_INVALID_ARG;
  int status = GMRES_NOT_CONVERGED;
  const int rc = brun([&] {
    auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = b->stream;
    // the private stream is non-blocking: order it after the caller's stream (NULL = legacy)
    BCK(cudaEventRecord(b->ev, b->user_stream));
    BCK(cudaStreamWaitEvent(s, b->ev, 0));
    const size_t bytes = (size_t)b->total_n * kP * sizeof(double);
    const int rows_grid = (b->N + 255) / 256;
    BCK(cudaMemcpyAsync(b->stage, Bin, bytes, cudaMemcpyDefault, s));
    kb_pack<<<rows_grid, 256, 0, s>>>(b->stage, b->B, b->N, b->tile_sys, b->sd, b->soff);
    BCK(cudaMemcpyAsync(b->stage, Xio, bytes, cudaMemcpyDefault, s));
    kb_pack<<<rows_grid, 256, 0, s>>>(b->stage, b->X, b->N, b->tile_sys, b->sd, b->soff);
    // fresh per-system state
    std::vector<SysState> init(b->nsys);
    for (auto& x : init) {
      std::memset(&x, 0, sizeof(x));
      x.first = 1;
    }
    BCK(cudaMemcpyAsync(b->S.st, init.data(), b->nsys * sizeof(SysState), cudaMemcpyHostToDevice, s));
    const Csr<double> A64{b->N, 0, b->rowptr, b->col, b->v64};
    launch_compact(*b, s);   // every system active
    kb_residual<<<b->grid_res, kTile, 0, s>>>(A64, b->X, b->B, b->W, b->tile_sys, active(*b), b->S);
    kb_sys_residual<<<b->nsys, 256, 0, s>>>(b->S, tol);
    launch_compact(*b, s);   // the systems the first cycle runs
    BCK(cudaGetLastError());
    int64_t launches = 6;   // kernels so far: two packs, two compactions, residual, convergence
    int cycles = 0;
    double tk[4] = {0, 0, 0, 0};
    int64_t cl[4] = {0, 0, 0, 0};
    for (;;) {
      BCK(cudaMemcpyAsync(b->st_host, b->S.st, b->nsys * sizeof(SysState), cudaMemcpyDeviceToHost, s));
      BCK(cudaStreamSynchronize(s));
      int ndone = 0, expired = 0;
      for (int i = 0; i < b->nsys; ++i) {
        ndone += b->st_host[i].done ? 1 : 0;
        expired |= b->st_host[i].breakdowns >= kTimeoutMark;
      }
      if (expired) {   // a bulk-copy wait ran out: the iterates of that cycle are not trusted
        status = GMRES_TIMEOUT;
        break;
      }
      if (ndone == b->nsys) {
        status = GMRES_OK;
        break;
      }
      if (cycles >= max_cycles) break;
      if (b->profiling) {   // direct launches, kernel classes timed with events
        launches += launch_cycle(*b, tol, tk, cl);
        ++cycles;
        continue;
      }
      if (!b->graph) {
        cudaGraph_t g;
        BCK(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        int n = 0;
        try {
          n = launch_cycle(*b, tol);
        } catch (...) {
          cudaStreamEndCapture(s, &g);
          if (g) cudaGraphDestroy(g);
          throw;
        }
        BCK(cudaStreamEndCapture(s, &g));
        const cudaError_t e = cudaGraphInstantiate(&b->graph, g, 0);
        cudaGraphDestroy(g);
        BCK(e);
        b->graph_launches = n;
      }
      BCK(cudaGraphLaunch(b->graph, s));
      launches += b->graph_launches;
      ++cycles;
    }
    kb_unpack<<<rows_grid, 256, 0, s>>>(b->X, b->stage, b->N, b->tile_sys, b->sd, b->soff);
    BCK(cudaGetLastError());
    BCK(cudaMemcpyAsync(Xio, b->stage, bytes, cudaMemcpyDefault, s));
    BCK(cudaEventRecord(b->ev, s));
    BCK(cudaStreamWaitEvent(b->user_stream, b->ev, 0));
    BCK(cudaStreamSynchronize(s));
    if (stats) {
      gmres_batch_stats_t& S = *stats;
      S.status = status;
      S.cycles = cycles;
      S.kernel_launches = launches + 1;   // + the unpack kernel
      for (int i = 0; i < 4; ++i) {
        S.t_kernel[i] = tk[i];
        S.class_launches[i] = cl[i];
      }
      S.solve_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      S.max_rel_res = 0.0;
      S.converged_systems = 0;
      S.block_steps = 0;
      S.breakdowns = 0;
      for (int i = 0; i < b->nsys; ++i) {
        const SysState& x = b->st_host[i];
        for (int c = 0; c < kP; ++c) S.max_rel_res = std::max(S.max_rel_res, x.rel[c]);
        S.converged_systems += x.done ? 1 : 0;
        S.block_steps += x.iters;
        S.breakdowns += x.breakdowns >= kTimeoutMark ? 0 : x.breakdowns;
        if (S.per_system_rel && i < S.per_system_cap) {
          double mx = 0.0;
          for (int c = 0; c < kP; ++c) mx = std::max(mx, x.rel[c]);
          S.per_system_rel[i] = mx;
        }
        if (S.per_system_cycles && i < S.per_system_cap) S.per_system_cycles[i] = x.cycles;
      }
    }
  });
  if (rc != GMRES_OK) {
    if (stats) stats->status = rc;
    return rc;
  }
  return status;
}

int gmres_batch_autotune(gmres_batch_t b, const double* Bin, double tol, int max_cycles,
                         gmres_batch_tuning_t* best, double* best_seconds, double* default_seconds) {
  if (!b || !Bin || !(tol >= 0.0) || max_cycles < 1) return GMRES_ERR_INVALID_ARG;
  const gmres_batch_tuning_t saved = b->tuning;
  const int saved_prof = b->profiling;
  b->profiling = 0;
  double* X = nullptr;
  const size_t bytes = (size_t)b->total_n * kP * sizeof(double);
  gmres_batch_tuning_t chosen = saved;
  double t_best = 0.0, t_default = 0.0;
  int rc = brun([&] { BCK(cudaMalloc(&X, bytes)); });
  static const int chunk[] = {0, 8, 32};
  static const int pipe[][2] = {{0, 0}, {100, 4}, {220, 8}};   // {smem budget KB, stage cap}
  bool have = false;
  for (int c : chunk) {
    for (const auto& p : pipe) {
      if (rc != GMRES_OK) break;
      const gmres_batch_tuning_t cand{c, p[0], p[1], 0};
      rc = gmres_batch_set_tuning(b, &cand);
      if (rc != GMRES_OK) break;
      double el = 0.0;
      for (int rep = 0; rep < 2 && rc == GMRES_OK; ++rep) {   // rep 0 captures the graph
        rc = brun([&] { BCK(cudaMemsetAsync(X, 0, bytes, b->stream)); });
        if (rc != GMRES_OK) break;
        gmres_batch_stats_t st{};
        const int r = gmres_batch_ir_solve(b, Bin, X, tol, rep == 0 ? 1 : max_cycles, &st);
        if (r < 0) rc = r;
        el = st.solve_seconds;
      }
      if (rc != GMRES_OK) break;
      if (c == 0 && p[0] == 0 && p[1] == 0) t_default = el;
      if (!have || el < t_best) {
        have = true;
        t_best = el;
        chosen = cand;
      }
    }
  }
  if (X) cudaFree(X);
  b->profiling = saved_prof;
  const int rc2 = gmres_batch_set_tuning(b, rc == GMRES_OK ? &chosen : &saved);
  if (rc != GMRES_OK) return rc;
  if (rc2 != GMRES_OK) return rc2;
  if (best) *best = chosen;
  if (best_seconds) *best_seconds = t_best;
  if (default_seconds) *default_seconds = t_default;
  return GMRES_OK;
}

}  // extern "C"
