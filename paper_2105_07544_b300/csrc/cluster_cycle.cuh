// One GMRES restart cycle of a small system in one thread-block cluster (sm_90+ clusters with
// distributed shared memory).
//
// A system whose Krylov basis fits in the shared memory of the cluster's CTAs (up to 16 CTAs of
// 256 threads, 256 or 512 rows each) runs a whole cycle -- the m Arnoldi steps with CGS2
// (Section III-A), the Givens least squares, x += V y and the FP64 residual of the next cycle
// (Algorithm 2 for GMRES-IR, Algorithm 1 for FP64 GMRES) -- in one launch.  The per-step kernels
// pay a launch, a pipeline fill and a two-level cross-CTA sum through global memory several
// times per step; here each CTA keeps its rows of the matrix and of every basis column in shared
// memory, the SpMV reads the other CTAs' rows of the current column through distributed shared
// memory, and every global reduction is one cluster barrier: each CTA writes its partial sums to
// its own shared memory, and after the barrier every CTA adds all CTAs' partials in rank order,
// so the sums (and every decision taken from them) are the same in every CTA without a second
// barrier.
//
// Every CTA runs the same number of cluster barriers whatever the data: 3 per step for the
// cycle's jmax steps (a stopped cycle skips the work, not the barriers), then 3 at the cycle end.
// A ninth warp takes the FP64 Givens chain off the row warps' path (B300's FP64 unit makes each
// dependent FP64 operation cost on the order of a hundred cycles): it arrives at a step's first
// barrier early and rotates the previous column while the row warps work, so the decision to stop
// reaches them one barrier later; the work they start meanwhile is discarded if the cycle stopped
// (only the first k columns and the first k rotations are ever used).
//
// Arithmetic is that of the per-step kernels: the inner SpMV w = s_j A V_j sums in ACC and then
// scales; projections accumulate in ACC within a CTA and in FP64 across CTAs (fixed order);
// w' = w - V (s h1), w'' = w' - V (s h2) in ACC, column by column; H[:, j] = h1 + h2 and the
// Givens rotation, stop tests and state bookkeeping as in the update sweep's last CTA; the
// solution update accumulates V (s y) in FP64; the residual r = b - A x in FP64 with the FP64
// values, stored as TV in column 0 with s_0 = 1 / ||TV(r)||.
#pragma once

#include "kernels.cuh"

namespace gmresb3 {

constexpr int kClusterMax = 16;   // CTAs (non-portable cluster size; 8 is the portable limit)

__device__ __forceinline__ void cluster_arrive() {
  asm volatile("barrier.cluster.arrive.release;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() {
  asm volatile("barrier.cluster.wait.acquire;" ::: "memory");
}
__device__ __forceinline__ void cluster_barrier() {
  cluster_arrive();
  cluster_wait();
}
__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
// Generic address of the same shared-memory location in CTA `rank` of the cluster.
template <typename T> __device__ __forceinline__ T* dsmem_ptr(T* p, unsigned rank) {
  uint64_t out;
  asm volatile("mapa.u64 %0, %1, %2;" : "=l"(out) : "l"(p), "r"(rank));
  return reinterpret_cast<T*>(out);
}

struct ClusterShape {
  int n;        // rows
  int nctas;    // CTAs of the cluster (= grid)
  int mcap;     // columns of the shared basis: mcap + 1
  int nnzcap;   // staged nonzeros per CTA (the most in one block of RS rows)
  long vts;     // tile stride of the global tile-blocked basis
};

// Threads: 8 row warps (kThreads, one or two rows each) and one scalar warp that runs the
// Givens chain of step j while the row warps start step j + 1.
constexpr int kClusterThreads = kThreads + 32;

// Shared-memory layout (bytes from the dynamic base), RS = kThreads * RPT rows per CTA.
template <typename TA, typename TV, typename ACC, int RPT> struct ClusterSmem {
  static constexpr int RS = kThreads * RPT;
  static __host__ __device__ size_t slots(int mcap) { return (size_t)mcap + 4; }
  static __host__ __device__ size_t x_off(int mcap) {
    return align16((size_t)(mcap + 1) * RS * sizeof(TV));
  }
  static __host__ __device__ size_t part_off(int mcap) { return x_off(mcap) + (size_t)RS * 8; }
  static __host__ __device__ size_t red_off(int mcap) {
    return part_off(mcap) + 3 * slots(mcap) * 8;
  }
  static __host__ __device__ size_t small_off(int mcap) {
    return align16(red_off(mcap) + (size_t)kWarps * slots(mcap) * sizeof(ACC));
  }
  // small: h1, h2, s, g, cs, sn, c, col, coef1, coef2 (slots each) + R ((mcap + 1) x mcap)
  static __host__ __device__ size_t csr_off(int mcap) {
    return align16(small_off(mcap) + (10 * slots(mcap) + (size_t)(mcap + 1) * mcap) * 8);
  }
  // staged CSR rows: local row offsets (RS + 1), column indices, values
  static __host__ __device__ size_t col_off(int mcap) {
    return align16(csr_off(mcap) + (size_t)(RS + 1) * 4);
  }
  static __host__ __device__ size_t val_off(int mcap, int nnzcap) {
    return align16(col_off(mcap) + (size_t)nnzcap * 4);
  }
  static __host__ __device__ size_t bytes(int mcap, int nnzcap) {
    return val_off(mcap, nnzcap) + (size_t)nnzcap * sizeof(TA) + 64;
  }
};

// Barrier of the 8 row warps only (named barrier 1): the scalar warp runs on meanwhile.
__device__ __forceinline__ void row_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kThreads) : "memory"); }

template <typename T> __device__ __forceinline__ T row_block_sum(T v, T* red /* kWarps */) {
  v = warp_sum(v);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  row_sync();
  if (l == 0) red[w] = v;
  row_sync();
  T s = 0;
#pragma unroll
  for (int i = 0; i < kWarps; ++i) s += red[i];
  return s;
}

// Row warps: block sums of the ncols column products p_i = sum over the thread's rows of
// V_i[r] w[r] (16-column batches, summed over each warp by a reduce-scatter), per warp in
// red[warp][i]; then thread i <= ncols adds the warps in order into part[i] (FP64); slot ncols
// takes the sum of `extra`.
template <typename ACC, typename TV, int RPT>
__device__ __forceinline__ void cluster_project(const TV* __restrict__ Vs, const ACC (&w)[RPT],
                                                int ncols, ACC extra, ACC* __restrict__ red,
                                                double* __restrict__ part, int nslot_ld) {
  constexpr int RS = kThreads * RPT;
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  const int nb = (ncols + 15) >> 4;
  for (int q = 0; q < nb; ++q) {
    ACC p[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      const int c = 16 * q + k;
      ACC s = 0;
      if (c < ncols) {
#pragma unroll
        for (int u = 0; u < RPT; ++u) s += cv<ACC>(Vs[(size_t)c * RS + t + kThreads * u]) * w[u];
      }
      p[k] = s;
    }
    const ACC tot = reduce_scatter16(p);
    const int c = 16 * q + (lane >> 1);
    if ((lane & 1) == 0 && c < ncols) red[wid * nslot_ld + c] = tot;
  }
  const ACC e = warp_sum(extra);
  if (lane == 0) red[wid * nslot_ld + ncols] = e;
  row_sync();
  for (int i = t; i <= ncols; i += kThreads) {
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kWarps; ++k) s += (double)red[k * nslot_ld + i];
    part[i] = s;
  }
}

// Sum over the cluster's CTAs of slot i of part: all loads in flight, then a fixed pairwise tree
// (ranks past nctas add zero), so every CTA gets the same value from a short dependent chain.
__device__ __forceinline__ double cluster_slot_sum(double* part, int i, int nctas) {
  double v[kClusterMax];
#pragma unroll
  for (int r = 0; r < kClusterMax; ++r) v[r] = (r < nctas) ? *dsmem_ptr(part + i, (unsigned)r) : 0.0;
#pragma unroll
  for (int w = 1; w < kClusterMax; w *= 2) {
#pragma unroll
    for (int r = 0; r + w < kClusterMax; r += 2 * w) v[r] += v[r + w];
  }
  return v[0];
}

template <typename TA, typename TV, typename ACC, int RPT>
__global__ void __launch_bounds__(kClusterThreads, 1)
    k_cycle_cluster(Csr<TA> A, Csr<double> A64, const double* __restrict__ b,
                    double* __restrict__ x, TV* __restrict__ Vg, Krylov K, ClusterShape cs) {
  using L = ClusterSmem<TA, TV, ACC, RPT>;
  constexpr int RS = L::RS;
  constexpr int kRsShift = (RPT == 1) ? 8 : 9;   // log2(RS)
  static_assert(RS == (1 << kRsShift), "rows per CTA");
  extern __shared__ __align__(128) unsigned char smem[];
  const int mcap = cs.mcap;
  const int nsl = (int)L::slots(mcap);
  TV* Vs = (TV*)smem;
  double* xs = (double*)(smem + L::x_off(mcap));
  double* part = (double*)(smem + L::part_off(mcap));   // 3 buffers of nsl slots
  ACC* red = (ACC*)(smem + L::red_off(mcap));
  double* sm = (double*)(smem + L::small_off(mcap));
  double* h1 = sm;
  double* h2 = h1 + nsl;
  double* sc = h2 + nsl;       // column scales s_i
  double* g = sc + nsl;
  double* rc = g + nsl;        // Givens cosines
  double* rsn = rc + nsl;      // Givens sines
  double* cy = rsn + nsl;      // solution coefficients s_i y_i
  double* col = cy + nsl;      // the scalar warp's working column; col[nsl - 1]: ||A z_j||^2
  ACC* coef1 = (ACC*)(col + nsl);
  ACC* coef2 = (ACC*)(col + 2 * nsl);
  double* Rm = col + 3 * nsl;  // rotated Hessenberg columns, column j at Rm[j (mcap + 1)]
  int* rp_s = (int*)(smem + L::csr_off(mcap));
  int* col_s = (int*)(smem + L::col_off(mcap));
  TA* val_s = (TA*)(smem + L::val_off(mcap, cs.nnzcap));
  // stop flags, cumulative over the cycle's steps: flag[j & 1] = stopped at or before step j
  // (the scalar warp writes one slot while the row warps read the other)
  __shared__ int s_flag[2], s_k, s_reason;
  __shared__ double s_implicit, s_red[kWarps];

  CycleState* st = K.st;
  const int t = threadIdx.x, lane = t & 31;
  const bool row_thread = t < kThreads;            // warp-uniform
  const unsigned rank = cluster_rank();
  const int n = cs.n, nctas = cs.nctas;
  const long row0 = (long)rank * RS;
  const int nrows = (int)max(0L, min((long)RS, (long)n - row0));
  const bool leader = rank == 0;

  // ---- cycle state, column 0 (written by the previous residual) and this CTA's matrix rows ----
  const int jmax = st->jmax;
  const int implicit_fp64 = st->implicit_fp64;
  const double uround = st->uround, tol = st->tol, bnorm = st->bnorm;
  const double inner_tol = st->inner_tol, gamma = st->gamma;
  if (t == 0) {
    s_flag[0] = s_flag[1] = st->stop;
    s_k = 0;
    s_reason = 0;
    s_implicit = st->implicit;
  }
  for (int i = t; i < nsl; i += kClusterThreads) {
    sc[i] = (i == 0) ? K.s[0] : 0.0;
    g[i] = (i == 0) ? K.g[0] : 0.0;
  }
  const int base = (nrows > 0) ? __ldg(A.rowptr + row0) : 0;
  const int lnnz = (nrows > 0) ? __ldg(A.rowptr + row0 + nrows) - base : 0;
  for (int i = t; i <= RS; i += kClusterThreads)
    rp_s[i] = (i <= nrows) ? __ldg(A.rowptr + row0 + i) - base : lnnz;
  for (int p = t; p < lnnz; p += kClusterThreads) {
    col_s[p] = __ldg(A.col + base + p);
    val_s[p] = A.val[base + p];
  }
  if (row_thread) {
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const long r = row0 + t + kThreads * u;
      Vs[t + kThreads * u] = (r < n) ? Vg[(size_t)(r >> kTileShift) * cs.vts + (r & (kTile - 1))]
                                     : cv<TV>(0.0);
    }
  }
  cluster_barrier();   // every CTA's column 0 and staged rows are in place
  if (!row_thread && jmax > 0) cluster_arrive();                      // (1) of step 0

  // ---- the Arnoldi steps: 3 cluster barriers each, jmax steps whatever the data ----
  for (int j = 0; j < jmax; ++j) {
    const int ncols = j + 1;
    double* p1 = part;
    double* p2 = part + nsl;
    double* p3 = part + 2 * nsl;
    if (row_thread) {
      // the decision of step j - 1 may still be in the making: start if nothing stopped by j - 2
      const bool pre = s_flag[j & 1] == 0;   // slot (j - 2) & 1
      ACC w[RPT];
      if (pre) {
        ACC az = 0;
        const ACC scale = (ACC)sc[j];
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
          const int lr = t + kThreads * u;
          ACC s = 0;
          if (lr < nrows) {
            const int a = rp_s[lr], e = rp_s[lr + 1];
            for (int p = a; p < e; ++p) {
              const int c = col_s[p];
              const TV* src = dsmem_ptr(Vs + (size_t)j * RS + (c & (RS - 1)), (unsigned)(c >> kRsShift));
              s += cv<ACC>(val_s[p]) * cv<ACC>(*src);
            }
          }
          w[u] = s * scale;
          az += w[u] * w[u];
        }
        cluster_project<ACC, TV, RPT>(Vs, w, ncols, az, red, p1, nsl);
      }
      cluster_barrier();                                              // (1) first projection
      if (pre) {   // (speculative: the decision of step j - 1 is read after barrier (2))
        for (int i = t; i <= ncols; i += kThreads) {
          const double v = cluster_slot_sum(p1, i, nctas);
          if (i < ncols) {
            h1[i] = sc[i] * v;
            coef1[i] = (ACC)(sc[i] * h1[i]);
          } else {
            col[nsl - 1] = v;                                          // ||A z_j||^2
          }
        }
        row_sync();
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
          ACC s = 0;
          for (int i = 0; i < ncols; ++i) s += cv<ACC>(Vs[(size_t)i * RS + t + kThreads * u]) * coef1[i];
          w[u] -= s;                                                   // w' = w - V (s h1)
        }
        cluster_project<ACC, TV, RPT>(Vs, w, ncols, ACC(0), red, p2, nsl);
      }
      cluster_barrier();                                              // (2) second projection
      const bool active = pre && s_flag[(j + 1) & 1] == 0;            // slot (j - 1) & 1
      if (active) {
        for (int i = t; i < ncols; i += kThreads) {
          h2[i] = sc[i] * cluster_slot_sum(p2, i, nctas);
          coef2[i] = (ACC)(sc[i] * h2[i]);
        }
        row_sync();
        ACC q2 = 0;
#pragma unroll
        for (int u = 0; u < RPT; ++u) {
          ACC s = 0;
          for (int i = 0; i < ncols; ++i) s += cv<ACC>(Vs[(size_t)i * RS + t + kThreads * u]) * coef2[i];
          const bool in = t + kThreads * u < nrows;
          const TV qv = cv<TV>(w[u] - s);                              // v_{j+1} = w'' unscaled
          Vs[(size_t)ncols * RS + t + kThreads * u] = in ? qv : cv<TV>(0.0);
          const ACC qa = in ? cv<ACC>(qv) : ACC(0);
          q2 += qa * qa;
        }
        const double nb = (double)row_block_sum(q2, (ACC*)s_red);
        if (t == 0) p3[0] = nb;
      }
      cluster_barrier();                                              // (3) norm of w''
      if (active && t == 0) sc[ncols] = 1.0 / sqrt(cluster_slot_sum(p3, 0, nctas));
      row_sync();                                                      // s_{j+1} for step j + 1
    } else {
      // ---- scalar warp: step j's barriers, then the Hessenberg column j, its Givens rotation
      // and the stop tests.  It takes what it needs from the row warps (the norm's partials, h1,
      // h2, ||A z_j||) before arriving at barrier (1) of step j + 1, and runs the rotation chain
      // between that arrival and its wait, while the row warps compute step j + 1; its decision
      // is read by them after barrier (2) of step j + 1.
      cluster_wait();                                                 // (1), arrived earlier
      cluster_arrive();
      cluster_wait();                                                 // (2)
      cluster_arrive();
      cluster_wait();                                                 // (3)
      const bool active = s_flag[(j + 1) & 1] == 0;                   // stopped by step j - 1?
      double qn = 0.0, az2 = 0.0;
      if (active) {
        qn = sqrt(cluster_slot_sum(p3, 0, nctas));
        az2 = col[nsl - 1];
        for (int i = lane; i <= j; i += 32) col[i] = h1[i] + h2[i];
      }
      __syncwarp();
      if (j + 1 < jmax) cluster_arrive();                              // (1) of step j + 1
      int stop_now = active ? 0 : 1;
      if (active) {
        const double hn = qn;
        if (leader) {
          const int m1 = K.m + 1;
          for (int i = lane; i <= j; i += 32) K.H[(size_t)j * m1 + i] = col[i];
          if (lane == 0) K.H[(size_t)j * m1 + j + 1] = hn;
        }
        __syncwarp();
        // the earlier rotations applied to column j by the whole warp (givens_apply_warp)
        double xr = givens_apply_warp(col, rc, rsn, j);
        if (lane == 0) {
          const double gj = g[j];
          const double r = givens_radius(xr, hn);
          double c = 1.0, sgn = 0.0;
          if (r != 0.0) {
            const double ir = 1.0 / r;
            c = xr * ir;
            sgn = hn * ir;
          }
          rc[j] = c;
          rsn[j] = sgn;
          col[j] = r;
          col[j + 1] = 0.0;
          g[j + 1] = -sgn * gj;
          g[j] = c * gj;
          const double imp = fabs(sgn * gj);
          int reason = 0;
          if (!finite_d(hn) || !finite_d(imp) || !finite_d(r)) {
            reason = 3;
          } else if (hn <= 10.0 * uround * sqrt(az2)) {
            reason = 2;
          } else {
            const double thr = implicit_fp64 ? tol * bnorm : inner_tol * gamma;
            if (imp <= thr) reason = 1;
            else if (j + 1 >= jmax) reason = 4;
          }
          s_implicit = imp;
          s_k = j + 1;
          if (reason) {
            s_reason = reason;
            stop_now = 1;
          }
          if (leader) {
            K.cs[j] = c;
            K.sn[j] = sgn;
            K.g[j] = g[j];
            K.g[j + 1] = g[j + 1];
            K.s[j + 1] = 1.0 / qn;
            st->implicit = imp;
            st->k = j + 1;
            if (reason == 3) st->nan = 1;
            if (reason == 2) st->breakdowns += 1;
            if (reason) {
              st->reason = reason;
              st->stop = 1;
            }
          }
        }
        __syncwarp();
        for (int i = lane; i <= j + 1; i += 32) Rm[(size_t)j * (mcap + 1) + i] = col[i];
        stop_now = __shfl_sync(0xffffffffu, stop_now, 0);
      }
      if (lane == 0) s_flag[j & 1] = stop_now;   // read by the row warps after barrier (2) of j + 1
      __syncwarp();
    }
  }
  __syncthreads();   // the scalar warp's last column is done

  // ---- cycle end: y = R^{-1} g (scalar warp), x += V (s y) (row warps) ----
  const int k = s_k;
  if (!row_thread) {
    // column-oriented back substitution by one warp (the order of the per-step solve kernel)
    for (int i = lane; i < k; i += 32) col[i] = g[i];
    __syncwarp();
    for (int i = k - 1; i >= 0; --i) {
      const double yi = col[i] / Rm[(size_t)i * (mcap + 1) + i];
      __syncwarp();
      for (int r = lane; r < i; r += 32) col[r] -= Rm[(size_t)i * (mcap + 1) + r] * yi;
      if (lane == 0) {
        cy[i] = sc[i] * yi;
        if (leader) K.c[i] = cy[i];
      }
      __syncwarp();
    }
  }
  __syncthreads();
  if (row_thread) {
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const long r = row0 + t + kThreads * u;
      double xv = 0.0;
      if (r < n) {
        xv = x[r];
        if (k > 0) {
          double s = 0.0;
          for (int i = 0; i < k; ++i) s += cy[i] * cv<double>(Vs[(size_t)i * RS + t + kThreads * u]);
          xv += s;
          x[r] = xv;
        }
      }
      xs[t + kThreads * u] = xv;
    }
  }
  cluster_barrier();                                                // (4) x in place

  // ---- FP64 residual of the next cycle: r = b - A x, column 0 = TV(r) ----
  if (row_thread) {
    double r2 = 0.0, q2 = 0.0;
#pragma unroll
    for (int u = 0; u < RPT; ++u) {
      const long r = row0 + t + kThreads * u;
      if (r < n) {
        const int a = __ldg(A64.rowptr + r), e = __ldg(A64.rowptr + r + 1);
        double ax = 0.0;
        for (int p = a; p < e; ++p) {
          const int c = __ldg(A64.col + p);
          ax += A64.val[p] * *dsmem_ptr(xs + (c & (RS - 1)), (unsigned)(c >> kRsShift));
        }
        const double rr = b[r] - ax;
        r2 += rr * rr;
        const TV q = cv<TV>(rr);
        const double qd = cv<double>(q);
        q2 += qd * qd;
        Vg[(size_t)(r >> kTileShift) * cs.vts + (r & (kTile - 1))] = q;
      }
    }
    const double r2b = row_block_sum(r2, s_red);
    const double q2b = row_block_sum(q2, s_red);
    if (t == 0) {
      part[0] = r2b;
      part[1] = q2b;
    }
  }
  cluster_barrier();                                                // (5) residual norms
  if (t == 0) {
    const double r2t = cluster_slot_sum(part, 0, nctas);
    const double q2t = cluster_slot_sum(part, 1, nctas);
    if (leader) {
      const double rel = sqrt(r2t) / bnorm;
      const double gam = sqrt(q2t);
      st->last_k = k;
      st->last_reason = s_reason;
      st->last_implicit = s_implicit;
      if (implicit_fp64 && s_reason == 1 && !(rel <= tol)) st->loa += 1;
      st->rel_res = rel;
      st->gamma = gam;
      st->converged = (rel <= tol) ? 1 : 0;
      if (!finite_d(rel) || !finite_d(gam)) st->nan = 1;
      K.s[0] = 1.0 / gam;
      K.g[0] = gam;
      st->k = 0;
      st->reason = 0;
      st->implicit = gam;
      st->stop = (st->converged || st->nan || gam == 0.0) ? 1 : 0;
    }
  }
  cluster_barrier();   // (6) no CTA leaves while another still reads its shared memory
}

}  // namespace gmresb3
