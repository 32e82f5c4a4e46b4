// Learned GMRES-IR parameter controller for C callers (include/gmresb3.h, gmres_controller_*).
//
// The paper picks the restart length (Section V-E), the inner tolerance and the polynomial
// degree (Section V-F) by hand.  This file gives C callers the trained network's choice:
//   gmres_controller_load     : read a CRC32-checked checkpoint (network parameters, feature
//                               standardisation, and in version 2 the best fixed setting of the
//                               training sweep); the network lives in an MLP context on the GPU
//   gmres_controller_features : the 12 features of a system, on the GPU: one pass of a row kernel
//                               over the handle's CSR (sizes, diagonal dominance, nonsymmetry,
//                               upwind strength, Gershgorin bounds), a 10-step FP64 Arnoldi run
//                               and one timed default GMRES-IR cycle on a temporary handle
//   gmres_controller_decide   : network forward pass (the library's MLP kernels) and the rule
//                               that falls back to the default or to the best fixed setting
//   gmres_controller_suggest  : features, then decide
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gmresb3.h"
#include "handle_view.h"
#include "poly_host.h"

namespace {

constexpr int kFeat = 12;
constexpr int kOut = 9;
constexpr int kMClass[3] = {25, 50, 100};
constexpr int kDClass[4] = {0, 10, 25, 40};
constexpr int kDefaultM = 50;
constexpr double kFallbackRatio = 0.95;

// CRC-32 (the reflected polynomial 0xEDB88320, initial value and final xor 0xFFFFFFFF), as in
// zlib and PNG; table built once.
uint32_t crc32_of(const unsigned char* p, size_t n) {
  static uint32_t table[256];
  static bool ready = false;
  if (!ready) {
    for (uint32_t i = 0; i < 256; ++i) {
      uint32_t c = i;
      for (int k = 0; k < 8; ++k) c = (c & 1u) ? 0xEDB88320u ^ (c >> 1) : (c >> 1);
      table[i] = c;
    }
    ready = true;
  }
  uint32_t c = 0xFFFFFFFFu;
  for (size_t i = 0; i < n; ++i) c = table[(c ^ p[i]) & 0xFFu] ^ (c >> 8);
  return c ^ 0xFFFFFFFFu;
}

template <typename T> T read_le(const unsigned char* p) {
  T v;
  std::memcpy(&v, p, sizeof(T));   // the checkpoint is little-endian, like every CUDA host
  return v;
}

// ---- row features ------------------------------------------------------------------------------
// Per CTA, over its rows (grid-stride): [0] sum of nonzeros, [1] max nonzeros per row,
// [2] min |a_ii| / sum_{j != i} |a_ij|, [3] sum |a_ii|, [4] min (a_ii - off_i), [5] max (a_ii +
// off_i), [6] sum a_ij^2, [7] sum over stored (i, j) of the (A - A^T) entries it accounts for
// (d^2 with d = a_ij - a_ji when (j, i) is stored, 2 a_ij^2 otherwise), [8] max |d|.
constexpr int kRowStats = 9;

__global__ void __launch_bounds__(256) k_row_features(int n, const int* __restrict__ rp,
                                                      const int* __restrict__ ci,
                                                      const double* __restrict__ va,
                                                      double* __restrict__ part) {
  double s_cnt = 0, m_cnt = 0, m_dom = INFINITY, s_dg = 0, m_gmin = INFINITY, m_gmax = -INFINITY;
  double s_f2 = 0, s_d2 = 0, m_d = 0;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const int a = rp[i], e = rp[i + 1];
    double diag = 0, off = 0;
    for (int p = a; p < e; ++p) {
      const int j = ci[p];
      const double v = va[p];
      s_f2 += v * v;
      if (j == i) {
        diag += v;
        continue;
      }
      off += fabs(v);
      double vt = 0;
      bool found = false;
      for (int q = rp[j]; q < rp[j + 1]; ++q)
        if (ci[q] == (int)i) {
          vt += va[q];
          found = true;
        }
      const double d = v - vt;
      s_d2 += found ? d * d : 2.0 * v * v;
      m_d = fmax(m_d, fabs(d));
    }
    s_cnt += e - a;
    m_cnt = fmax(m_cnt, (double)(e - a));
    m_dom = fmin(m_dom, fabs(diag) / fmax(off, 1e-300));
    s_dg += fabs(diag);
    m_gmin = fmin(m_gmin, diag - off);
    m_gmax = fmax(m_gmax, diag + off);
  }
  double v[kRowStats] = {s_cnt, m_cnt, m_dom, s_dg, m_gmin, m_gmax, s_f2, s_d2, m_d};
  __shared__ double red[kRowStats][8];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int k = 0; k < kRowStats; ++k) {
    double x = v[k];
    for (int o = 16; o > 0; o >>= 1) {
      const double y = __shfl_xor_sync(0xffffffffu, x, o);
      x = (k == 2 || k == 4) ? fmin(x, y) : (k == 1 || k == 5 || k == 8) ? fmax(x, y) : x + y;
    }
    if (lane == 0) red[k][w] = x;
  }
  __syncthreads();
  if (threadIdx.x < kRowStats) {
    const int k = threadIdx.x;
    double x = red[k][0];
    for (int q = 1; q < (int)(blockDim.x / 32); ++q) {
      const double y = red[k][q];
      x = (k == 2 || k == 4) ? fmin(x, y) : (k == 1 || k == 5 || k == 8) ? fmax(x, y) : x + y;
    }
    part[(size_t)k * gridDim.x + blockIdx.x] = x;
  }
}

struct Fail {
  int code;
};
#define CC(call)                                                        \
  do {                                                                  \
    const cudaError_t e_ = (call);                                      \
    if (e_ != cudaSuccess) {                                            \
      cudaGetLastError();                                               \
      throw Fail{e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA}; \
    }                                                                   \
  } while (0)
#define CG(call)                                \
  do {                                          \
    const int r_ = (call);                      \
    if (r_ < 0) throw Fail{r_};                 \
  } while (0)

template <typename T> struct DevBuf {
  T* p = nullptr;
  explicit DevBuf(size_t n) { CC(cudaMalloc(&p, std::max<size_t>(n, 1) * sizeof(T))); }
  ~DevBuf() { cudaFree(p); }
};

struct TempHandle {
  gmres_handle_t h = nullptr;
  ~TempHandle() { gmres_destroy(h); }
};

void compute_features(gmres_handle_t h, const double* b, double* f) {
  const gmresb3::HandleView M = gmresb3::handle_view(h);
  const int n = (int)M.n;
  int prev = -1;
  CC(cudaGetDevice(&prev));
  if (prev != M.dev) CC(cudaSetDevice(M.dev));
  struct Restore {
    int d, cur;
    ~Restore() {
      if (d != cur) cudaSetDevice(d);
    }
  } restore{prev, M.dev};
  cudaStream_t s = (cudaStream_t)M.user_stream;
  // (1) row statistics of the handle's FP64 matrix
  const int grid = std::max(1, std::min(M.sms * 4, (n + 255) / 256));
  DevBuf<double> part((size_t)kRowStats * grid);
  k_row_features<<<grid, 256, 0, s>>>(n, M.rowptr, M.col, M.val, part.p);
  CC(cudaGetLastError());
  std::vector<double> hp((size_t)kRowStats * grid);
  CC(cudaMemcpyAsync(hp.data(), part.p, hp.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
  CC(cudaStreamSynchronize(s));
  double st[kRowStats];
  for (int k = 0; k < kRowStats; ++k) {
    double x = hp[(size_t)k * grid];
    for (int g = 1; g < grid; ++g) {
      const double y = hp[(size_t)k * grid + g];
      x = (k == 2 || k == 4) ? std::min(x, y) : (k == 1 || k == 5 || k == 8) ? std::max(x, y) : x + y;
    }
    st[k] = x;
  }
  double dscale = st[3] / n;
  if (!(dscale > 0.0)) dscale = 1.0;
  const double pe = st[8] / dscale;
  f[0] = std::log10((double)n);
  f[1] = st[0] / n;
  f[2] = st[1];
  f[3] = st[2];
  f[4] = std::sqrt(st[7]) / std::max(std::sqrt(st[6]), 1e-300);
  f[5] = std::log10(pe + 1e-12);
  f[6] = st[4] / dscale;
  f[7] = st[5] / dscale;
  // (2) a temporary handle with the default parameters (FP32 basis, m = 50, no polynomial)
  DevBuf<double> bd(n), xd(n);
  CC(cudaMemcpyAsync(bd.p, b, (size_t)n * sizeof(double), cudaMemcpyDefault, s));
  CC(cudaStreamSynchronize(s));
  gmres_csr_t csr{M.n, M.nnz, M.rowptr, M.col, M.val, 1};
  const gmres_precisions_t prec{GMRES_F32, GMRES_F32, GMRES_F32, GMRES_F32};
  TempHandle T;
  CG(gmres_create(&csr, kDefaultM, 0, prec, nullptr, &T.h));
  CG(gmres_set_stream(T.h, M.user_stream));
  // 10-step FP64 Arnoldi from b: the extreme Ritz values (eigenvalues of H_k)
  const int k = n > 1 ? std::min(10, n - 1) : 1;
  std::vector<double> H((size_t)(k + 1) * k);
  int steps = 0;
  CG(gmres_arnoldi(T.h, GMRES_F64, k, bd.p, H.data(), nullptr, &steps));
  const int kk = std::max(1, steps);
  std::vector<std::complex<double>> ev;
  if (!gmresb3::hessenberg_eigvals(kk, H.data(), k + 1, ev)) throw Fail{GMRES_ERR_INVALID_ARG};
  double emax = 0.0, emin = INFINITY;
  for (const auto& z : ev) {
    emax = std::max(emax, std::abs(z));
    emin = std::min(emin, std::abs(z));
  }
  f[8] = emax / dscale;
  f[9] = emin / dscale;
  // one default GMRES-IR cycle: the first run captures the cycle graph, the second is timed
  gmres_params_t P;
  gmres_default_params(&P);
  P.maxiter = kDefaultM;
  CG(gmres_set_params(T.h, &P));
  double hist[4] = {0, 0, 0, 0};
  gmres_stats_t S{};
  S.res_history = hist;
  S.res_history_cap = 4;
  CC(cudaMemsetAsync(xd.p, 0, (size_t)n * sizeof(double), s));
  CG(gmres_ir_solve(T.h, bd.p, xd.p, 1e-10, &S));
  CC(cudaMemsetAsync(xd.p, 0, (size_t)n * sizeof(double), s));
  CC(cudaStreamSynchronize(s));
  S = gmres_stats_t{};
  S.res_history = hist;
  S.res_history_cap = 4;
  const auto t0 = std::chrono::steady_clock::now();
  CG(gmres_ir_solve(T.h, bd.p, xd.p, 1e-10, &S));
  CC(cudaStreamSynchronize(s));
  const double el = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  const double drop = (S.res_history_len > 1 && hist[0] > 0.0) ? hist[1] / hist[0] : 1.0;
  f[10] = std::log10(std::max(drop, 1e-30));
  f[11] = std::log10(std::max(el, 1e-6));
}

template <class F> int guarded(F fn) {
  try {
    fn();
    return GMRES_OK;
  } catch (const Fail& e) {
    return e.code;
  } catch (const std::bad_alloc&) {
    return GMRES_ERR_OOM;
  } catch (...) {
    return GMRES_ERR_CUDA;
  }
}

}  // namespace

struct gmres_ctrl_ctx {
  gmres_mlp_t net = nullptr;
  double mean[kFeat], std_[kFeat];
  int has_fixed = 0;            // version 2: the best fixed setting of the training sweep
  int fixed_m = 0, fixed_d = 0;
  double fixed_tol = 0.0, fixed_ratio = 0.0;
  ~gmres_ctrl_ctx() { gmres_mlp_destroy(net); }
};

extern "C" {

int gmres_controller_load(const char* path, gmres_ctrl_t* out) {
  if (!path || !out) return GMRES_ERR_INVALID_ARG;
  *out = nullptr;
  std::vector<unsigned char> raw;
  {
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return GMRES_ERR_INVALID_ARG;
    unsigned char buf[65536];
    size_t got;
    while ((got = std::fread(buf, 1, sizeof(buf), fp)) > 0) raw.insert(raw.end(), buf, buf + got);
    std::fclose(fp);
  }
  const int np = gmres_mlp_num_params();
  const size_t base = 8 + 8 + 2 * kFeat * 8 + (size_t)np * 4;   // magic .. parameters
  if (raw.size() < base + 4 || std::memcmp(raw.data(), "GMRESMLP", 8) != 0)
    return GMRES_ERR_INVALID_ARG;
  const unsigned char* body = raw.data() + 8;
  const size_t body_len = raw.size() - 12;
  if (crc32_of(body, body_len) != read_le<uint32_t>(raw.data() + raw.size() - 4))
    return GMRES_ERR_INVALID_ARG;
  const uint32_t ver = read_le<uint32_t>(body), npar = read_le<uint32_t>(body + 4);
  if ((ver != 1 && ver != 2) || (int)npar != np) return GMRES_ERR_INVALID_ARG;
  const size_t want = base + (ver == 2 ? 4 + 8 + 4 + 8 : 0) + 4;
  if (raw.size() != want) return GMRES_ERR_INVALID_ARG;
  gmres_ctrl_ctx* c = new (std::nothrow) gmres_ctrl_ctx();
  if (!c) return GMRES_ERR_OOM;
  for (int i = 0; i < kFeat; ++i) {
    c->mean[i] = read_le<double>(body + 8 + 8 * i);
    c->std_[i] = read_le<double>(body + 8 + 8 * kFeat + 8 * i);
  }
  std::vector<float> params((size_t)np);
  std::memcpy(params.data(), body + 8 + 16 * kFeat, (size_t)np * 4);
  if (ver == 2) {
    const unsigned char* q = body + 8 + 16 * kFeat + (size_t)np * 4;
    c->fixed_m = read_le<int32_t>(q);
    c->fixed_tol = read_le<double>(q + 4);
    c->fixed_d = read_le<int32_t>(q + 12);
    c->fixed_ratio = read_le<double>(q + 16);
    c->has_fixed = c->fixed_m > 0 && c->fixed_ratio > 0.0;
  }
  const int rc = gmres_mlp_create(params.data(), &c->net);
  if (rc != GMRES_OK) {
    delete c;
    return rc;
  }
  *out = c;
  return GMRES_OK;
}

int gmres_controller_destroy(gmres_ctrl_t c) {
  delete c;
  return GMRES_OK;
}

int gmres_controller_features(gmres_handle_t h, const double* b, double* features) {
  if (!h || !b || !features) return GMRES_ERR_INVALID_ARG;
  return guarded([&] { compute_features(h, b, features); });
}

int gmres_controller_decide(gmres_ctrl_t c, const double* features, gmres_suggestion_t* out) {
  if (!c || !features || !out) return GMRES_ERR_INVALID_ARG;
  float x[kFeat], y[kOut];
  for (int i = 0; i < kFeat; ++i) {
    if (!std::isfinite(features[i])) return GMRES_ERR_INVALID_ARG;
    x[i] = (float)((features[i] - c->mean[i]) / c->std_[i]);
  }
  const int rc = gmres_mlp_forward(c->net, x, 1, y);
  if (rc != GMRES_OK) return rc;
  gmres_suggestion_t S{};
  for (int i = 0; i < kFeat; ++i) S.features[i] = features[i];
  for (int i = 0; i < kOut; ++i) S.outputs[i] = y[i];
  S.predicted_ratio = std::exp((double)y[8]);
  const double y8 = (double)y[8];
  if (y8 >= std::log(kFallbackRatio)) {                  // no gain predicted over the default
    S.m = kDefaultM;
    S.inner_tol = 0.0;
    S.poly_degree = 0;
    S.choice = 1;
  } else if (c->has_fixed && y8 >= std::log(c->fixed_ratio / kFallbackRatio)) {
    // the network's predicted gain is not clearly beyond what the best fixed setting reaches on
    // the training data: take that setting
    S.m = c->fixed_m;
    S.inner_tol = c->fixed_tol;
    S.poly_degree = c->fixed_d;
    S.choice = 2;
  } else {
    int im = 0, id = 0;
    for (int i = 1; i < 3; ++i)
      if (y[i] > y[im]) im = i;
    for (int i = 1; i < 4; ++i)
      if (y[4 + i] > y[4 + id]) id = i;
    S.m = kMClass[im];
    S.poly_degree = kDClass[id];
    S.inner_tol = std::pow(10.0, std::min(-2.0, std::max(-6.0, (double)y[3])));
    S.choice = 0;
  }
  *out = S;
  return GMRES_OK;
}

int gmres_controller_suggest(gmres_ctrl_t c, gmres_handle_t h, const double* b,
                             gmres_suggestion_t* out) {
  if (!c || !h || !b || !out) return GMRES_ERR_INVALID_ARG;
  double f[kFeat];
  const int rc = gmres_controller_features(h, b, f);
  if (rc != GMRES_OK) return rc;
  return gmres_controller_decide(c, f, out);
}

}  // extern "C"
