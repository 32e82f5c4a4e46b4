// The learned GMRES-IR parameter controller: a small MLP with its own FP32 forward, backward and
// Adam kernels.  The paper tunes restart length, inner tolerance and polynomial degree by hand
// (Sections V-E and V-F); this network proposes them from cheap matrix features and the residual
// history of a first cycle.
//
// Architecture: 12 features -> 64 (ReLU) -> 64 (ReLU) -> 9 outputs:
//   [0..2] logits of the restart length class m in {25, 50, 100}            (cross-entropy)
//   [3]    log10 of the inner tolerance                                     (squared error)
//   [4..7] logits of the polynomial degree class d in {0, 10, 25, 40}       (cross-entropy)
//   [8]    log of the predicted time ratio against the default parameters  (squared error)
// Parameters (one flat FP32 array): W1[64][12], b1[64], W2[64][64], b2[64], W3[9][64], b3[9].
//
// Kernels: forward (one thread per sample, weights in shared memory), backward through the
// activations (one thread per sample), parameter gradients (one thread per parameter, summing the
// batch in a fixed order: deterministic), loss reduction and Adam.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/gmresb3.h"

namespace gmresb3 {
namespace mlp {

constexpr int kIn = 12, kH = 64, kOut = 9;
constexpr int oW1 = 0, oB1 = oW1 + kH * kIn, oW2 = oB1 + kH, oB2 = oW2 + kH * kH, oW3 = oB2 + kH,
              oB3 = oW3 + kOut * kH, kParams = oB3 + kOut;
constexpr int kMaxBatch = 1 << 16;

__global__ void __launch_bounds__(128)
    k_fwd(const float* __restrict__ P, const float* __restrict__ X, int B, float* __restrict__ H1,
          float* __restrict__ H2, float* __restrict__ Y) {
  __shared__ float w[kParams];
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = P[i];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float x[kIn], h1[kH];
  for (int j = 0; j < kIn; ++j) x[j] = X[(size_t)b * kIn + j];
  for (int i = 0; i < kH; ++i) {
    float s = w[oB1 + i];
    for (int j = 0; j < kIn; ++j) s += w[oW1 + i * kIn + j] * x[j];
    h1[i] = fmaxf(s, 0.f);
    if (H1) H1[(size_t)b * kH + i] = h1[i];
  }
  float h2[kH];
  for (int i = 0; i < kH; ++i) {
    float s = w[oB2 + i];
    for (int j = 0; j < kH; ++j) s += w[oW2 + i * kH + j] * h1[j];
    h2[i] = fmaxf(s, 0.f);
    if (H2) H2[(size_t)b * kH + i] = h2[i];
  }
  for (int o = 0; o < kOut; ++o) {
    float s = w[oB3 + o];
    for (int j = 0; j < kH; ++j) s += w[oW3 + o * kH + j] * h2[j];
    Y[(size_t)b * kOut + o] = s;
  }
}

// Loss terms per sample and gradients with respect to outputs and hidden activations.
// Labels: mc (class of m, -1 = none), tl (log10 inner tol), dc (class of d, -1 = none),
// rt (log time ratio); every term is averaged over the batch.
__global__ void __launch_bounds__(128)
    k_bwd_act(const float* __restrict__ P, int B, const float* __restrict__ H1,
              const float* __restrict__ H2, const float* __restrict__ Y, const int* __restrict__ mc,
              const float* __restrict__ tl, const int* __restrict__ dc, const float* __restrict__ rt,
              float* __restrict__ dY, float* __restrict__ dH1, float* __restrict__ dH2,
              float* __restrict__ lparts) {
  __shared__ float w[kParams];
  for (int i = threadIdx.x; i < kParams; i += blockDim.x) w[i] = P[i];
  __syncthreads();
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  const float inv = 1.f / (float)B;
  float y[kOut], dy[kOut];
  for (int o = 0; o < kOut; ++o) {
    y[o] = Y[(size_t)b * kOut + o];
    dy[o] = 0.f;
  }
  float l[4] = {0.f, 0.f, 0.f, 0.f};
  // cross-entropy heads: softmax over a slice
  auto ce = [&](int lo, int nc, int label, float& loss) {
    if (label < 0 || label >= nc) return;  // no label (or out of range): no term
    float mx = y[lo];
    for (int c = 1; c < nc; ++c) mx = fmaxf(mx, y[lo + c]);
    float z = 0.f;
    for (int c = 0; c < nc; ++c) z += expf(y[lo + c] - mx);
    for (int c = 0; c < nc; ++c) {
      const float p = expf(y[lo + c] - mx) / z;
      dy[lo + c] = (p - (c == label ? 1.f : 0.f)) * inv;
    }
    loss = -(y[lo + label] - mx - logf(z));
  };
  ce(0, 3, mc[b], l[0]);
  ce(4, 4, dc[b], l[2]);
  const float e3 = y[3] - tl[b], e8 = y[8] - rt[b];
  l[1] = e3 * e3;
  dy[3] = 2.f * e3 * inv;
  l[3] = e8 * e8;
  dy[8] = 2.f * e8 * inv;
  for (int o = 0; o < kOut; ++o) dY[(size_t)b * kOut + o] = dy[o];
  for (int q = 0; q < 4; ++q) lparts[(size_t)b * 4 + q] = l[q];
  float d2[kH];
  for (int j = 0; j < kH; ++j) {
    float s = 0.f;
    for (int o = 0; o < kOut; ++o) s += w[oW3 + o * kH + j] * dy[o];
    d2[j] = H2[(size_t)b * kH + j] > 0.f ? s : 0.f;
    dH2[(size_t)b * kH + j] = d2[j];
  }
  for (int j = 0; j < kH; ++j) {
    float s = 0.f;
    for (int i = 0; i < kH; ++i) s += w[oW2 + i * kH + j] * d2[i];
    dH1[(size_t)b * kH + j] = H1[(size_t)b * kH + j] > 0.f ? s : 0.f;
  }
}

// One thread per parameter: the batch sum of its gradient contributions, in sample order.
__global__ void k_grad(const float* __restrict__ X, const float* __restrict__ H1,
                       const float* __restrict__ H2, const float* __restrict__ dY,
                       const float* __restrict__ dH1, const float* __restrict__ dH2, int B,
                       float* __restrict__ G) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  float s = 0.f;
  if (p < oB1) {
    const int i = (p - oW1) / kIn, j = (p - oW1) % kIn;
    for (int b = 0; b < B; ++b) s += dH1[(size_t)b * kH + i] * X[(size_t)b * kIn + j];
  } else if (p < oW2) {
    const int i = p - oB1;
    for (int b = 0; b < B; ++b) s += dH1[(size_t)b * kH + i];
  } else if (p < oB2) {
    const int i = (p - oW2) / kH, j = (p - oW2) % kH;
    for (int b = 0; b < B; ++b) s += dH2[(size_t)b * kH + i] * H1[(size_t)b * kH + j];
  } else if (p < oW3) {
    const int i = p - oB2;
    for (int b = 0; b < B; ++b) s += dH2[(size_t)b * kH + i];
  } else if (p < oB3) {
    const int o = (p - oW3) / kH, j = (p - oW3) % kH;
    for (int b = 0; b < B; ++b) s += dY[(size_t)b * kOut + o] * H2[(size_t)b * kH + j];
  } else {
    const int o = p - oB3;
    for (int b = 0; b < B; ++b) s += dY[(size_t)b * kOut + o];
  }
  G[p] = s;
}

// Batch means of the four loss terms (one warp, fixed order).
__global__ void k_loss(const float* __restrict__ lparts, int B, float* __restrict__ L) {
  const int q = threadIdx.x;
  if (q >= 4) return;
  float s = 0.f;
  for (int b = 0; b < B; ++b) s += lparts[(size_t)b * 4 + q];
  L[q] = s / (float)B;
}

__global__ void k_adam(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                       float* __restrict__ V, float lr, float b1, float b2, float eps, float c1,
                       float c2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kParams) return;
  const float g = G[p];
  const float m = b1 * M[p] + (1.f - b1) * g;
  const float v = b2 * V[p] + (1.f - b2) * g * g;
  M[p] = m;
  V[p] = v;
  P[p] -= lr * (m / c1) / (sqrtf(v / c2) + eps);
}

}  // namespace mlp
}  // namespace gmresb3

using namespace gmresb3::mlp;

struct gmres_mlp_ctx {
  cudaStream_t stream = nullptr;
  float *P = nullptr, *G = nullptr, *M = nullptr, *V = nullptr, *L = nullptr;
  float *H1 = nullptr, *H2 = nullptr, *Y = nullptr, *dY = nullptr, *dH1 = nullptr, *dH2 = nullptr;
  float* lparts = nullptr;
  float *X = nullptr, *tl = nullptr, *rt = nullptr;  // staged inputs (callers pass host or device)
  int *mc = nullptr, *dc = nullptr;
  int cap = 0;     // batch capacity of the activation and staging buffers
  int64_t step = 0;
  ~gmres_mlp_ctx() {
    void* ptrs[] = {P, G, M, V, L, H1, H2, Y, dY, dH1, dH2, lparts, X, tl, rt, mc, dc};
    for (void* p : ptrs) cudaFree(p);
    if (stream) cudaStreamDestroy(stream);
  }
};

namespace {

bool ensure_cap(gmres_mlp_ctx* c, int B) {
  if (B <= c->cap) return true;
  void** bufs[] = {(void**)&c->H1, (void**)&c->H2,  (void**)&c->Y,  (void**)&c->dY,
                   (void**)&c->dH1, (void**)&c->dH2, (void**)&c->lparts, (void**)&c->X,
                   (void**)&c->tl, (void**)&c->rt,  (void**)&c->mc, (void**)&c->dc};
  const size_t sizes[] = {kH, kH, kOut, kOut, kH, kH, 4, kIn, 1, 1, 1, 1};  // 4-byte words
  c->cap = 0;
  for (int i = 0; i < 12; ++i) {
    cudaFree(*bufs[i]);
    *bufs[i] = nullptr;
  }
  for (int i = 0; i < 12; ++i)
    if (cudaMalloc(bufs[i], sizes[i] * B * 4) != cudaSuccess) return false;
  c->cap = B;
  return true;
}

int mlp_err(cudaError_t e) {
  if (e == cudaSuccess) return GMRES_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA;
}

}  // namespace

extern "C" {

int gmres_mlp_create(const float* params, gmres_mlp_t* out) {
  if (!out || !params) return GMRES_ERR_INVALID_ARG;
  *out = nullptr;
  gmres_mlp_ctx* c = new (std::nothrow) gmres_mlp_ctx();
  if (!c) return GMRES_ERR_OOM;
  cudaError_t e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
  float** bufs[] = {&c->P, &c->G, &c->M, &c->V};
  for (auto b : bufs)
    if (e == cudaSuccess) e = cudaMalloc(b, kParams * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&c->L, 4 * sizeof(float));
  // on the private stream: it is non-blocking and would not wait for legacy-stream copies
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c->P, params, kParams * sizeof(float), cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->M, 0, kParams * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->V, 0, kParams * sizeof(float), c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    delete c;
    return mlp_err(e);
  }
  *out = c;
  return GMRES_OK;
}

int gmres_mlp_destroy(gmres_mlp_t c) {
  if (!c) return GMRES_OK;
  cudaStreamSynchronize(c->stream);
  delete c;
  return GMRES_OK;
}

int gmres_mlp_num_params(void) { return kParams; }

int gmres_mlp_get_params(gmres_mlp_t c, float* params) {
  if (!c || !params) return GMRES_ERR_INVALID_ARG;
  cudaError_t e =
      cudaMemcpyAsync(params, c->P, kParams * sizeof(float), cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return mlp_err(e);
}

int gmres_mlp_forward(gmres_mlp_t c, const float* X, int B, float* Y) {
  if (!c || !X || !Y || B < 1 || B > kMaxBatch) return GMRES_ERR_INVALID_ARG;
  if (!ensure_cap(c, B)) return GMRES_ERR_OOM;
  cudaError_t e =
      cudaMemcpyAsync(c->X, X, (size_t)B * kIn * sizeof(float), cudaMemcpyDefault, c->stream);
  if (e != cudaSuccess) return mlp_err(e);
  k_fwd<<<(B + 127) / 128, 128, 0, c->stream>>>(c->P, c->X, B, c->H1, c->H2, c->Y);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(Y, c->Y, (size_t)B * kOut * sizeof(float), cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return mlp_err(e);
}

static int mlp_backward(gmres_mlp_t c, const float* X, const int* mc, const float* tl,
                        const int* dc, const float* rt, int B) {
  if (!ensure_cap(c, B)) return GMRES_ERR_OOM;
  const void* src[] = {X, mc, tl, dc, rt};
  void* dst[] = {c->X, c->mc, c->tl, c->dc, c->rt};
  const size_t words[] = {(size_t)kIn, 1, 1, 1, 1};
  for (int i = 0; i < 5; ++i) {
    cudaError_t e = cudaMemcpyAsync(dst[i], src[i], words[i] * B * 4, cudaMemcpyDefault, c->stream);
    if (e != cudaSuccess) return mlp_err(e);
  }
  const int g = (B + 127) / 128;
  k_fwd<<<g, 128, 0, c->stream>>>(c->P, c->X, B, c->H1, c->H2, c->Y);
  k_bwd_act<<<g, 128, 0, c->stream>>>(c->P, B, c->H1, c->H2, c->Y, c->mc, c->tl, c->dc, c->rt,
                                      c->dY, c->dH1, c->dH2, c->lparts);
  k_grad<<<(kParams + 255) / 256, 256, 0, c->stream>>>(c->X, c->H1, c->H2, c->dY, c->dH1, c->dH2, B,
                                                       c->G);
  k_loss<<<1, 32, 0, c->stream>>>(c->lparts, B, c->L);
  return mlp_err(cudaGetLastError());
}

int gmres_mlp_gradient(gmres_mlp_t c, const float* X, const int* mc, const float* tl, const int* dc,
                       const float* rt, int B, float* grad, float* loss4) {
  if (!c || !X || !mc || !tl || !dc || !rt || !grad || B < 1 || B > kMaxBatch)
    return GMRES_ERR_INVALID_ARG;
  int rc = mlp_backward(c, X, mc, tl, dc, rt, B);
  if (rc != GMRES_OK) return rc;
  cudaError_t e = cudaMemcpyAsync(grad, c->G, kParams * sizeof(float), cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess && loss4)
    e = cudaMemcpyAsync(loss4, c->L, 4 * sizeof(float), cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return mlp_err(e);
}

int gmres_mlp_train_step(gmres_mlp_t c, const float* X, const int* mc, const float* tl,
                         const int* dc, const float* rt, int B, float lr, float* loss4) {
  if (!c || !X || !mc || !tl || !dc || !rt || B < 1 || B > kMaxBatch || !(lr > 0.f))
    return GMRES_ERR_INVALID_ARG;
  int rc = mlp_backward(c, X, mc, tl, dc, rt, B);
  if (rc != GMRES_OK) return rc;
  c->step += 1;
  const float b1 = 0.9f, b2 = 0.999f;
  const float c1 = 1.f - powf(b1, (float)c->step), c2 = 1.f - powf(b2, (float)c->step);
  k_adam<<<(kParams + 255) / 256, 256, 0, c->stream>>>(c->P, c->G, c->M, c->V, lr, b1, b2, 1e-8f,
                                                       c1, c2);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && loss4)
    e = cudaMemcpyAsync(loss4, c->L, 4 * sizeof(float), cudaMemcpyDefault, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  return mlp_err(e);
}

}  // extern "C"
