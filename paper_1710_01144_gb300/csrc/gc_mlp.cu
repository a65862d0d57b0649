// Kernels and C ABI of the candidate-proposal network (gc_mlp.cuh):
// features, forward, backward (activations + weight-gradient reductions),
// Adam, and a minibatch training loop -- all hand-written float32 kernels on
// CUDA cores (the network is 4801 parameters; there is no dense contraction
// large enough for tensor cores to matter).
#include <limits.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "gc_device.cuh"
#include "gc_internal.cuh"
#include "gc_mlp.cuh"

struct gc_mlp {
  int32_t max_batch = 0;
  cudaStream_t stream = nullptr;
  float *params = nullptr;  // [kMlpParams]
  float *grad = nullptr;    // [kMlpParams]
  float *adam_m = nullptr, *adam_v = nullptr;
  float *h1 = nullptr, *h2 = nullptr, *dh1 = nullptr, *dh2 = nullptr;  // [max_batch][64]
  float *dout = nullptr;                                              // [max_batch]
  double *loss = nullptr;                                             // device accumulator
  double *h_loss = nullptr;                                           // pinned
  int64_t t = 0;                                                      // Adam step count
};

namespace gc {

constexpr int kMlpThreads = 256;

// features of list[i] (i < *m_dev or m) into X[i][8]
__global__ void k_features(const int32_t *__restrict__ list, int32_t m, const int32_t *m_dev,
                           const int32_t *__restrict__ rp, const int32_t *__restrict__ dS,
                           const long long *__restrict__ ub, const int32_t *__restrict__ stamp,
                           const long long *__restrict__ two_hop, const int32_t *__restrict__ mx, int32_t round,
                           long long prev_gain, float *X) {
  const int cnt = m_dev ? *m_dev : m;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
    float f[kMlpIn];
    cand_features(list[i], rp, dS, ub, stamp, two_hop, mx, round, prev_gain, f);
#pragma unroll
    for (int j = 0; j < kMlpIn; ++j) X[(size_t)i * kMlpIn + j] = f[j];
  }
}

__global__ void __launch_bounds__(kMlpThreads) k_mlp_forward(const float *__restrict__ W,
                                                             const float *__restrict__ X, int32_t m,
                                                             float *__restrict__ out) {
  __shared__ float sw[kMlpParams];
  __shared__ float sh[kMlpThreads / 32][kMlpHidden];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sw[i] = W[i];
  cta_sync();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wid, nw = gridDim.x * (blockDim.x >> 5);
  for (int s = gw; s < m; s += nw) {
    float x[kMlpIn];
#pragma unroll
    for (int f = 0; f < kMlpIn; ++f) x[f] = X[(size_t)s * kMlpIn + f];
    const float o = mlp_forward_warp(sw, x, sh[wid]);
    if (lane == 0) out[s] = o;
  }
}

// Per-sample forward and backward of L = (1/m) sum (out - y)^2: stores h1, h2,
// dL/dz1 (dh1), dL/dz2 (dh2) and dL/dout; accumulates the loss.
__global__ void __launch_bounds__(kMlpThreads) k_mlp_fwdbwd(const float *__restrict__ W,
                                                            const float *__restrict__ X,
                                                            const float *__restrict__ y, int32_t m, float *H1,
                                                            float *H2, float *DH1, float *DH2, float *DOUT,
                                                            double *loss) {
  __shared__ float sw[kMlpParams];
  __shared__ float sh1[kMlpThreads / 32][kMlpHidden];
  __shared__ float sd2[kMlpThreads / 32][kMlpHidden];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sw[i] = W[i];
  cta_sync();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wid, nw = gridDim.x * (blockDim.x >> 5);
  double lsum = 0;
  for (int s = gw; s < m; s += nw) {
    float x[kMlpIn];
#pragma unroll
    for (int f = 0; f < kMlpIn; ++f) x[f] = X[(size_t)s * kMlpIn + f];
    // forward, keeping pre-activations for the ReLU masks
    float z10 = sw[kOffB1 + lane], z11 = sw[kOffB1 + lane + 32];
#pragma unroll
    for (int f = 0; f < kMlpIn; ++f) {
      z10 = fmaf(x[f], sw[kOffW1 + f * kMlpHidden + lane], z10);
      z11 = fmaf(x[f], sw[kOffW1 + f * kMlpHidden + lane + 32], z11);
    }
    const float h10 = fmaxf(z10, 0.f), h11 = fmaxf(z11, 0.f);
    sh1[wid][lane] = h10;
    sh1[wid][lane + 32] = h11;
    __syncwarp();
    float z20 = sw[kOffB2 + lane], z21 = sw[kOffB2 + lane + 32];
    for (int i = 0; i < kMlpHidden; ++i) {
      const float h = sh1[wid][i];
      z20 = fmaf(h, sw[kOffW2 + i * kMlpHidden + lane], z20);
      z21 = fmaf(h, sw[kOffW2 + i * kMlpHidden + lane + 32], z21);
    }
    const float h20 = fmaxf(z20, 0.f), h21 = fmaxf(z21, 0.f);
    float o = h20 * sw[kOffW3 + lane] + h21 * sw[kOffW3 + lane + 32];
#pragma unroll
    for (int q = 16; q > 0; q >>= 1) o += __shfl_xor_sync(0xffffffffu, o, q);
    o += sw[kOffB3];
    const float diff = o - y[s];
    const float dout = 2.f * diff / (float)m;
    if (lane == 0) lsum += (double)diff * (double)diff;
    // backward
    const float d20 = z20 > 0.f ? dout * sw[kOffW3 + lane] : 0.f;
    const float d21 = z21 > 0.f ? dout * sw[kOffW3 + lane + 32] : 0.f;
    sd2[wid][lane] = d20;
    sd2[wid][lane + 32] = d21;
    __syncwarp();
    float e0 = 0.f, e1 = 0.f;  // dL/dh1 for i = lane, lane + 32
    for (int j = 0; j < kMlpHidden; ++j) {
      const float d = sd2[wid][j];
      e0 = fmaf(d, sw[kOffW2 + lane * kMlpHidden + j], e0);
      e1 = fmaf(d, sw[kOffW2 + (lane + 32) * kMlpHidden + j], e1);
    }
    const size_t row = (size_t)s * kMlpHidden;
    H1[row + lane] = h10;
    H1[row + lane + 32] = h11;
    H2[row + lane] = h20;
    H2[row + lane + 32] = h21;
    DH2[row + lane] = d20;
    DH2[row + lane + 32] = d21;
    DH1[row + lane] = z10 > 0.f ? e0 : 0.f;
    DH1[row + lane + 32] = z11 > 0.f ? e1 : 0.f;
    if (lane == 0) DOUT[s] = dout;
    __syncwarp();
  }
  if (lane == 0 && lsum != 0) atomicAdd(loss, lsum / (double)m);
}

// Weight gradients: one thread per parameter, summing over the batch.
__global__ void k_mlp_wgrad(const float *__restrict__ X, const float *__restrict__ H1,
                            const float *__restrict__ H2, const float *__restrict__ DH1,
                            const float *__restrict__ DH2, const float *__restrict__ DOUT, int32_t m,
                            float *__restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  float acc = 0.f;
  if (p < kOffB1) {  // W1[f][i] = sum_b X[b][f] * dh1[b][i]
    const int f = p / kMlpHidden, i = p % kMlpHidden;
    for (int b = 0; b < m; ++b) acc = fmaf(X[(size_t)b * kMlpIn + f], DH1[(size_t)b * kMlpHidden + i], acc);
  } else if (p < kOffW2) {
    const int i = p - kOffB1;
    for (int b = 0; b < m; ++b) acc += DH1[(size_t)b * kMlpHidden + i];
  } else if (p < kOffB2) {  // W2[i][j] = sum_b h1[b][i] * dh2[b][j]
    const int q = p - kOffW2, i = q / kMlpHidden, j = q % kMlpHidden;
    for (int b = 0; b < m; ++b)
      acc = fmaf(H1[(size_t)b * kMlpHidden + i], DH2[(size_t)b * kMlpHidden + j], acc);
  } else if (p < kOffW3) {
    const int j = p - kOffB2;
    for (int b = 0; b < m; ++b) acc += DH2[(size_t)b * kMlpHidden + j];
  } else if (p < kOffB3) {
    const int j = p - kOffW3;
    for (int b = 0; b < m; ++b) acc = fmaf(H2[(size_t)b * kMlpHidden + j], DOUT[b], acc);
  } else {
    for (int b = 0; b < m; ++b) acc += DOUT[b];
  }
  grad[p] = acc;
}

__global__ void k_adam(float *p, const float *g, float *m, float *v, float lr, float b1, float b2, float eps,
                       float c1, float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= kMlpParams) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// Training data for the proposal: the features each evaluated candidate had
// when it was selected (before its bound is replaced) and log1p of the exact
// gain the pruned BFS found.  Appended at *count, up to cap rows.
__global__ void k_record(const int32_t *__restrict__ list, const int32_t *n_sel, const long long *__restrict__ lgain,
                         const int32_t *__restrict__ rp, const int32_t *__restrict__ dS,
                         const long long *__restrict__ ub, const int32_t *__restrict__ stamp,
                         const long long *__restrict__ two_hop, const int32_t *__restrict__ mx, int32_t round,
                         long long prev_gain, float *X, float *y, int32_t cap, int32_t *count) {
  const int m = *n_sel;
  const int base = *(volatile int32_t *)count;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
    const int row = base + i;
    if (row >= cap) break;
    float f[kMlpIn];
    cand_features(list[i], rp, dS, ub, stamp, two_hop, mx, round, prev_gain, f);
#pragma unroll
    for (int j = 0; j < kMlpIn; ++j) X[(size_t)row * kMlpIn + j] = f[j];
    y[row] = log1pf((float)lgain[i]);
  }
}

__global__ void k_record_advance(const int32_t *n_sel, int32_t cap, int32_t *count) {
  const int c = *count + *n_sel;
  *count = c < cap ? c : cap;
}

int launch_record(gc_graph *g, int32_t round, long long prev_gain) {
  if (!g->rec_X || g->rec_cap <= 0) return GC_OK;
  g->launches += 2;
  k_record<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->list, &g->sctl->n_sel, g->lgain, g->rp, g->dS, g->ub,
                                                         g->stamp, g->two_hop, g->mx, round, prev_gain, g->rec_X,
                                                         g->rec_y, g->rec_cap, g->rec_count);
  k_record_advance<<<1, 1, 0, g->stream>>>(&g->sctl->n_sel, g->rec_cap, g->rec_count);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

// Round-1 proposal (one CTA): the candidates list[0 .. *n_sel) (at most
// kProposeMax, the largest two-hop bounds) are scored by the network -- one
// warp per candidate, weights in shared memory -- and the kLanes with the
// largest predicted gain (ties: larger bound, then smaller id) are written
// back to list[0 .. 64) with *n_sel = min(64, count).  Only which candidates
// the first exact batch of round 1 holds changes; every other candidate is
// still compared with that batch's best exact gain by its bound.
constexpr int kProposeMax = 1024;
__global__ void __launch_bounds__(1024) k_round1_propose(int32_t *list, int32_t *n_sel, const float *__restrict__ W,
                                                        const int32_t *__restrict__ rp, const int32_t *__restrict__ dS,
                                                        const long long *__restrict__ ub,
                                                        const int32_t *__restrict__ stamp,
                                                        const long long *__restrict__ two_hop,
                                                        const int32_t *__restrict__ mx, long long prev_gain) {
  __shared__ float sw[kMlpParams];
  __shared__ float sh[32][kMlpHidden];
  __shared__ float s_key[kProposeMax];
  __shared__ long long s_ub[kProposeMax];
  __shared__ int s_id[kProposeMax];
  const int m = min(*n_sel, kProposeMax);
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sw[i] = W[i];
  for (int i = threadIdx.x; i < kProposeMax; i += blockDim.x) {
    s_id[i] = i < m ? list[i] : INT_MAX;
    s_ub[i] = i < m ? ub[s_id[i]] : LLONG_MIN;
    s_key[i] = -INFINITY;
  }
  cta_sync();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int i = wid; i < m; i += blockDim.x >> 5) {
    float f[kMlpIn];
    cand_features(s_id[i], rp, dS, ub, stamp, two_hop, mx, 1, prev_gain, f);
    const float o = mlp_forward_warp(sw, f, sh[wid]);
    if (lane == 0) s_key[i] = o;
  }
  cta_sync();
  // bitonic sort of (key desc, ub desc, id asc) over kProposeMax entries
  for (int size = 2; size <= kProposeMax; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      const int i = threadIdx.x, j = i ^ stride;
      if (j > i && i < kProposeMax) {
        const bool up = (i & size) == 0;  // this pair sorts "first = better"
        const bool ib = s_key[i] > s_key[j] || (s_key[i] == s_key[j] &&
                        (s_ub[i] > s_ub[j] || (s_ub[i] == s_ub[j] && s_id[i] < s_id[j])));
        if (ib != up) {
          const float tk = s_key[i]; s_key[i] = s_key[j]; s_key[j] = tk;
          const long long tu = s_ub[i]; s_ub[i] = s_ub[j]; s_ub[j] = tu;
          const int ti = s_id[i]; s_id[i] = s_id[j]; s_id[j] = ti;
        }
      }
      cta_sync();
    }
  }
  if (threadIdx.x < kLanes && threadIdx.x < m) list[threadIdx.x] = s_id[threadIdx.x];
  if (threadIdx.x == 0) *n_sel = min(m, kLanes);
}

int launch_round1_propose(gc_graph *g, long long prev_gain) {
  if (!g->prop_params) return GC_EINVAL;
  ++g->launches;
  k_round1_propose<<<1, 1024, 0, g->stream>>>(g->list, &g->sctl->n_sel, g->prop_params, g->rp, g->dS, g->ub,
                                              g->stamp, g->two_hop, g->mx, prev_gain);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_features(gc_graph *g, const int32_t *list, int32_t m, const int32_t *m_dev, int32_t round,
                    long long prev_gain, float *X) {
  ++g->launches;
  k_features<<<g->red_blocks, kRedThreads, 0, g->stream>>>(list, m, m_dev, g->rp, g->dS, g->ub, g->stamp,
                                                           g->two_hop, g->mx, round, prev_gain, X);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

static int mlp_grad_async(gc_mlp *h, const float *X, const float *y, int32_t m) {
  GC_CUDA(cudaMemsetAsync(h->loss, 0, sizeof(double), h->stream));
  const int blocks = std::max(1, std::min(1024, (m + (kMlpThreads / 32) - 1) / (kMlpThreads / 32)));
  k_mlp_fwdbwd<<<blocks, kMlpThreads, 0, h->stream>>>(h->params, X, y, m, h->h1, h->h2, h->dh1, h->dh2,
                                                      h->dout, h->loss);
  k_mlp_wgrad<<<(kMlpParams + 255) / 256, 256, 0, h->stream>>>(X, h->h1, h->h2, h->dh1, h->dh2, h->dout, m,
                                                               h->grad);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

static int mlp_adam_async(gc_mlp *h, float lr) {
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  h->t += 1;
  const float c1 = 1.f - powf(b1, (float)h->t), c2 = 1.f - powf(b2, (float)h->t);
  k_adam<<<(kMlpParams + 255) / 256, 256, 0, h->stream>>>(h->params, h->grad, h->adam_m, h->adam_v, lr, b1, b2,
                                                          eps, c1, c2);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

}  // namespace gc

using namespace gc;

extern "C" {

int gc_mlp_create(int32_t max_batch, void *stream, gc_mlp **out) {
  if (!out || max_batch < 1) {
    set_error("bad argument to gc_mlp_create");
    return GC_EINVAL;
  }
  *out = nullptr;
  gc_mlp *h = new gc_mlp();
  h->max_batch = max_batch;
  h->stream = (cudaStream_t)stream;
  const size_t act = (size_t)max_batch * kMlpHidden * sizeof(float);
  void **bufs[] = {(void **)&h->params, (void **)&h->grad, (void **)&h->adam_m, (void **)&h->adam_v};
  bool ok = true;
  for (void **b : bufs) ok = ok && cudaMalloc(b, kMlpParams * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc((void **)&h->h1, act) == cudaSuccess && cudaMalloc((void **)&h->h2, act) == cudaSuccess &&
       cudaMalloc((void **)&h->dh1, act) == cudaSuccess && cudaMalloc((void **)&h->dh2, act) == cudaSuccess &&
       cudaMalloc((void **)&h->dout, (size_t)max_batch * sizeof(float)) == cudaSuccess &&
       cudaMalloc((void **)&h->loss, sizeof(double)) == cudaSuccess &&
       cudaMallocHost((void **)&h->h_loss, sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    gc_mlp_free(h);
    set_error("gc_mlp_create: allocation failed");
    return GC_ENOMEM;
  }
  cudaMemsetAsync(h->params, 0, kMlpParams * sizeof(float), h->stream);
  cudaMemsetAsync(h->adam_m, 0, kMlpParams * sizeof(float), h->stream);
  cudaMemsetAsync(h->adam_v, 0, kMlpParams * sizeof(float), h->stream);
  *out = h;
  return GC_OK;
}

int gc_mlp_free(gc_mlp *h) {
  if (!h) return GC_OK;
  cudaStreamSynchronize(h->stream);
  void *bufs[] = {h->params, h->grad, h->adam_m, h->adam_v, h->h1, h->h2, h->dh1, h->dh2, h->dout, h->loss};
  for (void *b : bufs)
    if (b) cudaFree(b);
  if (h->h_loss) cudaFreeHost(h->h_loss);
  delete h;
  return GC_OK;
}

int gc_mlp_set_params(gc_mlp *h, const float *params) {
  if (!h || !params) {
    set_error("bad argument to gc_mlp_set_params");
    return GC_EINVAL;
  }
  GC_CUDA(cudaMemcpyAsync(h->params, params, kMlpParams * sizeof(float), cudaMemcpyHostToDevice, h->stream));
  GC_CUDA(cudaMemsetAsync(h->adam_m, 0, kMlpParams * sizeof(float), h->stream));
  GC_CUDA(cudaMemsetAsync(h->adam_v, 0, kMlpParams * sizeof(float), h->stream));
  h->t = 0;
  GC_CUDA(cudaStreamSynchronize(h->stream));
  return GC_OK;
}

int gc_mlp_get_params(gc_mlp *h, float *params) {
  if (!h || !params) {
    set_error("bad argument to gc_mlp_get_params");
    return GC_EINVAL;
  }
  GC_CUDA(cudaMemcpyAsync(params, h->params, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(cudaStreamSynchronize(h->stream));
  return GC_OK;
}

int gc_mlp_forward(gc_mlp *h, const float *X, int32_t m, float *out) {
  if (!h || m < 0 || (m > 0 && (!X || !out))) {
    set_error("bad argument to gc_mlp_forward");
    return GC_EINVAL;
  }
  if (m == 0) return GC_OK;
  const int blocks = std::max(1, std::min(4096, (m + 7) / 8));
  k_mlp_forward<<<blocks, kMlpThreads, 0, h->stream>>>(h->params, X, m, out);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int gc_mlp_grad(gc_mlp *h, const float *X, const float *y, int32_t m, float *grad, double *loss) {
  if (!h || !X || !y || m < 1 || m > h->max_batch) {
    set_error("bad argument to gc_mlp_grad (1 <= m <= max_batch)");
    return GC_EINVAL;
  }
  int rc = mlp_grad_async(h, X, y, m);
  if (rc) return rc;
  if (grad)
    GC_CUDA(cudaMemcpyAsync(grad, h->grad, kMlpParams * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(cudaMemcpyAsync(h->h_loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  GC_CUDA(cudaStreamSynchronize(h->stream));
  if (loss) *loss = *h->h_loss;
  return GC_OK;
}

int gc_mlp_adam_step(gc_mlp *h, const float *X, const float *y, int32_t m, float lr) {
  if (!h || !X || !y || m < 1 || m > h->max_batch || !(lr > 0)) {
    set_error("bad argument to gc_mlp_adam_step");
    return GC_EINVAL;
  }
  int rc = mlp_grad_async(h, X, y, m);
  if (!rc) rc = mlp_adam_async(h, lr);
  return rc;
}

int gc_mlp_train(gc_mlp *h, const float *X, const float *y, int32_t m, int32_t epochs, int32_t batch, float lr,
                 uint64_t seed, double *final_loss) {
  if (!h || !X || !y || m < 1 || epochs < 1 || batch < 1 || batch > h->max_batch || !(lr > 0)) {
    set_error("bad argument to gc_mlp_train");
    return GC_EINVAL;
  }
  const int32_t nb = (m + batch - 1) / batch;
  std::vector<int32_t> order(nb);
  uint64_t s = seed * 0x9E3779B97F4A7C15ULL + 1;
  for (int32_t e = 0; e < epochs; ++e) {
    for (int32_t i = 0; i < nb; ++i) order[i] = i;
    for (int32_t i = nb - 1; i > 0; --i) {  // Fisher-Yates on the minibatch order (xorshift64)
      s ^= s << 13;
      s ^= s >> 7;
      s ^= s << 17;
      std::swap(order[i], order[(int32_t)(s % (uint64_t)(i + 1))]);
    }
    for (int32_t i = 0; i < nb; ++i) {
      const int32_t off = order[i] * batch, len = std::min(batch, m - off);
      int rc = mlp_grad_async(h, X + (size_t)off * kMlpIn, y + off, len);
      if (!rc) rc = mlp_adam_async(h, lr);
      if (rc) return rc;
    }
  }
  if (final_loss) {
    // loss over the whole set, one batch at a time
    double tot = 0;
    for (int32_t off = 0; off < m; off += batch) {
      const int32_t len = std::min(batch, m - off);
      int rc = mlp_grad_async(h, X + (size_t)off * kMlpIn, y + off, len);
      if (rc) return rc;
      GC_CUDA(cudaMemcpyAsync(h->h_loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
      GC_CUDA(cudaStreamSynchronize(h->stream));
      tot += *h->h_loss * len;
    }
    *final_loss = tot / m;
  }
  GC_CUDA(cudaStreamSynchronize(h->stream));
  return GC_OK;
}

int gc_candidate_features(const int32_t *row_ptr, const int32_t *dS, const int64_t *ub, const int32_t *stamp,
                          const int64_t *two_hop, const int32_t *mx, const int32_t *cand, int32_t m, int32_t round,
                          int64_t prev_gain, float *X, void *stream) {
  if (!row_ptr || !dS || !ub || !stamp || !two_hop || m < 0 || (m > 0 && (!cand || !X))) {
    set_error("bad argument to gc_candidate_features");
    return GC_EINVAL;
  }
  if (m == 0) return GC_OK;
  k_features<<<std::min(1024, (m + 255) / 256), 256, 0, (cudaStream_t)stream>>>(
      cand, m, nullptr, row_ptr, dS, (const long long *)ub, stamp, (const long long *)two_hop, mx, round,
      (long long)prev_gain, X);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int gc_set_proposal(gc_graph *g, const gc_mlp *h, int32_t fill) {
  if (!g || fill < 0 || fill > kLanes - 1) {
    set_error("bad argument to gc_set_proposal (0 <= fill < 64)");
    return GC_EINVAL;
  }
  g->prop_params = h ? h->params : nullptr;
  g->prop_fill = h ? fill : 0;  // 0: round 1's first batch only
  return GC_OK;
}

int gc_set_recorder(gc_graph *g, float *X, float *y, int32_t cap) {
  if (!g || cap < 0 || (cap > 0 && (!X || !y))) {
    set_error("bad argument to gc_set_recorder");
    return GC_EINVAL;
  }
  g->rec_X = cap ? X : nullptr;
  g->rec_y = cap ? y : nullptr;
  g->rec_cap = cap;
  if (g->rec_count) GC_CUDA(cudaMemsetAsync(g->rec_count, 0, sizeof(int32_t), g->stream));
  return GC_OK;
}

int64_t gc_recorded(gc_graph *g) {
  if (!g || !g->rec_count) return -1;
  int32_t c = 0;
  if (cudaMemcpyAsync(&c, g->rec_count, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream) != cudaSuccess ||
      cudaStreamSynchronize(g->stream) != cudaSuccess)
    return -1;
  return c;
}

}  // extern "C"
