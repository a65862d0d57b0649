// Candidate-proposal network (not part of the paper's method): per-vertex
// features and a 8 -> 64 -> 64 -> 1 ReLU MLP in float32.  It only orders which
// candidates get an exact pruned-BFS evaluation; acceptance stays the exact
// lazy rule of Sec. 4.2, so the greedy group never depends on it.
//
// Parameter vector (kMlpParams floats): W1[8][64], b1[64], W2[64][64], b2[64],
// W3[64], b3.
#pragma once

#include <stdint.h>

namespace gc {

constexpr int kMlpIn = 8;
constexpr int kMlpHidden = 64;
constexpr int kMlpParams = kMlpIn * kMlpHidden + kMlpHidden + kMlpHidden * kMlpHidden + kMlpHidden +
                           kMlpHidden + 1;  // 4801
constexpr int kOffW1 = 0, kOffB1 = kOffW1 + kMlpIn * kMlpHidden, kOffW2 = kOffB1 + kMlpHidden,
              kOffB2 = kOffW2 + kMlpHidden * kMlpHidden, kOffW3 = kOffB2 + kMlpHidden,
              kOffB3 = kOffW3 + kMlpHidden;

// Features of candidate v in round `round` (see the file comment of
// oracle-side reference for the same list):
//   0 log1p(deg)  1 d_S  2 log1p(max(ub,0))  3 round - stamp  4 log1p(two_hop)
//   5 mx - d_S    6 log1p(prev_gain)          7 f2 - f6
__device__ __forceinline__ void cand_features(int v, const int32_t *__restrict__ rp,
                                              const int32_t *dS, const long long *ub,
                                              const int32_t *stamp,
                                              const long long *__restrict__ two_hop,
                                              const int32_t *__restrict__ mx, int32_t round, long long prev_gain,
                                              float *f) {
  const float d = (float)dS[v];
  const long long u = ub[v];
  f[0] = log1pf((float)(rp[v + 1] - rp[v]));
  f[1] = d;
  f[2] = log1pf((float)(u > 0 ? u : 0));
  f[3] = (float)(round - stamp[v]);
  f[4] = log1pf((float)two_hop[v]);
  f[5] = (mx ? (float)mx[v] : d) - d;
  f[6] = log1pf((float)(prev_gain > 0 ? prev_gain : 0));
  f[7] = f[2] - f[6];
}

// One sample's forward pass by one warp; the weights are in shared memory
// (sw, kMlpParams floats), h1 is a per-warp shared buffer of 64 floats.
// Every lane returns the network output.
__device__ __forceinline__ float mlp_forward_warp(const float *sw, const float *x, float *h1) {
  const int lane = threadIdx.x & 31;
  float a0 = sw[kOffB1 + lane], a1 = sw[kOffB1 + lane + 32];
#pragma unroll
  for (int f = 0; f < kMlpIn; ++f) {
    a0 = fmaf(x[f], sw[kOffW1 + f * kMlpHidden + lane], a0);
    a1 = fmaf(x[f], sw[kOffW1 + f * kMlpHidden + lane + 32], a1);
  }
  h1[lane] = fmaxf(a0, 0.f);
  h1[lane + 32] = fmaxf(a1, 0.f);
  __syncwarp();
  float c0 = sw[kOffB2 + lane], c1 = sw[kOffB2 + lane + 32];
#pragma unroll 8
  for (int i = 0; i < kMlpHidden; ++i) {
    const float h = h1[i];
    c0 = fmaf(h, sw[kOffW2 + i * kMlpHidden + lane], c0);
    c1 = fmaf(h, sw[kOffW2 + i * kMlpHidden + lane + 32], c1);
  }
  float o = fmaxf(c0, 0.f) * sw[kOffW3 + lane] + fmaxf(c1, 0.f) * sw[kOffW3 + lane + 32];
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) o += __shfl_xor_sync(0xffffffffu, o, s);
  __syncwarp();
  return o + sw[kOffB3];
}

}  // namespace gc
