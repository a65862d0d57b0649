// bitGreedy++ (Sec. 4.3, Theorem 1): Greedy with per-vertex bit vectors.
//
// b^i_u is the set of vertices within distance i of u (b^0_u = {u}, and b^i_u
// is b^{i-1}_u together with b^{i-1}_v of every neighbour v: the closed
// neighbourhood, see the reading of the recurrence).  Theorem 1 gives the
// marginal gain of every vertex at once: Delta(u | S) = sum_i |b^i_u AND NOT
// b^i_S|, where b^i_S holds the vertices w with d_S[w] <= i; and with S empty
// the farness f({u}) = sum_i (n - |b^i_u|) (the vertices farther than i, summed
// over i), so round 0 is the same sweep.
//
// Memory.  n-bit vectors for all n vertices need n^2 bits.  Because distances
// are symmetric, bit t of b^i_u says d(u, t) <= i, so the targets t can be
// taken in chunks of 64 W: for one chunk every vertex holds W words (bit j of
// word q: target base + 64 q + j), the sweep level by level computes those
// words for all u, and the per-vertex sums add up over the chunks.  Two
// buffers of n x W words are the whole memory (the memory limit the paper
// leaves open, with W = 32 at most: 2048 targets per chunk), plus one byte
// per vertex and buffer saying whether its row holds any bit: a level loads
// the words of a neighbour only when its row is nonzero (32 neighbours' flags
// are gathered and balloted at once).
//
// Pruning.  A target t adds to no sum at levels i >= d_S[t] (its bit is
// masked out there), so its bit is dropped from the words from that level on:
// the sweep for target t is a BFS from t cut at depth d_S[t] - 1, the pruned
// SSSP of Sec. 4.1 seen from the other end.
//
// One cooperative launch per round; every level ends with a grid barrier.
#include <limits.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "gc_device.cuh"
#include "gc_internal.cuh"

namespace gc {

typedef unsigned long long u64;

constexpr int kBitsThreads = 256;

// MODE 0: out[u] += sum_i (cs - |b^i_u|) over the chunk (farness, S empty).
// MODE 1: out[u] += sum_i |b^i_u AND NOT b^i_S| over the chunk (gains).
template <int MODE>
__global__ void __launch_bounds__(kBitsThreads) k_bits_round(const int32_t *__restrict__ rp,
                                                             const int32_t *__restrict__ ci, int32_t n,
                                                             const int32_t *dS, int W, u64 *B0, u64 *B1,
                                                             unsigned char *A0, unsigned char *A1,
                                                             long long *out, BitsCtl *ctl,
                                                             unsigned long long tns) {
  __shared__ u64 s_mask[32];
  __shared__ int s_live;
  const int tid = threadIdx.x, lane = tid & 31, b = blockIdx.x, G = gridDim.x, T = blockDim.x;
  const int gw = (b * T + tid) >> 5, nw = (G * T) >> 5;
  const int chunk = 64 * W;
  int32_t *err = &ctl->err;
  u64 lev_total = 0;
  for (int base = 0; base < n; base += chunk) {
    const int cs = min(chunk, n - base);
    // level 0: every target's own bit (gains: only targets outside S)
    for (size_t x = (size_t)b * T + tid; x < (size_t)n * W; x += (size_t)G * T) B0[x] = 0ull;
    for (int u = b * T + tid; u < n; u += G * T) A0[u] = 0;
    if (!grid_sync(&ctl->bar, err, tns)) return;
    for (int j = b * T + tid; j < cs; j += G * T) {
      const int t = base + j;
      if (MODE == 0 || dS[t] > 0) {
        B0[(size_t)t * W + (j >> 6)] = 1ull << (j & 63);
        A0[t] = 1;
        if (MODE == 1) out[t] += 1;  // |b^0_t AND NOT b^0_S| = [d_S[t] > 0]
      }
    }
    if (MODE == 0)  // level 0: every target but u itself is farther than 0
      for (int u = b * T + tid; u < n; u += G * T) out[u] += cs - ((u >= base && u < base + cs) ? 1 : 0);
    if (b == 0 && tid == 0) ctl->changed[0] = ctl->changed[1] = ctl->changed[2] = 0u;
    if (!grid_sync(&ctl->bar, err, tns)) return;
    u64 *cur = B0, *nxt = B1;
    unsigned char *acur = A0, *anxt = A1;  // row nonzero, per vertex
    for (int i = 1;; ++i) {
      // the targets still counted at level i
      if (tid < W) {
        u64 m = 0ull;
        for (int q = 0; q < 64; ++q) {
          const int j = tid * 64 + q;
          if (j < cs && (MODE == 0 || dS[base + j] > i)) m |= 1ull << q;
        }
        s_mask[tid] = m;
      }
      if (tid == 0) s_live = 0;
      cta_sync();
      if (tid < W && s_mask[tid]) atomicOr(&s_live, 1);
      cta_sync();
      if (!s_live || i > n) break;  // no target left (the same decision in every CTA); i > n: never on a connected graph
      if (b == 0 && tid == 0) ctl->changed[(i + 1) % 3] = 0u;  // read two levels from now
      unsigned int chg = 0u;
      for (int u = gw; u < n; u += nw) {
        const u64 own = (lane < W && acur[u]) ? cur[(size_t)u * W + lane] : 0ull;
        u64 x = own;
        for (int e0 = rp[u]; e0 < rp[u + 1]; e0 += 32) {
          // 32 neighbours at once: their row flags, then only the nonzero rows
          const int cnt = min(32, rp[u + 1] - e0);
          const int mine = lane < cnt ? ci[e0 + lane] : 0;
          unsigned live = __ballot_sync(0xffffffffu, lane < cnt && acur[mine] != 0);
          while (live) {
            const int q = __ffs(live) - 1;
            live &= live - 1;
            const int v = __shfl_sync(0xffffffffu, mine, q);
            if (lane < W) x |= cur[(size_t)v * W + lane];
          }
        }
        int pc = 0;
        if (lane < W) {
          x &= s_mask[lane];
          nxt[(size_t)u * W + lane] = x;
          pc = __popcll(x);
          chg |= x != (own & s_mask[lane]);
        }
        const bool nz = __ballot_sync(0xffffffffu, lane < W && x != 0ull) != 0u;
        pc = warp_sum(pc);
        if (lane == 0) {
          anxt[u] = nz ? 1 : 0;
          out[u] += MODE == 1 ? (long long)pc : (long long)(cs - pc);
        }
      }
      if (MODE == 0 && __any_sync(0xffffffffu, chg) && lane == 0) atomicOr(&ctl->changed[i % 3], 1u);
      if (!grid_sync(&ctl->bar, err, tns)) return;
      ++lev_total;
      u64 *t = cur;
      cur = nxt;
      nxt = t;
      unsigned char *ta = acur;
      acur = anxt;
      anxt = ta;
      // farness: once no word changed, every later level adds cs - |b_u| = 0
      // (connected graph: all of the chunk is reached)
      if (MODE == 0 && *(volatile unsigned int *)&ctl->changed[i % 3] == 0u) break;
    }
    if (!grid_sync(&ctl->bar, err, tns)) return;  // the chunk's buffers are reused
  }
  if (b == 0 && tid == 0) ctl->levels = lev_total;
}

// Packed arg-best over the sums: MODE 0 the smallest farness (ties: smaller
// id), MODE 1 the largest gain among u with d_S[u] > 0 (ties: smaller id).
// Values below 2^31 (checked by the host: n <= kBitsMaxN).
template <int MODE>
__global__ void __launch_bounds__(kBitsThreads) k_bits_argbest(const long long *out, const int32_t *dS, int32_t n,
                                                               BitsCtl *ctl) {
  u64 best = 0ull;
  for (int u = blockIdx.x * blockDim.x + threadIdx.x; u < n; u += gridDim.x * blockDim.x) {
    if (MODE == 1 && dS[u] <= 0) continue;
    const long long v = out[u];
    const u64 val = MODE == 0 ? (u64)(v >= 0x7fffffffll ? 0ll : 0x7fffffffll - v) : (u64)v;
    const u64 key = (val << 32) | (u64)(0xffffffffu - (unsigned)u);
    best = best > key ? best : key;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const u64 x = __shfl_xor_sync(0xffffffffu, best, o);
    best = best > x ? best : x;
  }
  if ((threadIdx.x & 31) == 0 && best) atomicMax(&ctl->best, best);
}

static int bits_occupancy(int *blocks_per_sm) {
  int a = 0, b = 0;
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_bits_round<0>, kBitsThreads, 0));
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_bits_round<1>, kBitsThreads, 0));
  *blocks_per_sm = std::min(a, b);
  return GC_OK;
}

int launch_bits_round(gc_graph *g, int mode, unsigned long long *B, long long *out, BitsCtl *ctl, int W,
                      int64_t tns) {
  int occ = 0;
  const int rc = bits_occupancy(&occ);
  if (rc != GC_OK) return rc;
  const int grid = std::min(kMaxGridCtas, std::max(1, occ) * g->num_sms);
  const int32_t *rp = g->rp, *ci = g->ci, *dS = g->dS;
  int32_t n = g->n;
  u64 *B0 = B, *B1 = B + (size_t)n * W;
  unsigned char *A0 = (unsigned char *)(B + 2 * (size_t)n * W), *A1 = A0 + n;
  unsigned long long t = (unsigned long long)tns;
  void *args[] = {(void *)&rp, (void *)&ci, (void *)&n, (void *)&dS, (void *)&W, (void *)&B0, (void *)&B1,
                  (void *)&A0, (void *)&A1, (void *)&out, (void *)&ctl, (void *)&t};
  GC_CUDA(cudaMemsetAsync(ctl, 0, sizeof(BitsCtl), g->stream));
  GC_CUDA(cudaMemsetAsync(out, 0, (size_t)n * sizeof(long long), g->stream));
  g->launches += 2;
  GC_CUDA(cudaLaunchCooperativeKernel(mode == 0 ? (const void *)k_bits_round<0> : (const void *)k_bits_round<1>,
                                      dim3(grid), dim3(kBitsThreads), args, 0, g->stream));
  const int rb = std::min(g->num_sms * 4, std::max(1, (n + kBitsThreads - 1) / kBitsThreads));
  if (mode == 0) k_bits_argbest<0><<<rb, kBitsThreads, 0, g->stream>>>(out, g->dS, n, ctl);
  else k_bits_argbest<1><<<rb, kBitsThreads, 0, g->stream>>>(out, g->dS, n, ctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

}  // namespace gc
