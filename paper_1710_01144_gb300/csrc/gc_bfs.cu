// Grid-wide BFS kernels of libgc: the distance-to-group array d_S
// (Algorithm 2: SSSP from s0, then d_S <- min(d_S, d(s, .)) after each pick,
// done as a pruned SSSP per Sec. 4.1), group farness (Sec. 2), the round-0
// lower bound, and CSR validation.
#include <cooperative_groups.h>

#include <algorithm>

#include "gc_device.cuh"
#include "gc_grid.cuh"
#include "gc_internal.cuh"

namespace gc {

__global__ void k_fill_i32(int32_t *p, int32_t v, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}
__global__ void k_fill_i64(long long *p, long long v, int64_t count) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = v;
}

// Relabel BFS (cooperative, one launch for all levels).  Level L+1 labels go to
// every neighbour w of the level-L frontier with L+1 < dist[w]; only relabelled
// vertices enter the next frontier.  With dist = kInf this is a plain
// (multi-source) BFS; with dist = d_S and one seed s it is the pruned SSSP of
// Sec. 4.1 that turns d_S into min(d_S, d(s, .)): a vertex not strictly closer
// to s than to S keeps its label and is not expanded.  ctl->decrease collects
// sum(old - new) over relabelled vertices with a finite old label, i.e. the
// farness decrease Delta(s | S).
__global__ void __launch_bounds__(kBfsThreads) k_bfs_relabel(
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n, int32_t *dist,
    const int32_t *__restrict__ seeds, int32_t n_seeds, int32_t *q0, int32_t *q1, int32_t *st0, int32_t *st1,
    BfsCtl *ctl, unsigned long long timeout_ns, const int32_t *__restrict__ c3) {
  grid_relabel_bfs(rp, ci, n, dist, seeds, n_seeds, q0, q1, ctl->pk, &ctl->levels, &ctl->decrease,
                   &ctl->relabelled, st0, st1, &ctl->bar, &ctl->err, timeout_ns, nullptr, c3);
}

// sum(dist) and the count of unreached vertices; the last CTA to finish folds
// the per-CTA partials (ticket pattern, no waiting) into ctl->sum / ctl->count.
__global__ void __launch_bounds__(kRedThreads) k_sum_dist(const int32_t *__restrict__ dist, int32_t n,
                                                         long long *partial, SelCtl *ctl) {
  __shared__ long long sh[32];
  __shared__ bool last;
  long long s = 0, c = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int d = dist[i];
    if (d >= kInf) ++c;
    else s += d;
  }
  s = block_sum(s, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = s;
    partial[2 * blockIdx.x + 1] = c;
    __threadfence();
    last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
  }
  cta_sync();
  if (!last) return;
  __threadfence();
  s = 0;
  c = 0;
  for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    s += ((volatile long long *)partial)[2 * b];
    c += ((volatile long long *)partial)[2 * b + 1];
  }
  s = block_sum(s, sh);
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    ctl->sum = s;
    ctl->count = c;
    ctl->ticket = 0;
  }
}

// Round-0 lower bound on f({v}) (the BFScut idea of Sec. 3.1 with a degree
// bound for the second level): the deg(v) neighbours sit at distance 1; at
// most c2 = min(sum_{w in N(v)} (deg(w) - 1), n - 1 - deg(v)) vertices sit at
// distance 2 (every neighbour has v among its own neighbours); everything else
// is at least 3 away.  key[v] = -(deg + 2 c2 + 3 (n - 1 - deg - c2)).
// Row-wise kernels give a warp to each row up to kHeavyRow entries; longer
// rows (hubs) go to a whole CTA in a companion kernel, so that no warp walks a
// hub's row alone while the rest of the grid has finished.  The companions
// walk the list of long rows built once per graph (k_heavy_rows).

// heavy[0..*nh) = the rows with more than kHeavyRow entries (any order)
__global__ void __launch_bounds__(kRedThreads) k_heavy_rows(const int32_t *__restrict__ rp, int32_t n,
                                                            int32_t *heavy, int32_t *nh) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    if (rp[v + 1] - rp[v] > kHeavyRow) heavy[atomicAdd(nh, 1)] = v;
}

__global__ void __launch_bounds__(kRedThreads) k_round0_keys(const int32_t *__restrict__ rp,
                                                             const int32_t *__restrict__ ci,
                                                             int32_t n, long long *key, long long *two_hop) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int v = gwarp; v < n; v += nwarps) {
    const int beg = rp[v], end = rp[v + 1];
    if (end - beg > kHeavyRow) continue;  // k_round0_keys_heavy
    long long x = 0;
    for (int e = beg + lane; e < end; e += 32) {
      const int w = ci[e];
      x += (long long)(rp[w + 1] - rp[w] - 1);
    }
    x = warp_sum(x);
    if (lane == 0) {
      const long long deg = end - beg;
      long long rest = (long long)n - 1 - deg;
      if (rest < 0) rest = 0;
      const long long c2 = x < rest ? x : rest;
      key[v] = -(deg + 2 * c2 + 3 * (rest - c2));
      if (two_hop) two_hop[v] = x;
    }
  }
}

__global__ void __launch_bounds__(1024) k_round0_keys_heavy(const int32_t *__restrict__ rp,
                                                           const int32_t *__restrict__ ci, int32_t n,
                                                           long long *key, long long *two_hop, const int32_t *__restrict__ heavy, const int32_t *__restrict__ nh) {
  __shared__ long long s_red[32];
  for (int i = blockIdx.x; i < *nh; i += gridDim.x) {
    const int v = heavy[i];
    const int beg = rp[v], end = rp[v + 1];
    long long x = 0;
    for (int e = beg + threadIdx.x; e < end; e += 1024) {
      const int w = ci[e];
      x += (long long)(rp[w + 1] - rp[w] - 1);
    }
    x = block_sum(x, s_red);
    if (threadIdx.x == 0) {
      const long long deg = end - beg;
      long long rest = (long long)n - 1 - deg;
      if (rest < 0) rest = 0;
      const long long c2 = x < rest ? x : rest;
      key[v] = -(deg + 2 * c2 + 3 * (rest - c2));
      if (two_hop) two_hop[v] = x;
    }
  }
}

// Pivot lower bound for round 0.  For any vertex p and every w,
// d(v, w) >= |d(p, w) - d(p, v)| (triangle inequality), so with n_l vertices
// at distance l from p,
//   f({v}) >= LB_p(v) = sum_l n_l * |l - d(p, v)|,
// which prefix counts C[x] = sum_{l<x} n_l and prefix sums M[x] = sum_{l<x} l n_l
// give in O(1) per vertex:  x C[x] - M[x] + (M[D+1] - M[x+1]) - x (n - C[x+1]).
// The bound only decides which vertices still need an exact search.
__global__ void __launch_bounds__(kRedThreads) k_level_hist(const int32_t *__restrict__ dist, int32_t n,
                                                            unsigned long long *cnt, int32_t *maxlev) {
  int mloc = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const int x = dist[v];
    if (x >= 0 && x < n) {
      atomicAdd(&cnt[x], 1ull);
      mloc = max(mloc, x);
    }
  }
  for (int o = 16; o > 0; o >>= 1) mloc = max(mloc, __shfl_xor_sync(0xffffffffu, mloc, o));
  if ((threadIdx.x & 31) == 0) atomicMax(maxlev, mloc);
}

// One CTA: cnt[0..D] -> C[0..D+1] (exclusive prefix counts, in place of cnt
// shifted by one) and M[0..D+1]; D = *maxlev.  cnt is cleared for the next use.
__global__ void __launch_bounds__(1024) k_level_prefix(unsigned long long *cnt, const int32_t *maxlev,
                                                       unsigned long long *C, unsigned long long *M) {
  __shared__ unsigned long long s_c[1024], s_m[1024];
  __shared__ unsigned long long carry_c, carry_m;
  const int D = *maxlev;
  if (threadIdx.x == 0) {
    carry_c = 0;
    carry_m = 0;
  }
  cta_sync();
  for (int base = 0; base <= D; base += 1024) {
    const int l = base + threadIdx.x;
    const unsigned long long c = l <= D ? cnt[l] : 0ull;
    s_c[threadIdx.x] = c;
    s_m[threadIdx.x] = c * (unsigned long long)(l <= D ? l : 0);
    cta_sync();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive Hillis-Steele scan
      unsigned long long a = 0, b = 0;
      if (threadIdx.x >= o) {
        a = s_c[threadIdx.x - o];
        b = s_m[threadIdx.x - o];
      }
      cta_sync();
      s_c[threadIdx.x] += a;
      s_m[threadIdx.x] += b;
      cta_sync();
    }
    if (l <= D) {
      C[l + 1] = carry_c + s_c[threadIdx.x];
      M[l + 1] = carry_m + s_m[threadIdx.x];
      cnt[l] = 0;
    }
    cta_sync();
    if (threadIdx.x == 1023) {
      carry_c += s_c[1023];
      carry_m += s_m[1023];
    }
    cta_sync();
  }
  if (threadIdx.x == 0) {
    C[0] = 0;
    M[0] = 0;
  }
}

// key[v] = -max(LB(v), LB_p(v)) for vertices still undecided (key != INT64_MIN).
__global__ void __launch_bounds__(kRedThreads) k_pivot_bound(const int32_t *__restrict__ dist, int32_t n,
                                                             const unsigned long long *__restrict__ C,
                                                             const unsigned long long *__restrict__ M,
                                                             const int32_t *maxlev, long long *key) {
  const int D = *maxlev;
  const long long Mt = (long long)M[D + 1];
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const long long k0 = key[v];
    const int x = dist[v];
    if (k0 == LLONG_MIN || x < 0 || x > D) continue;
    const long long cx = (long long)C[x], cx1 = (long long)C[x + 1];
    const long long lb = (long long)x * cx - (long long)M[x] + (Mt - (long long)M[x + 1]) - (long long)x * ((long long)n - cx1);
    if (-lb < k0) key[v] = -lb;
  }
}

// Pruned adjacency for the rounds after round 0.  A neighbour w of u can be
// claimed (or relabelled) at level L+1 only if d_S[w] > L+1 >= 1, and d_S only
// decreases, so entries with d_S[w] <= 1 at the time of the build are useless
// in every later round.  The pruned row of u keeps the entries with d_S[w] >= 2,
// those with d_S[w] >= 3 first; c3[u] counts them.  Level 0 scans the whole
// pruned row, levels >= 1 (where d_S[w] > 2 is needed) only its first c3[u].
__global__ void __launch_bounds__(kRedThreads) k_prune_count(const int32_t *__restrict__ rp,
                                                             const int32_t *__restrict__ ci, int32_t n,
                                                             const int32_t *__restrict__ dS, int32_t *cnt2,
                                                             int32_t *c3) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int u = gwarp; u < n; u += nwarps) {
    const int r0 = rp[u], r1 = rp[u + 1];
    if (r1 - r0 > kHeavyRow) continue;  // k_prune_count_heavy
    int a2 = 0, a3 = 0;
    for (int e = r0 + lane; e < r1; e += 32) {
      const int d = dS[ci[e]];
      a2 += d >= 2;
      a3 += d >= 3;
    }
    a2 = warp_sum(a2);
    a3 = warp_sum(a3);
    if (lane == 0) {
      cnt2[u] = a2;
      c3[u] = a3;
    }
  }
}

// The long rows of k_prune_count, a CTA per row.
__global__ void __launch_bounds__(1024) k_prune_count_heavy(const int32_t *__restrict__ rp,
                                                           const int32_t *__restrict__ ci, int32_t n,
                                                           const int32_t *__restrict__ dS, int32_t *cnt2,
                                                           int32_t *c3, const int32_t *__restrict__ heavy, const int32_t *__restrict__ nh) {
  __shared__ long long s_red[32];
  for (int i = blockIdx.x; i < *nh; i += gridDim.x) {
    const int u = heavy[i];
    const int r0 = rp[u], r1 = rp[u + 1];
    long long a2 = 0, a3 = 0;
    for (int e = r0 + threadIdx.x; e < r1; e += 1024) {
      const int d = dS[ci[e]];
      a2 += d >= 2;
      a3 += d >= 3;
    }
    a2 = block_sum(a2, s_red);
    a3 = block_sum(a3, s_red);
    if (threadIdx.x == 0) {
      cnt2[u] = (int32_t)a2;
      c3[u] = (int32_t)a3;
    }
  }
}

// One pass per row, two cursors: entries with d_S >= 3 go to the front of the
// pruned row, entries with d_S == 2 after the c3[u] of them.  A warp per row;
// rows longer than kHeavyRow are left to k_prune_fill_heavy.
__global__ void __launch_bounds__(kRedThreads) k_prune_fill(const int32_t *__restrict__ rp,
                                                            const int32_t *__restrict__ ci, int32_t n,
                                                            const int32_t *__restrict__ dS,
                                                            const int32_t *__restrict__ rpf,
                                                            const int32_t *__restrict__ c3, int32_t *cif) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int u = gwarp; u < n; u += nwarps) {
    const int r0 = rp[u], r1 = rp[u + 1];
    if (r1 - r0 > kHeavyRow) continue;
    int p3 = rpf[u], p2 = p3 + c3[u];
    for (int e0 = r0; e0 < r1; e0 += 32) {
      const int e = e0 + lane;
      int w = 0, d = 0;
      if (e < r1) {
        w = ci[e];
        d = dS[w];
      }
      const unsigned m3 = __ballot_sync(0xffffffffu, e < r1 && d >= 3);
      const unsigned m2 = __ballot_sync(0xffffffffu, e < r1 && d == 2);
      const unsigned below = (1u << lane) - 1u;
      if (e < r1 && d >= 3) cif[p3 + __popc(m3 & below)] = w;
      if (e < r1 && d == 2) cif[p2 + __popc(m2 & below)] = w;
      p3 += __popc(m3);
      p2 += __popc(m2);
    }
  }
}

// The long rows of k_prune_fill: each CTA takes whole rows, 1024 entries at a
// time, with block scans for the two cursors.
__global__ void __launch_bounds__(1024) k_prune_fill_heavy(const int32_t *__restrict__ rp,
                                                          const int32_t *__restrict__ ci, int32_t n,
                                                          const int32_t *__restrict__ dS,
                                                          const int32_t *__restrict__ rpf,
                                                          const int32_t *__restrict__ c3, int32_t *cif, const int32_t *__restrict__ heavy, const int32_t *__restrict__ nh) {
  __shared__ int s_scan[33];
  for (int i = blockIdx.x; i < *nh; i += gridDim.x) {
    const int u = heavy[i];
    const int r0 = rp[u], r1 = rp[u + 1];
    int p3 = rpf[u], p2 = p3 + c3[u];
    for (int e0 = r0; e0 < r1; e0 += 1024) {
      const int e = e0 + threadIdx.x;
      int w = 0, d = 0;
      if (e < r1) {
        w = ci[e];
        d = dS[w];
      }
      const int f3 = e < r1 && d >= 3, f2 = e < r1 && d == 2;
      int t3, t2;
      const int x3 = block_excl_scan(f3, s_scan, &t3);
      const int x2 = block_excl_scan(f2, s_scan, &t2);
      if (f3) cif[p3 + x3] = w;
      if (f2) cif[p2 + x2] = w;
      p3 += t3;
      p2 += t2;
    }
  }
}

// Exclusive prefix sum of cnt[0..n) into out[0..n] (out[n] = total), three
// launches: per-tile sums, a one-CTA scan of the tile sums, per-tile scans.
constexpr int kScanTile = 4096;

__global__ void __launch_bounds__(1024) k_scan_tiles(const int32_t *__restrict__ cnt, int32_t n,
                                                    long long *tile_sum) {
  __shared__ long long s[32];
  long long a = 0;
  const int base = blockIdx.x * kScanTile;
  for (int i = threadIdx.x; i < kScanTile; i += 1024)
    if (base + i < n) a += cnt[base + i];
  a = block_sum(a, s);
  if (threadIdx.x == 0) tile_sum[blockIdx.x] = a;
}

__global__ void __launch_bounds__(1024) k_scan_tops(long long *tile_sum, int32_t tiles) {
  __shared__ int s_scan[33];
  long long carry = 0;
  for (int base = 0; base < tiles; base += 1024) {
    const int i = base + threadIdx.x;
    const long long v = i < tiles ? tile_sum[i] : 0;
    int tot;
    // tile sums fit int32 here: the CSR has fewer than 2^31 entries
    const int ex = block_excl_scan((int)v, s_scan, &tot);
    if (i < tiles) tile_sum[i] = carry + ex;
    carry += tot;
    cta_sync();
  }
}

__global__ void __launch_bounds__(1024) k_scan_apply(const int32_t *__restrict__ cnt, int32_t n,
                                                    const long long *__restrict__ tile_sum, int32_t *out) {
  __shared__ int s_scan[33];
  const int base = blockIdx.x * kScanTile;
  long long carry = tile_sum[blockIdx.x];
  for (int off = 0; off < kScanTile; off += 1024) {
    const int i = base + off + threadIdx.x;
    const int v = i < n ? cnt[i] : 0;
    int tot;
    const int ex = block_excl_scan(v, s_scan, &tot);
    if (i < n) out[i] = (int32_t)(carry + ex);
    if (i == n - 1) out[n] = (int32_t)(carry + ex + v);
    carry += tot;
    cta_sync();
  }
}

// mx[u] = max over neighbours w of d_S[w].  d_S only decreases as the group
// grows, so the value stays an upper bound; a frontier vertex u at level L can
// claim a neighbour only if that neighbour's d_S exceeds L+1, so mx[u] <= L+1
// means expanding u is useless (the pruning test of Sec. 4.1 applied one level
// ahead).
__global__ void __launch_bounds__(kRedThreads) k_max_nbr(const int32_t *__restrict__ rp,
                                                         const int32_t *__restrict__ ci, int32_t n,
                                                         const int32_t *__restrict__ dS, int32_t *mx) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int v = gwarp; v < n; v += nwarps) {
    if (rp[v + 1] - rp[v] > kHeavyRow) continue;  // k_max_nbr_heavy
    int m = 0;
    for (int e = rp[v] + lane; e < rp[v + 1]; e += 32) m = max(m, dS[ci[e]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    if (lane == 0) mx[v] = m;
  }
}

__global__ void __launch_bounds__(1024) k_max_nbr_heavy(const int32_t *__restrict__ rp,
                                                       const int32_t *__restrict__ ci, int32_t n,
                                                       const int32_t *__restrict__ dS, int32_t *mx, const int32_t *__restrict__ heavy, const int32_t *__restrict__ nh) {
  __shared__ int s_m[32];
  for (int i = blockIdx.x; i < *nh; i += gridDim.x) {
    const int v = heavy[i];
    int m = 0;
    for (int e = rp[v] + threadIdx.x; e < rp[v + 1]; e += 1024) m = max(m, dS[ci[e]]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
    cta_sync();
    if ((threadIdx.x & 31) == 0) s_m[threadIdx.x >> 5] = m;
    cta_sync();
    if (threadIdx.x < 32) {
      m = s_m[threadIdx.x];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (threadIdx.x == 0) mx[v] = m;
    }
  }
}

// Round-1 upper bounds.  With S = {s0} and d_S = d(s0, .), every candidate v
// satisfies
//   Delta(v|S) <= d_S[v] + sum_{w in N(v)} ((d_S[w] - 1)^+ + c3[w]) + G3,
//   G3 = sum_u (d_S[u] - 3)^+,
// because a vertex u at distance 1 from v gains at most d_S[u] - 1; one at
// distance 2 gains at most (d_S[u] - 2)^+ = [d_S[u] >= 3] + (d_S[u] - 3)^+,
// and each such u with d_S[u] >= 3 is a neighbour of some w in N(v), counted
// by c3[w] (neighbours of w with d_S >= 3); farther vertices gain at most
// (d_S[u] - 3)^+; and the (d_S - 3)^+ terms of all of them sum to at most G3.
// A neighbour w with d_S[w] <= 1 adds nothing (its own term is 0 and its
// neighbours have d_S <= 2), so the pruned rows (d_S[w] >= 2) suffice.  The
// bounds replace the +infinity of round 1 (Sec. 4.2 gives none), so the lazy
// rule of round 1 evaluates only the candidates whose bound reaches the best
// exact gain.  ub[v] <- the bound (members of S: -1), stamp[v] <- 0.
__global__ void __launch_bounds__(kRedThreads) k_excess3(const int32_t *__restrict__ dS, int32_t n,
                                                         unsigned long long *g3) {
  __shared__ long long sh[32];
  long long s = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int d = dS[i];
    if (d > 3) s += d - 3;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0 && s) atomicAdd(g3, (unsigned long long)s);
}

// A warp per row; rows longer than kHeavyRow (full adjacency) are left to
// k_round1_bound_heavy.
__global__ void __launch_bounds__(kRedThreads) k_round1_bound(const int32_t *__restrict__ rpf,
                                                              const int32_t *__restrict__ cif,
                                                              const int32_t *__restrict__ rp, int32_t n,
                                                              const int32_t *__restrict__ dS,
                                                              const int32_t *__restrict__ c3,
                                                              const unsigned long long *__restrict__ g3,
                                                              long long *ub, int32_t *stamp) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const long long G3 = (long long)*g3;
  for (int v = gwarp; v < n; v += nwarps) {
    if (rp[v + 1] - rp[v] > kHeavyRow) continue;  // k_round1_bound_heavy
    long long s = 0;
    for (int e = rpf[v] + lane; e < rpf[v + 1]; e += 32) {
      const int w = cif[e];
      s += (long long)max(dS[w] - 1, 0) + (long long)c3[w];
    }
    s = warp_sum(s);
    if (lane == 0) {
      const int dv = dS[v];
      ub[v] = dv == 0 ? -1ll : (long long)dv + s + G3;
      stamp[v] = 0;
    }
  }
}

// The long rows of k_round1_bound, a CTA per row.
__global__ void __launch_bounds__(1024) k_round1_bound_heavy(const int32_t *__restrict__ rpf,
                                                            const int32_t *__restrict__ cif,
                                                            const int32_t *__restrict__ dS,
                                                            const int32_t *__restrict__ c3,
                                                            const unsigned long long *__restrict__ g3,
                                                            long long *ub, int32_t *stamp,
                                                            const int32_t *__restrict__ heavy,
                                                            const int32_t *__restrict__ nh) {
  __shared__ long long s_red[32];
  const long long G3 = (long long)*g3;
  for (int i = blockIdx.x; i < *nh; i += gridDim.x) {
    const int v = heavy[i];
    long long s = 0;
    for (int e = rpf[v] + threadIdx.x; e < rpf[v + 1]; e += 1024) {
      const int w = cif[e];
      s += (long long)max(dS[w] - 1, 0) + (long long)c3[w];
    }
    s = block_sum(s, s_red);
    if (threadIdx.x == 0) {
      const int dv = dS[v];
      ub[v] = dv == 0 ? -1ll : (long long)dv + s + G3;
      stamp[v] = 0;
    }
  }
}

// Bound refresh for later rounds.  The inequality of k_round1_bound holds for
// any group S with d_S, c3 and G3 taken for that S, and it tightens as S grows.
// k_count3 recounts, for the current d_S, the neighbours with d_S >= 3 of every
// vertex (they are all in the pruned rows: d_S only decreases); k_bound_refresh
// lowers every candidate's bound to the recomputed value.  A candidate already
// evaluated in the current round keeps its exact gain (the bound is above it).
__global__ void __launch_bounds__(kRedThreads) k_count3(const int32_t *__restrict__ rpf,
                                                        const int32_t *__restrict__ cif,
                                                        const int32_t *__restrict__ rp, int32_t n,
                                                        const int32_t *__restrict__ dS, int32_t *c3s) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int u = gwarp; u < n; u += nwarps) {
    if (rp[u + 1] - rp[u] > kHeavyRow) continue;  // k_count3_heavy
    int a = 0;
    for (int e = rpf[u] + lane; e < rpf[u + 1]; e += 32) a += dS[cif[e]] >= 3;
    a = warp_sum(a);
    if (lane == 0) c3s[u] = a;
  }
}

__global__ void __launch_bounds__(1024) k_count3_heavy(const int32_t *__restrict__ rpf,
                                                      const int32_t *__restrict__ cif,
                                                      const int32_t *__restrict__ dS, int32_t *c3s,
                                                      const int32_t *__restrict__ heavy,
                                                      const int32_t *__restrict__ nh) {
  __shared__ long long s_red[32];
  for (int i = blockIdx.x; i < *nh; i += gridDim.x) {
    const int u = heavy[i];
    long long a = 0;
    for (int e = rpf[u] + threadIdx.x; e < rpf[u + 1]; e += 1024) a += dS[cif[e]] >= 3;
    a = block_sum(a, s_red);
    if (threadIdx.x == 0) c3s[u] = (int32_t)a;
  }
}

__global__ void __launch_bounds__(kRedThreads) k_bound_refresh(const int32_t *__restrict__ rpf,
                                                               const int32_t *__restrict__ cif,
                                                               const int32_t *__restrict__ rp, int32_t n,
                                                               const int32_t *__restrict__ dS,
                                                               const int32_t *__restrict__ c3s,
                                                               const unsigned long long *__restrict__ g3,
                                                               long long *ub) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  const long long G3 = (long long)*g3;
  for (int v = gwarp; v < n; v += nwarps) {
    if (rp[v + 1] - rp[v] > kHeavyRow) continue;  // k_bound_refresh_heavy
    if (ub[v] < 0) continue;                       // a member (warp-uniform: one v per warp)
    long long s = 0;
    for (int e = rpf[v] + lane; e < rpf[v + 1]; e += 32) {
      const int w = cif[e];
      s += (long long)max(dS[w] - 1, 0) + (long long)c3s[w];
    }
    s = warp_sum(s);
    if (lane == 0) {
      const long long b = (long long)dS[v] + s + G3;
      if (b < ub[v]) ub[v] = b;
    }
  }
}

__global__ void __launch_bounds__(1024) k_bound_refresh_heavy(const int32_t *__restrict__ rpf,
                                                             const int32_t *__restrict__ cif,
                                                             const int32_t *__restrict__ dS,
                                                             const int32_t *__restrict__ c3s,
                                                             const unsigned long long *__restrict__ g3,
                                                             long long *ub, const int32_t *__restrict__ heavy,
                                                             const int32_t *__restrict__ nh) {
  __shared__ long long s_red[32];
  const long long G3 = (long long)*g3;
  for (int i = blockIdx.x; i < *nh; i += gridDim.x) {
    const int v = heavy[i];
    if (ub[v] < 0) continue;  // block-uniform
    long long s = 0;
    for (int e = rpf[v] + threadIdx.x; e < rpf[v + 1]; e += 1024) {
      const int w = cif[e];
      s += (long long)max(dS[w] - 1, 0) + (long long)c3s[w];
    }
    s = block_sum(s, s_red);
    if (threadIdx.x == 0) {
      const long long b = (long long)dS[v] + s + G3;
      if (b < ub[v]) ub[v] = b;
    }
  }
}

// CSR validation, part 1: row_ptr monotone within [0, nnz].
__global__ void k_validate_rowptr(const int32_t *__restrict__ rp, int32_t n, int64_t nnz,
                                  SelCtl *ctl) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int a = rp[i], b = rp[i + 1];
    if (a < 0 || b < a || (int64_t)b > nnz) atomicExch(&ctl->err, GC_EINVAL);
  }
}

// CSR validation, part 2 (only after part 1 passed): ids in range, no
// self-loop, strictly increasing rows, and every edge (u, w) mirrored by
// (w, u) (binary search in the sorted row of w).
__global__ void k_validate_rows(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                int32_t n, SelCtl *ctl) {
  const int lane = threadIdx.x & 31;
  const int gwarp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int nwarps = (gridDim.x * blockDim.x) >> 5;
  for (int u = gwarp; u < n; u += nwarps) {
    const int beg = rp[u], end = rp[u + 1];
    for (int e = beg + lane; e < end; e += 32) {
      const int w = ci[e];
      bool bad = (w < 0 || w >= n || w == u || (e > beg && ci[e - 1] >= w));
      if (!bad) {
        int lo = rp[w], hi = rp[w + 1];
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (ci[mid] < u) lo = mid + 1;
          else hi = mid;
        }
        bad = !(lo < rp[w + 1] && ci[lo] == u);
      }
      if (bad) atomicExch(&ctl->err, GC_EINVAL);
    }
  }
}

// ------------------------------------------------------------- launchers ----
static int grid_for(int64_t count, int threads, int cap) {
  int64_t b = (count + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > cap) b = cap;
  return (int)b;
}

int launch_fill_i32(gc_graph *g, int32_t *p, int32_t v, int64_t count) {
  if (count <= 0) return GC_OK;
  ++g->launches;
  k_fill_i32<<<grid_for(count, 256, g->num_sms * 8), 256, 0, g->stream>>>(p, v, count);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}
int launch_fill_i64(gc_graph *g, long long *p, long long v, int64_t count) {
  if (count <= 0) return GC_OK;
  ++g->launches;
  k_fill_i64<<<grid_for(count, 256, g->num_sms * 8), 256, 0, g->stream>>>(p, v, count);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_bfs_relabel(gc_graph *g, int32_t *dist, const int32_t *seeds, int32_t n_seeds,
                       int64_t timeout_ns, bool pruned) {
  GC_CUDA(cudaMemsetAsync(g->bctl, 0, sizeof(BfsCtl), g->stream));
  const int32_t *rp = pruned ? g->rpf : g->rp, *ci = pruned ? g->cif : g->ci;
  const int32_t *c3 = pruned ? g->c3 : nullptr;
  int32_t n = g->n;
  int32_t *q0 = g->bq0, *q1 = g->bq1, *st0 = g->goff, *st1 = g->gx;
  BfsCtl *ctl = g->bctl;
  unsigned long long tns = (unsigned long long)timeout_ns;
  void *args[] = {(void *)&rp,      (void *)&ci, (void *)&n,  (void *)&dist, (void *)&seeds,
                  (void *)&n_seeds, (void *)&q0, (void *)&q1, (void *)&st0, (void *)&st1, (void *)&ctl,
                  (void *)&tns, (void *)&c3};
  ++g->launches;
  GC_CUDA(cudaLaunchCooperativeKernel((const void *)k_bfs_relabel, dim3(std::min(g->bfs_ctas, kMaxGridCtas)),
                                      dim3(kBfsThreads), args, 0, g->stream));
  return GC_OK;
}

int bfs_kernel_occupancy(int *blocks_per_sm) {
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_bfs_relabel, kBfsThreads, 0));
  return GC_OK;
}

int launch_sum_dist(gc_graph *g, const int32_t *dist) {
  ++g->launches;
  k_sum_dist<<<g->red_blocks, kRedThreads, 0, g->stream>>>(dist, g->n, g->partial, g->sctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_round0_keys(gc_graph *g) {
  ++g->launches;
  k_round0_keys<<<grid_for((int64_t)g->n * 32, kRedThreads, g->num_sms * 8), kRedThreads, 0,
                  g->stream>>>(g->rp, g->ci, g->n, g->key, g->two_hop);
  ++g->launches;
  k_round0_keys_heavy<<<g->num_sms * 2, 1024, 0, g->stream>>>(g->rp, g->ci, g->n, g->key, g->two_hop,
                                                              g->heavy, g->n_heavy);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_pivot_bound(gc_graph *g) {
  g->launches += 3;
  GC_CUDA(cudaMemsetAsync(g->lev_max, 0, sizeof(int32_t), g->stream));
  k_level_hist<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->dS, g->n, g->lev_cnt, g->lev_max);
  k_level_prefix<<<1, 1024, 0, g->stream>>>(g->lev_cnt, g->lev_max, g->lev_C, g->lev_M);
  k_pivot_bound<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->dS, g->n, g->lev_C, g->lev_M, g->lev_max,
                                                              g->key);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_prune_csr(gc_graph *g) {
  const int n = g->n;
  const int tiles = (n + kScanTile - 1) / kScanTile;
  const int grid = grid_for((int64_t)n * 32, kRedThreads, g->num_sms * 8);
  g->launches += 7;
  k_prune_count<<<grid, kRedThreads, 0, g->stream>>>(g->rp, g->ci, n, g->dS, g->io_a, g->c3);
  k_prune_count_heavy<<<g->num_sms * 2, 1024, 0, g->stream>>>(g->rp, g->ci, n, g->dS, g->io_a, g->c3, g->heavy,
                                                              g->n_heavy);
  k_scan_tiles<<<tiles, 1024, 0, g->stream>>>(g->io_a, n, g->lgain);
  k_scan_tops<<<1, 1024, 0, g->stream>>>(g->lgain, tiles);
  k_scan_apply<<<tiles, 1024, 0, g->stream>>>(g->io_a, n, g->lgain, g->rpf);
  k_prune_fill<<<grid, kRedThreads, 0, g->stream>>>(g->rp, g->ci, n, g->dS, g->rpf, g->c3, g->cif);
  k_prune_fill_heavy<<<g->num_sms * 2, 1024, 0, g->stream>>>(g->rp, g->ci, n, g->dS, g->rpf, g->c3, g->cif,
                                                             g->heavy, g->n_heavy);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_round1_bound(gc_graph *g) {
  const int n = g->n;
  g->launches += 3;
  GC_CUDA(cudaMemsetAsync(g->g3, 0, sizeof(unsigned long long), g->stream));
  k_excess3<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->dS, n, g->g3);
  k_round1_bound<<<grid_for((int64_t)n * 32, kRedThreads, g->num_sms * 8), kRedThreads, 0, g->stream>>>(
      g->rpf, g->cif, g->rp, n, g->dS, g->c3, g->g3, g->ub, g->stamp);
  k_round1_bound_heavy<<<g->num_sms * 2, 1024, 0, g->stream>>>(g->rpf, g->cif, g->dS, g->c3, g->g3, g->ub,
                                                               g->stamp, g->heavy, g->n_heavy);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

// Round-0 work estimate: the sum over list[0..m) of two_hop[v] (sum over the
// neighbours of v of deg - 1), the adjacency entries a search from v scans to
// reach distance 2.  Accumulated into *out (zeroed by the caller).
__global__ void k_sum_two_hop(const int32_t *__restrict__ list, const int32_t *m_dev,
                              const long long *__restrict__ two_hop, unsigned long long *out) {
  __shared__ long long sh[32];
  const int m = *m_dev;
  long long s = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) s += two_hop[list[i]];
  s = block_sum(s, sh);
  if (threadIdx.x == 0 && s) atomicAdd(out, (unsigned long long)s);
}

int launch_sum_two_hop(gc_graph *g, unsigned long long *out) {
  ++g->launches;
  GC_CUDA(cudaMemsetAsync(out, 0, sizeof(unsigned long long), g->stream));
  k_sum_two_hop<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->list, &g->sctl->n_sel, g->two_hop, out);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

// ub[v] = -1 for members (d_S[v] = 0), +infinity for every other vertex: the
// starting point of k_bound_refresh when no earlier bound exists.
__global__ void k_init_ub(const int32_t *__restrict__ dS, int32_t n, long long *ub) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    ub[v] = dS[v] == 0 ? -1ll : LLONG_MAX;
}

int launch_init_ub(gc_graph *g) {
  ++g->launches;
  k_init_ub<<<grid_for(g->n, 256, g->num_sms * 8), 256, 0, g->stream>>>(g->dS, g->n, g->ub);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_bound_refresh(gc_graph *g) {
  const int n = g->n;
  const int grid = grid_for((int64_t)n * 32, kRedThreads, g->num_sms * 8);
  g->launches += 5;
  GC_CUDA(cudaMemsetAsync(g->g3, 0, sizeof(unsigned long long), g->stream));
  k_excess3<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->dS, n, g->g3);
  k_count3<<<grid, kRedThreads, 0, g->stream>>>(g->rpf, g->cif, g->rp, n, g->dS, g->c3s);
  k_count3_heavy<<<g->num_sms * 2, 1024, 0, g->stream>>>(g->rpf, g->cif, g->dS, g->c3s, g->heavy, g->n_heavy);
  k_bound_refresh<<<grid, kRedThreads, 0, g->stream>>>(g->rpf, g->cif, g->rp, n, g->dS, g->c3s, g->g3, g->ub);
  k_bound_refresh_heavy<<<g->num_sms * 2, 1024, 0, g->stream>>>(g->rpf, g->cif, g->dS, g->c3s, g->g3, g->ub,
                                                                g->heavy, g->n_heavy);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_heavy_rows(gc_graph *g) {
  ++g->launches;
  GC_CUDA(cudaMemsetAsync(g->n_heavy, 0, sizeof(int32_t), g->stream));
  k_heavy_rows<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->rp, g->n, g->heavy, g->n_heavy);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_max_nbr(gc_graph *g) {
  ++g->launches;
  k_max_nbr<<<grid_for((int64_t)g->n * 32, kRedThreads, g->num_sms * 8), kRedThreads, 0, g->stream>>>(
      g->rp, g->ci, g->n, g->dS, g->mx_buf);
  ++g->launches;
  k_max_nbr_heavy<<<g->num_sms * 2, 1024, 0, g->stream>>>(g->rp, g->ci, g->n, g->dS, g->mx_buf, g->heavy,
                                                          g->n_heavy);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_validate(gc_graph *g) {
  GC_CUDA(cudaMemsetAsync(&g->sctl->err, 0, sizeof(int32_t), g->stream));
  ++g->launches;
  k_validate_rowptr<<<grid_for(g->n, 256, g->num_sms * 8), 256, 0, g->stream>>>(g->rp, g->n, g->nnz,
                                                                                 g->sctl);
  GC_CUDA(cudaGetLastError());
  GC_CUDA(cudaMemcpyAsync(&g->h_sctl->err, &g->sctl->err, sizeof(int32_t), cudaMemcpyDeviceToHost,
                          g->stream));
  GC_CUDA(cudaStreamSynchronize(g->stream));
  if (g->h_sctl->err) return GC_EINVAL;
  ++g->launches;
  k_validate_rows<<<grid_for((int64_t)g->n * 32, 256, g->num_sms * 8), 256, 0, g->stream>>>(
      g->rp, g->ci, g->n, g->sctl);
  GC_CUDA(cudaGetLastError());
  GC_CUDA(cudaMemcpyAsync(&g->h_sctl->err, &g->sctl->err, sizeof(int32_t), cudaMemcpyDeviceToHost,
                          g->stream));
  GC_CUDA(cudaStreamSynchronize(g->stream));
  return g->h_sctl->err ? GC_EINVAL : GC_OK;
}

}  // namespace gc
