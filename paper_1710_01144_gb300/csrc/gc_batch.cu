// Batched Greedy++ over many graphs in ONE persistent cooperative launch.
//
// The batch is stored as one block-diagonal union CSR (global vertex ids;
// graph g owns ids [off[g], off[g+1])).  Distances never cross components, so
// the multi-source relabel BFS computes every graph's BFS at once (one seed
// per graph), and 64-lane gain batches stay inside one graph.  What is per
// graph -- round-0 cut thresholds, argmin/argmax, the lazy round state and its
// acceptance test (Sec. 4.2), the group -- lives in per-graph arrays.
//
// Phases (bounded grid barriers between them):
//   P0  lower bounds LB(v) and, per graph, the vertex v_a of smallest bound
//   P1  BFS from all v_a; per-graph farness f_a
//   P2  every v with LB(v) <= f_a evaluated by the 64-lane BFS in farness
//       mode with per-graph cuts (graph-aligned batches from a dynamic task
//       counter over all CTAs); per graph s0 = argmin (f, id)
//   P3  BFS from all s0 (d_S), per-graph farness, neighbour bound mx
//   P4  round 1: every candidate of every graph, graph-aligned 64-lane batches
//       from a dynamic task counter; per-graph argmax; picks; BFS from picks
//   P5  per graph (one CTA): active list of the largest bounds
//   P6  lazy rounds: each CTA runs its graphs' rounds to completion -- fold,
//       decide, select 64, evaluate them (64-lane BFS), and on acceptance a
//       CTA-local pruned BFS from the pick -- so no graph waits for another.
//   P7  check: one BFS from every graph's whole group; each graph's farness
//       must equal f(s0) minus the sum of its accepted gains.
#include <limits.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <string>
#include <vector>

#include "gc_cta.cuh"
#include "gc_lazy.cuh"

namespace gc {

struct BatchCtl {
  GridBar bar;
  int32_t err;
  int32_t remaining;  // graphs that still need lazy rounds
  int32_t nseeds;     // seeds of the next relabel BFS
  int32_t task;       // dynamic task counter of P4
  int32_t pad0;
  unsigned long long pk[3];  // relabel BFS frontiers (see BfsCtl)
  int32_t pad;
  unsigned long long decrease;
  long long iterations;
  long long dbg[4];  // first failed check: phase, graph, expected, found
  unsigned long long ns_ph[6];  // end of round 0 (P2), round 1 (P5), lazy rounds (P6), check (P7),
                                // start and end of the round-1 gains (P4)
  unsigned long long ns_lazy[3];  // lazy rounds, summed over graphs: selection (with list
                                  // rebuilds), gain batches, d_S updates
  int32_t blk_tot[kMaxGridCtas];
};

static __device__ void check_fail(BatchCtl *c, int phase, int g, long long want, long long got) {
  if (atomicCAS((unsigned long long *)&c->dbg[0], 0ull, (unsigned long long)phase) == 0ull) {
    c->dbg[1] = g;
    c->dbg[2] = want;
    c->dbg[3] = got;
  }
  atomicExch(&c->err, GC_EINTERNAL);
}

struct BatchArgs {
  const int32_t *rp, *ci;
  int32_t N;
  int32_t count;
  const int32_t *gid, *off, *ng, *kk, *iota;
  const int32_t *bstart;  // round-1 task prefix per graph ([count+1])
  int32_t lanes1;         // candidates per round-1 batch
  int32_t max_n;          // vertices of the largest graph (workspace layout)
  int32_t *dS, *mx, *stamp, *q0, *q1, *goff, *st1;
  int32_t *rpf, *cif, *c3;  // pruned adjacency for rounds >= 1 (built in P3)
  int32_t *dS1;             // d(s0, .) as of P3, never written after: round 1 reads it read-only
  long long *ub, *key, *f0;
  unsigned char *ws;
  size_t ws_stride;
  unsigned long long *packed;
  long long *fa, *farness, *bestf;
  LazyCtl *lc;
  int32_t *act, *act_n, *full;
  int32_t A;
  int32_t kmax;
  int32_t *picks;
  long long *pgain;
  int32_t *seeds;  // [max(count, sum k)]
  int32_t *slist;  // round-0 survivors, graph-aligned [N]
  int32_t *scount, *tstart;  // per-graph survivor counts, task prefix [count+1]
  BatchCtl *ctl;
  GainCtl *gctl;
  GridGainCtl *gg;    // grid-wide batches of the big graphs' lazy rounds
  GridSelScratch *gsel;  // their grid-wide selection
  int32_t *gx;        // their scratch: 3 * max_n
  int32_t grid_min_n; // graphs with at least this many vertices run their lazy rounds grid-wide
  int32_t bounded;    // round 1 with two-hop bounds (batch_round1_bounded) and the refresh after it
  long long *g3;      // [2 * count]: sum of (d - 3)^+ per graph for round 1, then for the refresh
  unsigned long long tns;
};

constexpr int kBatchThreads = kGainThreads;
// lazy rounds grid-wide from this many vertices.  On the 256-graph mix
// (10^4 to 5 x 10^5 vertices per graph) the whole solve took 1.72 s with
// 65,536, 1.70 s with 262,144 and 1.56 s with every graph CTA-local: one CTA
// per graph in parallel beats graphs of that size taking the grid in turn, so
// only much larger graphs go grid-wide
constexpr int32_t kBatchGridMinN = 1 << 21;

static __device__ __forceinline__ bool bsync(const BatchArgs &a) { return grid_sync(&a.ctl->bar, &a.ctl->err, a.tns); }

// The pruned adjacency of the single-graph path (k_prune_count in gc_bfs.cu)
// over the union CSR, built inside the solve once d_S = d(s0, .) is known:
// rows keep the neighbours with d_S >= 2, those with d_S >= 3 first (c3 of
// them).  Count per vertex into a.q0 (free here), scan across CTAs (each
// CTA owns a contiguous vertex range), fill.  Three grid barriers.
static __device__ bool batch_prune(const BatchArgs &a) {
  __shared__ int s_scan[33];
  __shared__ long long s_off[kMaxGridCtas + 1];
  const int tid = threadIdx.x, lane = tid & 31, T = blockDim.x, G = gridDim.x, b = blockIdx.x;
  const int gw = (b * T + tid) >> 5, nw = (G * T) >> 5;
  for (int u = gw; u < a.N; u += nw) {
    int a2 = 0, a3 = 0;
    for (int e = a.rp[u] + lane; e < a.rp[u + 1]; e += 32) {
      const int d = a.dS[a.ci[e]];
      a2 += d >= 2;
      a3 += d >= 3;
    }
    a2 = warp_sum(a2);
    a3 = warp_sum(a3);
    if (lane == 0) {
      a.q0[u] = a2;
      a.c3[u] = a3;
    }
  }
  if (!bsync(a)) return false;
  const int P = (a.N + G - 1) / G;
  const int lo = min(a.N, b * P), hi = min(a.N, lo + P);
  long long mine = 0;
  for (int v = lo + tid; v < hi; v += T) mine += a.q0[v];
  mine = block_sum(mine, (long long *)s_off);
  if (tid == 0) a.ctl->blk_tot[b] = (int32_t)mine;  // < 2^31: the CSR has fewer entries
  if (!bsync(a)) return false;
  long long run = 0;
  for (int base = 0; base < G; base += T) {
    const int j = base + tid;
    const int v = j < G ? ((volatile int32_t *)a.ctl->blk_tot)[j] : 0;
    int total;
    const int off = block_excl_scan(v, s_scan, &total);
    if (j < G) s_off[j] = run + off;
    run += total;
    cta_sync();
  }
  long long carry = s_off[b];
  cta_sync();
  for (int base = lo; base < hi; base += T) {
    const int v = base + tid;
    const int x = v < hi ? a.q0[v] : 0;
    int total;
    const int off = block_excl_scan(x, s_scan, &total);
    if (v < hi) a.rpf[v] = (int32_t)(carry + off);
    carry += total;
  }
  if (b == G - 1 && tid == 0) a.rpf[a.N] = (int32_t)run;
  if (!bsync(a)) return false;
  for (int u = gw; u < a.N; u += nw) {
    int pos = a.rpf[u];
    for (int pass = 0; pass < 2; ++pass) {  // d_S >= 3 first, then d_S == 2
      for (int e0 = a.rp[u]; e0 < a.rp[u + 1]; e0 += 32) {
        const int e = e0 + lane;
        int w = 0;
        bool keep = false;
        if (e < a.rp[u + 1]) {
          w = a.ci[e];
          const int d = a.dS[w];
          keep = pass == 0 ? d >= 3 : d == 2;
        }
        const unsigned m = __ballot_sync(0xffffffffu, keep);
        if (keep) a.cif[pos + __popc(m & ((1u << lane) - 1u))] = w;
        pos += __popc(m);
      }
    }
  }
  return bsync(a);
}


static __device__ bool grid_refresh_graph(const BatchArgs &a, int g);
static __device__ void cta_build_list(const BatchArgs &a, int g);

// Lazy rounds (Sec. 4.2) of one big graph g by the whole grid: every CTA
// takes part in each step's decision and selection (grid_lazy_step) over the
// graph's active list (built in P5), evaluates the 64 selected as one
// grid-wide 64-lane batch, and each pick updates d_S by the grid relabel BFS,
// checked against the pick's gain.  When the list cannot certify a pick, the
// graph's bounds are refreshed and the list rebuilt; a second failure in the
// same round lists every candidate from then on.  Every CTA runs the same loop.
static __device__ bool batch_grid_lazy(const BatchArgs &a, int g) {
  const int tid = threadIdx.x, b = blockIdx.x;
  LazyCtl *lc = &a.lc[g];
  const int o = a.off[g], ng = a.ng[g];
  bool every = false, fold = false;
  int rebuilt = -1;  // round of the last rebuild
  unsigned long long t_ph[3] = {0, 0, 0}, t_mark = global_ns();  // CTA 0's phase clocks
  auto lap = [&](int q) {
    if (b == 0 && tid == 0) {
      const unsigned long long now = global_ns();
      t_ph[q] += now - t_mark;
      t_mark = now;
    }
    __syncwarp();  // reconverge warp 0 before the warp-synchronous code that follows
  };
  for (;;) {
    const int r = *(volatile int32_t *)&lc->round;
    if (r >= a.kk[g]) break;
    const int32_t *list = every ? a.iota + o : a.act + (size_t)g * a.A;
    const int m = every ? ng : *(volatile int32_t *)&a.act_n[g];
    int dec;
    if (!grid_lazy_step(list, m, a.ub, a.stamp, nullptr, nullptr, lc, a.gg, fold, lc->sel, lc->selpos,
                        lc->gsel, kLanes, a.gsel, &a.ctl->bar, &a.ctl->err, a.tns, &dec))
      return false;
    if (!bsync(a)) return false;
    lap(0);
    if (dec == 2) {
      if (every) {  // cannot happen with every candidate listed
        if (b == 0 && tid == 0) check_fail(a.ctl, 6, g, 1, 2);
        return false;
      }
      if (rebuilt == r) {
        every = true;
        if (b == 0 && tid == 0) lc->theta = LLONG_MIN;
      } else {
        rebuilt = r;
        if (!grid_refresh_graph(a, g)) return false;
        if (b == 0) cta_build_list(a, g);
      }
      if (!bsync(a)) return false;
      lap(0);
      fold = false;
      continue;
    }
    if (dec == 0) {
      if (!grid_gain_batch<kModeGain>(a.rpf, a.cif, a.N, a.dS, lc->sel, 0, &lc->n_sel, lc->gsel, a.ws, a.gx,
                                      a.goff, a.gg, a.gctl, &a.ctl->bar, &a.ctl->err, a.tns, a.mx, a.c3, o,
                                      a.max_n))
        return false;
      if (b == 0 && tid == 0 && *(volatile int32_t *)&a.gg->err)
        atomicExch(&a.ctl->err, *(volatile int32_t *)&a.gg->err);
      if (!bsync(a)) return false;  // workspace clean, gains visible
      lap(1);
      fold = true;
      continue;
    }
    // accept the round's best and update d_S from it
    fold = false;
    if (b == 0 && tid == 0) {
      a.ctl->pk[0] = a.ctl->pk[1] = a.ctl->pk[2] = 0;
      a.ctl->decrease = 0;
    }
    if (!bsync(a)) return false;
    if (!grid_relabel_bfs(a.rpf, a.cif, a.N, a.dS, &lc->best_id, 1, a.q0, a.q1, a.ctl->pk, nullptr,
                          &a.ctl->decrease, nullptr, a.goff, a.st1, &a.ctl->bar, &a.ctl->err, a.tns, nullptr,
                          a.c3))
      return false;
    if (!bsync(a)) return false;
    if (b == 0 && tid == 0) {
      const int pick = lc->best_id;
      const long long gain = lc->best_gain;
      a.ctl->pk[0] = a.ctl->pk[1] = a.ctl->pk[2] = 0;
      if ((long long)a.ctl->decrease != gain) check_fail(a.ctl, 6, g, gain, (long long)a.ctl->decrease);
      a.picks[(size_t)g * a.kmax + r] = pick;
      a.pgain[(size_t)g * a.kmax + r] = gain;
      a.ub[pick] = -1;
      lc->last_gain = gain;
      lc->best_id = -1;
      lc->best_gain = -1;
      lc->round = r + 1;
    }
    if (!bsync(a)) return false;
    lap(2);
  }
  if (b == 0 && tid == 0) {
    atomicAdd((unsigned long long *)&a.ctl->iterations, (unsigned long long)lc->steps);
    for (int q = 0; q < 3; ++q) atomicAdd(&a.ctl->ns_lazy[q], t_ph[q]);
  }
  return true;
}

// per-graph sum of d over all vertices (warp-aggregated when a warp's vertices
// share a graph); unreached vertices raise GC_EDISCONNECTED
static __device__ void seg_sum_dist(const BatchArgs &a, long long *out) {
  const int lane = threadIdx.x & 31;
  for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < a.N; base += gridDim.x * blockDim.x) {
    const int v = base + lane;
    long long d = 0;
    int g = -1;
    if (v < a.N) {
      const int x = a.dS[v];
      if (x >= kInf) atomicExch(&a.ctl->err, GC_EDISCONNECTED);
      else d = x;
      g = a.gid[v];
    }
    const int g0 = __shfl_sync(0xffffffffu, g, 0);
    const bool uniform = __all_sync(0xffffffffu, g == g0 || g < 0);
    if (uniform) {
      const long long s = warp_sum(d);
      if (lane == 0 && g0 >= 0 && s) atomicAdd((unsigned long long *)&out[g0], (unsigned long long)s);
    } else if (g >= 0 && d) {
      atomicAdd((unsigned long long *)&out[g], (unsigned long long)d);
    }
  }
}

// one CTA: argmin (f0, local id) over graph g's vertices with f0 >= 0
static __device__ int cta_argmin_f0(const BatchArgs &a, int g) {
  __shared__ long long s_v[32];
  __shared__ int s_id[32];
  const int o = a.off[g], n = a.ng[g];
  long long bv = LLONG_MAX;
  int bid = -1;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const long long f = a.f0[o + i];
    if (f >= 0 && better_min(f, i, bv, bid)) {
      bv = f;
      bid = i;
    }
  }
  // block arg-min through the arg-max helper on negated values
  long long nv = bv == LLONG_MAX ? LLONG_MIN : -bv;
  block_argmax_all(nv, bid, s_v, s_id);
  return bid;
}

// One CTA: the want-th largest of graph g's bounds ub >= 0, by a radix select
// over their bytes (256-bin shared histograms, most significant byte first).
// *c gets how many bounds are >= 0; when *c <= want the result is -1.  *need
// gets how many of the bounds equal to the result belong to the top `want`
// (the others above it: want - *need of them).
static __device__ long long cta_kth_bound(const long long *ub, int o, int n, int want, long long *c,
                                          int *need) {
  __shared__ int s_hist[256];
  __shared__ int s_pick[2];
  __shared__ long long s_ll[32];
  const int tid = threadIdx.x, T = blockDim.x;
  long long umax = -1, cnt = 0;
  for (int i = tid; i < n; i += T) {
    const long long u = ub[o + i];
    if (u >= 0) {
      umax = max(umax, u);
      ++cnt;
    }
  }
  umax = block_max_ll(umax, s_ll);
  cnt = block_sum(cnt, s_ll);
  *c = cnt;
  *need = 0;
  if (cnt <= want) return -1;
  unsigned long long prefix = 0, mask = 0;
  int nd = want;
  const int top = umax > 0 ? 63 - __clzll((unsigned long long)umax) : 0;
  for (int shift = (top / 8) * 8; shift >= 0; shift -= 8) {
    for (int j = tid; j < 256; j += T) s_hist[j] = 0;
    cta_sync();
    for (int i = tid; i < n; i += T) {
      const long long u = ub[o + i];
      if (u >= 0 && ((unsigned long long)u & mask) == prefix)
        atomicAdd(&s_hist[((unsigned long long)u >> shift) & 255], 1);
    }
    cta_sync();
    if (tid == 0) {  // the bin holding the nd-th largest of the matching values
      int acc = 0, bin = 255;
      for (; bin > 0; --bin) {
        if (acc + s_hist[bin] >= nd) break;
        acc += s_hist[bin];
      }
      s_pick[0] = bin;
      s_pick[1] = acc;
    }
    cta_sync();
    prefix |= (unsigned long long)s_pick[0] << shift;
    mask |= 255ull << shift;
    nd -= s_pick[1];
    cta_sync();
  }
  *need = nd;
  return (long long)prefix;
}

// One CTA: the `want` candidates of graph g with the largest bounds, ordered by
// (ub desc, id asc) with ub >= 0, written to out[] in id order; returns their
// count.  Every candidate above the want-th largest bound T is taken, then the
// smallest ids of those equal to T.
static __device__ int cta_top_bounds(const long long *ub, int o, int n, int want, int32_t *out) {
  __shared__ int s_scan[33];
  const int tid = threadIdx.x, T = blockDim.x;
  long long c;
  int need;
  const long long thr = cta_kth_bound(ub, o, n, want, &c, &need);  // -1: take every ub >= 0
  int carry = 0, eq_seen = 0;
  for (int base = 0; base < n; base += T) {
    const int i = base + tid;
    const long long u = i < n ? ub[o + i] : -1;
    const int eq = u >= 0 && u == thr;
    int eq_total;
    const int eq_pos = block_excl_scan(eq, s_scan, &eq_total);
    const int take = (u >= 0 && u > thr) || (eq && eq_seen + eq_pos < need);
    int total;
    const int pos = block_excl_scan(take, s_scan, &total);
    if (take) out[carry + pos] = o + i;
    carry += total;
    eq_seen += eq_total;
  }
  return carry;
}

// One CTA: graph g's active list = {ub >= L} (ids in increasing order, at most
// A of them) with L the smallest value whose list fits, and theta = the
// largest bound left out, plus one (LLONG_MIN when nothing is left out): every
// candidate outside the list has ub < theta.
static __device__ void cta_build_list(const BatchArgs &a, int g) {
  __shared__ long long s_ll[32];
  __shared__ int s_scan[33];
  const int tid = threadIdx.x, T = blockDim.x;
  const int o = a.off[g], n = a.ng[g];
  long long c;
  int need;
  const long long kth = cta_kth_bound(a.ub, o, n, a.A, &c, &need);
  long long L = 0, theta = LLONG_MIN;
  if (c > a.A) {
    // the bounds equal to kth that the top A leaves out decide whether kth fits
    long long eq = 0, below = -1;
    for (int i = tid; i < n; i += T) {
      const long long u = a.ub[o + i];
      eq += u == kth;
      if (u >= 0 && u < kth) below = max(below, u);
    }
    eq = block_sum(eq, s_ll);
    below = block_max_ll(below, s_ll);
    if (eq > need) {
      L = kth + 1;
      theta = kth + 1;
    } else {
      L = kth;
      theta = below + 1;  // c > A leaves some bound below kth
    }
  }
  int32_t *act = a.act + (size_t)g * a.A;
  int carry = 0;
  for (int base = 0; base < n; base += T) {
    const int i = base + tid;
    const int f = i < n && a.ub[o + i] >= 0 && a.ub[o + i] >= L;
    int total;
    const int pos = block_excl_scan(f, s_scan, &total);
    if (f && carry + pos < a.A) act[carry + pos] = o + i;
    carry += total;
  }
  if (carry > a.A) {  // cannot happen (count(ub >= L) <= A); never write past the list
    if (tid == 0) check_fail(a.ctl, 5, g, a.A, carry);
    carry = a.A;
  }
  if (tid == 0) {
    a.act_n[g] = carry;
    a.lc[g].theta = theta;
  }
  cta_sync();
}

// Two-hop upper bound of Delta(v|S) for the group whose distances are d (the
// inequality and its derivation are those of k_round1_bound in gc_bfs.cu):
// d[v] + sum over the pruned row of v of ((d[w] - 1)^+ + c3[w]), plus the
// graph's G3 = sum_u (d[u] - 3)^+ added by the caller.  One warp per v.
static __device__ __forceinline__ long long warp_two_hop(const BatchArgs &a, const int32_t *d, const int32_t *c3,
                                                         int v) {
  const int lane = threadIdx.x & 31;
  long long s = 0;
  for (int e = a.rpf[v] + lane; e < a.rpf[v + 1]; e += 32) {
    const int w = a.cif[e];
    s += (long long)max(d[w] - 1, 0) + (long long)c3[w];
  }
  return warp_sum(s) + (long long)d[v];
}

// per-graph sum of (d - 3)^+ into out[g] (warp-aggregated like seg_sum_dist)
static __device__ void seg_sum_excess3(const BatchArgs &a, const int32_t *d, long long *out) {
  const int lane = threadIdx.x & 31;
  for (int base = (blockIdx.x * blockDim.x + threadIdx.x) & ~31; base < a.N; base += gridDim.x * blockDim.x) {
    const int v = base + lane;
    long long x = 0;
    int g = -1;
    if (v < a.N) {
      x = max(d[v] - 3, 0);
      g = a.gid[v];
    }
    const int g0 = __shfl_sync(0xffffffffu, g, 0);
    if (__all_sync(0xffffffffu, g == g0 || g < 0)) {
      const long long s = warp_sum(x);
      if (lane == 0 && g0 >= 0 && s) atomicAdd((unsigned long long *)&out[g0], (unsigned long long)s);
    } else if (g >= 0 && x) {
      atomicAdd((unsigned long long *)&out[g], (unsigned long long)x);
    }
  }
}

// Round 1 with two-hop bounds (the single-graph path's round 1, per graph):
// every candidate gets the bound for S = {s0}; the 64 largest bounds of each
// graph are evaluated as one CTA batch, then every candidate whose bound
// reaches that batch's best exact gain.  After that no unevaluated candidate
// can beat the best exact gain (its bound is below it), so the lazy rule of
// Sec. 4.2 accepts the best one.  Evaluated candidates get stamp 1 and their
// exact gain in ub; the rest keep stamp 0 and their bound.
static __device__ bool batch_round1_bounded(const BatchArgs &a, const GainWs &myws, GainCounters &cnt,
                                            long long *s_out) {
  __shared__ int s_task;
  __shared__ long long s_ll[32];
  __shared__ int s_scan[33];
  const int tid = threadIdx.x, b = blockIdx.x, G = gridDim.x, T = blockDim.x;
  seg_sum_excess3(a, a.dS1, a.g3);
  if (!bsync(a)) return false;
  {
    const int lane = tid & 31, gw = (b * T + tid) >> 5, nw = (G * T) >> 5;
    for (int v = gw; v < a.N; v += nw) {
      const long long s = warp_two_hop(a, a.dS1, a.c3, v);
      if (lane == 0) {
        a.ub[v] = a.dS1[v] == 0 ? -1ll : s + a.g3[a.gid[v]];
        a.stamp[v] = 0;
      }
    }
  }
  if (!bsync(a)) return false;
  // the first batch of each graph: its 64 largest bounds
  for (int g = b; g < a.count; g += G) {
    const int m = a.kk[g] >= 2 ? cta_top_bounds(a.ub, a.off[g], a.ng[g], kLanes, a.slist + a.off[g]) : 0;
    if (tid == 0) a.scount[g] = m;
    cta_sync();
  }
  if (!bsync(a)) return false;
  for (;;) {
    if (tid == 0) s_task = atomicAdd(&a.ctl->task, 1);
    cta_sync();
    const int g = s_task;
    cta_sync();
    if (g >= a.count) break;
    const int m = a.scount[g], o = a.off[g];
    if (m == 0) continue;
    cta_gain_batch<kModeGain, true, true>(a.rpf, a.cif, a.N, a.dS1, a.slist + o, m, s_out, myws, a.gctl, a.mx,
                                          LaneGraphs(), cnt, o, a.c3);
    if (tid < m) {
      const int v = a.slist[o + tid];
      a.ub[v] = s_out[tid];
      a.stamp[v] = 1;
    }
    const long long best = block_max_ll(tid < m ? s_out[tid] : -1ll, s_ll);
    if (tid == 0) a.bestf[g] = best;
    cta_sync();
  }
  if (!bsync(a)) return false;
  // every other candidate whose bound reaches the first batch's best
  for (int g = b; g < a.count; g += G) {
    const int o = a.off[g], n = a.ng[g];
    const long long b1 = a.bestf[g];
    int carry = 0;
    if (a.kk[g] >= 2) {
      for (int base = 0; base < n; base += T) {
        const int i = base + tid;
        int flag = 0;
        if (i < n) {
          const long long u = a.ub[o + i];
          flag = u >= 0 && u >= b1 && a.stamp[o + i] == 0;
        }
        int total;
        const int pos = block_excl_scan(flag, s_scan, &total);
        if (flag) a.slist[o + carry + pos] = o + i;
        carry += total;
      }
    }
    if (tid == 0) a.scount[g] = carry;
    cta_sync();
  }
  if (!bsync(a)) return false;
  if (b == 0 && tid == 0) {
    int acc = 0;
    for (int g = 0; g < a.count; ++g) {
      a.tstart[g] = acc;
      acc += (a.scount[g] + kLanes - 1) / kLanes;
    }
    a.tstart[a.count] = acc;
    a.ctl->task = 0;
  }
  if (!bsync(a)) return false;
  const int n_tasks = a.tstart[a.count];
  for (;;) {
    if (tid == 0) s_task = atomicAdd(&a.ctl->task, 1);
    cta_sync();
    const int t = s_task;
    cta_sync();
    if (t >= n_tasks) break;
    int lo = 0, hi = a.count - 1;  // graph with tstart[g] <= t < tstart[g+1] (non-empty)
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.tstart[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const int g = lo, o = a.off[g], first = (t - a.tstart[g]) * kLanes;
    const int nl = min(kLanes, a.scount[g] - first);
    cta_gain_batch<kModeGain, true, true>(a.rpf, a.cif, a.N, a.dS1, a.slist + o + first, nl, s_out, myws, a.gctl,
                                          a.mx, LaneGraphs(), cnt, o, a.c3);
    if (tid < nl) {
      const int v = a.slist[o + first + tid];
      a.ub[v] = s_out[tid];
      a.stamp[v] = 1;
    }
    cta_sync();
  }
  return bsync(a);
}

// Bound refresh before the lazy rounds: the two-hop bound for the group after
// round 1 (d = the current d_S, c3 recounted into q0, G3 into g3[count + g])
// lowers every candidate's bound, as before each persistent launch of the
// single-graph path.
static __device__ bool batch_bound_refresh(const BatchArgs &a) {
  const int tid = threadIdx.x, lane = tid & 31, b = blockIdx.x, G = gridDim.x, T = blockDim.x;
  const int gw = (b * T + tid) >> 5, nw = (G * T) >> 5;
  for (int u = gw; u < a.N; u += nw) {
    int c = 0;
    for (int e = a.rpf[u] + lane; e < a.rpf[u + 1]; e += 32) c += a.dS[a.cif[e]] >= 3;
    c = warp_sum(c);
    if (lane == 0) a.q0[u] = c;
  }
  seg_sum_excess3(a, a.dS, a.g3 + a.count);
  if (!bsync(a)) return false;
  for (int v = gw; v < a.N; v += nw) {
    const int g = a.gid[v];
    if (a.kk[g] <= 2 || a.ub[v] < 0) continue;  // warp-uniform: one v per warp
    const long long s = warp_two_hop(a, a.dS, a.q0, v) + a.g3[a.count + g];
    if (lane == 0 && s < a.ub[v]) a.ub[v] = s;
  }
  return bsync(a);
}

// Refresh of one graph's bounds in the lazy rounds, when its active list can no
// longer certify a pick (the single-graph path refreshes before each rebuild
// of its list the same way): c3 for the current d_S into q0, G3 of the graph,
// then every candidate's bound lowered to the two-hop bound for the current
// group.  The CTA form runs inside one CTA (P6b); the grid form is spread over
// every CTA, with three grid barriers (P6a).
static __device__ void cta_refresh_graph(const BatchArgs &a, int g) {
  __shared__ long long s_ll[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  const int o = a.off[g], n = a.ng[g];
  long long x3 = 0;
  for (int i = tid; i < n; i += blockDim.x) x3 += max(a.dS[o + i] - 3, 0);
  for (int u = o + wid; u < o + n; u += nw) {
    int c = 0;
    for (int e = a.rpf[u] + lane; e < a.rpf[u + 1]; e += 32) c += a.dS[a.cif[e]] >= 3;
    c = warp_sum(c);
    if (lane == 0) a.q0[u] = c;
  }
  const long long G3 = block_sum(x3, s_ll);  // its barriers also publish q0
  for (int v = o + wid; v < o + n; v += nw) {
    if (a.ub[v] < 0) continue;  // a member (warp-uniform)
    const long long s = warp_two_hop(a, a.dS, a.q0, v) + G3;
    if (lane == 0 && s < a.ub[v]) a.ub[v] = s;
  }
  cta_sync();
}

static __device__ bool grid_refresh_graph(const BatchArgs &a, int g) {
  __shared__ long long s_ll[32];
  const int tid = threadIdx.x, lane = tid & 31, b = blockIdx.x, G = gridDim.x, T = blockDim.x;
  const int gw = (b * T + tid) >> 5, nw = (G * T) >> 5;
  const int o = a.off[g], n = a.ng[g];
  long long *g3 = a.g3 + a.count + g;
  if (b == 0 && tid == 0) *g3 = 0;
  if (!bsync(a)) return false;
  long long x3 = 0;
  for (int i = b * T + tid; i < n; i += G * T) x3 += max(a.dS[o + i] - 3, 0);
  x3 = block_sum(x3, s_ll);
  if (tid == 0 && x3) atomicAdd((unsigned long long *)g3, (unsigned long long)x3);
  for (int u = o + gw; u < o + n; u += nw) {
    int c = 0;
    for (int e = a.rpf[u] + lane; e < a.rpf[u + 1]; e += 32) c += a.dS[a.cif[e]] >= 3;
    c = warp_sum(c);
    if (lane == 0) a.q0[u] = c;
  }
  if (!bsync(a)) return false;
  const long long G3 = *(volatile long long *)g3;
  for (int v = o + gw; v < o + n; v += nw) {
    if (a.ub[v] < 0) continue;  // a member (warp-uniform)
    const long long s = warp_two_hop(a, a.dS, a.q0, v) + G3;
    if (lane == 0 && s < a.ub[v]) a.ub[v] = s;
  }
  return bsync(a);
}

// Two CTAs per SM (64 registers, no spills): the CTA-local phases are latency
// bound and gain from the second resident CTA.
__global__ void __launch_bounds__(kBatchThreads, 2) k_batch_solve(const BatchArgs a) {
  __shared__ long long s_out[kLanes];
  __shared__ int s_task;
  __shared__ int s_scan[33];
  __shared__ unsigned long long s_red[32];
  const int tid = threadIdx.x, lane = tid & 31, b = blockIdx.x, G = gridDim.x, T = blockDim.x;
  GainCounters cnt;
  const unsigned long long t_start = global_ns();
  const GainWs myws = gain_ws(a.ws, a.ws_stride, a.max_n, b);  // this CTA's workspace, sized for the largest graph
  // ---- P0: lower bounds, per-graph argmin ----
  {
    const int gw = (b * T + tid) >> 5, nw = (G * T) >> 5;
    for (int v = gw; v < a.N; v += nw) {
      const int beg = a.rp[v], end = a.rp[v + 1];
      long long x = 0;
      for (int e = beg + lane; e < end; e += 32) {
        const int w = a.ci[e];
        x += (long long)(a.rp[w + 1] - a.rp[w] - 1);
      }
      x = warp_sum(x);
      if (lane == 0) {
        const int g = a.gid[v];
        const long long deg = end - beg;
        long long rest = (long long)a.ng[g] - 1 - deg;
        if (rest < 0) rest = 0;
        const long long c2 = x < rest ? x : rest;
        const long long lb = deg + 2 * c2 + 3 * (rest - c2);
        a.key[v] = -lb;
        a.f0[v] = -1;
        a.dS[v] = kInf;
        a.stamp[v] = 0;
        a.ub[v] = LLONG_MAX;
        atomicMin(&a.packed[g], ((unsigned long long)lb << 32) | (unsigned long long)(v - a.off[g]));
      }
    }
  }
  for (int g = b * T + tid; g < 2 * a.count; g += G * T) a.g3[g] = 0;
  if (!bsync(a)) return;
  // ---- P1: BFS from all v_a ----
  for (int g = b * T + tid; g < a.count; g += G * T) a.seeds[g] = a.off[g] + (int)(a.packed[g] & 0xffffffffull);
  if (!bsync(a)) return;
  if (!grid_relabel_bfs(a.rp, a.ci, a.N, a.dS, a.seeds, a.count, a.q0, a.q1, a.ctl->pk, nullptr,
                        &a.ctl->decrease, nullptr, a.goff, a.st1, &a.ctl->bar, &a.ctl->err, a.tns))
    return;
  if (!bsync(a)) return;
  seg_sum_dist(a, a.fa);
  if (b == 0 && tid == 0) a.ctl->pk[0] = a.ctl->pk[1] = a.ctl->pk[2] = 0;
  if (!bsync(a)) return;
  // ---- P2: round-0 survivors (every v with LB(v) <= f_a) ----
  // P2a, one CTA per graph: compact the graph's survivors into its own region
  // of slist (graph-aligned, so batches never mix graphs)
  for (int g = b; g < a.count; g += G) {
    const int o = a.off[g], n = a.ng[g];
    const long long fa = a.fa[g];
    const int va = a.seeds[g];
    if (tid == 0) {
      a.bestf[g] = fa;
      a.f0[va] = fa;
      a.key[va] = LLONG_MIN;
    }
    cta_sync();
    int carry = 0;
    for (int base = 0; base < n; base += T) {
      const int i = base + tid;
      int flag = 0;
      if (i < n) {
        const long long k = a.key[o + i];
        flag = k != LLONG_MIN && -k <= fa;
      }
      int total;
      const int pos = block_excl_scan(flag, s_scan, &total);
      if (flag) a.slist[o + carry + pos] = o + i;
      carry += total;
    }
    if (tid == 0) a.scount[g] = carry;
    cta_sync();
  }
  if (!bsync(a)) return;
  // P2b: task prefix over graphs (64 survivors per task)
  if (b == 0 && tid == 0) {
    int acc = 0;
    for (int g = 0; g < a.count; ++g) {
      a.tstart[g] = acc;
      acc += (a.scount[g] + kLanes - 1) / kLanes;
    }
    a.tstart[a.count] = acc;
    a.ctl->task = 0;
  }
  if (!bsync(a)) return;
  // P2c: every CTA takes survivor batches from a dynamic counter
  {
    const int n_tasks = a.tstart[a.count];
    const LaneGraphs lg{a.gid, a.ng, a.bestf};
    for (;;) {
      if (tid == 0) s_task = atomicAdd(&a.ctl->task, 1);
      cta_sync();
      const int t = s_task;
      cta_sync();
      if (t >= n_tasks) break;
      int lo = 0, hi = a.count - 1;  // graph with tstart[g] <= t < tstart[g+1] (non-empty)
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (a.tstart[mid] <= t) lo = mid;
        else hi = mid - 1;
      }
      const int g = lo, o = a.off[g], first = (t - a.tstart[g]) * kLanes;
      const int nl = min(kLanes, a.scount[g] - first);
      cta_gain_batch<kModeFarness, true, false>(a.rp, a.ci, a.N, a.dS, a.slist + o + first, nl, s_out, myws, a.gctl, nullptr,
                                   lg, cnt, o);
      if (tid < nl) a.f0[a.slist[o + first + tid]] = s_out[tid];
      cta_sync();
    }
  }
  if (!bsync(a)) return;
  // P2d, one CTA per graph: s0 = argmin (f, id) over the exact farness values
  for (int g = b; g < a.count; g += G) {
    const int s0 = cta_argmin_f0(a, g);
    if (tid == 0) a.seeds[g] = a.off[g] + (s0 >= 0 ? s0 : 0);
    cta_sync();
  }
  if (!bsync(a)) return;
  if (b == 0 && tid == 0) a.ctl->ns_ph[0] = global_ns() - t_start;
  // ---- P3: d_S = BFS from all s0; farness; neighbour bound ----
  for (int v = b * T + tid; v < a.N; v += G * T) a.dS[v] = kInf;
  if (!bsync(a)) return;
  if (!grid_relabel_bfs(a.rp, a.ci, a.N, a.dS, a.seeds, a.count, a.q0, a.q1, a.ctl->pk, nullptr,
                        &a.ctl->decrease, nullptr, a.goff, a.st1, &a.ctl->bar, &a.ctl->err, a.tns))
    return;
  if (!bsync(a)) return;
  seg_sum_dist(a, a.farness);
  for (int v = b * T + tid; v < a.N; v += G * T) a.dS1[v] = a.dS[v];  // round 1's read-only d_S
  {
    const int gw = (b * T + tid) >> 5, nw = (G * T) >> 5;
    for (int v = gw; v < a.N; v += nw) {
      int m = 0;
      for (int e = a.rp[v] + lane; e < a.rp[v + 1]; e += 32) m = max(m, a.dS[a.ci[e]]);
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 16));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 8));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 4));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 2));
      m = max(m, __shfl_xor_sync(0xffffffffu, m, 1));
      if (lane == 0) a.mx[v] = m;
    }
  }
  if (b == 0 && tid == 0) {
    a.ctl->pk[0] = a.ctl->pk[1] = a.ctl->pk[2] = 0;
    a.ctl->task = 0;
  }
  if (!bsync(a)) return;
  if (!batch_prune(a)) return;
  for (int g = b * T + tid; g < a.count; g += G * T) {
    const int s0 = a.seeds[g];
    if (a.f0[s0] != a.farness[g]) check_fail(a.ctl, 3, g, a.f0[s0], a.farness[g]);
    a.picks[(size_t)g * a.kmax] = s0;
    a.pgain[(size_t)g * a.kmax] = a.farness[g];
    a.packed[g] = 0;  // reused as the round-1 arg-max key
  }
  // ---- P4: round 1 (graph-aligned batches from a dynamic counter) ----
  if (b == 0 && tid == 0) a.ctl->ns_ph[4] = global_ns() - t_start;
  if (a.bounded) {
    if (!bsync(a)) return;  // the pruned adjacency's c3 and the picks above are in place
    if (!batch_round1_bounded(a, myws, cnt, s_out)) return;
  }
  const int n_tasks = a.bounded ? 0 : a.bstart[a.count];
  for (;;) {
    if (tid == 0) s_task = atomicAdd(&a.ctl->task, 1);
    cta_sync();
    const int t = s_task;
    cta_sync();
    if (t >= n_tasks) break;
    int lo = 0, hi = a.count - 1;  // graph with bstart[g] <= t < bstart[g+1]
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (a.bstart[mid] <= t) lo = mid;
      else hi = mid - 1;
    }
    const int g = lo;
    if (a.kk[g] < 2) continue;
    const int o = a.off[g], first = (t - a.bstart[g]) * a.lanes1;
    const int nl = min(a.lanes1, a.ng[g] - first);
    cta_gain_batch<kModeGain, true, true>(a.rpf, a.cif, a.N, a.dS1, a.iota + o + first, nl, a.ub + o + first, myws,
                                          a.gctl, a.mx, LaneGraphs(), cnt, o, a.c3);
  }
  if (!bsync(a)) return;
  if (b == 0 && tid == 0) a.ctl->ns_ph[5] = global_ns() - t_start;
  if (!a.bounded)  // every candidate was evaluated in round 1
    for (int v = b * T + tid; v < a.N; v += G * T) a.stamp[v] = 1;
  for (int g = b * T + tid; g < a.count; g += G * T) a.ub[a.seeds[g]] = -1;  // s0 is a member
  if (!bsync(a)) return;
  // per-graph argmax (gain desc, id asc) of round 1
  for (int base = (b * T + tid) & ~31; base < a.N; base += G * T) {
    const int v = base + lane;
    unsigned long long key = 0;
    int g = -1;
    if (v < a.N) {
      g = a.gid[v];
      const long long u = a.ub[v];
      if (u >= 0 && a.kk[g] >= 2 && a.stamp[v] == 1) {  // exact round-1 gains only
        if (u >= (1ll << 31)) atomicExch(&a.ctl->err, GC_ERANGE);
        key = ((unsigned long long)u << 32) | (0xffffffffull - (unsigned long long)(v - a.off[g]));
      }
    }
    const int g0 = __shfl_sync(0xffffffffu, g, 0);
    if (__all_sync(0xffffffffu, g == g0 || g < 0)) {
      unsigned long long m = key;
#pragma unroll
      for (int s = 16; s > 0; s >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, s));
      if (lane == 0 && g0 >= 0 && m) atomicMax(&a.packed[g0], m);
    } else if (g >= 0 && key) {
      atomicMax(&a.packed[g], key);
    }
  }
  if (!bsync(a)) return;
  if (b == 0) {
    if (tid == 0) {
      a.ctl->nseeds = 0;
      a.ctl->remaining = 0;
    }
    cta_sync();
    for (int g = tid; g < a.count; g += T) {
      if (a.kk[g] < 2) {
        a.lc[g].round = a.kk[g];  // nothing after round 0
        continue;
      }
      const unsigned long long key = a.packed[g];
      const int v = a.off[g] + (int)(0xffffffffull - (key & 0xffffffffull));
      const long long gain = (long long)(key >> 32);
      a.picks[(size_t)g * a.kmax + 1] = v;
      a.pgain[(size_t)g * a.kmax + 1] = gain;
      a.ub[v] = -1;
      a.seeds[atomicAdd(&a.ctl->nseeds, 1)] = v;
      LazyCtl *lc = &a.lc[g];
      lc->round = 2;
      lc->best_id = -1;
      lc->best_gain = -1;
      lc->last_gain = gain;
      lc->pad = 0;  // fold flag
      if (a.kk[g] > 2) atomicAdd(&a.ctl->remaining, 1);
    }
  }
  if (!bsync(a)) return;
  if (!grid_relabel_bfs(a.rpf, a.cif, a.N, a.dS, a.seeds, *(volatile int32_t *)&a.ctl->nseeds, a.q0, a.q1,
                        a.ctl->pk, nullptr, &a.ctl->decrease, nullptr, a.goff, a.st1, &a.ctl->bar,
                        &a.ctl->err, a.tns, nullptr, a.c3))
    return;
  if (!bsync(a)) return;
  if (b == 0 && tid == 0) {
    a.ctl->pk[0] = a.ctl->pk[1] = a.ctl->pk[2] = 0;
    a.ctl->nseeds = 0;
  }
  if (a.bounded && !batch_bound_refresh(a)) return;
  // ---- P5: active lists (one CTA per graph) ----
  for (int g = b; g < a.count; g += G) {
    if (a.kk[g] <= 2) continue;
    cta_build_list(a, g);
    if (tid == 0) a.full[g] = 0;
  }
  if (!bsync(a)) return;
  if (b == 0 && tid == 0) a.ctl->ns_ph[1] = global_ns() - t_start;
  // ---- P6a: lazy rounds of the big graphs, one graph at a time by the grid ----
  for (int g = 0; g < a.count; ++g)
    if (a.ng[g] >= a.grid_min_n && a.kk[g] > 2 && !batch_grid_lazy(a, g)) return;
  // ---- P6b: the other graphs' lazy rounds; each CTA runs its graphs to
  // completion (no grid barrier: a graph never waits for another graph's step) ----
  {
    __shared__ int s_stop;
    for (int g = b; g < a.count; g += G) {
      if (a.ng[g] >= a.grid_min_n) continue;  // done in P6a
      LazyCtl *lc = &a.lc[g];
      const int o = a.off[g];
      unsigned long long t_ph[3] = {0, 0, 0}, t_mark = global_ns();  // thread 0's phase clocks
      for (;;) {
        if (tid == 0) s_stop = (lc->round >= a.kk[g]) || (*(volatile int32_t *)&a.ctl->err != 0);
        cta_sync();
        if (s_stop) break;
        const bool full = a.full[g] == 1;  // 0: list, 2 + r: list rebuilt in round r, 1: every candidate
        const int32_t *act = full ? a.iota + o : a.act + (size_t)g * a.A;
        const int m = full ? a.ng[g] : a.act_n[g];
        if (full && tid == 0) lc->theta = LLONG_MIN;
        cta_sync();
        lazy_cta0_step(act, m, a.ub, a.stamp, lc, nullptr, lc->pad != 0, nullptr, 0);
        cta_sync();
        const int dec = *(volatile int32_t *)&lc->dec;
        if (tid == 0) {
          const unsigned long long now = global_ns();
          t_ph[0] += now - t_mark;
          t_mark = now;
        }
        int ph = 0;  // the rest of the step: 0 list rebuild, 1 gain batch, 2 d_S update
        if (dec == 0) {  // evaluate the selected batch
          cta_gain_batch<kModeGain, true, false>(a.rpf, a.cif, a.N, a.dS, lc->sel, lc->n_sel, lc->gsel, myws,
                                                 a.gctl, a.mx, LaneGraphs(), cnt, o, a.c3);
          if (tid == 0) lc->pad = 1;  // fold it next step
          ph = 1;
        } else if (dec == 1) {  // accept: record, then update d_S from the pick
          ph = 2;
          const int pick = lc->best_id;
          const long long gain = lc->best_gain;
          const int r = lc->round;
          cta_sync();
          const long long decr = cta_relabel_bfs(a.rpf, a.cif, a.dS, pick, myws.qv0, myws.qv1);
          if (tid == 0) {
            if (decr != gain) check_fail(a.ctl, 6, g, gain, decr);
            a.picks[(size_t)g * a.kmax + r] = pick;
            a.pgain[(size_t)g * a.kmax + r] = gain;
            a.ub[pick] = -1;
            lc->last_gain = gain;
            lc->best_id = -1;
            lc->best_gain = -1;
            lc->pad = 0;
            lc->round = r + 1;
            lc->steps += 0;
          }
        } else {  // the list cannot certify: refresh the bounds and rebuild it
          const int r = lc->round;
          const bool again = a.full[g] == 2 + r;
          cta_sync();
          if (!again) {
            cta_refresh_graph(a, g);
            cta_build_list(a, g);
          }
          if (tid == 0) {
            a.full[g] = again ? 1 : 2 + r;  // a second failure in one round: every candidate
            lc->pad = 0;
          }
        }
        if (tid == 0) {
          const unsigned long long now = global_ns();
          t_ph[ph] += now - t_mark;
          t_mark = now;
          if (now - t_start > 6ull * a.tns) atomicExch(&a.ctl->err, GC_ETIMEOUT);
        }
        cta_sync();
      }
      if (tid == 0) {
        atomicAdd((unsigned long long *)&a.ctl->iterations, (unsigned long long)lc->steps);
        for (int q = 0; q < 3; ++q) atomicAdd(&a.ctl->ns_lazy[q], t_ph[q]);
      }
    }
  }
  if (!bsync(a)) return;
  if (b == 0 && tid == 0) a.ctl->ns_ph[2] = global_ns() - t_start;
  // ---- P7: check every group's farness with one BFS ----
  for (int v = b * T + tid; v < a.N; v += G * T) a.dS[v] = kInf;
  if (b == 0) {
    if (tid == 0) {
      a.ctl->nseeds = 0;
      a.ctl->pk[0] = a.ctl->pk[1] = a.ctl->pk[2] = 0;  // the grid lazy rounds leave them set
    }
    cta_sync();
    for (int g = tid; g < a.count; g += T) {
      long long f = a.pgain[(size_t)g * a.kmax];
      for (int r = 1; r < a.kk[g]; ++r) f -= a.pgain[(size_t)g * a.kmax + r];
      a.fa[g] = f;  // farness implied by the accepted gains
      a.farness[g] = 0;
    }
  }
  if (!bsync(a)) return;
  if (b == 0) {
    for (int g = 0; g < a.count; ++g) {
      for (int r = tid; r < a.kk[g]; r += T) a.seeds[atomicAdd(&a.ctl->nseeds, 1)] = a.picks[(size_t)g * a.kmax + r];
    }
  }
  if (!bsync(a)) return;
  if (!grid_relabel_bfs(a.rp, a.ci, a.N, a.dS, a.seeds, *(volatile int32_t *)&a.ctl->nseeds, a.q0, a.q1,
                        a.ctl->pk, nullptr, &a.ctl->decrease, nullptr, a.goff, a.st1, &a.ctl->bar,
                        &a.ctl->err, a.tns))
    return;
  if (!bsync(a)) return;
  seg_sum_dist(a, a.farness);
  if (!bsync(a)) return;
  for (int g = b * T + tid; g < a.count; g += G * T)
    if (a.farness[g] != a.fa[g]) check_fail(a.ctl, 7, g, a.fa[g], a.farness[g]);
  if (b == 0 && tid == 0) a.ctl->ns_ph[3] = global_ns() - t_start;
  // work counters
  u64 c_scalar = block_sum(cnt.scalar, s_red);
  u64 c_union = block_sum(cnt.uni, s_red);
  u64 c_front = block_sum(cnt.front, s_red);
  u64 c_push = block_sum(cnt.push, s_red);
  if (tid == 0) {
    atomicAdd(&a.gctl->edges_scalar, c_scalar);
    atomicAdd(&a.gctl->edges_union, c_union);
    atomicAdd(&a.gctl->frontier, c_front);
    atomicAdd(&a.gctl->pushes, c_push);
    atomicAdd(&a.gctl->levels, cnt.levels);
    atomicAdd(&a.gctl->batches, cnt.batches);
    atomicAdd(&a.gctl->lanes, cnt.lanes);
  }
}

__global__ void k_iota(int32_t *p, int32_t n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

// union CSR: shift graph g's row pointers by its first edge and its neighbour
// ids by its first vertex; gid[v] = graph of v
__global__ void k_union_fix(int32_t *rp, int32_t *ci, int32_t *gid, const int32_t *off, const int64_t *eoff,
                            int32_t count, int32_t N, int64_t nnz) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t v = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; v < N; v += stride) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (off[mid] <= v) lo = mid;
      else hi = mid - 1;
    }
    gid[v] = lo;
    rp[v] += (int32_t)eoff[lo];
  }
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nnz; e += stride) {
    int lo = 0, hi = count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (eoff[mid] <= e) lo = mid;
      else hi = mid - 1;
    }
    ci[e] += off[lo];
  }
}

}  // namespace gc

using namespace gc;

struct gc_batch {
  int32_t count = 0;
  int32_t N = 0;
  int64_t nnz = 0;
  int32_t max_n = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0, ctas = 0;
  std::vector<int32_t> h_off, h_n;
  int32_t *rp = nullptr, *ci = nullptr, *gid = nullptr, *off = nullptr, *ng = nullptr, *iota = nullptr;
  int32_t *dS = nullptr, *mx = nullptr, *stamp = nullptr, *q0 = nullptr, *q1 = nullptr, *goff = nullptr,
          *st1 = nullptr;
  int32_t *rpf = nullptr, *cif = nullptr, *c3 = nullptr, *gx = nullptr, *dS1 = nullptr;
  GridGainCtl *gg = nullptr;
  GridSelScratch *gsel = nullptr;
  long long *ub = nullptr, *key = nullptr, *f0 = nullptr;
  unsigned char *ws = nullptr;
  size_t ws_stride = 0;
  unsigned long long *packed = nullptr;
  long long *fa = nullptr, *farness = nullptr, *bestf = nullptr, *g3 = nullptr;
  LazyCtl *lc = nullptr;
  int32_t *act = nullptr, *act_n = nullptr, *full = nullptr, *kk = nullptr, *bstart = nullptr;
  int32_t A = 0, act_cap = 0;
  int32_t kcap = 0;
  int32_t *picks = nullptr;
  long long *pgain = nullptr;
  int32_t *seeds = nullptr;
  int32_t seeds_cap = 0;
  int32_t *slist = nullptr, *scount = nullptr, *tstart = nullptr;
  BatchCtl *ctl = nullptr, *h_ctl = nullptr;
  GainCtl *gctl = nullptr, *h_gctl = nullptr;
  // captured launch sequence
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  cudaStream_t cap_stream = nullptr;  // private stream the sequence is captured on
  std::vector<int32_t> cap_k;
  int32_t cap_A = 0, cap_lanes = 0, cap_grid_min_n = 0;
  uint32_t cap_flags = 0;
  std::vector<int32_t> h_picks;
  std::vector<long long> h_pgain, h_far;
  int32_t *h_picks_pinned = nullptr;
  long long *h_far_pinned = nullptr;
  int32_t *h_k_pinned = nullptr, *h_bstart_pinned = nullptr;  // sources of the captured copies
};

static void batch_release(gc_batch *b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  void *dev[] = {b->rp, b->ci, b->gid, b->off, b->ng, b->iota, b->dS, b->mx, b->stamp, b->q0, b->q1, b->goff, b->st1,
                 b->ub, b->key, b->f0, b->ws, b->packed, b->fa, b->farness, b->bestf, b->lc, b->act, b->act_n,
                 b->full, b->kk, b->bstart, b->picks, b->pgain, b->seeds, b->ctl, b->gctl, b->slist,
                 b->scount, b->tstart, b->rpf, b->cif, b->c3, b->gx, b->gg, b->gsel, b->dS1, b->g3};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (b->h_ctl) cudaFreeHost(b->h_ctl);
  if (b->h_gctl) cudaFreeHost(b->h_gctl);
  if (b->h_picks_pinned) cudaFreeHost(b->h_picks_pinned);
  if (b->h_far_pinned) cudaFreeHost(b->h_far_pinned);
  if (b->h_k_pinned) cudaFreeHost(b->h_k_pinned);
  if (b->h_bstart_pinned) cudaFreeHost(b->h_bstart_pinned);
  delete b;
}

template <typename T>
static bool balloc(T **p, size_t count) {
  if (count == 0) count = 1;
  if (cudaMalloc((void **)p, count * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  return true;
}

// The union CSR of `count` graphs.  Host arrays (nnzs == nullptr: the entry
// counts are read from row_ptrs[g][ns[g]]), or device arrays of existing
// handles (nnzs given; the handles were checked when they were loaded).  The
// copies use cudaMemcpyDefault, which takes either kind of pointer.
static int batch_load_impl(int32_t count, const int32_t *const *row_ptrs, const int32_t *const *col_idxs,
                           const int32_t *ns, const int64_t *nnzs, void *stream, gc_batch **out) {
  if (!out || count < 1 || !row_ptrs || !col_idxs || !ns) {
    set_error("bad argument to gc_batch_load");
    return GC_EINVAL;
  }
  *out = nullptr;
  gc_batch *b = new gc_batch();
  b->count = count;
  b->stream = (cudaStream_t)stream;
  b->h_off.resize(count + 1);
  b->h_n.assign(ns, ns + count);
  std::vector<int64_t> eoff(count + 1);
  int64_t N = 0, E = 0;
  for (int32_t g = 0; g < count; ++g) {
    const int64_t e = nnzs ? nnzs[g] : (ns[g] >= 1 && row_ptrs[g] ? row_ptrs[g][ns[g]] : -1);
    if (ns[g] < 1 || !row_ptrs[g] || e < 0 || (!nnzs && row_ptrs[g][0] != 0) || (e > 0 && !col_idxs[g])) {
      batch_release(b);
      set_error("gc_batch_load: graph " + std::to_string(g) + " is malformed");
      return GC_EINVAL;
    }
    b->h_off[g] = (int32_t)N;
    eoff[g] = E;
    N += ns[g];
    E += e;
    b->max_n = std::max(b->max_n, ns[g]);
    if (N >= INT32_MAX || E >= INT32_MAX) {
      batch_release(b);
      set_error("gc_batch_load: the union exceeds int32 CSR limits");
      return GC_ERANGE;
    }
  }
  b->h_off[count] = (int32_t)N;
  eoff[count] = E;
  b->N = (int32_t)N;
  b->nnz = E;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_batch_solve, kBatchThreads, 0) != cudaSuccess || occ < 1) {
    batch_release(b);
    set_error("gc_batch_load: the batch kernel cannot be resident");
    return GC_ECUDA;
  }
  b->ctas = std::min(kMaxGridCtas, occ * b->num_sms);
  const size_t Nn = (size_t)N;
  bool ok = balloc(&b->rp, Nn + 1) && balloc(&b->ci, (size_t)E) && balloc(&b->gid, Nn) &&
            balloc(&b->off, (size_t)count + 1) && balloc(&b->ng, (size_t)count) && balloc(&b->iota, Nn) &&
            balloc(&b->dS, Nn) && balloc(&b->mx, Nn) && balloc(&b->stamp, Nn) && balloc(&b->q0, Nn) &&
            balloc(&b->q1, Nn) && balloc(&b->goff, Nn + 1) && balloc(&b->st1, Nn) && balloc(&b->ub, Nn) && balloc(&b->key, Nn) &&
            balloc(&b->f0, Nn) && balloc(&b->packed, (size_t)count) && balloc(&b->fa, (size_t)count) &&
            balloc(&b->farness, (size_t)count) && balloc(&b->bestf, (size_t)count) &&
            balloc(&b->lc, (size_t)count) && balloc(&b->act_n, (size_t)count) && balloc(&b->full, (size_t)count) &&
            balloc(&b->kk, (size_t)count) && balloc(&b->bstart, (size_t)count + 1) && balloc(&b->ctl, 1) &&
            balloc(&b->slist, Nn) && balloc(&b->scount, (size_t)count) && balloc(&b->tstart, (size_t)count + 1) &&
            balloc(&b->rpf, Nn + 1) && balloc(&b->cif, std::max<size_t>(1, (size_t)E)) && balloc(&b->c3, Nn) &&
            balloc(&b->dS1, Nn) && balloc(&b->g3, 2 * (size_t)count) &&
            balloc(&b->gx, 3 * (size_t)std::max<int32_t>(1, b->max_n)) && balloc(&b->gg, 1) && balloc(&b->gsel, 1) &&
            balloc(&b->gctl, 1) && cudaMallocHost((void **)&b->h_ctl, sizeof(BatchCtl)) == cudaSuccess &&
            cudaMallocHost((void **)&b->h_gctl, sizeof(GainCtl)) == cudaSuccess;
  int64_t *d_eoff = nullptr;
  ok = ok && balloc(&d_eoff, (size_t)count + 1);
  // one workspace per CTA, sized for the largest graph
  b->ws_stride = gain_ws_stride(b->max_n);
  ok = ok && balloc(&b->ws, b->ws_stride * (size_t)b->ctas);
  if (!ok) {
    cudaFree(d_eoff);
    batch_release(b);
    set_error("gc_batch_load: device allocation failed");
    return GC_ENOMEM;
  }
  cudaStream_t st = b->stream;
  bool cp = true;
  for (int32_t g = 0; g < count; ++g) {
    cp = cp && cudaMemcpyAsync(b->rp + b->h_off[g], row_ptrs[g], (size_t)ns[g] * sizeof(int32_t),
                               cudaMemcpyDefault, st) == cudaSuccess;
    const int64_t e = eoff[g + 1] - eoff[g];
    if (e) cp = cp && cudaMemcpyAsync(b->ci + eoff[g], col_idxs[g], (size_t)e * sizeof(int32_t),
                                      cudaMemcpyDefault, st) == cudaSuccess;
  }
  const int32_t last = (int32_t)E;
  cp = cp && cudaMemcpyAsync(b->rp + N, &last, sizeof(int32_t), cudaMemcpyHostToDevice, st) == cudaSuccess &&
       cudaMemcpyAsync(b->off, b->h_off.data(), ((size_t)count + 1) * sizeof(int32_t), cudaMemcpyHostToDevice,
                       st) == cudaSuccess &&
       cudaMemcpyAsync(b->ng, ns, (size_t)count * sizeof(int32_t), cudaMemcpyHostToDevice, st) == cudaSuccess &&
       cudaMemcpyAsync(d_eoff, eoff.data(), ((size_t)count + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st) ==
           cudaSuccess &&
       cudaMemsetAsync(b->ws, 0, b->ws_stride * (size_t)b->ctas, st) == cudaSuccess;
  if (cp) {
    k_union_fix<<<b->num_sms * 8, 256, 0, st>>>(b->rp, b->ci, b->gid, b->off, d_eoff, count, (int32_t)N, E);
    k_iota<<<b->num_sms * 8, 256, 0, st>>>(b->iota, (int32_t)N);
    cp = cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(st) == cudaSuccess;
  }
  cudaFree(d_eoff);
  if (!cp) {
    batch_release(b);
    set_error("gc_batch_load: copy to the device failed");
    return GC_ECUDA;
  }
  *out = b;
  return GC_OK;
}

extern "C" {

int gc_batch_load(int32_t count, const int32_t *const *row_ptrs, const int32_t *const *col_idxs, const int32_t *ns,
                  uint32_t flags, void *stream, gc_batch **out) {
  (void)flags;
  return batch_load_impl(count, row_ptrs, col_idxs, ns, nullptr, stream, out);
}

int gc_batch_free(gc_batch *b) {
  if (b) {
    cudaStreamSynchronize(b->stream);
    batch_release(b);
  }
  return GC_OK;
}

int64_t gc_batch_vertices(const gc_batch *b) { return b ? b->N : -1; }

int gc_batch_greedy(gc_batch *b, const int32_t *ks, const gc_opts *opts_in, int32_t *groups, int64_t *farness,
                    gc_stats *stats) {
  if (!b || !ks || !groups || !farness) {
    set_error("bad argument to gc_batch_greedy");
    return GC_EINVAL;
  }
  gc_opts opts;
  if (opts_in) opts = *opts_in;
  else gc_opts_default(&opts);
  int32_t kmax = 1;
  int64_t ksum = 0;
  for (int32_t g = 0; g < b->count; ++g) {
    if (ks[g] < 1 || ks[g] > b->h_n[g]) {
      set_error("gc_batch_greedy: k of graph " + std::to_string(g) + " outside [1, n]");
      return GC_EINVAL;
    }
    kmax = std::max(kmax, ks[g]);
    ksum += ks[g];
  }
  const int32_t A = opts.active_target > 0 ? opts.active_target : 1024;
  const int32_t lanes1 = (opts.step_lanes > 0 && opts.step_lanes <= kLanes) ? opts.step_lanes : kLanes;
  const bool capture = (opts.flags & GC_OPT_CAPTURE) != 0;
  auto t0 = std::chrono::steady_clock::now();
  cudaStream_t st = b->stream;
  // (re)size per-call buffers; a resize invalidates a captured sequence
  bool resized = false;
  if (kmax > b->kcap) {
    cudaFree(b->picks);
    cudaFree(b->pgain);
    b->picks = nullptr;
    b->pgain = nullptr;
    if (!balloc(&b->picks, (size_t)b->count * kmax) || !balloc(&b->pgain, (size_t)b->count * kmax)) {
      set_error("gc_batch_greedy: allocation failed");
      return GC_ENOMEM;
    }
    b->kcap = kmax;
    resized = true;
    if (b->h_picks_pinned) cudaFreeHost(b->h_picks_pinned);
    if (cudaMallocHost((void **)&b->h_picks_pinned, (size_t)b->count * kmax * sizeof(int32_t)) != cudaSuccess) {
      set_error("gc_batch_greedy: pinned allocation failed");
      return GC_ENOMEM;
    }
  }
  if (!b->h_far_pinned && cudaMallocHost((void **)&b->h_far_pinned, (size_t)b->count * sizeof(long long)) != cudaSuccess) {
    set_error("gc_batch_greedy: pinned allocation failed");
    return GC_ENOMEM;
  }
  const int64_t need_seeds = std::max<int64_t>(b->count, ksum);
  if (need_seeds > b->seeds_cap) {
    cudaFree(b->seeds);
    if (!balloc(&b->seeds, (size_t)need_seeds)) {
      set_error("gc_batch_greedy: allocation failed");
      return GC_ENOMEM;
    }
    b->seeds_cap = (int32_t)need_seeds;
    resized = true;
  }
  if (A > b->act_cap) {
    cudaFree(b->act);
    if (!balloc(&b->act, (size_t)b->count * A)) {
      set_error("gc_batch_greedy: allocation failed");
      return GC_ENOMEM;
    }
    b->act_cap = A;
    resized = true;
  }
  if (!b->h_k_pinned && (cudaMallocHost((void **)&b->h_k_pinned, (size_t)b->count * sizeof(int32_t)) != cudaSuccess ||
                         cudaMallocHost((void **)&b->h_bstart_pinned, ((size_t)b->count + 1) * sizeof(int32_t)) !=
                             cudaSuccess)) {
    set_error("gc_batch_greedy: pinned allocation failed");
    return GC_ENOMEM;
  }
  std::vector<int32_t> bstart(b->count + 1, 0);
  for (int32_t g = 0; g < b->count; ++g) bstart[g + 1] = bstart[g] + (b->h_n[g] + lanes1 - 1) / lanes1;
  const bool same = b->exec && !resized && b->cap_k == std::vector<int32_t>(ks, ks + b->count) && b->cap_A == A && b->cap_grid_min_n == opts.batch_grid_min_n && b->cap_flags == opts.flags &&
                    b->cap_lanes == lanes1;
  BatchArgs a;
  a.rp = b->rp;
  a.ci = b->ci;
  a.N = b->N;
  a.count = b->count;
  a.gid = b->gid;
  a.off = b->off;
  a.ng = b->ng;
  a.kk = b->kk;
  a.iota = b->iota;
  a.bstart = b->bstart;
  a.lanes1 = lanes1;
  a.max_n = b->max_n;
  a.dS = b->dS;
  a.mx = b->mx;
  a.stamp = b->stamp;
  a.q0 = b->q0;
  a.q1 = b->q1;
  a.goff = b->goff;
  a.st1 = b->st1;
  a.rpf = b->rpf;
  a.cif = b->cif;
  a.c3 = b->c3;
  a.dS1 = b->dS1;
  a.gg = b->gg;
  a.gsel = b->gsel;
  a.gx = b->gx;
  a.bounded = (opts.flags & GC_OPT_NO_ROUND1_BOUND) ? 0 : 1;
  a.g3 = b->g3;
  a.grid_min_n = opts.batch_grid_min_n == 0 ? kBatchGridMinN
                 : (opts.batch_grid_min_n < 0 ? INT32_MAX : opts.batch_grid_min_n);
  a.ub = b->ub;
  a.key = b->key;
  a.f0 = b->f0;
  a.ws = b->ws;
  a.ws_stride = b->ws_stride;
  a.packed = b->packed;
  a.fa = b->fa;
  a.farness = b->farness;
  a.bestf = b->bestf;
  a.lc = b->lc;
  a.act = b->act;
  a.act_n = b->act_n;
  a.full = b->full;
  a.A = A;
  a.kmax = kmax;
  a.picks = b->picks;
  a.pgain = b->pgain;
  a.seeds = b->seeds;
  a.slist = b->slist;
  a.scount = b->scount;
  a.tstart = b->tstart;
  a.ctl = b->ctl;
  a.gctl = b->gctl;
  a.tns = opts.timeout_us > 0 ? (unsigned long long)opts.timeout_us * 1000ull
                              : (unsigned long long)((opts.timeout_ms > 0 ? opts.timeout_ms : 10000) * 1000000LL);
  auto enqueue = [&](cudaStream_t st) -> cudaError_t {
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b->kk, b->h_k_pinned, (size_t)b->count * sizeof(int32_t), cudaMemcpyHostToDevice, st)))
      return e;
    if ((e = cudaMemcpyAsync(b->bstart, b->h_bstart_pinned, bstart.size() * sizeof(int32_t), cudaMemcpyHostToDevice,
                             st)))
      return e;
    if ((e = cudaMemsetAsync(b->packed, 0xff, (size_t)b->count * sizeof(unsigned long long), st))) return e;
    if ((e = cudaMemsetAsync(b->fa, 0, (size_t)b->count * sizeof(long long), st))) return e;
    if ((e = cudaMemsetAsync(b->farness, 0, (size_t)b->count * sizeof(long long), st))) return e;
    if ((e = cudaMemsetAsync(b->lc, 0, (size_t)b->count * sizeof(LazyCtl), st))) return e;
    if ((e = cudaMemsetAsync(b->ctl, 0, sizeof(BatchCtl), st))) return e;
    if ((e = cudaMemsetAsync(b->gctl, 0, sizeof(GainCtl), st))) return e;
    if ((e = cudaMemsetAsync(b->gg, 0, sizeof(GridGainCtl), st))) return e;
    if ((e = cudaMemsetAsync(b->gsel, 0, sizeof(GridSelScratch), st))) return e;
    void *args[] = {(void *)&a};
    if ((e = cudaLaunchCooperativeKernel((const void *)k_batch_solve, dim3(b->ctas), dim3(kBatchThreads), args, 0,
                                         st)))
      return e;
    if ((e = cudaMemcpyAsync(b->h_picks_pinned, b->picks, (size_t)b->count * kmax * sizeof(int32_t),
                             cudaMemcpyDeviceToHost, st)))
      return e;
    if ((e = cudaMemcpyAsync(b->h_far_pinned, b->farness, (size_t)b->count * sizeof(long long),
                             cudaMemcpyDeviceToHost, st)))
      return e;
    if ((e = cudaMemcpyAsync(b->h_ctl, b->ctl, sizeof(BatchCtl), cudaMemcpyDeviceToHost, st))) return e;
    return cudaMemcpyAsync(b->h_gctl, b->gctl, sizeof(GainCtl), cudaMemcpyDeviceToHost, st);
  };
  bool used_graph = false;
  if (!(capture && same)) {  // a replay reads the pinned buffers it was captured from (same contents)
    cudaStreamSynchronize(st);  // no earlier copy may still read them
    memcpy(b->h_k_pinned, ks, (size_t)b->count * sizeof(int32_t));
    memcpy(b->h_bstart_pinned, bstart.data(), bstart.size() * sizeof(int32_t));
  }
  if (capture && same) {
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaGraphLaunch");
    used_graph = true;
  } else if (capture) {
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
    }
    b->cap_k.assign(ks, ks + b->count);
    b->cap_A = A;
    b->cap_lanes = lanes1;
    b->cap_grid_min_n = opts.batch_grid_min_n;
    b->cap_flags = opts.flags;
    // capture on a private non-blocking stream (the legacy default stream
    // cannot be captured); the graph is then launched on the caller's stream
    cudaError_t e = cudaSuccess;
    if (!b->cap_stream) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      e = enqueue(b->cap_stream);
      cudaGraph_t graph = nullptr;
      const cudaError_t e2 = cudaStreamEndCapture(b->cap_stream, &graph);
      if (e == cudaSuccess) e = e2;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, graph, 0);
      b->graph = graph;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      if (b->exec) cudaGraphExecDestroy(b->exec);
      if (b->graph) cudaGraphDestroy(b->graph);
      b->exec = nullptr;
      b->graph = nullptr;
      return cuda_fail(e, "capture of the batched solve");
    }
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return cuda_fail(cudaGetLastError(), "cudaGraphLaunch");
    used_graph = true;
  } else {
    const cudaError_t e = enqueue(st);
    if (e != cudaSuccess) return cuda_fail(e, "batched solve launch");
  }
  GC_CUDA(cudaStreamSynchronize(st));
  if (b->h_ctl->err) {
    cudaMemsetAsync(b->ws, 0, b->ws_stride * (size_t)b->ctas, st);
    cudaStreamSynchronize(st);
    const int e = b->h_ctl->err;
    set_error(e == GC_ETIMEOUT ? "device-side wait timed out" : e == GC_EDISCONNECTED ? "a graph is disconnected"
              : e == GC_ERANGE ? "a gain exceeds the batched solver's 31-bit key"
                               : "device-side check failed (phase " + std::to_string(b->h_ctl->dbg[0]) + ", graph " +
                                     std::to_string(b->h_ctl->dbg[1]) + ": expected " +
                                     std::to_string(b->h_ctl->dbg[2]) + ", found " +
                                     std::to_string(b->h_ctl->dbg[3]) + ")");
    return e;
  }
  int64_t pos = 0;
  for (int32_t g = 0; g < b->count; ++g) {
    for (int32_t r = 0; r < ks[g]; ++r) groups[pos + r] = b->h_picks_pinned[(size_t)g * kmax + r];
    for (int32_t r = 0; r < ks[g]; ++r) groups[pos + r] -= b->h_off[g];  // local ids
    pos += ks[g];
    farness[g] = b->h_far_pinned[g];
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->rounds = ksum;
    stats->steps = b->h_ctl->iterations;
    stats->batches = (int64_t)b->h_gctl->batches;
    stats->edges_scalar = (int64_t)b->h_gctl->edges_scalar;
    stats->edges_union = (int64_t)b->h_gctl->edges_union;
    stats->levels = (int64_t)b->h_gctl->levels;
    stats->frontier = (int64_t)b->h_gctl->frontier;
    stats->pushes = (int64_t)b->h_gctl->pushes;
    stats->lanes = (int64_t)b->h_gctl->lanes;
    stats->kernel_launches = 1;
    stats->graph_replay = used_graph ? 1 : 0;
    // phases of the solve (CTA 0's clock): rounds 0, 1, the lazy rounds, the check
    const unsigned long long *ph = b->h_ctl->ns_ph;
    stats->ms_round0 = ph[0] * 1e-6;
    stats->ms_round1 = (ph[1] - ph[0]) * 1e-6;
    stats->ms_lazy_kernel = (ph[2] - ph[1]) * 1e-6;  // the lazy rounds of every graph (P6)
    stats->ms_lazy_select = b->h_ctl->ns_lazy[0] * 1e-6;  // their phases, summed over graphs
    stats->ms_lazy_gain = b->h_ctl->ns_lazy[1] * 1e-6;
    stats->ms_lazy_update = b->h_ctl->ns_lazy[2] * 1e-6;
    stats->ms_gain_kernel = (ph[5] - ph[4]) * 1e-6;  // round-1 gains of every graph (P4)
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return GC_OK;
}

// gc_greedy_batch: the batched solve over graphs already loaded as handles.
// Their device CSRs are gathered into one union (device-to-device copies), the
// union is solved by gc_batch_greedy, and each group is handed back through its
// own output pointer.
int gc_greedy_batch(gc_graph *const *gs, const int32_t *ks, int32_t count, const gc_opts *opts,
                    int32_t *const *out_groups, int64_t *out_farness, gc_stats *stats) {
  if (!gs || !ks || count < 1 || !out_groups || !out_farness) {
    set_error("bad argument to gc_greedy_batch");
    return GC_EINVAL;
  }
  std::vector<const int32_t *> rps(count), cis(count);
  std::vector<int32_t> ns(count);
  std::vector<int64_t> nnz(count);
  int64_t ksum = 0;
  for (int32_t g = 0; g < count; ++g) {
    if (!gs[g] || !out_groups[g] || gs[g]->device != gs[0]->device) {
      set_error("gc_greedy_batch: graph " + std::to_string(g) +
                " is NULL, has no output array, or lives on another device");
      return GC_EINVAL;
    }
    rps[g] = gs[g]->rp;
    cis[g] = gs[g]->ci;
    ns[g] = gs[g]->n;
    nnz[g] = gs[g]->nnz;
    ksum += ks[g] > 0 ? ks[g] : 0;
  }
  // the handles' own streams may still be writing their CSRs (adopted arrays)
  for (int32_t g = 0; g < count; ++g)
    if (cudaStreamSynchronize(gs[g]->stream) != cudaSuccess) {
      set_error("gc_greedy_batch: a handle's stream failed");
      return GC_ECUDA;
    }
  gc_batch *b = nullptr;
  int rc = batch_load_impl(count, rps.data(), cis.data(), ns.data(), nnz.data(), gs[0]->stream, &b);
  if (rc != GC_OK) return rc;
  std::vector<int32_t> flat((size_t)std::max<int64_t>(1, ksum));
  rc = gc_batch_greedy(b, ks, opts, flat.data(), out_farness, stats);
  gc_batch_free(b);
  if (rc != GC_OK) return rc;
  size_t pos = 0;
  for (int32_t g = 0; g < count; ++g) {
    memcpy(out_groups[g], flat.data() + pos, (size_t)ks[g] * sizeof(int32_t));
    pos += (size_t)ks[g];
  }
  return GC_OK;
}

}  // extern "C"
