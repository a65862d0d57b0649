// Candidate selection and round bookkeeping of the lazy greedy (Sec. 4.2).
//
// Supermodularity of farness makes the gain computed for v in an earlier round
// an upper bound ub[v] on its gain now.  A round evaluates exactly the
// candidates with the largest bounds first and accepts the best exact gain g*
// (vertex v*, smallest id among equal gains) once no candidate left
// unevaluated in this round has ub > g*, or ub == g* with a smaller id -- the
// plain greedy's choice under the smallest-id rule.  Which candidates a step
// evaluates only changes the work, never the pick.
//
// Selection without sorting: a key range [lo, hi] is cut into kHistBins bins;
// one pass counts keys per bin, a one-CTA kernel walks the bins from the top
// until `want` candidates are covered and either fixes the threshold tau or
// narrows [lo, hi] to the boundary bin for another pass.  The compaction that
// follows is order-preserving (per-block counts, one scan, one write pass).
#include <limits.h>

#include "gc_device.cuh"
#include "gc_internal.cuh"

namespace gc {

// key of vertex v for the selection, or LLONG_MIN if v is not selectable
template <int MODE>
__device__ __forceinline__ long long sel_key(int v, const long long *__restrict__ ub,
                                             const int32_t *__restrict__ stamp, int32_t round,
                                             const long long *__restrict__ key) {
  if (MODE == kSelLazy) {
    const long long u = ub[v];
    return (u >= 0 && stamp[v] != round) ? u : LLONG_MIN;
  }
  if (MODE == kSelActive) {
    const long long u = ub[v];
    return u >= 0 ? u : LLONG_MIN;
  }
  return key[v];
}

// Reduce (max key, count) of selectable vertices; the last CTA writes
// ctl->hi, ctl->lo (= min key) and resets the threshold search.
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_sel_range(int32_t n, const long long *ub,
                                                           const int32_t *stamp, int32_t round,
                                                           const long long *key, long long *partial,
                                                           SelCtl *ctl) {
  __shared__ long long sh[32];
  __shared__ long long smx[32], smn[32];
  __shared__ bool last;
  long long mx = LLONG_MIN, mn = LLONG_MAX, c = 0;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const long long k = sel_key<MODE>(v, ub, stamp, round, key);
    if (k == LLONG_MIN) continue;
    mx = max(mx, k);
    mn = min(mn, k);
    ++c;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  if (lane == 0) {
    smx[wid] = mx;
    smn[wid] = mn;
  }
  c = block_sum(c, sh);
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) {
      mx = max(mx, smx[w]);
      mn = min(mn, smn[w]);
    }
    partial[3 * blockIdx.x] = mx;
    partial[3 * blockIdx.x + 1] = mn;
    partial[3 * blockIdx.x + 2] = c;
    __threadfence();
    last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
  }
  cta_sync();
  if (!last) return;
  __threadfence();
  mx = LLONG_MIN;
  mn = LLONG_MAX;
  c = 0;
  for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    mx = max(mx, ((volatile long long *)partial)[3 * b]);
    mn = min(mn, ((volatile long long *)partial)[3 * b + 1]);
    c += ((volatile long long *)partial)[3 * b + 2];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    mn = min(mn, __shfl_xor_sync(0xffffffffu, mn, o));
  }
  cta_sync();
  if (lane == 0) {
    smx[wid] = mx;
    smn[wid] = mn;
  }
  c = block_sum(c, sh);
  if (threadIdx.x != 0) return;
  for (int w = 1; w < nw; ++w) {
    mx = max(mx, smx[w]);
    mn = min(mn, smn[w]);
  }
  ctl->hi = mx;
  ctl->lo = mn;
  ctl->sel_count = c;
  ctl->done = c == 0;  // nothing selectable: select nothing
  ctl->tau = c == 0 ? LLONG_MAX : mn;
  ctl->ticket = 0;
}

// Histogram pass over [lo, hi] (skipped once the threshold is fixed).
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_sel_hist(int32_t n, const long long *ub,
                                                          const int32_t *stamp, int32_t round,
                                                          const long long *key, unsigned int *hist,
                                                          SelCtl *ctl) {
  __shared__ unsigned int sh[kHistBins];
  if (*(volatile int32_t *)&ctl->done) return;
  const long long lo = ctl->lo, hi = ctl->hi;
  // width = ceil((hi - lo + 1) / bins) in unsigned arithmetic (range may span 2^63)
  const unsigned long long span = (unsigned long long)hi - (unsigned long long)lo + 1ull;
  const unsigned long long width = span / kHistBins + ((span % kHistBins) ? 1ull : 0ull);
  for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) sh[i] = 0;
  cta_sync();
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const long long k = sel_key<MODE>(v, ub, stamp, round, key);
    if (k == LLONG_MIN || k < lo || k > hi) continue;
    const unsigned long long b = ((unsigned long long)k - (unsigned long long)lo) / width;
    atomicAdd(&sh[b], 1u);
  }
  cta_sync();
  for (int i = threadIdx.x; i < kHistBins; i += blockDim.x)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// One CTA: walk bins from the top until `want` keys are covered.  Fix tau if
// the boundary bin keeps the selection within `cap` or is one key wide;
// otherwise narrow [lo, hi] to the boundary bin (want reduced by what lies
// above) for another pass.  Clears the histogram for the next pass.
__global__ void __launch_bounds__(1024) k_sel_pick(unsigned int *hist, SelCtl *ctl, int32_t cap,
                                                   int32_t *want_dev) {
  static_assert(kHistBins == 2048, "two bins per thread of a 1024-thread CTA");
  __shared__ int sh[33];
  __shared__ int s_b;
  __shared__ long long s_above, s_here;
  const bool done = *(volatile int32_t *)&ctl->done;
  if (!done) {
    const long long want = *want_dev;
    // thread t owns bins b0 = 2047 - 2t and b1 = b0 - 1 (walking down from the top)
    const int b0 = kHistBins - 1 - 2 * (int)threadIdx.x, b1 = b0 - 1;
    const int h0 = (int)hist[b0], h1 = (int)hist[b1];
    if (threadIdx.x == 0) {
      s_b = 0;
      s_above = 0;
      s_here = 0;
    }
    int total;
    const long long above0 = block_excl_scan(h0 + h1, sh, &total);  // keys in bins > b0
    if (above0 < want && above0 + h0 >= want) {
      s_b = b0;
      s_above = above0;
      s_here = h0;
    } else if (above0 + h0 < want && above0 + h0 + h1 >= want) {
      s_b = b1;
      s_above = above0 + h0;
      s_here = h1;
    }
    if (threadIdx.x == 0 && (long long)total < want) {  // everything fits: select all
      s_b = 0;
      s_above = total - (long long)hist[0];
      s_here = hist[0];
    }
    cta_sync();
    if (threadIdx.x == 0) {
      const unsigned long long lo = (unsigned long long)ctl->lo, hi = (unsigned long long)ctl->hi;
      const unsigned long long span = hi - lo + 1ull;
      const unsigned long long width = span / kHistBins + ((span % kHistBins) ? 1ull : 0ull);
      const int b = s_b;
      const long long above = s_above, here = s_here;
      const unsigned long long bin_lo = lo + width * (unsigned long long)b;
      ctl->tau = (long long)bin_lo;
      if (above + here <= cap || width == 1ull || (b == 0 && above + here < want)) {
        ctl->done = 1;
      } else {
        const unsigned long long room = hi - bin_lo;  // keys above bin_lo still in range
        ctl->lo = (long long)bin_lo;
        ctl->hi = (long long)(bin_lo + (width - 1ull < room ? width - 1ull : room));
        *want_dev = (int32_t)(want - above);
      }
    }
  }
  for (int i = threadIdx.x; i < kHistBins; i += blockDim.x) hist[i] = 0;
}

// Compaction, pass 1: per-block counts of selectable keys >= tau.
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_compact_count(int32_t n, const long long *ub,
                                                               const int32_t *stamp, int32_t round,
                                                               const long long *key, SelCtl *ctl,
                                                               int32_t *blk) {
  __shared__ long long sh[32];
  const long long tau = ctl->tau;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int beg = blockIdx.x * per, end = min(n, beg + per);
  long long c = 0;
  for (int v = beg + threadIdx.x; v < end; v += blockDim.x) {
    const long long k = sel_key<MODE>(v, ub, stamp, round, key);
    c += (k != LLONG_MIN && k >= tau);
  }
  c = block_sum(c, sh);
  if (threadIdx.x == 0) blk[blockIdx.x] = (int32_t)c;
}

// Compaction, pass 2 (one CTA): exclusive scan of block counts; total -> n_sel.
__global__ void __launch_bounds__(1024) k_compact_scan(int32_t *blk, int32_t nblk, SelCtl *ctl) {
  __shared__ int sh[33];
  int carry = 0;
  for (int base = 0; base < nblk; base += blockDim.x) {
    const int i = base + threadIdx.x;
    const int v = i < nblk ? blk[i] : 0;
    int total;
    const int ex = block_excl_scan(v, sh, &total);
    if (i < nblk) blk[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) ctl->n_sel = carry;
}

// Compaction, pass 3: write the selected ids in vertex order.
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_compact_write(int32_t n, const long long *ub,
                                                               const int32_t *stamp, int32_t round,
                                                               const long long *key, SelCtl *ctl,
                                                               const int32_t *blk, int32_t *list) {
  __shared__ int sh[33];
  const long long tau = ctl->tau;
  const int per = (n + gridDim.x - 1) / gridDim.x;
  const int beg = blockIdx.x * per, end = min(n, beg + per);
  int off = blk[blockIdx.x];
  for (int base = beg; base < end; base += blockDim.x) {
    const int v = base + threadIdx.x;
    int f = 0;
    if (v < end) {
      const long long k = sel_key<MODE>(v, ub, stamp, round, key);
      f = (k != LLONG_MIN && k >= tau);
    }
    int total;
    const int ex = block_excl_scan(f, sh, &total);
    if (f) list[off + ex] = v;
    off += total;
  }
}

// (value, id) arg-reduction helper for one CTA; thread 0 gets the result.
template <bool MAX>
__device__ __forceinline__ void block_arg(long long &v, int &id, long long *sv, int *sid) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oid = __shfl_xor_sync(0xffffffffu, id, o);
    if (MAX ? better_max(ov, oid, v, id) : better_min(ov, oid, v, id)) {
      v = ov;
      id = oid;
    }
  }
  cta_sync();
  if (lane == 0) {
    sv[wid] = v;
    sid[wid] = id;
  }
  cta_sync();
  if (threadIdx.x == 0)
    for (int w = 1; w < nw; ++w)
      if (MAX ? better_max(sv[w], sid[w], v, id) : better_min(sv[w], sid[w], v, id)) {
        v = sv[w];
        id = sid[w];
      }
}

// After a lazy step: ub[v] <- exact gain, stamp[v] <- round; fold the step's
// best (gain desc, id asc) into ctl->best_gain / best_id; count evaluations.
__global__ void __launch_bounds__(kRedThreads) k_after_eval_lazy(const int32_t *list,
                                                                 const long long *lgain,
                                                                 long long *ub, int32_t *stamp,
                                                                 int32_t round, long long *partial,
                                                                 SelCtl *ctl) {
  __shared__ long long sv[32];
  __shared__ int sid[32];
  __shared__ bool last;
  const int n_list = ctl->n_sel;
  long long bv = -1;
  int bid = -1;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_list; i += gridDim.x * blockDim.x) {
    const int v = list[i];
    const long long gv = lgain[i];
    ub[v] = gv;
    stamp[v] = round;
    if (better_max(gv, v, bv, bid)) {
      bv = gv;
      bid = v;
    }
  }
  block_arg<true>(bv, bid, sv, sid);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = bv;
    partial[2 * blockIdx.x + 1] = bid;
    __threadfence();
    last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
  }
  cta_sync();
  if (!last) return;
  __threadfence();
  bv = ctl->best_gain;
  bid = ctl->best_id;
  for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const long long v = ((volatile long long *)partial)[2 * b];
    const int id = (int)((volatile long long *)partial)[2 * b + 1];
    if (id >= 0 && better_max(v, id, bv, bid)) {
      bv = v;
      bid = id;
    }
  }
  block_arg<true>(bv, bid, sv, sid);
  if (threadIdx.x != 0) return;
  ctl->best_gain = bv;
  ctl->best_id = bid;
  ctl->evals += n_list;  // evaluations of the call
  ctl->steps += 1;       // steps of the call
  ctl->ticket = 0;
}

// Best bound among candidates not evaluated in this round, and the acceptance
// test of the lazy greedy: accept (best_gain, best_id) iff it beats that bound
// in the (value desc, id asc) order.
__global__ void __launch_bounds__(kRedThreads) k_unevaluated_best(int32_t n, const long long *ub,
                                                                  const int32_t *stamp, int32_t round,
                                                                  long long *partial, SelCtl *ctl) {
  __shared__ long long sv[32];
  __shared__ int sid[32];
  __shared__ bool last;
  long long bv = LLONG_MIN;
  int bid = -1;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const long long u = ub[v];
    if (u < 0 || stamp[v] == round) continue;
    if (better_max(u, v, bv, bid)) {
      bv = u;
      bid = v;
    }
  }
  block_arg<true>(bv, bid, sv, sid);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = bv;
    partial[2 * blockIdx.x + 1] = bid;
    __threadfence();
    last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
  }
  cta_sync();
  if (!last) return;
  __threadfence();
  bv = LLONG_MIN;
  bid = -1;
  for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const long long v = ((volatile long long *)partial)[2 * b];
    const int id = (int)((volatile long long *)partial)[2 * b + 1];
    if (id >= 0 && better_max(v, id, bv, bid)) {
      bv = v;
      bid = id;
    }
  }
  block_arg<true>(bv, bid, sv, sid);
  if (threadIdx.x != 0) return;
  ctl->unev_ub = bv;
  ctl->unev_id = bid;
  ctl->accepted = ctl->best_id >= 0 && (bid < 0 || better_max(ctl->best_gain, ctl->best_id, bv, bid));
  ctl->ticket = 0;
}

// Round 0 bookkeeping: f0[v] <- exact farness or -1 (cut), key[v] <- done.
__global__ void k_after_eval_round0(const int32_t *list, const long long *lgain, long long *f0,
                                    long long *key, const SelCtl *ctl) {
  const int n_list = ctl->n_sel;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_list; i += gridDim.x * blockDim.x) {
    const int v = list[i];
    f0[v] = lgain[i];
    key[v] = LLONG_MIN;
  }
}

// argmin (value, id): MODE 0 over exactly evaluated f0 (s0 of round 0);
// MODE 1 over the round-0 lower bounds -key (the vertex whose BFS seeds the
// cut threshold).  Result -> ctl->arg_val / arg_id.
template <int MODE>
__global__ void __launch_bounds__(kRedThreads) k_argmin(int32_t n, const long long *arr,
                                                        long long *partial, SelCtl *ctl) {
  __shared__ long long sv[32];
  __shared__ int sid[32];
  __shared__ bool last;
  long long bv = LLONG_MAX;
  int bid = -1;
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
    const long long a = arr[v];
    const bool valid = MODE == 0 ? a >= 0 : a != LLONG_MIN;
    const long long f = MODE == 0 ? a : -a;
    if (valid && better_min(f, v, bv, bid)) {
      bv = f;
      bid = v;
    }
  }
  block_arg<false>(bv, bid, sv, sid);
  if (threadIdx.x == 0) {
    partial[2 * blockIdx.x] = bv;
    partial[2 * blockIdx.x + 1] = bid;
    __threadfence();
    last = atomicAdd(&ctl->ticket, 1u) == gridDim.x - 1;
  }
  cta_sync();
  if (!last) return;
  __threadfence();
  bv = LLONG_MAX;
  bid = -1;
  for (int b = threadIdx.x; b < gridDim.x; b += blockDim.x) {
    const long long v = ((volatile long long *)partial)[2 * b];
    const int id = (int)((volatile long long *)partial)[2 * b + 1];
    if (id >= 0 && better_min(v, id, bv, bid)) {
      bv = v;
      bid = id;
    }
  }
  block_arg<false>(bv, bid, sv, sid);
  if (threadIdx.x != 0) return;
  ctl->arg_val = bv;
  ctl->arg_id = bid;
  ctl->ticket = 0;
}

// Round 0 after the BFS from the lowest-bound vertex v_a: its exact farness
// (ctl->sum) becomes f0[v_a], the cut threshold best_f, and the selection
// threshold tau = -best_f (every vertex whose bound does not exceed it).
__global__ void k_round0_seed(long long *f0, long long *key, SelCtl *ctl, GainCtl *gctl) {
  const int v = ctl->arg_id;
  const long long f = ctl->sum;
  if (v >= 0) {
    f0[v] = f;
    key[v] = LLONG_MIN;
  }
  gctl->best_f = f;
  ctl->tau = -f;
}

__global__ void k_round0_pivot(long long *f0, long long *key, SelCtl *ctl, GainCtl *gctl) {
  const int v = ctl->arg_id;
  const long long f = ctl->sum;
  if (v >= 0) {
    f0[v] = f;
    key[v] = LLONG_MIN;
  }
  if (f < gctl->best_f) gctl->best_f = f;
  ctl->tau = -gctl->best_f;
}

// Top-k closeness: the selection key of every exactly searched vertex is its
// negated farness (the k largest keys are the k smallest farness values);
// vertices never searched, or cut, are not selectable.
__global__ void k_topk_keys(const long long *f0, int32_t n, long long *key) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    key[v] = f0[v] >= 0 ? -f0[v] : LLONG_MIN;
}

// lgain[i] <- f0[list[i]] for the selected list
__global__ void k_gather_f0(const int32_t *list, const long long *f0, long long *lgain, const SelCtl *ctl) {
  const int m = ctl->n_sel;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) lgain[i] = f0[list[i]];
}

// Start of a lazy round: clear the round's best and the acceptance flag.
__global__ void k_round_begin(SelCtl *ctl) {
  ctl->best_gain = -1;
  ctl->best_id = -1;
  ctl->accepted = 0;
}

// Round 1 work estimate: key[v] = deg(v) for non-members, LLONG_MIN for members.
__global__ void k_degree_keys(const int32_t *__restrict__ rp, int32_t n, const long long *__restrict__ ub,
                              long long *key) {
  for (int v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x)
    key[v] = ub[v] >= 0 ? (long long)(rp[v + 1] - rp[v]) : LLONG_MIN;
}

// Keep at most `cap` entries of the compacted list (the list is in vertex
// order; the dropped tail stays unevaluated and keeps its bound).
__global__ void k_clamp_nsel(SelCtl *ctl, int32_t cap) {
  if (ctl->n_sel > cap) ctl->n_sel = cap;
}

// End of a lazy round: remove the pick from the candidates.
__global__ void k_round_end(long long *ub, const SelCtl *ctl) {
  const int v = ctl->best_id;
  if (v >= 0) ub[v] = -1;
}

// ------------------------------------------------------------- launchers ----
template <int MODE>
static int select_impl(gc_graph *g, int32_t round, int32_t want, int tau_mode, long long tau) {
  const int rb = g->red_blocks;
  if (tau_mode == kTauHost) {
    // tau given: no range/histogram passes
    GC_CUDA(cudaMemcpyAsync(&g->sctl->tau, &tau, sizeof(long long), cudaMemcpyHostToDevice, g->stream));
  } else if (tau_mode == kTauHistogram || tau_mode == kTauHistogramTheta) {
    GC_CUDA(cudaMemcpyAsync(g->blk + rb, &want, sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
    ++g->launches;
    k_sel_range<MODE><<<rb, kRedThreads, 0, g->stream>>>(g->n, g->ub, g->stamp, round, g->key, g->partial,
                                                         g->sctl);
    GC_CUDA(cudaGetLastError());
    for (int pass = 0; pass < 3; ++pass) {
      ++g->launches;
      k_sel_hist<MODE><<<rb, kRedThreads, 0, g->stream>>>(g->n, g->ub, g->stamp, round, g->key, g->hist,
                                                          g->sctl);
      ++g->launches;
      k_sel_pick<<<1, 1024, 0, g->stream>>>(g->hist, g->sctl, 2 * want, g->blk + rb);
      GC_CUDA(cudaGetLastError());
    }
    if (tau_mode == kTauHistogramTheta) {
      const int rc = launch_active_theta(g);
      if (rc != GC_OK) return rc;
    }
  }
  ++g->launches;
  k_compact_count<MODE><<<rb, kRedThreads, 0, g->stream>>>(g->n, g->ub, g->stamp, round, g->key, g->sctl,
                                                           g->blk);
  ++g->launches;
  k_compact_scan<<<1, 1024, 0, g->stream>>>(g->blk, rb, g->sctl);
  ++g->launches;
  k_compact_write<MODE><<<rb, kRedThreads, 0, g->stream>>>(g->n, g->ub, g->stamp, round, g->key, g->sctl,
                                                           g->blk, g->list);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_select(gc_graph *g, int mode, int32_t round, int32_t want, int tau_mode, long long tau) {
  if (mode == kSelLazy) return select_impl<kSelLazy>(g, round, want, tau_mode, tau);
  if (mode == kSelActive) return select_impl<kSelActive>(g, round, want, tau_mode, tau);
  return select_impl<kSelKey>(g, round, want, tau_mode, tau);
}

int launch_after_eval(gc_graph *g, int32_t round, int32_t n_list) {
  (void)n_list;
  ++g->launches;
  if (round == 0)
    k_after_eval_round0<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->list, g->lgain, g->f0, g->key,
                                                                      g->sctl);
  else
    k_after_eval_lazy<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->list, g->lgain, g->ub, g->stamp,
                                                                    round, g->partial, g->sctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_unevaluated_best(gc_graph *g, int32_t round) {
  ++g->launches;
  k_unevaluated_best<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->n, g->ub, g->stamp, round,
                                                                   g->partial, g->sctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_argmin_f0(gc_graph *g) {
  ++g->launches;
  k_argmin<0><<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->n, g->f0, g->partial, g->sctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_argmin_lb(gc_graph *g) {
  ++g->launches;
  k_argmin<1><<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->n, g->key, g->partial, g->sctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_topk_keys(gc_graph *g) {
  ++g->launches;
  k_topk_keys<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->f0, g->n, g->key);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_gather_f0(gc_graph *g) {
  ++g->launches;
  k_gather_f0<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->list, g->f0, g->lgain, g->sctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_round0_seed(gc_graph *g) {
  ++g->launches;
  k_round0_seed<<<1, 1, 0, g->stream>>>(g->f0, g->key, g->sctl, g->gctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_round0_pivot(gc_graph *g) {
  ++g->launches;
  k_round0_pivot<<<1, 1, 0, g->stream>>>(g->f0, g->key, g->sctl, g->gctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_round_begin(gc_graph *g) {
  ++g->launches;
  k_round_begin<<<1, 1, 0, g->stream>>>(g->sctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_degree_keys(gc_graph *g) {
  ++g->launches;
  k_degree_keys<<<g->red_blocks, kRedThreads, 0, g->stream>>>(g->rp, g->n, g->ub, g->key);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_clamp_nsel(gc_graph *g, int32_t cap) {
  ++g->launches;
  k_clamp_nsel<<<1, 1, 0, g->stream>>>(g->sctl, cap);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_round_end(gc_graph *g) {
  ++g->launches;
  k_round_end<<<1, 1, 0, g->stream>>>(g->ub, g->sctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

}  // namespace gc
