// Device-side pieces of the lazy greedy (Sec. 4.2) shared by the persistent
// single-graph kernel (gc_lazy.cu) and the batched multi-graph solver
// (gc_batch.cu): exact top-K selection by one CTA, the per-step decision of a
// graph's lazy round, and proposal scoring.
#pragma once

#include <limits.h>

#include "gc_grid.cuh"
#include "gc_mlp.cuh"

namespace gc {

constexpr int kLazyBins = 1024;  // two bins per thread of a 512-thread CTA

static __device__ __forceinline__ long long block_min_ll(long long v, long long *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  cta_sync();
  if (lane == 0) sh[wid] = v;
  cta_sync();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) v = min(v, sh[w]);
    sh[0] = v;
  }
  cta_sync();
  v = sh[0];
  cta_sync();
  return v;
}

static __device__ __forceinline__ long long block_max_ll(long long v, long long *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  cta_sync();
  if (lane == 0) sh[wid] = v;
  cta_sync();
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w) v = max(v, sh[w]);
    sh[0] = v;
  }
  cta_sync();
  v = sh[0];
  cta_sync();
  return v;
}

// (value, id) block arg-max; every thread gets the result.
static __device__ __forceinline__ void block_argmax_all(long long &v, int &id, long long *sv, int *sid) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oid = __shfl_xor_sync(0xffffffffu, id, o);
    if (better_max(ov, oid, v, id)) {
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
  if (threadIdx.x == 0) {
    for (int w = 1; w < nw; ++w)
      if (better_max(sv[w], sid[w], v, id)) {
        v = sv[w];
        id = sid[w];
      }
    sv[0] = v;
    sid[0] = id;
  }
  cta_sync();
  v = sv[0];
  id = sid[0];
  cta_sync();
}

// CTA 0's sorted view of its shared-memory list (lean steps): the positions
// of the entries with a bound >= 0 in the order (bound desc, position asc) --
// position order is id order, so this is the selection's order, ties to the
// smaller id.  A step's batch is then the first 64 entries not evaluated in
// the round, the same set the histogram selection finds.  A fold changes the
// bounds of its batch only (exact gains), so the view is kept by one merge of
// the re-sorted batch into the other entries; members (bound -1) leave it at
// the next fold.  ord and tmp hold kCta0SelectMax entries, mark as many bytes
// (zero between folds), *nord the view's length.
struct SortedView {
  uint16_t *ord, *tmp;
  unsigned char *mark;
  int *nord;
};

// a precedes b in the view
static __device__ __forceinline__ bool sv_before(const long long *sk, int a, int b) {
  const long long ka = sk[a], kb = sk[b];
  return ka > kb || (ka == kb && a < b);
}

// The view of sk[0..m): the positions with sk >= 0, bitonic-sorted (padding
// positions 0xffff go last).  Whole CTA.
static __device__ void sv_build(const long long *sk, int m, const SortedView &v) {
  __shared__ int s_scan[33];
  const int tid = threadIdx.x, T = blockDim.x;
  int nv = 0;
  for (int base = 0; base < m; base += T) {
    const int i = base + tid;
    const int e = (i < m && sk[i] >= 0) ? 1 : 0;
    if (i < m) v.mark[i] = 0;
    int tot;
    const int off = block_excl_scan(e, s_scan, &tot);
    if (e) v.ord[nv + off] = (uint16_t)i;
    nv += tot;
  }
  int N = 1;
  while (N < nv) N <<= 1;
  for (int i = nv + tid; i < N; i += T) v.ord[i] = 0xffffu;
  cta_sync();
  for (int k = 2; k <= N; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = tid; i < N; i += T) {
        const int ixj = i ^ j;
        if (ixj > i) {
          const int a = v.ord[i], b = v.ord[ixj];
          const bool b_first = b != 0xffff && (a == 0xffff || sv_before(sk, b, a));
          const bool a_first = a != 0xffff && (b == 0xffff || sv_before(sk, a, b));
          if ((i & k) == 0 ? b_first : a_first) {
            v.ord[i] = (uint16_t)b;
            v.ord[ixj] = (uint16_t)a;
          }
        }
      }
      cta_sync();
    }
  if (tid == 0) *v.nord = nv;
  cta_sync();
}

// After a fold: the batch's entries (list positions pos[0..ns), their bounds
// in sk already the exact gains) leave the view, entries with sk < 0 are
// dropped, and the batch, sorted by rank counting, is merged back.  Whole CTA.
static __device__ void sv_refold(const long long *sk, const int32_t *pos, int ns, const SortedView &v) {
  __shared__ uint16_t s_nb[kLanes];
  __shared__ int s_scan[33];
  const int tid = threadIdx.x, T = blockDim.x;
  if (tid < ns) v.mark[pos[tid]] = 1;
  cta_sync();
  const int nord = *v.nord;
  // the kept entries, in order, to tmp: contiguous chunks per thread
  const int C = (nord + T - 1) / T;
  const int i0 = min(nord, tid * C), i1 = min(nord, i0 + C);
  int keep = 0;
  for (int i = i0; i < i1; ++i) {
    const int p = v.ord[i];
    keep += (!v.mark[p] && sk[p] >= 0) ? 1 : 0;
  }
  int nkeep;
  int at = block_excl_scan(keep, s_scan, &nkeep);
  for (int i = i0; i < i1; ++i) {
    const int p = v.ord[i];
    if (!v.mark[p] && sk[p] >= 0) v.tmp[at++] = (uint16_t)p;
  }
  if (tid < ns) {  // the batch in view order
    const int p = pos[tid];
    int rk = 0;
    for (int j = 0; j < ns; ++j) rk += sv_before(sk, pos[j], p) ? 1 : 0;
    s_nb[rk] = (uint16_t)p;
  }
  cta_sync();
  if (tid < ns) v.mark[pos[tid]] = 0;
  // merge: each entry's rank is its index plus the entries of the other run
  // before it (binary search)
  for (int i = tid; i < nkeep; i += T) {
    const int p = v.tmp[i];
    int lo = 0, hi = ns;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sv_before(sk, s_nb[mid], p)) lo = mid + 1;
      else hi = mid;
    }
    v.ord[i + lo] = (uint16_t)p;
  }
  if (tid < ns) {
    const int p = s_nb[tid];
    int lo = 0, hi = nkeep;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sv_before(sk, v.tmp[mid], p)) lo = mid + 1;
      else hi = mid;
    }
    v.ord[tid + lo] = (uint16_t)p;
  }
  if (tid == 0) *v.nord = nkeep + ns;
  cta_sync();
}

// The first `need` entries of the view not evaluated in round r (and with a
// bound >= 0) to sel/selpos, in view order; *umax/*vmax get the first one's
// bound and id (LLONG_MIN / -1 if none).  Returns how many were taken.
// Whole CTA; *scanned counts the view entries read.
static __device__ int sv_select(const long long *sk, const int32_t *sa, const int32_t *ss, int r,
                                const SortedView &v, int need, int32_t *sel, int32_t *selpos, long long *umax,
                                int *vmax, unsigned long long *scanned) {
  __shared__ int s_scan[33];
  __shared__ long long s_u;
  __shared__ int s_v;
  const int tid = threadIdx.x, T = blockDim.x;
  const int nord = *v.nord;
  if (tid == 0) {
    s_u = LLONG_MIN;
    s_v = -1;
  }
  int taken = 0, base = 0;
  for (; base < nord && taken < need; base += T) {
    const int i = base + tid;
    const int p = i < nord ? v.ord[i] : 0;
    const bool e = i < nord && sk[p] >= 0 && ss[p] != r;
    int tot;
    const int off = block_excl_scan(e ? 1 : 0, s_scan, &tot);
    if (e && taken + off < need) {
      sel[taken + off] = sa[p];
      selpos[taken + off] = p;
      if (taken + off == 0) {
        s_u = sk[p];
        s_v = sa[p];
      }
    }
    taken += tot;
  }
  cta_sync();
  *umax = s_u;
  *vmax = s_v;
  if (tid == 0 && scanned) atomicAdd(scanned, (unsigned long long)min(base, nord));
  return taken < need ? taken : need;
}

// The per-step statistics of CTA 0's list scan in one exchange: the best
// (value, id) pair, the smallest value and the count, each reduced over the
// warp by shuffles, then over the warps by every thread from shared memory.
// One CTA barrier: the arrays are this function's own, and a caller runs other
// barriers between two calls.
static __device__ __forceinline__ void block_scan_stats(long long &umax, int &vmax, long long &umin,
                                                        long long &cnt) {
  __shared__ long long s_mx[32], s_mn[32], s_ct[32];
  __shared__ int s_id[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const long long ov = __shfl_xor_sync(0xffffffffu, umax, o);
    const int oid = __shfl_xor_sync(0xffffffffu, vmax, o);
    if (better_max(ov, oid, umax, vmax)) {
      umax = ov;
      vmax = oid;
    }
    umin = min(umin, __shfl_xor_sync(0xffffffffu, umin, o));
    cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
  }
  if (lane == 0) {
    s_mx[wid] = umax;
    s_id[wid] = vmax;
    s_mn[wid] = umin;
    s_ct[wid] = cnt;
  }
  cta_sync();
  umax = s_mx[0];
  vmax = s_id[0];
  umin = s_mn[0];
  cnt = s_ct[0];
  for (int w = 1; w < nw; ++w) {
    if (better_max(s_mx[w], s_id[w], umax, vmax)) {
      umax = s_mx[w];
      vmax = s_id[w];
    }
    umin = min(umin, s_mn[w]);
    cnt += s_ct[w];
  }
}

// Exact top-`need` of the list entries by key (larger first; ties by list
// order, i.e. smaller id), written to sel[base..cap) and, when selpos is
// given, their list positions to selpos[base..cap).  key(i, v) returns LLONG_MIN
// for entries that are not eligible; kmin/kmax/cnt describe the eligible keys.
// Histogram passes over [kmin, kmax] fix the threshold value; every key above it
// is taken, then keys equal to it in list order.  Returns the number taken.
template <class KeyFn>
static __device__ int cta_topk(const int32_t *act, int32_t m, KeyFn key, long long kmin, long long kmax,
                        long long cnt, int need, int32_t *sel, int base, unsigned int *s_hist,
                        int32_t *selpos = nullptr, unsigned long long *scanned = nullptr, int cap = kLanes) {
  __shared__ int s_scan[33];
  __shared__ int s_b;
  __shared__ long long s_ab;
  const int tid = threadIdx.x, T = blockDim.x;
  if (need <= 0 || cnt <= 0) return 0;
  if (need > cnt) need = (int)cnt;
  long long tau = kmin, above = 0;  // above = eligible keys > tau
  if (cnt > need) {
    unsigned long long lo = (unsigned long long)kmin, hi = (unsigned long long)kmax;
    long long want = need, acc = 0;
    for (int pass = 0; pass < 8; ++pass) {
      const unsigned long long span = hi - lo + 1ull;
      const unsigned long long width = span / kLazyBins + ((span % kLazyBins) ? 1ull : 0ull);
      for (int i = tid; i < kLazyBins; i += T) s_hist[i] = 0;
      if (scanned && tid == 0) *scanned += (unsigned long long)m;
      cta_sync();
      for (int i = tid; i < m; i += T) {
        const long long k = key(i, act[i]);
        if (k == LLONG_MIN) continue;
        const unsigned long long uu = (unsigned long long)k;
        if (uu - lo > hi - lo) continue;  // outside [lo, hi] (unsigned wrap)
        atomicAdd(&s_hist[(uu - lo) / width], 1u);
      }
      cta_sync();
      // walk down from the top bin: thread t owns bins 1023-2t and 1022-2t
      const int b0 = kLazyBins - 1 - 2 * tid, b1 = b0 - 1;
      const int h0 = tid < kLazyBins / 2 ? (int)s_hist[b0] : 0;
      const int h1 = tid < kLazyBins / 2 ? (int)s_hist[b1] : 0;
      if (tid == 0) {
        s_b = 0;
        s_ab = 0;
      }
      int total;
      const long long a0 = block_excl_scan(h0 + h1, s_scan, &total);
      if (tid < kLazyBins / 2) {
        if (a0 < want && a0 + h0 >= want) {
          s_b = b0;
          s_ab = a0;
        } else if (a0 + h0 < want && a0 + h0 + h1 >= want) {
          s_b = b1;
          s_ab = a0 + h0;
        }
      }
      cta_sync();
      const int bb = s_b;
      const long long ab = s_ab;
      const unsigned long long bin_lo = lo + width * (unsigned long long)bb;
      if (width == 1ull) {
        tau = (long long)bin_lo;
        above = acc + ab;
        break;
      }
      acc += ab;
      want -= ab;
      const unsigned long long room = hi - bin_lo;
      lo = bin_lo;
      hi = bin_lo + (width - 1ull < room ? width - 1ull : room);
      cta_sync();
    }
  }
  // Selection in list order.  Thread t owns the contiguous entries [t C, t C + C):
  // one pass counts its keys above and equal to tau, two block scans give the
  // counts before its first entry, a second pass writes its taken entries at
  // rank (entries above tau before it) + min(entries equal before it, eq_take).
  const int eq_take = (int)(need - above);  // equal keys taken, the first ones in list order
  const int C = (m + T - 1) / T;
  const int i0 = min(m, tid * C), i1 = min(m, i0 + C);
  int ngt = 0, neq = 0;
  for (int i = i0; i < i1; ++i) {
    const long long k = key(i, act[i]);
    if (k == LLONG_MIN) continue;
    ngt += k > tau;
    neq += k == tau;
  }
  if (scanned && tid == 0) *scanned += (unsigned long long)m;
  int tot_gt, tot_eq;
  int gt_before = block_excl_scan(ngt, s_scan, &tot_gt);
  int eq_before = block_excl_scan(neq, s_scan, &tot_eq);
  if (ngt > 0 || (neq > 0 && eq_before < eq_take)) {
    for (int i = i0; i < i1; ++i) {
      const int v = act[i];
      const long long k = key(i, v);
      if (k == LLONG_MIN) continue;
      const bool gt = k > tau, eq = k == tau;
      if (gt || (eq && eq_before < eq_take)) {
        const int pos = gt_before + min(eq_before, eq_take);
        if (base + pos < cap) {
          sel[base + pos] = v;
          if (selpos) selpos[base + pos] = i;
        }
      }
      gt_before += gt;
      eq_before += eq;
    }
  }
  cta_sync();
  const int taken = tot_gt + min(tot_eq, eq_take);
  return taken < need ? taken : need;
}

// CTA 0's part of a step (see the file comment).  Writes lc->dec (0 evaluate
// lc->sel[0..n_sel), 1 accept lc->best_id, 2 rebuild the list).  With compact
// keys (akey/ast non-null: ub and stamp of list entry i at position i, kept in
// step with ub/stamp), every scan of the list reads contiguous words instead of
// gathering ub[v] and stamp[v]; lc->selpos/best_pos then hold list positions.
// With wcap > 0 (wide steps) a step selects up to wcap candidates into
// wsel/wpos (their gains come back in wgain) instead of 64 into lc->sel.  With a
// proposal network (score != nullptr), `fill` of the 64 lanes go to the
// unevaluated candidates whose bound most exceeds the network's predicted
// gain: evaluating them tightens the bounds later rounds must beat.
static __device__ void lazy_cta0_step(const int32_t *act, int32_t m, long long *ub, int32_t *stamp,
                               LazyCtl *lc, GridGainCtl *gg, bool fold, const float *score, int fill,
                               long long *akey = nullptr, int32_t *ast = nullptr, int32_t *wsel = nullptr,
                               long long *wgain = nullptr, int32_t *wpos = nullptr, int wcap = 0) {
  __shared__ long long s_v[32];
  __shared__ int s_id[32];
  __shared__ long long s_ll[32];
  __shared__ unsigned int s_hist[kLazyBins];
  __shared__ int s_bpos, s_blane;
  const int tid = threadIdx.x;
  const int T = blockDim.x;
  const int r = lc->round;

  if (fold) {  // the batch just evaluated: exact gains become the bounds
    const int ns = lc->n_sel;
    const int32_t *fsel = wcap ? wsel : lc->sel, *fpos = wcap ? wpos : lc->selpos;
    const long long *fgain = wcap ? wgain : lc->gsel;
    long long bv = -1;
    int bid = -1, mypos = -1, mylane = -1;
    for (int i = tid; i < ns; i += T) {
      const int v = fsel[i];
      const long long gv = fgain[i];
      ub[v] = gv;
      stamp[v] = r;
      const int p = akey ? fpos[i] : -1;
      if (akey) {
        akey[p] = gv;
        ast[p] = r;
      }
      if (better_max(gv, v, bv, bid)) {
        bv = gv;
        bid = v;
        mypos = p;
        mylane = i;
      }
    }
    const int mine = bid;
    block_argmax_all(bv, bid, s_v, s_id);
    if (mine >= 0 && mine == bid) {
      s_bpos = mypos;
      s_blane = mylane;
    }
    cta_sync();
    if (tid == 0) {
      // the batch's claim-log entries: [log_mark, log_n)
      const unsigned long long l1 = *(volatile unsigned long long *)&lc->log_n;
      if (bid >= 0 && better_max(bv, bid, lc->best_gain, lc->best_id)) {
        lc->best_gain = bv;
        lc->best_id = bid;
        lc->best_pos = s_bpos;
        lc->best_lane = wcap ? -1 : s_blane;  // wide steps keep no log
        lc->best_seg0 = lc->log_mark;
        lc->best_seg1 = l1;
      }
      lc->log_mark = l1;
      lc->steps += 1;
      lc->evals += ns;
    }
    cta_sync();
  }
  const long long gb = *(volatile long long *)&lc->best_gain;
  const int vb = *(volatile int32_t *)&lc->best_id;
  const long long theta = lc->theta;

  // best unevaluated bound, smallest bound, count
  long long umax = LLONG_MIN, umin = LLONG_MAX, cnt = 0;
  int vmax = -1;
  for (int i = tid; i < m; i += T) {
    const int v = act[i];
    const long long u = akey ? akey[i] : ub[v];
    if (u < 0 || (akey ? ast[i] : stamp[v]) == r) continue;
    if (better_max(u, v, umax, vmax)) {
      umax = u;
      vmax = v;
    }
    umin = min(umin, u);
    ++cnt;
  }
  if (akey && tid == 0) lc->sel_scanned += (unsigned long long)m;
  block_scan_stats(umax, vmax, umin, cnt);
  int dec;
  if (vb >= 0 && (cnt == 0 || better_max(gb, vb, umax, vmax))) dec = gb >= theta ? 1 : 2;
  else if (cnt == 0) dec = 2;
  else dec = 0;
  if (dec != 0) {
    if (tid == 0) lc->dec = dec;
    return;
  }
  // the largest bounds (all 64 lanes without a proposal; wcap in wide steps)
  const int need1 = wcap ? wcap : (score ? kLanes - fill : kLanes);
  auto by_bound = [=] __device__(int i, int v) -> long long {
    const long long u = akey ? akey[i] : ub[v];
    return (u >= 0 && (akey ? ast[i] : stamp[v]) != r) ? u : LLONG_MIN;
  };
  int32_t *selpos = akey ? lc->selpos : nullptr;
  unsigned long long *scanned = akey ? &lc->sel_scanned : nullptr;
  if (wcap) {
    const int taken = cta_topk(act, m, by_bound, umin, umax, cnt, need1, wsel, 0, s_hist, akey ? wpos : nullptr,
                               scanned, wcap);
    if (tid == 0) {
      lc->n_sel = taken < wcap ? taken : wcap;
      lc->dec = 0;
    }
    return;
  }
  int taken = cta_topk(act, m, by_bound, umin, umax, cnt, need1, lc->sel, 0, s_hist, selpos, scanned);
  if (score && taken < kLanes && cnt > taken) {
    // mark the bound picks as evaluated in this round (their fold does it again)
    if (tid < taken) {
      stamp[lc->sel[tid]] = r;
      if (akey) ast[lc->selpos[tid]] = r;
    }
    cta_sync();
    auto by_slack = [=] __device__(int i, int v) -> long long {
      const long long u = akey ? akey[i] : ub[v];
      if (u < 0 || (akey ? ast[i] : stamp[v]) == r) return LLONG_MIN;
      float p = expm1f(score[i]);
      p = p < 0.f ? 0.f : (p > (float)u ? (float)u : p);
      return u - (long long)p;
    };
    long long smin = LLONG_MAX, smax = LLONG_MIN, scnt = 0;
    for (int i = tid; i < m; i += T) {
      const long long k = by_slack(i, act[i]);
      if (k == LLONG_MIN) continue;
      smin = min(smin, k);
      smax = max(smax, k);
      ++scnt;
    }
    smin = block_min_ll(smin, s_ll);
    smax = block_max_ll(smax, s_ll);
    scnt = block_sum(scnt, s_ll);
    taken += cta_topk(act, m, by_slack, smin, smax, scnt, kLanes - taken, lc->sel, taken, s_hist, selpos,
                      scanned);
  }
  // a fresh grid-batch control block for the evaluation (grid form only)
  if (gg && tid < kLanes) {
    gg->gain[tid] = 0;
    gg->cnt[tid] = 0;
  }
  if (tid == 0) {
    lc->n_sel = taken < kLanes ? taken : kLanes;
    lc->dec = 0;
    if (gg) {
      gg->pk[0] = 0;
      gg->pk[1] = 0;
      gg->pk[2] = 0;
      gg->touched = 0;
    }
  }
}

// CTA 0's state in lean steps, in its shared memory: CTA 0 alone selects,
// runs level 0, reads the batch's gains and folds them, so it keeps the batch
// (ids, list positions, gains), the decision and the round's best here and
// publishes to LazyCtl only what the other CTAs read (dec, n_sel, best_*,
// log_mark).  Every read on CTA 0's path of a step is then a shared-memory
// read but one (the claim log's length).
struct Cta0State {
  int32_t sel[kLanes], selpos[kLanes];
  long long gout[kLanes];
  int nsel, dec, bid, bpos;
  long long bgain, theta;
  unsigned long long log_mark;
};

// One lean step of CTA 0 (list in shared memory: ids act, bounds akey, stamps
// ast, all at list positions; its sorted view): fold the batch just evaluated
// (exact gains become bounds, the round's best is updated), then decide --
// accept the best, ask for a longer list, or evaluate the head of the view --
// exactly as lazy_cta0_step does with its histogram selection.
static __device__ void lean_step(const int32_t *act, long long *ub, int32_t *stamp, LazyCtl *lc,
                                 GridGainCtl *gg, bool fold, int r, long long *akey, int32_t *ast,
                                 const SortedView &view, Cta0State &st) {
  __shared__ long long s_bv[2];
  __shared__ int s_bid[2], s_bpos[2], s_blane[2];
  const int tid = threadIdx.x, lane = tid & 31;
  if (fold) {
    const int ns = st.nsel;
    long long bv = -1;
    int bid = -1, bpos = -1, blane = -1;
    if (tid < ns) {
      const int v = st.sel[tid], p = st.selpos[tid];
      const long long gv = st.gout[tid];
      ub[v] = gv;
      stamp[v] = r;
      akey[p] = gv;
      ast[p] = r;
      bv = gv;
      bid = v;
      bpos = p;
      blane = tid;
    }
    if (tid < kLanes) {  // arg-best of the batch: warps 0 and 1, then thread 0
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oid = __shfl_xor_sync(0xffffffffu, bid, o);
        const int op = __shfl_xor_sync(0xffffffffu, bpos, o), ol = __shfl_xor_sync(0xffffffffu, blane, o);
        if (oid >= 0 && (bid < 0 || better_max(ov, oid, bv, bid))) {
          bv = ov;
          bid = oid;
          bpos = op;
          blane = ol;
        }
      }
      if (lane == 0) {
        s_bv[tid >> 5] = bv;
        s_bid[tid >> 5] = bid;
        s_bpos[tid >> 5] = bpos;
        s_blane[tid >> 5] = blane;
      }
    }
    cta_sync();
    if (tid == 0) {
      if (s_bid[1] >= 0 && (bid < 0 || better_max(s_bv[1], s_bid[1], bv, bid))) {
        bv = s_bv[1];
        bid = s_bid[1];
        bpos = s_bpos[1];
        blane = s_blane[1];
      }
      // the batch's claim-log entries: [log_mark, log_n)
      const unsigned long long l1 = *(volatile unsigned long long *)&lc->log_n;
      if (bid >= 0 && better_max(bv, bid, st.bgain, st.bid)) {
        st.bgain = bv;
        st.bid = bid;
        st.bpos = bpos;
        lc->best_gain = bv;
        lc->best_id = bid;
        lc->best_pos = bpos;
        lc->best_lane = blane;
        lc->best_seg0 = st.log_mark;
        lc->best_seg1 = l1;
      }
      st.log_mark = l1;
      lc->log_mark = l1;
      atomicAdd(reinterpret_cast<unsigned long long *>(&lc->steps), 1ull);
      atomicAdd(reinterpret_cast<unsigned long long *>(&lc->evals), (unsigned long long)ns);
    }
    sv_refold(akey, st.selpos, ns, view);
  }
  long long vmx;
  int vid;
  const int taken = sv_select(akey, act, ast, r, view, kLanes, st.sel, st.selpos, &vmx, &vid, &lc->sel_scanned);
  const long long gb = st.bgain;
  const int vb = st.bid;
  int dec;
  if (vb >= 0 && (taken == 0 || better_max(gb, vb, vmx, vid))) dec = gb >= st.theta ? 1 : 2;
  else if (taken == 0) dec = 2;
  else dec = 0;
  if (dec == 0 && tid < kLanes) {  // a fresh grid-batch control block
    gg->gain[tid] = 0;
    gg->cnt[tid] = 0;
  }
  if (tid == 0) {
    st.dec = dec;
    lc->dec = dec;
    if (dec == 0) {
      st.nsel = taken;
      lc->n_sel = taken;
      gg->pk[0] = 0;
      gg->pk[1] = 0;
      gg->pk[2] = 0;
      gg->touched = 0;
    }
  }
}

// One step of the lazy loop (Sec. 4.2) by every CTA of the grid: the lazy
// state lives in *lc, the list is act[0..m) (ids in increasing order), its
// bounds are akey/ast at list positions (compact copies) or ub/stamp by
// vertex (akey == nullptr).  CTA b owns the list slice [b P, b P + P).
//   1. fold: the gains of the last evaluated batch (sel/selpos/gsel, n_sel of
//      them) become bounds; each CTA applies those in its slice and every CTA
//      computes the round's best exact gain the same way;
//   2. scan: per-CTA (largest unevaluated bound, its id), smallest bound, count;
//   3. decision, taken identically by every CTA: accept the best (dec 1), ask
//      for a longer list (dec 2: no unevaluated entry, or the best is below
//      theta), or evaluate (dec 0);
//   4. threshold: histogram passes over [umin, umax] (1024 bins, summed over
//      CTAs in global memory) find the key of the need-th largest entry;
//   5. selection: entries above it and, in list order, enough equal to it.
// Returns false if a barrier gave up; *dec_out gets the decision.  The caller
// synchronises the grid before using the selection.
static __device__ bool grid_lazy_step(const int32_t *act, int32_t m, long long *ub, int32_t *stamp,
                                      long long *akey, int32_t *ast, LazyCtl *lc, GridGainCtl *gg, bool fold,
                                      int32_t *sel, int32_t *selpos, const long long *gsel, int cap,
                                      GridSelScratch *sc, GridBar *bar, int32_t *err, unsigned long long tns,
                                      int *dec_out) {
  __shared__ long long s_v[32];
  __shared__ int s_id[32];
  __shared__ long long s_ll[32];
  __shared__ unsigned int s_hist[kSelBins];
  __shared__ int s_scan[33];
  __shared__ int s_b, s_lane;
  __shared__ long long s_ab;
  const int tid = threadIdx.x, T = blockDim.x, G = gridDim.x, b = blockIdx.x;
  const int r = *(volatile int32_t *)&lc->round;
  const int P = (m + G - 1) / G;
  const int lo = min(m, b * P), hi = min(m, lo + P);
  auto key_of = [&](int i) -> long long {
    const int v = act[i];
    const long long u = akey ? akey[i] : ub[v];
    const int st = akey ? ast[i] : stamp[v];
    return (u >= 0 && st != r) ? u : LLONG_MIN;
  };

  // ---- 1. fold ----
  long long gb = *(volatile long long *)&lc->best_gain;
  int vb = *(volatile int32_t *)&lc->best_id;
  int bpos = *(volatile int32_t *)&lc->best_pos;
  if (fold) {
    const int ns = *(volatile int32_t *)&lc->n_sel;
    long long fv = -1;
    int fid = -1, fpos = -1, flane = -1;
    for (int j = tid; j < ns; j += T) {
      const int v = sel[j], p = selpos[j];
      const long long gv = gsel[j];
      if (p >= lo && p < hi) {  // this CTA's slice: the bound becomes exact
        ub[v] = gv;
        stamp[v] = r;
        if (akey) {
          akey[p] = gv;
          ast[p] = r;
        }
      }
      if (better_max(gv, v, fv, fid)) {
        fv = gv;
        fid = v;
        fpos = p;
        flane = j;
      }
    }
    const int mine = fid;
    block_argmax_all(fv, fid, s_v, s_id);
    if (mine >= 0 && mine == fid) {
      s_b = fpos;
      s_lane = flane;
    }
    cta_sync();
    bool improved = false;
    if (fid >= 0 && better_max(fv, fid, gb, vb)) {
      gb = fv;
      vb = fid;
      bpos = s_b;
      improved = true;
    }
    if (b == 0 && tid == 0) {
      // the batch's claim-log entries: [log_mark, log_n)
      const unsigned long long l1 = *(volatile unsigned long long *)&lc->log_n;
      if (improved) {
        lc->best_lane = s_lane;
        lc->best_seg0 = lc->log_mark;
        lc->best_seg1 = l1;
      }
      lc->log_mark = l1;
      lc->best_gain = gb;
      lc->best_id = vb;
      lc->best_pos = bpos;
      lc->steps += 1;
      lc->evals += ns;
    }
    cta_sync();
  }
  // ---- 2. scan of this CTA's slice ----
  long long umax = LLONG_MIN, umin = LLONG_MAX, cnt = 0;
  int vmax = -1;
  for (int i = lo + tid; i < hi; i += T) {
    const long long k = key_of(i);
    if (k == LLONG_MIN) continue;
    const int v = act[i];
    if (better_max(k, v, umax, vmax)) {
      umax = k;
      vmax = v;
    }
    umin = min(umin, k);
    ++cnt;
  }
  block_argmax_all(umax, vmax, s_v, s_id);
  umin = block_min_ll(umin, s_ll);
  cnt = block_sum(cnt, s_ll);
  if (tid == 0) {
    sc->umax[b] = umax;
    sc->vmax[b] = vmax;
    sc->umin[b] = umin;
    sc->cnt[b] = cnt;
  }
  if (!grid_sync(bar, err, tns)) return false;
  // ---- 3. decision (every CTA the same) ----
  umax = LLONG_MIN;
  vmax = -1;
  umin = LLONG_MAX;
  cnt = 0;
  for (int c = tid; c < G; c += T) {
    const long long u = ((volatile long long *)sc->umax)[c];
    const int v = ((volatile int32_t *)sc->vmax)[c];
    if (v >= 0 && better_max(u, v, umax, vmax)) {
      umax = u;
      vmax = v;
    }
    umin = min(umin, ((volatile long long *)sc->umin)[c]);
    cnt += ((volatile long long *)sc->cnt)[c];
  }
  block_argmax_all(umax, vmax, s_v, s_id);
  umin = block_min_ll(umin, s_ll);
  cnt = block_sum(cnt, s_ll);
  const long long theta = *(volatile long long *)&lc->theta;
  int dec;
  if (vb >= 0 && (cnt == 0 || better_max(gb, vb, umax, vmax))) dec = gb >= theta ? 1 : 2;
  else if (cnt == 0) dec = 2;
  else dec = 0;
  *dec_out = dec;
  if (dec != 0) {
    if (b == 0 && tid == 0) lc->dec = dec;
    return true;
  }
  // ---- 4. threshold: key of the need-th largest eligible entry ----
  const int need = (int)((long long)cap < cnt ? (long long)cap : cnt);
  long long tau = umin, above = 0;  // above = eligible keys > tau
  int last_hist = -1;
  if (cnt > need) {
    unsigned long long lo2 = (unsigned long long)umin, hi2 = (unsigned long long)umax;
    long long want = need, acc = 0;
    for (int pass = 0; pass < 8; ++pass) {
      const int hb = pass % 3;
      unsigned int *gh = sc->hist[hb];
      const unsigned long long span = hi2 - lo2 + 1ull;
      const unsigned long long width = span / kSelBins + ((span % kSelBins) ? 1ull : 0ull);
      for (int i = tid; i < kSelBins; i += T) s_hist[i] = 0;
      if (b == 0)  // the next pass's buffer (read two passes ago by everyone)
        for (int i = tid; i < kSelBins; i += T) sc->hist[(pass + 1) % 3][i] = 0;
      cta_sync();
      for (int i = lo + tid; i < hi; i += T) {
        const long long k = key_of(i);
        if (k == LLONG_MIN) continue;
        const unsigned long long uu = (unsigned long long)k;
        if (uu - lo2 > hi2 - lo2) continue;  // outside [lo2, hi2]
        atomicAdd(&s_hist[(uu - lo2) / width], 1u);
      }
      cta_sync();
      for (int i = tid; i < kSelBins; i += T)
        if (s_hist[i]) atomicAdd(&gh[i], s_hist[i]);
      if (!grid_sync(bar, err, tns)) return false;
      last_hist = hb;
      // walk down from the top bin: thread t owns bins 1023-2t and 1022-2t
      const int b0 = kSelBins - 1 - 2 * tid, b1 = b0 - 1;
      const int h0 = tid < kSelBins / 2 ? (int)((volatile unsigned int *)gh)[b0] : 0;
      const int h1 = tid < kSelBins / 2 ? (int)((volatile unsigned int *)gh)[b1] : 0;
      if (tid == 0) {
        s_b = 0;
        s_ab = 0;
      }
      int total;
      const long long a0 = block_excl_scan(h0 + h1, s_scan, &total);
      if (tid < kSelBins / 2) {
        if (a0 < want && a0 + h0 >= want) {
          s_b = b0;
          s_ab = a0;
        } else if (a0 + h0 < want && a0 + h0 + h1 >= want) {
          s_b = b1;
          s_ab = a0 + h0;
        }
      }
      cta_sync();
      const int bb = s_b;
      const long long ab = s_ab;
      cta_sync();
      const unsigned long long bin_lo = lo2 + width * (unsigned long long)bb;
      if (width == 1ull) {
        tau = (long long)bin_lo;
        above = acc + ab;
        break;
      }
      acc += ab;
      want -= ab;
      const unsigned long long room = hi2 - bin_lo;
      lo2 = bin_lo;
      hi2 = bin_lo + (width - 1ull < room ? width - 1ull : room);
    }
  }
  // ---- 5. selection: counts per slice, then positions in list order ----
  int n_gt = 0, n_eq = 0;
  for (int i = lo + tid; i < hi; i += T) {
    const long long k = key_of(i);
    if (k == LLONG_MIN) continue;
    n_gt += k > tau;
    n_eq += k == tau;
  }
  n_gt = (int)block_sum((long long)n_gt, s_ll);
  n_eq = (int)block_sum((long long)n_eq, s_ll);
  if (tid == 0) {
    sc->gt[b] = n_gt;
    sc->eq[b] = n_eq;
  }
  if (!grid_sync(bar, err, tns)) return false;
  if (b == 0 && last_hist >= 0)  // every histogram has been read: all three zero for the next step
    for (int i = tid; i < 3 * kSelBins; i += T) (&sc->hist[0][0])[i] = 0;
  long long gt_off = 0, eq_off = 0, gt_tot = 0;
  for (int c = tid; c < G; c += T) {
    const long long g1 = ((volatile int32_t *)sc->gt)[c], e1 = ((volatile int32_t *)sc->eq)[c];
    gt_tot += g1;
    if (c < b) {
      gt_off += g1;
      eq_off += e1;
    }
  }
  gt_off = block_sum(gt_off, s_ll);
  eq_off = block_sum(eq_off, s_ll);
  gt_tot = block_sum(gt_tot, s_ll);
  (void)above;
  const long long quota = (long long)need - gt_tot;  // entries equal to tau still to take, in list order
  int gt_seen = 0, eq_seen = 0;
  for (int base = lo; base < hi; base += T) {
    const int i = base + tid;
    int gt = 0, eq = 0;
    if (i < hi) {
      const long long k = key_of(i);
      if (k != LLONG_MIN) {
        gt = k > tau;
        eq = k == tau;
      }
    }
    int tg, te;
    const int rg = block_excl_scan(gt, s_scan, &tg);
    const int re = block_excl_scan(eq, s_scan, &te);
    long long pos = -1;
    if (gt) pos = gt_off + gt_seen + rg;
    else if (eq && eq_off + eq_seen + re < quota) pos = gt_tot + eq_off + eq_seen + re;
    if (pos >= 0 && pos < cap) {
      sel[pos] = act[i];
      selpos[pos] = i;
    }
    gt_seen += tg;
    eq_seen += te;
  }
  if (b == 0 && tid == 0) {
    lc->n_sel = need;
    lc->dec = 0;
    if (gg) {
      gg->pk[0] = 0;
      gg->pk[1] = 0;
      gg->pk[2] = 0;
      gg->touched = 0;
    }
  }
  if (b == 0 && gg && tid < kLanes) {
    gg->gain[tid] = 0;
    gg->cnt[tid] = 0;
  }
  return true;
}

// Proposal scores of the active list for this round (every CTA, one warp per
// candidate): score[i] = network output on the candidate's features.
static __device__ void lazy_score(const int32_t *act, int32_t m, const float *__restrict__ prop,
                           const int32_t *__restrict__ rp, const int32_t *dS,
                           const long long *ub, const int32_t *stamp,
                           const long long *__restrict__ two_hop, const int32_t *__restrict__ mx, int32_t round,
                           long long prev_gain, float *score) {
  __shared__ float sw[kMlpParams];
  __shared__ float sh[kGridGainThreads / 32][kMlpHidden];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) sw[i] = prop[i];
  cta_sync();
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = blockIdx.x * (blockDim.x >> 5) + wid, nw = gridDim.x * (blockDim.x >> 5);
  for (int i = gw; i < m; i += nw) {
    float f[kMlpIn];
    cand_features(act[i], rp, dS, ub, stamp, two_hop, mx, round, prev_gain, f);
    const float o = mlp_forward_warp(sw, f, sh[wid]);
    if (lane == 0) score[i] = o;
  }
  cta_sync();
}

}  // namespace gc
