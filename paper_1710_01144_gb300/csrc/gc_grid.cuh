// Device-side bodies of the grid-wide kernels (cooperative launches): the
// 64-lane pruned multi-source BFS for one batch (see gc_gain_grid.cu) and the
// relabel BFS that maintains d_S (see gc_bfs.cu).  Both synchronise through a
// caller-supplied bounded grid barrier, so they can run as phases of a larger
// persistent kernel (gc_lazy.cu).
// The adjacency (rp, ci, c3) and the neighbour bound mx are read through the
// read-only data path: callers never change them while a kernel that runs
// these functions can read them (inside a persistent kernel they are written
// before, in an earlier phase, and never after).  d_S and the lane words are
// read with ordinary loads: they change between phases.
#pragma once

#include "gc_device.cuh"
#include "gc_internal.cuh"

namespace gc {

typedef unsigned long long u64;

constexpr int kGridIlp = 2;  // adjacency entries in flight per thread (grid forms)

// Length of the row that vertex w scans when expanded at level lev: the whole
// row at level 0, the first c3[w] entries of a pruned row later.
static __device__ __forceinline__ int row_len(const int32_t *__restrict__ rp, const int32_t *__restrict__ c3, int w,
                                              int lev) {
  return (c3 && lev > 0) ? __ldg(c3 + w) : __ldg(rp + w + 1) - __ldg(rp + w);
}

// Largest x in [0, F) with start[x] <= e, for one warp; start is
// non-decreasing and start[0] <= e.  A 32-ary search: about log32(F) rounds
// of one coalesced probe each.
static __device__ __forceinline__ int warp_find_start(const int32_t *start, int F, long long e) {
  const int lane = threadIdx.x & 31;
  __syncwarp();  // callers reach it right after thread 0's bookkeeping: reconverge first
  int lo = 0, hi = F - 1;
  while (hi - lo >= 32) {
    const int step = (hi - lo + 32) / 32;  // 32 probes cover [lo, hi]
    const int idx = min(hi, lo + lane * step);
    const unsigned ok = __ballot_sync(0xffffffffu, (long long)start[idx] <= e);
    const int j = 31 - __clz(ok);  // ok holds lane 0 (start[lo] <= e)
    const int next = lo + (j + 1) * step;  // first probe past the answer, if any
    const int nlo = min(hi, lo + j * step);
    if (j < 31 && next <= hi) hi = next - 1;
    lo = nlo;
  }
  const int idx = lo + lane;
  const unsigned ok = __ballot_sync(0xffffffffu, idx <= hi && (long long)start[min(idx, hi)] <= e);
  return lo + 31 - __clz(ok);
}

// One batch of nl <= 64 candidates advanced by every CTA of the grid, with one
// grid barrier per BFS level.  ctl must hold zeros in pk, touched, gain and
// cnt on entry; the workspace's lane words must be zero and are zero again
// when the function returns (in every CTA).  gx holds 3n int32
// (entry offsets by level parity, a third frontier list).  Returns false if a
// barrier gave up (the error code is in *err / gctl->err).
//
// Claims work as in the CTA form (gc_cta.cuh): atomicOr on the visited word
// decides.  Claim words cycle through three per vertex (level L mod 3): level
// L reads word L, claims into word L+1, and clears word L-1 of the previous
// frontier, which nobody reads any more.  A vertex entering the next frontier
// takes its list slot and the start of its adjacency range in the level's
// edge space with one packed atomicAdd (count << 32 | degree), so the list is
// born sorted by range start: every CTA takes an equal slice of the level's
// adjacency entries right after the barrier, finds its first entry by one
// warp-wide search, stages the entries covering its slice in shared memory
// and expands them edge by edge.  A vertex with nothing left to claim (gain
// mode: every neighbour's d_S <= its level + 1) is counted but never queued.
// With c3 (pruned adjacency, see k_prune_count) rp/ci are the pruned rows and
// levels >= 1 scan only their first c3[u] entries.  With voff/ws_n (one graph
// of a block-diagonal union) the vertices are [voff, voff + ws_n): workspace 0
// and gx are laid out for ws_n vertices and indexed by w - voff.
// `phase` (gain mode only) splits off level 0, which one warp does: kBatchLevel0
// runs just that part in the calling CTA and returns without a barrier (a
// persistent kernel's selecting CTA does it right after choosing the batch);
// kBatchRest then runs the rest in every CTA, after a grid barrier the caller
// placed between the two.  kBatchAll does both with a barrier of its own.
// With `log` (gain mode), every claim that wins lanes at level L >= 1 appends
// {w, L, lanes won} at *log_n (one warp-aggregated slot per claim round); slots
// at or past log_cap are counted in *log_n but not written.
// With `acc`, each thread adds its work counts (scalar and union adjacency
// entries, frontier entries, pushes) to *acc instead of the batch summing them
// over the CTA and into gctl (a persistent caller sums them once at its end).
constexpr int kBatchAll = 0, kBatchLevel0 = 1, kBatchRest = 2;
struct GridCounts {
  u64 scalar = 0, uni = 0, front = 0, push = 0;
};
template <int MODE>
static __device__ __forceinline__ bool grid_gain_batch(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                int32_t n, const int32_t *dS, const int32_t *cand, int32_t nl_arg,
                                const int32_t *nl_dev, long long *out, unsigned char *ws_base, int32_t *gx,
                                int32_t *__restrict__ goff, GridGainCtl *ctl, GainCtl *gctl, GridBar *bar,
                                int32_t *err, unsigned long long timeout_ns, const int32_t *__restrict__ mx,
                                const int32_t *__restrict__ c3 = nullptr, int voff = 0, int ws_n = -1,
                                int phase = kBatchAll, ClaimRec *log = nullptr,
                                unsigned long long *log_n = nullptr, unsigned long long log_cap = 0,
                                GridCounts *acc = nullptr) {
  constexpr int T = kGridGainThreads;
  __shared__ u64 s_gain[kLanes];
  __shared__ unsigned int s_cnt[kLanes];
  __shared__ int s_go[T + 1];  // staged entries: start of each entry's range in the level's edge space
  __shared__ int s_rs[T];
  __shared__ u64 s_sm[T];
  __shared__ int s_x0;
  __shared__ u64 s_red[32];
  // farness mode: running per-lane distance sums and counts, the same in every
  // CTA (each adds the same per-level totals), so that every CTA takes the
  // same BFScut decisions
  __shared__ u64 s_tg[kLanes], s_tc[kLanes];
  (void)goff;

  const int tid = threadIdx.x, lane = tid & 31;
  const int G = gridDim.x, b = blockIdx.x;
  const int nl = nl_dev ? min(kLanes, *(volatile const int32_t *)nl_dev) : nl_arg;
  if (ws_n < 0) ws_n = n;
  const GainWs ws = gain_ws(ws_base, 0, ws_n, 0);
  // frontier lists by level mod 3 and range starts by level parity (selected,
  // not indexed, so that nothing lands in local memory)
  int32_t *const list2 = gx + 2 * (size_t)ws_n;
  auto list_of = [&](int r) -> int32_t * { return r == 0 ? ws.qv0 : (r == 1 ? ws.qv1 : list2); };
  auto starts_of = [&](int p) -> int32_t * { return p ? gx + (size_t)ws_n : gx; };
  auto words_of = [&](int r) -> LaneWords { return r == 0 ? ws.nx[0] : (r == 1 ? ws.nx[1] : ws.nx[2]); };
  u64 c_scalar = 0, c_union = 0, c_front = 0, c_push = 0;
  if (tid < kLanes) {
    s_gain[tid] = 0;
    s_cnt[tid] = 0;
  }
  u64 alive = nl >= kLanes ? ~0ull : ((1ull << nl) - 1ull);

  if (MODE != kModeGain) phase = kBatchAll;
  // ---- level 0 (warps 0 and 1 of CTA 0, or of the calling CTA): lanes reach
  // their candidates; thread j takes lane j.  Per warp three rounds of memory
  // traffic: the candidates' labels, bounds and rows; the visited and claim
  // words; the touched-list and frontier slots. ----
  if (phase != kBatchRest && (b == 0 || phase == kBatchLevel0) && tid < kLanes) {
    // the caller may arrive with the warp split by a single-thread branch: the
    // warp-synchronous code below needs it converged
    __syncwarp();
    const int j = tid;
    const int c = j < nl ? cand[j] : -1;
    const bool valid = j < nl && c >= 0 && c < n && c - voff >= 0 && c - voff < ws_n;
    if (j < nl && !valid) atomicExch(&ctl->err, GC_EINVAL);  // outside the graph
    int dc = 1, mxc = INT_MAX, deg = 0;
    if (valid) {
      if (MODE == kModeGain) dc = dS[c];
      if (MODE == kModeGain && mx) mxc = __ldg(mx + c);
      deg = row_len(rp, c3, c, 0);
    }
    const bool reach = valid && dc > 0;
    if (reach) {
      if (MODE == kModeGain) ctl->gain[j] = (u64)dc;
      else ctl->dcnt[0][j] = 1;
    }
    const u64 bit = 1ull << j;
    const bool expand = reach && (MODE != kModeGain || mxc > 1);
    const u64 ov = reach ? atomicOr(&ws.vis[c - voff], bit) : ~0ull;
    const u64 on = expand ? atomicOr(&ws.nx[0][c - voff], bit) : ~0ull;
    const bool fresh = ov == 0ull, q = on == 0ull;
    const unsigned fm = __ballot_sync(0xffffffffu, fresh), qm = __ballot_sync(0xffffffffu, q);
    if (!q) deg = 0;
    int incl = deg;  // inclusive prefix of the degrees over the queueing lanes
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int sum = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long bq = 0;
    int bf = 0;
    if (lane == 0) {
      if (qm) bq = atomicAdd(&ctl->pk[0], ((unsigned long long)__popc(qm) << 32) | (unsigned long long)sum);
      if (fm) bf = atomicAdd(&ctl->touched, __popc(fm));
    }
    const unsigned below = (1u << lane) - 1u;
    bq = __shfl_sync(0xffffffffu, bq, 0);
    bf = __shfl_sync(0xffffffffu, bf, 0);
    if (fresh) ws.touched[bf + __popc(fm & below)] = c;
    if (q) {
      const int slot = (int)(bq >> 32) + __popc(qm & below);
      list_of(0)[slot] = c;
      starts_of(0)[slot] = (int)(bq & 0xffffffffull) + incl - deg;
    }
    c_push += lane == 0 ? (u64)__popc(qm) : 0ull;
    if (phase == kBatchLevel0) {
      if (c_push) atomicAdd(&gctl->pushes, c_push);
      return true;
    }
  }
  if (phase == kBatchLevel0) return true;
  bool ok = true;
  if (phase == kBatchRest) cta_sync();  // s_gain and s_cnt are zero
  else ok = grid_sync(bar, err, timeout_ns);
  // invalid candidate ids leave their lanes empty
  if (ok && MODE == kModeFarness) {
    if (tid < kLanes) {
      s_tg[tid] = 0;
      s_tc[tid] = tid < nl ? ((volatile u64 *)ctl->dcnt[0])[tid] : 0ull;
    }
    cta_sync();
    for (int j = 0; j < nl; ++j)
      if (s_tc[j] == 0) alive &= ~(1ull << j);
  }

  int L = 0, F_prev = 0;
  for (; ok; ++L) {
    const unsigned long long pk = *(volatile unsigned long long *)&ctl->pk[L % 3];
    const int F = (int)(pk >> 32);
    const long long E = (long long)(pk & 0xffffffffull);
    // clear the claim words of the previous frontier (read by nobody now)
    if (L > 0) {
      const LaneWords prev = words_of((L + 2) % 3);
      const int32_t *pl = list_of((L + 2) % 3);
      for (int i = b * T + tid; i < F_prev; i += G * T) prev[pl[i] - voff] = 0;
    }
    if (F == 0) break;
    if (b == 0 && tid == 0) ctl->pk[(L + 2) % 3] = 0;  // the frontier after next (read two levels ago)
    if (MODE == kModeFarness && b == 0 && tid < kLanes) {
      // the totals of distance L + 2 (read by every CTA after the barrier of level L - 2)
      ctl->dgain[(L + 2) % 3][tid] = 0;
      ctl->dcnt[(L + 2) % 3][tid] = 0;
    }
    const int32_t *qcur_v = list_of(L % 3);
    const int32_t *qstart = starts_of(L & 1);
    const LaneWords cur = words_of(L % 3), nxt = words_of((L + 1) % 3);
    const int nlev = L + 1;
    const long long es = E * b / G, ee = E * (b + 1) / G;
    if (es < ee) {
      // the first entry whose range holds edge es: a warp-wide search, unless
      // one staging pass covers the whole frontier (then it starts at 0)
      if (F > T && tid < 32) {
        const int x = warp_find_start(qstart, F, es);
        if (tid == 0) s_x0 = x;
      }
      cta_sync();
      int x = F > T ? s_x0 : 0;
      while (x < F) {
        // stage up to T entries from x: range starts, row starts, lane masks
        const int xi = x + tid;
        const int cntx = min(T, F - x);
        if (xi < F) {
          const int u = qcur_v[xi];
          u64 m = cur[u - voff];
          if (MODE == kModeFarness) m &= alive;
          s_go[tid] = qstart[xi];
          s_sm[tid] = m;
          s_rs[tid] = __ldg(rp + u);
          if (s_go[tid] >= es && s_go[tid] < ee) {  // counted once: by the CTA holding the entry's first edge
            const int deg = (c3 && L > 0) ? __ldg(c3 + u) : __ldg(rp + u + 1) - s_rs[tid];
            c_union += (u64)deg;
            c_scalar += (u64)__popcll(m) * (u64)deg;
            c_front += 1;
          }
        }
        if (tid == 0) s_go[cntx] = (x + cntx < F) ? qstart[x + cntx] : (int)E;
        cta_sync();
        const long long a0 = max((long long)s_go[0], es), a1 = min((long long)s_go[cntx], ee);
        for (long long e0 = a0 + (long long)(tid & ~31) * kGridIlp; e0 < a1; e0 += (long long)T * kGridIlp) {
          // kGridIlp entries per thread: loads of all are issued before any claim
          int w[kGridIlp], sl[kGridIlp];
#pragma unroll
          for (int k = 0; k < kGridIlp; ++k) {
            const long long e = e0 + k * 32 + lane;
            w[k] = -1;
            sl[k] = 0;
            if (e < a1) {
              int l = 0, h = cntx - 1;  // staged entry holding e (every entry's range is non-empty)
              while (l < h) {
                const int mid = (l + h + 1) >> 1;
                if (s_go[mid] <= e) l = mid;
                else h = mid - 1;
              }
              sl[k] = l;
              w[k] = __ldg(ci + s_rs[l] + (int)(e - s_go[l]));
            }
          }
          // everything indexed by the neighbour is loaded at once: d_S, the
          // neighbour bound, the row length it would scan next level and its
          // visited word (from L2: it holds every lane that reached w before
          // this level)
          int dw[kGridIlp], mxw[kGridIlp], lw[kGridIlp];
          u64 vp[kGridIlp];
#pragma unroll
          for (int k = 0; k < kGridIlp; ++k) {
            const bool ok = w[k] >= 0;
            dw[k] = (MODE == kModeGain && ok) ? dS[w[k]] : 0;
            mxw[k] = (MODE == kModeGain && mx && ok) ? __ldg(mx + w[k]) : INT_MAX;
            lw[k] = ok ? row_len(rp, c3, w[k], nlev) : 0;
            vp[k] = ok ? __ldcg(&ws.vis[w[k] - voff]) : 0ull;
          }
          u64 nb[kGridIlp];
#pragma unroll
          for (int k = 0; k < kGridIlp; ++k) {
            // pruned unless w is strictly closer to the lane's candidate than
            // to S; lanes that reached w at an earlier level are left out
            const bool live = w[k] >= 0 && (MODE != kModeGain || dw[k] > nlev);
            nb[k] = live ? (s_sm[sl[k]] & ~vp[k]) : 0ull;
          }
          // Both claims at once.  The visited word decides which lanes this
          // thread wins (its gains) and whether w is new to the batch.  The
          // claim word of level nlev receives all of nb: every bit of it is a
          // lane that reaches w at this level (won here or by a concurrent
          // claim), and the thread that finds the word empty queues w.  w is
          // expanded at level nlev only if some neighbour may still be claimed.
          u64 ov[kGridIlp], on[kGridIlp];
#pragma unroll
          for (int k = 0; k < kGridIlp; ++k) {
            ov[k] = nb[k] ? atomicOr(&ws.vis[w[k] - voff], nb[k]) : ~0ull;
            on[k] = (nb[k] && mxw[k] > nlev + 1) ? atomicOr(&nxt[w[k] - voff], nb[k]) : ~0ull;
          }
#pragma unroll
          for (int k = 0; k < kGridIlp; ++k) {
            u64 won = nb[k] & ~ov[k];
            const bool fresh = won && ov[k] == 0;
            const bool q = on[k] == 0ull;
            // the warp's appends -- next frontier (slot and range start),
            // touched list, claim log -- take their slots by atomics that lane
            // 0 issues together, so that their round trips overlap
            const unsigned qm = __ballot_sync(0xffffffffu, q), fm = __ballot_sync(0xffffffffu, fresh);
            const unsigned lm = (MODE == kModeGain && log) ? __ballot_sync(0xffffffffu, won != 0ull) : 0u;
            const int deg = q ? lw[k] : 0;
            int incl = deg;  // inclusive prefix of the degrees over the queueing lanes
            if (qm) {
#pragma unroll
              for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += y;
              }
            }
            const int sum = __shfl_sync(0xffffffffu, incl, 31);
            unsigned long long bq = 0, bl = 0;
            int bf = 0;
            if (lane == 0) {
              if (qm) bq = atomicAdd(&ctl->pk[nlev % 3], ((unsigned long long)__popc(qm) << 32) | (unsigned long long)sum);
              if (fm) bf = atomicAdd(&ctl->touched, __popc(fm));
              if (lm) bl = atomicAdd(log_n, (unsigned long long)__popc(lm));
              c_push += (u64)__popc(qm);
            }
            const unsigned below = (1u << lane) - 1u;
            if (qm) {
              bq = __shfl_sync(0xffffffffu, bq, 0);
              if (q) {
                const int slot = (int)(bq >> 32) + __popc(qm & below);
                list_of(nlev % 3)[slot] = w[k];
                starts_of(nlev & 1)[slot] = (int)(bq & 0xffffffffull) + incl - deg;
              }
            }
            if (fm) {
              bf = __shfl_sync(0xffffffffu, bf, 0);
              if (fresh) ws.touched[bf + __popc(fm & below)] = w[k];
            }
            if (lm) {
              bl = __shfl_sync(0xffffffffu, bl, 0) + (unsigned long long)__popc(lm & below);
              if (won && bl < log_cap)
                *reinterpret_cast<int4 *>(log + bl) =
                    make_int4(w[k], nlev, (int)(unsigned)won, (int)(unsigned)(won >> 32));
            }
            // per-lane sums: claims that won one lane (the common case: a
            // row's entries all carry the lane of the vertex being expanded)
            // are summed over the threads of the warp that won the same lane,
            // and one thread adds the sum; claims of several lanes add each
            const u64 wt = MODE == kModeGain ? (u64)(dw[k] - nlev) : (u64)nlev;
            const bool one = won != 0ull && (won & (won - 1ull)) == 0ull;
            const int j1 = one ? __ffsll((long long)won) - 1 : -1;  // (the -1 group adds nothing here)
            const unsigned grp = __match_any_sync(0xffffffffu, j1);
            if (one) {
              // wt < 2^31: two 16-bit halves keep the 32-lane sums exact
              const unsigned lo = __reduce_add_sync(grp, (unsigned)(wt & 0xffffu));
              const unsigned hi = __reduce_add_sync(grp, (unsigned)(wt >> 16));
              if (lane == __ffs(grp) - 1) {
                atomicAdd(&s_gain[j1], (u64)lo + ((u64)hi << 16));
                if (MODE == kModeFarness) atomicAdd(&s_cnt[j1], (unsigned)__popc(grp));
              }
            } else if (won) {
              do {
                const int j = __ffsll((long long)won) - 1;
                won &= won - 1;
                atomicAdd(&s_gain[j], wt);
                if (MODE == kModeFarness) atomicAdd(&s_cnt[j], 1u);
              } while (won);
            }
          }
        }
        const int done_end = s_go[cntx];
        cta_sync();  // the staged arrays are reused
        if ((long long)done_end >= ee) break;
        x += cntx;
      }
    }
    if (MODE == kModeFarness) {
      cta_sync();
      if (tid < kLanes) {  // the vertices claimed at distance L + 1
        if (s_gain[tid]) atomicAdd(&ctl->dgain[(L + 1) % 3][tid], s_gain[tid]);
        if (s_cnt[tid]) atomicAdd(&ctl->dcnt[(L + 1) % 3][tid], (u64)s_cnt[tid]);
        s_gain[tid] = 0;
        s_cnt[tid] = 0;
      }
    }
    F_prev = F;
    ok = grid_sync(bar, err, timeout_ns);
    if (!ok) break;
    if (MODE == kModeFarness) {
      // the same BFScut test in every CTA: all vertices within L+1 are
      // counted, the rest are at least L+2 away
      // (the running totals come from the per-distance buffers, which no CTA
      // changes until the next barrier: the cumulative sums would already be
      // growing with the next level in faster CTAs)
      const int Fn = (int)(*(volatile unsigned long long *)&ctl->pk[(L + 1) % 3] >> 32);
      const long long best = *(volatile long long *)&gctl->best_f;
      if (tid < nl) {
        s_tg[tid] += ((volatile u64 *)ctl->dgain[(L + 1) % 3])[tid];
        s_tc[tid] += ((volatile u64 *)ctl->dcnt[(L + 1) % 3])[tid];
      }
      cta_sync();
      for (int j = 0; j < nl; ++j) {
        if (!((alive >> j) & 1ull)) continue;
        const long long s = (long long)s_tg[j];
        const long long c = (long long)s_tc[j];
        if (Fn > 0 && s + (long long)(L + 2) * ((long long)n - c) > best) alive &= ~(1ull << j);
      }
      if (alive == 0) {
        // every lane is cut: clear the claim words of this frontier and of the
        // next one, which is not expanded
        const LaneWords lw0 = cur, lw1 = nxt;
        const int32_t *l0 = list_of(L % 3), *l1 = list_of((L + 1) % 3);
        for (int i = b * T + tid; i < F; i += G * T) lw0[l0[i] - voff] = 0;
        for (int i = b * T + tid; i < Fn; i += G * T) lw1[l1[i] - voff] = 0;
        F_prev = 0;
        ++L;
        break;
      }
    }
  }
  // L = levels expanded
  // ---- results ----
  if (MODE == kModeGain) {
    cta_sync();
    if (tid < kLanes && s_gain[tid]) atomicAdd(&ctl->gain[tid], s_gain[tid]);
  }
  // leave the workspace zero: the touched list is complete once the last
  // level's barrier has passed, and the barrier below publishes the clearing
  {
    const int nt = *(volatile int32_t *)&ctl->touched;
    for (int i = b * T + tid; i < nt; i += G * T) ws.vis[ws.touched[i] - voff] = 0;
  }
  if (acc) {
    acc->scalar += c_scalar;
    acc->uni += c_union;
    acc->front += c_front;
    acc->push += c_push;
  } else {
    c_scalar = block_sum(c_scalar, s_red);
    c_union = block_sum(c_union, s_red);
    c_front = block_sum(c_front, s_red);
    c_push = block_sum(c_push, s_red);
  }
  if (tid == 0) {
    if (!acc) {
      atomicAdd(&gctl->edges_scalar, c_scalar);
      atomicAdd(&gctl->edges_union, c_union);
      atomicAdd(&gctl->frontier, c_front);
      atomicAdd(&gctl->pushes, c_push);
    }
    if (b == 0) {
      atomicAdd(&gctl->levels, (u64)L);
      atomicAdd(&gctl->batches, 1ull);
      atomicAdd(&gctl->lanes, (u64)nl);
    }
  }
  const bool ok2 = grid_sync(bar, err, timeout_ns);
  if (b == 0 && tid < nl) {
    const int c = cand[tid];
    long long r;
    if (!ok2 || c < 0 || c >= n) {
      r = -1;
    } else if (MODE == kModeGain) {
      r = (long long)((volatile u64 *)ctl->gain)[tid];
    } else if (!((alive >> tid) & 1ull)) {
      r = -1;
    } else if ((long long)s_tc[tid] != n) {
      r = -1;
      gctl->short_vertex = c;
      gctl->short_count = (long long)s_tc[tid];
      atomicExch(&gctl->err, GC_EDISCONNECTED);
    } else {
      r = (long long)s_tg[tid];
      if (!gctl->fixed_best) atomicMin(&gctl->best_f, r);
    }
    out[tid] = r;
  }
  if (!ok2 && b == 0 && tid == 0) atomicExch(&gctl->err, GC_ETIMEOUT);
  return ok2;
}

// Relabel BFS over the whole grid: dist[w] <- min(dist[w], level) from the
// seeds, expanding only where the label decreased (the pruned SSSP of Sec. 4.1
// when dist holds d_S).  pk[0..2] must be zero on entry (the frontier of level
// L by L mod 3: entries << 32 | adjacency entries).  *decrease collects
// sum(old - new) over relabelled vertices with a finite old label.
// One grid barrier per level, as in grid_gain_batch: a relabelled vertex takes
// its slot in the next list and the start of its adjacency range with one
// packed atomicAdd, so every CTA takes an equal slice of the level's adjacency
// entries right away (a hub row is shared by all CTAs instead of serialising
// one warp).  q0/q1 are the lists and st0/st1 the range starts by level
// parity, n entries each.  With `work` given, CTA 0 adds the frontier entries
// and adjacency entries of every level to work[0], work[1].  With c3 (pruned
// adjacency, valid when dist holds d_S) levels >= 1 scan only the first c3[u]
// entries of the pruned rows rp/ci.
static __device__ __forceinline__ bool grid_relabel_bfs(
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n, int32_t *dist,
    const int32_t *seeds, int32_t n_seeds, int32_t *q0, int32_t *q1, unsigned long long *pk, int32_t *levels_out,
    unsigned long long *decrease, unsigned long long *relabelled, int32_t *st0, int32_t *st1,
    GridBar *bar, int32_t *err, unsigned long long timeout_ns, unsigned long long *work = nullptr,
    const int32_t *__restrict__ c3 = nullptr) {
  constexpr int kT = 1024;  // staging capacity (blockDim.x <= 1024)
  __shared__ unsigned long long sh_bfs[32];
  __shared__ int s_go[kT + 1];
  __shared__ int s_rs[kT];
  __shared__ int s_x0;
  const int tid = threadIdx.x, lane = tid & 31, T = blockDim.x;
  const int G = gridDim.x, b = blockIdx.x;
  unsigned long long dec = 0, rel = 0;

  // queue w for level lev: warp-aggregated slot and range start (whole warp)
  auto enqueue = [&](bool q, int w, int lev, int deg) {
    const unsigned qm = __ballot_sync(0xffffffffu, q);
    if (!qm) return;
    if (!q) deg = 0;
    int incl = deg;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    const int sum = __shfl_sync(0xffffffffu, incl, 31);
    const int leader = __ffs(qm) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(&pk[lev % 3], ((unsigned long long)__popc(qm) << 32) | (unsigned long long)sum);
    base = __shfl_sync(0xffffffffu, base, leader);
    if (q) {
      const int slot = (int)(base >> 32) + __popc(qm & ((1u << lane) - 1u));
      ((lev & 1) ? q1 : q0)[slot] = w;
      ((lev & 1) ? st1 : st0)[slot] = (int)(base & 0xffffffffull) + incl - deg;
    }
  };

  for (int base = b * T; base < n_seeds; base += G * T) {  // warp-uniform trip count
    const int i = base + tid;
    bool q = false;
    int s = 0;
    if (i < n_seeds) {
      s = ((volatile const int32_t *)seeds)[i];
      if (s < 0 || s >= n) {
        atomicExch(err, GC_EINVAL);
      } else {
        const int old = atomicMin(&dist[s], 0);
        if (old > 0) {
          q = true;
          if (old < kInf) dec += (unsigned long long)old;
          ++rel;
        }
      }
    }
    enqueue(q, s, 0, q ? row_len(rp, c3, s, 0) : 0);
  }
  bool ok = grid_sync(bar, err, timeout_ns);
  for (int L = 0; ok; ++L) {
    const unsigned long long pkl = *(volatile unsigned long long *)&pk[L % 3];
    const int F = (int)(pkl >> 32);
    const long long E = (long long)(pkl & 0xffffffffull);
    if (F == 0) break;
    if (b == 0 && tid == 0) pk[(L + 2) % 3] = 0;  // the frontier after next (read two levels ago)
    if (work && b == 0 && tid == 0) {
      work[0] += (unsigned long long)F;
      work[1] += (unsigned long long)E;
    }
    const int32_t *qc = (L & 1) ? q1 : q0;
    const int32_t *qs = (L & 1) ? st1 : st0;
    const int nl = L + 1;
    const long long es = E * b / G, ee = E * (b + 1) / G;
    if (es < ee) {
      if (tid < 32) {
        const int x = warp_find_start(qs, F, es);
        if (tid == 0) s_x0 = x;
      }
      cta_sync();
      int x = s_x0;
      while (x < F) {
        const int xi = x + tid;
        const int cntx = min(T, F - x);
        if (xi < F) {
          s_go[tid] = qs[xi];
          s_rs[tid] = __ldg(rp + qc[xi]);
        }
        if (tid == 0) s_go[cntx] = (x + cntx < F) ? qs[x + cntx] : (int)E;
        cta_sync();
        const long long a0 = max((long long)s_go[0], es), a1 = min((long long)s_go[cntx], ee);
        for (long long e0 = a0 + (tid & ~31); e0 < a1; e0 += T) {  // warp-uniform trip count
          const long long e = e0 + lane;
          bool q = false;
          int w = 0, lw = 0;
          if (e < a1) {
            int l = 0, h = cntx - 1;  // staged entry holding e (every entry's range is non-empty)
            while (l < h) {
              const int mid = (l + h + 1) >> 1;
              if (s_go[mid] <= e) l = mid;
              else h = mid - 1;
            }
            w = __ldg(ci + s_rs[l] + (int)(e - s_go[l]));
            const int dcur = dist[w];
            lw = row_len(rp, c3, w, nl);  // with the label: no load waits in enqueue
            if (nl < dcur) {
              const int old = atomicMin(&dist[w], nl);
              if (old > nl) {
                q = true;
                if (old < kInf) dec += (unsigned long long)(old - nl);
                ++rel;
              }
            }
          }
          enqueue(q, w, nl, lw);
        }
        const int done_end = s_go[cntx];
        cta_sync();  // the staged arrays are reused
        if ((long long)done_end >= ee) break;
        x += cntx;
      }
    }
    ok = grid_sync(bar, err, timeout_ns);
    if (ok && b == 0 && tid == 0 && levels_out) *levels_out = L + 1;
  }
  dec = block_sum(dec, sh_bfs);
  rel = block_sum(rel, sh_bfs);
  if (tid == 0) {
    if (dec) atomicAdd(decrease, dec);
    if (rel && relabelled) atomicAdd(relabelled, rel);
  }
  return ok;
}

}  // namespace gc
