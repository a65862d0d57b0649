// The CTA-per-batch form of the 64-lane pruned multi-source BFS (see
// gc_gain.cu for the method and layout), as a device function so that the
// batched multi-graph solver can run it inside a persistent kernel.
#pragma once

#include "gc_device.cuh"
#include "gc_internal.cuh"

namespace gc {

typedef unsigned long long u64;

struct GainCounters {
  u64 scalar = 0, uni = 0, levels = 0, batches = 0, front = 0, push = 0, lanes = 0;
};

// One batch of nl <= 64 candidates (cand[0..nl)) by the whole CTA, results to
// out[0..nl).  The workspace's lane words are zero on entry and on exit.
//
// Lane words of vertex w: vis (every lane that has reached w) and the claims
// of the current and the next level, nx[L & 1] and nx[(L + 1) & 1].  A lane
// claims w at level L + 1 by setting its bit in vis with atomicOr: the bit
// was clear exactly for the lanes that reach w first here, and those lanes
// are then recorded in nx[(L + 1) & 1][w].  Level L + 1 expands w with the
// lanes of that word, which the expanding thread reads and clears; so no
// separate commit pass is needed between levels.
//
// With c3 (the pruned adjacency, see k_prune_count), rp/ci are the pruned
// rows: level 0 scans a whole row, later levels only its first c3[u] entries.
//
// RO_GRAPH / RO_DS: read rp, ci, c3, mx / dS through the read-only data path.
// Only for data that no thread changes while the calling kernel can still
// read it through that path (inside a persistent kernel: written before and
// never after); it lets the column, d_S and bound loads of independent
// adjacency entries overlap freely, three times faster on hub-heavy batches.
template <int MODE, bool RO_GRAPH = true, bool RO_DS = true>
__device__ __forceinline__ void cta_gain_batch(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                               int32_t n, const int32_t *dS,
                                               const int32_t *cand, int nl,
                                               long long *__restrict__ out, const GainWs &ws, GainCtl *ctl,
                                               const int32_t *__restrict__ mx, const LaneGraphs lg,
                                               GainCounters &cnt, int voff = 0,
                                               const int32_t *__restrict__ c3 = nullptr) {
  constexpr int T = kGainThreads;
  __shared__ u64 s_gain[kLanes];
  __shared__ int s_cnt[kLanes];
  __shared__ int s_cand[kLanes];
  __shared__ int s_nlane[kLanes];
  __shared__ long long s_best[kLanes];
  __shared__ int s_off[T + 1];
  __shared__ int s_rs[T];
  __shared__ u64 s_m[T];
  __shared__ int s_scan[33];
  __shared__ int s_qn, s_touched;
  __shared__ u64 s_alive;

  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < kLanes) {
    s_gain[tid] = 0;
    s_cnt[tid] = 0;
    const int c = tid < nl ? cand[tid] : -1;
    s_cand[tid] = c;
    if (MODE == kModeFarness) {
      const int g = (lg.gid && c >= 0 && c < n) ? lg.gid[c] : -1;
      s_nlane[tid] = g >= 0 ? lg.ng[g] : n;
      s_best[tid] = g >= 0 ? *(volatile long long *)&lg.best_f[g] : 0;
    }
  }
  if (tid == 0) {
    s_qn = 0;
    s_touched = 0;
    s_alive = nl >= kLanes ? ~0ull : ((1ull << nl) - 1ull);
  }
  cta_sync();
  int32_t *qcur_v = ws.qv0, *qnxt_v = ws.qv1;

  // level 0: lane j reaches its candidate
  if (tid < nl) {
    const int c = s_cand[tid];
    const u64 bit = 1ull << tid;
    bool reach = false;
    if (c < 0 || c >= n) {
      s_cand[tid] = -2;  // invalid id
      atomicAnd(&s_alive, ~bit);
    } else if (MODE == kModeGain) {
      const int dc = ld_ro<RO_DS>(dS + c);
      if (dc > 0) {  // v not in S: it contributes d_S[v] - 0 and expands
        s_gain[tid] = (u64)dc;
        reach = true;
      }
    } else {
      s_cnt[tid] = 1;
      reach = true;
    }
    if (reach) {
      const u64 ov = atomicOr(&ws.vis[c - voff], bit);
      if (ov == 0) ws.touched[atomicAdd(&s_touched, 1)] = c;
      const u64 on = atomicOr(&ws.nx[0][c - voff], bit);
      if (on == 0) qcur_v[atomicAdd(&s_qn, 1)] = c;
    }
  }
  cta_sync();
  int F = s_qn;
  cta_sync();
  if (tid == 0) s_qn = 0;
  cta_sync();

  int L = 0;
  for (; F > 0; ++L) {
    const int nlev = L + 1;
    // (selected, not indexed: a dynamic index would put ws in local memory)
    const LaneWords cur = (L & 1) ? ws.nx[1] : ws.nx[0], nxt = (L & 1) ? ws.nx[0] : ws.nx[1];
    // ---- expand level L into level L+1 ----
    for (int chunk = 0; chunk < F; chunk += T) {
      const int i = chunk + tid;
      int deg = 0, rs = 0;
      u64 m = 0;
      if (i < F) {
        const int u = qcur_v[i];
        // the lanes that reached u at level L; the word is free for level L+2
        m = cur[u - voff];
        cur[u - voff] = 0;
        if (MODE == kModeFarness) m &= s_alive;
        const int r0 = ld_ro<RO_GRAPH>(rp + u);
        const int r1 = (c3 && L > 0) ? r0 + ld_ro<RO_GRAPH>(c3 + u) : ld_ro<RO_GRAPH>(rp + u + 1);
        // no neighbour of u can still be claimed: skip the scan
        if (MODE == kModeGain && mx && ld_ro<RO_GRAPH>(mx + u) <= nlev) m = 0;
        if (m) {
          rs = r0;
          deg = r1 - r0;
        }
        cnt.uni += (u64)deg;
        cnt.scalar += (u64)__popcll(m) * (u64)deg;
        cnt.front += (m != 0);
      }
      int total;
      const int off = block_excl_scan(deg, s_scan, &total);
      s_off[tid] = off;
      s_rs[tid] = rs;
      s_m[tid] = m;
      if (tid == T - 1) s_off[T] = total;
      cta_sync();
      // kEdgeIlp adjacency entries per thread are in flight at once: the
      // column, d_S, visited-word loads and the claiming atomics of
      // independent entries are issued before any result is used.
      // (the trip count is the same for the 32 threads of a warp: the
      // warp-wide sums and appends below need them converged)
      for (int e0 = tid; e0 - (tid & 31) < total; e0 += kEdgeIlp * T) {
        int w[kEdgeIlp], sl[kEdgeIlp];
#pragma unroll
        for (int k = 0; k < kEdgeIlp; ++k) {
          const int e = e0 + k * T;
          w[k] = -1;
          sl[k] = 0;
          if (e < total) {
            int lo = 0, hi = T - 1;  // largest j with s_off[j] <= e (its row is non-empty)
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (s_off[mid] <= e) lo = mid;
              else hi = mid - 1;
            }
            sl[k] = lo;
            w[k] = ld_ro<RO_GRAPH>(ci + s_rs[lo] + (e - s_off[lo]));
          }
        }
        int dw[kEdgeIlp];
#pragma unroll
        for (int k = 0; k < kEdgeIlp; ++k) dw[k] = (MODE == kModeGain && w[k] >= 0) ? ld_ro<RO_DS>(dS + w[k]) : 0;
        u64 nb[kEdgeIlp];
#pragma unroll
        for (int k = 0; k < kEdgeIlp; ++k) {
          // pruned unless w is strictly closer to the lane's candidate than to S
          const bool live = w[k] >= 0 && (MODE != kModeGain || dw[k] > nlev);
          nb[k] = live ? (s_m[sl[k]] & ~ws.vis[w[k] - voff]) : 0ull;
        }
        u64 ov[kEdgeIlp];
#pragma unroll
        for (int k = 0; k < kEdgeIlp; ++k) ov[k] = nb[k] ? atomicOr(&ws.vis[w[k] - voff], nb[k]) : ~0ull;
        u64 on[kEdgeIlp];
#pragma unroll
        for (int k = 0; k < kEdgeIlp; ++k) {
          const u64 won = nb[k] & ~ov[k];
          on[k] = won ? atomicOr(&nxt[w[k] - voff], won) : ~0ull;
        }
#pragma unroll
        for (int k = 0; k < kEdgeIlp; ++k) {
          u64 won = nb[k] & ~ov[k];
          // touched list and next frontier: one shared-memory slot reservation
          // per warp for each
          const bool fresh = won && ov[k] == 0, q = won && on[k] == 0;
          const unsigned fm = __ballot_sync(0xffffffffu, fresh), qm = __ballot_sync(0xffffffffu, q);
          int bt = 0, bq = 0;
          if (lane == 0) {
            if (fm) bt = atomicAdd(&s_touched, __popc(fm));
            if (qm) bq = atomicAdd(&s_qn, __popc(qm));
          }
          const unsigned below = (1u << lane) - 1u;
          bt = __shfl_sync(0xffffffffu, bt, 0);
          bq = __shfl_sync(0xffffffffu, bq, 0);
          if (fresh) ws.touched[bt + __popc(fm & below)] = w[k];
          if (q) {
            qnxt_v[bq + __popc(qm & below)] = w[k];
            ++cnt.push;
          }
          // per-lane sums: a claim of one lane (the common case: a row's
          // entries carry the lane of the vertex being expanded) is summed over
          // the warp's threads that won the same lane, one thread adds the sum
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
              if (MODE == kModeFarness) atomicAdd(&s_cnt[j1], __popc(grp));
            }
          } else if (won) {
            do {
              const int j = __ffsll((long long)won) - 1;
              won &= won - 1;
              atomicAdd(&s_gain[j], wt);
              if (MODE == kModeFarness) atomicAdd(&s_cnt[j], 1);
            } while (won);
          }
        }
      }
      cta_sync();
    }
    const int Fn = s_qn;
    if (MODE == kModeFarness && tid < kLanes && ((s_alive >> tid) & 1ull)) {
      // every vertex within distance L+1 is counted; the rest are >= L+2 away
      const long long lb = (long long)s_gain[tid] + (long long)(L + 2) * (long long)(s_nlane[tid] - s_cnt[tid]);
      const long long best = lg.gid ? s_best[tid] : *(volatile long long *)&ctl->best_f;
      if (Fn > 0 && lb > best) atomicAnd(&s_alive, ~(1ull << tid));
    }
    cta_sync();
    if (tid == 0) s_qn = 0;
    { int32_t *t = qcur_v; qcur_v = qnxt_v; qnxt_v = t; }
    F = Fn;
    cta_sync();
    if (MODE == kModeFarness && s_alive == 0) {
      // every lane is cut: clear the claims of the frontier that is not expanded
      for (int i = tid; i < F; i += T) nxt[qcur_v[i] - voff] = 0;
      break;
    }
  }
  cnt.levels += (u64)L;
  ++cnt.batches;
  cnt.lanes += (u64)nl;

  if (tid < nl) {
    const int c = s_cand[tid];
    long long r;
    if (c == -2) {
      r = -1;
      atomicExch(&ctl->err, GC_EINVAL);
    } else if (MODE == kModeGain) {
      r = (long long)s_gain[tid];
    } else if (!((s_alive >> tid) & 1ull)) {
      r = -1;  // cut: cannot beat the best farness
    } else if (s_cnt[tid] != s_nlane[tid]) {
      r = -1;
      ctl->short_vertex = c;
      ctl->short_count = s_cnt[tid];
      atomicExch(&ctl->err, GC_EDISCONNECTED);
    } else {
      r = (long long)s_gain[tid];
      if (lg.gid) atomicMin(&lg.best_f[lg.gid[c]], r);
      else if (!ctl->fixed_best) atomicMin(&ctl->best_f, r);
    }
    out[tid] = r;
  }
  const int nt = s_touched;
  for (int i = tid; i < nt; i += T) ws.vis[ws.touched[i] - voff] = 0;
  cta_sync();
}

// CTA-local pruned relabel BFS from seed s (the pruned SSSP of Sec. 4.1 that
// turns d_S into min(d_S, d(s, .))): only vertices whose label improves are
// relabelled and expanded.  q0/q1 are queues of at least the component's size.
// Returns the farness decrease sum(old - new) (every thread gets it).
static __device__ __noinline__ long long cta_relabel_bfs(const int32_t *__restrict__ rp,
                                                        const int32_t *__restrict__ ci, int32_t *dist, int s,
                                                        int32_t *q0, int32_t *q1) {
  constexpr int T = kGainThreads;
  __shared__ int s_off[T + 1];
  __shared__ int s_rs[T];
  __shared__ int s_scan[33];
  __shared__ int s_qn, s_F;
  __shared__ long long s_red[32];
  const int tid = threadIdx.x;
  long long dec = 0;
  if (tid == 0) {
    s_qn = 0;
    s_F = 0;
    const int old = dist[s];
    if (old > 0) {
      dec = old;
      dist[s] = 0;
      q0[0] = s;
      s_F = 1;
    }
  }
  cta_sync();
  int32_t *qc = q0, *qn = q1;
  for (int L = 0; s_F > 0; ++L) {
    const int F = s_F;
    const int nl = L + 1;
    for (int chunk = 0; chunk < F; chunk += T) {
      const int i = chunk + tid;
      int deg = 0, rs = 0;
      if (i < F) {
        const int u = qc[i];
        rs = rp[u];
        deg = rp[u + 1] - rs;
      }
      int total;
      const int off = block_excl_scan(deg, s_scan, &total);
      s_off[tid] = off;
      s_rs[tid] = rs;
      if (tid == T - 1) s_off[T] = total;
      cta_sync();
      for (int e = tid; e < total; e += T) {
        int lo = 0, hi = T - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_off[mid] <= e) lo = mid;
          else hi = mid - 1;
        }
        const int w = ci[s_rs[lo] + (e - s_off[lo])];
        if (nl < dist[w]) {
          const int old = atomicMin(&dist[w], nl);
          if (old > nl) {
            dec += (long long)(old - nl);
            qn[atomicAdd(&s_qn, 1)] = w;
          }
        }
      }
      cta_sync();
    }
    if (tid == 0) {
      s_F = s_qn;
      s_qn = 0;
    }
    cta_sync();
    int32_t *t = qc;
    qc = qn;
    qn = t;
  }
  return block_sum(dec, s_red);
}

}  // namespace gc
