// Device-side bodies of the grid-wide kernels (cooperative launches): the
// 64-lane pruned multi-source BFS for one batch (see gc_gain_grid.cu) and the
// relabel BFS that maintains d_S (see gc_bfs.cu).  Both synchronise through a
// caller-supplied bounded grid barrier, so they can run as phases of a larger
// persistent kernel (gc_lazy.cu).
#pragma once

#include "gc_device.cuh"
#include "gc_internal.cuh"

namespace gc {

typedef unsigned long long u64;

constexpr int kGridIlp = 2;  // adjacency entries in flight per thread (grid forms)

// Per-level frontier layout of the grid forms: CTA b owns the contiguous
// slice [b*P, min(F, b*P + P)) of the frontier list (P = ceil(F / G)) and
// writes the slice-local exclusive prefix of its entries' degrees to goff;
// blkoff (shared, per CTA) is the exclusive prefix of the slices' totals.
// Entry x then owns the global adjacency indices starting at
// blkoff[x / P] + goff[x].  grid_find_entry returns, for one warp, the
// largest x whose start is <= e (an entry with a non-empty range).
static __device__ __forceinline__ int grid_find_entry(long long e, const long long *blkoff, int G,
                                                      const int32_t *__restrict__ goff, int F, int P) {
  int a = 0, z = G - 1;  // largest slice with blkoff <= e (non-empty)
  while (a < z) {
    const int mid = (a + z + 1) >> 1;
    if (blkoff[mid] <= e) a = mid;
    else z = mid - 1;
  }
  const int local = (int)(e - blkoff[a]);
  const int lane = threadIdx.x & 31;
  int lo = min(F, a * P), hi = min(F, a * P + P) - 1;
  // 32-ary search: goff is non-decreasing in the slice
  while (hi - lo >= 32) {
    const int step = (hi - lo + 32) / 32;  // 32 probes cover [lo, hi]
    const int idx = min(hi, lo + lane * step);
    const unsigned ok = __ballot_sync(0xffffffffu, goff[idx] <= local);
    const int j = 31 - __clz(ok);  // ok holds lane 0 (goff[lo] <= local)
    const int next = lo + (j + 1) * step;  // first probe past the answer, if any
    const int nlo = min(hi, lo + j * step);
    if (j < 31 && next <= hi) hi = next - 1;
    lo = nlo;
  }
  const int idx = lo + lane;
  const unsigned ok = __ballot_sync(0xffffffffu, idx <= hi && goff[min(idx, hi)] <= local);
  return lo + 31 - __clz(ok);
}

// One batch of nl <= 64 candidates advanced by every CTA of the grid.  ctl
// must hold zeros in F, qn, touched, gain and cnt on entry (blk_tot is
// overwritten); the workspace's lane words must be zero and are zero again
// when the last CTA passes the caller's next barrier.  qm holds 2n words (the
// lane masks of the frontier lists).  Returns false if a barrier gave up (the
// error code is in *err / gctl->err).
//
// Claims work as in the CTA form (gc_cta.cuh): atomicOr on the visited word
// decides, and the claim words of levels L and L+1 alternate, so a level needs
// two grid barriers: after the degree scan of the frontier (which also moves
// each entry's claim word into qm and clears it) and after the expansion.
template <int MODE>
static __device__ __forceinline__ bool grid_gain_batch(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                int32_t n, const int32_t *__restrict__ dS, const int32_t *cand, int32_t nl_arg,
                                const int32_t *nl_dev, long long *out, unsigned char *ws_base, u64 *qm,
                                int32_t *__restrict__ goff, GridGainCtl *ctl, GainCtl *gctl, GridBar *bar,
                                int32_t *err, unsigned long long timeout_ns, const int32_t *__restrict__ mx) {
  constexpr int T = kGridGainThreads;
  __shared__ u64 s_gain[kLanes];
  __shared__ unsigned int s_cnt[kLanes];
  __shared__ int s_scan[33];
  __shared__ long long s_blkoff[kMaxGridCtas + 1];
  __shared__ int s_go[T + 1];  // staged entries: start of each entry's range, relative to the level
  __shared__ int s_rs[T];
  __shared__ u64 s_sm[T];
  __shared__ int s_x0;
  __shared__ u64 s_red[32];
  __shared__ int s_qn, s_touched;

  const int tid = threadIdx.x, lane = tid & 31;
  const int G = gridDim.x, b = blockIdx.x;
  const int nl = nl_dev ? min(kLanes, *(volatile const int32_t *)nl_dev) : nl_arg;
  const GainWs ws = gain_ws(ws_base, 0, n, 0);
  u64 c_scalar = 0, c_union = 0, c_front = 0, c_push = 0;
  if (tid < kLanes) {
    s_gain[tid] = 0;
    s_cnt[tid] = 0;
  }
  u64 alive = nl >= kLanes ? ~0ull : ((1ull << nl) - 1ull);

  // ---- level 0 (CTA 0): lanes reach their candidates ----
  if (b == 0) {
    if (tid == 0) {
      s_qn = 0;
      s_touched = 0;
    }
    __syncthreads();
    if (tid < nl) {
      const int c = cand[tid];
      const u64 bit = 1ull << tid;
      bool reach = false;
      if (c < 0 || c >= n) {
        atomicExch(&ctl->err, GC_EINVAL);
      } else if (MODE == kModeGain) {
        const int dc = dS[c];
        if (dc > 0) {
          ctl->gain[tid] = (u64)dc;
          reach = true;
        }
      } else {
        ctl->cnt[tid] = 1;
        reach = true;
      }
      if (reach) {
        if (atomicOr(&ws.vis[c], bit) == 0) ws.touched[atomicAdd(&s_touched, 1)] = c;
        if (atomicOr(&ws.nx[0][c], bit) == 0) ws.qv0[atomicAdd(&s_qn, 1)] = c;
      }
    }
    __syncthreads();
    if (tid == 0) {
      ctl->qn[0] = s_qn;
      ctl->touched = s_touched;
    }
  }
  bool ok = grid_sync(bar, err, timeout_ns);
  // invalid candidate ids leave their lanes empty
  if (ok && MODE == kModeFarness) {
    for (int j = 0; j < nl; ++j)
      if (((volatile unsigned long long *)ctl->cnt)[j] == 0) alive &= ~(1ull << j);
  }

  int L = 0;
  for (; ok; ++L) {
    const int F = *(volatile int32_t *)&ctl->qn[L & 1];
    if (F == 0) break;
    const int32_t *qcur_v = (L & 1) ? ws.qv1 : ws.qv0;
    int32_t *qnxt_v = (L & 1) ? ws.qv0 : ws.qv1;
    u64 *qcur_m = qm + (size_t)(L & 1) * (size_t)n;
    int32_t *qn_ctr = &ctl->qn[(L + 1) & 1];
    const LaneWords cur = (L & 1) ? ws.nx[1] : ws.nx[0], nxt = (L & 1) ? ws.nx[0] : ws.nx[1];
    const int nlev = L + 1;
    // ---- phase 1: masks and degree offsets of this CTA's frontier slice ----
    const int P = (F + G - 1) / G;
    const int lo = min(F, b * P), hi = min(F, lo + P);
    int carry = 0;
    for (int base = lo; base < hi; base += T) {
      const int i = base + tid;
      int deg = 0;
      if (i < hi) {
        const int u = qcur_v[i];
        u64 m = cur[u];
        cur[u] = 0;  // free for level L+2
        const int r0 = rp[u], r1 = rp[u + 1];
        if (MODE == kModeFarness) m &= alive;
        if (MODE == kModeGain && mx && mx[u] <= nlev) m = 0;  // nothing left to claim
        if (m) deg = r1 - r0;
        qcur_m[i] = m;
        c_union += (u64)deg;
        c_scalar += (u64)__popcll(m) * (u64)deg;
        c_front += (m != 0);
      }
      int total;
      const int off = block_excl_scan(deg, s_scan, &total);
      if (i < hi) goff[i] = carry + off;
      carry += total;
    }
    if (tid == 0) {
      ctl->blk_tot[b] = carry;
      if (b == 0) *qn_ctr = 0;
    }
    ok = grid_sync(bar, err, timeout_ns);
    if (!ok) break;
    // ---- phase 2: expand an equal slice of the level's adjacency entries ----
    {
      long long run = 0;
      for (int base = 0; base < G; base += T) {
        const int j = base + tid;
        const int v = j < G ? ((volatile int32_t *)ctl->blk_tot)[j] : 0;
        int total;
        const int off = block_excl_scan(v, s_scan, &total);
        if (j < G) s_blkoff[j] = run + off;
        run += total;
      }
      if (tid == 0) s_blkoff[G] = run;
      __syncthreads();
    }
    const long long E = s_blkoff[G];
    const long long es = E * b / G, ee = E * (b + 1) / G;
    if (es < ee) {
      if (tid < 32) {
        const int x = grid_find_entry(es, s_blkoff, G, goff, F, P);
        if (tid == 0) s_x0 = x;
      }
      __syncthreads();
      int x = s_x0;
      if (x < 0 || x >= F) {  // cannot happen for a consistent frontier; never index with it
        if (tid == 0) atomicExch(err, GC_EINTERNAL);
        x = F;
      }
      while (x < F) {
        // stage up to T entries from x: range starts, row starts, lane masks
        const int xi = x + tid;
        if (xi < F) {
          const u64 m = qcur_m[xi];
          s_go[tid] = (int)(s_blkoff[xi / P] + goff[xi]);
          s_sm[tid] = m;
          s_rs[tid] = m ? rp[qcur_v[xi]] : 0;
        }
        const int cntx = min(T, F - x);
        if (tid == 0) s_go[cntx] = (x + cntx < F) ? (int)(s_blkoff[(x + cntx) / P] + goff[x + cntx]) : (int)E;
        __syncthreads();
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
              int l = 0, h = cntx - 1;  // staged entry holding e (non-empty range)
              while (l < h) {
                const int mid = (l + h + 1) >> 1;
                if (s_go[mid] <= e) l = mid;
                else h = mid - 1;
              }
              sl[k] = l;
              w[k] = ci[s_rs[l] + (int)(e - s_go[l])];
            }
          }
          int dw[kGridIlp];
#pragma unroll
          for (int k = 0; k < kGridIlp; ++k) dw[k] = (MODE == kModeGain && w[k] >= 0) ? dS[w[k]] : 0;
          u64 nb[kGridIlp];
#pragma unroll
          for (int k = 0; k < kGridIlp; ++k) {
            // pruned unless w is strictly closer to the lane's candidate than to S
            const bool live = w[k] >= 0 && (MODE != kModeGain || dw[k] > nlev);
            nb[k] = live ? (s_sm[sl[k]] & ~ws.vis[w[k]]) : 0ull;
          }
          u64 ov[kGridIlp];
#pragma unroll
          for (int k = 0; k < kGridIlp; ++k) ov[k] = nb[k] ? atomicOr(&ws.vis[w[k]], nb[k]) : ~0ull;
#pragma unroll
          for (int k = 0; k < kGridIlp; ++k) {
            u64 won = nb[k] & ~ov[k];
            const bool fresh = won && ov[k] == 0;
            bool push = false;
            if (won) {
              push = atomicOr(&nxt[w[k]], won) == 0;
              const u64 wt = MODE == kModeGain ? (u64)(dw[k] - nlev) : (u64)nlev;
              do {
                const int j = __ffsll((long long)won) - 1;
                won &= won - 1;
                atomicAdd(&s_gain[j], wt);
                if (MODE == kModeFarness) atomicAdd(&s_cnt[j], 1u);
              } while (won);
            }
            const unsigned pm = __ballot_sync(0xffffffffu, push);
            if (pm) {
              const int leader = __ffs(pm) - 1;
              int pos = 0;
              if (lane == leader) pos = atomicAdd(qn_ctr, __popc(pm));
              pos = __shfl_sync(0xffffffffu, pos, leader);
              if (push) qnxt_v[pos + __popc(pm & ((1u << lane) - 1u))] = w[k];
              c_push += (lane == leader) ? (u64)__popc(pm) : 0ull;
            }
            const unsigned fm = __ballot_sync(0xffffffffu, fresh);
            if (fm) {
              const int leader = __ffs(fm) - 1;
              int pos = 0;
              if (lane == leader) pos = atomicAdd(&ctl->touched, __popc(fm));
              pos = __shfl_sync(0xffffffffu, pos, leader);
              if (fresh) ws.touched[pos + __popc(fm & ((1u << lane) - 1u))] = w[k];
            }
          }
        }
        const int done_end = s_go[cntx];
        __syncthreads();  // the staged arrays are reused
        if ((long long)done_end >= ee) break;
        x += cntx;
      }
    }
    if (MODE == kModeFarness) {
      __syncthreads();
      if (tid < kLanes) {
        if (s_gain[tid]) atomicAdd(&ctl->gain[tid], s_gain[tid]);
        if (s_cnt[tid]) atomicAdd(&ctl->cnt[tid], (u64)s_cnt[tid]);
        s_gain[tid] = 0;
        s_cnt[tid] = 0;
      }
    }
    ok = grid_sync(bar, err, timeout_ns);
    if (!ok) break;
    if (MODE == kModeFarness) {
      // the same BFScut test in every CTA: all vertices within L+1 are
      // counted, the rest are at least L+2 away
      const int Fn = *(volatile int32_t *)qn_ctr;
      const long long best = *(volatile long long *)&gctl->best_f;
      for (int j = 0; j < nl; ++j) {
        if (!((alive >> j) & 1ull)) continue;
        const long long s = (long long)((volatile u64 *)ctl->gain)[j];
        const long long c = (long long)((volatile u64 *)ctl->cnt)[j];
        if (Fn > 0 && s + (long long)(L + 2) * ((long long)n - c) > best) alive &= ~(1ull << j);
      }
      if (alive == 0) {
        // every lane is cut: clear the claims of the frontier that is not expanded
        for (int i = b * T + tid; i < Fn; i += G * T) nxt[qnxt_v[i]] = 0;
        break;
      }
    }
  }
  // ---- results ----
  if (MODE == kModeGain) {
    __syncthreads();
    if (tid < kLanes && s_gain[tid]) atomicAdd(&ctl->gain[tid], s_gain[tid]);
  }
  c_scalar = block_sum(c_scalar, s_red);
  c_union = block_sum(c_union, s_red);
  c_front = block_sum(c_front, s_red);
  c_push = block_sum(c_push, s_red);
  if (tid == 0) {
    atomicAdd(&gctl->edges_scalar, c_scalar);
    atomicAdd(&gctl->edges_union, c_union);
    atomicAdd(&gctl->frontier, c_front);
    atomicAdd(&gctl->pushes, c_push);
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
    } else if ((long long)((volatile u64 *)ctl->cnt)[tid] != n) {
      r = -1;
      atomicExch(&gctl->err, GC_EDISCONNECTED);
    } else {
      r = (long long)((volatile u64 *)ctl->gain)[tid];
      atomicMin(&gctl->best_f, r);
    }
    out[tid] = r;
  }
  // leave the workspace zero for the next launch
  const int nt = *(volatile int32_t *)&ctl->touched;
  for (int i = b * T + tid; i < nt; i += G * T) ws.vis[ws.touched[i]] = 0;
  if (!ok2 && b == 0 && tid == 0) atomicExch(&gctl->err, GC_ETIMEOUT);
  return ok2;
}

// Relabel BFS over the whole grid: dist[w] <- min(dist[w], level) from the
// seeds, expanding only where the label decreased (the pruned SSSP of Sec. 4.1
// when dist holds d_S).  qsize[0..2] must be zero on entry.  *decrease collects
// sum(old - new) over relabelled vertices with a finite old label.
// Each level is edge-balanced like grid_gain_batch: CTA slices of the frontier
// scan their degrees into goff (phase 1), then every CTA takes an equal slice
// of the level's adjacency entries (phase 2), so a hub row is shared by all
// CTAs instead of serialising one warp.  With `work` given, CTA 0 adds the
// frontier entries and adjacency entries of every level to work[0], work[1].
static __device__ __forceinline__ bool grid_relabel_bfs(
    const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n, int32_t *dist,
    const int32_t *seeds, int32_t n_seeds, int32_t *q0, int32_t *q1, int32_t *qsize, int32_t *levels_out,
    unsigned long long *decrease, unsigned long long *relabelled, int32_t *__restrict__ goff,
    int32_t *blk_tot, GridBar *bar, int32_t *err, unsigned long long timeout_ns,
    unsigned long long *work = nullptr) {
  __shared__ unsigned long long sh_bfs[32];
  __shared__ int s_scan_b[33];
  __shared__ long long s_boff[kMaxGridCtas + 1];
  const int tid = threadIdx.x, lane = tid & 31, T = blockDim.x;
  const int G = gridDim.x, b = blockIdx.x;
  unsigned long long dec = 0, rel = 0;
  for (int i = b * T + tid; i < n_seeds; i += G * T) {
    const int s = ((volatile const int32_t *)seeds)[i];
    if (s < 0 || s >= n) {
      atomicExch(err, GC_EINVAL);
      continue;
    }
    const int old = atomicMin(&dist[s], 0);
    if (old > 0) {
      const int p = atomicAdd(&qsize[0], 1);
      q0[p] = s;
      if (old < kInf) dec += (unsigned long long)old;
      ++rel;
    }
  }
  bool ok = grid_sync(bar, err, timeout_ns);
  for (int L = 0; ok; ++L) {
    const int F = *(volatile int32_t *)&qsize[L % 3];
    if (F == 0) break;
    const int32_t *qc = (L & 1) ? q1 : q0;
    int32_t *qn = (L & 1) ? q0 : q1;
    int32_t *qn_size = &qsize[(L + 1) % 3];
    const int nl = L + 1;
    // phase 1: degree offsets of this CTA's contiguous frontier slice
    const int P = (F + G - 1) / G;
    const int lo = min(F, b * P), hi = min(F, lo + P);
    int carry = 0;
    for (int base = lo; base < hi; base += T) {
      const int i = base + tid;
      const int deg = i < hi ? rp[qc[i] + 1] - rp[qc[i]] : 0;
      int total;
      const int off = block_excl_scan(deg, s_scan_b, &total);
      if (i < hi) goff[i] = carry + off;
      carry += total;
    }
    if (tid == 0) {
      blk_tot[b] = carry;
      if (b == 0) qsize[(L + 2) % 3] = 0;
    }
    ok = grid_sync(bar, err, timeout_ns);
    if (!ok) break;
    // phase 2: an equal slice of the level's adjacency entries per CTA
    {
      long long run = 0;
      for (int base = 0; base < G; base += T) {
        const int j = base + tid;
        const int v = j < G ? ((volatile int32_t *)blk_tot)[j] : 0;
        int total;
        const int off = block_excl_scan(v, s_scan_b, &total);
        if (j < G) s_boff[j] = run + off;
        run += total;
      }
      if (tid == 0) s_boff[G] = run;
      __syncthreads();
    }
    const long long E = s_boff[G];
    if (work && b == 0 && tid == 0) {
      work[0] += (unsigned long long)F;
      work[1] += (unsigned long long)E;
    }
    const long long es = E * b / G, ee = E * (b + 1) / G;
    for (long long e0 = es + (tid & ~31); e0 < ee; e0 += T) {
      const long long e = e0 + lane;
      bool push = false;
      int w = 0;
      if (e < ee) {
        int a = 0, z = G - 1;
        while (a < z) {
          const int mid = (a + z + 1) >> 1;
          if (s_boff[mid] <= e) a = mid;
          else z = mid - 1;
        }
        const int local = (int)(e - s_boff[a]);
        int x = min(F, a * P), y = min(F, a * P + P) - 1;
        while (x < y) {
          const int mid = (x + y + 1) >> 1;
          if (goff[mid] <= local) x = mid;
          else y = mid - 1;
        }
        w = ci[rp[qc[x]] + (local - goff[x])];
        if (nl < dist[w]) {
          const int old = atomicMin(&dist[w], nl);
          if (old > nl) {
            push = true;
            if (old < kInf) dec += (unsigned long long)(old - nl);
            ++rel;
          }
        }
      }
      const unsigned m = __ballot_sync(0xffffffffu, push);
      if (m) {
        const int leader = __ffs(m) - 1;
        int pos = 0;
        if (lane == leader) pos = atomicAdd(qn_size, __popc(m));
        pos = __shfl_sync(0xffffffffu, pos, leader);
        if (push) qn[pos + __popc(m & ((1u << lane) - 1u))] = w;
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
