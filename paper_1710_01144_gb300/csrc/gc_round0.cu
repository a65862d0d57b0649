// Round 0 on shallow graphs: f({v}) for many round-0 survivors at once, with
// the BFScut of Sec. 3.1 (Algorithm 3 with k = 1), by a bit-parallel
// multi-source BFS of B = 64 W lanes per batch that runs on the whole GPU.
//
// Why a separate kernel.  On small-world graphs (R-MAT, social networks) the
// round-0 degree bound leaves the vertices next to the hubs: their two-hop
// counts are large.  Each of them reaches most of the graph at distance 2, so
// its search scans the hub rows before its cut can fire.  Batches of 64 lanes
// on one CTA re-read those rows once per batch (the scale-24 R-MAT graph: 867
// batches, 210G adjacency entries, 23 s).  Here one batch holds up to 512
// candidates and every level after the first is expanded bottom-up: each
// vertex with lanes still missing ORs the lane words of its neighbours that are
// in the current frontier (a 1-bit-per-vertex bitmap decides which words to
// read) until no missing lane is left.  One pass over the adjacency then serves
// every lane of the batch, and the pass is a coalesced stream over the CSR.
//
// Level 0 -> 1 (the candidates' own rows) is top-down: atomicOr of the lane
// bit into the neighbour's visited and claim words.  Rows longer than
// kHeavyRow entries are split into chunks of kHeavyRow that any warp can
// take; their partial ORs meet in a per-row accumulator that a second phase
// applies.  Rows of up to 32 entries are scanned by one thread, longer light
// rows by a whole warp.
//
// Lane words: vis[w] (the lanes that reached w) and three claim buffers used in
// rotation: the frontier of distance d is buf[d mod 3] with bitmap fb[d mod 3];
// while distance d + 1 is claimed, the buffer of distance d - 1 is cleared.
// Claim buffers and bitmaps are zero between batches; vis is cleared at the
// end of every batch.
//
// Per-lane counts of each level come from warp ballots (one ballot per lane
// bit over 32 vertices), summed per CTA in shared memory and per level in
// global memory.  After each level every CTA applies the same BFScut test to
// its own copy of the lane state, from the same global totals:
//   lane j, all vertices within distance d counted (cnt_j of them, distance
//   sum sum_j):  f({v_j}) >= sum_j + (d + 1) (n - cnt_j);  cut if > best.
// best only decreases (completed lanes), so every CTA keeps the same copy.
//
// The first bottom-up level (distance 2) reads the short rows in stages (the
// far-vertex probe): a vertex whose whole row holds none of a lane's missing
// bits is at distance >= 3 from that lane's candidate, and counting such
// vertices raises the lane's bound above the usual "every unvisited vertex at
// d + 1" form.  Most round-0 survivors of R-MAT graphs are at distance >= 3
// from most vertices, so a stage or two cut a whole batch before its longer
// rows and hub chunks are read.
//
// Survivors are taken in list order while their lower bound is at most the
// best farness so far.  A batch whose live lanes fall below `defer_below`
// after the distance-2 cut hands them to a deferred list and ends, so that a
// few surviving lanes do not pay full passes over the graph alone; the
// deferred candidates run afterwards in full batches of their own.
#include <limits.h>
#include <string.h>

#include <algorithm>

#include "gc_device.cuh"
#include "gc_internal.cuh"

namespace gc {

typedef unsigned long long u64;

constexpr int kR0Threads = 512;
constexpr int kR0Ilp = 4;  // adjacency entries in flight per thread in the bottom-up passes

// Lane words and bitmaps change from level to level and are written by other
// SMs; they are read with ordinary loads after the grid barrier, whose
// release/acquire pair orders every write before it (other CTAs included)
// before every read after it, so hot lines (hub frontier words, bitmap words)
// can be served by L1 within a level.
template <int W>
__device__ __forceinline__ void ld_words(const u64 *p, u64 (&x)[W]) {
  if (W == 1) {
    x[0] = *p;
  } else {
#pragma unroll
    for (int k = 0; k < W; k += 2) {
      const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p + k);
      x[k] = v.x;
      x[k + (W > 1 ? 1 : 0)] = v.y;
    }
  }
}

template <int W>
__device__ __forceinline__ void st_words(u64 *p, const u64 (&x)[W]) {
  if (W == 1) {
    *p = x[0];
  } else {
#pragma unroll
    for (int k = 0; k < W; k += 2) {
      ulonglong2 v;
      v.x = x[k];
      v.y = x[k + (W > 1 ? 1 : 0)];
      *reinterpret_cast<ulonglong2 *>(p + k) = v;
    }
  }
}

// acc |= the lane words at p, loading only the words marked in `open` (pairs of
// words share one 16-byte load)
template <int W>
__device__ __forceinline__ void gather_open(const u64 *p, unsigned open, u64 (&acc)[W]) {
  if (W == 1) {
    if (open & 1u) acc[0] |= *p;
  } else {
#pragma unroll
    for (int k = 0; k < W; k += 2) {
      if (!((open >> k) & 3u)) continue;
      const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p + k);
      acc[k] |= v.x;
      acc[k + (W > 1 ? 1 : 0)] |= v.y;
    }
  }
}

__device__ __forceinline__ u64 warp_or64(u64 x) {
  const unsigned lo = __reduce_or_sync(0xffffffffu, (unsigned)x);
  const unsigned hi = __reduce_or_sync(0xffffffffu, (unsigned)(x >> 32));
  return ((u64)hi << 32) | lo;
}

__device__ __forceinline__ long long r0_block_min(long long v, long long *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  cta_sync();
  if (lane == 0) sh[wid] = v;
  cta_sync();
  v = LLONG_MAX;
  for (int w = 0; w < nw; ++w) v = min(v, sh[w]);
  cta_sync();
  return v;
}

__device__ __forceinline__ bool in_frontier(const uint32_t *fb, int u) { return (fb[u >> 5] >> (u & 31)) & 1u; }

// Zero the words of every vertex marked in bitmap fb, and (clear_bitmap) the
// bitmap.
template <int W>
__device__ __forceinline__ void clear_frontier(u64 *buf, uint32_t *fb, int nbw, bool clear_bitmap = true) {
  const int T = blockDim.x;
  for (int x = blockIdx.x * T + threadIdx.x; x < nbw; x += gridDim.x * T) {
    uint32_t bits = fb[x];
    if (!bits) continue;
    if (clear_bitmap) fb[x] = 0;
    const u64 z[W] = {};
    do {
      const int b = __ffs(bits) - 1;
      bits &= bits - 1;
      st_words<W>(buf + (size_t)(32 * x + b) * W, z);
    } while (bits);
  }
}

template <int W>
__device__ __forceinline__ void count_lanes(bool has, const u64 (&xw)[W], int lane, unsigned int (&lc)[2 * W]);

// The end of a vertex chunk in a bottom-up pass: lane w (if `want`) has found
// the missing lanes `nw` among its frontier neighbours; record them in its
// visited and next-frontier words and the next bitmap, and add them to this
// thread's per-lane counts (lc[2k + h] counts lane 64k + 32h + (thread lane))
// through one warp ballot per lane bit.
template <int W>
__device__ __forceinline__ void claim_words(int w, int base, int lane, bool want, const u64 (&nw)[W], u64 *vis,
                                            u64 *nxt, uint32_t *fbn, unsigned int (&lc)[2 * W],
                                            unsigned int &claims, bool write) {
  bool has = false;
#pragma unroll
  for (int k = 0; k < W; ++k) has |= want && nw[k] != 0;
  if (has && write) {  // only this thread writes w's words during the level
    u64 vw[W];
    ld_words<W>(vis + (size_t)w * W, vw);
#pragma unroll
    for (int k = 0; k < W; ++k) vw[k] |= nw[k];
    st_words<W>(vis + (size_t)w * W, vw);
    st_words<W>(nxt + (size_t)w * W, nw);
    ++claims;
  }
  const unsigned hm = __ballot_sync(0xffffffffu, has);
  if (write && lane == 0 && hm) atomicOr(&fbn[base >> 5], hm);  // both passes may mark this word
  count_lanes<W>(has, nw, lane, lc);
}

// Per-lane counts of the bits of x over the warp (only where `has`):
// lc[2k + h] += the number of threads whose word k holds bit 32h + (this
// thread's lane), one warp ballot per lane bit.
template <int W>
__device__ __forceinline__ void count_lanes(bool has, const u64 (&xw)[W], int lane, unsigned int (&lc)[2 * W]) {
#pragma unroll
  for (int k = 0; k < W; ++k) {
    const u64 x = has ? xw[k] : 0ull;
    if (!__any_sync(0xffffffffu, x != 0)) continue;
    unsigned c0 = 0, c1 = 0;
#pragma unroll
    for (int bt = 0; bt < 32; ++bt) {
      const unsigned b0 = __ballot_sync(0xffffffffu, (x >> bt) & 1ull);
      const unsigned b1 = __ballot_sync(0xffffffffu, (x >> (bt + 32)) & 1ull);
      if (lane == bt) {
        c0 = __popc(b0);
        c1 = __popc(b1);
      }
    }
    lc[2 * k] += c0;
    lc[2 * k + 1] += c1;
  }
}

template <int W>
__global__ void __launch_bounds__(kR0Threads, W <= 4 ? 2 : 1)
    k_round0_wide(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n,
                  const int32_t *__restrict__ list, int32_t m, const long long *__restrict__ key, long long *lgain,
                  int32_t *defer, R0Ctl *ctl, GainCtl *gctl, u64 *vis, u64 *buf_a, u64 *buf_b, u64 *buf_c,
                  uint32_t *fb_a, uint32_t *fb_b, uint32_t *fb_c, const int32_t *__restrict__ heavy, int32_t nh,
                  const int32_t *__restrict__ hcp, u64 *hacc, int32_t defer_below, int32_t allow_count_only,
                  int32_t probe_stride, unsigned long long tns) {
  constexpr int B = 64 * W;
  constexpr int T = kR0Threads;
  __shared__ int s_cand[B], s_pos[B];
  __shared__ long long s_sum[B], s_cnt[B], s_fin[B];
  __shared__ unsigned int s_lc[B], s_fc[B];
  __shared__ int s_eoff[B + 1];
  __shared__ u64 s_alive[W];
  __shared__ int s_scan[33];
  __shared__ long long s_red[32];
  const int tid = threadIdx.x, lane = tid & 31, G = gridDim.x, b = blockIdx.x;
  const int gw = b * (T / 32) + (tid >> 5), nwarps = G * (T / 32);
  const int nbw = (n + 31) >> 5;
  int32_t *err = &gctl->err;
  const bool fixed_best = *(volatile int32_t *)&gctl->fixed_best != 0;  // top-k: the cut stays at its start
  u64 *bufs[3] = {buf_a, buf_b, buf_c};
  uint32_t *fbs[3] = {fb_a, fb_b, fb_c};
  const int C = nh > 0 ? hcp[nh] : 0;  // heavy-row chunks
  u64 w_batches = 0, w_levels = 0, w_lanes = 0, w_td = 0, w_scan = 0, w_gath = 0, w_claim = 0;
  u64 w_vert = 0, w_visr = 0;  // bottom-up: row-pointer pairs and visited words read
  const bool timer = b == 0 && tid == 0;
  u64 t_prev = timer ? global_ns() : 0, t_ph[4] = {0, 0, 0, 0};
  auto lap = [&](int i) {
    if (timer) {
      const u64 t = global_ns();
      t_ph[i] += t - t_prev;
      t_prev = t;
    }
  };

  for (;;) {
    // ---------- batch selection (warp 0 of CTA 0) ----------
    if (b == 0 && tid < 32) {
      const long long bf = ctl->best_f;
      int phase = ctl->phase, nb = 0;
      while (phase < 2 && nb < B) {
        const int end = phase == 0 ? m : ctl->n_defer;
        int cur = phase == 0 ? ctl->cursor : ctl->dcursor;
        while (cur < end && nb < B) {
          const int i = cur + lane;
          int v = -1, pos = -1;
          bool ok = false;
          if (i < end) {
            if (phase == 0) {
              v = list[i];
              pos = i;
            } else {
              v = defer[2 * i];
              pos = defer[2 * i + 1];
            }
            ok = -key[v] <= bf;  // lower bound at most the best farness so far
          }
          const unsigned okm = __ballot_sync(0xffffffffu, ok);
          const int room = B - nb;
          // entries consumed: all up to the room-th accepted one
          int take_upto = 32;  // lanes [0, take_upto) are consumed
          if (__popc(okm) > room) {
            unsigned mm = okm;
            for (int r = 0; r < room; ++r) mm &= mm - 1;
            take_upto = __ffs(mm) - 1;  // the first accepted entry that does not fit
          }
          if (i < end && lane < take_upto) {
            if (ok) {
              const int slot = nb + __popc(okm & ((1u << lane) - 1u));
              ctl->cand[slot] = v;
              ctl->pos[slot] = pos;
            } else {
              lgain[pos] = -1;  // cannot beat the best farness: never searched
            }
          }
          nb += __popc(okm & (take_upto == 32 ? 0xffffffffu : ((1u << take_upto) - 1u)));
          cur += min(take_upto, end - cur);
          __syncwarp();
        }
        if (lane == 0) {
          if (phase == 0) ctl->cursor = cur;
          else ctl->dcursor = cur;
        }
        if (nb < B && cur >= end) ++phase;  // this list is exhausted
        else break;
      }
      if (lane == 0) {
        ctl->phase = phase;
        ctl->nb = nb;
        // count distance 2 only while at most a quarter of such lanes survive
        // their distance-2 cut (the survivors are rerun in full batches)
        ctl->count_only = allow_count_only && phase == 0 && 4 * ctl->co_surv <= ctl->co_lanes + 64;
      }
      for (int i = lane; i < 3 * B; i += 32) ctl->tot[i / B][i % B] = 0;  // rows are kR0MaxLanes apart
      for (int i = lane; i < B; i += 32) ctl->far[i] = 0;
    }
    if (!grid_sync(&ctl->bar, err, tns)) break;
    lap(0);
    const int nb = *(volatile int32_t *)&ctl->nb;
    if (nb == 0) break;
    const int phase = *(volatile int32_t *)&ctl->phase;
    const bool co = *(volatile int32_t *)&ctl->count_only != 0;
    bool wrote = false;  // a bottom-up level wrote visited words (else they are sparse)
    long long bf = *(volatile long long *)&ctl->best_f;
    // ---------- lane state (every CTA keeps the same copy) ----------
    for (int j = tid; j < B; j += T) {
      const int c = j < nb ? ((volatile int32_t *)ctl->cand)[j] : -1;
      s_cand[j] = c;
      s_pos[j] = j < nb ? ((volatile int32_t *)ctl->pos)[j] : -1;
      s_sum[j] = 0;
      s_cnt[j] = 1;  // the candidate itself
      s_fin[j] = -1;
      s_lc[j] = 0;
      s_fc[j] = 0;
    }
    if (tid < W) {
      const int lo = 64 * tid;
      s_alive[tid] = nb >= lo + 64 ? ~0ull : (nb > lo ? ((1ull << (nb - lo)) - 1ull) : 0ull);
    }
    cta_sync();
    // ---------- distance 1: the candidates' rows, top-down ----------
    {
      const int j = tid;
      const int deg = (j < nb) ? __ldg(rp + s_cand[j] + 1) - __ldg(rp + s_cand[j]) : 0;
      int total;
      const int ex = block_excl_scan(j < B ? deg : 0, s_scan, &total);
      if (j < B) s_eoff[j] = ex;
      if (j == 0) s_eoff[B] = total;
      cta_sync();
      if (b == 0 && j < nb) {  // level 0: each lane reaches its candidate
        const int c = s_cand[j];
        atomicOr(&vis[(size_t)c * W + (j >> 6)], 1ull << (j & 63));
      }
      const int E = s_eoff[B];
      w_td += (u64)E;
      u64 *nx1 = bufs[1];
      uint32_t *fb1 = fbs[1];
      for (int e = b * T + tid; e < E; e += G * T) {
        int lo = 0, hi = nb - 1;  // lane holding e (largest lo with s_eoff[lo] <= e)
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (s_eoff[mid] <= e) lo = mid;
          else hi = mid - 1;
        }
        const int c = s_cand[lo];
        const int w = __ldg(ci + __ldg(rp + c) + (e - s_eoff[lo]));
        const u64 bit = 1ull << (lo & 63);
        const size_t at = (size_t)w * W + (lo >> 6);
        const u64 old = atomicOr(&vis[at], bit);
        if (!(old & bit)) {
          if (!co) atomicOr(&nx1[at], bit);  // (a count-only pass reads vis instead, see below)
          atomicOr(&fb1[w >> 5], 1u << (w & 31));
          atomicAdd(&s_lc[lo], 1u);
        }
      }
      cta_sync();
      for (int j2 = tid; j2 < nb; j2 += T)
        if (s_lc[j2]) {
          atomicAdd(&ctl->tot[1][j2], (u64)s_lc[j2]);
          s_lc[j2] = 0;
        }
    }
    bool ok = grid_sync(&ctl->bar, err, tns);
    if (!ok) break;
    lap(1);
    ++w_batches;
    w_lanes += (u64)nb;
    int d = 1;  // the distance whose claims were just counted
    bool any_alive = true;
    for (;;) {
      // ---------- fold the counts of distance d; BFScut (same in every CTA) ----------
      const volatile u64 *tot = (const volatile u64 *)ctl->tot[d % 3];
      long long fmin = LLONG_MAX;
      for (int j = tid; j < nb; j += T) {
        if (!((s_alive[j >> 6] >> (j & 63)) & 1ull)) continue;
        const long long c = (long long)tot[j];
        s_cnt[j] += c;
        s_sum[j] += (long long)d * c;
        if (c == 0 || s_cnt[j] == n) {  // search complete
          if (s_cnt[j] == n) {
            s_fin[j] = s_sum[j];
            fmin = min(fmin, s_sum[j]);
          } else {
            s_fin[j] = -2;  // ended short of n: the graph is disconnected
          }
        }
      }
      fmin = r0_block_min(fmin, s_red);
      if (!fixed_best) bf = min(bf, fmin);
      for (int j = tid; j < nb; j += T) {
        if (!((s_alive[j >> 6] >> (j & 63)) & 1ull)) continue;
        bool drop = false;
        long long out = 0;
        bool write = false;
        if (s_fin[j] != -1) {
          drop = true;
          write = true;
          out = s_fin[j] >= 0 ? s_fin[j] : -1;
          if (s_fin[j] == -2 && b == 0) {
            gctl->short_vertex = s_cand[j];
            gctl->short_count = s_cnt[j];
            atomicExch(&gctl->err, GC_EDISCONNECTED);
          }
        } else if (s_sum[j] + (long long)(d + 1) * ((long long)n - s_cnt[j]) > bf) {
          drop = true;  // cut: cannot beat the best farness
          write = true;
          out = -1;
        }
        if (drop) atomicAnd(&s_alive[j >> 6], ~(1ull << (j & 63)));
        if (write && b == 0) lgain[s_pos[j]] = out;
      }
      cta_sync();
      if (b == 0)  // the next level's totals (read two folds ago by every CTA)
        for (int j = tid; j < B; j += T) ctl->tot[(d + 1) % 3][j] = 0;
      int alive_cnt = 0;
#pragma unroll
      for (int k = 0; k < W; ++k) alive_cnt += __popcll(s_alive[k]);
      if (alive_cnt > 0 && phase == 0 && d >= 2 && (co || alive_cnt < defer_below)) {
        // few live lanes, or a count-only batch (no distance-2 frontier was
        // written): run them later in full batches of their own
        if (b == 0 && tid == 0) {
          int at = ctl->n_defer;
          for (int j = 0; j < nb; ++j)
            if ((s_alive[j >> 6] >> (j & 63)) & 1ull) {
              defer[2 * at] = s_cand[j];
              defer[2 * at + 1] = s_pos[j];
              ++at;
            }
          ctl->n_defer = at;
        }
        if (co && b == 0 && tid == 0) ctl->co_surv += (unsigned long long)alive_cnt;
        alive_cnt = 0;
      }
      if (co && d == 2 && b == 0 && tid == 0) ctl->co_lanes += (unsigned long long)nb;
      cta_sync();
      if (alive_cnt == 0) {
        any_alive = false;
        break;
      }
      ++w_levels;
      // ---------- claims of distance d + 1, bottom-up ----------
      // (a count-only batch counts distance 2 and writes nothing: its lanes
      // end or are deferred at the next fold)
      const bool write_lv = !(co && d == 1);
      wrote |= write_lv;
      // The frontier words of distance d.  A count-only pass writes no visited
      // word, so at distance 1 it reads vis (lanes within distance 1) for the
      // frontier's words: a lane j that vis adds beyond the distance-1 claims
      // has the frontier vertex as its candidate, so every neighbour u of it
      // is within distance 1 of v_j and lane j is not missing at u.  The
      // top-down level then skips the claim words of distance 1.
      const u64 *cur = (co && d == 1) ? vis : bufs[d % 3];
      const uint32_t *fbc = fbs[d % 3];
      u64 *nxt = bufs[(d + 1) % 3];
      uint32_t *fbn = fbs[(d + 1) % 3];
      clear_frontier<W>(bufs[(d + 2) % 3], fbs[(d + 2) % 3], nbw);  // distance d - 1
      unsigned int lc[2 * W];
#pragma unroll
      for (int k = 0; k < 2 * W; ++k) lc[k] = 0;
      unsigned int l_scan = 0, l_gath = 0, l_claim = 0, l_vert = 0, l_visr = 0;
      // One window of 32 vertices, its rows of at most 32 entries: one thread
      // each, kR0Ilp entries in flight; a lane word is loaded only while some
      // of its missing lanes are unfound, and the scan stops once none is
      // left.  With fc, also counts per lane the vertices whose whole row held
      // none of their missing lanes: those are at distance >= d + 2.
      auto short_window = [&](int base, bool with_far, unsigned int(&fc)[2 * W]) {
        const int w = base + lane;
        int r0 = 0, r1 = 0;
        u64 miss[W];
        bool want = false;
        if (w < n) {
          r0 = __ldg(rp + w);
          r1 = __ldg(rp + w + 1);
          ++l_vert;
        }
        if (r1 - r0 <= 32 && r1 > r0) {
          ++l_visr;
          ld_words<W>(vis + (size_t)w * W, miss);
#pragma unroll
          for (int k = 0; k < W; ++k) {
            miss[k] = s_alive[k] & ~miss[k];
            want |= miss[k] != 0;
          }
        }
        if (!__any_sync(0xffffffffu, want)) return;
        u64 acc[W];
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] = 0;
        if (want) {
          unsigned open = 0;  // words with lanes still unfound
#pragma unroll
          for (int k = 0; k < W; ++k) open |= (miss[k] != 0 ? 1u : 0u) << k;
          for (int e = r0; e < r1 && open; e += kR0Ilp) {
            int u[kR0Ilp];
#pragma unroll
            for (int q = 0; q < kR0Ilp; ++q) u[q] = e + q < r1 ? __ldg(ci + e + q) : -1;
            bool fr[kR0Ilp];
#pragma unroll
            for (int q = 0; q < kR0Ilp; ++q) fr[q] = u[q] >= 0 && in_frontier(fbc, u[q]);
#pragma unroll
            for (int q = 0; q < kR0Ilp; ++q) {
              if (!fr[q]) continue;
              ++l_gath;
              gather_open<W>(cur + (size_t)u[q] * W, open, acc);
            }
            l_scan += (unsigned)min(kR0Ilp, r1 - e);
#pragma unroll
            for (int k = 0; k < W; ++k)
              if ((acc[k] & miss[k]) == miss[k]) open &= ~(1u << k);
          }
#pragma unroll
          for (int k = 0; k < W; ++k) acc[k] &= miss[k];
        }
        claim_words<W>(w, base, lane, want, acc, vis, nxt, fbn, lc, l_claim, write_lv);
        if (with_far) {
          u64 far[W];
#pragma unroll
          for (int k = 0; k < W; ++k) far[k] = miss[k] & ~acc[k];
          count_lanes<W>(want, far, lane, fc);
        }
      };
      // Pass A, the short rows, in probe_stride stages at distance 2 (the
      // first bottom-up level): stage s takes the windows i with
      // i mod probe_stride == s.  A vertex whose whole row held none of a
      // lane's missing bits is at distance >= 3 from that lane's candidate,
      // so after each stage, with far_j such vertices counted over the grid,
      //   f({v_j}) >= sum_j + (d + 1) (n - cnt_j - far_j) + (d + 2) far_j,
      // and a lane whose bound exceeds the best farness is cut (BFScut,
      // Sec. 3.1) before the remaining windows, the longer rows and the hub
      // chunks are read.  On R-MAT most vertices are at distance >= 3 from
      // every round-0 survivor, so the first stage or two usually cut the
      // whole batch.  A count-only batch then defers what is left (those
      // lanes rerun in full batches) instead of reading the longer rows.
      const bool probe = d == 1 && probe_stride > 0;
      const int S = probe ? probe_stride : 1;
      bool live = true;
      for (int st = 0; st < S && live; ++st) {
        unsigned int fc[2 * W];
#pragma unroll
        for (int k = 0; k < 2 * W; ++k) fc[k] = 0;
        for (int base = (gw * S + st) * 32; base < n; base += nwarps * S * 32) short_window(base, probe, fc);
        if (!probe) break;
#pragma unroll
        for (int k = 0; k < 2 * W; ++k)
          if (fc[k]) atomicAdd(&s_fc[64 * (k >> 1) + 32 * (k & 1) + lane], fc[k]);
        cta_sync();
        for (int j = tid; j < nb; j += T)
          if (s_fc[j]) {
            atomicAdd(&ctl->far[j], (u64)s_fc[j]);
            s_fc[j] = 0;
          }
        ok = grid_sync(&ctl->bar, err, tns);
        if (!ok) break;
        const volatile u64 *farc = ctl->far;
        for (int j = tid; j < nb; j += T) {
          if (!((s_alive[j >> 6] >> (j & 63)) & 1ull)) continue;
          const long long fj = (long long)farc[j];
          const long long lb =
              s_sum[j] + (long long)(d + 1) * ((long long)n - s_cnt[j] - fj) + (long long)(d + 2) * fj;
          if (lb > bf) {
            atomicAnd(&s_alive[j >> 6], ~(1ull << (j & 63)));
            if (b == 0) {
              lgain[s_pos[j]] = -1;  // cut: cannot beat the best farness
              atomicAdd(&ctl->probe_cut, 1ull);
            }
          }
        }
        if (b == 0 && tid == 0) ++ctl->probe_levels;
        cta_sync();
        live = false;
#pragma unroll
        for (int k = 0; k < W; ++k) live |= s_alive[k] != 0;
      }
      if (!ok) break;
      if (probe && co && live) {
        // count-only: the lanes the short rows could not cut run later in
        // full batches of their own
        if (b == 0 && tid == 0) {
          int at = ctl->n_defer, cnt = 0;
          for (int j = 0; j < nb; ++j)
            if ((s_alive[j >> 6] >> (j & 63)) & 1ull) {
              defer[2 * at] = s_cand[j];
              defer[2 * at + 1] = s_pos[j];
              ++at;
              ++cnt;
            }
          ctl->n_defer = at;
          ctl->co_surv += (unsigned long long)cnt;
        }
        cta_sync();
        if (tid < W) s_alive[tid] = 0ull;
        cta_sync();
        live = false;
      }
      // Pass B: rows of 33 .. kHeavyRow entries, the whole warp on one vertex
      // at a time (coalesced column loads, kR0Ilp per lane in flight).
      for (int base = gw * 32; live && base < n; base += nwarps * 32) {
        const int w = base + lane;
        int r0 = 0, r1 = 0;
        u64 miss[W];
        bool want = false;
        if (w < n) {
          r0 = __ldg(rp + w);
          r1 = __ldg(rp + w + 1);
          ++l_vert;
        }
        if (r1 - r0 > 32 && r1 - r0 <= kHeavyRow) {
          ++l_visr;
          ld_words<W>(vis + (size_t)w * W, miss);
#pragma unroll
          for (int k = 0; k < W; ++k) {
            miss[k] = s_alive[k] & ~miss[k];
            want |= miss[k] != 0;
          }
        }
        unsigned mm = __ballot_sync(0xffffffffu, want);
        if (!mm) continue;
        u64 acc[W];
#pragma unroll
        for (int k = 0; k < W; ++k) acc[k] = 0;
        while (mm) {
          const int t = __ffs(mm) - 1;
          mm &= mm - 1;
          const int a0 = __shfl_sync(0xffffffffu, r0, t), a1 = __shfl_sync(0xffffffffu, r1, t);
          u64 ms[W], ac[W];
          unsigned open = 0;
#pragma unroll
          for (int k = 0; k < W; ++k) {
            ms[k] = __shfl_sync(0xffffffffu, miss[k], t);
            ac[k] = 0;
            open |= (ms[k] != 0 ? 1u : 0u) << k;
          }
          for (int e0 = a0; e0 < a1 && open; e0 += 32 * kR0Ilp) {
            int u[kR0Ilp];
#pragma unroll
            for (int q = 0; q < kR0Ilp; ++q) {
              const int e = e0 + q * 32 + lane;
              u[q] = e < a1 ? __ldg(ci + e) : -1;
            }
            bool fr[kR0Ilp];
#pragma unroll
            for (int q = 0; q < kR0Ilp; ++q) {
              fr[q] = u[q] >= 0 && in_frontier(fbc, u[q]);
              l_scan += u[q] >= 0;
            }
#pragma unroll
            for (int q = 0; q < kR0Ilp; ++q) {
              if (!fr[q]) continue;
              ++l_gath;
              gather_open<W>(cur + (size_t)u[q] * W, open, ac);
            }
#pragma unroll
            for (int k = 0; k < W; ++k) {
              if (!((open >> k) & 1u)) continue;  // (open is warp-uniform)
              ac[k] = warp_or64(ac[k]);
              if ((ac[k] & ms[k]) == ms[k]) open &= ~(1u << k);
            }
          }
          if (lane == t) {
#pragma unroll
            for (int k = 0; k < W; ++k) acc[k] = ac[k] & ms[k];
          }
        }
        claim_words<W>(w, base, lane, want, acc, vis, nxt, fbn, lc, l_claim, write_lv);
      }
      u64 al[W];
#pragma unroll
      for (int k = 0; k < W; ++k) al[k] = s_alive[k];
      // heavy rows: chunks of kHeavyRow entries, partial ORs into hacc
      for (int c = gw; live && c < C; c += nwarps) {
        int lo = 0, hi = nh - 1;  // heavy row holding chunk c
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (hcp[mid] <= c) lo = mid;
          else hi = mid - 1;
        }
        const int h = heavy[lo];
        const int a0 = __ldg(rp + h) + (c - hcp[lo]) * kHeavyRow;
        const int a1 = min(__ldg(rp + h + 1), a0 + kHeavyRow);
        u64 vh[W], ms[W], ac[W];
        ld_words<W>(vis + (size_t)h * W, vh);
        ++l_visr;
        bool any = false;
#pragma unroll
        for (int k = 0; k < W; ++k) {
          ms[k] = al[k] & ~vh[k];
          any |= ms[k] != 0;
          ac[k] = 0;
        }
        if (!any) continue;
        for (int e0 = a0; e0 < a1; e0 += 32 * kR0Ilp) {
          int u[kR0Ilp];
#pragma unroll
          for (int q = 0; q < kR0Ilp; ++q) {
            const int e = e0 + q * 32 + lane;
            u[q] = e < a1 ? __ldg(ci + e) : -1;
          }
          bool fr[kR0Ilp];
#pragma unroll
          for (int q = 0; q < kR0Ilp; ++q) {
            fr[q] = u[q] >= 0 && in_frontier(fbc, u[q]);
            l_scan += u[q] >= 0;
            l_gath += fr[q];
          }
#pragma unroll
          for (int q = 0; q < kR0Ilp; ++q) {
            if (!fr[q]) continue;
            u64 f[W];
            ld_words<W>(cur + (size_t)u[q] * W, f);
#pragma unroll
            for (int k = 0; k < W; ++k) ac[k] |= f[k];
          }
          if (((e0 - a0) & 255) == 128 || e0 + 32 * kR0Ilp >= a1) {  // every 256 entries: stop once nothing is missing
            bool done = true;
#pragma unroll
            for (int k = 0; k < W; ++k) {
              ac[k] = warp_or64(ac[k]);
              done &= (ac[k] & ms[k]) == ms[k];
            }
            if (done) break;
          }
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < W; ++k)
            if (ac[k] & ms[k]) atomicOr(&hacc[(size_t)lo * W + k], ac[k] & ms[k]);
        }
      }
#pragma unroll
      for (int k = 0; k < 2 * W; ++k)
        if (lc[k]) atomicAdd(&s_lc[64 * (k >> 1) + 32 * (k & 1) + lane], lc[k]);
      w_scan += l_scan;
      w_gath += l_gath;
      w_vert += l_vert;
      w_visr += l_visr;
      ok = grid_sync(&ctl->bar, err, tns);
      if (!ok) break;
      // heavy rows: apply the accumulated lanes
      for (int i = b * T + tid; i < nh; i += G * T) {
        u64 a[W];
        ld_words<W>(hacc + (size_t)i * W, a);
        bool any = false;
#pragma unroll
        for (int k = 0; k < W; ++k) any |= a[k] != 0;
        if (!any) continue;
        const u64 z[W] = {};
        st_words<W>(hacc + (size_t)i * W, z);
        const int h = heavy[i];
        u64 vh[W], nw[W];
        ld_words<W>(vis + (size_t)h * W, vh);
        bool has = false;
#pragma unroll
        for (int k = 0; k < W; ++k) {
          nw[k] = a[k] & al[k] & ~vh[k];
          has |= nw[k] != 0;
          vh[k] |= nw[k];
        }
        if (!has) continue;
        if (write_lv) {
          ++l_claim;
          st_words<W>(vis + (size_t)h * W, vh);
          st_words<W>(nxt + (size_t)h * W, nw);
          atomicOr(&fbn[h >> 5], 1u << (h & 31));
        }
#pragma unroll
        for (int k = 0; k < W; ++k) {
          u64 x = nw[k];
          while (x) {
            const int bt = __ffsll((long long)x) - 1;
            x &= x - 1;
            atomicAdd(&s_lc[64 * k + bt], 1u);
          }
        }
      }
      w_claim += l_claim;
      cta_sync();
      for (int j = tid; j < nb; j += T)
        if (s_lc[j]) {
          atomicAdd(&ctl->tot[(d + 1) % 3][j], (u64)s_lc[j]);
          s_lc[j] = 0;
        }
      ok = grid_sync(&ctl->bar, err, tns);
      if (!ok) break;
      ++d;
    }
    if (!ok) break;
    lap(2);
    (void)any_alive;
    // ---------- batch end: every lane word back to zero ----------
    if (!wrote) {
      // only the candidates and the distance-1 frontier (bitmap 1) carry
      // visited bits: clear those words, then the frontier
      if (b == 0)
        for (int j = tid; j < nb; j += T) {
          const u64 z[W] = {};
          st_words<W>(vis + (size_t)s_cand[j] * W, z);
        }
      clear_frontier<W>(vis, fbs[1], nbw, co);  // (count-only: no distance-1 claim words to clear)
      cta_sync();
      if (!grid_sync(&ctl->bar, err, tns)) break;
    }
    clear_frontier<W>(bufs[d % 3], fbs[d % 3], nbw);
    clear_frontier<W>(bufs[(d + 2) % 3], fbs[(d + 2) % 3], nbw);
    if (wrote) {
      const size_t words = (size_t)n * W;
      for (size_t i = ((size_t)b * T + tid) * 2; i < words; i += (size_t)G * T * 2) {
        if (i + 1 < words) *reinterpret_cast<ulonglong2 *>(vis + i) = make_ulonglong2(0ull, 0ull);
        else vis[i] = 0;
      }
      if (b == 0 && tid == 0) ++ctl->dense_clears;
    }
    if (b == 0 && tid == 0) ctl->best_f = bf;
    if (!grid_sync(&ctl->bar, err, tns)) break;
    lap(3);
  }
  w_scan = block_sum(w_scan, (u64 *)s_red);
  w_gath = block_sum(w_gath, (u64 *)s_red);
  w_claim = block_sum(w_claim, (u64 *)s_red);
  w_vert = block_sum(w_vert, (u64 *)s_red);
  w_visr = block_sum(w_visr, (u64 *)s_red);
  if (tid == 0) {
    atomicAdd(&ctl->bu_vertices, w_vert);
    atomicAdd(&ctl->bu_visreads, w_visr);
    atomicAdd(&ctl->bu_scanned, w_scan);
    atomicAdd(&ctl->bu_gathers, w_gath);
    atomicAdd(&ctl->bu_rows, w_claim);
  }
  if (b == 0 && tid == 0) {
    if (ctl->best_f < gctl->best_f) gctl->best_f = ctl->best_f;
    ctl->batches += w_batches;
    ctl->levels += w_levels;
    ctl->lanes += w_lanes;
    ctl->td_edges += w_td;
    for (int i = 0; i < 4; ++i) ctl->ns[i] += t_ph[i];
  }
}

static size_t round0_dyn_smem(int) { return 0; }

static const void *round0_fn(int W) {
  return W == 1 ? (const void *)k_round0_wide<1>
       : W == 2 ? (const void *)k_round0_wide<2>
       : W == 4 ? (const void *)k_round0_wide<4>
                : (const void *)k_round0_wide<8>;
}

int round0_wide_occupancy(int W, int *blocks_per_sm) {
  const void *fn = round0_fn(W);
  GC_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)round0_dyn_smem(W)));
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, fn, kR0Threads, round0_dyn_smem(W)));
  return GC_OK;
}

__global__ void k_heavy_chunks(const int32_t *__restrict__ rp, const int32_t *__restrict__ heavy,
                               const int32_t *__restrict__ nh_dev, int32_t *hcp) {
  // one CTA: hcp[i] = sum over heavy rows before i of ceil(deg / kHeavyRow)
  __shared__ int s_scan[33];
  const int nh = *nh_dev;
  int carry = 0;
  for (int base = 0; base < nh; base += blockDim.x) {
    const int i = base + threadIdx.x;
    int c = 0;
    if (i < nh) {
      const int h = heavy[i];
      c = (rp[h + 1] - rp[h] + kHeavyRow - 1) / kHeavyRow;
    }
    int total;
    const int ex = block_excl_scan(c, s_scan, &total);
    if (i < nh) hcp[i] = carry + ex;
    carry += total;
  }
  if (threadIdx.x == 0) hcp[nh] = carry;
}

// Allocate (once per handle and lane width) the lane words, bitmaps and heavy
// chunk index of the wide round-0 kernel; everything starts at zero.
static int round0_workspace(gc_graph *g, int W) {
  if (g->r0_w >= W && g->r0_vis) return GC_OK;
  if (g->r0_vis) {
    cudaFree(g->r0_vis);
    g->r0_vis = nullptr;
  }
  int32_t nh = 0;
  GC_CUDA(cudaMemcpyAsync(&nh, g->n_heavy, sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
  GC_CUDA(cudaStreamSynchronize(g->stream));
  const size_t n = (size_t)g->n, nbw = ((n + 31) / 32 + 63) & ~(size_t)63;
  const size_t words = ws_align(n * W * 8);
  const size_t bitmap = ws_align(nbw * 4);
  const size_t bytes = 4 * words + 3 * bitmap + ws_align(((size_t)nh + 1) * 4) + ws_align((size_t)nh * W * 8 + 8) +
                      ws_align(2 * n * 4) + ws_align(sizeof(R0Ctl));
  unsigned char *p = nullptr;
  cudaError_t e = cudaMalloc((void **)&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return cuda_fail(e, "cudaMalloc (round-0 lane words)");
  }
  GC_CUDA(cudaMemsetAsync(p, 0, bytes, g->stream));
  g->r0_vis = (unsigned long long *)p;
  g->r0_bytes = bytes;
  g->r0_w = W;
  g->r0_nh = nh;
  unsigned char *q = p + words;
  for (int i = 0; i < 3; ++i) {
    g->r0_buf[i] = (unsigned long long *)q;
    q += words;
  }
  for (int i = 0; i < 3; ++i) {
    g->r0_fb[i] = (uint32_t *)q;
    q += bitmap;
  }
  g->r0_hcp = (int32_t *)q;
  q += ws_align(((size_t)nh + 1) * 4);
  g->r0_hacc = (unsigned long long *)q;
  q += ws_align((size_t)nh * W * 8 + 8);
  g->r0_defer = (int32_t *)q;
  q += ws_align(2 * n * 4);
  g->r0_ctl = (R0Ctl *)q;
  ++g->launches;
  k_heavy_chunks<<<1, 1024, 0, g->stream>>>(g->rp, g->heavy, g->n_heavy, g->r0_hcp);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_round0_wide(gc_graph *g, const int32_t *list, int32_t m, long long *lgain, int W, int32_t defer_below,
                       bool count_only, int64_t timeout_ns, int32_t probe_stride) {
  if (m <= 0) return GC_OK;
  if (W != 1 && W != 2 && W != 4 && W != 8) return GC_EINVAL;
  int rc = round0_workspace(g, W);
  if (rc != GC_OK) return rc;
  // the control block: batch cursors, best farness, per-level lane totals
  GC_CUDA(cudaMemsetAsync(g->r0_ctl, 0, sizeof(R0Ctl), g->stream));
  GC_CUDA(cudaMemcpyAsync(&g->r0_ctl->best_f, &g->gctl->best_f, sizeof(long long), cudaMemcpyDeviceToDevice,
                          g->stream));
  int occ = 0;
  if ((rc = round0_wide_occupancy(W, &occ)) != GC_OK) return rc;
  const int grid = std::min(kMaxGridCtas, std::max(1, occ) * g->num_sms);
  const int32_t *rp = g->rp, *ci = g->ci, *key_list = list;
  int32_t n = g->n;
  const long long *key = g->key;
  int32_t *defer = g->r0_defer;
  R0Ctl *ctl = g->r0_ctl;
  GainCtl *gctl = g->gctl;
  // a workspace allocated for a wider W serves a narrower one: its words are
  // laid out with stride W of this launch, inside the larger buffers
  unsigned long long *vis = g->r0_vis, *b0 = g->r0_buf[0], *b1 = g->r0_buf[1], *b2 = g->r0_buf[2];
  uint32_t *f0 = g->r0_fb[0], *f1 = g->r0_fb[1], *f2 = g->r0_fb[2];
  const int32_t *heavy = g->heavy, *hcp = g->r0_hcp;
  int32_t nh = g->r0_nh;
  unsigned long long *hacc = g->r0_hacc;
  unsigned long long tns = (unsigned long long)timeout_ns;
  int32_t allow_co = count_only ? 1 : 0;
  void *args[] = {(void *)&rp,   (void *)&ci,   (void *)&n,    (void *)&key_list, (void *)&m,     (void *)&key,
                  (void *)&lgain, (void *)&defer, (void *)&ctl, (void *)&gctl,     (void *)&vis,   (void *)&b0,
                  (void *)&b1,   (void *)&b2,   (void *)&f0,   (void *)&f1,       (void *)&f2,    (void *)&heavy,
                  (void *)&nh,   (void *)&hcp,  (void *)&hacc, (void *)&defer_below, (void *)&allow_co,
                  (void *)&probe_stride, (void *)&tns};
  ++g->launches;
  GC_CUDA(cudaLaunchCooperativeKernel(round0_fn(W), dim3(grid), dim3(kR0Threads), args, round0_dyn_smem(W),
                                      g->stream));
  return GC_OK;
}

}  // namespace gc
