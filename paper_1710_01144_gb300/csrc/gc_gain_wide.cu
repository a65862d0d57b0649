// Exact marginal gains Delta(v | S) of B = 64 W candidates per batch (W = 2
// or 4 words of lane bits per vertex: 128 or 256 candidates), one CTA per
// batch.  The method is the 64-lane kernel's (gc_gain.cu): a bit-parallel,
// level-synchronous multi-source BFS from the batch's candidates, pruned at
// d_S (Sec. 4.1), in which every vertex w that a lane reaches strictly before
// d_S[w] adds d_S[w] - d(v, w) to that lane's gain (Theorem 1, Sec. 4.3).
// One scan of a frontier vertex's row serves every lane that reached it at
// the same level, so a wider word shares each scan among more candidates.
//
// Workspace record of vertex w (32 W bytes, sector aligned):
//   words [0, W)       vis: the lanes that have reached w
//   words [W, 2W)      claims of even levels
//   words [2W, 3W)     claims of odd levels
//   word 3W            flags: kTouched (w is on the touched list), kQueued0 /
//                      kQueued1 (w is on the frontier queue of an even / odd
//                      level); the rest of the record is padding
// A lane claims w at level L + 1 by setting its bit in vis with atomicOr: the
// bit was clear exactly for the lanes that reach w first here.  With several
// words per vertex no single word tells whether w is new to the batch or to
// the next frontier, so one atomicOr on the flags word decides both, once per
// claiming thread.  Expanding w at level L reads and clears its claim words of
// that level's parity and its queued flag.  Records are zero between batches:
// the batch's end clears vis and flags of every touched vertex; every claim
// word was cleared when its vertex was expanded.
//
// Candidates are taken in batches of B from a global counter by persistent
// CTAs, as in the 64-lane kernel; ragged tails run as partial batches.
#include <algorithm>

#include "gc_cta.cuh"  // GainCounters, and the helpers of gc_device.cuh

namespace gc {

namespace {

typedef unsigned long long u64;

constexpr unsigned kTouched = 1u, kQueued0 = 2u, kQueued1 = 4u;

// record of vertex v: 4 W words (W = 2: 64 bytes, W = 4: 128 bytes)
template <int W>
__device__ __forceinline__ u64 *rec_of(u64 *rec, int v) {
  return rec + (size_t)v * (4 * W);
}

template <int W>
__device__ __forceinline__ void ld_w(const u64 *p, u64 (&x)[W]) {
#pragma unroll
  for (int k = 0; k < W; k += 2) {
    const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(p + k);
    x[k] = v.x;
    x[k + 1] = v.y;
  }
}

template <int W>
__device__ __forceinline__ void st_zero(u64 *p) {
#pragma unroll
  for (int k = 0; k < W; k += 2) *reinterpret_cast<ulonglong2 *>(p + k) = make_ulonglong2(0ull, 0ull);
}

template <int W>
__device__ __forceinline__ void wide_gain_batch(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                int32_t n, const int32_t *__restrict__ dS,
                                                const int32_t *__restrict__ cand, int nl,
                                                long long *__restrict__ out, u64 *rec, int32_t *q0, int32_t *q1,
                                                int32_t *touched, GainCtl *ctl, const int32_t *__restrict__ mx,
                                                const int32_t *__restrict__ c3, GainCounters &cnt) {
  constexpr int B = 64 * W;
  constexpr int T = kGainThreads;
  __shared__ u64 s_gain[B];
  __shared__ int s_cand[B];
  __shared__ int s_off[T + 1];
  __shared__ int s_rs[T];
  __shared__ u64 s_m[W][T];
  __shared__ int s_scan[33];
  __shared__ int s_qn, s_touched;

  const int tid = threadIdx.x, lane = tid & 31;
  for (int j = tid; j < B; j += T) {
    s_gain[j] = 0;
    s_cand[j] = j < nl ? cand[j] : -1;
  }
  if (tid == 0) {
    s_qn = 0;
    s_touched = 0;
  }
  cta_sync();
  int32_t *qcur = q0, *qnxt = q1;

  // level 0: lane j reaches its candidate (a member of S reaches nothing)
  for (int j = tid; j < nl; j += T) {
    const int c = s_cand[j];
    if (c < 0 || c >= n) {
      s_cand[j] = -2;
      continue;
    }
    const int dc = dS[c];
    if (dc <= 0) continue;
    s_gain[j] = (u64)dc;
    u64 *r = rec_of<W>(rec, c);
    const u64 bit = 1ull << (j & 63);
    atomicOr(&r[j >> 6], bit);
    atomicOr(&r[W + (j >> 6)], bit);
    const unsigned old = atomicOr(reinterpret_cast<unsigned *>(&r[3 * W]), kTouched | kQueued0);
    if (!(old & kTouched)) touched[atomicAdd(&s_touched, 1)] = c;
    if (!(old & kQueued0)) qcur[atomicAdd(&s_qn, 1)] = c;
  }
  cta_sync();
  int F = s_qn;
  cta_sync();
  if (tid == 0) s_qn = 0;
  cta_sync();

  int L = 0;
  for (; F > 0; ++L) {
    const int nlev = L + 1;
    const int cw = W * (1 + (L & 1)), nw = W * (1 + ((L + 1) & 1));  // claim words of L and L + 1
    const unsigned qc = (L & 1) ? kQueued1 : kQueued0, qn = (L & 1) ? kQueued0 : kQueued1;
    for (int chunk = 0; chunk < F; chunk += T) {
      const int i = chunk + tid;
      int deg = 0, rs = 0;
      u64 m[W];
#pragma unroll
      for (int k = 0; k < W; ++k) m[k] = 0;
      if (i < F) {
        const int u = qcur[i];
        u64 *r = rec_of<W>(rec, u);
        ld_w<W>(r + cw, m);  // the lanes that reached u at level L
        st_zero<W>(r + cw);
        atomicAnd(reinterpret_cast<unsigned *>(&r[3 * W]), ~qc);
        const int r0 = __ldg(rp + u);
        const int r1 = (c3 && L > 0) ? r0 + __ldg(c3 + u) : __ldg(rp + u + 1);
        bool any = false;
        int pc = 0;
#pragma unroll
        for (int k = 0; k < W; ++k) {
          any |= m[k] != 0;
          pc += __popcll(m[k]);
        }
        // no neighbour of u can still be claimed: skip the scan
        if (mx && __ldg(mx + u) <= nlev) any = false;
        if (any) {
          rs = r0;
          deg = r1 - r0;
        } else {
#pragma unroll
          for (int k = 0; k < W; ++k) m[k] = 0;
          pc = 0;
        }
        cnt.uni += (u64)deg;
        cnt.scalar += (u64)pc * (u64)deg;
        cnt.front += any;
      }
      int total;
      const int off = block_excl_scan(deg, s_scan, &total);
      s_off[tid] = off;
      s_rs[tid] = rs;
#pragma unroll
      for (int k = 0; k < W; ++k) s_m[k][tid] = m[k];
      if (tid == T - 1) s_off[T] = total;
      cta_sync();
      // kEdgeIlp adjacency entries per thread in flight; the trip count is
      // the same for the 32 threads of a warp (the ballots below need them)
      for (int e0 = tid; e0 - lane < total; e0 += kEdgeIlp * T) {
        int w[kEdgeIlp], sl[kEdgeIlp];
#pragma unroll
        for (int q = 0; q < kEdgeIlp; ++q) {
          const int e = e0 + q * T;
          w[q] = -1;
          sl[q] = 0;
          if (e < total) {
            int lo = 0, hi = T - 1;  // largest j with s_off[j] <= e (its row is non-empty)
            while (lo < hi) {
              const int mid = (lo + hi + 1) >> 1;
              if (s_off[mid] <= e) lo = mid;
              else hi = mid - 1;
            }
            sl[q] = lo;
            w[q] = __ldg(ci + s_rs[lo] + (e - s_off[lo]));
          }
        }
        int dw[kEdgeIlp];
#pragma unroll
        for (int q = 0; q < kEdgeIlp; ++q) dw[q] = w[q] >= 0 ? __ldg(dS + w[q]) : 0;
        u64 nb[kEdgeIlp][W];
#pragma unroll
        for (int q = 0; q < kEdgeIlp; ++q) {
          // pruned unless w is strictly closer to the lane's candidate than to S
          const bool live = w[q] >= 0 && dw[q] > nlev;
          if (live) {
            // the frontier lanes of the expanded vertex, and w's visited words
            // for those of them (a pair of words per 16-byte load)
            const u64 *vw = rec_of<W>(rec, w[q]);
#pragma unroll
            for (int k = 0; k < W; k += 2) {
              const u64 m0 = s_m[k][sl[q]], m1 = s_m[k + 1][sl[q]];
              if (m0 | m1) {
                const ulonglong2 v = *reinterpret_cast<const ulonglong2 *>(vw + k);
                nb[q][k] = m0 & ~v.x;
                nb[q][k + 1] = m1 & ~v.y;
              } else {
                nb[q][k] = 0;
                nb[q][k + 1] = 0;
              }
            }
          } else {
#pragma unroll
            for (int k = 0; k < W; ++k) nb[q][k] = 0;
          }
        }
#pragma unroll
        for (int q = 0; q < kEdgeIlp; ++q)
#pragma unroll
          for (int k = 0; k < W; ++k)
            if (nb[q][k]) nb[q][k] &= ~atomicOr(rec_of<W>(rec, w[q]) + k, nb[q][k]);  // the lanes won here
#pragma unroll
        for (int q = 0; q < kEdgeIlp; ++q) {
          bool won = false;
          int pc = 0, j1 = -1;
#pragma unroll
          for (int k = 0; k < W; ++k) {
            won |= nb[q][k] != 0;
            pc += __popcll(nb[q][k]);
            if (nb[q][k]) j1 = 64 * k + __ffsll((long long)nb[q][k]) - 1;
          }
          unsigned old = kTouched | qn;
          if (won) {
            u64 *r = rec_of<W>(rec, w[q]);
#pragma unroll
            for (int k = 0; k < W; ++k)
              if (nb[q][k]) atomicOr(r + nw + k, nb[q][k]);
            old = atomicOr(reinterpret_cast<unsigned *>(&r[3 * W]), kTouched | qn);
          }
          // touched list and next frontier: one shared-memory slot
          // reservation per warp for each
          const bool fresh = !(old & kTouched), push = !(old & qn);
          const unsigned fm = __ballot_sync(0xffffffffu, fresh), qm = __ballot_sync(0xffffffffu, push);
          int bt = 0, bq = 0;
          if (lane == 0) {
            if (fm) bt = atomicAdd(&s_touched, __popc(fm));
            if (qm) bq = atomicAdd(&s_qn, __popc(qm));
          }
          const unsigned below = (1u << lane) - 1u;
          bt = __shfl_sync(0xffffffffu, bt, 0);
          bq = __shfl_sync(0xffffffffu, bq, 0);
          if (fresh) touched[bt + __popc(fm & below)] = w[q];
          if (push) {
            qnxt[bq + __popc(qm & below)] = w[q];
            ++cnt.push;
          }
          // per-lane sums: claims of a single lane are summed over the warp's
          // threads that won the same lane, and one thread adds the sum
          const u64 wt = (u64)(dw[q] - nlev);
          const bool one = pc == 1;
          const int jj = one ? j1 : -1;
          const unsigned grp = __match_any_sync(0xffffffffu, jj);
          if (one) {
            // wt < 2^30: two 16-bit halves keep the 32-lane sums exact
            const unsigned lo = __reduce_add_sync(grp, (unsigned)(wt & 0xffffu));
            const unsigned hi = __reduce_add_sync(grp, (unsigned)(wt >> 16));
            if (lane == __ffs(grp) - 1) atomicAdd(&s_gain[jj], (u64)lo + ((u64)hi << 16));
          } else if (won) {
#pragma unroll
            for (int k = 0; k < W; ++k) {
              u64 x = nb[q][k];
              while (x) {
                const int b = __ffsll((long long)x) - 1;
                x &= x - 1;
                atomicAdd(&s_gain[64 * k + b], wt);
              }
            }
          }
        }
      }
      cta_sync();
    }
    const int Fn = s_qn;
    cta_sync();
    if (tid == 0) s_qn = 0;
    { int32_t *t = qcur; qcur = qnxt; qnxt = t; }
    F = Fn;
    cta_sync();
  }
  cnt.levels += (u64)L;
  ++cnt.batches;
  cnt.lanes += (u64)nl;

  for (int j = tid; j < nl; j += T) {
    long long r = (long long)s_gain[j];
    if (s_cand[j] == -2) {
      r = -1;
      atomicExch(&ctl->err, GC_EINVAL);
    }
    out[j] = r;
  }
  // every touched record back to zero (its claim words already are)
  const int nt = s_touched;
  for (int i = tid; i < nt; i += T) {
    u64 *r = rec_of<W>(rec, touched[i]);
    st_zero<W>(r);
    r[3 * W] = 0ull;
  }
  cta_sync();
}

// (W = 4 at two CTAs per SM spills registers and measured slower)
template <int W>
__global__ void __launch_bounds__(kGainThreads, W <= 2 ? 2 : 1)
    k_gains_wide(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n,
                 const int32_t *__restrict__ dS, const int32_t *__restrict__ cand, int32_t n_cand_arg,
                 const int32_t *__restrict__ n_cand_dev, long long *__restrict__ out, unsigned char *ws_base,
                 size_t ws_stride, GainCtl *ctl, const int32_t *__restrict__ mx, const int32_t *__restrict__ c3) {
  constexpr int B = 64 * W;
  __shared__ int s_batch;
  __shared__ u64 s_red[32];
  const int tid = threadIdx.x;
  unsigned char *p = ws_base + ws_stride * (size_t)blockIdx.x;
  const size_t arec = ws_align((size_t)n * 32 * W), a4 = ws_align((size_t)n * sizeof(int32_t));
  u64 *rec = reinterpret_cast<u64 *>(p);
  int32_t *q0 = reinterpret_cast<int32_t *>(p + arec);
  int32_t *q1 = reinterpret_cast<int32_t *>(p + arec + a4);
  int32_t *touched = reinterpret_cast<int32_t *>(p + arec + 2 * a4);
  const int n_cand = n_cand_dev ? *n_cand_dev : n_cand_arg;
  const int n_batches = (n_cand + B - 1) / B;
  GainCounters cnt;
  for (;;) {
    if (tid == 0) s_batch = (int)atomicAdd(&ctl->batch_next, 1u);
    cta_sync();
    const int b = s_batch;
    cta_sync();
    if (b >= n_batches) break;
    const int base = b * B;
    wide_gain_batch<W>(rp, ci, n, dS, cand + base, min(B, n_cand - base), out + base, rec, q0, q1, touched, ctl,
                       mx, c3, cnt);
  }
  const u64 c_scalar = block_sum(cnt.scalar, s_red);
  const u64 c_union = block_sum(cnt.uni, s_red);
  const u64 c_front = block_sum(cnt.front, s_red);
  const u64 c_push = block_sum(cnt.push, s_red);
  if (tid == 0) {
    atomicAdd(&ctl->edges_scalar, c_scalar);
    atomicAdd(&ctl->edges_union, c_union);
    atomicAdd(&ctl->levels, cnt.levels);
    atomicAdd(&ctl->batches, cnt.batches);
    atomicAdd(&ctl->frontier, c_front);
    atomicAdd(&ctl->pushes, c_push);
    atomicAdd(&ctl->lanes, cnt.lanes);
    atomicAdd(&ctl->k_front, c_front);
    atomicAdd(&ctl->k_union, c_union);
    atomicAdd(&ctl->k_push, c_push);
    atomicAdd(&ctl->k_lanes, cnt.lanes);
  }
}

}  // namespace

size_t gain_wide_ws_stride(int32_t n, int W) {
  return ws_align((size_t)n * 32 * W) + 3 * ws_align((size_t)n * sizeof(int32_t));
}

// Workspaces of the wide kernel at W words: allocated on first use (and again
// when W changes), one per resident CTA within 40% of free memory and 16 GB.
static int wide_workspace(gc_graph *g, int W) {
  if (g->x_ws && g->x_w == W) return GC_OK;
  if (g->x_ws) {  // (an earlier launch on the handle's stream may still use it)
    GC_CUDA(cudaStreamSynchronize(g->stream));
    cudaFree(g->x_ws);
    g->x_ws = nullptr;
    g->x_w = 0;
    g->x_ctas = 0;
  }
  int occ = 0;
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, W <= 2 ? k_gains_wide<2> : k_gains_wide<4>, kGainThreads, 0));
  const size_t stride = gain_wide_ws_stride(g->n, W);
  size_t free_b = 0, total_b = 0;
  GC_CUDA(cudaMemGetInfo(&free_b, &total_b));
  const size_t budget = std::min<size_t>(free_b / 10 * 4, (size_t)16 << 30);
  int want = std::max(1, occ) * g->num_sms;
  if ((size_t)want * stride > budget) want = (int)std::max<size_t>(1, budget / stride);
  if (cudaMalloc((void **)&g->x_ws, (size_t)want * stride) != cudaSuccess) {
    cudaGetLastError();
    g->x_ws = nullptr;
    set_error("workspace of the wide gain kernel: allocation failed");
    return GC_ENOMEM;
  }
  GC_CUDA(cudaMemsetAsync(g->x_ws, 0, (size_t)want * stride, g->stream));
  g->x_w = W;
  g->x_ctas = want;
  g->x_stride = stride;
  return GC_OK;
}

int launch_gains_wide(gc_graph *g, const int32_t *cand, int32_t n_cand, const int32_t *n_cand_dev,
                      long long *out, int max_ctas, bool pruned) {
  const int W = g->gain_lanes >= 256 ? 4 : 2;
  const int rc = wide_workspace(g, W);
  if (rc != GC_OK) return rc;
  GC_CUDA(cudaMemsetAsync(&g->gctl->batch_next, 0, sizeof(unsigned int), g->stream));
  int ctas = g->x_ctas;
  if (max_ctas > 0 && max_ctas < ctas) ctas = max_ctas;
  if (!n_cand_dev) {
    const int n_batches = (n_cand + 64 * W - 1) / (64 * W);
    if (ctas > n_batches) ctas = n_batches;
  }
  ++g->launches;
  const int32_t *rp = pruned ? g->rpf : g->rp, *ci = pruned ? g->cif : g->ci, *c3 = pruned ? g->c3 : nullptr;
  if (W == 2)
    k_gains_wide<2><<<ctas, kGainThreads, 0, g->stream>>>(rp, ci, g->n, g->dS, cand, n_cand, n_cand_dev, out,
                                                          g->x_ws, g->x_stride, g->gctl, g->mx, c3);
  else
    k_gains_wide<4><<<ctas, kGainThreads, 0, g->stream>>>(rp, ci, g->n, g->dS, cand, n_cand, n_cand_dev, out,
                                                          g->x_ws, g->x_stride, g->gctl, g->mx, c3);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

}  // namespace gc
