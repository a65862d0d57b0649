// The hot kernel of libgc: exact marginal gains Delta(v | S) of 64 candidates
// at once by a bit-parallel, level-synchronous, pruned multi-source BFS.
//
// Paper basis.  Sec. 4.1: the SSSP from a candidate v only needs the vertices
// w with d(v, w) < d_S[w]; a vertex that fails the test is not expanded, and
// neither is its subtree.  Sec. 4.3 / Theorem 1: Delta(v | S) =
// sum_i |b^i_v AND NOT b^i_S|, i.e. each vertex w with d(v,w) < d_S[w] adds
// d_S[w] - d(v, w).  Bit j of a 64-bit word stands for candidate j of the batch,
// so one word per vertex carries 64 BFSs; one adjacency scan serves every lane
// that reached the vertex at the same level.
//
// Pruning is lane-independent here: whether w can contribute at level L+1
// depends only on d_S[w] > L+1, so a neighbour failing it is skipped before
// any bitmask traffic; the frontier of level L only holds vertices with
// d_S > L, all of which expand.  Each (vertex, lane) pair is claimed by exactly
// one thread through atomicOr on the next-level word; that thread adds the
// contribution d_S[w] - (L+1) to the lane's int64 gain.
//
// Farness mode (round 0, top-1 closeness, Sec. 3.1 / Algorithm 3): no pruning,
// each claimed (w, lane) adds L+1 and counts one visited vertex; after every
// level a lane whose bound  sum + (L+2)(n - visited)  exceeds the best exact
// farness found so far (any CTA) is cut, as BFScut does.
//
// Layout.  One persistent CTA per workspace; a CTA takes 64-candidate batches
// from a global counter.  Per-CTA workspace in HBM: vis[n], nxt[n] (uint64
// lane words, zero between batches), two frontier queues of (vertex, word) and
// a touched list used to zero vis after the batch.  Frontier expansion is
// edge-balanced across the CTA: a block scan of the frontier's degrees, then
// every thread takes adjacency entries at stride blockDim and finds its
// frontier slot by binary search, so hub rows and tiny rows share the work.
#include "gc_device.cuh"
#include "gc_internal.cuh"

namespace gc {

typedef unsigned long long u64;

struct GainWs {
  u64 *vis, *nxt, *qm0, *qm1;
  int32_t *qv0, *qv1, *touched;
};

__host__ __device__ inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t gain_ws_stride(int32_t n) {
  return 4 * align256((size_t)n * sizeof(u64)) + 3 * align256((size_t)n * sizeof(int32_t));
}

__device__ __forceinline__ GainWs gain_ws(unsigned char *base, size_t stride, int32_t n, int idx) {
  unsigned char *p = base + stride * (size_t)idx;
  const size_t a8 = align256((size_t)n * sizeof(u64)), a4 = align256((size_t)n * sizeof(int32_t));
  GainWs w;
  w.vis = (u64 *)p;
  w.nxt = (u64 *)(p + a8);
  w.qm0 = (u64 *)(p + 2 * a8);
  w.qm1 = (u64 *)(p + 3 * a8);
  w.qv0 = (int32_t *)(p + 4 * a8);
  w.qv1 = (int32_t *)(p + 4 * a8 + a4);
  w.touched = (int32_t *)(p + 4 * a8 + 2 * a4);
  return w;
}

template <int MODE>
__global__ void __launch_bounds__(kGainThreads, 2)
    k_gains64(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n,
              const int32_t *__restrict__ dS, const int32_t *__restrict__ cand, int32_t n_cand_arg,
              const int32_t *__restrict__ n_cand_dev, long long *__restrict__ out,
              unsigned char *ws_base, size_t ws_stride, GainCtl *ctl, int lanes,
              const int32_t *__restrict__ mx) {
  constexpr int T = kGainThreads;
  __shared__ u64 s_gain[kLanes];
  __shared__ int s_cnt[kLanes];
  __shared__ int s_cand[kLanes];
  __shared__ int s_off[T + 1];
  __shared__ int s_rs[T];
  __shared__ u64 s_m[T];
  __shared__ int s_scan[33];
  __shared__ int s_batch, s_qn, s_touched;
  __shared__ u64 s_alive;
  __shared__ u64 s_red[32];

  const int tid = threadIdx.x;
  const GainWs ws = gain_ws(ws_base, ws_stride, n, blockIdx.x);
  const int n_cand = n_cand_dev ? *n_cand_dev : n_cand_arg;
  const int n_batches = (n_cand + lanes - 1) / lanes;
  u64 c_scalar = 0, c_union = 0, c_levels = 0, c_batches = 0, c_front = 0, c_push = 0, c_lanes = 0;

  for (;;) {
    if (tid == 0) s_batch = (int)atomicAdd(&ctl->batch_next, 1u);
    __syncthreads();
    const int b = s_batch;
    if (b >= n_batches) break;
    const int base = b * lanes;
    const int nl = min(lanes, n_cand - base);
    if (tid < kLanes) {
      s_gain[tid] = 0;
      s_cnt[tid] = 0;
      s_cand[tid] = tid < nl ? cand[base + tid] : -1;
    }
    if (tid == 0) {
      s_qn = 0;
      s_touched = 0;
      s_alive = nl >= kLanes ? ~0ull : ((1ull << nl) - 1ull);
    }
    __syncthreads();
    int32_t *qcur_v = ws.qv0, *qnxt_v = ws.qv1;
    u64 *qcur_m = ws.qm0, *qnxt_m = ws.qm1;

    // level 0: lane j starts at its candidate
    if (tid < nl) {
      const int c = s_cand[tid];
      const u64 bit = 1ull << tid;
      bool push = false;
      if (c < 0 || c >= n) {
        s_cand[tid] = -2;  // invalid id
        atomicAnd(&s_alive, ~bit);
      } else if (MODE == kModeGain) {
        const int dc = dS[c];
        if (dc > 0) {  // v not in S: it contributes d_S[v] - 0 and expands
          s_gain[tid] = (u64)dc;
          push = true;
        }
      } else {
        s_cnt[tid] = 1;
        push = true;
      }
      if (push) {
        const u64 old = atomicOr(&ws.nxt[c], bit);
        if (old == 0) qnxt_v[atomicAdd(&s_qn, 1)] = c;
      }
    }
    __syncthreads();
    int F = s_qn;
    for (int i = tid; i < F; i += T) {  // commit level 0
      const int w = qnxt_v[i];
      const u64 m = ws.nxt[w];
      ws.nxt[w] = 0;
      ws.vis[w] = m;
      ws.touched[atomicAdd(&s_touched, 1)] = w;
      qnxt_m[i] = m;
    }
    __syncthreads();
    if (tid == 0) s_qn = 0;
    { int32_t *t = qcur_v; qcur_v = qnxt_v; qnxt_v = t; }
    { u64 *t = qcur_m; qcur_m = qnxt_m; qnxt_m = t; }
    __syncthreads();

    int L = 0;
    for (; F > 0; ++L) {
      const int nlev = L + 1;
      // ---- expand level L into level L+1 ----
      for (int chunk = 0; chunk < F; chunk += T) {
        const int i = chunk + tid;
        int deg = 0, rs = 0;
        u64 m = 0;
        if (i < F) {
          const int u = qcur_v[i];
          m = qcur_m[i];
          if (MODE == kModeFarness) m &= s_alive;
          // no neighbour of u can still be claimed: skip the scan
          if (MODE == kModeGain && mx && mx[u] <= nlev) m = 0;
          if (m) {
            rs = rp[u];
            deg = rp[u + 1] - rs;
          }
          c_union += (u64)deg;
          c_scalar += (u64)__popcll(m) * (u64)deg;
          c_front += (m != 0);
        }
        int total;
        const int off = block_excl_scan(deg, s_scan, &total);
        s_off[tid] = off;
        s_rs[tid] = rs;
        s_m[tid] = m;
        if (tid == T - 1) s_off[T] = total;
        __syncthreads();
        for (int e = tid; e < total; e += T) {
          int lo = 0, hi = T - 1;  // largest j with s_off[j] <= e (its row is non-empty)
          while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (s_off[mid] <= e) lo = mid;
            else hi = mid - 1;
          }
          const int w = ci[s_rs[lo] + (e - s_off[lo])];
          int dw = 0;
          if (MODE == kModeGain) {
            dw = dS[w];
            if (dw <= nlev) continue;  // pruned: w cannot be strictly closer to v than to S
          }
          const u64 nb = s_m[lo] & ~ws.vis[w];
          if (!nb) continue;
          const u64 old = atomicOr(&ws.nxt[w], nb);
          u64 won = nb & ~old;
          if (won) {
            const u64 wt = MODE == kModeGain ? (u64)(dw - nlev) : (u64)nlev;
            do {
              const int j = __ffsll((long long)won) - 1;
              won &= won - 1;
              atomicAdd(&s_gain[j], wt);
              if (MODE == kModeFarness) atomicAdd(&s_cnt[j], 1);
            } while (won);
          }
          if (old == 0) {
            qnxt_v[atomicAdd(&s_qn, 1)] = w;
            ++c_push;
          }
        }
        __syncthreads();
      }
      // ---- commit level L+1: fold the claimed words into vis ----
      const int Fn = s_qn;
      for (int i = tid; i < Fn; i += T) {
        const int w = qnxt_v[i];
        const u64 m = ws.nxt[w];
        ws.nxt[w] = 0;
        const u64 ov = ws.vis[w];
        ws.vis[w] = ov | m;
        if (ov == 0) ws.touched[atomicAdd(&s_touched, 1)] = w;
        qnxt_m[i] = m;
      }
      __syncthreads();
      if (MODE == kModeFarness && tid < kLanes && ((s_alive >> tid) & 1ull)) {
        // every vertex within distance L+1 is counted; the rest are >= L+2 away
        const long long lb = (long long)s_gain[tid] + (long long)(L + 2) * (long long)(n - s_cnt[tid]);
        const long long best = *(volatile long long *)&ctl->best_f;
        if (Fn > 0 && lb > best) atomicAnd(&s_alive, ~(1ull << tid));
      }
      if (tid == 0) s_qn = 0;
      { int32_t *t = qcur_v; qcur_v = qnxt_v; qnxt_v = t; }
      { u64 *t = qcur_m; qcur_m = qnxt_m; qnxt_m = t; }
      F = Fn;
      __syncthreads();
      if (MODE == kModeFarness && s_alive == 0) break;
    }
    c_levels += (u64)L;
    ++c_batches;
    c_lanes += (u64)nl;

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
      } else if (s_cnt[tid] != n) {
        r = -1;
        atomicExch(&ctl->err, GC_EDISCONNECTED);
      } else {
        r = (long long)s_gain[tid];
        atomicMin(&ctl->best_f, r);
      }
      out[base + tid] = r;
    }
    const int nt = s_touched;
    for (int i = tid; i < nt; i += T) ws.vis[ws.touched[i]] = 0;
    __syncthreads();
  }
  c_scalar = block_sum(c_scalar, s_red);
  c_union = block_sum(c_union, s_red);
  c_front = block_sum(c_front, s_red);
  c_push = block_sum(c_push, s_red);
  if (tid == 0) {
    atomicAdd(&ctl->edges_scalar, c_scalar);
    atomicAdd(&ctl->edges_union, c_union);
    atomicAdd(&ctl->levels, c_levels);
    atomicAdd(&ctl->batches, c_batches);
    atomicAdd(&ctl->frontier, c_front);
    atomicAdd(&ctl->pushes, c_push);
    atomicAdd(&ctl->lanes, c_lanes);
  }
}

int gain_kernel_occupancy(int *blocks_per_sm) {
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_gains64<kModeGain>,
                                                        kGainThreads, 0));
  int b2 = 0;
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, k_gains64<kModeFarness>,
                                                        kGainThreads, 0));
  if (b2 < *blocks_per_sm) *blocks_per_sm = b2;
  return GC_OK;
}

int launch_gains(gc_graph *g, int mode, const int32_t *cand, int32_t n_cand,
                 const int32_t *n_cand_dev, long long *out, int max_ctas, int lanes) {
  if (!n_cand_dev && n_cand <= 0) return GC_OK;
  if (lanes < 1 || lanes > kLanes) lanes = kLanes;
  GC_CUDA(cudaMemsetAsync(&g->gctl->batch_next, 0, sizeof(unsigned int), g->stream));
  int ctas = g->gain_ctas;
  if (max_ctas > 0 && max_ctas < ctas) ctas = max_ctas;
  if (!n_cand_dev) {
    const int n_batches = (n_cand + lanes - 1) / lanes;
    if (ctas > n_batches) ctas = n_batches;
  }
  ++g->launches;
  if (mode == kModeGain)
    k_gains64<kModeGain><<<ctas, kGainThreads, 0, g->stream>>>(
        g->rp, g->ci, g->n, g->dS, cand, n_cand, n_cand_dev, out, g->ws, g->ws_stride, g->gctl, lanes, g->mx);
  else
    k_gains64<kModeFarness><<<ctas, kGainThreads, 0, g->stream>>>(
        g->rp, g->ci, g->n, g->dS, cand, n_cand, n_cand_dev, out, g->ws, g->ws_stride, g->gctl, lanes, nullptr);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

}  // namespace gc
