// Weighted graphs (positive integer edge weights): the paper's Greedy with
// every SSSP a shortest-path search instead of a BFS (Sec. 3.2: Dijkstra,
// O(kn(m + n log n))), and the pruning of Sec. 4.1, which carries over: if
// d(v, w) < d_S[w] then every vertex x on a shortest v-w path has d(v, x) <
// d_S[x] (d(v, x) = d(v, w) - d(x, w) < d_S[w] - d(x, w) <= d_S[x]), so
// relaxing only into vertices the candidate would bring strictly closer finds
// the exact distance of every vertex that contributes to the gain.
//
// One search per CTA: a frontier-based label-correcting SSSP (parallel
// Bellman-Ford).  A warp takes a frontier vertex and its row; a relaxation
// lowers dist[w] with atomicMin and, if it lowered it, puts w into the next
// frontier once (a queue flag).  A vertex lowered after its warp read it is
// queued again, so the search ends with exact distances.  Workspace per CTA:
// dist, two frontier queues, the touched list and the queue flags (20 bytes
// per vertex); dist is kInf and the flags zero between searches.
//
// Modes: kWFarness  f({v}) of each listed source (a full search),
//        kWGain     Delta(v | S) of each listed candidate against d_S,
//        kWRelabel  d_S <- min(d_S, d(s, .)) in place from one source (the
//                   d_S update), the decrease summed for the gain check.
#include <limits.h>

#include <algorithm>

#include "gc_device.cuh"
#include "gc_internal.cuh"

namespace gc {

constexpr int kWThreads = 512;

struct WWs {
  int32_t *dist, *q0, *q1, *touched;
  unsigned int *inq;
};

__device__ __forceinline__ WWs wws(unsigned char *base, size_t stride, int32_t n, int idx) {
  unsigned char *p = base + stride * (size_t)idx;
  const size_t a4 = ws_align((size_t)n * 4);
  WWs w;
  w.dist = (int32_t *)p;
  w.q0 = (int32_t *)(p + a4);
  w.q1 = (int32_t *)(p + 2 * a4);
  w.touched = (int32_t *)(p + 3 * a4);
  w.inq = (unsigned int *)(p + 4 * a4);
  return w;
}

size_t wws_stride(int32_t n) { return 5 * ws_align((size_t)n * 4); }

// One search from s by the whole CTA.  d is the distance array the search
// lowers (the workspace's dist, or d_S itself in kWRelabel); dS (kWGain) the
// group's distances the search must beat.  Returns, in every thread, the
// search's sum: farness, gain, or the decrease of d_S.  *reached (thread 0)
// gets the number of vertices the search lowered from kInf.
template <int MODE>
static __device__ long long cta_wsssp(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                      const int32_t *__restrict__ wt, int32_t *d, const int32_t *dS,
                                      const WWs &ws, int s, long long *reached) {
  __shared__ int s_F, s_nt;
  __shared__ long long s_red[32];
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
  long long acc = 0;  // kWRelabel: this thread's share of the decrease
  if (tid == 0) {
    s_nt = 0;
    const int old = d[s];
    d[s] = 0;
    if (MODE == kWRelabel && old < kInf) acc += old;
    if (MODE != kWRelabel) ws.touched[s_nt++] = s;
    ws.q0[0] = s;
    s_F = 1;
  }
  cta_sync();
  int32_t *cur = ws.q0, *nxt = ws.q1;
  for (;;) {
    const int F = s_F;
    if (F == 0) break;
    for (int i = tid; i < F; i += blockDim.x) ws.inq[cur[i]] = 0u;  // may be queued again below
    cta_sync();
    if (tid == 0) s_F = 0;
    cta_sync();
    for (int i = wid; i < F; i += nw) {
      const int u = cur[i];
      const int du = __ldcg(&d[u]);  // the latest value (a lower one requeues u)
      for (int e = rp[u] + lane; e < rp[u + 1]; e += 32) {
        const int w = ci[e];
        const int nd = du + wt[e];
        if (MODE == kWGain && nd >= dS[w]) continue;  // pruned (Sec. 4.1)
        if (nd >= __ldcg(&d[w])) continue;
        const int old = atomicMin(&d[w], nd);
        if (nd < old) {
          if (MODE == kWRelabel) {
            if (old < kInf) acc += old - nd;
          } else if (old == kInf) {
            ws.touched[atomicAdd(&s_nt, 1)] = w;
          }
          if (atomicExch(&ws.inq[w], 1u) == 0u) nxt[atomicAdd(&s_F, 1)] = w;
        }
      }
    }
    cta_sync();
    int32_t *t = cur;
    cur = nxt;
    nxt = t;
  }
  long long r = 0;
  if (MODE == kWRelabel) {
    r = acc;
  } else {
    const int nt = s_nt;
    for (int i = tid; i < nt; i += blockDim.x) {
      const int w = ws.touched[i];
      const int dw = __ldcg(&d[w]);
      r += MODE == kWFarness ? (long long)dw : (long long)(dS[w] - dw);
    }
  }
  r = block_sum(r, s_red);
  if (tid == 0 && reached) *reached = s_nt;
  if (MODE != kWRelabel) {  // the workspace back to kInf for the next search
    const int nt = s_nt;
    for (int i = tid; i < nt; i += blockDim.x) d[ws.touched[i]] = kInf;
  }
  cta_sync();
  return r;
}

// Every listed source, one CTA per search, from a task counter.  out[i]: the
// farness (-1 if the search reached fewer than n vertices: disconnected) or
// the gain (0 for a member of S).
template <int MODE>
__global__ void __launch_bounds__(kWThreads) k_wsssp(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                                                     const int32_t *__restrict__ wt, int32_t n, const int32_t *dS,
                                                     const int32_t *list, const int32_t *m_dev, long long *out,
                                                     unsigned char *ws_base, size_t ws_stride, unsigned int *task,
                                                     int32_t *err) {
  __shared__ int s_i;
  const WWs ws = wws(ws_base, ws_stride, n, blockIdx.x);
  const int m = *m_dev;
  for (;;) {
    if (threadIdx.x == 0) s_i = (int)atomicAdd(task, 1u);
    cta_sync();
    const int i = s_i;
    cta_sync();
    if (i >= m) break;
    const int s = list[i];
    if (s < 0 || s >= n) {
      if (threadIdx.x == 0) {
        out[i] = -1;
        atomicExch(err, GC_EINVAL);
      }
      continue;
    }
    if (MODE == kWGain && dS[s] == 0) {  // a member: no gain
      if (threadIdx.x == 0) out[i] = 0;
      continue;
    }
    long long reached = 0;
    const long long r = cta_wsssp<MODE>(rp, ci, wt, ws.dist, dS, ws, s, &reached);
    if (threadIdx.x == 0) {
      if (MODE == kWFarness && reached != n) {
        out[i] = -1;
        atomicExch(err, GC_EDISCONNECTED);
      } else {
        out[i] = r;
      }
    }
  }
}

// d_S update from one source by one CTA, in place; *decrease gets the sum of
// (old - new) over the lowered labels with a finite old label.
__global__ void __launch_bounds__(kWThreads) k_wrelabel(const int32_t *__restrict__ rp,
                                                        const int32_t *__restrict__ ci,
                                                        const int32_t *__restrict__ wt, int32_t *dS,
                                                        const int32_t *src, unsigned char *ws_base,
                                                        size_t ws_stride, int32_t n,
                                                        unsigned long long *decrease) {
  const WWs ws = wws(ws_base, ws_stride, n, 0);
  const long long r = cta_wsssp<kWRelabel>(rp, ci, wt, dS, nullptr, ws, *src, nullptr);
  if (threadIdx.x == 0) *decrease = (unsigned long long)r;
}

// weights: w >= 1 everywhere, the same in both rows of an edge (binary search
// of the mirror entry in its sorted row), and the largest below max_w_out
__global__ void k_wcheck(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                         const int32_t *__restrict__ wt, int32_t n, int check_mirror, int32_t *bad,
                         int32_t *max_w) {
  const int lane = threadIdx.x & 31;
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
  int mx = 0;
  for (int u = gw; u < n; u += nw) {
    for (int e = rp[u] + lane; e < rp[u + 1]; e += 32) {
      const int w = wt[e];
      mx = max(mx, w);
      bool ok = w >= 1;
      if (ok && check_mirror) {
        const int x = ci[e];
        int lo = rp[x], hi = rp[x + 1];
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (ci[mid] < u) lo = mid + 1;
          else hi = mid;
        }
        ok = lo < rp[x + 1] && ci[lo] == u && wt[lo] == w;
      }
      if (!ok) atomicExch(bad, 1);
    }
  }
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 16));
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 8));
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 4));
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 2));
  mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, 1));
  if (lane == 0 && mx) atomicMax(max_w, mx);
}

int launch_wsssp(gc_graph *g, int mode, const int32_t *list, const int32_t *m_dev, long long *out,
                 unsigned int *task) {
  GC_CUDA(cudaMemsetAsync(task, 0, sizeof(unsigned int), g->stream));
  ++g->launches;
  const int grid = g->w_ctas;
  if (mode == kWFarness)
    k_wsssp<kWFarness><<<grid, kWThreads, 0, g->stream>>>(g->rp, g->ci, g->wt, g->n, g->dS, list, m_dev, out,
                                                          g->w_ws, g->w_stride, task, &g->sctl->err);
  else
    k_wsssp<kWGain><<<grid, kWThreads, 0, g->stream>>>(g->rp, g->ci, g->wt, g->n, g->dS, list, m_dev, out,
                                                       g->w_ws, g->w_stride, task, &g->sctl->err);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_wrelabel(gc_graph *g, const int32_t *src, unsigned long long *decrease) {
  ++g->launches;
  k_wrelabel<<<1, kWThreads, 0, g->stream>>>(g->rp, g->ci, g->wt, g->dS, src, g->w_ws, g->w_stride, g->n,
                                             decrease);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_wcheck(gc_graph *g, bool mirror, int32_t *bad, int32_t *max_w) {
  ++g->launches;
  k_wcheck<<<g->num_sms * 8, 256, 0, g->stream>>>(g->rp, g->ci, g->wt, g->n, mirror ? 1 : 0, bad, max_w);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

__global__ void k_w_iota(int32_t *p, int32_t n) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) p[i] = i;
}

int launch_iota(gc_graph *g, int32_t *p, int32_t n) {
  ++g->launches;
  k_w_iota<<<g->num_sms * 4, 256, 0, g->stream>>>(p, n);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int wsssp_occupancy(int *blocks_per_sm) {
  int a = 0, b = 0;
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_wsssp<kWFarness>, kWThreads, 0));
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_wsssp<kWGain>, kWThreads, 0));
  *blocks_per_sm = std::min(a, b);
  return GC_OK;
}

}  // namespace gc
