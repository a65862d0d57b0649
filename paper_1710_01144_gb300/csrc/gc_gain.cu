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
// one thread through atomicOr on the vertex's visited word; that thread adds
// the contribution d_S[w] - (L+1) to the lane's int64 gain and records the
// lane in w's claim word of level L+1.
//
// Farness mode (round 0, top-1 closeness, Sec. 3.1 / Algorithm 3): no pruning,
// each claimed (w, lane) adds L+1 and counts one visited vertex; after every
// level a lane whose bound  sum + (L+2)(n - visited)  exceeds the best exact
// farness found so far (any CTA) is cut, as BFScut does.
//
// Layout.  One persistent CTA per workspace; a CTA takes 64-candidate batches
// from a global counter.  Per-CTA workspace in HBM: one 32-byte record of lane
// words per vertex (visited, claims of even and of odd levels; zero between
// batches), two frontier queues of vertex ids and a touched list used to zero
// the visited words after the batch.  Frontier expansion is
// edge-balanced across the CTA: a block scan of the frontier's degrees, then
// every thread takes adjacency entries at stride blockDim and finds its
// frontier slot by binary search, so hub rows and tiny rows share the work.
#include "gc_cta.cuh"

namespace gc {

size_t gain_ws_stride(int32_t n) { return gain_ws_bytes(n); }

template <int MODE>
__global__ void __launch_bounds__(kGainThreads, 2)
    k_gains64(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n,
              const int32_t *__restrict__ dS, const int32_t *__restrict__ cand, int32_t n_cand_arg,
              const int32_t *__restrict__ n_cand_dev, long long *__restrict__ out,
              unsigned char *ws_base, size_t ws_stride, GainCtl *ctl, int lanes,
              const int32_t *__restrict__ mx, const LaneGraphs lg, const int32_t *__restrict__ c3) {
  __shared__ int s_batch;
  __shared__ u64 s_red[32];
  const int tid = threadIdx.x;
  const GainWs ws = gain_ws(ws_base, ws_stride, n, blockIdx.x);
  const int n_cand = n_cand_dev ? *n_cand_dev : n_cand_arg;
  const int n_batches = (n_cand + lanes - 1) / lanes;
  GainCounters cnt;
  for (;;) {
    if (tid == 0) s_batch = (int)atomicAdd(&ctl->batch_next, 1u);
    cta_sync();
    const int b = s_batch;
    cta_sync();
    if (b >= n_batches) break;
    const int base = b * lanes;
    cta_gain_batch<MODE, true, true>(rp, ci, n, dS, cand + base, min(lanes, n_cand - base), out + base, ws, ctl, mx,
                                     lg, cnt, 0, c3);
  }
  u64 c_scalar = block_sum(cnt.scalar, s_red);
  u64 c_union = block_sum(cnt.uni, s_red);
  u64 c_front = block_sum(cnt.front, s_red);
  u64 c_push = block_sum(cnt.push, s_red);
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
                 const int32_t *n_cand_dev, long long *out, int max_ctas, int lanes, bool pruned) {
  if (!n_cand_dev && n_cand <= 0) return GC_OK;
  if (lanes < 1 || lanes > kLanes) lanes = kLanes;
  // full batches of gains at the handle's width above 64: the wide kernel
  if (mode == kModeGain && lanes == kLanes && g->gain_lanes > kLanes)
    return launch_gains_wide(g, cand, n_cand, n_cand_dev, out, max_ctas, pruned);
  GC_CUDA(cudaMemsetAsync(&g->gctl->batch_next, 0, sizeof(unsigned int), g->stream));
  int ctas = g->gain_ctas;
  if (max_ctas > 0 && max_ctas < ctas) ctas = max_ctas;
  if (!n_cand_dev) {
    const int n_batches = (n_cand + lanes - 1) / lanes;
    if (ctas > n_batches) ctas = n_batches;
  }
  ++g->launches;
  const bool pr = pruned && mode == kModeGain;
  const int32_t *rp = pr ? g->rpf : g->rp, *ci = pr ? g->cif : g->ci, *c3 = pr ? g->c3 : nullptr;
  if (mode == kModeGain)
    k_gains64<kModeGain><<<ctas, kGainThreads, 0, g->stream>>>(
        rp, ci, g->n, g->dS, cand, n_cand, n_cand_dev, out, g->ws, g->ws_stride, g->gctl, lanes, g->mx,
        LaneGraphs(), c3);
  else
    k_gains64<kModeFarness><<<ctas, kGainThreads, 0, g->stream>>>(
        g->rp, g->ci, g->n, g->dS, cand, n_cand, n_cand_dev, out, g->ws, g->ws_stride, g->gctl, lanes, nullptr,
        g->lane_graphs, nullptr);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

}  // namespace gc
