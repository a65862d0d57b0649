// Grid-wide form of the 64-lane pruned multi-source BFS (see gc_gain.cu for
// the method): ONE batch of up to 64 candidates advanced by every CTA of a
// cooperative launch, for candidates whose searches are large -- the hubs that
// survive the round-0 bound, and the top-bound candidates of a lazy step.
//
// Per level, two phases separated by bounded grid barriers:
//   1. each CTA takes a contiguous slice of the frontier, moves each entry's
//      claim word (the lanes that reached it at this level) into the mask list
//      and clears it, and scans the entries' degrees (degree 0 where no lane
//      can claim anything), giving slice-local offsets;
//   2. every CTA prefix-sums the per-CTA totals and takes an equal slice of
//      the level's adjacency entries.  It locates the first frontier entry of
//      its slice with one warp-wide search, stages the entries that cover the
//      slice in shared memory (start, row, mask) and expands them edge by edge,
//      claiming (neighbour, lane) pairs with atomicOr on the visited word as the
//      CTA-per-batch kernel does; pushes are aggregated per warp.  In farness
//      mode per-lane sums and counts of each level are folded into a buffer of
//      that distance (three, by distance mod 3); after the barrier every CTA
//      adds the same buffer to its running totals and applies the same BFScut
//      test to its copy of the live-lane mask.
// Per-lane gains accumulate in shared memory and reach global memory once per
// CTA (gain mode) or once per level (farness mode, where the cut needs them).
#include "gc_grid.cuh"

namespace gc {

template <int MODE>
__global__ void __launch_bounds__(kGridGainThreads, 2)
    k_gains_grid(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n,
                 const int32_t *__restrict__ dS, const int32_t *__restrict__ cand, int32_t nl_arg,
                 const int32_t *__restrict__ nl_dev, long long *__restrict__ out, unsigned char *ws_base,
                 int32_t *gx, int32_t *__restrict__ goff, GridGainCtl *ctl, GainCtl *gctl,
                 unsigned long long timeout_ns, const int32_t *__restrict__ mx, const int32_t *__restrict__ c3) {
  grid_gain_batch<MODE>(rp, ci, n, dS, cand, nl_arg, nl_dev, out, ws_base, gx, goff, ctl, gctl, &ctl->bar,
                        &ctl->err, timeout_ns, mx, c3);
}

int grid_gain_occupancy(int *blocks_per_sm) {
  int a = 0, c = 0;
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_gains_grid<kModeGain>, kGridGainThreads, 0));
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&c, k_gains_grid<kModeFarness>, kGridGainThreads, 0));
  *blocks_per_sm = a < c ? a : c;
  return GC_OK;
}

int launch_gains_grid(gc_graph *g, int mode, const int32_t *cand, int32_t nl, const int32_t *nl_dev,
                      long long *out, int64_t timeout_ns, bool pruned) {
  if (!nl_dev && nl <= 0) return GC_OK;
  if (nl > kLanes) return GC_EINVAL;
  GC_CUDA(cudaMemsetAsync(g->ggctl, 0, sizeof(GridGainCtl), g->stream));
  const bool pr = pruned && mode == kModeGain;
  const int32_t *rp = pr ? g->rpf : g->rp, *ci = pr ? g->cif : g->ci, *dS = g->dS;
  const int32_t *c3 = pr ? g->c3 : nullptr;
  int32_t n = g->n;
  unsigned char *ws = g->ws;
  int32_t *gx = g->gx;
  int32_t *goff = g->goff;
  GridGainCtl *ctl = g->ggctl;
  GainCtl *gctl = g->gctl;
  unsigned long long tns = (unsigned long long)timeout_ns;
  const int32_t *mx = mode == kModeGain ? g->mx : nullptr;
  void *args[] = {(void *)&rp,  (void *)&ci,   (void *)&n,   (void *)&dS,  (void *)&cand,
                  (void *)&nl,  (void *)&nl_dev, (void *)&out, (void *)&ws, (void *)&gx, (void *)&goff,
                  (void *)&ctl, (void *)&gctl, (void *)&tns, (void *)&mx, (void *)&c3};
  ++g->launches;
  if (mode == kModeGain)
    GC_CUDA(cudaLaunchCooperativeKernel((const void *)k_gains_grid<kModeGain>, dim3(g->grid_ctas),
                                        dim3(kGridGainThreads), args, 0, g->stream));
  else
    GC_CUDA(cudaLaunchCooperativeKernel((const void *)k_gains_grid<kModeFarness>, dim3(g->grid_ctas),
                                        dim3(kGridGainThreads), args, 0, g->stream));
  return GC_OK;
}

}  // namespace gc
