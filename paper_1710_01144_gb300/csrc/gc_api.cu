// C ABI of libgc (declared in include/gc.h): handle management and the host
// side of Greedy++ (Algorithm 2 with the pruned SSSP of Sec. 4.1 and the lazy
// bounds of Sec. 4.2).  The host only sequences kernels; every distance, gain,
// bound, selection and arg-reduction is computed on the device.
#include <limits.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <chrono>
#include <string>
#include <vector>

#include "gc_internal.cuh"

namespace gc {

static thread_local std::string g_last_error;

void set_error(const std::string &msg) { g_last_error = msg; }

int cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string("CUDA error in ") + what + ": " + cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? GC_ENOMEM : GC_ECUDA;
}

static int fail(int code, const std::string &msg) {
  set_error(msg);
  return code;
}

constexpr int32_t kRound0GridMax = 256;  // round-0 survivors handled by grid-wide batches
constexpr int kRound0Pivots = 8;         // round 0: at most this many pivot bounds
constexpr int32_t kShallowLevels = 32;   // round 0: wide bottom-up batches up to this BFS depth
constexpr int32_t kR1Propose = 1024;     // round 1: candidates the proposal chooses the first batch from

#define GC_TRY(expr)              \
  do {                            \
    int rc_ = (expr);             \
    if (rc_ != GC_OK) return rc_; \
  } while (0)

template <typename T>
static int dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(GC_ENOMEM, std::string("cudaMalloc of ") + std::to_string(count * sizeof(T)) +
                               " bytes failed: " + cudaGetErrorString(e));
  }
  return GC_OK;
}

static void release(gc_graph *g) {
  if (!g) return;
  if (g->owns_csr) {
    cudaFree(g->rp);
    cudaFree(g->ci);
  }
  void *dev[] = {g->dS, g->ub, g->stamp, g->key, g->f0, g->list, g->lgain, g->bq0, g->bq1,
                 g->blk, g->partial, g->hist, g->io_a, g->io_b, g->bctl, g->gctl, g->sctl,
                 g->ws, g->dec, g->ggctl, g->goff, g->lctl, g->picks, g->pgain, g->pdec, g->mx_buf,
                 g->two_hop, g->score, g->rec_count, g->akey, g->ast, g->gx, g->wsel, g->wpos, g->wgain,
                 g->lev_cnt, g->lev_C, g->lev_M, g->lev_max, g->rpf, g->cif, g->c3, g->gsel, g->heavy, g->n_heavy,
                 g->g3, g->c3s, g->r0_vis, g->wt, g->w_ws, g->clog, g->x_ws};
  for (void *p : dev)
    if (p) cudaFree(p);
  if (g->h_sctl) cudaFreeHost(g->h_sctl);
  if (g->h_gctl) cudaFreeHost(g->h_gctl);
  if (g->h_bctl) cudaFreeHost(g->h_bctl);
  if (g->h_lctl) cudaFreeHost(g->h_lctl);
  for (cudaEvent_t e : g->events) cudaEventDestroy(e);
  delete g;
}

static int64_t timeout_ns(const gc_opts *o) {
  if (o && o->timeout_us > 0) return (int64_t)o->timeout_us * 1000LL;
  const int64_t ms = (o && o->timeout_ms > 0) ? o->timeout_ms : 10000;
  return ms * 1000000LL;
}

// Events bracketing gain-kernel launches (pairs), reused across calls.
static int gain_event(gc_graph *g, size_t idx, cudaEvent_t *ev) {
  while (g->events.size() <= idx) {
    cudaEvent_t e;
    GC_CUDA(cudaEventCreate(&e));
    g->events.push_back(e);
  }
  *ev = g->events[idx];
  return GC_OK;
}

static int sync(gc_graph *g) {
  GC_CUDA(cudaStreamSynchronize(g->stream));
  return GC_OK;
}

static int read_ctl(gc_graph *g) {
  GC_CUDA(cudaMemcpyAsync(g->h_sctl, g->sctl, sizeof(SelCtl), cudaMemcpyDeviceToHost, g->stream));
  GC_CUDA(cudaMemcpyAsync(g->h_gctl, g->gctl, sizeof(GainCtl), cudaMemcpyDeviceToHost, g->stream));
  GC_CUDA(cudaMemcpyAsync(g->h_bctl, g->bctl, sizeof(BfsCtl), cudaMemcpyDeviceToHost, g->stream));
  return sync(g);
}

static int device_errors(gc_graph *g) {
  const int e = g->h_gctl->err ? g->h_gctl->err : g->h_bctl->err ? g->h_bctl->err : g->h_sctl->err;
  if (!e) return GC_OK;
  // a kernel that gave up may have left lane words and selection histograms
  // behind: clear every scratch that must be zero at rest
  cudaMemsetAsync(g->ws, 0, (size_t)g->ws_count * g->ws_stride, g->stream);
  cudaMemsetAsync(g->gctl, 0, sizeof(GainCtl), g->stream);
  if (g->gsel) cudaMemsetAsync(g->gsel, 0, sizeof(GridSelScratch), g->stream);
  if (g->r0_vis) {  // the wide round-0 kernel's words: reallocated (zeroed) on next use
    cudaStreamSynchronize(g->stream);
    cudaFree(g->r0_vis);
    g->r0_vis = nullptr;
    g->r0_w = 0;
  }
  cudaStreamSynchronize(g->stream);
  std::string what = e == GC_ETIMEOUT ? "device-side wait timed out"
                     : e == GC_EDISCONNECTED ? "graph is disconnected"
                     : e == GC_EINVAL ? "invalid vertex id on the device"
                                      : "device-side consistency check failed";
  if (e == GC_EDISCONNECTED && g->h_gctl->err == GC_EDISCONNECTED)
    what += ": the search from vertex " + std::to_string(g->h_gctl->short_vertex) + " reached " +
            std::to_string(g->h_gctl->short_count) + " of " + std::to_string(g->n) + " vertices";
  return fail(e, what);
}

// d_S <- BFS from the device array seeds[0..n_seeds); checks connectivity.
static int distances_from(gc_graph *g, const int32_t *seeds_dev, int32_t n_seeds, int64_t tns,
                          int64_t *farness) {
  GC_TRY(launch_fill_i32(g, g->dS, kInf, g->n));
  GC_TRY(launch_bfs_relabel(g, g->dS, seeds_dev, n_seeds, tns));
  GC_TRY(launch_sum_dist(g, g->dS));
  GC_TRY(read_ctl(g));
  if (g->h_bctl->err) return device_errors(g);
  if (g->h_sctl->count != 0)
    return fail(GC_EDISCONNECTED, "graph is disconnected: the BFS from " + std::to_string(n_seeds) +
                                      " seed(s) left " + std::to_string(g->h_sctl->count) + " of " +
                                      std::to_string(g->n) + " vertices unreached");
  if (farness) *farness = g->h_sctl->sum;
  return GC_OK;
}

static int check_ids(const gc_graph *g, const int32_t *a, int32_t len, const char *what) {
  for (int32_t i = 0; i < len; ++i)
    if (a[i] < 0 || a[i] >= g->n)
      return fail(GC_EINVAL, std::string(what) + " holds a vertex id outside [0, n)");
  return GC_OK;
}

}  // namespace gc

using namespace gc;

extern "C" {

int gc_opts_default(gc_opts *o) {
  if (!o) return fail(GC_EINVAL, "opts is NULL");
  memset(o, 0, sizeof(*o));
  o->timeout_ms = 10000;
  return GC_OK;
}

const char *gc_last_error(void) { return g_last_error.c_str(); }

int64_t gc_num_vertices(const gc_graph *g) { return g ? g->n : -1; }
int64_t gc_num_entries(const gc_graph *g) { return g ? g->nnz : -1; }

int gc_free(gc_graph *g) {
  if (g) {
    cudaStreamSynchronize(g->stream);
    release(g);
  }
  return GC_OK;
}

int gc_load_csr(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, uint32_t flags,
                void *stream, gc_graph **out) {
  if (!out) return fail(GC_EINVAL, "out is NULL");
  *out = nullptr;
  if (n < 1 || !row_ptr) return fail(GC_EINVAL, "n < 1 or row_ptr is NULL");
  if ((flags & GC_ADOPT) && !(flags & GC_DEVICE_PTRS))
    return fail(GC_EINVAL, "GC_ADOPT requires GC_DEVICE_PTRS");
  const bool dev = flags & GC_DEVICE_PTRS;
  cudaStream_t st = (cudaStream_t)stream;
  int32_t ends[2];
  if (dev) {
    GC_CUDA(cudaMemcpyAsync(&ends[0], row_ptr, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GC_CUDA(cudaMemcpyAsync(&ends[1], row_ptr + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    GC_CUDA(cudaStreamSynchronize(st));
  } else {
    ends[0] = row_ptr[0];
    ends[1] = row_ptr[n];
  }
  if (ends[0] != 0) return fail(GC_EINVAL, "row_ptr[0] != 0");
  if (ends[1] < 0) return fail(GC_ERANGE, "row_ptr[n] is negative (nnz out of int32 range)");
  const int64_t nnz = ends[1];
  if (nnz > 0 && !col_idx) return fail(GC_EINVAL, "col_idx is NULL");
  if (!dev) {  // host arrays: check monotone row_ptr and id range here, cheaply
    if (flags & GC_VALIDATE)
      for (int32_t i = 0; i < n; ++i)
        if (row_ptr[i + 1] < row_ptr[i]) return fail(GC_EINVAL, "row_ptr is not monotone");
  }

  gc_graph *g = new gc_graph();
  g->n = n;
  g->nnz = nnz;
  g->stream = st;
  int rc = GC_OK;
  auto bail = [&](int code) {
    release(g);
    return code;
  };
  if (cudaGetDevice(&g->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess)
    return bail(fail(GC_ECUDA, "no CUDA device"));
  // CSR
  if (flags & GC_ADOPT) {
    g->owns_csr = false;
    g->rp = const_cast<int32_t *>(row_ptr);
    g->ci = const_cast<int32_t *>(col_idx);
  } else {
    if ((rc = dalloc(&g->rp, (size_t)n + 1)) || (rc = dalloc(&g->ci, (size_t)nnz))) return bail(rc);
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (cudaMemcpyAsync(g->rp, row_ptr, ((size_t)n + 1) * sizeof(int32_t), kind, st) != cudaSuccess ||
        (nnz && cudaMemcpyAsync(g->ci, col_idx, (size_t)nnz * sizeof(int32_t), kind, st) != cudaSuccess))
      return bail(fail(GC_ECUDA, "copy of the CSR failed"));
  }
  // launch geometry
  int occ = 0;
  if ((rc = gain_kernel_occupancy(&occ))) return bail(rc);
  g->gain_ctas = std::max(1, occ) * g->num_sms;
  if ((rc = bfs_kernel_occupancy(&occ))) return bail(rc);
  g->bfs_ctas = std::max(1, occ) * g->num_sms;
  if ((rc = grid_gain_occupancy(&occ))) return bail(rc);
  g->grid_ctas = std::min(kMaxGridCtas, std::max(1, occ) * g->num_sms);
  // persistent lazy kernel: one CTA per SM (its steps are short and barrier
  // bound; a second CTA per SM measured slower on R-MAT and grid graphs)
  if ((rc = lazy_occupancy(&occ))) return bail(rc);
  g->lazy_ctas = std::min(kMaxGridCtas, std::min(std::max(1, occ), 1) * g->num_sms);
  g->wcap = (int32_t)std::min<long long>((long long)n, (long long)g->lazy_ctas * kLanes);
  g->red_blocks = g->num_sms * 4;
  // per-vertex arrays
  const size_t N = (size_t)n;
  if ((rc = dalloc(&g->dS, N)) || (rc = dalloc(&g->ub, N)) || (rc = dalloc(&g->stamp, N)) ||
      (rc = dalloc(&g->key, N)) || (rc = dalloc(&g->f0, N)) || (rc = dalloc(&g->list, N)) ||
      (rc = dalloc(&g->lgain, N)) || (rc = dalloc(&g->bq0, N)) || (rc = dalloc(&g->bq1, N)) ||
      (rc = dalloc(&g->io_a, N)) || (rc = dalloc(&g->io_b, N)) ||
      (rc = dalloc(&g->blk, (size_t)g->red_blocks + 8)) ||
      (rc = dalloc(&g->partial, 3 * (size_t)g->red_blocks + 8)) ||
      (rc = dalloc(&g->hist, (size_t)kHistBins)) || (rc = dalloc(&g->bctl, 1)) ||
      (rc = dalloc(&g->gctl, 1)) || (rc = dalloc(&g->sctl, 1)) || (rc = dalloc(&g->ggctl, 1)) ||
      (rc = dalloc(&g->goff, N + 1)) || (rc = dalloc(&g->lctl, 1)) || (rc = dalloc(&g->picks, N)) ||
      (rc = dalloc(&g->pgain, N)) || (rc = dalloc(&g->pdec, N)) ||
      (rc = dalloc(&g->mx_buf, N)) || (rc = dalloc(&g->two_hop, N)) || (rc = dalloc(&g->score, N)) ||
      (rc = dalloc(&g->akey, N)) || (rc = dalloc(&g->ast, N)) || (rc = dalloc(&g->gx, 3 * N)) ||
      (rc = dalloc(&g->rpf, N + 1)) || (rc = dalloc(&g->cif, std::max<size_t>(1, (size_t)nnz))) ||
      (rc = dalloc(&g->c3, N)) || (rc = dalloc(&g->lev_cnt, N)) || (rc = dalloc(&g->heavy, N)) ||
      (rc = dalloc(&g->n_heavy, 1)) || (rc = dalloc(&g->lev_C, N + 1)) || (rc = dalloc(&g->lev_M, N + 1)) ||
      (rc = dalloc(&g->lev_max, 1)) || (rc = dalloc(&g->gsel, 1)) || (rc = dalloc(&g->g3, 1)) ||
      (rc = dalloc(&g->c3s, N)) ||
      (rc = dalloc(&g->wsel, (size_t)g->wcap)) || (rc = dalloc(&g->wpos, (size_t)g->wcap)) ||
      (rc = dalloc(&g->wgain, (size_t)g->wcap)) ||
      (rc = dalloc(&g->rec_count, 1)))
    return bail(rc);
  // claim log of the persistent lazy kernel: 2n entries (16 bytes each),
  // at least 2^20 and at most 2^24; a round that outgrows it falls back to the
  // relabel BFS for its d_S update
  g->clog_cap = std::min<long long>(1ll << 24, std::max<long long>(1ll << 20, 2ll * n));
  if ((rc = dalloc(&g->clog, (size_t)g->clog_cap))) return bail(rc);
  if (cudaMallocHost((void **)&g->h_sctl, sizeof(SelCtl)) != cudaSuccess ||
      cudaMallocHost((void **)&g->h_gctl, sizeof(GainCtl)) != cudaSuccess ||
      cudaMallocHost((void **)&g->h_bctl, sizeof(BfsCtl)) != cudaSuccess ||
      cudaMallocHost((void **)&g->h_lctl, sizeof(LazyCtl)) != cudaSuccess)
    return bail(fail(GC_ENOMEM, "pinned host allocation failed"));
  // gain-kernel workspaces: one per resident CTA, within 40% of free memory
  // and 16 GB (large shallow graphs use the wide round-0 kernel, not these)
  g->ws_stride = gain_ws_stride(n);
  size_t free_b = 0, total_b = 0;
  if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) return bail(fail(GC_ECUDA, "cudaMemGetInfo"));
  const size_t budget = std::min<size_t>(free_b / 10 * 4, (size_t)16 << 30);
  int want = g->gain_ctas;
  if ((size_t)want * g->ws_stride > budget) want = (int)std::max<size_t>(1, budget / g->ws_stride);
  g->gain_ctas = want;
  g->ws_count = want;
  if ((rc = dalloc(&g->ws, (size_t)want * g->ws_stride))) return bail(rc);
  if (cudaMemsetAsync(g->ws, 0, (size_t)want * g->ws_stride, st) != cudaSuccess ||
      cudaMemsetAsync(g->hist, 0, kHistBins * sizeof(unsigned int), st) != cudaSuccess ||
      cudaMemsetAsync(g->lev_cnt, 0, N * sizeof(unsigned long long), st) != cudaSuccess ||
      cudaMemsetAsync(g->gsel, 0, sizeof(GridSelScratch), st) != cudaSuccess ||
      cudaMemsetAsync(g->sctl, 0, sizeof(SelCtl), st) != cudaSuccess ||
      cudaMemsetAsync(g->gctl, 0, sizeof(GainCtl), st) != cudaSuccess)
    return bail(fail(GC_ECUDA, "memset failed"));
  if ((rc = launch_heavy_rows(g))) return bail(rc);
  if (flags & GC_VALIDATE) {
    if ((rc = launch_validate(g))) return bail(rc == GC_EINVAL ? fail(GC_EINVAL, "CSR validation failed") : rc);
    int32_t zero = 0;
    if ((rc = dalloc(&g->dec, 1))) return bail(rc);
    cudaMemcpy(g->dec, &zero, sizeof(int32_t), cudaMemcpyHostToDevice);
    int64_t f;
    rc = distances_from(g, g->dec, 1, 10000000000LL, &f);
    cudaFree(g->dec);
    g->dec = nullptr;
    if (rc) return bail(rc);
  }
  if (cudaStreamSynchronize(st) != cudaSuccess) return bail(fail(GC_ECUDA, "load failed"));
  *out = g;
  return GC_OK;
}

int gc_group_farness(gc_graph *g, const int32_t *S, int32_t s_len, int64_t *out_farness) {
  if (!g || !S || !out_farness || s_len < 1 || s_len > g->n)
    return fail(GC_EINVAL, "bad argument to gc_group_farness");
  GC_TRY(check_ids(g, S, s_len, "S"));
  GC_CUDA(cudaMemcpyAsync(g->io_a, S, (size_t)s_len * sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
  GC_CUDA(cudaMemsetAsync(g->bctl, 0, sizeof(BfsCtl), g->stream));
  return distances_from(g, g->io_a, s_len, timeout_ns(nullptr), out_farness);
}

static int gains_core(gc_graph *g, const int32_t *S_dev, int32_t s_len, const int32_t *cand_dev,
                      int32_t n_cand, long long *out_dev, bool check) {
  g->mx = nullptr;  // a fresh d_S: no neighbour bound
  GC_CUDA(cudaMemsetAsync(g->gctl, 0, sizeof(GainCtl), g->stream));
  if (check) {
    GC_TRY(distances_from(g, S_dev, s_len, timeout_ns(nullptr), nullptr));
  } else {
    GC_TRY(launch_fill_i32(g, g->dS, kInf, g->n));
    GC_TRY(launch_bfs_relabel(g, g->dS, S_dev, s_len, timeout_ns(nullptr)));
  }
  return launch_gains(g, kModeGain, cand_dev, n_cand, nullptr, out_dev, 0);
}

int gc_marginal_gains(gc_graph *g, const int32_t *S, int32_t s_len, const int32_t *cand,
                      int32_t n_cand, int64_t *out_gain, gc_stats *stats) {
  if (!g || !S || s_len < 1 || s_len > g->n || n_cand < 0 || (n_cand > 0 && (!cand || !out_gain)))
    return fail(GC_EINVAL, "bad argument to gc_marginal_gains");
  GC_TRY(check_ids(g, S, s_len, "S"));
  GC_TRY(check_ids(g, cand, n_cand, "cand"));
  g->mx = nullptr;  // a fresh d_S: no neighbour bound
  auto t0 = std::chrono::steady_clock::now();
  const int64_t launches0 = g->launches;
  GC_CUDA(cudaMemcpyAsync(g->io_a, S, (size_t)s_len * sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
  GC_CUDA(cudaMemsetAsync(g->gctl, 0, sizeof(GainCtl), g->stream));
  GC_TRY(distances_from(g, g->io_a, s_len, timeout_ns(nullptr), nullptr));
  float ms_k = 0.f;
  int64_t launches = 0;
  for (int32_t off = 0; off < n_cand; off += g->n) {
    const int32_t len = std::min<int32_t>(g->n, n_cand - off);
    GC_CUDA(cudaMemcpyAsync(g->list, cand + off, (size_t)len * sizeof(int32_t), cudaMemcpyHostToDevice,
                            g->stream));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GC_TRY(gain_event(g, 0, &e0));
    GC_TRY(gain_event(g, 1, &e1));
    GC_CUDA(cudaEventRecord(e0, g->stream));
    GC_TRY(launch_gains(g, kModeGain, g->list, len, nullptr, g->lgain, 0));
    GC_CUDA(cudaEventRecord(e1, g->stream));
    GC_CUDA(cudaMemcpyAsync(out_gain + off, g->lgain, (size_t)len * sizeof(long long),
                            cudaMemcpyDeviceToHost, g->stream));
    GC_TRY(sync(g));
    float ms = 0.f;
    GC_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    ms_k += ms;
    ++launches;
  }
  GC_TRY(read_ctl(g));
  GC_TRY(device_errors(g));
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->evals = n_cand;
    stats->batches = (int64_t)g->h_gctl->batches;
    stats->edges_scalar = (int64_t)g->h_gctl->edges_scalar;
    stats->edges_union = (int64_t)g->h_gctl->edges_union;
    stats->levels = (int64_t)g->h_gctl->levels;
    stats->frontier = (int64_t)g->h_gctl->frontier;
    stats->pushes = (int64_t)g->h_gctl->pushes;
    stats->lanes = (int64_t)g->h_gctl->lanes;
    stats->ms_gain_kernel = ms_k;
    stats->gain_launches = launches;
    stats->kernel_launches = g->launches - launches0;
    stats->ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return GC_OK;
}

int gc_set_gain_lanes(gc_graph *g, int32_t lanes) {
  if (!g || (lanes != 64 && lanes != 128 && lanes != 256))
    return fail(GC_EINVAL, "gc_set_gain_lanes: lanes must be 64, 128 or 256");
  g->gain_lanes = lanes;
  return GC_OK;
}

int gc_marginal_gains_device(gc_graph *g, const int32_t *S_dev, int32_t s_len, const int32_t *cand_dev,
                             int32_t n_cand, int64_t *out_gain_dev) {
  if (!g || !S_dev || s_len < 1 || n_cand < 0 || (n_cand > 0 && (!cand_dev || !out_gain_dev)))
    return fail(GC_EINVAL, "bad argument to gc_marginal_gains_device");
  return gains_core(g, S_dev, s_len, cand_dev, n_cand, (long long *)out_gain_dev, false);
}

int gc_gain_upper_bounds(gc_graph *g, const int32_t *S, int32_t s_len, int64_t *out_ub) {
  if (!g || !S || !out_ub || s_len < 1 || s_len > g->n) return fail(GC_EINVAL, "bad argument to gc_gain_upper_bounds");
  GC_TRY(check_ids(g, S, s_len, "S"));
  g->mx = nullptr;
  // S goes to io_b: the pruned-adjacency build uses io_a as scratch
  GC_CUDA(cudaMemcpyAsync(g->io_b, S, (size_t)s_len * sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
  // pruned rows from the distances of S[0] alone: every group containing S[0]
  // has d_S <= d(S[0], .), so the rows keep every neighbour it can still use
  GC_TRY(distances_from(g, g->io_b, 1, timeout_ns(nullptr), nullptr));
  GC_TRY(launch_prune_csr(g));
  if (s_len == 1) {
    GC_TRY(launch_round1_bound(g));
  } else {
    GC_TRY(distances_from(g, g->io_b, s_len, timeout_ns(nullptr), nullptr));
    GC_TRY(launch_init_ub(g));
    GC_TRY(launch_bound_refresh(g));
  }
  GC_CUDA(cudaMemcpyAsync(out_ub, g->ub, (size_t)g->n * sizeof(long long), cudaMemcpyDeviceToHost, g->stream));
  GC_TRY(sync(g));
  return GC_OK;
}

// Top-k closeness (Sec. 3.1, Algorithm 3 with general k): the k vertices of
// smallest farness f({v}), ordered by (farness, id).  The round-0 machinery of
// gc_greedy with one change: the BFScut threshold is fixed at an upper bound
// T of the k-th smallest farness instead of following the best farness found.
//   1. lower bounds LB(v) (the round-0 keys); one BFS from the vertex of
//      smallest bound, whose depth picks the search path and whose levels
//      tighten the bounds of deep graphs (pivot bound);
//   2. probes: at least k vertices of smallest bound, searched to the end;
//      T = the k-th smallest of their farness values (>= the true k-th);
//   3. every other vertex with LB(v) <= T, searched with the cut fixed at T:
//      a vertex of the true top k has LB <= f <= T, so it is never cut;
//   4. the k smallest (farness, id) among the vertices searched exactly.
int gc_top_closeness(gc_graph *g, int32_t k, const gc_opts *opts_in, int32_t *out_ids, int64_t *out_farness,
                     gc_stats *stats) {
  if (!g || !out_ids || !out_farness || k < 1 || k > g->n)
    return fail(GC_EINVAL, "bad argument to gc_top_closeness (need 1 <= k <= n)");
  gc_opts opts;
  if (opts_in) opts = *opts_in;
  else gc_opts_default(&opts);
  const int64_t tns = timeout_ns(&opts);
  auto t0 = std::chrono::steady_clock::now();
  const int64_t launches0 = g->launches;
  g->mx = nullptr;
  GC_CUDA(cudaMemsetAsync(g->sctl, 0, sizeof(SelCtl), g->stream));
  GC_CUDA(cudaMemsetAsync(g->gctl, 0, sizeof(GainCtl), g->stream));
  GC_CUDA(cudaMemsetAsync(g->bctl, 0, sizeof(BfsCtl), g->stream));
  GC_TRY(launch_fill_i64(g, g->f0, -1, g->n));
  GC_TRY(launch_round0_keys(g));
  GC_TRY(launch_argmin_lb(g));
  GC_TRY(distances_from(g, &g->sctl->arg_id, 1, tns, nullptr));
  const int32_t ecc = g->h_bctl->levels;
  if (ecc > kShallowLevels) GC_TRY(launch_pivot_bound(g));
  // 2. probes, searched with no cut (threshold +infinity, kept fixed)
  struct {
    long long best_f;
    int32_t fixed;
  } thr = {LLONG_MAX, 1};
  GC_CUDA(cudaMemcpyAsync(&g->gctl->best_f, &thr.best_f, sizeof(long long), cudaMemcpyHostToDevice, g->stream));
  GC_CUDA(cudaMemcpyAsync(&g->gctl->fixed_best, &thr.fixed, sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
  GC_TRY(launch_select(g, kSelKey, 0, k, kTauHistogram, 0));
  GC_TRY(read_ctl(g));
  const int32_t n_probe = std::min<int32_t>(g->h_sctl->n_sel, (k + kLanes - 1) / kLanes * kLanes);
  if (n_probe < k) return fail(GC_EINTERNAL, "top-k closeness: fewer probes than k");
  GC_TRY(launch_clamp_nsel(g, n_probe));
  if (n_probe <= kRound0GridMax) {
    for (int32_t off = 0; off < n_probe; off += kLanes)
      GC_TRY(launch_gains_grid(g, kModeFarness, g->list + off, std::min<int32_t>(kLanes, n_probe - off), nullptr,
                               g->lgain + off, tns, false));
  } else {
    GC_TRY(launch_gains(g, kModeFarness, g->list, n_probe, nullptr, g->lgain, opts.max_ctas, kLanes, false));
  }
  GC_TRY(launch_after_eval(g, 0, 0));
  std::vector<long long> pf(n_probe);
  GC_CUDA(cudaMemcpyAsync(pf.data(), g->lgain, (size_t)n_probe * sizeof(long long), cudaMemcpyDeviceToHost,
                          g->stream));
  GC_TRY(read_ctl(g));
  GC_TRY(device_errors(g));
  std::sort(pf.begin(), pf.end());
  if (pf[0] < 0) return fail(GC_EINTERNAL, "top-k closeness: a probe search did not complete");
  const long long T = pf[k - 1];
  // 3. every vertex whose bound reaches at most T, cut at T (fixed)
  thr.best_f = T;
  GC_CUDA(cudaMemcpyAsync(&g->gctl->best_f, &thr.best_f, sizeof(long long), cudaMemcpyHostToDevice, g->stream));
  GC_TRY(launch_select(g, kSelKey, 0, 0, kTauHost, -T));
  GC_TRY(read_ctl(g));
  const int32_t n_surv = g->h_sctl->n_sel;
  int r0_w = 0;
  if (n_surv > 0 && opts.round0_lanes >= 0 && ecc <= kShallowLevels) {
    const int want = opts.round0_lanes > 0 ? opts.round0_lanes : (n_surv > 128 ? 256 : n_surv > 64 ? 128 : 64);
    r0_w = want >= 512 ? 8 : want >= 256 ? 4 : want >= 128 ? 2 : 1;
    if (opts.round0_lanes == 0) {  // the same choice as round 0 of gc_greedy
      GC_TRY(launch_sum_two_hop(g, (unsigned long long *)g->g3));
      unsigned long long two_hop_sum = 0;
      GC_CUDA(cudaMemcpyAsync(&two_hop_sum, g->g3, sizeof(two_hop_sum), cudaMemcpyDeviceToHost, g->stream));
      GC_TRY(sync(g));
      const double passes = std::ceil((double)n_surv / (64.0 * r0_w));
      if ((double)two_hop_sum < passes * (double)g->nnz) r0_w = 0;
    }
  }
  float ms_wide = 0.f;
  if (n_surv > 0) {
    if (r0_w > 0) {
      cudaEvent_t e0 = nullptr, e1 = nullptr;
      GC_TRY(gain_event(g, 0, &e0));
      GC_TRY(gain_event(g, 1, &e1));
      GC_CUDA(cudaEventRecord(e0, g->stream));
      GC_TRY(launch_round0_wide(g, g->list, n_surv, g->lgain, r0_w, 8 * r0_w,
                                !(opts.flags & GC_OPT_R0_FULL_LEVELS), tns,
                                (opts.flags & GC_OPT_R0_NO_PROBE) ? 0 : kR0ProbeStride));
      GC_CUDA(cudaEventRecord(e1, g->stream));
      GC_TRY(sync(g));
      GC_CUDA(cudaEventElapsedTime(&ms_wide, e0, e1));
    } else if (n_surv <= kRound0GridMax) {
      for (int32_t off = 0; off < n_surv; off += kLanes)
        GC_TRY(launch_gains_grid(g, kModeFarness, g->list + off, std::min<int32_t>(kLanes, n_surv - off), nullptr,
                                 g->lgain + off, tns, false));
    } else {
      GC_TRY(launch_gains(g, kModeFarness, g->list, n_surv, nullptr, g->lgain, opts.max_ctas, kLanes, false));
    }
    GC_TRY(launch_after_eval(g, 0, 0));
  }
  GC_TRY(read_ctl(g));
  GC_TRY(device_errors(g));
  // 4. the k smallest (farness, id): every vertex at or below the selection
  // threshold, then sorted here (ties at the threshold add a few entries)
  GC_TRY(launch_topk_keys(g));
  GC_TRY(launch_select(g, kSelKey, 0, k, kTauHistogram, 0));
  GC_TRY(launch_gather_f0(g));
  GC_TRY(read_ctl(g));
  const int32_t m = g->h_sctl->n_sel;
  if (m < k) return fail(GC_EINTERNAL, "top-k closeness: fewer exact results than k");
  std::vector<int32_t> ids(m);
  std::vector<long long> fs(m);
  GC_CUDA(cudaMemcpyAsync(ids.data(), g->list, (size_t)m * sizeof(int32_t), cudaMemcpyDeviceToHost, g->stream));
  GC_CUDA(cudaMemcpyAsync(fs.data(), g->lgain, (size_t)m * sizeof(long long), cudaMemcpyDeviceToHost, g->stream));
  GC_TRY(sync(g));
  std::vector<int32_t> ord(m);
  for (int32_t i = 0; i < m; ++i) ord[i] = i;
  std::sort(ord.begin(), ord.end(), [&](int32_t a, int32_t b) {
    return fs[a] < fs[b] || (fs[a] == fs[b] && ids[a] < ids[b]);
  });
  for (int32_t i = 0; i < k; ++i) {
    out_ids[i] = ids[ord[i]];
    out_farness[i] = fs[ord[i]];
  }
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->round0_evals = (int64_t)n_probe + n_surv;
    stats->batches = (int64_t)g->h_gctl->batches;
    stats->edges_union = (int64_t)g->h_gctl->edges_union;
    stats->levels = (int64_t)g->h_gctl->levels;
    stats->lanes = (int64_t)g->h_gctl->lanes;
    stats->ms_round0_wide = ms_wide;
    stats->r0_width = r0_w * 64;
    stats->kernel_launches = g->launches - launches0;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    stats->ms_round0 = stats->ms_total;
  }
  return GC_OK;
}

// Edge weights for the weighted entry points (gc_weighted.cu).  Checked on the
// device: every weight >= 1, the same in both rows of an edge (with
// GC_VALIDATE), and (n - 1) * max weight below kInf, so that no path length
// can overflow the int32 distances.
int gc_set_weights(gc_graph *g, const int32_t *weights, uint32_t flags) {
  if (!g || (g->nnz > 0 && !weights)) return fail(GC_EINVAL, "bad argument to gc_set_weights");
  if (!g->wt && g->nnz > 0) {
    int rc = dalloc(&g->wt, (size_t)g->nnz);
    if (rc) return rc;
  }
  if (g->nnz == 0) return GC_OK;
  const cudaMemcpyKind kind = (flags & GC_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  GC_CUDA(cudaMemcpyAsync(g->wt, weights, (size_t)g->nnz * sizeof(int32_t), kind, g->stream));
  int32_t zero2[2] = {0, 0}, h[2] = {0, 0};
  GC_CUDA(cudaMemcpyAsync(g->io_b, zero2, sizeof(zero2), cudaMemcpyHostToDevice, g->stream));
  GC_TRY(launch_wcheck(g, (flags & GC_VALIDATE) != 0, g->io_b, g->io_b + 1));
  GC_CUDA(cudaMemcpyAsync(h, g->io_b, sizeof(h), cudaMemcpyDeviceToHost, g->stream));
  GC_TRY(sync(g));
  g->w_ok = false;
  if (h[0]) return fail(GC_EINVAL, (flags & GC_VALIDATE) ? "a weight is below 1 or differs between the two rows of an edge"
                                                         : "a weight is below 1");
  if ((int64_t)(g->n - 1) * (int64_t)h[1] >= (int64_t)kInf)
    return fail(GC_ERANGE, "(n - 1) * max weight reaches 2^30: path lengths could overflow");
  g->w_ok = true;
  return GC_OK;
}

// Weighted Greedy: Algorithm 2 with every SSSP a shortest-path search (the
// paper's weighted case) and the pruning of Sec. 4.1 and the lazy bounds of
// Sec. 4.2 unchanged.  Round 0 evaluates f({v}) of every vertex by a full
// search (a label-correcting search has no distance order to cut on);
// later rounds take host-driven lazy steps, one candidate per CTA; d_S is
// updated in place from each pick and its decrease must equal the pick's gain.
int gc_greedy_weighted(gc_graph *g, int32_t k, const gc_opts *opts_in, int32_t *out_group, int64_t *out_farness,
                       gc_stats *stats) {
  if (!g || !out_group || !out_farness || k < 1 || k > g->n)
    return fail(GC_EINVAL, "bad argument to gc_greedy_weighted (need 1 <= k <= n)");
  if (!g->w_ok) return fail(GC_EINVAL, "gc_greedy_weighted: no weights set (gc_set_weights)");
  gc_opts opts;
  if (opts_in) opts = *opts_in;
  else gc_opts_default(&opts);
  (void)opts;
  auto t0 = std::chrono::steady_clock::now();
  const int64_t launches0 = g->launches;
  const int32_t n = g->n;
  if (!g->w_ws) {  // per-CTA search workspaces: within 40% of free memory and 16 GB
    int occ = 0;
    GC_TRY(wsssp_occupancy(&occ));
    g->w_stride = wws_stride(n);
    size_t free_b = 0, total_b = 0;
    GC_CUDA(cudaMemGetInfo(&free_b, &total_b));
    const size_t budget = std::min<size_t>(free_b / 10 * 4, (size_t)16 << 30);
    int want = std::max(1, occ) * g->num_sms;
    if ((size_t)want * g->w_stride > budget) want = (int)std::max<size_t>(1, budget / g->w_stride);
    const size_t bytes = (size_t)want * g->w_stride + 256;
    if (cudaMalloc((void **)&g->w_ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      g->w_ws = nullptr;
      return fail(GC_ENOMEM, "gc_greedy_weighted: workspace allocation failed");
    }
    g->w_ctas = want;
    g->w_task = (unsigned int *)(g->w_ws + (size_t)want * g->w_stride);
    // queue flags 0, then every workspace's dist = kInf
    for (int c = 0; c < want; ++c) {
      unsigned char *p = g->w_ws + (size_t)c * g->w_stride;
      GC_CUDA(cudaMemsetAsync(p, 0, g->w_stride, g->stream));
    }
    for (int c = 0; c < want; ++c)
      GC_TRY(launch_fill_i32(g, (int32_t *)(g->w_ws + (size_t)c * g->w_stride), kInf, n));
  }
  GC_CUDA(cudaMemsetAsync(g->sctl, 0, sizeof(SelCtl), g->stream));
  // ---- round 0: f({v}) of every vertex, s0 = argmin (f, id) ----
  GC_TRY(launch_iota(g, g->list, n));
  GC_CUDA(cudaMemcpyAsync(&g->sctl->n_sel, &n, sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
  GC_TRY(launch_wsssp(g, kWFarness, g->list, &g->sctl->n_sel, g->f0, g->w_task));
  GC_TRY(launch_argmin_f0(g));
  GC_TRY(read_ctl(g));
  if (g->h_sctl->err) return fail(g->h_sctl->err, g->h_sctl->err == GC_EDISCONNECTED ? "graph is disconnected"
                                                                                      : "weighted search failed");
  const int32_t s0 = g->h_sctl->arg_id;
  const long long f_s0 = g->h_sctl->arg_val;
  if (s0 < 0 || s0 >= n) return fail(GC_EINTERNAL, "gc_greedy_weighted: round 0 produced no vertex");
  // d_S = d(s0, .) by the in-place search from s0; its sum must equal f_s0
  GC_TRY(launch_fill_i32(g, g->dS, kInf, n));
  GC_CUDA(cudaMemcpyAsync(g->io_a, &s0, sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
  GC_TRY(launch_wrelabel(g, g->io_a, &g->bctl->decrease));
  GC_TRY(launch_sum_dist(g, g->dS));
  GC_TRY(read_ctl(g));
  if (g->h_sctl->count != 0 || (long long)g->h_sctl->sum != f_s0)
    return fail(GC_EINTERNAL, "gc_greedy_weighted: farness of s0 disagrees between round 0 and d_S");
  long long f = f_s0;
  out_group[0] = s0;
  // ---- rounds 1..k-1: host-driven lazy steps, one candidate per CTA ----
  GC_TRY(launch_fill_i64(g, g->ub, LLONG_MAX, n));
  GC_TRY(launch_fill_i64(g, g->ub + s0, -1, 1));
  GC_TRY(launch_fill_i32(g, g->stamp, 0, n));
  const int32_t step_want = g->w_ctas;
  int64_t steps = 0, evals = 0;
  for (int32_t r = 1; r < k; ++r) {
    GC_TRY(launch_round_begin(g));
    for (;;) {
      GC_TRY(launch_select(g, kSelLazy, r, step_want, kTauHistogram, 0));
      GC_TRY(launch_wsssp(g, kWGain, g->list, &g->sctl->n_sel, g->lgain, g->w_task));
      GC_TRY(launch_after_eval(g, r, 0));
      GC_TRY(launch_unevaluated_best(g, r));
      GC_TRY(read_ctl(g));
      if (g->h_sctl->err) return fail(g->h_sctl->err, "weighted search failed");
      ++steps;
      evals += g->h_sctl->n_sel;
      if (g->h_sctl->accepted) break;
      if (g->h_sctl->n_sel == 0) return fail(GC_EINTERNAL, "gc_greedy_weighted: lazy step selected no candidate");
    }
    const int32_t pick = g->h_sctl->best_id;
    const long long gain = g->h_sctl->best_gain;
    GC_TRY(launch_round_end(g));
    GC_CUDA(cudaMemcpyAsync(g->io_a, &pick, sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
    GC_TRY(launch_wrelabel(g, g->io_a, &g->bctl->decrease));
    GC_TRY(read_ctl(g));
    if ((long long)g->h_bctl->decrease != gain)
      return fail(GC_EINTERNAL, "gc_greedy_weighted: gain of the pick disagrees with the d_S update (round " +
                                    std::to_string(r) + ")");
    f -= gain;
    out_group[r] = pick;
  }
  *out_farness = f;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->rounds = k;
    stats->steps = steps;
    stats->evals = evals;
    stats->round0_evals = n;
    stats->kernel_launches = g->launches - launches0;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return GC_OK;
}

// bitGreedy++ (Sec. 4.3, Theorem 1): every round scores every vertex by the
// bit-vector sweep of gc_bits.cu (round 0: the farness of every vertex; later
// rounds: every marginal gain against d_S), takes the best (ties: smaller id)
// and updates d_S by the pruned relabel BFS, whose decrease must equal the
// pick's gain.  The group equals gc_greedy's.
int gc_greedy_bits(gc_graph *g, int32_t k, const gc_opts *opts_in, int32_t *out_group, int64_t *out_farness,
                   gc_stats *stats) {
  if (!g || !out_group || !out_farness || k < 1 || k > g->n)
    return fail(GC_EINVAL, "bad argument to gc_greedy_bits (need 1 <= k <= n)");
  if (g->n > kBitsMaxN)
    return fail(GC_ERANGE, "gc_greedy_bits: n above " + std::to_string(kBitsMaxN) +
                               " (the bit-vector variant is for small graphs)");
  gc_opts opts;
  if (opts_in) opts = *opts_in;
  else gc_opts_default(&opts);
  const int64_t tns = timeout_ns(&opts);
  auto t0 = std::chrono::steady_clock::now();
  const int64_t launches0 = g->launches;
  const int32_t n = g->n;
  const int W = std::min(32, (n + 63) / 64);  // 64 W targets per chunk
  const size_t bytes_B = 2 * (size_t)n * W * sizeof(unsigned long long) + 2 * (size_t)n;  // words, row flags
  const size_t bytes = ws_align(bytes_B) + ws_align((size_t)n * sizeof(long long)) + ws_align(sizeof(BitsCtl));
  unsigned char *mem = nullptr;
  if (cudaMalloc((void **)&mem, bytes) != cudaSuccess) {
    cudaGetLastError();
    return fail(GC_ENOMEM, "gc_greedy_bits: device allocation failed");
  }
  unsigned long long *B = (unsigned long long *)mem;
  long long *out = (long long *)(mem + ws_align(bytes_B));
  BitsCtl *ctl = (BitsCtl *)(mem + ws_align(bytes_B) + ws_align((size_t)n * sizeof(long long)));
  BitsCtl h;
  auto done = [&](int rc) {
    cudaStreamSynchronize(g->stream);
    cudaFree(mem);
    return rc;
  };
  auto sweep = [&](int mode) -> int {
    GC_TRY(launch_bits_round(g, mode, B, out, ctl, W, tns));
    GC_CUDA(cudaMemcpyAsync(&h, ctl, sizeof(BitsCtl), cudaMemcpyDeviceToHost, g->stream));
    GC_TRY(sync(g));
    if (h.err) return fail(h.err, h.err == GC_ETIMEOUT ? "device-side wait timed out" : "bit-vector sweep failed");
    if (h.best == 0ull) return fail(GC_EINTERNAL, "gc_greedy_bits: no vertex to pick");
    return GC_OK;
  };
  int64_t levels = 0;
  int rc = sweep(0);  // round 0: s0 = argmin (farness, id)
  if (rc != GC_OK) return done(rc);
  levels += (int64_t)h.levels;
  const int32_t s0 = (int32_t)(0xffffffffu - (unsigned)(h.best & 0xffffffffull));
  const long long f_s0 = 0x7fffffffll - (long long)(h.best >> 32);
  GC_CUDA(cudaMemcpyAsync(g->io_a, &s0, sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
  GC_CUDA(cudaMemsetAsync(g->bctl, 0, sizeof(BfsCtl), g->stream));
  int64_t f = 0;
  if ((rc = distances_from(g, g->io_a, 1, tns, &f)) != GC_OK) return done(rc);
  if (f != f_s0) return done(fail(GC_EINTERNAL, "gc_greedy_bits: farness of s0 disagrees between the sweep and the BFS"));
  out_group[0] = s0;
  for (int32_t r = 1; r < k; ++r) {
    if ((rc = sweep(1)) != GC_OK) return done(rc);
    levels += (int64_t)h.levels;
    const int32_t pick = (int32_t)(0xffffffffu - (unsigned)(h.best & 0xffffffffull));
    const long long gain = (long long)(h.best >> 32);
    // d_S <- min(d_S, d(pick, .)) by the pruned relabel BFS; its decrease is the gain
    GC_CUDA(cudaMemcpyAsync(g->io_a, &pick, sizeof(int32_t), cudaMemcpyHostToDevice, g->stream));
    if ((rc = launch_bfs_relabel(g, g->dS, g->io_a, 1, tns)) != GC_OK) return done(rc);
    if ((rc = read_ctl(g)) != GC_OK) return done(rc);
    if (g->h_bctl->err) return done(device_errors(g));
    if ((long long)g->h_bctl->decrease != gain)
      return done(fail(GC_EINTERNAL, "gc_greedy_bits: gain of the pick disagrees with the d_S update (round " +
                                         std::to_string(r) + ")"));
    f -= gain;
    out_group[r] = pick;
  }
  *out_farness = f;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->rounds = k;
    stats->levels = levels;
    stats->evals = (int64_t)n * k;
    stats->kernel_launches = g->launches - launches0;
    stats->ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return done(GC_OK);
}

int gc_greedy(gc_graph *g, int32_t k, const gc_opts *opts_in, int32_t *out_group, int64_t *out_farness,
              gc_stats *stats) {
  if (!g || !out_group || !out_farness || k < 1 || k > g->n)
    return fail(GC_EINVAL, "bad argument to gc_greedy (need 1 <= k <= n)");
  gc_opts opts;
  if (opts_in) opts = *opts_in;
  else gc_opts_default(&opts);
  if (opts.use_proposal && !g->prop_params) return fail(GC_EINVAL, "no proposal network is set (gc_set_proposal)");
  const int64_t tns = timeout_ns(&opts);
  auto t0 = std::chrono::steady_clock::now();
  const int64_t launches0 = g->launches;
  memset(g->h_lctl, 0, sizeof(LazyCtl));  // the stats read it whether or not the lazy kernel runs
  size_t ev_used = 0;
  int64_t r0_stats[3] = {0, 0, 0};  // wide round-0 kernel: batches, bottom-up levels, top-down entries
  double r0_ms[4] = {0, 0, 0, 0};     // and its phases: selection, top-down, bottom-up, clears
  int64_t r0_bu[4] = {0, 0, 0, 0};    // its bottom-up claiming rows, entries read, words gathered, dense clears
  int64_t r0_probe[4] = {0, 0, 0, 0};  // its probe stages, the lanes they cut, row-pointer pairs and visited words read
  bool pruned = false;  // the pruned adjacency is built after round 0
  std::vector<char> ev_k64;  // per event pair: 1 = CTA-batched gain kernel, 0 = grid-wide, 2 = persistent
  auto gains_timed = [&](int mode, const int32_t *cand, int32_t n_cand, const int32_t *n_dev,
                         int lanes) -> int {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GC_TRY(gain_event(g, ev_used, &e0));
    GC_TRY(gain_event(g, ev_used + 1, &e1));
    ev_used += 2;
    ev_k64.push_back(1);
    GC_CUDA(cudaEventRecord(e0, g->stream));
    GC_TRY(launch_gains(g, mode, cand, n_cand, n_dev, g->lgain, opts.max_ctas, lanes, pruned));
    GC_CUDA(cudaEventRecord(e1, g->stream));
    return GC_OK;
  };
  auto grid_timed = [&](int mode, const int32_t *cand, int32_t nl, const int32_t *nl_dev,
                        long long *out) -> int {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GC_TRY(gain_event(g, ev_used, &e0));
    GC_TRY(gain_event(g, ev_used + 1, &e1));
    ev_used += 2;
    ev_k64.push_back(0);
    GC_CUDA(cudaEventRecord(e0, g->stream));
    GC_TRY(launch_gains_grid(g, mode, cand, nl, nl_dev, out, tns, pruned));
    GC_CUDA(cudaEventRecord(e1, g->stream));
    return GC_OK;
  };
  g->mx = nullptr;
  GC_CUDA(cudaMemsetAsync(g->sctl, 0, sizeof(SelCtl), g->stream));
  GC_CUDA(cudaMemsetAsync(g->gctl, 0, sizeof(GainCtl), g->stream));
  GC_CUDA(cudaMemsetAsync(g->bctl, 0, sizeof(BfsCtl), g->stream));

  // ---- round 0: s0 = argmin_v f({v}) (top-1 closeness, Sec. 3.1) ----
  // A lower bound LB(v) for every vertex; one grid-wide BFS from the vertex
  // with the smallest bound gives an exact farness f_a that serves as the cut
  // threshold; then every vertex with LB(v) <= f_a is evaluated by the
  // bit-parallel BFS with per-level cuts (BFScut).  Vertices above the bound
  // cannot beat f_a and are never searched.
  GC_TRY(launch_fill_i64(g, g->f0, -1, g->n));
  GC_TRY(launch_round0_keys(g));
  GC_TRY(launch_argmin_lb(g));
  GC_TRY(distances_from(g, &g->sctl->arg_id, 1, tns, nullptr));
  int32_t ds_src = g->h_sctl->arg_id;  // the vertex whose BFS distances are in d_S
  GC_TRY(launch_round0_seed(g));
  GC_TRY(launch_select(g, kSelKey, 0, 0, kTauDevice, 0));
  GC_TRY(read_ctl(g));
  int32_t n_surv = g->h_sctl->n_sel;
  // Shallow graphs (the BFS just run has few levels, as in social networks):
  // the survivors go to the wide bottom-up kernel, whose batches of up to 512
  // candidates read the graph once per level for all of them.  Pivot bounds
  // (triangle inequality) are weak there and are skipped.
  const int32_t ecc_a = g->h_bctl->levels;
  int r0_w = 0;
  if (opts.round0_lanes >= 0 && ecc_a <= kShallowLevels && n_surv > 0) {
    // automatic: 256 lanes at most (measured on R-MAT scale 24: 512 lanes are no
    // faster, their wider gathers cancel the halved batch count)
    const int want = opts.round0_lanes > 0 ? opts.round0_lanes : (n_surv > 128 ? 256 : n_surv > 64 ? 128 : 64);
    r0_w = want >= 512 ? 8 : want >= 256 ? 4 : want >= 128 ? 2 : 1;
    if (opts.round0_lanes == 0) {
      // The wide batches pay about one pass over the adjacency per batch;
      // the 64-lane top-down searches pay about the survivors' two-hop counts
      // (their scans to distance 2, where most searches are cut).  Take the
      // wide batches only when those counts are the larger: survivors next to
      // hubs (R-MAT), not flat graphs whose every vertex survives (BA).
      GC_TRY(launch_sum_two_hop(g, (unsigned long long *)g->g3));
      unsigned long long two_hop_sum = 0;
      GC_CUDA(cudaMemcpyAsync(&two_hop_sum, g->g3, sizeof(two_hop_sum), cudaMemcpyDeviceToHost, g->stream));
      GC_TRY(sync(g));
      const double passes = std::ceil((double)n_surv / (64.0 * r0_w));
      if ((double)two_hop_sum < passes * (double)g->nnz) r0_w = 0;
    }
  }
  // Many survivors (deep graphs, where the degree bound is weak): tighten the
  // bounds with the BFS levels of pivots (triangle inequality, see
  // k_pivot_bound).  The first pivot is the vertex just searched; each further
  // pivot is the undecided vertex of smallest bound, searched exactly, so it
  // may also lower the threshold.
  for (int piv = 0; r0_w == 0 && n_surv > kRound0GridMax && piv < kRound0Pivots; ++piv) {
    if (piv > 0) {
      GC_TRY(launch_argmin_lb(g));
      GC_TRY(distances_from(g, &g->sctl->arg_id, 1, tns, nullptr));
      ds_src = g->h_sctl->arg_id;
      GC_TRY(launch_round0_pivot(g));
    }
    GC_TRY(launch_pivot_bound(g));
    GC_TRY(launch_select(g, kSelKey, 0, 0, kTauDevice, 0));
    GC_TRY(read_ctl(g));
    n_surv = g->h_sctl->n_sel;
  }
  int64_t r0_wide_lanes = 0;
  if (r0_w > 0) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    GC_TRY(gain_event(g, ev_used, &e0));
    GC_TRY(gain_event(g, ev_used + 1, &e1));
    ev_used += 2;
    ev_k64.push_back(3);
    GC_CUDA(cudaEventRecord(e0, g->stream));
    GC_TRY(launch_round0_wide(g, g->list, n_surv, g->lgain, r0_w, 8 * r0_w, !(opts.flags & GC_OPT_R0_FULL_LEVELS),
                              tns, (opts.flags & GC_OPT_R0_NO_PROBE) ? 0 : kR0ProbeStride));
    GC_CUDA(cudaEventRecord(e1, g->stream));
    R0Ctl r0c;
    GC_CUDA(cudaMemcpyAsync(&r0c.batches, &g->r0_ctl->batches, 18 * sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, g->stream));
    GC_TRY(sync(g));
    r0_wide_lanes = (int64_t)r0c.lanes;
    r0_stats[0] = (int64_t)r0c.batches;
    r0_stats[1] = (int64_t)r0c.levels;
    r0_stats[2] = (int64_t)r0c.td_edges;
    for (int i = 0; i < 4; ++i) r0_ms[i] = r0c.ns[i] * 1e-6;
    r0_bu[0] = (int64_t)r0c.bu_rows;
    r0_bu[1] = (int64_t)r0c.bu_scanned;
    r0_bu[2] = (int64_t)r0c.bu_gathers;
    r0_bu[3] = (int64_t)r0c.dense_clears;
    r0_probe[0] = (int64_t)r0c.probe_levels;
    r0_probe[1] = (int64_t)r0c.probe_cut;
    r0_probe[2] = (int64_t)r0c.bu_vertices;
    r0_probe[3] = (int64_t)r0c.bu_visreads;
  } else if (n_surv <= kRound0GridMax) {
    // few survivors (hubs with large searches): one grid-wide batch per 64
    for (int32_t off = 0; off < n_surv; off += kLanes)
      GC_TRY(grid_timed(kModeFarness, g->list + off, std::min<int32_t>(kLanes, n_surv - off), nullptr,
                        g->lgain + off));
  } else {
    GC_TRY(gains_timed(kModeFarness, g->list, n_surv, nullptr, kLanes));
  }
  GC_TRY(launch_after_eval(g, 0, 0));
  GC_TRY(launch_argmin_f0(g));
  GC_TRY(read_ctl(g));
  GC_TRY(device_errors(g));
  const int32_t s0 = g->h_sctl->arg_id;
  const long long f_s0 = g->h_sctl->arg_val;
  const int64_t round0_evals = (int64_t)g->h_gctl->lanes + r0_wide_lanes + 1;
  if (s0 < 0) return fail(GC_EINTERNAL, "round 0 produced no vertex");
  int64_t f = f_s0;
  if (s0 != ds_src) {  // d_S = d(s0, .) unless s0's BFS is the one already in d_S
    GC_TRY(distances_from(g, &g->sctl->arg_id, 1, tns, &f));
    if (f != f_s0) return fail(GC_EINTERNAL, "farness of s0 disagrees between round 0 and the BFS");
  }
  // neighbour bound for the pruning of useless expansions in every later round
  if (!(opts.flags & GC_OPT_NO_EXPAND_BOUND)) {
    GC_TRY(launch_max_nbr(g));
    g->mx = g->mx_buf;
  }
  // pruned adjacency: drop the entries no later round can use (d_S[w] <= 1)
  if (!(opts.flags & GC_OPT_FULL_ADJACENCY)) {
    GC_TRY(launch_prune_csr(g));
    pruned = true;
  }
  const double ms_round0 =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  double ms_round1 = 0;
  out_group[0] = s0;

  // ---- rounds 1..k-1: lazy greedy with exact pruned gains ----
  // later rounds: few candidates per step, spread over CTAs in small batches
  const int32_t step_want = opts.eval_per_step > 0 ? opts.eval_per_step : 128;
  const int step_lanes = (opts.step_lanes > 0 && opts.step_lanes <= kLanes) ? opts.step_lanes : 8;
  const bool grid_steps = opts.step_mode == 2;
  const bool persistent = opts.step_mode == 0 || opts.step_mode == 3;
  // round-1 bounds (k_round1_bound, from the pruned adjacency's counts): round
  // 1 evaluates the 64 largest bounds, then only the candidates whose bound
  // reaches the best exact gain found, instead of every vertex
  const bool round1_bound = persistent && pruned && !(opts.flags & GC_OPT_NO_ROUND1_BOUND);
  if (k > 1) {
    if (round1_bound) {
      GC_TRY(launch_round1_bound(g));
    } else {
      GC_TRY(launch_fill_i64(g, g->ub, LLONG_MAX, g->n));
      GC_TRY(launch_fill_i64(g, g->ub + s0, -1, 1));
      GC_TRY(launch_fill_i32(g, g->stamp, 0, g->n));
    }
  }
  const int32_t heavy = opts.round1_heavy < 0 ? 0 : (opts.round1_heavy == 0 ? 1024 : opts.round1_heavy);
  // measured on R-MAT graphs: the grid-wide forms win, so both default off
  // lazy step form: wide (one 64-lane batch per CTA) on deep graphs, where a
  // grid-wide batch pays a grid barrier for each of its many levels
  int step_form = opts.step_form;
  const long long local_max = opts.local_update_max_gain <= 0 ? -1 : opts.local_update_max_gain;
  int64_t lazy_steps = 0, lazy_evals = 0, lazy_launches = 0;
  GainCtl lazy0, lazy1;  // gain counters around the persistent kernel
  memset(&lazy0, 0, sizeof(lazy0));
  memset(&lazy1, 0, sizeof(lazy1));
  double lazy_ms[3] = {0, 0, 0};
  std::vector<long long> gains_picked(k, 0), decreases(k, 0);
  gains_picked[0] = f;
  for (int32_t r = 1; r < k; ++r) {
    if (r >= 2 && persistent) {
      // rounds r..k-1 on the device: persistent kernel over an active list
      LazyCtl init;
      memset(&init, 0, sizeof(init));
      init.round = r;
      init.best_id = -1;
      init.best_pos = -1;
      init.best_gain = -1;
      init.best_lane = -1;
      init.last_gain = gains_picked[r - 1];
      init.scored_round = -1;
      *g->h_lctl = init;
      GC_CUDA(cudaMemcpyAsync(g->lctl, g->h_lctl, sizeof(LazyCtl), cudaMemcpyHostToDevice, g->stream));
      GC_TRY(read_ctl(g));
      lazy0 = *g->h_gctl;
      if (step_form == 0)  // levels per 64-lane batch so far (rounds 0 and 1)
        step_form = lazy0.batches && lazy0.levels > kWideLevels * lazy0.batches ? 2 : 1;
      // active list: short for 64-candidate steps (its scans are the selection's
      // cost), at least two wide steps for wide ones
      int32_t target = opts.active_target > 0 ? opts.active_target
                                              : (step_form == 2 ? std::max<int32_t>(4096, 2 * g->wcap) : 2048);
      for (;;) {
        // two-hop bounds for the current group, before every (re)launch: the
        // candidates round 1 skipped would otherwise keep their round-1 bounds
        if (round1_bound) GC_TRY(launch_bound_refresh(g));
        GC_TRY(launch_select(g, kSelActive, 0, target, kTauHistogramTheta, 0));
        cudaEvent_t le0 = nullptr, le1 = nullptr;
        GC_TRY(gain_event(g, ev_used, &le0));
        GC_TRY(gain_event(g, ev_used + 1, &le1));
        ev_used += 2;
        ev_k64.push_back(2);
        GC_CUDA(cudaEventRecord(le0, g->stream));
        GC_TRY(launch_lazy_rounds(g, k, tns, opts.use_proposal && g->prop_fill > 0 ? g->prop_params : nullptr,
                                  g->prop_fill,
                                  step_form == 2, local_max, opts.lazy_ctas, pruned,
                                  !(opts.flags & GC_OPT_NO_CLAIM_LOG), opts.claim_log_cap));
        GC_CUDA(cudaEventRecord(le1, g->stream));
        ++lazy_launches;
        GC_CUDA(cudaMemcpyAsync(g->h_lctl, g->lctl, sizeof(LazyCtl), cudaMemcpyDeviceToHost, g->stream));
        GC_TRY(read_ctl(g));
        if (g->h_lctl->err) {
          g->h_gctl->err = g->h_lctl->err;
          return device_errors(g);
        }
        if (g->h_lctl->round >= k) break;
        if (g->h_lctl->dec != 2) return fail(GC_EINTERNAL, "persistent lazy kernel stopped early");
        target = target > (1 << 28) ? g->n : target * 4;
      }
      lazy1 = *g->h_gctl;
      lazy_steps = g->h_lctl->steps;
      lazy_evals = g->h_lctl->evals;
      lazy_ms[0] = g->h_lctl->ns_select * 1e-6;
      lazy_ms[1] = g->h_lctl->ns_gain * 1e-6;
      lazy_ms[2] = g->h_lctl->ns_update * 1e-6;
      std::vector<int32_t> pk(k);
      std::vector<long long> pg(k), pd(k);
      GC_CUDA(cudaMemcpyAsync(pk.data() + r, g->picks + r, (size_t)(k - r) * sizeof(int32_t),
                              cudaMemcpyDeviceToHost, g->stream));
      GC_CUDA(cudaMemcpyAsync(pg.data() + r, g->pgain + r, (size_t)(k - r) * sizeof(long long),
                              cudaMemcpyDeviceToHost, g->stream));
      GC_CUDA(cudaMemcpyAsync(pd.data() + r, g->pdec + r, (size_t)(k - r) * sizeof(long long),
                              cudaMemcpyDeviceToHost, g->stream));
      GC_TRY(sync(g));
      for (int32_t q = r; q < k; ++q) {
        if (pg[q] != pd[q])
          return fail(GC_EINTERNAL, "gain of the pick disagrees with the d_S update (round " +
                                        std::to_string(q) + ")");
        f -= pg[q];
        out_group[q] = pk[q];
      }
      break;
    }
    GC_TRY(launch_round_begin(g));
    for (int step = 0;; ++step) {
      if (r == 1 && round1_bound) {
        if (step == 0 && g->rec_X && g->rec_cap > 0) {
          // recording run (training data for the proposal): the 1024 largest
          // bounds, every one evaluated exactly and recorded with the
          // features it had when it was chosen
          GC_TRY(launch_select(g, kSelLazy, r, kR1Propose, kTauHistogram, 0));
          GC_TRY(launch_clamp_nsel(g, kR1Propose));
          GC_TRY(read_ctl(g));
          const int32_t m1 = g->h_sctl->n_sel;
          for (int32_t off = 0; off < m1; off += kLanes)
            GC_TRY(grid_timed(kModeGain, g->list + off, std::min<int32_t>(kLanes, m1 - off), nullptr,
                              g->lgain + off));
          GC_TRY(launch_record(g, r, gains_picked[0]));
        } else if (step == 0) {
          // the first batch: its best exact gain is the level every other
          // candidate's bound must reach.  Without the proposal, the 64
          // largest bounds; with it, the 64 of the 1024 largest bounds whose
          // predicted gain is largest
          if (opts.use_proposal) {
            GC_TRY(launch_select(g, kSelLazy, r, kR1Propose, kTauHistogram, 0));
            GC_TRY(launch_clamp_nsel(g, kR1Propose));
            GC_TRY(launch_round1_propose(g, gains_picked[0]));
          } else {
            GC_TRY(launch_select(g, kSelLazy, r, kLanes, kTauHistogram, 0));
            GC_TRY(launch_clamp_nsel(g, kLanes));
          }
          GC_TRY(grid_timed(kModeGain, g->list, 0, &g->sctl->n_sel, g->lgain));
        } else {
          // every unevaluated candidate whose bound reaches the best exact
          // gain so far, in 64-lane batches, one CTA each
          GC_TRY(launch_select(g, kSelLazy, r, 0, kTauHost, g->h_sctl->best_gain));
          GC_TRY(gains_timed(kModeGain, g->list, 0, &g->sctl->n_sel, kLanes));
        }
      } else if (r == 1) {  // no bounds: all of V \ S
        if (heavy > 0) {
          // the highest-degree candidates have the largest searches: one
          // grid-wide batch per 64 of them, so no CTA is left with a hub batch
          GC_TRY(launch_degree_keys(g));
          GC_TRY(launch_select(g, kSelKey, 0, heavy, kTauHistogram, 0));
          GC_TRY(read_ctl(g));
          const int32_t nh = std::min<int32_t>(g->h_sctl->n_sel, 4 * heavy);
          for (int32_t off = 0; off < nh; off += kLanes)
            GC_TRY(grid_timed(kModeGain, g->list + off, std::min<int32_t>(kLanes, nh - off), nullptr,
                              g->lgain + off));
          GC_TRY(launch_clamp_nsel(g, nh));
          GC_TRY(launch_after_eval(g, r, 0));
        }
        // the rest in 64-lane batches, one CTA each
        GC_TRY(launch_select(g, kSelLazy, r, 0, kTauHost, 0));
        GC_TRY(gains_timed(kModeGain, g->list, 0, &g->sctl->n_sel, kLanes));
      } else if (grid_steps) {  // the top-64 bounds as one grid-wide batch
        GC_TRY(launch_select(g, kSelLazy, r, kLanes, kTauHistogram, 0));
        GC_TRY(launch_clamp_nsel(g, kLanes));
        GC_TRY(grid_timed(kModeGain, g->list, 0, &g->sctl->n_sel, g->lgain));
        GC_TRY(launch_record(g, r, gains_picked[r - 1]));
      } else {
        GC_TRY(launch_select(g, kSelLazy, r, step_want, kTauHistogram, 0));
        GC_TRY(gains_timed(kModeGain, g->list, 0, &g->sctl->n_sel, step_lanes));
        GC_TRY(launch_record(g, r, gains_picked[r - 1]));
      }
      GC_TRY(launch_after_eval(g, r, 0));
      GC_TRY(launch_unevaluated_best(g, r));
      GC_CUDA(cudaMemcpyAsync(g->h_sctl, g->sctl, sizeof(SelCtl), cudaMemcpyDeviceToHost, g->stream));
      GC_TRY(sync(g));
      if (g->h_sctl->accepted) break;
      if (g->h_sctl->n_sel == 0) return fail(GC_EINTERNAL, "lazy step selected no candidate");
    }
    const int32_t pick = g->h_sctl->best_id;
    gains_picked[r] = g->h_sctl->best_gain;
    GC_TRY(launch_round_end(g));
    GC_CUDA(cudaMemsetAsync(g->bctl, 0, sizeof(BfsCtl), g->stream));
    GC_TRY(launch_bfs_relabel(g, g->dS, &g->sctl->best_id, 1, tns, pruned));
    GC_CUDA(cudaMemcpyAsync(&g->h_bctl->decrease, &g->bctl->decrease, sizeof(unsigned long long),
                            cudaMemcpyDeviceToHost, g->stream));
    GC_TRY(sync(g));
    decreases[r] = (long long)g->h_bctl->decrease;
    if (decreases[r] != gains_picked[r])
      return fail(GC_EINTERNAL, "gain of the pick disagrees with the d_S update (round " +
                                    std::to_string(r) + ")");
    f -= gains_picked[r];
    out_group[r] = pick;
    if (r == 1)
      ms_round1 = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count() -
                  ms_round0;
  }
  g->mx = nullptr;
  GC_TRY(read_ctl(g));
  GC_TRY(device_errors(g));
  *out_farness = f;
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->rounds = k;
    stats->steps = g->h_sctl->steps + lazy_steps;
    stats->evals = g->h_sctl->evals + lazy_evals;
    stats->batches = (int64_t)g->h_gctl->batches;
    stats->edges_scalar = (int64_t)g->h_gctl->edges_scalar;
    stats->edges_union = (int64_t)g->h_gctl->edges_union;
    stats->levels = (int64_t)g->h_gctl->levels;
    stats->frontier = (int64_t)g->h_gctl->frontier;
    stats->pushes = (int64_t)g->h_gctl->pushes;
    stats->lanes = (int64_t)g->h_gctl->lanes;
    stats->round0_evals = round0_evals;
    stats->ms_round0 = ms_round0;
    stats->ms_round1 = ms_round1;
    for (size_t i = 0; i + 1 < ev_used; i += 2) {
      float ms = 0.f;
      GC_CUDA(cudaEventElapsedTime(&ms, g->events[i], g->events[i + 1]));
      const int kind = ev_k64[i / 2];
      if (kind == 2) {
        stats->ms_lazy_kernel += ms;
        ++stats->lazy_launches;
        continue;
      }
      if (kind == 3) {
        stats->ms_round0_wide += ms;
        continue;
      }
      stats->ms_gain_kernel += ms;
      ++stats->gain_launches;
      if (kind == 1) {
        stats->ms_gain64 += ms;
        ++stats->gain64_launches;
      }
    }
    stats->gain64_frontier = (int64_t)g->h_gctl->k_front;
    stats->gain64_edges = (int64_t)g->h_gctl->k_union;
    stats->gain64_pushes = (int64_t)g->h_gctl->k_push;
    stats->gain64_lanes = (int64_t)g->h_gctl->k_lanes;
    stats->lazy_frontier = (int64_t)(lazy1.frontier - lazy0.frontier);
    stats->lazy_edges = (int64_t)(lazy1.edges_union - lazy0.edges_union);
    stats->lazy_pushes = (int64_t)(lazy1.pushes - lazy0.pushes);
    stats->lazy_lanes = (int64_t)(lazy1.lanes - lazy0.lanes);
    stats->lazy_upd_frontier = (int64_t)g->h_lctl->upd_work[0];
    stats->lazy_upd_edges = (int64_t)g->h_lctl->upd_work[1];
    stats->lazy_upd_relabels = (int64_t)g->h_lctl->upd_relabels;
    stats->lazy_sel_scanned = (int64_t)g->h_lctl->sel_scanned;
    stats->lazy_log_picks = (int64_t)g->h_lctl->log_picks;
    stats->lazy_upd_log = (int64_t)g->h_lctl->upd_log;
    stats->lazy_log_entries = (int64_t)g->h_lctl->log_written;
    stats->r0_batches = r0_stats[0];
    stats->r0_levels = r0_stats[1];
    stats->r0_td_edges = r0_stats[2];
    stats->ms_r0_select = r0_ms[0];
    stats->ms_r0_topdown = r0_ms[1];
    stats->ms_r0_bottomup = r0_ms[2];
    stats->ms_r0_clear = r0_ms[3];
    stats->r0_bu_rows = r0_bu[0];
    stats->r0_bu_scanned = r0_bu[1];
    stats->r0_bu_gathers = r0_bu[2];
    stats->r0_width = r0_w * kLanes;
    stats->r0_dense_clears = r0_bu[3];
    stats->r0_probes = r0_probe[0];
    stats->r0_probe_cut = r0_probe[1];
    stats->r0_bu_vertices = r0_probe[2];
    stats->r0_bu_visreads = r0_probe[3];
    stats->ms_lazy_select = lazy_ms[0];
    stats->ms_lazy_gain = lazy_ms[1];
    stats->ms_lazy_update = lazy_ms[2];
    stats->kernel_launches = g->launches - launches0;
    stats->ms_total =
        std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  }
  return GC_OK;
}

}  // extern "C"
