// gc_marginal_gains_static: marginal gains without any device allocation.
//
// Who needs this: callers that cannot call cudaMalloc -- plugins that must
// live inside a host application's fixed device-memory budget or its own
// allocator (a raw cudaMalloc would bypass both), and latency-critical
// services that forbid allocator calls on their request path (cudaMalloc and
// cudaFree can synchronise the device and take unbounded time).  gc_load_csr
// allocates a handle's arrays, so such callers cannot use gc_marginal_gains;
// this entry point takes plain device pointers instead and keeps all of its
// scratch in one fixed array compiled into the library.
//
// The scratch is a file-scope __device__ array of kStaticScratchBytes (64 MiB).
// Every GPU that loads the library reserves it until the process exits.  It
// holds the control words, then 20 bytes per vertex (d(., S), two BFS queues
// and two range-start lists), then as many per-CTA gain workspaces (44 bytes
// per vertex each) as fit.  A graph needs at least one workspace, so n is at
// most kStaticMaxVertices = 1,048,496 (64 bytes per vertex plus 256-byte
// alignment of each part).  Fewer vertices leave room for more workspaces and
// so more CTAs: about 14 at n = 100,000, one at n = 646,000.
//
// Errors found on the device cannot reach the host without a synchronisation,
// which this entry point avoids.  Instead, when the BFS from S fails (an id of
// S outside [0, n), a device-side wait that timed out, or a vertex that S does
// not reach), a last kernel overwrites every output with -1.
//
// Host code cannot use the array's name as a device address; on the first
// call on each device (with that device current) the library looks the
// address up once with cudaGetSymbolAddress and caches it.  That first call
// should therefore happen before any stream capture.  The kernels are the
// library's ordinary BFS and 64-lane gain kernels, pointed at the array.
#include <mutex>

#include "gc_internal.cuh"

namespace gc {

size_t gain_ws_stride(int32_t n);
int gain_kernel_occupancy(int *blocks_per_sm);
int bfs_kernel_occupancy(int *blocks_per_sm);

constexpr size_t kStaticScratchBytes = 64ull << 20;
constexpr int32_t kStaticMaxVertices = 1048496;  // largest n whose layout fits (see above)
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

namespace {
std::mutex g_static_mu;
unsigned char *g_static_ptr[kMaxDevices];  // device address of the array, per device
int g_static_sms[kMaxDevices];
int g_static_gain_occ[kMaxDevices];
int g_static_bfs_occ[kMaxDevices];

size_t round_up(size_t x) { return (x + 255) & ~(size_t)255; }
}  // namespace

// Outputs become -1 when the BFS that computed d(., S) did not finish cleanly:
// an error code (bad id of S, wait timeout) or fewer than n vertices labelled
// (S does not reach every vertex, so d(., S) is undefined somewhere).
__global__ void k_static_poison(const BfsCtl *__restrict__ ctl, int32_t n, long long *out, int32_t n_cand) {
  const bool bad = ctl->err != 0 || ctl->relabelled != (unsigned long long)n;
  if (!bad) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_cand; i += gridDim.x * blockDim.x) out[i] = -1;
}

// Set-up once per device: the array's device address and the launch geometry.
static int static_setup(int dev) {
  std::lock_guard<std::mutex> lock(g_static_mu);
  if (g_static_ptr[dev]) return GC_OK;
  void *p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
  if (e != cudaSuccess || !p) {
    cudaGetLastError();
    set_error(std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
    return GC_ECUDA;
  }
  int sms = 0, occ_g = 0, occ_b = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_error("cudaDeviceGetAttribute failed");
    return GC_ECUDA;
  }
  int rc = gain_kernel_occupancy(&occ_g);
  if (rc == GC_OK) rc = bfs_kernel_occupancy(&occ_b);
  if (rc != GC_OK) return rc;
  g_static_sms[dev] = sms;
  g_static_gain_occ[dev] = occ_g > 0 ? occ_g : 1;
  g_static_bfs_occ[dev] = occ_b > 0 ? occ_b : 1;
  g_static_ptr[dev] = (unsigned char *)p;
  return GC_OK;
}

}  // namespace gc

using namespace gc;

extern "C" int gc_marginal_gains_static(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                                        const int32_t *S, int32_t s_len, const int32_t *cand,
                                        int32_t n_cand, int64_t *out_gain, void *stream) {
  if (n < 1 || !row_ptr || !col_idx || !S || s_len < 1 || n_cand < 0 || (n_cand > 0 && (!cand || !out_gain))) {
    set_error("bad argument to gc_marginal_gains_static");
    return GC_EINVAL;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    set_error("no usable CUDA device");
    return GC_ECUDA;
  }
  int rc = static_setup(dev);
  if (rc != GC_OK) return rc;

  // carve the array: control words, d(., S), BFS queues, then workspaces
  const size_t stride = gain_ws_stride(n);
  const size_t a4 = round_up((size_t)n * sizeof(int32_t));
  const size_t head = round_up(sizeof(BfsCtl)) + round_up(sizeof(GainCtl)) + 4 * a4 +
                      round_up(((size_t)n + 1) * sizeof(int32_t));
  if (n > kStaticMaxVertices || head + stride > kStaticScratchBytes) {
    set_error("gc_marginal_gains_static: n = " + std::to_string(n) + " needs " +
              std::to_string(head + stride) + " bytes of scratch, the static array holds " +
              std::to_string(kStaticScratchBytes));
    return GC_ERANGE;
  }
  unsigned char *base = g_static_ptr[dev];
  gc_graph g;  // a view over caller memory and the static array: nothing is allocated
  g.n = n;
  g.device = dev;
  g.num_sms = g_static_sms[dev];
  g.stream = (cudaStream_t)stream;
  g.owns_csr = false;
  g.rp = const_cast<int32_t *>(row_ptr);
  g.ci = const_cast<int32_t *>(col_idx);
  unsigned char *p = base;
  g.bctl = (BfsCtl *)p;
  p += round_up(sizeof(BfsCtl));
  g.gctl = (GainCtl *)p;
  p += round_up(sizeof(GainCtl));
  g.dS = (int32_t *)p;
  p += a4;
  g.bq0 = (int32_t *)p;
  p += a4;
  g.bq1 = (int32_t *)p;
  p += a4;
  g.goff = (int32_t *)p;
  p += round_up(((size_t)n + 1) * sizeof(int32_t));
  g.gx = (int32_t *)p;  // second range-start list of the relabel BFS
  p += a4;
  g.ws = p;
  g.ws_stride = stride;
  const int fit = (int)((kStaticScratchBytes - head) / stride);
  const int resident = g_static_gain_occ[dev] * g.num_sms;
  g.gain_ctas = fit < resident ? fit : resident;
  g.ws_count = g.gain_ctas;
  g.bfs_ctas = g_static_bfs_occ[dev] * g.num_sms;

  // The array keeps whatever the previous call left (possibly for another n):
  // zero the control words and every workspace this call will use.
  if (cudaMemsetAsync(base, 0, round_up(sizeof(BfsCtl)) + round_up(sizeof(GainCtl)), g.stream) != cudaSuccess ||
      cudaMemsetAsync(g.ws, 0, (size_t)g.gain_ctas * stride, g.stream) != cudaSuccess) {
    cudaGetLastError();
    set_error("cudaMemsetAsync on the static scratch failed");
    return GC_ECUDA;
  }
  if ((rc = launch_fill_i32(&g, g.dS, kInf, n)) != GC_OK) return rc;
  if ((rc = launch_bfs_relabel(&g, g.dS, S, s_len, 10000000000LL)) != GC_OK) return rc;
  if ((rc = launch_gains(&g, kModeGain, cand, n_cand, nullptr, (long long *)out_gain, 0)) != GC_OK) return rc;
  if (n_cand > 0) {
    const int blocks = (n_cand + 255) / 256 < 4 * g.num_sms ? (n_cand + 255) / 256 : 4 * g.num_sms;
    k_static_poison<<<blocks, 256, 0, g.stream>>>(g.bctl, n, (long long *)out_gain, n_cand);
    if (cudaGetLastError() != cudaSuccess) {
      set_error("launch of the output check failed");
      return GC_ECUDA;
    }
  }
  return GC_OK;
}
