// Device helpers shared by the libgc kernels: bounded grid barrier, timers,
// warp/block reductions.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "gc_internal.cuh"

namespace gc {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// CTA barrier.  __syncthreads() is an aligned barrier: it counts a warp
// correctly only if the warp arrives converged.  A warp still split by an
// earlier single-thread branch (thread 0's bookkeeping, a poll) could be
// counted at the wrong barrier, after which its warps run one barrier apart;
// __syncwarp() first reconverges it.  Every CTA barrier of the library goes
// through here.
__device__ __forceinline__ void cta_sync() {
  __syncwarp();
  __syncthreads();
}

// Grid barrier for cooperative launches (all CTAs co-resident).  One 32-bit
// word per barrier: in every episode CTA 0 adds 2^31 - (G - 1) and each other
// CTA adds 1 (G = gridDim.x), so the episode adds exactly 2^31: bit 31 of the
// word flips at the last arrival and the low 31 bits come back to zero, ready
// for the next episode (of any grid size).  Arrival is a release atomic by
// thread 0, the wait an acquire poll of bit 31; the CTA barriers on both sides
// extend the ordering to every thread.  The poll is bounded twice: by
// `timeout_ns` of global time and by an iteration cap.  On expiry the CTA
// records GC_ETIMEOUT in *err and the barrier returns false; every caller then
// leaves its kernel.  Returns false as well when *err is already set.  A word
// left mid-episode by such an exit must be zeroed before its next launch.
__device__ __forceinline__ bool grid_sync(GridBar *bar, int32_t *err,
                                          unsigned long long timeout_ns) {
  __shared__ int s_ok;
  cta_sync();
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned int add = blockIdx.x == 0 ? 0x80000000u - (gridDim.x - 1u) : 1u;
    unsigned int old;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(&bar->count), "r"(add) : "memory");
    const unsigned long long t0 = global_ns();
    unsigned int it = 0;
    for (;;) {
      unsigned int cur;
      asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(cur) : "l"(&bar->count) : "memory");
      if ((cur ^ old) & 0x80000000u) break;
      ++it;
      if ((it & 3u) == 0 && (global_ns() - t0 > timeout_ns || it > (1u << 30))) {
        atomicExch(err, GC_ETIMEOUT);
        ok = 0;
        break;
      }
    }
    s_ok = ok && (*(volatile int32_t *)err == 0);
  }
  cta_sync();
  return s_ok != 0;
}

// A load through the read-only data path when RO (the data must not change
// while the kernel can still read it), else a plain load.  For the same reason
// no pointer to data that a persistent kernel rewrites (d_S, bounds, stamps,
// selected candidates, active lists) is declared const __restrict__: the
// compiler may then load it through the non-coherent read-only path, which a
// grid barrier does not refresh.
template <bool RO>
__device__ __forceinline__ int32_t ld_ro(const int32_t *p) {
  if (RO) return __ldg(p);
  return *p;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum; every thread gets the result.  `sh` needs 32 entries.
template <typename T>
__device__ __forceinline__ T block_sum(T v, T *sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  cta_sync();
  if (lane == 0) sh[wid] = v;
  cta_sync();
  const int nw = (blockDim.x + 31) >> 5;
  T r = (threadIdx.x < nw) ? sh[threadIdx.x] : T(0);
  if (wid == 0) r = warp_sum(r);
  if (threadIdx.x == 0) sh[0] = r;
  cta_sync();
  r = sh[0];
  cta_sync();
  return r;
}

// Block-wide exclusive scan of int32 (blockDim.x <= 1024); returns the
// exclusive prefix, *total gets the block total.  `sh` needs 33 entries.
__device__ __forceinline__ int block_excl_scan(int v, int *sh, int *total) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    int y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  cta_sync();
  if (lane == 31) sh[wid] = x;
  cta_sync();
  if (wid == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    int s = (lane < nw) ? sh[lane] : 0;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    if (lane < nw) sh[lane] = s;  // inclusive prefix of warp totals
    if (lane == nw - 1) sh[32] = s;
  }
  cta_sync();
  const int warp_off = wid ? sh[wid - 1] : 0;
  *total = sh[32];
  const int r = warp_off + x - v;
  cta_sync();
  return r;
}

// (value, id) pairs ordered by larger value, then smaller id.
__device__ __forceinline__ bool better_max(long long v, int id, long long bv, int bid) {
  return v > bv || (v == bv && (unsigned)id < (unsigned)bid);
}
// (value, id) pairs ordered by smaller value, then smaller id.
__device__ __forceinline__ bool better_min(long long v, int id, long long bv, int bid) {
  return v < bv || (v == bv && (unsigned)id < (unsigned)bid);
}

}  // namespace gc
