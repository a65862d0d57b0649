// Persistent lazy greedy (Sec. 4.2) for rounds >= 2: one cooperative launch
// runs round after round on the device -- select, evaluate, certify, update
// d_S -- with no host round trip.
//
// Candidates live in an "active list" (vertex ids in increasing order) that
// holds every non-member whose bound ub is at least theta; every candidate
// outside it has ub < theta.  Each step, CTA 0
//   * folds the gains of the batch just evaluated (ub <- exact gain, stamp <-
//     round) into the round's best (gain desc, id asc);
//   * finds the best bound (ub desc, id asc) among active candidates not yet
//     evaluated in this round.  If the round's best beats it and is >= theta,
//     the best is the plain greedy's choice (nothing outside the list can
//     reach theta): accept.  If it beats the list but is below theta, the list
//     is too short: the kernel stops and the host rebuilds it with a lower
//     theta.  Otherwise
//   * selects exactly the 64 largest (ub, smaller id first) unevaluated active
//     candidates: histogram passes over the bounds fix the threshold value,
//     ties at the threshold go to the smallest ids (list order).
// Then every CTA runs the 64-lane pruned BFS on that batch (grid_gain_batch).
// On acceptance d_S becomes min(d_S, d(pick, .)) and the round advances.  The
// vertices whose label drops are exactly those the pick's lane reached in its
// pruned search, at the distances it reached them (Sec. 4.1), so the update
// reads them from the claim log the batches of the round wrote: one pass over
// the batch's entries by every CTA, no BFS levels.  If the log ran out of room
// (or in wide steps, which keep none) every CTA runs the relabel BFS from the
// pick instead (the pruned SSSP of Sec. 4.1).
#include <algorithm>

#include "gc_cta.cuh"
#include "gc_lazy.cuh"

namespace gc {

// One CTA per SM (the launch uses one), so the register budget is 128.
__global__ void __launch_bounds__(kGridGainThreads, 1)
    k_lazy_rounds(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, int32_t n, int32_t *dS,
                  long long *ub, int32_t *stamp, const int32_t *__restrict__ act, const int32_t *m_dev,
                  int32_t k, int32_t *picks, long long *pgain, long long *pdec, unsigned char *ws,
                  int32_t *goff, GridGainCtl *gg, LazyCtl *lc, GainCtl *gctl, int32_t *bq0, int32_t *bq1,
                  unsigned long long tns, const int32_t *__restrict__ mx, const float *__restrict__ prop,
                  int32_t fill, const long long *__restrict__ two_hop, float *score, size_t ws_stride,
                  int32_t wide, long long local_max, long long *akey, int32_t *ast,
                  int32_t *gx, int32_t *wsel, long long *wgain, int32_t *wpos, int32_t wcap,
                  const int32_t *__restrict__ rp_full, const int32_t *__restrict__ c3, GridSelScratch *gsel,
                  ClaimRec *clog, unsigned long long clog_cap) {
  __shared__ unsigned long long s_red[32];
  extern __shared__ __align__(16) unsigned char s_list[];  // kLazyListSmem bytes
  const int m = *m_dev;
  // CTA 0 keeps a list of at most kCta0SelectMax entries in shared memory (ids,
  // bounds, stamps): it alone selects from such a list, so every scan of a
  // step reads shared memory instead of L2.  Longer lists keep compact copies
  // in global memory (akey/ast), read by the grid-wide selection.
  const bool local = m <= kCta0SelectMax;
  const int32_t *lact = act;
  long long *lkey = akey;
  int32_t *lst = ast;
  __shared__ Cta0State s_st;  // CTA 0's step state in lean steps
  {  // the copies of the bounds of the (new) active list, and best_id's position
    const int b0 = *(volatile int32_t *)&lc->best_id;
    if (local) {
      if (blockIdx.x == 0) {
        long long *sk = reinterpret_cast<long long *>(s_list);
        int32_t *sa = reinterpret_cast<int32_t *>(sk + kCta0SelectMax), *ss = sa + kCta0SelectMax;
        if (threadIdx.x == 0) s_st.bpos = -1;
        cta_sync();
        for (int i = threadIdx.x; i < m; i += blockDim.x) {
          const int v = act[i];
          sa[i] = v;
          sk[i] = ub[v];
          ss[i] = stamp[v];
          if (v == b0) {
            lc->best_pos = i;
            s_st.bpos = i;
          }
        }
        lact = sa;
        lkey = sk;
        lst = ss;
      }
    } else {
      for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < m; i += gridDim.x * blockDim.x) {
        const int v = act[i];
        akey[i] = ub[v];
        ast[i] = stamp[v];
        if (v == b0) lc->best_pos = i;
      }
    }
  }
  // CTA 0's sorted view of a shared-memory list (lean steps)
  __shared__ int s_nord;
  SortedView view;
  view.ord = reinterpret_cast<uint16_t *>(s_list + (size_t)kCta0SelectMax * 16);
  view.tmp = view.ord + kCta0SelectMax;
  view.mark = reinterpret_cast<unsigned char *>(view.tmp + kCta0SelectMax);
  view.nord = &s_nord;
  const bool use_view = local && !prop && !wide;
  if (use_view && blockIdx.x == 0) {
    if (threadIdx.x == 0) {  // the lean state, carried over from an earlier launch of the round
      s_st.bid = *(volatile int32_t *)&lc->best_id;
      s_st.bgain = *(volatile long long *)&lc->best_gain;
      s_st.theta = *(volatile long long *)&lc->theta;
      s_st.log_mark = *(volatile unsigned long long *)&lc->log_mark;
      s_st.nsel = 0;
      s_st.dec = 0;
    }
    sv_build(lkey, m, view);
  }
  if (!grid_sync(&lc->bar, &lc->err, tns)) return;
  const bool timer = blockIdx.x == 0 && threadIdx.x == 0;
  const GainWs myws = gain_ws(ws, ws_stride, n, blockIdx.x);  // this CTA's own workspace
  GainCounters cnt;
  GridCounts gcnt;  // this thread's work counts of the grid-wide batches
  unsigned long long t0 = timer ? global_ns() : 0, t1;
  bool fold = false;
  // CTA 0 selects for short lists (a few scans of m entries cost less than the
  // grid barriers of the grid-wide selection), with proposal lanes and in wide
  // steps; otherwise every CTA takes part.  With CTA 0 selecting 64-lane grid
  // batches it also runs level 0 of the batch and the accept bookkeeping before
  // the step's barrier, and fewer barriers are needed per step and per round.
  const bool cta0_sel = prop || wide || m <= kCta0SelectMax;
  const bool lean = cta0_sel && !prop && !wide;  // (then also use_view: the list is local)
  // the batch as CTA 0 sees it in lean steps (shared memory) and as the others do
  const bool st0 = lean && blockIdx.x == 0;
  const int32_t *bsel = st0 ? s_st.sel : lc->sel;
  const int32_t *bnsel = st0 ? &s_st.nsel : &lc->n_sel;
  long long *bout = st0 ? s_st.gout : lc->gsel;
  int r = *(volatile int32_t *)&lc->round;  // every CTA counts the rounds itself
  for (;;) {
    if (r >= k) break;
    if (prop && *(volatile int32_t *)&lc->scored_round != r) {
      lazy_score(act, m, prop, rp_full, dS, ub, stamp, two_hop, mx, r, lc->last_gain, score);
      if (!grid_sync(&lc->bar, &lc->err, tns)) break;
      if (blockIdx.x == 0 && threadIdx.x == 0) lc->scored_round = r;
    }
    if (cta0_sel) {
      if (blockIdx.x == 0) {
        if (lean) {
          lean_step(lact, ub, stamp, lc, gg, fold, r, lkey, lst, view, s_st);
          cta_sync();  // s_st.dec, the batch and the reset batch control block
          const int d = s_st.dec;
          if (d == 0) {
            grid_gain_batch<kModeGain>(rp, ci, n, dS, s_st.sel, 0, &s_st.nsel, s_st.gout, ws, gx, goff, gg, gctl,
                                       &lc->bar, &lc->err, tns, mx, c3, 0, -1, kBatchLevel0, clog, &lc->log_n,
                                       clog_cap);
          } else if (d == 1 && threadIdx.x == 0) {
            picks[r] = s_st.bid;
            pgain[r] = s_st.bgain;
            lc->pk[0] = lc->pk[1] = lc->pk[2] = 0;
            lc->decrease = 0;
          }
        } else {
          lazy_cta0_step(lact, m, ub, stamp, lc, wide ? nullptr : gg, fold, (prop && !wide) ? score : nullptr, fill,
                         lkey, lst, wsel, wgain, wpos, wide ? wcap : 0);
        }
      }
    } else {  // every CTA takes part in the selection
      int dec_local;
      if (!grid_lazy_step(act, m, ub, stamp, akey, ast, lc, gg, fold, lc->sel, lc->selpos, lc->gsel, kLanes, gsel,
                          &lc->bar, &lc->err, tns, &dec_local))
        break;
    }
    if (!grid_sync(&lc->bar, &lc->err, tns)) break;
    if (timer) {
      t1 = global_ns();
      lc->ns_select += t1 - t0;
      t0 = t1;
    }
    const int dec = *(volatile int32_t *)&lc->dec;
    if (dec == 2) break;  // the host lowers theta and relaunches
    if (dec == 0) {
      // wide steps (deep graphs): one 64-lane batch per CTA, no grid barrier
      // inside; otherwise the whole grid on one 64-lane batch.
      bool ok;
      if (wide) {
        const int ns = *(volatile int32_t *)&lc->n_sel;
        const int nb = (ns + kLanes - 1) / kLanes;
        for (int bi = blockIdx.x; bi < nb; bi += gridDim.x)
          cta_gain_batch<kModeGain, true, false>(rp, ci, n, dS, wsel + bi * kLanes, min(kLanes, ns - bi * kLanes),
                                    wgain + bi * kLanes, myws, gctl, mx, LaneGraphs(), cnt, 0, c3);
        ok = grid_sync(&lc->bar, &lc->err, tns);  // gains visible to CTA 0
      } else {
        ok = grid_gain_batch<kModeGain>(rp, ci, n, dS, bsel, 0, bnsel, bout, ws, gx, goff, gg, gctl, &lc->bar,
                                        &lc->err, tns, mx, c3, 0, -1, lean ? kBatchRest : kBatchAll, clog,
                                        &lc->log_n, clog_cap, &gcnt);
        // the gains are in lc->gsel, written by CTA 0: only a grid-wide fold
        // needs them published
        if (!lean) ok = ok && grid_sync(&lc->bar, &lc->err, tns);
      }
      if (!ok) break;
      if (timer) {
        t1 = global_ns();
        lc->ns_gain += t1 - t0;
        t0 = t1;
      }
      fold = true;
      continue;
    }
    // accept the round's best: record it and update d_S from it
    fold = false;
    if (!lean) {
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        picks[r] = lc->best_id;
        pgain[r] = lc->best_gain;
        lc->pk[0] = lc->pk[1] = lc->pk[2] = 0;
        lc->decrease = 0;
      }
      if (!grid_sync(&lc->bar, &lc->err, tns)) break;
    }
    bool ok = true;
    const int blane = *(volatile int32_t *)&lc->best_lane;
    const unsigned long long s0 = *(volatile unsigned long long *)&lc->best_seg0;
    const unsigned long long s1 = *(volatile unsigned long long *)&lc->best_seg1;
    if (clog && !wide && blane >= 0 && blane < kLanes && s0 <= s1 && s1 <= clog_cap) {
      // from the claim log: the pick's lane, in the entries of its batch
      const u64 bit = 1ull << blane;
      u64 dec = 0, rel = 0;
      for (unsigned long long i = s0 + (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < s1;
           i += (unsigned long long)gridDim.x * blockDim.x) {
        const int4 e = *reinterpret_cast<const int4 *>(clog + i);
        const u64 won = (u64)(unsigned)e.z | ((u64)(unsigned)e.w << 32);
        if (!(won & bit)) continue;
        const int old = atomicMin(&dS[e.x], e.y);  // each vertex once per lane
        if (old > e.y) {
          if (old < kInf) dec += (u64)(old - e.y);
          ++rel;
        }
      }
      if (blockIdx.x == 0 && threadIdx.x == 0) {  // the pick itself (level 0)
        const int old = atomicMin(&dS[*(volatile int32_t *)&lc->best_id], 0);
        if (old > 0) {
          if (old < kInf) dec += (u64)old;
          ++rel;
        }
        lc->upd_log += s1 - s0;
        lc->log_picks += 1;
      }
      dec = block_sum(dec, s_red);
      rel = block_sum(rel, s_red);
      if (threadIdx.x == 0) {
        if (dec) atomicAdd(&lc->decrease, dec);
        if (rel) atomicAdd(&lc->upd_relabels, rel);
      }
    } else if (*(volatile long long *)&lc->best_gain <= local_max) {  // small region: CTA 0 alone
      if (blockIdx.x == 0) {
        const long long d = cta_relabel_bfs(rp, ci, dS, *(volatile int32_t *)&lc->best_id, myws.qv0, myws.qv1);
        if (threadIdx.x == 0) lc->decrease = (unsigned long long)d;
      }
    } else {
      ok = grid_relabel_bfs(rp, ci, n, dS, &lc->best_id, 1, bq0, bq1, lc->pk, nullptr, &lc->decrease,
                            &lc->upd_relabels, goff, gx, &lc->bar, &lc->err, tns, lc->upd_work, c3);
    }
    ok = ok && grid_sync(&lc->bar, &lc->err, tns);
    if (!ok) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      const int bid = lean ? s_st.bid : lc->best_id;
      const long long bgain = lean ? s_st.bgain : lc->best_gain;
      const int bp = lean ? s_st.bpos : lc->best_pos;
      const unsigned long long ln = *(volatile unsigned long long *)&lc->log_n;
      pdec[r] = (long long)*(volatile unsigned long long *)&lc->decrease;
      lc->log_written += ln < clog_cap ? ln : clog_cap;
      lc->last_gain = bgain;
      ub[bid] = -1;  // a member: never a candidate again
      if (bp >= 0 && bp < m && lact[bp] == bid) lkey[bp] = -1;
      lc->best_id = -1;
      lc->best_gain = -1;
      lc->best_lane = -1;
      lc->log_n = 0;  // the next round's log (its first batch starts after a barrier)
      lc->log_mark = 0;
      if (lean) {
        s_st.bid = -1;
        s_st.bgain = -1;
        s_st.bpos = -1;
        s_st.log_mark = 0;
      }
      atomicAdd(&lc->rounds_done, 1);
      lc->round = r + 1;
    }
    ++r;
    // the other CTAs read none of the bookkeeping before the next step's
    // barrier unless they select or score too; CTA 0's own threads do
    if (lean) cta_sync();
    else if (!grid_sync(&lc->bar, &lc->err, tns)) break;
    if (timer) {
      t1 = global_ns();
      lc->ns_update += t1 - t0;
      t0 = t1;
    }
  }
  // work counters: the wide steps' (per CTA) and the grid-wide batches' (per
  // thread, summed here once instead of after every batch)
  const u64 c_scalar = block_sum(cnt.scalar + gcnt.scalar, s_red), c_union = block_sum(cnt.uni + gcnt.uni, s_red);
  const u64 c_front = block_sum(cnt.front + gcnt.front, s_red), c_push = block_sum(cnt.push + gcnt.push, s_red);
  if (threadIdx.x == 0) {
    if (c_scalar) atomicAdd(&gctl->edges_scalar, c_scalar);
    if (c_union) atomicAdd(&gctl->edges_union, c_union);
    if (c_front) atomicAdd(&gctl->frontier, c_front);
    if (c_push) atomicAdd(&gctl->pushes, c_push);
    if (cnt.batches) {
      atomicAdd(&gctl->levels, cnt.levels);
      atomicAdd(&gctl->batches, cnt.batches);
      atomicAdd(&gctl->lanes, cnt.lanes);
    }
  }
}

// After a threshold pass over the bounds: never let theta exceed the round's
// best exact gain (so that the rebuilt list can certify it), then record theta.
__global__ void k_active_theta(SelCtl *sc, LazyCtl *lc) {
  long long tau = sc->tau;
  if (lc->best_id >= 0 && lc->best_gain < tau) tau = lc->best_gain;
  if (sc->sel_count == 0) tau = LLONG_MAX;
  sc->tau = tau;
  lc->theta = tau;
}

int lazy_occupancy(int *blocks_per_sm) {
  GC_CUDA(cudaFuncSetAttribute(k_lazy_rounds, cudaFuncAttributeMaxDynamicSharedMemorySize, kLazyListSmem));
  GC_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_lazy_rounds, kGridGainThreads,
                                                        kLazyListSmem));
  return GC_OK;
}

int launch_active_theta(gc_graph *g) {
  ++g->launches;
  k_active_theta<<<1, 1, 0, g->stream>>>(g->sctl, g->lctl);
  GC_CUDA(cudaGetLastError());
  return GC_OK;
}

int launch_lazy_rounds(gc_graph *g, int32_t k, int64_t timeout_ns, const float *prop, int32_t fill,
                       bool wide_steps, long long local_max, int ctas, bool pruned, bool use_log,
                       long long log_cap) {
  // one CTA per SM; wide steps give every CTA a gain workspace of its own, so
  // there the grid is also capped by the workspaces allocated (on large graphs
  // fewer than the SMs); grid-wide steps use workspace 0 and CTA 0's only
  int grid = wide_steps ? std::min(g->lazy_ctas, g->ws_count) : g->lazy_ctas;
  if (ctas > 0 && ctas < grid) grid = ctas;
  int32_t wide = wide_steps ? 1 : 0;
  int32_t wcap = std::min(g->wcap, grid * kLanes);
  int32_t *wsel = g->wsel, *wpos = g->wpos;
  long long *wgain = g->wgain;
  const int32_t *rp = pruned ? g->rpf : g->rp, *ci = pruned ? g->cif : g->ci;
  const int32_t *rp_full = g->rp, *c3 = pruned ? g->c3 : nullptr;
  GridSelScratch *gsel = g->gsel;
  int32_t n = g->n;
  int32_t *dS = g->dS;
  long long *ub = g->ub;
  int32_t *stamp = g->stamp;
  const int32_t *act = g->list;
  const int32_t *m_dev = &g->sctl->n_sel;
  int32_t *picks = g->picks;
  long long *pgain = g->pgain, *pdec = g->pdec;
  unsigned char *ws = g->ws;
  int32_t *goff = g->goff;
  GridGainCtl *gg = g->ggctl;
  LazyCtl *lc = g->lctl;
  GainCtl *gctl = g->gctl;
  int32_t *q0 = g->bq0, *q1 = g->bq1;
  unsigned long long tns = (unsigned long long)timeout_ns;
  const int32_t *mx = g->mx;
  const long long *two_hop = g->two_hop;
  float *score = g->score;
  size_t ws_stride = g->ws_stride;
  long long *akey = g->akey;
  int32_t *ast = g->ast;
  int32_t *gx = g->gx;
  ClaimRec *clog = use_log ? g->clog : nullptr;
  unsigned long long clog_cap =
      use_log ? (unsigned long long)(log_cap > 0 ? std::min(log_cap, g->clog_cap) : g->clog_cap) : 0ull;
  void *args[] = {(void *)&rp,    (void *)&ci,    (void *)&n,    (void *)&dS,   (void *)&ub,
                  (void *)&stamp, (void *)&act,   (void *)&m_dev, (void *)&k,   (void *)&picks,
                  (void *)&pgain, (void *)&pdec,  (void *)&ws,   (void *)&goff, (void *)&gg,
                  (void *)&lc,    (void *)&gctl,  (void *)&q0,   (void *)&q1,   (void *)&tns,
                  (void *)&mx,    (void *)&prop,  (void *)&fill, (void *)&two_hop, (void *)&score,
                  (void *)&ws_stride, (void *)&wide, (void *)&local_max, (void *)&akey,
                  (void *)&ast, (void *)&gx, (void *)&wsel, (void *)&wgain, (void *)&wpos, (void *)&wcap,
                  (void *)&rp_full, (void *)&c3, (void *)&gsel, (void *)&clog, (void *)&clog_cap};
  ++g->launches;
  GC_CUDA(cudaLaunchCooperativeKernel((const void *)k_lazy_rounds, dim3(grid), dim3(kGridGainThreads), args,
                                      kLazyListSmem, g->stream));
  return GC_OK;
}

}  // namespace gc
