// Internal declarations of libgc: handle layout, device helpers, kernels.
// Group-closeness Greedy++ (arXiv:1710.01144) on sm_103a.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/gc.h"

namespace gc {

constexpr int32_t kInf = 0x3fffffff;  // "unreached" distance (d + 1 cannot overflow)
constexpr int kLanes = 64;            // candidates per bit-parallel batch (one uint64 word)
constexpr int kGainThreads = 512;     // threads per CTA of the gain kernel
constexpr int kCta0SelectMax = 4096;  // lazy selection by CTA 0 up to this list length, grid-wide above
// CTA 0's shared-memory copy of such a list: bound (int64), id and stamp
// (int32); its sorted view: two position arrays (uint16) and a mark byte
constexpr int kLazyListSmem = kCta0SelectMax * 16 + kCta0SelectMax * 5;
constexpr int kWideLevels = 16;       // lazy steps go wide above this many BFS levels per batch
constexpr int kEdgeIlp = 4;           // adjacency entries in flight per thread (CTA gain batch)
constexpr int kBfsThreads = 256;      // threads per CTA of the grid-wide BFS
constexpr int kRedThreads = 256;      // threads per CTA of reductions / scans
constexpr int kHistBins = 2048;       // bins of the selection histogram
constexpr int kGridGainThreads = 512; // threads per CTA of the grid-wide gain kernel
constexpr int kMaxGridCtas = 1024;    // cap on CTAs of cooperative launches
constexpr int kHeavyRow = 2048;       // rows longer than this are split over CTAs / warps
constexpr int kR0MaxLanes = 512;      // lanes of the widest round-0 batch

// ----------------------------------------------------------- control words --
// Lane words of a gain workspace: one 32-byte record per vertex w holding its
// visited word (4w) and three claim words (4w + 1 .. 4w + 3).  The CTA form
// alternates the first two between even and odd levels; the grid form cycles
// through all three.  A claim reads the visited word and sets two words of the
// same record, so it touches one 32-byte sector.
struct LaneWords {
  unsigned long long *p;
  __device__ __forceinline__ unsigned long long &operator[](long long i) const { return p[4 * i]; }
};

// A gain workspace: the lane-word records, two frontier queues (vertex ids)
// and a touched list.  One per CTA of the CTA-batched kernel; workspace 0 also
// serves the grid-wide batch.  All lane words are zero between batches.
struct GainWs {
  LaneWords vis, nx[3];
  int32_t *qv0, *qv1, *touched;
};

__host__ __device__ inline size_t ws_align(size_t x) { return (x + 255) & ~(size_t)255; }

// bytes of one workspace for n vertices (44 per vertex, each part 256-aligned)
__host__ __device__ inline size_t gain_ws_bytes(int32_t n) {
  return ws_align((size_t)n * 32) + 3 * ws_align((size_t)n * sizeof(int32_t));
}

__device__ __forceinline__ GainWs gain_ws(unsigned char *base, size_t stride, int32_t n, int idx) {
  unsigned char *p = base + stride * (size_t)idx;
  const size_t a32 = ws_align((size_t)n * 32), a4 = ws_align((size_t)n * sizeof(int32_t));
  GainWs w;
  w.vis.p = (unsigned long long *)p;
  w.nx[0].p = (unsigned long long *)p + 1;
  w.nx[1].p = (unsigned long long *)p + 2;
  w.nx[2].p = (unsigned long long *)p + 3;
  w.qv0 = (int32_t *)(p + a32);
  w.qv1 = (int32_t *)(p + a32 + a4);
  w.touched = (int32_t *)(p + a32 + 2 * a4);
  return w;
}

// Scratch of the grid-wide lazy step (gc_lazy.cuh, grid_lazy_step): per-CTA
// partials of the decision scan and of the selection counts, and three
// threshold histograms that are all zero between steps.
constexpr int kSelBins = 1024;
struct GridSelScratch {
  long long umax[1024];
  int32_t vmax[1024];
  long long umin[1024];
  long long cnt[1024];
  int32_t gt[1024];
  int32_t eq[1024];
  unsigned int hist[3][kSelBins];
};

// Bounded grid barrier used by cooperative kernels: one arrival word whose
// bit 31 flips once per episode (`gen` is padding).  Every wait gives up
// after a time limit and reports GC_ETIMEOUT.
struct GridBar {
  unsigned int count;
  unsigned int gen;
};

// Grid-wide BFS control block (zeroed before each launch).
struct BfsCtl {
  GridBar bar;
  unsigned long long pk[3];  // frontier by level mod 3: entries << 32 | adjacency entries
  int32_t err;          // GC_* code set by the device, 0 = fine
  int32_t levels;       // levels completed
  unsigned long long decrease;  // sum over relabelled vertices of (old - new), old finite
  unsigned long long relabelled;
  int32_t blk_tot[kMaxGridCtas];  // per-CTA adjacency totals of the level
};

// Gain-kernel control block.  batch_next is zeroed before every launch; err,
// best_f and the counters live across the launches of one API call.
struct GainCtl {
  unsigned int batch_next;  // next batch to take (persistent CTAs)
  int32_t err;
  long long best_f;         // farness mode: best exact farness seen (atomicMin), cut threshold
  unsigned long long edges_scalar;  // sum over lanes of adjacency entries a 1-source BFS scans
  unsigned long long edges_union;   // adjacency entries scanned (once per frontier word)
  unsigned long long levels;        // BFS levels summed over batches
  unsigned long long batches;
  unsigned long long frontier;      // frontier entries expanded
  unsigned long long pushes;        // vertices that entered a next frontier
  unsigned long long lanes;         // candidate lanes processed
  // the same counters, added by the CTA-batched kernel (k_gains64) alone
  unsigned long long k_front, k_union, k_push, k_lanes;
  // farness mode, GC_EDISCONNECTED: a candidate whose search ended short and
  // the vertices it reached (for the error message)
  long long short_vertex, short_count;
  // farness mode: nonzero keeps best_f fixed (top-k closeness cuts at the
  // k-th best, not at the best farness a search completes with)
  int32_t fixed_best;
  int32_t pad;
};

// Grid-wide gain kernel control block (zeroed before each launch).
struct GridGainCtl {
  GridBar bar;
  int32_t err;
  int32_t F;          // (unused)
  int32_t qn[2];      // (unused)
  int32_t touched;    // vertices with a non-zero visited word
  int32_t pad;
  // frontier of level L, by L mod 3: entries (high 32 bits) and adjacency
  // entries (low 32 bits), both taken by one atomicAdd per push
  unsigned long long pk[3];
  unsigned long long gain[kLanes];  // gain mode: per-lane gain
  unsigned long long cnt[kLanes];   // (unused in farness mode, see dgain/dcnt)
  int32_t blk_tot[kMaxGridCtas];    // per-CTA adjacency totals of the level
  // farness mode: per-lane distance sums and counts of the vertices claimed at
  // distance d, in dgain/dcnt[d mod 3] (written during one level, read by every
  // CTA after its barrier, cleared two levels later)
  unsigned long long dgain[3][kLanes];
  unsigned long long dcnt[3][kLanes];
};

// Control block of the bit-vector sweep (gc_bits.cu), zeroed before each launch.
struct BitsCtl {
  GridBar bar;
  int32_t err;
  int32_t pad;
  unsigned int changed[3];  // farness sweep: some word changed at level i (by i mod 3)
  int32_t pad2;
  unsigned long long best;    // packed arg-best of the round
  unsigned long long levels;  // levels swept, summed over the target chunks
};
constexpr int32_t kBitsMaxN = 65536;  // bit-vector variant: packed 32-bit values (farness < 2^31)

// One entry of the claim log of the persistent lazy kernel: at BFS level
// `lev` of a 64-lane gain batch, the lanes `won` reached vertex w for the first
// time.  A lane's entries are its whole pruned search (Sec. 4.1): the vertices
// with d(candidate, w) < d_S[w], each once, at that distance.
struct __align__(16) ClaimRec {
  int32_t w;
  int32_t lev;
  unsigned long long won;
};

// Persistent lazy-rounds kernel control block (gc_lazy.cu).
struct LazyCtl {
  GridBar bar;
  int32_t err;
  int32_t dec;          // step decision: 0 evaluate, 1 accept, 2 rebuild the active list
  int32_t round;        // current round (in/out across launches)
  int32_t n_sel;        // candidates of the current batch
  int32_t best_id;      // round's best exact gain so far (-1 none)
  int32_t rounds_done;
  long long best_gain;
  long long theta;      // every candidate outside the active list has ub < theta
  int32_t pad;          // fold flag of the batched solver
  int32_t pad3;
  unsigned long long pk[3];  // relabel BFS frontiers (see BfsCtl)
  unsigned long long decrease;
  long long steps, evals;
  unsigned long long ns_select, ns_gain, ns_update;  // time in each phase (CTA 0's clock)
  long long last_gain;  // gain of the previous pick (proposal feature)
  int32_t scored_round;  // round whose proposal scores are in g->score
  int32_t best_pos;     // list position of best_id (compact keys only)
  int32_t sel[kLanes];
  long long gsel[kLanes];
  int32_t selpos[kLanes];  // list positions of sel[] (compact keys only)
  // work of the persistent kernel's update and selection phases
  unsigned long long upd_work[2];  // relabel BFS: frontier entries, adjacency entries
  unsigned long long upd_relabels; // relabel BFS: vertices whose d_S decreased
  unsigned long long sel_scanned;  // selection: active-list entries read
  // claim log of the current round (entries [0, log_n); past the capacity
  // nothing is written but log_n still counts): the entries of the batches
  // folded so far end at log_mark; the round's best came from lane best_lane
  // of the batch whose entries are [best_seg0, best_seg1) (-1: no log)
  unsigned long long log_n, log_mark, best_seg0, best_seg1;
  int32_t best_lane;
  int32_t pad4;
  unsigned long long upd_log;    // d_S updates from the log: entries read
  unsigned long long log_picks;  // picks whose d_S update came from the log
  unsigned long long log_written;  // log entries written (summed over rounds)
};

// Control block of the wide round-0 kernel (gc_round0.cu), zeroed before each
// launch except best_f.
struct R0Ctl {
  GridBar bar;
  int32_t phase;    // 0: survivor list, 1: deferred candidates, 2: done
  int32_t nb;       // lanes of the current batch
  int32_t cursor;   // next survivor-list position
  int32_t dcursor;  // next deferred position
  int32_t n_defer;  // deferred candidates
  int32_t count_only;  // this batch: distance 2 counted without writing lane words (see gc_round0.cu)
  long long best_f;  // best exact farness (written by CTA 0 between batches)
  int32_t cand[kR0MaxLanes];  // the batch: candidate ids and their list positions
  int32_t pos[kR0MaxLanes];
  unsigned long long tot[3][kR0MaxLanes];  // claims per lane at distance d, in tot[d mod 3]
  unsigned long long far[kR0MaxLanes];     // probe: vertices proven at distance >= 3, per lane
  unsigned long long batches, levels, lanes;  // work counters
  unsigned long long td_edges;                 // adjacency entries of the top-down levels
  unsigned long long ns[4];  // CTA 0's clock: selection, top-down level, bottom-up levels with folds, clears
  unsigned long long bu_rows, bu_scanned, bu_gathers;  // bottom-up: vertices that claimed lanes, entries read, frontier words gathered
  unsigned long long co_lanes, co_surv;  // lanes of count-only batches, and those of them deferred
  unsigned long long dense_clears;       // batches that cleared every visited word
  unsigned long long probe_levels, probe_cut;  // probe stages run, and lanes they cut
  unsigned long long bu_vertices, bu_visreads;  // bottom-up: row-pointer pairs and visited words read
};

// Selection / reduction control block (lives across a whole greedy call).
struct SelCtl {
  // threshold search (keys are compared as int64; differences in uint64)
  long long lo, hi;      // key range of the current histogram pass
  long long tau;         // selection: key >= tau
  long long sel_count;   // selectable vertices
  int32_t done;          // threshold fixed
  int32_t n_sel;         // size of the compacted list
  // lazy round state
  long long best_gain;   // best exact gain of the current round (-1 = none)
  int32_t best_id;
  int32_t accepted;      // 1 once the round's pick is certified
  long long unev_ub;     // best bound among candidates not evaluated this round
  int32_t unev_id;
  int32_t pad0;
  // reductions
  unsigned int ticket;   // last-CTA ticket of the reductions
  int32_t err;
  long long sum, count;  // k_sum_dist: sum of distances, unreached vertices
  long long arg_val;     // k_argmin_f0
  int32_t arg_id;
  int32_t pad1;
  long long evals, steps;  // lazy-step counters of the call
};

// Per-lane graph data for gain batches that mix graphs of a block-diagonal
// union (farness mode): lane j's vertex count and cut threshold come from its
// graph.  Empty (gid == nullptr) for a single graph.
struct LaneGraphs {
  const int32_t *gid = nullptr;  // graph of each vertex
  const int32_t *ng = nullptr;   // vertex count of each graph
  long long *best_f = nullptr;   // per-graph best exact farness (atomicMin)
};

// --------------------------------------------------------------- handle ----
}  // namespace gc

struct gc_graph {
  int32_t n = 0;
  int64_t nnz = 0;
  int device = 0;
  int num_sms = 0;
  cudaStream_t stream = nullptr;
  bool owns_csr = true;
  int32_t *rp = nullptr;  // row_ptr[n+1]
  int32_t *ci = nullptr;  // col_idx[nnz]
  int32_t *dS = nullptr;  // distance to the current group
  int32_t *mx = nullptr;  // mx[u] >= max over neighbours w of d_S[w] (or nullptr: no pruning)
  int32_t *mx_buf = nullptr;
  long long *two_hop = nullptr;            // sum over neighbours of (deg - 1), feature input
  // weighted graphs (gc_set_weights, gc_weighted.cu): weights aligned with ci,
  // the per-CTA search workspaces (allocated on first use) and their task counter
  int32_t *wt = nullptr;
  bool w_ok = false;  // weights set and checked
  unsigned char *w_ws = nullptr;
  size_t w_stride = 0;
  int w_ctas = 0;
  unsigned int *w_task = nullptr;
  // candidates per batch of the CTA-batched gain kernel (gc_set_gain_lanes):
  // 64, or 128 / 256 for the wide kernel (gc_gain_wide.cu), whose per-CTA
  // workspaces are allocated on first use
  int32_t gain_lanes = 64;
  unsigned char *x_ws = nullptr;
  size_t x_stride = 0;
  int x_ctas = 0, x_w = 0;
  float *score = nullptr;                  // proposal scores of the active list [n]
  // learned proposal (caller-owned weights) and training-data recorder
  const float *prop_params = nullptr;
  int32_t prop_fill = 0;
  float *rec_X = nullptr, *rec_y = nullptr;
  int32_t rec_cap = 0;
  int32_t *rec_count = nullptr;            // device counter
  long long *ub = nullptr;     // lazy bound / exact gain of the round in stamp
  int32_t *stamp = nullptr;    // round of the last exact evaluation (0 = never)
  long long *key = nullptr;    // round-0 selection key (-lower bound), INT64_MIN = done
  long long *f0 = nullptr;     // round 0: exact f({v}) or -1
  int32_t *list = nullptr;     // compacted candidate list [n]
  long long *lgain = nullptr;  // gains/farness of list entries [n]
  int32_t *gx = nullptr;       // grid-wide gain batch: entry offsets by level parity, third list [3n]
  int32_t *rpf = nullptr, *cif = nullptr, *c3 = nullptr;  // pruned adjacency after round 0 [n+1], [nnz], [n]
  int32_t *heavy = nullptr, *n_heavy = nullptr;           // rows with more than 2048 entries (built at load)
  unsigned long long *lev_cnt = nullptr;  // round-0 pivot bound: level counts [n] (zero between uses)
  unsigned long long *lev_C = nullptr, *lev_M = nullptr;  // prefix counts / level sums [n + 1]
  int32_t *lev_max = nullptr;
  unsigned long long *g3 = nullptr;  // round-1 bounds: sum over u of (d_S[u] - 3)^+
  int32_t *c3s = nullptr;            // bound refresh: neighbours with the current d_S >= 3 [n]
  gc::GridSelScratch *gsel = nullptr;  // grid-wide lazy selection scratch (histograms zero at rest)
  gc::ClaimRec *clog = nullptr;  // persistent lazy kernel: claim log [clog_cap]
  long long clog_cap = 0;
  int32_t *wsel = nullptr;     // wide lazy steps: candidates, list positions, gains [wcap]
  int32_t *wpos = nullptr;
  long long *wgain = nullptr;
  int32_t wcap = 0;
  long long *akey = nullptr;   // persistent lazy kernel: ub of list entry i [n]
  int32_t *ast = nullptr;      // persistent lazy kernel: stamp of list entry i [n]
  int32_t *bq0 = nullptr, *bq1 = nullptr;  // grid BFS queues [n]
  int32_t *blk = nullptr;                  // per-block counts / offsets
  long long *partial = nullptr;            // per-block partial reductions (x4)
  unsigned int *hist = nullptr;            // selection histogram [kHistBins]
  int32_t *io_a = nullptr;                 // staging for small host arrays [n]
  int32_t *io_b = nullptr;
  gc::BfsCtl *bctl = nullptr;
  gc::GridGainCtl *ggctl = nullptr;
  gc::LazyCtl *lctl = nullptr;
  gc::LazyCtl *h_lctl = nullptr;           // pinned host mirror
  int32_t *picks = nullptr;                // per-round picks / gains / d_S decreases [n]
  long long *pgain = nullptr, *pdec = nullptr;
  int32_t *goff = nullptr;                 // grid gain kernel: frontier offsets [n+1]
  gc::GainCtl *gctl = nullptr;
  gc::SelCtl *sctl = nullptr;
  gc::SelCtl *h_sctl = nullptr;  // pinned host mirror
  gc::GainCtl *h_gctl = nullptr;
  gc::BfsCtl *h_bctl = nullptr;
  // gain-kernel workspaces: one per resident CTA
  unsigned char *ws = nullptr;
  size_t ws_stride = 0;
  int ws_count = 0;
  int gain_ctas = 0;       // resident CTAs of the gain kernel
  int bfs_ctas = 0;        // resident CTAs of the cooperative BFS
  int grid_ctas = 0;       // resident CTAs of the grid-wide gain kernel
  int lazy_ctas = 0;       // resident CTAs of the persistent lazy kernel
  int red_blocks = 0;      // grid size of reductions
  // wide round-0 kernel (one allocation, made on first use): lane words
  // vis/buf[3] of r0_w 64-bit words per vertex, frontier bitmaps, heavy-row
  // chunk index and accumulators, deferred candidates, control block
  unsigned long long *r0_vis = nullptr, *r0_buf[3] = {nullptr, nullptr, nullptr}, *r0_hacc = nullptr;
  uint32_t *r0_fb[3] = {nullptr, nullptr, nullptr};
  int32_t *r0_hcp = nullptr, *r0_defer = nullptr;
  gc::R0Ctl *r0_ctl = nullptr;
  int r0_w = 0;
  int32_t r0_nh = 0;
  size_t r0_bytes = 0;
  int32_t *dec = nullptr;                  // scratch word
  int64_t launches = 0;                    // kernels launched through this handle
  gc::LaneGraphs lane_graphs;              // set for block-diagonal graph batches
  std::vector<cudaEvent_t> events;         // gain-kernel timing events (pairs)
};

namespace gc {

// ------------------------------------------------------------ errors -------
void set_error(const std::string &msg);
int cuda_fail(cudaError_t e, const char *what);

#define GC_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return gc::cuda_fail(e_, #call); \
  } while (0)

// ------------------------------------------------------------ launches -----
// Grid-wide relabel BFS: dist[w] <- min(dist[w], level) from the seeds,
// expanding only where the label decreased.  dist must already hold either
// kInf (fresh BFS) or the current d_S (pruned update, Sec. 4.1).
// pruned: use the pruned adjacency (g->rpf, g->cif, g->c3; valid only for
// d_S updates after it was built from an earlier d_S) instead of the full CSR.
int launch_bfs_relabel(gc_graph *g, int32_t *dist, const int32_t *seeds, int32_t n_seeds,
                       int64_t timeout_ns, bool pruned = false);
int launch_fill_i32(gc_graph *g, int32_t *p, int32_t v, int64_t count);
int launch_fill_i64(gc_graph *g, long long *p, long long v, int64_t count);
// sum of dist and count of unreached -> sctl->sum, sctl->count
int launch_sum_dist(gc_graph *g, const int32_t *dist);
// round-0 lower bound key[v] = -LB(v) (two-level degree bound)
int launch_round0_keys(gc_graph *g);
// validation: returns GC_OK / GC_EINVAL via sctl->err
int launch_validate(gc_graph *g);

enum GainMode { kModeGain = 0, kModeFarness = 1 };
// Evaluate cand[0..n_cand) in 64-lane batches.  Gain mode: out = Delta(v|S) with
// dS; farness mode: out = f({v}) or -1 if cut by gctl->best_f.
// n_cand_dev (optional) overrides n_cand with a count held in device memory.
// lanes: candidates per batch (1..64); fewer lanes spread one step's work
// over more CTAs.
// pruned (gain mode only): the pruned adjacency, as for launch_bfs_relabel.
int launch_gains(gc_graph *g, int mode, const int32_t *cand, int32_t n_cand,
                 const int32_t *n_cand_dev, long long *out, int max_ctas, int lanes = kLanes,
                 bool pruned = false);
size_t gain_ws_stride(int32_t n);
// Gain mode with 128 or 256 candidates per batch (g->gain_lanes), one CTA per
// batch; the same contract as launch_gains at 64 lanes.
int launch_gains_wide(gc_graph *g, const int32_t *cand, int32_t n_cand, const int32_t *n_cand_dev,
                      long long *out, int max_ctas, bool pruned);
size_t gain_wide_ws_stride(int32_t n, int W);
// One batch of nl <= 64 candidates with every CTA (cooperative launch);
// nl_dev (optional) gives min(64, *nl_dev) instead.
int launch_gains_grid(gc_graph *g, int mode, const int32_t *cand, int32_t nl, const int32_t *nl_dev,
                      long long *out, int64_t timeout_ns, bool pruned = false);
int grid_gain_occupancy(int *blocks_per_sm);
int gain_kernel_occupancy(int *blocks_per_sm);

// selection
// kSelLazy: bound of a candidate not evaluated in `round`; kSelKey: round-0
// key; kSelActive: bound of any non-member (active-list build)
enum SelMode { kSelLazy = 0, kSelKey = 1, kSelActive = 2 };
// tau_mode: kTauHistogram (find tau covering `want` keys), kTauHost (tau given),
// kTauDevice (tau already in sctl->tau)
enum TauMode { kTauHistogram = 0, kTauHost = 1, kTauDevice = 2, kTauHistogramTheta = 3 };
int launch_select(gc_graph *g, int mode, int32_t round, int32_t want, int tau_mode, long long tau);
int launch_after_eval(gc_graph *g, int32_t round, int32_t n_list);
int launch_unevaluated_best(gc_graph *g, int32_t round);
int launch_argmin_f0(gc_graph *g);
int launch_argmin_lb(gc_graph *g);
int launch_round0_seed(gc_graph *g);
// top-k closeness: key <- -f0 for searched vertices; lgain[i] <- f0[list[i]]
int launch_topk_keys(gc_graph *g);
// weighted searches (gc_weighted.cu): kWFarness f({v}) of each listed source,
// kWGain Delta(v|S) of each listed candidate (one CTA per search, out[i] per
// list entry); kWRelabel d_S <- min(d_S, d(s, .)) in place (one CTA)
enum WMode { kWFarness = 0, kWGain = 1, kWRelabel = 2 };
size_t wws_stride(int32_t n);
int wsssp_occupancy(int *blocks_per_sm);
int launch_wsssp(gc_graph *g, int mode, const int32_t *list, const int32_t *m_dev, long long *out,
                 unsigned int *task);
int launch_wrelabel(gc_graph *g, const int32_t *src, unsigned long long *decrease);
int launch_wcheck(gc_graph *g, bool mirror, int32_t *bad, int32_t *max_w);
int launch_iota(gc_graph *g, int32_t *p, int32_t n);
// bitGreedy++ sweep (gc_bits.cu): mode 0 farness of every vertex, mode 1 gain
// of every vertex against d_S; B holds 2 n W words and then 2 n bytes (row
// flags), out n int64; ctl->best
// gets the packed arg-best (see k_bits_argbest)
int launch_bits_round(gc_graph *g, int mode, unsigned long long *B, long long *out, BitsCtl *ctl, int W,
                      int64_t tns);
int launch_gather_f0(gc_graph *g);
int launch_round_begin(gc_graph *g);
int launch_round_end(gc_graph *g);
int launch_clamp_nsel(gc_graph *g, int32_t cap);
int launch_degree_keys(gc_graph *g);
// features of list entries + log1p(gain) targets appended to the recorder
int launch_record(gc_graph *g, int32_t round, long long prev_gain);
// round 1 with the proposal: of the candidates in g->list (n_sel of them, the
// largest bounds, at most 1024), keep the 64 with the largest predicted gain
int launch_round1_propose(gc_graph *g, long long prev_gain);
// mx[u] = max_{w in N(u)} d_S[w] into g->mx_buf (an upper bound for every later d_S)
int launch_max_nbr(gc_graph *g);
// the list of long rows used by the row-wise kernels' CTA-per-row companions
int launch_heavy_rows(gc_graph *g);
// pruned adjacency (g->rpf, g->cif, g->c3) from the d_S now in g->dS
int launch_prune_csr(gc_graph *g);
int launch_round1_bound(gc_graph *g);
// the same bound for the group whose distances are in d_S, over the pruned rows
// of an earlier d_S (any group contained in the current one); lowers ub[v]
int launch_bound_refresh(gc_graph *g);
// ub[v] = -1 where d_S[v] = 0, else +infinity
int launch_init_ub(gc_graph *g);
// *out = sum of two_hop[v] over the selected list g->list[0 .. sctl->n_sel)
int launch_sum_two_hop(gc_graph *g, unsigned long long *out);
// round 0: key[v] = -max(LB(v), LB_p(v)) with p the source of the BFS now in d_S
int launch_pivot_bound(gc_graph *g);
// round 0: an exactly evaluated pivot (sctl->arg_id, farness sctl->sum) becomes
// decided; best_f and tau follow the smallest exact farness so far
int launch_round0_pivot(gc_graph *g);
int launch_active_theta(gc_graph *g);
// prop: proposal weights (nullptr = plain bound order); fill: lanes it chooses
// wide: steps of one 64-lane batch per CTA (else one grid-wide 64-lane batch);
// local_max: largest pick gain whose d_S update runs on one CTA (above it,
// grid-wide)
int launch_lazy_rounds(gc_graph *g, int32_t k, int64_t timeout_ns, const float *prop, int32_t fill,
                       bool wide, long long local_max, int ctas, bool pruned, bool use_log,
                       long long log_cap);
int lazy_occupancy(int *blocks_per_sm);
// round 0 on shallow graphs: f({v}) or -1 (cut / bound above the best) into
// lgain[i] for list[0..m), B = 64 W lanes per batch (W in {1, 2, 4, 8}); a batch
// whose live lanes drop below defer_below after distance 2 defers them;
// count_only lets first-pass batches count distance 2 without writing it;
// probe_stride > 0: those batches first probe the short rows of every
// probe_stride-th window for vertices at distance >= 3 (0 = no probe)
constexpr int32_t kR0ProbeStride = 8;
int launch_round0_wide(gc_graph *g, const int32_t *list, int32_t m, long long *lgain, int W, int32_t defer_below,
                       bool count_only, int64_t timeout_ns, int32_t probe_stride = kR0ProbeStride);
int bfs_kernel_occupancy(int *blocks_per_sm);

}  // namespace gc
