/*
 * gc.h -- C ABI of the GB300 group-closeness library (libgc.so).
 *
 * Greedy++ group-closeness maximization after Bergamini, Gonser and
 * Meyerhenke, "Scaling up Group Closeness Maximization" (arXiv:1710.01144).
 * All compute runs in CUDA kernels for sm_103a on the current device; there
 * is no CPU fallback.  Every entry point returns GC_OK (0) or a negative
 * error code; gc_last_error() gives a thread-local message for the last
 * failure.
 *
 * Definitions (Sec. 2 of the paper; the readings are the library's):
 *   G = (V, E) simple, undirected, unweighted, connected; n = |V|.
 *   d(u, S) = min_{s in S} d(u, s)   (BFS distance, Sec. 2)
 *   farness f(S) = sum_{u in V} d(u, S), an int64.  The paper's closeness is
 *     c(S) = n / f(S); its 1/n normalisation is dropped.  Members contribute 0.
 *   gain Delta(v | S) = f(S) - f(S + {v}) = sum_u max(0, d(u,S) - d(v,u)) >= 0,
 *     the decrease of farness when v joins S (Sec. 4.2 writes the same
 *     quantity with the opposite sign).  Delta(v | S) = 0 for v in S.
 *   Ties between equal gains or equal farness always go to the smaller id.
 *
 * Graph format: int32 CSR.  row_ptr[n+1] with row_ptr[0] = 0 and
 * non-decreasing entries; col_idx[row_ptr[n]] neighbour ids in [0, n); each
 * undirected edge is stored in both rows.  nnz = row_ptr[n] < 2^31.
 *
 * Streams: every call is ordered on the stream given to gc_load_csr (a
 * cudaStream_t passed as void*, NULL = legacy default stream).  Calls that
 * return host results synchronise that stream before returning.
 * A handle must not be used from two threads at once.
 */
#ifndef GC_H_
#define GC_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------------------------------------------------- error codes -- */
#define GC_OK 0
#define GC_EINVAL (-1)        /* bad argument: NULL pointer, k < 1 or k > n,
                                 id outside [0, n), empty group, malformed CSR */
#define GC_EDISCONNECTED (-2) /* some vertex is unreachable (farness undefined) */
#define GC_ERANGE (-3)        /* size limit exceeded (nnz >= 2^31, scratch cap) */
#define GC_ENOMEM (-4)        /* device allocation failed */
#define GC_ECUDA (-5)         /* a CUDA runtime call failed */
#define GC_ETIMEOUT (-6)      /* a device-side wait exceeded its time limit; the
                                 kernel gave up, the context stays usable */
#define GC_EINTERNAL (-7)     /* a device-side consistency check failed */

/* ------------------------------------------------------ gc_load_csr flags -- */
#define GC_DEVICE_PTRS 0x1u /* row_ptr / col_idx are device pointers */
#define GC_ADOPT 0x2u       /* with GC_DEVICE_PTRS: use the caller's device
                               arrays in place (no copy); they must stay alive
                               and unchanged until gc_free */
#define GC_VALIDATE 0x4u    /* check the CSR on the device: row_ptr monotone,
                               ids in range, no self-loops, neighbour lists
                               strictly increasing (so no duplicates), every
                               edge present in both directions, and the graph
                               connected.  Failures return GC_EINVAL or
                               GC_EDISCONNECTED. */

typedef struct gc_graph gc_graph; /* opaque: device CSR + distance/bound arrays + scratch */

/* gc_opts.flags */
#define GC_OPT_NO_EXPAND_BOUND 0x1u
#define GC_OPT_CAPTURE 0x2u /* gc_batch_greedy: record the launch sequence in a
                               CUDA graph once and replay it while ks and the
                               options stay the same */
#define GC_OPT_FULL_ADJACENCY 0x4u /* gc_greedy: scan the full adjacency in rounds
                               >= 1 instead of the pruned one built after round 0
                               (rows without neighbours at d_S <= 1); work only,
                               the group is the same */
#define GC_OPT_R0_FULL_LEVELS 0x10u /* gc_greedy round 0 (wide batches): write every
                               bottom-up level's lane words instead of counting
                               distance 2 only in first-pass batches; work only */
#define GC_OPT_NO_ROUND1_BOUND 0x8u /* gc_greedy, gc_batch_greedy: evaluate every
                               vertex in round 1 instead of only those whose
                               two-hop upper bound reaches the best exact
                               gain, and skip the bound refresh; work only */
#define GC_OPT_NO_CLAIM_LOG 0x20u /* gc_greedy, persistent lazy rounds: update d_S
                               by the relabel BFS from each pick (Sec. 4.1)
                               instead of from the claim log of the pick's
                               gain batch (the same vertices at the same
                               distances); work only */
#define GC_OPT_R0_NO_PROBE 0x40u /* gc_greedy, gc_top_closeness round 0 (wide
                               batches): no far-vertex probe before the
                               count-only distance-2 pass (the probe reads the
                               short rows of every 8th window of 32 vertices
                               first and cuts every lane whose BFScut bound,
                               with the vertices proven at distance >= 3,
                               already exceeds the best farness); work only */

/* Options of gc_greedy; zero-initialise and set what you need
 * (gc_opts_default fills the defaults). */
typedef struct gc_opts {
  int32_t eval_per_step;   /* candidates evaluated exactly per lazy step
                              (rounded up to a multiple of 64); 0 = autotuned */
  int32_t use_proposal;    /* 1: let the learned proposal network set by
                              gc_set_proposal choose part of every batch; the
                              accepted vertex and the group are unchanged */
  int32_t max_ctas;        /* cap on resident CTAs of the gain kernel; 0 = all */
  int32_t timeout_ms;      /* limit of every device-side wait; 0 = 10000 */
  int32_t step_lanes;      /* candidates per 64-lane batch in rounds >= 2 (1..64);
                              fewer lanes spread a step over more CTAs; 0 = 8 */
  int32_t step_mode;       /* rounds >= 2: 0 = default (3), 1 = host-driven steps of
                              eval_per_step candidates in CTA-per-batch form,
                              2 = host-driven steps of one grid-wide batch of the
                              64 largest bounds, 3 = one persistent device kernel
                              for all remaining rounds (grid-wide batches of the
                              64 largest bounds, certification and d_S update on
                              the device) */
  int32_t active_target;   /* step_mode 3: initial size of its candidate list
                              (grown x4 when the list cannot certify a pick);
                              0 = 2048 for grid-wide steps, max(4096, two wide
                              steps) for wide ones */
  int32_t round1_heavy;    /* round 1: this many highest-degree candidates are
                              evaluated by the grid-wide kernel before the
                              CTA-per-batch sweep over the rest; 0 = 1024,
                              negative = none */
  uint32_t flags;          /* GC_OPT_NO_EXPAND_BOUND: do not skip expansions by the
                              neighbour bound (work only; the group is the same) */
  int32_t step_form;       /* step_mode 3: 0 = automatic (wide when the batches of
                              rounds 0-1 averaged more than 16 BFS levels), 1 = one
                              grid-wide 64-lane batch per step, 2 = wide steps: up
                              to 64 candidates per CTA, one CTA-local batch each */
  int32_t local_update_max_gain; /* step_mode 3: a pick whose gain is at most this
                              updates d_S on one CTA; 0 or negative = never */
  int32_t lazy_ctas;       /* step_mode 3: CTAs of the persistent kernel (fewer
                              CTAs make its grid barriers cheaper); 0 = one per
                              SM; clamped to that */
  int32_t batch_grid_min_n; /* gc_batch_greedy: graphs with at least this many
                              vertices run their lazy rounds grid-wide, one
                              graph at a time; the others CTA-locally;
                              0 = 2097152, negative = none */
  int32_t round0_lanes;    /* gc_greedy round 0 on shallow graphs (the BFS from
                              the lowest-bound vertex has at most 32 levels):
                              candidates per wide bottom-up batch, 64, 128, 256
                              or 512; 0 = automatic; negative = the 64-lane
                              batches used for deep graphs */
  int32_t timeout_us;      /* if > 0: the limit of every device-side wait in
                              microseconds, overriding timeout_ms (a limit
                              that short makes the waits give up with
                              GC_ETIMEOUT; the handle stays usable) */
  int32_t claim_log_cap;   /* if > 0: at most this many claim-log entries per
                              round of the persistent lazy kernel (default: the
                              log allocated at load, 2n entries clamped to
                              [2^20, 2^24]); a round whose log outgrows it
                              updates d_S by the relabel BFS; work only */
} gc_opts;

/* Work counters of the last gc_greedy / gc_marginal_gains call. */
typedef struct gc_stats {
  int64_t rounds;          /* greedy rounds completed (= k) */
  int64_t steps;           /* lazy evaluation steps over all rounds >= 1 */
  int64_t evals;           /* exact gains computed (rounds >= 1) */
  int64_t batches;         /* 64-lane batches run by the gain kernel */
  int64_t edges_scalar;    /* adjacency entries a one-source pruned BFS per
                              candidate would scan (sum over lanes) */
  int64_t edges_union;     /* adjacency entries the 64-lane kernel scanned */
  int64_t levels;          /* BFS levels summed over batches */
  int64_t frontier;        /* frontier entries (vertex, lane word) expanded */
  int64_t pushes;          /* vertices that entered a next-level frontier */
  int64_t lanes;           /* candidate lanes processed (all launches) */
  int64_t round0_evals;    /* candidates evaluated (exactly or cut) in round 0 */
  double ms_round0;        /* time of round 0 (top-1 closeness + d_S) */
  double ms_round1;        /* time of round 1 */
  double ms_total;         /* time of the whole call */
  double ms_gain_kernel;   /* summed duration of gain-kernel launches (host-driven
                              steps; the persistent kernel's phases are below) */
  double ms_lazy_select;   /* persistent kernel: candidate selection and certification */
  double ms_lazy_gain;     /* persistent kernel: grid-wide 64-lane gain batches */
  double ms_lazy_update;   /* persistent kernel: d_S updates from the picks */
  int64_t gain_launches;   /* gain-kernel launches */
  int64_t kernel_launches; /* all kernel launches of the call */
  int64_t graph_replay;    /* gc_batch_greedy: 1 if the solve ran from a captured CUDA graph */
  /* gc_greedy: the CTA-batched 64-lane gain kernel alone (its launches are a
     subset of gain_launches; the grid-wide batches are the rest) */
  int64_t gain64_launches; /* its launches */
  double ms_gain64;        /* their summed duration (CUDA events on the launch stream) */
  int64_t gain64_frontier; /* frontier entries they expanded */
  int64_t gain64_edges;    /* adjacency entries they scanned */
  int64_t gain64_pushes;   /* vertices they pushed into a next-level frontier */
  int64_t gain64_lanes;    /* candidate lanes they processed */
  /* gc_greedy: gain phases of the persistent lazy kernel (time: ms_lazy_gain) */
  int64_t lazy_frontier;
  int64_t lazy_edges;
  int64_t lazy_pushes;
  int64_t lazy_lanes;
  /* gc_greedy: the persistent lazy kernel as a whole */
  int64_t lazy_launches;     /* its launches (1 + list rebuilds) */
  double ms_lazy_kernel;     /* their summed duration (CUDA events on the launch stream) */
  int64_t lazy_upd_frontier; /* d_S updates: frontier entries expanded */
  int64_t lazy_upd_edges;    /* d_S updates: adjacency entries scanned */
  int64_t lazy_upd_relabels; /* d_S updates: labels lowered */
  int64_t lazy_sel_scanned;  /* selection: active-list entries read */
  /* gc_greedy round 0: the wide bottom-up kernel (shallow graphs) */
  double ms_round0_wide;     /* its duration (CUDA events on the launch stream) */
  int64_t r0_batches;        /* its batches */
  int64_t r0_levels;         /* bottom-up levels summed over batches */
  int64_t r0_td_edges;       /* adjacency entries of its top-down levels */
  double ms_r0_select;       /* its phases by the clock of its first CTA: batch selection, */
  double ms_r0_topdown;      /* the top-down first level, */
  double ms_r0_bottomup;     /* the bottom-up levels with their BFScut folds, */
  double ms_r0_clear;        /* and the clearing of the lane words after each batch */
  int64_t r0_bu_rows;        /* bottom-up: vertices whose words a claim wrote */
  int64_t r0_bu_scanned;     /* bottom-up: adjacency entries read */
  int64_t r0_bu_gathers;     /* bottom-up: frontier lane words gathered */
  int64_t r0_width;          /* its candidates per batch (0: not used) */
  int64_t r0_dense_clears;   /* its batches that cleared every visited word */
  /* gc_greedy: d_S updates of the persistent lazy kernel taken from the claim
   * log (the rest ran the relabel BFS) */
  int64_t lazy_log_picks;    /* picks updated from the log */
  int64_t lazy_upd_log;      /* log entries those updates read */
  int64_t lazy_log_entries;  /* log entries the gain phases wrote (16 bytes each) */
  int64_t r0_probes;         /* round 0, wide batches: far-vertex probe stages run */
  int64_t r0_probe_cut;      /* and the lanes they cut */
  int64_t r0_bu_vertices;    /* bottom-up: vertices whose row pointers were read */
  int64_t r0_bu_visreads;    /* bottom-up: visited lane words read (per vertex) */
} gc_stats;

/* gc_opts_default: fill *opts with the defaults.  Returns GC_OK or GC_EINVAL. */
int gc_opts_default(gc_opts *opts);

/* gc_load_csr -- create a graph handle.
 * n        : vertex count, 1 <= n < 2^31.
 * row_ptr  : int32[n+1]; col_idx : int32[row_ptr[n]]; host pointers unless
 *            flags has GC_DEVICE_PTRS.  Without GC_ADOPT the arrays are copied
 *            and the caller keeps ownership of its buffers.
 * flags    : GC_DEVICE_PTRS | GC_ADOPT | GC_VALIDATE.
 * stream   : cudaStream_t (as void*) on which this handle's work is ordered.
 * out      : receives the handle; release it with gc_free.
 * Errors   : GC_EINVAL (NULL, n < 1, row_ptr[0] != 0, GC_ADOPT without
 *            GC_DEVICE_PTRS, or a GC_VALIDATE failure), GC_ERANGE (nnz out of
 *            int32 range), GC_EDISCONNECTED (GC_VALIDATE only), GC_ENOMEM,
 *            GC_ECUDA.  Nothing is allocated on failure. */
int gc_load_csr(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, uint32_t flags,
                void *stream, gc_graph **out);

/* gc_free -- release the handle and its device memory (adopted arrays are left
 * alone).  NULL is accepted.  Returns GC_OK. */
int gc_free(gc_graph *g);

/* gc_num_vertices / gc_num_entries -- n and nnz of a handle (-1 on NULL). */
int64_t gc_num_vertices(const gc_graph *g);
int64_t gc_num_entries(const gc_graph *g);

/* gc_group_farness -- f(S) = sum_u d(u, S) (Sec. 2) by one multi-source BFS.
 * S        : host int32[s_len] vertex ids (duplicates allowed), s_len >= 1.
 * out      : host int64.
 * Errors   : GC_EINVAL (NULL, s_len < 1, id out of range), GC_EDISCONNECTED. */
int gc_group_farness(gc_graph *g, const int32_t *S, int32_t s_len, int64_t *out_farness);

/* gc_marginal_gains -- Delta(v | S) for each candidate v (Sec. 4.1 pruned SSSP,
 * evaluated 64 candidates at a time (128 or 256 after gc_set_gain_lanes) by
 * a bit-parallel multi-source BFS in the form of Theorem 1, Sec. 4.3).
 * S        : host int32[s_len], s_len >= 1 (d(., empty set) is undefined).
 * cand     : host int32[n_cand], any ids in [0, n), repeats allowed, n_cand >= 0.
 * out_gain : host int64[n_cand]; 0 for candidates in S.
 * stats    : optional (NULL), filled with the kernel's work counters.
 * Errors   : GC_EINVAL, GC_EDISCONNECTED. */
int gc_marginal_gains(gc_graph *g, const int32_t *S, int32_t s_len, const int32_t *cand,
                      int32_t n_cand, int64_t *out_gain, gc_stats *stats);

/* gc_set_gain_lanes -- candidates per batch of the CTA-batched gain kernel:
 * the width of the lane words of the bit-parallel pruned BFS (Sec. 4.1 with
 * the bit vectors of Theorem 1, Sec. 4.3; one bit per candidate, one scan of
 * a frontier vertex's row for every candidate that reached it at that level).
 * lanes    : 64 (default: one uint64 word per vertex), 128 or 256 (two or four
 *            words per vertex, 64 or 128 bytes of lane words and flags per
 *            vertex in each CTA's workspace, allocated on the first call that
 *            uses it and kept until gc_free).
 * Applies to every later gain evaluation of the handle that runs whole batches
 * one per CTA: gc_marginal_gains, gc_marginal_gains_device, and gc_greedy's
 * round-1 sweep and host-driven lazy steps (step_mode 1 with step_lanes 64).
 * Batches of fewer lanes, grid-wide batches
 * and the persistent lazy kernel keep 64 lanes.  Results never depend on it.
 * Errors   : GC_EINVAL (NULL handle, lanes not 64, 128 or 256). */
int gc_set_gain_lanes(gc_graph *g, int32_t lanes);

/* gc_marginal_gains_device -- as gc_marginal_gains with device pointers for
 * S, cand and out_gain; asynchronous on the handle's stream (no sync, no
 * host-visible error for bad ids: ids are checked on the device and an
 * out-of-range id yields gain -1 for that candidate). */
int gc_marginal_gains_device(gc_graph *g, const int32_t *S_dev, int32_t s_len,
                             const int32_t *cand_dev, int32_t n_cand, int64_t *out_gain_dev);

/* gc_marginal_gains_static -- the gains of gc_marginal_gains for callers that
 * cannot allocate device memory: plugins confined to a host application's own
 * allocator or fixed memory budget (a raw cudaMalloc would bypass both), and
 * request paths where allocator calls are not allowed (cudaMalloc and cudaFree
 * can synchronise the device and take unbounded time).  The paper has no
 * counterpart; this is a deployment variant.
 * It calls no cudaMalloc/cudaFree and creates no handle: all scratch lives in
 * one 64 MiB array compiled into the library, which every GPU that loads the
 * library keeps until the process exits.
 * n, row_ptr, col_idx : the CSR as device pointers (same format as above).
 * S, cand, out_gain   : device int32[s_len], int32[n_cand], int64[n_cand];
 *            s_len >= 1; out_gain[i] = Delta(cand[i] | S), or -1 for an id
 *            outside [0, n).
 * stream   : cudaStream_t (as void*); the call is asynchronous on it.
 * Device-side failures: when the BFS from S fails -- an id of S outside
 *            [0, n), a device-side wait that timed out, or a vertex that S does
 *            not reach (a disconnected graph) -- every out_gain entry is -1.
 *            Nothing is reported to the host, since that needs a
 *            synchronisation.
 * Limits   : n <= 1,048,496 (64 bytes of scratch per vertex: 20 for d(., S)
 *            and the BFS queues, 44 for one gain workspace, each part 256-byte
 *            aligned); a larger n returns GC_ERANGE before anything runs.
 *            Smaller graphs get more workspaces and so more parallel CTAs
 *            (about 14 at n = 100,000; one at n = 646,000).
 * Sharing  : all calls in the process share the one array, which keeps what the
 *            last call left.  Each call zeroes the parts it uses, so calls
 *            ordered on one stream are safe, but calls that overlap on the GPU
 *            (different streams or threads) race and give wrong results.
 * Set-up   : the first call on a device (with that device current) looks up the
 *            array's device address once with cudaGetSymbolAddress; make that
 *            first call before any stream capture begins.
 * Errors   : GC_EINVAL (NULL or bad sizes), GC_ERANGE (n too large), GC_ECUDA. */
int gc_marginal_gains_static(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                             const int32_t *S, int32_t s_len, const int32_t *cand, int32_t n_cand,
                             int64_t *out_gain, void *stream);

/* gc_gain_upper_bounds -- for every vertex v, an upper bound on Delta(v | S)
 * that needs no search from v (the paper gives no bound before a candidate's
 * first exact evaluation; this is the library's own, used to start the lazy
 * rounds of gc_greedy at round 1 and to tighten the bounds later):
 *   Delta(v | S) <= d_S[v] + sum_{w in N(v)} ((d_S[w] - 1)^+ + c3[w])
 *                   + sum_u (d_S[u] - 3)^+,
 * with d_S = d(., S) and c3[w] = #{u in N(w) : d_S[u] >= 3}.  A vertex at
 * distance 1 from v gains at most d_S - 1, one at distance 2 at most
 * [d_S >= 3] + (d_S - 3)^+ (and it is a neighbour of some w in N(v)), any other
 * at most (d_S - 3)^+.
 * S        : host int32[s_len] vertex ids, s_len >= 1.
 * out_ub   : host int64[n]; -1 for members of S.
 * Errors   : GC_EINVAL, GC_EDISCONNECTED. */
int gc_gain_upper_bounds(gc_graph *g, const int32_t *S, int32_t s_len, int64_t *out_ub);

/* gc_greedy -- Greedy++ (Algorithm 2 with pruned SSSPs, Sec. 4.1, and the lazy
 * supermodular bounds, Sec. 4.2): s0 = argmin_v f({v}) (top-1 closeness,
 * Sec. 3.1), then k-1 rounds adding argmax_v Delta(v | S).
 * k          : 1 <= k <= n.
 * opts       : NULL = defaults.
 * out_group  : host int32[k], vertices in pick order (s0 first).
 * out_farness: host int64, f(S) of the final group.
 * stats      : optional work counters.
 * The group equals the plain greedy of Algorithm 2 with smallest-id ties.
 * Errors   : GC_EINVAL, GC_EDISCONNECTED, GC_ETIMEOUT, GC_ENOMEM, GC_ECUDA. */
int gc_greedy(gc_graph *g, int32_t k, const gc_opts *opts, int32_t *out_group,
              int64_t *out_farness, gc_stats *stats);

/* gc_top_closeness -- top-k closeness (Sec. 3.1, Algorithm 3 with general k):
 * the k vertices of smallest single-vertex farness f({v}) = sum_u d(v, u), in
 * increasing order of (farness, id).  Bit-parallel BFScut searches as in round
 * 0 of gc_greedy, with the cut fixed at an upper bound of the k-th smallest
 * farness (the k-th best of at least k exact probe searches), so no vertex of
 * the result is ever cut.  k = 1 gives s0 of gc_greedy.
 * k          : 1 <= k <= n.
 * opts       : NULL = defaults (round0_lanes, max_ctas, timeout, flags
 *              GC_OPT_R0_FULL_LEVELS are used).
 * out_ids    : host int32[k], the vertices in order.
 * out_farness: host int64[k], their farness values.
 * stats      : optional; round0_evals = vertices searched (probes and
 *              survivors of the bound), ms_total, kernel_launches.
 * Errors   : GC_EINVAL, GC_EDISCONNECTED, GC_ETIMEOUT, GC_ENOMEM, GC_ECUDA. */
int gc_top_closeness(gc_graph *g, int32_t k, const gc_opts *opts, int32_t *out_ids, int64_t *out_farness,
                     gc_stats *stats);

/* gc_set_weights -- attach positive integer edge weights to a handle, for the
 * weighted entry points (the paper's weighted case: every SSSP a
 * shortest-path search, Sec. 3.2).
 * weights : int32[nnz] aligned with col_idx, host (copied) or device
 *           (flags & GC_DEVICE_PTRS, copied); every weight >= 1 and the same
 *           in both rows of an edge.
 * flags   : GC_DEVICE_PTRS | GC_VALIDATE (also check the two rows agree).
 * Errors  : GC_EINVAL (a weight below 1, or rows that disagree under
 *           GC_VALIDATE), GC_ERANGE ((n - 1) x max weight >= 2^30: path
 *           lengths could overflow the int32 distances), GC_ENOMEM, GC_ECUDA. */
int gc_set_weights(gc_graph *g, const int32_t *weights, uint32_t flags);

/* gc_greedy_weighted -- Greedy on the weighted graph: Algorithm 2 with weighted
 * distances, the pruned searches of Sec. 4.1 (valid for positive weights) and
 * the lazy bounds of Sec. 4.2; s0 = argmin f({v}) by a full search from every
 * vertex; ties to the smallest id.  Farness = sum of weighted distances (int64).
 * Requires gc_set_weights.  k, opts, out_group, out_farness, stats: as
 * gc_greedy (stats: rounds, steps, evals, round0_evals, ms_total, launches).
 * Errors   : GC_EINVAL (no weights, bad k), GC_EDISCONNECTED, GC_ENOMEM,
 *            GC_ECUDA. */
int gc_greedy_weighted(gc_graph *g, int32_t k, const gc_opts *opts, int32_t *out_group, int64_t *out_farness,
                       gc_stats *stats);

/* gc_greedy_bits -- bitGreedy++ (Sec. 4.3, Theorem 1): the same group as
 * gc_greedy, with every round scoring EVERY vertex by bit vectors: b^i_u (the
 * vertices within distance i of u) built level by level by ORs over the
 * neighbours, the gain of u being sum_i |b^i_u AND NOT b^i_S| and, in round 0,
 * the farness of u being sum_i (n - |b^i_u|).  The vectors are held for 64 W
 * target vertices at a time (W <= 32 words per vertex, two buffers of n x W
 * words: the memory limit), and a target's bit is dropped once d_S of the
 * target is reached (pruning).  No lazy bounds: every round is a full sweep.
 * For small graphs: n <= 65536.
 * k, opts, out_group, out_farness, stats: as gc_greedy (stats: rounds, levels
 * swept, evals = n k, ms_total, kernel_launches).
 * Errors   : GC_EINVAL, GC_ERANGE (n > 65536), GC_EDISCONNECTED, GC_ETIMEOUT,
 *            GC_ENOMEM, GC_ECUDA. */
int gc_greedy_bits(gc_graph *g, int32_t k, const gc_opts *opts, int32_t *out_group, int64_t *out_farness,
                   gc_stats *stats);

/* ------------------------------------------------- learned proposal ---- */
/* A small network that only ORDERS exact evaluations (not part of the paper;
 * the acceptance rule of Sec. 4.2 is unchanged, so the group is identical with
 * or without it).  Network: 8 float features -> 64 -> 64 (ReLU) -> 1, float32,
 * GC_MLP_PARAMS parameters in the order W1[8][64], b1[64], W2[64][64], b2[64],
 * W3[64], b3.  Features of candidate v in round r: log1p(deg v), d_S[v],
 * log1p(stale bound), r - (round of its last evaluation), log1p(sum over
 * neighbours of (deg - 1)), max d_S over neighbours - d_S[v], log1p(gain of
 * the previous pick), and feature 2 - feature 6.  Trained (mean squared error
 * on log1p of exact gains, Adam) by the library's own kernels. */
#define GC_MLP_IN 8
#define GC_MLP_HIDDEN 64
#define GC_MLP_PARAMS 4801

typedef struct gc_mlp gc_mlp; /* opaque: parameters, Adam state, activation scratch */

/* gc_mlp_create -- a network with zero parameters; max_batch bounds the
 * minibatch of gc_mlp_grad / gc_mlp_adam_step / gc_mlp_train.  stream as in
 * gc_load_csr.  Errors: GC_EINVAL, GC_ENOMEM. */
int gc_mlp_create(int32_t max_batch, void *stream, gc_mlp **out);
/* gc_mlp_free -- release (NULL accepted). */
int gc_mlp_free(gc_mlp *mlp);
/* gc_mlp_set_params / gc_mlp_get_params -- host float[GC_MLP_PARAMS]; setting
 * resets the Adam state.  Synchronous. */
int gc_mlp_set_params(gc_mlp *mlp, const float *params);
int gc_mlp_get_params(gc_mlp *mlp, float *params);
/* gc_mlp_forward -- out[i] = network(X[i]) for device float X[m][8], out[m];
 * asynchronous on the network's stream. */
int gc_mlp_forward(gc_mlp *mlp, const float *X, int32_t m, float *out);
/* gc_mlp_grad -- gradient of L = (1/m) sum (out_i - y_i)^2 with respect to the
 * parameters, for device X[m][8], y[m], 1 <= m <= max_batch; grad is a host
 * float[GC_MLP_PARAMS] (may be NULL), loss a host double (may be NULL).
 * Synchronous. */
int gc_mlp_grad(gc_mlp *mlp, const float *X, const float *y, int32_t m, float *grad, double *loss);
/* gc_mlp_adam_step -- one Adam step (beta1 0.9, beta2 0.999, eps 1e-8) on the
 * minibatch X[m][8], y[m] (device); asynchronous. */
int gc_mlp_adam_step(gc_mlp *mlp, const float *X, const float *y, int32_t m, float lr);
/* gc_mlp_train -- `epochs` passes over device X[m][8], y[m] in minibatches of
 * `batch` (<= max_batch) taken in a seeded random order; final_loss (host, may be
 * NULL) gets the mean squared error over the whole set afterwards. */
int gc_mlp_train(gc_mlp *mlp, const float *X, const float *y, int32_t m, int32_t epochs, int32_t batch,
                 float lr, uint64_t seed, double *final_loss);
/* gc_candidate_features -- the network's input rows X[m][8] (device float) for
 * candidates cand[m] given the per-vertex device arrays row_ptr[n+1], d_S[n],
 * bound ub[n], evaluation round stamp[n], two_hop[n] (sum over neighbours of
 * deg - 1) and mx[n] (max d_S over neighbours; NULL = d_S itself), the round
 * and the previous pick's gain.  Asynchronous on `stream`. */
int gc_candidate_features(const int32_t *row_ptr, const int32_t *dS, const int64_t *ub, const int32_t *stamp,
                          const int64_t *two_hop, const int32_t *mx, const int32_t *cand, int32_t m, int32_t round,
                          int64_t prev_gain, float *X, void *stream);
/* gc_set_proposal -- let gc_greedy (opts.use_proposal = 1) use the network:
 * round 1's first exact batch becomes the 64 of the 1024 largest two-hop
 * bounds with the largest predicted gain (instead of the 64 largest bounds);
 * its best exact gain is the level every other round-1 candidate's bound must
 * reach.  With fill > 0, `fill` of every 64-candidate batch of the persistent
 * lazy rounds also go to the unevaluated candidates whose stale bound most
 * exceeds the predicted gain, the rest to the largest bounds.  The network
 * must outlive its use; NULL disables.  Errors: GC_EINVAL (fill outside
 * [0, 63]). */
int gc_set_proposal(gc_graph *g, const gc_mlp *mlp, int32_t fill);
/* gc_set_recorder -- while set (cap > 0), gc_greedy appends training samples
 * for the proposal: each candidate's features at selection time to X[cap][8]
 * and log1p(exact gain) to y[cap] (device arrays owned by the caller), for
 * the host-driven lazy steps of rounds >= 2 (opts.step_mode 1 or 2) and, with
 * the round-1 bounds, for the 1024 largest round-1 bounds (all evaluated
 * exactly in such a recording call); gc_recorded returns the row count. */
int gc_set_recorder(gc_graph *g, float *X, float *y, int32_t cap);
int64_t gc_recorded(gc_graph *g);

/* ------------------------------------------------- batched solving ----- */
/* Many graphs solved together: the batch is held as one block-diagonal union
 * graph on the device and solved by ONE persistent cooperative kernel (round 0,
 * round 1 and every lazy round of every graph, no host round trip), optionally
 * replayed from a captured CUDA graph (opts.flags & GC_OPT_CAPTURE).  Each
 * graph's group equals gc_greedy's on that graph alone. */
typedef struct gc_batch gc_batch; /* opaque: union CSR + per-graph state */

/* gc_batch_load -- count graphs given by host CSR arrays row_ptrs[g],
 * col_idxs[g] with ns[g] vertices (each connected, format as for gc_load_csr).
 * flags: reserved (0).  Errors: GC_EINVAL, GC_ERANGE (union beyond int32 CSR),
 * GC_ENOMEM, GC_ECUDA. */
int gc_batch_load(int32_t count, const int32_t *const *row_ptrs, const int32_t *const *col_idxs, const int32_t *ns,
                  uint32_t flags, void *stream, gc_batch **out);
int gc_batch_free(gc_batch *b);
int64_t gc_batch_vertices(const gc_batch *b);
/* gc_batch_greedy -- ks[count] group sizes (1 <= ks[g] <= ns[g]).  groups
 * (host int32[sum ks]) receives each graph's group in pick order, graph after
 * graph, in the graph's own vertex ids; farness (host int64[count]) each
 * group's farness.  opts: active_target = per-graph candidate-list capacity
 * (0 = 1024), step_lanes = candidates per round-1 batch (0 = 64), timeout_ms,
 * flags (GC_OPT_CAPTURE).  Errors: GC_EINVAL, GC_EDISCONNECTED, GC_ETIMEOUT,
 * GC_ERANGE (a gain >= 2^31), GC_ENOMEM, GC_ECUDA. */
int gc_batch_greedy(gc_batch *b, const int32_t *ks, const gc_opts *opts, int32_t *groups, int64_t *farness,
                    gc_stats *stats);

/* gc_greedy_batch -- the batched solve of gc_batch_greedy over graphs already
 * loaded with gc_load_csr (all on the current device).  gs[count] handles;
 * ks[count] group sizes (1 <= ks[g] <= n of graph g); opts as for
 * gc_batch_greedy; out_groups[g] (host int32[ks[g]]) receives graph g's group
 * in pick order, out_farness (host int64[count]) each group's farness.  Each
 * group equals gc_greedy's on that graph alone.  Every call gathers the
 * handles' CSRs into one union on the device (one device-to-device copy of
 * each CSR plus the batch's scratch): repeated solves of the same graphs are
 * cheaper through gc_batch_load + gc_batch_greedy.  The handles are not
 * changed.  Synchronous.  Errors: as gc_batch_greedy. */
int gc_greedy_batch(gc_graph *const *gs, const int32_t *ks, int32_t count, const gc_opts *opts,
                    int32_t *const *out_groups, int64_t *out_farness, gc_stats *stats);

/* gc_last_error -- thread-local description of the last failure ("" if none). */
const char *gc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GC_H_ */
