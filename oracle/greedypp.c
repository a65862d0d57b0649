/*
 * CPU oracle, part 2 ("O2"): the paper's Greedy++ on the CPU, for graphs too
 * large for the plain oracle of oracle.c.
 *
 * TEST INFRASTRUCTURE ONLY (tests, smoke check, CPU-baseline leg of the
 * benchmark).  Shares no code with the CUDA library.
 *
 * Steps in the paper's order:
 *   s0       : top-1 closeness (Sec. 3.1, Algorithm 3 with k=1): vertices in
 *              decreasing degree order (ties: smaller id first); each BFS is
 *              cut once the bound "every unvisited vertex sits at distance
 *              d+1" already shows it cannot beat the best found so far.  The
 *              cut is tie-safe: a vertex is cut only if (bound, id) exceeds
 *              (best farness, best id) lexicographically, so the smallest-id
 *              minimiser survives.
 *   d_S      : BFS from s0 (Algorithm 2).
 *   rounds   : every vertex not in S is scored by a pruned SSSP (Sec. 4.1: a
 *              vertex w reached at distance L contributes d_S[w] - L when
 *              L < d_S[w] and only then has its neighbours enqueued); scores
 *              from earlier rounds are upper bounds (Sec. 4.2, supermodularity
 *              of farness), so candidates are visited in decreasing bound order
 *              and the round stops once the best exact gain beats every
 *              remaining bound.  Ties: larger gain, then smaller id.
 *   update   : d_S <- min(d_S, d(pick, .)) by a pruned SSSP from the pick
 *              (Sec. 4.1: pruning leaves d_S unchanged).
 * The first round scores every vertex (no bound exists yet); it runs as an
 * OpenMP parallel loop, as in the paper's parallel Greedy++ (Sec. 6.4).
 * Its result must equal or_greedy_plain bit for bit (Sec. 4.1, Sec. 4.2 with
 * the smallest-id tie rule); the tests check that on small graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t *dist;    /* -1 = unvisited */
  int32_t *queue;   /* vertices to expand, in BFS order */
  int32_t *touched; /* every visited vertex, for the reset */
} bfs_ws;

static int ws_init(bfs_ws *w, int32_t n) {
  w->dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  w->queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  w->touched = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!w->dist || !w->queue || !w->touched) {
    free(w->dist); free(w->queue); free(w->touched); return -1;
  }
  for (int32_t i = 0; i < n; ++i) w->dist[i] = -1;
  return 0;
}
static void ws_free(bfs_ws *w) { free(w->dist); free(w->queue); free(w->touched); }

/* Pruned SSSP from v (Sec. 4.1).  Returns Delta(v|S); adds the number of
 * scanned adjacency entries to *edges.  Leaves w->dist all -1 on return. */
static int64_t pruned_gain(const int32_t *row_ptr, const int32_t *col_idx, const int32_t *dS,
                           int32_t v, bfs_ws *w, int64_t *edges) {
  if (dS[v] == 0) return 0;
  int64_t head = 0, tail = 0, nt = 0, g = 0, scanned = 0;
  w->dist[v] = 0; w->touched[nt++] = v; w->queue[tail++] = v;
  g += dS[v];
  while (head < tail) {
    int32_t u = w->queue[head++];
    int32_t du = w->dist[u];
    /* the queue only holds vertices with du < dS[u] */
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t x = col_idx[e];
      ++scanned;
      if (w->dist[x] >= 0) continue;
      w->dist[x] = du + 1;
      w->touched[nt++] = x;
      if (du + 1 < dS[x]) {  /* strictly closer to v than to S: counts, expands */
        g += dS[x] - (du + 1);
        w->queue[tail++] = x;
      }                        /* otherwise visited, pruned: no neighbours enqueued */
    }
  }
  for (int64_t i = 0; i < nt; ++i) w->dist[w->touched[i]] = -1;
  if (edges) *edges += scanned;
  return g;
}

/* d_S <- min(d_S, d(s,.)) by a pruned SSSP from s: only vertices strictly
 * closer to s than to S are relabelled and expanded.  Returns the decrease of
 * farness (= Delta(s|S) before the update). */
static int64_t pruned_update(const int32_t *row_ptr, const int32_t *col_idx, int32_t *dS, int32_t s,
                             int32_t *queue) {
  if (dS[s] == 0) return 0;
  int64_t head = 0, tail = 0, g = dS[s];
  dS[s] = 0; queue[tail++] = s;
  while (head < tail) {
    int32_t u = queue[head++];
    int32_t du = dS[u];
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t x = col_idx[e];
      if (du + 1 < dS[x]) { g += dS[x] - (du + 1); dS[x] = du + 1; queue[tail++] = x; }
    }
  }
  return g;
}

/* BFS from v with the Algorithm-3 cut against (best_f, best_id).
 * Returns f({v}) if the BFS completed, or -1 if it was cut. */
static int64_t bfscut(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t v,
                      int64_t best_f, int32_t best_id, bfs_ws *w) {
  int64_t head = 0, tail = 0, sum = 0, cut = 0;
  w->dist[v] = 0; w->queue[tail++] = v;
  int32_t level = 0;
  while (head < tail) {
    /* level `level` is complete in queue[head..tail): every vertex at
     * distance <= level is visited; the rest are at least level+1 away */
    if (best_f >= 0) {
      int64_t lb = sum + (int64_t)(level + 1) * (n - tail);
      if (lb > best_f || (lb == best_f && v > best_id)) { cut = 1; break; }
    }
    int64_t lvl_end = tail;
    while (head < lvl_end) {
      int32_t u = w->queue[head++];
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
        int32_t x = col_idx[e];
        if (w->dist[x] < 0) { w->dist[x] = level + 1; sum += level + 1; w->queue[tail++] = x; }
      }
    }
    ++level;
  }
  for (int64_t i = 0; i < tail; ++i) w->dist[w->queue[i]] = -1;
  if (cut) return -1;
  if (tail != n) return -2; /* disconnected */
  return sum;
}

typedef struct {
  int64_t evals;        /* pruned SSSPs run in rounds >= 1 */
  int64_t edges;        /* adjacency entries scanned by them */
  int64_t round0_full;  /* BFScut runs that completed */
} or_gpp_stats;

/* Top-1 closeness: s0 = argmin f({v}), ties -> smallest id. */
int or_top1_closeness(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t nthreads,
                      int32_t *s0_out, int64_t *f0_out, int64_t *n_full) {
  int nt = nthreads > 0 ? nthreads : 1;
  int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!order) return -2;
  /* decreasing degree, then increasing id: counting sort by degree */
  int32_t maxd = 0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t d = row_ptr[v + 1] - row_ptr[v];
    if (d > maxd) maxd = d;
  }
  int64_t *cnt = (int64_t *)calloc((size_t)maxd + 2, sizeof(int64_t));
  if (!cnt) { free(order); return -2; }
  for (int32_t v = 0; v < n; ++v) cnt[maxd - (row_ptr[v + 1] - row_ptr[v]) + 1]++;
  for (int32_t d = 1; d <= maxd + 1; ++d) cnt[d] += cnt[d - 1];
  for (int32_t v = 0; v < n; ++v) order[cnt[maxd - (row_ptr[v + 1] - row_ptr[v])]++] = v;
  free(cnt);

  int64_t best_f = -1;
  int32_t best_id = -1;
  int64_t full = 0;
  int err = 0;
#pragma omp parallel num_threads(nt)
  {
    bfs_ws w;
    int ok = ws_init(&w, n) == 0;
    if (!ok) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = 0; i < n; ++i) {
      if (!ok) continue;
      int32_t v = order[i];
      int64_t bf;
      int32_t bi;
#pragma omp critical(gpp_best)
      { bf = best_f; bi = best_id; }
      int64_t f = bfscut(n, row_ptr, col_idx, v, bf, bi, &w);
      if (f == -2) {
#pragma omp atomic write
        err = 2;
      }
      if (f >= 0) {
#pragma omp atomic
        full++;
#pragma omp critical(gpp_best)
        {
          if (best_f < 0 || f < best_f || (f == best_f && v < best_id)) { best_f = f; best_id = v; }
        }
      }
    }
    if (ok) ws_free(&w);
  }
  free(order);
  if (err) return err == 1 ? -2 : -1;
  *s0_out = best_id; *f0_out = best_f;
  if (n_full) *n_full = full;
  return 0;
}

/* Top-k closeness (Sec. 3.1, Algorithm 3 with general k): the k vertices of
 * smallest farness f({v}), ordered by (farness, id).  Vertices are searched in
 * decreasing degree order (ties: smaller id first).  While fewer than k
 * searches have completed nothing is cut; afterwards a BFS is cut once its
 * bound exceeds the k-th best (farness, id) pair found so far, lexicographically
 * (tie-safe, as in the top-1 search).  A completed search replaces the k-th best
 * when it is smaller.  ids_out / f_out receive the k results in order.
 * Returns 0, -1 (disconnected or k outside [1, n]) or -2 (allocation). */
int or_topk_closeness(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t k, int32_t nthreads,
                      int32_t *ids_out, int64_t *f_out, int64_t *n_full) {
  if (k < 1 || k > n) return -1;
  int nt = nthreads > 0 ? nthreads : 1;
  int32_t *order = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int64_t *top_f = (int64_t *)malloc((size_t)k * sizeof(int64_t));
  int32_t *top_id = (int32_t *)malloc((size_t)k * sizeof(int32_t));
  if (!order || !top_f || !top_id) { free(order); free(top_f); free(top_id); return -2; }
  int32_t maxd = 0;
  for (int32_t v = 0; v < n; ++v) {
    int32_t d = row_ptr[v + 1] - row_ptr[v];
    if (d > maxd) maxd = d;
  }
  int64_t *cnt = (int64_t *)calloc((size_t)maxd + 2, sizeof(int64_t));
  if (!cnt) { free(order); free(top_f); free(top_id); return -2; }
  for (int32_t v = 0; v < n; ++v) cnt[maxd - (row_ptr[v + 1] - row_ptr[v]) + 1]++;
  for (int32_t d = 1; d <= maxd + 1; ++d) cnt[d] += cnt[d - 1];
  for (int32_t v = 0; v < n; ++v) order[cnt[maxd - (row_ptr[v + 1] - row_ptr[v])]++] = v;
  free(cnt);

  int32_t have = 0;  /* results so far, kept sorted by (farness, id) in top_f / top_id */
  int64_t full = 0;
  int err = 0;
#pragma omp parallel num_threads(nt)
  {
    bfs_ws w;
    int ok = ws_init(&w, n) == 0;
    if (!ok) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = 0; i < n; ++i) {
      if (!ok) continue;
      int32_t v = order[i];
      int64_t bf = -1;  /* no cut until k searches have completed */
      int32_t bi = -1;
#pragma omp critical(gpp_topk)
      {
        if (have == k) { bf = top_f[k - 1]; bi = top_id[k - 1]; }
      }
      int64_t f = bfscut(n, row_ptr, col_idx, v, bf, bi, &w);
      if (f == -2) {
#pragma omp atomic write
        err = 2;
      }
      if (f >= 0) {
#pragma omp atomic
        full++;
#pragma omp critical(gpp_topk)
        {
          /* insert (f, v) if the list is short or it beats the k-th entry */
          if (have < k || f < top_f[k - 1] || (f == top_f[k - 1] && v < top_id[k - 1])) {
            int32_t j = have < k ? have++ : k - 1;
            while (j > 0 && (top_f[j - 1] > f || (top_f[j - 1] == f && top_id[j - 1] > v))) {
              top_f[j] = top_f[j - 1];
              top_id[j] = top_id[j - 1];
              --j;
            }
            top_f[j] = f;
            top_id[j] = v;
          }
        }
      }
    }
    if (ok) ws_free(&w);
  }
  free(order);
  if (!err) {
    for (int32_t j = 0; j < k; ++j) { ids_out[j] = top_id[j]; f_out[j] = top_f[j]; }
    if (n_full) *n_full = full;
  }
  free(top_f);
  free(top_id);
  if (err) return err == 1 ? -2 : -1;
  return 0;
}

/* Greedy++ (pruned SSSPs + supermodular lazy bounds), farness form.
 * Outputs as or_greedy_plain; stats may be NULL.  Returns 0 / -1 / -2. */
int or_greedypp(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t k,
                int32_t *group, int64_t *farness_trace, int64_t *gain_trace, int32_t nthreads,
                or_gpp_stats *stats) {
  if (k < 1 || k > n) return -1;
  int nt = nthreads > 0 ? nthreads : 1;
  or_gpp_stats st = {0, 0, 0};
  int32_t s0;
  int64_t f0;
  int rc = or_top1_closeness(n, row_ptr, col_idx, nt, &s0, &f0, &st.round0_full);
  if (rc) return rc;
  int32_t *dS = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int64_t *ub = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int32_t *stamp = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  /* max-heap of (ub desc, id asc) */
  int32_t *heap = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!dS || !queue || !ub || !stamp || !heap) {
    free(dS); free(queue); free(ub); free(stamp); free(heap); return -2;
  }
  for (int32_t u = 0; u < n; ++u) dS[u] = -1;
  {
    /* d_S = BFS(s0) */
    int64_t head = 0, tail = 0;
    dS[s0] = 0; queue[tail++] = s0;
    while (head < tail) {
      int32_t u = queue[head++];
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
        if (dS[col_idx[e]] < 0) { dS[col_idx[e]] = dS[u] + 1; queue[tail++] = col_idx[e]; }
    }
  }
  group[0] = s0; farness_trace[0] = f0; gain_trace[0] = f0;
  int64_t f = f0;
  if (k > 1) {
    /* round 1: exact pruned gains of every vertex (no bounds yet) */
    int64_t ev = 0, ed = 0;
    int err = 0;
#pragma omp parallel num_threads(nt) reduction(+ : ev, ed)
    {
      bfs_ws w;
      int ok = ws_init(&w, n) == 0;
      if (!ok) {
#pragma omp atomic write
        err = 1;
      }
#pragma omp for schedule(dynamic, 64)
      for (int32_t v = 0; v < n; ++v) {
        if (!ok) continue;
        ub[v] = pruned_gain(row_ptr, col_idx, dS, v, &w, &ed);
        stamp[v] = 1;
        ++ev;
      }
      if (ok) ws_free(&w);
    }
    if (err) { free(dS); free(queue); free(ub); free(stamp); free(heap); return -2; }
    st.evals += ev; st.edges += ed;
  }
  /* heap over vertices not in S */
  int32_t hn = 0;
#define HBETTER(a, b) (ub[a] > ub[b] || (ub[a] == ub[b] && (a) < (b)))
  for (int32_t v = 0; v < n; ++v)
    if (v != s0) {
      int32_t i = hn++;
      heap[i] = v;
      while (i > 0) {
        int32_t p = (i - 1) / 2;
        if (!HBETTER(heap[i], heap[p])) break;
        int32_t t = heap[i]; heap[i] = heap[p]; heap[p] = t; i = p;
      }
    }
  bfs_ws w;
  if (ws_init(&w, n)) { free(dS); free(queue); free(ub); free(stamp); free(heap); return -2; }
  for (int32_t r = 1; r < k; ++r) {
    for (;;) {
      int32_t top = heap[0];
      if (stamp[top] == r) break; /* exact for this round and >= every other bound */
      ub[top] = pruned_gain(row_ptr, col_idx, dS, top, &w, &st.edges);
      stamp[top] = r;
      st.evals++;
      /* sift down (the key can only decrease) */
      int32_t i = 0;
      for (;;) {
        int32_t l = 2 * i + 1, rr = l + 1, m = i;
        if (l < hn && HBETTER(heap[l], heap[m])) m = l;
        if (rr < hn && HBETTER(heap[rr], heap[m])) m = rr;
        if (m == i) break;
        int32_t t = heap[i]; heap[i] = heap[m]; heap[m] = t; i = m;
      }
    }
    int32_t pick = heap[0];
    /* pop */
    heap[0] = heap[--hn];
    {
      int32_t i = 0;
      for (;;) {
        int32_t l = 2 * i + 1, rr = l + 1, m = i;
        if (l < hn && HBETTER(heap[l], heap[m])) m = l;
        if (rr < hn && HBETTER(heap[rr], heap[m])) m = rr;
        if (m == i) break;
        int32_t t = heap[i]; heap[i] = heap[m]; heap[m] = t; i = m;
      }
    }
    int64_t g = pruned_update(row_ptr, col_idx, dS, pick, queue);
    f -= g;
    group[r] = pick; gain_trace[r] = g; farness_trace[r] = f;
  }
#undef HBETTER
  ws_free(&w);
  free(dS); free(queue); free(ub); free(stamp); free(heap);
  if (stats) *stats = st;
  return 0;
}

/* Cost sample (used only to time the oracle on a bounded part of a workload
 * whose answer is known, for the benchmark's CPU baseline): for each vertex in
 * cand[0..m), the two steps of this file that dominate Greedy++ on large
 * graphs -- the round-0 BFScut of Sec. 3.1 / Algorithm 3 against the fixed
 * threshold (f_best, id_best), and the round-1 pruned SSSP of Sec. 4.1 against
 * S = {s0} -- run exactly as or_greedypp runs them, in parallel over the
 * candidates.  out[0] and out[1] receive the wall seconds of the two parts;
 * out[2] the adjacency entries the pruned SSSPs scanned.  Returns 0, or -2 on
 * allocation failure. */
int or_greedypp_cost_sample(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t s0,
                            int64_t f_best, int32_t id_best, const int32_t *cand, int32_t m, int32_t nthreads,
                            double *out) {
  int nt = nthreads > 0 ? nthreads : 1;
  int32_t *dS = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *queue = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!dS || !queue) { free(dS); free(queue); return -2; }
  for (int32_t u = 0; u < n; ++u) dS[u] = -1;
  {
    int64_t head = 0, tail = 0;
    dS[s0] = 0; queue[tail++] = s0;
    while (head < tail) {
      int32_t u = queue[head++];
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
        if (dS[col_idx[e]] < 0) { dS[col_idx[e]] = dS[u] + 1; queue[tail++] = col_idx[e]; }
    }
  }
  int err = 0;
  int64_t scanned = 0;
  double t0 = omp_get_wtime();
#pragma omp parallel num_threads(nt)
  {
    bfs_ws w;
    int ok = ws_init(&w, n) == 0;
    if (!ok) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = 0; i < m; ++i)
      if (ok) (void)bfscut(n, row_ptr, col_idx, cand[i], f_best, id_best, &w);
    if (ok) ws_free(&w);
  }
  double t1 = omp_get_wtime();
#pragma omp parallel num_threads(nt) reduction(+ : scanned)
  {
    bfs_ws w;
    int ok = ws_init(&w, n) == 0;
    if (!ok) {
#pragma omp atomic write
      err = 1;
    }
#pragma omp for schedule(dynamic, 64)
    for (int32_t i = 0; i < m; ++i)
      if (ok) (void)pruned_gain(row_ptr, col_idx, dS, cand[i], &w, &scanned);
    if (ok) ws_free(&w);
  }
  double t2 = omp_get_wtime();
  free(dS); free(queue);
  if (err) return -2;
  out[0] = t1 - t0;
  out[1] = t2 - t1;
  out[2] = (double)scanned;
  return 0;
}
