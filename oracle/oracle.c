/*
 * CPU oracle for group-closeness maximization (Bergamini, Gonser, Meyerhenke,
 * "Scaling up Group Closeness Maximization", arXiv:1710.01144).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing on the product path may call this file;
 * it is linked by the tests, by the package entry's smoke check and by the
 * benchmark's CPU-baseline leg.  It shares no code with the CUDA library.
 *
 * Part 1 (this file) is the plain, slow, obviously correct reference "O1":
 * every quantity is computed from its definition with full breadth-first
 * searches -- no pruning, no laziness, no bounds.
 *
 *   distance d(u,v)        : Sec. 2, unweighted graph => SSSP is a BFS
 *   d(u,S) = min_s d(u,s)  : Sec. 2
 *   farness f(S)           : Sec. 2 / Sec. 3.2 (farness view of Greedy); read as
 *                            the integer sum_{u in V} d(u,S) with the 1/n and
 *                            |S|-normalisations dropped (they do not move any
 *                            argmin/argmax); members contribute d = 0.
 *   gain Delta(v|S)        : f(S) - f(S u {v}) = sum_u max(0, d(u,S) - d(v,u)),
 *                            the positive decrease of farness (Sec. 4.2 uses the
 *                            negated difference; the sign is a reading).
 *   plain greedy           : Algorithm 2 in the farness form: s0 = argmin_v f({v})
 *                            (the node of maximum closeness, Sec. 3.1 / Alg. 3 with
 *                            k=1), then k-1 rounds that score every v not in S by a
 *                            full SSSP and add the best; d_S updated by a full SSSP
 *                            from the pick.  Ties go to the smallest vertex id.
 *   brute-force optimum    : min f(S) over all C(n,k) subsets (stands in for the
 *                            ILP of Sec. 5, Eq. 2, on graphs of <= ~24 vertices).
 *   bit-parallel gain      : Theorem 1 (Sec. 4.3): sum_i |b^i_v AND NOT b^i_S| with
 *                            b^i_u = b^{i-1}_u OR (OR_{w in N(u)} b^{i-1}_w), an
 *                            independent second formula for Delta(v|S).
 *
 * Graphs are int32 CSR (row_ptr[n+1], col_idx[nnz]), undirected (each edge
 * stored in both rows).  Unreachable distance is -1.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- BFS ---- */

/* Multi-source BFS: dist[u] = min_{s in src} d(s,u), -1 where unreachable.
 * Returns the number of reached vertices, or -1 on a bad source id. */
int64_t or_bfs_multi(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                     const int32_t *src, int32_t n_src, int32_t *dist) {
  int32_t *queue = (int32_t *)malloc((size_t)(n > 0 ? n : 1) * sizeof(int32_t));
  if (!queue) return -2;
  for (int32_t u = 0; u < n; ++u) dist[u] = -1;
  int64_t head = 0, tail = 0;
  for (int32_t i = 0; i < n_src; ++i) {
    int32_t s = src[i];
    if (s < 0 || s >= n) { free(queue); return -1; }
    if (dist[s] != 0) { dist[s] = 0; queue[tail++] = s; }
  }
  while (head < tail) {
    int32_t u = queue[head++];
    for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
      int32_t w = col_idx[e];
      if (dist[w] < 0) { dist[w] = dist[u] + 1; queue[tail++] = w; }
    }
  }
  free(queue);
  return tail;
}

int64_t or_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t src, int32_t *dist) {
  return or_bfs_multi(n, row_ptr, col_idx, &src, 1, dist);
}

/* f(S) = sum_u d(u,S); -1 if some vertex is unreachable from S or S is bad. */
int64_t or_farness(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                   const int32_t *S, int32_t s_len) {
  if (s_len <= 0) return -1;
  int32_t *d = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!d) return -2;
  int64_t reached = or_bfs_multi(n, row_ptr, col_idx, S, s_len, d);
  int64_t f = 0;
  if (reached != n) f = -1;
  else for (int32_t u = 0; u < n; ++u) f += d[u];
  free(d);
  return f;
}

/* Delta(v|S) from a FULL BFS out of v, given dS[u] = d(u,S).
 * dist is caller scratch of n int32. */
static int64_t gain_full_bfs(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                             const int32_t *dS, int32_t v, int32_t *dist) {
  or_bfs(n, row_ptr, col_idx, v, dist);
  int64_t g = 0;
  for (int32_t u = 0; u < n; ++u)
    if (dist[u] >= 0 && dS[u] > dist[u]) g += (int64_t)(dS[u] - dist[u]);
  return g;
}

/* gains[i] = Delta(cand[i] | S) for each candidate (0 for members of S).
 * Returns 0, or -1 on bad input. */
int or_gains(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *S,
             int32_t s_len, const int32_t *cand, int32_t n_cand, int64_t *gains, int32_t nthreads) {
  if (s_len <= 0) return -1;
  int32_t *dS = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!dS) return -2;
  if (or_bfs_multi(n, row_ptr, col_idx, S, s_len, dS) < 0) { free(dS); return -1; }
  for (int32_t i = 0; i < n_cand; ++i)
    if (cand[i] < 0 || cand[i] >= n) { free(dS); return -1; }
  int bad = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
  {
    int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    if (!dist) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = 0; i < n_cand; ++i)
      if (dist) gains[i] = gain_full_bfs(n, row_ptr, col_idx, dS, cand[i], dist);
    free(dist);
  }
  free(dS);
  return bad ? -2 : 0;
}

/* Plain greedy (Algorithm 2, farness form, full SSSPs, no pruning/laziness).
 * group[0..k-1] in pick order; farness_trace[i] = f({group[0..i]});
 * gain_trace[i] = Delta(group[i] | group[0..i-1]) for i >= 1, and
 * gain_trace[0] = f({s0}).  Returns 0, or -1 on bad input / disconnected. */
int or_greedy_plain(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t k,
                    int32_t *group, int64_t *farness_trace, int64_t *gain_trace, int32_t nthreads) {
  if (k < 1 || k > n) return -1;
  int nt = nthreads > 0 ? nthreads : 1;
  int64_t *score = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int32_t *dS = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  int32_t *dnew = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  char *in_S = (char *)calloc((size_t)n, 1);
  if (!score || !dS || !dnew || !in_S) { free(score); free(dS); free(dnew); free(in_S); return -2; }
  int rc = 0;

  /* round 0: s0 = argmin_v f({v}) by n full BFSs, ties -> smallest id */
#pragma omp parallel num_threads(nt)
  {
    int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
#pragma omp for schedule(dynamic, 4)
    for (int32_t v = 0; v < n; ++v) {
      if (!dist) { score[v] = -2; continue; }
      int64_t reached = or_bfs(n, row_ptr, col_idx, v, dist);
      int64_t f = 0;
      for (int32_t u = 0; u < n; ++u) f += dist[u];
      score[v] = (reached == n) ? f : -1;
    }
    free(dist);
  }
  int32_t s0 = -1;
  for (int32_t v = 0; v < n; ++v) {
    if (score[v] < 0) { rc = -1; break; }
    if (s0 < 0 || score[v] < score[s0]) s0 = v;
  }
  if (s0 < 0) rc = -1;
  if (rc == 0) {
    group[0] = s0; in_S[s0] = 1;
    or_bfs(n, row_ptr, col_idx, s0, dS);
    int64_t f = 0;
    for (int32_t u = 0; u < n; ++u) f += dS[u];
    farness_trace[0] = f;
    gain_trace[0] = f;
    for (int32_t r = 1; r < k; ++r) {
      /* score every v not in S by a full SSSP */
#pragma omp parallel num_threads(nt)
      {
        int32_t *dist = (int32_t *)malloc((size_t)n * sizeof(int32_t));
#pragma omp for schedule(dynamic, 4)
        for (int32_t v = 0; v < n; ++v)
          score[v] = (in_S[v] || !dist) ? -1 : gain_full_bfs(n, row_ptr, col_idx, dS, v, dist);
        free(dist);
      }
      int32_t best = -1;
      for (int32_t v = 0; v < n; ++v)
        if (!in_S[v] && (best < 0 || score[v] > score[best])) best = v;
      if (best < 0 || score[best] < 0) { rc = -2; break; }
      group[r] = best; in_S[best] = 1;
      /* d_S <- min(d_S, d(best, .)) by a full SSSP */
      or_bfs(n, row_ptr, col_idx, best, dnew);
      for (int32_t u = 0; u < n; ++u)
        if (dnew[u] < dS[u]) dS[u] = dnew[u];
      f = 0;
      for (int32_t u = 0; u < n; ++u) f += dS[u];
      gain_trace[r] = farness_trace[r - 1] - f;
      farness_trace[r] = f;
    }
  }
  free(score); free(dS); free(dnew); free(in_S);
  return rc;
}

/* Brute-force optimum: min over all k-subsets of f(S), from an all-pairs
 * distance table.  best_group gets the lexicographically first optimal set.
 * Returns the optimal farness, or -1 on bad input (n > 24 refused). */
int64_t or_opt_bruteforce(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, int32_t k,
                          int32_t *best_group) {
  if (k < 1 || k > n || n > 24) return -1;
  int32_t *D = (int32_t *)malloc((size_t)n * n * sizeof(int32_t));
  if (!D) return -2;
  for (int32_t s = 0; s < n; ++s)
    if (or_bfs(n, row_ptr, col_idx, s, D + (size_t)s * n) != n) { free(D); return -1; }
  int32_t idx[24];
  for (int32_t i = 0; i < k; ++i) idx[i] = i;
  int64_t best = -1;
  for (;;) {
    int64_t f = 0;
    for (int32_t u = 0; u < n; ++u) {
      int32_t m = D[(size_t)idx[0] * n + u];
      for (int32_t i = 1; i < k; ++i) {
        int32_t d = D[(size_t)idx[i] * n + u];
        if (d < m) m = d;
      }
      f += m;
    }
    if (best < 0 || f < best) {
      best = f;
      for (int32_t i = 0; i < k; ++i) best_group[i] = idx[i];
    }
    /* next combination in lexicographic order */
    int32_t i = k - 1;
    while (i >= 0 && idx[i] == n - k + i) --i;
    if (i < 0) break;
    idx[i]++;
    for (int32_t j = i + 1; j < k; ++j) idx[j] = idx[j - 1] + 1;
  }
  free(D);
  return best;
}

/* Theorem 1 (Sec. 4.3): for every vertex v,
 *   gains[v] = sum_{i>=0} |b^i_v AND NOT b^i_S|
 * where b^i_u is the bit vector of vertices within distance i of u, built by
 * the recurrence b^i_u = b^{i-1}_u OR (OR over neighbours w of b^{i-1}_w)
 * (the neighbourhood read as closed, so that b^i_u keeps u), and b^i_S is the
 * OR of b^i_s over s in S.  Members of S get 0 (the theorem ranges over
 * V \ S).  Iterates until no vector changes.  Memory Theta(n^2) bits, as in
 * the paper; refuses n > 16384.  Returns 0 or -1. */
int or_gains_bitparallel(int32_t n, const int32_t *row_ptr, const int32_t *col_idx,
                         const int32_t *S, int32_t s_len, int64_t *gains) {
  if (n > 16384 || s_len <= 0) return -1;
  const int32_t W = (n + 63) / 64;
  uint64_t *prev = (uint64_t *)calloc((size_t)n * W, sizeof(uint64_t));
  uint64_t *cur = (uint64_t *)calloc((size_t)n * W, sizeof(uint64_t));
  uint64_t *bS = (uint64_t *)calloc((size_t)W, sizeof(uint64_t));
  char *in_S = (char *)calloc((size_t)n, 1);
  if (!prev || !cur || !bS || !in_S) { free(prev); free(cur); free(bS); free(in_S); return -2; }
  for (int32_t i = 0; i < s_len; ++i) {
    if (S[i] < 0 || S[i] >= n) { free(prev); free(cur); free(bS); free(in_S); return -1; }
    in_S[S[i]] = 1;
  }
  for (int32_t u = 0; u < n; ++u) { prev[(size_t)u * W + u / 64] = 1ULL << (u % 64); gains[u] = 0; }
  for (int iter = 0;; ++iter) {
    /* b^i_S and the level-i terms, i = iter, from prev (= b^i) */
    memset(bS, 0, (size_t)W * sizeof(uint64_t));
    for (int32_t u = 0; u < n; ++u)
      if (in_S[u])
        for (int32_t w = 0; w < W; ++w) bS[w] |= prev[(size_t)u * W + w];
    for (int32_t u = 0; u < n; ++u) {
      if (in_S[u]) continue;
      int64_t c = 0;
      for (int32_t w = 0; w < W; ++w) c += __builtin_popcountll(prev[(size_t)u * W + w] & ~bS[w]);
      gains[u] += c;
    }
    /* b^{i+1} */
    int changed = 0;
    for (int32_t u = 0; u < n; ++u) {
      uint64_t *dst = cur + (size_t)u * W;
      memcpy(dst, prev + (size_t)u * W, (size_t)W * sizeof(uint64_t));
      for (int32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
        const uint64_t *src = prev + (size_t)col_idx[e] * W;
        for (int32_t w = 0; w < W; ++w) dst[w] |= src[w];
      }
      for (int32_t w = 0; w < W && !changed; ++w) changed |= dst[w] != prev[(size_t)u * W + w];
    }
    uint64_t *t = prev; prev = cur; cur = t;
    if (!changed) break;
  }
  free(prev); free(cur); free(bS); free(in_S);
  return 0;
}

/* ------------------------------------------------------ weighted graphs ---- */
/* The paper's weighted case (Sec. 3.2: every SSSP becomes a Dijkstra search,
 * O(kn(m + n log n)) for the greedy): positive integer edge weights w[e] >= 1
 * aligned with col_idx (the same weight in both rows of an edge), distances in
 * int64, unreachable -1.  Farness, gain and plain greedy are the definitions
 * above with d the weighted distance. */

typedef struct { int64_t d; int32_t v; } wh_item;

/* binary min-heap on (d, v) */
static void wh_push(wh_item *h, int64_t *size, int64_t d, int32_t v) {
  int64_t i = (*size)++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (h[p].d < d || (h[p].d == d && h[p].v <= v)) break;
    h[i] = h[p];
    i = p;
  }
  h[i].d = d; h[i].v = v;
}

static wh_item wh_pop(wh_item *h, int64_t *size) {
  wh_item top = h[0], last = h[--(*size)];
  int64_t i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= *size) break;
    if (c + 1 < *size && (h[c + 1].d < h[c].d || (h[c + 1].d == h[c].d && h[c + 1].v < h[c].v))) ++c;
    if (last.d < h[c].d || (last.d == h[c].d && last.v <= h[c].v)) break;
    h[i] = h[c];
    i = c;
  }
  h[i] = last;
  return top;
}

/* Multi-source Dijkstra: dist[u] = min_{s in src} d(s,u), -1 where
 * unreachable.  Returns the number of reached vertices, -1 on a bad source
 * id, -3 on a weight below 1, -2 on allocation failure. */
int64_t or_dijkstra_multi(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w,
                          const int32_t *src, int32_t n_src, int64_t *dist) {
  int64_t nnz = row_ptr[n];
  wh_item *heap = (wh_item *)malloc((size_t)(nnz + n_src + 1) * sizeof(wh_item));
  char *done = (char *)calloc((size_t)(n > 0 ? n : 1), 1);
  if (!heap || !done) { free(heap); free(done); return -2; }
  for (int32_t u = 0; u < n; ++u) dist[u] = -1;
  int64_t size = 0, reached = 0;
  for (int32_t i = 0; i < n_src; ++i) {
    int32_t s = src[i];
    if (s < 0 || s >= n) { free(heap); free(done); return -1; }
    if (dist[s] != 0) { dist[s] = 0; wh_push(heap, &size, 0, s); }
  }
  while (size > 0) {
    wh_item it = wh_pop(heap, &size);
    if (done[it.v]) continue;  /* a stale entry */
    done[it.v] = 1;
    ++reached;
    for (int32_t e = row_ptr[it.v]; e < row_ptr[it.v + 1]; ++e) {
      if (w[e] < 1) { free(heap); free(done); return -3; }
      int32_t x = col_idx[e];
      int64_t nd = it.d + w[e];
      if (!done[x] && (dist[x] < 0 || nd < dist[x])) { dist[x] = nd; wh_push(heap, &size, nd, x); }
    }
  }
  free(heap); free(done);
  return reached;
}

/* f(S) = sum_u d(u,S) with weighted distances; -1 if unreachable / bad S. */
int64_t or_wfarness(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w,
                    const int32_t *S, int32_t s_len) {
  if (s_len <= 0) return -1;
  int64_t *d = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!d) return -2;
  int64_t reached = or_dijkstra_multi(n, row_ptr, col_idx, w, S, s_len, d);
  int64_t f = 0;
  if (reached != n) f = -1;
  else for (int32_t u = 0; u < n; ++u) f += d[u];
  free(d);
  return f;
}

/* Delta(v|S) = sum_u max(0, dS[u] - d(v,u)) from a FULL Dijkstra out of v. */
static int64_t wgain_full(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w,
                          const int64_t *dS, int32_t v, int64_t *dist) {
  or_dijkstra_multi(n, row_ptr, col_idx, w, &v, 1, dist);
  int64_t g = 0;
  for (int32_t u = 0; u < n; ++u)
    if (dist[u] >= 0 && dS[u] > dist[u]) g += dS[u] - dist[u];
  return g;
}

/* gains[i] = Delta(cand[i] | S), weighted.  Returns 0, -1 on bad input. */
int or_wgains(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w, const int32_t *S,
              int32_t s_len, const int32_t *cand, int32_t n_cand, int64_t *gains, int32_t nthreads) {
  if (s_len <= 0) return -1;
  int64_t *dS = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  if (!dS) return -2;
  if (or_dijkstra_multi(n, row_ptr, col_idx, w, S, s_len, dS) < 0) { free(dS); return -1; }
  for (int32_t i = 0; i < n_cand; ++i)
    if (cand[i] < 0 || cand[i] >= n) { free(dS); return -1; }
  int bad = 0;
#pragma omp parallel num_threads(nthreads > 0 ? nthreads : 1)
  {
    int64_t *dist = (int64_t *)malloc((size_t)n * sizeof(int64_t));
    if (!dist) {
#pragma omp atomic write
      bad = 1;
    }
#pragma omp for schedule(dynamic, 1)
    for (int32_t i = 0; i < n_cand; ++i)
      if (dist) gains[i] = wgain_full(n, row_ptr, col_idx, w, dS, cand[i], dist);
    free(dist);
  }
  free(dS);
  return bad ? -2 : 0;
}

/* Plain weighted greedy: or_greedy_plain with Dijkstra for every SSSP.
 * Outputs as or_greedy_plain.  Returns 0, -1 (bad input / disconnected). */
int or_wgreedy_plain(int32_t n, const int32_t *row_ptr, const int32_t *col_idx, const int32_t *w, int32_t k,
                     int32_t *group, int64_t *farness_trace, int64_t *gain_trace, int32_t nthreads) {
  if (k < 1 || k > n) return -1;
  int nt = nthreads > 0 ? nthreads : 1;
  int64_t *score = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *dS = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  int64_t *dnew = (int64_t *)malloc((size_t)n * sizeof(int64_t));
  char *in_S = (char *)calloc((size_t)n, 1);
  if (!score || !dS || !dnew || !in_S) { free(score); free(dS); free(dnew); free(in_S); return -2; }
  int rc = 0;
  /* round 0: s0 = argmin_v f({v}) by n full Dijkstra searches, ties -> smallest id */
#pragma omp parallel num_threads(nt)
  {
    int64_t *dist = (int64_t *)malloc((size_t)n * sizeof(int64_t));
#pragma omp for schedule(dynamic, 4)
    for (int32_t v = 0; v < n; ++v) {
      if (!dist) { score[v] = -2; continue; }
      int64_t reached = or_dijkstra_multi(n, row_ptr, col_idx, w, &v, 1, dist);
      int64_t f = 0;
      for (int32_t u = 0; u < n; ++u) f += dist[u];
      score[v] = (reached == n) ? f : -1;
    }
    free(dist);
  }
  int32_t s0 = -1;
  for (int32_t v = 0; v < n; ++v) {
    if (score[v] < 0) { rc = -1; break; }
    if (s0 < 0 || score[v] < score[s0]) s0 = v;
  }
  if (s0 < 0) rc = -1;
  if (rc == 0) {
    group[0] = s0; in_S[s0] = 1;
    or_dijkstra_multi(n, row_ptr, col_idx, w, &s0, 1, dS);
    int64_t f = 0;
    for (int32_t u = 0; u < n; ++u) f += dS[u];
    farness_trace[0] = f;
    gain_trace[0] = f;
    for (int32_t r = 1; r < k; ++r) {
#pragma omp parallel num_threads(nt)
      {
        int64_t *dist = (int64_t *)malloc((size_t)n * sizeof(int64_t));
#pragma omp for schedule(dynamic, 4)
        for (int32_t v = 0; v < n; ++v)
          score[v] = (in_S[v] || !dist) ? -1 : wgain_full(n, row_ptr, col_idx, w, dS, v, dist);
        free(dist);
      }
      int32_t best = -1;
      for (int32_t v = 0; v < n; ++v)
        if (!in_S[v] && (best < 0 || score[v] > score[best])) best = v;
      if (best < 0 || score[best] < 0) { rc = -2; break; }
      group[r] = best; in_S[best] = 1;
      or_dijkstra_multi(n, row_ptr, col_idx, w, &best, 1, dnew);
      for (int32_t u = 0; u < n; ++u)
        if (dnew[u] < dS[u]) dS[u] = dnew[u];
      f = 0;
      for (int32_t u = 0; u < n; ++u) f += dS[u];
      gain_trace[r] = farness_trace[r - 1] - f;
      farness_trace[r] = f;
    }
  }
  free(score); free(dS); free(dnew); free(in_S);
  return rc;
}
