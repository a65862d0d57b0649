/*
 * Seeded synthetic graph generators: Barabasi-Albert, R-MAT, damaged grid
 * with diagonal shortcuts, and a mixed batch.  Output is a simple undirected
 * graph (no self-loops, no duplicate edges) restricted to its largest
 * connected component, as an int32 CSR with sorted neighbour lists.
 *
 * This module only shapes inputs.  It holds none of the group-closeness
 * arithmetic (no distances, farness or gains); both the CPU oracle's tests and
 * the GPU path take their graphs from here.  The paper evaluates on real
 * social/road networks (Sec. 6); these generators stand in for them.
 *
 * Randomness: splitmix64 seeds xoshiro256** (Vigna's published definitions),
 * one stream per fixed-size chunk of samples, so that the result does not
 * depend on the number of OpenMP threads.  Floating point is used only for
 * comparisons of exactly representable uniforms against the R-MAT quadrant
 * probabilities, so x86-64 and aarch64 give identical graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ rng -- */
static uint64_t sm64_next(uint64_t *x) {
  uint64_t z = (*x += 0x9E3779B97F4A7C15ULL);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}
typedef struct { uint64_t s[4]; } xo_t;
static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }
static void xo_seed(xo_t *r, uint64_t seed, uint64_t stream) {
  uint64_t x = seed ^ (stream * 0xD1B54A32D192ED03ULL);
  for (int i = 0; i < 4; ++i) r->s[i] = sm64_next(&x);
}
static inline uint64_t xo_next(xo_t *r) {
  uint64_t *s = r->s;
  const uint64_t out = rotl64(s[1] * 5, 7) * 9;
  const uint64_t t = s[1] << 17;
  s[2] ^= s[0]; s[3] ^= s[1]; s[1] ^= s[2]; s[0] ^= s[3];
  s[2] ^= t; s[3] = rotl64(s[3], 45);
  return out;
}
/* uniform integer in [0, bound) by the multiply-high method */
static inline uint64_t xo_below(xo_t *r, uint64_t bound) {
  return (uint64_t)(((unsigned __int128)xo_next(r) * bound) >> 64);
}
/* uniform double in [0,1) with 53 random bits (exact) */
static inline double xo_unit(xo_t *r) { return (double)(xo_next(r) >> 11) * (1.0 / 9007199254740992.0); }

/* ------------------------------------------------------------- edge list -- */
typedef struct { int32_t *u, *v; int64_t len, cap; } elist;
static int el_push(elist *e, int32_t a, int32_t b) {
  if (e->len == e->cap) {
    int64_t nc = e->cap ? e->cap * 2 : 1024;
    int32_t *nu = (int32_t *)realloc(e->u, nc * sizeof(int32_t));
    if (!nu) return -1;
    e->u = nu;
    int32_t *nv = (int32_t *)realloc(e->v, nc * sizeof(int32_t));
    if (!nv) return -1;
    e->v = nv;
    e->cap = nc;
  }
  e->u[e->len] = a; e->v[e->len] = b; e->len++;
  return 0;
}
static void el_free(elist *e) { free(e->u); free(e->v); memset(e, 0, sizeof(*e)); }

/* ---------------------------------------------------------------- output -- */
typedef struct gg_graph {
  int32_t n;
  int64_t nnz;
  int32_t *row_ptr; /* n+1 */
  int32_t *col_idx; /* nnz */
  int32_t n_raw;    /* vertex count before the LCC restriction */
} gg_graph;

void gg_free(gg_graph *g) {
  if (!g) return;
  free(g->row_ptr); free(g->col_idx); free(g);
}
int32_t gg_n(const gg_graph *g) { return g->n; }
int64_t gg_nnz(const gg_graph *g) { return g->nnz; }
int32_t gg_n_raw(const gg_graph *g) { return g->n_raw; }
void gg_copy(const gg_graph *g, int32_t *row_ptr, int32_t *col_idx) {
  memcpy(row_ptr, g->row_ptr, (size_t)(g->n + 1) * sizeof(int32_t));
  memcpy(col_idx, g->col_idx, (size_t)g->nnz * sizeof(int32_t));
}

static int cmp_i32(const void *a, const void *b) {
  int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
  return (x > y) - (x < y);
}
static void sort_i32(int32_t *a, int64_t len) {
  if (len < 32) {
    for (int64_t i = 1; i < len; ++i) {
      int32_t x = a[i]; int64_t j = i - 1;
      while (j >= 0 && a[j] > x) { a[j + 1] = a[j]; --j; }
      a[j + 1] = x;
    }
  } else {
    qsort(a, (size_t)len, sizeof(int32_t), cmp_i32);
  }
}

static int32_t uf_find(int32_t *p, int32_t x) {
  while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
  return x;
}

/* Symmetrise, drop self-loops and duplicates, keep the largest connected
 * component (ties: the component holding the smallest vertex id), relabel its
 * vertices in increasing original order.  Returns NULL on allocation failure
 * or if the result would not fit int32 CSR. */
static gg_graph *build_csr(int32_t n, const elist *e, int keep_lcc) {
  int64_t *deg = (int64_t *)calloc((size_t)n + 1, sizeof(int64_t));
  if (!deg) return NULL;
  for (int64_t i = 0; i < e->len; ++i) {
    if (e->u[i] == e->v[i]) continue;
    deg[e->u[i]]++; deg[e->v[i]]++;
  }
  int64_t *off = (int64_t *)malloc(((size_t)n + 1) * sizeof(int64_t));
  if (!off) { free(deg); return NULL; }
  off[0] = 0;
  for (int32_t i = 0; i < n; ++i) off[i + 1] = off[i] + deg[i];
  int64_t tot = off[n];
  int32_t *col = (int32_t *)malloc((size_t)(tot ? tot : 1) * sizeof(int32_t));
  if (!col) { free(deg); free(off); return NULL; }
  memset(deg, 0, ((size_t)n + 1) * sizeof(int64_t));
  for (int64_t i = 0; i < e->len; ++i) {
    int32_t a = e->u[i], b = e->v[i];
    if (a == b) continue;
    col[off[a] + deg[a]++] = b;
    col[off[b] + deg[b]++] = a;
  }
  /* sort + dedup each row; new degree into deg[] */
#pragma omp parallel for schedule(dynamic, 1024)
  for (int32_t i = 0; i < n; ++i) {
    int32_t *r = col + off[i];
    int64_t len = off[i + 1] - off[i];
    sort_i32(r, len);
    int64_t w = 0;
    for (int64_t j = 0; j < len; ++j)
      if (w == 0 || r[w - 1] != r[j]) r[w++] = r[j];
    deg[i] = w;
  }
  /* components by union-find over the deduplicated rows */
  int32_t *keep_id = (int32_t *)malloc((size_t)n * sizeof(int32_t));
  if (!keep_id) { free(deg); free(off); free(col); return NULL; }
  int32_t n_keep = 0;
  if (keep_lcc) {
    int32_t *par = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *cnt = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!par || !cnt) { free(par); free(cnt); free(deg); free(off); free(col); free(keep_id); return NULL; }
    for (int32_t i = 0; i < n; ++i) par[i] = i;
    for (int32_t i = 0; i < n; ++i)
      for (int64_t j = 0; j < deg[i]; ++j) {
        int32_t a = uf_find(par, i), b = uf_find(par, col[off[i] + j]);
        if (a != b) { if (a < b) par[b] = a; else par[a] = b; }
      }
    int32_t best = -1, best_cnt = 0;
    for (int32_t i = 0; i < n; ++i) cnt[uf_find(par, i)]++;
    for (int32_t i = 0; i < n; ++i)
      if (cnt[i] > best_cnt) { best_cnt = cnt[i]; best = i; }
    for (int32_t i = 0; i < n; ++i) keep_id[i] = (uf_find(par, i) == best) ? n_keep++ : -1;
    free(par); free(cnt);
  } else {
    for (int32_t i = 0; i < n; ++i) keep_id[i] = n_keep++;
  }
  int64_t nnz = 0;
  for (int32_t i = 0; i < n; ++i)
    if (keep_id[i] >= 0) nnz += deg[i];
  gg_graph *g = (gg_graph *)calloc(1, sizeof(gg_graph));
  if (!g || nnz >= (int64_t)INT32_MAX) { free(g); free(deg); free(off); free(col); free(keep_id); return NULL; }
  g->n = n_keep; g->nnz = nnz; g->n_raw = n;
  g->row_ptr = (int32_t *)malloc(((size_t)n_keep + 1) * sizeof(int32_t));
  g->col_idx = (int32_t *)malloc((size_t)(nnz ? nnz : 1) * sizeof(int32_t));
  if (!g->row_ptr || !g->col_idx) { gg_free(g); free(deg); free(off); free(col); free(keep_id); return NULL; }
  int64_t w = 0;
  g->row_ptr[0] = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (keep_id[i] < 0) continue;
    for (int64_t j = 0; j < deg[i]; ++j) g->col_idx[w++] = keep_id[col[off[i] + j]];
    g->row_ptr[keep_id[i] + 1] = (int32_t)w;
  }
  free(deg); free(off); free(col); free(keep_id);
  return g;
}

/* ------------------------------------------------------- Barabasi-Albert -- */
/* Seed clique on m+1 vertices; every later vertex attaches to m distinct
 * earlier vertices drawn from the list of edge endpoints (preferential
 * attachment by the endpoint-list method). */
gg_graph *gg_barabasi_albert(int32_t n, int32_t m, uint64_t seed) {
  if (m < 1 || n < m + 1) return NULL;
  elist e = {0};
  int64_t n_end = (int64_t)m * (m + 1) + 2LL * (n - m - 1) * m;
  int32_t *ends = (int32_t *)malloc((size_t)n_end * sizeof(int32_t));
  int32_t *pick = (int32_t *)malloc((size_t)m * sizeof(int32_t));
  if (!ends || !pick) { free(ends); free(pick); return NULL; }
  int64_t ne = 0;
  for (int32_t a = 0; a <= m; ++a)
    for (int32_t b = a + 1; b <= m; ++b) {
      if (el_push(&e, a, b)) goto fail;
      ends[ne++] = a; ends[ne++] = b;
    }
  xo_t r; xo_seed(&r, seed, 0xBA);
  for (int32_t v = m + 1; v < n; ++v) {
    int32_t got = 0;
    while (got < m) {
      int32_t t = ends[xo_below(&r, (uint64_t)ne)];
      int dup = 0;
      for (int32_t q = 0; q < got; ++q) dup |= (pick[q] == t);
      if (!dup) pick[got++] = t;
    }
    for (int32_t q = 0; q < m; ++q) {
      if (el_push(&e, v, pick[q])) goto fail;
      ends[ne++] = v; ends[ne++] = pick[q];
    }
  }
  free(ends); free(pick);
  gg_graph *g = build_csr(n, &e, 1);
  el_free(&e);
  return g;
fail:
  free(ends); free(pick); el_free(&e);
  return NULL;
}

/* ----------------------------------------------------------------- R-MAT -- */
/* n_samples = edge_factor * 2^scale ordered pairs, each chosen by descending
 * the 2x2 recursive quadrant split with probabilities (a, b, c, 1-a-b-c) at
 * each of the `scale` levels.  Pairs with an endpoint >= n_keep are dropped
 * (n_keep <= 2^scale; used for the mixed batch). */
#define GG_CHUNK 65536
gg_graph *gg_rmat(int32_t scale, double edge_factor, double a, double b, double c,
                  uint64_t seed, int32_t n_keep) {
  if (scale < 1 || scale > 30) return NULL;
  int64_t nv = (int64_t)1 << scale;
  if (n_keep <= 0 || n_keep > nv) n_keep = (int32_t)nv;
  int64_t ns = (int64_t)llround(edge_factor * (double)nv);
  elist e = {0};
  e.u = (int32_t *)malloc((size_t)(ns ? ns : 1) * sizeof(int32_t));
  e.v = (int32_t *)malloc((size_t)(ns ? ns : 1) * sizeof(int32_t));
  if (!e.u || !e.v) { el_free(&e); return NULL; }
  e.cap = ns; e.len = ns;
  const double ab = a + b, abc = a + b + c;
  int64_t nchunk = (ns + GG_CHUNK - 1) / GG_CHUNK;
#pragma omp parallel for schedule(dynamic, 1)
  for (int64_t ch = 0; ch < nchunk; ++ch) {
    xo_t r; xo_seed(&r, seed, 0x52A7000000000000ULL + (uint64_t)ch);
    int64_t lo = ch * GG_CHUNK, hi = lo + GG_CHUNK < ns ? lo + GG_CHUNK : ns;
    for (int64_t i = lo; i < hi; ++i) {
      int64_t u = 0, v = 0;
      for (int32_t l = 0; l < scale; ++l) {
        double x = xo_unit(&r);
        int bu = x >= ab, bv = (x >= a && x < ab) || x >= abc;
        u = (u << 1) | bu; v = (v << 1) | bv;
      }
      e.u[i] = (int32_t)u; e.v[i] = (int32_t)v;
    }
  }
  if (n_keep < nv) { /* drop pairs outside [0, n_keep) */
    int64_t w = 0;
    for (int64_t i = 0; i < ns; ++i)
      if (e.u[i] < n_keep && e.v[i] < n_keep) { e.u[w] = e.u[i]; e.v[w] = e.v[i]; ++w; }
    e.len = w;
  }
  gg_graph *g = build_csr(n_keep, &e, 1);
  el_free(&e);
  return g;
}

/* ------------------------------------------------------------- road-like -- */
/* rows x cols 4-neighbour grid (row-major ids); each grid edge deleted
 * independently with probability p_del; then round(diag_frac * E0) diagonal
 * shortcuts (i,j)-(i+1,j+-1) drawn uniformly (duplicates merge), E0 = the
 * grid's original edge count. */
gg_graph *gg_grid_road(int32_t rows, int32_t cols, double p_del, double diag_frac, uint64_t seed) {
  if (rows < 2 || cols < 2 || (int64_t)rows * cols >= INT32_MAX) return NULL;
  int64_t e0 = (int64_t)rows * (cols - 1) + (int64_t)(rows - 1) * cols;
  elist e = {0};
  xo_t r; xo_seed(&r, seed, 0x6121D);
  for (int32_t i = 0; i < rows; ++i)
    for (int32_t j = 0; j < cols; ++j) {
      int32_t id = i * cols + j;
      if (j + 1 < cols && xo_unit(&r) >= p_del)
        if (el_push(&e, id, id + 1)) goto fail;
      if (i + 1 < rows && xo_unit(&r) >= p_del)
        if (el_push(&e, id, id + cols)) goto fail;
    }
  int64_t nd = (int64_t)llround(diag_frac * (double)e0);
  for (int64_t q = 0; q < nd;) {
    int32_t i = (int32_t)xo_below(&r, (uint64_t)(rows - 1));
    int32_t j = (int32_t)xo_below(&r, (uint64_t)cols);
    int32_t j2 = j + (xo_below(&r, 2) ? 1 : -1);
    if (j2 < 0 || j2 >= cols) continue;
    if (el_push(&e, i * cols + j, (i + 1) * cols + j2)) goto fail;
    ++q;
  }
  {
    gg_graph *g = build_csr(rows * cols, &e, 1);
    el_free(&e);
    return g;
  }
fail:
  el_free(&e);
  return NULL;
}

/* ---------------------------------------------------------- mixed batch -- */
/* Parameters of graph `index` of a mixed batch: family (0 = BA, 1 = R-MAT),
 * vertex count log-uniform in [n_lo, n_hi], average degree uniform in
 * [deg_lo, deg_hi], group size uniform integer in [k_lo, k_hi]. */
void gg_batch_params(uint64_t seed, int32_t index, int32_t n_lo, int32_t n_hi, double deg_lo,
                     double deg_hi, int32_t k_lo, int32_t k_hi, int32_t *family, int32_t *n,
                     double *avg_deg, int32_t *k, uint64_t *graph_seed) {
  xo_t r; xo_seed(&r, seed, 0xBA7C000000000000ULL + (uint64_t)index);
  *family = (int32_t)xo_below(&r, 2);
  /* log-uniform on a 4096-step geometric grid: ratio^(i/4096) is a product of
   * repeated square roots, so only correctly rounded IEEE operations are used
   * (no libm exp/log) and every platform draws the same n. */
  double q = (double)n_hi / (double)n_lo, root[12], f = 1.0;
  for (int b = 11; b >= 0; --b) { q = sqrt(q); root[b] = q; }
  uint32_t i = (uint32_t)xo_below(&r, 4097);
  if (i == 4096) f = (double)n_hi / (double)n_lo;
  else for (int b = 0; b < 12; ++b) if (i >> b & 1) f *= root[b];
  int32_t nn = (int32_t)llround((double)n_lo * f);
  if (nn < n_lo) nn = n_lo;
  if (nn > n_hi) nn = n_hi;
  *n = nn;
  *avg_deg = deg_lo + (deg_hi - deg_lo) * xo_unit(&r);
  *k = k_lo + (int32_t)xo_below(&r, (uint64_t)(k_hi - k_lo + 1));
  *graph_seed = xo_next(&r);
}
