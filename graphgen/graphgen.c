/*
 * Seeded synthetic graph generators for the MFBC workloads.
 *
 * This module only produces inputs: CSR adjacency (row pointers, column
 * indices, optional integer weights) and sampled source lists.  It holds none
 * of the betweenness-centrality arithmetic and is shared, as an input source
 * only, by the CPU oracle and the CUDA library.
 *
 * Workloads follow the paper's experimental section (Sec. 6): R-MAT graphs
 * (power-law, Chakrabarti et al.), Erdos-Renyi uniform random graphs, and
 * (for the serving pool) weighted 2D grids.  Randomness is counter based
 * (splitmix64, Steele/Lea/Flood 2014): every draw is a pure function of
 * (seed, stream, index), so outputs do not depend on the thread count or on
 * the host architecture (integer arithmetic only, except the geometric skip
 * of the G(n,p) generator, which uses log()).
 *
 * Conventions (shared by every generator):
 *  - no self-loops; duplicate arcs are merged keeping the minimum weight;
 *  - undirected graphs store both arcs with the same weight;
 *  - rows are sorted by column index;
 *  - weights are integers in [wlo, whi]; wlo == whi == 0 means unweighted
 *    (no weight array is produced).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

static inline uint64_t sm64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

/* draw number k of stream `stream` under `seed` */
static inline uint64_t draw(uint64_t seed, uint64_t stream, uint64_t k) {
  return sm64(sm64(seed ^ (stream * 0xD1B54A32D192ED03ull)) + k * 0x9E3779B97F4A7C15ull);
}

/* uniform integer in [lo, hi] from a 64-bit draw (multiply-shift) */
static inline int32_t uni_int(uint64_t r, int32_t lo, int32_t hi) {
  uint64_t range = (uint64_t)((int64_t)hi - (int64_t)lo + 1);
  return (int32_t)((int64_t)lo + (int64_t)(((r >> 32) * range) >> 32));
}

typedef struct {
  int64_t m;        /* arcs stored */
  int32_t* src;
  int32_t* dst;
  int32_t* w;       /* may be NULL */
} arcs_t;

static int cmp_pair(const void* a, const void* b) {
  const int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
  return (x > y) - (x < y);
}

/* Counting sort of the arc list by source, per-row sort by (dst, w), merge of
 * duplicates keeping the minimum weight.  Output arrays are malloc'ed. */
static int build_csr(int32_t n, arcs_t* a, int64_t** rowptr_out, int32_t** col_out,
                     int32_t** w_out, int64_t* nnz_out) {
  int64_t* cnt = (int64_t*)calloc((size_t)n + 1, sizeof(int64_t));
  if (!cnt) return -1;
  for (int64_t e = 0; e < a->m; e++) cnt[a->src[e] + 1]++;
  for (int32_t v = 0; v < n; v++) cnt[v + 1] += cnt[v];
  int64_t* key = (int64_t*)malloc(sizeof(int64_t) * (size_t)(a->m ? a->m : 1));
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!key || !pos) { free(cnt); free(key); free(pos); return -1; }
  memcpy(pos, cnt, sizeof(int64_t) * ((size_t)n + 1));
  for (int64_t e = 0; e < a->m; e++) {
    int64_t wv = a->w ? (int64_t)a->w[e] : 0;
    key[pos[a->src[e]]++] = ((int64_t)a->dst[e] << 32) | wv;
  }
  free(pos);
  /* sort each row and merge duplicates in place */
  int64_t out = 0;
  int64_t* rowptr = (int64_t*)malloc(sizeof(int64_t) * ((size_t)n + 1));
  if (!rowptr) { free(cnt); free(key); return -1; }
  rowptr[0] = 0;
  for (int32_t v = 0; v < n; v++) {
    int64_t b = cnt[v], e = cnt[v + 1];
    if (e - b > 1) qsort(key + b, (size_t)(e - b), sizeof(int64_t), cmp_pair);
    int64_t last = -1;
    for (int64_t i = b; i < e; i++) {
      int64_t d = key[i] >> 32;
      if (d == last) continue;            /* same dst: first has min weight */
      key[out++] = key[i];
      last = d;
    }
    rowptr[v + 1] = out;
  }
  free(cnt);
  int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(out ? out : 1));
  int32_t* w = a->w ? (int32_t*)malloc(sizeof(int32_t) * (size_t)(out ? out : 1)) : NULL;
  if (!col || (a->w && !w)) { free(key); free(rowptr); free(col); free(w); return -1; }
  for (int64_t i = 0; i < out; i++) {
    col[i] = (int32_t)(key[i] >> 32);
    if (w) w[i] = (int32_t)(key[i] & 0xffffffffll);
  }
  free(key);
  *rowptr_out = rowptr; *col_out = col; *w_out = w; *nnz_out = out;
  return 0;
}

/* ---------------------------------------------------------------- R-MAT -- */

typedef struct {
  int scale; uint64_t seed; int64_t e0, e1;
  uint32_t ta, tab, tabc;             /* cumulative quadrant thresholds (2^32 scale) */
  const int32_t* perm; int directed; int32_t wlo, whi;
  int32_t *src, *dst, *w; int64_t* kept; /* per-draw output slot (-1 = dropped) */
} rmat_job_t;

static void* rmat_worker(void* p) {
  rmat_job_t* j = (rmat_job_t*)p;
  for (int64_t e = j->e0; e < j->e1; e++) {
    uint32_t u = 0, v = 0;
    for (int l = 0; l < j->scale; l += 2) {
      uint64_t r = draw(j->seed, 1, (uint64_t)e * 16 + (uint64_t)(l >> 1));
      for (int h = 0; h < 2 && l + h < j->scale; h++) {
        uint32_t x = (uint32_t)(h ? (r >> 32) : r);
        uint32_t bu, bv;
        if (x < j->ta) { bu = 0; bv = 0; }
        else if (x < j->tab) { bu = 0; bv = 1; }
        else if (x < j->tabc) { bu = 1; bv = 0; }
        else { bu = 1; bv = 1; }
        u = (u << 1) | bu; v = (v << 1) | bv;
      }
    }
    int32_t pu = j->perm[u], pv = j->perm[v];
    j->src[e] = pu; j->dst[e] = pv;
    if (j->w) j->w[e] = uni_int(draw(j->seed, 2, (uint64_t)e), j->wlo, j->whi);
  }
  return NULL;
}

/* random permutation of 0..n-1 (Fisher-Yates, counter-based draws) */
static int32_t* make_perm(int32_t n, uint64_t seed) {
  int32_t* p = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  if (!p) return NULL;
  for (int32_t i = 0; i < n; i++) p[i] = i;
  for (int32_t i = n - 1; i > 0; i--) {
    uint64_t r = draw(seed, 3, (uint64_t)i);
    int32_t k = (int32_t)(((r >> 32) * (uint64_t)(i + 1)) >> 32);
    int32_t t = p[i]; p[i] = p[k]; p[k] = t;
  }
  return p;
}

int gg_rmat(int scale, int64_t nedges, double a, double b, double c, int directed,
            int32_t wlo, int32_t whi, uint64_t seed, int nthreads,
            int64_t** rowptr, int32_t** col, int32_t** w, int64_t* nnz) {
  if (scale < 1 || scale > 30 || nedges < 0) return -2;
  int32_t n = (int32_t)(1u << scale);
  int weighted = !(wlo == 0 && whi == 0);
  if (weighted && (wlo < 1 || whi < wlo)) return -2;
  int32_t* perm = make_perm(n, seed);
  int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nedges ? nedges : 1));
  int32_t* d = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nedges ? nedges : 1));
  int32_t* ww = weighted ? (int32_t*)malloc(sizeof(int32_t) * (size_t)(nedges ? nedges : 1)) : NULL;
  if (!perm || !s || !d || (weighted && !ww)) { free(perm); free(s); free(d); free(ww); return -1; }
  if (nthreads < 1) nthreads = 1;
  if (nthreads > 256) nthreads = 256;
  pthread_t th[256];
  rmat_job_t jobs[256];
  const double scl = 4294967296.0;
  for (int t = 0; t < nthreads; t++) {
    rmat_job_t* j = &jobs[t];
    j->scale = scale; j->seed = seed;
    j->e0 = nedges * t / nthreads; j->e1 = nedges * (t + 1) / nthreads;
    j->ta = (uint32_t)(a * scl); j->tab = (uint32_t)((a + b) * scl);
    j->tabc = (uint32_t)((a + b + c) * scl);
    j->perm = perm; j->directed = directed; j->wlo = wlo; j->whi = whi;
    j->src = s; j->dst = d; j->w = ww; j->kept = NULL;
    pthread_create(&th[t], NULL, rmat_worker, j);
  }
  for (int t = 0; t < nthreads; t++) pthread_join(th[t], NULL);
  free(perm);
  /* drop self-loops; undirected: store both arcs */
  int64_t m = 0;
  int64_t cap = directed ? nedges : 2 * nedges;
  arcs_t A;
  A.src = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap ? cap : 1));
  A.dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap ? cap : 1));
  A.w = weighted ? (int32_t*)malloc(sizeof(int32_t) * (size_t)(cap ? cap : 1)) : NULL;
  if (!A.src || !A.dst || (weighted && !A.w)) { free(s); free(d); free(ww); return -1; }
  for (int64_t e = 0; e < nedges; e++) {
    if (s[e] == d[e]) continue;
    A.src[m] = s[e]; A.dst[m] = d[e]; if (A.w) A.w[m] = ww[e]; m++;
    if (!directed) { A.src[m] = d[e]; A.dst[m] = s[e]; if (A.w) A.w[m] = ww[e]; m++; }
  }
  free(s); free(d); free(ww);
  A.m = m;
  int rc = build_csr(n, &A, rowptr, col, w, nnz);
  free(A.src); free(A.dst); free(A.w);
  return rc;
}

/* ------------------------------------------------------- Erdos-Renyi G(n,p) */
/* Geometric skipping over the pairs (Batagelj & Brandes, Phys. Rev. E 71, 2005):
 * the gap to the next present pair is floor(log(1-U)/log(1-p)). */
int gg_er(int32_t n, double avg_deg, int directed, int32_t wlo, int32_t whi, uint64_t seed,
          int64_t** rowptr, int32_t** col, int32_t** w, int64_t* nnz) {
  if (n < 0) return -2;
  int weighted = !(wlo == 0 && whi == 0);
  if (weighted && (wlo < 1 || whi < wlo)) return -2;
  double p = (n > 1) ? avg_deg / (double)(n - 1) : 0.0;
  if (p < 0) p = 0;
  if (p > 1) p = 1;
  int64_t cap = 1024;
  arcs_t A; A.m = 0;
  A.src = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  A.dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  A.w = weighted ? (int32_t*)malloc(sizeof(int32_t) * (size_t)cap) : NULL;
  if (!A.src || !A.dst || (weighted && !A.w)) return -1;
  uint64_t k = 0, pairs_done = 0;
  double lq = (p < 1.0) ? log(1.0 - p) : 0.0;
  /* undirected: pairs (v,u) with u < v, row-major; directed: all (v,u), u != v */
  int64_t v = directed ? 0 : 1, u = -1;
  if (p > 0.0 && n > 1) {
    for (;;) {
      uint64_t r = draw(seed, 4, k++);
      double U = (double)(r >> 11) * (1.0 / 9007199254740992.0);
      int64_t skip = (p >= 1.0) ? 0 : (int64_t)floor(log(1.0 - U) / lq);
      u += 1 + skip;
      if (directed) {
        while (v < n && u >= (int64_t)n - 1) { u -= (int64_t)n - 1; v++; }
      } else {
        while (v < n && u >= v) { u -= v; v++; }
      }
      if (v >= n) break;
      int32_t uu = (int32_t)u;
      if (directed && uu >= v) uu++;      /* skip the diagonal */
      int32_t wv = weighted ? uni_int(draw(seed, 5, pairs_done), wlo, whi) : 0;
      pairs_done++;
      int64_t need = A.m + 2;
      if (need > cap) {
        cap *= 2;
        A.src = (int32_t*)realloc(A.src, sizeof(int32_t) * (size_t)cap);
        A.dst = (int32_t*)realloc(A.dst, sizeof(int32_t) * (size_t)cap);
        if (weighted) A.w = (int32_t*)realloc(A.w, sizeof(int32_t) * (size_t)cap);
        if (!A.src || !A.dst || (weighted && !A.w)) return -1;
      }
      A.src[A.m] = (int32_t)v; A.dst[A.m] = uu; if (weighted) A.w[A.m] = wv; A.m++;
      if (!directed) { A.src[A.m] = uu; A.dst[A.m] = (int32_t)v; if (weighted) A.w[A.m] = wv; A.m++; }
    }
  }
  int rc = build_csr(n, &A, rowptr, col, w, nnz);
  free(A.src); free(A.dst); free(A.w);
  return rc;
}

/* ------------------------------------------------------ 2D 4-neighbour grid */
int gg_grid(int32_t L, int32_t wlo, int32_t whi, uint64_t seed,
            int64_t** rowptr, int32_t** col, int32_t** w, int64_t* nnz) {
  if (L < 1 || (int64_t)L * L > 0x7fffffffll) return -2;
  int weighted = !(wlo == 0 && whi == 0);
  int32_t n = L * L;
  int64_t cap = 4ll * n;
  arcs_t A; A.m = 0;
  A.src = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  A.dst = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
  A.w = weighted ? (int32_t*)malloc(sizeof(int32_t) * (size_t)cap) : NULL;
  if (!A.src || !A.dst || (weighted && !A.w)) return -1;
  for (int32_t r = 0; r < L; r++)
    for (int32_t c = 0; c < L; c++) {
      int32_t v = r * L + c;
      for (int dir = 0; dir < 2; dir++) {
        int32_t rr = r + (dir == 1), cc = c + (dir == 0);
        if (rr >= L || cc >= L) continue;
        int32_t u = rr * L + cc;
        int32_t wv = weighted ? uni_int(draw(seed, 6, (uint64_t)v * 2 + (uint64_t)dir), wlo, whi) : 0;
        A.src[A.m] = v; A.dst[A.m] = u; if (weighted) A.w[A.m] = wv; A.m++;
        A.src[A.m] = u; A.dst[A.m] = v; if (weighted) A.w[A.m] = wv; A.m++;
      }
    }
  int rc = build_csr(n, &A, rowptr, col, w, nnz);
  free(A.src); free(A.dst); free(A.w);
  return rc;
}

/* ----------------------------------------------------------- source picks */
/* k sources drawn uniformly without replacement from vertices with
 * out-degree >= 1 (partial Fisher-Yates).  Returns -3 if too few exist. */
int gg_sample_sources(int32_t n, const int64_t* rowptr, int32_t k, uint64_t seed, int32_t* out) {
  int32_t* cand = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n ? n : 1));
  if (!cand) return -1;
  int32_t c = 0;
  for (int32_t v = 0; v < n; v++) if (rowptr[v + 1] > rowptr[v]) cand[c++] = v;
  if (k > c) { free(cand); return -3; }
  for (int32_t i = 0; i < k; i++) {
    uint64_t r = draw(seed, 7, (uint64_t)i);
    int32_t j = i + (int32_t)(((r >> 32) * (uint64_t)(c - i)) >> 32);
    int32_t t = cand[i]; cand[i] = cand[j]; cand[j] = t;
    out[i] = cand[i];
  }
  free(cand);
  return 0;
}

void gg_free(void* p) { free(p); }
