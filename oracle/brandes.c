/*
 * CPU oracle for MFBC -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, __graft_entry__.smoke() and the CPU-baseline /
 * reference legs of bench.py may load or run this code.  The CUDA library
 * never calls it and shares no code with it.
 *
 * What it computes (paper Sec. 2.4, "Brandes' Algorithm", and Table 1):
 *   tau(s,v)       shortest-path distance from s to v;
 *   sigma_bar(s,v) number of shortest s-v paths (sigma_bar(s,s) = 1);
 *   delta(s,v)     dependency of s on v, sum over t of sigma(s,t,v)/sigma_bar(s,t),
 *                  with sigma(s,s,v) = sigma(s,t,s) = sigma(s,t,t) = 0;
 *   lambda(v)      sum over the listed sources s (ordered pairs) of delta(s,v).
 * Theorem 1 states that MFBC (Algorithms 1-3) returns exactly this lambda, so
 * the oracle is Brandes' algorithm written plainly:
 *   - forward: breadth-first search for unit weights (Sec. 2.3) or Dijkstra
 *     with a binary heap for integer weights >= 1; sigma_bar of a vertex is
 *     the sum of sigma_bar over its predecessors on shortest paths, i.e. the
 *     vertices u with an arc u->v and tau(s,u) + A(u,v) = tau(s,v);
 *   - backward: in reverse settling order (non-increasing distance),
 *     delta(s,v) = sum over arcs v->w with tau(s,w) = tau(s,v) + A(v,w)
 *     of sigma_bar(s,v)/sigma_bar(s,w) * (1 + delta(s,w))      (Sec. 2.4);
 *   - lambda(v) += delta(s,v) for every v != s.
 * Unreachable vertices have sigma_bar = 0 and delta = 0.  Everything is FP64;
 * sigma_bar is also counted exactly in a saturating unsigned 128-bit shadow so
 * that a path count at or above 2^53 (where FP64 stops being exact) is flagged.
 *
 * Graph input: CSR of A (row v lists arcs v -> col[k] with weight w[k]);
 * w == NULL means every arc weighs 1.  No validation beyond what the tests
 * need: callers pass well-formed graphs.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define ORACLE_INF INT32_MAX
typedef unsigned __int128 u128;
static const u128 U128_MAX = ~(u128)0;
static const u128 TWO53 = (u128)1 << 53;

typedef struct {
  int32_t n;
  const int64_t* rowptr;
  const int32_t* col;
  const int32_t* w;
} graph_t;

typedef struct {            /* per-thread scratch for one single-source run */
  int32_t* dist;
  double* sigma;
  u128* sig128;
  int32_t* order;           /* vertices in settling order */
  double* delta;
  int64_t* heap_d;          /* binary heap of (distance, vertex) */
  int32_t* heap_v;
  int64_t heap_cap;
} scratch_t;

static int scratch_init(scratch_t* S, int32_t n, int64_t nnz) {
  size_t nn = (size_t)(n ? n : 1);
  S->dist = (int32_t*)malloc(sizeof(int32_t) * nn);
  S->sigma = (double*)malloc(sizeof(double) * nn);
  S->sig128 = (u128*)malloc(sizeof(u128) * nn);
  S->order = (int32_t*)malloc(sizeof(int32_t) * nn);
  S->delta = (double*)malloc(sizeof(double) * nn);
  S->heap_cap = nnz + 2;
  S->heap_d = (int64_t*)malloc(sizeof(int64_t) * (size_t)S->heap_cap);
  S->heap_v = (int32_t*)malloc(sizeof(int32_t) * (size_t)S->heap_cap);
  return (S->dist && S->sigma && S->sig128 && S->order && S->delta && S->heap_d && S->heap_v) ? 0 : -1;
}

static void scratch_free(scratch_t* S) {
  free(S->dist); free(S->sigma); free(S->sig128); free(S->order); free(S->delta);
  free(S->heap_d); free(S->heap_v);
}

static inline u128 sat_add(u128 a, u128 b) { return (a > U128_MAX - b) ? U128_MAX : a + b; }

/* ---- binary min-heap on (distance, vertex), lazy deletion ---- */
static void heap_push(scratch_t* S, int64_t* sz, int64_t d, int32_t v) {
  int64_t i = (*sz)++;
  while (i > 0) {
    int64_t p = (i - 1) / 2;
    if (S->heap_d[p] <= d) break;
    S->heap_d[i] = S->heap_d[p]; S->heap_v[i] = S->heap_v[p];
    i = p;
  }
  S->heap_d[i] = d; S->heap_v[i] = v;
}

static void heap_pop(scratch_t* S, int64_t* sz, int64_t* d, int32_t* v) {
  *d = S->heap_d[0]; *v = S->heap_v[0];
  int64_t last = --(*sz);
  int64_t ld = S->heap_d[last]; int32_t lv = S->heap_v[last];
  int64_t i = 0;
  for (;;) {
    int64_t c = 2 * i + 1;
    if (c >= last) break;
    if (c + 1 < last && S->heap_d[c + 1] < S->heap_d[c]) c++;
    if (S->heap_d[c] >= ld) break;
    S->heap_d[i] = S->heap_d[c]; S->heap_v[i] = S->heap_v[c];
    i = c;
  }
  S->heap_d[i] = ld; S->heap_v[i] = lv;
}

/* Forward pass from s: fills dist, sigma, sig128 and the settling order.
 * Returns the number of settled (reachable) vertices. */
static int32_t forward(const graph_t* G, scratch_t* S, int32_t s) {
  const int32_t n = G->n;
  for (int32_t v = 0; v < n; v++) { S->dist[v] = ORACLE_INF; S->sigma[v] = 0.0; S->sig128[v] = 0; }
  S->dist[s] = 0; S->sigma[s] = 1.0; S->sig128[s] = 1;
  int32_t cnt = 0;
  if (!G->w) {
    /* breadth-first search: the queue is the settling order */
    int32_t head = 0;
    S->order[cnt++] = s;
    while (head < cnt) {
      int32_t v = S->order[head++];
      for (int64_t k = G->rowptr[v]; k < G->rowptr[v + 1]; k++) {
        int32_t u = G->col[k];
        if (S->dist[u] == ORACLE_INF) { S->dist[u] = S->dist[v] + 1; S->order[cnt++] = u; }
        if (S->dist[u] == S->dist[v] + 1) {
          S->sigma[u] += S->sigma[v];
          S->sig128[u] = sat_add(S->sig128[u], S->sig128[v]);
        }
      }
    }
  } else {
    /* Dijkstra with a binary heap; a vertex's sigma is final when it is popped
     * because every predecessor is strictly closer (weights >= 1). */
    unsigned char* done = (unsigned char*)calloc((size_t)(n ? n : 1), 1);
    int64_t hs = 0;
    heap_push(S, &hs, 0, s);
    while (hs > 0) {
      int64_t d; int32_t v;
      heap_pop(S, &hs, &d, &v);
      if (done[v] || d != S->dist[v]) continue;
      done[v] = 1;
      S->order[cnt++] = v;
      for (int64_t k = G->rowptr[v]; k < G->rowptr[v + 1]; k++) {
        int32_t u = G->col[k];
        int64_t nd = d + (int64_t)G->w[k];
        if (nd < S->dist[u]) {
          S->dist[u] = (int32_t)nd; S->sigma[u] = S->sigma[v]; S->sig128[u] = S->sig128[v];
          if (hs >= S->heap_cap) {
            S->heap_cap *= 2;
            S->heap_d = (int64_t*)realloc(S->heap_d, sizeof(int64_t) * (size_t)S->heap_cap);
            S->heap_v = (int32_t*)realloc(S->heap_v, sizeof(int32_t) * (size_t)S->heap_cap);
          }
          heap_push(S, &hs, nd, u);
        } else if (nd == S->dist[u]) {
          S->sigma[u] += S->sigma[v];
          S->sig128[u] = sat_add(S->sig128[u], S->sig128[v]);
        }
      }
    }
    free(done);
  }
  return cnt;
}

/* Backward pass (Brandes' dependency recurrence) over the settling order. */
static void backward(const graph_t* G, scratch_t* S, int32_t cnt) {
  for (int32_t i = 0; i < cnt; i++) S->delta[S->order[i]] = 0.0;
  for (int32_t i = cnt - 1; i >= 0; i--) {
    int32_t v = S->order[i];
    double acc = 0.0;
    for (int64_t k = G->rowptr[v]; k < G->rowptr[v + 1]; k++) {
      int32_t wv = G->col[k];
      int32_t a = G->w ? G->w[k] : 1;
      if (S->dist[wv] != ORACLE_INF && (int64_t)S->dist[wv] == (int64_t)S->dist[v] + a)
        acc += S->sigma[v] / S->sigma[wv] * (1.0 + S->delta[wv]);
    }
    S->delta[v] = acc;
  }
}

static int any_inexact(const scratch_t* S, int32_t cnt) {
  for (int32_t i = 0; i < cnt; i++) if (S->sig128[S->order[i]] >= TWO53) return 1;
  return 0;
}

typedef struct {
  const graph_t* G;
  const int32_t* sources;
  int32_t i0, i1;           /* source range handled by this thread */
  double* lambda;           /* per-thread partial lambda (bc) */
  int32_t* dist_out;        /* sssp rows */
  double* sigma_out;
  uint8_t* inexact;
  int mode;                 /* 0 = bc, 1 = sssp */
  int rc;
} job_t;

static void* worker(void* p) {
  job_t* J = (job_t*)p;
  const graph_t* G = J->G;
  scratch_t S;
  J->rc = 0;
  if (scratch_init(&S, G->n, G->rowptr[G->n]) != 0) { J->rc = -1; scratch_free(&S); return NULL; }
  for (int32_t i = J->i0; i < J->i1; i++) {
    int32_t s = J->sources[i];
    int32_t cnt = forward(G, &S, s);
    if (J->inexact) J->inexact[i] = (uint8_t)any_inexact(&S, cnt);
    if (J->mode == 1) {
      memcpy(J->dist_out + (size_t)i * G->n, S.dist, sizeof(int32_t) * (size_t)G->n);
      if (J->sigma_out) memcpy(J->sigma_out + (size_t)i * G->n, S.sigma, sizeof(double) * (size_t)G->n);
    } else {
      backward(G, &S, cnt);
      for (int32_t k = 0; k < cnt; k++) {
        int32_t v = S.order[k];
        if (v != s) J->lambda[v] += S.delta[v];
      }
    }
  }
  scratch_free(&S);
  return NULL;
}

static int run(const graph_t* G, const int32_t* sources, int32_t nsrc, int nthreads, int mode,
               double* lambda_out, int32_t* dist_out, double* sigma_out, uint8_t* inexact_out) {
  if (nthreads < 1) nthreads = 1;
  if (nthreads > nsrc) nthreads = nsrc > 0 ? nsrc : 1;
  if (nthreads > 512) nthreads = 512;
  pthread_t th[512];
  job_t jobs[512];
  double* partial = NULL;
  if (mode == 0) {
    partial = (double*)calloc((size_t)nthreads * (size_t)(G->n ? G->n : 1), sizeof(double));
    if (!partial) return -1;
  }
  for (int t = 0; t < nthreads; t++) {
    job_t* J = &jobs[t];
    J->G = G; J->sources = sources;
    J->i0 = (int32_t)((int64_t)nsrc * t / nthreads);
    J->i1 = (int32_t)((int64_t)nsrc * (t + 1) / nthreads);
    J->lambda = partial ? partial + (size_t)t * (size_t)G->n : NULL;
    J->dist_out = dist_out; J->sigma_out = sigma_out; J->inexact = inexact_out;
    J->mode = mode;
    pthread_create(&th[t], NULL, worker, J);
  }
  int rc = 0;
  for (int t = 0; t < nthreads; t++) { pthread_join(th[t], NULL); if (jobs[t].rc) rc = jobs[t].rc; }
  if (mode == 0) {
    for (int32_t v = 0; v < G->n; v++) {
      double acc = 0.0;
      for (int t = 0; t < nthreads; t++) acc += partial[(size_t)t * (size_t)G->n + v];
      lambda_out[v] = acc;
    }
    free(partial);
  }
  return rc;
}

/* lambda_out[v] = sum over sources[i] of delta(sources[i], v), v != source. */
int oracle_bc(int32_t n, const int64_t* rowptr, const int32_t* col, const int32_t* w,
              const int32_t* sources, int32_t nsrc, int nthreads,
              double* lambda_out, uint8_t* inexact_out) {
  graph_t G = {n, rowptr, col, w};
  return run(&G, sources, nsrc, nthreads, 0, lambda_out, NULL, NULL, inexact_out);
}

/* Row i of dist_out / sigma_out holds tau(sources[i], .) / sigma_bar(sources[i], .);
 * unreachable: INT32_MAX and 0. */
int oracle_sssp(int32_t n, const int64_t* rowptr, const int32_t* col, const int32_t* w,
                const int32_t* sources, int32_t nsrc, int nthreads,
                int32_t* dist_out, double* sigma_out, uint8_t* inexact_out) {
  graph_t G = {n, rowptr, col, w};
  return run(&G, sources, nsrc, nthreads, 1, NULL, dist_out, sigma_out, inexact_out);
}

/* delta(s, .) for one source (diagnostics and the per-source tests). */
int oracle_delta(int32_t n, const int64_t* rowptr, const int32_t* col, const int32_t* w,
                 int32_t s, double* delta_out) {
  graph_t G = {n, rowptr, col, w};
  scratch_t S;
  if (scratch_init(&S, n, rowptr[n]) != 0) { scratch_free(&S); return -1; }
  int32_t cnt = forward(&G, &S, s);
  backward(&G, &S, cnt);
  for (int32_t v = 0; v < n; v++) delta_out[v] = 0.0;
  for (int32_t i = 0; i < cnt; i++) delta_out[S.order[i]] = S.delta[S.order[i]];
  scratch_free(&S);
  return 0;
}
