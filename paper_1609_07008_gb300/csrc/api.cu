// C ABI of the MFBC library: argument checks, choice of kernel family and
// batch width, scratch management, and the batch loop of Algorithm 3.
#include <algorithm>
#include <cstring>
#include <chrono>
#include <mutex>
#include <optional>
#include <string>

#include "internal.cuh"

using namespace mfbc;

struct mfbc_graph {
  DevGraph g;
  void* ws = nullptr;              // cached scratch (cudaMalloc), grown on demand
  size_t ws_bytes = 0;
  uint32_t* h_ctr = nullptr;       // pinned counter mirror
  uint32_t flags = 0;
  std::mutex mu;
  // autotuner results (mfbc_autotune): batch width per kernel family
  // (0 = not tuned), the family AUTO picks, and the general kernels' arcs
  // per step (0 = by average degree); force_arcs overrides it while tuning
  int tuned_nb[4] = {0, 0, 0, 0};   // level, general, distance, persistent small-graph kernels
  int tuned_arcs = 0;
  int tuned_path = 0;               // kernel family for MFBC_PATH_AUTO (0 = by weights)
  int force_arcs = 0;
  int tuned_accum = 0;              // general kernels' accumulator for MFBC_ACCUM_AUTO (0 = per product)
};

static thread_local std::string t_err;

static mfbc_status fail(mfbc_status s, const std::string& msg) {
  t_err = msg;
  return s;
}

extern "C" const char* mfbc_status_string(mfbc_status s) {
  switch (s) {
    case MFBC_OK: return "ok";
    case MFBC_ERR_INVALID: return "invalid argument";
    case MFBC_ERR_OOM: return "out of memory";
    case MFBC_ERR_CUDA: return "CUDA error";
    case MFBC_ERR_OVERFLOW: return "distance overflow";
    case MFBC_ERR_NO_CONVERGENCE: return "no convergence";
    case MFBC_ERR_TIMEOUT: return "device wait timed out";
  }
  return "unknown status";
}

extern "C" const char* mfbc_last_error(void) { return t_err.c_str(); }

extern "C" const char* mfbc_version(void) { return "mfbc-gb300 0.1 (sm_103a)"; }

// ------------------------------------------------------------------ graphs
// Arrays given in CSC orientation hold the rows of A^T (row v lists the tails
// of the arcs into v).  For a directed graph they are checked as rows
// (row pointers, column range, strictly increasing columns: the checks that
// the transposition itself relies on) and turned into the rows of A by a
// stable counting sort, which leaves every row of A sorted; graph_build then
// validates A as usual.  An undirected A equals A^T: nothing to do.
static mfbc_status csc_to_csr(int32_t n, int64_t nnz, const int64_t* rp, const int32_t* col, const int32_t* w,
                              std::vector<int64_t>& orp, std::vector<int32_t>& ocol, std::vector<int32_t>& ow) {
  for (int32_t v = 0; v < n; v++)
    if (rp[v + 1] < rp[v] || rp[v + 1] > nnz)
      return fail(MFBC_ERR_INVALID, "rowptr must start at 0, be non-decreasing and end at nnz");
  orp.assign((size_t)n + 1, 0);
  for (int32_t v = 0; v < n; v++)
    for (int64_t k = rp[v]; k < rp[v + 1]; k++) {
      const int32_t u = col[k];
      if (u < 0 || u >= n) return fail(MFBC_ERR_INVALID, "column index out of range [0, n)");
      if (k > rp[v] && col[k - 1] >= u) return fail(MFBC_ERR_INVALID, "rows must be sorted by column without duplicate arcs");
      orp[(size_t)u + 1]++;
    }
  for (int32_t u = 0; u < n; u++) orp[(size_t)u + 1] += orp[(size_t)u];
  ocol.resize((size_t)nnz);
  if (w) ow.resize((size_t)nnz);
  std::vector<int64_t> pos(orp.begin(), orp.end() - 1);
  for (int32_t v = 0; v < n; v++)            // rows of A^T in order: each row of A receives its heads sorted
    for (int64_t k = rp[v]; k < rp[v + 1]; k++) {
      const int64_t p = pos[(size_t)col[k]]++;
      ocol[(size_t)p] = v;
      if (w) ow[(size_t)p] = w[k];
    }
  return MFBC_OK;
}

static mfbc_status create_common(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                                 const int32_t* w, uint32_t flags, void* stream, mfbc_graph** out) {
  std::vector<int64_t> trp;
  std::vector<int32_t> tcol, tw;
  if ((flags & MFBC_CSC) && !(flags & MFBC_UNDIRECTED)) {
    mfbc_status s = csc_to_csr(n, nnz, rowptr, col, w, trp, tcol, tw);
    if (s) return s;
    rowptr = trp.data();
    col = tcol.data();
    w = w ? tw.data() : nullptr;
  }
  auto* G = new (std::nothrow) mfbc_graph();
  if (!G) return fail(MFBC_ERR_OOM, "host allocation of the graph handle failed");
  std::string err;
  mfbc_status s = graph_build(n, nnz, rowptr, col, w, flags, (cudaStream_t)stream, &G->g, &err);
  if (s == MFBC_OK) {
    cudaError_t e = cudaMallocHost((void**)&G->h_ctr, 64);
    if (e != cudaSuccess) { s = MFBC_ERR_OOM; err = "cudaMallocHost of the counter mirror failed"; }
  }
  if (s != MFBC_OK) {
    graph_free(&G->g);
    if (G->h_ctr) cudaFreeHost(G->h_ctr);
    delete G;
    cudaGetLastError();
    return fail(s, err);
  }
  G->flags = flags;
  *out = G;
  t_err.clear();
  return MFBC_OK;
}

static mfbc_status check_create_args(int32_t n, int64_t nnz, const void* rowptr, const void* col,
                                     uint32_t flags, mfbc_graph** out) {
  if (!out) return fail(MFBC_ERR_INVALID, "out must not be NULL");
  *out = nullptr;
  if (n < 0) return fail(MFBC_ERR_INVALID, "n must be >= 0");
  if (nnz < 0) return fail(MFBC_ERR_INVALID, "nnz must be >= 0");
  if (!rowptr) return fail(MFBC_ERR_INVALID, "rowptr must not be NULL");
  if (nnz > 0 && !col) return fail(MFBC_ERR_INVALID, "col must not be NULL when nnz > 0");
  if (flags & ~(MFBC_CSC | MFBC_UNDIRECTED)) return fail(MFBC_ERR_INVALID, "unknown flag bits");
  return MFBC_OK;
}

extern "C" mfbc_status mfbc_graph_create(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                                         const int32_t* w, uint32_t flags, void* stream, mfbc_graph** out) {
  mfbc_status s = check_create_args(n, nnz, rowptr, col, flags, out);
  if (s) return s;
  if (rowptr[0] != 0 || rowptr[n] != nnz) return fail(MFBC_ERR_INVALID, "rowptr[0] must be 0 and rowptr[n] == nnz");
  return create_common(n, nnz, rowptr, col, w, flags, stream, out);
}

extern "C" mfbc_status mfbc_graph_create_device(int32_t n, int64_t nnz, const int64_t* rowptr,
                                                const int32_t* col, const int32_t* w, uint32_t flags,
                                                void* stream, mfbc_graph** out) {
  mfbc_status s = check_create_args(n, nnz, rowptr, col, flags, out);
  if (s) return s;
  // stage through the host: construction also needs the row pointers there
  std::vector<int64_t> rp((size_t)n + 1);
  std::vector<int32_t> c((size_t)nnz), ww(w ? (size_t)nnz : 0);
  cudaStream_t st = (cudaStream_t)stream;
  if (cudaMemcpyAsync(rp.data(), rowptr, sizeof(int64_t) * rp.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      (nnz && cudaMemcpyAsync(c.data(), col, sizeof(int32_t) * c.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      (w && nnz && cudaMemcpyAsync(ww.data(), w, sizeof(int32_t) * ww.size(), cudaMemcpyDeviceToHost, st) != cudaSuccess) ||
      cudaStreamSynchronize(st) != cudaSuccess) {
    cudaGetLastError();
    return fail(MFBC_ERR_CUDA, "copying the device graph arrays failed");
  }
  if (rp[0] != 0 || rp[(size_t)n] != nnz) return fail(MFBC_ERR_INVALID, "rowptr[0] must be 0 and rowptr[n] == nnz");
  return create_common(n, nnz, rp.data(), c.data(), w ? ww.data() : nullptr, flags, stream, out);
}

extern "C" void mfbc_graph_destroy(mfbc_graph* G) {
  if (!G) return;
  graph_free(&G->g);
  if (G->ws) cudaFree(G->ws);
  if (G->h_ctr) cudaFreeHost(G->h_ctr);
  delete G;
}

extern "C" mfbc_status mfbc_graph_release_scratch(mfbc_graph* G) {
  if (!G) return fail(MFBC_ERR_INVALID, "graph must not be NULL");
  std::lock_guard<std::mutex> lock(G->mu);
  if (G->ws) {
    // calls return once their work is complete, so nothing of this handle
    // runs here; synchronise anyway before giving the memory back
    if (cudaDeviceSynchronize() != cudaSuccess || cudaFree(G->ws) != cudaSuccess) {
      cudaGetLastError();
      return fail(MFBC_ERR_CUDA, "freeing the cached scratch failed");
    }
    G->ws = nullptr;
    G->ws_bytes = 0;
  }
  t_err.clear();
  return MFBC_OK;
}

extern "C" mfbc_status mfbc_graph_info(const mfbc_graph* G, int32_t* n, int64_t* nnz, uint32_t* flags,
                                       int32_t* unit) {
  if (!G) return fail(MFBC_ERR_INVALID, "graph must not be NULL");
  if (n) *n = G->g.n;
  if (nnz) *nnz = G->g.nnz;
  if (flags) *flags = G->flags;
  if (unit) *unit = G->g.unit ? 1 : 0;
  return MFBC_OK;
}

// ------------------------------------------------------------------ planning
struct Plan {
  int path = MFBC_PATH_GENERAL;
  int nb = 32;
  int groups = 0;                  // persistent small-graph kernel: block groups
  int64_t table_batches = 1;       //   and the batches its table holds
  int Lcap = 0;
  int64_t list_cap = 0;
  size_t state_bytes = 0;          // kernel-family state
  size_t extra_bytes = 0;          // lambda, device sources, sssp staging
  size_t total = 0;
};

static inline size_t al256(size_t b) { return (b + 255) & ~size_t(255); }

static size_t extras(const DevGraph& g, int32_t nsrc, int mode, int nb, bool host_io, int path) {
  size_t b = 0;
  if (path == MFBC_PATH_SMALL) {             // the call's batch table: sources, lambda rows, packed columns
    const size_t nbatch = std::max<size_t>(1, ((size_t)nsrc + nb - 1) / nb);
    b += 2 * al256(sizeof(int32_t) * nbatch * nb) + al256(sizeof(int32_t) * nbatch * (nb / 32));
  }
  if (mode == 0) b += al256(sizeof(double) * (size_t)std::max(g.n, 1));        // device lambda
  if (host_io) b += al256(sizeof(int32_t) * (size_t)std::max(nsrc, 1));        // device sources
  if (mode == 0) b += al256(sizeof(int32_t) * (size_t)std::max(nsrc, 1));      // reordered sources
  if (mode == 1 && host_io) b += al256((sizeof(int32_t) + sizeof(double)) * (size_t)nb * std::max(g.n, 1));
  if (mode == 2) b += 2 * al256(sizeof(int32_t) * (size_t)nb);                 // packed batch columns
  return b;
}

static void level_caps(const DevGraph& g, int nb, int* Lcap, int64_t* list_cap) {
  (void)nb;
  const int64_t n = g.n;
  *Lcap = (int)std::min<int64_t>(n + 2, 48);
  *list_cap = n * std::min<int64_t>(*Lcap, 24) + 64;
}

static size_t plan_bytes(const DevGraph& g, int path, int nb, int32_t nsrc, int mode, bool host_io,
                         Plan* p) {
  p->path = path;
  p->nb = nb;
  if (path == MFBC_PATH_LEVEL) {
    level_caps(g, nb, &p->Lcap, &p->list_cap);
    // room for the general kernels at n_b = 32 too: the fallback used when
    // a batch is deeper than the level capacity runs in the same scratch
    p->state_bytes = std::max(level_bytes(g, nb, p->Lcap, p->list_cap), general_bytes(g.n, 32));
  } else if (path == MFBC_PATH_DIST) {
    p->state_bytes = dist_bytes(g.n, nb, g.wmax + 1);
  } else if (path == MFBC_PATH_SMALL) {
    // batches too deep for the kernel's byte levels are redone by the general
    // kernels at n_b = 32 in the same scratch
    const int nbatch = (int)std::max<int64_t>(1, ((int64_t)nsrc + nb - 1) / nb);
    p->table_batches = nbatch;
    p->groups = small_groups(g.n, nb, mode == 1 ? 1 : nbatch);
    p->state_bytes = std::max(small_bytes(g.n, nb, p->groups), general_bytes(g.n, 32));
  } else {
    p->state_bytes = general_bytes(g.n, nb);
  }
  p->extra_bytes = extras(g, nsrc, mode, nb, host_io, path);
  p->total = p->state_bytes + p->extra_bytes;
  return p->total;
}

// Kernel family for MFBC_PATH_AUTO without tuning: level kernels for unit
// weights; distance-ordered kernels for weights <= 128 on graphs without hubs
// (no degree above max(64, 4x the average): each distance step waits for its
// longest adjacency list, so hubs make the steps slow -- weighted R-MAT 16,
// 4096 sources: 3661 ms against 281 ms on the general kernels -- while grids
// and uniform random graphs gain: weighted 256^2 grid 313 against 2883 ms,
// Erdos-Renyi n = 2^16, k = 1024, 256 sources 153 against 326 ms); general
// kernels otherwise.
// Unit-weight graphs small enough for the persistent kernel to win: its
// levels scan every (vertex, word) and every in-arc of an open vertex, which
// costs more than the per-product kernels as the graph grows (R-MAT 14,
// 16384 vertices, 4096 sources: 45 ms), while on small graphs the
// per-product kernels wait on launches (Erdos-Renyi n = 1024, all sources:
// 0.75 ms here against 14.7 ms).  mfbc_autotune compares the two.
static bool small_graph(const DevGraph& g) { return g.n <= (1 << 13) && g.nnz <= (1 << 18); }
// graphs on which mfbc_autotune also times the persistent kernel
static bool small_tunable(const DevGraph& g) { return g.n <= (1 << 15) && g.nnz <= (1 << 19); }

static int default_path(const DevGraph& g) {
  if (g.unit) return small_graph(g) ? MFBC_PATH_SMALL : MFBC_PATH_LEVEL;
  const int64_t avg = g.n ? g.nnz / g.n : 0;
  const int64_t deg_cap = std::max<int64_t>(64, 4 * avg);
  if (g.wmax <= 128 && std::max(g.max_deg, g.max_in_deg) <= deg_cap && (uint64_t)g.n * 128u <= 0xffffffffull)
    return MFBC_PATH_DIST;
  return MFBC_PATH_GENERAL;
}

static int tuned_slot(int path) {
  return path == MFBC_PATH_LEVEL ? 0 : path == MFBC_PATH_GENERAL ? 1 : path == MFBC_PATH_DIST ? 2 : 3;
}

static mfbc_status make_plan(const mfbc_graph* G, int32_t nsrc, int mode, const mfbc_options* opt,
                             bool host_io, Plan* p) {
  const DevGraph& g = G->g;
  int path = opt ? opt->path : MFBC_PATH_AUTO;
  if (path == MFBC_PATH_AUTO) path = G->tuned_path ? G->tuned_path : default_path(g);
  else if ((path == MFBC_PATH_LEVEL || path == MFBC_PATH_SMALL) && !g.unit)
    return fail(MFBC_ERR_INVALID, path == MFBC_PATH_LEVEL ? "MFBC_PATH_LEVEL needs unit weights"
                                                          : "MFBC_PATH_SMALL needs unit weights");
  else if (path == MFBC_PATH_DIST && g.wmax + 1 > DIST_MAX_BUCKETS)
    return fail(MFBC_ERR_INVALID, "MFBC_PATH_DIST needs weights <= 4096");
  else if (path == MFBC_PATH_DIST && (uint64_t)g.n * 128u > 0xffffffffull)
    return fail(MFBC_ERR_INVALID, "MFBC_PATH_DIST needs n < 2^25");
  else if (path != MFBC_PATH_GENERAL && path != MFBC_PATH_LEVEL && path != MFBC_PATH_DIST &&
           path != MFBC_PATH_SMALL)
    return fail(MFBC_ERR_INVALID, "unknown path");
  int maxnb = path == MFBC_PATH_LEVEL ? LEVEL_MAX_NB : (path == MFBC_PATH_SMALL ? 1024 : 4096);
  if (path == MFBC_PATH_DIST) {
    // the distance kernels' settled list holds up to n * n_b (vertex, word)
    // entries addressed by 32-bit offsets: n * n_b must stay below 2^32
    const int64_t cap = ((int64_t)0xfffffffe / std::max<int64_t>(g.n, 1)) / 32 * 32;
    maxnb = (int)std::min<int64_t>(maxnb, cap);
    if (maxnb < 32) return fail(MFBC_ERR_INVALID, "MFBC_PATH_DIST needs n < 2^27");
  }
  // the level kernels move 128 columns (four 32-column words) at a time
  const int gran = path == MFBC_PATH_LEVEL ? 128 : 32;
  int req = opt ? opt->n_b : 0;
  if (req < 0) return fail(MFBC_ERR_INVALID, "n_b must be >= 0");
  if (path == MFBC_PATH_LEVEL && (int64_t)g.n * (LEVEL_MAX_NB / 128) >= (1ll << 31))
    // pair records name a row as vertex * (n_b / 128) + quad in 31 bits
    maxnb = (int)std::max<int64_t>(128, (((1ll << 31) - 1) / std::max<int64_t>(g.n, 1)) * 128);
  if (path == MFBC_PATH_LEVEL && (int64_t)g.n * (maxnb / 128) >= (1ll << 31))
    return fail(MFBC_ERR_INVALID, "graph too large for the level kernels' 31-bit pair row indices");
  if (req > 0) {
    int nb = (req + gran - 1) / gran * gran;
    if (nb > maxnb) return fail(MFBC_ERR_INVALID, "n_b too large for this path (max " + std::to_string(maxnb) + ")");
    plan_bytes(g, path, nb, nsrc, mode, host_io, p);
    return MFBC_OK;
  }
  // auto: widest batch (<= number of sources, <= the tuned width) whose
  // scratch fits the budget
  const int tuned = G->tuned_nb[tuned_slot(path)];
  size_t budget;
  if (opt && opt->workspace) budget = opt->workspace_bytes;
  else {
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) { cudaGetLastError(); return fail(MFBC_ERR_CUDA, "cudaMemGetInfo failed"); }
    budget = (size_t)(0.80 * (double)(fr + G->ws_bytes));
  }
  // the persistent small-graph kernel runs batches side by side: 128 columns
  // per batch leave it several batches to spread over its block groups.  On
  // dense graphs (average degree >= 64) the distance kernels check one
  // 4-byte distance per in-arc and pair, each in its own 32-byte sector, so
  // a batch whose distances stay in the L2 wins: dense weighted ER n = 2^16,
  // k = 1024, 4096 sources, n_b 256 / 512 / 1024 / 4096: 64.9 / 66.0 /
  // 62.3 / 51.5 GTEPS
  const bool dense_dist = path == MFBC_PATH_DIST && g.nnz >= 64 * (int64_t)std::max(g.n, 1);
  const int widest = tuned > 0 ? tuned : (path == MFBC_PATH_SMALL ? 128 : dense_dist ? std::min(maxnb, 512) : maxnb);
  int nb = std::min(widest, std::max(gran, (nsrc + gran - 1) / gran * gran));
  while (true) {
    plan_bytes(g, path, nb, nsrc, mode, host_io, p);
    if (p->total <= budget || nb == gran) break;
    nb -= gran;
  }
  return MFBC_OK;
}

extern "C" mfbc_status mfbc_workspace_size(const mfbc_graph* G, int32_t nsrc, int32_t mode,
                                           const mfbc_options* opt, uint64_t* bytes) {
  if (!G || !bytes) return fail(MFBC_ERR_INVALID, "graph and bytes must not be NULL");
  if (nsrc < 0 || mode < 0 || mode > 2) return fail(MFBC_ERR_INVALID, "bad nsrc or mode");
  Plan p;
  mfbc_options o = opt ? *opt : mfbc_options{};
  o.workspace = nullptr;
  mfbc_status s = make_plan(G, nsrc, mode, &o, mode != 2, &p);
  if (s) return s;
  *bytes = p.total;
  return MFBC_OK;
}

// ------------------------------------------------------------------ runner
namespace {

struct Run {
  mfbc_graph* G;
  const mfbc_options* opt;
  cudaStream_t st;
  Profiler prof;
  std::string err;
  Plan plan;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  const int32_t* req_off = nullptr;  // mode 2: host offsets of the requests in the source list
  int32_t nreq = 0;
};

mfbc_status get_workspace(Run& R) {
  const mfbc_options* opt = R.opt;
  if (opt && opt->workspace) {
    if ((uintptr_t)opt->workspace & 255u) return fail(MFBC_ERR_INVALID, "workspace must be 256-byte aligned");
    if (opt->workspace_bytes < R.plan.total)
      return fail(MFBC_ERR_INVALID, "workspace too small: need " + std::to_string(R.plan.total) + " bytes");
    R.ws = (char*)opt->workspace;
    R.ws_bytes = opt->workspace_bytes;
    return MFBC_OK;
  }
  mfbc_graph* G = R.G;
  if (G->ws_bytes < R.plan.total) {
    if (G->ws) { cudaStreamSynchronize(R.st); cudaFree(G->ws); G->ws = nullptr; G->ws_bytes = 0; }
    cudaError_t e = cudaMalloc(&G->ws, R.plan.total);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(MFBC_ERR_OOM, "cudaMalloc of " + std::to_string(R.plan.total) + " scratch bytes failed");
    }
    G->ws_bytes = R.plan.total;
  }
  R.ws = (char*)G->ws;
  R.ws_bytes = G->ws_bytes;
  return MFBC_OK;
}

void finish_profile(Run& R, mfbc_profile* out, int64_t batches, int64_t fi, int64_t bi, Counters* ctr) {
  if (!out) return;
  R.prof.drain();
  unsigned long long bytes[K_NUM], stat[4];
  if (cudaMemcpy(bytes, ctr->bytes, sizeof(bytes), cudaMemcpyDeviceToHost) != cudaSuccess ||
      cudaMemcpy(stat, ctr->stat, sizeof(stat), cudaMemcpyDeviceToHost) != cudaSuccess) {
    cudaGetLastError();
    memset(bytes, 0, sizeof(bytes));
    memset(stat, 0, sizeof(stat));
  }
  for (int i = 0; i < 4; i++) out->stat[i] = stat[i];
  out->nkernels = 0;
  for (int i = 0; i < K_NUM && out->nkernels < MFBC_MAX_KSTATS; i++) {
    KStat& k = R.prof.k[i];
    if (!k.launches) continue;
    mfbc_kernel_stat& o = out->k[out->nkernels++];
    memset(o.name, 0, sizeof(o.name));
    strncpy(o.name, k.name, sizeof(o.name) - 1);
    o.launches = k.launches;
    o.ms = k.ms;
    o.bytes = k.bytes + (double)bytes[i];
  }
  out->batches = (uint64_t)batches;
  out->fwd_iters = (uint64_t)fi;
  out->bwd_iters = (uint64_t)bi;
  out->n_b = R.plan.nb;
  out->path = R.plan.path;
}

// Ordering key of each source: its distances to the K landmarks (rows[k][v],
// capped at 0xffff) followed by its BFS parent toward landmark 0 (the
// smallest-id neighbour one level closer; itself for the landmark or when
// unreachable).  One warp per source.
__global__ void k_order_keys(const int32_t* __restrict__ src, int32_t nsrc, const int64_t* __restrict__ rowptr,
                             const int32_t* __restrict__ col, const int32_t* __restrict__ rows, int32_t n, int K,
                             int32_t* keys) {
  const uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  if (gw >= (uint64_t)nsrc) return;
  const int32_t s = src[gw];
  int32_t* key = keys + gw * (uint64_t)(K + 1);
  for (int k = (int)lane; k < K; k += 32) key[k] = min(rows[(size_t)k * n + s], 0xffff);
  const int32_t ds = rows[s];
  int32_t best = 0x7fffffff;
  if (ds > 0 && ds != 0x7fffffff)
    for (int64_t k = rowptr[s] + lane; k < rowptr[s + 1]; k += 32) {
      const int32_t u = col[k];
      if (rows[u] == ds - 1 && u < best) best = u;
    }
  for (int o = 16; o; o >>= 1) best = min(best, __shfl_xor_sync(0xffffffffu, best, o));
  if (lane == 0) key[K] = best == 0x7fffffff ? s : best;
}

// Group sources of similar distance profile into the same batches (level
// kernels, undirected graphs): one MFBF pass from the K highest-degree
// vertices gives every vertex's distances to them, and the sources are sorted
// by that vector (lexicographically), then by BFS parent.  Sources at equal
// distances from many well-connected vertices reach most other vertices at
// the same levels, so their frontier bits share words and sectors.  Writes the
// permuted list to d_out; leaves the order alone when it does not apply.  The
// level state's sv array serves as scratch.
mfbc_status order_sources(RunCtx& rc, LevelState& ls, const int32_t* d_src, int32_t nsrc, int32_t* d_out,
                          bool* applied) {
  const DevGraph& g = *rc.g;
  const int32_t n = g.n;
  const int K = (int)g.landmarks.size();
  *applied = false;
  const size_t rows_bytes = al256(sizeof(int32_t) * (size_t)K * n);
  const size_t need = rows_bytes + sizeof(int32_t) * (size_t)(K + 1) * nsrc;
  if (g.directed || K == 0 || K > ls.nb || K > nsrc || need > sizeof(double) * (size_t)n * ls.nb) return MFBC_OK;
  int32_t* rows = (int32_t*)ls.sv;
  int32_t* keys = (int32_t*)((char*)ls.sv + rows_bytes);
  MFBC_CUDA_TRY(cudaMemcpyAsync(d_out, g.landmarks.data(), sizeof(int32_t) * K, cudaMemcpyHostToDevice, rc.stream),
                rc.err);
  int levels = -1;
  bool exceeded = false;
  mfbc_status s = level_batch(rc, ls, d_out, K, nullptr, false, &levels, &exceeded, nullptr, nullptr);
  if (s != MFBC_OK) {
    if (!exceeded) return s;
    return MFBC_OK;                    // too deep for the level masks: keep the given order
  }
  level_output(rc, ls, levels, K, rows, nullptr);
  level_reset(rc, ls, levels);
  k_order_keys<<<(unsigned)(((uint64_t)nsrc * 32 + 255) / 256), 256, 0, rc.stream>>>(d_src, nsrc, g.rowptr, g.col,
                                                                                    rows, n, K, keys);
  std::vector<int32_t> hk((size_t)(K + 1) * nsrc);
  std::vector<int32_t> hs((size_t)nsrc), out((size_t)nsrc), idx((size_t)nsrc);
  MFBC_CUDA_TRY(cudaMemcpyAsync(hk.data(), keys, sizeof(int32_t) * hk.size(), cudaMemcpyDeviceToHost, rc.stream),
                rc.err);
  MFBC_CUDA_TRY(cudaMemcpyAsync(hs.data(), d_src, sizeof(int32_t) * nsrc, cudaMemcpyDeviceToHost, rc.stream), rc.err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(rc.stream), rc.err);
  for (int32_t i = 0; i < nsrc; i++) idx[i] = i;
  std::sort(idx.begin(), idx.end(), [&](int32_t a, int32_t b) {
    const int32_t* x = &hk[(size_t)a * (K + 1)];
    const int32_t* y = &hk[(size_t)b * (K + 1)];
    for (int k = 0; k <= K; k++)
      if (x[k] != y[k]) return x[k] < y[k];
    return a < b;
  });
  for (int32_t i = 0; i < nsrc; i++) out[i] = hs[(size_t)idx[i]];
  MFBC_CUDA_TRY(cudaMemcpyAsync(d_out, out.data(), sizeof(int32_t) * nsrc, cudaMemcpyHostToDevice, rc.stream), rc.err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(rc.stream), rc.err);
  *applied = true;
  return MFBC_OK;
}

// out[j] = src[colidx[j]] for the packed columns of one batch, -1 where empty.
__global__ void k_gather_sources(const int32_t* __restrict__ src, const int32_t* __restrict__ colidx, int nb,
                                 int32_t* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < nb) out[j] = colidx[j] >= 0 ? src[colidx[j]] : -1;
}

// Column layout of several requests packed into batches of nb columns:
// requests in the given order, each starting on a 32-column word boundary,
// spilling into the next batch when one fills.  colidx[b*nb + j] is the
// index into the source list of batch b's column j (-1 empty), wreq[b*W + w]
// the request owning word w (-1 empty), used[b] the columns up to the last
// filled one.
struct Packing {
  std::vector<int32_t> colidx, wreq, used;
  int64_t batches = 0;
};
static Packing pack_requests(const int32_t* off, int32_t nreq, int nb, const int32_t* rows) {
  Packing p;
  const int W = nb / 32;
  auto open_batch = [&]() {
    p.colidx.resize((size_t)(p.batches + 1) * nb, -1);
    p.wreq.resize((size_t)(p.batches + 1) * W, -1);
    p.used.push_back(0);
    p.batches++;
  };
  int col = nb;                                  // no batch open yet
  for (int32_t r = 0; r < nreq; r++) {
    int64_t i = off[r];
    const int64_t e = off[r + 1];
    if (i == e) continue;
    col = (col + 31) / 32 * 32;
    while (i < e) {
      if (col >= nb) { open_batch(); col = 0; }
      const int64_t b = p.batches - 1;
      const int take = (int)std::min<int64_t>(e - i, nb - col);
      for (int t = 0; t < take; t++) p.colidx[(size_t)b * nb + col + t] = (int32_t)(i + t);
      for (int w = col / 32; w <= (col + take - 1) / 32; w++) p.wreq[(size_t)b * W + w] = rows ? rows[r] : r;
      col += take;
      i += take;
      p.used[(size_t)b] = col;
    }
  }
  return p;
}

// Sources outside [0, n) in the batch table become padding (-1) and raise
// FLAG_BAD_SOURCE, so no kernel indexes with them.
__global__ void k_check_table(int32_t* tab, size_t count, int32_t n, Counters* ctr) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count && (tab[i] < -1 || tab[i] >= n)) {
    tab[i] = -1;
    atomicOr(&ctr->flags, FLAG_BAD_SOURCE);
  }
}

// Every batch of the call on the persistent small-graph kernel (one launch
// for modes 0 and 2; mode 1 launches per batch so that host outputs go
// through the one-batch staging rows).  Batches the kernel hands back (deeper
// than its byte levels, or path counts >= 2^58) are recomputed by the
// general kernels at n_b = 32 in the same scratch.
mfbc_status small_path(mfbc_graph* G, Run& R, RunCtx& rc, SmallState& ss, const int32_t* d_src, int32_t nsrc,
                       int mode, double* d_lambda, int32_t* dist_out, double* sigma_out, bool out_on_host,
                       const Packing& pk, int64_t nbatches, char* tab, int32_t* stage_d, double* stage_s,
                       uint32_t* warn, int64_t* fi, int64_t* bi) {
  const DevGraph& g = G->g;
  const Plan& P = R.plan;
  const int nb = P.nb, W = nb / 32;
  const bool multi = mode == 2;
  const size_t nbt = (size_t)P.table_batches;
  int32_t* d_all = (int32_t*)tab;
  int32_t* d_col = (int32_t*)(tab + al256(sizeof(int32_t) * nbt * nb));
  int32_t* d_wreq = (int32_t*)(tab + 2 * al256(sizeof(int32_t) * nbt * nb));
  if ((size_t)nbatches > nbt) { *rc.err = "packed batches exceed the batch table"; return MFBC_ERR_INVALID; }
  if (nbatches == 0) return MFBC_OK;       // no sources: nothing to launch
  if (multi) {
    MFBC_CUDA_TRY(cudaMemcpyAsync(d_col, pk.colidx.data(), sizeof(int32_t) * pk.colidx.size(), cudaMemcpyHostToDevice,
                                  R.st), rc.err);
    const size_t cols = (size_t)nbatches * nb;
    k_gather_sources<<<(unsigned)((cols + 255) / 256), 256, 0, R.st>>>(d_src, d_col, (int)cols, d_all);
    MFBC_CUDA_TRY(cudaMemcpyAsync(d_wreq, pk.wreq.data(), sizeof(int32_t) * pk.wreq.size(), cudaMemcpyHostToDevice,
                                  R.st), rc.err);
  } else {
    fill_i32(d_all, -1, (size_t)nbatches * nb, R.st);
    if (nsrc)
      MFBC_CUDA_TRY(cudaMemcpyAsync(d_all, d_src, sizeof(int32_t) * (size_t)nsrc, cudaMemcpyDeviceToDevice, R.st),
                    rc.err);
  }
  // sources out of [0, n) become padding and fail the call after the launch
  k_check_table<<<(unsigned)(((size_t)nbatches * nb + 255) / 256), 256, 0, R.st>>>(d_all, (size_t)nbatches * nb,
                                                                                  g.n, ss.ctr);
  const uint32_t oflags = R.opt ? R.opt->flags : 0u;
  std::vector<int32_t> redo, part;
  if (mode == 1) {
    for (int64_t b = 0; b < nbatches; b++) {
      const int32_t b0 = (int32_t)(b * nb);
      const int na = std::min(nb, nsrc - b0);
      int32_t* dd = out_on_host ? stage_d : dist_out + (size_t)b0 * g.n;
      double* dsg = sigma_out ? (out_on_host ? stage_s : sigma_out + (size_t)b0 * g.n) : nullptr;
      mfbc_status s = small_run(rc, ss, d_all + (size_t)b * nb, nullptr, 1, nullptr, dd, dsg, na, oflags, &part);
      if (s) return s;
      if (!part.empty()) redo.push_back((int32_t)b);
      else if (out_on_host) {
        MFBC_CUDA_TRY(cudaMemcpyAsync(dist_out + (size_t)b0 * g.n, stage_d, sizeof(int32_t) * (size_t)na * g.n,
                                      cudaMemcpyDeviceToHost, R.st), rc.err);
        if (sigma_out)
          MFBC_CUDA_TRY(cudaMemcpyAsync(sigma_out + (size_t)b0 * g.n, stage_s, sizeof(double) * (size_t)na * g.n,
                                        cudaMemcpyDeviceToHost, R.st), rc.err);
        MFBC_CUDA_TRY(cudaStreamSynchronize(R.st), rc.err);
      }
    }
  } else {
    mfbc_status s = small_run(rc, ss, d_all, multi ? d_wreq : nullptr, (int)nbatches, d_lambda, nullptr, nullptr, 0,
                              oflags, &redo);
    if (s) return s;
  }
  if (rc.h_ctr[0] & FLAG_BAD_SOURCE) { *rc.err = "source id out of range"; return MFBC_ERR_INVALID; }
  if (rc.h_ctr[0] & FLAG_SIGMA_INEXACT) *warn |= MFBC_WARN_SIGMA_INEXACT;
  if (fi) *fi += nbatches - (int64_t)redo.size();
  if (bi) *bi += nbatches - (int64_t)redo.size();
  if (redo.empty()) return MFBC_OK;
  // general kernels for the batches handed back
  Carver c2(R.ws, P.state_bytes);
  GeneralState gs;
  general_carve(c2, g.n, 32, gs);
  MFBC_CUDA_TRY(cudaMemsetAsync(gs.ctr, 0, sizeof(Counters), R.st), rc.err);
  for (int32_t b : redo) {
    const int32_t b0 = (int32_t)((int64_t)b * nb);
    const int na = multi ? nb : std::min(nb, nsrc - b0);
    for (int sb = 0; sb < na; sb += 32) {
      const int nsa = std::min(32, na - sb);
      rc.word_req = multi ? &pk.wreq[(size_t)b * W + sb / 32] : nullptr;
      mfbc_status s = general_batch(rc, gs, d_all + (size_t)b * nb + sb, nsa, mode == 1 ? nullptr : d_lambda, fi, bi);
      if (s) return s;
      if (mode == 1) {
        int32_t* dd = out_on_host ? stage_d + (size_t)sb * g.n : dist_out + (size_t)(b0 + sb) * g.n;
        double* dsg = sigma_out ? (out_on_host ? stage_s + (size_t)sb * g.n : sigma_out + (size_t)(b0 + sb) * g.n)
                                : nullptr;
        general_output(rc, gs, nsa, dd, dsg);
      }
    }
    if (mode == 1 && out_on_host) {
      MFBC_CUDA_TRY(cudaMemcpyAsync(dist_out + (size_t)b0 * g.n, stage_d, sizeof(int32_t) * (size_t)na * g.n,
                                    cudaMemcpyDeviceToHost, R.st), rc.err);
      if (sigma_out)
        MFBC_CUDA_TRY(cudaMemcpyAsync(sigma_out + (size_t)b0 * g.n, stage_s, sizeof(double) * (size_t)na * g.n,
                                      cudaMemcpyDeviceToHost, R.st), rc.err);
      MFBC_CUDA_TRY(cudaStreamSynchronize(R.st), rc.err);
    }
  }
  rc.word_req = nullptr;
  // the general batches flag inexact counts in their own counters
  MFBC_CUDA_TRY(cudaMemcpyAsync(G->h_ctr, &gs.ctr->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, R.st), rc.err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(R.st), rc.err);
  if (G->h_ctr[0] & FLAG_SIGMA_INEXACT) *warn |= MFBC_WARN_SIGMA_INEXACT;
  return MFBC_OK;
}

// mode 0: lambda (d_lambda device, n doubles, overwritten); mode 1: sssp rows;
// mode 2: one lambda row per request (d_lambda device, nreq * n doubles).
mfbc_status run(mfbc_graph* G, const int32_t* d_src, int32_t nsrc, int mode, double* d_lambda,
                int32_t* dist_out, double* sigma_out, bool out_on_host, Run& R, char* extra, int32_t* d_sorted) {
  const DevGraph& g = G->g;
  const Plan& P = R.plan;
  const int nb = P.nb;
  int64_t batches = 0, fi = 0, bi = 0;
  RunCtx rc{&g, R.st, &R.prof, G->h_ctr, &R.err};
  rc.arcs = G->force_arcs ? G->force_arcs : G->tuned_arcs;
  rc.accum = R.opt && R.opt->accumulator ? R.opt->accumulator : G->tuned_accum;
  rc.small_rounds = R.opt && (R.opt->flags & MFBC_OPT_TEST_SMALL_ROUNDS);
  Carver c(R.ws, R.ws_bytes);
  GeneralState gs;
  LevelState ls;
  DistState ds;
  Counters* ctr;
  SmallState ss;
  if (P.path == MFBC_PATH_LEVEL) { level_carve(c, g, nb, P.Lcap, P.list_cap, ls); ctr = ls.ctr; }
  else if (P.path == MFBC_PATH_DIST) { dist_carve(c, g.n, nb, g.wmax + 1, ds); ctr = ds.ctr; }
  else if (P.path == MFBC_PATH_SMALL) { small_carve(c, g.n, nb, P.groups, ss); ctr = ss.ctr; }
  else { general_carve(c, g.n, nb, gs); ctr = gs.ctr; }
  int32_t* stage_d = nullptr;
  double* stage_s = nullptr;
  char* small_tab = extra;
  if (P.path == MFBC_PATH_SMALL) {          // batch table first (see extras)
    const size_t nbatch = (size_t)P.table_batches;
    extra += 2 * al256(sizeof(int32_t) * nbatch * nb) + al256(sizeof(int32_t) * nbatch * (nb / 32));
  }
  if (mode == 1 && out_on_host) {
    stage_d = (int32_t*)extra;
    stage_s = (double*)(extra + al256(sizeof(int32_t) * (size_t)nb * std::max(g.n, 1)));
  }
  MFBC_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(Counters), R.st), &R.err);
  const bool multi = mode == 2;
  const bool want_lambda = mode != 1;
  const int32_t* lrows = multi && R.opt ? R.opt->lambda_rows : nullptr;
  if (want_lambda && g.n && !(R.opt && (R.opt->flags & MFBC_OPT_ACCUMULATE))) {
    if (lrows) {
      for (int32_t r = 0; r < R.nreq; r++)
        MFBC_CUDA_TRY(cudaMemsetAsync(d_lambda + (size_t)lrows[r] * g.n, 0, sizeof(double) * (size_t)g.n, R.st),
                      &R.err);
    } else {
      const size_t rows = multi ? (size_t)R.nreq : 1;
      MFBC_CUDA_TRY(cudaMemsetAsync(d_lambda, 0, sizeof(double) * rows * (size_t)g.n, R.st), &R.err);
    }
  }
  Packing pk;
  int32_t* d_colidx = nullptr;
  int32_t* d_batch = nullptr;
  if (multi) {
    pk = pack_requests(R.req_off, R.nreq, nb, lrows);
    d_colidx = (int32_t*)extra;
    d_batch = (int32_t*)(extra + al256(sizeof(int32_t) * (size_t)nb));
  }
  const int64_t nbatches = multi ? pk.batches : ((int64_t)nsrc + nb - 1) / nb;
  uint32_t warn = 0;
  if (P.path == MFBC_PATH_SMALL) {
    mfbc_status s = small_path(G, R, rc, ss, d_src, nsrc, mode, d_lambda, dist_out, sigma_out, out_on_host, pk,
                               nbatches, small_tab, stage_d, stage_s, &warn, &fi, &bi);
    if (s) return fail(s, R.err.empty() ? std::string(mfbc_status_string(s)) : R.err);
    batches = nbatches;
  }
  if (P.path == MFBC_PATH_LEVEL && g.n) {
    // masks start clean; each batch returns them to zero
    MFBC_CUDA_TRY(cudaMemsetAsync(ls.V, 0, sizeof(uint32_t) * (size_t)g.n * ls.W, R.st), &R.err);
    MFBC_CUDA_TRY(cudaMemsetAsync(ls.F, 0, sizeof(uint32_t) * (size_t)ls.Lcap * g.n * ls.W, R.st), &R.err);
    MFBC_CUDA_TRY(cudaMemsetAsync(ls.member, 0, sizeof(uint32_t) * (size_t)ls.Lcap * ls.mw, R.st), &R.err);
    if (g.items_out.nhub)
      MFBC_CUDA_TRY(cudaMemsetAsync(ls.zacc, 0, sizeof(double) * (size_t)g.items_out.nhub * nb, R.st), &R.err);
  }
  if (mode == 0 && P.path == MFBC_PATH_LEVEL && nsrc > nb && !(R.opt && (R.opt->flags & MFBC_OPT_KEEP_ORDER))) {
    bool applied = false;
    mfbc_status so = order_sources(rc, ls, d_src, nsrc, d_sorted, &applied);
    if (so) return fail(so, R.err.empty() ? std::string(mfbc_status_string(so)) : R.err);
    if (applied) d_src = d_sorted;
  }
  for (int64_t bx = 0; bx < (P.path == MFBC_PATH_SMALL ? 0 : nbatches); bx++) {
    const int32_t b0 = multi ? 0 : (int32_t)(bx * nb);
    int na;
    const int32_t* bsrc;
    const int32_t* bwreq = nullptr;
    if (multi) {
      MFBC_CUDA_TRY(cudaMemcpyAsync(d_colidx, &pk.colidx[(size_t)bx * nb], sizeof(int32_t) * nb,
                                    cudaMemcpyHostToDevice, R.st), &R.err);
      k_gather_sources<<<(nb + 255) / 256, 256, 0, R.st>>>(d_src, d_colidx, nb, d_batch);
      bsrc = d_batch;
      na = pk.used[(size_t)bx];
      bwreq = &pk.wreq[(size_t)bx * (nb / 32)];
    } else {
      bsrc = d_src + b0;
      na = std::min(nb, nsrc - b0);
    }
    rc.word_req = bwreq;
    batches++;
    mfbc_status s;
    bool fallback = false;
    if (P.path == MFBC_PATH_LEVEL) {
      int levels = -1;
      bool exceeded = false;
      s = level_batch(rc, ls, bsrc, na, want_lambda ? d_lambda : nullptr, want_lambda, &levels, &exceeded,
                      &fi, &bi);
      if (s == MFBC_OK) {
        if (mode == 1) {
          int32_t* dd = out_on_host ? stage_d : dist_out + (size_t)b0 * g.n;
          double* ds = sigma_out ? (out_on_host ? stage_s : sigma_out + (size_t)b0 * g.n) : nullptr;
          level_output(rc, ls, levels, na, dd, ds);
          // exactness check reads the staged per-source rows
          if (ds) check_sigma_exact(ds, (size_t)na * g.n, ls.ctr, R.st);
        }
        level_reset(rc, ls, levels);
      } else if (exceeded) {
        fallback = true;
      }
    }
    if (P.path == MFBC_PATH_DIST) {
      s = dist_batch(rc, ds, bsrc, na, want_lambda ? d_lambda : nullptr, &fi, &bi);
      if (s == MFBC_OK && mode == 1) {
        int32_t* dd = out_on_host ? stage_d : dist_out + (size_t)b0 * g.n;
        double* dsg = sigma_out ? (out_on_host ? stage_s : sigma_out + (size_t)b0 * g.n) : nullptr;
        dist_output(rc, ds, na, dd, dsg);
      }
      if (s == MFBC_OK) {
        MFBC_CUDA_TRY(cudaMemcpyAsync(G->h_ctr, &ds.ctr->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, R.st),
                      &R.err);
        MFBC_CUDA_TRY(cudaStreamSynchronize(R.st), &R.err);
        if (G->h_ctr[0] & FLAG_SIGMA_INEXACT) warn |= MFBC_WARN_SIGMA_INEXACT;
      }
    }
    if (P.path == MFBC_PATH_GENERAL || fallback) {
      // general kernels; when falling back from the level path, run this batch
      // in sub-batches that fit the scratch already held
      GeneralState* gp = &gs;
      GeneralState fb;
      int nbg = nb;
      if (fallback) {
        Carver c2(R.ws, P.state_bytes);
        nbg = nb;
        while (nbg > 32 && general_bytes(g.n, nbg) > P.state_bytes) nbg -= 32;
        if (general_bytes(g.n, nbg) > P.state_bytes)
          return fail(MFBC_ERR_OOM, "level capacity exceeded and the general path does not fit the scratch");
        general_carve(c2, g.n, nbg, fb);
        gp = &fb;
        // the level state is overwritten: start its masks again afterwards
        MFBC_CUDA_TRY(cudaMemsetAsync(fb.ctr, 0, sizeof(Counters), R.st), &R.err);
      }
      for (int sb = 0; sb < na; sb += nbg) {
        const int nsa = std::min(nbg, na - sb);
        rc.word_req = bwreq ? bwreq + sb / 32 : nullptr;
        s = general_batch(rc, *gp, bsrc + sb, nsa, want_lambda ? d_lambda : nullptr, &fi, &bi);
        if (s) break;
        if (mode == 1) {
          int32_t* dd = out_on_host ? stage_d + (size_t)sb * g.n : dist_out + (size_t)(b0 + sb) * g.n;
          double* ds = sigma_out ? (out_on_host ? stage_s + (size_t)sb * g.n : sigma_out + (size_t)(b0 + sb) * g.n)
                                 : nullptr;
          general_output(rc, *gp, nsa, dd, ds);
        }
        MFBC_CUDA_TRY(cudaMemcpyAsync(G->h_ctr, &gp->ctr->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, R.st), &R.err);
        MFBC_CUDA_TRY(cudaStreamSynchronize(R.st), &R.err);
        if (G->h_ctr[0] & FLAG_SIGMA_INEXACT) warn |= MFBC_WARN_SIGMA_INEXACT;
      }
      if (fallback && s == MFBC_OK) {
        // restore the level masks for the next batch
        Carver c3(R.ws, R.ws_bytes);
        level_carve(c3, g, nb, P.Lcap, P.list_cap, ls);
        MFBC_CUDA_TRY(cudaMemsetAsync(ls.V, 0, sizeof(uint32_t) * (size_t)g.n * ls.W, R.st), &R.err);
        MFBC_CUDA_TRY(cudaMemsetAsync(ls.F, 0, sizeof(uint32_t) * (size_t)ls.Lcap * g.n * ls.W, R.st), &R.err);
        MFBC_CUDA_TRY(cudaMemsetAsync(ls.member, 0, sizeof(uint32_t) * (size_t)ls.Lcap * ls.mw, R.st), &R.err);
        if (g.items_out.nhub)
          MFBC_CUDA_TRY(cudaMemsetAsync(ls.zacc, 0, sizeof(double) * (size_t)g.items_out.nhub * nb, R.st), &R.err);
        MFBC_CUDA_TRY(cudaMemsetAsync(ls.ctr, 0, sizeof(Counters), R.st), &R.err);
      }
    }
    if (s) return fail(s, R.err.empty() ? std::string(mfbc_status_string(s)) : R.err);
    if (mode == 1 && out_on_host) {
      MFBC_CUDA_TRY(cudaMemcpyAsync(dist_out + (size_t)b0 * g.n, stage_d, sizeof(int32_t) * (size_t)na * g.n,
                                    cudaMemcpyDeviceToHost, R.st), &R.err);
      if (sigma_out)
        MFBC_CUDA_TRY(cudaMemcpyAsync(sigma_out + (size_t)b0 * g.n, stage_s, sizeof(double) * (size_t)na * g.n,
                                      cudaMemcpyDeviceToHost, R.st), &R.err);
    }
  }
  if (P.path != MFBC_PATH_SMALL) {            // the small path read its flags already
    MFBC_CUDA_TRY(cudaMemcpyAsync(G->h_ctr, &ctr->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, R.st), &R.err);
    MFBC_CUDA_TRY(cudaStreamSynchronize(R.st), &R.err);
    if (G->h_ctr[0] & FLAG_SIGMA_INEXACT) warn |= MFBC_WARN_SIGMA_INEXACT;
  }
  MFBC_CUDA_TRY(cudaGetLastError(), &R.err);
  if (R.opt && R.opt->warn_out) *R.opt->warn_out = warn;
  if (R.opt && R.opt->profile) finish_profile(R, R.opt->profile, batches, fi, bi, ctr);
  return MFBC_OK;
}

// The level gathers read scattered 32-byte sectors; with the context's
// default L2 fetch granularity (64 bytes) a miss also brings in the
// neighbouring sector, which is mostly not needed (measured: 5 % slower on
// R-MAT 22).  A call sets the hint to 32 bytes while it runs and restores the
// previous value when it returns (its work is complete by then).
struct L2FetchHint {
  size_t prev = 0;
  bool set = false;
  L2FetchHint() {
    if (cudaDeviceGetLimit(&prev, cudaLimitMaxL2FetchGranularity) == cudaSuccess && prev != 32 &&
        cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, 32) == cudaSuccess)
      set = true;
    else
      cudaGetLastError();
  }
  ~L2FetchHint() {
    if (set && cudaDeviceSetLimit(cudaLimitMaxL2FetchGranularity, prev) != cudaSuccess) cudaGetLastError();
  }
};

mfbc_status entry(const mfbc_graph* Gc, const int32_t* sources, int32_t nsrc, int mode, double* lambda_out,
                  int32_t* dist_out, double* sigma_out, const mfbc_options* opt, bool host_io,
                  const int32_t* req_off = nullptr, int32_t nreq = 0) {
  if (!Gc) return fail(MFBC_ERR_INVALID, "graph must not be NULL");
  if (nsrc < 0) return fail(MFBC_ERR_INVALID, "nsrc must be >= 0");
  if (nsrc > 0 && !sources) return fail(MFBC_ERR_INVALID, "sources must not be NULL");
  if (mode != 1 && Gc->g.n > 0 && !lambda_out) return fail(MFBC_ERR_INVALID, "lambda_out must not be NULL");
  if (mode == 2) {
    if (nreq < 1 || !req_off) return fail(MFBC_ERR_INVALID, "need nreq >= 1 and req_offsets");
    if (req_off[0] != 0 || req_off[nreq] != nsrc)
      return fail(MFBC_ERR_INVALID, "req_offsets must start at 0 and end at nsrc");
    for (int32_t r = 0; r < nreq; r++)
      if (req_off[r + 1] < req_off[r]) return fail(MFBC_ERR_INVALID, "req_offsets must be non-decreasing");
    if (opt && opt->lambda_rows)
      for (int32_t r = 0; r < nreq; r++)
        if (opt->lambda_rows[r] < 0) return fail(MFBC_ERR_INVALID, "lambda_rows must be >= 0");
  }
  if (mode == 1 && nsrc > 0 && Gc->g.n > 0 && !dist_out) return fail(MFBC_ERR_INVALID, "dist_out must not be NULL");
  mfbc_graph* G = const_cast<mfbc_graph*>(Gc);
  std::lock_guard<std::mutex> lock(G->mu);
  const int32_t n = G->g.n;
  if (host_io && nsrc > 0) {
    for (int32_t i = 0; i < nsrc; i++)
      if (sources[i] < 0 || sources[i] >= n) return fail(MFBC_ERR_INVALID, "source id out of range");
  }
  if (opt && (opt->accumulator < MFBC_ACCUM_AUTO || opt->accumulator > MFBC_ACCUM_HASH))
    return fail(MFBC_ERR_INVALID, "unknown accumulator");
  if (opt && opt->warn_out) *opt->warn_out = 0;
  t_err.clear();
  Run R;
  R.G = G;
  R.opt = opt;
  R.req_off = req_off;
  R.nreq = nreq;
  R.st = opt ? (cudaStream_t)opt->stream : nullptr;
  int32_t plan_cols = nsrc;                  // mode 2: each request rounded up to 32 columns
  if (mode == 2) {
    int64_t cols = 0;
    for (int32_t r = 0; r < nreq; r++) cols += (req_off[r + 1] - req_off[r] + 31) / 32 * 32;
    plan_cols = (int32_t)std::min<int64_t>(cols, 0x7fffffff);
  }
  mfbc_status s = make_plan(G, plan_cols, mode, opt, host_io, &R.plan);
  if (s) return s;
  s = get_workspace(R);
  if (s) return s;
  // only the level kernels' gathers gain from the 32-byte fetch hint; setting
  // and restoring it costs two driver calls that small calls would feel
  std::optional<L2FetchHint> l2hint;
  if (R.plan.path == MFBC_PATH_LEVEL) l2hint.emplace();
  R.prof.on = opt && opt->profile;
  R.prof.count_bytes = R.prof.on && (opt->flags & MFBC_OPT_COUNT_BYTES);
  R.prof.stream = R.st;
  char* extra = R.ws + R.plan.state_bytes;
  double* d_lambda = lambda_out;
  const int32_t* d_src = sources;
  if (mode == 0 && host_io) { d_lambda = (double*)extra; extra += al256(sizeof(double) * (size_t)std::max(n, 1)); }
  else if (mode == 0) extra += al256(sizeof(double) * (size_t)std::max(n, 1));
  if (mode == 0 && host_io && n > 0 && opt && (opt->flags & MFBC_OPT_ACCUMULATE)) {
    cudaError_t e = cudaMemcpyAsync(d_lambda, lambda_out, sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, R.st);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(MFBC_ERR_CUDA, "copying lambda failed"); }
  }
  if (host_io) {
    int32_t* ds = (int32_t*)extra;
    extra += al256(sizeof(int32_t) * (size_t)std::max(nsrc, 1));
    if (nsrc) {
      cudaError_t e = cudaMemcpyAsync(ds, sources, sizeof(int32_t) * (size_t)nsrc, cudaMemcpyHostToDevice, R.st);
      if (e != cudaSuccess) { cudaGetLastError(); return fail(MFBC_ERR_CUDA, "copying sources failed"); }
    }
    d_src = ds;
  } else if (nsrc > 0 && R.plan.path != MFBC_PATH_SMALL) {
    // device sources: validate the range on the host copy (the persistent
    // small-graph path checks them on the device, without a round trip)
    std::vector<int32_t> hs((size_t)nsrc);
    if (cudaMemcpyAsync(hs.data(), sources, sizeof(int32_t) * (size_t)nsrc, cudaMemcpyDeviceToHost, R.st) != cudaSuccess ||
        cudaStreamSynchronize(R.st) != cudaSuccess) {
      cudaGetLastError();
      return fail(MFBC_ERR_CUDA, "reading device sources failed");
    }
    for (int32_t v : hs) if (v < 0 || v >= n) return fail(MFBC_ERR_INVALID, "source id out of range");
  }
  int32_t* d_sorted = nullptr;
  if (mode == 0) { d_sorted = (int32_t*)extra; extra += al256(sizeof(int32_t) * (size_t)std::max(nsrc, 1)); }
  s = run(G, d_src, nsrc, mode, d_lambda, dist_out, sigma_out, host_io, R, extra, d_sorted);
  if (s == MFBC_OK && mode == 0 && host_io && n > 0) {
    cudaError_t e = cudaMemcpyAsync(lambda_out, d_lambda, sizeof(double) * (size_t)n, cudaMemcpyDeviceToHost, R.st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(R.st);
    if (e != cudaSuccess) { cudaGetLastError(); s = fail(MFBC_ERR_CUDA, std::string("copying lambda failed: ") + cudaGetErrorString(e)); }
  }
  R.prof.release();
  if (s == MFBC_OK) t_err.clear();
  else {
    if (!R.err.empty() && t_err.empty()) t_err = R.err;
    cudaGetLastError();
  }
  return s;
}

}  // namespace

extern "C" mfbc_status mfbc_bc(const mfbc_graph* g, const int32_t* sources, int32_t nsrc, double* lambda_out,
                               const mfbc_options* opt) {
  return entry(g, sources, nsrc, 0, lambda_out, nullptr, nullptr, opt, true);
}

extern "C" mfbc_status mfbc_bc_device(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                                      double* lambda_out, const mfbc_options* opt) {
  return entry(g, sources, nsrc, 0, lambda_out, nullptr, nullptr, opt, false);
}

extern "C" mfbc_status mfbc_bc_multi_device(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                                            const int32_t* req_offsets, int32_t nreq, double* lambda_out,
                                            const mfbc_options* opt) {
  return entry(g, sources, nsrc, 2, lambda_out, nullptr, nullptr, opt, false, req_offsets, nreq);
}

extern "C" mfbc_status mfbc_autotune(mfbc_graph* G, const int32_t* sources, int32_t nsrc, const mfbc_options* opt,
                                     mfbc_tuning* out) {
  if (!G || !out) return fail(MFBC_ERR_INVALID, "graph and out must not be NULL");
  if (nsrc < 1 || !sources) return fail(MFBC_ERR_INVALID, "need at least one source");
  const int req_path = opt ? opt->path : MFBC_PATH_AUTO;
  const bool dist_ok = G->g.wmax + 1 <= DIST_MAX_BUCKETS;
  std::vector<int> paths;
  if (req_path == MFBC_PATH_AUTO) {
    if (G->g.unit) paths = small_tunable(G->g) ? std::vector<int>{MFBC_PATH_LEVEL, MFBC_PATH_SMALL}
                                             : std::vector<int>{MFBC_PATH_LEVEL};
    else paths = dist_ok ? std::vector<int>{MFBC_PATH_GENERAL, MFBC_PATH_DIST} : std::vector<int>{MFBC_PATH_GENERAL};
  } else if (req_path == MFBC_PATH_LEVEL) {
    if (!G->g.unit) return fail(MFBC_ERR_INVALID, "MFBC_PATH_LEVEL needs unit weights");
    paths = {MFBC_PATH_LEVEL};
  } else if (req_path == MFBC_PATH_GENERAL) {
    paths = {MFBC_PATH_GENERAL};
  } else if (req_path == MFBC_PATH_DIST) {
    if (!dist_ok) return fail(MFBC_ERR_INVALID, "MFBC_PATH_DIST needs weights <= 4096");
    paths = {MFBC_PATH_DIST};
  } else if (req_path == MFBC_PATH_SMALL) {
    if (!G->g.unit) return fail(MFBC_ERR_INVALID, "MFBC_PATH_SMALL needs unit weights");
    paths = {MFBC_PATH_SMALL};
  } else {
    return fail(MFBC_ERR_INVALID, "unknown path");
  }
  std::vector<double> lam((size_t)std::max(G->g.n, 1));
  mfbc_options o = opt ? *opt : mfbc_options{};
  o.profile = nullptr;
  o.warn_out = nullptr;
  double best = 0.0;
  int best_nb = 0, best_arcs = 0, best_path = 0, best_accum = 0, tried = 0;
  bool best_widest = false;
  for (int path : paths) {
    const bool level = path == MFBC_PATH_LEVEL;
    std::vector<int> widths = level ? std::vector<int>{128, 256, 512, 1024}
                              : path == MFBC_PATH_SMALL ? std::vector<int>{32, 64, 128, 256}
                                                        : std::vector<int>{128, 256, 512, 1024, 2048, 4096};
    const int gran = level ? 128 : 32;
    const int cols = (nsrc + gran - 1) / gran * gran;
    while (widths.size() > 1 && widths.back() > cols) widths.pop_back();
    // general kernels: atomic products walking 1 or 8 arcs per step, the
    // segmented products, the hash-combined products, and the per-product
    // choice between atomic and segmented
    struct Var { int arcs, accum; };
    const std::vector<Var> vars = path == MFBC_PATH_GENERAL
        ? std::vector<Var>{{1, MFBC_ACCUM_ATOMIC}, {8, MFBC_ACCUM_ATOMIC}, {0, MFBC_ACCUM_SEGMENTED},
                           {0, MFBC_ACCUM_HASH}, {0, MFBC_ACCUM_AUTO}}
        : std::vector<Var>{{0, MFBC_ACCUM_AUTO}};
    o.path = path;
    for (int nb : widths)
      for (const Var& var : vars) {
        const int a = var.arcs;
        o.n_b = nb;
        o.accumulator = var.accum;
        {
          std::lock_guard<std::mutex> lock(G->mu);
          G->force_arcs = a;
        }
        // one untimed call (scratch growth, first touch), then the timed one
        mfbc_status s = entry(G, sources, nsrc, 0, lam.data(), nullptr, nullptr, &o, true);
        const auto t0 = std::chrono::steady_clock::now();
        if (s == MFBC_OK) s = entry(G, sources, nsrc, 0, lam.data(), nullptr, nullptr, &o, true);
        const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        if (s == MFBC_ERR_OOM) continue;           // too wide for this device: not a candidate
        if (s != MFBC_OK) {
          std::lock_guard<std::mutex> lock(G->mu);
          G->force_arcs = 0;
          return s;
        }
        tried++;
        if (best_nb == 0 || ms < best) {
          best = ms; best_nb = nb; best_arcs = a; best_path = path; best_accum = var.accum;
          best_widest = nb == widths.back();
        }
      }
  }
  std::lock_guard<std::mutex> lock(G->mu);
  G->force_arcs = 0;
  if (!best_nb) return fail(MFBC_ERR_OOM, "no candidate batch width fits the device");
  // a width is kept as a cap only when a wider one was tried and lost
  G->tuned_nb[tuned_slot(best_path)] = best_widest ? 0 : best_nb;
  if (best_path == MFBC_PATH_GENERAL) {
    G->tuned_arcs = best_arcs;
    G->tuned_accum = best_accum;
  }
  if (req_path == MFBC_PATH_AUTO) G->tuned_path = best_path;
  out->n_b = best_nb;
  out->path = best_path;
  out->arcs = best_arcs;
  out->tried = tried;
  out->ms_per_source = best / nsrc;
  out->accumulator = best_path == MFBC_PATH_GENERAL ? best_accum : 0;
  t_err.clear();
  return MFBC_OK;
}

extern "C" mfbc_status mfbc_sssp_batch(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                                       int32_t* dist_out, double* sigma_out, const mfbc_options* opt) {
  return entry(g, sources, nsrc, 1, nullptr, dist_out, sigma_out, opt, true);
}

extern "C" mfbc_status mfbc_sssp_batch_device(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                                              int32_t* dist_out, double* sigma_out, const mfbc_options* opt) {
  return entry(g, sources, nsrc, 1, nullptr, dist_out, sigma_out, opt, false);
}

// Accessors for entry points defined in other translation units.
namespace mfbc {
const DevGraph* graph_device_view(const mfbc_graph* G) { return G ? &G->g : nullptr; }
uint32_t* graph_counter_mirror(const mfbc_graph* G) { return G ? G->h_ctr : nullptr; }
void graph_lock(const mfbc_graph* G) { const_cast<mfbc_graph*>(G)->mu.lock(); }
void graph_unlock(const mfbc_graph* G) { const_cast<mfbc_graph*>(G)->mu.unlock(); }
void set_last_error(const std::string& msg) { t_err = msg; }
}  // namespace mfbc
