// Graph construction: upload of the CSR adjacency (Sec. 2.1; the paper's
// bulk Tensor::write of the input, Sec. 6.1), validation on the device, the
// transposed adjacency A^T that Algorithm 2's products use, and the work-item
// lists of the level kernels.
//
// Validation (a graph that fails any check is rejected with INVALID):
//   rowptr[0] == 0, non-decreasing, rowptr[n] == nnz;
//   0 <= col < n, strictly increasing within a row (no duplicate arcs),
//   no self-loops, weights >= 1;
//   UNDIRECTED: every arc v->u has a reverse arc u->v of equal weight.
// Distances are int32, so (n-1)*max_w + max_w must stay below INT32_MAX
// (OVERFLOW otherwise): every finite distance and every candidate tau + w of
// the MFBF product then fits.
#include <algorithm>
#include <cstring>

#include "internal.cuh"

namespace mfbc {

struct ValFlags {
  unsigned int bad_rowptr, bad_col, unsorted, self_loop, bad_weight, asym, non_unit;
  int wmax;
};

__global__ void k_check_rowptr(int32_t n, int64_t nnz, const int64_t* __restrict__ rowptr, ValFlags* f) {
  int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v > n) return;
  int64_t r = rowptr[v];
  bool bad = (r < 0 || r > nnz) || (v == 0 && r != 0) || (v == n && r != nnz) ||
             (v < n && rowptr[v + 1] < r);
  if (bad) atomicOr(&f->bad_rowptr, 1u);
}

// One warp per row.
__global__ void k_check_arcs(int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const int32_t* __restrict__ w, bool undirected, ValFlags* f) {
  uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  int wmax = 1;
  unsigned bc = 0, uns = 0, sl = 0, bw = 0, asy = 0, nu = 0;
  for (; gw < (uint64_t)n; gw += nw) {
    const int32_t v = (int32_t)gw;
    const int64_t beg = rowptr[v], end = rowptr[v + 1];
    for (int64_t k = beg + lane; k < end; k += 32) {
      const int32_t c = col[k];
      if (c < 0 || c >= n) { bc = 1; continue; }
      if (c == v) sl = 1;
      if (k > beg && col[k - 1] >= c) uns = 1;
      int32_t wk = 1;
      if (w) {
        wk = w[k];
        if (wk < 1) { bw = 1; continue; }
        if (wk != 1) nu = 1;
        wmax = max(wmax, wk);
      }
      if (undirected) {
        // binary search for v in row c (rows are sorted when valid; an
        // unsorted row just makes the search miss, and is flagged above)
        int64_t lo = rowptr[c], hi = rowptr[c + 1];
        bool found = false;
        while (lo < hi) {
          int64_t mid = (lo + hi) >> 1;
          int32_t x = col[mid];
          if (x == v) { found = (w ? w[mid] == wk : true); break; }
          if (x < v) lo = mid + 1; else hi = mid;
        }
        if (!found) asy = 1;
      }
    }
  }
  if (bc) atomicOr(&f->bad_col, 1u);
  if (uns) atomicOr(&f->unsorted, 1u);
  if (sl) atomicOr(&f->self_loop, 1u);
  if (bw) atomicOr(&f->bad_weight, 1u);
  if (asy) atomicOr(&f->asym, 1u);
  if (nu) atomicOr(&f->non_unit, 1u);
  if (w) atomicMax(&f->wmax, wmax);
}

template <class T>
static mfbc_status dev_alloc(DevGraph* g, T** p, size_t count, std::string* err) {
  *p = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
  if (e != cudaSuccess) {
    if (err) *err = std::string("cudaMalloc(graph): ") + cudaGetErrorString(e);
    cudaGetLastError();
    return MFBC_ERR_OOM;
  }
  g->owned.push_back((void*)*p);
  return MFBC_OK;
}

#define TRY(x)                  \
  do {                          \
    mfbc_status _s = (x);       \
    if (_s != MFBC_OK) return _s; \
  } while (0)

// empty_rows: give every row without arcs one empty item.  The MFBr gather
// must visit DAG sinks too (their frontier value 1/sigma_bar is written by
// that visit); in an undirected graph a vertex without arcs can only be a
// source, so only directed graphs need it.
static mfbc_status build_items(DevGraph* g, const std::vector<int64_t>& rp, ItemList* L, bool empty_rows,
                               cudaStream_t st, std::string* err) {
  const int32_t n = g->n;
  if (rp[n] >= (1ll << 40)) { *err = "graphs with 2^40 or more arcs are not supported"; return MFBC_ERR_INVALID; }
  std::vector<int32_t> iv;
  std::vector<int64_t> ib;
  std::vector<int32_t> hub_of((size_t)n, -1), hubs;
  for (int32_t v = 0; v < n; v++) {
    const int64_t deg = rp[v + 1] - rp[v];
    if (deg > CHUNK) { hub_of[v] = (int32_t)hubs.size(); hubs.push_back(v); }
    // item metadata: first arc (bits 0..39), arc count (40..45), multi-item row (46)
    const int64_t multi = deg > CHUNK ? (1ll << 46) : 0;
    for (int64_t b = rp[v]; b < rp[v + 1]; b += CHUNK) {
      iv.push_back(v);
      ib.push_back(b | (std::min<int64_t>(CHUNK, rp[v + 1] - b) << 40) | multi);
    }
    if (deg == 0 && empty_rows) { iv.push_back(v); ib.push_back(rp[v]); }
  }
  L->count = (int64_t)iv.size();
  L->nhub = (int32_t)hubs.size();
  TRY(dev_alloc(g, &L->v, iv.size(), err));
  TRY(dev_alloc(g, &L->beg, ib.size(), err));
  TRY(dev_alloc(g, &L->hub_of, (size_t)n, err));
  TRY(dev_alloc(g, &L->hubs, hubs.size(), err));
  MFBC_CUDA_TRY(cudaMemcpyAsync(L->v, iv.data(), sizeof(int32_t) * iv.size(), cudaMemcpyHostToDevice, st), err);
  MFBC_CUDA_TRY(cudaMemcpyAsync(L->beg, ib.data(), sizeof(int64_t) * ib.size(), cudaMemcpyHostToDevice, st), err);
  MFBC_CUDA_TRY(cudaMemcpyAsync(L->hub_of, hub_of.data(), sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, st), err);
  if (!hubs.empty())
    MFBC_CUDA_TRY(cudaMemcpyAsync(L->hubs, hubs.data(), sizeof(int32_t) * hubs.size(), cudaMemcpyHostToDevice, st), err);
  // the host vectors die at return: finish the copies first
  MFBC_CUDA_TRY(cudaStreamSynchronize(st), err);
  return MFBC_OK;
}

// Targets where the push products' candidates meet often enough for the
// hash accumulator to combine them in shared memory: vertices whose row in
// rp (in-arcs for MFBF targets, out-arcs for MFBr targets) holds at least
// max(16, 2 x the average degree) arcs.  One bit per vertex.
static mfbc_status upload_hot_targets(DevGraph* g, const std::vector<int64_t>& rp, uint32_t** out, cudaStream_t st,
                                      std::string* err) {
  const int32_t n = g->n;
  const int64_t avg2 = n ? 2 * g->nnz / n : 0;
  const int64_t thr = std::max<int64_t>(16, avg2);
  std::vector<uint32_t> bits(((size_t)n + 31) / 32 + 1, 0u);
  for (int32_t v = 0; v < n; v++)
    if (rp[(size_t)v + 1] - rp[v] >= thr) bits[(size_t)v >> 5] |= 1u << (v & 31);
  TRY(dev_alloc(g, out, bits.size(), err));
  MFBC_CUDA_TRY(cudaMemcpyAsync(*out, bits.data(), sizeof(uint32_t) * bits.size(), cudaMemcpyHostToDevice, st), err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(st), err);
  return MFBC_OK;
}

mfbc_status graph_build(int32_t n, int64_t nnz, const int64_t* h_rowptr, const int32_t* h_col,
                        const int32_t* h_w, uint32_t flags, cudaStream_t st, DevGraph* g,
                        std::string* err) {
  g->n = n;
  g->nnz = nnz;
  g->directed = !(flags & MFBC_UNDIRECTED);
  TRY(dev_alloc(g, &g->rowptr, (size_t)n + 1, err));
  TRY(dev_alloc(g, &g->col, (size_t)nnz, err));
  if (h_w) TRY(dev_alloc(g, &g->w, (size_t)nnz, err));
  ValFlags* d_f;
  TRY(dev_alloc(g, &d_f, 1, err));
  MFBC_CUDA_TRY(cudaMemcpyAsync(g->rowptr, h_rowptr, sizeof(int64_t) * ((size_t)n + 1), cudaMemcpyHostToDevice, st), err);
  if (nnz) MFBC_CUDA_TRY(cudaMemcpyAsync(g->col, h_col, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, st), err);
  if (h_w && nnz) MFBC_CUDA_TRY(cudaMemcpyAsync(g->w, h_w, sizeof(int32_t) * (size_t)nnz, cudaMemcpyHostToDevice, st), err);
  MFBC_CUDA_TRY(cudaMemsetAsync(d_f, 0, sizeof(ValFlags), st), err);
  k_check_rowptr<<<(unsigned)((n + 1 + 255) / 256), 256, 0, st>>>(n, nnz, g->rowptr, d_f);
  ValFlags f;
  MFBC_CUDA_TRY(cudaMemcpyAsync(&f, d_f, sizeof(f), cudaMemcpyDeviceToHost, st), err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(st), err);
  if (f.bad_rowptr) { *err = "rowptr must start at 0, be non-decreasing and end at nnz"; return MFBC_ERR_INVALID; }
  if (n) {
    unsigned blocks = (unsigned)std::min<int64_t>(((int64_t)n + 7) / 8, 152 * 32);
    k_check_arcs<<<blocks, 256, 0, st>>>(n, g->rowptr, g->col, g->w, !g->directed, d_f);
  }
  // While the GPU checks the arcs, the host prepares what depends on the
  // (already checked) row pointers alone; the result is read further down.
  // host copy of the row pointers for the work-item lists
  std::vector<int64_t> rp(h_rowptr, h_rowptr + (size_t)n + 1);
  std::vector<uint32_t> hot(((size_t)n + 31) / 32 + 1, 0u);
  {
    // landmarks for source ordering: the highest out-degree vertices
    // (degree descending, then id), isolated vertices excluded
    std::vector<int32_t> ids;
    ids.reserve((size_t)n);
    for (int32_t v = 0; v < n; v++) {
      if (rp[v + 1] > rp[v]) ids.push_back(v);
      g->max_deg = std::max<int64_t>(g->max_deg, rp[v + 1] - rp[v]);
    }
    // the HOT_ROWS highest degrees also mark the rows the level gathers ask
    // the L2 to keep (their values are read along most DAG arcs)
    const size_t k = std::min<size_t>(ids.size(), (size_t)std::max(ORDER_LANDMARKS, HOT_ROWS));
    auto higher = [&](int32_t a, int32_t b) {
      const int64_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
      return da != db ? da > db : a < b;
    };
    std::nth_element(ids.begin(), ids.begin() + k, ids.end(), higher);
    std::sort(ids.begin(), ids.begin() + k, higher);
    g->landmarks.assign(ids.begin(), ids.begin() + std::min<size_t>(k, (size_t)ORDER_LANDMARKS));
    for (size_t i = 0; i < std::min<size_t>(k, (size_t)HOT_ROWS); i++) hot[(size_t)ids[i] >> 5] |= 1u << (ids[i] & 31);
    TRY(dev_alloc(g, &g->hot, hot.size(), err));
    MFBC_CUDA_TRY(cudaMemcpyAsync(g->hot, hot.data(), sizeof(uint32_t) * hot.size(), cudaMemcpyHostToDevice, st), err);
  }
  if (!g->directed) {
    g->max_in_deg = g->max_deg;
    TRY(build_items(g, rp, &g->items_in, false, st, err));      // (waits for the stream)
    g->items_out = g->items_in;
    TRY(upload_hot_targets(g, rp, &g->hot_in, st, err));
    g->hot_out = g->hot_in;
  }
  MFBC_CUDA_TRY(cudaMemcpyAsync(&f, d_f, sizeof(f), cudaMemcpyDeviceToHost, st), err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(st), err);
  MFBC_CUDA_TRY(cudaGetLastError(), err);
  if (f.bad_col) { *err = "column index out of range [0, n)"; return MFBC_ERR_INVALID; }
  if (f.self_loop) { *err = "self-loops are not allowed"; return MFBC_ERR_INVALID; }
  if (f.unsorted) { *err = "rows must be sorted by column without duplicate arcs"; return MFBC_ERR_INVALID; }
  if (f.bad_weight) { *err = "weights must be integers >= 1"; return MFBC_ERR_INVALID; }
  if (f.asym) { *err = "UNDIRECTED graph is not symmetric with symmetric weights"; return MFBC_ERR_INVALID; }
  g->wmax = h_w ? std::max(1, f.wmax) : 1;
  if ((int64_t)n * (int64_t)g->wmax >= (int64_t)INF) {
    *err = "(n-1)*max_w + max_w must be below 2^31-1 for int32 distances";
    return MFBC_ERR_OVERFLOW;
  }
  g->unit = !f.non_unit;
  if (g->unit && g->w) { g->w = nullptr; }   // all ones: treat as unweighted (array still owned)
  if (g->directed) {
    // A^T by a stable counting sort on the host: rows of A^T are sorted by
    // source vertex, so the transposed graph is deterministic.
    std::vector<int64_t> rpt((size_t)n + 1, 0);
    for (int64_t k = 0; k < nnz; k++) rpt[(size_t)h_col[k] + 1]++;
    for (int32_t v = 0; v < n; v++) {
      g->max_in_deg = std::max<int64_t>(g->max_in_deg, rpt[v + 1]);
      rpt[v + 1] += rpt[v];
    }
    std::vector<int32_t> ct((size_t)nnz), wtv(g->w ? (size_t)nnz : 0);
    std::vector<int64_t> pos(rpt.begin(), rpt.end() - 1);
    for (int32_t v = 0; v < n; v++)
      for (int64_t k = rp[v]; k < rp[v + 1]; k++) {
        int64_t p = pos[h_col[k]]++;
        ct[p] = v;
        if (g->w) wtv[p] = h_w[k];
      }
    TRY(dev_alloc(g, &g->rowptr_t, (size_t)n + 1, err));
    TRY(dev_alloc(g, &g->col_t, (size_t)nnz, err));
    if (g->w) TRY(dev_alloc(g, &g->w_t, (size_t)nnz, err));
    MFBC_CUDA_TRY(cudaMemcpyAsync(g->rowptr_t, rpt.data(), sizeof(int64_t) * rpt.size(), cudaMemcpyHostToDevice, st), err);
    if (nnz) MFBC_CUDA_TRY(cudaMemcpyAsync(g->col_t, ct.data(), sizeof(int32_t) * ct.size(), cudaMemcpyHostToDevice, st), err);
    if (g->w && nnz) MFBC_CUDA_TRY(cudaMemcpyAsync(g->w_t, wtv.data(), sizeof(int32_t) * wtv.size(), cudaMemcpyHostToDevice, st), err);
    MFBC_CUDA_TRY(cudaStreamSynchronize(st), err);
    TRY(build_items(g, rpt, &g->items_in, false, st, err));
    TRY(build_items(g, rp, &g->items_out, true, st, err));
    TRY(upload_hot_targets(g, rpt, &g->hot_in, st, err));
    TRY(upload_hot_targets(g, rp, &g->hot_out, st, err));
  } else {
    g->rowptr_t = g->rowptr;
    g->col_t = g->col;
    g->w_t = g->w;
  }
  return MFBC_OK;
}

void graph_free(DevGraph* g) {
  for (void* p : g->owned) cudaFree(p);
  g->owned.clear();
}

}  // namespace mfbc
