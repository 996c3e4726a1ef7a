// Internal declarations of the MFBC CUDA library (sm_103a).
//
// State layout (both kernel families): every per-(source, vertex) array of a
// batch is VERTEX-MAJOR, x[v * nb + j] for vertex v and batch column j, so that
// one warp touching 32 consecutive columns of one vertex reads or writes one
// contiguous 128-byte (int32) or 256-byte (FP64) segment.  Frontier and
// visited sets are bit masks, 32 columns per uint32 word, mask[v * W + j/32]
// with W = nb / 32.  Column j of a batch belongs to source src[j]; src[j] < 0
// marks a padding column (Theorem 1's padding of the last batch).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/mfbc.h"

namespace mfbc {

constexpr int32_t INF = 0x7fffffff;
constexpr int WARP = 32;
constexpr int CHUNK = 32;          // neighbours per work item of the level kernels

// ------------------------------------------------------------------ graph
struct ItemList {                  // work items of <= CHUNK arcs of one row
  int64_t count = 0;
  int32_t* v = nullptr;            // row (vertex) of the item
  int64_t* beg = nullptr;          // first arc | arc count << 40 | multi-item row << 46
  int32_t nhub = 0;                // vertices whose row spans more than one item
  int32_t* hub_of = nullptr;       // [n] hub index or -1
  int32_t* hubs = nullptr;         // [nhub] vertex ids
};

struct DevGraph {
  int32_t n = 0;
  int64_t nnz = 0;
  bool directed = true;
  bool unit = true;                // every arc weighs 1 (w == NULL or all ones)
  int32_t wmax = 1;
  std::vector<int32_t> landmarks;   // highest out-degree vertices, descending (source ordering)
  uint32_t* hot = nullptr;         // [n/32] bits: the HOT_ROWS highest out-degree vertices
  uint32_t* hot_in = nullptr;      // [n/32] bits: in-degree >= max(16, 2 x average) (hash accumulator)
  uint32_t* hot_out = nullptr;     // [n/32] bits: the same for out-degree (aliases hot_in when undirected)
  int64_t max_deg = 0;             // largest out-degree
  int64_t max_in_deg = 0;          // largest in-degree
  int64_t* rowptr = nullptr;       // CSR of A (out-arcs)
  int32_t* col = nullptr;
  int32_t* w = nullptr;            // nullptr when unit
  int64_t* rowptr_t = nullptr;     // CSR of A^T (in-arcs); aliases CSR when undirected
  int32_t* col_t = nullptr;
  int32_t* w_t = nullptr;
  ItemList items_in;               // over A^T rows (MFBF pull gathers in-arcs)
  ItemList items_out;              // over A rows   (MFBr pull gathers out-arcs)
  std::vector<void*> owned;        // device allocations to free
};

// ------------------------------------------------------------- profiling
struct KStat {
  const char* name;
  uint64_t launches = 0;
  double ms = 0.0;
  double bytes = 0.0;
};

enum KId {
  K_FILL = 0, K_SEED, K_RELAX_MIN, K_RELAX_TIE, K_ACCUM, K_COUNTERS, K_PROPAGATE, K_FINAL,
  K_LAMBDA, K_CLEAR, K_LVL_FWD, K_LVL_VISIT, K_LVL_BWD, K_LVL_HUB, K_LVL_RESET, K_OUTPUT,
  K_LVL_FWD_G, K_LVL_BWD_G, K_LVL_SPLIT, K_DP_FWD, K_DP_BWD, K_SMALL, K_PULL_FWD, K_PULL_BWD,
  K_HASH_MIN, K_HASH_TIE, K_HASH_PROP, K_NUM
};

// Bits of Counters::flags, set by kernels and read by the host drivers.
constexpr uint32_t FLAG_LEVEL_LIST = 1u;     // level kernels: a per-level vertex list overflowed
constexpr uint32_t FLAG_SIGMA_INEXACT = 2u;  // some sigma_bar >= 2^53 (FP64 output may be rounded)
constexpr uint32_t FLAG_BAD_SOURCE = 4u;     // mfbc_bc_static: a source id outside [0, n)
constexpr uint32_t FLAG_COUNT_WRAP = 8u;     // level kernels: a path count reached 2^58 (batch redone)
constexpr uint32_t FLAG_TIMEOUT = 16u;       // a bounded device-side wait ran out (MFBC_ERR_TIMEOUT)
constexpr uint32_t FLAG_ROUND_ABORT = 32u;   // level kernels: a round's pair buffers overflowed; the
                                             // launches queued after it return at once until cleared

// Device-side counters of algorithmic bytes, one slot per kernel id.
struct Counters {
  unsigned long long bytes[K_NUM];
  unsigned long long stat[4];      // (counting pass) pairs fwd/bwd, gathered values fwd/bwd
  uint32_t list_count[4];          // frontier / touched list sizes
  uint32_t flags;                  // FLAG_* bits
  uint32_t work[4];                // level kernels: pairs, segments, gather group counter, overflow
  uint32_t abort_level;            // level kernels: highest MFBr level whose round overflowed
  uint32_t visit_count;            // level kernels: vertices of the next level's visit (0 after an overflow)
};

class Profiler {
 public:
  bool on = false;                 // record CUDA events around launches
  bool count_bytes = false;        // kernels add their algorithmic bytes on the device
  cudaStream_t stream = nullptr;
  KStat k[K_NUM];
  Profiler();
  void begin(KId id);              // record start event of a launch of kernel id
  void end(KId id);                // record stop event
  void drain();                    // accumulate finished event pairs (stream synchronised)
  void release();
 private:
  struct Pending { KId id; cudaEvent_t a, b; };
  std::vector<Pending> pend;
  std::vector<cudaEvent_t> pool;
  cudaEvent_t get();
};

// ------------------------------------------------------------- workspaces
struct Carver {
  char* base; size_t off = 0, cap;
  Carver(void* b, size_t c) : base((char*)b), cap(c) {}
  template <class T> T* take(size_t count) {
    size_t bytes = (count * sizeof(T) + 255) & ~size_t(255);
    T* p = (T*)(base ? base + off : nullptr);
    off += bytes;
    return p;
  }
};

// General (any integer weight) path: Algorithms 1 and 2 with the two-phase
// monoid product.  See general.cu.
struct GeneralState {
  int nb = 0, W = 0;
  int32_t* dist;      // T.w            [n][nb]
  double* sig;        // T.m            [n][nb]
  int32_t* cw;        // product weight / MFBr counter Z.c   [n][nb]
  double* cm;         // product mult.  / MFBr factor Z.p    [n][nb]
  double* fm;         // frontier mult. / MFBr frontier value [n][nb]
  uint32_t* fmask;    // frontier bits  [n][W]
  uint32_t* tmask;    // touched bits   [n][W]
  uint32_t* vflag;    // per-vertex enqueue flags [n]
  uint32_t* fmem;     // frontier membership bits, one per vertex [n/32] (pull products)
  int32_t* listA;     // frontier vertex lists [n]
  int32_t* listB;
  int32_t* src;       // [nb]
  int32_t* word_req;  // [W] request of each word (lambda row), see RunCtx
  Counters* ctr;
};
size_t general_bytes(int32_t n, int nb);
void general_carve(Carver& c, int32_t n, int nb, GeneralState& s);

// Level-synchronous path for unit weights: Algorithms 1 and 2 with the
// frontiers kept as per-level bit masks.  See level.cu.
constexpr int LEVEL_MAX_NB = 1024;   // widest batch of the level kernels
constexpr int ORDER_LANDMARKS = 128; // distance profile length used to order sources
constexpr int HOT_ROWS = 4096;       // rows the level gathers load with the L2 evict-last hint
struct LevelState {
  int nb = 0, W = 0, Lcap = 0;
  double* sv;         // sigma_bar, then zeta + 1/sigma_bar (in place)  [n][nb]
  uint32_t* V;        // visited bits [n][W]
  uint32_t* F;        // per-level frontier bits, level l at F + l*n*W
  uint32_t* member;   // per-level vertex bitmaps, level l at member + l*mw
  uint32_t* full;     // vertices visited by every active column  [mw]
  int32_t* lists;     // per-level vertex lists, concatenated
  int64_t list_cap;
  double* zacc;       // [nhub_out][nb] backward partial sums of multi-item vertices
  uint32_t* prow;     // pairs of one product round: row index u*Q + quad
  uint4* pmask;       //   and the pair's 128-column mask
  uint4* segs;        // segment headers of one product round
  uint32_t pair_cap, seg_cap;
  int32_t* src;       // [nb]
  uint32_t* colmask;  // [W] columns of the batch that hold a source
  int32_t* word_req;  // [W] request of each word (lambda row), see RunCtx
  int32_t* quad_req;  // [W/4] request of each quad, -1 none, -2 mixed
  Counters* ctr;
  int64_t mw;         // words per vertex bitmap
};
size_t level_bytes(const DevGraph& g, int nb, int Lcap, int64_t list_cap);
void level_carve(Carver& c, const DevGraph& g, int nb, int Lcap, int64_t list_cap, LevelState& s);

// Distance path for small integer weights: Algorithms 1 and 2 stepped in
// order of distance value.  See dist.cu.
constexpr int DIST_MAX_BUCKETS = 4097;   // w_max + 1 at most
// Step bookkeeping of the distance kernels (one per batch workspace, zeroed
// before a batch): the forward step kernels read the distance value to
// process here, and the last block of each step advances it.
struct DpSync {
  uint32_t done;         // blocks finished with the current step
  int32_t d;             // distance value of the next forward step
  uint32_t off;          // settled-list offset at the start of that step
  uint32_t k;            // steps recorded since the host last read them
  uint32_t stop;         // 1: no bucket holds items
  uint32_t steps;        // forward steps processed (statistics)
};
constexpr int DP_STEP_RECORDS = 32; // >= the forward steps of one round between host reads
constexpr int DP_CSTRIDE = 32;      // uint32 per bucket counter: one 128-byte line each

struct DistState {
  int nb = 0, W = 0, B = 0, BW = 0;
  int32_t* dist;      // tau  [n][nb]
  double* sig;        // sigma_bar [n][nb]
  double* val;        // MFBr value zeta + 1/sigma_bar [n][nb]
  uint32_t* mlist;    // (vertex * W + word) items settled per step, concatenated
  size_t mcap;
  uint32_t* blist;    // [B][bcap] ring of bucket lists of (vertex * W + word) items
  uint32_t* bflag;    // [n * W][BW] bucket membership bits per item
  size_t bcap;        // n * W
  uint32_t* bcount;   // [B + 1] bucket counts, then the settled-list count, DP_CSTRIDE apart
  DpSync* sy;
  int32_t* sd;        // [DP_STEP_RECORDS] distance value of each recorded step
  uint32_t* soff;     // [DP_STEP_RECORDS] its first settled-list entry
  int32_t* src;       // [nb]
  int32_t* word_req;  // [W]
  Counters* ctr;
};
size_t dist_bytes(int32_t n, int nb, int B);
void dist_carve(Carver& c, int32_t n, int nb, int B, DistState& s);

// Persistent path for small unit-weight graphs: whole batches inside one
// cooperative launch, block groups taking batches from a device queue.  See
// small.cu.
struct SmallGroupCtl {  // one per block group, on its own 128-byte line
  uint32_t arrive;      // barrier arrivals of the group's blocks (monotonic)
  uint32_t batch;       // batch the group works on
  uint32_t wrap;        // a path count of the batch reached 2^58
  uint32_t any[3];      // a pair entered level l + 1 during product l (slot l % 3)
  uint32_t pad[26];
};
struct SmallState {
  int nb = 0, W = 0, G = 0;
  uint8_t* lvl;         // [G][n][nb] tau, 255 = unreached
  uint64_t* sv;         // [G][n][nb] sigma_bar, then zeta + 1/sigma_bar (double-float)
  SmallGroupCtl* ctl;   // [G]
  uint32_t* head;       // [0] batch queue head, [1] batches listed in redo
  int32_t* redo;        // batches left to the general kernels (too deep or counts >= 2^58)
  Counters* ctr;
};
size_t small_bytes(int32_t n, int nb, int groups);
void small_carve(Carver& c, int32_t n, int nb, int groups, SmallState& s);
// groups a call launches for nbatch batches (bounded by a quarter of the co-resident blocks)
int small_groups(int32_t n, int nb, int nbatch);

// --------------------------------------------------------------- drivers
struct RunCtx {
  const DevGraph* g;
  cudaStream_t stream;
  Profiler* prof;
  uint32_t* h_ctr;                 // pinned host mirror of Counters::list_count / flags
  std::string* err;
  // Requests packed into the current batch (host array, one entry per
  // 32-column word: the request owning the word's columns, -1 for none).
  // Request r adds into lambda + r * n.  nullptr: the whole batch is
  // request 0.
  const int32_t* word_req = nullptr;
  // general kernels: arcs walked per step (1 or 8); 0 = by average degree
  int arcs = 0;
  // general kernels: how a product reduces its candidates (MFBC_ACCUM_*)
  int accum = 0;
  // level kernels: test hook MFBC_OPT_TEST_SMALL_ROUNDS (small pair buffers)
  bool small_rounds = false;
};

// Request of the batch as a whole: r >= 0 when every used word belongs to
// request r (or word_req is null: 0), -2 when the batch mixes requests.
int batch_uniform_request(const int32_t* word_req, int W);

// One batch of the general path.  lambda != nullptr: full MFBC batch adding
// into lambda; otherwise MFBF only.  Returns MFBC_OK or an error status.
mfbc_status general_batch(RunCtx& rc, GeneralState& s, const int32_t* d_src_batch, int nactive,
                          double* lambda, int64_t* fwd_iters, int64_t* bwd_iters);
// Transposed copy of the general state's dist/sig into per-source rows.
mfbc_status general_output(RunCtx& rc, GeneralState& s, int nactive, int32_t* dist_out,
                           double* sigma_out);

// One batch of the level path.  Returns MFBC_OK, an error, or
// MFBC_ERR_NO_CONVERGENCE with *levels_exceeded set when Lcap was too small.
mfbc_status level_batch(RunCtx& rc, LevelState& s, const int32_t* d_src_batch, int nactive,
                        double* lambda, bool backward, int* levels_out, bool* levels_exceeded,
                        int64_t* fwd_iters, int64_t* bwd_iters);
mfbc_status level_output(RunCtx& rc, LevelState& s, int levels, int nactive, int32_t* dist_out,
                         double* sigma_out);

// One batch of the distance path (lambda != nullptr: full MFBC batch).
mfbc_status dist_batch(RunCtx& rc, DistState& s, const int32_t* d_src_batch, int nactive, double* lambda,
                       int64_t* fwd_iters, int64_t* bwd_iters);
mfbc_status dist_output(RunCtx& rc, DistState& s, int nactive, int32_t* dist_out, double* sigma_out);

// All batches of a call on the persistent small-graph kernel.  d_src_all:
// [nbatch][nb] columns' sources (-1 padding); d_wreq: [nbatch][W] lambda row
// of each word or null (row 0).  lambda null: MFBF only, writing sssp rows
// b*nb + j < out_rows of dist_out / sigma_out.  Batches the kernel could not
// finish (too deep, or counts >= 2^58) are returned in redo, untouched.
mfbc_status small_run(RunCtx& rc, SmallState& s, const int32_t* d_src_all, const int32_t* d_wreq, int nbatch,
                      double* lambda, int32_t* dist_out, double* sigma_out, int32_t out_rows, uint32_t opt_flags,
                      std::vector<int32_t>* redo);
void level_reset(RunCtx& rc, LevelState& s, int levels);

// Graph construction helpers (graph.cu).
mfbc_status graph_build(int32_t n, int64_t nnz, const int64_t* h_rowptr, const int32_t* h_col,
                        const int32_t* h_w, uint32_t flags, cudaStream_t st, DevGraph* g,
                        std::string* err);
void graph_free(DevGraph* g);

// Graph-handle accessors (api.cu).
const DevGraph* graph_device_view(const mfbc_graph* G);
uint32_t* graph_counter_mirror(const mfbc_graph* G);
void graph_lock(const mfbc_graph* G);
void graph_unlock(const mfbc_graph* G);
void set_last_error(const std::string& msg);

// Small device utilities (util.cu).
void fill_i32(int32_t* p, int32_t v, size_t count, cudaStream_t st);
void fill_f64(double* p, double v, size_t count, cudaStream_t st);
void check_sigma_exact(const double* sig, size_t count, Counters* ctr, cudaStream_t st);
void transpose_i32(const int32_t* in, int32_t* out, int32_t n, int nb, int nactive, int64_t out_ld,
                   cudaStream_t st);
void transpose_f64(const double* in, double* out, int32_t n, int nb, int nactive, int64_t out_ld,
                   cudaStream_t st);

// ------------------------------------------------------------ device helpers
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

}  // namespace mfbc

namespace mfbc {
inline mfbc_status cuda_fail(std::string* errp, const char* what, cudaError_t e) {
  if (errp) *errp = std::string(what) + ": " + cudaGetErrorString(e);
  return MFBC_ERR_CUDA;
}
}  // namespace mfbc

#define MFBC_CUDA_TRY(expr, errp)                                 \
  do {                                                            \
    cudaError_t _e = (expr);                                      \
    if (_e != cudaSuccess) return mfbc::cuda_fail((errp), #expr, _e); \
  } while (0)
