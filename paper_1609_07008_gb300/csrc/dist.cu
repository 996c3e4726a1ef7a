// Distance path: MFBF (Algorithm 1) and MFBr (Algorithm 2) for small integer
// weights, processed in order of distance value instead of Bellman-Ford
// products.
//
// With integer weights >= 1, every (s,v) at distance d has all its shortest-
// path predecessors at distances < d and all its DAG successors at distances
// > d.  So, stepping d = 0, 1, 2, ... over the distance values that occur:
//   * the pairs with tentative distance d are final (no later step can offer
//     less than d + 1);
//   * sigma_bar(s,v) = sum of sigma_bar(s,u) over in-neighbours u with
//     tau(s,u) + w(u,v) = d, all final (a pull: no multiplicity atomics);
//   * the pairs push candidates d + w to their out-neighbours (atomicMin on
//     the tentative distance), which can only land on values d+1 .. d+w_max.
// MFBr runs the same steps in decreasing order: zeta(s,v) is the sum over
// out-neighbours x with tau(s,x) = d + w(v,x) of zeta(s,x) + 1/sigma_bar(s,x)
// (Sec. 4.2.1), lambda(v) += zeta * sigma_bar (Algorithm 3), and the slot of
// (s,v) takes the value zeta + 1/sigma_bar.  Each (s,v) is settled once,
// whereas the Bellman-Ford products of the general kernels may improve a
// pair several times (weighted grids: about 540 products per batch).
//
// (Vertex, 32-column word) items waiting for a distance value are kept in a
// ring of w_max + 1 buckets (an item list and one flag bit per item each), so
// a step visits only the words that received a candidate for its distance.
// A step reads each item's 32 distances with one warp and works the pairs at
// its distance one per lane; the items that settle pairs are appended to one
// list with per-step offsets, which the backward pass replays in reverse.
#include <algorithm>

#include "internal.cuh"

namespace mfbc {

size_t dist_bytes(int32_t n, int nb, int B) {
  Carver c(nullptr, 0);
  DistState s;
  dist_carve(c, n, nb, B, s);
  return c.off;
}

void dist_carve(Carver& c, int32_t n, int nb, int B, DistState& s) {
  const size_t cells = (size_t)n * nb;
  s.nb = nb;
  s.W = nb / 32;
  s.B = B;
  s.BW = (B + 31) / 32;
  s.dist = c.take<int32_t>(cells);
  s.sig = c.take<double>(cells);
  s.val = c.take<double>(cells);
  // a (vertex, word) settles at most once per column; offsets into this list
  // are 32-bit, so the planner keeps n * n_b below 2^32
  s.mcap = cells + 1;
  s.mlist = c.take<uint32_t>(s.mcap);
  s.bcap = (size_t)n * s.W;                  // (vertex, word) items a bucket can hold
  s.blist = c.take<uint32_t>((size_t)B * s.bcap);
  s.bflag = c.take<uint32_t>(s.bcap * s.BW);
  s.bcount = c.take<uint32_t>(((size_t)B + 1) * DP_CSTRIDE);  // B bucket counts, settled-list count
  s.sy = c.take<DpSync>(1);
  s.sd = c.take<int32_t>(DP_STEP_RECORDS);
  s.soff = c.take<uint32_t>(DP_STEP_RECORDS);
  s.src = c.take<int32_t>((size_t)nb);
  s.word_req = c.take<int32_t>((size_t)s.W);
  s.ctr = c.take<Counters>(1);
}

// Level 0: (s_j, s_j) at distance 0 with sigma_bar 1, in bucket 0.
__global__ void k_dp_seed(const int32_t* __restrict__ src, int nb, int W, int BW, int32_t* dist, double* sig,
                          uint32_t* bflag, uint32_t* blist, uint32_t* bcount) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int32_t s = src[j];
  if (s < 0) return;
  dist[(size_t)s * nb + j] = 0;
  sig[(size_t)s * nb + j] = 1.0;
  const uint32_t item = (uint32_t)s * (uint32_t)W + (uint32_t)(j >> 5);
  if (!(atomicOr(&bflag[(size_t)item * BW], 1u) & 1u)) blist[atomicAdd(&bcount[0], 1u)] = item;  // bucket 0
}

// ------------------------------------------------------------ step kernels
// The steps of a batch are small (a weighted 256^2 grid has about 2200
// distance values, each settling about 15 000 pairs at 512 columns: under 500
// passes of 32 pairs over the whole GPU), so the host never waits between
// them.  The forward step reads its distance value
// from sy on the device, and the last block to finish it does the step's
// bookkeeping: it empties the bucket, records the step for MFBr, and moves
// sy->d to the next distance value with queued items (or sets sy->stop).  A
// round of DP_ROUND such launches is captured once per batch as a CUDA graph
// and replayed until sy->stop; launches after the last step return at once.
// (A persistent cooperative form with a grid barrier between steps was no
// faster alone, and its grid, holding every SM, stopped concurrent batches of
// other requests from overlapping.)
constexpr int DP_ROUND = 32;
static_assert(DP_ROUND <= DP_STEP_RECORDS, "a round records at most one step per launch");

struct DpFwd {
  uint32_t* blist;       // [B][bcap] bucket item lists
  uint32_t* bflag;       // [n * W][BW] bucket membership bits
  uint32_t* bcount;      // [B + 1] bucket counts, settled-list count (DP_CSTRIDE apart)
  uint32_t* mlist;       // settled (vertex, word) items in step order
  int32_t* dist;         // tau [n][nb]
  double* sig;           // sigma_bar [n][nb]
  const int64_t* rp; const int32_t* col; const int32_t* wt;     // A (out-arcs)
  const int64_t* rpt; const int32_t* colt; const int32_t* wtt;  // A^T (in-arcs)
  size_t bcap;
  int B, BW, W, nb;
  DpSync* sy;
  int32_t* sd;           // step records: distance value, first settled entry
  uint32_t* soff;
  unsigned long long* bytes;  // algorithmic bytes (counting runs only)
};

// A step's (vertex, word) items rarely have all 32 columns at its distance
// (on a weighted grid usually one: the word's sources are at different
// distances from the vertex).  So a warp reads an item's 32 distances, keeps
// the columns at distance d as (vertex, column) pairs in a per-warp queue, and
// works the queue 32 pairs at a time, one pair per lane: each lane walks its
// own vertex's arcs.
struct DpQueue {
  int32_t v[64];
  uint16_t j[64];        // column (n_b <= 4096)
  uint32_t m[32];        // settled items waiting for one settled-list reservation
};

// Arcs of one pair taken together: their loads and atomics are issued before
// any result is used, so a step's latency is a few memory round trips rather
// than a few per arc (the steps of small batches are latency chains).  Four
// arcs beat one and eight on grids and on dense graphs (measured when a warp
// still took one item, 32 columns, per pass).
constexpr int DP_ILP = 4;

// Appends the lanes with isM, as (v, column) pairs, to the warp's queue (whole warp).
__device__ __forceinline__ void dp_enqueue(DpQueue& q, int& qn, int32_t v, int j, bool isM, unsigned lane) {
  const uint32_t bal = __ballot_sync(0xffffffffu, isM);
  const int at = qn + __popc(bal & ((1u << lane) - 1u));
  __syncwarp();
  if (isM) { q.v[at] = v; q.j[at] = (uint16_t)j; }
  qn += __popc(bal);
  __syncwarp();
}

// Drops the first 32 entries of the queue (whole warp).
__device__ __forceinline__ void dp_shift(DpQueue& q, int& qn, unsigned lane) {
  int32_t v = 0;
  uint16_t j = 0;
  const bool keep = (int)lane < qn - 32;
  if (keep) { v = q.v[32 + lane]; j = q.j[32 + lane]; }
  __syncwarp();
  if (keep) { q.v[lane] = v; q.j[lane] = j; }
  qn -= 32;
  __syncwarp();
}

// Appends the warp's buffered settled items to the settled list with one
// reservation (whole warp).
__device__ __forceinline__ void dp_flush_settled(const DpFwd& a, DpQueue& q, int& mn, unsigned lane) {
  __syncwarp();
  uint32_t at = 0;
  if (lane == 0) at = atomicAdd(&a.bcount[(size_t)a.B * DP_CSTRIDE], (uint32_t)mn);
  at = __shfl_sync(0xffffffffu, at, 0);
  if ((int)lane < mn) a.mlist[at + lane] = q.m[lane];
  mn = 0;
  __syncwarp();
}

// Items are read SCAN at a time per warp, with their 32 distances each
// loaded before any is used.  Four suit graphs of small degree, where an item
// costs little more than these loads; one suits dense graphs, where the
// items' arc walks dominate and are better spread over more warps (weighted
// 256^2 grid, 4096 sources: 353 ms with one, 313 with four; Erdos-Renyi
// n = 2^16, k = 1024, 256 sources: 154 ms with one, 186 with four).
constexpr uint32_t DP_NO_ITEM = 0xffffffffu;   // items are < n * W <= 2^32 / 4

template <int SCAN>
__device__ __forceinline__ void dp_scan_load(const uint32_t* list, uint64_t count, uint64_t base, int W, int nb,
                                             const int32_t* dist, unsigned lane, uint32_t (&it)[SCAN],
                                             int32_t (&dv)[SCAN]) {
  const uint32_t mine = lane < (unsigned)SCAN && base + lane < count ? list[base + lane] : DP_NO_ITEM;
#pragma unroll
  for (int t = 0; t < SCAN; t++) {
    it[t] = __shfl_sync(0xffffffffu, mine, t);
    const int32_t v = (int32_t)(it[t] / (uint32_t)W);
    const int j = (int)(it[t] % (uint32_t)W) * 32 + (int)lane;
    dv[t] = it[t] != DP_NO_ITEM ? dist[(size_t)v * nb + j] : -1;
  }
}

// Forward pairs at distance d, lane i < cnt takes queue entry i.  The pair is
// final: sigma_bar is the sum over in-neighbours u one arc short of d
// (integers below 2^53, exact in any order), and it offers d + w to its
// out-neighbours; an out-neighbour's (vertex, word) item joins the bucket of
// d + w unless it is there already.
__device__ __forceinline__ void dp_fwd_pairs(const DpFwd& a, const DpQueue& q, int cnt, int32_t d, unsigned lane,
                                             unsigned long long& nbytes) {
  if ((int)lane >= cnt) return;
  const int32_t v = q.v[lane];
  const int j = q.j[lane];
  if (d > 0) {
    double acc = 0.0;
    const int64_t b = __ldg(&a.rpt[v]), e = __ldg(&a.rpt[v + 1]);
    for (int64_t k0 = b; k0 < e; k0 += DP_ILP) {
      size_t uj[DP_ILP];
      int32_t du[DP_ILP], want[DP_ILP];
#pragma unroll
      for (int t = 0; t < DP_ILP; t++) {
        const bool in = k0 + t < e;
        const int32_t u = in ? __ldg(&a.colt[k0 + t]) : 0;
        const int32_t w = in ? (a.wtt ? __ldg(&a.wtt[k0 + t]) : 1) : INF;
        const bool ok = in && w <= d;
        uj[t] = (size_t)u * a.nb + j;
        want[t] = d - w;
        du[t] = ok ? a.dist[uj[t]] : INF;       // want[t] < INF: never matches
        if (a.bytes && ok) nbytes += 4;
      }
#pragma unroll
      for (int t = 0; t < DP_ILP; t++)
        if (du[t] == want[t]) { acc += a.sig[uj[t]]; if (a.bytes) nbytes += 8; }
    }
    a.sig[(size_t)v * a.nb + j] = acc;
    if (a.bytes) nbytes += 8;
  }
  const uint32_t word = (uint32_t)j >> 5;
  const int64_t b = __ldg(&a.rp[v]), e = __ldg(&a.rp[v + 1]);
  for (int64_t k0 = b; k0 < e; k0 += DP_ILP) {
    int32_t x[DP_ILP], cand[DP_ILP], cur[DP_ILP];
#pragma unroll
    for (int t = 0; t < DP_ILP; t++) {
      const bool in = k0 + t < e;
      x[t] = in ? __ldg(&a.col[k0 + t]) : 0;
      cand[t] = d + (in ? (a.wt ? __ldg(&a.wt[k0 + t]) : 1) : 0);
      cur[t] = in ? a.dist[(size_t)x[t] * a.nb + j] : -1;  // cand[t] >= 0: never better
      if (a.bytes && in) nbytes += 4;
    }
#pragma unroll
    for (int t = 0; t < DP_ILP; t++) {
      if (cand[t] < cur[t]) {
        if (a.bytes) nbytes += 4;
        if (atomicMin(&a.dist[(size_t)x[t] * a.nb + j], cand[t]) > cand[t]) {
          const int s2 = cand[t] % a.B;
          const uint32_t bit = 1u << (s2 & 31);
          const uint32_t xi = (uint32_t)x[t] * (uint32_t)a.W + word;
          if (!(atomicOr(&a.bflag[(size_t)xi * a.BW + s2 / 32], bit) & bit)) {
            // one reservation per bucket among the lanes here
            const unsigned act = __activemask();
            const unsigned grp = __match_any_sync(act, s2);
            const int leader = __ffs(grp) - 1;
            uint32_t at = 0;
            if ((int)lane == leader) at = atomicAdd(&a.bcount[(size_t)s2 * DP_CSTRIDE], (uint32_t)__popc(grp));
            at = __shfl_sync(grp, at, leader) + __popc(grp & ((1u << lane) - 1u));
            a.blist[(size_t)s2 * a.bcap + at] = xi;
          }
        }
      }
    }
  }
}

// MFBF step at distance sy->d.  The candidates of step d land on d + 1 ..
// d + w_max, never in bucket d, so the last block can empty that bucket and
// look for the next non-empty one among the other w_max.
template <int SCAN>
__global__ void __launch_bounds__(256, 4) k_dp_fwd(DpFwd a) {
  __shared__ int32_t s_d;
  __shared__ uint32_t s_cnt, s_stop, s_last, s_j;
  const unsigned lane = lane_id();
  volatile DpSync* vs = a.sy;
  if (threadIdx.x == 0) {
    s_stop = vs->stop;
    s_d = vs->d;
    s_cnt = s_stop ? 0u : __ldcg(&a.bcount[(size_t)(s_d % a.B) * DP_CSTRIDE]);
  }
  __syncthreads();
  if (s_stop) return;
  const int32_t d = s_d;
  const int slot = d % a.B;
  const uint32_t count = s_cnt;
  const uint32_t* list = a.blist + (size_t)slot * a.bcap;
  const uint64_t nw = (gridDim.x * blockDim.x) >> 5;
  unsigned long long nbytes = 0;
  __shared__ DpQueue dq[8];
  DpQueue& q = dq[threadIdx.x >> 5];
  int qn = 0;                                  // warp-uniform queue length (< 32 between items)
  int mn = 0;                                  // warp-uniform count of settled items not yet listed
  for (uint64_t base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * SCAN; base < count;
       base += nw * SCAN) {
    uint32_t it[SCAN];
    int32_t dv[SCAN];
    dp_scan_load(list, count, base, a.W, a.nb, a.dist, lane, it, dv);
#pragma unroll
    for (int t = 0; t < SCAN; t++) {
      if (it[t] == DP_NO_ITEM) break;
      const int32_t v = (int32_t)(it[t] / (uint32_t)a.W);
      const int j = (int)(it[t] % (uint32_t)a.W) * 32 + (int)lane;
      if (lane == 0) atomicAnd(&a.bflag[(size_t)it[t] * a.BW + slot / 32], ~(1u << (slot & 31)));
      const bool isM = dv[t] == d;
      if (a.bytes) nbytes += 4;
      if (!__any_sync(0xffffffffu, isM)) continue;
      if (lane == 0) q.m[mn] = it[t];
      if (++mn == 32) dp_flush_settled(a, q, mn, lane);
      dp_enqueue(q, qn, v, j, isM, lane);
      if (qn >= 32) {
        dp_fwd_pairs(a, q, 32, d, lane, nbytes);
        __syncwarp();
        dp_shift(q, qn, lane);
      }
    }
  }
  if (qn > 0) dp_fwd_pairs(a, q, qn, d, lane, nbytes);
  __syncwarp();
  if (mn > 0) dp_flush_settled(a, q, mn, lane);
  if (a.bytes) {
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0 && nbytes) atomicAdd(a.bytes, nbytes);
  }
  // the last block to finish the step does its bookkeeping
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();                           // publish this block's writes
    s_last = atomicAdd(&a.sy->done, 1u) == gridDim.x - 1;
    s_j = 0xffffffffu;
  }
  __syncthreads();
  if (!s_last) return;
  __threadfence();                             // see every block's writes
  for (uint32_t j = 1 + threadIdx.x; j < (uint32_t)a.B; j += blockDim.x)
    if (__ldcg(&a.bcount[(size_t)((d + (int32_t)j) % a.B) * DP_CSTRIDE])) atomicMin(&s_j, j);
  __syncthreads();
  if (threadIdx.x == 0) {
    a.bcount[(size_t)slot * DP_CSTRIDE] = 0;
    const uint32_t end = __ldcg(&a.bcount[(size_t)a.B * DP_CSTRIDE]);
    const uint32_t k = vs->k;
    vs->steps = vs->steps + 1;
    if (end != vs->off && k < (uint32_t)DP_STEP_RECORDS) {  // the step settled pairs: record it
      a.sd[k] = d;
      a.soff[k] = vs->off;
      vs->k = k + 1;
      vs->off = end;
    }
    if (s_j == 0xffffffffu) vs->stop = 1;
    else vs->d = d + (int32_t)s_j;
    vs->done = 0;
  }
}

struct DpBwd {
  const uint32_t* items;  // the step's settled (vertex, word) items
  uint32_t count;
  int32_t d;
  const int64_t* rp; const int32_t* col; const int32_t* wt;
  const int32_t* dist; const double* sig;  // final, read-only in MFBr
  double* val;           // zeta + 1/sigma_bar [n][nb]
  const int32_t* src;
  double* lambda;
  const int32_t* word_req;
  int W, nb;
  int32_t n;
  unsigned long long* bytes;
};

// Backward pairs at distance d, lane i < cnt takes queue entry i: zeta is
// the sum over out-neighbours x at d + w of their value zeta + 1/sigma_bar
// (Sec. 4.2.1), the slot takes zeta + 1/sigma_bar, and lambda(v) gains
// zeta * sigma_bar (Algorithm 3), summed over each item's pairs (they sit
// next to each other in the queue, and an item occurs once per step).
__device__ __forceinline__ void dp_bwd_pairs(const DpBwd& a, const DpQueue& q, int cnt, int32_t d, unsigned lane,
                                             unsigned long long& nbytes) {
  const bool has = (int)lane < cnt;
  const int32_t v = has ? q.v[lane] : -1;
  const int j = has ? q.j[lane] : 0;
  const int r = has ? (a.word_req ? __ldg(&a.word_req[j >> 5]) : 0) : -1;
  double lam = 0.0;
  if (has) {
    double acc = 0.0;
    const int64_t b = __ldg(&a.rp[v]), e = __ldg(&a.rp[v + 1]);
    for (int64_t k0 = b; k0 < e; k0 += DP_ILP) {
      size_t xj[DP_ILP];
      int32_t dx[DP_ILP], want[DP_ILP];
#pragma unroll
      for (int t = 0; t < DP_ILP; t++) {
        const bool in = k0 + t < e;
        const int32_t x = in ? __ldg(&a.col[k0 + t]) : 0;
        want[t] = d + (in ? (a.wt ? __ldg(&a.wt[k0 + t]) : 1) : 0);
        xj[t] = (size_t)x * a.nb + j;
        dx[t] = in ? __ldg(&a.dist[xj[t]]) : -1;  // want[t] >= 1: never matches
        if (a.bytes && in) nbytes += 4;
      }
#pragma unroll
      for (int t = 0; t < DP_ILP; t++)
        if (dx[t] == want[t]) { acc += a.val[xj[t]]; if (a.bytes) nbytes += 8; }
    }
    const size_t vj = (size_t)v * a.nb + j;
    const double sg = __ldg(&a.sig[vj]);
    if (__ldg(&a.src[j]) != v) lam = acc * sg;
    a.val[vj] = acc + 1.0 / sg;
    if (a.bytes) nbytes += 20;
  }
  // segmented sum over runs of one item (vertex, word); the run's last lane
  // adds it
  const int wd = j >> 5;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const double y = __shfl_up_sync(0xffffffffu, lam, o);
    const int32_t vo = __shfl_up_sync(0xffffffffu, v, o);
    const int wo = __shfl_up_sync(0xffffffffu, wd, o);
    if ((int)lane >= o && vo == v && wo == wd) lam += y;
  }
  const int32_t vn = __shfl_down_sync(0xffffffffu, v, 1);
  const int wn = __shfl_down_sync(0xffffffffu, wd, 1);
  const bool last = lane == 31 || vn != v || wn != wd;
  if (has && last && r >= 0 && lam != 0.0) atomicAdd(&a.lambda[(size_t)r * a.n + v], lam);
}

// MFBr step at distance a.d over the items that settled there.
template <int SCAN>
__global__ void __launch_bounds__(256, 4) k_dp_bwd(DpBwd a) {
  __shared__ DpQueue dq[8];
  DpQueue& q = dq[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  const uint64_t nw = (gridDim.x * blockDim.x) >> 5;
  unsigned long long nbytes = 0;
  int qn = 0;
  for (uint64_t base = ((blockIdx.x * blockDim.x + threadIdx.x) >> 5) * SCAN; base < a.count;
       base += nw * SCAN) {
    uint32_t it[SCAN];
    int32_t dv[SCAN];
    dp_scan_load(a.items, a.count, base, a.W, a.nb, a.dist, lane, it, dv);
#pragma unroll
    for (int t = 0; t < SCAN; t++) {
      if (it[t] == DP_NO_ITEM) break;
      const int32_t v = (int32_t)(it[t] / (uint32_t)a.W);
      const int j = (int)(it[t] % (uint32_t)a.W) * 32 + (int)lane;
      dp_enqueue(q, qn, v, j, dv[t] == a.d, lane);
      if (qn >= 32) {
        dp_bwd_pairs(a, q, 32, a.d, lane, nbytes);
        dp_shift(q, qn, lane);
      }
    }
  }
  if (qn > 0) dp_bwd_pairs(a, q, qn, a.d, lane, nbytes);
  if (a.bytes) {
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0 && nbytes) atomicAdd(a.bytes, nbytes);
  }
}

#define PROF(id, ...)             \
  do {                            \
    rc.prof->begin(id);           \
    __VA_ARGS__;                  \
    rc.prof->end(id);             \
  } while (0)

// One wave of blocks: each item is a chain of dependent loads, so a step
// wants every warp the SMs hold, and blocks beyond one wave would only read
// the count and leave.
static unsigned dp_blocks(const void* kern) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess) return 0;
  return (unsigned)(sms * std::max(per_sm, 1));
}

static inline unsigned dp_grid(uint64_t warps, unsigned cap) {
  const uint64_t b = (warps + 7) / 8;
  return (unsigned)(b < 1 ? 1 : (b > cap ? cap : b));
}

// A round of DP_ROUND forward step launches as an executable CUDA graph,
// captured on a private stream of the calling thread (capture is not
// possible on the legacy default stream, which callers may pass).
struct DpRound {
  cudaGraphExec_t exec = nullptr;
  ~DpRound() { if (exec) cudaGraphExecDestroy(exec); }
  cudaError_t build(const void* kern, const DpFwd& fa, unsigned grid) {
    static thread_local cudaStream_t cap = nullptr;
    cudaError_t e = cudaSuccess;
    if (!cap && (e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking)) != cudaSuccess) return e;
    if ((e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal)) != cudaSuccess) return e;
    void* args[] = {const_cast<DpFwd*>(&fa)};
    cudaError_t le = cudaSuccess;
    for (int k = 0; k < DP_ROUND && le == cudaSuccess; k++) le = cudaLaunchKernel(kern, grid, 256, args, 0, cap);
    cudaGraph_t gr = nullptr;
    e = cudaStreamEndCapture(cap, &gr);         // ends the capture in every case
    if (le != cudaSuccess) e = le;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, gr, 0);
    if (gr) cudaGraphDestroy(gr);
    return e;
  }
};

mfbc_status dist_batch(RunCtx& rc, DistState& s, const int32_t* d_src_batch, int nactive, double* lambda,
                       int64_t* fwd_iters, int64_t* bwd_iters) {
  const DevGraph& g = *rc.g;
  const int32_t n = g.n;
  const int nb = s.nb, W = s.W, B = s.B;
  cudaStream_t st = rc.stream;
  const size_t cells = (size_t)n * nb;
  unsigned long long* B_ = rc.prof->count_bytes ? s.ctr->bytes : nullptr;
  if (n == 0) return MFBC_OK;

  fill_i32(s.src, -1, (size_t)nb, st);
  if (nactive)
    MFBC_CUDA_TRY(cudaMemcpyAsync(s.src, d_src_batch, sizeof(int32_t) * nactive, cudaMemcpyDeviceToDevice, st),
                  rc.err);
  PROF(K_FILL, {
    fill_i32(s.dist, INF, cells, st);
    cudaMemsetAsync(s.sig, 0, sizeof(double) * cells, st);
    cudaMemsetAsync(s.bflag, 0, sizeof(uint32_t) * s.bcap * s.BW, st);
    cudaMemsetAsync(s.bcount, 0, sizeof(uint32_t) * ((size_t)B + 1) * DP_CSTRIDE, st);
    cudaMemsetAsync(s.sy, 0, sizeof(DpSync), st);
  });
  rc.prof->k[K_FILL].bytes += 12.0 * cells + 4.0 * s.bcap * s.BW;
  PROF(K_SEED, (k_dp_seed<<<(nb + 127) / 128, 128, 0, st>>>(s.src, nb, W, s.BW, s.dist, s.sig, s.bflag, s.blist,
                                                          s.bcount)));

  // ---- MFBF in increasing distance order, DP_ROUND steps between host reads
  const DpFwd fa{s.blist, s.bflag, s.bcount, s.mlist, s.dist, s.sig, g.rowptr, g.col, g.w, g.rowptr_t, g.col_t,
                 g.w_t, s.bcap, B, s.BW, W, nb, s.sy, s.sd, s.soff, B_ ? B_ + K_DP_FWD : nullptr};
  const bool dense = g.nnz >= 32 * (int64_t)n;  // scan one item at a time (see SCAN)
  const void* fk = dense ? (const void*)k_dp_fwd<1> : (const void*)k_dp_fwd<4>;
  const unsigned fgrid = dp_blocks(fk);
  if (!fgrid) return cuda_fail(rc.err, "occupancy of the distance kernels", cudaGetLastError());
  DpRound round;
  MFBC_CUDA_TRY(round.build(fk, fa, fgrid), rc.err);
  std::vector<int32_t> hd, kd((size_t)DP_STEP_RECORDS);
  std::vector<uint32_t> hoff, koff((size_t)DP_STEP_RECORDS);
  DpSync hs{};
  const int64_t max_rounds = (int64_t)n * (int64_t)std::max(1, g.wmax) / DP_ROUND + 2;
  for (int64_t r = 0;; r++) {
    cudaError_t e;
    PROF(K_DP_FWD, e = cudaGraphLaunch(round.exec, st));
    MFBC_CUDA_TRY(e, rc.err);
    rc.prof->k[K_DP_FWD].launches += DP_ROUND - 1;   // kernels, not graph launches
    MFBC_CUDA_TRY(cudaMemcpyAsync(&hs, s.sy, sizeof(DpSync), cudaMemcpyDeviceToHost, st), rc.err);
    MFBC_CUDA_TRY(cudaMemcpyAsync(kd.data(), s.sd, sizeof(int32_t) * DP_STEP_RECORDS, cudaMemcpyDeviceToHost, st),
                  rc.err);
    MFBC_CUDA_TRY(
        cudaMemcpyAsync(koff.data(), s.soff, sizeof(uint32_t) * DP_STEP_RECORDS, cudaMemcpyDeviceToHost, st),
        rc.err);
    MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
    rc.prof->drain();
    hd.insert(hd.end(), kd.begin(), kd.begin() + hs.k);
    hoff.insert(hoff.end(), koff.begin(), koff.begin() + hs.k);
    if (hs.stop) break;
    if (r >= max_rounds) {
      if (rc.err) *rc.err = "distance steps did not terminate";
      return MFBC_ERR_NO_CONVERGENCE;
    }
    hs.k = 0;                                  // the next round records from the start
    MFBC_CUDA_TRY(cudaMemcpyAsync(s.sy, &hs, sizeof(DpSync), cudaMemcpyHostToDevice, st), rc.err);
  }
  if (fwd_iters) *fwd_iters += hs.steps;
  check_sigma_exact(s.sig, cells, s.ctr, st);
  if (!lambda) return MFBC_OK;

  // ---- MFBr in decreasing distance order (distance 0 holds the sources only)
  const int32_t* wreq = nullptr;
  const int urq = rc.word_req ? batch_uniform_request(rc.word_req, W) : 0;
  if (rc.word_req && urq < 0) {
    MFBC_CUDA_TRY(cudaMemcpyAsync(s.word_req, rc.word_req, sizeof(int32_t) * W, cudaMemcpyHostToDevice, st),
                  rc.err);
    wreq = s.word_req;
  }
  double* lam0 = wreq ? lambda : lambda + (size_t)(urq < 0 ? 0 : urq) * n;
  const void* bk = dense ? (const void*)k_dp_bwd<1> : (const void*)k_dp_bwd<4>;
  const unsigned bcap = dp_blocks(bk);
  if (!bcap) return cuda_fail(rc.err, "occupancy of the distance kernels", cudaGetLastError());
  DpBwd ba{nullptr, 0, 0, g.rowptr, g.col, g.w, s.dist, s.sig, s.val, s.src, lam0, wreq, W, nb, n,
           B_ ? B_ + K_DP_BWD : nullptr};
  for (int64_t i = (int64_t)hd.size() - 1; i >= 0; i--) {
    if (hd[(size_t)i] <= 0) continue;
    const uint32_t end = (size_t)i + 1 < hoff.size() ? hoff[(size_t)i + 1] : hs.off;
    ba.items = s.mlist + hoff[(size_t)i];
    ba.count = end - hoff[(size_t)i];
    ba.d = hd[(size_t)i];
    void* args[] = {&ba};
    cudaError_t e;
    PROF(K_DP_BWD, e = cudaLaunchKernel(bk, dp_grid(ba.count, bcap), 256, args, 0, st));
    MFBC_CUDA_TRY(e, rc.err);
    if (bwd_iters) (*bwd_iters)++;
  }
  MFBC_CUDA_TRY(cudaGetLastError(), rc.err);
  return MFBC_OK;
}

mfbc_status dist_output(RunCtx& rc, DistState& s, int nactive, int32_t* dist_out, double* sigma_out) {
  const int32_t n = rc.g->n;
  PROF(K_OUTPUT, {
    transpose_i32(s.dist, dist_out, n, s.nb, nactive, n, rc.stream);
    if (sigma_out) transpose_f64(s.sig, sigma_out, n, s.nb, nactive, n, rc.stream);
  });
  return MFBC_OK;
}

}  // namespace mfbc
