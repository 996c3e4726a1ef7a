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
// A step runs one warp per item; the items that settle pairs are appended to
// one list with per-step offsets, which the backward pass replays in
// reverse.
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
  s.mcap = cells + 1;                        // a (vertex, word) settles at most once per column
  s.mlist = c.take<uint32_t>(s.mcap);
  s.bcap = (size_t)n * s.W;                  // (vertex, word) items a bucket can hold
  s.blist = c.take<uint32_t>((size_t)B * s.bcap);
  s.bflag = c.take<uint32_t>(s.bcap * s.BW);
  s.bcount = c.take<uint32_t>((size_t)B + 1); // B bucket counts, then the settled-list count
  s.sy = c.take<DpSync>(1);
  s.sd = c.take<int32_t>(DP_STEPS);
  s.soff = c.take<uint32_t>(DP_STEPS);
  s.scnt = c.take<uint32_t>(DP_STEPS);
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
  if (!(atomicOr(&bflag[(size_t)item * BW], 1u) & 1u)) blist[atomicAdd(&bcount[0], 1u)] = item;
}

// ------------------------------------------------ persistent step kernels
// The steps of a batch are tiny (a weighted 256^2 grid has about 2000 distance
// values, each holding a few hundred items per 512 columns), so both passes
// run as one cooperative launch whose resident blocks take the steps one
// after another, separated by a grid-wide barrier, instead of one launch per
// step.  The block that reaches a barrier last does the step's bookkeeping
// while the others wait.  Every wait is bounded: past DP_WAIT_NS the waiting
// block sets sy->err, every block leaves its loop, and the host reports
// MFBC_ERR_TIMEOUT.  Buffers that other blocks write during the launch are
// read with plain (or L2-only) loads after the barrier's fences, never through
// the read-only data path.
constexpr uint64_t DP_WAIT_NS = 10ull * 1000 * 1000 * 1000;

__device__ __forceinline__ uint64_t dp_clock_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid-wide barrier.  `serial` runs in all threads of the block that arrives
// last, after every block has finished the work before the barrier and
// before any block continues.  Returns false in every block once a wait has
// timed out (here or in another block).
template <class Serial>
__device__ __forceinline__ bool dp_barrier(DpSync* sy, Serial serial) {
  __shared__ uint32_t s_last, s_gen, s_err;
  volatile DpSync* vs = sy;
  __syncthreads();                             // this block's work of the step is done
  if (threadIdx.x == 0) {
    s_gen = vs->gen;                           // cannot advance before this block arrives
    __threadfence();                           // publish the block's writes
    s_last = atomicAdd(&sy->arrive, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (s_last) {
    __threadfence();
    serial();
    __syncthreads();
    if (threadIdx.x == 0) {
      vs->arrive = 0;
      __threadfence();
      vs->gen = s_gen + 1;                     // release the waiting blocks
    }
  } else if (threadIdx.x == 0) {
    const uint64_t t0 = dp_clock_ns();
    while (vs->gen == s_gen) {
      if (dp_clock_ns() - t0 > DP_WAIT_NS) { atomicOr(&sy->err, 1u); break; }
      __nanosleep(32);
    }
    __threadfence();                           // acquire what the other blocks wrote
  }
  if (threadIdx.x == 0) s_err = vs->err;
  __syncthreads();
  return s_err == 0;
}

struct DpFwd {
  uint32_t* blist;       // [B][bcap] bucket item lists
  uint32_t* bflag;       // [n * W][BW] bucket membership bits
  uint32_t* bcount;      // [B + 1] bucket counts, settled-list count
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

// Arcs of one item taken together: their loads and atomics are issued before
// any result is used, so a step's latency is a few memory round trips rather
// than a few per arc (the steps of small batches are latency chains).  Four
// arcs (58-61 registers) beat one and eight on grids and on dense graphs.
constexpr int DP_ILP = 4;

// One forward item at distance d: the warp's lanes are the 32 columns of word
// `word` of vertex v.  Pairs at distance d are final: their sigma_bar is the
// sum over in-neighbours u one arc short of d (integers below 2^53, exact in
// any order), and they offer d + w to their out-neighbours.
__device__ __forceinline__ void dp_fwd_item(const DpFwd& a, uint32_t item, int32_t d, int slot, unsigned lane,
                                            unsigned long long& nbytes) {
  const int32_t v = (int32_t)(item / (uint32_t)a.W);
  const int word = (int)(item % (uint32_t)a.W);
  if (lane == 0) atomicAnd(&a.bflag[(size_t)item * a.BW + slot / 32], ~(1u << (slot & 31)));
  const int j = word * 32 + (int)lane;
  const size_t vj = (size_t)v * a.nb + j;
  const bool isM = a.dist[vj] == d;
  if (a.bytes) nbytes += 4;
  if (!__ballot_sync(0xffffffffu, isM)) return;
  if (lane == 0) a.mlist[atomicAdd(&a.bcount[a.B], 1u)] = item;
  if (d > 0) {
    double acc = 0.0;
    const int64_t b = __ldg(&a.rpt[v]), e = __ldg(&a.rpt[v + 1]);
    for (int64_t k0 = b; k0 < e; k0 += 32) {
      const int64_t k = k0 + lane;
      const int32_t myu = k < e ? __ldg(&a.colt[k]) : 0;
      const int32_t myw = k < e ? (a.wtt ? __ldg(&a.wtt[k]) : 1) : INF;
      const int cnt = (int)(e - k0 < 32 ? e - k0 : 32);
      for (int t0 = 0; t0 < cnt; t0 += DP_ILP) {
        size_t uj[DP_ILP];
        int32_t du[DP_ILP], want[DP_ILP];
#pragma unroll
        for (int q = 0; q < DP_ILP; q++) {
          const int32_t u = __shfl_sync(0xffffffffu, myu, (t0 + q) & 31);
          const int32_t w = __shfl_sync(0xffffffffu, myw, (t0 + q) & 31);
          const bool ok = isM && t0 + q < cnt && w <= d;
          uj[q] = (size_t)u * a.nb + j;
          want[q] = d - w;
          du[q] = ok ? a.dist[uj[q]] : INF;      // want[q] < INF: never matches
          if (a.bytes && ok) nbytes += 4;
        }
#pragma unroll
        for (int q = 0; q < DP_ILP; q++)
          if (du[q] == want[q]) { acc += a.sig[uj[q]]; if (a.bytes) nbytes += 8; }
      }
    }
    if (isM) { a.sig[vj] = acc; if (a.bytes) nbytes += 8; }
  }
  const int64_t b = __ldg(&a.rp[v]), e = __ldg(&a.rp[v + 1]);
  for (int64_t k0 = b; k0 < e; k0 += 32) {
    const int64_t k = k0 + lane;
    const int32_t myx = k < e ? __ldg(&a.col[k]) : 0;
    const int32_t myw = k < e ? (a.wt ? __ldg(&a.wt[k]) : 1) : 0;
    const int cnt = (int)(e - k0 < 32 ? e - k0 : 32);
    for (int t0 = 0; t0 < cnt; t0 += DP_ILP) {
      int32_t x[DP_ILP], cand[DP_ILP], cur[DP_ILP];
#pragma unroll
      for (int q = 0; q < DP_ILP; q++) {
        x[q] = __shfl_sync(0xffffffffu, myx, (t0 + q) & 31);
        cand[q] = d + __shfl_sync(0xffffffffu, myw, (t0 + q) & 31);
        const bool ok = isM && t0 + q < cnt;
        cur[q] = ok ? a.dist[(size_t)x[q] * a.nb + j] : -1;  // cand[q] >= 1: never better
        if (a.bytes && ok) nbytes += 4;
      }
      unsigned imp = 0;                        // bit q: arc t0 + q improved some column
#pragma unroll
      for (int q = 0; q < DP_ILP; q++) {
        const bool better = cand[q] < cur[q] && atomicMin(&a.dist[(size_t)x[q] * a.nb + j], cand[q]) > cand[q];
        if (a.bytes && cand[q] < cur[q]) nbytes += 4;
        if (__ballot_sync(0xffffffffu, better)) imp |= 1u << q;
      }
      // lane q queues (x, word) of arc t0 + q for distance cand
      int32_t xq = 0, cq = 0;
#pragma unroll
      for (int q = 0; q < DP_ILP; q++)
        if ((int)lane == q) { xq = x[q]; cq = cand[q]; }
      if (lane < (unsigned)DP_ILP && ((imp >> lane) & 1u)) {
        const int s2 = cq % a.B;
        const uint32_t bit = 1u << (s2 & 31);
        const uint32_t xi = (uint32_t)xq * (uint32_t)a.W + (uint32_t)word;
        if (!(atomicOr(&a.bflag[(size_t)xi * a.BW + s2 / 32], bit) & bit))
          a.blist[(size_t)s2 * a.bcap + atomicAdd(&a.bcount[s2], 1u)] = xi;
      }
    }
  }
}

// MFBF: steps d = sy->d, then the next distance value with queued items, ...
// until no bucket holds items (stop 1) or DP_STEPS steps with settled items
// have been recorded (stop 2; the host launches again from sy->d).  The
// candidates of step d land on d + 1 .. d + w_max, i.e. never in bucket d, so
// the last block to finish step d can empty that bucket and look for the next
// non-empty one among the other w_max.
__global__ void __launch_bounds__(256) k_dp_fwd(DpFwd a) {
  __shared__ int32_t s_d;
  __shared__ uint32_t s_cnt, s_stop, s_j;
  const unsigned lane = lane_id();
  const uint64_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint64_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  unsigned long long nbytes = 0;
  volatile DpSync* vs = a.sy;
  for (;;) {
    if (threadIdx.x == 0) {
      s_stop = vs->stop | vs->err;
      s_d = vs->d;
      s_cnt = s_stop ? 0u : __ldcg(&a.bcount[s_d % a.B]);
    }
    __syncthreads();
    if (s_stop) break;
    const int32_t d = s_d;
    const int slot = d % a.B;
    const uint32_t count = s_cnt;
    const uint32_t* list = a.blist + (size_t)slot * a.bcap;
    for (uint64_t gw = w0; gw < count; gw += nw) dp_fwd_item(a, list[gw], d, slot, lane, nbytes);
    const bool ok = dp_barrier(a.sy, [&] {
      if (threadIdx.x == 0) s_j = 0xffffffffu;
      __syncthreads();
      for (uint32_t j = 1 + threadIdx.x; j < (uint32_t)a.B; j += blockDim.x)
        if (__ldcg(&a.bcount[(d + (int32_t)j) % a.B])) atomicMin(&s_j, j);
      __syncthreads();
      if (threadIdx.x == 0) {
        a.bcount[slot] = 0;
        const uint32_t end = __ldcg(&a.bcount[a.B]);
        const uint32_t k = vs->k;
        vs->steps = vs->steps + 1;
        if (end != vs->off) {                  // the step settled pairs: record it
          a.sd[k] = d;
          a.soff[k] = vs->off;
          vs->k = k + 1;
          vs->off = end;
        }
        if (s_j == 0xffffffffu) vs->stop = 1;
        else {
          vs->d = d + (int32_t)s_j;
          if (vs->k == (uint32_t)DP_STEPS) vs->stop = 2;
        }
      }
    });
    if (!ok) break;
  }
  if (a.bytes) {
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0) atomicAdd(a.bytes, nbytes);
  }
}

struct DpBwd {
  const uint32_t* mlist;
  const int32_t* sd;     // [nsteps] distance values, decreasing
  const uint32_t* soff;  // [nsteps] first settled-list entry of each step
  const uint32_t* scnt;  // [nsteps] its length
  int nsteps;
  const int64_t* rp; const int32_t* col; const int32_t* wt;
  const int32_t* dist; const double* sig;  // final, read-only during the launch
  double* val;           // zeta + 1/sigma_bar [n][nb]
  const int32_t* src;
  double* lambda;
  const int32_t* word_req;
  int W, nb;
  int32_t n;
  DpSync* sy;
  unsigned long long* bytes;
};

// One backward item at distance d: zeta of the pairs settled at d is the sum
// over out-neighbours x at d + w of their value zeta + 1/sigma_bar (Sec.
// 4.2.1); lambda(v) += zeta * sigma_bar over the word's columns (Algorithm 3).
__device__ __forceinline__ void dp_bwd_item(const DpBwd& a, uint32_t it, int32_t d, unsigned lane,
                                            unsigned long long& nbytes) {
  const int32_t v = (int32_t)(it / (uint32_t)a.W);
  const int word = (int)(it % (uint32_t)a.W);
  const int r = a.word_req ? __ldg(&a.word_req[word]) : 0;
  const int j = word * 32 + (int)lane;
  const size_t vj = (size_t)v * a.nb + j;
  const bool isM = __ldg(&a.dist[vj]) == d;
  double acc = 0.0;
  const int64_t b = __ldg(&a.rp[v]), e = __ldg(&a.rp[v + 1]);
  for (int64_t k0 = b; k0 < e; k0 += 32) {
    const int64_t k = k0 + lane;
    const int32_t myx = k < e ? __ldg(&a.col[k]) : 0;
    const int32_t myw = k < e ? (a.wt ? __ldg(&a.wt[k]) : 1) : 0;
    const int cnt = (int)(e - k0 < 32 ? e - k0 : 32);
    for (int t0 = 0; t0 < cnt; t0 += DP_ILP) {
      size_t xj[DP_ILP];
      int32_t dx[DP_ILP], want[DP_ILP];
#pragma unroll
      for (int q = 0; q < DP_ILP; q++) {
        const int32_t x = __shfl_sync(0xffffffffu, myx, (t0 + q) & 31);
        const int32_t w = __shfl_sync(0xffffffffu, myw, (t0 + q) & 31);
        const bool ok = isM && t0 + q < cnt;
        xj[q] = (size_t)x * a.nb + j;
        want[q] = d + w;
        dx[q] = ok ? __ldg(&a.dist[xj[q]]) : -1;  // want[q] >= 1: never matches
        if (a.bytes && ok) nbytes += 4;
      }
#pragma unroll
      for (int q = 0; q < DP_ILP; q++)
        if (dx[q] == want[q]) { acc += a.val[xj[q]]; if (a.bytes) nbytes += 8; }
    }
  }
  double lam = 0.0;
  if (isM) {
    const double sg = __ldg(&a.sig[vj]);
    if (__ldg(&a.src[j]) != v) lam = acc * sg;
    a.val[vj] = acc + 1.0 / sg;
    if (a.bytes) nbytes += 20;
  }
  for (int o = 16; o; o >>= 1) lam += __shfl_xor_sync(0xffffffffu, lam, o);
  if (lane == 0 && r >= 0 && lam != 0.0) atomicAdd(&a.lambda[(size_t)r * a.n + v], lam);
}

// MFBr: the recorded steps in decreasing distance order, one barrier apart.
__global__ void __launch_bounds__(256) k_dp_bwd(DpBwd a) {
  const unsigned lane = lane_id();
  const uint64_t nw = (gridDim.x * blockDim.x) >> 5;
  const uint64_t w0 = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  unsigned long long nbytes = 0;
  for (int k = 0; k < a.nsteps; k++) {
    const int32_t d = __ldg(&a.sd[k]);
    const uint32_t* items = a.mlist + __ldg(&a.soff[k]);
    const uint32_t count = __ldg(&a.scnt[k]);
    for (uint64_t gw = w0; gw < count; gw += nw) dp_bwd_item(a, __ldg(&items[gw]), d, lane, nbytes);
    if (k + 1 < a.nsteps && !dp_barrier(a.sy, [] {})) break;
  }
  if (a.bytes) {
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0) atomicAdd(a.bytes, nbytes);
  }
}

#define PROF(id, ...)             \
  do {                            \
    rc.prof->begin(id);           \
    __VA_ARGS__;                  \
    rc.prof->end(id);             \
  } while (0)

// Blocks of a cooperative launch: as many as the SMs hold at once (each item
// is a chain of dependent loads, so the steps need every resident warp; two
// blocks per SM made small batches 1.3x and dense graphs 2.5x slower).
static unsigned dp_blocks(const void* kern) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, 0) != cudaSuccess) return 0;
  return (unsigned)(sms * per_sm);
}

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
    cudaMemsetAsync(s.bcount, 0, sizeof(uint32_t) * ((size_t)B + 1), st);
    cudaMemsetAsync(s.sy, 0, sizeof(DpSync), st);
  });
  rc.prof->k[K_FILL].bytes += 12.0 * cells + 4.0 * s.bcap * s.BW;
  PROF(K_SEED, (k_dp_seed<<<(nb + 127) / 128, 128, 0, st>>>(s.src, nb, W, s.BW, s.dist, s.sig, s.bflag, s.blist,
                                                          s.bcount)));

  // ---- MFBF in increasing distance order, DP_STEPS recorded steps per launch
  DpFwd fa{s.blist, s.bflag, s.bcount, s.mlist, s.dist, s.sig, g.rowptr, g.col, g.w, g.rowptr_t, g.col_t, g.w_t,
           s.bcap, B, s.BW, W, nb, s.sy, s.sd, s.soff, B_ ? B_ + K_DP_FWD : nullptr};
  const unsigned fgrid = dp_blocks((const void*)k_dp_fwd);
  if (!fgrid) return cuda_fail(rc.err, "occupancy of the distance kernels", cudaGetLastError());
  std::vector<int32_t> hd, kd((size_t)DP_STEPS);
  std::vector<uint32_t> hoff, koff((size_t)DP_STEPS);
  DpSync hs{};
  const int64_t max_launches = (int64_t)n * (int64_t)std::max(1, g.wmax) / DP_STEPS + 2;
  for (int64_t launch = 0;; launch++) {
    void* args[] = {&fa};
    cudaError_t e;
    PROF(K_DP_FWD, e = cudaLaunchCooperativeKernel((const void*)k_dp_fwd, fgrid, 256, args, 0, st));
    MFBC_CUDA_TRY(e, rc.err);
    MFBC_CUDA_TRY(cudaMemcpyAsync(&hs, s.sy, sizeof(DpSync), cudaMemcpyDeviceToHost, st), rc.err);
    MFBC_CUDA_TRY(cudaMemcpyAsync(kd.data(), s.sd, sizeof(int32_t) * DP_STEPS, cudaMemcpyDeviceToHost, st), rc.err);
    MFBC_CUDA_TRY(cudaMemcpyAsync(koff.data(), s.soff, sizeof(uint32_t) * DP_STEPS, cudaMemcpyDeviceToHost, st),
                  rc.err);
    MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
    rc.prof->drain();
    if (hs.err) {
      if (rc.err) *rc.err = "a grid barrier of the distance kernels waited past its limit";
      return MFBC_ERR_TIMEOUT;
    }
    hd.insert(hd.end(), kd.begin(), kd.begin() + hs.k);
    hoff.insert(hoff.end(), koff.begin(), koff.begin() + hs.k);
    if (hs.stop == 1) break;
    if (hs.stop != 2 || launch >= max_launches) {
      if (rc.err) *rc.err = "distance steps did not terminate";
      return MFBC_ERR_NO_CONVERGENCE;
    }
    hs.k = 0;                                  // continue from hs.d with empty step records
    hs.stop = 0;
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
  std::vector<int32_t> bd;
  std::vector<uint32_t> boff, bcnt;
  for (int64_t i = (int64_t)hd.size() - 1; i >= 0; i--) {
    if (hd[(size_t)i] <= 0) continue;
    const uint32_t end = (size_t)i + 1 < hoff.size() ? hoff[(size_t)i + 1] : hs.off;
    bd.push_back(hd[(size_t)i]);
    boff.push_back(hoff[(size_t)i]);
    bcnt.push_back(end - hoff[(size_t)i]);
  }
  DpBwd ba{s.mlist, s.sd, s.soff, s.scnt, 0, g.rowptr, g.col, g.w, s.dist, s.sig, s.val, s.src, lam0, wreq, W, nb,
           n, s.sy, B_ ? B_ + K_DP_BWD : nullptr};
  const unsigned bgrid = dp_blocks((const void*)k_dp_bwd);
  if (!bgrid) return cuda_fail(rc.err, "occupancy of the distance kernels", cudaGetLastError());
  for (size_t c0 = 0; c0 < bd.size(); c0 += DP_STEPS) {
    const size_t c = std::min(bd.size() - c0, (size_t)DP_STEPS);
    MFBC_CUDA_TRY(cudaMemcpyAsync(s.sd, bd.data() + c0, sizeof(int32_t) * c, cudaMemcpyHostToDevice, st), rc.err);
    MFBC_CUDA_TRY(cudaMemcpyAsync(s.soff, boff.data() + c0, sizeof(uint32_t) * c, cudaMemcpyHostToDevice, st),
                  rc.err);
    MFBC_CUDA_TRY(cudaMemcpyAsync(s.scnt, bcnt.data() + c0, sizeof(uint32_t) * c, cudaMemcpyHostToDevice, st),
                  rc.err);
    ba.nsteps = (int)c;
    void* args[] = {&ba};
    cudaError_t e;
    PROF(K_DP_BWD, e = cudaLaunchCooperativeKernel((const void*)k_dp_bwd, bgrid, 256, args, 0, st));
    MFBC_CUDA_TRY(e, rc.err);
    if (bwd_iters) *bwd_iters += (int64_t)c;
  }
  MFBC_CUDA_TRY(cudaMemcpyAsync(&hs, s.sy, sizeof(DpSync), cudaMemcpyDeviceToHost, st), rc.err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
  rc.prof->drain();
  if (hs.err) {
    if (rc.err) *rc.err = "a grid barrier of the distance kernels waited past its limit";
    return MFBC_ERR_TIMEOUT;
  }
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
