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
  s.marks = c.take<uint32_t>(64);               // settled-list offsets of the queued steps
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

// Forward step at distance d over the (vertex, word) items listed in bucket
// `slot`: one warp per item, lane = column.  The items that hold pairs at
// distance d are appended to the settled list, which the backward pass
// replays.
__global__ void __launch_bounds__(256) k_dp_fwd(
    const uint32_t* __restrict__ list, const uint32_t* count_p, int32_t d, int slot, int B, int BW, int W, int nb,
    size_t bcap,
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const int32_t* __restrict__ wt,
    const int64_t* __restrict__ rpt, const int32_t* __restrict__ colt, const int32_t* __restrict__ wtt,
    int32_t* dist, double* sig, uint32_t* bflag, uint32_t* blist, uint32_t* bcount, uint32_t* mlist,
    unsigned long long* bytes) {
  const unsigned lane = lane_id();
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long nbytes = 0;               // algorithmic bytes of this lane (counting runs only)
  const uint32_t count = *count_p;             // items queued for distance d by the earlier steps
  for (uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < count; gw += nw) {
    const uint32_t item = list[gw];
    const int32_t v = (int32_t)(item / (uint32_t)W);
    const int word = (int)(item % (uint32_t)W);
    if (lane == 0) atomicAnd(&bflag[(size_t)item * BW + slot / 32], ~(1u << (slot & 31)));
    const int j = word * 32 + (int)lane;
    const size_t vj = (size_t)v * nb + j;
    const bool isM = dist[vj] == d;
    if (bytes) nbytes += 4;
    if (!__ballot_sync(0xffffffffu, isM)) continue;
    if (lane == 0) mlist[atomicAdd(&bcount[B], 1u)] = item;
    if (d > 0) {
      // sigma_bar from the final in-neighbours one arc short of d
      double acc = 0.0;
      const int64_t b = rpt[v], e = rpt[v + 1];
      for (int64_t k0 = b; k0 < e; k0 += 32) {
        const int64_t k = k0 + lane;
        const int32_t myu = k < e ? colt[k] : 0;
        const int32_t myw = k < e ? (wtt ? wtt[k] : 1) : 0;
        const int cnt = (int)(e - k0 < 32 ? e - k0 : 32);
        for (int t = 0; t < cnt; t++) {
          const int32_t u = __shfl_sync(0xffffffffu, myu, t);
          const int32_t w = __shfl_sync(0xffffffffu, myw, t);
          if (isM && w <= d) {
            const size_t uj = (size_t)u * nb + j;
            if (dist[uj] == d - w) { acc += sig[uj]; if (bytes) nbytes += 8; }
            if (bytes) nbytes += 4;
          }
        }
      }
      if (isM) { sig[vj] = acc; if (bytes) nbytes += 8; }
    }
    // candidates d + w to the out-neighbours
    const int64_t b = rp[v], e = rp[v + 1];
    for (int64_t k0 = b; k0 < e; k0 += 32) {
      const int64_t k = k0 + lane;
      const int32_t myx = k < e ? col[k] : 0;
      const int32_t myw = k < e ? (wt ? wt[k] : 1) : 0;
      const int cnt = (int)(e - k0 < 32 ? e - k0 : 32);
      for (int t = 0; t < cnt; t++) {
        const int32_t x = __shfl_sync(0xffffffffu, myx, t);
        const int32_t cand = d + __shfl_sync(0xffffffffu, myw, t);
        bool improved = false;
        if (isM) {
          int32_t* dx = &dist[(size_t)x * nb + j];
          if (cand < *dx) { improved = atomicMin(dx, cand) > cand; if (bytes) nbytes += 4; }
          if (bytes) nbytes += 4;
        }
        if (__ballot_sync(0xffffffffu, improved) && lane == 0) {
          const int s2 = cand % B;
          const uint32_t bit = 1u << (s2 & 31);
          const uint32_t xi = (uint32_t)x * (uint32_t)W + (uint32_t)word;
          if (!(atomicOr(&bflag[(size_t)xi * BW + s2 / 32], bit) & bit))
            blist[(size_t)s2 * bcap + atomicAdd(&bcount[s2], 1u)] = xi;
        }
      }
    }
  }
  if (bytes) {
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0) atomicAdd(bytes, nbytes);
  }
}

// Backward step at distance d over the (vertex, word) items settled at d.
__global__ void __launch_bounds__(256) k_dp_bwd(
    const uint32_t* __restrict__ items, uint32_t count, int32_t d, int W, int nb, int32_t n,
    const int64_t* __restrict__ rp, const int32_t* __restrict__ col, const int32_t* __restrict__ wt,
    const int32_t* __restrict__ dist, const double* __restrict__ sig, double* val, const int32_t* __restrict__ src,
    double* lambda, const int32_t* __restrict__ word_req, unsigned long long* bytes) {
  const unsigned lane = lane_id();
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long nbytes = 0;
  for (uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < count; gw += nw) {
    const uint32_t it = items[gw];
    const int32_t v = (int32_t)(it / (uint32_t)W);
    const int word = (int)(it % (uint32_t)W);
    const int r = word_req ? word_req[word] : 0;
    const int j = word * 32 + (int)lane;
    const size_t vj = (size_t)v * nb + j;
    const bool isM = dist[vj] == d;
    double acc = 0.0;
    const int64_t b = rp[v], e = rp[v + 1];
    for (int64_t k0 = b; k0 < e; k0 += 32) {
      const int64_t k = k0 + lane;
      const int32_t myx = k < e ? col[k] : 0;
      const int32_t myw = k < e ? (wt ? wt[k] : 1) : 0;
      const int cnt = (int)(e - k0 < 32 ? e - k0 : 32);
      for (int t = 0; t < cnt; t++) {
        const int32_t x = __shfl_sync(0xffffffffu, myx, t);
        const int32_t w = __shfl_sync(0xffffffffu, myw, t);
        if (isM) {
          const size_t xj = (size_t)x * nb + j;
          if (dist[xj] == d + w) { acc += val[xj]; if (bytes) nbytes += 8; }
          if (bytes) nbytes += 4;
        }
      }
    }
    double lam = 0.0;
    if (isM) {
      const double sg = sig[vj];
      if (src[j] != v) lam = acc * sg;
      val[vj] = acc + 1.0 / sg;
      if (bytes) nbytes += 20;
    }
    for (int o = 16; o; o >>= 1) lam += __shfl_xor_sync(0xffffffffu, lam, o);
    if (lane == 0 && r >= 0 && lam != 0.0) atomicAdd(&lambda[(size_t)r * n + v], lam);
  }
  if (bytes) {
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0) atomicAdd(bytes, nbytes);
  }
}

#define PROF(id, ...)             \
  do {                            \
    rc.prof->begin(id);           \
    __VA_ARGS__;                  \
    rc.prof->end(id);             \
  } while (0)

static inline unsigned dp_grid(uint64_t warps) {
  uint64_t b = (warps + 7) / 8;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
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
  });
  rc.prof->k[K_FILL].bytes += 12.0 * cells + 4.0 * s.bcap * s.BW;
  PROF(K_SEED, (k_dp_seed<<<(nb + 127) / 128, 128, 0, st>>>(s.src, nb, W, s.BW, s.dist, s.sig, s.bflag, s.blist,
                                                          s.bcount)));

  // ---- MFBF in increasing distance order.  Steps are queued without waiting:
  // each kernel reads its bucket's count on the device, and the host looks at
  // the counts once every DP_CHECK distance values (done when every bucket is
  // empty), collecting the settled list's offset at the start of each step.
  constexpr int DP_CHECK = 32;
  std::vector<uint32_t> cnt((size_t)B + 1), mk((size_t)DP_CHECK), marks;
  const int64_t max_steps = (int64_t)n * (int64_t)std::max(1, g.wmax) + DP_CHECK + 1;
  int64_t steps = 0;
  int32_t d = 0;
  while (true) {
    for (int k = 0; k < DP_CHECK; k++, d++) {
      const int slot = d % B;
      MFBC_CUDA_TRY(cudaMemcpyAsync(&s.marks[k], &s.bcount[B], sizeof(uint32_t), cudaMemcpyDeviceToDevice, st),
                    rc.err);
      PROF(K_DP_FWD, (k_dp_fwd<<<152 * 16, 256, 0, st>>>(
                         s.blist + (size_t)slot * s.bcap, &s.bcount[slot], d, slot, B, s.BW, W, nb, s.bcap,
                         g.rowptr, g.col, g.w, g.rowptr_t, g.col_t, g.w_t, s.dist, s.sig, s.bflag, s.blist,
                         s.bcount, s.mlist, B_ ? B_ + K_DP_FWD : nullptr)));
      MFBC_CUDA_TRY(cudaMemsetAsync(&s.bcount[slot], 0, sizeof(uint32_t), st), rc.err);
    }
    steps += DP_CHECK;
    MFBC_CUDA_TRY(cudaMemcpyAsync(mk.data(), s.marks, sizeof(uint32_t) * DP_CHECK, cudaMemcpyDeviceToHost, st),
                  rc.err);
    MFBC_CUDA_TRY(cudaMemcpyAsync(cnt.data(), s.bcount, sizeof(uint32_t) * cnt.size(), cudaMemcpyDeviceToHost, st),
                  rc.err);
    MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
    rc.prof->drain();
    marks.insert(marks.end(), mk.begin(), mk.end());
    bool pending = false;
    for (int k = 0; k < B; k++) pending |= cnt[(size_t)k] != 0;
    if (!pending) break;
    if (steps > max_steps) {
      if (rc.err) *rc.err = "distance steps did not terminate";
      return MFBC_ERR_NO_CONVERGENCE;
    }
  }
  marks.push_back(cnt[(size_t)B]);              // end of the last step's items
  if (fwd_iters) *fwd_iters += steps;
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
  for (int64_t dd = (int64_t)marks.size() - 2; dd >= 1; dd--) {
    const uint32_t off = marks[(size_t)dd], cntd = marks[(size_t)dd + 1] - off;
    if (!cntd) continue;
    PROF(K_DP_BWD, (k_dp_bwd<<<dp_grid(cntd), 256, 0, st>>>(
                       s.mlist + off, cntd, (int32_t)dd, W, nb, n, g.rowptr, g.col, g.w, s.dist, s.sig, s.val,
                       s.src, lam0, wreq, B_ ? B_ + K_DP_BWD : nullptr)));
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
