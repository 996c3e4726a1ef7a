// General path: MFBF (Algorithm 1) and MFBr (Algorithm 2) for any integer
// weights >= 1 over the vertex-major batch state.  A product reduces the
// candidates that meet at one (vertex, column) in one of three ways
// (MFBC_ACCUM_*): pushed from the frontier with atomics at the targets (the
// kernels right below), pulled per target row and reduced in registers
// (segmented, further down), or pushed and first combined in a per-block
// shared-memory hash table (hash, further down).
//
// Push form:
// One warp owns one (frontier vertex u, 32-column word) pair; lane l is batch
// column 32*word + l.  The warp walks u's arc list once, broadcasting 32 arcs
// at a time by shuffle, and every lane whose column is in the frontier
// applies the monoid action to its own column of the target row.  The 32
// lanes of a warp therefore always touch one contiguous 128-byte (int32) or
// 256-byte (FP64) segment of the target vertex's row.
//
// MFBF iteration i (Algorithm 1, with the readings of the seed and of the
// frontier filter listed in the design notes):
//   relax_min  product weight:  cw(s,v) = min over frontier (s,u), arcs u->v,
//              of tau_i(s,u) + A(u,v)      [the (+) of the multpath monoid,
//              Sec. 4.1.1, applied to f(a,w) = (a.w + w, a.m), Sec. 4.1.2];
//              candidates heavier than the current T(s,v).w cannot survive the
//              filter and are not offered;
//   relax_tie  product multiplicity: cm(s,v) = sum of frontier multiplicities
//              over the arcs that attain cw(s,v) (ties summed);
//   accumulate T := T (+) product; the new frontier keeps every product entry
//              whose weight equals the accumulated weight, carrying the
//              product's multiplicity (the increment).
// MFBr (Algorithm 2):
//   counters_leaves  Z(s,v).c = number of successors u of v on shortest paths
//              (arcs v->u with tau(s,u) = tau(s,v) + A(v,u)); leaves (c = 0)
//              form the first frontier with value 1/sigma_bar(s,v);
//   propagate  push over A^T: each frontier (s,u) adds its value to Z(s,v).p of
//              every predecessor v (the Brandes action g(a,w) = (a.w - w, a.p,
//              a.c) keeps exactly those v with tau(s,v) = tau(s,u) - A(v,u)) and
//              decrements Z(s,v).c; the lane that takes a counter to zero
//              enqueues (s,v) -- exactly once, so no retirement pass is needed;
//   next_frontier  value of a new frontier entry: Z(s,v).p + 1/sigma_bar(s,v).
// lambda (Algorithm 3): lambda(v) += sum_j zeta(src_j, v) * sigma_bar(src_j, v)
//   over active columns with src_j != v.
#include "internal.cuh"

namespace mfbc {

size_t general_bytes(int32_t n, int nb) {
  Carver c(nullptr, 0);
  GeneralState s;
  general_carve(c, n, nb, s);
  return c.off;
}

void general_carve(Carver& c, int32_t n, int nb, GeneralState& s) {
  size_t cells = (size_t)n * nb;
  s.nb = nb;
  s.W = nb / 32;
  s.dist = c.take<int32_t>(cells);
  s.sig = c.take<double>(cells);
  s.cw = c.take<int32_t>(cells);
  s.cm = c.take<double>(cells);
  s.fm = c.take<double>(cells);
  s.fmask = c.take<uint32_t>((size_t)n * s.W);
  s.tmask = c.take<uint32_t>((size_t)n * s.W);
  s.vflag = c.take<uint32_t>((size_t)n);
  s.fmem = c.take<uint32_t>(((size_t)n + 31) / 32);
  s.listA = c.take<int32_t>((size_t)n);
  s.listB = c.take<int32_t>((size_t)n);
  s.src = c.take<int32_t>((size_t)nb);
  s.word_req = c.take<int32_t>((size_t)s.W);
  s.ctr = c.take<Counters>(1);
}

// ---------------------------------------------------------------- kernels
__device__ __forceinline__ void enqueue_once(uint32_t* vflag, int32_t* list, uint32_t* count,
                                             int32_t v) {
  if (*((volatile uint32_t*)&vflag[v]) == 0 && atomicExch(&vflag[v], 1u) == 0u)
    list[atomicAdd(count, 1u)] = v;
}

// The arc kernels come in two widths: ARCS = 8 walks a row's arcs eight at a
// time with their loads issued together (rows of high-degree graphs), ARCS =
// 1 one at a time (rows of a few arcs, e.g. grids, where the batching costs
// more than it hides); the host picks by the average degree.
//
// Per-warp append buffer (shared memory, 40 entries): vertices to add to a
// list are gathered and written 32 at a time with one atomic on the list
// counter (a single counter shared by all warps is an L2 hot spot).
__device__ __forceinline__ void wl_push(int32_t* buf, int& n, bool mine, int32_t v, int32_t* list,
                                        uint32_t* count) {
  const unsigned lane = lane_id();
  const uint32_t m = __ballot_sync(0xffffffffu, mine);
  if (mine) buf[n + __popc(m & ((1u << lane) - 1u))] = v;
  n += __popc(m);
  __syncwarp();
  if (n >= 32) {
    uint32_t b = 0;
    if (lane == 0) b = atomicAdd(count, 32u);
    b = __shfl_sync(0xffffffffu, b, 0);
    list[b + lane] = buf[lane];
    __syncwarp();
    if ((int)lane < n - 32) buf[lane] = buf[32 + lane];
    __syncwarp();
    n -= 32;
  }
}
__device__ __forceinline__ void wl_flush(int32_t* buf, int n, int32_t* list, uint32_t* count) {
  if (!n) return;
  uint32_t b = 0;
  if (lane_id() == 0) b = atomicAdd(count, (uint32_t)n);
  b = __shfl_sync(0xffffffffu, b, 0);
  if ((int)lane_id() < n) list[b + lane_id()] = buf[lane_id()];
}
// true for the caller that first flags v (exactly one caller per vertex)
__device__ __forceinline__ bool claim_vertex(uint32_t* vflag, int32_t v) {
  return *((volatile uint32_t*)&vflag[v]) == 0 && atomicExch(&vflag[v], 1u) == 0u;
}

// Seed (Algorithm 1 start, read as T(s,s) = (0,1), frontier {(s,s)}).
__global__ void k_gp_seed(const int32_t* __restrict__ src, int nb, int W, int32_t* dist, double* sig,
                          double* fm, uint32_t* fmask, uint32_t* fmem, uint32_t* vflag, int32_t* list,
                          uint32_t* count) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  int32_t s = src[j];
  if (s < 0) return;
  size_t idx = (size_t)s * nb + j;
  dist[idx] = 0;
  sig[idx] = 1.0;
  fm[idx] = 1.0;
  atomicOr(&fmask[(size_t)s * W + (j >> 5)], 1u << (j & 31));
  atomicOr(&fmem[s >> 5], 1u << (s & 31));
  enqueue_once(vflag, list, count, s);
}

__global__ void k_clear_flags(const int32_t* __restrict__ list, uint32_t count, uint32_t* vflag) {
  uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) vflag[list[i]] = 0;
}

// MFBF product, phase 1: minimum candidate weight per (s, v).  One warp per
// (frontier vertex u, 32-column word); the arcs of u are walked ARCS at a
// time.
template <int ARCS>
__global__ void __launch_bounds__(256, ARCS > 1 ? 4 : 8) k_gp_relax_min(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ wt,
    const int32_t* __restrict__ flist, uint32_t fcount, int W, int nb,
    const uint32_t* __restrict__ fmask, const int32_t* __restrict__ dist, int32_t* cw, uint32_t* tmask,
    uint32_t* vflag, int32_t* tlist, uint32_t* tcount, unsigned long long* bytes, int64_t min_arcs) {
  __shared__ int32_t qbuf[8][40];
  int32_t* q = qbuf[threadIdx.x >> 5];
  uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= (uint64_t)fcount * W) return;
  const unsigned lane = lane_id();
  const int word = (int)(gw % W);
  const int32_t u = flist[gw / W];
  const uint32_t m = fmask[(size_t)u * W + word];
  if (!m) return;
  const int j = word * 32 + lane;
  const bool active = (m >> lane) & 1u;
  const int64_t beg = rowptr[u], end = rowptr[u + 1];
  if (end - beg < min_arcs) return;              // short rows: the hash kernels' share
  const int32_t du = active ? dist[(size_t)u * nb + j] : 0;
  unsigned long long nb_bytes = 0;
  int qn = 0;
  for (int64_t k0 = beg; k0 < end; k0 += 32) {
    const int64_t k = k0 + lane;
    const int32_t myv = k < end ? col[k] : 0;
    const int32_t myw = k < end ? (wt ? wt[k] : 1) : 0;
    const int cnt = (int)(end - k0 < 32 ? end - k0 : 32);
    for (int t0 = 0; t0 < cnt; t0 += ARCS) {
      int32_t v8[ARCS], w8[ARCS], d8[ARCS], c8[ARCS];
#pragma unroll
      for (int r = 0; r < ARCS; r++) {
        v8[r] = __shfl_sync(0xffffffffu, myv, (t0 + r) & 31);
        w8[r] = __shfl_sync(0xffffffffu, myw, (t0 + r) & 31);
      }
#pragma unroll
      for (int r = 0; r < ARCS; r++) {
        d8[r] = 0;
        c8[r] = 0;
        if (active && t0 + r < cnt) {
          const size_t idx = (size_t)v8[r] * nb + j;
          d8[r] = __ldg(&dist[idx]);
          c8[r] = cw[idx];
        }
      }
      bool mine = false;
      int32_t mv = 0;
#pragma unroll
      for (int r = 0; r < ARCS; r++) {
        if (t0 + r < cnt) {
          const int32_t cand = du + w8[r];
          const bool touch = active && cand <= d8[r];
          if (touch && cand < c8[r]) atomicMin(&cw[(size_t)v8[r] * nb + j], cand);
          const uint32_t tb = __ballot_sync(0xffffffffu, touch);
          if (tb && (int)lane == r) {
            atomicOr(&tmask[(size_t)v8[r] * W + word], tb);
            if (claim_vertex(vflag, v8[r])) { mine = true; mv = v8[r]; }
          }
          if (bytes) nb_bytes += 4ull * __popc(m) + 8ull * __popc(tb);
        }
      }
      if constexpr (ARCS == 1) {
        if (mine) tlist[atomicAdd(tcount, 1u)] = mv;
      } else {
        wl_push(q, qn, mine, mv, tlist, tcount);
      }
    }
  }
  if constexpr (ARCS > 1) wl_flush(q, qn, tlist, tcount);
  if (bytes && lane == 0) atomicAdd(bytes, nb_bytes + 8ull * (end - beg) / W + 4ull * __popc(m));
}

// MFBF product, phase 2: sum the frontier multiplicities that attain the minimum.
template <int ARCS>
__global__ void __launch_bounds__(256, ARCS > 1 ? 4 : 8) k_gp_relax_tie(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ wt,
    const int32_t* __restrict__ flist, uint32_t fcount, int W, int nb,
    const uint32_t* __restrict__ fmask, const int32_t* __restrict__ dist, const double* __restrict__ fm,
    const int32_t* __restrict__ cw, double* cm, unsigned long long* bytes, int64_t min_arcs) {
  uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= (uint64_t)fcount * W) return;
  const unsigned lane = lane_id();
  const int word = (int)(gw % W);
  const int32_t u = flist[gw / W];
  const uint32_t m = fmask[(size_t)u * W + word];
  if (!m) return;
  const int j = word * 32 + lane;
  const bool active = (m >> lane) & 1u;
  const int64_t beg = rowptr[u], end = rowptr[u + 1];
  if (end - beg < min_arcs) return;
  const int32_t du = active ? dist[(size_t)u * nb + j] : 0;
  const double mu = active ? fm[(size_t)u * nb + j] : 0.0;
  unsigned long long nb_bytes = 0;
  for (int64_t k0 = beg; k0 < end; k0 += 32) {
    const int64_t k = k0 + lane;
    const int32_t myv = k < end ? col[k] : 0;
    const int32_t myw = k < end ? (wt ? wt[k] : 1) : 0;
    const int cnt = (int)(end - k0 < 32 ? end - k0 : 32);
    for (int t0 = 0; t0 < cnt; t0 += ARCS) {
      int32_t v8[ARCS], w8[ARCS], c8[ARCS];
#pragma unroll
      for (int r = 0; r < ARCS; r++) {
        v8[r] = __shfl_sync(0xffffffffu, myv, (t0 + r) & 31);
        w8[r] = __shfl_sync(0xffffffffu, myw, (t0 + r) & 31);
      }
#pragma unroll
      for (int r = 0; r < ARCS; r++)
        c8[r] = (active && t0 + r < cnt) ? __ldg(&cw[(size_t)v8[r] * nb + j]) : -1;
#pragma unroll
      for (int r = 0; r < ARCS; r++) {
        if (t0 + r < cnt) {
          const bool hit = active && du + w8[r] == c8[r];
          if (hit) atomicAdd(&cm[(size_t)v8[r] * nb + j], mu);
          if (bytes) nb_bytes += 4ull * __popc(m) + 16ull * __popc(__ballot_sync(0xffffffffu, hit));
        }
      }
    }
  }
  if (bytes && lane == 0) atomicAdd(bytes, nb_bytes + 8ull * (end - beg) / W + 12ull * __popc(m));
}

// Zero the frontier rows of the listed vertices and their membership bits.
__global__ void k_clear_mask_rows(const int32_t* __restrict__ list, uint32_t count, int W, uint32_t* mask,
                                  uint32_t* mem) {
  uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (uint64_t)count * W) return;
  const int32_t v = list[i / W];
  mask[(size_t)v * W + (i % W)] = 0u;
  if (mem && i % W == 0) atomicAnd(&mem[v >> 5], ~(1u << (v & 31)));
}

// T := T (+) product, frontier filter, compaction of the next frontier.
__global__ void __launch_bounds__(256) k_gp_accumulate(
    const int32_t* __restrict__ tlist, const uint32_t* tcount_p, int W, int nb, int32_t* dist,
    double* sig, int32_t* cw, double* cm, double* fm, uint32_t* fmask, uint32_t* tmask, uint32_t* vflag,
    uint32_t* fmem, int32_t* nlist, uint32_t* ncount, unsigned long long* bytes) {
  __shared__ int32_t qbuf[8][40];
  int32_t* q = qbuf[threadIdx.x >> 5];
  int qn = 0;
  const uint32_t tcount = *tcount_p;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < tcount; gw += nw) {
  const unsigned lane = lane_id();
  const int32_t v = tlist[gw];
  bool any = false;
  unsigned long long nbytes = 0;
  for (int word = 0; word < W; word++) {
    const size_t mi = (size_t)v * W + word;
    const uint32_t t = tmask[mi];
    if (!t) continue;
    const bool on = (t >> lane) & 1u;
    bool keep = false;
    if (on) {
      const size_t idx = (size_t)v * nb + word * 32 + lane;
      const int32_t c = cw[idx], d = dist[idx];
      const double mm = cm[idx];
      if (c < d) { dist[idx] = c; sig[idx] = mm; keep = true; }
      else if (c == d) { sig[idx] += mm; keep = true; }
      if (keep) fm[idx] = mm;
      cw[idx] = INF;
      cm[idx] = 0.0;
    }
    const uint32_t kb = __ballot_sync(0xffffffffu, keep);
    if (lane == 0) { fmask[mi] = kb; tmask[mi] = 0u; }
    any |= (kb != 0u);
    nbytes += 8ull + 48ull * __popc(t);
  }
  if (lane == 0) {
    vflag[v] = 0u;
    if (any) atomicOr(&fmem[v >> 5], 1u << (v & 31));
    if (bytes) atomicAdd(bytes, nbytes + 8ull);
  }
  wl_push(q, qn, lane == 0 && any, v, nlist, ncount);
  }
  wl_flush(q, qn, nlist, ncount);
}

// Algorithm 2 initialisation: successor counters and the leaf frontier.
template <int ARCS>
__global__ void __launch_bounds__(256, ARCS > 1 ? 4 : 6) k_gp_counters(
    int32_t n, const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const int32_t* __restrict__ wt, int W, int nb, const int32_t* __restrict__ src,
    const int32_t* __restrict__ dist, const double* __restrict__ sig, int32_t* cnt, double* zp, double* fv,
    uint32_t* fmask, uint32_t* fmem, int32_t* flist, uint32_t* fcount, unsigned long long* bytes) {
  uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= (uint64_t)n) return;
  const unsigned lane = lane_id();
  const int32_t v = (int32_t)gw;
  const int64_t beg = rowptr[v], end = rowptr[v + 1];
  bool any = false;
  unsigned long long nbytes = 0;
  for (int word = 0; word < W; word++) {
    const int j = word * 32 + lane;
    const size_t idx = (size_t)v * nb + j;
    const double sv = sig[idx];
    const bool reach = (src[j] >= 0) && (sv > 0.0);
    const uint32_t rb = __ballot_sync(0xffffffffu, reach);
    if (!rb) continue;
    const int32_t dv = reach ? dist[idx] : 0;
    int32_t c = 0;
    for (int64_t k0 = beg; k0 < end; k0 += 32) {
      const int64_t k = k0 + lane;
      const int32_t myu = k < end ? col[k] : 0;
      const int32_t myw = k < end ? (wt ? wt[k] : 1) : 0;
      const int cntk = (int)(end - k0 < 32 ? end - k0 : 32);
      for (int t0 = 0; t0 < cntk; t0 += ARCS) {
        int32_t u8[ARCS], w8[ARCS], d8[ARCS];
#pragma unroll
        for (int r = 0; r < ARCS; r++) {
          u8[r] = __shfl_sync(0xffffffffu, myu, (t0 + r) & 31);
          w8[r] = __shfl_sync(0xffffffffu, myw, (t0 + r) & 31);
        }
#pragma unroll
        for (int r = 0; r < ARCS; r++)
          d8[r] = (reach && t0 + r < cntk) ? __ldg(&dist[(size_t)u8[r] * nb + j]) : -1;
#pragma unroll
        for (int r = 0; r < ARCS; r++)
          if (t0 + r < cntk && d8[r] == dv + w8[r]) c++;
      }
    }
    if (reach) {
      cnt[idx] = c;
      zp[idx] = 0.0;
      if (c == 0) fv[idx] = 1.0 / sv;
    }
    const uint32_t lb = __ballot_sync(0xffffffffu, reach && c == 0);
    if (lane == 0) fmask[(size_t)v * W + word] = lb;
    any |= (lb != 0u);
    nbytes += 4ull * __popc(rb) * (end - beg) + 24ull * __popc(rb);
  }
  if (lane == 0) {
    if (any) {
      flist[atomicAdd(fcount, 1u)] = v;
      atomicOr(&fmem[v >> 5], 1u << (v & 31));
    }
    if (bytes) atomicAdd(bytes, nbytes + 8ull * (end - beg));
  }
}

// MFBr product over A^T with counter decrement and exactly-once enqueue.
template <int ARCS>
__global__ void __launch_bounds__(256, ARCS > 1 ? 4 : 6) k_gp_propagate(
    const int64_t* __restrict__ rowptr_t, const int32_t* __restrict__ col_t,
    const int32_t* __restrict__ wt_t, const int32_t* __restrict__ flist, uint32_t fcount, int W, int nb,
    const uint32_t* __restrict__ fmask, const int32_t* __restrict__ dist, const double* __restrict__ fv,
    double* zp, int32_t* cnt, uint32_t* tmask, uint32_t* vflag, int32_t* tlist, uint32_t* tcount,
    unsigned long long* bytes, int64_t min_arcs) {
  __shared__ int32_t qbuf[8][40];
  int32_t* q = qbuf[threadIdx.x >> 5];
  int qn = 0;
  uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= (uint64_t)fcount * W) return;
  const unsigned lane = lane_id();
  const int word = (int)(gw % W);
  const int32_t u = flist[gw / W];
  const uint32_t m = fmask[(size_t)u * W + word];
  if (!m) return;
  const int j = word * 32 + lane;
  const bool active = (m >> lane) & 1u;
  const int64_t beg = rowptr_t[u], end = rowptr_t[u + 1];
  if (end - beg < min_arcs) return;
  const int32_t du = active ? dist[(size_t)u * nb + j] : 0;
  const double val = active ? fv[(size_t)u * nb + j] : 0.0;
  unsigned long long nb_bytes = 0;
  for (int64_t k0 = beg; k0 < end; k0 += 32) {
    const int64_t k = k0 + lane;
    const int32_t myv = k < end ? col_t[k] : 0;
    const int32_t myw = k < end ? (wt_t ? wt_t[k] : 1) : 0;
    const int cntk = (int)(end - k0 < 32 ? end - k0 : 32);
    for (int t0 = 0; t0 < cntk; t0 += ARCS) {
      int32_t v8[ARCS], w8[ARCS], d8[ARCS], o8[ARCS];
#pragma unroll
      for (int r = 0; r < ARCS; r++) {
        v8[r] = __shfl_sync(0xffffffffu, myv, (t0 + r) & 31);
        w8[r] = __shfl_sync(0xffffffffu, myw, (t0 + r) & 31);
      }
#pragma unroll
      for (int r = 0; r < ARCS; r++)
        d8[r] = (active && t0 + r < cntk) ? __ldg(&dist[(size_t)v8[r] * nb + j]) : INT32_MIN;
#pragma unroll
      for (int r = 0; r < ARCS; r++) {
        o8[r] = 0;
        if (t0 + r < cntk && d8[r] == du - w8[r]) {
          const size_t idx = (size_t)v8[r] * nb + j;
          atomicAdd(&zp[idx], val);
          o8[r] = atomicSub(&cnt[idx], 1);
        }
      }
      bool mine = false;
      int32_t mv = 0;
#pragma unroll
      for (int r = 0; r < ARCS; r++) {
        if (t0 + r < cntk) {
          const uint32_t rb = __ballot_sync(0xffffffffu, o8[r] == 1);
          if (rb && (int)lane == r) {
            atomicOr(&tmask[(size_t)v8[r] * W + word], rb);
            if (claim_vertex(vflag, v8[r])) { mine = true; mv = v8[r]; }
          }
          if (bytes) nb_bytes += 4ull * __popc(m) + 24ull * __popc(__ballot_sync(0xffffffffu, d8[r] == du - w8[r]));
        }
      }
      if constexpr (ARCS == 1) {
        if (mine) tlist[atomicAdd(tcount, 1u)] = mv;
      } else {
        wl_push(q, qn, mine, mv, tlist, tcount);
      }
    }
  }
  if constexpr (ARCS > 1) wl_flush(q, qn, tlist, tcount);
  if (bytes && lane == 0) atomicAdd(bytes, nb_bytes + 8ull * (end - beg) / W + 16ull * __popc(m));
}

// New MFBr frontier entries: value Z.p + 1/sigma_bar.
__global__ void __launch_bounds__(256) k_gp_next_frontier(
    const int32_t* __restrict__ tlist, const uint32_t* tcount_p, int W, int nb,
    const double* __restrict__ sig, const double* __restrict__ zp, double* fv, uint32_t* fmask,
    uint32_t* tmask, uint32_t* vflag, uint32_t* fmem, int32_t* nlist, uint32_t* ncount, unsigned long long* bytes) {
  __shared__ int32_t qbuf[8][40];
  int32_t* q = qbuf[threadIdx.x >> 5];
  int qn = 0;
  const uint32_t tcount = *tcount_p;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; gw < tcount; gw += nw) {
  const unsigned lane = lane_id();
  const int32_t v = tlist[gw];
  unsigned long long nbytes = 0;
  for (int word = 0; word < W; word++) {
    const size_t mi = (size_t)v * W + word;
    const uint32_t r = tmask[mi];
    if (!r) continue;
    if ((r >> lane) & 1u) {
      const size_t idx = (size_t)v * nb + word * 32 + lane;
      fv[idx] = zp[idx] + 1.0 / sig[idx];
    }
    if (lane == 0) { fmask[mi] = r; tmask[mi] = 0u; }
    nbytes += 8ull + 24ull * __popc(r);
  }
  if (lane == 0) {
    vflag[v] = 0u;
    atomicOr(&fmem[v >> 5], 1u << (v & 31));
    if (bytes) atomicAdd(bytes, nbytes);
  }
  wl_push(q, qn, lane == 0, v, nlist, ncount);
  }
  wl_flush(q, qn, nlist, ncount);
}

// Algorithm 3 accumulation, one warp per vertex, no atomics.
// word_req: request (lambda row) of each 32-column word, or nullptr when the
// whole batch adds into row 0.
__global__ void __launch_bounds__(256) k_gp_lambda(int32_t n, int W, int nb, const int32_t* __restrict__ src,
                                                   const double* __restrict__ zp,
                                                   const double* __restrict__ sig, double* lambda,
                                                   const int32_t* __restrict__ word_req) {
  uint64_t gw = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gw >= (uint64_t)n) return;
  const unsigned lane = lane_id();
  const int32_t v = (int32_t)gw;
  double acc = 0.0;
  int cur = word_req ? -1 : 0;
  for (int word = 0; word < W; word++) {
    if (word_req) {
      const int r = word_req[word];
      if (r != cur) {                          // a new request's words begin: flush the previous one
        for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0 && cur >= 0) lambda[(size_t)cur * n + v] += acc;
        acc = 0.0;
        cur = r;
      }
      if (r < 0) continue;
    }
    const int j = word * 32 + lane;
    const size_t idx = (size_t)v * nb + j;
    const int32_t s = src[j];
    const double sg = sig[idx];
    if (s >= 0 && s != v && sg > 0.0) acc += zp[idx] * sg;
  }
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0 && cur >= 0) lambda[(size_t)cur * n + v] += acc;
}

// ---------------------------------------------------------- hash accumulator
// The push products above, with the reduction at the targets done first in
// shared memory.  A block takes 8 * HASH_ITEMS (frontier vertex, word) items,
// ordered word-major, so its warps work on the same 32 columns of different
// frontier vertices.  Candidates for a hot target (a vertex of high in-degree
// for MFBF, out-degree for MFBr: where many frontier vertices meet) go to the
// slot of the key (target, word) in the block's open-addressing table
// (HASH_PROBES linear probes); each lane reduces its own column there with
// shared-memory atomics.  Once the block's arcs are walked, every occupied
// slot is merged into the batch state with one global operation per column,
// so the global atomics at a hub column fall from one per arc to one per
// block.  Other targets, and keys that find no free slot, take the atomic
// path unchanged.  The reductions are the monoid's own (minimum; sums of
// integer multiplicities, exact in FP64 in any order; sums of MFBr values,
// whose order only rounds), so the results are those of the atomic path.
constexpr int HASH_SLOTS = 128;      // keys per block (a power of two)
constexpr int HASH_PROBES = 8;
constexpr int HASH_ITEMS = 4;        // (frontier vertex, word) items per warp
constexpr int HASH_ROW_MAX = 128;    // longer frontier rows go to the atomic kernels: a block
                                     // waits at its barrier for its longest row
constexpr unsigned long long HASH_EMPTY = ~0ull;

struct HashSmem {
  unsigned long long key[HASH_SLOTS];  // (vertex * W + word) or HASH_EMPTY
  int32_t mn[HASH_SLOTS][32];          // MFBF: the block's minimum candidate; MFBr: its tight-arc count
  double sum[HASH_SLOTS][32];          // MFBF ties: multiplicity sum (as uint64); MFBr: value sum
  uint32_t take[HASH_SLOTS];           // MFBF ties: columns whose block minimum is the product's
  int32_t q[8][40];                    // per-warp list append buffers
};

__device__ __forceinline__ bool hot_bit(const uint32_t* __restrict__ bits, int32_t v) {
  return (__ldg(&bits[v >> 5]) >> (v & 31)) & 1u;
}
__device__ __forceinline__ uint32_t hash_home(unsigned long long key) {
  return (uint32_t)((key * 0x9E3779B97F4A7C15ull) >> 57) & (HASH_SLOTS - 1);   // Fibonacci hashing, 7 bits
}
// slot of key, inserting it when absent; -1 when its probes find no room
__device__ __forceinline__ int hash_insert(unsigned long long* keys, unsigned long long key) {
  const uint32_t h = hash_home(key);
  for (int p = 0; p < HASH_PROBES; p++) {
    const int s = (int)((h + (uint32_t)p) & (HASH_SLOTS - 1));
    unsigned long long k = *((volatile unsigned long long*)&keys[s]);
    if (k == HASH_EMPTY) k = atomicCAS(&keys[s], HASH_EMPTY, key);
    if (k == HASH_EMPTY || k == key) return s;
  }
  return -1;
}
// slot of key in a table no longer written; -1 when absent
__device__ __forceinline__ int hash_find(const unsigned long long* keys, unsigned long long key) {
  const uint32_t h = hash_home(key);
  for (int p = 0; p < HASH_PROBES; p++) {
    const int s = (int)((h + (uint32_t)p) & (HASH_SLOTS - 1));
    const unsigned long long k = keys[s];
    if (k == key) return s;
    if (k == HASH_EMPTY) return -1;
  }
  return -1;
}

__device__ __forceinline__ void hash_clear(HashSmem& hs, int32_t mn0) {
  for (int i = threadIdx.x; i < HASH_SLOTS; i += blockDim.x) {
    hs.key[i] = HASH_EMPTY;
    hs.take[i] = 0u;
  }
  for (int i = threadIdx.x; i < HASH_SLOTS * 32; i += blockDim.x) {
    (&hs.mn[0][0])[i] = mn0;
    (&hs.sum[0][0])[i] = 0.0;
  }
}

// The item of warp `warp`, step `it` of this block: word-major order.
__device__ __forceinline__ bool hash_item(uint32_t fcount, int W, int it, uint64_t* i_out) {
  const uint64_t i = ((uint64_t)blockIdx.x * HASH_ITEMS + (uint64_t)it) * 8 + (threadIdx.x >> 5);
  *i_out = i;
  return i < (uint64_t)fcount * W;
}

// Slots of the arcs t0 .. t0+ARCS-1 of the current 32-arc chunk (lane t holds
// arc t): the arc's own lane looks its key up when `want` is set for it.
template <int ARCS>
__device__ __forceinline__ void hash_slots(HashSmem& hs, bool insert, int t0, int cnt, int32_t myv, int W, int word,
                                           const uint32_t* __restrict__ hot, uint32_t want, int (&s8)[ARCS]) {
  const int lane = (int)lane_id();
  const int r = lane - t0;
  int slot = -1;
  if (r >= 0 && r < ARCS && lane < cnt && ((want >> r) & 1u) && hot_bit(hot, myv)) {
    const unsigned long long key = (unsigned long long)myv * (unsigned)W + (unsigned)word;
    slot = insert ? hash_insert(hs.key, key) : hash_find(hs.key, key);
  }
#pragma unroll
  for (int k = 0; k < ARCS; k++) s8[k] = __shfl_sync(0xffffffffu, slot, (t0 + k) & 31);
}

// MFBF product, phase 1 (minimum candidate per (s, v)), hash form.
template <int ARCS>
__global__ void __launch_bounds__(256, 4) k_gp_hash_min(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ wt,
    const uint32_t* __restrict__ hot, const int32_t* __restrict__ flist, uint32_t fcount, int W, int nb,
    const uint32_t* __restrict__ fmask, const int32_t* __restrict__ dist, int32_t* cw, uint32_t* tmask,
    uint32_t* vflag, int32_t* tlist, uint32_t* tcount, unsigned long long* bytes) {
  extern __shared__ __align__(16) unsigned char hash_raw[];
  HashSmem& hs = *reinterpret_cast<HashSmem*>(hash_raw);
  const unsigned lane = lane_id();
  int32_t* q = hs.q[threadIdx.x >> 5];
  int qn = 0;
  unsigned long long nbytes = 0;
  hash_clear(hs, INF);
  __syncthreads();
  for (int it = 0; it < HASH_ITEMS; it++) {
    uint64_t i;
    if (!hash_item(fcount, W, it, &i)) break;
    const int word = (int)(i / fcount);
    const int32_t u = flist[i % fcount];
    const uint32_t m = fmask[(size_t)u * W + word];
    if (!m) continue;
    const int j = word * 32 + (int)lane;
    const bool active = (m >> lane) & 1u;
    const int32_t du = active ? dist[(size_t)u * nb + j] : 0;
    const int64_t beg = rowptr[u], end = rowptr[u + 1];
    if (end - beg > HASH_ROW_MAX) continue;
    for (int64_t k0 = beg; k0 < end; k0 += 32) {
      const int64_t k = k0 + lane;
      const int32_t myv = k < end ? col[k] : 0;
      const int32_t myw = k < end ? (wt ? wt[k] : 1) : 0;
      const int cnt = (int)(end - k0 < 32 ? end - k0 : 32);
      for (int t0 = 0; t0 < cnt; t0 += ARCS) {
        int32_t v8[ARCS], w8[ARCS], d8[ARCS], c8[ARCS];
        int s8[ARCS];
        hash_slots<ARCS>(hs, true, t0, cnt, myv, W, word, hot, 0xffffffffu, s8);
#pragma unroll
        for (int r = 0; r < ARCS; r++) {
          v8[r] = __shfl_sync(0xffffffffu, myv, (t0 + r) & 31);
          w8[r] = __shfl_sync(0xffffffffu, myw, (t0 + r) & 31);
        }
#pragma unroll
        for (int r = 0; r < ARCS; r++) {
          d8[r] = 0;
          c8[r] = 0;
          if (active && t0 + r < cnt && s8[r] < 0) {
            const size_t idx = (size_t)v8[r] * nb + j;
            d8[r] = __ldg(&dist[idx]);
            c8[r] = cw[idx];
          }
        }
        bool mine = false;
        int32_t mv = 0;
#pragma unroll
        for (int r = 0; r < ARCS; r++) {
          if (t0 + r < cnt) {
            const int32_t cand = du + w8[r];
            if (s8[r] >= 0) {
              if (active) atomicMin(&hs.mn[s8[r]][lane], cand);
            } else {
              const bool touch = active && cand <= d8[r];
              if (touch && cand < c8[r]) atomicMin(&cw[(size_t)v8[r] * nb + j], cand);
              const uint32_t tb = __ballot_sync(0xffffffffu, touch);
              if (tb && (int)lane == r) {
                atomicOr(&tmask[(size_t)v8[r] * W + word], tb);
                if (claim_vertex(vflag, v8[r])) { mine = true; mv = v8[r]; }
              }
              if (bytes) nbytes += 4ull * __popc(m) + 8ull * __popc(tb);
            }
          }
        }
        wl_push(q, qn, mine, mv, tlist, tcount);
      }
    }
    if (bytes) nbytes += 8ull * (end - beg) / W + 4ull * __popc(m) + 4ull;
  }
  __syncthreads();
  // merge: one warp per slot, one lane per column
  for (int sl = (int)(threadIdx.x >> 5); sl < HASH_SLOTS; sl += 8) {
    const unsigned long long key = hs.key[sl];
    if (key == HASH_EMPTY) continue;
    const int32_t v = (int32_t)(key / (unsigned)W);
    const int word = (int)(key % (unsigned)W);
    const int32_t mn = hs.mn[sl][lane];
    bool touch = false;
    if (mn != INF) {
      const size_t idx = (size_t)v * nb + word * 32 + lane;
      touch = mn <= dist[idx];
      if (touch && mn < cw[idx]) atomicMin(&cw[idx], mn);
    }
    const uint32_t tb = __ballot_sync(0xffffffffu, touch);
    bool mine = false;
    if (tb && lane == 0) {
      atomicOr(&tmask[(size_t)v * W + word], tb);
      mine = claim_vertex(vflag, v);
    }
    wl_push(q, qn, mine, v, tlist, tcount);
    if (bytes) nbytes += 12ull * __popc(__ballot_sync(0xffffffffu, mn != INF));
  }
  wl_flush(q, qn, tlist, tcount);
  if (bytes && lane == 0) atomicAdd(bytes, nbytes);
}

// MFBF product, phase 2 (sum of the multiplicities that attain the minimum),
// hash form: the block first finds its own minimum per slot and column
// (shared memory only), keeps the columns where it equals the product's
// minimum cw, then sums the frontier multiplicities of the candidates that
// attain it and adds each slot column to cm once.
template <int ARCS>
__global__ void __launch_bounds__(256, 4) k_gp_hash_tie(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ wt,
    const uint32_t* __restrict__ hot, const int32_t* __restrict__ flist, uint32_t fcount, int W, int nb,
    const uint32_t* __restrict__ fmask, const int32_t* __restrict__ dist, const double* __restrict__ fm,
    const int32_t* __restrict__ cw, double* cm, unsigned long long* bytes) {
  extern __shared__ __align__(16) unsigned char hash_raw[];
  HashSmem& hs = *reinterpret_cast<HashSmem*>(hash_raw);
  const unsigned lane = lane_id();
  unsigned long long nbytes = 0;
  hash_clear(hs, INF);
  __syncthreads();
  for (int pass = 0; pass < 2; pass++) {
    for (int it = 0; it < HASH_ITEMS; it++) {
      uint64_t i;
      if (!hash_item(fcount, W, it, &i)) break;
      const int word = (int)(i / fcount);
      const int32_t u = flist[i % fcount];
      const uint32_t m = fmask[(size_t)u * W + word];
      if (!m) continue;
      const int j = word * 32 + (int)lane;
      const bool active = (m >> lane) & 1u;
      const int32_t du = active ? dist[(size_t)u * nb + j] : 0;
      const double mu = (pass == 1 && active) ? fm[(size_t)u * nb + j] : 0.0;
      const int64_t beg = rowptr[u], end = rowptr[u + 1];
      if (end - beg > HASH_ROW_MAX) continue;
      for (int64_t k0 = beg; k0 < end; k0 += 32) {
        const int64_t k = k0 + lane;
        const int32_t myv = k < end ? col[k] : 0;
        const int32_t myw = k < end ? (wt ? wt[k] : 1) : 0;
        const int cnt = (int)(end - k0 < 32 ? end - k0 : 32);
        for (int t0 = 0; t0 < cnt; t0 += ARCS) {
          int32_t v8[ARCS], w8[ARCS], c8[ARCS];
          int s8[ARCS];
          hash_slots<ARCS>(hs, pass == 0, t0, cnt, myv, W, word, hot, 0xffffffffu, s8);
#pragma unroll
          for (int r = 0; r < ARCS; r++) {
            v8[r] = __shfl_sync(0xffffffffu, myv, (t0 + r) & 31);
            w8[r] = __shfl_sync(0xffffffffu, myw, (t0 + r) & 31);
          }
          if (pass == 0) {
#pragma unroll
            for (int r = 0; r < ARCS; r++)
              if (t0 + r < cnt && s8[r] >= 0 && active) atomicMin(&hs.mn[s8[r]][lane], du + w8[r]);
            continue;
          }
#pragma unroll
          for (int r = 0; r < ARCS; r++)
            c8[r] = (active && t0 + r < cnt && s8[r] < 0) ? __ldg(&cw[(size_t)v8[r] * nb + j]) : -1;
#pragma unroll
          for (int r = 0; r < ARCS; r++) {
            if (t0 + r < cnt) {
              const int32_t cand = du + w8[r];
              if (s8[r] >= 0) {
                // integer multiplicities below 2^53 sum exactly as 64-bit
                // integers (a slot column takes at most one per item);
                // larger ones, rounded in FP64 anyway, go to cm directly
                if (active && ((hs.take[s8[r]] >> lane) & 1u) && cand == hs.mn[s8[r]][lane]) {
                  if (mu < 9007199254740992.0)
                    atomicAdd(reinterpret_cast<unsigned long long*>(&hs.sum[s8[r]][lane]),
                              (unsigned long long)mu);
                  else
                    atomicAdd(&cm[(size_t)v8[r] * nb + j], mu);
                }
              } else {
                const bool hit = active && cand == c8[r];
                if (hit) atomicAdd(&cm[(size_t)v8[r] * nb + j], mu);
                if (bytes) nbytes += 4ull * __popc(m) + 16ull * __popc(__ballot_sync(0xffffffffu, hit));
              }
            }
          }
        }
      }
      if (bytes && pass == 1) nbytes += 8ull * (end - beg) / W + 12ull * __popc(m) + 4ull;
    }
    __syncthreads();
    if (pass == 0) {
      // columns where the block's minimum is the product's minimum
      for (int sl = (int)(threadIdx.x >> 5); sl < HASH_SLOTS; sl += 8) {
        const unsigned long long key = hs.key[sl];
        if (key == HASH_EMPTY) continue;
        const int32_t v = (int32_t)(key / (unsigned)W);
        const int word = (int)(key % (unsigned)W);
        const int32_t mn = hs.mn[sl][lane];
        const bool take = mn != INF && mn == cw[(size_t)v * nb + word * 32 + lane];
        const uint32_t tb = __ballot_sync(0xffffffffu, take);
        if (lane == 0) hs.take[sl] = tb;
        if (bytes) nbytes += 4ull * __popc(__ballot_sync(0xffffffffu, mn != INF));
      }
      __syncthreads();
    }
  }
  for (int sl = (int)(threadIdx.x >> 5); sl < HASH_SLOTS; sl += 8) {
    if (hs.key[sl] == HASH_EMPTY) continue;
    const uint32_t tb = hs.take[sl];
    if (!tb) continue;
    const unsigned long long key = hs.key[sl];
    const int32_t v = (int32_t)(key / (unsigned)W);
    const int word = (int)(key % (unsigned)W);
    const unsigned long long sm = reinterpret_cast<const unsigned long long*>(&hs.sum[sl][0])[lane];
    if (((tb >> lane) & 1u) && sm) atomicAdd(&cm[(size_t)v * nb + word * 32 + lane], (double)sm);
    if (bytes) nbytes += 8ull * __popc(tb);
  }
  if (bytes && lane == 0) atomicAdd(bytes, nbytes);
}

// MFBr product over A^T (counter decrement, exactly-once enqueue), hash
// form: per slot column the block sums the values and counts the tight arcs,
// then adds the sum to Z.p and takes the count off the counter with one
// atomic each; the lane whose subtraction takes the counter to zero enqueues.
template <int ARCS>
__global__ void __launch_bounds__(256, 4) k_gp_hash_prop(
    const int64_t* __restrict__ rowptr_t, const int32_t* __restrict__ col_t, const int32_t* __restrict__ wt_t,
    const uint32_t* __restrict__ hot, const int32_t* __restrict__ flist, uint32_t fcount, int W, int nb,
    const uint32_t* __restrict__ fmask, const int32_t* __restrict__ dist, const double* __restrict__ fv,
    double* zp, int32_t* cnt, uint32_t* tmask, uint32_t* vflag, int32_t* tlist, uint32_t* tcount,
    unsigned long long* bytes) {
  extern __shared__ __align__(16) unsigned char hash_raw[];
  HashSmem& hs = *reinterpret_cast<HashSmem*>(hash_raw);
  const unsigned lane = lane_id();
  int32_t* q = hs.q[threadIdx.x >> 5];
  int qn = 0;
  unsigned long long nbytes = 0;
  hash_clear(hs, 0);
  __syncthreads();
  for (int it = 0; it < HASH_ITEMS; it++) {
    uint64_t i;
    if (!hash_item(fcount, W, it, &i)) break;
    const int word = (int)(i / fcount);
    const int32_t u = flist[i % fcount];
    const uint32_t m = fmask[(size_t)u * W + word];
    if (!m) continue;
    const int j = word * 32 + (int)lane;
    const bool active = (m >> lane) & 1u;
    const int32_t du = active ? dist[(size_t)u * nb + j] : 0;
    const double val = active ? fv[(size_t)u * nb + j] : 0.0;
    const int64_t beg = rowptr_t[u], end = rowptr_t[u + 1];
    if (end - beg > HASH_ROW_MAX) continue;
    for (int64_t k0 = beg; k0 < end; k0 += 32) {
      const int64_t k = k0 + lane;
      const int32_t myv = k < end ? col_t[k] : 0;
      const int32_t myw = k < end ? (wt_t ? wt_t[k] : 1) : 0;
      const int cntk = (int)(end - k0 < 32 ? end - k0 : 32);
      for (int t0 = 0; t0 < cntk; t0 += ARCS) {
        int32_t v8[ARCS], w8[ARCS], d8[ARCS], o8[ARCS];
        int s8[ARCS];
#pragma unroll
        for (int r = 0; r < ARCS; r++) {
          v8[r] = __shfl_sync(0xffffffffu, myv, (t0 + r) & 31);
          w8[r] = __shfl_sync(0xffffffffu, myw, (t0 + r) & 31);
        }
#pragma unroll
        for (int r = 0; r < ARCS; r++)
          d8[r] = (active && t0 + r < cntk) ? __ldg(&dist[(size_t)v8[r] * nb + j]) : INT32_MIN;
        // only arcs that are tight in some column take a slot
        uint32_t want = 0u;
#pragma unroll
        for (int r = 0; r < ARCS; r++)
          want |= (__ballot_sync(0xffffffffu, t0 + r < cntk && d8[r] == du - w8[r]) ? 1u : 0u) << r;
        hash_slots<ARCS>(hs, true, t0, cntk, myv, W, word, hot, want, s8);
#pragma unroll
        for (int r = 0; r < ARCS; r++) {
          o8[r] = 0;
          if (t0 + r < cntk && d8[r] == du - w8[r]) {
            if (s8[r] >= 0) {
              atomicAdd(&hs.sum[s8[r]][lane], val);
              atomicAdd(&hs.mn[s8[r]][lane], 1);
            } else {
              const size_t idx = (size_t)v8[r] * nb + j;
              atomicAdd(&zp[idx], val);
              o8[r] = atomicSub(&cnt[idx], 1);
            }
          }
        }
        bool mine = false;
        int32_t mv = 0;
#pragma unroll
        for (int r = 0; r < ARCS; r++) {
          if (t0 + r < cntk) {
            const uint32_t rb = __ballot_sync(0xffffffffu, o8[r] == 1);
            if (rb && (int)lane == r) {
              atomicOr(&tmask[(size_t)v8[r] * W + word], rb);
              if (claim_vertex(vflag, v8[r])) { mine = true; mv = v8[r]; }
            }
            if (bytes)
              nbytes += 4ull * __popc(m) +
                        (s8[r] < 0 ? 24ull * __popc(__ballot_sync(0xffffffffu, d8[r] == du - w8[r])) : 0ull);
          }
        }
        wl_push(q, qn, mine, mv, tlist, tcount);
      }
    }
    if (bytes) nbytes += 8ull * (end - beg) / W + 16ull * __popc(m) + 4ull;
  }
  __syncthreads();
  for (int sl = (int)(threadIdx.x >> 5); sl < HASH_SLOTS; sl += 8) {
    const unsigned long long key = hs.key[sl];
    if (key == HASH_EMPTY) continue;
    const int32_t v = (int32_t)(key / (unsigned)W);
    const int word = (int)(key % (unsigned)W);
    const int32_t c = hs.mn[sl][lane];
    bool zero = false;
    if (c > 0) {
      const size_t idx = (size_t)v * nb + word * 32 + lane;
      atomicAdd(&zp[idx], hs.sum[sl][lane]);
      zero = atomicSub(&cnt[idx], c) == c;
    }
    const uint32_t rb = __ballot_sync(0xffffffffu, zero);
    bool mine = false;
    if (rb && lane == 0) {
      atomicOr(&tmask[(size_t)v * W + word], rb);
      mine = claim_vertex(vflag, v);
    }
    wl_push(q, qn, mine, v, tlist, tcount);
    if (bytes) nbytes += 16ull * __popc(__ballot_sync(0xffffffffu, c > 0));
  }
  wl_flush(q, qn, tlist, tcount);
  if (bytes && lane == 0) atomicAdd(bytes, nbytes);
}

// ------------------------------------------------------ segmented (pull) products
// The same products as the push kernels above, with the roles reversed: the
// candidates that meet at one (vertex v, 32-column word) -- those of v's arcs
// whose other end is in the frontier -- form one segment, and the warp that
// owns (v, word) reduces it in registers, so no two threads update one
// (vertex, column) and no atomics are needed.  Frontier membership is one bit
// per vertex (fmem), so a vertex with no frontier neighbour costs a row of
// bit tests.  Rows of more than PULL_ROW_MAX arcs (hubs) are reduced by a
// block: its warps split the row and combine their partial results through
// shared memory.
//
// FWD (MFBF, Algorithm 1's product over A^T rows = in-arcs): per column the
// minimum of tau(s,u) + A(u,v) over frontier (s,u), and the sum of the
// frontier multiplicities that attain it (the multpath monoid, Sec. 4.1.1);
// a minimum <= T(s,v).w is written to cw / cm and its bit to tmask, for
// k_gp_accumulate.
// BWD (MFBr, over A rows = out-arcs): for columns whose counter is still
// positive, the sum of the frontier values of successors u with
// tau(s,u) = tau(s,v) + A(v,u) (the centpath monoid, Sec. 4.2) and their
// number; zeta += sum, counter -= number; a counter reaching zero puts (s,v)
// in the next frontier (tmask), for k_gp_next_frontier.
constexpr int PULL_ROW_MAX = 256;

struct PullArgs {
  const int64_t* rowptr;   // FWD: A^T rows (in-arcs); BWD: A rows (out-arcs)
  const int32_t* col;
  const int32_t* wt;       // nullptr: unit weights
  int32_t n;
  int W, nb;
  const uint32_t* fmem;    // frontier membership bits
  const uint32_t* fmask;   // frontier columns [n][W]
  const int32_t* dist;     // T.w
  const double* fval;      // FWD: frontier multiplicities; BWD: frontier values zeta + 1/sigma_bar
  int32_t* cw;             // FWD: product weight out;  BWD: counters (in/out)
  double* cm;              // FWD: product multiplicity out;  BWD: zeta (in/out)
  uint32_t* tmask;
  uint32_t* vflag;
  int32_t* tlist;
  uint32_t* tcount;
  const int32_t* hubs;     // vertices whose row may exceed PULL_ROW_MAX (the block kernel's list)
  int32_t nhub;
  unsigned long long* bytes;
};

// Per-lane reduction state of one column.
template <bool FWD> struct PullAcc;
template <> struct PullAcc<true> {
  int32_t best = INF;
  double sum = 0.0;
  __device__ __forceinline__ void add(int32_t c, double m) {
    if (c < best) { best = c; sum = m; }
    else if (c == best) sum += m;
  }
  __device__ __forceinline__ void merge(const PullAcc& o) { add(o.best, o.sum); }
};
template <> struct PullAcc<false> {
  double sum = 0.0;
  int32_t hits = 0;
  __device__ __forceinline__ void merge(const PullAcc& o) { sum += o.sum; hits += o.hits; }
};

// Reduce the arcs [k0, k1) of v's row into this lane's column j.  FWD: act is
// "the column holds a source"; BWD: "the counter of (s,v) is positive", dv =
// tau(s,v).
template <bool FWD>
__device__ __forceinline__ void pull_span(const PullArgs& a, int64_t k0, int64_t k1, int word, int j, bool act,
                                          int32_t dv, PullAcc<FWD>& acc, unsigned long long& nbytes) {
  const unsigned lane = threadIdx.x & 31u;
  for (int64_t c0 = k0; c0 < k1; c0 += 32) {
    const int64_t k = c0 + lane;
    const int32_t myu = k < k1 ? __ldg(&a.col[k]) : -1;
    const int32_t myw = k < k1 ? (a.wt ? __ldg(&a.wt[k]) : 1) : 0;
    const bool mem = myu >= 0 && ((__ldg(&a.fmem[myu >> 5]) >> (myu & 31)) & 1u);
    uint32_t mm = __ballot_sync(0xffffffffu, mem);
    if (a.bytes && lane == 0) nbytes += 8ull * (uint64_t)(k1 - c0 < 32 ? k1 - c0 : 32);
    while (mm) {                                   // four frontier neighbours in flight
      int q[4];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        q[r] = mm ? __ffs(mm) - 1 : -1;
        mm &= mm ? mm - 1 : 0u;
      }
      int32_t u[4], w[4];
      uint32_t fw[4];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        u[r] = __shfl_sync(0xffffffffu, myu, q[r] & 31);
        w[r] = __shfl_sync(0xffffffffu, myw, q[r] & 31);
        fw[r] = q[r] >= 0 ? __ldg(&a.fmask[(size_t)u[r] * a.W + word]) : 0u;
      }
      int32_t d[4];
      double x[4];
      bool on[4];
#pragma unroll
      for (int r = 0; r < 4; r++) {
        on[r] = act && ((fw[r] >> lane) & 1u);
        d[r] = on[r] ? __ldg(&a.dist[(size_t)u[r] * a.nb + j]) : 0;
      }
#pragma unroll
      for (int r = 0; r < 4; r++) {
        if (!FWD) on[r] = on[r] && d[r] == dv + w[r];      // arc v -> u on a shortest path
        x[r] = on[r] ? __ldg(&a.fval[(size_t)u[r] * a.nb + j]) : 0.0;
      }
#pragma unroll
      for (int r = 0; r < 4; r++) {
        if (on[r]) {
          if constexpr (FWD) acc.add(d[r] + w[r], x[r]);
          else { acc.sum += x[r]; acc.hits++; }
        }
        if (a.bytes && q[r] >= 0) nbytes += 4ull * (lane == 0) + 12ull * on[r];
      }
    }
  }
}

// Write the reduced segment of (v, word): FWD the product entry, BWD the
// counter and zeta; set the touched bits and list v once.
template <bool FWD>
__device__ __forceinline__ void pull_finish(const PullArgs& a, int32_t v, int word, int j, int32_t dv,
                                            const PullAcc<FWD>& acc, bool& mine, unsigned long long& nbytes) {
  const unsigned lane = threadIdx.x & 31u;
  const size_t idx = (size_t)v * a.nb + j;
  bool touch;
  if constexpr (FWD) {
    touch = acc.best != INF && acc.best <= dv;     // heavier candidates cannot pass the filter
    if (touch) { a.cw[idx] = acc.best; a.cm[idx] = acc.sum; }
  } else {
    touch = false;
    if (acc.hits) {
      a.cm[idx] += acc.sum;
      const int32_t c = a.cw[idx] - acc.hits;
      a.cw[idx] = c;
      touch = c == 0;
    }
  }
  const uint32_t tb = __ballot_sync(0xffffffffu, touch);
  if (a.bytes && lane == 0) nbytes += 4ull + (FWD ? 12ull : 24ull) * __popc(tb);
  if (tb && lane == 0) {
    atomicOr(&a.tmask[(size_t)v * a.W + word], tb);
    if (claim_vertex(a.vflag, v)) mine = true;
  }
}

// One warp per (vertex, word) for rows of at most PULL_ROW_MAX arcs.
template <bool FWD>
__global__ void __launch_bounds__(256) k_gp_pull_rows(PullArgs a) {
  __shared__ int32_t qbuf[8][40];
  int32_t* q = qbuf[threadIdx.x >> 5];
  int qn = 0;
  const unsigned lane = threadIdx.x & 31u;
  const uint64_t tasks = (uint64_t)a.n * a.W;
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  unsigned long long nbytes = 0;
  for (uint64_t t = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; t < tasks; t += nw) {
    const int32_t v = (int32_t)(t / a.W);
    const int word = (int)(t % a.W);
    const int64_t k0 = __ldg(&a.rowptr[v]), k1 = __ldg(&a.rowptr[v + 1]);
    bool mine = false;
    if (k1 > k0 && k1 - k0 <= PULL_ROW_MAX) {
      const int j = word * 32 + (int)lane;
      const int32_t dv = __ldg(&a.dist[(size_t)v * a.nb + j]);
      const bool act = FWD ? true : (dv != INF && a.cw[(size_t)v * a.nb + j] > 0);
      if (__any_sync(0xffffffffu, act)) {
        PullAcc<FWD> acc;
        pull_span<FWD>(a, k0, k1, word, j, act, dv, acc, nbytes);
        pull_finish<FWD>(a, v, word, j, dv, acc, mine, nbytes);
      }
    }
    wl_push(q, qn, mine, v, a.tlist, a.tcount);
  }
  wl_flush(q, qn, a.tlist, a.tcount);
  if (a.bytes) {
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0 && nbytes) atomicAdd(a.bytes, nbytes);
  }
}

// One block of 8 warps per (hub, word) for rows of more than PULL_ROW_MAX arcs.
template <bool FWD>
__global__ void __launch_bounds__(256) k_gp_pull_hubs(PullArgs a) {
  __shared__ PullAcc<FWD> part[8][32];
  const unsigned lane = threadIdx.x & 31u;
  const int wid = (int)(threadIdx.x >> 5);
  unsigned long long nbytes = 0;
  const uint64_t tasks = (uint64_t)a.nhub * a.W;
  for (uint64_t t = blockIdx.x; t < tasks; t += gridDim.x) {
    const int32_t v = __ldg(&a.hubs[t / a.W]);
    const int word = (int)(t % a.W);
    const int64_t k0 = __ldg(&a.rowptr[v]), k1 = __ldg(&a.rowptr[v + 1]);
    if (k1 - k0 <= PULL_ROW_MAX) continue;         // uniform over the block
    const int j = word * 32 + (int)lane;
    const int32_t dv = __ldg(&a.dist[(size_t)v * a.nb + j]);
    const bool act = FWD ? true : (dv != INF && a.cw[(size_t)v * a.nb + j] > 0);
    PullAcc<FWD> acc;
    if (__syncthreads_or(act)) {
      // warp w takes the 32-arc chunks w, w + 8, ...
      for (int64_t c0 = k0 + 32 * wid; c0 < k1; c0 += 32 * 8)
        pull_span<FWD>(a, c0, c0 + 32 < k1 ? c0 + 32 : k1, word, j, act, dv, acc, nbytes);
      part[wid][lane] = acc;
      __syncthreads();
      if (wid == 0) {
        for (int r = 1; r < 8; r++) acc.merge(part[r][lane]);
        bool mine = false;
        pull_finish<FWD>(a, v, word, j, dv, acc, mine, nbytes);
        if (mine) a.tlist[atomicAdd(a.tcount, 1u)] = v;
      }
    }
    __syncthreads();
  }
  if (a.bytes) {
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0 && nbytes) atomicAdd(a.bytes, nbytes);
  }
}

// ------------------------------------------------------------------ driver
static inline unsigned warp_blocks(uint64_t warps) { return (unsigned)((warps + 7) / 8); }
// grid for kernels whose item count is only known on the device (grid-stride)
static inline unsigned stride_blocks(uint64_t max_warps) {
  uint64_t b = (max_warps + 7) / 8;
  return (unsigned)(b < 1 ? 1 : (b > 152 * 16 ? 152 * 16 : b));
}

// blocks of the hub kernels: one per (hub, word) task, at most 8 per SM
static inline unsigned hub_blocks(int32_t nhub, int W) {
  const uint64_t t = (uint64_t)nhub * W;
  return (unsigned)(t < 152 * 8 ? (t ? t : 1) : 152 * 8);
}

// Segmented (pull) or atomic (push) reduction for a product whose frontier
// holds fcount vertices: MFBC_ACCUM_AUTO pulls once the frontier holds 1/64 of
// the vertices (the pull kernels visit every vertex; the push kernels only
// the frontier's arcs, but meet in atomics at hub columns).
static inline bool use_pull(const RunCtx& rc, uint32_t fcount, int32_t n) {
  if (rc.accum == MFBC_ACCUM_SEGMENTED) return true;
  if (rc.accum == MFBC_ACCUM_ATOMIC || rc.accum == MFBC_ACCUM_HASH) return false;
  return (uint64_t)fcount * 64 >= (uint64_t)n;
}

static mfbc_status read_counts(RunCtx& rc, Counters* ctr) {
  MFBC_CUDA_TRY(cudaMemcpyAsync(rc.h_ctr, ctr->list_count, sizeof(uint32_t) * 5,
                                cudaMemcpyDeviceToHost, rc.stream), rc.err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(rc.stream), rc.err);
  rc.prof->drain();
  return MFBC_OK;
}

// arc kernels: eight arcs per step on graphs of average degree >= 8
#define GP_LAUNCH(kern, grid, ...)                                        \
  do {                                                                    \
    if (wide) kern<8><<<grid, 256, 0, st>>>(__VA_ARGS__);                 \
    else kern<1><<<grid, 256, 0, st>>>(__VA_ARGS__);                      \
  } while (0)

// hash accumulator kernels: one block per 8 * HASH_ITEMS items, the table
// in dynamic shared memory
static inline unsigned hash_blocks(uint64_t items) {
  const uint64_t b = (items + 8 * HASH_ITEMS - 1) / (8 * HASH_ITEMS);
  return (unsigned)(b < 1 ? 1 : b);
}
static void hash_smem_attrs() {
  static bool done = false;
  if (done) return;
  const int sz = (int)sizeof(HashSmem);
  cudaFuncSetAttribute(k_gp_hash_min<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
  cudaFuncSetAttribute(k_gp_hash_min<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
  cudaFuncSetAttribute(k_gp_hash_tie<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
  cudaFuncSetAttribute(k_gp_hash_tie<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
  cudaFuncSetAttribute(k_gp_hash_prop<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
  cudaFuncSetAttribute(k_gp_hash_prop<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, sz);
  done = true;
}
#define GP_HASH(kern, grid, ...)                                                   \
  do {                                                                             \
    if (wide) kern<8><<<grid, 256, sizeof(HashSmem), st>>>(__VA_ARGS__);           \
    else kern<1><<<grid, 256, sizeof(HashSmem), st>>>(__VA_ARGS__);                \
  } while (0)

#define PROF(id, ...)             \
  do {                            \
    rc.prof->begin(id);           \
    __VA_ARGS__;                  \
    rc.prof->end(id);             \
  } while (0)

mfbc_status general_batch(RunCtx& rc, GeneralState& s, const int32_t* d_src_batch, int nactive,
                          double* lambda, int64_t* fwd_iters, int64_t* bwd_iters) {
  const DevGraph& g = *rc.g;
  const int32_t n = g.n;
  const int nb = s.nb, W = s.W;
  cudaStream_t st = rc.stream;
  const size_t cells = (size_t)n * nb;
  unsigned long long* B = rc.prof->count_bytes ? s.ctr->bytes : nullptr;
  if (n == 0) return MFBC_OK;
  // eight arcs per step on graphs of average degree >= 8, unless tuned
  const bool wide = rc.arcs ? rc.arcs > 1 : g.nnz >= 8 * (int64_t)n;

  // batch sources: active columns then padding
  fill_i32(s.src, -1, (size_t)nb, st);
  if (nactive)
    MFBC_CUDA_TRY(cudaMemcpyAsync(s.src, d_src_batch, sizeof(int32_t) * nactive,
                                  cudaMemcpyDeviceToDevice, st), rc.err);
  PROF(K_FILL, {
    fill_i32(s.dist, INF, cells, st);
    fill_i32(s.cw, INF, cells, st);
    cudaMemsetAsync(s.sig, 0, sizeof(double) * cells, st);
    cudaMemsetAsync(s.cm, 0, sizeof(double) * cells, st);
    cudaMemsetAsync(s.fmask, 0, sizeof(uint32_t) * (size_t)n * W, st);
    cudaMemsetAsync(s.tmask, 0, sizeof(uint32_t) * (size_t)n * W, st);
    cudaMemsetAsync(s.vflag, 0, sizeof(uint32_t) * (size_t)n, st);
    cudaMemsetAsync(s.fmem, 0, sizeof(uint32_t) * (((size_t)n + 31) / 32), st);
    cudaMemsetAsync(s.ctr->list_count, 0, sizeof(uint32_t) * 4, st);
  });
  rc.prof->k[K_FILL].bytes += 24.0 * cells + 8.0 * n * W + 4.0 * n;

  int32_t* cur = s.listA;
  int32_t* nxt = s.listB;
  PROF(K_SEED, (k_gp_seed<<<(nb + 127) / 128, 128, 0, st>>>(s.src, nb, W, s.dist, s.sig, s.fm, s.fmask,
                                                          s.fmem, s.vflag, cur, &s.ctr->list_count[0])));
  mfbc_status e = read_counts(rc, s.ctr);
  if (e) return e;
  uint32_t fcount = rc.h_ctr[0];
  if (fcount) k_clear_flags<<<(fcount + 255) / 256, 256, 0, st>>>(cur, fcount, s.vflag);

  // ---- MFBF (Algorithm 1)
  int64_t iters = 0;
  while (fcount) {
    if (++iters > (int64_t)n + 1) {
      if (rc.err) *rc.err = "MFBF did not converge within n+1 products";
      return MFBC_ERR_NO_CONVERGENCE;
    }
    MFBC_CUDA_TRY(cudaMemsetAsync(s.ctr->list_count, 0, sizeof(uint32_t) * 4, st), rc.err);
    const uint64_t wp = (uint64_t)fcount * W;
    if (use_pull(rc, fcount, n)) {
      const PullArgs pa{g.rowptr_t, g.col_t, g.w_t, n, W, nb, s.fmem, s.fmask, s.dist, s.fm, s.cw, s.cm,
                        s.tmask, s.vflag, nxt, &s.ctr->list_count[1], g.items_in.hubs, g.items_in.nhub,
                        B ? B + K_PULL_FWD : nullptr};
      PROF(K_PULL_FWD, {
        k_gp_pull_rows<true><<<stride_blocks((uint64_t)n * W), 256, 0, st>>>(pa);
        if (g.items_in.nhub) k_gp_pull_hubs<true><<<hub_blocks(g.items_in.nhub, W), 256, 0, st>>>(pa);
      });
    } else if (rc.accum == MFBC_ACCUM_HASH) {
      hash_smem_attrs();
      // rows of at most HASH_ROW_MAX arcs in the hash kernels, longer ones
      // on the atomic kernels; both minimum passes precede both tie passes
      const bool longrows = g.max_deg > HASH_ROW_MAX;
      PROF(K_HASH_MIN, {
        GP_HASH(k_gp_hash_min, hash_blocks(wp), g.rowptr, g.col, g.w, g.hot_in, cur, fcount, W, nb, s.fmask,
                s.dist, s.cw, s.tmask, s.vflag, nxt, &s.ctr->list_count[1], B ? B + K_HASH_MIN : nullptr);
        if (longrows)
          GP_LAUNCH(k_gp_relax_min, warp_blocks(wp), g.rowptr, g.col, g.w, cur, fcount, W, nb, s.fmask, s.dist,
                    s.cw, s.tmask, s.vflag, nxt, &s.ctr->list_count[1], B ? B + K_HASH_MIN : nullptr,
                    (int64_t)HASH_ROW_MAX + 1);
      });
      PROF(K_HASH_TIE, {
        GP_HASH(k_gp_hash_tie, hash_blocks(wp), g.rowptr, g.col, g.w, g.hot_in, cur, fcount, W, nb, s.fmask,
                s.dist, s.fm, s.cw, s.cm, B ? B + K_HASH_TIE : nullptr);
        if (longrows)
          GP_LAUNCH(k_gp_relax_tie, warp_blocks(wp), g.rowptr, g.col, g.w, cur, fcount, W, nb, s.fmask, s.dist,
                    s.fm, s.cw, s.cm, B ? B + K_HASH_TIE : nullptr, (int64_t)HASH_ROW_MAX + 1);
      });
    } else {
      PROF(K_RELAX_MIN, GP_LAUNCH(k_gp_relax_min, warp_blocks(wp),
                            g.rowptr, g.col, g.w, cur, fcount, W, nb, s.fmask, s.dist, s.cw, s.tmask,
                            s.vflag, nxt, &s.ctr->list_count[1], B ? B + K_RELAX_MIN : nullptr, (int64_t)0));
      PROF(K_RELAX_TIE, GP_LAUNCH(k_gp_relax_tie, warp_blocks(wp),
                            g.rowptr, g.col, g.w, cur, fcount, W, nb, s.fmask, s.dist, s.fm, s.cw, s.cm,
                            B ? B + K_RELAX_TIE : nullptr, (int64_t)0));
    }
    PROF(K_CLEAR, (k_clear_mask_rows<<<(unsigned)((wp + 255) / 256), 256, 0, st>>>(cur, fcount, W,
                                                                                   s.fmask, s.fmem)));
    // the touched list lives in nxt; compact the next frontier into cur
    PROF(K_ACCUM, (k_gp_accumulate<<<stride_blocks((uint64_t)n), 256, 0, st>>>(
                      nxt, &s.ctr->list_count[1], W, nb, s.dist, s.sig, s.cw, s.cm, s.fm, s.fmask,
                      s.tmask, s.vflag, s.fmem, cur, &s.ctr->list_count[0], B ? B + K_ACCUM : nullptr)));
    e = read_counts(rc, s.ctr);
    if (e) return e;
    fcount = rc.h_ctr[0];
  }
  if (fwd_iters) *fwd_iters += iters;
  check_sigma_exact(s.sig, cells, s.ctr, st);
  if (!lambda) return MFBC_OK;

  // ---- MFBr (Algorithm 2): cw holds the counters, cm the factors Z.p, fm the values
  MFBC_CUDA_TRY(cudaMemsetAsync(s.ctr->list_count, 0, sizeof(uint32_t) * 4, st), rc.err);
  PROF(K_COUNTERS, GP_LAUNCH(k_gp_counters, warp_blocks((uint64_t)n),
                       n, g.rowptr, g.col, g.w, W, nb, s.src, s.dist, s.sig, s.cw, s.cm, s.fm, s.fmask,
                       s.fmem, cur, &s.ctr->list_count[0], B ? B + K_COUNTERS : nullptr));
  e = read_counts(rc, s.ctr);
  if (e) return e;
  fcount = rc.h_ctr[0];
  iters = 0;
  while (fcount) {
    if (++iters > (int64_t)n + 1) {
      if (rc.err) *rc.err = "MFBr did not converge within n+1 products";
      return MFBC_ERR_NO_CONVERGENCE;
    }
    MFBC_CUDA_TRY(cudaMemsetAsync(s.ctr->list_count, 0, sizeof(uint32_t) * 4, st), rc.err);
    const uint64_t wp = (uint64_t)fcount * W;
    if (use_pull(rc, fcount, n)) {
      const PullArgs pb{g.rowptr, g.col, g.w, n, W, nb, s.fmem, s.fmask, s.dist, s.fm, s.cw, s.cm,
                        s.tmask, s.vflag, nxt, &s.ctr->list_count[1], g.items_out.hubs, g.items_out.nhub,
                        B ? B + K_PULL_BWD : nullptr};
      PROF(K_PULL_BWD, {
        k_gp_pull_rows<false><<<stride_blocks((uint64_t)n * W), 256, 0, st>>>(pb);
        if (g.items_out.nhub) k_gp_pull_hubs<false><<<hub_blocks(g.items_out.nhub, W), 256, 0, st>>>(pb);
      });
    } else if (rc.accum == MFBC_ACCUM_HASH) {
      hash_smem_attrs();
      PROF(K_HASH_PROP, {
        GP_HASH(k_gp_hash_prop, hash_blocks(wp), g.rowptr_t, g.col_t, g.w_t, g.hot_out, cur, fcount, W, nb,
                s.fmask, s.dist, s.fm, s.cm, s.cw, s.tmask, s.vflag, nxt, &s.ctr->list_count[1],
                B ? B + K_HASH_PROP : nullptr);
        if (g.max_in_deg > HASH_ROW_MAX)
          GP_LAUNCH(k_gp_propagate, warp_blocks(wp), g.rowptr_t, g.col_t, g.w_t, cur, fcount, W, nb, s.fmask,
                    s.dist, s.fm, s.cm, s.cw, s.tmask, s.vflag, nxt, &s.ctr->list_count[1],
                    B ? B + K_HASH_PROP : nullptr, (int64_t)HASH_ROW_MAX + 1);
      });
    } else {
      PROF(K_PROPAGATE, GP_LAUNCH(k_gp_propagate, warp_blocks(wp),
                            g.rowptr_t, g.col_t, g.w_t, cur, fcount, W, nb, s.fmask, s.dist, s.fm, s.cm,
                            s.cw, s.tmask, s.vflag, nxt, &s.ctr->list_count[1],
                            B ? B + K_PROPAGATE : nullptr, (int64_t)0));
    }
    PROF(K_CLEAR, (k_clear_mask_rows<<<(unsigned)((wp + 255) / 256), 256, 0, st>>>(cur, fcount, W,
                                                                                   s.fmask, s.fmem)));
    PROF(K_FINAL, (k_gp_next_frontier<<<stride_blocks((uint64_t)n), 256, 0, st>>>(
                      nxt, &s.ctr->list_count[1], W, nb, s.sig, s.cm, s.fm, s.fmask, s.tmask, s.vflag,
                      s.fmem, cur, &s.ctr->list_count[0], B ? B + K_FINAL : nullptr)));
    e = read_counts(rc, s.ctr);
    if (e) return e;
    fcount = rc.h_ctr[0];
  }
  if (bwd_iters) *bwd_iters += iters;
  const int32_t* wreq = nullptr;
  if (rc.word_req && batch_uniform_request(rc.word_req, W) < 0) {
    MFBC_CUDA_TRY(cudaMemcpyAsync(s.word_req, rc.word_req, sizeof(int32_t) * W, cudaMemcpyHostToDevice, st), rc.err);
    wreq = s.word_req;
  }
  const int urq = rc.word_req ? batch_uniform_request(rc.word_req, W) : 0;
  double* lam0 = wreq ? lambda : lambda + (size_t)(urq < 0 ? 0 : urq) * n;
  PROF(K_LAMBDA, (k_gp_lambda<<<warp_blocks((uint64_t)n), 256, 0, st>>>(n, W, nb, s.src, s.cm, s.sig,
                                                                         lam0, wreq)));
  rc.prof->k[K_LAMBDA].bytes += 16.0 * cells + 16.0 * n;
  return MFBC_OK;
}

mfbc_status general_output(RunCtx& rc, GeneralState& s, int nactive, int32_t* dist_out,
                           double* sigma_out) {
  const int32_t n = rc.g->n;
  PROF(K_OUTPUT, {
    transpose_i32(s.dist, dist_out, n, s.nb, nactive, n, rc.stream);
    if (sigma_out) transpose_f64(s.sig, sigma_out, n, s.nb, nactive, n, rc.stream);
  });
  return MFBC_OK;
}

}  // namespace mfbc
