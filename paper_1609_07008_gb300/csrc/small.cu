// Persistent path for small unit-weight graphs: MFBF (Algorithm 1) and MFBr
// (Algorithm 2) of whole batches inside one cooperative launch.
//
// On a graph of a few thousand vertices a level of the per-product kernels
// (level.cu) is a few microseconds of work behind a launch and a host
// round trip, so a batch is bound by launch latency.  Here the batches of a
// call form a device queue; the launch holds G groups of P blocks, and each
// group takes the next batch from the queue, runs all of its levels with the
// group's blocks meeting at a barrier after each level, adds its lambda terms,
// and takes the next batch until the queue is empty.  One launch per call,
// no host round trip between levels.  The grid is small (G * P blocks), so
// other streams keep the rest of the GPU.
//
// State of a group (vertex-major like the other kernel families):
//   lvl[v][j]  uint8, tau(s_j, v), or LVL_NONE while unreached;
//   sv[v][j]   sigma_bar(s_j, v) as an exact 64-bit integer after MFBF, then
//              the MFBr value zeta + 1/sigma_bar as a double-float pair
//              (dfloat.cuh), written once the pair's level is finished.
// MFBF product of level l (the multpath product over unit weights, Sec.
// 4.1): for every (v, j) still unreached, sigma_bar(s_j, v) = sum of
// sigma_bar(s_j, u) over in-neighbours u at level l; a non-zero sum puts
// (s_j, v) at level l + 1 (Lemma 1: the frontier of product l is exactly the
// pairs at distance l).  MFBr level l, from the deepest level down to 1
// (Sec. 4.2.1): zeta(s_j, v) = sum over out-neighbours u at level l + 1 of
// (zeta + 1/sigma_bar)(s_j, u); lambda(v) += zeta * sigma_bar (Algorithm 3;
// level 0 holds only the source, which is skipped).
//
// Barriers: arrival counters in global memory, one per group.  A group's
// blocks are co-resident (cooperative launch), so a wait ends as soon as the
// slowest block finishes its level; every wait still has a clock64 budget,
// after which the block sets MFBC's timeout flag and the whole launch returns
// (the call reports MFBC_ERR_TIMEOUT).
//
// A batch deeper than SMALL_MAX_LEVEL levels, or whose path counts reach
// 2^58, is listed for recomputation by the general kernels (FP64 counts, no
// depth limit); its MFBr is skipped, so it adds nothing to lambda here.
#include <algorithm>

#include "dfloat.cuh"
#include "internal.cuh"

namespace mfbc {

constexpr int SMALL_THREADS = 256;
constexpr int SMALL_WARPS = SMALL_THREADS / 32;
constexpr uint8_t LVL_NONE = 255;
constexpr int SMALL_MAX_LEVEL = 254;           // deepest level an uint8 holds (255 = unreached)

size_t small_bytes(int32_t n, int nb, int groups) {
  Carver c(nullptr, 0);
  SmallState s;
  small_carve(c, n, nb, groups, s);
  return c.off;
}

void small_carve(Carver& c, int32_t n, int nb, int groups, SmallState& s) {
  s.nb = nb;
  s.W = nb / 32;
  s.G = groups;
  const size_t cells = (size_t)n * nb;
  s.lvl = c.take<uint8_t>(cells * groups);
  s.sv = c.take<uint64_t>(cells * groups);
  s.ctl = c.take<SmallGroupCtl>((size_t)groups);
  s.head = c.take<uint32_t>(64);
  s.redo = c.take<int32_t>(4096);
  s.ctr = c.take<Counters>(1);
}

__device__ __forceinline__ uint32_t ld_acquire(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ uint32_t ld_relaxed(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

struct SmallArgs {
  int32_t n;
  int nb, W, P;
  const int64_t* rp_in;                // rows of A^T (in-arcs): MFBF gathers over them
  const int32_t* col_in;
  const int64_t* rp_out;               // rows of A (out-arcs): MFBr gathers over them
  const int32_t* col_out;
  const int32_t* src;                  // [nbatch][nb] source of each column, -1 padding
  const int32_t* wreq;                 // [nbatch][W] lambda row of each word (-1 none), or null: row 0
  int32_t nbatch;
  double* lambda;                      // rows of n; null: MFBF only
  int32_t* dist_out;                   // sssp rows [out_rows][n] (row b*nb + j), or null
  double* sigma_out;
  int32_t out_rows;
  uint8_t* lvl;                        // [G][n][nb]
  uint64_t* sv;                        // [G][n][nb]
  SmallGroupCtl* ctl;                  // [G]
  uint32_t* head;                      // batch queue head, then the redo count
  int32_t* redo;                       // batches for the general kernels
  int32_t redo_cap;
  uint32_t* flags;                     // FLAG_* bits (Counters::flags)
  long long budget;                    // clock64 cycles a barrier wait may take
  uint32_t stall;                      // test hook: a barrier waits for one arrival too many
  unsigned long long* bytes;           // algorithmic bytes (byte-counting runs), or null
};

// Barrier of the P blocks of one group.  Returns false (every block of the
// launch then returns) when the wait ran out of budget or another block
// already flagged a timeout.
__device__ __forceinline__ bool group_barrier(const SmallArgs& a, SmallGroupCtl* c, uint32_t& epoch,
                                              uint32_t& s_ok) {
  __syncthreads();
  if (threadIdx.x == 0) {
    ++epoch;
    const uint32_t target = epoch * (uint32_t)a.P + a.stall;
    __threadfence();
    atomicAdd(&c->arrive, 1u);
    const long long t0 = clock64();
    uint32_t ok = 1;
    while (ld_acquire(&c->arrive) < target) {
      if ((ld_relaxed(a.flags) & FLAG_TIMEOUT) || clock64() - t0 > a.budget) {
        atomicOr(a.flags, FLAG_TIMEOUT);
        ok = 0;
        break;
      }
      __nanosleep(64);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// MFBF product of level l over the group's share of (vertex, word) tasks.
// Sets *any when a pair entered level l + 1, *wrap when a count reached 2^58.
__device__ __forceinline__ void small_fwd_level(const SmallArgs& a, const int32_t* __restrict__ src, uint8_t* lvl,
                                                uint64_t* sv, int l, int gw, int GW, uint32_t* any, uint32_t* wrap,
                                                unsigned long long& nbytes) {
  const unsigned lane = threadIdx.x & 31u;
  const int nb = a.nb, W = a.W;
  const uint64_t tasks = (uint64_t)a.n * W;
  bool big = false;
  for (uint64_t t = (uint64_t)gw; t < tasks; t += (uint64_t)GW) {
    const int32_t v = (int32_t)(t / W);
    const int j = (int)(t % W) * 32 + (int)lane;
    const size_t me = (size_t)v * nb + j;
    const bool open = lvl[me] == LVL_NONE && __ldg(&src[j]) >= 0;
    if (a.bytes) nbytes += 32;
    if (!__any_sync(0xffffffffu, open)) continue;
    const int64_t beg = __ldg(&a.rp_in[v]), end = __ldg(&a.rp_in[v + 1]);
    uint64_t acc = 0;
    bool ovf = false;
    for (int64_t k0 = beg; k0 < end; k0 += 32) {
      const int cnt = (int)(end - k0 < 32 ? end - k0 : 32);
      const int32_t myu = (int)lane < cnt ? __ldg(&a.col_in[k0 + lane]) : 0;
      for (int q0 = 0; q0 < cnt; q0 += 4) {
        int32_t u[4];
        uint8_t x[4];
#pragma unroll
        for (int q = 0; q < 4; q++) {
          u[q] = __shfl_sync(0xffffffffu, myu, (q0 + q) & 31);
          x[q] = q0 + q < cnt ? lvl[(size_t)u[q] * nb + j] : LVL_NONE;
        }
        uint64_t y[4];
#pragma unroll
        for (int q = 0; q < 4; q++) y[q] = (open && x[q] == (uint8_t)l) ? sv[(size_t)u[q] * nb + j] : 0ull;
#pragma unroll
        for (int q = 0; q < 4; q++) {
          const uint64_t s = acc + y[q];
          ovf |= s < acc;
          acc = s;
          if (a.bytes) nbytes += (q0 + q < cnt ? 32 : 0) + 8ull * __popc(__ballot_sync(0xffffffffu, y[q] != 0ull));
        }
      }
      if (a.bytes) nbytes += 4ull * cnt;
    }
    const bool hit = open && acc != 0ull;
    if (hit) {
      lvl[me] = (uint8_t)(l + 1);
      sv[me] = acc;
      big |= acc >= (1ull << 53);
      ovf |= acc >= (1ull << 58);
    }
    const uint32_t hm = __ballot_sync(0xffffffffu, hit);
    if (a.bytes) nbytes += 9ull * __popc(hm);
    if (hm && lane == 0) atomicOr(any, 1u);
    if (__any_sync(0xffffffffu, ovf) && lane == 0) atomicOr(wrap, 1u);
  }
  if (__any_sync(0xffffffffu, big) && lane == 0) atomicOr(a.flags, FLAG_SIGMA_INEXACT);
}

// MFBr of level l (1 <= l <= deepest) over the group's share of tasks.
__device__ __forceinline__ void small_bwd_level(const SmallArgs& a, uint8_t* lvl, uint64_t* sv, int l, bool deepest,
                                                const int32_t* __restrict__ wreq, int gw, int GW,
                                                unsigned long long& nbytes) {
  const unsigned lane = threadIdx.x & 31u;
  const int nb = a.nb, W = a.W;
  const uint64_t tasks = (uint64_t)a.n * W;
  for (uint64_t t = (uint64_t)gw; t < tasks; t += (uint64_t)GW) {
    const int32_t v = (int32_t)(t / W);
    const int word = (int)(t % W);
    const int j = word * 32 + (int)lane;
    const size_t me = (size_t)v * nb + j;
    const bool mine = lvl[me] == (uint8_t)l;
    if (a.bytes) nbytes += 32;
    if (!__any_sync(0xffffffffu, mine)) continue;
    float zs = 0.f, zc = 0.f;                            // compensated zeta sum of this lane's column
    if (!deepest) {                                      // the deepest level has no successors
      const int64_t beg = __ldg(&a.rp_out[v]), end = __ldg(&a.rp_out[v + 1]);
      for (int64_t k0 = beg; k0 < end; k0 += 32) {
        const int cnt = (int)(end - k0 < 32 ? end - k0 : 32);
        const int32_t myu = (int)lane < cnt ? __ldg(&a.col_out[k0 + lane]) : 0;
        for (int q0 = 0; q0 < cnt; q0 += 4) {
          int32_t u[4];
          uint8_t x[4];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            u[q] = __shfl_sync(0xffffffffu, myu, (q0 + q) & 31);
            x[q] = q0 + q < cnt ? lvl[(size_t)u[q] * nb + j] : LVL_NONE;
          }
          uint64_t y[4];
          bool h[4];
#pragma unroll
          for (int q = 0; q < 4; q++) {
            h[q] = mine && x[q] == (uint8_t)(l + 1);
            y[q] = h[q] ? sv[(size_t)u[q] * nb + j] : 0ull;
          }
#pragma unroll
          for (int q = 0; q < 4; q++) {
            if (h[q]) acc_add(zs, zc, y[q]);
            if (a.bytes) nbytes += (q0 + q < cnt ? 32 : 0) + 8ull * __popc(__ballot_sync(0xffffffffu, h[q]));
          }
        }
        if (a.bytes) nbytes += 4ull * cnt;
      }
    }
    float ls = 0.f, lc = 0.f;
    if (mine) sv[me] = finish_col(acc_value(zs, zc), sv[me], ls, lc);
    if (a.bytes) nbytes += 16ull * __popc(__ballot_sync(0xffffffffu, mine));
    if (a.lambda && __any_sync(0xffffffffu, ls != 0.f)) {
      const double lam = warp_acc_sum(ls, lc);
      const int row = wreq ? __ldg(&wreq[word]) : 0;
      if (lane == 0 && row >= 0) atomicAdd(&a.lambda[(size_t)row * a.n + v], lam);
      if (a.bytes) nbytes += 8;
    }
  }
}

__global__ void __launch_bounds__(SMALL_THREADS, 4) k_small_bc(SmallArgs a) {
  __shared__ uint32_t s_ok;
  const int g = (int)blockIdx.x / a.P, r = (int)blockIdx.x % a.P;
  SmallGroupCtl* c = a.ctl + g;
  uint32_t epoch = 0;
  const int gw = r * SMALL_WARPS + (int)(threadIdx.x >> 5);   // warp within the group
  const int GW = a.P * SMALL_WARPS;
  const int gt = r * SMALL_THREADS + (int)threadIdx.x;         // thread within the group
  const int GT = a.P * SMALL_THREADS;
  const size_t cells = (size_t)a.n * a.nb;
  uint8_t* lvl = a.lvl + (size_t)g * cells;
  uint64_t* sv = a.sv + (size_t)g * cells;
  unsigned long long nbytes = 0;
  for (;;) {
    if (r == 0 && threadIdx.x == 0) {
      c->batch = atomicAdd(a.head, 1u);
      c->wrap = 0u;
      c->any[0] = c->any[1] = c->any[2] = 0u;
    }
    if (!group_barrier(a, c, epoch, s_ok)) break;
    const uint32_t b = ld_relaxed(&c->batch);
    if (b >= (uint32_t)a.nbatch) break;
    const int32_t* src = a.src + (size_t)b * a.nb;
    const int32_t* wreq = a.wreq ? a.wreq + (size_t)b * a.W : nullptr;
    // every pair unreached, every count zero (16-byte stores; n_b is a multiple of 32)
    for (size_t i = (size_t)gt; i < cells / 16; i += (size_t)GT)
      reinterpret_cast<uint4*>(lvl)[i] = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
    for (size_t i = (size_t)gt; i < cells / 2; i += (size_t)GT) reinterpret_cast<uint4*>(sv)[i] = make_uint4(0, 0, 0, 0);
    if (a.bytes && gt == 0) nbytes += 9ull * cells;
    if (!group_barrier(a, c, epoch, s_ok)) break;
    // seed: T(s_j, s_j) = (0, 1), frontier {(s_j, s_j)} (Algorithm 1's start);
    // the first product is pushed from the seed by the column's thread: every
    // out-neighbour of s_j is at level 1 with one path (no self-loops, so
    // the two levels never meet in one column)
    {
      bool any1 = false;
      for (int j = gt; j < a.nb; j += GT) {
        const int32_t s = src[j];
        if (s < 0) continue;
        lvl[(size_t)s * a.nb + j] = 0;
        sv[(size_t)s * a.nb + j] = 1ull;
        for (int64_t k = __ldg(&a.rp_out[s]); k < __ldg(&a.rp_out[s + 1]); k++) {
          const int32_t v = __ldg(&a.col_out[k]);
          lvl[(size_t)v * a.nb + j] = 1;
          sv[(size_t)v * a.nb + j] = 1ull;
          any1 = true;
          if (a.bytes) nbytes += 13;
        }
      }
      if (__syncthreads_or(any1) && threadIdx.x == 0) atomicOr(&c->any[0], 1u);
    }
    if (!group_barrier(a, c, epoch, s_ok)) break;
    // MFBF, level by level until a product adds no pair (slot 0 holds the
    // seed's flag; every block reads it here, before the barrier after which
    // block 0 may clear that slot for level 3)
    int deepest = 0;
    bool redo = false, quit = false;
    const bool level1 = ld_relaxed(&c->any[0]) != 0u;
    for (int l = 1; level1; l++) {
      if (l >= SMALL_MAX_LEVEL) { redo = true; break; }
      // the flag of level l + 1 shares its slot with level l - 2, which every
      // block has read before arriving at the barrier of level l - 1
      if (r == 0 && threadIdx.x == 0) c->any[(l + 1) % 3] = 0u;
      small_fwd_level(a, src, lvl, sv, l, gw, GW, &c->any[l % 3], &c->wrap, nbytes);
      if (!group_barrier(a, c, epoch, s_ok)) { quit = true; break; }
      if (ld_relaxed(&c->wrap)) { redo = true; break; }
      if (!ld_relaxed(&c->any[l % 3])) { deepest = l; break; }
    }
    if (quit) break;
    if (redo) {
      if (r == 0 && threadIdx.x == 0) {
        const uint32_t k = atomicAdd(&a.head[1], 1u);
        if ((int32_t)k < a.redo_cap) a.redo[k] = (int32_t)b;
      }
    } else {
      if (a.dist_out) {                      // MFBF alone: per-source rows of tau and sigma_bar
        for (int j = 0; j < a.nb; j++) {
          const int64_t row = (int64_t)b * a.nb + j;
          if (row >= a.out_rows || src[j] < 0) continue;
          for (int32_t v = gt; v < a.n; v += GT) {
            const uint8_t x = lvl[(size_t)v * a.nb + j];
            a.dist_out[row * a.n + v] = x == LVL_NONE ? INF : (int32_t)x;
            if (a.sigma_out) a.sigma_out[row * a.n + v] = (double)sv[(size_t)v * a.nb + j];
          }
        }
      }
      if (a.lambda) {
        for (int l = deepest; l >= 1; l--) {
          small_bwd_level(a, lvl, sv, l, l == deepest, wreq, gw, GW, nbytes);
          if (!group_barrier(a, c, epoch, s_ok)) { quit = true; break; }
        }
        if (quit) break;
      }
    }
    // every block is done with this batch's state before the next clear
    if (!group_barrier(a, c, epoch, s_ok)) break;
  }
  if (a.bytes) {
    const unsigned lane = threadIdx.x & 31u;
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0 && nbytes) atomicAdd(a.bytes, nbytes);
  }
}

// Blocks per group: about 16 (vertex, word) tasks per warp and level, at
// most 32 blocks.
static int small_group_blocks(int32_t n, int W) {
  const int64_t tasks = (int64_t)n * W;
  const int64_t p = (tasks + SMALL_WARPS * 16 - 1) / (SMALL_WARPS * 16);
  return (int)std::max<int64_t>(1, std::min<int64_t>(32, p));
}

// Co-resident blocks of k_small_bc on the current device (looked up once per device).
static int small_resident_blocks() {
  static int cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0) { cudaGetLastError(); return 1; }
  if (dev < 64 && cache[dev]) return cache[dev];
  int per_sm = 0, sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_small_bc, SMALL_THREADS, 0) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  const int r = std::max(1, per_sm * sms);
  if (dev < 64) cache[dev] = r;
  return r;
}

int small_groups(int32_t n, int nb, int nbatch) {
  const int P = small_group_blocks(n, nb / 32);
  // half of the co-resident blocks at most: other streams keep the rest
  const int cap = std::max(1, small_resident_blocks() / 2 / P);
  return std::max(1, std::min(nbatch, cap));
}

mfbc_status small_run(RunCtx& rc, SmallState& s, const int32_t* d_src_all, const int32_t* d_wreq, int nbatch,
                      double* lambda, int32_t* dist_out, double* sigma_out, int32_t out_rows, uint32_t opt_flags,
                      std::vector<int32_t>* redo) {
  const DevGraph& g = *rc.g;
  redo->clear();
  if (g.n == 0 || nbatch == 0) return MFBC_OK;
  cudaStream_t st = rc.stream;
  SmallArgs a;
  a.n = g.n;
  a.nb = s.nb;
  a.W = s.W;
  a.P = small_group_blocks(g.n, s.W);
  a.rp_in = g.rowptr_t;
  a.col_in = g.col_t;
  a.rp_out = g.rowptr;
  a.col_out = g.col;
  a.src = d_src_all;
  a.wreq = d_wreq;
  a.nbatch = nbatch;
  a.lambda = lambda;
  a.dist_out = dist_out;
  a.sigma_out = sigma_out;
  a.out_rows = out_rows;
  a.lvl = s.lvl;
  a.sv = s.sv;
  a.ctl = s.ctl;
  a.head = s.head;
  a.redo = s.redo;
  a.redo_cap = 4096;
  a.flags = &s.ctr->flags;
  static int khz_cache[64];
  int khz = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); dev = -1; }
  if (dev >= 0 && dev < 64 && khz_cache[dev]) khz = khz_cache[dev];
  else if (dev < 0 || cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev) != cudaSuccess || khz <= 0) {
    cudaGetLastError();
    khz = 2000000;
  } else if (dev < 64) khz_cache[dev] = khz;
  // a wait ends when the group's slowest block finishes its level; one
  // second is far beyond any level of a graph this path takes.  The test
  // hook makes every wait run out, and a short budget keeps that test quick.
  const double wait_s = (opt_flags & MFBC_OPT_TEST_STALL) ? 0.02 : 1.0;
  a.budget = (long long)(wait_s * 1e3 * (double)khz);
  a.stall = (opt_flags & MFBC_OPT_TEST_STALL) ? 1u : 0u;
  a.bytes = rc.prof->count_bytes ? &s.ctr->bytes[K_SMALL] : nullptr;
  const int G = std::min(s.G, std::max(1, nbatch));
  MFBC_CUDA_TRY(cudaMemsetAsync(s.ctl, 0, sizeof(SmallGroupCtl) * (size_t)s.G, st), rc.err);
  MFBC_CUDA_TRY(cudaMemsetAsync(s.head, 0, sizeof(uint32_t) * 2, st), rc.err);
  void* args[] = {&a};
  rc.prof->begin(K_SMALL);
  cudaError_t e = cudaLaunchCooperativeKernel((void*)k_small_bc, dim3((unsigned)(G * a.P)), dim3(SMALL_THREADS),
                                              args, 0, st);
  rc.prof->end(K_SMALL);
  if (e != cudaSuccess) return cuda_fail(rc.err, "cudaLaunchCooperativeKernel(k_small_bc)", e);
  uint32_t h[2];
  MFBC_CUDA_TRY(cudaMemcpyAsync(h, s.head, sizeof(h), cudaMemcpyDeviceToHost, st), rc.err);
  MFBC_CUDA_TRY(cudaMemcpyAsync(rc.h_ctr, &s.ctr->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), rc.err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
  rc.prof->drain();
  if (rc.h_ctr[0] & FLAG_TIMEOUT) {
    if (rc.err) *rc.err = "a block-group barrier of the persistent small-graph kernel waited past its budget";
    return MFBC_ERR_TIMEOUT;
  }
  const int nredo = (int)std::min<uint32_t>(h[1], 4096u);
  if (h[1] > 4096u) {
    if (rc.err) *rc.err = "too many batches need the general kernels";
    return MFBC_ERR_NO_CONVERGENCE;
  }
  if (nredo) {
    redo->resize((size_t)nredo);
    MFBC_CUDA_TRY(cudaMemcpy(redo->data(), s.redo, sizeof(int32_t) * (size_t)nredo, cudaMemcpyDeviceToHost), rc.err);
    std::sort(redo->begin(), redo->end());
  }
  return MFBC_OK;
}

}  // namespace mfbc
