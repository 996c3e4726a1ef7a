// Level path: MFBF (Algorithm 1) and MFBr (Algorithm 2) for unit weights.
//
// With every arc of weight 1 the multpath frontier of MFBF iteration l holds
// exactly the pairs (s,v) with tau(s,v) = l (Lemma 1: the frontier after
// j-1 products carries the shortest paths of exactly j edges), each once.
// The frontier is therefore stored as one bit per (column, vertex) and level,
// F_l[v] (W words of 32 columns), plus a one-bit-per-vertex membership bitmap
// and a vertex list per level.  Multiplicities live in one FP64 array
// sv[v][j] (vertex-major).
//
// MFBF product of level l (gather form of the product F_l (+).f A): for every
// vertex v not yet reached by all columns, and every in-neighbour u of v that
// is in F_l,
//     new(s,v)        = [s in F_l(u)] and not visited(s,v)
//     sigma_bar(s,v) += sigma_bar(s,u)          for those s.
// Over unit weights every candidate of the product has weight l+1, so the
// monoid's minimum is decided by "not yet visited" alone and every candidate
// is a tie that is summed (Sec. 4.1.1); the filter of Algorithm 1 keeps
// exactly the new pairs, which form F_{l+1}.
//
// MFBr (Algorithm 2) over unit weights: a pair (s,v) at level l has its DAG
// successors among the pairs (s,u), u an out-neighbour of v, at level l+1.
// Processing levels in decreasing order makes every counter of Algorithm 2
// reach zero at the level's turn, so the counters need not be stored: level
// l gathers, for each (s,v) in F_l,
//     zeta(s,v) = sum over out-neighbours u with (s,u) in F_{l+1} of
//                 (zeta(s,u) + 1/sigma_bar(s,u))
// (Sec. 4.2.1), adds zeta(s,v) * sigma_bar(s,v) to lambda(v) (Algorithm 3),
// and overwrites sv(s,v) with the frontier value zeta + 1/sigma_bar that its
// predecessors gather one level later.
//
// Work decomposition: the adjacency rows are cut into work items of at most
// CHUNK = 32 arcs, and a product round is two kernels.  The pair kernel gives
// a warp a group of items; lane k reads arc k of an item, membership of the
// neighbour in the level is one bit test per lane, and the member
// neighbours' frontier rows are read whole (lane = 32-column word).  For
// every 128-column quad with a candidate it writes a segment header and one
// pair record (neighbour row, 128-bit column mask) per member neighbour whose
// mask is non-zero there.  The gather kernel takes segments in groups; per
// pair, each lane owns four columns of the quad and issues one 32-byte load
// (one DRAM sector) when its 4-bit slice of the mask is set, summing exact
// 64-bit path counts (MFBF) or compensated double-float values (MFBr).  Rows
// longer than one item ("hubs") combine their items with atomics (sv for
// MFBF, a per-hub FP64 accumulator for MFBr finalised by k_lvl_hub_final).
// Rounds are queued without host reads; a one-thread gate between the two
// kernels turns a round whose pair buffers overflowed into a no-op for the
// host to redo over halves of its items.
#include <algorithm>

#include "dfloat.cuh"
#include "internal.cuh"

namespace mfbc {

constexpr int LVL_WARPS = 8;                 // warps per block
#ifndef MFBC_PAIR_MIN_BLOCKS
#define MFBC_PAIR_MIN_BLOCKS 4
#endif
constexpr unsigned PAIR_GRID = 152u * MFBC_PAIR_MIN_BLOCKS;   // resident blocks of the pair kernels
constexpr uint32_t PAIR_CHUNK = 2048;        // pair slots a warp reserves at a time (> 32 Q = 256)
constexpr uint32_t SEG_CHUNK = 64;           // segment slots a warp reserves at a time (at most)
constexpr uint32_t SEG_DUMMY = 0xffffffffu;  // vertex field of a filler segment

size_t level_bytes(const DevGraph& g, int nb, int Lcap, int64_t list_cap) {
  Carver c(nullptr, 0);
  LevelState s;
  level_carve(c, g, nb, Lcap, list_cap, s);
  return c.off;
}

void level_carve(Carver& c, const DevGraph& g, int nb, int Lcap, int64_t list_cap, LevelState& s) {
  const int32_t n = g.n;
  s.nb = nb;
  s.W = nb / 32;
  s.Lcap = Lcap;
  s.mw = ((int64_t)n + 31) / 32;
  s.sv = c.take<double>((size_t)n * nb);
  s.V = c.take<uint32_t>((size_t)n * s.W);
  s.F = c.take<uint32_t>((size_t)Lcap * n * s.W);
  s.member = c.take<uint32_t>((size_t)Lcap * s.mw);
  s.full = c.take<uint32_t>((size_t)s.mw);
  s.list_cap = list_cap;
  s.lists = c.take<int32_t>((size_t)list_cap);
  s.zacc = c.take<double>((size_t)(g.items_out.nhub > 0 ? g.items_out.nhub : 1) * nb);
  // pair / segment buffers of one product round, sized so that no round
  // overflows them unless the 2^31 clamp binds (a round that overflows is
  // redone over halves of the item range).  A round uses at most Q pairs per
  // arc and Q segments per item.  Warps reserve slots in chunks, and an
  // item whose P pairs (at most 32 Q) do not fit the rest of its warp's
  // chunk leaves that rest unused: each reservation but a warp's first
  // fills at least C - 32 Q + 1 slots before it wastes at most 32 Q - 1, and
  // a warp's last chunk may stay almost empty.  Likewise for segments, whose
  // chunks hold at least 2 Q.
  const int64_t items = std::max(g.items_in.count, g.items_out.count);
  const int64_t Q = std::max(1, s.W / 4);
  const int64_t warps = (int64_t)PAIR_GRID * LVL_WARPS;
  const int64_t pmax = 32 * Q, pairs = std::max<int64_t>(1 << 16, g.nnz * Q);
  const int64_t pair_need = pairs + (pmax - 1) * (warps + pairs / (PAIR_CHUNK - pmax + 1)) + warps * PAIR_CHUNK;
  const int64_t segs = std::max<int64_t>(1 << 16, items * Q);
  const int64_t seg_need = segs + (Q - 1) * (warps + segs / (Q + 1)) + warps * (SEG_CHUNK + Q);
  s.pair_cap = (uint32_t)std::min<int64_t>(0x7fffffff, pair_need);
  s.seg_cap = (uint32_t)std::min<int64_t>(0x7fffffff, seg_need);
  s.prow = c.take<uint32_t>((size_t)s.pair_cap);
  s.pmask = c.take<uint4>((size_t)s.pair_cap);
  s.segs = c.take<uint4>((size_t)s.seg_cap);
  s.src = c.take<int32_t>((size_t)nb);
  s.colmask = c.take<uint32_t>((size_t)s.W);
  s.word_req = c.take<int32_t>((size_t)s.W);
  s.quad_req = c.take<int32_t>((size_t)std::max(1, s.W / 4));
  s.ctr = c.take<Counters>(1);
}

__device__ __forceinline__ bool test_bit(const uint32_t* bm, int32_t v) {
  return (__ldg(&bm[v >> 5]) >> (v & 31)) & 1u;
}

constexpr int NO_REQ = 0x7fffffff;           // key of a lane without a column

__global__ void k_clear_flag_bits(uint32_t* flags, uint32_t bits) { atomicAnd(flags, ~bits); }

// sv rows of multi-item vertices start at zero (MFBF adds into them).
// One warp per row, 32 bytes per lane and store (n_b is a multiple of 128).
__global__ void k_lvl_zero_hubs(const int32_t* __restrict__ hubs, int32_t nhub, int nb, double* sv) {
  const unsigned lane = lane_id();
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t h = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; h < (uint64_t)nhub; h += nw) {
    double* row = sv + (size_t)hubs[h] * nb;
    for (int c = 4 * (int)lane; c < nb; c += 128)
      asm volatile("st.global.v4.u64 [%0], {%1,%1,%1,%1};" ::"l"(row + c), "l"(0ull) : "memory");
  }
}

// Level 0: F_0(s_j) holds column j, sigma_bar(s_j, s_j) = 1.
__global__ void k_lvl_seed(const int32_t* __restrict__ src, int nb, int W, double* sv, uint32_t* F0,
                           uint32_t* member0, int32_t* list0, uint32_t* count) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nb) return;
  const int32_t s = src[j];
  if (s < 0) return;
  reinterpret_cast<uint64_t*>(sv)[(size_t)s * nb + j] = 1ull;   // sigma_bar as an exact integer
  atomicOr(&F0[(size_t)s * W + (j >> 5)], 1u << (j & 31));
  const uint32_t bit = 1u << (s & 31);
  if (!(atomicOr(&member0[s >> 5], bit) & bit)) list0[atomicAdd(count, 1u)] = s;
}

// colmask[w] = the columns of word w whose source is set (one warp per word).
__global__ void k_lvl_colmask(const int32_t* __restrict__ src, int W, uint32_t* colmask) {
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  if (w >= W) return;
  const uint32_t m = __ballot_sync(0xffffffffu, src[w * 32 + (int)lane_id()] >= 0);
  if (lane_id() == 0) colmask[w] = m;
}

// visited |= F_l for the vertices of level l; mark vertices reached by every
// column that holds a source (colmask).
__device__ __forceinline__ void visit_rows(const int32_t* __restrict__ list, uint32_t count, int W,
                                           const uint32_t* __restrict__ colmask, const uint32_t* __restrict__ Fl,
                                           uint32_t* V, uint32_t* full) {
  const unsigned lane = lane_id();
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += nw) {
    const int32_t v = list[i];
    bool ok = true;
    if ((int)lane < W) {
      const size_t r = (size_t)v * W + lane;
      const uint32_t x = V[r] | Fl[r];
      V[r] = x;
      const uint32_t am = colmask[lane];
      ok = (x & am) == am;
    }
    if (__all_sync(0xffffffffu, ok) && lane == 0) atomicOr(&full[v >> 5], 1u << (v & 31));
  }
}
__global__ void k_lvl_visit(const int32_t* __restrict__ list, uint32_t count, int W,
                            const uint32_t* __restrict__ colmask, const uint32_t* __restrict__ Fl, uint32_t* V,
                            uint32_t* full) {
  visit_rows(list, count, W, colmask, Fl, V, full);
}

// The visit of the next level, run by the MFBF gather of the current one
// after its segments (the gather neither reads V nor full, and the next pair
// kernel starts after it), which saves a launch per level.
struct VisitNext {
  const int32_t* list;       // the next level's vertices
  const uint32_t* count;     // their number (device, written by the pair kernel); nullptr: no visit here
  int64_t cap;               // room of the list (a longer count is clamped; the batch is then redone)
  int W;
  const uint32_t* colmask;
  const uint32_t* Fn;        // the next level's frontier rows
  uint32_t* V;
  uint32_t* full;
};

// Segments per group when the host left it open (0): the host's rule (see
// group_size), from the count the pair kernel left on the device.
__device__ __forceinline__ int seg_group_of(uint32_t nseg, int given) {
  if (given > 0) return given;
  int g = 32;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  while (g > 1 && (uint64_t)nseg < (uint64_t)g * warps * 4) g >>= 1;
  return g;
}

// Between the pair kernel and the gather of a round queued without a host
// read (one thread): when the pair buffers overflowed (work[3]), or an earlier
// round of the same MFBr sweep did (flags bit FLAG_ROUND_ABORT, kept until the
// host clears it), the gather is given no segment and the MFBF gather no
// visit; an MFBr overflow sets the flag and records its level.  The host
// finds the overflow at its next read of the counters and redoes the round
// over halves of the items; the skipped round wrote nothing.
__global__ void k_lvl_round_gate(uint32_t* work, const uint32_t* list_count, uint32_t* flags, uint32_t* abort_level,
                                 uint32_t* visit_count, int level, int bwd) {
  const bool ovf = work[3] != 0u;
  if (ovf && bwd) {
    atomicOr(flags, FLAG_ROUND_ABORT);
    atomicMax(abort_level, (uint32_t)level);
  }
  const bool skip = ovf || (*flags & FLAG_ROUND_ABORT);
  if (skip) work[1] = 0u;
  *visit_count = skip ? 0u : *list_count;
}

// Per-warp shared memory of the pair kernels.
struct WarpSmem {
  int32_t su[32];                            // member neighbour ids of the item
  int32_t newv[32];                          // vertices entering the next level, not yet appended
  uint32_t sF[32][33];                       // member q's masked frontier word j (padded: no bank conflicts)
};
constexpr size_t LVL_SMEM = sizeof(WarpSmem) * LVL_WARPS;

#ifndef MFBC_GATHER_U
#define MFBC_GATHER_U 4
#endif
constexpr int GATHER_U = MFBC_GATHER_U;      // gather loads in flight per warp
#ifndef MFBC_GATHER_MIN_BLOCKS
#define MFBC_GATHER_MIN_BLOCKS 4
#endif
#ifndef MFBC_BWD_GATHER_MIN_BLOCKS
#define MFBC_BWD_GATHER_MIN_BLOCKS MFBC_GATHER_MIN_BLOCKS
#endif

// Item metadata: first arc (bits 0..39), arc count (bits 40..45), multi-item row (bit 46).
__device__ __forceinline__ int64_t meta_beg(int64_t m) { return m & ((1ll << 40) - 1); }
__device__ __forceinline__ int meta_len(int64_t m) { return (int)((m >> 40) & 63); }
__device__ __forceinline__ bool meta_multi(int64_t m) { return (m >> 46) & 1; }

// Gathers move 128 columns at a time ("quads"): lane l of a warp covers the
// four columns 4l..4l+3 of the quad, i.e. exactly one 32-byte sector of a
// vertex row, so a lane loads a sector only when one of its four columns is
// needed.  n_b is a multiple of 128 on the level path; Q = n_b / 128 quads
// per row, and row index u*Q + d names quad d of vertex u.
//
// Pair record: row index (uint32) and the 128-column mask (uint4, word w of
// the quad in component w).  Segment header: (v, first pair, count | quad << 8
// | multi-item row << 16, 0); a segment is one (vertex, quad) of one work item.
__device__ __forceinline__ uint4 make_seg(int32_t v, uint32_t pb, int cnt, int d, bool multi) {
  return make_uint4((uint32_t)v, pb, (uint32_t)cnt | ((uint32_t)d << 8) | ((uint32_t)multi << 16), 0u);
}

__device__ __forceinline__ uint32_t quad_or(const WarpSmem& w, int q, int d) {
  return w.sF[q][4 * d] | w.sF[q][4 * d + 1] | w.sF[q][4 * d + 2] | w.sF[q][4 * d + 3];
}

// Pair and segment slots reserved by one warp.  Slots are taken from the
// round's counters in chunks (one atomic per chunk rather than two per item:
// the counters sit in one L2 slice).  Pair slots left at the end of a chunk
// are never referenced; segment slots left over when a warp takes a new
// chunk or finishes are filled with headers whose vertex is SEG_DUMMY, which
// the gathers skip.
struct SlotCursor { uint32_t p = 0, pe = 0, s = 0, se = 0; };

// Reserve max(need, chunk) slots; false (cursor emptied, overflow flagged)
// when the buffer cannot hold them.
__device__ __forceinline__ bool reserve_slots(uint32_t* counter, uint32_t need, uint32_t chunk, uint32_t cap,
                                              uint32_t* overflow, uint32_t& b, uint32_t& e) {
  const uint32_t sz = need > chunk ? need : chunk;
  uint32_t x = 0;
  if (lane_id() == 0) x = atomicAdd(counter, sz);
  x = __shfl_sync(0xffffffffu, x, 0);
  if ((uint64_t)x + sz > cap) {
    if (lane_id() == 0) atomicOr(overflow, 1u);
    b = e = 0;
    return false;
  }
  b = x;
  e = x + sz;
  return true;
}

__device__ __forceinline__ void fill_dummy_segs(uint4* segs, uint32_t b, uint32_t e) {
  for (uint32_t i = b + lane_id(); i < e; i += 32) segs[i] = make_uint4(SEG_DUMMY, 0u, 0u, 0u);
}

// Emit the (member, mask) pairs of one item, quad by quad over `quads`
// (ascending), as segments.  Returns false (writing nothing) when the
// buffers are full.
__device__ __forceinline__ bool emit_quads(const WarpSmem& w, int nm, int32_t v, bool multi, uint32_t quads, int Q,
                                           const uint32_t* __restrict__ hot, uint32_t* prow, uint4* pmask,
                                           uint4* segs, uint32_t* work,
                                           uint32_t pair_cap, uint32_t seg_cap, SlotCursor& cur,
                                           unsigned long long* npairs, uint32_t seg_chunk) {
  const unsigned lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  int mycnt = 0;
  for (uint32_t ql = quads; ql; ql &= ql - 1) {
    const int d = __ffs(ql) - 1;
    const uint32_t mk = __ballot_sync(0xffffffffu, ((int)lane < nm) && quad_or(w, lane, d) != 0u);
    if ((int)lane == d) mycnt = __popc(mk);
  }
  int incl = mycnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  const int excl = incl - mycnt;
  const uint32_t P = (uint32_t)__shfl_sync(0xffffffffu, incl, 31);
  const uint32_t S = (uint32_t)__popc(quads);
  if (cur.p + P > cur.pe && !reserve_slots(&work[0], P, PAIR_CHUNK, pair_cap, &work[3], cur.p, cur.pe))
    return false;
  if (cur.s + S > cur.se) {
    fill_dummy_segs(segs, cur.s, cur.se);
    if (!reserve_slots(&work[1], S, seg_chunk, seg_cap, &work[3], cur.s, cur.se)) return false;
  }
  const uint32_t pb = cur.p, sb = cur.s;
  cur.p += P;
  cur.s += S;
  // bit 31 of a pair's row index: the row belongs to a high-degree vertex
  const uint32_t hotbit = ((int)lane < nm && hot && test_bit(hot, w.su[lane])) ? 0x80000000u : 0u;
  if (npairs) *npairs += P + (uint64_t)S * (1ull << 32);   // pairs in the low word, segments in the high
  int r = 0;
  for (uint32_t ql = quads; ql; ql &= ql - 1, r++) {
    const int d = __ffs(ql) - 1;
    const bool nz = ((int)lane < nm) && quad_or(w, lane, d) != 0u;
    const uint32_t mk = __ballot_sync(0xffffffffu, nz);
    const uint32_t off = (uint32_t)__shfl_sync(0xffffffffu, excl, d);
    if (nz) {
      const uint32_t at = pb + off + __popc(mk & lt);
      prow[at] = ((uint32_t)w.su[lane] * (uint32_t)Q + (uint32_t)d) | hotbit;
      pmask[at] = make_uint4(w.sF[lane][4 * d], w.sF[lane][4 * d + 1], w.sF[lane][4 * d + 2], w.sF[lane][4 * d + 3]);
    }
    if (lane == 0) segs[sb + r] = make_seg(v, pb + off, __popc(mk), d, multi);
  }
  return true;
}

// quads (bit d) touched by the non-zero words of a word ballot
__device__ __forceinline__ uint32_t quads_of_words(uint32_t words, int Q) {
  uint32_t q = 0;
  for (int d = 0; d < Q; d++)
    if ((words >> (4 * d)) & 0xfu) q |= 1u << d;
  return q;
}

// Work items are handed out in groups of ig <= 32 (hub items cost far more
// than leaf items); the group counter is zeroed before each launch.  ig is 32
// unless the range is too short to give every resident warp several groups
// (small graphs), where smaller groups spread it over more warps.  (Handing
// out 4 to 16 groups per atomic was measured slower: balance matters more
// than the counter.)
#define FOR_ITEM_GROUPS(ib, ie, counter, ig)                                                \
  for (;;) {                                                                              \
    uint32_t grp_ = 0;                                                                    \
    if (lane == 0) grp_ = atomicAdd(counter, 1u);                                         \
    const uint64_t base = (uint64_t)(ib) + (uint64_t)__shfl_sync(0xffffffffu, grp_, 0) * (uint64_t)(ig); \
    if (base >= (uint64_t)(ie)) break;

// MFBF pairs of level l (see file comment): for items [ib, ie) of rows not yet
// reached by every column, the masks F_l(u) & ~visited(v) of the in-neighbours
// u in F_l, the next frontier bits F_{l+1}(v), and the level-(l+1) list.
__global__ void __launch_bounds__(LVL_WARPS * 32, MFBC_PAIR_MIN_BLOCKS) k_lvl_fwd_pairs(
    int64_t ib, int64_t ie, const int32_t* __restrict__ item_v, const int64_t* __restrict__ item_meta,
    const int32_t* __restrict__ col_t, int W, const uint32_t* __restrict__ full, const uint32_t* __restrict__ V,
    const uint32_t* __restrict__ Fl, const uint32_t* __restrict__ mem_l, uint32_t* Fn, uint32_t* mem_n,
    int32_t* list_n, uint32_t* count_n, int64_t cap_n, uint32_t* flags, uint32_t* next_group, uint32_t* prow,
    uint4* pmask, uint4* segs, uint32_t* work, uint32_t pair_cap, uint32_t seg_cap, const uint32_t* __restrict__ hot,
    unsigned long long* bytes, unsigned long long* stat, int ig, uint32_t seg_chunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem& sm = reinterpret_cast<WarpSmem*>(smem_raw)[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  const int Q = W / 4;
  unsigned long long nbytes = 0, npairs = 0;
  SlotCursor cur;
  int nnew = 0;                                    // entries of sm.newv
  if (*((volatile const uint32_t*)flags) & FLAG_ROUND_ABORT) return;
  // append sm.newv to the level-(l+1) list with one atomic
  auto flush_new = [&]() {
    uint32_t b = 0;
    if (lane == 0) b = atomicAdd(count_n, (uint32_t)nnew);
    b = __shfl_sync(0xffffffffu, b, 0);
    __syncwarp();
    if ((int)lane < nnew) {
      const uint32_t pos = b + lane;
      if ((int64_t)pos < cap_n) list_n[pos] = sm.newv[lane];
      else atomicOr(flags, FLAG_LEVEL_LIST);
    }
    __syncwarp();
    nnew = 0;
  };
  FOR_ITEM_GROUPS(ib, ie, next_group, ig)
    // lane-parallel precheck of the group's items: skip rows already reached by every column
    const uint64_t myit = base + lane;
    int32_t myv = 0;
    int64_t mymeta = 0;
    bool act = false;
    if ((int)lane < ig && myit < (uint64_t)ie) {
      myv = item_v[myit];
      mymeta = item_meta[myit];
      act = !test_bit(full, myv);
    }
    uint32_t am = __ballot_sync(0xffffffffu, act);
    // the next active item's neighbour ids and visited row are loaded one item ahead
    int32_t nv = 0, nu = -1;
    int64_t nmeta = 0;
    uint32_t nVv = 0xffffffffu;
    if (am) {
      const int t = __ffs(am) - 1;
      nv = __shfl_sync(0xffffffffu, myv, t);
      nmeta = __shfl_sync(0xffffffffu, mymeta, t);
      nu = (int)lane < meta_len(nmeta) ? __ldg(&col_t[meta_beg(nmeta) + lane]) : -1;
      nVv = (int)lane < W ? V[(size_t)nv * W + lane] : 0xffffffffu;
      am &= am - 1;
    }
    for (bool have = __ballot_sync(0xffffffffu, act) != 0u; have;) {
      const int32_t v = nv;
      const int64_t meta = nmeta;
      const int32_t u = nu;
      const uint32_t Vv = nVv;
      have = am != 0u;
      if (have) {
        const int t = __ffs(am) - 1;
        nv = __shfl_sync(0xffffffffu, myv, t);
        nmeta = __shfl_sync(0xffffffffu, mymeta, t);
        nu = (int)lane < meta_len(nmeta) ? __ldg(&col_t[meta_beg(nmeta) + lane]) : -1;
        nVv = (int)lane < W ? V[(size_t)nv * W + lane] : 0xffffffffu;
        am &= am - 1;
      }
      const int len = meta_len(meta);
      const bool multi = meta_multi(meta);
      const bool isMem = u >= 0 && test_bit(mem_l, u);
      const uint32_t mm = __ballot_sync(0xffffffffu, isMem);
      if (bytes) nbytes += 4ull * len + 12ull;
      if (!mm) continue;
      const int nm = __popc(mm);
      if (isMem) sm.su[__popc(mm & lt)] = u;
      __syncwarp();
      uint32_t cand = 0;
      for (int q0 = 0; q0 < nm; q0 += 8) {          // eight frontier rows in flight
        uint32_t f[8];
#pragma unroll
        for (int t = 0; t < 8; t++)
          f[t] = (q0 + t < nm && (int)lane < W) ? __ldg(&Fl[(size_t)sm.su[q0 + t] * W + lane]) : 0u;
#pragma unroll
        for (int t = 0; t < 8; t++) {
          if (q0 + t < nm) {
            const uint32_t mk = f[t] & ~Vv;
            sm.sF[q0 + t][lane] = mk;
            cand |= mk;
          }
        }
      }
      __syncwarp();
      if (bytes) nbytes += 4ull * W * (nm + 1);
      const uint32_t cw = __ballot_sync(0xffffffffu, cand != 0u);
      if (!cw) continue;
      emit_quads(sm, nm, v, multi, quads_of_words(cw, Q), Q, hot, prow, pmask, segs, work, pair_cap, seg_cap, cur,
                 bytes ? &npairs : nullptr, seg_chunk);
      if ((int)lane < W && cand) {
        if (multi) atomicOr(&Fn[(size_t)v * W + lane], cand);
        else Fn[(size_t)v * W + lane] = cand;
      }
      uint32_t isnew = 0;
      if (lane == 0) {
        const uint32_t bit = 1u << (v & 31);
        isnew = !(atomicOr(&mem_n[v >> 5], bit) & bit);
        if (isnew) sm.newv[nnew] = v;
      }
      nnew += (int)__shfl_sync(0xffffffffu, isnew, 0);
      __syncwarp();
      if (nnew == 32) flush_new();
    }
  }
  if (nnew) flush_new();
  fill_dummy_segs(segs, cur.s, cur.se);
  if (bytes && lane == 0) {
    const unsigned long long np = npairs & 0xffffffffull, ns = npairs >> 32;
    atomicAdd(bytes, nbytes + 20ull * np + 16ull * ns);
    atomicAdd(&stat[0], np);
  }
}

// MFBr pairs of level l >= 1: for items [ib, ie) of rows with a column at
// level l, the masks F_{l+1}(u) & F_l(v) of the out-neighbours u in F_{l+1}.
// Every level-l quad of a single-item row gets a segment (its columns are
// finalised by the gather even without successors); multi-item rows only emit
// quads with pairs (their finalisation is k_lvl_hub_final).
__global__ void __launch_bounds__(LVL_WARPS * 32, MFBC_PAIR_MIN_BLOCKS) k_lvl_bwd_pairs(
    int64_t ib, int64_t ie, const int32_t* __restrict__ item_v, const int64_t* __restrict__ item_meta,
    const int32_t* __restrict__ col, int W, const uint32_t* __restrict__ Fl, const uint32_t* __restrict__ mem_l,
    const uint32_t* __restrict__ Fn, const uint32_t* __restrict__ mem_n, uint32_t* next_group, uint32_t* prow,
    uint4* pmask, uint4* segs, uint32_t* work, uint32_t pair_cap, uint32_t seg_cap, const uint32_t* __restrict__ hot,
    unsigned long long* bytes, unsigned long long* stat, int ig, const uint32_t* flags, uint32_t seg_chunk) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  WarpSmem& sm = reinterpret_cast<WarpSmem*>(smem_raw)[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  const int Q = W / 4;
  unsigned long long nbytes = 0, npairs = 0;
  SlotCursor cur;
  if (*((volatile const uint32_t*)flags) & FLAG_ROUND_ABORT) return;
  FOR_ITEM_GROUPS(ib, ie, next_group, ig)
    // lane-parallel precheck of the group's items: only rows with a column at level l
    const uint64_t myit = base + lane;
    int32_t myv = 0;
    int64_t mymeta = 0;
    bool act = false;
    if ((int)lane < ig && myit < (uint64_t)ie) {
      myv = item_v[myit];
      mymeta = item_meta[myit];
      act = test_bit(mem_l, myv);
    }
    uint32_t am = __ballot_sync(0xffffffffu, act);
    // the next active item's neighbour ids and frontier row are loaded one item ahead
    int32_t nv = 0, nu = -1;
    int64_t nmeta = 0;
    uint32_t nFv = 0u;
    if (am) {
      const int t = __ffs(am) - 1;
      nv = __shfl_sync(0xffffffffu, myv, t);
      nmeta = __shfl_sync(0xffffffffu, mymeta, t);
      nu = (int)lane < meta_len(nmeta) ? __ldg(&col[meta_beg(nmeta) + lane]) : -1;
      nFv = (int)lane < W ? __ldg(&Fl[(size_t)nv * W + lane]) : 0u;
      am &= am - 1;
    }
    for (bool have = __ballot_sync(0xffffffffu, act) != 0u; have;) {
      const int32_t v = nv;
      const int64_t meta = nmeta;
      const int32_t u = nu;
      const uint32_t Fv = nFv;
      have = am != 0u;
      if (have) {
        const int t = __ffs(am) - 1;
        nv = __shfl_sync(0xffffffffu, myv, t);
        nmeta = __shfl_sync(0xffffffffu, mymeta, t);
        nu = (int)lane < meta_len(nmeta) ? __ldg(&col[meta_beg(nmeta) + lane]) : -1;
        nFv = (int)lane < W ? __ldg(&Fl[(size_t)nv * W + lane]) : 0u;
        am &= am - 1;
      }
      const int len = meta_len(meta);
      const bool multi = meta_multi(meta);
      const bool isMem = u >= 0 && test_bit(mem_n, u);
      const uint32_t mm = __ballot_sync(0xffffffffu, isMem);
      if (bytes) nbytes += 4ull * len + 12ull;
      if (multi && !mm) continue;                    // nothing to add to the hub accumulator
      const int nm = __popc(mm);
      if (isMem) sm.su[__popc(mm & lt)] = u;
      __syncwarp();
      uint32_t any = 0;
      for (int q0 = 0; q0 < nm; q0 += 8) {          // eight frontier rows in flight
        uint32_t f[8];
#pragma unroll
        for (int t = 0; t < 8; t++)
          f[t] = (q0 + t < nm && (int)lane < W) ? __ldg(&Fn[(size_t)sm.su[q0 + t] * W + lane]) : 0u;
#pragma unroll
        for (int t = 0; t < 8; t++) {
          if (q0 + t < nm) {
            sm.sF[q0 + t][lane] = f[t] & Fv;
            any |= f[t] & Fv;
          }
        }
      }
      __syncwarp();
      if (bytes) nbytes += 4ull * W * (nm + 1);
      const uint32_t words = __ballot_sync(0xffffffffu, multi ? any != 0u : Fv != 0u);
      if (words) emit_quads(sm, nm, v, multi, quads_of_words(words, Q), Q, hot, prow, pmask, segs, work, pair_cap,
                            seg_cap, cur, bytes ? &npairs : nullptr, seg_chunk);
      __syncwarp();
    }
  }
  fill_dummy_segs(segs, cur.s, cur.se);
  if (bytes && lane == 0) {
    const unsigned long long np = npairs & 0xffffffffull, ns = npairs >> 32;
    atomicAdd(bytes, nbytes + 20ull * np + 16ull * ns);
    atomicAdd(&stat[1], np);
  }
}

// Per-warp shared staging of one chunk of 32 pairs in the gather kernels.
struct GatherSmem {
  uint4 mask[32];
  uint32_t row[32];
  int32_t seg[32];
};

__device__ __forceinline__ void ld4(const double* p, double& a, double& b, double& c, double& d) {
  asm volatile("ld.global.nc.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(a), "=d"(b), "=d"(c), "=d"(d) : "l"(p));
}
__device__ __forceinline__ void ld4_coherent(const double* p, double& a, double& b, double& c, double& d) {
  asm volatile("ld.global.v4.f64 {%0,%1,%2,%3}, [%4];" : "=d"(a), "=d"(b), "=d"(c), "=d"(d) : "l"(p) : "memory");
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
  asm volatile("st.global.v4.f64 [%0], {%1,%2,%3,%4};" ::"l"(p), "d"(a), "d"(b), "d"(c), "d"(d) : "memory");
}

// Gather over a group of up to 32 segments (lane k holds segment k's header).
// The group's pairs are flattened with a warp scan and staged 32 at a time in
// shared memory; each pair costs every lane one broadcast row read, one mask
// word read and, when one of its four columns is set, one 32-byte load.
// FLUSH(k, acc) is called once per segment with pairs, in order, by the whole
// warp, with the lane's four column sums and the OR of its 4-bit slices.
template <bool COUNT>
__device__ __forceinline__ void stage_chunk(const uint4& myseg, int excl, int incl, int T, int p0,
                                            const uint32_t* __restrict__ prow, const uint4* __restrict__ pmask,
                                            GatherSmem& gs, uint32_t* lastmask) {
  const unsigned lane = lane_id();
  const int p = p0 + (int)lane;
  int t = 0;
#pragma unroll
  for (int step = 16; step; step >>= 1) {            // largest t with excl_t <= p
    const int e = __shfl_sync(0xffffffffu, excl, t + step > 31 ? 31 : t + step);
    if (t + step <= 31 && e <= p) t += step;
  }
  // excl is non-decreasing and empty segments share their successor's excl,
  // so the largest such t is the segment that holds pair p
  const uint32_t tpb = __shfl_sync(0xffffffffu, myseg.y, t);
  const int texcl = __shfl_sync(0xffffffffu, excl, t);
  const int tincl = __shfl_sync(0xffffffffu, incl, t);
  __syncwarp();
  if (p < T) {
    const uint32_t at = tpb + (uint32_t)(p - texcl);
    gs.mask[lane] = pmask[at];
    gs.row[lane] = prow[at];
    gs.seg[lane] = t;
  }
  *lastmask = __ballot_sync(0xffffffffu, p < T && p + 1 == tincl);
  __syncwarp();
}

// Gather load of one 32-byte sector (four columns of one vertex row of sv).
//
// Other warps of the same launch write sv while the gathers read it, so the
// loads are ordinary coherent loads that skip L1 allocation.  No element is
// both read and written by one launch (the MFBF gather of level l reads
// sigma_bar of level-l pairs and writes level-(l+1) pairs; the MFBr gather of
// level l reads level-(l+1) values and overwrites level-l pairs), but a loaded
// sector can hold a column that the launch writes, since a vertex has columns
// at several levels.  The columns a gather uses (the pair's mask) are never
// written during the launch, so the read-only path (-DMFBC_GATHER_NC=1) gives
// the same results; on R-MAT 22 both run at the same speed (311.2 GTEPS).
#ifndef MFBC_GATHER_NC
#define MFBC_GATHER_NC 0
#endif
// Rows of high-degree vertices (bit 31 of the pair's row index) are loaded
// with the L2 evict-last priority: most DAG arcs end there, so their sectors
// are read again and again within a level, while the rows of the many
// low-degree vertices stream through.  A hint only; results do not depend on it.
#ifndef MFBC_HOT_HINT
#define MFBC_HOT_HINT 1
#endif
__device__ __forceinline__ void ld4u_keep(const uint64_t* p, uint64_t& a, uint64_t& b, uint64_t& c, uint64_t& d) {
  asm volatile("ld.global.L1::no_allocate.L2::evict_last.v4.u64 {%0,%1,%2,%3}, [%4];"
               : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
}
__device__ __forceinline__ void ld4u(const uint64_t* p, uint64_t& a, uint64_t& b, uint64_t& c, uint64_t& d) {
#if MFBC_GATHER_NC
  asm volatile("ld.global.nc.L1::no_allocate.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
#else
  asm volatile("ld.global.L1::no_allocate.v4.u64 {%0,%1,%2,%3}, [%4];" : "=l"(a), "=l"(b), "=l"(c), "=l"(d) : "l"(p));
#endif
}

// Gather over a group of up to 32 segments (lane k holds segment k's header).
// The group's pairs are flattened with a warp scan and staged 32 at a time in
// shared memory; each pair costs every lane one broadcast row read, one mask
// word read and, when one of its four columns is set, one 32-byte load.
// MFBF (INT = true) sums exact 64-bit path counts; MFBr sums double-float
// values with compensation.  FLUSH(k, ...) is called once per segment with
// pairs, in order, by the whole warp, with the lane's four column sums and
// the OR of its 4-bit slices.
template <bool COUNT, bool INT, class Flush>
__device__ __forceinline__ void gather_group(const uint4& myseg, int nin, const uint32_t* __restrict__ prow,
                                             const uint4* __restrict__ pmask, GatherSmem& gs, const uint64_t* sv,
                                             unsigned long long& nvals, unsigned long long& nvals_rec, uint32_t& ovf,
                                             Flush flush) {
  const unsigned lane = lane_id();
  const int mycnt = (int)lane < nin ? (int)(myseg.z & 0xffu) : 0;
  int incl = mycnt;
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if ((int)lane >= o) incl += y;
  }
  const int excl = incl - mycnt;
  const int T = __shfl_sync(0xffffffffu, incl, 31);
  // algorithmic bytes of the group's records: 16 B per segment header and
  // 20 B per pair (row index + mask), counted once (by lane 0)
  if (COUNT) {
    const uint32_t real = __ballot_sync(0xffffffffu, (int)lane < nin && myseg.x != SEG_DUMMY);
    if (lane == 0) nvals_rec += 16ull * __popc(real) + 20ull * T;
  }
  const int shift = 4 * (int)(lane & 7u);
  const int mword = (int)(lane >> 3);
  uint64_t i0 = 0, i1 = 0, i2 = 0, i3 = 0;                 // MFBF sums
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;            // MFBr sums
  float c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;            //   and their compensations
  uint32_t cs = 0;
  for (int p0 = 0; p0 < T; p0 += 32) {
    uint32_t lastmask;
    stage_chunk<COUNT>(myseg, excl, incl, T, p0, prow, pmask, gs, &lastmask);
    const int nq = T - p0 < 32 ? T - p0 : 32;
    for (int q0 = 0; q0 < nq; q0 += GATHER_U) {
      uint64_t x[GATHER_U][4];
      uint32_t sl[GATHER_U];
#pragma unroll
      for (int r = 0; r < GATHER_U; r++) {
        const int q = q0 + r;
        sl[r] = 0u;
        x[r][0] = x[r][1] = x[r][2] = x[r][3] = 0ull;
        if (q < nq) {
          const uint32_t mw = reinterpret_cast<const uint32_t*>(&gs.mask[q])[mword];
          sl[r] = (mw >> shift) & 0xfu;
          if (sl[r]) {
            const uint32_t rr = gs.row[q];
            const uint64_t* p = sv + (size_t)(rr & 0x7fffffffu) * 128 + 4 * lane;
            if (rr >> 31) ld4u_keep(p, x[r][0], x[r][1], x[r][2], x[r][3]);
            else ld4u(p, x[r][0], x[r][1], x[r][2], x[r][3]);
            if (COUNT) nvals += __popc(sl[r]);
          }
        }
      }
#pragma unroll
      for (int r = 0; r < GATHER_U; r++) {
        const int q = q0 + r;
        if (q < nq) {
          if (INT) {
            // no wrap check per add: stored counts stay below 2^58 (larger
            // sums are flagged at the flush), and a segment adds <= 32 of them
            if (sl[r] & 1u) i0 += x[r][0];
            if (sl[r] & 2u) i1 += x[r][1];
            if (sl[r] & 4u) i2 += x[r][2];
            if (sl[r] & 8u) i3 += x[r][3];
          } else {
            if (sl[r] & 1u) acc_add(s0, c0, x[r][0]);
            if (sl[r] & 2u) acc_add(s1, c1, x[r][1]);
            if (sl[r] & 4u) acc_add(s2, c2, x[r][2]);
            if (sl[r] & 8u) acc_add(s3, c3, x[r][3]);
          }
          cs |= sl[r];
          if ((lastmask >> q) & 1u) {
            flush(gs.seg[q], i0, i1, i2, i3, s0, s1, s2, s3, c0, c1, c2, c3, cs);
            i0 = i1 = i2 = i3 = 0ull;
            s0 = s1 = s2 = s3 = c0 = c1 = c2 = c3 = 0.f;
            cs = 0u;
          }
        }
      }
    }
  }
}

// Segments are handed out in groups of gs <= 32 (lane k holds segment k of
// the group); gs < 32 only when there are too few segments to give every
// resident warp several groups.
#define FOR_SEGMENT_GROUPS(nseg, counter, gs)                                                \
  for (;;) {                                                                               \
    uint32_t grp_ = 0;                                                                     \
    if (lane == 0) grp_ = atomicAdd(counter, 1u);                                          \
    const uint64_t base = (uint64_t)__shfl_sync(0xffffffffu, grp_, 0) * (uint64_t)(gs);    \
    if (base >= (uint64_t)(nseg)) break;                                                   \
    const int nin = (uint64_t)(nseg) - base < (uint64_t)(gs) ? (int)((uint64_t)(nseg) - base) : (gs); \
    uint4 myseg = make_uint4(0u, 0u, 0u, 0u);                                              \
    if ((int)lane < nin) myseg = segs[base + lane];

// MFBF gather of level l: sigma_bar(s,v) = sum over the segment's pairs
// (exact 64-bit integers).  flags: bit 1 some sigma_bar >= 2^53, bit 3 a sum
// passed 2^64 (the batch is then recomputed by the general kernels).
template <bool COUNT, bool G32>
__global__ void __launch_bounds__(256, MFBC_GATHER_MIN_BLOCKS) k_lvl_fwd_gather(
    const uint4* __restrict__ segs, const uint32_t* nseg_p, const uint32_t* __restrict__ prow,
    const uint4* __restrict__ pmask, int nb, double* svd, uint32_t* flags, uint32_t* next_group,
    unsigned long long* bytes, unsigned long long* stat, VisitNext vn, int seg_group) {
  __shared__ GatherSmem gsm[8];
  GatherSmem& gs = gsm[threadIdx.x >> 5];
  uint64_t* sv = reinterpret_cast<uint64_t*>(svd);
  const unsigned lane = lane_id();
  const uint32_t nseg = *nseg_p;
  if (!G32) seg_group = seg_group_of(nseg, seg_group);
  unsigned long long nvals = 0, nw = 0, nrec = 0;
  uint32_t ovf = 0, big = 0;
  FOR_SEGMENT_GROUPS(nseg, next_group, G32 ? 32 : seg_group)
    gather_group<COUNT, true>(myseg, nin, prow, pmask, gs, sv, nvals, nrec, ovf,
        [&](int k, uint64_t a0, uint64_t a1, uint64_t a2, uint64_t a3, float, float, float, float, float, float,
            float, float, uint32_t cs) {
      const int32_t v = (int32_t)__shfl_sync(0xffffffffu, myseg.x, k);
      const uint32_t z = __shfl_sync(0xffffffffu, myseg.z, k);
      const int d = (int)((z >> 8) & 0xffu);
      if (cs) {
        uint64_t* dst = sv + (size_t)v * nb + 128 * d + 4 * lane;
        uint64_t t0 = a0, t1 = a1, t2 = a2, t3 = a3;
        if ((z >> 16) & 1u) {
          unsigned long long* da = reinterpret_cast<unsigned long long*>(dst);
          if (cs & 1u) { const uint64_t o = atomicAdd(da + 0, (unsigned long long)a0); t0 = o + a0; ovf |= t0 < o; }
          if (cs & 2u) { const uint64_t o = atomicAdd(da + 1, (unsigned long long)a1); t1 = o + a1; ovf |= t1 < o; }
          if (cs & 4u) { const uint64_t o = atomicAdd(da + 2, (unsigned long long)a2); t2 = o + a2; ovf |= t2 < o; }
          if (cs & 8u) { const uint64_t o = atomicAdd(da + 3, (unsigned long long)a3); t3 = o + a3; ovf |= t3 < o; }
        } else if (cs == 0xfu) {
          asm volatile("st.global.v4.u64 [%0], {%1,%2,%3,%4};" ::"l"(dst), "l"(a0), "l"(a1), "l"(a2), "l"(a3)
                       : "memory");
        } else {
          if (cs & 1u) dst[0] = a0;
          if (cs & 2u) dst[1] = a1;
          if (cs & 4u) dst[2] = a2;
          if (cs & 8u) dst[3] = a3;
        }
        // bit 1: a count reached 2^53 (FP64 output inexact); bit 3: a count
        // reached 2^58 (later sums could wrap 2^64: the batch is redone by the
        // general kernels)
        const uint64_t m = ((cs & 1u) ? t0 : 0ull) | ((cs & 2u) ? t1 : 0ull) | ((cs & 4u) ? t2 : 0ull) |
                           ((cs & 8u) ? t3 : 0ull);
        big |= (uint32_t)(m >= (1ull << 53));
        ovf |= (uint32_t)(m >= (1ull << 58));
        if (COUNT) nw += __popc(cs);
      }
    });
  }
  if (__any_sync(0xffffffffu, big != 0u) && lane == 0) atomicOr(flags, FLAG_SIGMA_INEXACT);
  if (__any_sync(0xffffffffu, ovf != 0u) && lane == 0) atomicOr(flags, FLAG_COUNT_WRAP);
  // (the gate's count: 0 after an overflow, whose redo must see the old visited rows)
  if (vn.count) {
    const uint32_t c = *((volatile const uint32_t*)vn.count);
    visit_rows(vn.list, (int64_t)c < vn.cap ? c : (uint32_t)vn.cap, vn.W, vn.colmask, vn.Fn, vn.V, vn.full);
  }
  if (COUNT) {
    for (int o = 16; o; o >>= 1) {
      nvals += __shfl_xor_sync(0xffffffffu, nvals, o);
      nw += __shfl_xor_sync(0xffffffffu, nw, o);
    }
    for (int o = 16; o; o >>= 1) nrec += __shfl_xor_sync(0xffffffffu, nrec, o);
    if (lane == 0) {
      atomicAdd(bytes, 8ull * (nvals + nw) + nrec);
      atomicAdd(&stat[2], nvals);
    }
  }
}

// Per-warp staging of one segment's frontier columns in the MFBr gather.
struct FinishSmem {
  float s[128], c[128];                      // compensated zeta sum of the column
  uint8_t col[128];                          // column within the quad
};

// Finalisation of a segment whose quad holds columns of several requests
// (packed batches): lambda terms are summed per request (runs of words) by a
// segmented warp reduction over the compacted columns.  Kept out of line so
// that the common single-request path keeps its registers.  Returns the
// number of lambda updates made (on lane 0's count).
__device__ __noinline__ int finish_mixed(const FinishSmem& fm, int total, uint64_t* row, double* lambda, int32_t n,
                                         int32_t v, const int32_t* __restrict__ quad_words_req) {
  const unsigned lane = lane_id();
  int adds = 0;
  for (int i0 = 0; i0 < total; i0 += 32) {
    const int i = i0 + (int)lane;
    float ls = 0.f, lc = 0.f;
    int key = NO_REQ;
    if (i < total) {
      const int c = fm.col[i];
      uint64_t* slot = row + c;
      *slot = finish_col(acc_value(fm.s[i], fm.c[i]), *slot, ls, lc);
      key = __ldg(&quad_words_req[c >> 5]);
    }
    const bool last = warp_acc_seg_sum(ls, lc, key) && key != NO_REQ && ls != 0.f;
    if (last) atomicAdd(&lambda[(size_t)key * n + v], (double)ls + (double)lc);
    adds += __popc(__ballot_sync(0xffffffffu, last));
  }
  return adds;
}

// MFBr gather of level l: zeta(s,v) = sum over the segment's pairs of the
// successors' values (double-float, compensated).  Single-item rows are
// finalised here: lambda(v) += zeta * sigma_bar and the slot of (s,v) takes
// the value zeta + 1/sigma_bar; multi-item rows add their partial zeta into
// the row's FP64 accumulator.  Only the columns of v's level-l frontier are
// finalised (about one in six of the quad on R-MAT inputs), so they are
// first compacted through shared memory and then finalised one per lane.
template <bool COUNT, bool G32>
__global__ void __launch_bounds__(256, MFBC_BWD_GATHER_MIN_BLOCKS) k_lvl_bwd_gather(
    const uint4* __restrict__ segs, const uint32_t* nseg_p, const uint32_t* __restrict__ prow,
    const uint4* __restrict__ pmask, int nb, int W, const uint32_t* __restrict__ Fl,
    const int32_t* __restrict__ hub_of, double* svd, double* zacc, double* lambda, int32_t n, int uniform_req,
    const int32_t* __restrict__ quad_req, const int32_t* __restrict__ word_req, uint32_t* next_group,
    unsigned long long* bytes, unsigned long long* stat, int seg_group) {
  __shared__ GatherSmem gsm[8];
  __shared__ FinishSmem fsm[8];
  GatherSmem& gs = gsm[threadIdx.x >> 5];
  FinishSmem& fm = fsm[threadIdx.x >> 5];
  uint64_t* sv = reinterpret_cast<uint64_t*>(svd);
  const unsigned lane = lane_id();
  const uint32_t lt = (1u << lane) - 1u;
  const uint32_t nseg = *nseg_p;
  if (!G32) seg_group = seg_group_of(nseg, seg_group);
  const int shift = 4 * (int)(lane & 7u);
  unsigned long long nvals = 0, nw = 0, nrec = 0;
  uint32_t ovf = 0;
  FOR_SEGMENT_GROUPS(nseg, next_group, G32 ? 32 : seg_group)
    auto finish = [&](int k, uint64_t, uint64_t, uint64_t, uint64_t, float s0, float s1, float s2, float s3, float c0,
                      float c1, float c2, float c3, uint32_t) {
      const int32_t v = (int32_t)__shfl_sync(0xffffffffu, myseg.x, k);
      const uint32_t z = __shfl_sync(0xffffffffu, myseg.z, k);
      const int d = (int)((z >> 8) & 0xffu);
      // this lane's four columns of v's level-l frontier
      const uint32_t fs = (__ldg(&Fl[(size_t)v * W + 4 * d + (lane >> 3)]) >> shift) & 0xfu;
      const uint32_t b0 = __ballot_sync(0xffffffffu, fs & 1u), b1 = __ballot_sync(0xffffffffu, fs & 2u);
      const uint32_t b2 = __ballot_sync(0xffffffffu, fs & 4u), b3 = __ballot_sync(0xffffffffu, fs & 8u);
      const int total = __popc(b0) + __popc(b1) + __popc(b2) + __popc(b3);
      if (total == 0) return;
      int at = __popc(b0 & lt) + __popc(b1 & lt) + __popc(b2 & lt) + __popc(b3 & lt);
      __syncwarp();                                   // the previous segment's entries are consumed
      if (fs & 1u) { fm.s[at] = s0; fm.c[at] = c0; fm.col[at] = (uint8_t)(4 * lane + 0); at++; }
      if (fs & 2u) { fm.s[at] = s1; fm.c[at] = c1; fm.col[at] = (uint8_t)(4 * lane + 1); at++; }
      if (fs & 4u) { fm.s[at] = s2; fm.c[at] = c2; fm.col[at] = (uint8_t)(4 * lane + 2); at++; }
      if (fs & 8u) { fm.s[at] = s3; fm.c[at] = c3; fm.col[at] = (uint8_t)(4 * lane + 3); }
      __syncwarp();
      if ((z >> 16) & 1u) {
        double* za = zacc + (size_t)hub_of[v] * nb + 128 * d;
        for (int i = (int)lane; i < total; i += 32) atomicAdd(za + fm.col[i], (double)fm.s[i] + (double)fm.c[i]);
        if (COUNT && lane == 0) nw += (unsigned long long)total;
      } else {
        // this segment is the only writer of these slots in this launch
        uint64_t* row = sv + (size_t)v * nb + 128 * d;
        const int rq = uniform_req >= 0 ? uniform_req : __ldg(&quad_req[d]);
        if (COUNT && lane == 0) nw += 2ull * (unsigned long long)total;
        if (rq >= 0) {                                // one request: one lambda(v) sum
          float ls = 0.f, lc = 0.f;                   // lambda(v) terms of this lane's columns
          for (int i = (int)lane; i < total; i += 32) {
            uint64_t* slot = row + fm.col[i];
            *slot = finish_col(acc_value(fm.s[i], fm.c[i]), *slot, ls, lc);
          }
          if (__any_sync(0xffffffffu, ls != 0.f)) {
            const double lam = warp_acc_sum(ls, lc);
            if (lane == 0) atomicAdd(&lambda[(size_t)rq * n + v], lam);
            if (COUNT && lane == 0) nrec += 8ull;
          }
        } else {                                      // requests meet in this quad: sum per request
          const int adds = finish_mixed(fm, total, row, lambda, n, v, word_req + 4 * d);
          if (COUNT) nrec += 8ull * adds;
        }
      }
    };
    gather_group<COUNT, false>(myseg, nin, prow, pmask, gs, sv, nvals, nrec, ovf, finish);
    // segments without successor pairs: zeta = 0
    uint32_t empty = __ballot_sync(0xffffffffu, (int)lane < nin && (myseg.z & 0xffu) == 0u && myseg.x != SEG_DUMMY);
    while (empty) {
      const int k = __ffs(empty) - 1;
      empty &= empty - 1;
      finish(k, 0, 0, 0, 0, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0u);
    }
  }
  if (COUNT) {
    for (int o = 16; o; o >>= 1) {
      nvals += __shfl_xor_sync(0xffffffffu, nvals, o);
      nw += __shfl_xor_sync(0xffffffffu, nw, o);
    }
    for (int o = 16; o; o >>= 1) nrec += __shfl_xor_sync(0xffffffffu, nrec, o);
    if (lane == 0) {
      atomicAdd(bytes, 8ull * (nvals + nw) + nrec);
      atomicAdd(&stat[3], nvals);
    }
  }
}

// Finalise the multi-item vertices of level l: zeta from the row's FP64
// accumulator, lambda(v) += zeta * sigma_bar, slot value zeta + 1/sigma_bar
// (double-float), accumulator reset.  32 hubs are tested per warp at once;
// the level-l columns of a hub (lane j holds frontier word j) are compacted
// into shared memory and finalised one per lane.
__global__ void __launch_bounds__(LVL_WARPS * 32) k_lvl_hub_final(
    const int32_t* __restrict__ hubs, int32_t nhub, int W, int nb, const uint32_t* __restrict__ Fl,
    const uint32_t* __restrict__ mem_l, double* svd, double* zacc, double* lambda, int32_t n, int uniform_req,
    const int32_t* __restrict__ word_req, unsigned long long* bytes, int hc, const uint32_t* flags) {
  __shared__ uint16_t cols_all[LVL_WARPS][LEVEL_MAX_NB];
  uint16_t* cols = cols_all[threadIdx.x >> 5];
  const unsigned lane = lane_id();
  if (*((volatile const uint32_t*)flags) & FLAG_ROUND_ABORT) return;   // the level's gather did not run
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  uint64_t* sv = reinterpret_cast<uint64_t*>(svd);
  unsigned long long nbytes = 0;
  // hc <= 32 hubs per warp and round (fewer when there are few hubs)
  for (uint64_t base = (((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * hc; base < (uint64_t)nhub;
       base += nw * hc) {
    const uint64_t myh = base + lane;
    const int32_t myv = (int)lane < hc && myh < (uint64_t)nhub ? hubs[myh] : 0;
    uint32_t am = __ballot_sync(0xffffffffu, (int)lane < hc && myh < (uint64_t)nhub && test_bit(mem_l, myv));
    while (am) {
      const int t = __ffs(am) - 1;
      am &= am - 1;
      const uint64_t h = base + t;
      const int32_t v = __shfl_sync(0xffffffffu, myv, t);
      uint32_t x = (int)lane < W ? Fl[(size_t)v * W + lane] : 0u;
      const int cnt = __popc(x);
      int incl = cnt;
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, incl, o);
        if ((int)lane >= o) incl += y;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      int at = incl - cnt;
      __syncwarp();                                   // the previous hub's columns are consumed
      while (x) {
        cols[at++] = (uint16_t)(32 * lane + (__ffs(x) - 1));
        x &= x - 1;
      }
      __syncwarp();
      double* za = zacc + (size_t)h * nb;
      uint64_t* row = sv + (size_t)v * nb;
      if (uniform_req >= 0) {
        float ls = 0.f, lc = 0.f;
        for (int i = (int)lane; i < total; i += 32) {
          const int c = cols[i];
          row[c] = finish_col(df_of_double(za[c]), row[c], ls, lc);
          za[c] = 0.0;
        }
        const double lam = warp_acc_sum(ls, lc);
        if (lane == 0) lambda[(size_t)uniform_req * n + v] += lam;
      } else {
        // several requests in the batch: sum per request (runs of words)
        for (int i0 = 0; i0 < total; i0 += 32) {
          const int i = i0 + (int)lane;
          float ls = 0.f, lc = 0.f;
          int key = NO_REQ;
          if (i < total) {
            const int c = cols[i];
            row[c] = finish_col(df_of_double(za[c]), row[c], ls, lc);
            za[c] = 0.0;
            key = __ldg(&word_req[c >> 5]);
          }
          if (warp_acc_seg_sum(ls, lc, key) && key != NO_REQ && ls != 0.f)
            atomicAdd(&lambda[(size_t)key * n + v], (double)ls + (double)lc);
        }
      }
      if (bytes && lane == 0) nbytes += 32ull * total + 4ull * W + 16ull;
    }
  }
  if (bytes) {
    for (int o = 16; o; o >>= 1) nbytes += __shfl_xor_sync(0xffffffffu, nbytes, o);
    if (lane == 0) atomicAdd(bytes, nbytes);
  }
}

// Return the bit masks touched by a batch to zero (F rows, visited rows).
__global__ void k_lvl_clear_rows(const int32_t* __restrict__ list, uint32_t count, int W, uint32_t* Fl,
                                 uint32_t* V) {
  const uint64_t total = (uint64_t)count * W;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const size_t r = (size_t)list[i / W] * W + (i % W);
    Fl[r] = 0u;
    V[r] = 0u;
  }
}

// Per-source rows of tau and sigma_bar from the level masks (sssp output).
__global__ void k_lvl_output(const int32_t* __restrict__ list, uint32_t count, int level, int W, int nb,
                             int nactive, int32_t n, const uint32_t* __restrict__ Fl,
                             const double* __restrict__ sv, int32_t* dist_out, double* sigma_out) {
  const unsigned lane = lane_id();
  const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
  for (uint64_t i = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += nw) {
    const int32_t v = list[i];
    for (int j = 0; j < W; j++) {
      const uint32_t fj = Fl[(size_t)v * W + j];
      const int c = j * 32 + lane;
      if (((fj >> lane) & 1u) && c < nactive) {
        dist_out[(size_t)c * n + v] = level;
        if (sigma_out) sigma_out[(size_t)c * n + v] = (double)reinterpret_cast<const uint64_t*>(sv)[(size_t)v * nb + c];
      }
    }
  }
}

// ------------------------------------------------------------------ driver
#define PROF(id, ...)             \
  do {                            \
    rc.prof->begin(id);           \
    __VA_ARGS__;                  \
    rc.prof->end(id);             \
  } while (0)

// one warp per 32 items (the precheck group)
static inline unsigned grid_for_items(int64_t items, unsigned cap) {
  uint64_t warps = ((uint64_t)items + 31) / 32;
  uint64_t b = (warps + LVL_WARPS - 1) / LVL_WARPS;
  if (b < 1) b = 1;
  return (unsigned)(b > cap ? cap : b);
}

static void set_smem_attrs() {
  static bool done = false;
  if (done) return;
  cudaFuncSetAttribute(k_lvl_fwd_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LVL_SMEM);
  cudaFuncSetAttribute(k_lvl_bwd_pairs, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LVL_SMEM);
  done = true;
}

// Units per group (<= 32, a power of two) so that a launch of `warps`
// resident warps gets at least four groups per warp where the work allows,
// and the blocks that launch with such groups (at most cap).
static inline int group_size(uint64_t units, uint64_t warps) {
  int g = 32;
  while (g > 1 && units < (uint64_t)g * warps * 4) g >>= 1;
  return g;
}
static inline unsigned grid_for_groups(uint64_t units, int g, unsigned cap) {
  const uint64_t warps = (units + (uint64_t)g - 1) / (uint64_t)g;
  uint64_t b = (warps + LVL_WARPS - 1) / LVL_WARPS;
  if (b < 1) b = 1;
  return (unsigned)(b > cap ? cap : b);
}

static inline unsigned grid_for_warps(uint64_t warps, unsigned cap) {
  uint64_t b = (warps + LVL_WARPS - 1) / LVL_WARPS;
  if (b < 1) b = 1;
  return (unsigned)(b > cap ? cap : b);
}

struct LevelPlan {                 // host-side level bookkeeping of one batch
  std::vector<int64_t> off;        // list offset of each level
  std::vector<uint32_t> cnt;       // list length of each level
};
static thread_local LevelPlan tl_plan;

static const unsigned kGatherGrid = 152u * MFBC_GATHER_MIN_BLOCKS;   // resident blocks of the gather kernels
static const unsigned kBwdGatherGrid = 152u * MFBC_BWD_GATHER_MIN_BLOCKS;

static mfbc_status level_round_halves(RunCtx& rc, LevelState& s, bool fwd, int l, int64_t ib, int64_t ie,
                                      int uniform_req, int64_t off_n, double* lambda);

// One MFBF (fwd) or MFBr product of level l over the items [ib, ie): the pair
// kernel, then the gather kernel.
//
// checked = false: both are queued without waiting, with a one-thread gate
// between them.  The gather reads the segment count the pair kernel left on
// the device, which the gate sets to 0 when the pair buffers overflowed (an
// MFBr overflow also sets FLAG_ROUND_ABORT, so the launches queued after it
// in the sweep do nothing); the host finds out at its next read of the
// counters and redoes the round over halves.
// checked = true: the host reads the pair kernel's counters first; when the
// buffers overflowed the range is split in halves.  The pair kernels' side
// effects (frontier bits, membership, list appends) are idempotent, so a
// re-run of a range is harmless.
// visited_next (MFBF): the gather also runs the next level's visit.
static mfbc_status level_round(RunCtx& rc, LevelState& s, bool fwd, int l, int64_t ib, int64_t ie,
                               int uniform_req, int64_t off_n, double* lambda, bool checked,
                               bool* visited_next = nullptr) {
  if (visited_next) *visited_next = false;
  const DevGraph& g = *rc.g;
  const int32_t n = g.n;
  const int nb = s.nb, W = s.W;
  cudaStream_t st = rc.stream;
  unsigned long long* B = rc.prof->count_bytes ? s.ctr->bytes : nullptr;
  const uint32_t* Fl = s.F + (size_t)l * n * W;
  const uint32_t* Ml = s.member + (size_t)l * s.mw;
  uint32_t* Fn = s.F + (size_t)(l + 1) * n * W;
  uint32_t* Mn = s.member + (size_t)(l + 1) * s.mw;
  // test hook: buffers of 2^16 slots make rounds overflow and split
  const uint32_t pair_cap = rc.small_rounds ? std::min<uint32_t>(s.pair_cap, 1u << 16) : s.pair_cap;
  const uint32_t seg_cap = rc.small_rounds ? std::min<uint32_t>(s.seg_cap, 1u << 16) : s.seg_cap;
  MFBC_CUDA_TRY(cudaMemsetAsync(s.ctr->work, 0, sizeof(uint32_t) * 4, st), rc.err);
  MFBC_CUDA_TRY(cudaMemsetAsync(&s.ctr->list_count[2], 0, sizeof(uint32_t), st), rc.err);
  const int ig = group_size((uint64_t)(ie - ib), (uint64_t)PAIR_GRID * LVL_WARPS);
  const unsigned pgrid = grid_for_groups((uint64_t)(ie - ib), ig, PAIR_GRID);
  // row indices u * Q + quad need bit 31 free for the hot-row flag
  const int Qn = std::max(1, W / 4);
  // segment slots per reservation: with small item groups a warp emits few
  // segments, and the unused rest of its chunk only adds filler segments that
  // the gather walks past
  const uint32_t seg_chunk =
      ig == 32 ? SEG_CHUNK : std::max<uint32_t>(2u * Qn, std::min<uint32_t>(SEG_CHUNK, 2u * ig * Qn));
  const uint32_t* hot = MFBC_HOT_HINT && (uint64_t)n * (uint64_t)Qn < (1ull << 31) ? g.hot : nullptr;
  if (fwd)
    PROF(K_LVL_FWD, (k_lvl_fwd_pairs<<<pgrid, LVL_WARPS * 32, LVL_SMEM, st>>>(
                        ib, ie, g.items_in.v, g.items_in.beg, g.col_t, W, s.full, s.V, Fl, Ml, Fn, Mn,
                        s.lists + off_n, &s.ctr->list_count[0], s.list_cap - off_n, &s.ctr->flags,
                        &s.ctr->list_count[2], s.prow, s.pmask, s.segs, s.ctr->work, pair_cap, seg_cap, hot,
                        B ? B + K_LVL_FWD : nullptr, s.ctr->stat, ig, seg_chunk)));
  else
    PROF(K_LVL_BWD, (k_lvl_bwd_pairs<<<pgrid, LVL_WARPS * 32, LVL_SMEM, st>>>(
                        ib, ie, g.items_out.v, g.items_out.beg, g.col, W, Fl, Ml, Fn, Mn,
                        &s.ctr->list_count[2], s.prow, s.pmask, s.segs, s.ctr->work, pair_cap, seg_cap, hot,
                        B ? B + K_LVL_BWD : nullptr, s.ctr->stat, ig, &s.ctr->flags, seg_chunk)));
  // segments per gather group: from the count, which unchecked rounds leave
  // to the gather (0), checked ones read first
  const unsigned gcap = fwd ? kGatherGrid : kBwdGatherGrid;
  int gs = 0;
  unsigned ggrid = gcap;
  if (checked) {
    MFBC_CUDA_TRY(cudaMemcpyAsync(rc.h_ctr, s.ctr->list_count, sizeof(uint32_t) * 9, cudaMemcpyDeviceToHost, st),
                  rc.err);
    MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
    rc.prof->drain();
    if (rc.h_ctr[8]) return level_round_halves(rc, s, fwd, l, ib, ie, uniform_req, off_n, lambda);
    const uint32_t nseg = rc.h_ctr[6];
    if (!nseg) return MFBC_OK;
    gs = group_size(nseg, (uint64_t)gcap * 8);
    ggrid = grid_for_groups(nseg, gs, gcap);
  }
  if (!checked)
    k_lvl_round_gate<<<1, 1, 0, st>>>(s.ctr->work, &s.ctr->list_count[0], &s.ctr->flags, &s.ctr->abort_level,
                                      &s.ctr->visit_count, l, fwd ? 0 : 1);
  // the next level's visit rides on this gather (the count is the gate's,
  // clamped to the list's room)
  VisitNext vn{s.lists + off_n, nullptr, s.list_cap - off_n, W, s.colmask, Fn, s.V, s.full};
  if (fwd && visited_next && !checked) {
    vn.count = &s.ctr->visit_count;
    *visited_next = true;
  }
  // groups of 32 segments compile to constants (G32): taken when the round
  // has that many segments (checked) or the graph is large enough that its
  // wide levels do (unchecked: a quad per item and quad is at least 8x the
  // segments that 32 per group need)
  const int64_t items = fwd ? g.items_in.count : g.items_out.count;
  const bool g32 = checked ? gs == 32 : (uint64_t)items * (uint64_t)Qn >= 8ull * 32 * 4 * gcap * 8;
#define GATHER_LAUNCH(kern, C, ...)                                                   \
  do {                                                                                \
    if (g32) kern<C, true><<<ggrid, 256, 0, st>>>(__VA_ARGS__);                       \
    else kern<C, false><<<ggrid, 256, 0, st>>>(__VA_ARGS__);                          \
  } while (0)
  if (fwd) {
    if (B)
      PROF(K_LVL_FWD_G, GATHER_LAUNCH(k_lvl_fwd_gather, true, s.segs, &s.ctr->work[1], s.prow, s.pmask, nb, s.sv,
                                      &s.ctr->flags, &s.ctr->work[2], B + K_LVL_FWD_G, s.ctr->stat, vn, gs));
    else
      PROF(K_LVL_FWD_G, GATHER_LAUNCH(k_lvl_fwd_gather, false, s.segs, &s.ctr->work[1], s.prow, s.pmask, nb, s.sv,
                                      &s.ctr->flags, &s.ctr->work[2], nullptr, s.ctr->stat, vn, gs));
  } else {
    if (B)
      PROF(K_LVL_BWD_G, GATHER_LAUNCH(k_lvl_bwd_gather, true, s.segs, &s.ctr->work[1], s.prow, s.pmask, nb, W, Fl,
                                      g.items_out.hub_of, s.sv, s.zacc, lambda, n, uniform_req, s.quad_req,
                                      s.word_req, &s.ctr->work[2], B + K_LVL_BWD_G, s.ctr->stat, gs));
    else
      PROF(K_LVL_BWD_G, GATHER_LAUNCH(k_lvl_bwd_gather, false, s.segs, &s.ctr->work[1], s.prow, s.pmask, nb, W, Fl,
                                      g.items_out.hub_of, s.sv, s.zacc, lambda, n, uniform_req, s.quad_req,
                                      s.word_req, &s.ctr->work[2], nullptr, s.ctr->stat, gs));
  }
#undef GATHER_LAUNCH
  return MFBC_OK;
}

// A round known to overflow its buffers over [ib, ie), redone as checked
// rounds over the two halves.
static mfbc_status level_round_halves(RunCtx& rc, LevelState& s, bool fwd, int l, int64_t ib, int64_t ie,
                                      int uniform_req, int64_t off_n, double* lambda) {
  rc.prof->k[K_LVL_SPLIT].launches++;          // reported as "level_round_split"
  if (ie - ib <= 32) {
    if (rc.err) *rc.err = "level pair buffers cannot hold one group of 32 work items";
    return MFBC_ERR_OOM;
  }
  const int64_t mid = ib + ((ie - ib) / 2 + 31) / 32 * 32;
  mfbc_status e = level_round(rc, s, fwd, l, ib, mid, uniform_req, off_n, lambda, true);
  if (e) return e;
  return level_round(rc, s, fwd, l, mid, ie, uniform_req, off_n, lambda, true);
}

// Clear every level mask of the state (after a batch stopped at a list that
// overflowed: rows of vertices missing from the list may hold bits).
static mfbc_status level_clear_all(RunCtx& rc, LevelState& s) {
  const size_t n = (size_t)rc.g->n;
  cudaStream_t st = rc.stream;
  MFBC_CUDA_TRY(cudaMemsetAsync(s.V, 0, sizeof(uint32_t) * n * s.W, st), rc.err);
  MFBC_CUDA_TRY(cudaMemsetAsync(s.F, 0, sizeof(uint32_t) * (size_t)s.Lcap * n * s.W, st), rc.err);
  MFBC_CUDA_TRY(cudaMemsetAsync(s.member, 0, sizeof(uint32_t) * (size_t)s.Lcap * s.mw, st), rc.err);
  return MFBC_OK;
}

// One MFBr level: its round (halves: one known to overflow, redone over
// halves), then the finalisation of its multi-item rows.
static mfbc_status level_bwd(RunCtx& rc, LevelState& s, int l, int uniform_req, double* lambda, bool checked,
                             bool halves = false) {
  const DevGraph& g = *rc.g;
  unsigned long long* B = rc.prof->count_bytes ? s.ctr->bytes : nullptr;
  mfbc_status e = halves ? level_round_halves(rc, s, false, l, 0, g.items_out.count, uniform_req, 0, lambda)
                         : level_round(rc, s, false, l, 0, g.items_out.count, uniform_req, 0, lambda, checked);
  if (e) return e;
  if (g.items_out.nhub) {
    const int hc = group_size((uint64_t)g.items_out.nhub, 152ull * 8 * LVL_WARPS);
    PROF(K_LVL_HUB, (k_lvl_hub_final<<<grid_for_groups(g.items_out.nhub, hc, 152 * 8), LVL_WARPS * 32, 0,
                                       rc.stream>>>(
                        g.items_out.hubs, g.items_out.nhub, s.W, s.nb, s.F + (size_t)l * g.n * s.W,
                        s.member + (size_t)l * s.mw, s.sv, s.zacc, lambda, g.n, uniform_req, s.word_req,
                        B ? B + K_LVL_HUB : nullptr, hc, &s.ctr->flags)));
  }
  return MFBC_OK;
}

mfbc_status level_batch(RunCtx& rc, LevelState& s, const int32_t* d_src_batch, int nactive,
                        double* lambda, bool backward, int* levels_out, bool* levels_exceeded,
                        int64_t* fwd_iters, int64_t* bwd_iters) {
  const DevGraph& g = *rc.g;
  const int32_t n = g.n;
  const int nb = s.nb, W = s.W;
  cudaStream_t st = rc.stream;
  *levels_exceeded = false;
  *levels_out = -1;
  if (n == 0) return MFBC_OK;
  set_smem_attrs();

  fill_i32(s.src, -1, (size_t)nb, st);
  if (nactive)
    MFBC_CUDA_TRY(cudaMemcpyAsync(s.src, d_src_batch, sizeof(int32_t) * nactive, cudaMemcpyDeviceToDevice, st), rc.err);
  k_lvl_colmask<<<(unsigned)((W * 32 + 255) / 256), 256, 0, st>>>(s.src, W, s.colmask);
  // requests packed into this batch: per-word and per-quad lambda rows
  int uniform_req = 0;
  if (rc.word_req && lambda) {
    uniform_req = batch_uniform_request(rc.word_req, W);
    if (uniform_req < 0) {
      std::vector<int32_t> q((size_t)(W / 4));
      for (int d = 0; d < W / 4; d++) {
        int r = -1;
        for (int w = 4 * d; w < 4 * d + 4; w++) {
          const int x = rc.word_req[w];
          if (x >= 0) r = (r == -1 || r == x) ? x : -2;
        }
        q[(size_t)d] = r;
      }
      MFBC_CUDA_TRY(cudaMemcpyAsync(s.word_req, rc.word_req, sizeof(int32_t) * W, cudaMemcpyHostToDevice, st), rc.err);
      MFBC_CUDA_TRY(cudaMemcpyAsync(s.quad_req, q.data(), sizeof(int32_t) * q.size(), cudaMemcpyHostToDevice, st),
                    rc.err);
    }
  }
  MFBC_CUDA_TRY(cudaMemsetAsync(s.ctr->list_count, 0, sizeof(uint32_t) * 4, st), rc.err);
  MFBC_CUDA_TRY(cudaMemsetAsync(&s.ctr->abort_level, 0, sizeof(uint32_t), st), rc.err);
  MFBC_CUDA_TRY(cudaMemsetAsync(s.full, 0, sizeof(uint32_t) * s.mw, st), rc.err);
  if (g.items_in.nhub)
    PROF(K_FILL, (k_lvl_zero_hubs<<<152 * 4, 256, 0, st>>>(g.items_in.hubs, g.items_in.nhub, nb, s.sv)));
  rc.prof->k[K_FILL].bytes += 8.0 * g.items_in.nhub * nb;
  PROF(K_SEED, (k_lvl_seed<<<(nb + 127) / 128, 128, 0, st>>>(s.src, nb, W, s.sv, s.F, s.member, s.lists,
                                                           &s.ctr->list_count[0])));
  MFBC_CUDA_TRY(cudaMemcpyAsync(rc.h_ctr, s.ctr->list_count, sizeof(uint32_t) * 5, cudaMemcpyDeviceToHost, st), rc.err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
  LevelPlan& P = tl_plan;
  P.off.assign(1, 0);
  P.cnt.assign(1, rc.h_ctr[0]);
  auto Fl = [&](int l) { return s.F + (size_t)l * n * W; };

  // MFBF: one host read of the counters per level (the next level's size,
  // which ends the loop when it is 0, and the flags)
  int L = 0;
  bool visited = false;                  // level l's visit ran inside the previous gather
  for (int l = 0;; l++) {
    const uint32_t cl = P.cnt[l];
    if (!visited) {
      PROF(K_LVL_VISIT, (k_lvl_visit<<<grid_for_warps(cl, 152 * 16), LVL_WARPS * 32, 0, st>>>(
                            s.lists + P.off[l], cl, W, s.colmask, Fl(l), s.V, s.full)));
      rc.prof->k[K_LVL_VISIT].bytes += 12.0 * W * cl;
    }
    if (l + 1 >= s.Lcap) { *levels_exceeded = true; level_reset(rc, s, l); return MFBC_ERR_NO_CONVERGENCE; }
    const int64_t off_n = P.off[l] + cl;
    MFBC_CUDA_TRY(cudaMemsetAsync(&s.ctr->list_count[0], 0, sizeof(uint32_t), st), rc.err);
    mfbc_status e = level_round(rc, s, true, l, 0, g.items_in.count, uniform_req, off_n, nullptr, false, &visited);
    if (e) return e;
    MFBC_CUDA_TRY(cudaMemcpyAsync(rc.h_ctr, s.ctr->list_count, sizeof(uint32_t) * 9, cudaMemcpyDeviceToHost, st), rc.err);
    MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
    rc.prof->drain();
    if (rc.h_ctr[8]) {
      // the pair buffers overflowed: neither the gather nor the visit ran;
      // redo the round checked (split over halves of the items)
      k_clear_flag_bits<<<1, 1, 0, st>>>(&s.ctr->flags, FLAG_ROUND_ABORT);
      e = level_round_halves(rc, s, true, l, 0, g.items_in.count, uniform_req, off_n, nullptr);
      if (e) return e;
      visited = false;
      MFBC_CUDA_TRY(cudaMemcpyAsync(rc.h_ctr, s.ctr->list_count, sizeof(uint32_t) * 5, cudaMemcpyDeviceToHost, st),
                    rc.err);
      MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
      rc.prof->drain();
    }
    if (rc.h_ctr[4] & (FLAG_LEVEL_LIST | FLAG_COUNT_WRAP)) {
      // list capacity exceeded (bit 0) or a path count passed 2^64 (bit 3):
      // the general kernels redo this batch; rows of vertices missing from
      // the overflowed list may hold bits, so every mask is cleared
      k_clear_flag_bits<<<1, 1, 0, st>>>(&s.ctr->flags, FLAG_LEVEL_LIST | FLAG_COUNT_WRAP);
      *levels_exceeded = true;
      e = level_clear_all(rc, s);
      if (e) return e;
      return MFBC_ERR_NO_CONVERGENCE;
    }
    const uint32_t cn = rc.h_ctr[0];
    if (visited) rc.prof->k[K_LVL_FWD_G].bytes += 12.0 * W * cn;
    P.off.push_back(off_n);
    P.cnt.push_back(cn);
    if (fwd_iters) (*fwd_iters)++;
    if (cn == 0) { L = l; break; }
  }
  *levels_out = L;
  if (!backward) return MFBC_OK;

  // MFBr over levels L .. 1 (level L+1 is empty and all-zero), queued
  // without waiting; one read of the flags at the end.  If a round's pair
  // buffers overflowed, the sweep stopped there (every later launch returned
  // at once) and resumes from that level with checked rounds.
  for (int l = L; l >= 1; l--) {
    mfbc_status e = level_bwd(rc, s, l, uniform_req, lambda, false);
    if (e) return e;
    if (bwd_iters) (*bwd_iters)++;
  }
  MFBC_CUDA_TRY(cudaMemcpyAsync(rc.h_ctr, &s.ctr->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st), rc.err);
  MFBC_CUDA_TRY(cudaMemcpyAsync(rc.h_ctr + 1, &s.ctr->abort_level, sizeof(uint32_t), cudaMemcpyDeviceToHost, st),
                rc.err);
  MFBC_CUDA_TRY(cudaStreamSynchronize(st), rc.err);
  rc.prof->drain();
  if (rc.h_ctr[0] & FLAG_ROUND_ABORT) {
    const int l0 = (int)rc.h_ctr[1];
    k_clear_flag_bits<<<1, 1, 0, st>>>(&s.ctr->flags, FLAG_ROUND_ABORT);
    for (int l = l0; l >= 1; l--) {
      mfbc_status e = level_bwd(rc, s, l, uniform_req, lambda, true, l == l0);
      if (e) return e;
    }
  }
  return MFBC_OK;
}

void level_reset(RunCtx& rc, LevelState& s, int levels) {
  const LevelPlan& P = tl_plan;
  const int32_t n = rc.g->n;
  for (int l = 0; l <= levels && l < (int)P.cnt.size(); l++) {
    const uint32_t c = P.cnt[l];
    if (c)
      PROF(K_LVL_RESET, (k_lvl_clear_rows<<<grid_for_warps((uint64_t)c * s.W / 32 + 1, 152 * 8), 256, 0,
                                            rc.stream>>>(s.lists + P.off[l], c, s.W,
                                                         s.F + (size_t)l * n * s.W, s.V)));
    cudaMemsetAsync(s.member + (size_t)l * s.mw, 0, sizeof(uint32_t) * s.mw, rc.stream);
  }
  // the level after the last one may hold stray bits only if the list overflowed
  if (levels + 1 < s.Lcap)
    cudaMemsetAsync(s.member + (size_t)(levels + 1) * s.mw, 0, sizeof(uint32_t) * s.mw, rc.stream);
}

mfbc_status level_output(RunCtx& rc, LevelState& s, int levels, int nactive, int32_t* dist_out,
                         double* sigma_out) {
  const LevelPlan& P = tl_plan;
  const int32_t n = rc.g->n;
  PROF(K_OUTPUT, {
    fill_i32(dist_out, INF, (size_t)nactive * n, rc.stream);
    if (sigma_out) cudaMemsetAsync(sigma_out, 0, sizeof(double) * (size_t)nactive * n, rc.stream);
    for (int l = 0; l <= levels; l++) {
      const uint32_t c = P.cnt[l];
      if (!c) continue;
      k_lvl_output<<<grid_for_warps(c, 152 * 16), LVL_WARPS * 32, 0, rc.stream>>>(
          s.lists + P.off[l], c, l, s.W, s.nb, nactive, n, s.F + (size_t)l * n * s.W, s.sv, dist_out,
          sigma_out);
    }
  });
  return MFBC_OK;
}

}  // namespace mfbc
