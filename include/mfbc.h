/*
 * mfbc.h -- C ABI of the MFBC library (Maximal Frontier Betweenness
 * Centrality; Solomonik, Besta, Vella, Hoefler, SC17, arXiv:1609.07008).
 *
 * The library computes, on one GPU, the two sparse passes of the paper and
 * the centrality update that joins them:
 *   MFBF  (Sec. 4.1, Algorithm 1): distances tau(s,v) and shortest-path
 *         multiplicities sigma_bar(s,v) for a batch of n_b sources, as a
 *         repeated generalised product of a sparse n x n_b frontier with the
 *         adjacency matrix over the multpath monoid;
 *   MFBr  (Sec. 4.2, Algorithm 2): partial centrality factors
 *         zeta(s,v) = delta(s,v) / sigma_bar(s,v), propagated backwards from
 *         the leaves of the shortest-path DAG over the centpath monoid;
 *   MFBC  (Sec. 4.3, Algorithm 3): lambda(v) += sum_s zeta(s,v) sigma_bar(s,v)
 *         over batches of sources.
 *
 * Conventions shared by every call
 *  - Graphs are compressed rows of the adjacency matrix A of Sec. 2.1 (CSR:
 *    row v lists the arcs v -> col[k]) or of its transpose (CSC: row v lists
 *    the arcs col[k] -> v), with integer weights w[k] >= 1 (w == NULL: every
 *    arc weighs 1).  Vertex ids are 0..n-1.  Rows must be sorted by column
 *    with no duplicate arcs and no self-loops.
 *  - Distances are int32 with INT32_MAX meaning "unreachable" (the infinity
 *    of Sec. 2.1); path multiplicities and centralities are IEEE FP64.
 *    Multiplicities are exact integers while below 2^53.
 *  - Every call returns an mfbc_status; nothing aborts or throws.  On error
 *    the outputs are unspecified and mfbc_last_error() describes the cause.
 *  - "host" pointers are ordinary CPU memory (pinned memory makes copies
 *    faster); "device" pointers are CUDA global memory of the current device.
 *    The caller owns every buffer it passes; the library never keeps a
 *    pointer to caller memory after a call returns.
 *  - Calls on one graph handle must not overlap (the handle caches scratch
 *    memory); distinct handles are independent.
 *  - mfbc_bc[_device] and mfbc_sssp_batch[_device] set the current CUDA
 *    context's L2 fetch-granularity hint (cudaLimitMaxL2FetchGranularity) to
 *    32 bytes while they run and restore the previous value before returning;
 *    other work in the same context sees the hint meanwhile (performance
 *    only, never results).
 */
#ifndef MFBC_H
#define MFBC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  MFBC_OK = 0,
  MFBC_ERR_INVALID = 1,        /* bad argument or malformed graph */
  MFBC_ERR_OOM = 2,            /* device or host allocation failed */
  MFBC_ERR_CUDA = 3,           /* a CUDA runtime call failed */
  MFBC_ERR_OVERFLOW = 4,       /* (n-1) * max weight could overflow int32 distances */
  MFBC_ERR_NO_CONVERGENCE = 5, /* an MFBF/MFBr loop exceeded its iteration bound */
  MFBC_ERR_TIMEOUT = 6         /* a bounded device-side wait ran out of its budget (the
                                  persistent small-graph kernel's group barriers); the
                                  outputs are unspecified, the context stays usable */
} mfbc_status;

/* mfbc_graph_create flags: bit 0 = orientation of the arrays, bit 1 = symmetry */
#define MFBC_CSR        0u     /* row v of the arrays lists the out-arcs v -> col[k]: the adjacency
                                  matrix A itself, A(v, col[k]) = w[k] (Sec. 2.1) */
#define MFBC_CSC        1u     /* row v lists the in-arcs col[k] -> v: the arrays hold A^T, the
                                  operand of Algorithm 2's products (Sec. 4.2); A is built from it */
#define MFBC_DIRECTED   0u
#define MFBC_UNDIRECTED 2u     /* A is symmetric with symmetric weights (checked) */

/* bits written to *mfbc_options.warn_out */
#define MFBC_WARN_SIGMA_INEXACT 1u  /* some sigma_bar >= 2^53: FP64 counts may be rounded */

/* mfbc_options.path */
#define MFBC_PATH_AUTO    0    /* unit weights: the persistent small-graph kernel when n <= 2^13
                                  and nnz <= 2^18, else the level kernels; distance kernels for weights
                                  <= 128 when no in- or out-degree exceeds max(64, 4x the
                                  average degree); general kernels otherwise (or the family
                                  mfbc_autotune chose) */
#define MFBC_PATH_GENERAL 1    /* force the general (any integer weight) kernels */
#define MFBC_PATH_LEVEL   2    /* require the unit-weight level kernels (INVALID if weighted) */
#define MFBC_PATH_DIST    3    /* distance-ordered kernels for small integer weights
                                  (INVALID when the largest weight exceeds 4096); n_b is at
                                  most 4096 and n * n_b stays below 2^32 */
#define MFBC_PATH_SMALL   4    /* persistent kernel for small unit-weight graphs: every batch
                                  of the call in one launch (INVALID if weighted or when
                                  n * n_b * 9 bytes per group does not fit; see below) */

typedef struct mfbc_graph mfbc_graph;   /* opaque, device resident */

/* Per-kernel statistics, filled when mfbc_options.profile is non-NULL.
 * ms is the sum of CUDA-event durations of the kernel's launches; bytes is
 * the algorithmic (compulsory) DRAM traffic of those launches under the
 * model documented beside each kernel. */
#define MFBC_MAX_KSTATS 24
typedef struct {
  char name[40];
  uint64_t launches;
  double ms;
  double bytes;
} mfbc_kernel_stat;              /* launches counts kernels, also those run inside the
                                     CUDA graphs of the distance kernels' forward steps */

typedef struct {
  int32_t nkernels;
  mfbc_kernel_stat k[MFBC_MAX_KSTATS];
  uint64_t batches;
  uint64_t fwd_iters;          /* MFBF products over all batches (distance kernels: distance
                                  steps, including those that settle no pair) */
  uint64_t bwd_iters;          /* MFBr products over all batches (distance kernels: steps that
                                  settled pairs, distance 0 excepted) */
  int32_t n_b;                 /* batch width used */
  int32_t path;                /* MFBC_PATH_GENERAL, MFBC_PATH_LEVEL or MFBC_PATH_DIST */
  uint64_t stat[4];            /* with MFBC_OPT_COUNT_BYTES, level kernels: (neighbour, word)
                                  pairs gathered by MFBF / MFBr, values gathered by MFBF / MFBr */
} mfbc_profile;

typedef struct {
  int32_t n_b;                 /* sources per batch; 0 = largest that fits; rounded up to 32
                                  (general kernels) or 128 (level kernels) */
  int32_t path;                /* MFBC_PATH_* */
  void* stream;                /* cudaStream_t to run on; NULL = legacy default stream */
  void* workspace;             /* optional caller-owned device scratch, 256-byte aligned */
  uint64_t workspace_bytes;    /* its size; see mfbc_workspace_size */
  uint32_t* warn_out;          /* optional host pointer, receives MFBC_WARN_* bits */
  mfbc_profile* profile;       /* optional host pointer; enables per-kernel event timing */
  uint32_t flags;              /* MFBC_OPT_* bits */
  const int32_t* lambda_rows;  /* mfbc_bc_multi_device only, optional HOST int32[nreq]: the row of
                                  lambda_out that receives request r (NULL: row r); rows >= 0 */
  int32_t accumulator;         /* general kernels: MFBC_ACCUM_*, how a product reduces the
                                  candidates that meet at one (vertex, column) */
} mfbc_options;                /* zero-initialised = all defaults */

/* mfbc_options.accumulator (general kernels; the monoid reduction inside the
 * products of Algorithms 1 and 2, Sec. 3's generalised product) */
#define MFBC_ACCUM_AUTO      0   /* per product: segmented when the frontier holds at least
                                    1/64 of the vertices, else atomic (or what mfbc_autotune chose) */
#define MFBC_ACCUM_ATOMIC    1   /* push from the frontier: atomicMin on the distance, then an
                                    atomic add of the tied multiplicities (MFBr: atomic adds
                                    and counter decrements at the predecessors) */
#define MFBC_ACCUM_SEGMENTED 2   /* pull by target: the candidates of one (vertex, 32-column word)
                                    form one segment -- the vertex's arcs to the frontier -- and
                                    are reduced in registers by the warp that owns it (a block
                                    for rows of more than 256 arcs); no same-address atomics */
#define MFBC_ACCUM_HASH      3   /* push, reduced first in shared memory: a block's candidates for
                                    a high-degree target meet in one slot of the block's hash
                                    table (key = target vertex and word), and each slot column
                                    is merged into the batch state with one atomic per block */

/* mfbc_options.flags */
#define MFBC_OPT_COUNT_BYTES 1u  /* with profile: count algorithmic bytes on the device (slower) */
#define MFBC_OPT_KEEP_ORDER  2u  /* mfbc_bc*: batch the sources in the given order (see below) */
#define MFBC_OPT_ACCUMULATE  8u  /* mfbc_bc* and mfbc_bc_multi_device: add the result to the values
                                    already in lambda_out (its rows) instead of overwriting them;
                                    lambda is linear in the source list, so a request split over
                                    several calls accumulates to its whole answer */
#define MFBC_OPT_TEST_STALL  4u  /* test hook, MFBC_PATH_SMALL only: every group barrier waits
                                    for one arrival more than the group has, so each wait runs
                                    out of its (shortened, 20 ms) budget and the call returns
                                    MFBC_ERR_TIMEOUT; nothing faults and the context stays usable */
#define MFBC_OPT_TEST_SMALL_ROUNDS 16u  /* test hook, level kernels: product rounds get pair and
                                    segment buffers of 2^16 slots, so their rounds overflow and
                                    are redone over halves of the work items (the path a graph
                                    beyond 2^31 pairs per round takes); results are unchanged */

/* Build a device-resident graph from HOST compressed-row arrays (Sec. 2.1:
 * A(i,j) = w(i,j) for (i,j) in E; the paper's Tensor::write of the input,
 * Sec. 6.1).
 *   n       vertices (0 <= n < 2^31);  nnz = rowptr[n] arcs
 *   rowptr  int64[n+1], col int32[nnz], w int32[nnz] or NULL (unweighted)
 *   flags   (MFBC_CSR or MFBC_CSC) | (MFBC_DIRECTED or MFBC_UNDIRECTED).
 *           MFBC_CSR: the arrays are the rows of A (out-arcs); MFBC_CSC: they
 *           are the rows of A^T (row v lists the tails u of the arcs u -> v,
 *           with their weights).  Both describe the same graph; for an
 *           UNDIRECTED graph A = A^T and the two are the same arrays.
 *   stream  cudaStream_t or NULL; the construction (copies, validation
 *           kernels) is queued on it, and the call is complete on return.
 *           The paper's interface has no stream; it lets a caller keep the
 *           upload off the legacy default stream.
 * The arrays are copied; the library keeps both A and A^T (Algorithm 1's
 * products read in-arcs, Algorithm 2's out-arcs), building the one not given
 * (for directed graphs) by a stable counting sort, so rows stay sorted and the
 * result does not depend on the orientation passed.  Returns INVALID for
 * unsorted or out-of-range columns, duplicates, self-loops, weights < 1, an
 * asymmetric UNDIRECTED graph or unknown flag bits; OVERFLOW if
 * (n-1)*max_w + max_w >= 2^31-1. */
mfbc_status mfbc_graph_create(int32_t n, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                              const int32_t* w, uint32_t flags, void* stream, mfbc_graph** out);

/* Same as mfbc_graph_create (either orientation), from DEVICE arrays (copied;
 * caller keeps ownership). */
mfbc_status mfbc_graph_create_device(int32_t n, int64_t nnz, const int64_t* rowptr,
                                     const int32_t* col, const int32_t* w, uint32_t flags,
                                     void* stream, mfbc_graph** out);

/* Release the graph and any scratch cached on it.  NULL is ignored. */
void mfbc_graph_destroy(mfbc_graph* g);

/* Free the device scratch the handle cached for earlier calls (it grows to
 * the largest call made without opt->workspace); the next such call
 * allocates again.  The graph stays resident.  Every call has finished its
 * work when it returns; this one still synchronises the device before it
 * frees the memory. */
mfbc_status mfbc_graph_release_scratch(mfbc_graph* g);

/* n, nnz, flags and whether the graph has unit weights (out pointers may be NULL). */
mfbc_status mfbc_graph_info(const mfbc_graph* g, int32_t* n, int64_t* nnz, uint32_t* flags,
                            int32_t* unit_weights);

/* Betweenness centrality over a source list (Algorithm 3, Theorem 1):
 *   lambda_out[v] = sum over i < nsrc, v != sources[i], of
 *                   sum_t sigma(sources[i],t,v) / sigma_bar(sources[i],t)
 * (ordered pairs, Sec. 2.4; unreachable t contribute 0).  Sources may repeat
 * and are counted once per occurrence (lambda is linear in the list); with
 * every vertex listed once this is exact BC, otherwise the unscaled sum over
 * the sample.  HOST pointers: sources int32[nsrc], lambda_out double[n].
 * Sources are processed in batches of options->n_b (Algorithm 3's loop); a
 * short last batch is padded with inactive columns (Theorem 1's padding).
 * Unless MFBC_OPT_KEEP_ORDER is set, the unit-weight kernels on an
 * undirected graph with more sources than one batch first sort the sources
 * by their BFS distances to the 128 highest-degree vertices (one extra MFBF
 * pass), so that each batch holds sources of similar distance profile and
 * its frontier masks are denser; lambda is a sum over sources, so only the
 * floating-point summation order changes. */
mfbc_status mfbc_bc(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                    double* lambda_out, const mfbc_options* opt);

/* mfbc_bc with DEVICE sources int32[nsrc] and DEVICE lambda_out double[n]
 * (overwritten).  Work is queued on opt->stream; the call returns once the
 * result is complete on that stream. */
mfbc_status mfbc_bc_device(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                           double* lambda_out, const mfbc_options* opt);

/* Several betweenness requests in one pass.  The paper has no such call:
 * it serves callers that collect source lists of independent requests on one
 * graph (continuous batching) and packs their columns into shared batches of
 * Algorithm 3's loop.  DEVICE sources int32[nsrc] hold the requests' lists
 * back to back; HOST req_offsets int32[nreq+1] (req_offsets[0] = 0,
 * non-decreasing, req_offsets[nreq] = nsrc) delimit them: request r owns
 * sources[req_offsets[r] .. req_offsets[r+1]).  DEVICE lambda_out: row
 * lambda_rows[r] (row r when opt->lambda_rows is NULL; a row is n doubles at
 * lambda_out + row*n) receives request r's lambda exactly as mfbc_bc_device
 * would compute it for that list alone, up to the floating-point summation
 * order; the rows are overwritten, or added to with MFBC_OPT_ACCUMULATE (a
 * serving loop that splits a request over several calls keeps one row per
 * request and accumulates into it).  Each request starts on a 32-column
 * boundary of a batch and may continue into the next batch; sources are not
 * reordered.  Returns once lambda_out is complete on opt->stream. */
mfbc_status mfbc_bc_multi_device(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                                 const int32_t* req_offsets, int32_t nreq, double* lambda_out,
                                 const mfbc_options* opt);

/* Result of mfbc_autotune. */
typedef struct {
  int32_t n_b;            /* fastest batch width found */
  int32_t path;           /* MFBC_PATH_LEVEL, MFBC_PATH_GENERAL or MFBC_PATH_DIST */
  int32_t arcs;           /* general kernels: arcs walked per step (1 or 8); 0 on the level kernels */
  int32_t tried;          /* configurations timed */
  double ms_per_source;   /* wall time of the fastest configuration per source */
  int32_t accumulator;    /* general kernels: MFBC_ACCUM_* chosen; 0 on the other families */
} mfbc_tuning;

/* Autotuner (no counterpart in the paper, whose batch width and processor
 * grid come from its cost model, Sec. 5): times mfbc_bc on the HOST sources
 * int32[nsrc] for each candidate configuration and keeps the fastest on the
 * graph handle.  Candidates: n_b in {128, 256, 512, 1024} on the level kernels
 * and, for unit-weight graphs of at most 2^15 vertices and 2^19 arcs, n_b in
 * {32, 64, 128, 256} on the persistent small-graph kernel (AUTO itself takes
 * it up to 2^13 vertices and 2^18 arcs);
 * n_b in {128, 256, 512, 1024, 2048, 4096} on the general kernels (x the
 * atomic accumulator walking 1 or 8 arcs per step, the segmented accumulator,
 * the hash accumulator and the per-product choice) and on the distance
 * kernels; each at most nsrc
 * rounded up;
 * widths that do not fit the device are skipped.  With opt->path == AUTO a
 * weighted graph tries both the general and (weights <= 4096) the distance
 * kernels and later AUTO calls use the faster family; another path restricts
 * the search to it.  Each candidate runs twice (the first call untimed).
 * Later calls on this handle with opt->n_b == 0 use at most the tuned width
 * (no cap when the fastest width was the widest one tried), and the general
 * kernels use the tuned arcs per step (without tuning: 8 when the average
 * degree is at least 8, else 1) and, with opt->accumulator == AUTO, the tuned
 * accumulator.  n_b and accumulator in opt are ignored.  Results are
 * unaffected. */
mfbc_status mfbc_autotune(mfbc_graph* g, const int32_t* sources, int32_t nsrc, const mfbc_options* opt,
                          mfbc_tuning* out);

/* MFBF alone (Algorithm 1, Lemma 1): for each i < nsrc,
 *   dist_out [i*n + v] = tau(sources[i], v)        (INT32_MAX if unreachable)
 *   sigma_out[i*n + v] = sigma_bar(sources[i], v)  (0 if unreachable; sigma_bar(s,s) = 1)
 * HOST pointers; sigma_out may be NULL. */
mfbc_status mfbc_sssp_batch(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                            int32_t* dist_out, double* sigma_out, const mfbc_options* opt);

/* mfbc_sssp_batch with DEVICE sources, dist_out and sigma_out (sigma_out may be NULL). */
mfbc_status mfbc_sssp_batch_device(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                                   int32_t* dist_out, double* sigma_out,
                                   const mfbc_options* opt);

/* Device scratch (bytes) that mfbc_bc* (mode 0), mfbc_sssp_batch* (mode 1)
 * or mfbc_bc_multi_device (mode 2; nsrc = the packed columns, each request
 * rounded up to 32) needs for nsrc sources under *opt (n_b, path).  A caller that passes its
 * own opt->workspace of at least this size makes the call allocate nothing
 * on the device. */
mfbc_status mfbc_workspace_size(const mfbc_graph* g, int32_t nsrc, int32_t mode,
                                const mfbc_options* opt, uint64_t* bytes);

/* Allocation-free betweenness centrality.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate GPU memory at
 * call time -- a serving process whose device memory is fully partitioned by
 * its own pool, code inside an allocator callback or memory-pressure handler,
 * a plug-in whose host framework owns all device memory, or a latency-bound
 * loop that cannot absorb cudaMalloc's implicit synchronisation.
 * It computes the same lambda as mfbc_bc_device (DEVICE sources int32[nsrc],
 * DEVICE lambda_out double[n], overwritten; stream = cudaStream_t or NULL)
 * with the general kernels at n_b = 32, keeping all scratch in one file-scope
 * __device__ array of MFBC_STATIC_SCRATCH_BYTES that every GPU loading the
 * library holds until exit.  It calls no cudaMalloc, cudaFree or allocating
 * library routine.  The array's device address is looked up once per device
 * (cudaGetSymbolAddress, device current) by the first call on that device, so
 * make that first call before any stream capture.  Graphs with more than
 * mfbc_static_max_vertices() vertices are rejected with MFBC_ERR_INVALID.
 * All calls share the array and it keeps the last call's contents (each call
 * clears what must start at zero); calls that overlap on the GPU race.  The
 * call returns once lambda_out is complete on the stream.  warn_out (HOST,
 * may be NULL) receives the same MFBC_WARN_* bits as mfbc_options.warn_out:
 * MFBC_WARN_SIGMA_INEXACT when some sigma_bar reached 2^53. */
#define MFBC_STATIC_SCRATCH_BYTES (32u << 20)
mfbc_status mfbc_bc_static(const mfbc_graph* g, const int32_t* sources, int32_t nsrc,
                           double* lambda_out, void* stream, uint32_t* warn_out);

/* Largest vertex count mfbc_bc_static accepts. */
uint64_t mfbc_static_max_vertices(void);

const char* mfbc_status_string(mfbc_status s);

/* Detail of the last error on the calling thread ("" if none). */
const char* mfbc_last_error(void);

/* Library version string. */
const char* mfbc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MFBC_H */
