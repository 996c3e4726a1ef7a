// mfbc_bc_static: betweenness centrality without any allocation.
//
// Some callers cannot allocate GPU memory when they need the result: a
// serving process whose device memory is fully partitioned among tenants by
// its own pool, code running inside an allocator callback or a memory-pressure
// handler (where cudaMalloc could recurse or deadlock), a framework plug-in
// whose host framework owns every device byte, or a latency-bound loop that
// cannot afford cudaMalloc's implicit device synchronisation.  For them this
// entry point runs the general MFBF / MFBr / lambda kernels with their
// per-batch state carved from one file-scope __device__ array instead of
// from cudaMalloc'ed scratch: it calls no cudaMalloc, cudaFree or other
// allocating routine.  The caller still passes device inputs and outputs.
//
// The array is MFBC_STATIC_SCRATCH_BYTES large and is held by every GPU that
// loads the library until the process exits.  Its address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on that device; that first call should therefore happen
// before any stream capture.  All calls share the array and it keeps the last
// call's contents; everything that must start at zero is cleared by each
// call.  Calls whose work overlaps on the GPU (e.g. on two streams) race on
// the array: serialise them.
#include <mutex>

#include "internal.cuh"

namespace mfbc {

// Host code may not dereference or pass this symbol: on the host it is a
// stand-in, not a device address.  Use static_scratch_ptr().
static __device__ __align__(256) unsigned char g_static_scratch[MFBC_STATIC_SCRATCH_BYTES];

constexpr int kStaticNb = 32;          // batch width used by the static entry point
constexpr int kMaxDevices = 64;
static void* g_scratch_ptr[kMaxDevices];
static std::mutex g_static_mu;         // also serialises host-side use of the array

// Device address of the array on the current device (set up once per device).
static mfbc_status static_scratch_ptr(void** out, std::string* err) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(err, "cudaGetDevice", e);
  if (dev < 0 || dev >= kMaxDevices) {
    if (err) *err = "device ordinal out of range for the static scratch table";
    return MFBC_ERR_INVALID;
  }
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(g_static_scratch)", e);
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MFBC_OK;
}

__global__ void k_check_sources(const int32_t* __restrict__ src, int32_t nsrc, int32_t n, Counters* ctr) {
  int32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nsrc && (src[i] < 0 || src[i] >= n)) atomicOr(&ctr->flags, FLAG_BAD_SOURCE);
}

}  // namespace mfbc

using namespace mfbc;

extern "C" uint64_t mfbc_static_max_vertices(void) {
  // largest n whose general state at n_b = 32 fits the array
  uint64_t lo = 0, hi = (uint64_t)MFBC_STATIC_SCRATCH_BYTES;
  while (lo < hi) {
    uint64_t mid = (lo + hi + 1) / 2;
    if (general_bytes((int32_t)mid, kStaticNb) <= (size_t)MFBC_STATIC_SCRATCH_BYTES) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

extern "C" mfbc_status mfbc_bc_static(const mfbc_graph* G, const int32_t* sources, int32_t nsrc,
                                      double* lambda_out, void* stream, uint32_t* warn_out) {
  if (warn_out) *warn_out = 0;
  if (!G) { set_last_error("graph must not be NULL"); return MFBC_ERR_INVALID; }
  if (nsrc < 0) { set_last_error("nsrc must be >= 0"); return MFBC_ERR_INVALID; }
  if (nsrc > 0 && !sources) { set_last_error("sources must not be NULL"); return MFBC_ERR_INVALID; }
  const DevGraph* g = graph_device_view(G);
  if (g->n > 0 && !lambda_out) { set_last_error("lambda_out must not be NULL"); return MFBC_ERR_INVALID; }
  if (general_bytes(g->n, kStaticNb) > (size_t)MFBC_STATIC_SCRATCH_BYTES) {
    set_last_error("graph too large for mfbc_bc_static: n = " + std::to_string(g->n) + " exceeds " +
                   std::to_string(mfbc_static_max_vertices()) + " vertices (" +
                   std::to_string((unsigned long long)MFBC_STATIC_SCRATCH_BYTES) + "-byte scratch array)");
    return MFBC_ERR_INVALID;
  }
  std::lock_guard<std::mutex> lock(g_static_mu);
  graph_lock(G);
  std::string err;
  mfbc_status s = MFBC_OK;
  cudaStream_t st = (cudaStream_t)stream;
  uint32_t* h_ctr = graph_counter_mirror(G);
  void* base = nullptr;
  do {
    s = static_scratch_ptr(&base, &err);
    if (s) break;
    Carver c(base, MFBC_STATIC_SCRATCH_BYTES);
    GeneralState gs;
    general_carve(c, g->n, kStaticNb, gs);
    Profiler prof;                     // off: records no events
    RunCtx rc{g, st, &prof, h_ctr, &err};
    cudaError_t e = cudaMemsetAsync(gs.ctr, 0, sizeof(Counters), st);
    if (e != cudaSuccess) { s = cuda_fail(&err, "cudaMemsetAsync(counters)", e); break; }
    if (g->n) {
      e = cudaMemsetAsync(lambda_out, 0, sizeof(double) * (size_t)g->n, st);
      if (e != cudaSuccess) { s = cuda_fail(&err, "cudaMemsetAsync(lambda)", e); break; }
    }
    if (nsrc > 0) {
      k_check_sources<<<(nsrc + 255) / 256, 256, 0, st>>>(sources, nsrc, g->n, gs.ctr);
      e = cudaMemcpyAsync(h_ctr, &gs.ctr->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) { s = cuda_fail(&err, "checking sources", e); break; }
      if (h_ctr[0] & FLAG_BAD_SOURCE) { s = MFBC_ERR_INVALID; err = "source id out of range"; break; }
    }
    for (int32_t b0 = 0; b0 < nsrc && s == MFBC_OK; b0 += kStaticNb) {
      const int na = nsrc - b0 < kStaticNb ? nsrc - b0 : kStaticNb;
      s = general_batch(rc, gs, sources + b0, na, lambda_out, nullptr, nullptr);
    }
    if (s) break;
    // the general batches raise FLAG_SIGMA_INEXACT when a path count reaches
    // 2^53; report it like mfbc_bc_device does through warn_out
    e = cudaMemcpyAsync(h_ctr, &gs.ctr->flags, sizeof(uint32_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) { s = cuda_fail(&err, "mfbc_bc_static", e); break; }
    if (warn_out && (h_ctr[0] & FLAG_SIGMA_INEXACT)) *warn_out |= MFBC_WARN_SIGMA_INEXACT;
  } while (0);
  graph_unlock(G);
  if (s) { set_last_error(err.empty() ? mfbc_status_string(s) : err); cudaGetLastError(); }
  else set_last_error("");
  return s;
}
