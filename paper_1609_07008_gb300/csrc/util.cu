// Small device utilities: fills, the per-source transposed output copy, the
// FP64 path-count exactness check, and the event-based per-kernel profiler.
#include "internal.cuh"

namespace mfbc {

__global__ void k_fill_i32(int32_t* __restrict__ p, int32_t v, size_t count) {
  // scalar stores: p may be any 4-byte aligned pointer (e.g. a row offset
  // into a caller's output buffer)
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t k = i; k < count; k += stride) p[k] = v;
}

__global__ void k_fill_f64(double* __restrict__ p, double v, size_t count) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  for (size_t k = i; k < count; k += stride) p[k] = v;
}

static int fill_grid(size_t count) {
  size_t b = (count / 4 + 255) / 256;
  if (b < 1) b = 1;
  if (b > 152 * 16) b = 152 * 16;
  return (int)b;
}

void fill_i32(int32_t* p, int32_t v, size_t count, cudaStream_t st) {
  if (!count) return;
  k_fill_i32<<<fill_grid(count), 256, 0, st>>>(p, v, count);
}

void fill_f64(double* p, double v, size_t count, cudaStream_t st) {
  if (!count) return;
  k_fill_f64<<<fill_grid(count * 2), 256, 0, st>>>(p, v, count);
}

// flags bit1 is raised when any path count reaches 2^53 (FP64 may be inexact).
__global__ void k_sigma_exact(const double* __restrict__ s, size_t count, Counters* ctr) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  size_t stride = (size_t)gridDim.x * blockDim.x;
  bool big = false;
  for (size_t k = i; k < count; k += stride) big |= (s[k] >= 9007199254740992.0);
  if (__syncthreads_or(big) && threadIdx.x == 0) atomicOr(&ctr->flags, FLAG_SIGMA_INEXACT);
}

void check_sigma_exact(const double* sig, size_t count, Counters* ctr, cudaStream_t st) {
  if (!count) return;
  k_sigma_exact<<<fill_grid(count * 2), 256, 0, st>>>(sig, count, ctr);
}

// out[j * out_ld + v] = in[v * nb + j] for v < n, j < nactive (32x32 smem tiles)
template <class T>
__global__ void k_transpose(const T* __restrict__ in, T* __restrict__ out, int32_t n, int nb,
                            int nactive, int64_t out_ld) {
  __shared__ T tile[32][33];
  int64_t v0 = (int64_t)blockIdx.x * 32;
  int j0 = blockIdx.y * 32;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int64_t v = v0 + r;
    int j = j0 + threadIdx.x;
    if (v < n && j < nb) tile[r][threadIdx.x] = in[v * nb + j];
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    int j = j0 + r;
    int64_t v = v0 + threadIdx.x;
    if (v < n && j < nactive) out[(int64_t)j * out_ld + v] = tile[threadIdx.x][r];
  }
}

void transpose_i32(const int32_t* in, int32_t* out, int32_t n, int nb, int nactive, int64_t out_ld,
                   cudaStream_t st) {
  if (!n || !nactive) return;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((nactive + 31) / 32));
  k_transpose<int32_t><<<grid, dim3(32, 8), 0, st>>>(in, out, n, nb, nactive, out_ld);
}

void transpose_f64(const double* in, double* out, int32_t n, int nb, int nactive, int64_t out_ld,
                   cudaStream_t st) {
  if (!n || !nactive) return;
  dim3 grid((unsigned)((n + 31) / 32), (unsigned)((nactive + 31) / 32));
  k_transpose<double><<<grid, dim3(32, 8), 0, st>>>(in, out, n, nb, nactive, out_ld);
}

// ------------------------------------------------------------------ Profiler
static const char* kNames[K_NUM] = {
  "fill", "mfbf_seed", "mfbf_relax_min", "mfbf_relax_tie", "mfbf_accumulate",
  "mfbr_counters_leaves", "mfbr_propagate", "mfbr_next_frontier", "lambda_accumulate",
  "clear_masks", "level_mfbf_pairs", "level_visit", "level_mfbr_pairs", "level_mfbr_hub_final",
  "level_reset", "output_copy", "level_mfbf_gather", "level_mfbr_gather", "level_round_split",
  "dist_mfbf", "dist_mfbr", "small_persistent", "mfbf_pull", "mfbr_pull",
  "mfbf_hash_min", "mfbf_hash_tie", "mfbr_hash"};

Profiler::Profiler() {
  for (int i = 0; i < K_NUM; i++) k[i].name = kNames[i];
}

cudaEvent_t Profiler::get() {
  if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
  cudaEvent_t e;
  cudaEventCreate(&e);
  return e;
}

void Profiler::begin(KId id) {
  k[id].launches++;
  if (!on) return;
  Pending p{id, get(), get()};
  cudaEventRecord(p.a, stream);
  pend.push_back(p);
}

void Profiler::end(KId id) {
  if (!on || pend.empty()) return;
  cudaEventRecord(pend.back().b, stream);
  (void)id;
}

void Profiler::drain() {
  if (!on) return;
  for (auto& p : pend) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.a, p.b) == cudaSuccess) k[p.id].ms += ms;
    pool.push_back(p.a);
    pool.push_back(p.b);
  }
  pend.clear();
}

void Profiler::release() {
  drain();
  for (auto e : pool) cudaEventDestroy(e);
  pool.clear();
}

int batch_uniform_request(const int32_t* word_req, int W) {
  if (!word_req) return 0;
  int r = -1;
  for (int w = 0; w < W; w++) {
    const int x = word_req[w];
    if (x < 0) continue;
    if (r < 0) r = x;
    else if (r != x) return -2;
  }
  return r < 0 ? 0 : r;
}

}  // namespace mfbc
