#pragma once

#include "internal.cuh"

namespace mfbc {

// Double-float arithmetic of the unit-weight kernels (level.cu, small.cu).
//
// GB300 executes FP64 at a small fraction of its FP32 rate, so the hot loops
// avoid it: MFBF path counts are exact 64-bit integers, and MFBr values
// zeta + 1/sigma_bar are double-float pairs (hi + lo, about 48 significant
// bits) kept in the same 8-byte slots and combined on the FP32 pipes with
// error-free transformations (Fast2Sum, FMA-based products).  Every MFBr
// quantity is non-negative, so no sum cancels.
struct dfl { float hi, lo; };

__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {   // |a| >= |b|
  s = a + b;
  e = b - (s - a);
}
// An exact integer count x < 2^58 as hi + lo: hi = x rounded to FP32, lo =
// the remainder rounded to FP32.  Exact below 2^48; above, the remainder has
// more than 24 bits and lo is rounded, a relative error of at most 2^-48 of x
// (the MFBF counts stop at 2^58: a larger one sends the batch to the FP64
// kernels).
__device__ __forceinline__ dfl df_of_u64(uint64_t x) {
  const float h = __ull2float_rn(x);
  const long long r = (long long)(x - (uint64_t)h);
  return {h, __ll2float_rn(r)};
}
__device__ __forceinline__ dfl df_mul(dfl a, dfl b) {
  const float p = a.hi * b.hi;
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, e);
  e = fmaf(a.lo, b.hi, e);
  float s, t;
  fast_two_sum(p, e, s, t);
  return {s, t};
}
// 1/x for x >= 1: the FP32 reciprocal approximation (rcp.approx, relative
// error about 2^-23) refined by one Newton step in double-float, e = 1 - x r,
// 1/x = r (1 + e + e^2 + ...) ~ r + r e (error about e^2 ~ 2^-46).
__device__ __forceinline__ dfl df_rcp(dfl a) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a.hi));
  float e = fmaf(-a.hi, r, 1.0f);
  e = fmaf(-a.lo, r, e);
  float s, t;
  fast_two_sum(r, r * e, s, t);
  return {s, t};
}
// a + b for a, b >= 0: no cancellation, so Fast2Sum on the ordered high
// parts plus the low parts gives a relative error of a few 2^-48.
__device__ __forceinline__ dfl df_add_pos(dfl a, dfl b) {
  const float x = fmaxf(a.hi, b.hi), y = fminf(a.hi, b.hi);
  const float s = x + y;
  const float e = (y - (s - x)) + (a.lo + b.lo);
  float h, l;
  fast_two_sum(s, e, h, l);
  return {h, l};
}
__device__ __forceinline__ uint64_t df_pack(dfl a) {
  return (uint64_t)__float_as_uint(a.hi) | ((uint64_t)__float_as_uint(a.lo) << 32);
}
__device__ __forceinline__ dfl df_unpack(uint64_t u) {
  return {__uint_as_float((uint32_t)u), __uint_as_float((uint32_t)(u >> 32))};
}
__device__ __forceinline__ dfl df_of_double(double x) {
  const float h = __double2float_rn(x);
  return {h, __double2float_rn(x - (double)h)};
}
// compensated accumulation of non-negative double-float terms (hi, lo) into
// (s, c): Fast2Sum on the ordered pair (max, min) gives the exact rounding
// error of s + hi (Neumaier's summation without its branch)
__device__ __forceinline__ void acc_add(float& s, float& c, float hi, float lo) {
  const float a = fmaxf(s, hi), b = fminf(s, hi);
  const float t = a + b;
  c += (b - (t - a)) + lo;
  s = t;
}
__device__ __forceinline__ void acc_add(float& s, float& c, uint64_t x) {
  const dfl v = df_unpack(x);
  acc_add(s, c, v.hi, v.lo);
}
__device__ __forceinline__ dfl acc_value(float s, float c) {
  float h, l;
  fast_two_sum(s, c, h, l);
  return {h, l};
}

// One column of a finished level-l pair (s,v) with zeta(s,v) = zt: the
// lambda term zeta * sigma_bar(s,v) goes into the compensated sum (ls, lc),
// and the slot's new value zeta + 1/sigma_bar is returned (Sec. 4.2.1,
// Algorithm 3).  w holds sigma_bar(s,v) as an integer below 2^58.
__device__ __forceinline__ uint64_t finish_col(dfl zt, uint64_t w, float& ls, float& lc) {
  const dfl sg = df_of_u64(w);
  const dfl p = df_mul(zt, sg);
  acc_add(ls, lc, p.hi, p.lo);
  return df_pack(df_add_pos(zt, df_rcp(sg)));
}
// warp sum of non-negative compensated sums (s, c), as a double on every lane
__device__ __forceinline__ double warp_acc_sum(float s, float c) {
  for (int o = 16; o; o >>= 1) {
    const float s2 = __shfl_xor_sync(0xffffffffu, s, o), c2 = __shfl_xor_sync(0xffffffffu, c, o);
    acc_add(s, c, s2, c2);
  }
  return (double)s + (double)c;
}

// Segmented warp sum of non-negative compensated sums (s, c) over runs of
// equal, non-decreasing keys; true on the last lane of each run, which then
// holds the run's sum.
__device__ __forceinline__ bool warp_acc_seg_sum(float& s, float& c, int key) {
  const unsigned lane = lane_id();
  for (int o = 1; o < 32; o <<= 1) {
    const float s2 = __shfl_up_sync(0xffffffffu, s, o), c2 = __shfl_up_sync(0xffffffffu, c, o);
    const int k2 = __shfl_up_sync(0xffffffffu, key, o);
    if ((int)lane >= o && k2 == key) acc_add(s, c, s2, c2);
  }
  const int kn = __shfl_down_sync(0xffffffffu, key, 1);
  return lane == 31 || kn != key;
}
}  // namespace mfbc
