// Float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits with the exponent range of float.  The
// operations are built from the error-free transformations of Knuth
// (two_sum: a + b = s + e exactly) and Dekker (two_prod: a * b = p + e
// exactly, here through one FMA), as in the classical double-double
// literature (Dekker 1971; Hida, Li and Bailey 2001), at half the width.
// Every step uses the _rn intrinsics so that the compiler cannot contract a
// multiply and an add into an FMA, which would break the error terms.
//
// On this GPU an SM retires one FP64 warp instruction about every 19 cycles
// but four FP32 warp instructions per cycle, so a float-float operation
// (4 to 15 FP32 instructions) is far cheaper than the FP64 one it replaces.
#pragma once

#include <cuda_runtime.h>

namespace amm {

struct ff {
  float hi, lo;
};

__device__ __forceinline__ ff ff_make(float h, float l) {
  ff r;
  r.hi = h;
  r.lo = l;
  return r;
}
__device__ __forceinline__ ff ff_from(float x) { return ff_make(x, 0.f); }

// s + e = a + b exactly (any a, b)
__device__ __forceinline__ ff two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return ff_make(s, e);
}
// s + e = a + b exactly when |a| >= |b| (or a = 0)
__device__ __forceinline__ ff fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return ff_make(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ ff ff_neg(ff a) { return ff_make(-a.hi, -a.lo); }

__device__ __forceinline__ ff ff_add(ff a, ff b) {
  const ff s = two_sum(a.hi, b.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo)));
}

__device__ __forceinline__ ff ff_mul(ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);  // the rounding error of p, exactly
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  return fast_two_sum(p, e);
}

// a * b + c with one normalisation
__device__ __forceinline__ ff ff_fma(ff a, ff b, ff c) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = fmaf(a.hi, b.hi, -p);
  e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
  const ff s = two_sum(p, c.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(e, c.lo)));
}

// 1 / sqrt(x) for x > 0: the FP32 estimate r refined by one Newton step
// r + r (1 - x r^2) / 2 with the residual formed in float-float (the
// relative error goes from about 2^-23 to about 2^-44).
__device__ __forceinline__ ff ff_rsqrt(ff x) {
  const float r = rsqrtf(x.hi);
  const ff xrr = ff_mul(ff_mul(x, ff_from(r)), ff_from(r));
  const float h = __fsub_rn(__fsub_rn(1.f, xrr.hi), xrr.lo);
  return fast_two_sum(r, __fmul_rn(__fmul_rn(r, h), 0.5f));
}

}  // namespace amm

namespace amm {

// x rounded to float-float (hi = x rounded to float, lo = the rest rounded);
// NaN stays NaN in hi.
__device__ __forceinline__ ff ff_from_double(double x) {
  const float h = __double2float_rn(x);
  return ff_make(h, __double2float_rn(x - (double)h));
}
__device__ __forceinline__ double ff_to_double(ff a) { return (double)a.hi + (double)a.lo; }

// acc + a b with the product split exactly (a dot-product step)
__device__ __forceinline__ ff ff_dot_acc(ff acc, float a, float b) {
  const float p = __fmul_rn(a, b);
  const float e = fmaf(a, b, -p);
  const ff t = two_sum(acc.hi, p);
  return fast_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(e, acc.lo)));
}

__device__ __forceinline__ ff ff_shfl_xor(ff v, int m) {
  return ff_make(__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m));
}

// Sum over the block in float-float, a fixed order; every thread gets the
// same value.  redf must hold 2 * (warps + 1) floats.  Contains
// __syncthreads().
__device__ __forceinline__ ff block_sum_ff(ff v, float* redf) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = ff_add(v, ff_shfl_xor(v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = blockDim.x >> 5;
  __syncthreads();
  if (l == 0) {
    redf[2 * w] = v.hi;
    redf[2 * w + 1] = v.lo;
  }
  __syncthreads();
  ff s = ff_make(redf[0], redf[1]);
  for (int q = 1; q < nw; ++q) s = ff_add(s, ff_make(redf[2 * q], redf[2 * q + 1]));
  return s;
}

}  // namespace amm
