// FP32 error-free transforms and double-word FP32 arithmetic, shared by the
// cross-section fit and the ray tracer's precise decisions.
#pragma once

#include <cuda_runtime.h>

namespace hr {

// Knuth's TwoSum: returns s = fl(a + b) and sets e with s + e == a + b
// exactly (round to nearest, no overflow).  The _rn intrinsics keep the
// compiler from contracting or reordering the steps.
__device__ __forceinline__ float two_sum(float a, float b, float& e) {
  const float s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return s;
}

// Double-word FP32 numbers hi + lo, |lo| <= ulp(hi) / 2 (Dekker 1971; the
// accurate addition of Li et al., "Design, implementation and testing of
// extended and mixed precision BLAS", 2002): about 2^-44 relative error per
// operation, at a few FP32 operations each instead of one FP64 operation
// (1/64 of the FP32 rate on this GPU).
struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_fast(float a, float b) {  // |a| >= |b|
  const float s = __fadd_rn(a, b);
  return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ df df_add(df a, df b) {
  float e1, e2;
  const float s = two_sum(a.hi, b.hi, e1);
  const float t = two_sum(a.lo, b.lo, e2);
  const df u = df_fast(s, __fadd_rn(e1, t));
  return df_fast(u.hi, __fadd_rn(u.lo, e2));
}
__device__ __forceinline__ df df_sub(df a, df b) { return df_add(a, {-b.hi, -b.lo}); }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  const float e = fmaf(a.hi, b.hi, -p);
  return df_fast(p, fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e)));
}
__device__ __forceinline__ df df_mul(df a, float b) {
  const float p = __fmul_rn(a.hi, b);
  const float e = fmaf(a.hi, b, -p);
  return df_fast(p, fmaf(a.lo, b, e));
}
__device__ __forceinline__ float df_float(df a) { return __fadd_rn(a.hi, a.lo); }
__device__ __forceinline__ double df_double(df a) { return (double)a.hi + (double)a.lo; }
// Exact product: returns p = fl(a b) and sets e with p + e == a b (the FMA
// form of Dekker's TwoProduct).
__device__ __forceinline__ float two_prod(float a, float b, float& e) {
  const float p = __fmul_rn(a, b);
  e = fmaf(a, b, -p);
  return p;
}
__device__ __forceinline__ df df_add(df a, float b) {
  float e;
  const float s = two_sum(a.hi, b, e);
  return df_fast(s, __fadd_rn(e, a.lo));
}

}  // namespace hr
