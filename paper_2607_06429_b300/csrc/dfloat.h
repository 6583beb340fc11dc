// Double-float arithmetic on the FP32 pipe.  On B300 the FP64 pipe runs at about 1/64 of
// the FP32 rate, so sums that need more than FP32 accuracy but are dominated by
// multiply-adds (the correction SpMV, the FP64 multi-RHS contraction) carry each real
// number as an unevaluated pair hi + lo of floats (about 48 significant bits) and use the
// error-free transformations TwoSum (Knuth) and TwoProduct by fused multiply-add.
// Complex numbers are stored as float4 (re.hi, im.hi, re.lo, im.lo) and processed as
// packed (re, im) pairs with the FP32x2 instructions.
#pragma once

#include <cuda_runtime.h>

namespace vsie {

__device__ __forceinline__ float2 df_bc(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 df_neg(float2 a) { return make_float2(-a.x, -a.y); }

// complex128 -> (re.hi, im.hi, re.lo, im.lo)
__device__ __forceinline__ float4 df_pack(double2 v) {
  const float rh = __double2float_rn(v.x), ih = __double2float_rn(v.y);
  return make_float4(rh, ih, __double2float_rn(v.x - (double)rh), __double2float_rn(v.y - (double)ih));
}

// s + e = a + b exactly (componentwise)
__device__ __forceinline__ void df_two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = __fadd2_rn(a, b);
  const float2 z = __ffma2_rn(a, df_bc(-1.0f), s);          // s - a
  const float2 t = __ffma2_rn(z, df_bc(-1.0f), s);          // s - z
  e = __fadd2_rn(__ffma2_rn(t, df_bc(-1.0f), a), __ffma2_rn(z, df_bc(-1.0f), b));  // (a - t) + (b - z)
}

// (S, C) += v x for complex double-float v, x: the products by TwoProduct (FMA) plus the
// cross terms hi*lo, the sums by TwoSum, every rounding error collected in C.
__device__ __forceinline__ void df_cmac(float2& S, float2& C, float4 v, float4 x) {
  const float2 xh = make_float2(x.x, x.y), xl = make_float2(x.z, x.w);
  const float2 jh = make_float2(-x.y, x.x), jl = make_float2(-x.w, x.z);  // i x
  const float2 p1 = __fmul2_rn(df_bc(v.x), xh);                             // re(v) x
  float2 e1 = __ffma2_rn(df_bc(v.x), xh, df_neg(p1));
  e1 = __ffma2_rn(df_bc(v.x), xl, e1);
  e1 = __ffma2_rn(df_bc(v.z), xh, e1);
  const float2 p2 = __fmul2_rn(df_bc(v.y), jh);                             // im(v) i x
  float2 e2 = __ffma2_rn(df_bc(v.y), jh, df_neg(p2));
  e2 = __ffma2_rn(df_bc(v.y), jl, e2);
  e2 = __ffma2_rn(df_bc(v.w), jh, e2);
  float2 s, e;
  df_two_sum2(S, p1, s, e);
  C = __fadd2_rn(C, __fadd2_rn(e, e1));
  df_two_sum2(s, p2, S, e);
  C = __fadd2_rn(C, __fadd2_rn(e, e2));
}

// (S, C) <- S + C renormalised (hi carries the sum, lo the rounding error)
__device__ __forceinline__ void df_renorm2(float2& S, float2& C) {
  float2 s, e;
  df_two_sum2(S, C, s, e);
  S = s;
  C = e;
}

// (S, C) += (S2, C2)
__device__ __forceinline__ void df_add2(float2& S, float2& C, float2 S2, float2 C2) {
  float2 s, e;
  df_two_sum2(S, S2, s, e);
  S = s;
  C = __fadd2_rn(C, __fadd2_rn(C2, e));
}

__device__ __forceinline__ double2 df_value(float2 S, float2 C) {
  return make_double2((double)S.x + (double)C.x, (double)S.y + (double)C.y);
}

}  // namespace vsie
