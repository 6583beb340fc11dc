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

// ----------------------------------------------------------------- scalar double-float
// Real double-float numbers (h + l, |l| <= ulp(h)/2) for the FP64-accuracy far-field sums.
// All operations use the _rn intrinsics so the compiler never contracts or reorders them.

struct dfs {
  float h, l;
};

__device__ __forceinline__ dfs dfs_make(double v) {
  const float h = __double2float_rn(v);
  return dfs{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double dfs_value(dfs a) { return (double)a.h + (double)a.l; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ dfs dfs_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fsub_rn(s, a);
  return dfs{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}
// s + e = a + b exactly when |a| >= |b| or a = 0 (Dekker)
__device__ __forceinline__ dfs dfs_fast_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  return dfs{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfs dfs_add(dfs a, dfs b) {
  const dfs s = dfs_two_sum(a.h, b.h);
  return dfs_fast_sum(s.h, __fadd_rn(s.l, __fadd_rn(a.l, b.l)));
}
__device__ __forceinline__ dfs dfs_neg(dfs a) { return dfs{-a.h, -a.l}; }
__device__ __forceinline__ dfs dfs_sub(dfs a, dfs b) { return dfs_add(a, dfs_neg(b)); }
__device__ __forceinline__ dfs dfs_addf(dfs a, float b) {
  const dfs s = dfs_two_sum(a.h, b);
  return dfs_fast_sum(s.h, __fadd_rn(s.l, a.l));
}
// products: the high product's error by FMA (TwoProduct), plus the cross terms
__device__ __forceinline__ dfs dfs_mul(dfs a, dfs b) {
  const float p = __fmul_rn(a.h, b.h);
  float e = __fmaf_rn(a.h, b.h, -p);
  e = __fmaf_rn(a.h, b.l, e);
  e = __fmaf_rn(a.l, b.h, e);
  return dfs_fast_sum(p, e);
}
__device__ __forceinline__ dfs dfs_mulf(dfs a, float b) {
  const float p = __fmul_rn(a.h, b);
  float e = __fmaf_rn(a.h, b, -p);
  e = __fmaf_rn(a.l, b, e);
  return dfs_fast_sum(p, e);
}
__device__ __forceinline__ dfs dfs_sqr(dfs a) {
  const float p = __fmul_rn(a.h, a.h);
  float e = __fmaf_rn(a.h, a.h, -p);
  e = __fmaf_rn(__fmul_rn(2.0f, a.h), a.l, e);
  return dfs_fast_sum(p, e);
}

// 1/sqrt(a) for a > 0: the hardware estimate, one FP32 Newton step, then one Newton step
// whose residual 1 - a y^2 is formed exactly enough in double-float (quadratic convergence
// from ~2^-24 to ~2^-47).
__device__ __forceinline__ dfs dfs_rsqrt(dfs a) {
  float y = rsqrtf(a.h);
  y = __fmul_rn(y, __fmaf_rn(__fmul_rn(-0.5f, a.h), __fmul_rn(y, y), 1.5f));
  const float q = __fmul_rn(y, y);
  const dfs y2{q, __fmaf_rn(y, y, -q)};
  const dfs w = dfs_mul(a, y2);
  const float res = __fsub_rn(__fsub_rn(1.0f, w.h), w.l);  // 1 - w.h is exact (w.h near 1)
  return dfs_fast_sum(y, __fmul_rn(__fmul_rn(0.5f, y), res));
}

// Double-float constants: the float nearest to the value and the float nearest to the rest.
#define VSIE_DFC(name, hi, lo) __device__ __forceinline__ dfs name() { return dfs{hi, lo}; }
VSIE_DFC(dfc_two_pi, 0x1.921fb6p+2f, -0x1.777a5cp-23f)
VSIE_DFC(dfc_sqrt_half, 0x1.6a09e6p-1f, 0x1.9fcef4p-27f)
VSIE_DFC(dfc_inv3, 0x1.555556p-3f, -0x1.555556p-28f)    // 1/3!
VSIE_DFC(dfc_inv4, 0x1.555556p-5f, -0x1.555556p-30f)    // 1/4!
VSIE_DFC(dfc_inv5, 0x1.111112p-7f, -0x1.dddddep-32f)     // 1/5!
VSIE_DFC(dfc_inv6, 0x1.6c16c2p-10f, -0x1.27d27ep-35f)   // 1/6!
VSIE_DFC(dfc_inv7, 0x1.a01a02p-13f, -0x1.7f97fap-39f)   // 1/7!
VSIE_DFC(dfc_inv8, 0x1.a01a02p-16f, -0x1.7f97fap-42f)   // 1/8!
VSIE_DFC(dfc_inv9, 0x1.71de3ap-19f, 0x1.55b1ccp-45f)    // 1/9!
#undef VSIE_DFC

// (cos, sin)(2 pi f) for a double-float f with |f| <= 1/2 (plus rounding).  Reduction to
// the nearest multiple m of 1/8 (exact in float), g = f - m/8 with |2 pi g| <= pi/8, Taylor
// series of sin and cos in x = (2 pi g)^2 (terms through x^7: truncation below 2e-18),
// the terms below 1e-10 in plain float and the others in double-float Horner steps, then
// rotation by m pi/4 (a sum/difference scaled by sqrt(1/2) for odd m, a quarter-turn
// permutation with sign changes).
__device__ __forceinline__ void dfs_cossin_2pi(dfs f, dfs& c, dfs& s) {
  const float m = rintf(__fmul_rn(8.0f, f.h));
  const dfs g = dfs_two_sum(__fmaf_rn(-0.125f, m, f.h), f.l);
  const dfs th = dfs_mul(g, dfc_two_pi());
  const dfs x = dfs_sqr(th);
  const float xh = x.h;
  // sin(th) = th (1 - x/3! + x^2/5! - x^3/7! + x^4/9! - x^5/11! + x^6/13! - x^7/15!)
  const float ts = __fmul_rn(xh, __fmaf_rn(xh, __fmaf_rn(xh, -7.6471636e-13f, 1.6059044e-10f), -2.5052108e-08f));
  dfs p = dfs_addf(dfc_inv9(), ts);
  p = dfs_sub(dfs_mul(p, x), dfc_inv7());
  p = dfs_add(dfs_mul(p, x), dfc_inv5());
  p = dfs_sub(dfs_mul(p, x), dfc_inv3());
  p = dfs_addf(dfs_mul(p, x), 1.0f);
  const dfs sn = dfs_mul(p, th);
  // cos(th) = 1 - x/2! + x^2/4! - x^3/6! + x^4/8! - x^5/10! + x^6/12! - x^7/14!
  const float tc = __fmul_rn(xh, __fmaf_rn(xh, __fmaf_rn(xh, -1.1470745e-11f, 2.0876756e-09f), -2.7557320e-07f));
  dfs q = dfs_addf(dfc_inv8(), tc);
  q = dfs_sub(dfs_mul(q, x), dfc_inv6());
  q = dfs_add(dfs_mul(q, x), dfc_inv4());
  q = dfs_addf(dfs_mul(q, x), -0.5f);
  q = dfs_addf(dfs_mul(q, x), 1.0f);
  dfs cs = q;
  dfs sv = sn;
  const int mi = (int)m;  // -4 .. 4
  if (mi & 1) {  // rotate by pi/4: (c - s, c + s) sqrt(1/2)
    const dfs a = dfs_mul(dfs_sub(cs, sv), dfc_sqrt_half());
    const dfs b = dfs_mul(dfs_add(cs, sv), dfc_sqrt_half());
    cs = a;
    sv = b;
  }
  const int qd = ((mi - (mi & 1)) / 2) & 3;  // remaining quarter turns
  if (qd == 1) {
    const dfs t = cs;
    cs = dfs_neg(sv);
    sv = t;
  } else if (qd == 2) {
    cs = dfs_neg(cs);
    sv = dfs_neg(sv);
  } else if (qd == 3) {
    const dfs t = cs;
    cs = sv;
    sv = dfs_neg(t);
  }
  c = cs;
  s = sv;
}

struct DTgt {
  dfs x, y, z;
};

// d = t - y~ (y~ from records a = (x.h, y.h, z.h, *), b = (x.l, y.l, z.l, *)); rinv = 1/|d|
// (0 at d = 0), tt = |d| (revolutions), (cs, sn) = (cos, sin)(2 pi tt)
__device__ __forceinline__ void df_geometry(const DTgt& t, const float4& a, const float4& b, dfs& dx, dfs& dy,
                                            dfs& dz, dfs& rinv, dfs& tt, dfs& cs, dfs& sn) {
  dx = dfs_sub(t.x, dfs{a.x, b.x});
  dy = dfs_sub(t.y, dfs{a.y, b.y});
  dz = dfs_sub(t.z, dfs{a.z, b.z});
  const dfs r2 = dfs_add(dfs_add(dfs_sqr(dx), dfs_sqr(dy)), dfs_sqr(dz));
  const bool zero = !(r2.h > 0.0f);
  rinv = dfs_rsqrt(zero ? dfs{1.0f, 0.0f} : r2);
  if (zero) rinv = dfs{0.0f, 0.0f};
  tt = dfs_mul(r2, rinv);
  const float n = rintf(tt.h);
  const dfs f = dfs_two_sum(__fsub_rn(tt.h, n), tt.l);
  dfs_cossin_2pi(f, cs, sn);
}

__device__ __forceinline__ float4 df_c4(dfs re, dfs im) { return make_float4(re.h, im.h, re.l, im.l); }

// G coefficient e^{2 pi i t} / |d~|  and K coefficient e^{2 pi i t}(2 pi i t - 1)(d~ . n)/|d~|^3
// as double-float complex numbers (re.hi, im.hi, re.lo, im.lo)
__device__ __forceinline__ float4 df_coef_g(const DTgt& t, const float4& a, const float4& b) {
  dfs dx, dy, dz, rinv, tt, cs, sn;
  df_geometry(t, a, b, dx, dy, dz, rinv, tt, cs, sn);
  return df_c4(dfs_mul(cs, rinv), dfs_mul(sn, rinv));
}
__device__ __forceinline__ float4 df_coef_k(const DTgt& t, const float4& a, const float4& b, dfs nx, dfs ny,
                                            dfs nz) {
  dfs dx, dy, dz, rinv, tt, cs, sn;
  df_geometry(t, a, b, dx, dy, dz, rinv, tt, cs, sn);
  const dfs dn = dfs_add(dfs_add(dfs_mul(dx, nx), dfs_mul(dy, ny)), dfs_mul(dz, nz));
  const dfs g3 = dfs_mul(dfs_mul(dfs_sqr(rinv), rinv), dn);
  const dfs kr = dfs_mul(tt, dfc_two_pi());
  const dfs A = dfs_add(cs, dfs_mul(kr, sn));  // cos + kr sin
  const dfs Q = dfs_sub(dfs_mul(kr, cs), sn);  // kr cos - sin
  return df_c4(dfs_neg(dfs_mul(g3, A)), dfs_mul(g3, Q));
}

}  // namespace vsie
