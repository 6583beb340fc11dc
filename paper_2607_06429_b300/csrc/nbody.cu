// Far-field N-body sums of the discretised VSIE operator (Eq. vsie, Sec. 2.3.4).
//
// For a collocation point x and a far-field source point y with weights (s, v), the
// coefficient of the owning unknown p_e is
//     C(x, y) = G(r) [ -s + (i k r - 1) ((x - y) . v) / r^2 ],   G = e^{ikr}/(4 pi r),
// which covers the volume single layer (s = (beta - k0^2 alpha) w), the volume adjoint
// double layer (v = grad(alpha) w) and the interface double layer (v = -omega n w,
// since dG/dn_y = -grad_x G . n).  With charges q = -s p_e/(4 pi), u = v p_e/(4 pi):
//     y_i = sum_j (e^{ikr}/r) [ q_j + (i k r - 1) (d . u_j) / r^2 ],   r = 0 -> 0.
//
// Source classes (one kernel each, so no pair pays for terms it does not have):
//   G  volume points with v = 0:          y += (e^{ikr}/r) q
//   K  interface points (s = 0, v = sigma n):  y += e^{ikr} (ikr - 1)(d.n) c / r^3
//   F  volume points with grad(alpha) != 0:    the general form above
//
// Units: positions are stored pre-multiplied by kappa = k/(2 pi), so that
// t = |x~ - y~| = k r/(2 pi) is the phase in revolutions and 1/r = kappa/|x~ - y~|;
// the kappa powers are folded into the charges by the prescale kernels.  e^{ikr} is
// evaluated from f = t - round(t) in [-1/2, 1/2] (round by the 1.5*2^23 shifter, two
// adds on the FP32 pipe) so the hardware sine/cosine only sees |2 pi f| <= pi.
//
// Scheduling (B300, 148 SMs): a persistent grid of exactly the resident block count.
// The work is the list of (target tile of 512, source chunk of 1024) items in
// target-major order; block b takes the contiguous item range [b N/C, (b+1) N/C), so all
// blocks get the same number of pairs (+-1 chunk) and there is no tail wave.  A target
// tile that spans several blocks leaves its pieces in per-block slots, and a fix-up kernel
// adds them in block order (deterministic).  Within an item each thread owns 4 targets
// in registers; 128 source records at a time are staged in shared memory and read back
// as warp-wide broadcasts.  FP32 accumulation is compensated: each 128-source tile is
// summed in FP32 and folded into an FP32 (hi, lo) pair with an exact TwoSum.

#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "dfloat.h"
#include "vsie_internal.h"

namespace vsie {

constexpr int kBlock = 128;                 // threads per block, sources per smem tile
constexpr int kT = 4;                       // targets per thread
constexpr int kTile = kBlock * kT;          // targets per work item
constexpr int kChunk = 8 * kBlock;          // sources per work item (default; the autotuner may pick another)
constexpr double kTwoPi = 2.0 * kPi;

template <class R>
struct Vec4;
template <>
struct Vec4<float> {
  using type = float4;
};
template <>
struct Vec4<double> {
  using type = double4_32a;
};

// ----------------------------------------------------------------- phase helpers

// rinv = 1/|d~| (0 at d~ = 0), t = |d~| (revolutions), (cs, sn) = (cos, sin)(2 pi t)
__device__ __forceinline__ void phase(float r2, float& rinv, float& t, float& cs, float& sn) {
  rinv = (r2 > 0.0f) ? rsqrtf(r2) : 0.0f;
  t = r2 * rinv;
  const float shifter = 12582912.0f;  // 1.5 * 2^23: (t + s) - s rounds t to an integer
  const float rt = __fsub_rn(__fadd_rn(t, shifter), shifter);
  const float f = __fsub_rn(t, rt);
  __sincosf(f * 6.28318530717958647692f, &sn, &cs);
}
__device__ __forceinline__ void phase(double r2, double& rinv, double& t, double& cs, double& sn) {
  rinv = (r2 > 0.0) ? rsqrt(r2) : 0.0;
  t = r2 * rinv;
  const double f = t - rint(t);
  sincospi(2.0 * f, &sn, &cs);
}

// ----------------------------------------------------------------- accumulators

template <class R>
struct Acc;
template <>
struct Acc<float> {
  float hr, lr, hi, li;
  __device__ __forceinline__ void zero() { hr = lr = hi = li = 0.0f; }
  __device__ __forceinline__ static void two_sum(float& h, float& l, float a) {
    const float s = __fadd_rn(h, a);
    const float bp = __fsub_rn(s, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bp)), __fsub_rn(a, bp));
    h = s;
    l = __fadd_rn(l, e);
  }
  __device__ __forceinline__ void fold(float ar, float ai) {
    two_sum(hr, lr, ar);
    two_sum(hi, li, ai);
  }
  __device__ __forceinline__ double2 value() const {
    return make_double2((double)hr + (double)lr, (double)hi + (double)li);
  }
};
template <>
struct Acc<double> {
  double r, i;
  __device__ __forceinline__ void zero() { r = i = 0.0; }
  __device__ __forceinline__ void fold(double ar, double ai) {
    r += ar;
    i += ai;
  }
  __device__ __forceinline__ double2 value() const { return make_double2(r, i); }
};

// ----------------------------------------------------------------- pair policies

// G: records a = (x~, y~, z~, q~.re), b = q~.im;  y += e^{2 pi i t} rinv q~
template <class R>
struct PolG {
  using V = typename Vec4<R>::type;
  struct Smem {
    V a[kBlock];
    R b[kBlock];
  };
  struct Src {
    V a;
    R b;
  };
  struct Tgt {
    R x, y, z;
  };
  const V* __restrict__ tgt;  // target positions (scaled, or unscaled if tscale != 1)
  R tscale;
  const V* __restrict__ sa;
  const R* __restrict__ sb;

  __device__ __forceinline__ void load_target(int64_t i, bool ok, Tgt& t) const {
    if (ok) {
      const V p = tgt[i];
      t.x = p.x * tscale;
      t.y = p.y * tscale;
      t.z = p.z * tscale;
    } else {
      t.x = t.y = t.z = R(0);
    }
  }
  __device__ __forceinline__ void stage(Smem& sm, int64_t j, bool ok, int tid) const {
    if (ok) {
      sm.a[tid] = sa[j];
      sm.b[tid] = sb[j];
    } else {
      sm.a[tid] = V{};  // zero charge contributes exactly 0 wherever it sits
      sm.b[tid] = R(0);
    }
  }
  __device__ __forceinline__ Src get(const Smem& sm, int jj) const { return Src{sm.a[jj], sm.b[jj]}; }
  __device__ __forceinline__ void pair(const Src& s, const Tgt& t, R& ar, R& ai) const {
    const R dx = t.x - s.a.x, dy = t.y - s.a.y, dz = t.z - s.a.z;
    const R r2 = dx * dx + dy * dy + dz * dz;
    R rinv, tt, cs, sn;
    phase(r2, rinv, tt, cs, sn);
    const R er = cs * rinv, ei = sn * rinv;
    ar += er * s.a.w - ei * s.b;
    ai += er * s.b + ei * s.a.w;
  }
};

// K: records a = (x~, y~, z~, c~.re), b = (c~.im, nx, ny, nz);
//    y += e^{2 pi i t} (2 pi i t - 1) (d~ . n) rinv^3 c~
template <class R>
struct PolK {
  using V = typename Vec4<R>::type;
  struct Smem {
    V a[kBlock];
    V b[kBlock];
  };
  struct Src {
    V a, b;
  };
  using Tgt = typename PolG<R>::Tgt;
  const V* __restrict__ tgt;
  R tscale;
  const V* __restrict__ src;  // 2 records per source

  __device__ __forceinline__ void load_target(int64_t i, bool ok, Tgt& t) const {
    if (ok) {
      const V p = tgt[i];
      t.x = p.x * tscale;
      t.y = p.y * tscale;
      t.z = p.z * tscale;
    } else {
      t.x = t.y = t.z = R(0);
    }
  }
  __device__ __forceinline__ void stage(Smem& sm, int64_t j, bool ok, int tid) const {
    if (ok) {
      sm.a[tid] = src[2 * j];
      sm.b[tid] = src[2 * j + 1];
    } else {
      sm.a[tid] = V{};
      sm.b[tid] = V{};
    }
  }
  __device__ __forceinline__ Src get(const Smem& sm, int jj) const { return Src{sm.a[jj], sm.b[jj]}; }
  __device__ __forceinline__ void pair(const Src& s, const Tgt& t, R& ar, R& ai) const {
    const R dx = t.x - s.a.x, dy = t.y - s.a.y, dz = t.z - s.a.z;
    const R r2 = dx * dx + dy * dy + dz * dz;
    R rinv, tt, cs, sn;
    phase(r2, rinv, tt, cs, sn);
    const R dn = dx * s.b.y + dy * s.b.z + dz * s.b.w;
    const R g3 = rinv * rinv * rinv * dn;
    const R gr = cs * g3, gi = sn * g3;
    const R kr = tt * R(6.28318530717958647692);
    const R hr = -gr - kr * gi, hi = kr * gr - gi;
    ar += hr * s.a.w - hi * s.b.x;
    ai += hr * s.b.x + hi * s.a.w;
  }
};

// F: records a = (x~, y~, z~, q~.re), b = (q~.im, ux.re, ux.im, uy.re), c = (uy.im, uz.re, uz.im, 0)
//    y += e^{2 pi i t} rinv [q~ + (2 pi i t - 1)(d~ . u~) rinv^2]
template <class R>
struct PolF {
  using V = typename Vec4<R>::type;
  struct Smem {
    V a[kBlock];
    V b[kBlock];
    V c[kBlock];
  };
  struct Src {
    V a, b, c;
  };
  using Tgt = typename PolG<R>::Tgt;
  const V* __restrict__ tgt;
  R tscale;
  const V* __restrict__ src;  // 3 records per source

  __device__ __forceinline__ void load_target(int64_t i, bool ok, Tgt& t) const {
    if (ok) {
      const V p = tgt[i];
      t.x = p.x * tscale;
      t.y = p.y * tscale;
      t.z = p.z * tscale;
    } else {
      t.x = t.y = t.z = R(0);
    }
  }
  __device__ __forceinline__ void stage(Smem& sm, int64_t j, bool ok, int tid) const {
    if (ok) {
      sm.a[tid] = src[3 * j];
      sm.b[tid] = src[3 * j + 1];
      sm.c[tid] = src[3 * j + 2];
    } else {
      sm.a[tid] = V{};
      sm.b[tid] = V{};
      sm.c[tid] = V{};
    }
  }
  __device__ __forceinline__ Src get(const Smem& sm, int jj) const {
    return Src{sm.a[jj], sm.b[jj], sm.c[jj]};
  }
  __device__ __forceinline__ void pair(const Src& s, const Tgt& t, R& ar, R& ai) const {
    const R dx = t.x - s.a.x, dy = t.y - s.a.y, dz = t.z - s.a.z;
    const R r2 = dx * dx + dy * dy + dz * dz;
    R rinv, tt, cs, sn;
    phase(r2, rinv, tt, cs, sn);
    const R dur = dx * s.b.y + dy * s.b.w + dz * s.c.y;
    const R dui = dx * s.b.z + dy * s.c.x + dz * s.c.z;
    const R rinv2 = rinv * rinv;
    const R fi = (tt * R(6.28318530717958647692)) * rinv2;  // (2 pi i t - 1) rinv^2
    const R inr = s.a.w - rinv2 * dur - fi * dui;
    const R ini = s.b.x - rinv2 * dui + fi * dur;
    const R er = cs * rinv, ei = sn * rinv;
    ar += er * inr - ei * ini;
    ai += er * ini + ei * inr;
  }
};

// Adjoint F: targets are source points j with (y~, s) and v~ = kappa v; sources are
// collocation records a = (x~, c~.re), b = c~.im with c~ = kappa conj(lam)/(4 pi):
//   w_j += e^{2 pi i t} rinv c~ [-s + (2 pi i t - 1)((x~_i - y~_j) . v~) rinv^2]
template <class R>
struct PolAF {
  using V = typename Vec4<R>::type;
  using Smem = typename PolG<R>::Smem;
  using Src = typename PolG<R>::Src;
  struct Tgt {
    R x, y, z, s, vx, vy, vz;
  };
  const V* __restrict__ tps;  // (y~, s) scaled positions
  const V* __restrict__ tv;   // v~
  const V* __restrict__ sa;
  const R* __restrict__ sb;

  __device__ __forceinline__ void load_target(int64_t i, bool ok, Tgt& t) const {
    if (ok) {
      const V p = tps[i], v = tv[i];
      t.x = p.x;
      t.y = p.y;
      t.z = p.z;
      t.s = p.w;
      t.vx = v.x;
      t.vy = v.y;
      t.vz = v.z;
    } else {
      t.x = t.y = t.z = t.s = t.vx = t.vy = t.vz = R(0);
    }
  }
  __device__ __forceinline__ void stage(Smem& sm, int64_t j, bool ok, int tid) const {
    if (ok) {
      sm.a[tid] = sa[j];
      sm.b[tid] = sb[j];
    } else {
      sm.a[tid] = V{};
      sm.b[tid] = R(0);
    }
  }
  __device__ __forceinline__ Src get(const Smem& sm, int jj) const { return Src{sm.a[jj], sm.b[jj]}; }
  __device__ __forceinline__ void pair(const Src& s, const Tgt& t, R& ar, R& ai) const {
    const R dx = s.a.x - t.x, dy = s.a.y - t.y, dz = s.a.z - t.z;  // x_i - y_j
    const R r2 = dx * dx + dy * dy + dz * dz;
    R rinv, tt, cs, sn;
    phase(r2, rinv, tt, cs, sn);
    const R dv = dx * t.vx + dy * t.vy + dz * t.vz;
    const R rinv2 = rinv * rinv;
    const R mr = -t.s - rinv2 * dv;
    const R mi = (tt * R(6.28318530717958647692)) * rinv2 * dv;
    const R er = cs * rinv, ei = sn * rinv;
    const R gr = er * s.a.w - ei * s.b, gi = er * s.b + ei * s.a.w;
    ar += gr * mr - gi * mi;
    ai += gr * mi + gi * mr;
  }
};

// Block-level interface over a per-target policy: kT independent targets per thread.
template <class R, class B>
struct PerTarget : B {
  using typename B::Src;
  using typename B::Smem;
  struct Tgts {
    typename B::Tgt t[kT];
  };
  struct Part {
    R ar[kT], ai[kT];
  };
  __device__ __forceinline__ void load_targets(int64_t i0, int64_t nt, Tgts& tg) const {
#pragma unroll
    for (int t = 0; t < kT; ++t) {
      const int64_t i = i0 + (int64_t)t * kBlock;
      B::load_target(i, i < nt, tg.t[t]);
    }
  }
  __device__ __forceinline__ void zero(Part& q) const {
#pragma unroll
    for (int t = 0; t < kT; ++t) q.ar[t] = q.ai[t] = R(0);
  }
  __device__ __forceinline__ void accumulate(const Src& s, const Tgts& tg, Part& q) const {
#pragma unroll
    for (int t = 0; t < kT; ++t) B::pair(s, tg.t[t], q.ar[t], q.ai[t]);
  }
  __device__ __forceinline__ void unpack(const Part& q, R* ar, R* ai) const {
#pragma unroll
    for (int t = 0; t < kT; ++t) {
      ar[t] = q.ar[t];
      ai[t] = q.ai[t];
    }
  }
};

// ----------------------------------------------------------------- packed FP32 policies
// Blackwell's paired FP32 instructions (two lanes' worth of add/mul/fma per issue slot)
// evaluate two targets per instruction.  Targets (t0, t2) and (t1, t3) form the packed
// pairs; source records are staged in shared memory already duplicated (and negated
// where the formula subtracts), so every packed operand is a single 64-bit load.

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// e^{2 pi i t} for a packed pair, plus rinv = 1/|d~| (0 at coincidence) and t.
__device__ __forceinline__ void phase2(float2 r2, float2& rinv, float2& t, float2& cs, float2& sn) {
  rinv.x = (r2.x > 0.0f) ? rsqrtf(r2.x) : 0.0f;
  rinv.y = (r2.y > 0.0f) ? rsqrtf(r2.y) : 0.0f;
  t = __fmul2_rn(r2, rinv);
  const float2 u = __fadd2_rn(t, f2(12582912.0f));       // t + 1.5*2^23
  const float2 w = __fadd2_rn(u, f2(-12582912.0f));      // round(t)
  const float2 f = __ffma2_rn(w, f2(-1.0f), t);          // t - round(t), exact
  const float2 a = __fmul2_rn(f, f2(6.28318530717958647692f));
  __sincosf(a.x, &sn.x, &cs.x);
  __sincosf(a.y, &sn.y, &cs.y);
}

struct Tgts2 {
  float2 x[kT / 2], y[kT / 2], z[kT / 2];  // packed pair p holds targets (p, p + kT/2)
};

__device__ __forceinline__ void load_targets2(const float4* __restrict__ tgt, int64_t i0, int64_t nt,
                                              Tgts2& tg) {
#pragma unroll
  for (int p = 0; p < kT / 2; ++p) {
    const int64_t ia = i0 + (int64_t)p * kBlock, ib = i0 + (int64_t)(p + kT / 2) * kBlock;
    const float4 a = ia < nt ? tgt[ia] : make_float4(0, 0, 0, 0);
    const float4 b = ib < nt ? tgt[ib] : make_float4(0, 0, 0, 0);
    tg.x[p] = make_float2(a.x, b.x);
    tg.y[p] = make_float2(a.y, b.y);
    tg.z[p] = make_float2(a.z, b.z);
  }
}

struct Part2 {
  float2 ar[kT / 2], ai[kT / 2];
};

__device__ __forceinline__ void zero2(Part2& q) {
#pragma unroll
  for (int p = 0; p < kT / 2; ++p) q.ar[p] = q.ai[p] = make_float2(0.0f, 0.0f);
}

__device__ __forceinline__ void unpack2(const Part2& q, float* ar, float* ai) {
#pragma unroll
  for (int p = 0; p < kT / 2; ++p) {
    ar[p] = q.ar[p].x;
    ai[p] = q.ai[p].x;
    ar[p + kT / 2] = q.ar[p].y;
    ai[p + kT / 2] = q.ai[p].y;
  }
}

// Volume sources (G class), y += e^{2 pi i t} rinv q~.
// Smem per source: (-x, -x, -y, -y) (-z, -z, q.re, q.re) (q.im, q.im, -q.im, -q.im)
struct PolG2 {
  struct Smem {
    float4 a[kBlock], b[kBlock], c[kBlock];
  };
  struct Src {
    float4 a, b, c;
  };
  using Tgts = Tgts2;
  using Part = Part2;
  const float4* __restrict__ tgt;
  const float4* __restrict__ sa;
  const float* __restrict__ sb;

  __device__ __forceinline__ void load_targets(int64_t i0, int64_t nt, Tgts& tg) const {
    load_targets2(tgt, i0, nt, tg);
  }
  __device__ __forceinline__ void stage(Smem& sm, int64_t j, bool ok, int tid) const {
    float4 r = ok ? sa[j] : make_float4(0, 0, 0, 0);
    const float qi = ok ? sb[j] : 0.0f;
    sm.a[tid] = make_float4(-r.x, -r.x, -r.y, -r.y);
    sm.b[tid] = make_float4(-r.z, -r.z, r.w, r.w);
    sm.c[tid] = make_float4(qi, qi, -qi, -qi);
  }
  __device__ __forceinline__ Src get(const Smem& sm, int jj) const { return Src{sm.a[jj], sm.b[jj], sm.c[jj]}; }
  __device__ __forceinline__ void zero(Part& q) const { zero2(q); }
  __device__ __forceinline__ void unpack(const Part& q, float* ar, float* ai) const { unpack2(q, ar, ai); }
  __device__ __forceinline__ void accumulate(const Src& s, const Tgts& tg, Part& q) const {
    const float2 nx = make_float2(s.a.x, s.a.y), ny = make_float2(s.a.z, s.a.w);
    const float2 nz = make_float2(s.b.x, s.b.y), qr = make_float2(s.b.z, s.b.w);
    const float2 qi = make_float2(s.c.x, s.c.y), nqi = make_float2(s.c.z, s.c.w);
#pragma unroll
    for (int p = 0; p < kT / 2; ++p) {
      const float2 dx = __fadd2_rn(tg.x[p], nx), dy = __fadd2_rn(tg.y[p], ny), dz = __fadd2_rn(tg.z[p], nz);
      float2 r2 = __fmul2_rn(dx, dx);
      r2 = __ffma2_rn(dy, dy, r2);
      r2 = __ffma2_rn(dz, dz, r2);
      float2 rinv, t, cs, sn;
      phase2(r2, rinv, t, cs, sn);
      const float2 er = __fmul2_rn(cs, rinv), ei = __fmul2_rn(sn, rinv);
      q.ar[p] = __ffma2_rn(er, qr, q.ar[p]);
      q.ar[p] = __ffma2_rn(ei, nqi, q.ar[p]);
      q.ai[p] = __ffma2_rn(er, qi, q.ai[p]);
      q.ai[p] = __ffma2_rn(ei, qr, q.ai[p]);
    }
  }
};

// Interface sources (K class), y += e^{2 pi i t}(2 pi i t - 1)(d~ . n) rinv^3 c~.
// With A = cos + kr sin and Q = kr cos - sin (kr = 2 pi t):
//   re += -g3 (A c.re + Q c.im),  im += g3 (Q c.re - A c.im),  g3 = rinv^3 (d~ . n).
// Smem per source: (-x,-x,-y,-y) (-z,-z,nx,nx) (ny,ny,nz,nz) (-c.re,-c.re,-c.im,-c.im) (c.re,c.re,0,0)
struct PolK2 {
  struct Smem {
    float4 a[kBlock], b[kBlock], c[kBlock], d[kBlock], e[kBlock];
  };
  struct Src {
    float4 a, b, c, d, e;
  };
  using Tgts = Tgts2;
  using Part = Part2;
  const float4* __restrict__ tgt;
  const float4* __restrict__ src;  // 2 records per source: (x, y, z, c.re) (c.im, nx, ny, nz)

  __device__ __forceinline__ void load_targets(int64_t i0, int64_t nt, Tgts& tg) const {
    load_targets2(tgt, i0, nt, tg);
  }
  __device__ __forceinline__ void stage(Smem& sm, int64_t j, bool ok, int tid) const {
    const float4 r = ok ? src[2 * j] : make_float4(0, 0, 0, 0);
    const float4 v = ok ? src[2 * j + 1] : make_float4(0, 0, 0, 0);
    sm.a[tid] = make_float4(-r.x, -r.x, -r.y, -r.y);
    sm.b[tid] = make_float4(-r.z, -r.z, v.y, v.y);
    sm.c[tid] = make_float4(v.z, v.z, v.w, v.w);
    sm.d[tid] = make_float4(-r.w, -r.w, -v.x, -v.x);
    sm.e[tid] = make_float4(r.w, r.w, 0.0f, 0.0f);
  }
  __device__ __forceinline__ Src get(const Smem& sm, int jj) const {
    return Src{sm.a[jj], sm.b[jj], sm.c[jj], sm.d[jj], sm.e[jj]};
  }
  __device__ __forceinline__ void zero(Part& q) const { zero2(q); }
  __device__ __forceinline__ void unpack(const Part& q, float* ar, float* ai) const { unpack2(q, ar, ai); }
  __device__ __forceinline__ void accumulate(const Src& s, const Tgts& tg, Part& q) const {
    const float2 nx = make_float2(s.a.x, s.a.y), ny = make_float2(s.a.z, s.a.w);
    const float2 nz = make_float2(s.b.x, s.b.y), ux = make_float2(s.b.z, s.b.w);
    const float2 uy = make_float2(s.c.x, s.c.y), uz = make_float2(s.c.z, s.c.w);
    const float2 ncr = make_float2(s.d.x, s.d.y), nci = make_float2(s.d.z, s.d.w);
    const float2 cr = make_float2(s.e.x, s.e.y);
#pragma unroll
    for (int p = 0; p < kT / 2; ++p) {
      const float2 dx = __fadd2_rn(tg.x[p], nx), dy = __fadd2_rn(tg.y[p], ny), dz = __fadd2_rn(tg.z[p], nz);
      float2 r2 = __fmul2_rn(dx, dx);
      r2 = __ffma2_rn(dy, dy, r2);
      r2 = __ffma2_rn(dz, dz, r2);
      float2 rinv, t, cs, sn;
      phase2(r2, rinv, t, cs, sn);
      float2 dn = __fmul2_rn(dx, ux);
      dn = __ffma2_rn(dy, uy, dn);
      dn = __ffma2_rn(dz, uz, dn);
      const float2 ri2 = __fmul2_rn(rinv, rinv);
      const float2 g3 = __fmul2_rn(__fmul2_rn(ri2, rinv), dn);
      const float2 kr = __fmul2_rn(t, f2(6.28318530717958647692f));
      const float2 A = __ffma2_rn(kr, sn, cs);                        // cos + kr sin
      const float2 Q = __ffma2_rn(kr, cs, __fmul2_rn(sn, f2(-1.0f)));  // kr cos - sin
      const float2 gA = __fmul2_rn(g3, A), gQ = __fmul2_rn(g3, Q);
      q.ar[p] = __ffma2_rn(gA, ncr, q.ar[p]);   // - gA c.re
      q.ar[p] = __ffma2_rn(gQ, nci, q.ar[p]);   // - gQ c.im
      q.ai[p] = __ffma2_rn(gQ, cr, q.ai[p]);    // + gQ c.re
      q.ai[p] = __ffma2_rn(gA, nci, q.ai[p]);   // - gA c.im
    }
  }
};

// ----------------------------------------------------------------- double-float policies
// Precision 48: FP64-class accuracy (about 2^-47 per operation) with every operation on the
// FP32 pipe, for the residuals of iterative refinement (B300's FP64 pipe runs at 1/64 of
// the FP32 rate).  Positions (kappa-scaled), charges and normals are double-float records;
// d = x~ - y~, r^2, 1/r (hardware estimate + Newton steps), the phase t = r (revolutions),
// f = t - round(t) and (cos, sin)(2 pi f) (Taylor series after an octant reduction,
// dfloat.h) are double-float; each pair's coefficient times its charge is accumulated by
// the packed double-float complex multiply-add.  The partial sum of a 128-source tile is
// converted to FP64 and added to the target's FP64 accumulator.

template <int NREC>
struct DfBase {
  struct Smem {
    float4 r[NREC][kBlock];
  };
  struct Src {
    float4 r[NREC];
  };
  struct Tgts {
    DTgt t[kT];
  };
  struct Part {
    float2 S[kT], C[kT];
  };
  const float4* __restrict__ tgt;  // 2 records per target
  const float4* __restrict__ src;  // NREC records per source

  // One pair evaluation is several hundred instructions: the driver does not unroll the
  // source loop, and accumulate() walks the targets with one copy of the evaluation by
  // rotating them (and their sums) through slot 0, so the loop body stays small enough for
  // the instruction cache while every register index is a compile-time constant.
  static constexpr int kSrcUnroll = 1;
  __device__ __forceinline__ static void rotate(Tgts& tg, Part& q) {
    const DTgt t0 = tg.t[0];
    const float2 s0 = q.S[0], c0 = q.C[0];
#pragma unroll
    for (int t = 0; t + 1 < kT; ++t) {
      tg.t[t] = tg.t[t + 1];
      q.S[t] = q.S[t + 1];
      q.C[t] = q.C[t + 1];
    }
    tg.t[kT - 1] = t0;
    q.S[kT - 1] = s0;
    q.C[kT - 1] = c0;
  }

  __device__ __forceinline__ void load_targets(int64_t i0, int64_t nt, Tgts& tg) const {
#pragma unroll
    for (int t = 0; t < kT; ++t) {
      const int64_t i = i0 + (int64_t)t * kBlock;
      float4 a = make_float4(0, 0, 0, 0), b = a;
      if (i < nt) {
        a = tgt[2 * i];
        b = tgt[2 * i + 1];
      }
      tg.t[t] = DTgt{dfs{a.x, b.x}, dfs{a.y, b.y}, dfs{a.z, b.z}};
    }
  }
  __device__ __forceinline__ void stage(Smem& sm, int64_t j, bool ok, int tid) const {
#pragma unroll
    for (int q = 0; q < NREC; ++q) sm.r[q][tid] = ok ? src[(int64_t)NREC * j + q] : make_float4(0, 0, 0, 0);
  }
  __device__ __forceinline__ Src get(const Smem& sm, int jj) const {
    Src s;
#pragma unroll
    for (int q = 0; q < NREC; ++q) s.r[q] = sm.r[q][jj];
    return s;
  }
  __device__ __forceinline__ void zero(Part& q) const {
#pragma unroll
    for (int t = 0; t < kT; ++t) q.S[t] = q.C[t] = make_float2(0.0f, 0.0f);
  }
  __device__ __forceinline__ void unpack(Part& q, double* ar, double* ai) const {
#pragma unroll
    for (int t = 0; t < kT; ++t) {
      df_renorm2(q.S[t], q.C[t]);
      const double2 v = df_value(q.S[t], q.C[t]);
      ar[t] = v.x;
      ai[t] = v.y;
    }
  }
};

// G: records (x.h, y.h, z.h, q.re.h) (x.l, y.l, z.l, q.re.l) (q.im.h, q.im.l, 0, 0);
//    y += e^{2 pi i t} rinv q~
struct PolGdf : DfBase<3> {
  __device__ __forceinline__ void accumulate(const Src& s, Tgts& tg, Part& q) const {
    const float4 qv = make_float4(s.r[0].w, s.r[2].x, s.r[1].w, s.r[2].y);
#pragma unroll 1
    for (int t = 0; t < kT; ++t) {
      df_cmac(q.S[0], q.C[0], df_coef_g(tg.t[0], s.r[0], s.r[1]), qv);
      rotate(tg, q);
    }
  }
};

// K: records (x.h, y.h, z.h, c.re.h) (x.l, y.l, z.l, c.re.l) (nx.h, ny.h, nz.h, c.im.h)
//    (nx.l, ny.l, nz.l, c.im.l);  y += e^{2 pi i t}(2 pi i t - 1)(d~ . n) rinv^3 c~
struct PolKdf : DfBase<4> {
  __device__ __forceinline__ void accumulate(const Src& s, Tgts& tg, Part& q) const {
    const float4 cv = make_float4(s.r[0].w, s.r[2].w, s.r[1].w, s.r[3].w);
    const dfs nx{s.r[2].x, s.r[3].x}, ny{s.r[2].y, s.r[3].y}, nz{s.r[2].z, s.r[3].z};
#pragma unroll 1
    for (int t = 0; t < kT; ++t) {
      df_cmac(q.S[0], q.C[0], df_coef_k(tg.t[0], s.r[0], s.r[1], nx, ny, nz), cv);
      rotate(tg, q);
    }
  }
};

// F: records (x.h, y.h, z.h, q.re.h) (x.l, y.l, z.l, q.re.l) (q.im.h, q.im.l, ux.re.h, ux.re.l)
//    (ux.im.h, ux.im.l, uy.re.h, uy.re.l) (uy.im.h, uy.im.l, uz.re.h, uz.re.l) (uz.im.h, uz.im.l, 0, 0);
//    y += e^{2 pi i t} rinv [q~ + (2 pi i t - 1)(d~ . u~) rinv^2]
struct PolFdf : DfBase<6> {
  __device__ __forceinline__ void accumulate(const Src& s, Tgts& tg, Part& q) const {
    const dfs qr{s.r[0].w, s.r[1].w}, qi{s.r[2].x, s.r[2].y};
    const dfs uxr{s.r[2].z, s.r[2].w}, uxi{s.r[3].x, s.r[3].y}, uyr{s.r[3].z, s.r[3].w};
    const dfs uyi{s.r[4].x, s.r[4].y}, uzr{s.r[4].z, s.r[4].w}, uzi{s.r[5].x, s.r[5].y};
#pragma unroll 1
    for (int t = 0; t < kT; ++t) {
      dfs dx, dy, dz, rinv, tt, cs, sn;
      df_geometry(tg.t[0], s.r[0], s.r[1], dx, dy, dz, rinv, tt, cs, sn);
      const dfs dur = dfs_add(dfs_add(dfs_mul(dx, uxr), dfs_mul(dy, uyr)), dfs_mul(dz, uzr));
      const dfs dui = dfs_add(dfs_add(dfs_mul(dx, uxi), dfs_mul(dy, uyi)), dfs_mul(dz, uzi));
      const dfs ri2 = dfs_sqr(rinv);
      const dfs fi = dfs_mul(dfs_mul(tt, dfc_two_pi()), ri2);  // 2 pi t rinv^2
      const dfs inr = dfs_sub(dfs_sub(qr, dfs_mul(ri2, dur)), dfs_mul(fi, dui));
      const dfs ini = dfs_add(dfs_sub(qi, dfs_mul(ri2, dui)), dfs_mul(fi, dur));
      df_cmac(q.S[0], q.C[0], df_c4(dfs_mul(cs, rinv), dfs_mul(sn, rinv)), df_c4(inr, ini));
      rotate(tg, q);
    }
  }
};

// source-loop unroll factor of the driver: the policy's kSrcUnroll where it sets one, else 4
template <class P, class = void>
struct SrcUnroll {
  static constexpr int value = 4;
};
template <class P>
struct SrcUnroll<P, std::void_t<decltype(P::kSrcUnroll)>> {
  static constexpr int value = P::kSrcUnroll;
};

// ----------------------------------------------------------------- persistent driver

struct StreamK {
  int64_t nt, ns;
  int64_t chunk;                 // sources per work item (a multiple of kBlock)
  int64_t ntile, nchunk, nitems;
  int64_t grid;
};

__host__ __device__ __forceinline__ int64_t sk_begin(const StreamK& s, int64_t b) {
  return (b * s.nitems) / s.grid;
}

template <class R, class P>
__global__ void __launch_bounds__(kBlock) nbody_kernel(P p, StreamK sk, double2* __restrict__ out,
                                                       double2* __restrict__ slots, int mode) {
  __shared__ typename P::Smem sm;
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  const int64_t k0 = sk_begin(sk, b), k1 = sk_begin(sk, b + 1);
  int64_t k = k0;
  while (k < k1) {
    const int64_t tile = k / sk.nchunk;
    const int64_t c0 = k - tile * sk.nchunk;
    const int64_t c1 = min(sk.nchunk, c0 + (k1 - k));
    typename P::Tgts tg;
    Acc<R> acc[kT];
    p.load_targets(tile * kTile + tid, sk.nt, tg);
#pragma unroll
    for (int t = 0; t < kT; ++t) acc[t].zero();
    const int64_t j_begin = c0 * sk.chunk;
    const int64_t j_end = min(sk.ns, c1 * sk.chunk);
    for (int64_t j0 = j_begin; j0 < j_end; j0 += kBlock) {
      const int64_t j = j0 + tid;
      p.stage(sm, j, j < j_end, tid);
      __syncthreads();
      typename P::Part part;
      p.zero(part);
#pragma unroll(SrcUnroll<P>::value)
      for (int jj = 0; jj < kBlock; ++jj) p.accumulate(p.get(sm, jj), tg, part);
      __syncthreads();
      R ar[kT], ai[kT];
      p.unpack(part, ar, ai);
#pragma unroll
      for (int t = 0; t < kT; ++t) acc[t].fold(ar[t], ai[t]);
    }
    const bool complete = (c0 == 0 && c1 == sk.nchunk);
    const int64_t slot = (k == k0) ? 2 * b : 2 * b + 1;
#pragma unroll
    for (int t = 0; t < kT; ++t) {
      const int64_t i = tile * kTile + (int64_t)t * kBlock + tid;
      if (i < sk.nt) {
        const double2 v = acc[t].value();
        if (complete) {
          if (mode) {
            const double2 o = out[i];
            out[i] = make_double2(o.x + v.x, o.y + v.y);
          } else {
            out[i] = v;
          }
        } else {
          slots[slot * kTile + (int64_t)t * kBlock + tid] = v;
        }
      }
    }
    k = tile * sk.nchunk + c1;
  }
}

__device__ __forceinline__ int64_t sk_block_of(const StreamK& s, int64_t k) {
  int64_t b = (k * s.grid) / s.nitems;
  while (b + 1 < s.grid && sk_begin(s, b + 1) <= k) ++b;
  while (b > 0 && sk_begin(s, b) > k) --b;
  return b;
}

// Adds the pieces of target tiles that span several blocks, in block order.
__global__ void __launch_bounds__(kTile) fixup_kernel(StreamK sk, const double2* __restrict__ slots,
                                                      double2* __restrict__ out, int mode) {
  const int64_t tile = blockIdx.x;
  const int64_t kf = tile * sk.nchunk, kl = kf + sk.nchunk - 1;
  const int64_t bs = sk_block_of(sk, kf), be = sk_block_of(sk, kl);
  if (bs == be) return;  // the whole tile was summed (and written) by one block
  const int idx = threadIdx.x;
  const int64_t i = tile * kTile + idx;
  if (i >= sk.nt) return;
  double sr = 0.0, si = 0.0;
  for (int64_t b = bs; b <= be; ++b) {
    if (sk_begin(sk, b) == sk_begin(sk, b + 1)) continue;  // empty range
    const int64_t slot = (b == bs && sk_begin(sk, b) != kf) ? 2 * b + 1 : 2 * b;
    const double2 v = slots[slot * kTile + idx];
    sr += v.x;
    si += v.y;
  }
  if (mode) {
    const double2 o = out[i];
    out[i] = make_double2(o.x + sr, o.y + si);
  } else {
    out[i] = make_double2(sr, si);
  }
}

// ----------------------------------------------------------------- launch planning

template <class R, class P>
static int resident_per_sm() {
  static int cached = 0;  // per instantiation; identical on every B300
  if (!cached) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, nbody_kernel<R, P>, kBlock, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    cached = per_sm;
  }
  return cached;
}

// Work decomposition of one class sum: target tiles x source chunks, a persistent grid.
// FP32 sums of class cls (0 G, 1 K, 2 F) take the autotuned chunk and blocks per SM when
// set; explicit chunk / bps arguments (> 0) override both (the autotuner's candidates).
template <class R, class P>
static StreamK plan_sk(const vsie_handle* h, int64_t nt, int64_t ns, int cls = -1, int chunk = 0, int bps = 0) {
  StreamK s;
  s.nt = nt;
  s.ns = ns;
  const bool tuned = sizeof(R) == 4 && cls >= 0;
  if (chunk <= 0) chunk = (tuned && h->tune.chunk[cls] > 0) ? h->tune.chunk[cls] : kChunk;
  if (bps <= 0) bps = (tuned && h->tune.bps[cls] > 0) ? h->tune.bps[cls] : resident_per_sm<R, P>();
  bps = std::min(bps, resident_per_sm<R, P>());
  s.chunk = chunk;
  s.ntile = (nt + kTile - 1) / kTile;
  s.nchunk = (ns + s.chunk - 1) / s.chunk;
  s.nitems = s.ntile * s.nchunk;
  int64_t C = (int64_t)bps * (h->num_sms > 0 ? h->num_sms : 148);
  if (h->tile_override > 0) C = h->tile_override;
  s.grid = std::max<int64_t>(1, std::min<int64_t>(C, s.nitems));
  return s;
}

static size_t slot_elems(const StreamK& s) { return (size_t)(2 * s.grid) * kTile; }

template <class R, class P>
static vsie_status run_nbody(const P& p, const StreamK& sk, double2* out, int mode, double2* slots,
                             cudaStream_t st, int* launches) {
  if (sk.nt == 0 || sk.ns == 0) return VSIE_OK;
  nbody_kernel<R, P><<<(unsigned)sk.grid, kBlock, 0, st>>>(p, sk, out, slots, mode);
  fixup_kernel<<<(unsigned)sk.ntile, kTile, 0, st>>>(sk, slots, out, mode);
  if (launches) *launches += 2;
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

// Slot scratch of the handle, grown on demand.
static vsie_status handle_slots(vsie_handle* h, size_t elems, double2** out) {
  if (h->split_elems < elems) {
    double2* p = nullptr;
    VSIE_TRY(dalloc_t(h, &p, elems));
    h->split = p;
    h->split_elems = elems;
  }
  *out = h->split;
  return VSIE_OK;
}

// ----------------------------------------------------------------- prescale kernels

// G: a = kappa (y, q.re), b = kappa q.im,  q = -s p/(4 pi)
__global__ void prescale_g_kernel(const double4_32a* __restrict__ ps, const int32_t* __restrict__ own,
                                  const double2* __restrict__ p, int64_t n, double kap, int prec,
                                  float4* __restrict__ a32, float* __restrict__ b32,
                                  double4_32a* __restrict__ a64, double* __restrict__ b64) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  const double2 pe = p[own[j]];
  const double sc = -kap * y.w / kFourPi;
  const double qr = sc * pe.x, qi = sc * pe.y;
  if (prec == 32) {
    a32[j] = make_float4((float)(kap * y.x), (float)(kap * y.y), (float)(kap * y.z), (float)qr);
    b32[j] = (float)qi;
  } else {
    a64[j] = make_double4_32a(kap * y.x, kap * y.y, kap * y.z, qr);
    b64[j] = qi;
  }
}

// K: a = (kappa y, c~.re), b = (c~.im, n), c~ = kappa^2 sigma p/(4 pi), v = sigma n
__global__ void prescale_k_kernel(const double4_32a* __restrict__ ps, const double4_32a* __restrict__ nrm,
                                  const int32_t* __restrict__ own, const double2* __restrict__ p, int64_t n,
                                  double kap, int prec, float4* __restrict__ a32,
                                  double4_32a* __restrict__ a64) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  const double4_32a nn = nrm[j];
  const double2 pe = p[own[j]];
  const double sc = kap * kap * nn.w / kFourPi;
  const double cr = sc * pe.x, ci = sc * pe.y;
  if (prec == 32) {
    a32[2 * j] = make_float4((float)(kap * y.x), (float)(kap * y.y), (float)(kap * y.z), (float)cr);
    a32[2 * j + 1] = make_float4((float)ci, (float)nn.x, (float)nn.y, (float)nn.z);
  } else {
    a64[2 * j] = make_double4_32a(kap * y.x, kap * y.y, kap * y.z, cr);
    a64[2 * j + 1] = make_double4_32a(ci, nn.x, nn.y, nn.z);
  }
}

// F: a = (kappa y, kappa q.re), b = (kappa q.im, kappa^2 u...), c = (...)
__global__ void prescale_f_kernel(const double4_32a* __restrict__ ps, const double4_32a* __restrict__ vv,
                                  const int32_t* __restrict__ own, const double2* __restrict__ p,
                                  int64_t n, double kap, int prec, float4* __restrict__ a32,
                                  double4_32a* __restrict__ a64) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  const double4_32a v = vv[j];
  const double2 pe = p[own[j]];
  const double sc = -kap * y.w / kFourPi, vs = kap * kap / kFourPi;
  const double qr = sc * pe.x, qi = sc * pe.y;
  const double uxr = vs * v.x * pe.x, uxi = vs * v.x * pe.y;
  const double uyr = vs * v.y * pe.x, uyi = vs * v.y * pe.y;
  const double uzr = vs * v.z * pe.x, uzi = vs * v.z * pe.y;
  if (prec == 32) {
    a32[3 * j] = make_float4((float)(kap * y.x), (float)(kap * y.y), (float)(kap * y.z), (float)qr);
    a32[3 * j + 1] = make_float4((float)qi, (float)uxr, (float)uxi, (float)uyr);
    a32[3 * j + 2] = make_float4((float)uyi, (float)uzr, (float)uzi, 0.0f);
  } else {
    a64[3 * j] = make_double4_32a(kap * y.x, kap * y.y, kap * y.z, qr);
    a64[3 * j + 1] = make_double4_32a(qi, uxr, uxi, uyr);
    a64[3 * j + 2] = make_double4_32a(uyi, uzr, uzi, 0.0);
  }
}

// double-float records of the precision-48 sums (layouts as in PolGdf / PolKdf / PolFdf)
__device__ __forceinline__ float2 split_hl(double v) {
  const float h = __double2float_rn(v);
  return make_float2(h, __double2float_rn(v - (double)h));
}

__global__ void prescale_g_df_kernel(const double4_32a* __restrict__ ps, const int32_t* __restrict__ own,
                                     const double2* __restrict__ p, int64_t n, double kap, float4* __restrict__ r) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  const double2 pe = p[own[j]];
  const double sc = -kap * y.w / kFourPi;
  const float2 x = split_hl(kap * y.x), yy = split_hl(kap * y.y), z = split_hl(kap * y.z);
  const float2 qr = split_hl(sc * pe.x), qi = split_hl(sc * pe.y);
  r[3 * j] = make_float4(x.x, yy.x, z.x, qr.x);
  r[3 * j + 1] = make_float4(x.y, yy.y, z.y, qr.y);
  r[3 * j + 2] = make_float4(qi.x, qi.y, 0.0f, 0.0f);
}

__global__ void prescale_k_df_kernel(const double4_32a* __restrict__ ps, const double4_32a* __restrict__ nrm,
                                     const int32_t* __restrict__ own, const double2* __restrict__ p, int64_t n,
                                     double kap, float4* __restrict__ r) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  const double4_32a nn = nrm[j];
  const double2 pe = p[own[j]];
  const double sc = kap * kap * nn.w / kFourPi;
  const float2 x = split_hl(kap * y.x), yy = split_hl(kap * y.y), z = split_hl(kap * y.z);
  const float2 cr = split_hl(sc * pe.x), ci = split_hl(sc * pe.y);
  const float2 nx = split_hl(nn.x), ny = split_hl(nn.y), nz = split_hl(nn.z);
  r[4 * j] = make_float4(x.x, yy.x, z.x, cr.x);
  r[4 * j + 1] = make_float4(x.y, yy.y, z.y, cr.y);
  r[4 * j + 2] = make_float4(nx.x, ny.x, nz.x, ci.x);
  r[4 * j + 3] = make_float4(nx.y, ny.y, nz.y, ci.y);
}

__global__ void prescale_f_df_kernel(const double4_32a* __restrict__ ps, const double4_32a* __restrict__ vv,
                                     const int32_t* __restrict__ own, const double2* __restrict__ p, int64_t n,
                                     double kap, float4* __restrict__ r) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  const double4_32a v = vv[j];
  const double2 pe = p[own[j]];
  const double sc = -kap * y.w / kFourPi, vs = kap * kap / kFourPi;
  const float2 x = split_hl(kap * y.x), yy = split_hl(kap * y.y), z = split_hl(kap * y.z);
  const float2 qr = split_hl(sc * pe.x), qi = split_hl(sc * pe.y);
  const float2 uxr = split_hl(vs * v.x * pe.x), uxi = split_hl(vs * v.x * pe.y);
  const float2 uyr = split_hl(vs * v.y * pe.x), uyi = split_hl(vs * v.y * pe.y);
  const float2 uzr = split_hl(vs * v.z * pe.x), uzi = split_hl(vs * v.z * pe.y);
  r[6 * j] = make_float4(x.x, yy.x, z.x, qr.x);
  r[6 * j + 1] = make_float4(x.y, yy.y, z.y, qr.y);
  r[6 * j + 2] = make_float4(qi.x, qi.y, uxr.x, uxr.y);
  r[6 * j + 3] = make_float4(uxi.x, uxi.y, uyr.x, uyr.y);
  r[6 * j + 4] = make_float4(uyi.x, uyi.y, uzr.x, uzr.y);
  r[6 * j + 5] = make_float4(uzi.x, uzi.y, 0.0f, 0.0f);
}

// collocation records for the adjoint: c~ = kappa conj(lam)/(4 pi) at kappa x
__global__ void prescale_colloc_kernel(const double4_32a* __restrict__ tgt, const double2* __restrict__ lam,
                                       int64_t n, double kap, int prec, float4* __restrict__ a32,
                                       float* __restrict__ b32, double4_32a* __restrict__ a64,
                                       double* __restrict__ b64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4_32a x = tgt[i];
  const double cr = kap * lam[i].x / kFourPi, ci = -kap * lam[i].y / kFourPi;
  if (prec == 32) {
    a32[i] = make_float4((float)(kap * x.x), (float)(kap * x.y), (float)(kap * x.z), (float)cr);
    b32[i] = (float)ci;
  } else {
    a64[i] = make_double4_32a(kap * x.x, kap * x.y, kap * x.z, cr);
    b64[i] = ci;
  }
}

// static per-point target records for the adjoint: (kappa y, s) and (kappa v, 0)
__global__ void point_records_kernel(const double4_32a* __restrict__ ps, const double4_32a* __restrict__ vv,
                                     int64_t n, double kap, float4* __restrict__ p32,
                                     float4* __restrict__ v32, double4_32a* __restrict__ p64,
                                     double4_32a* __restrict__ v64) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  p32[j] = make_float4((float)(kap * y.x), (float)(kap * y.y), (float)(kap * y.z), (float)y.w);
  p64[j] = make_double4_32a(kap * y.x, kap * y.y, kap * y.z, y.w);
  if (vv) {
    const double4_32a v = vv[j];
    v32[j] = make_float4((float)(kap * v.x), (float)(kap * v.y), (float)(kap * v.z), 0.0f);
    v64[j] = make_double4_32a(kap * v.x, kap * v.y, kap * v.z, 0.0);
  }
}

// x_e = conj(sum_{j in e} scale_j w_j), scale_j = -s_j for the G class (w = a_j), 1 otherwise
__global__ void gather_adjoint_kernel(const double2* __restrict__ w, const double4_32a* __restrict__ ps,
                                      int use_s, const int32_t* __restrict__ first,
                                      const int32_t* __restrict__ elem, int64_t n_elem,
                                      double2* __restrict__ x) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  double sr = 0.0, si = 0.0;
  for (int32_t j = first[e]; j < first[e + 1]; ++j) {
    const double sc = use_s ? -ps[j].w : 1.0;
    sr += sc * w[j].x;
    si += sc * w[j].y;
  }
  x[elem[e]] = make_double2(sr, -si);
}

static inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

// ----------------------------------------------------------------- forward apply

vsie_status far_prescale(vsie_handle* h, const double2* x, int precision, cudaStream_t st,
                         int* launches) {
  const double kap = h->k0 / kTwoPi;
  Sources& G = h->G;
  Sources& F = h->F;
  Sources& K = h->K;
  if (precision == 48) {
    if (G.n) prescale_g_df_kernel<<<nblk(G.n), 256, 0, st>>>(G.pos_s, G.owner, x, G.n, kap, G.rdf);
    if (K.n) prescale_k_df_kernel<<<nblk(K.n), 256, 0, st>>>(K.pos_s, K.aux, K.owner, x, K.n, kap, K.rdf);
    if (F.n) prescale_f_df_kernel<<<nblk(F.n), 256, 0, st>>>(F.pos_s, F.vvec, F.owner, x, F.n, kap, F.rdf);
    if (launches) *launches += (G.n > 0) + (K.n > 0) + (F.n > 0);
    VSIE_CUDA(cudaGetLastError());
    return VSIE_OK;
  }
  if (G.n) {
    prescale_g_kernel<<<nblk(G.n), 256, 0, st>>>(G.pos_s, G.owner, x, G.n, kap, precision, G.r32a,
                                                 G.r32b, G.r64a, G.r64b);
    if (launches) ++*launches;
  }
  if (K.n) {
    prescale_k_kernel<<<nblk(K.n), 256, 0, st>>>(K.pos_s, K.aux, K.owner, x, K.n, kap, precision,
                                                 K.r32a, K.r64a);
    if (launches) ++*launches;
  }
  if (F.n) {
    prescale_f_kernel<<<nblk(F.n), 256, 0, st>>>(F.pos_s, F.vvec, F.owner, x, F.n, kap, precision,
                                                 F.r32a, F.r64a);
    if (launches) ++*launches;
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

// Plans of the three forward sums (stored/added in the order G, K, F).
struct ForwardPlans {
  StreamK g, k, f;
  size_t slots;
};

static ForwardPlans forward_plans(const vsie_handle* h, int precision) {
  ForwardPlans P;
  const int64_t n = h->n;
  if (precision == 48) {
    P.g = plan_sk<double, PolGdf>(h, n, h->G.n);
    P.k = plan_sk<double, PolKdf>(h, n, h->K.n);
    P.f = plan_sk<double, PolFdf>(h, n, h->F.n);
  } else if (precision == 32) {
    P.g = plan_sk<float, PolG2>(h, n, h->G.n, 0);
    P.k = plan_sk<float, PolK2>(h, n, h->K.n, 1);
    P.f = plan_sk<float, PerTarget<float, PolF<float>>>(h, n, h->F.n, 2);
  } else {
    P.g = plan_sk<double, PerTarget<double, PolG<double>>>(h, n, h->G.n);
    P.k = plan_sk<double, PerTarget<double, PolK<double>>>(h, n, h->K.n);
    P.f = plan_sk<double, PerTarget<double, PolF<double>>>(h, n, h->F.n);
  }
  P.slots = std::max(slot_elems(P.g), std::max(slot_elems(P.k), slot_elems(P.f)));
  return P;
}

template <class R>
struct PolicySet {
  using G = PerTarget<R, PolG<R>>;
  using K = PerTarget<R, PolK<R>>;
  using F = PerTarget<R, PolF<R>>;
};
template <>
struct PolicySet<float> {
  using G = PolG2;
  using K = PolK2;
  using F = PerTarget<float, PolF<float>>;
};

template <class R>
static typename PolicySet<R>::G make_g(const vsie_handle* h);
template <>
PolG2 make_g<float>(const vsie_handle* h) {
  return PolG2{h->tgt32, h->G.r32a, h->G.r32b};
}
template <>
PerTarget<double, PolG<double>> make_g<double>(const vsie_handle* h) {
  PerTarget<double, PolG<double>> p;
  p.tgt = h->tgt64;
  p.tscale = h->k0 / kTwoPi;
  p.sa = h->G.r64a;
  p.sb = h->G.r64b;
  return p;
}
template <class R>
static typename PolicySet<R>::K make_k(const vsie_handle* h);
template <>
PolK2 make_k<float>(const vsie_handle* h) {
  return PolK2{h->tgt32, h->K.r32a};
}
template <>
PerTarget<double, PolK<double>> make_k<double>(const vsie_handle* h) {
  PerTarget<double, PolK<double>> p;
  p.tgt = h->tgt64;
  p.tscale = h->k0 / kTwoPi;
  p.src = h->K.r64a;
  return p;
}
template <class R>
static PerTarget<R, PolF<R>> make_f(const vsie_handle* h) {
  PerTarget<R, PolF<R>> p;
  using V = typename Vec4<R>::type;
  const bool fp32 = sizeof(R) == 4;
  p.tgt = reinterpret_cast<const V*>(fp32 ? (const void*)h->tgt32 : (const void*)h->tgt64);
  p.tscale = fp32 ? R(1) : (R)(h->k0 / kTwoPi);
  p.src = reinterpret_cast<const V*>(fp32 ? (const void*)h->F.r32a : (const void*)h->F.r64a);
  return p;
}

template <class R>
static vsie_status forward_sums(vsie_handle* h, double2* y, const ForwardPlans& P, double2* slots,
                                cudaStream_t st, int phase_mask, int* launches) {
  using PS = PolicySet<R>;
  int mode = 0;
  if (h->G.n) {
    if (phase_mask & 1) VSIE_TRY((run_nbody<R, typename PS::G>(make_g<R>(h), P.g, y, mode, slots, st, launches)));
    mode = 1;
  }
  if (h->K.n) {
    if (phase_mask & 2) VSIE_TRY((run_nbody<R, typename PS::K>(make_k<R>(h), P.k, y, mode, slots, st, launches)));
    mode = 1;
  }
  if (h->F.n) {
    if (phase_mask & 4) VSIE_TRY((run_nbody<R, typename PS::F>(make_f<R>(h), P.f, y, mode, slots, st, launches)));
    mode = 1;
  }
  if (!mode && (phase_mask & 1)) VSIE_CUDA(cudaMemsetAsync(y, 0, sizeof(double2) * h->n, st));
  return VSIE_OK;
}

static vsie_status forward_sums_df(vsie_handle* h, double2* y, const ForwardPlans& P, double2* slots,
                                   cudaStream_t st, int phase_mask, int* launches) {
  int mode = 0;
  if (h->G.n) {
    if (phase_mask & 1)
      VSIE_TRY((run_nbody<double, PolGdf>(PolGdf{{h->tgtdf, h->G.rdf}}, P.g, y, mode, slots, st, launches)));
    mode = 1;
  }
  if (h->K.n) {
    if (phase_mask & 2)
      VSIE_TRY((run_nbody<double, PolKdf>(PolKdf{{h->tgtdf, h->K.rdf}}, P.k, y, mode, slots, st, launches)));
    mode = 1;
  }
  if (h->F.n) {
    if (phase_mask & 4)
      VSIE_TRY((run_nbody<double, PolFdf>(PolFdf{{h->tgtdf, h->F.rdf}}, P.f, y, mode, slots, st, launches)));
    mode = 1;
  }
  if (!mode && (phase_mask & 1)) VSIE_CUDA(cudaMemsetAsync(y, 0, sizeof(double2) * h->n, st));
  return VSIE_OK;
}

// y[i] += z[i], i < n (the concurrent K sum's output joined into y).
__global__ void add_into_kernel(double2* __restrict__ y, const double2* __restrict__ z, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    const double2 a = y[i], b = z[i];
    y[i] = make_double2(a.x + b.x, a.y + b.y);
  }
}

// The FP32 volume (G) and interface (K) sums over the first nt targets at the same time,
// with gbps and kbps resident blocks per SM: G stores into y on st while K stores into
// h->gk_y on the handle's second stream, forked from st and joined back into it with events
// (so the pair is captured into a CUDA graph like any other launch sequence); the
// heterogeneous-volume sum (F, with_f) follows G on st, and y += gk_y after the join.  The G tiles
// are bound by the MUFU pipe and the K tiles by the FMA pipe, so blocks of both on one SM
// keep both pipes busy.  slots: G's and F's split slots; K's are h->gk_split.
static vsie_status gk_concurrent(vsie_handle* h, const PolG2& pg, const PolK2& pk, int64_t nt, int gbps, int kbps,
                                 bool with_f, double2* y, double2* slots, cudaStream_t st, int* launches) {
  const StreamK g = plan_sk<float, PolG2>(h, nt, h->G.n, 0, 0, gbps);
  const StreamK k = plan_sk<float, PolK2>(h, nt, h->K.n, 1, 0, kbps);
  VSIE_CUDA(cudaEventRecord(h->gk_fork, st));
  VSIE_CUDA(cudaStreamWaitEvent(h->gk_stream, h->gk_fork, 0));
  VSIE_TRY((run_nbody<float, PolG2>(pg, g, y, 0, slots, st, launches)));
  VSIE_TRY((run_nbody<float, PolK2>(pk, k, h->gk_y, 0, h->gk_split, h->gk_stream, launches)));
  VSIE_CUDA(cudaEventRecord(h->gk_join, h->gk_stream));
  if (with_f && h->F.n) {
    const StreamK f = plan_sk<float, PerTarget<float, PolF<float>>>(h, nt, h->F.n, 2);
    VSIE_TRY((run_nbody<float, PerTarget<float, PolF<float>>>(make_f<float>(h), f, y, 1, slots, st, launches)));
  }
  VSIE_CUDA(cudaStreamWaitEvent(st, h->gk_join, 0));
  add_into_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(y, h->gk_y, nt);
  VSIE_CUDA(cudaGetLastError());
  if (launches) *launches += 1;
  return VSIE_OK;
}

// Slots the concurrent sums need on the main stream (G's with gbps blocks per SM, F's).
static size_t gk_main_slots(const vsie_handle* h, int64_t nt, int gbps) {
  size_t e = slot_elems(plan_sk<float, PolG2>(h, nt, h->G.n, 0, 0, gbps));
  if (h->F.n) e = std::max(e, slot_elems(plan_sk<float, PerTarget<float, PolF<float>>>(h, nt, h->F.n, 2)));
  return e;
}

// True when the autotuner chose the concurrent sums and their buffers are in place.
static bool gk_ready(const vsie_handle* h) {
  return h->tune.gk_bps[0] > 0 && h->tune.gk_bps[1] > 0 && h->G.n && h->K.n && h->gk_stream && h->gk_y &&
         h->gk_y_n >= h->n &&
         h->gk_split_elems >= slot_elems(plan_sk<float, PolK2>(h, h->n, h->K.n, 1, 0, h->tune.gk_bps[1]));
}

static vsie_status forward(vsie_handle* h, double2* y, int precision, double2* slots_given,
                           cudaStream_t st, int phase_mask, int* launches) {
  if (precision == 32 && phase_mask == 7 && !slots_given && gk_ready(h)) {
    double2* slots = nullptr;
    VSIE_TRY(handle_slots(h, gk_main_slots(h, h->n, h->tune.gk_bps[0]), &slots));
    return gk_concurrent(h, make_g<float>(h), make_k<float>(h), h->n, h->tune.gk_bps[0], h->tune.gk_bps[1], true,
                         y, slots, st, launches);
  }
  const ForwardPlans P = forward_plans(h, precision);
  double2* slots = slots_given;
  if (!slots) VSIE_TRY(handle_slots(h, P.slots, &slots));
  if (precision == 32) return forward_sums<float>(h, y, P, slots, st, phase_mask, launches);
  if (precision == 48) return forward_sums_df(h, y, P, slots, st, phase_mask, launches);
  return forward_sums<double>(h, y, P, slots, st, phase_mask, launches);
}

// The three class sums at m arbitrary points (the records written by far_prescale): the
// policies of the collocation sums with their target arrays replaced.
vsie_status far_sums_at(vsie_handle* h, const double2* x, const double4_32a* t64, const float4* t32,
                        const float4* tdf, int64_t m, double2* y, int precision, cudaStream_t st) {
  VSIE_TRY(far_prescale(h, x, precision, st, nullptr));
  StreamK g, k, f;
  if (precision == 48) {
    g = plan_sk<double, PolGdf>(h, m, h->G.n);
    k = plan_sk<double, PolKdf>(h, m, h->K.n);
    f = plan_sk<double, PolFdf>(h, m, h->F.n);
  } else if (precision == 32) {
    g = plan_sk<float, PolG2>(h, m, h->G.n, 0);
    k = plan_sk<float, PolK2>(h, m, h->K.n, 1);
    f = plan_sk<float, PerTarget<float, PolF<float>>>(h, m, h->F.n, 2);
  } else {
    g = plan_sk<double, PerTarget<double, PolG<double>>>(h, m, h->G.n);
    k = plan_sk<double, PerTarget<double, PolK<double>>>(h, m, h->K.n);
    f = plan_sk<double, PerTarget<double, PolF<double>>>(h, m, h->F.n);
  }
  double2* slots = nullptr;
  VSIE_TRY(handle_slots(h, std::max(slot_elems(g), std::max(slot_elems(k), slot_elems(f))), &slots));
  VSIE_CUDA(cudaMemsetAsync(y, 0, sizeof(double2) * m, st));
  const int mode = 1;  // every class adds into the zeroed y
  if (precision == 48) {
    if (h->G.n) VSIE_TRY((run_nbody<double, PolGdf>(PolGdf{{tdf, h->G.rdf}}, g, y, mode, slots, st, nullptr)));
    if (h->K.n) VSIE_TRY((run_nbody<double, PolKdf>(PolKdf{{tdf, h->K.rdf}}, k, y, mode, slots, st, nullptr)));
    if (h->F.n) VSIE_TRY((run_nbody<double, PolFdf>(PolFdf{{tdf, h->F.rdf}}, f, y, mode, slots, st, nullptr)));
  } else if (precision == 32) {
    PerTarget<float, PolF<float>> pf = make_f<float>(h);
    pf.tgt = t32;
    if (h->G.n) VSIE_TRY((run_nbody<float, PolG2>(PolG2{t32, h->G.r32a, h->G.r32b}, g, y, mode, slots, st, nullptr)));
    if (h->K.n) VSIE_TRY((run_nbody<float, PolK2>(PolK2{t32, h->K.r32a}, k, y, mode, slots, st, nullptr)));
    if (h->F.n) VSIE_TRY((run_nbody<float, PerTarget<float, PolF<float>>>(pf, f, y, mode, slots, st, nullptr)));
  } else {
    PerTarget<double, PolG<double>> pg = make_g<double>(h);
    PerTarget<double, PolK<double>> pk = make_k<double>(h);
    PerTarget<double, PolF<double>> pf = make_f<double>(h);
    pg.tgt = pk.tgt = pf.tgt = t64;
    if (h->G.n) VSIE_TRY((run_nbody<double, PerTarget<double, PolG<double>>>(pg, g, y, mode, slots, st, nullptr)));
    if (h->K.n) VSIE_TRY((run_nbody<double, PerTarget<double, PolK<double>>>(pk, k, y, mode, slots, st, nullptr)));
    if (h->F.n) VSIE_TRY((run_nbody<double, PerTarget<double, PolF<double>>>(pf, f, y, mode, slots, st, nullptr)));
  }
  return VSIE_OK;
}

// phase bits: 1 the volume (G) sum, 2 the interface (K) sum, 4 the heterogeneous-volume (F)
// sum; each phase stores into y if it is the first class present, else adds.
vsie_status far_sum_g(vsie_handle* h, double2* y, int precision, cudaStream_t st, int* launches) {
  return forward(h, y, precision, nullptr, st, 1, launches);
}
vsie_status far_sum_f(vsie_handle* h, double2* y, int precision, cudaStream_t st, int* launches) {
  return forward(h, y, precision, nullptr, st, 6, launches);
}

vsie_status far_apply(vsie_handle* h, const double2* x, double2* y, int precision,
                      cudaStream_t st) {
  VSIE_TRY(far_prescale(h, x, precision, st, nullptr));
  return forward(h, y, precision, nullptr, st, 7, nullptr);
}

// ----------------------------------------------------------------- autotuning

// Times the FP32 sum of class cls (records already prescaled) on the first nt targets with
// a candidate work shape (sources per item, blocks per SM): the best of `reps` runs.
template <class P>
static vsie_status time_class(vsie_handle* h, const P& p, int64_t nt, int64_t ns, int chunk, int bps,
                              double2* out, cudaStream_t st, int reps, float* best_ms) {
  const StreamK sk = plan_sk<float, P>(h, nt, ns, -1, chunk, bps);
  double2* slots = nullptr;
  VSIE_TRY(handle_slots(h, slot_elems(sk), &slots));
  cudaEvent_t e0, e1;
  VSIE_CUDA(cudaEventCreate(&e0));
  VSIE_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  vsie_status s = VSIE_OK;
  for (int r = 0; r <= reps && s == VSIE_OK; ++r) {  // the first run warms up
    cudaEventRecord(e0, st);
    s = run_nbody<float, P>(p, sk, out, 0, slots, st, nullptr);
    cudaEventRecord(e1, st);
    if (s == VSIE_OK && cudaEventSynchronize(e1) == cudaSuccess && r > 0) {
      float ms = 0.0f;
      cudaEventElapsedTime(&ms, e0, e1);
      best = std::min(best, ms);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *best_ms = best;
  return s;
}

// Picks sources per work item and blocks per SM of each FP32 class sum by timing the
// candidates on a sample of the targets (sized to about 4e10 pair evaluations per run, so
// a candidate costs tens of milliseconds at any mesh size), with x a random vector.
vsie_status far_autotune(vsie_handle* h, const double2* x, double2* scratch, cudaStream_t st, int cand_out[3][2],
                         double ms_out[3][2], int* candidates) {
  VSIE_TRY(far_prescale(h, x, 32, st, nullptr));
  static const int chunks[] = {512, 1024, 2048, 4096};
  for (int cls = 0; cls < 3; ++cls) {
    const int64_t ns = cls == 0 ? h->G.n : cls == 1 ? h->K.n : h->F.n;
    cand_out[cls][0] = cand_out[cls][1] = 0;
    ms_out[cls][0] = ms_out[cls][1] = 0.0;
    if (!ns || !h->n) continue;
    const int64_t want = std::max<int64_t>((int64_t)kTile * 2 * std::max(h->num_sms, 1),
                                           (int64_t)(4e10 / (double)ns));
    const int64_t nt = std::min<int64_t>(h->n, want);
    const int maxb = cls == 0 ? resident_per_sm<float, PolG2>()
                              : cls == 1 ? resident_per_sm<float, PolK2>()
                                         : resident_per_sm<float, PerTarget<float, PolF<float>>>();
    int bps_c[3] = {maxb, std::max(1, maxb / 2), std::max(1, (3 * maxb) / 4)};
    float best = 1e30f, dflt = 0.0f;
    int best_chunk = kChunk, best_bps = maxb;
    for (int c : chunks)
      for (int bi = 0; bi < 3; ++bi) {
        if (bi > 0 && bps_c[bi] == bps_c[0]) continue;
        float ms = 0.0f;
        if (cls == 0)
          VSIE_TRY(time_class(h, make_g<float>(h), nt, ns, c, bps_c[bi], scratch, st, 2, &ms));
        else if (cls == 1)
          VSIE_TRY(time_class(h, make_k<float>(h), nt, ns, c, bps_c[bi], scratch, st, 2, &ms));
        else
          VSIE_TRY(time_class(h, make_f<float>(h), nt, ns, c, bps_c[bi], scratch, st, 2, &ms));
        ++*candidates;
        if (c == kChunk && bi == 0) dflt = ms;
        if (ms < best) {
          best = ms;
          best_chunk = c;
          best_bps = bps_c[bi];
        }
      }
    h->tune.chunk[cls] = best_chunk;
    h->tune.bps[cls] = best_bps;
    cand_out[cls][0] = best_chunk;
    cand_out[cls][1] = best_bps;
    ms_out[cls][0] = best;
    ms_out[cls][1] = dflt;
  }
  return VSIE_OK;
}

// The second stream, the fork/join events, K's output (n values) and K's split slots of the
// concurrent G and K sums, sized for any split, and G's slots: created once per handle, here
// only, so that an apply never allocates for them.
static vsie_status gk_resources(vsie_handle* h) {
  const int maxg = resident_per_sm<float, PolG2>(), maxk = resident_per_sm<float, PolK2>();
  if (!h->gk_stream) VSIE_CUDA(cudaStreamCreateWithFlags(&h->gk_stream, cudaStreamNonBlocking));
  if (!h->gk_fork) VSIE_CUDA(cudaEventCreateWithFlags(&h->gk_fork, cudaEventDisableTiming));
  if (!h->gk_join) VSIE_CUDA(cudaEventCreateWithFlags(&h->gk_join, cudaEventDisableTiming));
  if (h->gk_y_n < h->n) {
    VSIE_TRY(dalloc_t(h, &h->gk_y, (size_t)h->n));
    h->gk_y_n = h->n;
  }
  const size_t kslots = slot_elems(plan_sk<float, PolK2>(h, h->n, h->K.n, 1, 0, maxk));
  if (h->gk_split_elems < kslots) {
    VSIE_TRY(dalloc_t(h, &h->gk_split, kslots));
    h->gk_split_elems = kslots;
  }
  double2* slots = nullptr;
  return handle_slots(h, std::max(gk_main_slots(h, h->n, maxg), forward_plans(h, 32).slots), &slots);
}

int far_gk_extra_launches(const vsie_handle* h, int precision) {
  return precision == 32 && gk_ready(h) ? 1 : 0;
}

vsie_status far_set_gk(vsie_handle* h, int gbps, int kbps) {
  h->tune.gk_bps[0] = h->tune.gk_bps[1] = 0;
  if (gbps <= 0 || kbps <= 0 || !h->G.n || !h->K.n) return VSIE_OK;
  VSIE_TRY(gk_resources(h));
  h->tune.gk_bps[0] = std::min(gbps, resident_per_sm<float, PolG2>());
  h->tune.gk_bps[1] = std::min(kbps, resident_per_sm<float, PolK2>());
  return VSIE_OK;
}

// Times the FP32 G and K sums (records prescaled by far_autotune) one after the other with
// their tuned shapes, and concurrently for every split of the resident blocks per SM
// between them; keeps the concurrent split if it is at least 2% faster.  The second stream,
// the events, K's output (n values) and K's slots are created here, the only place they
// are allocated, so that an apply never allocates for them.
vsie_status far_autotune_gk(vsie_handle* h, const double2* x, double2* scratch, cudaStream_t st, int out_bps[2],
                            double out_ms[2], int* candidates) {
  out_bps[0] = out_bps[1] = 0;
  out_ms[0] = out_ms[1] = 0.0;
  h->tune.gk_bps[0] = h->tune.gk_bps[1] = 0;
  if (!h->G.n || !h->K.n || !h->n) return VSIE_OK;
  VSIE_TRY(far_prescale(h, x, 32, st, nullptr));
  const int maxg = resident_per_sm<float, PolG2>(), maxk = resident_per_sm<float, PolK2>();
  if (maxg < 2 || maxk < 2) return VSIE_OK;
  VSIE_TRY(gk_resources(h));
  const int64_t want = std::max<int64_t>((int64_t)kTile * 2 * std::max(h->num_sms, 1),
                                         (int64_t)(4e10 / (double)(h->G.n + h->K.n)));
  const int64_t nt = std::min<int64_t>(h->n, want);
  double2* slots = h->split;
  const PolG2 pg = make_g<float>(h);
  const PolK2 pk = make_k<float>(h);
  cudaEvent_t e0, e1;
  VSIE_CUDA(cudaEventCreate(&e0));
  VSIE_CUDA(cudaEventCreate(&e1));
  // gbps == 0: sequential (G then K, tuned shapes)
  auto time_one = [&](int gbps, int kbps, float* best_ms) -> vsie_status {
    float best = 1e30f;
    for (int r = 0; r <= 2; ++r) {
      VSIE_CUDA(cudaEventRecord(e0, st));
      if (gbps == 0) {
        VSIE_TRY((run_nbody<float, PolG2>(pg, plan_sk<float, PolG2>(h, nt, h->G.n, 0), scratch, 0, slots, st,
                                          nullptr)));
        VSIE_TRY((run_nbody<float, PolK2>(pk, plan_sk<float, PolK2>(h, nt, h->K.n, 1), scratch, 1, slots, st,
                                          nullptr)));
      } else {
        VSIE_TRY(gk_concurrent(h, pg, pk, nt, gbps, kbps, false, scratch, slots, st, nullptr));
      }
      VSIE_CUDA(cudaEventRecord(e1, st));
      VSIE_CUDA(cudaEventSynchronize(e1));
      float ms = 0.0f;
      VSIE_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (r > 0) best = std::min(best, ms);
    }
    *best_ms = best;
    return VSIE_OK;
  };
  float seq = 0.0f, best = 1e30f;
  int bg = 0, bk = 0;
  vsie_status s = time_one(0, 0, &seq);
  ++*candidates;
  for (int gb = 1; gb < maxg && s == VSIE_OK; ++gb) {
    const int kb = std::max(1, (maxk * (maxg - gb)) / maxg);
    float ms = 0.0f;
    s = time_one(gb, kb, &ms);
    ++*candidates;
    if (s == VSIE_OK && ms < best) {
      best = ms;
      bg = gb;
      bk = kb;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  VSIE_TRY(s);
  out_ms[1] = seq;
  if (bg > 0 && best < 0.98f * seq) {
    h->tune.gk_bps[0] = out_bps[0] = bg;
    h->tune.gk_bps[1] = out_bps[1] = bk;
    out_ms[0] = best;
  } else {
    out_ms[0] = seq;
  }
  return VSIE_OK;
}

vsie_status far_sum_f_only(vsie_handle* h, const double2* x, double2* y, int precision, cudaStream_t st) {
  if (!h->F.n) return VSIE_OK;
  VSIE_TRY(far_prescale(h, x, precision, st, nullptr));
  return forward(h, y, precision, nullptr, st, 4, nullptr);
}

size_t far_split_elems(const vsie_handle* h, int precision) { return forward_plans(h, precision).slots; }

vsie_status far_sums_into(vsie_handle* h, double2* y, int precision, double2* scratch,
                          cudaStream_t st) {
  return forward(h, y, precision, scratch, st, 7, nullptr);
}

// ----------------------------------------------------------------- adjoint apply

// Per-point target records and collocation-record buffers of the adjoint sums (built on
// the first adjoint call).
static vsie_status adjoint_buffers(vsie_handle* h, cudaStream_t st) {
  const int64_t n = h->n;
  const double kap = h->k0 / kTwoPi;
  AdjRecords* A = &h->adj;
  Sources* cls[3] = {&h->G, &h->K, &h->F};
  if (A->w) return VSIE_OK;
  int64_t maxn = 1;
  for (Sources* S : cls) maxn = std::max<int64_t>(maxn, S->n);
  for (Sources* S : cls) {
    VSIE_TRY(dalloc_t(h, &S->adj_p32, (size_t)S->n));
    VSIE_TRY(dalloc_t(h, &S->adj_v32, (size_t)S->n));
    VSIE_TRY(dalloc_t(h, &S->adj_p64, (size_t)S->n));
    VSIE_TRY(dalloc_t(h, &S->adj_v64, (size_t)S->n));
    if (S->n)
      point_records_kernel<<<nblk(S->n), 256, 0, st>>>(S->pos_s, S->vvec, S->n, kap, S->adj_p32, S->adj_v32,
                                                        S->adj_p64, S->adj_v64);
  }
  VSIE_TRY(dalloc_t(h, &A->c_a32, (size_t)n));
  VSIE_TRY(dalloc_t(h, &A->c_b32, (size_t)n));
  VSIE_TRY(dalloc_t(h, &A->c_a64, (size_t)n));
  VSIE_TRY(dalloc_t(h, &A->c_b64, (size_t)n));
  VSIE_TRY(dalloc_t(h, &A->w, (size_t)maxn));
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

vsie_status far_adjoint(vsie_handle* h, const double2* lam, double2* x, int precision,
                        cudaStream_t st) {
  const int64_t n = h->n;
  const double kap = h->k0 / kTwoPi;
  AdjRecords* A = &h->adj;
  Sources* cls[3] = {&h->G, &h->K, &h->F};
  VSIE_TRY(adjoint_buffers(h, st));
  prescale_colloc_kernel<<<nblk(n), 256, 0, st>>>(h->tgt64, lam, n, kap, precision, A->c_a32, A->c_b32,
                                                  A->c_a64, A->c_b64);
  VSIE_CUDA(cudaGetLastError());
  for (int c = 0; c < 3; ++c) {
    Sources& S = *cls[c];
    if (!S.n) continue;
    double2* slots = nullptr;
    if (c == 0) {
      // G: w_j = sum_i (e^{ikr}/r) c_i, x_e = conj(sum_j -s_j w_j)
      if (precision == 32) {
        const StreamK sk = plan_sk<float, PolG2>(h, S.n, n);
        VSIE_TRY(handle_slots(h, slot_elems(sk), &slots));
        PolG2 p{S.adj_p32, A->c_a32, A->c_b32};
        VSIE_TRY((run_nbody<float, PolG2>(p, sk, A->w, 0, slots, st, nullptr)));
      } else {
        using PG = PerTarget<double, PolG<double>>;
        const StreamK sk = plan_sk<double, PG>(h, S.n, n);
        VSIE_TRY(handle_slots(h, slot_elems(sk), &slots));
        PG p;
        p.tgt = S.adj_p64;
        p.tscale = 1.0;
        p.sa = A->c_a64;
        p.sb = A->c_b64;
        VSIE_TRY((run_nbody<double, PG>(p, sk, A->w, 0, slots, st, nullptr)));
      }
      gather_adjoint_kernel<<<nblk(S.n_elem), 256, 0, st>>>(A->w, S.pos_s, 1, S.elem_first, S.elem_list,
                                                            S.n_elem, x);
    } else {
      // K and F: w_j = sum_i (e^{ikr}/r)[-s_j + (ikr - 1)((x_i - y_j).v_j)/r^2] c_i
      if (precision == 32) {
        using PA = PerTarget<float, PolAF<float>>;
        const StreamK sk = plan_sk<float, PA>(h, S.n, n);
        VSIE_TRY(handle_slots(h, slot_elems(sk), &slots));
        PA p;
        p.tps = S.adj_p32;
        p.tv = S.adj_v32;
        p.sa = A->c_a32;
        p.sb = A->c_b32;
        VSIE_TRY((run_nbody<float, PA>(p, sk, A->w, 0, slots, st, nullptr)));
      } else {
        using PA = PerTarget<double, PolAF<double>>;
        const StreamK sk = plan_sk<double, PA>(h, S.n, n);
        VSIE_TRY(handle_slots(h, slot_elems(sk), &slots));
        PA p;
        p.tps = S.adj_p64;
        p.tv = S.adj_v64;
        p.sa = A->c_a64;
        p.sb = A->c_b64;
        VSIE_TRY((run_nbody<double, PA>(p, sk, A->w, 0, slots, st, nullptr)));
      }
      gather_adjoint_kernel<<<nblk(S.n_elem), 256, 0, st>>>(A->w, S.pos_s, 0, S.elem_first, S.elem_list,
                                                            S.n_elem, x);
    }
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

// ----------------------------------------------------------------- gradient channels

// Target records of one channel pass over the source points of a class: (kappa y, s') with
// s' = -1 for Phi (the adjoint sum then equals sum_i e^{ikr}/(4 pi r) conj(lam_i)), else 0,
// and v' = the unit vector of axis ch - 1 (not scaled by kappa) for Psi.
__global__ void channel_records_kernel(const double4_32a* __restrict__ ps, int64_t n, double kap, int ch,
                                       float4* __restrict__ p32, float4* __restrict__ v32,
                                       double4_32a* __restrict__ p64, double4_32a* __restrict__ v64) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  const double s = ch == 0 ? -1.0 : 0.0;
  const double vx = ch == 1 ? 1.0 : 0.0, vy = ch == 2 ? 1.0 : 0.0, vz = ch == 3 ? 1.0 : 0.0;
  p32[j] = make_float4((float)(kap * y.x), (float)(kap * y.y), (float)(kap * y.z), (float)s);
  v32[j] = make_float4((float)vx, (float)vy, (float)vz, 0.0f);
  p64[j] = make_double4_32a(kap * y.x, kap * y.y, kap * y.z, s);
  v64[j] = make_double4_32a(vx, vy, vz, 0.0);
}

// Phi_j = conj(w_j);  Psi_j[ch - 1] = conj(kappa w_j) (the unit v' carried 1/kappa)
__global__ void channel_out_kernel(const double2* __restrict__ w, int64_t n, int ch, double kap,
                                   double2* __restrict__ phi, double2* __restrict__ psi) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double2 v = w[j];
  if (ch == 0)
    phi[j] = make_double2(v.x, -v.y);
  else
    psi[3 * j + ch - 1] = make_double2(kap * v.x, -kap * v.y);
}

// One-pass FP32 channels: every (source point j, collocation point i) pair is evaluated
// once and feeds four complex sums, two source points per packed FP32x2 instruction:
//   E = e^{2 pi i t} rinv c~_i,            Phi'_j += E,
//   Psi'_j += d~ rinv^2 (Re + kr Im, Im - kr Re)(E),   kr = 2 pi t,  d~ = x~_i - y~_j,
// so that sum_i conj(G) lam_i = conj(Phi') and sum_i conj(grad_x G) lam_i = -kappa conj(Psi')
// (E (i kr - 1) = -(E.re + kr E.im) - i (E.im - kr E.re)).  Work items (tile of 256 points x
// chunk of collocation points) as in the other sums, partial tiles to slots, fix-up after.
constexpr int kChT = 2;                  // source points per thread (one packed pair)
constexpr int kChTile = kBlock * kChT;   // source points per work item

__global__ void __launch_bounds__(kBlock) channels_kernel(const float4* __restrict__ pts, const float4* __restrict__ ca,
                                                          const float* __restrict__ cb, StreamK sk,
                                                          double2* __restrict__ out, double2* __restrict__ slots) {
  __shared__ float4 sa[kBlock], sb[kBlock], sc[kBlock];
  const int tid = threadIdx.x;
  const int64_t b = blockIdx.x;
  const int64_t k0 = sk_begin(sk, b), k1 = sk_begin(sk, b + 1);
  int64_t k = k0;
  while (k < k1) {
    const int64_t tile = k / sk.nchunk;
    const int64_t c0 = k - tile * sk.nchunk;
    const int64_t c1 = min(sk.nchunk, c0 + (k1 - k));
    const int64_t ia = tile * kChTile + tid, ib = ia + kBlock;
    const float4 pa = ia < sk.nt ? pts[ia] : make_float4(0, 0, 0, 0);
    const float4 pb = ib < sk.nt ? pts[ib] : make_float4(0, 0, 0, 0);
    const float2 ntx = make_float2(-pa.x, -pb.x), nty = make_float2(-pa.y, -pb.y), ntz = make_float2(-pa.z, -pb.z);
    Acc<float> acc[kChT][4];
#pragma unroll
    for (int t = 0; t < kChT; ++t)
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[t][c].zero();
    const int64_t j_begin = c0 * sk.chunk;
    const int64_t j_end = min(sk.ns, c1 * sk.chunk);
    for (int64_t j0 = j_begin; j0 < j_end; j0 += kBlock) {
      const int64_t j = j0 + tid;
      const bool ok = j < j_end;
      const float4 r = ok ? ca[j] : make_float4(0, 0, 0, 0);
      const float ci = ok ? cb[j] : 0.0f;
      sa[tid] = make_float4(r.x, r.x, r.y, r.y);
      sb[tid] = make_float4(r.z, r.z, r.w, r.w);
      sc[tid] = make_float4(ci, ci, -ci, -ci);
      __syncthreads();
      float2 phr = f2(0.0f), phi = phr, xr = phr, xi = phr, yr = phr, yi = phr, zr = phr, zi = phr;
#pragma unroll 4
      for (int jj = 0; jj < kBlock; ++jj) {
        const float4 A = sa[jj], Bv = sb[jj], C = sc[jj];
        const float2 dx = __fadd2_rn(make_float2(A.x, A.y), ntx);
        const float2 dy = __fadd2_rn(make_float2(A.z, A.w), nty);
        const float2 dz = __fadd2_rn(make_float2(Bv.x, Bv.y), ntz);
        float2 r2 = __fmul2_rn(dx, dx);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        float2 rinv, t, cs, sn;
        phase2(r2, rinv, t, cs, sn);
        const float2 er = __fmul2_rn(cs, rinv), ei = __fmul2_rn(sn, rinv);
        const float2 cr = make_float2(Bv.z, Bv.w), cim = make_float2(C.x, C.y), ncim = make_float2(C.z, C.w);
        const float2 Er = __ffma2_rn(ei, ncim, __fmul2_rn(er, cr));
        const float2 Ei = __ffma2_rn(ei, cr, __fmul2_rn(er, cim));
        phr = __fadd2_rn(phr, Er);
        phi = __fadd2_rn(phi, Ei);
        const float2 kr = __fmul2_rn(t, f2(6.28318530717958647692f));
        const float2 nkr = __fmul2_rn(t, f2(-6.28318530717958647692f));
        const float2 ri2 = __fmul2_rn(rinv, rinv);
        const float2 hr = __fmul2_rn(ri2, __ffma2_rn(kr, Ei, Er));     // rinv^2 (Re + kr Im)
        const float2 hi = __fmul2_rn(ri2, __ffma2_rn(nkr, Er, Ei));    // rinv^2 (Im - kr Re)
        xr = __ffma2_rn(dx, hr, xr);
        xi = __ffma2_rn(dx, hi, xi);
        yr = __ffma2_rn(dy, hr, yr);
        yi = __ffma2_rn(dy, hi, yi);
        zr = __ffma2_rn(dz, hr, zr);
        zi = __ffma2_rn(dz, hi, zi);
      }
      __syncthreads();
      acc[0][0].fold(phr.x, phi.x);
      acc[1][0].fold(phr.y, phi.y);
      acc[0][1].fold(xr.x, xi.x);
      acc[1][1].fold(xr.y, xi.y);
      acc[0][2].fold(yr.x, yi.x);
      acc[1][2].fold(yr.y, yi.y);
      acc[0][3].fold(zr.x, zi.x);
      acc[1][3].fold(zr.y, zi.y);
    }
    const bool complete = (c0 == 0 && c1 == sk.nchunk);
    const int64_t slot = (k == k0) ? 2 * b : 2 * b + 1;
#pragma unroll
    for (int t = 0; t < kChT; ++t) {
      const int64_t i = tile * kChTile + (int64_t)t * kBlock + tid;
      if (i < sk.nt) {
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const double2 v = acc[t][c].value();
          if (complete)
            out[(int64_t)c * sk.nt + i] = v;
          else
            slots[(slot * 4 + c) * kChTile + (int64_t)t * kBlock + tid] = v;
        }
      }
    }
    k = tile * sk.nchunk + c1;
  }
}

// Adds the pieces of point tiles that span several blocks, in block order (4 channels).
__global__ void __launch_bounds__(kChTile) channels_fixup_kernel(StreamK sk, const double2* __restrict__ slots,
                                                                 double2* __restrict__ out) {
  const int64_t tile = blockIdx.x;
  const int64_t kf = tile * sk.nchunk, kl = kf + sk.nchunk - 1;
  const int64_t bs = sk_block_of(sk, kf), be = sk_block_of(sk, kl);
  if (bs == be) return;
  const int idx = threadIdx.x;
  const int64_t i = tile * kChTile + idx;
  if (i >= sk.nt) return;
  for (int c = 0; c < 4; ++c) {
    double sr = 0.0, si = 0.0;
    for (int64_t bb = bs; bb <= be; ++bb) {
      if (sk_begin(sk, bb) == sk_begin(sk, bb + 1)) continue;
      const int64_t slot = (bb == bs && sk_begin(sk, bb) != kf) ? 2 * bb + 1 : 2 * bb;
      const double2 v = slots[(slot * 4 + c) * kChTile + idx];
      sr += v.x;
      si += v.y;
    }
    out[(int64_t)c * sk.nt + i] = make_double2(sr, si);
  }
}

// Phi_j = conj(Phi'_j);  Psi_j = -kappa conj(Psi'_j)
__global__ void channels_finish_kernel(const double2* __restrict__ w4, int64_t n, double kap,
                                       double2* __restrict__ phi, double2* __restrict__ psi) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double2 p = w4[j];
  phi[j] = make_double2(p.x, -p.y);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const double2 v = w4[(int64_t)(a + 1) * n + j];
    psi[3 * j + a] = make_double2(-kap * v.x, kap * v.y);
  }
}

static int channels_resident_per_sm() {
  static int cached = 0;
  if (!cached) {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, channels_kernel, kBlock, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
    cached = per_sm;
  }
  return cached;
}

static vsie_status channels_fp32(vsie_handle* h, const Sources& S, double2* phi, double2* psi, cudaStream_t st) {
  AdjRecords* A = &h->adj;
  const double kap = h->k0 / kTwoPi;
  StreamK sk;
  sk.nt = S.n;
  sk.ns = h->n;
  sk.chunk = kChunk;
  sk.ntile = (sk.nt + kChTile - 1) / kChTile;
  sk.nchunk = (sk.ns + sk.chunk - 1) / sk.chunk;
  sk.nitems = sk.ntile * sk.nchunk;
  int64_t C = (int64_t)channels_resident_per_sm() * (h->num_sms > 0 ? h->num_sms : 148);
  if (h->tile_override > 0) C = h->tile_override;
  sk.grid = std::max<int64_t>(1, std::min<int64_t>(C, sk.nitems));
  double2* slots = nullptr;
  VSIE_TRY(handle_slots(h, (size_t)(2 * sk.grid) * 4 * kChTile, &slots));
  channels_kernel<<<(unsigned)sk.grid, kBlock, 0, st>>>(S.adj_p32, A->c_a32, A->c_b32, sk, A->ch_out, slots);
  channels_fixup_kernel<<<(unsigned)sk.ntile, kChTile, 0, st>>>(sk, slots, A->ch_out);
  channels_finish_kernel<<<nblk(S.n), 256, 0, st>>>(A->ch_out, S.n, kap, phi, psi);
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

vsie_status gradient_channels(vsie_handle* h, const double2* lam, int precision, double2* phi, double2* psi,
                              cudaStream_t st) {
  const int64_t n = h->n;
  const double kap = h->k0 / kTwoPi;
  AdjRecords* A = &h->adj;
  VSIE_TRY(adjoint_buffers(h, st));
  Sources* cls[3] = {&h->G, &h->K, &h->F};
  int64_t maxn = 1;
  for (Sources* S : cls) maxn = std::max<int64_t>(maxn, S->n);
  if (!A->ch_p32) {
    VSIE_TRY(dalloc_t(h, &A->ch_p32, (size_t)maxn));
    VSIE_TRY(dalloc_t(h, &A->ch_v32, (size_t)maxn));
    VSIE_TRY(dalloc_t(h, &A->ch_p64, (size_t)maxn));
    VSIE_TRY(dalloc_t(h, &A->ch_v64, (size_t)maxn));
  }
  prescale_colloc_kernel<<<nblk(n), 256, 0, st>>>(h->tgt64, lam, n, kap, precision, A->c_a32, A->c_b32,
                                                  A->c_a64, A->c_b64);
  VSIE_CUDA(cudaGetLastError());
  int64_t off = 0;
  if (precision == 32) {
    if (!A->ch_out) VSIE_TRY(dalloc_t(h, &A->ch_out, 4 * (size_t)maxn));
    for (int c = 0; c < 3; ++c) {
      Sources& S = *cls[c];
      if (!S.n) continue;
      if (n) VSIE_TRY(channels_fp32(h, S, phi + off, psi + 3 * off, st));
      else {
        VSIE_CUDA(cudaMemsetAsync(phi + off, 0, sizeof(double2) * S.n, st));
        VSIE_CUDA(cudaMemsetAsync(psi + 3 * off, 0, sizeof(double2) * 3 * S.n, st));
      }
      off += S.n;
    }
    return VSIE_OK;
  }
  for (int c = 0; c < 3; ++c) {
    Sources& S = *cls[c];
    if (!S.n) continue;
    for (int ch = 0; ch < 4; ++ch) {
      channel_records_kernel<<<nblk(S.n), 256, 0, st>>>(S.pos_s, S.n, kap, ch, A->ch_p32, A->ch_v32, A->ch_p64,
                                                         A->ch_v64);
      double2* slots = nullptr;
      if (precision == 32) {
        using PA = PerTarget<float, PolAF<float>>;
        const StreamK sk = plan_sk<float, PA>(h, S.n, n);
        VSIE_TRY(handle_slots(h, slot_elems(sk), &slots));
        PA p;
        p.tps = A->ch_p32;
        p.tv = A->ch_v32;
        p.sa = A->c_a32;
        p.sb = A->c_b32;
        VSIE_TRY((run_nbody<float, PA>(p, sk, A->w, 0, slots, st, nullptr)));
      } else {
        using PA = PerTarget<double, PolAF<double>>;
        const StreamK sk = plan_sk<double, PA>(h, S.n, n);
        VSIE_TRY(handle_slots(h, slot_elems(sk), &slots));
        PA p;
        p.tps = A->ch_p64;
        p.tv = A->ch_v64;
        p.sa = A->c_a64;
        p.sb = A->c_b64;
        VSIE_TRY((run_nbody<double, PA>(p, sk, A->w, 0, slots, st, nullptr)));
      }
      channel_out_kernel<<<nblk(S.n), 256, 0, st>>>(A->w, S.n, ch, kap, phi + off, psi + 3 * off);
      VSIE_CUDA(cudaGetLastError());
    }
    off += S.n;
  }
  return VSIE_OK;
}

}  // namespace vsie
