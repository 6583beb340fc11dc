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
// Kernel design (B300, sm_103a): the sum is bound by the FP32 and MUFU pipes, not by
// memory.  Each thread owns T targets in registers; a block stages 128 source records
// into shared memory per tile (one coalesced 16-byte load per thread) and every thread
// reads them back as warp-wide broadcasts.  e^{ikr} uses an explicit range reduction
// t = r k/(2 pi), f = t - rint(t), so the hardware sine/cosine only ever sees |2 pi f| <= pi.
// Accumulation is compensated by blocking: each tile's 128 terms are summed in FP32 and
// the tile sums are added in FP64.  A second grid dimension splits the sources when the
// target count alone cannot fill the 148 SMs; partial sums then go to a scratch array and
// are reduced in a fixed order (deterministic).

#include <cuda_runtime.h>

#include <algorithm>

#include "vsie_internal.h"

namespace vsie {

constexpr int kBlock = 128;

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

// rinv = 1/r (0 at r = 0); (cs, sn) = (cos kr, sin kr).  kk = k/(2 pi).
__device__ __forceinline__ void phase(float r2, float kk, float& rinv, float& cs, float& sn) {
  rinv = (r2 > 0.0f) ? rsqrtf(r2) : 0.0f;
  const float t = r2 * rinv * kk;
  const float f = t - rintf(t);
  __sincosf(f * 6.28318530717958647692f, &sn, &cs);
}
__device__ __forceinline__ void phase(double r2, double kk, double& rinv, double& cs, double& sn) {
  rinv = (r2 > 0.0) ? rsqrt(r2) : 0.0;
  const double t = r2 * rinv * kk;
  const double f = t - rint(t);
  sincospi(2.0 * f, &sn, &cs);
}

// ---------------------------------------------------------------------------------
// G class: y_i += sum_j (e^{ikr}/r) q_j.  Source records: a = (x, y, z, q.re), b = q.im.
template <class R, int T>
__global__ void __launch_bounds__(kBlock) far_g_kernel(
    const typename Vec4<R>::type* __restrict__ tgt, int64_t nt,
    const typename Vec4<R>::type* __restrict__ sa, const R* __restrict__ sb, int64_t ns,
    int64_t chunk, R kk, double2* __restrict__ out, int mode) {
  using V = typename Vec4<R>::type;
  __shared__ V s_a[kBlock];
  __shared__ R s_b[kBlock];
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kBlock * T + tid;
  const int64_t j_begin = (int64_t)blockIdx.y * chunk;
  const int64_t j_end = min(ns, j_begin + chunk);
  R xt[T], yt[T], zt[T];
  double tr[T], ti[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int64_t i = base + (int64_t)t * kBlock;
    V p = (i < nt) ? tgt[i] : V{};
    xt[t] = p.x;
    yt[t] = p.y;
    zt[t] = p.z;
    tr[t] = 0.0;
    ti[t] = 0.0;
  }
  for (int64_t j0 = j_begin; j0 < j_end; j0 += kBlock) {
    const int64_t j = j0 + tid;
    if (j < j_end) {
      s_a[tid] = sa[j];
      s_b[tid] = sb[j];
    } else {
      s_a[tid] = V{};  // zero charge: contributes exactly 0 wherever it sits
      s_b[tid] = R(0);
    }
    __syncthreads();
    R ar[T], ai[T];
#pragma unroll
    for (int t = 0; t < T; ++t) ar[t] = ai[t] = R(0);
#pragma unroll 4
    for (int jj = 0; jj < kBlock; ++jj) {
      const V s = s_a[jj];
      const R qi = s_b[jj];
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const R dx = xt[t] - s.x, dy = yt[t] - s.y, dz = zt[t] - s.z;
        const R r2 = dx * dx + dy * dy + dz * dz;
        R rinv, cs, sn;
        phase(r2, kk, rinv, cs, sn);
        const R er = cs * rinv, ei = sn * rinv;
        ar[t] += er * s.w - ei * qi;
        ai[t] += er * qi + ei * s.w;
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < T; ++t) {
      tr[t] += (double)ar[t];
      ti[t] += (double)ai[t];
    }
  }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int64_t i = base + (int64_t)t * kBlock;
    if (i < nt) {
      double2* o = out + (int64_t)blockIdx.y * nt + i;
      if (mode) {
        double2 v = *o;
        *o = make_double2(v.x + tr[t], v.y + ti[t]);
      } else {
        *o = make_double2(tr[t], ti[t]);
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// F class: y_i += sum_j (e^{ikr}/r) [q_j + (ikr - 1)(d . u_j)/r^2].
// Records (3 per source): (x, y, z, q.re) (q.im, ux.re, ux.im, uy.re) (uy.im, uz.re, uz.im, 0)
template <class R, int T>
__global__ void __launch_bounds__(kBlock) far_f_kernel(
    const typename Vec4<R>::type* __restrict__ tgt, int64_t nt,
    const typename Vec4<R>::type* __restrict__ src, int64_t ns, int64_t chunk, R k, R kk,
    double2* __restrict__ out, int mode) {
  using V = typename Vec4<R>::type;
  __shared__ V s_r[3 * kBlock];
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kBlock * T + tid;
  const int64_t j_begin = (int64_t)blockIdx.y * chunk;
  const int64_t j_end = min(ns, j_begin + chunk);
  R xt[T], yt[T], zt[T];
  double tr[T], ti[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int64_t i = base + (int64_t)t * kBlock;
    V p = (i < nt) ? tgt[i] : V{};
    xt[t] = p.x;
    yt[t] = p.y;
    zt[t] = p.z;
    tr[t] = 0.0;
    ti[t] = 0.0;
  }
  for (int64_t j0 = j_begin; j0 < j_end; j0 += kBlock) {
    // 3*kBlock records, loaded as 3 coalesced passes
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      const int64_t idx = 3 * j0 + (int64_t)c * kBlock + tid;
      s_r[c * kBlock + tid] = (idx < 3 * j_end) ? src[idx] : V{};
    }
    __syncthreads();
    R ar[T], ai[T];
#pragma unroll
    for (int t = 0; t < T; ++t) ar[t] = ai[t] = R(0);
#pragma unroll 2
    for (int jj = 0; jj < kBlock; ++jj) {
      const V a = s_r[3 * jj], b = s_r[3 * jj + 1], c = s_r[3 * jj + 2];
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const R dx = xt[t] - a.x, dy = yt[t] - a.y, dz = zt[t] - a.z;
        const R r2 = dx * dx + dy * dy + dz * dz;
        R rinv, cs, sn;
        phase(r2, kk, rinv, cs, sn);
        const R dur = dx * b.y + dy * b.w + dz * c.y;
        const R dui = dx * b.z + dy * c.x + dz * c.z;
        const R rinv2 = rinv * rinv;
        const R fi = (r2 * rinv * k) * rinv2;  // (ikr - 1)/r^2 = -rinv2 + i kr rinv2
        const R inr = a.w - rinv2 * dur - fi * dui;
        const R ini = b.x - rinv2 * dui + fi * dur;
        const R er = cs * rinv, ei = sn * rinv;
        ar[t] += er * inr - ei * ini;
        ai[t] += er * ini + ei * inr;
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < T; ++t) {
      tr[t] += (double)ar[t];
      ti[t] += (double)ai[t];
    }
  }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int64_t i = base + (int64_t)t * kBlock;
    if (i < nt) {
      double2* o = out + (int64_t)blockIdx.y * nt + i;
      if (mode) {
        double2 v = *o;
        *o = make_double2(v.x + tr[t], v.y + ti[t]);
      } else {
        *o = make_double2(tr[t], ti[t]);
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Adjoint, F class: for every source point j (here the "target", with weights s_j, v_j)
//   w_j = sum_i (e^{ikr}/r) [-s_j + (ikr - 1)((x_i - y_j) . v_j)/r^2] c_i,
// with c_i = conj(lam_i)/(4 pi) at the collocation points; then
// sum_i conj(C_ij) lam_i = conj(w_j).  Collocation records: a = (x, y, z, c.re), b = c.im.
template <class R, int T>
__global__ void __launch_bounds__(kBlock) adj_f_kernel(
    const typename Vec4<R>::type* __restrict__ tps, const typename Vec4<R>::type* __restrict__ tv,
    int64_t nt, const typename Vec4<R>::type* __restrict__ sa, const R* __restrict__ sb,
    int64_t ns, int64_t chunk, R k, R kk, double2* __restrict__ out, int mode) {
  using V = typename Vec4<R>::type;
  __shared__ V s_a[kBlock];
  __shared__ R s_b[kBlock];
  const int tid = threadIdx.x;
  const int64_t base = (int64_t)blockIdx.x * kBlock * T + tid;
  const int64_t j_begin = (int64_t)blockIdx.y * chunk;
  const int64_t j_end = min(ns, j_begin + chunk);
  V pt[T], vt[T];
  double tr[T], ti[T];
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int64_t i = base + (int64_t)t * kBlock;
    pt[t] = (i < nt) ? tps[i] : V{};
    vt[t] = (i < nt) ? tv[i] : V{};
    tr[t] = 0.0;
    ti[t] = 0.0;
  }
  for (int64_t j0 = j_begin; j0 < j_end; j0 += kBlock) {
    const int64_t j = j0 + tid;
    if (j < j_end) {
      s_a[tid] = sa[j];
      s_b[tid] = sb[j];
    } else {
      s_a[tid] = V{};
      s_b[tid] = R(0);
    }
    __syncthreads();
    R ar[T], ai[T];
#pragma unroll
    for (int t = 0; t < T; ++t) ar[t] = ai[t] = R(0);
#pragma unroll 2
    for (int jj = 0; jj < kBlock; ++jj) {
      const V s = s_a[jj];
      const R ci = s_b[jj];
#pragma unroll
      for (int t = 0; t < T; ++t) {
        const R dx = s.x - pt[t].x, dy = s.y - pt[t].y, dz = s.z - pt[t].z;  // x_i - y_j
        const R r2 = dx * dx + dy * dy + dz * dz;
        R rinv, cs, sn;
        phase(r2, kk, rinv, cs, sn);
        const R dv = dx * vt[t].x + dy * vt[t].y + dz * vt[t].z;
        const R rinv2 = rinv * rinv;
        const R mr = -pt[t].w - rinv2 * dv;        // -s + (ikr - 1) dv / r^2
        const R mi = (r2 * rinv * k) * rinv2 * dv;
        const R er = cs * rinv, ei = sn * rinv;
        const R gr = er * s.w - ei * ci, gi = er * ci + ei * s.w;  // (e^{ikr}/r) c_i
        ar[t] += gr * mr - gi * mi;
        ai[t] += gr * mi + gi * mr;
      }
    }
    __syncthreads();
#pragma unroll
    for (int t = 0; t < T; ++t) {
      tr[t] += (double)ar[t];
      ti[t] += (double)ai[t];
    }
  }
#pragma unroll
  for (int t = 0; t < T; ++t) {
    const int64_t i = base + (int64_t)t * kBlock;
    if (i < nt) {
      double2* o = out + (int64_t)blockIdx.y * nt + i;
      if (mode) {
        double2 v = *o;
        *o = make_double2(v.x + tr[t], v.y + ti[t]);
      } else {
        *o = make_double2(tr[t], ti[t]);
      }
    }
  }
}

// ---------------------------------------------------------------------------------
// Charge prescale (per apply): q = -s p_e/(4 pi), u = v p_e/(4 pi).
__global__ void prescale_g_kernel(const double4_32a* __restrict__ ps, const int32_t* __restrict__ own,
                                  const double2* __restrict__ p, int64_t n, int prec,
                                  float4* __restrict__ a32, float* __restrict__ b32,
                                  double4_32a* __restrict__ a64, double* __restrict__ b64) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  const double2 pe = p[own[j]];
  const double sc = -y.w / kFourPi;
  const double qr = sc * pe.x, qi = sc * pe.y;
  if (prec == 32) {
    a32[j] = make_float4((float)y.x, (float)y.y, (float)y.z, (float)qr);
    b32[j] = (float)qi;
  } else {
    a64[j] = make_double4_32a(y.x, y.y, y.z, qr);
    b64[j] = qi;
  }
}

__global__ void prescale_f_kernel(const double4_32a* __restrict__ ps, const double4_32a* __restrict__ vv,
                                  const int32_t* __restrict__ own, const double2* __restrict__ p,
                                  int64_t n, int prec, float4* __restrict__ a32,
                                  double4_32a* __restrict__ a64) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  const double4_32a v = vv[j];
  const double2 pe = p[own[j]];
  const double sc = -y.w / kFourPi, vs = 1.0 / kFourPi;
  const double qr = sc * pe.x, qi = sc * pe.y;
  const double uxr = vs * v.x * pe.x, uxi = vs * v.x * pe.y;
  const double uyr = vs * v.y * pe.x, uyi = vs * v.y * pe.y;
  const double uzr = vs * v.z * pe.x, uzi = vs * v.z * pe.y;
  if (prec == 32) {
    a32[3 * j] = make_float4((float)y.x, (float)y.y, (float)y.z, (float)qr);
    a32[3 * j + 1] = make_float4((float)qi, (float)uxr, (float)uxi, (float)uyr);
    a32[3 * j + 2] = make_float4((float)uyi, (float)uzr, (float)uzi, 0.0f);
  } else {
    a64[3 * j] = make_double4_32a(y.x, y.y, y.z, qr);
    a64[3 * j + 1] = make_double4_32a(qi, uxr, uxi, uyr);
    a64[3 * j + 2] = make_double4_32a(uyi, uzr, uzi, 0.0);
  }
}

// collocation records for the adjoint: c = conj(lam)/(4 pi) at x_i
__global__ void prescale_colloc_kernel(const double4_32a* __restrict__ tgt, const double2* __restrict__ lam,
                                       int64_t n, int prec, float4* __restrict__ a32,
                                       float* __restrict__ b32, double4_32a* __restrict__ a64,
                                       double* __restrict__ b64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4_32a x = tgt[i];
  const double cr = lam[i].x / kFourPi, ci = -lam[i].y / kFourPi;
  if (prec == 32) {
    a32[i] = make_float4((float)x.x, (float)x.y, (float)x.z, (float)cr);
    b32[i] = (float)ci;
  } else {
    a64[i] = make_double4_32a(x.x, x.y, x.z, cr);
    b64[i] = ci;
  }
}

// static per-point target records for the adjoint: (x, y, z, s) and (vx, vy, vz, 0)
__global__ void point_records_kernel(const double4_32a* __restrict__ ps, const double4_32a* __restrict__ vv,
                                     int64_t n, float4* __restrict__ p32, float4* __restrict__ v32) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= n) return;
  const double4_32a y = ps[j];
  p32[j] = make_float4((float)y.x, (float)y.y, (float)y.z, (float)y.w);
  if (vv) {
    const double4_32a v = vv[j];
    v32[j] = make_float4((float)v.x, (float)v.y, (float)v.z, 0.0f);
  }
}

// sum of split partials (fixed order), stored or added into out
__global__ void reduce_split_kernel(const double2* __restrict__ part, int nsplit, int64_t n,
                                    double2* __restrict__ out, int mode) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double sr = 0.0, si = 0.0;
  for (int s = 0; s < nsplit; ++s) {
    const double2 v = part[(int64_t)s * n + i];
    sr += v.x;
    si += v.y;
  }
  if (mode) {
    const double2 v = out[i];
    out[i] = make_double2(v.x + sr, v.y + si);
  } else {
    out[i] = make_double2(sr, si);
  }
}

// x_e = sum_{j in e} conj(scale_j * w_j), scale_j = -s_j for the G class (w = a_j), 1 for F
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

// ---------------------------------------------------------------------------------
struct Launch {
  dim3 grid;
  int64_t chunk;
  int nsplit;
};

static Launch plan(const vsie_handle* h, int64_t nt, int64_t ns, int T) {
  Launch L;
  const int64_t bx = (nt + (int64_t)kBlock * T - 1) / ((int64_t)kBlock * T);
  const int64_t want = (int64_t)(h->num_sms > 0 ? h->num_sms : 148) * 8;
  int64_t nsplit = (bx >= want) ? 1 : (want + bx - 1) / bx;
  const int64_t max_split = (ns + kBlock - 1) / kBlock;
  if (nsplit > max_split) nsplit = max_split;
  if (nsplit < 1) nsplit = 1;
  if (h->tile_override > 0) nsplit = h->tile_override < 65535 ? h->tile_override : 65535;
  int64_t chunk = (ns + nsplit - 1) / nsplit;
  chunk = ((chunk + kBlock - 1) / kBlock) * kBlock;
  if (chunk < kBlock) chunk = kBlock;
  nsplit = (int)((ns + chunk - 1) / chunk);
  if (nsplit < 1) nsplit = 1;
  L.grid = dim3((unsigned)bx, (unsigned)nsplit, 1);
  L.chunk = chunk;
  L.nsplit = (int)nsplit;
  return L;
}

}  // namespace vsie

namespace vsie {

// Split-partial scratch, grown on demand and owned by the handle.
static vsie_status split_scratch(vsie_handle* h, size_t elems, double2** out) {
  if (h->split_elems < elems) {
    double2* p = nullptr;
    VSIE_TRY(dalloc_t(h, &p, elems));
    h->split = p;
    h->split_elems = elems;
  }
  *out = h->split;
  return VSIE_OK;
}

constexpr int kT = 4;

template <class R>
static vsie_status launch_g(vsie_handle* h, const typename Vec4<R>::type* tgt, int64_t nt,
                            const typename Vec4<R>::type* sa, const R* sb, int64_t ns, double2* out,
                            int mode, cudaStream_t st) {
  if (ns == 0 || nt == 0) return VSIE_OK;
  const R kk = (R)(h->k0 / (2.0 * kPi));
  Launch L = plan(h, nt, ns, kT);
  if (L.nsplit == 1) {
    far_g_kernel<R, kT><<<L.grid, kBlock, 0, st>>>(tgt, nt, sa, sb, ns, L.chunk, kk, out, mode);
  } else {
    double2* part;
    VSIE_TRY(split_scratch(h, (size_t)L.nsplit * nt, &part));
    far_g_kernel<R, kT><<<L.grid, kBlock, 0, st>>>(tgt, nt, sa, sb, ns, L.chunk, kk, part, 0);
    reduce_split_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(part, L.nsplit, nt, out, mode);
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

template <class R>
static vsie_status launch_f(vsie_handle* h, const typename Vec4<R>::type* tgt, int64_t nt,
                            const typename Vec4<R>::type* src, int64_t ns, double2* out, int mode,
                            cudaStream_t st) {
  if (ns == 0 || nt == 0) return VSIE_OK;
  const R k = (R)h->k0, kk = (R)(h->k0 / (2.0 * kPi));
  Launch L = plan(h, nt, ns, kT);
  if (L.nsplit == 1) {
    far_f_kernel<R, kT><<<L.grid, kBlock, 0, st>>>(tgt, nt, src, ns, L.chunk, k, kk, out, mode);
  } else {
    double2* part;
    VSIE_TRY(split_scratch(h, (size_t)L.nsplit * nt, &part));
    far_f_kernel<R, kT><<<L.grid, kBlock, 0, st>>>(tgt, nt, src, ns, L.chunk, k, kk, part, 0);
    reduce_split_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(part, L.nsplit, nt, out, mode);
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

static inline unsigned nblk(int64_t n, int b = 256) { return (unsigned)((n + b - 1) / b); }

vsie_status far_prescale(vsie_handle* h, const double2* x, int precision, cudaStream_t st,
                         int* launches) {
  Sources& G = h->G;
  Sources& F = h->F;
  if (G.n) {
    prescale_g_kernel<<<nblk(G.n), 256, 0, st>>>(G.pos_s, G.owner, x, G.n, precision, G.r32a,
                                                 G.r32b, G.r64a, G.r64b);
    if (launches) ++*launches;
  }
  if (F.n) {
    prescale_f_kernel<<<nblk(F.n), 256, 0, st>>>(F.pos_s, F.vvec, F.owner, x, F.n, precision,
                                                 F.r32a, F.r64a);
    if (launches) ++*launches;
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

static int launches_of(const vsie_handle* h, int64_t nt, int64_t ns) {
  if (ns == 0 || nt == 0) return 0;
  return plan(h, nt, ns, kT).nsplit > 1 ? 2 : 1;
}

vsie_status far_sum_g(vsie_handle* h, double2* y, int precision, cudaStream_t st, int* launches) {
  Sources& G = h->G;
  if (!G.n) return VSIE_OK;
  if (launches) *launches += launches_of(h, h->n, G.n);
  if (precision == 32) return launch_g<float>(h, h->tgt32, h->n, G.r32a, G.r32b, G.n, y, 0, st);
  return launch_g<double>(h, h->tgt64, h->n, G.r64a, G.r64b, G.n, y, 0, st);
}

vsie_status far_sum_f(vsie_handle* h, double2* y, int precision, cudaStream_t st, int* launches) {
  Sources& F = h->F;
  const int mode = h->G.n ? 1 : 0;
  if (!F.n) {
    if (!h->G.n) VSIE_CUDA(cudaMemsetAsync(y, 0, sizeof(double2) * h->n, st));
    return VSIE_OK;
  }
  if (launches) *launches += launches_of(h, h->n, F.n);
  if (precision == 32) return launch_f<float>(h, h->tgt32, h->n, F.r32a, F.n, y, mode, st);
  return launch_f<double>(h, h->tgt64, h->n, F.r64a, F.n, y, mode, st);
}

vsie_status far_apply(vsie_handle* h, const double2* x, double2* y, int precision,
                      cudaStream_t st) {
  VSIE_TRY(far_prescale(h, x, precision, st, nullptr));
  VSIE_TRY(far_sum_g(h, y, precision, st, nullptr));
  VSIE_TRY(far_sum_f(h, y, precision, st, nullptr));
  return VSIE_OK;
}

// ---------------------------------------------------------------------------------
// Far-field sums whose source-split partials go to caller-provided scratch instead of
// the handle's lazily grown buffer (used by the allocation-free apply).

size_t far_split_elems(const vsie_handle* h) {
  size_t need = 0;
  const Sources* cls[2] = {&h->G, &h->F};
  for (const Sources* S : cls) {
    if (!S->n || !h->n) continue;
    const Launch L = plan(h, h->n, S->n, kT);
    if (L.nsplit > 1) need = std::max(need, (size_t)L.nsplit * (size_t)h->n);
  }
  return need;
}

template <class R>
static void launch_g_into(const vsie_handle* h, const typename Vec4<R>::type* tgt, int64_t nt,
                          const typename Vec4<R>::type* sa, const R* sb, int64_t ns, double2* out,
                          int mode, double2* scratch, cudaStream_t st) {
  const R kk = (R)(h->k0 / (2.0 * kPi));
  const Launch L = plan(h, nt, ns, kT);
  if (L.nsplit == 1) {
    far_g_kernel<R, kT><<<L.grid, kBlock, 0, st>>>(tgt, nt, sa, sb, ns, L.chunk, kk, out, mode);
  } else {
    far_g_kernel<R, kT><<<L.grid, kBlock, 0, st>>>(tgt, nt, sa, sb, ns, L.chunk, kk, scratch, 0);
    reduce_split_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(scratch, L.nsplit, nt, out, mode);
  }
}

template <class R>
static void launch_f_into(const vsie_handle* h, const typename Vec4<R>::type* tgt, int64_t nt,
                          const typename Vec4<R>::type* src, int64_t ns, double2* out, int mode,
                          double2* scratch, cudaStream_t st) {
  const R k = (R)h->k0, kk = (R)(h->k0 / (2.0 * kPi));
  const Launch L = plan(h, nt, ns, kT);
  if (L.nsplit == 1) {
    far_f_kernel<R, kT><<<L.grid, kBlock, 0, st>>>(tgt, nt, src, ns, L.chunk, k, kk, out, mode);
  } else {
    far_f_kernel<R, kT><<<L.grid, kBlock, 0, st>>>(tgt, nt, src, ns, L.chunk, k, kk, scratch, 0);
    reduce_split_kernel<<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(scratch, L.nsplit, nt, out, mode);
  }
}

vsie_status far_sums_into(vsie_handle* h, double2* y, int precision, double2* scratch,
                          cudaStream_t st) {
  Sources& G = h->G;
  Sources& F = h->F;
  const int64_t n = h->n;
  if (!G.n && !F.n) {
    VSIE_CUDA(cudaMemsetAsync(y, 0, sizeof(double2) * n, st));
    return VSIE_OK;
  }
  if (G.n) {
    if (precision == 32)
      launch_g_into<float>(h, h->tgt32, n, G.r32a, G.r32b, G.n, y, 0, scratch, st);
    else
      launch_g_into<double>(h, h->tgt64, n, G.r64a, G.r64b, G.n, y, 0, scratch, st);
  }
  if (F.n) {
    const int mode = G.n ? 1 : 0;
    if (precision == 32)
      launch_f_into<float>(h, h->tgt32, n, F.r32a, F.n, y, mode, scratch, st);
    else
      launch_f_into<double>(h, h->tgt64, n, F.r64a, F.n, y, mode, scratch, st);
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

vsie_status far_adjoint(vsie_handle* h, const double2* lam, double2* x, int precision,
                        cudaStream_t st) {
  Sources& G = h->G;
  Sources& F = h->F;
  const int64_t n = h->n;
  AdjRecords* A = &h->adj;
  if (!A->w) {
    VSIE_TRY(dalloc_t(h, &A->g_p32, (size_t)G.n));
    VSIE_TRY(dalloc_t(h, &A->f_p32, (size_t)F.n));
    VSIE_TRY(dalloc_t(h, &A->f_v32, (size_t)F.n));
    VSIE_TRY(dalloc_t(h, &A->c_a32, (size_t)n));
    VSIE_TRY(dalloc_t(h, &A->c_b32, (size_t)n));
    VSIE_TRY(dalloc_t(h, &A->c_a64, (size_t)n));
    VSIE_TRY(dalloc_t(h, &A->c_b64, (size_t)n));
    VSIE_TRY(dalloc_t(h, &A->w, (size_t)(G.n > F.n ? G.n : F.n)));
    if (G.n) point_records_kernel<<<nblk(G.n), 256, 0, st>>>(G.pos_s, nullptr, G.n, A->g_p32, nullptr);
    if (F.n) point_records_kernel<<<nblk(F.n), 256, 0, st>>>(F.pos_s, F.vvec, F.n, A->f_p32, A->f_v32);
    VSIE_CUDA(cudaGetLastError());
  }
  prescale_colloc_kernel<<<nblk(n), 256, 0, st>>>(h->tgt64, lam, n, precision, A->c_a32, A->c_b32,
                                                  A->c_a64, A->c_b64);
  VSIE_CUDA(cudaGetLastError());
  const double k = h->k0, kk = h->k0 / (2.0 * kPi);
  // G class: w_j = sum_i (e^{ikr}/r) c_i, then x_e = conj(sum_j -s_j w_j)
  if (G.n) {
    if (precision == 32)
      VSIE_TRY(launch_g<float>(h, A->g_p32, G.n, A->c_a32, A->c_b32, n, A->w, 0, st));
    else
      VSIE_TRY(launch_g<double>(h, G.pos_s, G.n, A->c_a64, A->c_b64, n, A->w, 0, st));
    gather_adjoint_kernel<<<nblk(G.n_elem), 256, 0, st>>>(A->w, G.pos_s, 1, G.elem_first,
                                                          G.elem_list, G.n_elem, x);
  }
  if (F.n) {
    Launch L = plan(h, F.n, n, kT);
    double2* dst = A->w;
    double2* part = nullptr;
    if (L.nsplit > 1) {
      VSIE_TRY(split_scratch(h, (size_t)L.nsplit * F.n, &part));
      dst = part;
    }
    if (precision == 32)
      adj_f_kernel<float, kT><<<L.grid, kBlock, 0, st>>>(A->f_p32, A->f_v32, F.n, A->c_a32, A->c_b32, n,
                                                         L.chunk, (float)k, (float)kk, dst, 0);
    else
      adj_f_kernel<double, kT><<<L.grid, kBlock, 0, st>>>(F.pos_s, F.vvec, F.n, A->c_a64, A->c_b64, n,
                                                          L.chunk, k, kk, dst, 0);
    if (L.nsplit > 1)
      reduce_split_kernel<<<nblk(F.n), 256, 0, st>>>(part, L.nsplit, F.n, A->w, 0);
    gather_adjoint_kernel<<<nblk(F.n_elem), 256, 0, st>>>(A->w, F.pos_s, 0, F.elem_first,
                                                          F.elem_list, F.n_elem, x);
  }
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

}  // namespace vsie
