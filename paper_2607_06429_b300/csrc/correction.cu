// Near-field and self correction matrix Delta (FP64, built on the device) and its
// application y += m x + Delta x (Eq. mass_function for m, Sec. 2.3.4 for the self terms).
//
// The far-field kernels evaluate every (collocation point, source point) pair with the
// far rule.  Delta replaces, pair by pair, that far-rule value with an accurate one:
//   * a tetrahedron on its own centroid: -(beta - k0^2 alpha)_e S(a_e), the single layer
//     integrated over the ball of equal volume, S(a) = [e^{ika}(1 - ika) - 1]/k^2; the
//     adjoint double layer of that ball vanishes by symmetry (Sec. 2.3.4);
//   * a tetrahedron whose centroid lies within near_radius of the target (centroid far
//     rule only): the degree-2 four-point rule;
//   * a triangle whose centroid lies within tri_near_radius of the target: the double
//     layer split as G = G_0 + (G - G_0), the Laplace part integrated exactly through the
//     signed solid angle (Van Oosterom & Strackee), the bounded remainder by the
//     three-point rule; a triangle on its own centroid takes the principal value 0.
// Entry = accurate value - far-rule value, computed in FP64 and stored as double-float
// pairs.  Two value arrays are kept: val64 subtracts the far-rule value from the FP64
// coordinates (used with the FP64 far sum), val32 from the FP32 coordinates the FP32 far
// sum sees (float(kappa x)), so that near-singular pairs cancel to FP32 arithmetic error
// rather than to coordinate-rounding error.
//
// Neighbour search: uniform cell grids (cell >= radius) over tetrahedron and triangle
// centroids, sorted by cell with thrust; each target scans its 27 neighbouring cells.

#include <cuda_runtime.h>
#include <thrust/binary_search.h>
#include <thrust/device_ptr.h>
#include <thrust/execution_policy.h>
#include <thrust/iterator/counting_iterator.h>
#include <thrust/scan.h>
#include <thrust/sequence.h>
#include <thrust/sort.h>

#include <algorithm>
#include <cmath>

#include "dfloat.h"
#include "vsie_internal.h"

namespace vsie {



__device__ __forceinline__ int cell_coord(double p, double lo, double inv, int nc) {
  int c = (int)floor((p - lo) * inv);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

__global__ void cell_id_kernel(const double4_32a* __restrict__ pts, int64_t n, CellGrid g,
                               int64_t* __restrict__ key, int32_t* __restrict__ idx) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double4_32a p = pts[i];
  const int cx = cell_coord(p.x, g.lo[0], g.inv, g.nc[0]);
  const int cy = cell_coord(p.y, g.lo[1], g.inv, g.nc[1]);
  const int cz = cell_coord(p.z, g.lo[2], g.inv, g.nc[2]);
  key[i] = ((int64_t)cx * g.nc[1] + cy) * g.nc[2] + cz;
  idx[i] = (int32_t)i;
}

// ----------------------------------------------------------------- FP64 pair values

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// C(x, y) = G [-s + (ikr - 1)(d . v)/r^2], d = x - y, zero at r = 0.
__device__ double2 pair64(double dx, double dy, double dz, double s, double vx, double vy,
                          double vz, double k) {
  const double r2 = dx * dx + dy * dy + dz * dz;
  if (!(r2 > 0.0)) return make_double2(0.0, 0.0);
  const double r = sqrt(r2);
  double sn, cs;
  sincos(k * r, &sn, &cs);
  const double g = 1.0 / (kFourPi * r);
  const double dv = (dx * vx + dy * vy + dz * vz) / r2;
  // (-s - dv) + i (k r dv)
  const double2 m = make_double2(-s - dv, k * r * dv);
  return cmul(make_double2(g * cs, g * sn), m);
}

// The coordinate the FP32 far-field kernels see: x stored as float(kappa x), mapped back.
__device__ __forceinline__ double r32(double x, double kap) { return (double)(float)(kap * x) / kap; }

// sum over the tetrahedron's four-point rule (weights w/4)
__device__ double2 tet4(double x, double y, double z, const double4_32a* __restrict__ pts, double s4,
                        double4_32a g4, double k, bool round32) {
  const double kap = k / (2.0 * kPi);
  double2 acc = make_double2(0.0, 0.0);
  for (int q = 0; q < 4; ++q) {
    double4_32a p = pts[q];
    double xx = x, yy = y, zz = z;
    if (round32) {
      p.x = r32(p.x, kap); p.y = r32(p.y, kap); p.z = r32(p.z, kap);
      xx = r32(x, kap); yy = r32(y, kap); zz = r32(z, kap);
    }
    const double2 c = pair64(xx - p.x, yy - p.y, zz - p.z, s4, g4.x, g4.y, g4.z, k);
    acc.x += c.x;
    acc.y += c.y;
  }
  return acc;
}

// int_t dG/dn_y dS for a target near the flat triangle t (see file comment)
__device__ double2 dl_near(double x, double y, double z, const double4_32a* __restrict__ V,
                           const double4_32a* __restrict__ Q, double4_32a nrm, double k) {
  const double ax = V[0].x - x, ay = V[0].y - y, az = V[0].z - z;
  const double bx = V[1].x - x, by = V[1].y - y, bz = V[1].z - z;
  const double cx = V[2].x - x, cy = V[2].y - y, cz = V[2].z - z;
  const double la = sqrt(ax * ax + ay * ay + az * az);
  const double lb = sqrt(bx * bx + by * by + bz * bz);
  const double lc = sqrt(cx * cx + cy * cy + cz * cz);
  const double num = ax * (by * cz - bz * cy) + ay * (bz * cx - bx * cz) + az * (bx * cy - by * cx);
  const double den = la * lb * lc + (ax * bx + ay * by + az * bz) * lc +
                     (ax * cx + ay * cy + az * cz) * lb + (bx * cx + by * cy + bz * cz) * la;
  const double omega = 2.0 * atan2(num, den);
  double2 acc = make_double2(-omega / kFourPi, 0.0);
  const double w = nrm.w / 3.0;
  for (int q = 0; q < 3; ++q) {
    const double dx = x - Q[q].x, dy = y - Q[q].y, dz = z - Q[q].z;
    const double r2 = dx * dx + dy * dy + dz * dz;
    if (!(r2 > 0.0)) continue;
    const double r = sqrt(r2);
    double sn, cs;
    sincos(k * r, &sn, &cs);
    // g'(r) = (i k r e^{ikr} - e^{ikr} + 1) / (4 pi r^2)
    const double nr = -k * r * sn - cs + 1.0;
    const double ni = k * r * cs - sn;
    const double inv = 1.0 / (kFourPi * r2);
    const double dn = (dx * nrm.x + dy * nrm.y + dz * nrm.z) / r;
    acc.x += -nr * inv * dn * w;
    acc.y += -ni * inv * dn * w;
  }
  return acc;
}



// Visit the correction entries of row i: vol near set (or self only), then tri near set.
// fill == false: count only.
__global__ void corr_rows_kernel(CorrInputs in, const int64_t* __restrict__ row_ptr,
                                 int64_t* __restrict__ counts, int32_t* __restrict__ col,
                                 double2* __restrict__ v64, double2* __restrict__ v32, int fill) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= in.n) return;
  const double4_32a X = in.tgt[i];
  const double k = in.k;
  const int64_t si = in.self ? i : -1;  // the row's own unknown, if any
  int64_t pos = fill ? row_ptr[i] : 0;
  int64_t cnt = 0;
  auto emit = [&](int32_t c, double2 a64, double2 a32) {
    if (fill) {
      col[pos] = c;
      v64[pos] = a64;
      v32[pos] = a32;
      ++pos;
    }
    ++cnt;
  };
  auto vol_entry = [&](int64_t e) {
    const double vol = in.tet_vol[e];
    const double s = in.tet_s[e];
    const double4_32a ga = in.tet_ga[e];
    double2 acc, f64 = make_double2(0, 0), f32 = make_double2(0, 0);
    const double s4 = s * vol * 0.25;
    const double4_32a g4 = make_double4_32a(ga.x * vol * 0.25, ga.y * vol * 0.25, ga.z * vol * 0.25, 0);
    if (e == si) {
      // self: single layer over the equal-volume ball, adjoint double layer 0
      const double a = cbrt(3.0 * vol / kFourPi);
      double sn, cs;
      sincos(k * a, &sn, &cs);
      // e^{ika}(1 - ika) - 1
      const double re = cs + k * a * sn - 1.0, im = sn - k * a * cs;
      acc = make_double2(-s * re / (k * k), -s * im / (k * k));
      if (in.far_points == 4) {
        f64 = tet4(X.x, X.y, X.z, in.tet_pts + 4 * e, s4, g4, k, false);
        f32 = tet4(X.x, X.y, X.z, in.tet_pts + 4 * e, s4, g4, k, true);
      }
    } else {
      acc = tet4(X.x, X.y, X.z, in.tet_pts + 4 * e, s4, g4, k, false);
      const double4_32a c = in.tet_cen[e];
      f64 = pair64(X.x - c.x, X.y - c.y, X.z - c.z, s * vol, ga.x * vol, ga.y * vol, ga.z * vol, k);
      const double kap = k / (2.0 * kPi);
      f32 = pair64(r32(X.x, kap) - r32(c.x, kap), r32(X.y, kap) - r32(c.y, kap),
                   r32(X.z, kap) - r32(c.z, kap), s * vol, ga.x * vol, ga.y * vol, ga.z * vol, k);
    }
    emit((int32_t)e, make_double2(acc.x - f64.x, acc.y - f64.y),
         make_double2(acc.x - f32.x, acc.y - f32.y));
  };
  auto tri_entry = [&](int64_t t) {
    const double om = in.tri_omega[t];
    const double4_32a nr = in.tri_nrm[t];
    const double4_32a* Q = in.tri_pts + 3 * t;
    const double w = nr.w / 3.0;
    const double vx = -om * w * nr.x, vy = -om * w * nr.y, vz = -om * w * nr.z;
    double2 acc = make_double2(0, 0), f64 = make_double2(0, 0), f32 = make_double2(0, 0);
    const bool self = (si == in.n_tet + t);
    if (!self) {
      const double2 d = dl_near(X.x, X.y, X.z, in.tri_vtx + 3 * t, Q, nr, k);
      acc = make_double2(om * d.x, om * d.y);
    }
    const double kap = k / (2.0 * kPi);
    const double xr = r32(X.x, kap), yr = r32(X.y, kap), zr = r32(X.z, kap);
    for (int q = 0; q < 3; ++q) {
      const double2 c64 = pair64(X.x - Q[q].x, X.y - Q[q].y, X.z - Q[q].z, 0.0, vx, vy, vz, k);
      const double2 c32 = pair64(xr - r32(Q[q].x, kap), yr - r32(Q[q].y, kap), zr - r32(Q[q].z, kap),
                                 0.0, vx, vy, vz, k);
      f64.x += c64.x;
      f64.y += c64.y;
      f32.x += c32.x;
      f32.y += c32.y;
    }
    emit((int32_t)(in.n_tet + t), make_double2(acc.x - f64.x, acc.y - f64.y),
         make_double2(acc.x - f32.x, acc.y - f32.y));
  };

  // volume part
  if (in.R2v > 0.0) {
    const CellGrid& g = in.gv;
    const int cx = cell_coord(X.x, g.lo[0], g.inv, g.nc[0]);
    const int cy = cell_coord(X.y, g.lo[1], g.inv, g.nc[1]);
    const int cz = cell_coord(X.z, g.lo[2], g.inv, g.nc[2]);
    for (int ax = max(cx - 1, 0); ax <= min(cx + 1, g.nc[0] - 1); ++ax)
      for (int ay = max(cy - 1, 0); ay <= min(cy + 1, g.nc[1] - 1); ++ay)
        for (int az = max(cz - 1, 0); az <= min(cz + 1, g.nc[2] - 1); ++az) {
          const int64_t cell = ((int64_t)ax * g.nc[1] + ay) * g.nc[2] + az;
          for (int64_t p = g.start[cell]; p < g.start[cell + 1]; ++p) {
            const int32_t e = g.order[p];
            const double4_32a c = in.tet_cen[e];
            const double dx = X.x - c.x, dy = X.y - c.y, dz = X.z - c.z;
            if (dx * dx + dy * dy + dz * dz < in.R2v || e == si) vol_entry(e);
          }
        }
  } else if (si >= 0 && si < in.n_tet) {
    vol_entry(si);
  }
  // interface part
  if (in.R2t > 0.0) {
    const CellGrid& g = in.gt;
    const int cx = cell_coord(X.x, g.lo[0], g.inv, g.nc[0]);
    const int cy = cell_coord(X.y, g.lo[1], g.inv, g.nc[1]);
    const int cz = cell_coord(X.z, g.lo[2], g.inv, g.nc[2]);
    for (int ax = max(cx - 1, 0); ax <= min(cx + 1, g.nc[0] - 1); ++ax)
      for (int ay = max(cy - 1, 0); ay <= min(cy + 1, g.nc[1] - 1); ++ay)
        for (int az = max(cz - 1, 0); az <= min(cz + 1, g.nc[2] - 1); ++az) {
          const int64_t cell = ((int64_t)ax * g.nc[1] + ay) * g.nc[2] + az;
          for (int64_t p = g.start[cell]; p < g.start[cell + 1]; ++p) {
            const int32_t t = g.order[p];
            const double4_32a c = in.tri_cen[t];
            const double dx = X.x - c.x, dy = X.y - c.y, dz = X.z - c.z;
            if (dx * dx + dy * dy + dz * dz < in.R2t || si == in.n_tet + t) tri_entry(t);
          }
        }
  }
  if (!fill) counts[i] = cnt;
}

// ----------------------------------------------------------------- application


// The correction values are stored as double-float complex numbers (re.hi, im.hi, re.lo,
// im.lo): 16 bytes per entry like complex128, about 48 significant bits, so that the
// multiply-adds run on the FP32 pipe (dfloat.h) instead of B300's 1/64-rate FP64 pipe and
// the SpMV becomes bound by HBM bandwidth.

// complex128 -> double-float, in place (each 16-byte entry rewritten by the thread that reads it)
__global__ void to_df_inplace_kernel(double2* __restrict__ v, int64_t m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const float4 d = df_pack(v[i]);
  reinterpret_cast<float4*>(v)[i] = d;
}

__global__ void to_df_kernel(const double2* __restrict__ x, float4* __restrict__ xd, int64_t m) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) xd[i] = df_pack(x[i]);
}

__device__ __forceinline__ float2 shfl_down2(float2 v, int o) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, o), __shfl_down_sync(0xffffffffu, v.y, o));
}

// y_i += m_i x_i + sum_k Delta_ik x_col(k); one warp per row, lanes strided over the row's
// entries (coalesced value and column loads), double-float products and sums, a fixed
// reduction order (deterministic); xd is x in double-float.
__global__ void __launch_bounds__(256) corr_apply_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                         const float4* __restrict__ val, const double* __restrict__ mass,
                                                         const float4* __restrict__ xd, const double2* __restrict__ x,
                                                         double2* __restrict__ y, int64_t n) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  float2 S = make_float2(0.0f, 0.0f), C = S;
  const int64_t pe = rp[row + 1];
#pragma unroll 4
  for (int64_t p = rp[row] + lane; p < pe; p += 32) df_cmac(S, C, val[p], xd[col[p]]);
  df_renorm2(S, C);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) df_add2(S, C, shfl_down2(S, o), shfl_down2(C, o));
  if (lane == 0) {
    const double2 d = df_value(S, C);
    const double m = mass[row];
    const double2 q = x[row];
    const double2 o = y[row];
    y[row] = make_double2(o.x + m * q.x + d.x, o.y + m * q.y + d.y);
  }
}

// x_e += m_e lam_e (the mass is real)
__global__ void mass_adjoint_kernel(const double* __restrict__ mass, const double2* __restrict__ lam,
                                    double2* __restrict__ x, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double m = mass[i];
  const double2 l = lam[i];
  const double2 o = x[i];
  x[i] = make_double2(o.x + m * l.x, o.y + m * l.y);
}

// x_col += conj(Delta_ik) lam_i (scatter with FP64 atomics)
__global__ void corr_adjoint_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const float4* __restrict__ val, const double2* __restrict__ lam,
                                    double2* __restrict__ x, int64_t n) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  const double2 l = lam[row];
  for (int64_t p = rp[row] + lane; p < rp[row + 1]; p += 32) {
    const float4 d = val[p];
    const double vr = (double)d.x + (double)d.z, vi = (double)d.y + (double)d.w;
    double* dst = reinterpret_cast<double*>(x + col[p]);
    atomicAdd(dst, vr * l.x + vi * l.y);
    atomicAdd(dst + 1, vr * l.y - vi * l.x);
  }
}

vsie_status correction_apply(vsie_handle* h, const double2* x, double2* y, int precision,
                             cudaStream_t st) {
  const int64_t n = h->n;
  if (n == 0) return VSIE_OK;
  const float4* val = precision == 32 ? h->C.val32 : h->C.val64;
  to_df_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, h->C.xd, n);
  const unsigned blocks = (unsigned)((n * 32 + 255) / 256);
  corr_apply_kernel<<<blocks, 256, 0, st>>>(h->C.row_ptr, h->C.col, val, h->mass, h->C.xd, x, y, n);
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

// Rows [r0, r1) of the correction and mass: y_out[i - r0] += m_i x_i + (Delta x)_i.  The
// row pointers hold absolute offsets into the column and value arrays, and the columns are
// global unknowns, so the kernel of the full apply serves with its row arrays offset.
vsie_status correction_apply_rows(vsie_handle* h, const double2* x, double2* y_out, int64_t r0, int64_t r1,
                                  int precision, cudaStream_t st) {
  const int64_t n = h->n, m = r1 - r0;
  if (m <= 0) return VSIE_OK;
  const float4* val = precision == 32 ? h->C.val32 : h->C.val64;
  to_df_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x, h->C.xd, n);
  const unsigned blocks = (unsigned)((m * 32 + 255) / 256);
  corr_apply_kernel<<<blocks, 256, 0, st>>>(h->C.row_ptr + r0, h->C.col, val, h->mass + r0, h->C.xd, x + r0,
                                            y_out, m);
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

vsie_status correction_adjoint(vsie_handle* h, const double2* lam, double2* x, int precision,
                               cudaStream_t st) {
  const int64_t n = h->n;
  const float4* val = precision == 32 ? h->C.val32 : h->C.val64;
  mass_adjoint_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(h->mass, lam, x, n);
  corr_adjoint_kernel<<<(unsigned)((n * 32 + 255) / 256), 256, 0, st>>>(h->C.row_ptr, h->C.col, val,
                                                                          lam, x, n);
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

// ----------------------------------------------------------------- block application

// xt[c][r] = x[r][c] for a block of up to 64 columns: row-major, 64 entries per row (zero
// past the block), as float2 (FP32 path) or double-float float4 (FP64 path).  32 x 32
// tiles through shared memory, so both the reads and the writes are coalesced.
template <class T>
__device__ __forceinline__ T to_row(double2 v);
template <>
__device__ __forceinline__ float2 to_row<float2>(double2 v) {
  return make_float2((float)v.x, (float)v.y);
}
template <>
__device__ __forceinline__ float4 to_row<float4>(double2 v) {
  return df_pack(v);
}

template <class T>
__global__ void corr_transpose_kernel(const double2* __restrict__ x, int64_t n, int ncols, T* __restrict__ xt) {
  __shared__ double2 tile[32][33];
  const int64_t c0 = (int64_t)blockIdx.x * 32;
  const int r0 = blockIdx.y * 32;
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int r = r0 + k;
    const int64_t c = c0 + threadIdx.x;
    tile[k][threadIdx.x] = (r < ncols && c < n) ? x[(int64_t)r * n + c] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int k = threadIdx.y; k < 32; k += blockDim.y) {
    const int64_t c = c0 + k;
    if (c < n) xt[c * 64 + r0 + threadIdx.x] = to_row<T>(tile[threadIdx.x][k]);
  }
}

// Kahan step for the (re, im) pair: s - c carries the sum, c the lost low part
__device__ __forceinline__ void kahan2(float2& s, float2& c, float2 p) {
  const float2 yv = __fadd2_rn(p, make_float2(-c.x, -c.y));
  const float2 t = __fadd2_rn(s, yv);
  c = __fadd2_rn(__fadd2_rn(t, make_float2(-s.x, -s.y)), make_float2(-yv.x, -yv.y));
  s = t;
}

// y[r][i] += m_i x[r][i] + sum_k Delta_ik x[r][col_k] for the ncols columns of a block:
// one warp per row i, lane l owns columns l and l + 32.  The row's (value, column) pairs are
// loaded 32 at a time (coalesced) and broadcast by shuffles; each entry then costs one
// coalesced read of the charge row xt[col] (256 or 1024 bytes, L2-resident for mid-size
// meshes).  FP32 path (T = float2): the values' high parts, FP32 products, Kahan-compensated
// sums.  FP64 path (T = float4): double-float products and sums.
template <class T>
__global__ void __launch_bounds__(256) corr_block_kernel(const int64_t* __restrict__ rp,
                                                         const int32_t* __restrict__ col,
                                                         const float4* __restrict__ val,
                                                         const double* __restrict__ mass,
                                                         const T* __restrict__ xt,
                                                         const double2* __restrict__ x,
                                                         double2* __restrict__ y, int64_t n, int ncols) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  constexpr bool kDF = sizeof(T) == 16;
  float2 s0 = make_float2(0.0f, 0.0f), s1 = s0, c0 = s0, c1 = s0;
  const int64_t pb = rp[row], pe = rp[row + 1];
  for (int64_t p0 = pb; p0 < pe; p0 += 32) {
    const int cnt = (int)min((int64_t)32, pe - p0);
    float4 mv = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    int32_t mc = 0;
    if (lane < cnt) {
      mv = val[p0 + lane];
      mc = col[p0 + lane];
    }
#pragma unroll 4
    for (int q = 0; q < cnt; ++q) {
      float4 v;
      v.x = __shfl_sync(0xffffffffu, mv.x, q);
      v.y = __shfl_sync(0xffffffffu, mv.y, q);
      if constexpr (kDF) {
        v.z = __shfl_sync(0xffffffffu, mv.z, q);
        v.w = __shfl_sync(0xffffffffu, mv.w, q);
      }
      const int32_t cc = __shfl_sync(0xffffffffu, mc, q);
      const T a = xt[(int64_t)cc * 64 + lane], b = xt[(int64_t)cc * 64 + lane + 32];
      if constexpr (kDF) {
        df_cmac(s0, c0, v, a);
        df_cmac(s1, c1, v, b);
      } else {
        kahan2(s0, c0, make_float2(fmaf(v.x, a.x, -v.y * a.y), fmaf(v.x, a.y, v.y * a.x)));
        kahan2(s1, c1, make_float2(fmaf(v.x, b.x, -v.y * b.y), fmaf(v.x, b.y, v.y * b.x)));
      }
    }
    if constexpr (kDF) {
      df_renorm2(s0, c0);
      df_renorm2(s1, c1);
    }
  }
  const double m = mass[row];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int r = lane + 32 * h;
    if (r >= ncols) continue;
    const float2 sv = h ? s1 : s0, cv = h ? c1 : c0;
    const double2 d = kDF ? df_value(sv, cv) : make_double2((double)sv.x - (double)cv.x, (double)sv.y - (double)cv.y);
    const double2 q = x[(int64_t)r * n + row];
    double2* o = y + (int64_t)r * n + row;
    const double2 ov = *o;
    *o = make_double2(ov.x + m * q.x + d.x, ov.y + m * q.y + d.y);
  }
}

vsie_status correction_apply_block(vsie_handle* h, const double2* x, double2* y, int ncols, int precision,
                                   cudaStream_t st) {
  const int64_t n = h->n;
  if (n == 0 || ncols < 1) return VSIE_OK;
  const size_t xt_bytes = (size_t)n * 64 * (precision == 32 ? sizeof(float2) : sizeof(float4));
  if (h->batch.xt_bytes < xt_bytes) {
    unsigned char* p = nullptr;
    VSIE_TRY(dalloc_t(h, &p, xt_bytes));
    h->batch.xt = p;
    h->batch.xt_bytes = xt_bytes;
  }
  const dim3 tgrid((unsigned)((n + 31) / 32), 2), tblock(32, 8);
  const unsigned blocks = (unsigned)((n * 32 + 255) / 256);
  for (int r0 = 0; r0 < ncols; r0 += 64) {
    const int nc = std::min(64, ncols - r0);
    const double2* xb = x + (size_t)r0 * n;
    double2* yb = y + (size_t)r0 * n;
    if (precision == 32) {
      float2* xt = reinterpret_cast<float2*>(h->batch.xt);
      corr_transpose_kernel<float2><<<tgrid, tblock, 0, st>>>(xb, n, nc, xt);
      corr_block_kernel<float2><<<blocks, 256, 0, st>>>(h->C.row_ptr, h->C.col, h->C.val32, h->mass, xt, xb, yb,
                                                         n, nc);
    } else {
      float4* xt = reinterpret_cast<float4*>(h->batch.xt);
      corr_transpose_kernel<float4><<<tgrid, tblock, 0, st>>>(xb, n, nc, xt);
      corr_block_kernel<float4><<<blocks, 256, 0, st>>>(h->C.row_ptr, h->C.col, h->C.val64, h->mass, xt, xb, yb,
                                                         n, nc);
    }
    VSIE_CUDA(cudaGetLastError());
  }
  return VSIE_OK;
}

// ----------------------------------------------------------------- construction

static vsie_status make_grid(vsie_handle* h, const double4_32a* pts, int64_t np, double radius,
                             const double lo[3], const double hi[3], CellGrid* g,
                             std::vector<void*>* temps) {
  double cs = radius;
  for (;;) {
    int64_t total = 1;
    for (int d = 0; d < 3; ++d) {
      g->lo[d] = lo[d];
      g->nc[d] = (int)std::floor((hi[d] - lo[d]) / cs) + 1;
      total *= g->nc[d];
    }
    if (total <= (int64_t)1 << 24) {
      g->ncell = total;
      break;
    }
    cs *= 1.5;  // a coarser grid still finds every neighbour within one cell
  }
  g->inv = 1.0 / cs;
  int64_t* key;
  int32_t* order;
  int64_t* start;
  VSIE_CUDA(cudaMalloc(&key, sizeof(int64_t) * (np > 0 ? np : 1)));
  temps->push_back(key);
  // the sorted order and the cell starts stay with the handle (field evaluation reuses them)
  VSIE_TRY(dalloc_t(h, &order, (size_t)(np > 0 ? np : 1)));
  VSIE_TRY(dalloc_t(h, &start, (size_t)g->ncell + 1));
  if (np > 0) {
    cell_id_kernel<<<(unsigned)((np + 255) / 256), 256>>>(pts, np, *g, key, order);
    VSIE_CUDA(cudaGetLastError());
    thrust::stable_sort_by_key(thrust::device, thrust::device_ptr<int64_t>(key),
                               thrust::device_ptr<int64_t>(key + np),
                               thrust::device_ptr<int32_t>(order));
  }
  thrust::lower_bound(thrust::device, thrust::device_ptr<int64_t>(key),
                      thrust::device_ptr<int64_t>(key + np), thrust::counting_iterator<int64_t>(0),
                      thrust::counting_iterator<int64_t>(g->ncell + 1),
                      thrust::device_ptr<int64_t>(start));
  VSIE_CUDA(cudaGetLastError());
  g->order = order;
  g->start = start;
  return VSIE_OK;
}

vsie_status build_correction(vsie_handle* h, const double4_32a* d_tet_cen, const double4_32a* d_tet_pts,
                             const double* d_tet_s, const double4_32a* d_tet_ga, const double* d_tet_vol,
                             const double4_32a* d_tri_vtx, const double4_32a* d_tri_pts,
                             const double4_32a* d_tri_cen, const double4_32a* d_tri_nrm,
                             const double* d_tri_omega, const double lo[3], const double hi[3]) {
  CorrInputs in;
  in.tgt = h->tgt64;
  in.tet_cen = d_tet_cen;
  in.tet_pts = d_tet_pts;
  in.tet_s = d_tet_s;
  in.tet_ga = d_tet_ga;
  in.tet_vol = d_tet_vol;
  in.tri_vtx = d_tri_vtx;
  in.tri_pts = d_tri_pts;
  in.tri_cen = d_tri_cen;
  in.tri_nrm = d_tri_nrm;
  in.tri_omega = d_tri_omega;
  in.n_tet = h->n_tet;
  in.n_tri = h->n_tri;
  in.n = h->n;
  in.far_points = h->far_points;
  in.k = h->k0;
  const bool vol_near = h->far_points == 1 && h->near_radius > 0.0 && h->n_tet > 0;
  const bool tri_near = h->tri_near_radius > 0.0 && h->n_tri > 0;
  in.R2v = vol_near ? h->near_radius * h->near_radius : 0.0;
  in.R2t = tri_near ? h->tri_near_radius * h->tri_near_radius : 0.0;

  std::vector<void*> temps;
  auto cleanup = [&]() {
    for (void* p : temps) cudaFree(p);
  };
  vsie_status s = VSIE_OK;
  if (vol_near) s = make_grid(h, d_tet_cen, h->n_tet, h->near_radius, lo, hi, &in.gv, &temps);
  if (s == VSIE_OK && tri_near)
    s = make_grid(h, d_tri_cen, h->n_tri, h->tri_near_radius, lo, hi, &in.gt, &temps);
  if (s != VSIE_OK) {
    cleanup();
    return s;
  }
  const int64_t n = h->n;
  s = dalloc_t(h, &h->C.row_ptr, (size_t)n + 1);
  if (s != VSIE_OK) {
    cleanup();
    return s;
  }
  const unsigned blocks = (unsigned)((n + 127) / 128);
  cudaError_t e = cudaMemset(h->C.row_ptr, 0, sizeof(int64_t) * ((size_t)n + 1));
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "cudaMemset(row_ptr)", __FILE__, __LINE__);
  }
  corr_rows_kernel<<<blocks, 128>>>(in, nullptr, h->C.row_ptr, nullptr, nullptr, nullptr, 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "corr_rows_kernel(count)", __FILE__, __LINE__);
  }
  // counts -> exclusive prefix sum in place (row_ptr[n] = nnz)
  thrust::exclusive_scan(thrust::device, thrust::device_ptr<int64_t>(h->C.row_ptr),
                         thrust::device_ptr<int64_t>(h->C.row_ptr + n + 1),
                         thrust::device_ptr<int64_t>(h->C.row_ptr));
  int64_t nnz = 0;
  e = cudaMemcpy(&nnz, h->C.row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "cudaMemcpy(nnz)", __FILE__, __LINE__);
  }
  h->C.nnz = nnz;
  double2 *v64 = nullptr, *v32 = nullptr;
  if ((s = dalloc_t(h, &h->C.col, (size_t)nnz)) != VSIE_OK || (s = dalloc_t(h, &v64, (size_t)nnz)) != VSIE_OK ||
      (s = dalloc_t(h, &v32, (size_t)nnz)) != VSIE_OK || (s = dalloc_t(h, &h->C.xd, (size_t)n)) != VSIE_OK) {
    cleanup();
    return s;
  }
  corr_rows_kernel<<<blocks, 128>>>(in, h->C.row_ptr, nullptr, h->C.col, v64, v32, 1);
  e = cudaGetLastError();
  if (e == cudaSuccess && nnz > 0) {
    // the FP64 values become double-float pairs in place (16 bytes each either way)
    to_df_inplace_kernel<<<(unsigned)((nnz + 255) / 256), 256>>>(v64, nnz);
    to_df_inplace_kernel<<<(unsigned)((nnz + 255) / 256), 256>>>(v32, nnz);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  h->C.val64 = reinterpret_cast<float4*>(v64);
  h->C.val32 = reinterpret_cast<float4*>(v32);
  cleanup();
  if (e != cudaSuccess) return cuda_fail(e, "corr_rows_kernel(fill)", __FILE__, __LINE__);
  h->geo = in;
  return VSIE_OK;
}

// ----------------------------------------------------------------- field points

// y_r = -(y_r + sum_k Delta_rk x_col(k)): one warp per field point, the entries in
// double-float like corr_apply_kernel (no mass term: the points carry no unknown).
__global__ void __launch_bounds__(256) field_corr_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                                         const float4* __restrict__ val, const float4* __restrict__ xd,
                                                         double2* __restrict__ y, int64_t m) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= m) return;
  float2 S = make_float2(0.0f, 0.0f), C = S;
  const int64_t pe = rp[row + 1];
  for (int64_t p = rp[row] + lane; p < pe; p += 32) df_cmac(S, C, val[p], xd[col[p]]);
  df_renorm2(S, C);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) df_add2(S, C, shfl_down2(S, o), shfl_down2(C, o));
  if (lane == 0) {
    const double2 d = df_value(S, C);
    const double2 o = y[row];
    y[row] = make_double2(-(o.x + d.x), -(o.y + d.y));
  }
}

vsie_status field_correction(vsie_handle* h, const double4_32a* d_pts, int64_t m, const double2* x,
                             int nrhs, double2* y, int precision, cudaStream_t st) {
  if (m <= 0 || nrhs <= 0) return VSIE_OK;
  CorrInputs in = h->geo;
  in.tgt = d_pts;
  in.n = m;
  in.self = 0;
  int64_t* rp = nullptr;
  int32_t* col = nullptr;
  double2 *v64 = nullptr, *v32 = nullptr;
  auto cleanup = [&]() {
    cudaFree(rp);
    cudaFree(col);
    cudaFree(v64);
    cudaFree(v32);
  };
  auto fail = [&](cudaError_t e, const char* what) {
    cleanup();
    return cuda_fail(e, what, __FILE__, __LINE__);
  };
  cudaError_t e = cudaMalloc(&rp, sizeof(int64_t) * ((size_t)m + 1));
  if (e != cudaSuccess) return fail(e, "cudaMalloc(field row_ptr)");
  e = cudaMemsetAsync(rp, 0, sizeof(int64_t) * ((size_t)m + 1), st);
  if (e != cudaSuccess) return fail(e, "cudaMemsetAsync(field row_ptr)");
  const unsigned blocks = (unsigned)((m + 127) / 128);
  corr_rows_kernel<<<blocks, 128, 0, st>>>(in, nullptr, rp, nullptr, nullptr, nullptr, 0);
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "corr_rows_kernel(field count)");
  thrust::exclusive_scan(thrust::cuda::par.on(st), thrust::device_ptr<int64_t>(rp),
                         thrust::device_ptr<int64_t>(rp + m + 1), thrust::device_ptr<int64_t>(rp));
  int64_t nnz = 0;
  if ((e = cudaMemcpyAsync(&nnz, rp + m, sizeof(int64_t), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(e, "cudaMemcpyAsync(field nnz)");
  const size_t cap = (size_t)(nnz > 0 ? nnz : 1);
  if ((e = cudaMalloc(&col, sizeof(int32_t) * cap)) != cudaSuccess ||
      (e = cudaMalloc(&v64, sizeof(double2) * cap)) != cudaSuccess ||
      (e = cudaMalloc(&v32, sizeof(double2) * cap)) != cudaSuccess)
    return fail(e, "cudaMalloc(field rows)");
  corr_rows_kernel<<<blocks, 128, 0, st>>>(in, rp, nullptr, col, v64, v32, 1);
  if (nnz > 0) {
    to_df_inplace_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(v64, nnz);
    to_df_inplace_kernel<<<(unsigned)((nnz + 255) / 256), 256, 0, st>>>(v32, nnz);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "corr_rows_kernel(field fill)");
  const float4* val = reinterpret_cast<const float4*>(precision == 32 ? v32 : v64);
  const int64_t n = h->n;
  for (int c = 0; c < nrhs; ++c) {
    to_df_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(x + (size_t)c * n, h->C.xd, n);
    field_corr_kernel<<<(unsigned)((m * 32 + 255) / 256), 256, 0, st>>>(rp, col, val, h->C.xd,
                                                                         y + (size_t)c * m, m);
  }
  if ((e = cudaGetLastError()) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return fail(e, "field_corr_kernel");
  cleanup();
  return VSIE_OK;
}

}  // namespace vsie
