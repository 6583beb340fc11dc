// Incident plane waves (Eq. planewave) and the far-field pattern of the scattered field
// (Eq. vsie used as a representation formula in Omega_0, Sec. 2.3.1), both in FP64.

#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "vsie_internal.h"

namespace vsie {

// b[i + n d] = exp(i k0 x_i . dir_d)
__global__ void plane_wave_kernel(const double4_32a* __restrict__ tgt, int64_t n, const double4_32a* __restrict__ dirs,
                                  int ndir, double k0, double2* __restrict__ b) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int d = blockIdx.y;
  if (i >= n || d >= ndir) return;
  const double4_32a x = tgt[i], u = dirs[d];
  double sn, cs;
  sincos(k0 * (x.x * u.x + x.y * u.y + x.z * u.z), &sn, &cs);
  b[(int64_t)d * n + i] = make_double2(cs, sn);
}

// out[d + ndir r] = (1/4pi) sum_j e^{-ik xhat.y_j} (s_j - ik xhat.v_j) p_e(j)
struct FarClass {
  const double4_32a* ps;
  const double4_32a* v;  // null for the G class (v = 0)
  const int32_t* own;
  int64_t n;
};

__global__ void far_field_kernel(FarClass c0, FarClass c1, FarClass c2, const double2* __restrict__ p,
                                 int64_t n, const double4_32a* __restrict__ dirs, int ndir, double k,
                                 double2* __restrict__ out) {
  __shared__ double red[2][8];
  const int d = blockIdx.x, r = blockIdx.y;
  const double4_32a u = dirs[d];
  const double2* pr = p + (int64_t)r * n;
  double ar = 0.0, ai = 0.0;
  const int64_t total = c0.n + c1.n + c2.n;
  for (int64_t jj = threadIdx.x; jj < total; jj += blockDim.x) {
    const FarClass& c = jj < c0.n ? c0 : (jj < c0.n + c1.n ? c1 : c2);
    const int64_t j = jj < c0.n ? jj : (jj < c0.n + c1.n ? jj - c0.n : jj - c0.n - c1.n);
    const double4_32a y = c.ps[j];
    double vx = 0, vy = 0, vz = 0;
    if (c.v) {
      const double4_32a v = c.v[j];
      vx = v.x; vy = v.y; vz = v.z;
    }
    const int32_t e = c.own[j];
    double sn, cs;
    sincos(-k * (u.x * y.x + u.y * y.y + u.z * y.z), &sn, &cs);
    const double amr = y.w, ami = -k * (u.x * vx + u.y * vy + u.z * vz);
    const double tr = cs * amr - sn * ami, ti = cs * ami + sn * amr;
    const double2 q = pr[e];
    ar += tr * q.x - ti * q.y;
    ai += tr * q.y + ti * q.x;
  }
  for (int o = 16; o > 0; o >>= 1) {
    ar += __shfl_down_sync(0xffffffffu, ar, o);
    ai += __shfl_down_sync(0xffffffffu, ai, o);
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) {
    red[0][wid] = ar;
    red[1][wid] = ai;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sr = 0, si = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      sr += red[0][w];
      si += red[1][w];
    }
    out[(int64_t)r * ndir + d] = make_double2(sr / kFourPi, si / kFourPi);
  }
}

// x_e = (1/4pi) sum_{j in e} sum_d e^{+ik xhat_d.y_j}(s_j + ik xhat_d.v_j) r_d  (F^H r);
// one thread per element (its quadrature points are contiguous in its class).
__global__ void far_field_adjoint_kernel(FarClass c, const int32_t* __restrict__ first,
                                         const int32_t* __restrict__ elem, int64_t n_elem,
                                         const double2* __restrict__ r, int ndir, int64_t n,
                                         const double4_32a* __restrict__ dirs, double k, int nrhs,
                                         double2* __restrict__ x) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  for (int q = 0; q < nrhs; ++q) {
    const double2* rq = r + (int64_t)q * ndir;
    double ar = 0.0, ai = 0.0;
    for (int32_t j = first[e]; j < first[e + 1]; ++j) {
      const double4_32a y = c.ps[j];
      double vx = 0, vy = 0, vz = 0;
      if (c.v) {
        const double4_32a v = c.v[j];
        vx = v.x; vy = v.y; vz = v.z;
      }
      for (int d = 0; d < ndir; ++d) {
        const double4_32a u = dirs[d];
        double sn, cs;
        sincos(k * (u.x * y.x + u.y * y.y + u.z * y.z), &sn, &cs);
        const double amr = y.w, ami = k * (u.x * vx + u.y * vy + u.z * vz);
        const double tr = cs * amr - sn * ami, ti = cs * ami + sn * amr;
        const double2 rr = rq[d];
        ar += tr * rr.x - ti * rr.y;
        ai += tr * rr.y + ti * rr.x;
      }
    }
    x[(int64_t)q * n + elem[e]] = make_double2(ar / kFourPi, ai / kFourPi);
  }
}

static vsie_status upload_dirs(const double* h_dirs, int ndir, double4_32a** d_dirs, cudaStream_t st) {
  std::vector<double4_32a> u(ndir);
  for (int d = 0; d < ndir; ++d) {
    const double x = h_dirs[3 * d], y = h_dirs[3 * d + 1], z = h_dirs[3 * d + 2];
    const double nrm = std::sqrt(x * x + y * y + z * z);
    if (!(nrm > 0.0) || !std::isfinite(nrm)) {
      set_error("direction vectors must be nonzero and finite");
      return VSIE_ERR_ARG;
    }
    u[d] = make_double4_32a(x / nrm, y / nrm, z / nrm, 0.0);
  }
  VSIE_CUDA(cudaMalloc(d_dirs, sizeof(double4_32a) * ndir));
  cudaError_t e = cudaMemcpyAsync(*d_dirs, u.data(), sizeof(double4_32a) * ndir, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    cudaFree(*d_dirs);
    return cuda_fail(e, "upload directions", __FILE__, __LINE__);
  }
  return VSIE_OK;
}

}  // namespace vsie

using namespace vsie;

extern "C" vsie_status vsie_plane_wave_rhs(vsie_handle* h, const double* h_dirs, int32_t ndir, void* d_b,
                                           void* stream) {
  clear_error();
  TraceRange trace("vsie_plane_wave_rhs");
  if (!h || !h_dirs || !d_b || ndir < 1 || ndir > 65535) {
    set_error("vsie_plane_wave_rhs: invalid argument");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double4_32a* dirs;
  VSIE_TRY(upload_dirs(h_dirs, ndir, &dirs, st));
  dim3 grid((unsigned)((h->n + 255) / 256), (unsigned)ndir);
  plane_wave_kernel<<<grid, 256, 0, st>>>(h->tgt64, h->n, dirs, ndir, h->k0, (double2*)d_b);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dirs);
  if (e != cudaSuccess) return cuda_fail(e, "plane_wave_kernel", __FILE__, __LINE__);
  return VSIE_OK;
}

extern "C" vsie_status vsie_far_field(vsie_handle* h, const void* d_p, int32_t nrhs, const double* h_dirs,
                                      int32_t ndir, void* d_out, void* stream) {
  clear_error();
  TraceRange trace("vsie_far_field");
  if (!h || !d_p || !h_dirs || !d_out || ndir < 1 || nrhs < 1 || nrhs > 65535) {
    set_error("vsie_far_field: invalid argument");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double4_32a* dirs;
  VSIE_TRY(upload_dirs(h_dirs, ndir, &dirs, st));
  dim3 grid((unsigned)ndir, (unsigned)nrhs);
  const FarClass g{h->G.pos_s, nullptr, h->G.owner, h->G.n};
  const FarClass kc{h->K.pos_s, h->K.vvec, h->K.owner, h->K.n};
  const FarClass f{h->F.pos_s, h->F.vvec, h->F.owner, h->F.n};
  far_field_kernel<<<grid, 256, 0, st>>>(g, kc, f, (const double2*)d_p, h->n, dirs, ndir, h->k0,
                                         (double2*)d_out);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dirs);
  if (e != cudaSuccess) return cuda_fail(e, "far_field_kernel", __FILE__, __LINE__);
  return VSIE_OK;
}

extern "C" vsie_status vsie_far_field_adjoint(vsie_handle* h, const void* d_r, int32_t nrhs, const double* h_dirs,
                                              int32_t ndir, void* d_x, void* stream) {
  clear_error();
  TraceRange trace("vsie_far_field_adjoint");
  if (!h || !d_r || !h_dirs || !d_x || ndir < 1 || nrhs < 1) {
    set_error("vsie_far_field_adjoint: invalid argument");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double4_32a* dirs;
  VSIE_TRY(upload_dirs(h_dirs, ndir, &dirs, st));
  const Sources* cls[3] = {&h->G, &h->K, &h->F};
  cudaError_t e = cudaSuccess;
  for (const Sources* S : cls) {
    if (!S->n_elem) continue;
    const FarClass c{S->pos_s, S == &h->G ? nullptr : S->vvec, S->owner, S->n};
    far_field_adjoint_kernel<<<(unsigned)((S->n_elem + 127) / 128), 128, 0, st>>>(
        c, S->elem_first, S->elem_list, S->n_elem, (const double2*)d_r, ndir, h->n, dirs, h->k0, nrhs,
        (double2*)d_x);
    e = cudaGetLastError();
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(dirs);
  if (e != cudaSuccess) return cuda_fail(e, "far_field_adjoint_kernel", __FILE__, __LINE__);
  return VSIE_OK;
}
