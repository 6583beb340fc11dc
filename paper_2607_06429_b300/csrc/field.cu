// Field at points off the collocation grid (Sec. 2, Eq. vsie with m = 1 outside the
// scatterer): once the collocation values p solve A p = p_inc, the equation evaluated at an
// exterior point X gives p(X) = p_inc(X) - I(X) p, where I(X) p is the integral part of the
// operator at X: the far rule over every far-field source point plus, for the elements whose
// centroids lie within the near radii of X, the near rules in place of the far rule.  The
// scattered field is therefore p_s(X) = -I(X) p.  The far sums reuse the collocation
// kernels with the points as targets; the near rows are built for the points from the
// handle's geometry and neighbour grids (correction.cu).

#include <cmath>
#include <vector>

#include "vsie_internal.h"

using namespace vsie;

extern "C" vsie_status vsie_scattered_field(vsie_handle* h, const void* d_p, int32_t nrhs, const double* h_points,
                                            int64_t m, int32_t precision, void* d_out, void* stream) {
  clear_error();
  TraceRange trace("vsie_scattered_field");
  if (!h || !d_p || !h_points || !d_out || m < 1 || nrhs < 1 ||
      (precision != 32 && precision != 48 && precision != 64)) {
    set_error("vsie_scattered_field: invalid argument (handle, buffers, m >= 1, nrhs >= 1, precision 32/48/64)");
    return VSIE_ERR_ARG;
  }
  for (int64_t r = 0; r < 3 * m; ++r)
    if (!std::isfinite(h_points[r])) {
      set_error("vsie_scattered_field: non-finite point coordinate");
      return VSIE_ERR_ARG;
    }
  cudaStream_t st = (cudaStream_t)stream;
  const double kap = h->k0 / (2.0 * kPi);
  std::vector<double4_32a> t64((size_t)m);
  std::vector<float4> t32((size_t)m), tdf(2 * (size_t)m);
  for (int64_t r = 0; r < m; ++r) {
    const double* X = h_points + 3 * r;
    t64[r] = make_double4_32a(X[0], X[1], X[2], 0.0);
    float hi[3], lo[3];
    for (int d = 0; d < 3; ++d) {
      const double v = kap * X[d];
      hi[d] = (float)v;
      lo[d] = (float)(v - (double)hi[d]);
    }
    t32[r] = make_float4(hi[0], hi[1], hi[2], 0.0f);
    tdf[2 * r] = t32[r];
    tdf[2 * r + 1] = make_float4(lo[0], lo[1], lo[2], 0.0f);
  }
  double4_32a* d64 = nullptr;
  float4 *d32 = nullptr, *ddf = nullptr;
  auto cleanup = [&]() {
    cudaFree(d64);
    cudaFree(d32);
    cudaFree(ddf);
  };
  cudaError_t e;
  if ((e = cudaMalloc(&d64, sizeof(double4_32a) * m)) != cudaSuccess ||
      (e = cudaMalloc(&d32, sizeof(float4) * m)) != cudaSuccess ||
      (e = cudaMalloc(&ddf, sizeof(float4) * 2 * m)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d64, t64.data(), sizeof(double4_32a) * m, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(d32, t32.data(), sizeof(float4) * m, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ddf, tdf.data(), sizeof(float4) * 2 * m, cudaMemcpyHostToDevice, st)) != cudaSuccess) {
    cleanup();
    return cuda_fail(e, "vsie_scattered_field: point upload", __FILE__, __LINE__);
  }
  const double2* p = (const double2*)d_p;
  double2* out = (double2*)d_out;
  vsie_status s = VSIE_OK;
  for (int c = 0; c < nrhs && s == VSIE_OK; ++c)
    s = far_sums_at(h, p + (size_t)c * h->n, d64, d32, ddf, m, out + (size_t)c * m, precision, st);
  if (s == VSIE_OK) s = field_correction(h, d64, m, p, nrhs, out, precision, st);
  if (s == VSIE_OK && (e = cudaStreamSynchronize(st)) != cudaSuccess)
    s = cuda_fail(e, "vsie_scattered_field", __FILE__, __LINE__);
  cleanup();
  return s;
}
