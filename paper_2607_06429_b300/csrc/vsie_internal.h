// Internal declarations of libvsie (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "vsie.h"

namespace vsie {

constexpr double kPi = 3.14159265358979323846;
constexpr double kFourPi = 4.0 * kPi;

// Thread-local error text behind vsie_last_error().
void set_error(const std::string& msg);
void clear_error();

// Record a CUDA failure (with call site) and return VSIE_ERR_CUDA / VSIE_ERR_OOM.
vsie_status cuda_fail(cudaError_t e, const char* what, const char* file, int line);

#define VSIE_CUDA(call)                                                     \
  do {                                                                      \
    cudaError_t _e = (call);                                                \
    if (_e != cudaSuccess) return ::vsie::cuda_fail(_e, #call, __FILE__, __LINE__); \
  } while (0)

#define VSIE_TRY(call)                     \
  do {                                     \
    vsie_status _s = (call);               \
    if (_s != VSIE_OK) return _s;          \
  } while (0)

// Far-field source records.  Sources come in two classes:
//   G: volume quadrature points whose density is locally constant (v = 0): weight s only;
//   F: points with a vector weight v (interface points, and volume points with
//      grad(alpha) != 0), which may also carry s.
// Charges per apply: q = -s p/(4 pi) (complex), u = v p/(4 pi) (complex 3-vector).
// FP32 records (written per apply by the prescale kernels):
//   G: float4 (x, y, z, q.re) + float q.im
//   F: 3 x float4 (x, y, z, q.re) (q.im, ux.re, ux.im, uy.re) (uy.im, uz.re, uz.im, 0)
// FP64 records: the same layouts with double4_32a / double.
struct Sources {
  int64_t n = 0;
  double4_32a* pos_s = nullptr;   // (x, y, z, s) FP64, static
  double4_32a* vvec = nullptr;    // (vx, vy, vz, 0) FP64, static (class F only)
  int32_t* owner = nullptr;   // unknown index e(j)
  int32_t* elem_first = nullptr;  // CSR-like point ranges per owning element (adjoint)
  int32_t* elem_list = nullptr;   // owning unknown of each range
  int64_t n_elem = 0;
  // per-apply records
  float4* r32a = nullptr;     // G: n records; F: 3n records
  float* r32b = nullptr;      // G: q.im
  double4_32a* r64a = nullptr;
  double* r64b = nullptr;
};

struct Correction {
  int64_t nnz = 0;
  int64_t* row_ptr = nullptr;  // n + 1
  int32_t* col = nullptr;      // nnz
  double2* val64 = nullptr;    // accurate - far-rule value (FP64 coordinates)
  double2* val32 = nullptr;    // accurate - far-rule value (FP32-rounded coordinates)
};

// Static point records and per-call buffers of the adjoint far-field sum (built on
// first use).
struct AdjRecords {
  float4* g_p32 = nullptr;
  float4* f_p32 = nullptr;
  float4* f_v32 = nullptr;
  float4* c_a32 = nullptr;
  float* c_b32 = nullptr;
  double4_32a* c_a64 = nullptr;
  double* c_b64 = nullptr;
  double2* w = nullptr;
};

}  // namespace vsie

struct vsie_handle {
  int device = 0;
  int num_sms = 0;
  int64_t n_tet = 0, n_tri = 0, n = 0;
  double k0 = 0, rho0 = 1, c0 = 1;
  int far_points = 1;
  double near_radius = 0, tri_near_radius = 0;
  int tile_override = 0;

  double4_32a* tgt64 = nullptr;   // (x, y, z, 0) collocation points, FP64
  float4* tgt32 = nullptr;    // FP32-rounded copies
  double* mass = nullptr;     // mass function m at the collocation points

  vsie::Sources G, F;
  vsie::Correction C;

  // library-owned scratch
  double2* host_x = nullptr;  // device staging of vsie_apply_host
  double2* host_y = nullptr;
  int64_t host_cols = 0;
  double2* split = nullptr;   // source-split partial sums of the far-field kernels
  size_t split_elems = 0;
  vsie::AdjRecords adj;

  std::vector<void*> allocs;  // every device allocation, freed by vsie_destroy
};

namespace vsie {

vsie_status dalloc(vsie_handle* h, void** p, size_t bytes);
template <class T>
vsie_status dalloc_t(vsie_handle* h, T** p, size_t count) {
  return dalloc(h, reinterpret_cast<void**>(p), count * sizeof(T));
}

// Near-field / self correction matrix (built on the device at create time; blocking).
vsie_status build_correction(vsie_handle* h, const double4_32a* d_tet_cen,
                             const double4_32a* d_tet_pts /*4 per tet*/,
                             const double* d_tet_s /*(beta-k0^2 alpha) per tet*/,
                             const double4_32a* d_tet_ga /*grad alpha per tet*/,
                             const double* d_tet_vol, const double4_32a* d_tri_vtx /*3 per tri*/,
                             const double4_32a* d_tri_pts /*3 per tri*/, const double4_32a* d_tri_cen,
                             const double4_32a* d_tri_nrm /*(n, area)*/, const double* d_tri_omega,
                             const double lo[3], const double hi[3]);

// Far-field sums: y (+)= sum_j C(x_i, y_j) p_e(j) over the far-field source points.
vsie_status far_apply(vsie_handle* h, const double2* x, double2* y, int precision,
                      cudaStream_t st);
// The three phases of far_apply (launch counters optional).
vsie_status far_prescale(vsie_handle* h, const double2* x, int precision, cudaStream_t st,
                         int* launches);
vsie_status far_sum_g(vsie_handle* h, double2* y, int precision, cudaStream_t st, int* launches);
vsie_status far_sum_f(vsie_handle* h, double2* y, int precision, cudaStream_t st, int* launches);
// Both far-field sums with source-split partials in caller-provided scratch; the scratch
// must hold far_split_elems(h) double2 values (nothing is allocated).
size_t far_split_elems(const vsie_handle* h);
vsie_status far_sums_into(vsie_handle* h, double2* y, int precision, double2* scratch,
                          cudaStream_t st);
// x_e = sum_{j in e} sum_i conj(C_ij) lam_i (overwrites x).
vsie_status far_adjoint(vsie_handle* h, const double2* lam, double2* x, int precision,
                        cudaStream_t st);
// y += m x + Delta x  (Delta for the given precision's far sum)
vsie_status correction_apply(vsie_handle* h, const double2* x, double2* y, int precision,
                             cudaStream_t st);
// x += conj(m) lam + Delta^H lam
vsie_status correction_adjoint(vsie_handle* h, const double2* lam, double2* x,
                               int precision, cudaStream_t st);

vsie_status apply_one(vsie_handle* h, const double2* x, double2* y, int precision,
                      cudaStream_t st);


}  // namespace vsie
