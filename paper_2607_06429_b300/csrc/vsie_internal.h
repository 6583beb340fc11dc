// Internal declarations of libvsie (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "vsie.h"

namespace vsie {

constexpr double kPi = 3.14159265358979323846;
constexpr double kFourPi = 4.0 * kPi;

// A named range on the host timeline for profilers (NVTX): it brackets one call of an
// entry point or one phase of it; without an attached tool the push and pop do nothing.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};

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

// Far-field source points, in three classes (one kernel each):
//   G: volume quadrature points whose density is locally constant (v = 0): weight s;
//   K: interface quadrature points (s = 0, v = sigma n with sigma = -omega w);
//   F: volume points with grad(alpha) != 0 (both s and v).
// Static FP64 data: pos_s = (x, y, z, s), vvec = (vx, vy, vz, 0) (K and F), and for K
// aux = (nx, ny, nz, sigma).  Per-apply records written by the prescale kernels, with
// positions scaled by kappa = k0/(2 pi) and the kappa powers folded into the charges:
//   G: (x, y, z, q.re) + q.im                       (r32a n, r32b n)
//   K: (x, y, z, c.re) (c.im, nx, ny, nz)           (r32a 2n)
//   F: (x, y, z, q.re) (q.im, ux.re, ux.im, uy.re) (uy.im, uz.re, uz.im, 0)  (r32a 3n)
// and the same layouts in FP64 (r64a, r64b).
struct Sources {
  int64_t n = 0;
  double4_32a* pos_s = nullptr;
  double4_32a* vvec = nullptr;
  double4_32a* aux = nullptr;
  int32_t* owner = nullptr;       // unknown index e(j)
  int32_t* elem_first = nullptr;  // point ranges per owning element (n_elem + 1)
  int32_t* elem_list = nullptr;   // owning unknown of each range
  int64_t n_elem = 0;
  float4* r32a = nullptr;
  float* r32b = nullptr;
  float4* rdf = nullptr;          // double-float records of the precision-48 sums (3 G, 4 K, 6 F)
  double4_32a* r64a = nullptr;
  double* r64b = nullptr;
  // adjoint target records (built on first adjoint call): (kappa y, s), (kappa v, 0)
  float4* adj_p32 = nullptr;
  float4* adj_v32 = nullptr;
  double4_32a* adj_p64 = nullptr;
  double4_32a* adj_v64 = nullptr;
};

struct Correction {
  int64_t nnz = 0;
  int64_t* row_ptr = nullptr;  // n + 1
  int32_t* col = nullptr;      // nnz
  // accurate - far-rule value as double-float complex (re.hi, im.hi, re.lo, im.lo)
  float4* val64 = nullptr;     // far rule from the FP64 coordinates
  float4* val32 = nullptr;     // far rule from the FP32-rounded coordinates
  float4* xd = nullptr;        // n: the applied vector in double-float (scratch)
};

// Per-call buffers of the adjoint far-field sum (allocated on the first adjoint call).
struct AdjRecords {
  float4* c_a32 = nullptr;   // collocation records (kappa x, c.re), c = kappa conj(lam)/(4 pi)
  float* c_b32 = nullptr;
  double4_32a* c_a64 = nullptr;
  double* c_b64 = nullptr;
  double2* w = nullptr;      // per-source-point sums
  // target records of the gradient-channel passes (built per pass)
  float4* ch_p32 = nullptr;
  float4* ch_v32 = nullptr;
  double4_32a* ch_p64 = nullptr;
  double4_32a* ch_v64 = nullptr;
  double2* ch_out = nullptr;   // one-pass FP32 channels: 4 sums per source point (Phi, Psi x, y, z)
};

// Buffers of the tensor-core multi-RHS path (grown on demand).
struct BatchBuffers {
  unsigned char* img = nullptr;  // per-source-tile images (records + tf32 charge operands)
  size_t img_bytes = 0;
  double* slots = nullptr;       // per-CTA FP64 accumulators / partial tiles of the fix-up
  size_t slot_elems = 0;
  int* status = nullptr;         // set by a timed-out mbarrier wait
  float4* q64 = nullptr;         // FP64 multi-RHS charges [source][64] (double-float)
  size_t q64_elems = 0;
  double2* part64 = nullptr;     // FP64 multi-RHS partial sums of the source splits
  size_t part64_elems = 0;
  unsigned char* xt = nullptr;   // row-major charge block of the block correction
  size_t xt_bytes = 0;
};

// Uniform cell grid over element centroids (cell >= the search radius); elements sorted
// by cell.  Points outside the box clamp to its boundary cells, which still finds every
// element within one cell of them.
struct CellGrid {
  double lo[3] = {0, 0, 0};
  double inv = 0;   // 1 / cell size
  int nc[3] = {0, 0, 0};
  int64_t ncell = 0;
  const int32_t* order = nullptr;   // element ids sorted by cell
  const int64_t* start = nullptr;   // ncell + 1
};

// Geometry of the near-field rules (device arrays, kept for the life of the handle) and the
// targets whose correction rows are built: the collocation points (self = 1: a target is
// its own element's centroid) or arbitrary field points (self = 0).
struct CorrInputs {
  const double4_32a* tgt = nullptr;       // n targets
  const double4_32a* tet_cen = nullptr;   // n_tet
  const double4_32a* tet_pts = nullptr;   // 4 n_tet
  const double* tet_s = nullptr;
  const double4_32a* tet_ga = nullptr;
  const double* tet_vol = nullptr;
  const double4_32a* tri_vtx = nullptr;   // 3 n_tri
  const double4_32a* tri_pts = nullptr;   // 3 n_tri
  const double4_32a* tri_cen = nullptr;   // n_tri
  const double4_32a* tri_nrm = nullptr;   // (n, area)
  const double* tri_omega = nullptr;
  int64_t n_tet = 0, n_tri = 0, n = 0;
  int far_points = 1;
  int self = 1;
  double R2v = 0, R2t = 0;          // squared radii (0 = inactive)
  double k = 0;
  CellGrid gv, gt;
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
  int debug_flags = 0;

  double4_32a* tgt64 = nullptr;   // (x, y, z, 0) collocation points, FP64
  float4* tgt32 = nullptr;    // FP32 copies of kappa * x (kappa = k0/(2 pi))
  float4* tgtdf = nullptr;    // double-float kappa * x: (hi, hi, hi, 0) (lo, lo, lo, 0) per point
  double* mass = nullptr;     // mass function m at the collocation points

  vsie::Sources G, K, F;
  vsie::Correction C;
  vsie::CorrInputs geo;       // near-rule geometry and neighbour grids (field evaluation)

  // library-owned scratch
  double2* host_x = nullptr;  // device staging of vsie_apply_host
  double2* host_y = nullptr;
  int64_t host_cols = 0;
  double2* split = nullptr;   // per-block partial-tile slots of the far-field kernels
  size_t split_elems = 0;
  vsie::AdjRecords adj;
  vsie::BatchBuffers batch;
  // work shapes chosen by vsie_autotune (0 = built-in default)
  struct {
    int chunk[3] = {0, 0, 0};  // FP32 far sums (G, K, F): sources per work item
    int bps[3] = {0, 0, 0};    // FP32 far sums: resident blocks per SM
    int bt_chunk_tiles = 0;    // tensor-core batched sums: 32-source tiles per work item
    int gk_bps[2] = {0, 0};    // FP32 G and K sums run concurrently with these blocks per SM
                               // each (0: one after the other)
  } tune;
  // concurrent G and K sums: the K sum's stream, fork/join events, output and slots
  cudaStream_t gk_stream = nullptr;
  cudaEvent_t gk_fork = nullptr, gk_join = nullptr;
  double2* gk_y = nullptr;
  int64_t gk_y_n = 0;
  double2* gk_split = nullptr;
  size_t gk_split_elems = 0;

  std::vector<void*> allocs;  // every device allocation, freed by vsie_destroy

  // the creation inputs (host copies), from which vsie_set_frequency rebuilds the operator
  struct {
    int kind = 0;  // 0: tetrahedra and triangles (vsie_create); 1: cuboid grid (vsie_create_cuboid)
    std::vector<double> vert, rho, c, grad_alpha, tri_rho_in, tri_rho_out;
    std::vector<int32_t> tet, tri;
    std::vector<double> x_edges, y_edges, z_edges;
    bool has_opt = false, has_grad_alpha = false;
    vsie_options opt{};
  } inputs;
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
// Field points (not collocation points): y_r = -(y_r + sum_k Delta(X_r, k) x_k) for each of
// the nrhs columns (x: n x nrhs, y: m x nrhs), Delta = near-rule minus far-rule values at
// the points X (the near sets of the create-time radii, no self terms).  Builds the rows
// with the handle's geometry, applies them and frees them; blocking.
vsie_status field_correction(vsie_handle* h, const double4_32a* d_pts, int64_t m, const double2* x,
                             int nrhs, double2* y, int precision, cudaStream_t st);

// Far-field sums at m arbitrary points: y_r = sum_j C(X_r, y_j) p_e(j) (t64: (x, y, z, 0),
// t32: float(kappa X), tdf: double-float kappa X as (hi, lo) float4 pairs; the one of the
// precision used is read).  x: n.  Asynchronous on st.
vsie_status far_sums_at(vsie_handle* h, const double2* x, const double4_32a* t64, const float4* t32,
                        const float4* tdf, int64_t m, double2* y, int precision, cudaStream_t st);
// Far-field sums: y (+)= sum_j C(x_i, y_j) p_e(j) over the far-field source points.
vsie_status far_apply(vsie_handle* h, const double2* x, double2* y, int precision,
                      cudaStream_t st);
// The phases of far_apply (launch counters optional): prescale; the volume (G) sum;
// the interface (K) and heterogeneous-volume (F) sums.
vsie_status far_prescale(vsie_handle* h, const double2* x, int precision, cudaStream_t st,
                         int* launches);
vsie_status far_sum_g(vsie_handle* h, double2* y, int precision, cudaStream_t st, int* launches);
vsie_status far_sum_f(vsie_handle* h, double2* y, int precision, cudaStream_t st, int* launches);
// All far-field sums with the partial-tile slots in caller-provided scratch; the scratch
// must hold far_split_elems(h, precision) double2 values (nothing is allocated).
size_t far_split_elems(const vsie_handle* h, int precision);
// Looks up (and caches) the device address of the allocation-free apply's fixed array on
// the given device; called once an operator exists there.
void noalloc_prepare(int device);
vsie_status far_sums_into(vsie_handle* h, double2* y, int precision, double2* scratch,
                          cudaStream_t st);
// x_e = sum_{j in e} sum_i conj(C_ij) lam_i (overwrites x).
vsie_status far_adjoint(vsie_handle* h, const double2* lam, double2* x, int precision,
                        cudaStream_t st);
// y += m x + Delta x  (Delta for the given precision's far sum)
vsie_status correction_apply(vsie_handle* h, const double2* x, double2* y, int precision,
                             cudaStream_t st);
// rows [r0, r1) only: y_out[i - r0] += m_i x_i + (Delta x)_i  (x: all n unknowns)
vsie_status correction_apply_rows(vsie_handle* h, const double2* x, double2* y_out, int64_t r0, int64_t r1,
                                  int precision, cudaStream_t st);
// y[:, r] += m x[:, r] + Delta x[:, r] for ncols columns (n x ncols column-major), 64 at a
// time with one pass over the correction matrix per 64 columns
vsie_status correction_apply_block(vsie_handle* h, const double2* x, double2* y, int ncols, int precision,
                                   cudaStream_t st);
// Gradient channels at every far-field source point (classes G, K, F in order):
// phi_j = sum_i conj(G(x_i, y_j)) lam_i, psi_j = sum_i conj(grad_x G(x_i, y_j)) lam_i (3 per point)
vsie_status gradient_channels(vsie_handle* h, const double2* lam, int precision, double2* phi, double2* psi,
                              cudaStream_t st);
// x += conj(m) lam + Delta^H lam
vsie_status correction_adjoint(vsie_handle* h, const double2* lam, double2* x,
                               int precision, cudaStream_t st);

// y = A x at the given precision (an operator for the generic GMRES driver)
using ApplyFn = std::function<vsie_status(const double2* x, double2* y, int precision)>;
// GMRES (x0 = 0, or the iterate in x with opts->initial_guess) with, in mode 32, FP64
// iterative refinement: inner cycles with the inner_prec apply, true residuals with the
// res_prec apply; who names the entry point in error messages.  Blocking.
vsie_status gmres_solve(int64_t n, const ApplyFn& apply, const double2* b, double2* x,
                        const vsie_solve_opts* opts, vsie_solve_info* info, cudaStream_t st, int inner_prec,
                        int res_prec, const char* who);
vsie_status apply_one(vsie_handle* h, const double2* x, double2* y, int precision,
                      cudaStream_t st);

// Far-field sums over the G and K classes for nrhs columns on the tensor cores (FP32 tile
// evaluation, three-term TF32 contraction); y is overwritten.  batch_status reads (and
// clears) the timeout flag of those kernels, synchronising the stream.
vsie_status far_batched_gk(vsie_handle* h, const double2* x, double2* y, int nrhs, cudaStream_t st);
// The same for nop operators of equal work shape (one persistent launch per class and
// 64-column block for up to 16 operators); x[p], y[p] are operator p's blocks.
vsie_status far_batched_gk_multi(vsie_handle* const* hs, int nop, const double2* const* x, double2* const* y,
                                 int nrhs, cudaStream_t st);
vsie_status batch_status(vsie_handle* h, cudaStream_t st);
// The FP32 multi-operator batched apply without the final timeout-flag check (no host
// synchronisation, no allocation once the buffers exist: capturable in a CUDA graph), and
// the argument check shared by its entry points.
vsie_status check_multi_args(vsie_handle* const* hs, int32_t nop, const void* const* x, void* const* y,
                             int32_t nrhs, const char* who);
vsie_status apply_batched_multi_launch(vsie_handle* const* hs, int nop, const double2* const* x,
                                       double2* const* y, int nrhs, cudaStream_t st);
// The same sums in FP64 on the CUDA cores (each coefficient evaluated once per block of 64
// columns); y is overwritten.
vsie_status far_batched64_gk(vsie_handle* h, const double2* x, double2* y, int nrhs, cudaStream_t st);
// Autotuning of the FP32 far sums' work shapes (sets h->tune; x is a random vector,
// scratch holds n values): chosen (chunk, blocks per SM) and (chosen, default) times per class.
vsie_status far_autotune(vsie_handle* h, const double2* x, double2* scratch, cudaStream_t st, int cand_out[3][2],
                         double ms_out[3][2], int* candidates);
// Then the choice between the G and K sums one after the other and concurrently (resident
// blocks per SM split between them), timed on a target sample: sets h->tune.gk_bps;
// (chosen, sequential) times.
vsie_status far_autotune_gk(vsie_handle* h, const double2* x, double2* scratch, cudaStream_t st, int out_bps[2],
                            double out_ms[2], int* candidates);
// Sets the concurrent G and K sums with gbps and kbps resident blocks per SM (clamped to the
// kernels' occupancy), allocating their buffers; 0, 0: the sums one after the other.
vsie_status far_set_gk(vsie_handle* h, int gbps, int kbps);
// Kernels vsie_apply launches beyond the sequential sums' count (1 with the concurrent sums:
// the join's addition).
int far_gk_extra_launches(const vsie_handle* h, int precision);
// The same for the tensor-core batched sums' source tiles per work item (x: a block of 64
// random columns, y: n x 64 scratch).
vsie_status batch_autotune(vsie_handle* h, const double2* x, double2* y, cudaStream_t st, int* chunk_tiles,
                           double ms_out[2], int* candidates);
// Far-field sum of the F class only (added into y), for one column.
vsie_status far_sum_f_only(vsie_handle* h, const double2* x, double2* y, int precision, cudaStream_t st);


}  // namespace vsie
