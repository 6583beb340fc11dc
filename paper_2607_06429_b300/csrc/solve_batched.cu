// Lockstep GMRES for a block of right-hand sides: the same systems as vsie_solve (Sec. 3.1:
// GMRES from x0 = 0, no preconditioner, relative residual tolerance), one per column, with
// every operator application shared by the whole block.
//
//   mode 32: FP64 iterative refinement (true residual b - A x with the FP64 apply) around
//            inner GMRES cycles whose operator is the tensor-core multi-RHS FP32 apply,
//            one call for all active columns per Arnoldi step;
//   mode 64: FP64 GMRES with the FP64 multi-RHS apply (the plain FP64 solver run on the
//            same block, for time-to-solution comparisons).
//
// Each column keeps its own Krylov basis, Hessenberg matrix and Givens rotations; a column
// leaves the active set of a cycle when its residual estimate meets its target.  Arnoldi is
// CGS2 as in the single-column solver, with the multi-dot, update and scaling kernels
// batched over the active columns (grid.y = column) and one host synchronisation per step.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "vsie_internal.h"

namespace vsie {

namespace {

using cplx = std::complex<double>;

constexpr int kBThreads = 256;
constexpr int kMaxBasis = 1000;  // Krylov basis limit of the batched solver (host Hessenberg memory)

inline unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }

// partial[(y k + i) nbx + bx] = sum over slice bx of conj(v_i) w, for the k vectors
// v_i = V + col(y) ldc + i ldv of column slot y (col(y) = act[y], or y when act is null)
// and w = W + y ldw.
__global__ void __launch_bounds__(kBThreads) bmultidot_kernel(const double2* __restrict__ V, int64_t ldc,
                                                              int64_t ldv, int k, const int* __restrict__ act,
                                                              const double2* __restrict__ W, int64_t ldw,
                                                              int64_t n, double2* __restrict__ partial) {
  __shared__ double red[2][kBThreads / 32];
  const int nbx = gridDim.x, bx = blockIdx.x, y = blockIdx.y;
  const int64_t c = act ? act[y] : y;
  const int64_t per = (n + nbx - 1) / nbx;
  const int64_t i0 = (int64_t)bx * per, i1 = min(n, i0 + per);
  const double2* w = W + (int64_t)y * ldw;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int i = 0; i < k; ++i) {
    const double2* v = V + c * ldc + (int64_t)i * ldv;
    double ar = 0.0, ai = 0.0;
    for (int64_t t = i0 + threadIdx.x; t < i1; t += kBThreads) {
      const double2 a = v[t], b = w[t];
      ar += a.x * b.x + a.y * b.y;
      ai += a.x * b.y - a.y * b.x;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ar += __shfl_down_sync(0xffffffffu, ar, o);
      ai += __shfl_down_sync(0xffffffffu, ai, o);
    }
    if (lane == 0) {
      red[0][wid] = ar;
      red[1][wid] = ai;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      double sr = 0.0, si = 0.0;
      for (int q = 0; q < kBThreads / 32; ++q) {
        sr += red[0][q];
        si += red[1][q];
      }
      partial[((int64_t)y * k + i) * nbx + bx] = make_double2(sr, si);
    }
    __syncthreads();
  }
}

// out[t] = sum_b partial[t nbx + b] (fixed order), t < count
__global__ void breduce_kernel(const double2* __restrict__ partial, int nbx, int count, double2* __restrict__ out) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= count) return;
  double sr = 0.0, si = 0.0;
  for (int b = 0; b < nbx; ++b) {
    const double2 v = partial[(int64_t)t * nbx + b];
    sr += v.x;
    si += v.y;
  }
  out[t] = make_double2(sr, si);
}

// w_y -= sum_{i < k} v_i h[y k + i]   (the vectors of column act[y])
__global__ void bupdate_kernel(const double2* __restrict__ V, int64_t ldc, int64_t ldv, int k,
                               const int* __restrict__ act, const double2* __restrict__ hcoef,
                               double2* __restrict__ W, int64_t ldw, int64_t n) {
  extern __shared__ double2 hs[];
  const int y = blockIdx.y;
  for (int i = threadIdx.x; i < k; i += blockDim.x) hs[i] = hcoef[(int64_t)y * k + i];
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t c = act[y];
  double2* w = W + (int64_t)y * ldw;
  double2 acc = w[t];
  for (int i = 0; i < k; ++i) {
    const double2 v = V[c * ldc + (int64_t)i * ldv + t];
    const double2 q = hs[i];
    acc.x -= v.x * q.x - v.y * q.y;
    acc.y -= v.x * q.y + v.y * q.x;
  }
  w[t] = acc;
}

// dst[dcol(y) ldd + doff + t] = s[y] * src[scol(y) lds + soff + t]   (index arrays may be null: y)
__global__ void bcopy_scaled_kernel(const double2* __restrict__ src, int64_t lds, int64_t soff,
                                    const int* __restrict__ sidx, const double* __restrict__ s,
                                    double2* __restrict__ dst, int64_t ldd, int64_t doff,
                                    const int* __restrict__ didx, int64_t n) {
  const int y = blockIdx.y;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t sc = sidx ? sidx[y] : y, dc = didx ? didx[y] : y;
  const double f = s ? s[y] : 1.0;
  const double2 v = src[sc * lds + soff + t];
  dst[dc * ldd + doff + t] = make_double2(v.x * f, v.y * f);
}

// x_{col(y)} += sum_{i < kk[y]} v_i coef[y kmax + i]
__global__ void bcombine_kernel(const double2* __restrict__ V, int64_t ldc, int64_t ldv, const int* __restrict__ col,
                                const int* __restrict__ kk, int kmax, const double2* __restrict__ coef,
                                double2* __restrict__ X, int64_t ldx, int64_t n) {
  extern __shared__ double2 cs[];
  const int y = blockIdx.y, k = kk[y];
  for (int i = threadIdx.x; i < k; i += blockDim.x) cs[i] = coef[(int64_t)y * kmax + i];
  __syncthreads();
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t c = col[y];
  double2 acc = X[c * ldx + t];
  for (int i = 0; i < k; ++i) {
    const double2 v = V[c * ldc + (int64_t)i * ldv + t];
    const double2 q = cs[i];
    acc.x += v.x * q.x - v.y * q.y;
    acc.y += v.x * q.y + v.y * q.x;
  }
  X[c * ldx + t] = acc;
}

// r_{col(y)} = b_{col(y)} - t_y
__global__ void bresidual_kernel(const double2* __restrict__ B, const double2* __restrict__ T,
                                 const int* __restrict__ col, double2* __restrict__ R, int64_t n) {
  const int y = blockIdx.y;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int64_t c = col[y];
  const double2 b = B[c * n + t], v = T[(int64_t)y * n + t];
  R[c * n + t] = make_double2(b.x - v.x, b.y - v.y);
}

// host-side GMRES state of one column within a cycle
struct Column {
  int c = 0;                            // right-hand side index
  double target = 0.0;                  // absolute residual target of the cycle
  int limit = 0;                        // Arnoldi steps allowed in the cycle
  std::vector<std::vector<cplx>> R;     // rotated Hessenberg columns (upper triangle)
  std::vector<cplx> cs, sn, g;
  int k = 0;                            // steps taken
  double res = 0.0;
  bool breakdown = false;
};

struct Work {
  int64_t n = 0;
  int R = 0, m = 0;
  double2* V = nullptr;     // R x (m + 1) x n bases
  double2* X = nullptr;     // n x R gathered operator inputs
  double2* W = nullptr;     // n x R operator outputs / Arnoldi vectors
  double2* r = nullptr;     // n x R residuals
  double2* partial = nullptr;
  int nbx = 0;
  double2* h1 = nullptr;    // R x (m + 1)
  double2* h2 = nullptr;
  double2* nrm = nullptr;   // R
  int* idx_a = nullptr;     // R (active columns)
  int* idx_b = nullptr;     // R (source slots)
  int* idx_k = nullptr;     // R
  double* scale = nullptr;  // R
  double2* coef = nullptr;  // R x m
  double2* hbuf = nullptr;  // pinned host copy of h1, h2, nrm
};

// squared norms of the a columns W + y ldw -> host (synchronises)
vsie_status batched_norms(Work& S, const double2* W, int64_t ldw, int a, std::vector<double>& out,
                          cudaStream_t st) {
  bmultidot_kernel<<<dim3(S.nbx, a), kBThreads, 0, st>>>(W, ldw, 0, 1, nullptr, W, ldw, S.n, S.partial);
  breduce_kernel<<<(a + 127) / 128, 128, 0, st>>>(S.partial, S.nbx, a, S.nrm);
  VSIE_CUDA(cudaGetLastError());
  VSIE_CUDA(cudaMemcpyAsync(S.hbuf, S.nrm, sizeof(double2) * a, cudaMemcpyDeviceToHost, st));
  VSIE_CUDA(cudaStreamSynchronize(st));
  out.resize(a);
  for (int y = 0; y < a; ++y) out[y] = std::sqrt(std::max(S.hbuf[y].x, 0.0));
  return VSIE_OK;
}

// W[:, y] = A X[:, y] for a columns in the given precision, with the multi-RHS far-field
// sums (FP32: tensor cores; FP64: CUDA cores).  A block of 64 columns costs about as much
// as four (FP32) or five (FP64) single-column applies, so smaller sets of columns go
// through the single-column apply instead.
constexpr int kBatchMin32 = 4;
constexpr int kBatchMin64 = 5;

vsie_status block_apply(vsie_handle* h, const double2* X, double2* W, int a, int precision, cudaStream_t st,
                        vsie_solve_info* infos, const std::vector<int>& cols) {
  const int64_t n = h->n;
  if (a >= (precision == 32 ? kBatchMin32 : kBatchMin64)) {
    if (precision == 32)
      VSIE_TRY(far_batched_gk(h, X, W, a, st));
    else
      VSIE_TRY(far_batched64_gk(h, X, W, a, st));
    if (h->F.n)
      for (int y = 0; y < a; ++y)
        VSIE_TRY(far_sum_f_only(h, X + (size_t)y * n, W + (size_t)y * n, precision, st));
    VSIE_TRY(correction_apply_block(h, X, W, a, precision, st));
    if (precision == 32) VSIE_TRY(batch_status(h, st));
  } else {
    for (int y = 0; y < a; ++y) VSIE_TRY(apply_one(h, X + (size_t)y * n, W + (size_t)y * n, precision, st));
  }
  if (infos)
    for (int y = 0; y < a; ++y) {
      if (precision == 32)
        infos[cols[y]].fp32_applies += 1;
      else
        infos[cols[y]].fp64_applies += 1;
    }
  return VSIE_OK;
}

// One GMRES cycle for the given columns from d = 0 on A d = r_c (d is added to x_c).
vsie_status batched_cycle(vsie_handle* h, int precision, std::vector<Column>& cols, const std::vector<double>& r0n,
                          double2* x, Work& S, cudaStream_t st, vsie_solve_info* infos) {
  const int64_t n = S.n, ldc = (int64_t)(S.m + 1) * n;
  std::vector<int> act;  // positions in cols of the active columns
  std::vector<int> colid, srcslot;
  std::vector<double> sc;
  for (size_t q = 0; q < cols.size(); ++q) {
    Column& C = cols[q];
    C.R.clear();
    C.cs.assign(C.limit, 0.0);
    C.sn.assign(C.limit, 0.0);
    C.g.assign(C.limit + 1, 0.0);
    C.g[0] = r0n[q];
    C.k = 0;
    C.res = r0n[q];
    C.breakdown = false;
    if (C.limit > 0) {
      act.push_back((int)q);
      colid.push_back(C.c);
      sc.push_back(1.0 / r0n[q]);
    }
  }
  int a = (int)act.size();
  if (a > 0) {
    // v_0 = r_c / |r_c|
    VSIE_CUDA(cudaMemcpyAsync(S.idx_a, colid.data(), sizeof(int) * a, cudaMemcpyHostToDevice, st));
    VSIE_CUDA(cudaMemcpyAsync(S.scale, sc.data(), sizeof(double) * a, cudaMemcpyHostToDevice, st));
    bcopy_scaled_kernel<<<dim3(nb256(n), a), 256, 0, st>>>(S.r, n, 0, S.idx_a, S.scale, S.V, ldc, 0, S.idx_a, n);
    VSIE_CUDA(cudaGetLastError());
  }
  std::vector<int> cur_cols;
  for (int j = 0; a > 0; ++j) {
    cur_cols.assign(colid.begin(), colid.end());
    const int k = j + 1;
    // gather v_j of the active columns, apply the operator
    bcopy_scaled_kernel<<<dim3(nb256(n), a), 256, 0, st>>>(S.V, ldc, (int64_t)j * n, S.idx_a, nullptr, S.X, n, 0,
                                                           nullptr, n);
    VSIE_CUDA(cudaGetLastError());
    VSIE_TRY(block_apply(h, S.X, S.W, a, precision, st, infos, cur_cols));
    // CGS2: two passes of h = V^H w, w -= V h; then |w|
    for (int pass = 0; pass < 2; ++pass) {
      double2* hd = pass ? S.h2 : S.h1;
      bmultidot_kernel<<<dim3(S.nbx, a), kBThreads, 0, st>>>(S.V, ldc, n, k, S.idx_a, S.W, n, n, S.partial);
      breduce_kernel<<<(a * k + 127) / 128, 128, 0, st>>>(S.partial, S.nbx, a * k, hd);
      bupdate_kernel<<<dim3(nb256(n), a), 256, sizeof(double2) * k, st>>>(S.V, ldc, n, k, S.idx_a, hd, S.W, n, n);
      VSIE_CUDA(cudaGetLastError());
    }
    bmultidot_kernel<<<dim3(S.nbx, a), kBThreads, 0, st>>>(S.W, n, 0, 1, nullptr, S.W, n, n, S.partial);
    breduce_kernel<<<(a + 127) / 128, 128, 0, st>>>(S.partial, S.nbx, a, S.nrm);
    VSIE_CUDA(cudaGetLastError());
    double2* hb1 = S.hbuf;
    double2* hb2 = S.hbuf + (size_t)a * k;
    double2* hbn = S.hbuf + (size_t)2 * a * k;
    VSIE_CUDA(cudaMemcpyAsync(hb1, S.h1, sizeof(double2) * a * k, cudaMemcpyDeviceToHost, st));
    VSIE_CUDA(cudaMemcpyAsync(hb2, S.h2, sizeof(double2) * a * k, cudaMemcpyDeviceToHost, st));
    VSIE_CUDA(cudaMemcpyAsync(hbn, S.nrm, sizeof(double2) * a, cudaMemcpyDeviceToHost, st));
    VSIE_CUDA(cudaStreamSynchronize(st));
    std::vector<int> next_act, next_col, next_src;
    std::vector<double> next_sc;
    for (int y = 0; y < a; ++y) {
      Column& C = cols[act[y]];
      const double beta = std::sqrt(std::max(hbn[y].x, 0.0));
      if (!std::isfinite(beta)) {
        set_error("vsie_solve_batched: non-finite value in the Arnoldi process");
        return VSIE_ERR_NAN;
      }
      std::vector<cplx> col(k + 1);
      for (int i = 0; i < k; ++i)
        col[i] = cplx(hb1[(size_t)y * k + i].x + hb2[(size_t)y * k + i].x,
                      hb1[(size_t)y * k + i].y + hb2[(size_t)y * k + i].y);
      col[k] = beta;
      for (int i = 0; i < j; ++i) {
        const cplx p = col[i], q = col[i + 1];
        col[i] = std::conj(C.cs[i]) * p + std::conj(C.sn[i]) * q;
        col[i + 1] = -C.sn[i] * p + C.cs[i] * q;
      }
      const cplx p = col[j];
      const double bb = std::abs(col[j + 1]);
      const double den = std::sqrt(std::norm(p) + bb * bb);
      if (den == 0.0) {
        C.cs[j] = 1.0;
        C.sn[j] = 0.0;
      } else {
        C.cs[j] = p / den;
        C.sn[j] = col[j + 1] / den;
      }
      col[j] = den;
      col.resize(k);
      C.R.push_back(std::move(col));
      C.g[j + 1] = -C.sn[j] * C.g[j];
      C.g[j] = std::conj(C.cs[j]) * C.g[j];
      C.res = std::abs(C.g[j + 1]);
      C.k = k;
      bool finish = false;
      if (beta == 0.0) {
        C.breakdown = C.res > C.target;
        finish = true;
      } else if (C.res <= C.target || k >= C.limit) {
        finish = true;
      }
      if (!finish) {
        next_act.push_back(act[y]);
        next_col.push_back(C.c);
        next_src.push_back(y);
        next_sc.push_back(1.0 / beta);
      }
    }
    const int a2 = (int)next_act.size();
    if (a2 > 0) {
      // v_{j+1} = w / beta for the columns that continue
      VSIE_CUDA(cudaMemcpyAsync(S.idx_a, next_col.data(), sizeof(int) * a2, cudaMemcpyHostToDevice, st));
      VSIE_CUDA(cudaMemcpyAsync(S.idx_b, next_src.data(), sizeof(int) * a2, cudaMemcpyHostToDevice, st));
      VSIE_CUDA(cudaMemcpyAsync(S.scale, next_sc.data(), sizeof(double) * a2, cudaMemcpyHostToDevice, st));
      bcopy_scaled_kernel<<<dim3(nb256(n), a2), 256, 0, st>>>(S.W, n, 0, S.idx_b, S.scale, S.V, ldc,
                                                              (int64_t)(j + 1) * n, S.idx_a, n);
      VSIE_CUDA(cudaGetLastError());
    }
    act.swap(next_act);
    colid.swap(next_col);
    a = a2;
  }
  // back substitution R y = g per column, then x_c += V_c y
  std::vector<int> ccol, ck;
  std::vector<double2> coef((size_t)cols.size() * std::max(1, S.m));
  int kmax = 0;
  for (const Column& C : cols) kmax = std::max(kmax, C.k);
  if (kmax == 0) return VSIE_OK;
  for (const Column& C : cols) {
    if (C.k == 0) continue;
    std::vector<cplx> yv(C.k);
    for (int i = C.k - 1; i >= 0; --i) {
      cplx acc = C.g[i];
      for (int c2 = i + 1; c2 < C.k; ++c2) acc -= C.R[c2][i] * yv[c2];
      yv[i] = acc / C.R[i][i];
    }
    const size_t y = ccol.size();
    for (int i = 0; i < C.k; ++i) coef[y * kmax + i] = make_double2(yv[i].real(), yv[i].imag());
    ccol.push_back(C.c);
    ck.push_back(C.k);
  }
  const int nc = (int)ccol.size();
  VSIE_CUDA(cudaMemcpyAsync(S.idx_a, ccol.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st));
  VSIE_CUDA(cudaMemcpyAsync(S.idx_k, ck.data(), sizeof(int) * nc, cudaMemcpyHostToDevice, st));
  VSIE_CUDA(cudaMemcpyAsync(S.coef, coef.data(), sizeof(double2) * nc * kmax, cudaMemcpyHostToDevice, st));
  bcombine_kernel<<<dim3(nb256(n), nc), 256, sizeof(double2) * kmax, st>>>(S.V, ldc, n, S.idx_a, S.idx_k, kmax,
                                                                          S.coef, x, n, n);
  VSIE_CUDA(cudaGetLastError());
  VSIE_CUDA(cudaStreamSynchronize(st));
  return VSIE_OK;
}

}  // namespace

}  // namespace vsie

using namespace vsie;

extern "C" vsie_status vsie_solve_batched(vsie_handle* h, const void* d_b, void* d_x, int32_t nrhs,
                                          const vsie_solve_opts* opts, vsie_solve_info* infos, void* stream) {
  clear_error();
  TraceRange trace("vsie_solve_batched");
  if (!h || !d_b || !d_x || !opts || nrhs < 1 || nrhs > 65535) {
    set_error("vsie_solve_batched: null argument or nrhs outside [1, 65535]");
    return VSIE_ERR_ARG;
  }
  if ((opts->mode != 32 && opts->mode != 64) || !(opts->tol > 0.0) || opts->max_iters < 1 ||
      opts->restart < 0 || (opts->mode == 32 && !(opts->inner_tol > 0.0))) {
    set_error("vsie_solve_batched: invalid options");
    return VSIE_ERR_ARG;
  }
  if (opts->initial_guess) {
    set_error("vsie_solve_batched: initial_guess is not supported (use vsie_solve)");
    return VSIE_ERR_ARG;
  }
  if (opts->adjoint) {
    set_error("vsie_solve_batched: adjoint solves are not batched; use vsie_solve");
    return VSIE_ERR_ARG;
  }
  const int m = (opts->restart > 0 && opts->restart < opts->max_iters) ? opts->restart : opts->max_iters;
  if (m > kMaxBasis) {
    set_error("vsie_solve_batched: Krylov basis larger than 1000 columns; set restart <= 1000");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int64_t n = h->n;
  const double2* b = (const double2*)d_b;
  double2* x = (double2*)d_x;
  const int R = nrhs;
  std::vector<vsie_solve_info> local(R);
  vsie_solve_info* inf = infos ? infos : local.data();
  for (int c = 0; c < R; ++c) inf[c] = vsie_solve_info{};

  Work S;
  S.n = n;
  S.R = R;
  S.m = m;
  S.nbx = std::max(4, std::min(296, (2 * std::max(h->num_sms, 1) * 2 + R - 1) / R));
  std::vector<void*> temps;
  double2* hbuf = nullptr;
  auto cleanup = [&]() {
    for (void* p : temps) cudaFree(p);
    if (hbuf) cudaFreeHost(hbuf);
  };
  auto alloc = [&](void** p, size_t bytes) -> vsie_status {
    cudaError_t e = cudaMalloc(p, std::max<size_t>(bytes, 16));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(batched solver workspace)", __FILE__, __LINE__);
    temps.push_back(*p);
    return VSIE_OK;
  };
  vsie_status s = VSIE_OK;
  const size_t cols = (size_t)R * n;
  if ((s = alloc((void**)&S.V, sizeof(double2) * (size_t)(m + 1) * cols)) != VSIE_OK ||
      (s = alloc((void**)&S.X, sizeof(double2) * cols)) != VSIE_OK ||
      (s = alloc((void**)&S.W, sizeof(double2) * cols)) != VSIE_OK ||
      (s = alloc((void**)&S.r, sizeof(double2) * cols)) != VSIE_OK ||
      (s = alloc((void**)&S.partial, sizeof(double2) * (size_t)S.nbx * (m + 1) * R)) != VSIE_OK ||
      (s = alloc((void**)&S.h1, sizeof(double2) * (size_t)(m + 1) * R)) != VSIE_OK ||
      (s = alloc((void**)&S.h2, sizeof(double2) * (size_t)(m + 1) * R)) != VSIE_OK ||
      (s = alloc((void**)&S.nrm, sizeof(double2) * R)) != VSIE_OK ||
      (s = alloc((void**)&S.idx_a, sizeof(int) * R)) != VSIE_OK ||
      (s = alloc((void**)&S.idx_b, sizeof(int) * R)) != VSIE_OK ||
      (s = alloc((void**)&S.idx_k, sizeof(int) * R)) != VSIE_OK ||
      (s = alloc((void**)&S.scale, sizeof(double) * R)) != VSIE_OK ||
      (s = alloc((void**)&S.coef, sizeof(double2) * (size_t)m * R)) != VSIE_OK) {
    cleanup();
    return s;
  }
  if (cudaMallocHost((void**)&hbuf, sizeof(double2) * ((size_t)2 * (m + 1) * R + R)) != cudaSuccess) {
    cleanup();
    set_error("vsie_solve_batched: cudaMallocHost failed");
    return VSIE_ERR_OOM;
  }
  S.hbuf = hbuf;

  auto run = [&]() -> vsie_status {
    VSIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * cols, st));
    VSIE_CUDA(cudaMemcpyAsync(S.r, b, sizeof(double2) * cols, cudaMemcpyDeviceToDevice, st));
    std::vector<double> bnorm, rnorm;
    VSIE_TRY(batched_norms(S, b, n, R, bnorm, st));
    for (int c = 0; c < R; ++c)
      if (!std::isfinite(bnorm[c])) {
        set_error("vsie_solve_batched: non-finite right-hand side");
        return VSIE_ERR_NAN;
      }
    rnorm = bnorm;
    // 0 pending, 1 converged, 2 not converged, 3 breakdown
    std::vector<int> state(R, 0);
    for (int c = 0; c < R; ++c)
      if (bnorm[c] == 0.0) {
        state[c] = 1;
        inf[c].rel_residual = 0.0;
      }
    const int max_outer = opts->mode == 32 ? std::max(1, opts->max_refinements) : 1 << 30;
    for (int outer = 1;; ++outer) {
      std::vector<Column> cyc;
      std::vector<double> r0n;
      for (int c = 0; c < R; ++c) {
        if (state[c] != 0) continue;
        Column C;
        C.c = c;
        const double target = opts->tol * bnorm[c];
        C.target = opts->mode == 32 ? std::max(opts->inner_tol * rnorm[c], target) : target;
        C.limit = std::min(m, opts->max_iters - inf[c].iterations);
        cyc.push_back(std::move(C));
        r0n.push_back(rnorm[c]);
      }
      if (cyc.empty()) break;
      VSIE_TRY(batched_cycle(h, opts->mode, cyc, r0n, x, S, st, inf));
      // true residuals r_c = b_c - A x_c with the FP64 apply (gathered into X, A x into W)
      const int a = (int)cyc.size();
      std::vector<int> cc(a);
      for (int y = 0; y < a; ++y) cc[y] = cyc[y].c;
      VSIE_CUDA(cudaMemcpyAsync(S.idx_a, cc.data(), sizeof(int) * a, cudaMemcpyHostToDevice, st));
      bcopy_scaled_kernel<<<dim3(nb256(n), a), 256, 0, st>>>(x, n, 0, S.idx_a, nullptr, S.X, n, 0, nullptr, n);
      VSIE_CUDA(cudaGetLastError());
      VSIE_TRY(block_apply(h, S.X, S.W, a, 64, st, inf, cc));
      bresidual_kernel<<<dim3(nb256(n), a), 256, 0, st>>>(b, S.W, S.idx_a, S.r, n);
      bcopy_scaled_kernel<<<dim3(nb256(n), a), 256, 0, st>>>(S.r, n, 0, S.idx_a, nullptr, S.X, n, 0, nullptr, n);
      VSIE_CUDA(cudaGetLastError());
      std::vector<double> rn;
      VSIE_TRY(batched_norms(S, S.X, n, a, rn, st));
      for (int y = 0; y < a; ++y) {
        const Column& C = cyc[y];
        const int c = C.c;
        if (!std::isfinite(rn[y])) {
          set_error("vsie_solve_batched: non-finite residual");
          return VSIE_ERR_NAN;
        }
        rnorm[c] = rn[y];
        inf[c].iterations += C.k;
        inf[c].refinements = opts->mode == 32 ? outer : 0;
        inf[c].rel_residual = rn[y] / bnorm[c];
        if (rn[y] <= opts->tol * bnorm[c])
          state[c] = 1;
        else if (C.breakdown && C.k == 0)
          state[c] = 3;
        else if (inf[c].iterations >= opts->max_iters || outer >= max_outer)
          state[c] = 2;
      }
    }
    bool brk = false, nc = false;
    for (int c = 0; c < R; ++c) {
      brk |= state[c] == 3;
      nc |= state[c] == 2;
    }
    if (brk) {
      set_error("vsie_solve_batched: GMRES breakdown");
      return VSIE_ERR_BREAKDOWN;
    }
    if (nc) {
      set_error("vsie_solve_batched: tolerance not reached within the iteration limits");
      return VSIE_ERR_NOT_CONVERGED;
    }
    return VSIE_OK;
  };
  s = run();
  cudaStreamSynchronize(st);
  cleanup();
  return s;
}
