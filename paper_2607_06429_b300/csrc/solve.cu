// GMRES solve of the collocation system (Sec. 3.1: GMRES, x0 = 0, no preconditioner,
// relative residual tolerance) with FP64 Arnoldi on the device, and a mixed-precision
// variant: FP64 iterative refinement (true residual r = b - A x with the FP64 apply)
// around inner GMRES cycles that use the FP32 apply.
//
// Arnoldi uses classical Gram-Schmidt applied twice (CGS2): two passes of one fused
// multi-dot kernel (h = V^H w over all basis columns in one sweep of w) and one fused
// update kernel (w -= V h), so the basis is streamed from HBM four times per iteration
// instead of 2j times.  The small Hessenberg least-squares problem (Givens rotations)
// lives on the host in FP64.

#include <cuda_runtime.h>

#include <cmath>
#include <complex>
#include <vector>

#include "vsie_internal.h"

namespace vsie {

using cplx = std::complex<double>;

constexpr int kDotBlocks = 296;  // 2 per SM
constexpr int kDotThreads = 256;

// partial[c * nb + b] = sum_{i in slice b} conj(V[c][i]) w[i],  c < k
__global__ void __launch_bounds__(kDotThreads) multidot_kernel(const double2* __restrict__ V,
                                                               int64_t ld, int k,
                                                               const double2* __restrict__ w,
                                                               int64_t n, double2* __restrict__ partial) {
  __shared__ double red[2][kDotThreads / 32];
  const int nb = gridDim.x;
  const int64_t per = (n + nb - 1) / nb;
  const int64_t i0 = (int64_t)blockIdx.x * per;
  const int64_t i1 = min(n, i0 + per);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int c = 0; c < k; ++c) {
    const double2* v = V + (int64_t)c * ld;
    double ar = 0.0, ai = 0.0;
    for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
      const double2 a = v[i], b = w[i];
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
      for (int q = 0; q < kDotThreads / 32; ++q) {
        sr += red[0][q];
        si += red[1][q];
      }
      partial[(int64_t)c * nb + blockIdx.x] = make_double2(sr, si);
    }
    __syncthreads();
  }
}

// out[c] = sum_b partial[c * nb + b] (fixed order)
__global__ void reduce_partials_kernel(const double2* __restrict__ partial, int nb, int k,
                                       double2* __restrict__ out) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= k) return;
  double sr = 0.0, si = 0.0;
  for (int b = 0; b < nb; ++b) {
    const double2 v = partial[(int64_t)c * nb + b];
    sr += v.x;
    si += v.y;
  }
  out[c] = make_double2(sr, si);
}

// w -= sum_c V[c] h[c]
__global__ void update_kernel(const double2* __restrict__ V, int64_t ld, int k,
                              const double2* __restrict__ hcoef, double2* __restrict__ w, int64_t n) {
  extern __shared__ double2 hs[];
  for (int c = threadIdx.x; c < k; c += blockDim.x) hs[c] = hcoef[c];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 acc = w[i];
  for (int c = 0; c < k; ++c) {
    const double2 v = V[(int64_t)c * ld + i];
    const double2 q = hs[c];
    acc.x -= v.x * q.x - v.y * q.y;
    acc.y -= v.x * q.y + v.y * q.x;
  }
  w[i] = acc;
}

// x += sum_c V[c] y[c]
__global__ void combine_kernel(const double2* __restrict__ V, int64_t ld, int k,
                               const double2* __restrict__ ycoef, double2* __restrict__ x, int64_t n) {
  extern __shared__ double2 ys[];
  for (int c = threadIdx.x; c < k; c += blockDim.x) ys[c] = ycoef[c];
  __syncthreads();
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double2 acc = x[i];
  for (int c = 0; c < k; ++c) {
    const double2 v = V[(int64_t)c * ld + i];
    const double2 q = ys[c];
    acc.x += v.x * q.x - v.y * q.y;
    acc.y += v.x * q.y + v.y * q.x;
  }
  x[i] = acc;
}

__global__ void scale_kernel(const double2* __restrict__ w, double s, double2* __restrict__ v, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  v[i] = make_double2(w[i].x * s, w[i].y * s);
}

// r = b - y
__global__ void sub_kernel(const double2* __restrict__ b, const double2* __restrict__ y,
                           double2* __restrict__ r, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  r[i] = make_double2(b[i].x - y[i].x, b[i].y - y[i].y);
}

struct SolveWork {
  double2* V = nullptr;   // (m + 1) x n basis
  double2* w = nullptr;
  double2* r = nullptr;
  double2* t = nullptr;
  double2* partial = nullptr;
  double2* hdev = nullptr;
  int m = 0;
};

static inline unsigned nb256(int64_t n) { return (unsigned)((n + 255) / 256); }

// dot products of w with the first k columns of V, result copied to the host
static vsie_status multidot(const double2* V, int64_t ld, int k, const double2* w, int64_t n,
                            SolveWork& S, std::vector<cplx>& out, cudaStream_t st) {
  multidot_kernel<<<kDotBlocks, kDotThreads, 0, st>>>(V, ld, k, w, n, S.partial);
  reduce_partials_kernel<<<(k + 127) / 128, 128, 0, st>>>(S.partial, kDotBlocks, k, S.hdev);
  VSIE_CUDA(cudaGetLastError());
  out.resize(k);
  VSIE_CUDA(cudaMemcpyAsync(out.data(), S.hdev, sizeof(double2) * k, cudaMemcpyDeviceToHost, st));
  VSIE_CUDA(cudaStreamSynchronize(st));
  return VSIE_OK;
}

static vsie_status norm2(const double2* w, int64_t n, SolveWork& S, double* out, cudaStream_t st) {
  std::vector<cplx> d;
  VSIE_TRY(multidot(w, n, 1, w, n, S, d, st));
  *out = std::sqrt(std::max(d[0].real(), 0.0));
  return VSIE_OK;
}

// y = A x (adjoint == false) or y = A^H x (adjoint == true)
static vsie_status op_apply(vsie_handle* h, bool adjoint, const double2* x, double2* y, int precision,
                            cudaStream_t st) {
  if (!adjoint) return apply_one(h, x, y, precision, st);
  VSIE_TRY(far_adjoint(h, x, y, precision, st));
  return correction_adjoint(h, x, y, precision, st);
}

// One GMRES cycle for A d = r0 from d = 0 (d is ADDED to x).  Stops when the Arnoldi
// residual estimate drops below target_abs or after max_it iterations.
static vsie_status gmres_cycle(int64_t n, const ApplyFn& apply, int precision, const double2* r0,
                               double r0norm, double2* x, double target_abs, int max_it, SolveWork& S,
                               cudaStream_t st, int* iters, double* est, int* applies,
                               bool* breakdown, const char* who) {
  const int m = std::min(max_it, S.m);
  std::vector<cplx> H((size_t)(m + 1) * m, 0.0), cs(m), sn(m), g(m + 1, 0.0);
  g[0] = r0norm;
  scale_kernel<<<nb256(n), 256, 0, st>>>(r0, 1.0 / r0norm, S.V, n);
  VSIE_CUDA(cudaGetLastError());
  int j = 0;
  double res = r0norm;
  *breakdown = false;
  std::vector<cplx> h1, h2;
  for (j = 0; j < m; ++j) {
    double2* vj = S.V + (size_t)j * n;
    VSIE_TRY(apply(vj, S.w, precision));
    ++*applies;
    // CGS2
    // (multidot leaves the coefficients in S.hdev for the update kernel)
    VSIE_TRY(multidot(S.V, n, j + 1, S.w, n, S, h1, st));
    update_kernel<<<nb256(n), 256, sizeof(double2) * (j + 1), st>>>(S.V, n, j + 1, S.hdev, S.w, n);
    VSIE_CUDA(cudaGetLastError());
    VSIE_TRY(multidot(S.V, n, j + 1, S.w, n, S, h2, st));
    update_kernel<<<nb256(n), 256, sizeof(double2) * (j + 1), st>>>(S.V, n, j + 1, S.hdev, S.w, n);
    VSIE_CUDA(cudaGetLastError());
    double beta;
    VSIE_TRY(norm2(S.w, n, S, &beta, st));
    if (!std::isfinite(beta)) {
      set_error(std::string(who) + ": non-finite value in the Arnoldi process");
      return VSIE_ERR_NAN;
    }
    for (int i = 0; i <= j; ++i) H[(size_t)j * (m + 1) + i] = h1[i] + h2[i];
    H[(size_t)j * (m + 1) + j + 1] = beta;
    // apply previous rotations to column j
    cplx* col = &H[(size_t)j * (m + 1)];
    for (int i = 0; i < j; ++i) {
      const cplx a = col[i], b = col[i + 1];
      col[i] = std::conj(cs[i]) * a + std::conj(sn[i]) * b;
      col[i + 1] = -sn[i] * a + cs[i] * b;
    }
    // new rotation zeroing col[j+1]
    const cplx a = col[j];
    const double bb = std::abs(col[j + 1]);
    const double den = std::sqrt(std::norm(a) + bb * bb);
    if (den == 0.0) {
      cs[j] = 1.0;
      sn[j] = 0.0;
    } else {
      cs[j] = a / den;
      sn[j] = col[j + 1] / den;
    }
    col[j] = den;
    col[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = std::conj(cs[j]) * g[j];
    res = std::abs(g[j + 1]);
    if (beta == 0.0) {
      *breakdown = res > target_abs;
      ++j;
      break;
    }
    // v_{j+1} = w / beta  (column j+1 <= m exists: the basis has m + 1 columns)
    scale_kernel<<<nb256(n), 256, 0, st>>>(S.w, 1.0 / beta, S.V + (size_t)(j + 1) * n, n);
    VSIE_CUDA(cudaGetLastError());
    if (res <= target_abs) {
      ++j;
      break;
    }
  }
  const int k = std::min(j, m);
  // back substitution R y = g
  std::vector<cplx> y(k);
  for (int i = k - 1; i >= 0; --i) {
    cplx acc = g[i];
    for (int c = i + 1; c < k; ++c) acc -= H[(size_t)c * (m + 1) + i] * y[c];
    y[i] = acc / H[(size_t)i * (m + 1) + i];
  }
  if (k > 0) {
    VSIE_CUDA(cudaMemcpyAsync(S.hdev, y.data(), sizeof(double2) * k, cudaMemcpyHostToDevice, st));
    combine_kernel<<<nb256(n), 256, sizeof(double2) * k, st>>>(S.V, n, k, S.hdev, x, n);
    VSIE_CUDA(cudaGetLastError());
  }
  *iters = k;
  *est = res;
  return VSIE_OK;
}

// GMRES (x0 = 0 or the given iterate) with, in mode 32, FP64 iterative refinement: inner
// cycles with the inner_prec apply to inner_tol, true residuals with the res_prec apply.
vsie_status gmres_solve(int64_t n, const ApplyFn& apply, const double2* b, double2* x,
                        const vsie_solve_opts* opts, vsie_solve_info* info, cudaStream_t st, int inner_prec,
                        int res_prec, const char* who) {
  vsie_solve_info local{};
  vsie_solve_info& inf = info ? *info : local;
  inf = vsie_solve_info{};

  const int m = (opts->restart > 0 && opts->restart < opts->max_iters) ? opts->restart : opts->max_iters;
  if (m > 3000) {
    set_error(std::string(who) + ": Krylov basis larger than 3000 columns; set restart <= 3000");
    return VSIE_ERR_ARG;
  }
  std::vector<void*> temps;
  auto cleanup = [&]() {
    for (void* p : temps) cudaFree(p);
  };
  auto alloc = [&](double2** p, size_t count) -> vsie_status {
    cudaError_t e = cudaMalloc(p, sizeof(double2) * count);
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(solver workspace)", __FILE__, __LINE__);
    temps.push_back(*p);
    return VSIE_OK;
  };
  SolveWork S;
  S.m = m;
  vsie_status s;
  if ((s = alloc(&S.V, (size_t)(m + 1) * n)) != VSIE_OK || (s = alloc(&S.w, n)) != VSIE_OK ||
      (s = alloc(&S.r, n)) != VSIE_OK || (s = alloc(&S.t, n)) != VSIE_OK ||
      (s = alloc(&S.partial, (size_t)kDotBlocks * (m + 1))) != VSIE_OK ||
      (s = alloc(&S.hdev, (size_t)m + 1)) != VSIE_OK) {
    cleanup();
    return s;
  }
  auto run = [&]() -> vsie_status {
    if (!opts->initial_guess) VSIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * n, st));
    double bnorm;
    VSIE_TRY(norm2(b, n, S, &bnorm, st));
    if (!std::isfinite(bnorm)) {
      set_error(std::string(who) + ": non-finite right-hand side");
      return VSIE_ERR_NAN;
    }
    if (bnorm == 0.0) {  // the solution is 0 whatever the starting iterate
      VSIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double2) * n, st));
      inf.rel_residual = 0.0;
      return VSIE_OK;
    }
    const double target = opts->tol * bnorm;
    double rnorm = bnorm;
    if (opts->initial_guess) {
      // resume: r = b - A x from the given iterate
      VSIE_TRY(apply(x, S.t, res_prec));
      inf.fp64_applies += 1;
      sub_kernel<<<nb256(n), 256, 0, st>>>(b, S.t, S.r, n);
      VSIE_CUDA(cudaGetLastError());
      VSIE_TRY(norm2(S.r, n, S, &rnorm, st));
      if (!std::isfinite(rnorm)) {
        set_error(std::string(who) + ": non-finite residual of the initial guess");
        return VSIE_ERR_NAN;
      }
      inf.rel_residual = rnorm / bnorm;
      if (rnorm <= target) return VSIE_OK;
    } else {
      VSIE_CUDA(cudaMemcpyAsync(S.r, b, sizeof(double2) * n, cudaMemcpyDeviceToDevice, st));
    }
    const int max_outer = opts->mode == 32 ? std::max(1, opts->max_refinements) : 1 << 30;
    int outer = 0;
    while (true) {
      const double cycle_target =
          opts->mode == 32 ? std::max(opts->inner_tol * rnorm, target) : target;
      int it = 0, applies = 0;
      double est;
      bool brk;
      VSIE_TRY(gmres_cycle(n, apply, inner_prec, S.r, rnorm, x, cycle_target, opts->max_iters - inf.iterations,
                           S, st, &it, &est, &applies, &brk, who));
      inf.iterations += it;
      if (inner_prec == 32)
        inf.fp32_applies += applies;
      else
        inf.fp64_applies += applies;
      // true residual with the FP64-accuracy apply
      VSIE_TRY(apply(x, S.t, res_prec));
      inf.fp64_applies += 1;
      sub_kernel<<<nb256(n), 256, 0, st>>>(b, S.t, S.r, n);
      VSIE_CUDA(cudaGetLastError());
      VSIE_TRY(norm2(S.r, n, S, &rnorm, st));
      if (!std::isfinite(rnorm)) {
        set_error(std::string(who) + ": non-finite residual");
        return VSIE_ERR_NAN;
      }
      ++outer;
      inf.refinements = opts->mode == 32 ? outer : 0;
      inf.rel_residual = rnorm / bnorm;
      if (rnorm <= target) return VSIE_OK;
      if (brk && it == 0) {
        set_error(std::string(who) + ": GMRES breakdown");
        return VSIE_ERR_BREAKDOWN;
      }
      if (inf.iterations >= opts->max_iters || outer >= max_outer) {
        set_error(std::string(who) + ": tolerance not reached within the iteration limits");
        return VSIE_ERR_NOT_CONVERGED;
      }
    }
  };
  s = run();
  cudaStreamSynchronize(st);
  cleanup();
  return s;
}

}  // namespace vsie

using namespace vsie;

extern "C" vsie_status vsie_solve(vsie_handle* h, const void* d_b, void* d_x,
                                  const vsie_solve_opts* opts, vsie_solve_info* info, void* stream) {
  clear_error();
  TraceRange trace("vsie_solve");
  if (!h || !d_b || !d_x || !opts) {
    set_error("vsie_solve: null argument");
    return VSIE_ERR_ARG;
  }
  if ((opts->mode != 32 && opts->mode != 64) || !(opts->tol > 0.0) || opts->max_iters < 1 ||
      opts->restart < 0 || (opts->mode == 32 && !(opts->inner_tol > 0.0))) {
    set_error("vsie_solve: invalid options");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const bool adjoint = opts->adjoint != 0;
  // the apply that forms true residuals: the double-float sums (precision 48) in the
  // refinement of a forward solve, plain FP64 otherwise
  const int res_prec = (opts->mode == 32 && !adjoint) ? 48 : 64;
  const ApplyFn apply = [&](const double2* xx, double2* yy, int prec) {
    return op_apply(h, adjoint, xx, yy, prec, st);
  };
  return gmres_solve(h->n, apply, (const double2*)d_b, (double2*)d_x, opts, info, st, opts->mode, res_prec,
                     "vsie_solve");
}
