// Nested PMCHWT boundary element method (Sec. 2.4, the paper's comparison solver for
// piecewise-constant media): P1 Galerkin on triangulated interfaces, matrix-free.
//
// One apply of the lumped-mass-preconditioned PMCHWT operator (include/vsie_bem.h):
//   1. prolong   (per triangle): the P1 traces u, v at the far-rule points and the surface
//      curl of u, turned into per-layer source charges (weights, signs sigma_jl, rho_j,
//      k_j^2 and 1/(4 pi) folded in);
//   2. N-body    (per layer): at every far-rule point x of the interfaces bounding the
//      layer, the sums over the same points y of
//         S1 = sum G q + E ((x - y).n_y) u          (row of -K u + rho V v)
//         S2 = sum G (n_x.n_y) b + E ((x - y).n_x) c (k^2 part of W u / rho, and K' v)
//         A  = sum G a                               (curl part of W u / rho)
//      G = e^{ikr}/r, E = (ikr - 1) e^{ikr}/r^3 (so grad_x G = E (x - y) up to 1/(4 pi));
//      split over source chunks with per-chunk partial sums reduced in a fixed order and
//      multiplied by the target's sign sigma_jm;
//   3. restrict  (per triangle): the P1 test integrals of S1, S2 and A, plus the near
//      pairs' correction blocks times the trial triangles' nodal values;
//   4. gather    (per vertex): the triangles' local rows summed in triangle order and
//      divided by the lumped mass.
// The near correction of a pair (near rule minus far rule, every layer bounding both
// interfaces) is computed once at creation in FP64: closed-form potentials of linear
// densities on the trial triangle for the static kernel 1/(4 pi r) (edge integrals and
// the solid angle), the smooth remainder on the near rule.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "dfloat.h"
#include "vsie_bem.h"
#include "vsie_internal.h"

namespace vsie {

constexpr double kBPi = 3.14159265358979323846;
constexpr double kInv4Pi = 1.0 / (4.0 * kBPi);
constexpr int kBemMaxOrder = 8;
constexpr int kBemMaxQ = kBemMaxOrder * kBemMaxOrder;
constexpr int kBemThreads = 128;  // N-body block: sources per shared-memory tile
constexpr int kBemTgt = 2;        // targets per thread
constexpr int kSrcRec = 20;       // x y z nx ny nz | q uK b c (complex) | a (3 complex)
constexpr int kTgtRec = 6;        // x y z nx ny nz
constexpr int kOut = 10;          // S1, S2, A_x, A_y, A_z (complex)
constexpr int kDfTgt = 12;        // double-float target record: x y z nx ny nz (hi, lo each)
constexpr int kDfSrc = 40;        // double-float source record: the 20 values (hi, lo each)
constexpr int kDfThreads = 128;   // double-float N-body: one target per thread
constexpr int kDfTile = 64;       // sources per shared-memory tile

struct BemDomain {
  double k, rho;
  int sigma[2];  // per interface: +1 / -1, 0 if the layer does not touch it
  int64_t p0, np;  // its contiguous range of far-rule points (targets = sources)
};

// Quadrature rule on a triangle: barycentric coordinates and weights summing to 1.
struct BemRule {
  int q;
  double lam[kBemMaxQ][3];
  double w[kBemMaxQ];
};

// n-point Gauss-Legendre rule on [0, 1]: Newton's method on P_n from the Chebyshev-like
// initial guesses cos(pi (i + 3/4)/(n + 1/2)), weights 2 / ((1 - x^2) P_n'(x)^2) halved.
static void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double z = std::cos(kBPi * (i + 0.75) / (n + 0.5)), dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double pn = n == 0 ? 1.0 : (n == 1 ? z : p1);
      const double pm = n == 1 ? 1.0 : p0;
      dp = n * (z * pn - pm) / (z * z - 1.0);
      const double dz = pn / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (1.0 - z);
    w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Collapsed product rule: (u, v) in [0,1]^2 -> barycentric (1 - s - t, s, t) with s = u,
// t = (1 - u) v; weight 2 w_u w_v (1 - u).
static BemRule make_rule(int order) {
  BemRule r{};
  double x[kBemMaxOrder], w[kBemMaxOrder];
  gauss_legendre01(order, x, w);
  r.q = order * order;
  for (int a = 0; a < order; ++a)
    for (int b = 0; b < order; ++b) {
      const int i = a * order + b;
      const double s = x[a], t = (1.0 - x[a]) * x[b];
      r.lam[i][0] = 1.0 - s - t;
      r.lam[i][1] = s;
      r.lam[i][2] = t;
      r.w[i] = 2.0 * w[a] * w[b] * (1.0 - x[a]);
    }
  return r;
}

}  // namespace vsie

using namespace vsie;

struct vsie_bem {
  int device = 0;
  int nsurf = 0;
  int64_t nv_s[2] = {0, 0}, nt_s[2] = {0, 0}, v_off[2] = {0, 0}, t_off[2] = {0, 0};
  int64_t nv = 0, nt = 0, n = 0, nq = 0, nnear = 0;
  int ndom = 0;
  BemDomain dom[3];
  double k0 = 0.0, rho0 = 1.0, near_factor = 2.0;
  BemRule far{}, nearr{};
  BemRule* d_far = nullptr;
  BemRule* d_near = nullptr;
  // geometry
  double* vert = nullptr;       // nv x 3
  int* tri = nullptr;           // nt x 3 (global vertex indices)
  int* tsurf = nullptr;         // nt
  double* tgeo = nullptr;       // nt x 24: area, n(3), centroid(3), diam2, curl(3 x 3), pad
  int64_t* uidx = nullptr;      // nv: unknown index of u at the vertex (v at + nv_s)
  int64_t* vidx = nullptr;
  double* lmass = nullptr;      // nv
  int64_t* vt_ptr = nullptr;    // nv + 1
  int* vt_idx = nullptr;        // 3 nt entries: T * 3 + i
  // far-rule points
  double* qw = nullptr;         // nq: weight x area
  double* tgt64 = nullptr;      // nq x 6
  float* tgt32 = nullptr;
  double* src64[3] = {nullptr, nullptr, nullptr};  // per layer, nq x 20
  float* src32[3] = {nullptr, nullptr, nullptr};
  float* tgtdf = nullptr;                            // nq x 12
  float* srcdf[3] = {nullptr, nullptr, nullptr};   // per layer, nq x 40
  double* pout = nullptr;       // nq x 10 (the N-body sums, signed, all layers)
  double* part = nullptr;       // N-body chunk partials
  size_t part_elems = 0;
  double2* zloc = nullptr;      // nt x 6
  // near pairs
  int64_t* near_ptr = nullptr;  // nt + 1
  int* near_tp = nullptr;       // nnear
  double2* near_blk = nullptr;  // nnear x 36: rows (u_i, v_i) x columns (u_j, v_j)
  std::vector<void*> allocs;
};

namespace vsie {

static vsie_status balloc(vsie_bem* b, void** p, size_t bytes) {
  *p = nullptr;
  if (bytes == 0) bytes = 16;
  const cudaError_t e = cudaMalloc(p, bytes);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    set_error("vsie_bem: out of device memory");
    return VSIE_ERR_OOM;
  }
  if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc", __FILE__, __LINE__);
  b->allocs.push_back(*p);
  return VSIE_OK;
}
template <class T>
static vsie_status balloc_t(vsie_bem* b, T** p, size_t count) {
  return balloc(b, reinterpret_cast<void**>(p), count * sizeof(T));
}

static inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

// ----------------------------------------------------------------- geometry

// Per triangle: area, unit normal (right-hand), centroid ((a + b) + c)/3, largest squared
// edge, surface curls n x grad(lambda_i).  Rounded operations without contraction where the
// near-pair test reads them, so that its decisions match a plain evaluation.
__global__ void bem_geom_kernel(const double* __restrict__ vert, const int* __restrict__ tri, int64_t nt,
                                double* __restrict__ geo, int* __restrict__ bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double v[3][3];
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) v[i][d] = vert[3 * (int64_t)tri[3 * t + i] + d];
  double e1[3], e2[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = v[1][d] - v[0][d];
    e2[d] = v[2][d] - v[0][d];
  }
  double cr[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
  const double nn = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
  if (!(nn > 0.0)) {
    atomicExch(bad, 1);
    return;
  }
  double* g = geo + 24 * t;
  const double area = 0.5 * nn;
  double n[3] = {cr[0] / nn, cr[1] / nn, cr[2] / nn};
  g[0] = area;
  for (int d = 0; d < 3; ++d) {
    g[1 + d] = n[d];
    g[4 + d] = __ddiv_rn(__dadd_rn(__dadd_rn(v[0][d], v[1][d]), v[2][d]), 3.0);
  }
  double dm = 0.0;
  for (int e = 0; e < 3; ++e) {
    const double* p = v[e];
    const double* q = v[(e + 1) % 3];
    double s = 0.0;
    for (int d = 0; d < 3; ++d) {
      const double dd = __dsub_rn(q[d], p[d]);
      s = __dadd_rn(s, __dmul_rn(dd, dd));
    }
    dm = fmax(dm, s);
  }
  g[7] = dm;
  // grad lambda_i = n x (v_{i+2} - v_{i+1}) / (2A); curl = n x grad
  for (int i = 0; i < 3; ++i) {
    const double* p = v[(i + 1) % 3];
    const double* q = v[(i + 2) % 3];
    const double ed[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    double gr[3] = {(n[1] * ed[2] - n[2] * ed[1]) / nn, (n[2] * ed[0] - n[0] * ed[2]) / nn,
                    (n[0] * ed[1] - n[1] * ed[0]) / nn};
    g[8 + 3 * i + 0] = n[1] * gr[2] - n[2] * gr[1];
    g[8 + 3 * i + 1] = n[2] * gr[0] - n[0] * gr[2];
    g[8 + 3 * i + 2] = n[0] * gr[1] - n[1] * gr[0];
  }
}

// Far-rule points: weights and target records (position, triangle normal).
__global__ void bem_points_kernel(const double* __restrict__ vert, const int* __restrict__ tri,
                                  const double* __restrict__ geo, const BemRule* __restrict__ rule, int64_t nt,
                                  double* __restrict__ qw, double* __restrict__ tgt64, float* __restrict__ tgt32) {
  const int Q = rule->q;
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nt * Q) return;
  const int64_t t = p / Q;
  const int q = (int)(p - t * Q);
  double x[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) x[d] += rule->lam[q][i] * vert[3 * (int64_t)tri[3 * t + i] + d];
  const double* g = geo + 24 * t;
  qw[p] = rule->w[q] * g[0];
  for (int d = 0; d < 3; ++d) {
    tgt64[6 * p + d] = x[d];
    tgt64[6 * p + 3 + d] = g[1 + d];
    tgt32[6 * p + d] = (float)x[d];
    tgt32[6 * p + 3 + d] = (float)g[1 + d];
  }
}

// Source records: positions and normals (charges are written per apply).
template <class R>
__global__ void bem_src_geom_kernel(const double* __restrict__ tgt64, int64_t nq, R* __restrict__ src) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nq) return;
  for (int d = 0; d < 6; ++d) src[kSrcRec * p + d] = (R)tgt64[6 * p + d];
}

// Double-float records: positions and normals split into (hi, lo) floats, for the targets
// and the per-layer source arrays (charges are written per apply).
__global__ void bem_df_geom_kernel(const double* __restrict__ tgt64, int64_t nq, float* __restrict__ tgt,
                                   float* __restrict__ s0, float* __restrict__ s1, float* __restrict__ s2) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= nq) return;
  float* outs[3] = {s0, s1, s2};
  for (int d = 0; d < 6; ++d) {
    const dfs v = dfs_make(tgt64[6 * p + d]);
    tgt[kDfTgt * p + 2 * d] = v.h;
    tgt[kDfTgt * p + 2 * d + 1] = v.l;
    for (int j = 0; j < 3; ++j)
      if (outs[j]) {
        outs[j][kDfSrc * p + 2 * d] = v.h;
        outs[j][kDfSrc * p + 2 * d + 1] = v.l;
      }
  }
}

// Lumped mass per vertex: sum of A_T/3 over its triangles, in triangle order.
__global__ void bem_lumped_kernel(const int64_t* __restrict__ vt_ptr, const int* __restrict__ vt_idx,
                                  const double* __restrict__ geo, int64_t nv, double* __restrict__ m) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  double s = 0.0;
  for (int64_t k = vt_ptr[a]; k < vt_ptr[a + 1]; ++k) s += geo[24 * (vt_idx[k] / 3)] / 3.0;
  m[a] = s;
}

// ----------------------------------------------------------------- near pairs

__device__ __forceinline__ bool bem_is_near(const double* __restrict__ geo, const int* __restrict__ tri,
                                            int64_t t, int64_t u, double nf2) {
  const double* a = geo + 24 * t;
  const double* b = geo + 24 * u;
  double d2 = 0.0;
  for (int d = 0; d < 3; ++d) {
    const double dd = __dsub_rn(a[4 + d], b[4 + d]);
    d2 = __dadd_rn(d2, __dmul_rn(dd, dd));
  }
  if (d2 < __dmul_rn(nf2, fmax(a[7], b[7]))) return true;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      if (tri[3 * t + i] == tri[3 * u + j]) return true;
  return false;
}

// Pass 0 counts, pass 1 fills (in increasing T' order) the near triangles of each T among
// the triangles of interfaces that bound a common layer with T's (touch[sT][sT']).
__global__ void bem_near_kernel(const double* __restrict__ geo, const int* __restrict__ tri,
                                const int* __restrict__ tsurf, int64_t nt, double nf2, int touch01,
                                int64_t* __restrict__ count, const int64_t* __restrict__ ptr, int* __restrict__ list) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int st = tsurf[t];
  int64_t c = 0;
  int64_t o = list ? ptr[t] : 0;
  for (int64_t u = 0; u < nt; ++u) {
    const int su = tsurf[u];
    if (su != st && !touch01) continue;
    if (!bem_is_near(geo, tri, t, u, nf2)) continue;
    if (list)
      list[o++] = (int)u;
    else
      ++c;
  }
  if (!list) count[t] = c;
}

// Potentials of the static kernel over a flat triangle (v0, v1, v2) at x: for the three
// barycentric functions lambda_j,
//   IV_j = int lambda_j / R dy,   IK_j = int lambda_j (x - y).n / R^3 dy.
// With rho the projection of x on the plane, h = n.(x - v0) and per edge e (endpoints p, q,
// unit direction l, outward in-plane normal u = l x n, l-/l+ the endpoints' coordinates
// along l from rho, P0 = u.(p - rho), R0^2 = P0^2 + h^2, f_e = int dl / sqrt(l^2 + R0^2)):
//   S0 = int 1/R      = sum_e [P0 f_e - |h| (atan(P0 l+/(R0^2 + |h| R+)) - atan(P0 l-/(R0^2 + |h| R-)))]
//   S1 = int (y-rho)/R = sum_e u_e (R0^2 f_e + l+ R+ - l- R-)/2
//   D1 = int h (y-rho)/R^3 = -h sum_e u_e f_e
//   D0 = int h/R^3    = the solid angle of the triangle at x (signed with h)
// and lambda_j(y) = lambda_j(rho) + grad lambda_j . (y - rho).
__device__ void bem_static_potentials(const double x[3], const double v[3][3], bool skip_k, double IV[3],
                                      double IK[3]) {
  double e1[3], e2[3], n[3];
  for (int d = 0; d < 3; ++d) {
    e1[d] = v[1][d] - v[0][d];
    e2[d] = v[2][d] - v[0][d];
  }
  n[0] = e1[1] * e2[2] - e1[2] * e2[1];
  n[1] = e1[2] * e2[0] - e1[0] * e2[2];
  n[2] = e1[0] * e2[1] - e1[1] * e2[0];
  const double twoA = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
  for (int d = 0; d < 3; ++d) n[d] /= twoA;
  const double h = (x[0] - v[0][0]) * n[0] + (x[1] - v[0][1]) * n[1] + (x[2] - v[0][2]) * n[2];
  const double ah = fabs(h);
  double rho[3];
  for (int d = 0; d < 3; ++d) rho[d] = x[d] - h * n[d];
  double S0 = 0.0, S1[3] = {0.0, 0.0, 0.0}, D1[3] = {0.0, 0.0, 0.0};
  for (int e = 0; e < 3; ++e) {
    const double* p = v[e];
    const double* q = v[(e + 1) % 3];
    double L[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    const double ll = sqrt(L[0] * L[0] + L[1] * L[1] + L[2] * L[2]);
    for (int d = 0; d < 3; ++d) L[d] /= ll;
    const double u[3] = {L[1] * n[2] - L[2] * n[1], L[2] * n[0] - L[0] * n[2], L[0] * n[1] - L[1] * n[0]};
    double pr[3], qr[3];
    for (int d = 0; d < 3; ++d) {
      pr[d] = p[d] - rho[d];
      qr[d] = q[d] - rho[d];
    }
    const double lm = pr[0] * L[0] + pr[1] * L[1] + pr[2] * L[2];
    const double lp = qr[0] * L[0] + qr[1] * L[1] + qr[2] * L[2];
    const double P0 = pr[0] * u[0] + pr[1] * u[1] + pr[2] * u[2];
    const double R0sq = P0 * P0 + h * h;
    const double Rm = sqrt(lm * lm + R0sq), Rp = sqrt(lp * lp + R0sq);
    double f = 0.0;
    if (R0sq > 0.0) {
      if (lm >= 0.0)
        f = log((Rp + lp) / (Rm + lm));
      else if (lp <= 0.0)
        f = log((Rm - lm) / (Rp - lp));
      else
        f = log((Rp + lp) * (Rm - lm) / R0sq);
    }
    const double at = atan2(P0 * lp, R0sq + ah * Rp) - atan2(P0 * lm, R0sq + ah * Rm);
    S0 += P0 * f - ah * at;
    const double s1 = 0.5 * (R0sq * f + lp * Rp - lm * Rm);
    for (int d = 0; d < 3; ++d) {
      S1[d] += s1 * u[d];
      D1[d] += -h * f * u[d];
    }
  }
  double D0 = 0.0;
  if (!skip_k) {
    double A[3], B[3], C[3];
    for (int d = 0; d < 3; ++d) {
      A[d] = v[0][d] - x[d];
      B[d] = v[1][d] - x[d];
      C[d] = v[2][d] - x[d];
    }
    const double nA = sqrt(A[0] * A[0] + A[1] * A[1] + A[2] * A[2]);
    const double nB = sqrt(B[0] * B[0] + B[1] * B[1] + B[2] * B[2]);
    const double nC = sqrt(C[0] * C[0] + C[1] * C[1] + C[2] * C[2]);
    const double num = A[0] * (B[1] * C[2] - B[2] * C[1]) + A[1] * (B[2] * C[0] - B[0] * C[2]) +
                       A[2] * (B[0] * C[1] - B[1] * C[0]);
    const double den = nA * nB * nC + (A[0] * B[0] + A[1] * B[1] + A[2] * B[2]) * nC +
                       (A[0] * C[0] + A[1] * C[1] + A[2] * C[2]) * nB + (B[0] * C[0] + B[1] * C[1] + B[2] * C[2]) * nA;
    D0 = -2.0 * atan2(num, den);
  }
  for (int j = 0; j < 3; ++j) {
    const double* p = v[(j + 1) % 3];
    const double* q = v[(j + 2) % 3];
    const double ed[3] = {q[0] - p[0], q[1] - p[1], q[2] - p[2]};
    const double g[3] = {(n[1] * ed[2] - n[2] * ed[1]) / twoA, (n[2] * ed[0] - n[0] * ed[2]) / twoA,
                         (n[0] * ed[1] - n[1] * ed[0]) / twoA};
    const double lr = 1.0 + g[0] * (rho[0] - v[j][0]) + g[1] * (rho[1] - v[j][1]) + g[2] * (rho[2] - v[j][2]);
    IV[j] = lr * S0 + g[0] * S1[0] + g[1] * S1[1] + g[2] * S1[2];
    IK[j] = skip_k ? 0.0 : lr * D0 + g[0] * D1[0] + g[1] * D1[1] + g[2] * D1[2];
  }
}

struct C3 {
  double re[3][3], im[3][3];
};

// 3 x 3 blocks V3[i][j] = int int lambda_i(x) G lambda_j(y) and K3[i][j] = ... dG/dn_y ...
// over test triangle A (outer rule ro) and trial triangle B (inner rule ri), without the
// 1/(4 pi).  exact: the static part in closed form plus the smooth remainder
// (e^{ikr} - 1)/r on ri; else the full kernel on ri with zero-distance pairs dropped.
__device__ void bem_pair_blocks(const double va[3][3], double area_a, const double vb[3][3], double area_b,
                                const double nb[3], double k, const BemRule& ro, const BemRule& ri, bool exact,
                                bool same, C3& V3, C3& K3) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) V3.re[i][j] = V3.im[i][j] = K3.re[i][j] = K3.im[i][j] = 0.0;
  for (int q = 0; q < ro.q; ++q) {
    double x[3];
    for (int d = 0; d < 3; ++d) x[d] = ro.lam[q][0] * va[0][d] + ro.lam[q][1] * va[1][d] + ro.lam[q][2] * va[2][d];
    double vr[3] = {0, 0, 0}, vi[3] = {0, 0, 0}, kr_[3] = {0, 0, 0}, ki[3] = {0, 0, 0};
    for (int s = 0; s < ri.q; ++s) {
      double y[3];
      for (int d = 0; d < 3; ++d)
        y[d] = ri.lam[s][0] * vb[0][d] + ri.lam[s][1] * vb[1][d] + ri.lam[s][2] * vb[2][d];
      const double dx = x[0] - y[0], dy = x[1] - y[1], dz = x[2] - y[2];
      const double r = sqrt(dx * dx + dy * dy + dz * dz);
      const double dny = -(dx * nb[0] + dy * nb[1] + dz * nb[2]);  // (y - x).n_y
      double gr, gi, dr, di;
      if (r > 0.0) {
        const double kr = k * r;
        double sn, cs;
        sincos(kr, &sn, &cs);
        if (exact) {
          const double sh = sin(0.5 * kr);
          gr = -2.0 * sh * sh / r;
          gi = sn / r;
          const double r3 = r * r * r;
          dr = (2.0 * sh * sh - kr * sn) * dny / r3;
          di = (kr * cs - sn) * dny / r3;
        } else {
          gr = cs / r;
          gi = sn / r;
          const double r3 = r * r * r;
          dr = (-cs - kr * sn) * dny / r3;
          di = (kr * cs - sn) * dny / r3;
        }
      } else {
        gr = 0.0;
        gi = exact ? k : 0.0;
        dr = di = 0.0;
      }
      const double ws = ri.w[s] * area_b;
      for (int j = 0; j < 3; ++j) {
        const double lw = ws * ri.lam[s][j];
        vr[j] += gr * lw;
        vi[j] += gi * lw;
        kr_[j] += dr * lw;
        ki[j] += di * lw;
      }
    }
    if (exact) {
      double IV[3], IK[3];
      bem_static_potentials(x, vb, same, IV, IK);
      for (int j = 0; j < 3; ++j) {
        vr[j] += IV[j];
        kr_[j] += IK[j];
      }
    }
    const double wq = ro.w[q] * area_a;
    for (int i = 0; i < 3; ++i) {
      const double li = wq * ro.lam[q][i];
      for (int j = 0; j < 3; ++j) {
        V3.re[i][j] += li * vr[j];
        V3.im[i][j] += li * vi[j];
        K3.re[i][j] += li * kr_[j];
        K3.im[i][j] += li * ki[j];
      }
    }
  }
}

// Correction block of near pair p (T, T'): for every layer j bounding both interfaces,
//   dV = (V_near(T,T') + V_near(T',T)^T)/2 - V_far,  dK = K_near - K_far,
//   dK' = (K_near(T',T) - K_far(T',T))^T,
//   dW = (curl_i . curl'_j) sum(dV) - k_j^2 (n . n') dV,
// added with sigma_jm sigma_jl as [[-dK, rho_j dV], [dW/rho_j, dK']] (the 1/(4 pi) applied).
__global__ void bem_near_blocks_kernel(const double* __restrict__ vert, const int* __restrict__ tri,
                                       const int* __restrict__ tsurf, const double* __restrict__ geo,
                                       const int64_t* __restrict__ near_ptr, const int* __restrict__ near_tp,
                                       int64_t nt, const BemRule* __restrict__ rfar,
                                       const BemRule* __restrict__ rnear, BemDomain d0, BemDomain d1, BemDomain d2,
                                       int ndom, double2* __restrict__ blk) {
  const int64_t t = blockIdx.x;
  if (t >= nt) return;
  const BemDomain doms[3] = {d0, d1, d2};
  const BemRule& rf = *rfar;
  const BemRule& rn = *rnear;
  for (int64_t p = near_ptr[t] + threadIdx.x; p < near_ptr[t + 1]; p += blockDim.x) {
    const int64_t u = near_tp[p];
    double va[3][3], vb[3][3];
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) {
        va[i][d] = vert[3 * (int64_t)tri[3 * t + i] + d];
        vb[i][d] = vert[3 * (int64_t)tri[3 * u + i] + d];
      }
    const double* ga = geo + 24 * t;
    const double* gb = geo + 24 * u;
    const double na[3] = {ga[1], ga[2], ga[3]}, nb[3] = {gb[1], gb[2], gb[3]};
    const bool same = (t == u);
    const int sm = tsurf[t], sl = tsurf[u];
    double cre[6][6], cim[6][6];
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) cre[r][c] = cim[r][c] = 0.0;
    for (int j = 0; j < ndom; ++j) {
      const BemDomain& D = doms[j];
      const int sg = D.sigma[sm] * D.sigma[sl];
      if (sg == 0) continue;
      C3 dV, dK, dKp, tv, tk;
      bem_pair_blocks(va, ga[0], vb, gb[0], nb, D.k, rn, rn, true, same, tv, tk);
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          dV.re[a][c] = 0.5 * tv.re[a][c];
          dV.im[a][c] = 0.5 * tv.im[a][c];
          dK.re[a][c] = tk.re[a][c];
          dK.im[a][c] = tk.im[a][c];
        }
      bem_pair_blocks(vb, gb[0], va, ga[0], na, D.k, rn, rn, true, same, tv, tk);
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          dV.re[a][c] += 0.5 * tv.re[c][a];
          dV.im[a][c] += 0.5 * tv.im[c][a];
          dKp.re[a][c] = tk.re[c][a];
          dKp.im[a][c] = tk.im[c][a];
        }
      bem_pair_blocks(va, ga[0], vb, gb[0], nb, D.k, rf, rf, false, same, tv, tk);
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          dV.re[a][c] -= tv.re[a][c];
          dV.im[a][c] -= tv.im[a][c];
          dK.re[a][c] -= tk.re[a][c];
          dK.im[a][c] -= tk.im[a][c];
        }
      bem_pair_blocks(vb, gb[0], va, ga[0], na, D.k, rf, rf, false, same, tv, tk);
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          dKp.re[a][c] -= tk.re[c][a];
          dKp.im[a][c] -= tk.im[c][a];
        }
      double sre = 0.0, sim = 0.0;
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          sre += dV.re[a][c];
          sim += dV.im[a][c];
        }
      const double nn = na[0] * nb[0] + na[1] * nb[1] + na[2] * nb[2];
      const double s = sg * kInv4Pi, k2 = D.k * D.k;
      for (int a = 0; a < 3; ++a)
        for (int c = 0; c < 3; ++c) {
          const double cc = ga[8 + 3 * a] * gb[8 + 3 * c] + ga[9 + 3 * a] * gb[9 + 3 * c] +
                            ga[10 + 3 * a] * gb[10 + 3 * c];
          const double wre = cc * sre - k2 * nn * dV.re[a][c];
          const double wim = cc * sim - k2 * nn * dV.im[a][c];
          cre[a][c] += -s * dK.re[a][c];
          cim[a][c] += -s * dK.im[a][c];
          cre[a][3 + c] += s * D.rho * dV.re[a][c];
          cim[a][3 + c] += s * D.rho * dV.im[a][c];
          cre[3 + a][c] += s * wre / D.rho;
          cim[3 + a][c] += s * wim / D.rho;
          cre[3 + a][3 + c] += s * dKp.re[a][c];
          cim[3 + a][3 + c] += s * dKp.im[a][c];
        }
    }
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) blk[36 * p + 6 * r + c] = make_double2(cre[r][c], cim[r][c]);
  }
}

// ----------------------------------------------------------------- apply

// P1 traces at the far-rule points -> per-layer source charges (R precision), with the
// weight w, the sign sigma_jl, rho_j, k_j and 1/(4 pi):
//   q = rho sigma w v, uK = sigma w u, b = -k^2 sigma w u / rho, c = sigma w v,
//   a = sigma w curl(u) / rho.
// Charge k (0..13) of a source record: R precision, or (hi, lo) floats for the double-float
// records (tagged by R = dfs).
template <class R>
struct ChargeStore {
  using T = R;
  static __device__ __forceinline__ void put(R* o, int k, double v) { o[6 + k] = (R)v; }
  static constexpr int stride = kSrcRec;
};
template <>
struct ChargeStore<dfs> {
  using T = float;
  static __device__ __forceinline__ void put(float* o, int k, double v) {
    const dfs d = dfs_make(v);
    o[12 + 2 * k] = d.h;
    o[13 + 2 * k] = d.l;
  }
  static constexpr int stride = kDfSrc;
};

template <class R>
__global__ void bem_prolong_kernel(const double2* __restrict__ x, const int* __restrict__ tri,
                                   const int* __restrict__ tsurf, const int64_t* __restrict__ uidx,
                                   const int64_t* __restrict__ vidx, const double* __restrict__ geo,
                                   const double* __restrict__ qw, const BemRule* __restrict__ rule, int64_t nt,
                                   BemDomain d0, BemDomain d1, BemDomain d2, int ndom,
                                   typename ChargeStore<R>::T* __restrict__ s0,
                                   typename ChargeStore<R>::T* __restrict__ s1,
                                   typename ChargeStore<R>::T* __restrict__ s2) {
  using CS = ChargeStore<R>;
  using T = typename CS::T;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int Q = rule->q;
  double2 u[3], v[3];
  for (int i = 0; i < 3; ++i) {
    const int g = tri[3 * t + i];
    u[i] = x[uidx[g]];
    v[i] = x[vidx[g]];
  }
  const double* ge = geo + 24 * t;
  double cur[3][2];
  for (int d = 0; d < 3; ++d) {
    cur[d][0] = u[0].x * ge[8 + d] + u[1].x * ge[11 + d] + u[2].x * ge[14 + d];
    cur[d][1] = u[0].y * ge[8 + d] + u[1].y * ge[11 + d] + u[2].y * ge[14 + d];
  }
  const int sl = tsurf[t];
  const BemDomain doms[3] = {d0, d1, d2};
  T* outs[3] = {s0, s1, s2};
  for (int q = 0; q < Q; ++q) {
    const int64_t p = t * Q + q;
    double ur = 0, ui = 0, vr = 0, vi = 0;
    for (int i = 0; i < 3; ++i) {
      const double l = rule->lam[q][i];
      ur += l * u[i].x;
      ui += l * u[i].y;
      vr += l * v[i].x;
      vi += l * v[i].y;
    }
    for (int j = 0; j < ndom; ++j) {
      const BemDomain& D = doms[j];
      if (D.sigma[sl] == 0) continue;
      const double w = D.sigma[sl] * qw[p] * kInv4Pi;
      T* o = outs[j] + CS::stride * p;
      CS::put(o, 0, D.rho * w * vr);
      CS::put(o, 1, D.rho * w * vi);
      CS::put(o, 2, w * ur);
      CS::put(o, 3, w * ui);
      const double kb = -D.k * D.k * w / D.rho;
      CS::put(o, 4, kb * ur);
      CS::put(o, 5, kb * ui);
      CS::put(o, 6, w * vr);
      CS::put(o, 7, w * vi);
      for (int d = 0; d < 3; ++d) {
        CS::put(o, 8 + 2 * d, w * cur[d][0] / D.rho);
        CS::put(o, 9 + 2 * d, w * cur[d][1] / D.rho);
      }
    }
  }
}

template <class R>
__device__ __forceinline__ void bem_sincos_rev(R f, R* s, R* c);
template <>
__device__ __forceinline__ void bem_sincos_rev<float>(float f, float* s, float* c) {
  __sincosf(6.28318530717958647692f * f, s, c);
}
template <>
__device__ __forceinline__ void bem_sincos_rev<double>(double f, double* s, double* c) {
  sincospi(2.0 * f, s, c);
}
template <class R>
__device__ __forceinline__ R bem_rsqrt(R x);
template <>
__device__ __forceinline__ float bem_rsqrt<float>(float x) {
  return rsqrtf(x);
}
template <>
__device__ __forceinline__ double bem_rsqrt<double>(double x) {
  return rsqrt(x);
}

// N-body sums of one layer over its point range [p0, p0 + np): block (target block, source
// chunk); each thread kBemTgt targets; sources through shared memory in tiles of
// kBemThreads; per-tile sums in R folded into FP64.  part[chunk][i][10].
template <class R>
__global__ void __launch_bounds__(kBemThreads) bem_nbody_kernel(const R* __restrict__ tgt,
                                                                 const R* __restrict__ src, int64_t p0,
                                                                 int64_t np, R kappa, int64_t chunk,
                                                                 double* __restrict__ part) {
  __shared__ R sh[kBemThreads * kSrcRec];
  // the FP64 sums of this thread's targets live in shared memory (touched once per tile),
  // which keeps them out of the registers the pair loop needs
  __shared__ double acc[kBemTgt * kOut][kBemThreads];
  const int64_t tb = (int64_t)blockIdx.x * kBemThreads * kBemTgt;
  const int64_t c0 = (int64_t)blockIdx.y * chunk, c1 = min(np, c0 + chunk);
  R tx[kBemTgt][6];
  bool live[kBemTgt];
  for (int m = 0; m < kBemTgt; ++m) {
    const int64_t i = tb + threadIdx.x + m * kBemThreads;
    live[m] = i < np;
    for (int d = 0; d < 6; ++d) tx[m][d] = live[m] ? tgt[kTgtRec * (p0 + i) + d] : R(0);
    for (int o = 0; o < kOut; ++o) acc[m * kOut + o][threadIdx.x] = 0.0;
  }
  const R twopi = (R)6.28318530717958647692;
  for (int64_t s0 = c0; s0 < c1; s0 += kBemThreads) {
    const int ns = (int)((c1 - s0) < (int64_t)kBemThreads ? (c1 - s0) : (int64_t)kBemThreads);
    __syncthreads();
    if (threadIdx.x < ns) {
      const R* sp = src + kSrcRec * (p0 + s0 + threadIdx.x);
#pragma unroll
      for (int d = 0; d < kSrcRec; ++d) sh[kSrcRec * threadIdx.x + d] = sp[d];
    }
    __syncthreads();
    R a[kBemTgt][kOut];
    for (int m = 0; m < kBemTgt; ++m)
      for (int o = 0; o < kOut; ++o) a[m][o] = R(0);
    for (int j = 0; j < ns; ++j) {
      const R* s = sh + kSrcRec * j;
#pragma unroll
      for (int m = 0; m < kBemTgt; ++m) {
        const R dx = tx[m][0] - s[0], dy = tx[m][1] - s[1], dz = tx[m][2] - s[2];
        const R r2 = dx * dx + dy * dy + dz * dz;
        const R rinv = r2 > R(0) ? bem_rsqrt<R>(r2) : R(0);
        const R t = r2 * rinv * kappa;
        const R f = t - rint(t);
        R sn, cs;
        bem_sincos_rev<R>(f, &sn, &cs);
        const R Fr = cs * rinv, Fi = sn * rinv;
        const R rinv3 = rinv * rinv * rinv, kr = twopi * t;
        const R Er = (-cs - kr * sn) * rinv3, Ei = (kr * cs - sn) * rinv3;
        const R dns = dx * s[3] + dy * s[4] + dz * s[5];
        const R dnx = dx * tx[m][3] + dy * tx[m][4] + dz * tx[m][5];
        const R nn = tx[m][3] * s[3] + tx[m][4] * s[4] + tx[m][5] * s[5];
        // S1 += F q + E dns uK
        const R er1 = Er * dns, ei1 = Ei * dns;
        a[m][0] += Fr * s[6] - Fi * s[7] + er1 * s[8] - ei1 * s[9];
        a[m][1] += Fr * s[7] + Fi * s[6] + er1 * s[9] + ei1 * s[8];
        // S2 += F nn b + E dnx c
        const R fr2 = Fr * nn, fi2 = Fi * nn, er2 = Er * dnx, ei2 = Ei * dnx;
        a[m][2] += fr2 * s[10] - fi2 * s[11] + er2 * s[12] - ei2 * s[13];
        a[m][3] += fr2 * s[11] + fi2 * s[10] + er2 * s[13] + ei2 * s[12];
        // A += F a
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          a[m][4 + 2 * d] += Fr * s[14 + 2 * d] - Fi * s[15 + 2 * d];
          a[m][5 + 2 * d] += Fr * s[15 + 2 * d] + Fi * s[14 + 2 * d];
        }
      }
    }
    for (int m = 0; m < kBemTgt; ++m)
      for (int o = 0; o < kOut; ++o) acc[m * kOut + o][threadIdx.x] += (double)a[m][o];
  }
  for (int m = 0; m < kBemTgt; ++m) {
    const int64_t i = tb + threadIdx.x + m * kBemThreads;
    if (!live[m]) continue;
    double* out = part + ((int64_t)blockIdx.y * np + i) * kOut;
    for (int o = 0; o < kOut; ++o) out[o] = acc[m * kOut + o][threadIdx.x];
  }
}

// Double-float N-body sums of one layer (FP64-class accuracy on the FP32 pipe): one target
// per thread, every operation of the pair evaluation in double-float (positions,
// 1/r by a Newton-refined rsqrt, the phase kappa r reduced to revolutions, cos and sin of
// 2 pi f by the library's Taylor evaluation, the five complex sums), per-tile sums folded into
// FP64.  kappa = k/(2 pi) as a double-float.  part[chunk][i][10] as the other N-body kernels.
__global__ void __launch_bounds__(kDfThreads) bem_nbody_df_kernel(const float* __restrict__ tgt,
                                                                   const float* __restrict__ src, int64_t p0,
                                                                   int64_t np, float kap_h, float kap_l,
                                                                   int64_t chunk, double* __restrict__ part) {
  __shared__ float sh[kDfTile * kDfSrc];
  __shared__ double acc[kOut][kDfThreads];
  const int64_t i = (int64_t)blockIdx.x * kDfThreads + threadIdx.x;
  const int64_t c0 = (int64_t)blockIdx.y * chunk, c1 = min(np, c0 + chunk);
  const bool live = i < np;
  dfs t[6];
  for (int d = 0; d < 6; ++d)
    t[d] = live ? dfs{tgt[kDfTgt * (p0 + i) + 2 * d], tgt[kDfTgt * (p0 + i) + 2 * d + 1]} : dfs{0.0f, 0.0f};
  for (int o = 0; o < kOut; ++o) acc[o][threadIdx.x] = 0.0;
  const dfs kap{kap_h, kap_l};
  for (int64_t s0 = c0; s0 < c1; s0 += kDfTile) {
    const int ns = (int)((c1 - s0) < (int64_t)kDfTile ? (c1 - s0) : (int64_t)kDfTile);
    __syncthreads();
    for (int e = threadIdx.x; e < ns * kDfSrc; e += kDfThreads) sh[e] = src[kDfSrc * (p0 + s0) + e];
    __syncthreads();
    dfs a[kOut];
    for (int o = 0; o < kOut; ++o) a[o] = dfs{0.0f, 0.0f};
    for (int j = 0; j < ns; ++j) {
      const float* s = sh + kDfSrc * j;
      const dfs dx = dfs_sub(t[0], dfs{s[0], s[1]});
      const dfs dy = dfs_sub(t[1], dfs{s[2], s[3]});
      const dfs dz = dfs_sub(t[2], dfs{s[4], s[5]});
      const dfs r2 = dfs_add(dfs_add(dfs_sqr(dx), dfs_sqr(dy)), dfs_sqr(dz));
      if (!(r2.h > 0.0f)) continue;  // zero distance contributes nothing
      const dfs rinv = dfs_rsqrt(r2);
      const dfs tt = dfs_mul(dfs_mul(r2, rinv), kap);  // kr / (2 pi)
      const float nr = rintf(tt.h);
      dfs cs, sn;
      dfs_cossin_2pi(dfs_two_sum(__fsub_rn(tt.h, nr), tt.l), cs, sn);
      const dfs Fr = dfs_mul(cs, rinv), Fi = dfs_mul(sn, rinv);
      const dfs rinv3 = dfs_mul(dfs_sqr(rinv), rinv);
      const dfs kr = dfs_mul(tt, dfc_two_pi());
      const dfs Er = dfs_neg(dfs_mul(dfs_add(cs, dfs_mul(kr, sn)), rinv3));
      const dfs Ei = dfs_mul(dfs_sub(dfs_mul(kr, cs), sn), rinv3);
      const dfs snx{s[6], s[7]}, sny{s[8], s[9]}, snz{s[10], s[11]};
      const dfs dns = dfs_add(dfs_add(dfs_mul(dx, snx), dfs_mul(dy, sny)), dfs_mul(dz, snz));
      const dfs dnx = dfs_add(dfs_add(dfs_mul(dx, t[3]), dfs_mul(dy, t[4])), dfs_mul(dz, t[5]));
      const dfs nn = dfs_add(dfs_add(dfs_mul(t[3], snx), dfs_mul(t[4], sny)), dfs_mul(t[5], snz));
      // charge k at s[12 + 2k], s[13 + 2k]
#define BEM_CH(k) dfs{s[12 + 2 * (k)], s[13 + 2 * (k)]}
      // S1 += F q + (E dns) uK
      const dfs e1r = dfs_mul(Er, dns), e1i = dfs_mul(Ei, dns);
      a[0] = dfs_add(a[0], dfs_sub(dfs_add(dfs_mul(Fr, BEM_CH(0)), dfs_mul(e1r, BEM_CH(2))),
                                   dfs_add(dfs_mul(Fi, BEM_CH(1)), dfs_mul(e1i, BEM_CH(3)))));
      a[1] = dfs_add(a[1], dfs_add(dfs_add(dfs_mul(Fr, BEM_CH(1)), dfs_mul(Fi, BEM_CH(0))),
                                   dfs_add(dfs_mul(e1r, BEM_CH(3)), dfs_mul(e1i, BEM_CH(2)))));
      // S2 += (F nn) b + (E dnx) c
      const dfs f2r = dfs_mul(Fr, nn), f2i = dfs_mul(Fi, nn);
      const dfs e2r = dfs_mul(Er, dnx), e2i = dfs_mul(Ei, dnx);
      a[2] = dfs_add(a[2], dfs_sub(dfs_add(dfs_mul(f2r, BEM_CH(4)), dfs_mul(e2r, BEM_CH(6))),
                                   dfs_add(dfs_mul(f2i, BEM_CH(5)), dfs_mul(e2i, BEM_CH(7)))));
      a[3] = dfs_add(a[3], dfs_add(dfs_add(dfs_mul(f2r, BEM_CH(5)), dfs_mul(f2i, BEM_CH(4))),
                                   dfs_add(dfs_mul(e2r, BEM_CH(7)), dfs_mul(e2i, BEM_CH(6)))));
      // A += F a
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        a[4 + 2 * d] = dfs_add(a[4 + 2 * d], dfs_sub(dfs_mul(Fr, BEM_CH(8 + 2 * d)), dfs_mul(Fi, BEM_CH(9 + 2 * d))));
        a[5 + 2 * d] = dfs_add(a[5 + 2 * d], dfs_add(dfs_mul(Fr, BEM_CH(9 + 2 * d)), dfs_mul(Fi, BEM_CH(8 + 2 * d))));
      }
#undef BEM_CH
    }
    for (int o = 0; o < kOut; ++o) acc[o][threadIdx.x] += dfs_value(a[o]);
  }
  if (live) {
    double* out = part + ((int64_t)blockIdx.y * np + i) * kOut;
    for (int o = 0; o < kOut; ++o) out[o] = acc[o][threadIdx.x];
  }
}

// pout[p0 + i] += sigma(surface of the point) * sum_chunk part[chunk][i] (fixed order).
__global__ void bem_reduce_kernel(const double* __restrict__ part, int64_t np, int nchunk, int64_t p0,
                                  int64_t q_split, int sig0, int sig1, double* __restrict__ pout) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= np * kOut) return;
  double s = 0.0;
  for (int c = 0; c < nchunk; ++c) s += part[(int64_t)c * np * kOut + e];
  const int64_t p = p0 + e / kOut;
  const int sg = p < q_split ? sig0 : sig1;
  pout[p0 * kOut + e] += sg * s;
}

// Local P1 rows of triangle T: from the N-body sums at its points
//   Z1_i = sum_q w_q lambda_i S1,  Z2_i = curl_i . sum_q w_q A + sum_q w_q lambda_i S2,
// plus the near corrections C_{TT'} (u_T', v_T').
__global__ void bem_restrict_kernel(const double* __restrict__ pout, const double* __restrict__ qw,
                                    const BemRule* __restrict__ rule, const double* __restrict__ geo,
                                    const int64_t* __restrict__ near_ptr, const int* __restrict__ near_tp,
                                    const double2* __restrict__ blk, const double2* __restrict__ x,
                                    const int* __restrict__ tri, const int64_t* __restrict__ uidx,
                                    const int64_t* __restrict__ vidx, int64_t nt, double2* __restrict__ zloc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int Q = rule->q;
  double zr[6] = {0, 0, 0, 0, 0, 0}, zi[6] = {0, 0, 0, 0, 0, 0};
  double Ar[3] = {0, 0, 0}, Ai[3] = {0, 0, 0};
  for (int q = 0; q < Q; ++q) {
    const int64_t p = t * Q + q;
    const double w = qw[p];
    const double* o = pout + kOut * p;
    for (int i = 0; i < 3; ++i) {
      const double l = w * rule->lam[q][i];
      zr[i] += l * o[0];
      zi[i] += l * o[1];
      zr[3 + i] += l * o[2];
      zi[3 + i] += l * o[3];
    }
    for (int d = 0; d < 3; ++d) {
      Ar[d] += w * o[4 + 2 * d];
      Ai[d] += w * o[5 + 2 * d];
    }
  }
  const double* ge = geo + 24 * t;
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) {
      zr[3 + i] += ge[8 + 3 * i + d] * Ar[d];
      zi[3 + i] += ge[8 + 3 * i + d] * Ai[d];
    }
  for (int64_t k = near_ptr[t]; k < near_ptr[t + 1]; ++k) {
    const int u = near_tp[k];
    double2 y[6];
    for (int j = 0; j < 3; ++j) {
      const int g = tri[3 * (int64_t)u + j];
      y[j] = x[uidx[g]];
      y[3 + j] = x[vidx[g]];
    }
    const double2* C = blk + 36 * k;
    for (int r = 0; r < 6; ++r)
      for (int c = 0; c < 6; ++c) {
        const double2 m = C[6 * r + c];
        zr[r] += m.x * y[c].x - m.y * y[c].y;
        zi[r] += m.x * y[c].y + m.y * y[c].x;
      }
  }
  for (int r = 0; r < 6; ++r) zloc[6 * t + r] = make_double2(zr[r], zi[r]);
}

// y at the vertex's u and v unknowns: its triangles' local rows (in triangle order) / m_a.
__global__ void bem_gather_kernel(const double2* __restrict__ zloc, const int64_t* __restrict__ vt_ptr,
                                  const int* __restrict__ vt_idx, const double* __restrict__ lmass,
                                  const int64_t* __restrict__ uidx, const int64_t* __restrict__ vidx, int64_t nv,
                                  double2* __restrict__ y) {
  const int64_t a = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (a >= nv) return;
  double ur = 0, ui = 0, vr = 0, vi = 0;
  for (int64_t k = vt_ptr[a]; k < vt_ptr[a + 1]; ++k) {
    const int e = vt_idx[k];
    const int64_t t = e / 3;
    const int i = e - 3 * (int)t;
    const double2 zu = zloc[6 * t + i], zv = zloc[6 * t + 3 + i];
    ur += zu.x;
    ui += zu.y;
    vr += zv.x;
    vi += zv.y;
  }
  const double m = lmass[a];
  y[uidx[a]] = make_double2(ur / m, ui / m);
  y[vidx[a]] = make_double2(vr / m, vi / m);
}

// Local right-hand side rows: interface-1 triangles get
//   (sum_q w lambda_i p_inc, sum_q w lambda_i (i k0 d.n / rho0) p_inc); others zero.
__global__ void bem_rhs_kernel(const double* __restrict__ tgt64, const double* __restrict__ qw,
                               const BemRule* __restrict__ rule, const int* __restrict__ tsurf, int64_t nt,
                               double k0, double rho0, double dx, double dy, double dz, double2* __restrict__ zloc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double zr[6] = {0, 0, 0, 0, 0, 0}, zi[6] = {0, 0, 0, 0, 0, 0};
  if (tsurf[t] == 0) {
    const int Q = rule->q;
    for (int q = 0; q < Q; ++q) {
      const int64_t p = t * Q + q;
      const double* g = tgt64 + 6 * p;
      double sn, cs;
      sincos(k0 * (g[0] * dx + g[1] * dy + g[2] * dz), &sn, &cs);
      const double dn = k0 * (g[3] * dx + g[4] * dy + g[5] * dz) / rho0;  // i dn p_inc
      for (int i = 0; i < 3; ++i) {
        const double l = qw[p] * rule->lam[q][i];
        zr[i] += l * cs;
        zi[i] += l * sn;
        zr[3 + i] += -l * dn * sn;
        zi[3 + i] += l * dn * cs;
      }
    }
  }
  for (int r = 0; r < 6; ++r) zloc[6 * t + r] = make_double2(zr[r], zi[r]);
}

// p_inf(xhat_m) = (1/4 pi) sum over interface-1 points of w e^{-i k0 xhat.y}
// [-i k0 (xhat.n) u - rho0 v]; one block per direction, fixed-order tree reduction.
__global__ void bem_far_field_kernel(const double2* __restrict__ x, const double* __restrict__ tgt64,
                                     const double* __restrict__ qw, const BemRule* __restrict__ rule,
                                     const int* __restrict__ tri, const int64_t* __restrict__ uidx,
                                     const int64_t* __restrict__ vidx, int64_t nt1, const double* __restrict__ dirs,
                                     double k0, double rho0, double2* __restrict__ out) {
  __shared__ double sr[256], si[256];
  const int m = blockIdx.x;
  const double hx = dirs[3 * m], hy = dirs[3 * m + 1], hz = dirs[3 * m + 2];
  const int Q = rule->q;
  double ar = 0.0, ai = 0.0;
  for (int64_t p = threadIdx.x; p < nt1 * Q; p += blockDim.x) {
    const int64_t t = p / Q;
    const int q = (int)(p - t * Q);
    double ur = 0, ui = 0, vr = 0, vi = 0;
    for (int i = 0; i < 3; ++i) {
      const int g = tri[3 * t + i];
      const double l = rule->lam[q][i];
      const double2 a = x[uidx[g]], b = x[vidx[g]];
      ur += l * a.x;
      ui += l * a.y;
      vr += l * b.x;
      vi += l * b.y;
    }
    const double* g = tgt64 + 6 * p;
    double sn, cs;
    sincos(-k0 * (hx * g[0] + hy * g[1] + hz * g[2]), &sn, &cs);
    const double xn = k0 * (hx * g[3] + hy * g[4] + hz * g[5]);
    // amp = -i xn u - rho0 v
    const double amr = xn * ui - rho0 * vr, ami = -xn * ur - rho0 * vi;
    const double w = qw[p];
    ar += w * (cs * amr - sn * ami);
    ai += w * (cs * ami + sn * amr);
  }
  sr[threadIdx.x] = ar;
  si[threadIdx.x] = ai;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      sr[threadIdx.x] += sr[threadIdx.x + s];
      si[threadIdx.x] += si[threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[m] = make_double2(sr[0] * kInv4Pi, si[0] * kInv4Pi);
}

// ----------------------------------------------------------------- host side

// Source chunks of a layer's N-body launch: about two waves of 7 resident blocks on every
// SM, chunks of at least 512 sources.
static int bem_nchunk(int64_t np) {
  const int64_t tblocks = (np + kBemThreads * kBemTgt - 1) / (kBemThreads * kBemTgt);
  const int64_t want = (14 * 148 + tblocks - 1) / std::max<int64_t>(1, tblocks);
  const int64_t most = std::max<int64_t>(1, np / (4 * kBemThreads));
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, most, 64}));
}

// The same for the double-float launch (one target per thread, 128 per block).
static int bem_nchunk_df(int64_t np) {
  const int64_t tblocks = (np + kDfThreads - 1) / kDfThreads;
  const int64_t want = (8 * 148 + tblocks - 1) / std::max<int64_t>(1, tblocks);
  const int64_t most = std::max<int64_t>(1, np / (4 * kDfTile));
  return (int)std::max<int64_t>(1, std::min<int64_t>({want, most, 64}));
}

static vsie_status bem_apply_impl(vsie_bem* b, const double2* x, double2* y, int precision, cudaStream_t st) {
  const int64_t nt = b->nt;
  if (precision == 48)
    bem_prolong_kernel<dfs><<<nblk(nt, 128), 128, 0, st>>>(x, b->tri, b->tsurf, b->uidx, b->vidx, b->tgeo, b->qw,
                                                           b->d_far, nt, b->dom[0], b->dom[1], b->dom[2], b->ndom,
                                                           b->srcdf[0], b->srcdf[1], b->srcdf[2]);
  else if (precision == 32)
    bem_prolong_kernel<float><<<nblk(nt, 128), 128, 0, st>>>(x, b->tri, b->tsurf, b->uidx, b->vidx, b->tgeo, b->qw,
                                                             b->d_far, nt, b->dom[0], b->dom[1], b->dom[2], b->ndom,
                                                             b->src32[0], b->src32[1], b->src32[2]);
  else
    bem_prolong_kernel<double><<<nblk(nt, 128), 128, 0, st>>>(x, b->tri, b->tsurf, b->uidx, b->vidx, b->tgeo,
                                                              b->qw, b->d_far, nt, b->dom[0], b->dom[1], b->dom[2],
                                                              b->ndom, b->src64[0], b->src64[1], b->src64[2]);
  VSIE_CUDA(cudaGetLastError());
  VSIE_CUDA(cudaMemsetAsync(b->pout, 0, sizeof(double) * kOut * b->nq, st));
  for (int j = 0; j < b->ndom; ++j) {
    const BemDomain& D = b->dom[j];
    const bool df = precision == 48;
    const int nch = df ? bem_nchunk_df(D.np) : bem_nchunk(D.np);
    const int64_t chunk = (D.np + nch - 1) / nch;
    const dim3 grid((unsigned)(df ? (D.np + kDfThreads - 1) / kDfThreads
                                  : (D.np + kBemThreads * kBemTgt - 1) / (kBemThreads * kBemTgt)),
                    (unsigned)nch);
    const double kappa = D.k / (2.0 * kBPi);
    if (df) {
      const float kh = (float)kappa;
      bem_nbody_df_kernel<<<grid, kDfThreads, 0, st>>>(b->tgtdf, b->srcdf[j], D.p0, D.np, kh,
                                                       (float)(kappa - (double)kh), chunk, b->part);
    } else if (precision == 32)
      bem_nbody_kernel<float><<<grid, kBemThreads, 0, st>>>(b->tgt32, b->src32[j], D.p0, D.np, (float)kappa, chunk,
                                                            b->part);
    else
      bem_nbody_kernel<double><<<grid, kBemThreads, 0, st>>>(b->tgt64, b->src64[j], D.p0, D.np, kappa, chunk,
                                                             b->part);
    VSIE_CUDA(cudaGetLastError());
    const int64_t q_split = b->nsurf > 1 ? b->t_off[1] * b->far.q : b->nq;
    bem_reduce_kernel<<<nblk(D.np * kOut), 256, 0, st>>>(b->part, D.np, nch, D.p0, q_split, D.sigma[0],
                                                         D.sigma[1], b->pout);
    VSIE_CUDA(cudaGetLastError());
  }
  bem_restrict_kernel<<<nblk(nt, 128), 128, 0, st>>>(b->pout, b->qw, b->d_far, b->tgeo, b->near_ptr, b->near_tp,
                                                      b->near_blk, x, b->tri, b->uidx, b->vidx, nt, b->zloc);
  VSIE_CUDA(cudaGetLastError());
  bem_gather_kernel<<<nblk(b->nv), 256, 0, st>>>(b->zloc, b->vt_ptr, b->vt_idx, b->lmass, b->uidx, b->vidx, b->nv,
                                                 y);
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

static vsie_status bem_build(vsie_bem* b, const vsie_bem_desc* d) {
  // host arrays
  std::vector<double> vert(3 * b->nv);
  std::vector<int> tri(3 * b->nt), tsurf(b->nt);
  std::vector<int64_t> uidx(b->nv), vidx(b->nv);
  for (int m = 0; m < b->nsurf; ++m) {
    for (int64_t i = 0; i < 3 * b->nv_s[m]; ++i) vert[3 * b->v_off[m] + i] = d->h_vert[m][i];
    for (int64_t t = 0; t < b->nt_s[m]; ++t) {
      for (int i = 0; i < 3; ++i) tri[3 * (b->t_off[m] + t) + i] = (int)(d->h_tri[m][3 * t + i] + b->v_off[m]);
      tsurf[b->t_off[m] + t] = m;
    }
    for (int64_t a = 0; a < b->nv_s[m]; ++a) {
      uidx[b->v_off[m] + a] = 2 * b->v_off[m] + a;
      vidx[b->v_off[m] + a] = 2 * b->v_off[m] + b->nv_s[m] + a;
    }
  }
  // vertex -> (triangle, corner), triangles in increasing order
  std::vector<int64_t> vt_ptr(b->nv + 1, 0);
  for (int64_t e = 0; e < 3 * b->nt; ++e) ++vt_ptr[tri[e] + 1];
  for (int64_t a = 0; a < b->nv; ++a) vt_ptr[a + 1] += vt_ptr[a];
  std::vector<int> vt_idx(3 * b->nt);
  {
    std::vector<int64_t> fill(vt_ptr.begin(), vt_ptr.end() - 1);
    for (int64_t e = 0; e < 3 * b->nt; ++e) vt_idx[fill[tri[e]]++] = (int)e;
  }
  for (int64_t a = 0; a < b->nv; ++a)
    if (vt_ptr[a + 1] == vt_ptr[a]) {
      set_error("vsie_bem_create: a vertex belongs to no triangle (not a closed surface mesh)");
      return VSIE_ERR_MESH;
    }
  const int Q = b->far.q;
  b->nq = b->nt * Q;
  VSIE_TRY(balloc_t(b, &b->vert, vert.size()));
  VSIE_TRY(balloc_t(b, &b->tri, tri.size()));
  VSIE_TRY(balloc_t(b, &b->tsurf, tsurf.size()));
  VSIE_TRY(balloc_t(b, &b->uidx, uidx.size()));
  VSIE_TRY(balloc_t(b, &b->vidx, vidx.size()));
  VSIE_TRY(balloc_t(b, &b->vt_ptr, vt_ptr.size()));
  VSIE_TRY(balloc_t(b, &b->vt_idx, vt_idx.size()));
  VSIE_TRY(balloc_t(b, &b->tgeo, (size_t)24 * b->nt));
  VSIE_TRY(balloc_t(b, &b->lmass, (size_t)b->nv));
  VSIE_TRY(balloc_t(b, &b->d_far, 1));
  VSIE_TRY(balloc_t(b, &b->d_near, 1));
  VSIE_TRY(balloc_t(b, &b->qw, (size_t)b->nq));
  VSIE_TRY(balloc_t(b, &b->tgt64, (size_t)6 * b->nq));
  VSIE_TRY(balloc_t(b, &b->tgt32, (size_t)6 * b->nq));
  VSIE_TRY(balloc_t(b, &b->pout, (size_t)kOut * b->nq));
  VSIE_TRY(balloc_t(b, &b->zloc, (size_t)6 * b->nt));
  VSIE_TRY(balloc_t(b, &b->near_ptr, (size_t)b->nt + 1));
  VSIE_TRY(balloc_t(b, &b->tgtdf, (size_t)kDfTgt * b->nq));
  for (int j = 0; j < b->ndom; ++j) {
    VSIE_TRY(balloc_t(b, &b->src64[j], (size_t)kSrcRec * b->nq));
    VSIE_TRY(balloc_t(b, &b->src32[j], (size_t)kSrcRec * b->nq));
    VSIE_TRY(balloc_t(b, &b->srcdf[j], (size_t)kDfSrc * b->nq));
  }
  size_t part = 0;
  for (int j = 0; j < b->ndom; ++j)
    part = std::max(part, (size_t)std::max(bem_nchunk(b->dom[j].np), bem_nchunk_df(b->dom[j].np)) *
                              (size_t)b->dom[j].np * kOut);
  VSIE_TRY(balloc_t(b, &b->part, part));
  b->part_elems = part;
  int* d_bad = nullptr;
  VSIE_TRY(balloc_t(b, &d_bad, 1));
  int64_t* d_count = nullptr;
  VSIE_TRY(balloc_t(b, &d_count, (size_t)b->nt));
  VSIE_CUDA(cudaMemcpy(b->vert, vert.data(), sizeof(double) * vert.size(), cudaMemcpyHostToDevice));
  VSIE_CUDA(cudaMemcpy(b->tri, tri.data(), sizeof(int) * tri.size(), cudaMemcpyHostToDevice));
  VSIE_CUDA(cudaMemcpy(b->tsurf, tsurf.data(), sizeof(int) * tsurf.size(), cudaMemcpyHostToDevice));
  VSIE_CUDA(cudaMemcpy(b->uidx, uidx.data(), sizeof(int64_t) * uidx.size(), cudaMemcpyHostToDevice));
  VSIE_CUDA(cudaMemcpy(b->vidx, vidx.data(), sizeof(int64_t) * vidx.size(), cudaMemcpyHostToDevice));
  VSIE_CUDA(cudaMemcpy(b->vt_ptr, vt_ptr.data(), sizeof(int64_t) * vt_ptr.size(), cudaMemcpyHostToDevice));
  VSIE_CUDA(cudaMemcpy(b->vt_idx, vt_idx.data(), sizeof(int) * vt_idx.size(), cudaMemcpyHostToDevice));
  VSIE_CUDA(cudaMemcpy(b->d_far, &b->far, sizeof(BemRule), cudaMemcpyHostToDevice));
  VSIE_CUDA(cudaMemcpy(b->d_near, &b->nearr, sizeof(BemRule), cudaMemcpyHostToDevice));
  VSIE_CUDA(cudaMemset(d_bad, 0, sizeof(int)));
  bem_geom_kernel<<<nblk(b->nt), 256>>>(b->vert, b->tri, b->nt, b->tgeo, d_bad);
  VSIE_CUDA(cudaGetLastError());
  int bad = 0;
  VSIE_CUDA(cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost));
  if (bad) {
    set_error("vsie_bem_create: a triangle has zero area");
    return VSIE_ERR_MESH;
  }
  bem_points_kernel<<<nblk(b->nq), 256>>>(b->vert, b->tri, b->tgeo, b->d_far, b->nt, b->qw, b->tgt64, b->tgt32);
  bem_lumped_kernel<<<nblk(b->nv), 256>>>(b->vt_ptr, b->vt_idx, b->tgeo, b->nv, b->lmass);
  for (int j = 0; j < b->ndom; ++j) {
    bem_src_geom_kernel<double><<<nblk(b->nq), 256>>>(b->tgt64, b->nq, b->src64[j]);
    bem_src_geom_kernel<float><<<nblk(b->nq), 256>>>(b->tgt64, b->nq, b->src32[j]);
  }
  bem_df_geom_kernel<<<nblk(b->nq), 256>>>(b->tgt64, b->nq, b->tgtdf, b->srcdf[0], b->srcdf[1], b->srcdf[2]);
  VSIE_CUDA(cudaGetLastError());
  // near pairs: interfaces 0 and 1 bound a common layer when one layer touches both
  int touch01 = 0;
  for (int j = 0; j < b->ndom; ++j) touch01 |= (b->dom[j].sigma[0] != 0 && b->dom[j].sigma[1] != 0);
  const double nf2 = b->near_factor * b->near_factor;
  bem_near_kernel<<<nblk(b->nt, 128), 128>>>(b->tgeo, b->tri, b->tsurf, b->nt, nf2, touch01, d_count, nullptr,
                                              nullptr);
  VSIE_CUDA(cudaGetLastError());
  std::vector<int64_t> cnt(b->nt), ptr(b->nt + 1, 0);
  VSIE_CUDA(cudaMemcpy(cnt.data(), d_count, sizeof(int64_t) * b->nt, cudaMemcpyDeviceToHost));
  for (int64_t t = 0; t < b->nt; ++t) ptr[t + 1] = ptr[t] + cnt[t];
  b->nnear = ptr[b->nt];
  VSIE_CUDA(cudaMemcpy(b->near_ptr, ptr.data(), sizeof(int64_t) * ptr.size(), cudaMemcpyHostToDevice));
  VSIE_TRY(balloc_t(b, &b->near_tp, (size_t)b->nnear));
  VSIE_TRY(balloc_t(b, &b->near_blk, (size_t)36 * b->nnear));
  bem_near_kernel<<<nblk(b->nt, 128), 128>>>(b->tgeo, b->tri, b->tsurf, b->nt, nf2, touch01, nullptr, b->near_ptr,
                                              b->near_tp);
  VSIE_CUDA(cudaGetLastError());
  bem_near_blocks_kernel<<<(unsigned)b->nt, 32>>>(b->vert, b->tri, b->tsurf, b->tgeo, b->near_ptr, b->near_tp, b->nt,
                                                  b->d_far, b->d_near, b->dom[0], b->dom[1], b->dom[2], b->ndom,
                                                  b->near_blk);
  VSIE_CUDA(cudaGetLastError());
  VSIE_CUDA(cudaDeviceSynchronize());
  return VSIE_OK;
}

}  // namespace vsie

extern "C" vsie_status vsie_bem_create(const vsie_bem_desc* d, vsie_bem** out) {
  clear_error();
  TraceRange trace("vsie_bem_create");
  if (out) *out = nullptr;
  if (!d || !out) {
    set_error("vsie_bem_create: null argument");
    return VSIE_ERR_ARG;
  }
  if (d->n_interfaces != 1 && d->n_interfaces != 2) {
    set_error("vsie_bem_create: n_interfaces must be 1 or 2");
    return VSIE_ERR_ARG;
  }
  const int far_order = d->far_order ? d->far_order : 3, near_order = d->near_order ? d->near_order : 4;
  const double nf = d->near_factor > 0.0 ? d->near_factor : (d->near_factor == 0.0 ? 2.0 : -1.0);
  if (far_order < 1 || far_order > kBemMaxOrder || near_order < 1 || near_order > kBemMaxOrder || nf < 0.0) {
    set_error("vsie_bem_create: far_order and near_order must lie in 1..8 and near_factor must be >= 0");
    return VSIE_ERR_ARG;
  }
  if (!(d->k0 > 0.0) || !(d->rho0 > 0.0) || !(d->c0 > 0.0)) {
    set_error("vsie_bem_create: k0, rho0 and c0 must be positive");
    return VSIE_ERR_ARG;
  }
  for (int m = 0; m < d->n_interfaces; ++m) {
    if (!d->h_vert[m] || !d->h_tri[m]) {
      set_error("vsie_bem_create: null vertex or triangle array");
      return VSIE_ERR_ARG;
    }
    if (d->n_vert[m] < 4 || d->n_tri[m] < 4 || d->n_vert[m] > (1ll << 30) || d->n_tri[m] > (1ll << 30)) {
      set_error("vsie_bem_create: every interface needs at least 4 vertices and 4 triangles");
      return VSIE_ERR_ARG;
    }
    if (!(d->rho[m] > 0.0) || !(d->c[m] > 0.0)) {
      set_error("vsie_bem_create: layer densities and sound speeds must be positive");
      return VSIE_ERR_ARG;
    }
    for (int64_t e = 0; e < 3 * d->n_tri[m]; ++e)
      if (d->h_tri[m][e] < 0 || d->h_tri[m][e] >= d->n_vert[m]) {
        set_error("vsie_bem_create: a triangle's vertex index is out of range");
        return VSIE_ERR_MESH;
      }
  }
  vsie_bem* b = new vsie_bem();
  cudaGetDevice(&b->device);
  b->nsurf = d->n_interfaces;
  for (int m = 0; m < b->nsurf; ++m) {
    b->nv_s[m] = d->n_vert[m];
    b->nt_s[m] = d->n_tri[m];
    b->v_off[m] = m ? b->v_off[m - 1] + b->nv_s[m - 1] : 0;
    b->t_off[m] = m ? b->t_off[m - 1] + b->nt_s[m - 1] : 0;
  }
  b->nv = b->v_off[b->nsurf - 1] + b->nv_s[b->nsurf - 1];
  b->nt = b->t_off[b->nsurf - 1] + b->nt_s[b->nsurf - 1];
  b->n = 2 * b->nv;
  b->k0 = d->k0;
  b->rho0 = d->rho0;
  b->near_factor = nf;
  b->far = make_rule(far_order);
  b->nearr = make_rule(near_order);
  const double omega = d->k0 * d->c0;
  const int64_t Q = b->far.q;
  b->ndom = b->nsurf + 1;
  for (int j = 0; j < b->ndom; ++j) {
    BemDomain& D = b->dom[j];
    D.sigma[0] = D.sigma[1] = 0;
    if (j == 0) {
      D.k = d->k0;
      D.rho = d->rho0;
      D.sigma[0] = -1;
    } else {
      D.k = omega / d->c[j - 1];
      D.rho = d->rho[j - 1];
      D.sigma[j - 1] = +1;
      if (j < b->nsurf) D.sigma[j] = -1;
    }
    int lo = 2, hi = -1;
    for (int m = 0; m < b->nsurf; ++m)
      if (D.sigma[m]) {
        lo = std::min(lo, m);
        hi = std::max(hi, m);
      }
    D.p0 = b->t_off[lo] * Q;
    D.np = (b->t_off[hi] + b->nt_s[hi]) * Q - D.p0;
  }
  for (int j = b->ndom; j < 3; ++j) b->dom[j] = BemDomain{0.0, 1.0, {0, 0}, 0, 0};
  const vsie_status s = bem_build(b, d);
  if (s != VSIE_OK) {
    vsie_bem_destroy(b);
    return s;
  }
  *out = b;
  return VSIE_OK;
}

extern "C" void vsie_bem_destroy(vsie_bem* b) {
  if (!b) return;
  int prev = 0;
  cudaGetDevice(&prev);
  cudaSetDevice(b->device);
  for (void* p : b->allocs) cudaFree(p);
  cudaSetDevice(prev);
  delete b;
}

extern "C" vsie_status vsie_bem_sizes(const vsie_bem* b, int64_t* n_unknowns, int64_t* n_points,
                                      int64_t* n_near_pairs) {
  clear_error();
  if (!b) {
    set_error("vsie_bem_sizes: null handle");
    return VSIE_ERR_ARG;
  }
  if (n_unknowns) *n_unknowns = b->n;
  if (n_points) *n_points = b->nq;
  if (n_near_pairs) *n_near_pairs = b->nnear;
  return VSIE_OK;
}

extern "C" vsie_status vsie_bem_apply(vsie_bem* b, const void* d_x, void* d_y, int32_t precision, void* stream) {
  clear_error();
  TraceRange trace("vsie_bem_apply");
  if (!b || !d_x || !d_y || d_x == d_y || (precision != 32 && precision != 48 && precision != 64)) {
    set_error("vsie_bem_apply: null or aliased vectors, or precision not 32/48/64");
    return VSIE_ERR_ARG;
  }
  return bem_apply_impl(b, (const double2*)d_x, (double2*)d_y, precision, (cudaStream_t)stream);
}

extern "C" vsie_status vsie_bem_rhs(vsie_bem* b, const double* h_direction, void* d_b, void* stream) {
  clear_error();
  TraceRange trace("vsie_bem_rhs");
  if (!b || !h_direction || !d_b) {
    set_error("vsie_bem_rhs: null argument");
    return VSIE_ERR_ARG;
  }
  const double nd = std::sqrt(h_direction[0] * h_direction[0] + h_direction[1] * h_direction[1] +
                              h_direction[2] * h_direction[2]);
  if (!(nd > 0.0)) {
    set_error("vsie_bem_rhs: zero direction");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  bem_rhs_kernel<<<nblk(b->nt, 128), 128, 0, st>>>(b->tgt64, b->qw, b->d_far, b->tsurf, b->nt, b->k0, b->rho0,
                                                    h_direction[0] / nd, h_direction[1] / nd, h_direction[2] / nd,
                                                    b->zloc);
  VSIE_CUDA(cudaGetLastError());
  bem_gather_kernel<<<nblk(b->nv), 256, 0, st>>>(b->zloc, b->vt_ptr, b->vt_idx, b->lmass, b->uidx, b->vidx, b->nv,
                                                 (double2*)d_b);
  VSIE_CUDA(cudaGetLastError());
  return VSIE_OK;
}

extern "C" vsie_status vsie_bem_solve(vsie_bem* b, const void* d_b, void* d_x, const vsie_solve_opts* opts,
                                      vsie_solve_info* info, void* stream) {
  clear_error();
  TraceRange trace("vsie_bem_solve");
  if (!b || !d_b || !d_x || !opts || d_b == d_x) {
    set_error("vsie_bem_solve: null or aliased argument");
    return VSIE_ERR_ARG;
  }
  if ((opts->mode != 32 && opts->mode != 64) || !(opts->tol > 0.0) || opts->max_iters < 1 || opts->restart < 0 ||
      (opts->mode == 32 && !(opts->inner_tol > 0.0)) || opts->adjoint || opts->initial_guess) {
    set_error("vsie_bem_solve: invalid options (adjoint and initial_guess are not supported)");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  const ApplyFn apply = [&](const double2* x, double2* y, int prec) { return bem_apply_impl(b, x, y, prec, st); };
  // refinement residuals of mode 32 with the double-float sums (FP64-class on the FP32 pipe)
  return gmres_solve(b->n, apply, (const double2*)d_b, (double2*)d_x, opts, info, st, opts->mode,
                     opts->mode == 32 ? 48 : 64, "vsie_bem_solve");
}

extern "C" vsie_status vsie_bem_far_field(vsie_bem* b, const void* d_x, const double* h_dirs, int32_t ndir,
                                          void* d_out, void* stream) {
  clear_error();
  TraceRange trace("vsie_bem_far_field");
  if (!b || !d_x || !h_dirs || !d_out || ndir < 1) {
    set_error("vsie_bem_far_field: null argument or ndir < 1");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  double* d_dirs = nullptr;
  VSIE_CUDA(cudaMallocAsync(&d_dirs, sizeof(double) * 3 * ndir, st));
  cudaError_t e = cudaMemcpyAsync(d_dirs, h_dirs, sizeof(double) * 3 * ndir, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    bem_far_field_kernel<<<(unsigned)ndir, 256, 0, st>>>((const double2*)d_x, b->tgt64, b->qw, b->d_far, b->tri,
                                                         b->uidx, b->vidx, b->nt_s[0], d_dirs, b->k0, b->rho0,
                                                         (double2*)d_out);
    e = cudaGetLastError();
  }
  cudaFreeAsync(d_dirs, st);
  if (e != cudaSuccess) return cuda_fail(e, "vsie_bem_far_field", __FILE__, __LINE__);
  // the host directions must stay valid until the copy ran
  VSIE_CUDA(cudaStreamSynchronize(st));
  return VSIE_OK;
}
