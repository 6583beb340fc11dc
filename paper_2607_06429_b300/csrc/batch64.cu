// Multi-right-hand-side far-field sums in FP64 on the CUDA cores: the residual operator of
// the batched iterative refinement (the outer residual b - A x must be accurate to FP64
// level, which an FP32 tensor-core accumulator cannot give).
//
// Same sums as the FP64 single-column path (Eq. vsie; G and K source classes, positions
// scaled by kappa = k0/(2 pi), phase in revolutions), but each kernel coefficient C(x_i, y_j)
// is evaluated once (in double-float arithmetic on the FP32 pipe, about 2^-47 per
// operation, the same evaluator as the precision-48 sums) and applied to a block of up
// to 64 right-hand sides:
//     Y[i, r] = sum_j C(x_i, y_j) q_j^(r).
// One block owns 32 targets x 64 right-hand sides; per tile of 32 sources its 256 threads
// evaluate the 1024 coefficients into shared memory (4 per thread, own target), then each
// thread accumulates its target (its lane) against 8 right-hand sides (its warp's), reading
// the charges as warp-wide broadcasts.  The contraction runs in double-float arithmetic on the FP32 pipe
// (coefficients and charges as hi + lo float pairs, TwoProduct / TwoSum, about 48 bits):
// B300's FP64 pipe runs at 1/64 of the FP32 rate, so 4 DFMA per pair and right-hand side
// would cost five times the double-float multiply-add.  Source ranges are split over
// blockIdx.y when the target blocks alone do not fill the GPU; the partial sums are added
// in split order (deterministic).

#include <cuda_runtime.h>

#include <algorithm>

#include "dfloat.h"
#include "vsie_internal.h"

namespace vsie {

namespace {

constexpr int B64_T = 32;        // targets per block (one per lane)
constexpr int B64_S = 32;        // sources per tile
constexpr int B64_R = 64;        // right-hand sides per launch
constexpr int B64_THREADS = 256;
constexpr int B64_RPT = B64_R / (B64_THREADS / B64_T);  // right-hand sides per thread (8)
// shared memory: source positions and normals (double-float: hi and lo records), then the
// coefficient tile [S][T], then the charge tile [S][R]
constexpr size_t B64_SMEM_P = sizeof(float4) * 4 * B64_S;
constexpr size_t B64_SMEM_C = sizeof(float4) * B64_S * B64_T;
constexpr size_t B64_SMEM_Q = sizeof(float4) * B64_S * B64_R;
constexpr size_t B64_SMEM = B64_SMEM_P + B64_SMEM_C + B64_SMEM_Q;
static_assert(B64_SMEM <= 227 * 1024 && B64_SMEM_P % 16 == 0, "shared memory layout");

struct B64Args {
  const double4_32a* tgt;   // collocation points (FP64)
  const double4_32a* pos;   // source (x, y, z, s)
  const double4_32a* nrm;   // source (nx, ny, nz, sigma) (K class)
  const float4* q;          // charges [source][B64_R], double-float
  double kap;
  int64_t nt, ns, ntiles;
  int nsplit;
  double2* out;             // n x nrhs_out column-major
  int64_t ld_out;
  int nrhs_out;
  int mode;                 // 0 store, 1 add
  double2* part;            // [nsplit][B64_R][nt] when nsplit > 1
};

template <bool IsK>
__global__ void __launch_bounds__(B64_THREADS, 2) b64_kernel(B64Args a) {
  extern __shared__ __align__(16) unsigned char sm[];
  float4* sp = reinterpret_cast<float4*>(sm);  // [4][S]: kappa y hi, lo; normal hi, lo (K)
  float4* sC = reinterpret_cast<float4*>(sm + B64_SMEM_P);               // [S][T] coefficients (double-float)
  float4* sQ = reinterpret_cast<float4*>(sm + B64_SMEM_P + B64_SMEM_C);  // [S][R] charges (double-float)
  const int tid = threadIdx.x;
  const int t = tid & (B64_T - 1), rg = tid / B64_T;
  const int64_t i = (int64_t)blockIdx.x * B64_T + t;
  const bool tok = i < a.nt;
  DTgt tg{dfs{0.0f, 0.0f}, dfs{0.0f, 0.0f}, dfs{0.0f, 0.0f}};
  if (tok) {
    const double4_32a p = a.tgt[i];
    tg = DTgt{dfs_make(p.x * a.kap), dfs_make(p.y * a.kap), dfs_make(p.z * a.kap)};
  }
  float2 accS[B64_RPT], accC[B64_RPT];  // double-float sums: hi parts, collected rounding errors
#pragma unroll
  for (int r = 0; r < B64_RPT; ++r) accS[r] = accC[r] = make_float2(0.0f, 0.0f);
  const int sp_i = blockIdx.y;
  const int64_t tile0 = (a.ntiles * sp_i) / a.nsplit, tile1 = (a.ntiles * (sp_i + 1)) / a.nsplit;
  for (int64_t tile = tile0; tile < tile1; ++tile) {
    __syncthreads();
    const int64_t j0 = tile * B64_S;
    if (tid < B64_S) {
      const int64_t j = j0 + tid;
      float4 ph = make_float4(0, 0, 0, 0), pl = ph, nh = ph, nl = ph;
      if (j < a.ns) {
        const double4_32a q = a.pos[j];
        const dfs x = dfs_make(q.x * a.kap), y = dfs_make(q.y * a.kap), z = dfs_make(q.z * a.kap);
        ph = make_float4(x.h, y.h, z.h, 0.0f);
        pl = make_float4(x.l, y.l, z.l, 0.0f);
        if (IsK) {
          const double4_32a nv = a.nrm[j];
          const dfs nx = dfs_make(nv.x), ny = dfs_make(nv.y), nz = dfs_make(nv.z);
          nh = make_float4(nx.h, ny.h, nz.h, 0.0f);
          nl = make_float4(nx.l, ny.l, nz.l, 0.0f);
        }
      }
      sp[tid] = ph;
      sp[B64_S + tid] = pl;
      sp[2 * B64_S + tid] = nh;
      sp[3 * B64_S + tid] = nl;
    }
    for (int e = tid; e < B64_S * B64_R; e += B64_THREADS) {
      const int64_t j = j0 + e / B64_R;
      sQ[e] = (j < a.ns) ? a.q[j0 * B64_R + e] : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    __syncthreads();
#pragma unroll 2
    for (int q = 0; q < B64_S / (B64_THREADS / B64_T); ++q) {
      const int jj = rg + (B64_THREADS / B64_T) * q;
      if (IsK) {
        const float4 nh = sp[2 * B64_S + jj], nl = sp[3 * B64_S + jj];
        sC[jj * B64_T + t] =
            df_coef_k(tg, sp[jj], sp[B64_S + jj], dfs{nh.x, nl.x}, dfs{nh.y, nl.y}, dfs{nh.z, nl.z});
      } else {
        sC[jj * B64_T + t] = df_coef_g(tg, sp[jj], sp[B64_S + jj]);
      }
    }
    __syncthreads();
#pragma unroll 1
    for (int jj = 0; jj < B64_S; ++jj) {
      const float4 c = sC[jj * B64_T + t];
      const float4* qr = sQ + jj * B64_R + rg * B64_RPT;
#pragma unroll
      for (int r = 0; r < B64_RPT; ++r) df_cmac(accS[r], accC[r], c, qr[r]);
    }
#pragma unroll
    for (int r = 0; r < B64_RPT; ++r) df_renorm2(accS[r], accC[r]);
  }
  if (!tok) return;
#pragma unroll
  for (int r = 0; r < B64_RPT; ++r) {
    const int rr = rg * B64_RPT + r;
    if (rr >= a.nrhs_out) continue;
    const double2 v = df_value(accS[r], accC[r]);
    if (a.nsplit == 1) {
      double2* o = a.out + (int64_t)rr * a.ld_out + i;
      *o = a.mode ? make_double2(o->x + v.x, o->y + v.y) : v;
    } else {
      a.part[((int64_t)sp_i * B64_R + rr) * a.nt + i] = v;
    }
  }
}

// out (+)= sum over splits of part, in split order
__global__ void b64_reduce_kernel(B64Args a) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)a.nrhs_out * a.nt) return;
  const int64_t r = e / a.nt, i = e % a.nt;
  double sr = 0.0, si = 0.0;
  for (int s = 0; s < a.nsplit; ++s) {
    const double2 v = a.part[((int64_t)s * B64_R + r) * a.nt + i];
    sr += v.x;
    si += v.y;
  }
  double2* o = a.out + r * a.ld_out + i;
  *o = a.mode ? make_double2(o->x + sr, o->y + si) : make_double2(sr, si);
}

// charges of one block of right-hand sides: q[j][r] = sc_j p_r(e(j)), zero past nrhs
// G: sc = -kappa s / (4 pi);  K: sc = kappa^2 sigma / (4 pi)
__global__ void b64_charges_kernel(const double4_32a* __restrict__ pos, const double4_32a* __restrict__ aux,
                                   const int32_t* __restrict__ own, int64_t ns, const double2* __restrict__ x,
                                   int64_t ld_x, int nrhs, int r_base, double kap, int is_k,
                                   float4* __restrict__ q) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ns * B64_R) return;
  const int r = (int)(e % B64_R);
  const int64_t j = e / B64_R;
  const int rr = r_base + r;
  double2 v = make_double2(0.0, 0.0);
  if (rr < nrhs) {
    const double sc = is_k ? kap * kap * aux[j].w / kFourPi : -kap * pos[j].w / kFourPi;
    const double2 p = x[(int64_t)rr * ld_x + own[j]];
    v = make_double2(sc * p.x, sc * p.y);
  }
  q[e] = df_pack(v);
}

vsie_status b64_class(vsie_handle* h, const Sources& S, bool is_k, const double2* x, double2* y, int nrhs,
                      int r_base, int mode, cudaStream_t st) {
  const int64_t n = h->n;
  const size_t qn = (size_t)S.n * B64_R;
  if (h->batch.q64_elems < qn) {
    float4* p = nullptr;
    VSIE_TRY(dalloc_t(h, &p, qn));
    h->batch.q64 = p;
    h->batch.q64_elems = qn;
  }
  const double kap = h->k0 / (2.0 * kPi);
  b64_charges_kernel<<<(unsigned)((qn + 255) / 256), 256, 0, st>>>(S.pos_s, S.aux, S.owner, S.n, x, n, nrhs,
                                                                   r_base, kap, is_k ? 1 : 0, h->batch.q64);
  VSIE_CUDA(cudaGetLastError());
  B64Args a;
  a.tgt = h->tgt64;
  a.pos = S.pos_s;
  a.nrm = S.aux;
  a.q = h->batch.q64;
  a.kap = kap;
  a.nt = n;
  a.ns = S.n;
  a.ntiles = (S.n + B64_S - 1) / B64_S;
  const int64_t ntb = (n + B64_T - 1) / B64_T;
  const int64_t want = 4LL * 2 * std::max(h->num_sms, 1);  // four waves of two resident blocks per SM
  a.nsplit = (int)std::max<int64_t>(1, std::min<int64_t>(a.ntiles, (want + ntb - 1) / ntb));
  a.out = y + (int64_t)r_base * n;
  a.ld_out = n;
  a.nrhs_out = std::min(B64_R, nrhs - r_base);
  a.mode = mode;
  a.part = nullptr;
  if (a.nsplit > 1) {
    const size_t pn = (size_t)a.nsplit * B64_R * n;
    if (h->batch.part64_elems < pn) {
      double2* p = nullptr;
      VSIE_TRY(dalloc_t(h, &p, pn));
      h->batch.part64 = p;
      h->batch.part64_elems = pn;
    }
    a.part = h->batch.part64;
  }
  const dim3 grid((unsigned)ntb, (unsigned)a.nsplit);
  if (is_k) {
    VSIE_CUDA(cudaFuncSetAttribute(b64_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B64_SMEM));
    b64_kernel<true><<<grid, B64_THREADS, B64_SMEM, st>>>(a);
  } else {
    VSIE_CUDA(cudaFuncSetAttribute(b64_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)B64_SMEM));
    b64_kernel<false><<<grid, B64_THREADS, B64_SMEM, st>>>(a);
  }
  VSIE_CUDA(cudaGetLastError());
  if (a.nsplit > 1) {
    const int64_t e = (int64_t)a.nrhs_out * n;
    b64_reduce_kernel<<<(unsigned)((e + 255) / 256), 256, 0, st>>>(a);
    VSIE_CUDA(cudaGetLastError());
  }
  return VSIE_OK;
}

}  // namespace

// y[:, r] = (FP64 far-field sums over the G and K classes) for all columns r, 64 at a time
vsie_status far_batched64_gk(vsie_handle* h, const double2* x, double2* y, int nrhs, cudaStream_t st) {
  for (int r0 = 0; r0 < nrhs; r0 += B64_R) {
    int mode = 0;
    if (h->G.n) {
      VSIE_TRY(b64_class(h, h->G, false, x, y, nrhs, r0, mode, st));
      mode = 1;
    }
    if (h->K.n) {
      VSIE_TRY(b64_class(h, h->K, true, x, y, nrhs, r0, mode, st));
      mode = 1;
    }
    if (!mode) {
      const int cols = std::min(B64_R, nrhs - r0);
      VSIE_CUDA(cudaMemsetAsync(y + (int64_t)r0 * h->n, 0, sizeof(double2) * h->n * cols, st));
    }
  }
  return VSIE_OK;
}

}  // namespace vsie
