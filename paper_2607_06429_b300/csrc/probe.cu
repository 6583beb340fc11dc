// Issue-rate probe of the SM pipes the far-field sums are bound by: MUFU (rsqrt, sin), the
// FP32 pipe (scalar FFMA and paired FFMA2) and the FP64 pipe (DFMA).  The ALU rooflines of
// the far-sum kernels are stated from nominal unit counts and the sampled SM clock; this
// probe measures what one B300 sustains per clock and per SM, as evidence for those
// denominators.  (The paper has no counterpart; it reports no timings.)
//
// Each thread runs kChains independent dependency chains of one instruction for a fixed
// number of iterations; every block records its SM, and clock64() at its start and end.
// Per SM, rate = operations issued by its blocks / (last end - first start) in SM clocks.
// One wave: the grid is the SM count times the resident blocks per SM.

#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <vector>

#include "vsie_internal.h"

using namespace vsie;

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;

enum ProbeOp { kRsqrt = 0, kSin = 1, kFfma = 2, kFfma2 = 3, kDfma = 4, kNumOps = 5 };

__device__ __forceinline__ unsigned smid() {
  unsigned s;
  asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
  return s;
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) pipe_probe_kernel(int iters, float* __restrict__ sink,
                                                                   long long* __restrict__ stamps) {
  const int tid = threadIdx.x;
  const float seed = 1.0f + 1e-3f * (float)(tid & 31);
  __syncthreads();
  const long long t0 = clock64();
  float acc = 0.0f;
  if constexpr (OP == kRsqrt || OP == kSin || OP == kFfma) {
    float v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = seed + 0.01f * c;
    const float a = 0.9999f, b = 1e-4f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) {
        if constexpr (OP == kRsqrt) asm volatile("rsqrt.approx.ftz.f32 %0, %0;" : "+f"(v[c]));
        if constexpr (OP == kSin) asm volatile("sin.approx.ftz.f32 %0, %0;" : "+f"(v[c]));
        if constexpr (OP == kFfma) asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(v[c]) : "f"(a), "f"(b));
      }
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += v[c];
  } else if constexpr (OP == kFfma2) {
    float2 v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = make_float2(seed + 0.01f * c, seed - 0.01f * c);
    const float2 a = make_float2(0.9999f, 0.9998f), b = make_float2(1e-4f, 2e-4f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) v[c] = __ffma2_rn(v[c], a, b);
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += v[c].x + v[c].y;
  } else {
    double v[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) v[c] = (double)seed + 0.01 * c;
    const double a = 0.9999, b = 1e-4;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < kChains; ++c) asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(v[c]) : "d"(a), "d"(b));
    }
#pragma unroll
    for (int c = 0; c < kChains; ++c) acc += (float)v[c];
  }
  __syncthreads();
  const long long t1 = clock64();
  sink[(size_t)blockIdx.x * kProbeThreads + tid] = acc;
  if (tid == 0) {
    stamps[3 * (size_t)blockIdx.x] = t0;
    stamps[3 * (size_t)blockIdx.x + 1] = t1;
    stamps[3 * (size_t)blockIdx.x + 2] = (long long)smid();
  }
}

template <int OP>
vsie_status run_probe(int num_sms, int iters, cudaStream_t st, double* per_clk, double* mhz) {
  int bps = 0;
  VSIE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, pipe_probe_kernel<OP>, kProbeThreads, 0));
  bps = std::max(1, std::min(bps, 8));
  const int grid = num_sms * bps;
  float* sink = nullptr;
  long long* stamps = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  vsie_status s = VSIE_OK;
  std::vector<long long> hs(3 * (size_t)grid);
  float ms = 0.0f;
  cudaError_t e = cudaMalloc(&sink, sizeof(float) * (size_t)grid * kProbeThreads);
  if (e == cudaSuccess) e = cudaMalloc(&stamps, sizeof(long long) * 3 * (size_t)grid);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e == cudaSuccess) {
    pipe_probe_kernel<OP><<<grid, kProbeThreads, 0, st>>>(iters / 8, sink, stamps);  // warm-up
    e = cudaEventRecord(e0, st);
  }
  if (e == cudaSuccess) {
    pipe_probe_kernel<OP><<<grid, kProbeThreads, 0, st>>>(iters, sink, stamps);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaEventRecord(e1, st);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  if (e == cudaSuccess)
    e = cudaMemcpy(hs.data(), stamps, sizeof(long long) * hs.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) s = cuda_fail(e, "pipe probe", __FILE__, __LINE__);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  cudaFree(stamps);
  if (s != VSIE_OK) return s;
  // per SM: blocks' operations over the span of their clock stamps
  std::map<long long, std::pair<long long, long long>> span;
  std::map<long long, int> blocks;
  for (int b = 0; b < grid; ++b) {
    const long long t0 = hs[3 * b], t1 = hs[3 * b + 1], sm = hs[3 * b + 2];
    auto it = span.find(sm);
    if (it == span.end()) {
      span[sm] = {t0, t1};
    } else {
      it->second.first = std::min(it->second.first, t0);
      it->second.second = std::max(it->second.second, t1);
    }
    ++blocks[sm];
  }
  const double ops_per_block = (double)kProbeThreads * iters * kChains * (OP == kFfma2 ? 2.0 : 1.0);
  std::vector<double> rates, cycles;
  for (auto& kv : span) {
    const double cyc = (double)(kv.second.second - kv.second.first);
    if (cyc <= 0) continue;
    rates.push_back(ops_per_block * blocks[kv.first] / cyc);
    cycles.push_back(cyc);
  }
  if (rates.empty()) {
    set_error("pipe probe: no clock stamps");
    return VSIE_ERR_CUDA;
  }
  std::sort(rates.begin(), rates.end());
  std::sort(cycles.begin(), cycles.end());
  *per_clk = rates[rates.size() / 2];
  // the longest SM span against the event time of the launch: the SM clock under the probe
  if (mhz) *mhz = ms > 0.0f ? cycles.back() / (ms * 1e-3) / 1e6 : 0.0;
  return VSIE_OK;
}

}  // namespace

extern "C" vsie_status vsie_pipe_probe(double* per_clk_per_sm, double* sm_mhz, void* stream) {
  clear_error();
  TraceRange trace("vsie_pipe_probe");
  if (!per_clk_per_sm) {
    set_error("vsie_pipe_probe: null output");
    return VSIE_ERR_ARG;
  }
  int dev = 0, num_sms = 0;
  VSIE_CUDA(cudaGetDevice(&dev));
  VSIE_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  cudaStream_t st = (cudaStream_t)stream;
  double mhz[kNumOps] = {0, 0, 0, 0, 0};
  // iteration counts sized to tens of milliseconds per launch at the nominal rates
  VSIE_TRY(run_probe<kRsqrt>(num_sms, 32768, st, &per_clk_per_sm[kRsqrt], &mhz[kRsqrt]));
  VSIE_TRY(run_probe<kSin>(num_sms, 32768, st, &per_clk_per_sm[kSin], &mhz[kSin]));
  VSIE_TRY(run_probe<kFfma>(num_sms, 131072, st, &per_clk_per_sm[kFfma], &mhz[kFfma]));
  VSIE_TRY(run_probe<kFfma2>(num_sms, 131072, st, &per_clk_per_sm[kFfma2], &mhz[kFfma2]));
  VSIE_TRY(run_probe<kDfma>(num_sms, 4096, st, &per_clk_per_sm[kDfma], &mhz[kDfma]));
  if (sm_mhz) {
    double m = 0.0;
    for (int i = 0; i < kNumOps; ++i) m = std::max(m, mhz[i]);
    *sm_mhz = m;
  }
  return VSIE_OK;
}
