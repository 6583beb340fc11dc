// CUDA-graph plans of the multi-operator batched apply: the whole sequence of launches of
// vsie_apply_batched_multi (charge images, persistent tensor-core sums, fix-ups, F-class
// sums, block corrections) for fixed operators and buffers is recorded once by stream
// capture and replayed with a single cudaGraphLaunch.

#include <cuda_runtime.h>

#include <vector>

#include "vsie_internal.h"

struct vsie_graph {
  std::vector<vsie_handle*> hs;
  std::vector<const double2*> x;
  std::vector<double2*> y;
  int nrhs = 0;
  cudaStream_t capture = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

using namespace vsie;

extern "C" void vsie_graph_destroy(vsie_graph* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  if (g->capture) cudaStreamDestroy(g->capture);
  delete g;
}

extern "C" vsie_status vsie_graph_create_batched(vsie_handle* const* hs, int32_t nop, const void* const* d_x,
                                                 void* const* d_y, int32_t nrhs, vsie_graph** out) {
  clear_error();
  TraceRange trace("vsie_graph_create_batched");
  if (!out) {
    set_error("vsie_graph_create_batched: null output");
    return VSIE_ERR_ARG;
  }
  *out = nullptr;
  VSIE_TRY(check_multi_args(hs, nop, d_x, d_y, nrhs, "vsie_graph_create_batched"));
  vsie_graph* g = new vsie_graph;
  g->nrhs = nrhs;
  for (int p = 0; p < nop; ++p) {
    g->hs.push_back(hs[p]);
    g->x.push_back(static_cast<const double2*>(d_x[p]));
    g->y.push_back(static_cast<double2*>(d_y[p]));
  }
  auto fail = [&](vsie_status s) {
    vsie_graph_destroy(g);
    return s;
  };
  cudaError_t e = cudaStreamCreateWithFlags(&g->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamCreateWithFlags", __FILE__, __LINE__));
  // one uncaptured run allocates every scratch buffer and sets the kernel attributes
  vsie_status s = apply_batched_multi_launch(g->hs.data(), nop, g->x.data(), g->y.data(), nrhs, g->capture);
  for (int p = 0; p < nop && s == VSIE_OK; ++p) s = batch_status(g->hs[p], g->capture);
  if (s != VSIE_OK) return fail(s);
  e = cudaStreamBeginCapture(g->capture, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamBeginCapture", __FILE__, __LINE__));
  s = apply_batched_multi_launch(g->hs.data(), nop, g->x.data(), g->y.data(), nrhs, g->capture);
  e = cudaStreamEndCapture(g->capture, &g->graph);
  if (s != VSIE_OK) return fail(s);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__));
  e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  if (e != cudaSuccess) return fail(cuda_fail(e, "cudaGraphInstantiate", __FILE__, __LINE__));
  *out = g;
  return VSIE_OK;
}

extern "C" vsie_status vsie_graph_launch(vsie_graph* g, void* stream) {
  clear_error();
  TraceRange trace("vsie_graph_launch");
  if (!g || !g->exec) {
    set_error("vsie_graph_launch: null plan");
    return VSIE_ERR_ARG;
  }
  cudaStream_t st = (cudaStream_t)stream;
  VSIE_CUDA(cudaGraphLaunch(g->exec, st));
  for (vsie_handle* h : g->hs) VSIE_TRY(batch_status(h, st));
  return VSIE_OK;
}

extern "C" vsie_status vsie_graph_nodes(const vsie_graph* g, int64_t* nodes) {
  clear_error();
  if (!g || !g->graph || !nodes) {
    set_error("vsie_graph_nodes: null argument");
    return VSIE_ERR_ARG;
  }
  size_t cnt = 0;
  VSIE_CUDA(cudaGraphGetNodes(g->graph, nullptr, &cnt));
  *nodes = (int64_t)cnt;
  return VSIE_OK;
}
