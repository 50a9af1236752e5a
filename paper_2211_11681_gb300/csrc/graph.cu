// CUDA-graph capture of a masked product: the counter reset and the persistent product
// kernel of s_mul_masked recorded once and replayed with one graph launch.
#include <new>

#include "common.cuh"

struct s_graph_t {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  s_plan plan = nullptr;  // for the time-out record of the captured product
};

using namespace sf;

extern "C" s_status s_graph_capture_mul(s_plan plan, const void* A, const void* B, void* C, s_graph* out) {
  if (!out) return set_error(S_ERR_ARG, "s_graph_capture_mul: out is NULL");
  *out = nullptr;
  if (!plan || !A || !B || !C) return set_error(S_ERR_ARG, "s_graph_capture_mul: NULL argument");
  cudaStream_t cs;
  SF_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  s_graph_t* g = new (std::nothrow) s_graph_t();
  if (!g) {
    cudaStreamDestroy(cs);
    return set_error(S_ERR_NOMEM, "host allocation");
  }
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  s_status st = S_OK;
  if (e == cudaSuccess) {
    st = s_mul_masked(plan, A, B, C, cs);
    e = cudaStreamEndCapture(cs, &g->graph);
  }
  if (e == cudaSuccess && !st) e = cudaGraphInstantiate(&g->exec, g->graph, 0);
  cudaStreamDestroy(cs);
  if (st || e != cudaSuccess) {
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
    return st ? st : cuda_error(e, "s_graph_capture_mul");
  }
  g->plan = plan;
  *out = g;
  return S_OK;
}

extern "C" s_status s_graph_launch(s_graph g, void* stream) {
  if (!g) return set_error(S_ERR_ARG, "s_graph_launch: NULL graph");
  const s_status st = take_timeout(g->plan->fwd);
  if (st) return st;
  SF_CUDA(cudaGraphLaunch(g->exec, (cudaStream_t)stream));
  return S_OK;
}

extern "C" s_status s_graph_destroy(s_graph g) {
  if (!g) return S_OK;
  cudaGraphExecDestroy(g->exec);
  cudaGraphDestroy(g->graph);
  delete g;
  return S_OK;
}
