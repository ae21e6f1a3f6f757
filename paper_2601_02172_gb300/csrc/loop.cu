// Device-driven CG iteration loops: one CUDA graph holding, for each of one or several contexts,
// a conditional while node whose body is a round of that context's CG iterations (captured on
// the context's stream) followed by a one-thread condition kernel.  The loops of different
// contexts are independent branches of the graph, so each advances at its own pace; the host
// launches the graph once per inner solve instead of polling the activity flags every few
// iterations.
//
// Each loop is bounded three ways: the per-RHS iteration cap (the finalisation deactivates a
// right-hand side at maxit), a cap on the body's rounds, and a limit on the loop's device time
// (globaltimer nanoseconds) after which the condition kernel records a timeout and ends the loop.
// Nothing in it waits on another block, kernel or stream: each round is an ordinary sequence of
// kernel launches, so a loop always ends.
#include <cuda_runtime.h>

#include "xfft_kernels.h"

namespace xfft {

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void k_loop_start(LoopState* st) {
  if (threadIdx.x == 0) {
    st->t0 = global_ns();
    st->rounds = 0;
    st->timed_out = 0;
  }
}

// End of a round: continue while some right-hand side r < nr is active, fewer than max_rounds
// rounds have run and the loop has run for less than limit_ns (limit_ns < 0: no limit).
__global__ void k_loop_cond(cudaGraphConditionalHandle h, const int* __restrict__ act, int nr, LoopState* st,
                            unsigned max_rounds, long long limit_ns) {
  if (threadIdx.x != 0) return;
  int any = 0;
  for (int r = 0; r < nr; ++r) any |= act[r];
  const unsigned rounds = ++st->rounds;
  if (any && limit_ns >= 0 && (long long)(global_ns() - st->t0) >= limit_ns) {
    st->timed_out = 1;
    any = 0;
  }
  if (rounds >= max_rounds) any = 0;
  cudaGraphSetConditional(h, any ? 1u : 0u);
}

cudaError_t build_loop_graph(const std::vector<LoopSpec>& loops, cudaGraphExec_t* exec) {
  *exec = nullptr;
  cudaGraph_t G = nullptr;
  cudaError_t e = cudaGraphCreate(&G, 0);
  if (e != cudaSuccess) return e;
  for (const LoopSpec& L : loops) {
    cudaGraphNode_t start = nullptr, node = nullptr;
    cudaGraphConditionalHandle h = 0;
    {  // the start kernel: clock and counters of this loop
      cudaKernelNodeParams kp = {};
      LoopState* st = L.st;
      void* args[1] = {&st};
      kp.func = (void*)k_loop_start;
      kp.gridDim = dim3(1);
      kp.blockDim = dim3(32);
      kp.sharedMemBytes = 0;
      kp.kernelParams = args;
      e = cudaGraphAddKernelNode(&start, G, nullptr, 0, &kp);
    }
    cudaGraph_t bodyg = nullptr;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, G, 1u, cudaGraphCondAssignDefault);
    if (e == cudaSuccess) {
      cudaGraphNodeParams p = {};
      p.type = cudaGraphNodeTypeConditional;
      p.conditional.handle = h;
      p.conditional.type = cudaGraphCondTypeWhile;
      p.conditional.size = 1;
      e = cudaGraphAddNode(&node, G, &start, nullptr, 1, &p);
      if (e == cudaSuccess) bodyg = p.conditional.phGraph_out[0];
    }
    if (e == cudaSuccess)
      e = cudaStreamBeginCaptureToGraph(L.stream, bodyg, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
      cudaError_t eb = L.body(L.stream);
      if (eb == cudaSuccess) {
        k_loop_cond<<<1, 32, 0, L.stream>>>(h, L.act, L.nr, L.st, L.max_rounds, L.limit_ns);
        eb = cudaGetLastError();
      }
      cudaGraph_t captured = nullptr;
      e = cudaStreamEndCapture(L.stream, &captured);
      if (eb != cudaSuccess) e = eb;
    }
    if (e != cudaSuccess) break;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, G, 0);
  cudaGraphDestroy(G);
  if (e != cudaSuccess) {
    if (*exec) cudaGraphExecDestroy(*exec);
    *exec = nullptr;
  }
  return e;
}

}  // namespace xfft
