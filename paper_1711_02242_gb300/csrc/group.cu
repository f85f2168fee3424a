// Groups of independent runs replayed as one CUDA graph per block of steps.
#include <vector>

#include "kernels.cuh"
#include "state.cuh"

namespace afq {
int step_block(afqmc_state* s);  // api.cu: one graph block of steps, launched kernel by kernel
}

struct afqmc_group {
  std::vector<afqmc_state*> states;
  cudaStream_t root = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;  // fork + one join event per state
  int blk = 0;
  int64_t kernels = 0;
};

using namespace afq;

extern "C" int afqmc_group_create(afqmc_state* const* states, int32_t n, void* stream,
                                  afqmc_group** out) {
  if (!out || !states || n < 1) {
    set_error("group: bad arguments");
    return AFQMC_EINVAL;
  }
  *out = nullptr;
  int blk = -1;
  for (int i = 0; i < n; ++i) {
    afqmc_state* s = states[i];
    if (!s || !s->valid || !s->p.use_graph || s->graph_block <= 0) {
      set_error("group: state %d is invalid or has use_graph = 0", i);
      return AFQMC_EINVAL;
    }
    if (blk >= 0 && s->graph_block != blk) {
      set_error("group: graph blocks differ (%d vs %d)", s->graph_block, blk);
      return AFQMC_EINVAL;
    }
    blk = s->graph_block;
    for (int j = 0; j < i; ++j)
      if (states[j] == s || states[j]->st == s->st) {
        set_error("group: states %d and %d share a state or a stream", j, i);
        return AFQMC_EINVAL;
      }
  }
  afqmc_group* g = new afqmc_group();
  g->states.assign(states, states + n);
  g->root = static_cast<cudaStream_t>(stream);
  g->blk = blk;
  g->ev.resize(n + 1, nullptr);
  for (auto& e : g->ev) {
    if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
      for (auto& x : g->ev)
        if (x) cudaEventDestroy(x);
      delete g;
      set_error("group: cudaEventCreate failed");
      return AFQMC_ECUDA;
    }
  }
  *out = g;
  return AFQMC_OK;
}

static int capture_group(afqmc_group* g) {
  const int n = (int)g->states.size();
  std::vector<int64_t> h0(n);
  for (int i = 0; i < n; ++i) h0[i] = g->states[i]->h_step;
  const int64_t l0 = g_launches;
  AFQ_CUDA(cudaStreamBeginCapture(g->root, cudaStreamCaptureModeThreadLocal));
  int r = AFQMC_OK;
  cudaError_t e = cudaEventRecord(g->ev[0], g->root);
  for (int i = 0; i < n && r == AFQMC_OK && e == cudaSuccess; ++i) {
    afqmc_state* s = g->states[i];
    e = cudaStreamWaitEvent(s->st, g->ev[0], 0);
    if (e != cudaSuccess) break;
    s->t_fresh = false;
    r = step_block(s);
    if (r != AFQMC_OK) break;
    e = cudaEventRecord(g->ev[i + 1], s->st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(g->root, g->ev[i + 1], 0);
  }
  cudaGraph_t graph = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(g->root, &graph);
  for (int i = 0; i < n; ++i) g->states[i]->h_step = h0[i];  // nothing ran yet
  if (r != AFQMC_OK || e != cudaSuccess || e2 != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    if (r == AFQMC_OK) {
      set_error("group capture failed: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
      r = AFQMC_ECUDA;
    }
    return r;
  }
  e = cudaGraphInstantiate(&g->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    g->exec = nullptr;
    set_error("group graph instantiation failed: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  g->kernels = g_launches - l0;
  g_launches = l0;
  return AFQMC_OK;
}

extern "C" int afqmc_group_propagate(afqmc_group* g, int32_t nsteps) {
  if (!g || nsteps < 0 || nsteps % g->blk) {
    set_error("group: nsteps must be a non-negative multiple of the block (%d)", g ? g->blk : 0);
    return AFQMC_EINVAL;
  }
  for (afqmc_state* s : g->states)
    if (!s->valid || s->h_step % g->blk || s->prof.on || s->bp_on) {
      set_error("group: a state is invalid, profiling, in a back-propagation window, or off a "
                "block boundary");
      return AFQMC_ESTATE;
    }
  for (int done = 0; done < nsteps; done += g->blk) {
    if (!g->exec) AFQ_TRY(capture_group(g));
    AFQ_CUDA(cudaGraphLaunch(g->exec, g->root));
    g_launches += g->kernels;
    for (afqmc_state* s : g->states) {
      s->h_step += g->blk;
      s->t_fresh = false;
    }
  }
  return AFQMC_OK;
}

extern "C" int afqmc_group_destroy(afqmc_group* g) {
  if (!g) return AFQMC_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  delete g;
  return AFQMC_OK;
}
