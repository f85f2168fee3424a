// Groups of independent runs replayed as one CUDA graph per block of steps.
//
// Two ways to capture a block: every state's own kernel sequence on its own
// stream (branches of one graph), or - for mixed-precision states of one
// precision and the same periods - step by step in phases, where each of the
// step's four tensor-core contractions (force bias, V, the two half steps)
// of all states is ONE persistent launch over a work list of (state, tile)
// (TcGrouped, tile widths chosen by timing candidates on the group's own
// buffers), and the per-state kernels between them (fields, Taylor series,
// overlap / weights / periodic work) run on the states' streams.  In the
// default mode the group times its second and fourth blocks, one captured
// each way (results are bit-identical either way), and keeps the faster.
#include <vector>

#include "kernels.cuh"
#include "state.cuh"
#include "tc.cuh"

namespace afq {
// api.cu: one graph block of steps launched kernel by kernel, and the phases
// of a mixed-precision step
int step_block(afqmc_state* s);
int step_fields(afqmc_state* s);
int step_taylor(afqmc_state* s);
int step_after(afqmc_state* s);
void desc_force_bias(afqmc_state* s, TcJobDesc* d);
void desc_v(afqmc_state* s, TcJobDesc* d);
void desc_half1(afqmc_state* s, const double* phi_in, const void* phi_lo_in, TcJobDesc* d);
void desc_half2(afqmc_state* s, double* phi_out, void* phi_lo_out, TcJobDesc* d);
}  // namespace afq

struct afqmc_group {
  std::vector<afqmc_state*> states;
  cudaStream_t root = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaEvent_t> ev;  // fork + one join event per state
  int blk = 0;
  int64_t kernels = 0;
  // capture mode: 0 each state's own kernels, 1 grouped contractions, 2
  // choose by timing (trial: blocks replayed so far in the choice; ms of
  // the timed block of each mode)
  int mode = 2;
  int trial = 0;
  float trial_ms[2] = {0.f, 0.f};
  // grouped contractions: set up, and per phase (force bias, V, first half
  // step, last half step) the launch and its tile width
  bool grouped = false;
  afq::TcGrouped* gx[4] = {nullptr, nullptr, nullptr, nullptr};
  cudaEvent_t t0 = nullptr, t1 = nullptr;
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
  if (cudaEventCreate(&g->t0) != cudaSuccess || cudaEventCreate(&g->t1) != cudaSuccess) {
    for (auto& x : g->ev) cudaEventDestroy(x);
    if (g->t0) cudaEventDestroy(g->t0);
    delete g;
    set_error("group: cudaEventCreate failed");
    return AFQMC_ECUDA;
  }
  *out = g;
  return AFQMC_OK;
}

// Mixed states of one precision and the same periods, closed shell, single
// determinant, no back-propagation window.
static bool groupable(const afqmc_group* g) {
  const afqmc_state* s0 = g->states[0];
  for (const afqmc_state* s : g->states) {
    const afqmc_params& p = s->p;
    if (!s->b.mixed || s->b.lo_kind != s0->b.lo_kind || p.ndet || s->spin2 || s->bp_on ||
        p.qr_period != s0->p.qr_period || p.pc_period != s0->p.pc_period ||
        p.energy_period != s0->p.energy_period)
      return false;
  }
  return true;
}

static void free_grouped(afqmc_group* g) {
  for (auto& x : g->gx) {
    afq::tc_grouped_destroy(x);
    x = nullptr;
  }
  g->grouped = false;
}

// The four grouped launches; the force-bias and first-half-step tile widths
// timed on the states' buffers (scratch outputs only), the last half step
// taking the first's (same output shape; its epilogue writes the walkers).
static int setup_grouped(afqmc_group* g) {
  const int n = (int)g->states.size();
  for (afqmc_state* s : g->states) AFQ_CUDA(cudaStreamSynchronize(s->st));
  std::vector<TcJobDesc> d((size_t)n);
  int r = AFQMC_OK;
  for (int ph = 0; ph < 4 && r == AFQMC_OK; ++ph) {
    for (int i = 0; i < n; ++i) {
      afqmc_state* s = g->states[i];
      d[i] = TcJobDesc();
      if (ph == 0) afq::desc_force_bias(s, &d[i]);
      if (ph == 1) afq::desc_v(s, &d[i]);
      if (ph == 2) afq::desc_half1(s, s->b.phiT, s->b.phi_lo, &d[i]);
      if (ph == 3) afq::desc_half2(s, s->b.phiT, s->b.phi_lo, &d[i]);
    }
    if (ph == 3)
      r = afq::tc_grouped_create(d.data(), n, afq::tc_grouped_bn(g->gx[2]), &g->gx[3]);
    else
      r = afq::tc_grouped_tune(d.data(), n, g->root, &g->gx[ph]);
  }
  if (r == AFQMC_OK) r = cudaStreamSynchronize(g->root) == cudaSuccess ? AFQMC_OK : AFQMC_ECUDA;
  if (r != AFQMC_OK) {
    free_grouped(g);
    return r;
  }
  g->grouped = true;
  return AFQMC_OK;
}

// Run `fn` on every state's stream between a fork from and a join into root.
template <class F>
static int per_state(afqmc_group* g, F fn) {
  const int n = (int)g->states.size();
  AFQ_CUDA(cudaEventRecord(g->ev[0], g->root));
  for (int i = 0; i < n; ++i) {
    afqmc_state* s = g->states[i];
    AFQ_CUDA(cudaStreamWaitEvent(s->st, g->ev[0], 0));
    AFQ_TRY(fn(s));
    AFQ_CUDA(cudaEventRecord(g->ev[i + 1], s->st));
    AFQ_CUDA(cudaStreamWaitEvent(g->root, g->ev[i + 1], 0));
  }
  return AFQMC_OK;
}

// One block of steps in phases (captured on root).
static int grouped_block(afqmc_group* g) {
  for (int k = 0; k < g->blk; ++k) {
    const bool fb = !g->states[0]->t_fresh;
    for (afqmc_state* s : g->states)
      if (s->t_fresh != !fb) {
        afq::set_error("group: states disagree on the force bias of a step");
        return AFQMC_ESTATE;
      }
    if (fb) {
      AFQ_TRY(afq::tc_grouped_launch(g->gx[0], g->root));
      for (afqmc_state* s : g->states) s->t_fresh = true;
    }
    AFQ_TRY(per_state(g, [](afqmc_state* s) { return afq::step_fields(s); }));
    AFQ_TRY(afq::tc_grouped_launch(g->gx[1], g->root));
    AFQ_TRY(afq::tc_grouped_launch(g->gx[2], g->root));
    AFQ_TRY(per_state(g, [](afqmc_state* s) { return afq::step_taylor(s); }));
    AFQ_TRY(afq::tc_grouped_launch(g->gx[3], g->root));
    AFQ_TRY(per_state(g, [](afqmc_state* s) {
      AFQ_TRY(afq::step_after(s));
      return afq::join_side(s);
    }));
  }
  return AFQMC_OK;
}

static int capture_group(afqmc_group* g) {
  const int n = (int)g->states.size();
  std::vector<int64_t> h0(n);
  for (int i = 0; i < n; ++i) h0[i] = g->states[i]->h_step;
  const int64_t l0 = g_launches;
  const bool use_grouped = g->grouped;
  AFQ_CUDA(cudaStreamBeginCapture(g->root, cudaStreamCaptureModeThreadLocal));
  int r = AFQMC_OK;
  cudaError_t e = cudaSuccess;
  if (use_grouped) {
    for (afqmc_state* s : g->states) s->t_fresh = false;
    r = grouped_block(g);
  } else {
    e = cudaEventRecord(g->ev[0], g->root);
  }
  for (int i = 0; i < n && !use_grouped && r == AFQMC_OK && e == cudaSuccess; ++i) {
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
  const bool can_group = groupable(g);
  for (int done = 0; done < nsteps; done += g->blk) {
    // which capture this block replays: fixed, or the choice's trial
    // sequence (grouped, grouped timed, own kernels, own kernels timed)
    bool want = g->mode == 1;
    bool timed = false;
    if (g->mode == 2 && can_group && g->trial < 4) {
      want = g->trial < 2;
      timed = g->trial == 1 || g->trial == 3;
    } else if (g->mode == 2) {
      want = can_group && g->trial_ms[0] < g->trial_ms[1];
    }
    want = want && can_group;
    if (want != g->grouped || (want && !g->gx[0])) {
      if (g->exec) cudaGraphExecDestroy(g->exec);
      g->exec = nullptr;
      if (want) {
        AFQ_TRY(setup_grouped(g));
      } else {
        free_grouped(g);
      }
    }
    if (!g->exec) AFQ_TRY(capture_group(g));
    if (timed) AFQ_CUDA(cudaEventRecord(g->t0, g->root));
    AFQ_CUDA(cudaGraphLaunch(g->exec, g->root));
    if (timed) {
      AFQ_CUDA(cudaEventRecord(g->t1, g->root));
      AFQ_CUDA(cudaEventSynchronize(g->t1));
      AFQ_CUDA(cudaEventElapsedTime(&g->trial_ms[g->trial == 1 ? 0 : 1], g->t0, g->t1));
    }
    if (g->mode == 2 && can_group && g->trial < 4) ++g->trial;
    g_launches += g->kernels;
    for (afqmc_state* s : g->states) {
      s->h_step += g->blk;
      s->t_fresh = false;
    }
  }
  return AFQMC_OK;
}

extern "C" int afqmc_group_set_grouped(afqmc_group* g, int32_t mode) {
  if (!g || mode < 0 || mode > 2) {
    set_error("group: bad arguments");
    return AFQMC_EINVAL;
  }
  g->mode = mode;
  g->trial = 0;
  return AFQMC_OK;
}

extern "C" int afqmc_group_tiles(const afqmc_group* g, int32_t* bn) {
  if (!g || !bn) {
    set_error("group: bad arguments");
    return AFQMC_EINVAL;
  }
  for (int i = 0; i < 4; ++i) bn[i] = g->grouped ? afq::tc_grouped_bn(g->gx[i]) : 0;
  return g->grouped ? 1 : 0;
}

extern "C" int afqmc_group_destroy(afqmc_group* g) {
  if (!g) return AFQMC_OK;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  free_grouped(g);
  if (g->t0) cudaEventDestroy(g->t0);
  if (g->t1) cudaEventDestroy(g->t1);
  for (auto& e : g->ev)
    if (e) cudaEventDestroy(e);
  delete g;
  return AFQMC_OK;
}
