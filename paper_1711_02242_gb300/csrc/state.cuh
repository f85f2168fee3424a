// Host-side state of one AFQMC run (internal header).
#pragma once

#include <cmath>
#include <vector>

#include "kernels.cuh"

namespace afq {

enum { CTR_STEP = 0, CTR_RECORDS = 1, CTR_NONFINITE = 2, CTR_STATUS = 3 };

// Device buffers carved out of the caller's workspace.
struct Bufs {
  // constants of the run (all in the trial-adapted basis, see setup_device)
  double *LpT, *Lh, *hh, *c, *Bh, *VTt, *h1;
  // basis rotation: Qb[p][q] = Q_pq with Q[:, :N] the trial, QTb = Q^T
  double *Qb, *QTb;
  // walkers
  double *phiT, *thetaT, *ld, *ld_new, *wt, *S, *Sinv, *t, *x, *scal, *eloc, *part;
  double *cum, *wtot, *last, *records;
  int* parent;
  unsigned long long* counters;  // CTR_*
  // step scratch
  double *Y, *T0, *T1, *acc, *tmp_ld;
  // set-up scratch (aliases the step scratch); Ych: ych vectors of Q^T L_g
  double *Lfull, *L2, *cLp, *E0, *E1, *X, *red, *Ych;
  int ych = 0;
  int P, nchunk, gc;
  // mixed path: BF16 / TF32 operand copies and FP32 step buffers
  bool mixed = false;
  bool f32lu = false;  // S^-1, Theta and Gram-Schmidt in FP32 (the _F32LU precisions)
  bool theta32 = false;  // Theta = Phi S^-1 in FP32 (every mixed precision but _F64THETA)
  int lo_kind = 0, lo_bytes = 0, Gp = 0, Mp = 0;
  long Pp = 0;
  // LbT_lo: Cholesky vectors transposed over the upper 16 x 16 blocks (P <= Q)
  // of each Mp x Mp vector, rows blk * 256 + pp * 16 + qq, pitch Gp
  void *LbT_lo = nullptr, *Lh_lo = nullptr, *x_lo = nullptr, *th_lo = nullptr;
  int nblkV = 0;
  float* t32 = nullptr;
  // tensor-core propagation: exp(-dt v0'/2) as BF16/TF32 and TF32 [M][Mp],
  // V operand [W*M][2Mp], orbitals [W*2N][Mp], series sum [W*2N][Mp] FP32,
  // two Taylor-term operands [W*2N][2Mp]
  void *Bh_lo = nullptr, *V_lo = nullptr, *phi_lo = nullptr, *Tb0 = nullptr, *Tb1 = nullptr;
  float *Bh_tf = nullptr, *acc32 = nullptr;
  // the half steps' D_B = B_half - I as split pairs along K: [hi | lo] (the
  // first half step, BF16/TF32, segments of Kp1) and [hi | hi | lo | lo] (the
  // last one, TF32, segments of Mp)
  void* Bh_split = nullptr;
  float* Bh_split_tf = nullptr;
  int Kp1 = 0;
  int* status = nullptr;  // device status word (tensor-core waits)
  // back-propagation window (afqmc_params.bp_steps > 0): recorded fields
  // [bp_steps][W][2][G] float64 (mixed path: operand rows [W][2][Gp]), Psi_n and the back-propagated
  // orbitals [W][2][N][M], BP-PRes factors [W][2], cos dtheta [W], per-walker
  // weights [W][4], estimator slices [kBpSlices][2][M][M], R [4][M][M] and
  // the results [2][2][M][M] + 4 weight sums
  double *bp_hist = nullptr, *bp_psi = nullptr, *bp_phi = nullptr, *bp_f = nullptr;
  double *bp_cos = nullptr, *bp_part = nullptr, *bp_red = nullptr, *bp_R = nullptr;
  double* bp_out = nullptr;
  void* bp_phi_lo = nullptr;  // mixed path: operand copy of the back-propagated orbitals
  void* bp_tmp = nullptr;     // gather scratch: W rows of the largest recorded row
  // multi-determinant trial (afqmc_params.ndet >= 1), index ds = 2 d + spin:
  // orbitals V_ds^T [2nd][N][M], half-rotated vectors [2nd][G][N][M] and
  // one-body matrices [2nd][N][M], Theta_ds [2nd][W][2][N][M], log det S_ds
  // [W][2nd][2], weights w_d [W][nd][2], traces [2nd][2W][G], exchange
  // partials [2nd][W][nchunk][2], log A_d^* [nd][2]
  double *md_V = nullptr, *md_Lh = nullptr, *md_hh = nullptr, *md_theta = nullptr;
  double *md_ld = nullptr, *md_w = nullptr, *md_C = nullptr, *md_part = nullptr;
  double* md_logA = nullptr;
  // mixed path: Theta_ds rows [2nd][W][2N][Mp] and Lh_ds rows [2nd][G N][Mp]
  // as BF16/TF32, FP32 traces [2nd][2W][G]
  void *md_theta_lo = nullptr, *md_Lh_lo = nullptr;
  float* md_C32 = nullptr;
  // determinants taken relative to determinant 0 (holes and particles, see
  // multidet.cu): per (d, s) [k, particle offset, holes h_0..h_3, -, -],
  // particle rows (2 d + s) N + h of md_V / md_Lh / md_hh per spin
  // [2][kSmwMaxK nd], Xi_s = U_s^T Theta_0s [W][2][kSmwMaxK nd][N] complex,
  // energy partials [W][nchunk + 1][nd] complex
  int *smw_tab = nullptr, *smw_prow = nullptr;
  double *smw_xi = nullptr, *smw_part = nullptr;
};

constexpr int kSmwMaxK = 4;   // columns a determinant may differ from determinant 0 in, per spin
constexpr int kSmwMaxN = 32;  // orbitals per spin (one lane per column)
constexpr int kSmwGC = 8;     // Cholesky vectors per block of the low-rank kernels

constexpr int kBpSlices = 8;

size_t plan(const afqmc_params& p, Bufs* b, char* base);

}  // namespace afq

namespace afq {
// CUDA-event timing of the phases of a step (afqmc_profile_start/stop).
struct Profiler {
  bool on = false;
  int max_events = 0, used = 0;
  std::vector<cudaEvent_t> ev;  // pairs (begin, end)
  std::vector<int> phase;       // phase of each pair
  std::vector<int64_t> kern;    // kernels launched inside each pair
  int open_phase = -1;
  int64_t open_launch = 0;
};
}  // namespace afq

struct afqmc_state {
  afqmc_params p;
  cudaStream_t st = nullptr;
  char* ws = nullptr;
  size_t ws_bytes = 0;
  afq::Bufs b{};
  double E_T = 0, H0p = 0, e_shift = 0, wmax = 0, sdt = 0, elo = 0, ehi = 0;
  int64_t h_step = 0;
  bool t_fresh = false;
  bool valid = false;
  afq::Profiler prof;
  // CUDA graph of one block of steps (afqmc_params.use_graph)
  cudaGraphExec_t graph = nullptr;
  int graph_block = 0;
  int64_t graph_kernels = 0;
  // tile widths the autotuner chose for the V and force-bias contractions
  int bn_v = 0, bn_fb = 0;
  // back-propagation window: open, and steps recorded since it opened
  bool bp_on = false;
  int bp_m = 0;
  // spin blocks: p.N counts all orbital columns; the first nup are spin up.
  // Closed shell (one block standing for both spins): nup = p.N, sf = 2.
  bool spin2 = false;
  int nup = 0;
  double sf = 2.0;
  // population size of the last afqmc_comb_plan (sharded comb), 0 before one
  int64_t comb_nall = 0;
  // mixed path: Gram-Schmidt on a side stream, overlapping the work that does
  // not read the orbitals or log <Psi_T|Psi> (the energy evaluation, the next
  // step's force bias, fields and V); joined before the next reader
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_side = nullptr;
  bool side_pending = false;
  // multi-determinant trial evaluated relative to determinant 0 (float64),
  // with the particle count of each spin
  bool smw = false;
  int smw_np[2] = {0, 0};
};

namespace afq {
int bp_open(afqmc_state* s);
int bp_close(afqmc_state* s);
int bp_record_fields(afqmc_state* s);
int bp_step_factor(afqmc_state* s);
int bp_after_comb(afqmc_state* s);
int apply_b_f64(afqmc_state* s, const double* phi_in, double* phi_out, const double* mask);
int apply_b_mixed(afqmc_state* s, const double* phi_in, const void* phi_lo_in, double* phi_out,
                  void* phi_lo_out);
int md_overlap_update(afqmc_state* s, bool into_ld);
int md_force_bias(afqmc_state* s);
int md_local_energies(afqmc_state* s);
int md_setup(afqmc_state* s, const double* coef);
int smw_detect(afqmc_state* s, const double* up, const double* dn);
// Make the state's stream wait for a pending side-stream Gram-Schmidt.
int join_side(afqmc_state* s);
}  // namespace afq

namespace afq {
// Open / close a timed phase on the state's stream (no-ops unless profiling).
inline void prof_begin(afqmc_state* s, int phase) {
  Profiler& P = s->prof;
  if (!P.on || P.used >= P.max_events) return;
  cudaEventRecord(P.ev[2 * P.used], s->st);
  P.open_phase = phase;
  P.open_launch = g_launches;
}
inline void prof_end(afqmc_state* s) {
  Profiler& P = s->prof;
  if (!P.on || P.open_phase < 0) return;
  cudaEventRecord(P.ev[2 * P.used + 1], s->st);
  P.phase[P.used] = P.open_phase;
  P.kern[P.used] = g_launches - P.open_launch;
  P.used++;
  P.open_phase = -1;
}
}  // namespace afq
