// C ABI of the AFQMC library: workspace plan, set-up, step sequencing.
#include <cmath>
#include <cstdarg>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.cuh"
#include "state.cuh"
#include "tc.cuh"

namespace afq {

static thread_local char g_err[512] = "no error";
int64_t g_launches = 0;

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
}

// ----------------------------------------------------------- workspace plan --
namespace {
struct Bump {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~size_t(255);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};
}  // namespace

size_t plan(const afqmc_params& p, Bufs* b, char* base) {
  Bufs tmp;
  if (!b) b = &tmp;
  // N: orbital columns per walker (N_up + N_dn with two spin blocks)
  const size_t M = p.M, N = p.N + (p.Ndn > 0 ? p.Ndn : 0), G = p.nchol, W = p.nwalkers;
  const size_t P = M * (M + 1) / 2;
  const bool mixed = p.precision != AFQMC_FP64;
  size_t nchunk = (G + exchange_chunk((int)N, p.nchol) - 1) / exchange_chunk((int)N, p.nchol);
  if (mixed) nchunk = G;  // the tensor-core exchange leaves one partial per vector
  const size_t lo = (p.precision == AFQMC_MIXED_BF16 || p.precision == AFQMC_MIXED_BF16_F32LU ||
                     p.precision == AFQMC_MIXED_BF16_F64THETA)
                        ? 2
                        : 4;
  // pitches: 16-byte rows for TMA; Mp a multiple of 16 so that 16-column
  // epilogue chunks of the flattened (p, q) index never straddle rows
  const size_t Gp = (G + 7) / 8 * 8, Mp = (M + 15) / 16 * 16, Pp = (P + 3) / 4 * 4;
  Bump a{base};
  // constants
  b->LpT = a.take<double>(P * G);
  b->Lh = a.take<double>(G * N * M);
  b->hh = a.take<double>(N * M);
  b->c = a.take<double>(G);
  b->Bh = a.take<double>(M * M);
  b->VTt = a.take<double>(N * M);
  b->h1 = a.take<double>(M * M);
  b->Qb = a.take<double>(M * M);
  b->QTb = a.take<double>(M * M);
  // walkers
  b->phiT = a.take<double>(W * 2 * N * M);
  b->thetaT = a.take<double>(W * 2 * N * M);
  b->ld = a.take<double>(2 * W);
  b->ld_new = a.take<double>(2 * W);
  b->wt = a.take<double>(2 * W);
  b->S = a.take<double>(W * 2 * N * N);
  b->Sinv = a.take<double>(W * 2 * N * N);
  b->t = a.take<double>(W * 2 * G);
  b->x = a.take<double>(W * 2 * G);
  b->scal = a.take<double>(8 * W);
  b->eloc = a.take<double>(2 * W);
  b->part = a.take<double>(W * nchunk * 2);
  b->cum = a.take<double>(W);
  b->parent = a.take<int>(W);
  b->wtot = a.take<double>(8);
  b->last = a.take<double>(8);
  b->records = a.take<double>(4 * (size_t)(p.max_records > 0 ? p.max_records : 1));
  b->counters = a.take<unsigned long long>(8);
  if (p.ndet > 0) {
    const size_t nd2 = 2 * (size_t)p.ndet;
    b->md_V = a.take<double>(nd2 * N * M);
    b->md_Lh = a.take<double>(nd2 * G * N * M);
    b->md_hh = a.take<double>(nd2 * N * M);
    b->md_theta = a.take<double>(nd2 * W * 2 * N * M);
    b->md_ld = a.take<double>(W * nd2 * 2);
    b->md_w = a.take<double>(W * (size_t)p.ndet * 2);
    b->md_C = a.take<double>(nd2 * 2 * W * G);
    b->md_part = a.take<double>(nd2 * W * nchunk * 2);
    b->md_logA = a.take<double>(nd2);
    const size_t ks = (size_t)kSmwMaxK * p.ndet;
    const size_t nchk = (G + kSmwGC - 1) / kSmwGC;
    b->smw_tab = a.take<int>(nd2 * 8);
    b->smw_prow = a.take<int>(2 * ks);
    b->smw_xi = a.take<double>(W * 2 * ks * N * 2);
    b->smw_part = a.take<double>(W * (nchk + 1) * p.ndet * 2);
    if (mixed) {
      b->md_theta_lo = a.take<char>(nd2 * W * 2 * N * Mp * lo);
      b->md_Lh_lo = a.take<char>(nd2 * G * N * Mp * lo);
      b->md_C32 = a.take<float>(nd2 * 2 * W * G);
    }
  }
  if (p.bp_steps > 0) {
    // recorded fields: float64 [W][2][G], or the operand rows [W][2][Gp]
    b->bp_hist = mixed ? reinterpret_cast<double*>(a.take<char>((size_t)p.bp_steps * W * 2 * Gp * lo))
                       : a.take<double>((size_t)p.bp_steps * W * 2 * G);
    if (mixed) b->bp_phi_lo = a.take<char>(W * 2 * N * Mp * lo);
    b->bp_psi = a.take<double>(W * 2 * N * M);
    b->bp_phi = a.take<double>(W * 2 * N * M);
    b->bp_f = a.take<double>(2 * W);
    b->bp_cos = a.take<double>(W);
    b->bp_part = a.take<double>(4 * W);
    b->bp_red = a.take<double>((size_t)kBpSlices * 2 * M * M);
    b->bp_R = a.take<double>(4 * M * M);
    b->bp_out = a.take<double>(4 * M * M + 4);
    size_t row = sizeof(double) * 2 * N * M;
    const size_t frow = mixed ? 2 * Gp * lo : sizeof(double) * 2 * G;
    if (frow > row) row = frow;
    b->bp_tmp = a.take<char>(row * W);
  }
  b->mixed = mixed;
  b->f32lu = p.precision == AFQMC_MIXED_TF32_F32LU || p.precision == AFQMC_MIXED_BF16_F32LU;
  b->theta32 = mixed && p.precision != AFQMC_MIXED_TF32_F64THETA &&
               p.precision != AFQMC_MIXED_BF16_F64THETA;
  b->lo_kind = mixed ? (lo == 2 ? LO_BF16 : LO_TF32) : LO_NONE;
  b->lo_bytes = (int)lo;
  b->Gp = (int)Gp;
  b->Mp = (int)Mp;
  b->Pp = (long)Pp;
  if (mixed) {
    // Cholesky operand of V: the upper 16 x 16 blocks of each vector, 256 rows per block
    b->nblkV = (int)((Mp / 16) * (Mp / 16 + 1) / 2);
    b->LbT_lo = a.take<char>((size_t)b->nblkV * 256 * Gp * lo);
    b->Lh_lo = a.take<char>(G * N * Mp * lo);
    b->x_lo = a.take<char>(W * 2 * Gp * lo);
    b->th_lo = a.take<char>(W * 2 * N * Mp * lo);
    b->t32 = a.take<float>(W * 2 * G);
    b->Bh_lo = a.take<char>(M * Mp * lo);
    b->Bh_tf = a.take<float>(M * 2 * Mp);
    b->Kp1 = (int)((M + 128 / lo - 1) / (128 / lo) * (128 / lo));
    b->Bh_split = a.take<char>(M * 2 * (size_t)b->Kp1 * lo);
    b->Bh_split_tf = a.take<float>(M * 4 * Mp);
  }
  // scratch: the set-up and the step never run at the same time
  const size_t scratch_at = (a.off + 255) & ~size_t(255);
  Bump s1{base, scratch_at};
  if (mixed) {
    b->Y = nullptr;
    b->acc = nullptr;
    b->V_lo = s1.take<char>(W * M * 2 * Mp * lo);
    b->phi_lo = s1.take<char>(W * 2 * N * Mp * lo);
    b->acc32 = s1.take<float>(W * 2 * N * 2 * Mp);
    b->Tb0 = s1.take<char>(W * 2 * N * 2 * Mp * lo);
    b->Tb1 = s1.take<char>(W * 2 * N * 2 * Mp * lo);
  } else {
    b->Y = s1.take<double>(W * 2 * P);
    b->acc = s1.take<double>(W * 2 * N * M);
  }
  b->T0 = s1.take<double>(W * 2 * N * M);  // Taylor terms (FP64) / comb copies
  b->T1 = s1.take<double>(W * 2 * N * M);
  b->tmp_ld = s1.take<double>(2 * W);
  Bump s2{base, scratch_at};
  b->Lfull = s2.take<double>(G * M * M);
  b->L2 = s2.take<double>(M * M);
  b->cLp = s2.take<double>(P);
  b->E0 = s2.take<double>(M * M);
  b->E1 = s2.take<double>(M * M);
  b->X = s2.take<double>(M * M);
  b->red = s2.take<double>(8);
  b->ych = (int)(G < 32 ? G : 32);
  b->Ych = s2.take<double>((size_t)b->ych * M * M);
  b->P = (int)P;
  b->nchunk = (int)nchunk;
  b->gc = exchange_chunk((int)N, p.nchol);
  b->status = reinterpret_cast<int*>(b->counters + CTR_STATUS);
  return ((s1.off > s2.off ? s1.off : s2.off) + 255) & ~size_t(255);
}

// --------------------------------------------------------------- validation --
static int check_params(const afqmc_params* p) {
  if (!p) {
    set_error("params is NULL");
    return AFQMC_EINVAL;
  }
  if (p->M < 1 || p->N < 1 || p->N > p->M || p->nchol < 1 || p->nwalkers < 1) {
    set_error("bad sizes M=%d N=%d nchol=%d nwalkers=%d", p->M, p->N, p->nchol, p->nwalkers);
    return AFQMC_EINVAL;
  }
  if (p->N > 64) {
    set_error("N=%d: at most 64 electrons per spin are supported", p->N);
    return AFQMC_EUNSUPPORTED;
  }
  if (p->nwalkers > 65535) {
    // per-walker kernels put the walker index on the grid's y dimension
    set_error("nwalkers=%d: at most 65535 walkers per state are supported", p->nwalkers);
    return AFQMC_EUNSUPPORTED;
  }
  if (!(p->dt > 0.0) || !std::isfinite(p->dt)) {
    set_error("dt must be positive and finite");
    return AFQMC_EINVAL;
  }
  if (p->taylor_order < 1 || p->qr_period < 0 || p->pc_period < 0 || p->energy_period < 0 ||
      p->max_records < 1 || (p->use_graph != 0 && p->use_graph != 1)) {
    set_error("bad taylor_order / periods / max_records / use_graph");
    return AFQMC_EINVAL;
  }
  if (p->mode != AFQMC_PHASELESS && p->mode != AFQMC_FREE) {
    set_error("unknown mode %d", p->mode);
    return AFQMC_EINVAL;
  }
  if (p->mode == AFQMC_FREE && p->pc_period) {
    set_error("the comb needs real weights: pc_period must be 0 for free projection");
    return AFQMC_EINVAL;
  }
  if (p->precision < AFQMC_FP64 || p->precision > AFQMC_MIXED_BF16_F64THETA) {
    set_error("precision %d is not available in this build", p->precision);
    return AFQMC_EUNSUPPORTED;
  }
  if (p->bp_steps < 0 || p->ndet < 0 || p->Ndn < 0 || p->Ndn > p->M || p->walker0 < 0 ||
      (int64_t)p->walker0 + p->nwalkers > 0x7fffffffLL) {
    set_error("bp_steps < 0, ndet < 0, Ndn outside [0, M] or walker0 outside [0, 2^31 - nwalkers)");
    return AFQMC_EINVAL;
  }
  if (p->Ndn > 0) {
    if (p->N + p->Ndn > 64) {
      set_error("two spin blocks: N + Ndn = %d above 64", p->N + p->Ndn);
      return AFQMC_EUNSUPPORTED;
    }
    if (p->precision != AFQMC_FP64 || p->ndet || p->bp_steps) {
      set_error("two spin blocks run on the float64 path, with a single-determinant trial and "
                "no back-propagation window");
      return AFQMC_EUNSUPPORTED;
    }
  }
  if (p->ndet > 0 && (p->pc_period || p->bp_steps || p->mode != AFQMC_PHASELESS)) {
    set_error("a multi-determinant trial runs phaseless, without population control or "
              "back-propagation");
    return AFQMC_EUNSUPPORTED;
  }

  const double P = 0.5 * p->M * (p->M + 1.0);
  if ((double)p->nwalkers * 2 * p->N > 65535.0 * 64 || P * p->nchol > 4e10) {
    set_error("problem too large for this build");
    return AFQMC_EUNSUPPORTED;
  }
  if (!std::isfinite(p->H0) || !(std::isnan(p->e_shift) || std::isfinite(p->e_shift))) {
    set_error("H0 / e_shift not finite");
    return AFQMC_ENONFINITE;
  }
  return AFQMC_OK;
}

static int all_finite(const double* v, size_t n, const char* what) {
  for (size_t i = 0; i < n; ++i)
    if (!std::isfinite(v[i])) {
      set_error("%s[%zu] is not finite", what, i);
      return AFQMC_ENONFINITE;
    }
  return AFQMC_OK;
}

// ------------------------------------------------------------ step pieces ---
// The mixed path keeps phi_lo = BF16/TF32 copy of the orbitals (pitch Mp)
// current: the last half step writes both; every other change of the
// orbitals (Gram-Schmidt, comb, set-up, set_walkers, load) calls this.
int refresh_phi_lo(afqmc_state* s) {
  const Bufs& b = s->b;
  if (!b.mixed) return AFQMC_OK;
  const afqmc_params& p = s->p;
  return launch_convert_lo(b.phiT, 2L * p.N * p.nwalkers, p.M, p.M, b.phi_lo, b.Mp, b.lo_kind,
                           s->st);
}

// The same for the operand copy of Theta (pitch Mp), which the Theta kernel
// writes; the comb moves Theta without it.
int refresh_theta_lo(afqmc_state* s) {
  const Bufs& b = s->b;
  if (!b.mixed) return AFQMC_OK;
  const afqmc_params& p = s->p;
  return launch_convert_lo(b.thetaT, 2L * p.N * p.nwalkers, p.M, p.M, b.th_lo, b.Mp, b.lo_kind,
                           s->st);
}

int overlap_update(afqmc_state* s, bool into_ld, bool timed) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  if (p.ndet > 0) {
    if (timed) prof_begin(s, AFQMC_PH_OVERLAP);
    AFQ_TRY(md_overlap_update(s, into_ld));
    if (timed) prof_end(s);
    return AFQMC_OK;
  }
  // S = V_T^T Phi, S^-1, log det and Theta in one float64 kernel per walker
  OverlapArgs ov{p.nwalkers, p.M, p.N, b.VTt, b.phiT, b.thetaT, into_ld ? b.ld : b.ld_new, b.wt};
  // V_T' = [I_N; 0] in the trial-adapted basis; with two spin blocks only
  // the spin-up block is, and S = V_T'^T Phi' is formed per block
  ov.unit_trial = s->spin2 ? 0 : 1;
  ov.nup = s->nup;
  ov.sf = s->sf;
  ov.Sinv = reinterpret_cast<double2*>(b.Sinv);
  if (b.mixed) {
    ov.th_lo = b.th_lo;
    ov.lo_kind = b.lo_kind;
    ov.Mp = b.Mp;
    // FP32 elimination when asked for (_F32LU), else float64; the product
    // Theta = Phi S^-1 in FP32 unless the precision keeps it in float64
    if (b.f32lu) ov.Sinv32 = reinterpret_cast<float2*>(b.Sinv);
    ov.theta32 = b.theta32 ? 1 : 0;
  }
  if (timed) prof_begin(s, AFQMC_PH_OVERLAP);
  AFQ_TRY(launch_overlap(ov, s->st));
  if (timed) {
    prof_end(s);
    prof_begin(s, AFQMC_PH_THETA);
  }
  AFQ_TRY(launch_theta(ov, s->st));
  if (timed) prof_end(s);
  return AFQMC_OK;
}

// ---- the mixed path's per-step contractions as job descriptors --------------
// t[(w,c)][g] = 2 sum_(i,p) Theta^T_lo[(w,c)][(i,p)] Lh_lo[g][(i,p)] on tcgen05
void desc_force_bias(afqmc_state* s, TcJobDesc* d) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  d->kind = TC_JOB_STORE;
  d->g.m = 2 * p.nwalkers;
  d->g.n = p.nchol;
  d->g.k = p.N * b.Mp;
  d->g.A = b.th_lo;
  d->g.lda = (long)p.N * b.Mp;
  d->g.B = b.Lh_lo;
  d->g.ldb = (long)p.N * b.Mp;
  d->g.tf32 = b.lo_kind == LO_TF32;
  d->g.err = b.status;
  d->C = b.t32;
  d->ldc = p.nchol;
  d->alpha = 2.0f;
}

// V = i sqrt(dt) sum_g x_g L_g over the upper 16 x 16 blocks of the (p, q)
// grid (V is symmetric), each block and its mirror written straight into the
// [Re V | Im V] operand rows of the Taylor terms
void desc_v(afqmc_state* s, TcJobDesc* d) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  d->kind = TC_JOB_V;
  d->g.m = 2 * p.nwalkers;
  d->g.n = b.nblkV * 256;
  d->g.k = p.nchol;
  d->g.A = b.x_lo;
  d->g.lda = b.Gp;
  d->g.B = b.LbT_lo;
  d->g.ldb = b.Gp;
  d->g.tf32 = b.lo_kind == LO_TF32;
  d->g.err = b.status;
  d->V = b.V_lo;
  d->lo_kind = b.lo_kind;
  d->W = p.nwalkers;
  d->M = p.M;
  d->Mp = b.Mp;
  d->sdt = s->sdt;
}

// first half step: T_0 = (B_half Phi)^T = Phi^T + (Phi_lo D_B)^T, D_B =
// B_half - I (the identity part added in float64 orbitals by the epilogue),
// into columns [0, Mp) of the FP32 rows of acc (pitch 2 Mp) and, as the 0th
// Taylor operand, into Tb0
void desc_half1(afqmc_state* s, const double* phi_in, const void* phi_lo_in, TcJobDesc* d) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  d->kind = TC_JOB_PROP0;
  d->g.m = 2 * p.N * p.nwalkers;
  d->g.n = p.M;
  // D_B as [hi | lo] along K (segments of Kp1): Phi_lo (D_hi + D_lo)
  d->g.k = 2 * b.Kp1;
  d->g.ka = p.M;
  d->g.a_wrap = b.Kp1;
  d->g.A = phi_lo_in;
  d->g.lda = b.Mp;
  d->g.B = b.Bh_split;
  d->g.ldb = 2L * b.Kp1;
  d->g.tf32 = b.lo_kind == LO_TF32;
  d->g.err = b.status;
  d->acc = b.acc32;
  d->ldacc = 2L * b.Mp;
  d->tb = b.Tb0;
  d->phi_id = phi_in;
  d->lo_kind = b.lo_kind;
  d->N = p.N;
  d->M = p.M;
  d->Mp = b.Mp;
}

// last half step (TF32): Phi <- B_half (T_0 + S) = (T_0 + S) + [T_0 | S]
// [D_B | D_B] (one K = 2 Mp product; T_0 + S added in the epilogue); stored
// for live walkers
void desc_half2(afqmc_state* s, double* phi_out, void* phi_lo_out, TcJobDesc* d) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  d->kind = TC_JOB_PHI;
  d->g.m = 2 * p.N * p.nwalkers;
  d->g.n = p.M;
  // [T_0 | S] against [D_hi | D_hi | D_lo | D_lo] (segments of Mp)
  d->g.k = 4 * b.Mp;
  d->g.ka = 2 * b.Mp;
  d->g.a_wrap = 2 * b.Mp;
  d->g.A = b.acc32;
  d->g.lda = 2L * b.Mp;
  d->g.B = b.Bh_split_tf;
  d->g.ldb = 4L * b.Mp;
  d->g.tf32 = true;
  d->g.err = b.status;
  d->phiT = phi_out;
  d->wt = b.wt;
  d->N = p.N;
  d->M = p.M;
  d->phi_lo = phi_lo_out;
  d->lo_kind = b.lo_kind;
  d->Mp = b.Mp;
  d->acc_id = b.acc32;
}

int force_bias_gemm(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  if (p.ndet > 0) {
    AFQ_TRY(md_force_bias(s));
    s->t_fresh = true;
    return AFQMC_OK;
  }
  if (b.mixed) {
    TcJobDesc d;
    desc_force_bias(s, &d);
    AFQ_TRY(tc_job_launch(d, s->st));
    s->t_fresh = true;
    return AFQMC_OK;
  }
  GemmF64 g;
  g.m = 2 * p.nwalkers;
  g.n = p.nchol;
  g.k = p.N * p.M;
  g.alpha = s->sf;  // sum over spins: 2 Tr(Lh_g Theta) for the closed-shell block
  g.A = b.thetaT;
  g.lda = (long)p.N * p.M;
  g.B = b.Lh;
  g.ldb = (long)p.N * p.M;
  g.C = b.t;
  g.ldc = p.nchol;
  AFQ_TRY(gemm_nt_f64(g, s->st));
  s->t_fresh = true;
  return AFQMC_OK;
}

int energy_eval(afqmc_state* s, bool append, bool record = true) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  if (!s->t_fresh) AFQ_TRY(force_bias_gemm(s));
  if (p.ndet > 0) {
    AFQ_TRY(md_local_energies(s));
  } else if (b.mixed) {
    // T_g = Lh_g Theta for all (g, w) on tcgen05, sum_ij T_ij T_ji in the epilogue
    TcGemm g;
    g.m = p.nchol * p.N;
    g.n = 2 * p.N * p.nwalkers;
    g.k = p.M;
    g.A = b.Lh_lo;
    g.lda = b.Mp;
    g.B = b.th_lo;
    g.ldb = b.Mp;
    g.tf32 = b.lo_kind == LO_TF32;
    g.err = b.status;
    AFQ_TRY(tc_exchange(g, p.nchol, p.nwalkers, p.N, b.part, b.nchunk, s->st));
  } else {
    ExchArgs ex{p.nwalkers, p.M, p.N, p.nchol, b.gc, b.nchunk, b.Lh, b.thetaT, b.part, b.wt};
    ex.nup = s->nup;
    AFQ_TRY(launch_exchange(ex, s->st));
  }
  if (p.ndet == 0) {
    ElocArgs el{p.nwalkers, p.M, p.N, p.nchol, b.nchunk, p.H0, b.hh, b.thetaT, b.t, b.part, b.eloc,
                b.wt};
    el.t32 = b.mixed ? b.t32 : nullptr;
    el.sf = s->sf;
    AFQ_TRY(launch_eloc(el, s->st));
  }
  if (!record) return AFQMC_OK;
  RecordArgs rc;
  rc.W = p.nwalkers;
  rc.mode = p.mode;
  rc.max_records = p.max_records;
  rc.lo = s->elo;
  rc.hi = s->ehi;
  rc.eloc = b.eloc;
  rc.wt = b.wt;
  rc.records = append ? b.records : nullptr;
  rc.rec_count = b.counters + CTR_RECORDS;
  rc.last = b.last;
  rc.step = reinterpret_cast<const int64_t*>(b.counters + CTR_STEP);
  AFQ_TRY(launch_record(rc, s->st));
  return AFQMC_OK;
}

// Float64: phi_out <- B_half T_n(V) B_half phi_in with V = i sqrt(dt) sum_g x_g L_g
// for the fields in b.x (Eqs. primitive and hs2; Sec. 3.4.2); rows of walkers
// with W = 0 are not stored when mask is the weights.
int apply_b_f64(afqmc_state* s, const double* phi_in, double* phi_out, const double* mask) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, N = p.N, M = p.M, G = p.nchol;
  // Y = sum_g x_g L_g (packed), the dense contraction with K = N_gamma
  prof_begin(s, AFQMC_PH_V);
  GemmF64 g;
  g.m = 2 * W;
  g.n = b.P;
  g.k = G;
  g.A = b.x;
  g.lda = G;
  g.B = b.LpT;
  g.ldb = G;
  g.C = b.Y;
  g.ldc = b.P;
  AFQ_TRY(gemm_nt_f64(g, s->st));
  prof_end(s);
  // Phi <- B_half Phi  (Phi^T <- Phi^T B_half, B_half symmetric)
  prof_begin(s, AFQMC_PH_BHALF);
  GemmF64 bh;
  bh.m = 2 * N * W;
  bh.n = M;
  bh.k = M;
  bh.A = phi_in;
  bh.lda = M;
  bh.B = b.Bh;
  bh.ldb = M;
  bh.C = b.T0;
  bh.ldc = M;
  AFQ_TRY(gemm_nt_f64(bh, s->st));
  prof_end(s);
  // truncated Taylor series of exp(V)
  prof_begin(s, AFQMC_PH_TAYLOR);
  double* tin = b.T0;
  double* tout = b.T1;
  for (int k = 1; k <= p.taylor_order; ++k) {
    TaylorArgsT<double> ta{W, M, N, b.P, k, (long)b.P, s->sdt / k, b.Y, tin, tout, b.acc};
    AFQ_TRY(launch_taylor_term(ta, s->st));
    double* t_ = tin;
    tin = tout;
    tout = t_;
  }
  prof_end(s);
  // Phi <- B_half acc
  prof_begin(s, AFQMC_PH_BHALF);
  bh.A = b.acc;
  bh.C = phi_out;
  if (mask) {
    bh.mask = mask;
    bh.mask_rows = 2 * N;
  }
  AFQ_TRY(gemm_nt_f64(bh, s->st));
  prof_end(s);
  return AFQMC_OK;
}

static int propagate_f64(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, G = p.nchol;
  FieldArgs fa{W, G, p.mode, p.seed, s->sdt, p.fb_cap, b.t, b.c, b.wt, b.x, b.scal,
               reinterpret_cast<const int64_t*>(b.counters + CTR_STEP)};
  fa.w0 = p.walker0;
  prof_begin(s, AFQMC_PH_FIELDS);
  AFQ_TRY(launch_field(fa, s->st));
  prof_end(s);
  if (s->bp_on) AFQ_TRY(bp_record_fields(s));
  return apply_b_f64(s, b.phiT, b.phiT, b.wt);
}

// Mixed: the same product with every contraction on the tensor cores (BF16 or
// TF32 operands, FP32 accumulation) for the fields in b.x_lo: V, the first half
// step from the operand copy phi_lo_in, the Taylor series and the last half
// step (TF32), which stores float64 orbitals (walkers with W != 0) and their
// operand copy.
int join_side(afqmc_state* s) {
  if (!s->side_pending) return AFQMC_OK;
  AFQ_CUDA(cudaStreamWaitEvent(s->st, s->ev_side, 0));
  s->side_pending = false;
  return AFQMC_OK;
}

// terms k = 1..n of the Taylor series: S = T_1 + ... + T_n into columns
// [Mp, 2 Mp) of acc; the whole series in one launch when the term fits in
// shared memory, else one launch per term
int step_taylor(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  prof_begin(s, AFQMC_PH_TAYLOR);
  AFQ_TRY(taylor_apply(b.V_lo, b.Tb0, b.Tb1, b.acc32 + b.Mp, 2L * b.Mp, b.lo_kind, p.nwalkers, p.N,
                       p.M, b.Mp, p.taylor_order, false, b.status, s->st));
  prof_end(s);
  return AFQMC_OK;
}

int apply_b_mixed(afqmc_state* s, const double* phi_in, const void* phi_lo_in, double* phi_out,
                  void* phi_lo_out) {
  TcJobDesc d;
  prof_begin(s, AFQMC_PH_V);
  desc_v(s, &d);
  AFQ_TRY(tc_job_launch(d, s->st));
  prof_end(s);
  // the first half step reads the orbitals: a side-stream Gram-Schmidt must be done
  AFQ_TRY(join_side(s));
  prof_begin(s, AFQMC_PH_BHALF);
  d = TcJobDesc();
  desc_half1(s, phi_in, phi_lo_in, &d);
  AFQ_TRY(tc_job_launch(d, s->st));
  prof_end(s);
  AFQ_TRY(step_taylor(s));
  prof_begin(s, AFQMC_PH_BHALF);
  d = TcJobDesc();
  desc_half2(s, phi_out, phi_lo_out, &d);
  AFQ_TRY(tc_job_launch(d, s->st));
  prof_end(s);
  return AFQMC_OK;
}

// fields x = xi - xbar from the (fresh) force bias; on the mixed path also
// their BF16/TF32 operand rows
int step_fields(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, G = p.nchol;
  FieldArgs fa{W, G, p.mode, p.seed, s->sdt, p.fb_cap, nullptr, b.c, b.wt, nullptr, b.scal,
               reinterpret_cast<const int64_t*>(b.counters + CTR_STEP)};
  fa.w0 = p.walker0;
  fa.t32 = b.t32;
  fa.x_lo = b.x_lo;
  fa.lo_kind = b.lo_kind;
  fa.Gp = b.Gp;
  prof_begin(s, AFQMC_PH_FIELDS);
  AFQ_TRY(launch_field(fa, s->st));
  prof_end(s);
  if (s->bp_on) AFQ_TRY(bp_record_fields(s));
  return AFQMC_OK;
}

static int propagate_mixed(afqmc_state* s) {
  const Bufs& b = s->b;
  AFQ_TRY(step_fields(s));
  return apply_b_mixed(s, b.phiT, b.phi_lo, b.phiT, b.phi_lo);
}

int step_after(afqmc_state* s);

static int step_once(afqmc_state* s) {
  const Bufs& b = s->b;
  // force bias traces t = 2 Tr(Lh_g Theta) for every walker (Eq. precomputing2)
  if (!s->t_fresh) {
    prof_begin(s, AFQMC_PH_FORCE_BIAS);
    AFQ_TRY(force_bias_gemm(s));
    prof_end(s);
  }
  // fields, the force bias and x = xi - xbar; then exp(-dt v0'/2) T_n(V)
  // exp(-dt v0'/2) applied to every walker's orbitals
  AFQ_TRY(b.mixed ? propagate_mixed(s) : propagate_f64(s));
  return step_after(s);
}

// After the propagation: new overlap, log det, Theta; the weights (and step +=
// 1); then the periodic Gram-Schmidt, comb and energy record.
int step_after(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, N = p.N, M = p.M;
  AFQ_TRY(overlap_update(s, false, true));
  WeightArgs wa{W, p.mode, p.dt, s->sdt, s->H0p, s->e_shift, s->wmax, b.ld_new, b.ld, b.scal,
                b.wt, b.counters + CTR_NONFINITE,
                reinterpret_cast<int64_t*>(b.counters + CTR_STEP)};
  if (s->bp_on) wa.cosd = b.bp_cos;
  prof_begin(s, AFQMC_PH_WEIGHT);
  AFQ_TRY(launch_weight(wa, s->st));
  prof_end(s);
  s->t_fresh = false;
  s->h_step += 1;
  const int64_t n = s->h_step;
  if (s->bp_on) {
    // back-propagation window: this step's BP-PRes factor needs E_loc(Psi_k)
    // of every walker, taken before Gram-Schmidt (which leaves it unchanged)
    // and before a comb (which then copies factor and path together)
    AFQ_TRY(energy_eval(s, false, false));
    AFQ_TRY(bp_step_factor(s));
    s->bp_m += 1;
  }
  const bool qr_due = p.qr_period && n % p.qr_period == 0;
  const bool pc_due = p.pc_period && n % p.pc_period == 0;
  const bool e_due = p.energy_period && n % p.energy_period == 0;
  // Gram-Schmidt on the side stream when nothing of this step after it reads
  // the orbitals before the next first half step (no comb due): then the
  // energy evaluation, which reads neither Phi nor ld, is enqueued first so
  // that its persistent contraction takes the SMs and the sweep fills in
  const bool side = qr_due && !pc_due && s->side && !s->prof.on && !s->bp_on;
  if (side && e_due) {
    prof_begin(s, AFQMC_PH_ENERGY);
    AFQ_TRY(energy_eval(s, true));
    prof_end(s);
  }
  if (qr_due) {
    prof_begin(s, AFQMC_PH_QR);
    // Phi -> Q; Theta is unchanged and log det S drops by sum_k log r_kk,
    // which the kernel applies to ld (no new overlap needed)
    MgsArgs ma{W, M, N, b.phiT, b.wt, b.ld};
    ma.nup = s->nup;
    ma.sf = s->sf;
    if (b.mixed) {
      // the sweep (FP32 in shared memory when asked for, else float64) also
      // refreshes the operand copy of the orbitals
      ma.f32 = b.f32lu ? 1 : 0;
      ma.phi_lo = b.phi_lo;
      ma.lo_kind = b.lo_kind;
      ma.Mp = b.Mp;
    }
    if (side) {
      // join_side() before the next reader (the next first half step)
      AFQ_CUDA(cudaEventRecord(s->ev_fork, s->st));
      AFQ_CUDA(cudaStreamWaitEvent(s->side, s->ev_fork, 0));
      AFQ_TRY(launch_mgs(ma, s->side));
      AFQ_CUDA(cudaEventRecord(s->ev_side, s->side));
      s->side_pending = true;
    } else {
      AFQ_TRY(launch_mgs(ma, s->st));
    }
    prof_end(s);
  }
  if (pc_due) {
    AFQ_TRY(join_side(s));
    prof_begin(s, AFQMC_PH_COMB);
    CombArgs ca{W, M, N, p.seed, reinterpret_cast<const int64_t*>(b.counters + CTR_STEP),
                b.wt, b.cum, b.parent, b.phiT, b.thetaT, b.ld, b.T0, b.T1, b.tmp_ld, b.wtot};
    AFQ_TRY(launch_comb(ca, s->st));
    AFQ_TRY(refresh_phi_lo(s));
    AFQ_TRY(refresh_theta_lo(s));
    if (s->bp_on) AFQ_TRY(bp_after_comb(s));
    s->t_fresh = false;  // the walkers moved: their force-bias traces are stale
    prof_end(s);
  }
  if (e_due && !(side && e_due)) {
    prof_begin(s, AFQMC_PH_ENERGY);
    AFQ_TRY(energy_eval(s, true));
    prof_end(s);
  }
  return AFQMC_OK;
}

// One graph block of steps launched kernel by kernel (captured by groups).
int step_block(afqmc_state* s) {
  for (int i = 0; i < s->graph_block; ++i) AFQ_TRY(step_once(s));
  return join_side(s);
}

// B_half = exp(X), X = -dt v0'/2, by scaling and squaring of a degree-18
// Taylor polynomial evaluated by Horner's rule (all float64 GEMMs).
static int expm_device(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int M = p.M;
  AFQ_TRY(launch_norm1(b.X, b.red, M, s->st));
  double nrm = 0.0;
  AFQ_CUDA(cudaMemcpyAsync(&nrm, b.red, sizeof(double), cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  if (!std::isfinite(nrm)) {
    set_error("one-body operator is not finite");
    return AFQMC_ENONFINITE;
  }
  int sq = 0;
  while (nrm > 0.5 && sq < 60) {
    nrm *= 0.5;
    ++sq;
  }
  if (sq) AFQ_TRY(launch_scale(b.X, (long)M * M, std::ldexp(1.0, -sq), s->st));
  double* E = b.E0;
  double* F = b.E1;
  AFQ_TRY(launch_fill_identity(E, M, 1.0, s->st));
  for (int k = 18; k >= 1; --k) {
    AFQ_TRY(launch_fill_identity(F, M, 1.0, s->st));
    GemmF64 g;
    g.m = g.n = g.k = M;
    g.alpha = 1.0 / k;
    g.beta = 1.0;
    g.A = b.X;
    g.lda = M;
    g.B = E;
    g.ldb = M;
    g.C = F;
    g.ldc = M;
    AFQ_TRY(gemm_nt_f64(g, s->st));
    double* t_ = E;
    E = F;
    F = t_;
  }
  for (int i = 0; i < sq; ++i) {
    GemmF64 g;
    g.m = g.n = g.k = M;
    g.A = E;
    g.lda = M;
    g.B = E;
    g.ldb = M;
    g.C = F;
    g.ldc = M;
    AFQ_TRY(gemm_nt_f64(g, s->st));
    double* t_ = E;
    E = F;
    F = t_;
  }
  AFQ_CUDA(cudaMemcpyAsync(b.Bh, E, sizeof(double) * M * M, cudaMemcpyDeviceToDevice, s->st));
  return AFQMC_OK;
}

// An orthogonal M x M matrix (row-major) whose first N columns are the trial
// orbitals: the Householder QR of the trial (reflectors H_1 .. H_N) gives
// Q_H = H_1 ... H_N, whose first N columns span the trial and whose other
// columns are an orthonormal basis of the complement; the first N columns are
// then set to the trial itself.
static void complete_basis(const double* trial, int M, int N, std::vector<double>& q) {
  std::vector<double> a(trial, trial + (size_t)M * N);  // [M][N]
  std::vector<double> v((size_t)N * M, 0.0);           // reflector k: v[k][k .. M)
  for (int k = 0; k < N; ++k) {
    double nrm = 0.0;
    for (int r = k; r < M; ++r) nrm += a[(size_t)r * N + k] * a[(size_t)r * N + k];
    nrm = std::sqrt(nrm);
    double* vk = &v[(size_t)k * M];
    const double alpha = a[(size_t)k * N + k] >= 0.0 ? -nrm : nrm;
    for (int r = k; r < M; ++r) vk[r] = a[(size_t)r * N + k];
    vk[k] -= alpha;
    double vn = 0.0;
    for (int r = k; r < M; ++r) vn += vk[r] * vk[r];
    vn = std::sqrt(vn);
    if (vn > 0.0)
      for (int r = k; r < M; ++r) vk[r] /= vn;
    for (int j = k; j < N; ++j) {
      double d = 0.0;
      for (int r = k; r < M; ++r) d += vk[r] * a[(size_t)r * N + j];
      for (int r = k; r < M; ++r) a[(size_t)r * N + j] -= 2.0 * d * vk[r];
    }
  }
  q.assign((size_t)M * M, 0.0);
  for (int i = 0; i < M; ++i) q[(size_t)i * M + i] = 1.0;
  for (int k = N - 1; k >= 0; --k) {  // Q_H = H_1 (H_2 (... (H_N I)))
    const double* vk = &v[(size_t)k * M];
    for (int c = 0; c < M; ++c) {
      double d = 0.0;
      for (int r = k; r < M; ++r) d += vk[r] * q[(size_t)r * M + c];
      for (int r = k; r < M; ++r) q[(size_t)r * M + c] -= 2.0 * d * vk[r];
    }
  }
  for (int r = 0; r < M; ++r)
    for (int i = 0; i < N; ++i) q[(size_t)r * M + i] = trial[(size_t)r * N + i];
}

// C = A B^T for M x M float64 matrices batched over `batch` (strides 0 = shared).
static int gemm_sq(const double* A, long sA, const double* B, long sB, double* C, long sC, int M,
                   int batch, cudaStream_t st) {
  GemmF64 g;
  g.m = g.n = g.k = M;
  g.batch = batch;
  g.A = A;
  g.lda = M;
  g.sAb = sA;
  g.B = B;
  g.ldb = M;
  g.sBb = sB;
  g.C = C;
  g.ldc = M;
  g.sCb = sC;
  return gemm_nt_f64(g, st);
}

// The run works in the trial-adapted orthonormal basis {Q_p}: h' = Q^T h Q,
// L'_g = Q^T L_g Q and V_T' = Q^T V_T = [I_N; 0].  Energies, overlap ratios,
// weights and the fields' force bias are the same in any orthonormal basis;
// what changes is that S = V_T'^T Phi' is the top N x N block of Phi' (no
// product) and the top N rows of Theta' = Phi' S^-1 are the identity.
// Walkers cross the API in the caller's basis: Phi = Q Phi'.
// max |V^T V - I| of an M x N row-major matrix
static double orthonormality_error(const double* V, int M, int N) {
  double dev = 0.0;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j <= i; ++j) {
      double d = 0.0;
      for (int q = 0; q < M; ++q) d += V[(size_t)q * N + i] * V[(size_t)q * N + j];
      dev = std::fmax(dev, std::fabs(d - (i == j ? 1.0 : 0.0)));
    }
  return dev;
}

// md_coef / md_up / md_dn: a multi-determinant trial (p.ndet >= 1), whose
// leading spin-up orbitals md_up[0] are then the trial of the basis and of
// the initial walkers.
static int setup_device(afqmc_state* s, const double* h1, const double* L, const double* trial,
                        const double* trial_dn = nullptr, const double* md_coef = nullptr,
                        const double* md_up = nullptr, const double* md_dn = nullptr) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int M = p.M, N = p.N, G = p.nchol, W = p.nwalkers;
  const int nup = s->nup;  // spin-up columns (N unless two spin blocks)
  cudaStream_t st = s->st;
  const bool md = p.ndet > 0;
  if (md) trial = md_up;
  // the trial's columns must be orthonormal
  for (int ds = 0; ds < (md ? 2 * p.ndet : (s->spin2 ? 2 : 1)); ++ds) {
    const double* V = md ? ((ds & 1) ? md_dn : md_up) + (size_t)(ds >> 1) * M * N
                         : (ds ? trial_dn : trial);
    const int nc = md ? N : (ds ? N - nup : nup);
    const double dev = orthonormality_error(V, M, nc);
    if (!(dev < 1e-8)) {
      set_error("trial columns are not orthonormal (determinant %d spin %d: max |V^T V - I| = "
                "%.3g)", ds >> 1, ds & 1, dev);
      return AFQMC_EINVAL;
    }
  }
  std::vector<double> qh, qt((size_t)M * M), vtt((size_t)N * M, 0.0);
  complete_basis(trial, M, nup, qh);
  if (md) {
    // the determinants' orbitals in the run's basis, V' = Q^T V, stored as
    // rows i = column i: [2 ndet][N][M]
    std::vector<double> mv((size_t)2 * p.ndet * N * M, 0.0);
    for (int ds = 0; ds < 2 * p.ndet; ++ds) {
      const double* V = ((ds & 1) ? md_dn : md_up) + (size_t)(ds >> 1) * M * N;
      double* o = mv.data() + (size_t)ds * N * M;
      for (int r = 0; r < M; ++r)
        for (int i = 0; i < N; ++i) {
          const double v = V[(size_t)r * N + i];
          if (v == 0.0) continue;
          for (int q = 0; q < M; ++q) o[(size_t)i * M + q] += v * qh[(size_t)r * M + q];
        }
    }
    AFQ_CUDA(cudaMemcpyAsync(b.md_V, mv.data(), sizeof(double) * mv.size(),
                             cudaMemcpyHostToDevice, st));
    AFQ_CUDA(cudaStreamSynchronize(st));
    AFQ_TRY(smw_detect(s, md_up, md_dn));
  }
  for (int r = 0; r < M; ++r)
    for (int c = 0; c < M; ++c) qt[(size_t)c * M + r] = qh[(size_t)r * M + c];
  for (int i = 0; i < nup; ++i) vtt[(size_t)i * M + i] = 1.0;
  // two spin blocks: rows nup.. are the spin-down orbitals in this basis,
  // (Q^T V_dn)^T (the basis is adapted to the spin-up trial only)
  for (int i = nup; i < N; ++i)
    for (int r = 0; r < M; ++r) {
      const double v = trial_dn[(size_t)r * (N - nup) + (i - nup)];
      if (v == 0.0) continue;
      for (int q = 0; q < M; ++q) vtt[(size_t)i * M + q] += v * qh[(size_t)r * M + q];
    }
  // sf P = sf sum_i v_i v_i^T with v_i the trial's orbitals in the caller's
  // basis (the first nup columns of Q): c_g = Tr(L_g P) without the rotation
  std::vector<double> Pt;
  if (b.mixed && !md && !s->spin2) {
    Pt.assign((size_t)M * M, 0.0);
    for (int r = 0; r < M; ++r)
      for (int q = 0; q < M; ++q) {
        double v = 0.0;
        for (int i = 0; i < nup; ++i) v += qh[(size_t)r * M + i] * qh[(size_t)q * M + i];
        Pt[(size_t)r * M + q] = s->sf * v;
      }
  }
  AFQ_CUDA(cudaMemcpyAsync(b.Qb, qh.data(), sizeof(double) * M * M, cudaMemcpyHostToDevice, st));
  AFQ_CUDA(cudaMemcpyAsync(b.QTb, qt.data(), sizeof(double) * M * M, cudaMemcpyHostToDevice, st));
  AFQ_CUDA(cudaMemcpyAsync(b.VTt, vtt.data(), sizeof(double) * N * M, cudaMemcpyHostToDevice, st));
  AFQ_CUDA(cudaMemcpyAsync(b.X, h1, sizeof(double) * M * M, cudaMemcpyHostToDevice, st));
  AFQ_CUDA(cudaMemcpyAsync(b.Lfull, L, sizeof(double) * G * M * M, cudaMemcpyHostToDevice, st));
  {
    // the Cholesky vectors must be finite: one pass on the device (a scan on
    // the host would cost more than the rest of the set-up)
    auto* first = reinterpret_cast<unsigned long long*>(b.red + 4);
    AFQ_CUDA(cudaMemsetAsync(first, 0xff, sizeof(unsigned long long), st));
    AFQ_TRY(launch_first_nonfinite(b.Lfull, (long)G * M * M, first, st));
    unsigned long long bad = 0;
    AFQ_CUDA(cudaMemcpyAsync(&bad, first, sizeof(bad), cudaMemcpyDeviceToHost, st));
    AFQ_CUDA(cudaStreamSynchronize(st));
    if (bad != ~0ull) {
      set_error("L[%llu] is not finite", bad);
      return AFQMC_ENONFINITE;
    }
  }
  AFQ_CUDA(cudaMemsetAsync(b.counters, 0, 8 * sizeof(unsigned long long), st));
  // h' = Q^T h Q and L'_g = Q^T L_g Q (h, L_g symmetric: B = h reads h^T)
  AFQ_TRY(gemm_sq(b.QTb, 0, b.X, 0, b.E0, 0, M, 1, st));
  AFQ_TRY(gemm_sq(b.E0, 0, b.QTb, 0, b.h1, 0, M, 1, st));
  // Single-determinant mixed path (closed shell): the rotated L'_g only feed
  // the BF16/TF32 operands, Lh_lo and B_half (applied as BF16/TF32 high and
  // low parts), so they are rotated in FP32.  What stays float64 is taken in
  // the caller's basis first: c_g = Tr(L_g P) (the mean field, H0') and
  // sum_g c_g L_g, rotated as one M x M matrix.
  const bool f32_rot = !Pt.empty();
  const long nL = (long)G * M * M, cL = (long)b.ych * M * M;  // chunk: Ych's doubles
  float* Lf = reinterpret_cast<float*>(b.Lfull);
  if (f32_rot) {
    AFQ_CUDA(cudaMemcpyAsync(b.E1, Pt.data(), sizeof(double) * M * M, cudaMemcpyHostToDevice, st));
    AFQ_TRY(launch_rowdot(b.Lfull, b.E1, b.c, G, M * M, 1.0, st));
    const int nz = (int)std::min<long>(b.ych, G);
    AFQ_TRY(launch_wsum_rows(b.Lfull, b.c, G, (long)M * M, nz, b.Ych, st));
    AFQ_TRY(launch_sum_parts(b.Ych, nz, (long)M * M, b.X, st));  // sum_g c_g L_g
    AFQ_TRY(gemm_sq(b.QTb, 0, b.X, 0, b.E0, 0, M, 1, st));
    AFQ_TRY(gemm_sq(b.E0, 0, b.QTb, 0, b.E1, 0, M, 1, st));
    AFQ_TRY(launch_pack_transpose(b.E1, b.cLp, 1, M, st));  // packed, as v0p reads it
    // L and Q^T to FP32 (L in place: the FP32 array starts at Lfull)
    AFQ_TRY(launch_round_f32_inplace(b.Lfull, nL, cL, reinterpret_cast<float*>(b.Ych), st));
    AFQ_TRY(launch_round_f32(b.QTb, reinterpret_cast<float*>(b.E0), (long)M * M, st));
  }
  for (int g0 = 0; g0 < G; g0 += b.ych) {
    const int nb = G - g0 < b.ych ? G - g0 : b.ych;
    if (f32_rot) {
      float* Y = reinterpret_cast<float*>(b.Ych);
      const float* QTf = reinterpret_cast<const float*>(b.E0);
      float* Lg = Lf + (size_t)g0 * M * M;
      GemmNT<float, float, float> y;  // Q^T L_g
      y.m = y.n = y.k = M;
      y.batch = nb;
      y.A = QTf;
      y.lda = M;
      y.B = Lg;
      y.ldb = M;
      y.sBb = (long)M * M;
      y.C = Y;
      y.ldc = M;
      y.sCb = (long)M * M;
      AFQ_TRY(gemm_nt_fff(y, st));
      GemmNT<float, float, float> r = y;  // (Q^T L_g) Q, back into L_g's place
      r.A = Y;
      r.sAb = (long)M * M;
      r.B = QTf;
      r.sBb = 0;
      r.C = Lg;
      AFQ_TRY(gemm_nt_fff(r, st));
    } else {
      double* Lg = b.Lfull + (size_t)g0 * M * M;
      AFQ_TRY(gemm_sq(b.QTb, 0, Lg, (long)M * M, b.Ych, (long)M * M, M, nb, st));
      AFQ_TRY(gemm_sq(b.Ych, (long)M * M, b.QTb, 0, Lg, (long)M * M, M, nb, st));
    }
  }
  // packed, transposed Cholesky vectors for the float64 V contraction
  if (!f32_rot) AFQ_TRY(launch_pack_transpose(b.Lfull, b.LpT, G, M, st));
  // half-rotated vectors Lh_g = V_T^T L_g and hh = V_T^T h (Eq. precomputing2)
  {
    GemmF64 g;
    g.m = N;
    g.n = M;
    g.k = M;
    g.batch = G;
    g.A = b.VTt;
    g.lda = M;
    g.B = b.Lfull;
    g.ldb = M;
    g.sBb = (long)M * M;
    g.C = b.Lh;
    g.ldc = M;
    g.sCb = (long)N * M;
    if (f32_rot)  // V_T' = [I_N; 0]: the first N rows of each L'_g
      AFQ_TRY(launch_widen_rows(Lf, (long)M * M, (long)N * M, G, b.Lh, st));
    else
      AFQ_TRY(gemm_nt_f64(g, st));
    GemmF64 h;
    h.m = N;
    h.n = M;
    h.k = M;
    h.A = b.VTt;
    h.lda = M;
    h.B = b.h1;
    h.ldb = M;
    h.C = b.hh;
    h.ldc = M;
    AFQ_TRY(gemm_nt_f64(h, st));
  }
  // c_g = Tr(L_g P) = sf Tr(Lh_g V_T) summed over the spin blocks (2 Tr(Lh_g V_T)
  // closed shell): vbar_g = i c_g (Sec. 2.4); with a multi-determinant trial
  // the leading determinant's Tr(L_g (P_0u + P_0d))
  if (md)
    AFQ_TRY(md_setup(s, md_coef));
  else if (!f32_rot)
    AFQ_TRY(launch_rowdot(b.Lh, b.VTt, b.c, G, N * M, s->sf, st));
  // sum_g L_g L_g: one M x M output with K = G M would occupy a few dozen
  // CTAs, so the vectors go in ych - 1 equal chunks plus the remainder, each
  // chunk's sum a partial in Ych, the partials then added in order
  {
    const int np = b.ych > 1 ? b.ych - 1 : 1;
    const int chunk = G / np, rem = G - np * chunk;
    GemmF64 g;
    g.m = g.n = g.k = M;
    g.kb = chunk;
    g.batch = np;
    g.A = b.Lfull;
    g.lda = M;
    g.sAk = (long)M * M;
    g.sAb = (long)chunk * M * M;
    g.B = b.Lfull;
    g.ldb = M;
    g.sBk = (long)M * M;
    g.sBb = (long)chunk * M * M;
    g.C = b.Ych;
    g.ldc = M;
    g.sCb = (long)M * M;
    // (mixed path: the FP32 L', FP32 products summed in float64 across 16-term blocks)
    GemmNT<float, float, double> gf;
    gf.m = gf.n = gf.k = M;
    gf.kb = chunk;
    gf.batch = np;
    gf.A = gf.B = Lf;
    gf.lda = gf.ldb = M;
    gf.sAk = gf.sBk = (long)M * M;
    gf.sAb = gf.sBb = (long)chunk * M * M;
    gf.C = b.Ych;
    gf.ldc = M;
    gf.sCb = (long)M * M;
    if (chunk > 0) AFQ_TRY(f32_rot ? gemm_nt_ffd_split(gf, st) : gemm_nt_f64(g, st));
    if (rem > 0) {
      GemmF64 r = g;
      r.kb = rem;
      r.batch = 1;
      r.A = b.Lfull + (size_t)np * chunk * M * M;
      r.B = r.A;
      r.C = b.Ych + (size_t)np * M * M;
      GemmNT<float, float, double> rf = gf;
      rf.kb = rem;
      rf.batch = 1;
      rf.A = rf.B = Lf + (size_t)np * chunk * M * M;
      rf.C = r.C;
      AFQ_TRY(f32_rot ? gemm_nt_ffd_split(rf, st) : gemm_nt_f64(r, st));
    }
    AFQ_TRY(launch_sum_parts(chunk > 0 ? b.Ych : b.Ych + (size_t)np * M * M,
                             (chunk > 0 ? np : 0) + (rem > 0 ? 1 : 0), (long)M * M, b.L2, st));
  }
  // sum_g c_g L_g (packed: one dot over g per pair p <= q; the mixed path
  // formed it above)
  if (!f32_rot) AFQ_TRY(launch_rowdot(b.LpT, b.c, b.cLp, b.P, G, 1.0, st));
  AFQ_TRY(launch_v0p(b.h1, b.L2, b.cLp, b.X, M, -0.5 * p.dt, st));
  AFQ_TRY(launch_sumsq(b.c, b.red + 1, G, st));
  double sumc2 = 0.0;
  AFQ_CUDA(cudaMemcpyAsync(&sumc2, b.red + 1, sizeof(double), cudaMemcpyDeviceToHost, st));
  AFQ_TRY(expm_device(s));  // synchronises once
  s->H0p = p.H0 - 0.5 * sumc2;
  if (b.mixed) {
    // BF16 / TF32 copies of the contraction operands (zero-padded pitches)
    if (f32_rot)
      AFQ_TRY(launch_pack_blocks_lo(Lf, G, M, b.Mp, b.Gp, b.LbT_lo, b.lo_kind, st));
    else
      AFQ_TRY(launch_pack_blocks_lo(b.Lfull, G, M, b.Mp, b.Gp, b.LbT_lo, b.lo_kind, st));
    AFQ_TRY(launch_convert_lo(b.Lh, (long)G * N, M, M, b.Lh_lo, b.Mp, b.lo_kind, st));
    AFQ_CUDA(cudaMemsetAsync(b.th_lo, 0, (size_t)W * 2 * N * b.Mp * b.lo_bytes, st));
    AFQ_CUDA(cudaMemsetAsync(b.x_lo, 0, (size_t)W * 2 * b.Gp * b.lo_bytes, st));
    // D_B = B_half - I: the half steps apply the identity part exactly
    AFQ_TRY(launch_convert_lo(b.Bh, M, M, M, b.Bh_lo, b.Mp, b.lo_kind, st, 1.0));
    // [D_B | D_B] so that one K = 2 Mp product applies it to T_0 + S
    AFQ_TRY(launch_convert_lo(b.Bh, M, M, M, b.Bh_tf, 2L * b.Mp, LO_TF32, st, 1.0));
    AFQ_CUDA(cudaMemcpy2DAsync(b.Bh_tf + b.Mp, sizeof(float) * 2 * b.Mp, b.Bh_tf,
                               sizeof(float) * 2 * b.Mp, sizeof(float) * b.Mp, M,
                               cudaMemcpyDeviceToDevice, st));
    // rounded once, D_B would be the same slightly wrong one-body propagator
    // for every walker at every step: the half steps take it as a high and a
    // low part (twice the K, a product the half steps' memory traffic hides)
    AFQ_TRY(launch_split_lo(b.Bh, M, M, M, b.Bh_split, b.Kp1, 2, 0x2u, b.lo_kind, st, 1.0));
    AFQ_TRY(launch_split_lo(b.Bh, M, M, M, b.Bh_split_tf, b.Mp, 4, 0xCu, LO_TF32, st, 1.0));
  }
  // walkers at the trial, their overlaps, and the trial energy
  AFQ_TRY(launch_init_walkers(b.VTt, b.phiT, b.wt, W, N, M, st));
  AFQ_TRY(refresh_phi_lo(s));
  AFQ_TRY(overlap_update(s, true, false));
  s->t_fresh = false;
  s->elo = -INFINITY;
  s->ehi = INFINITY;
  AFQ_TRY(energy_eval(s, false));
  double e0[2];
  AFQ_CUDA(cudaMemcpyAsync(e0, b.eloc, sizeof(e0), cudaMemcpyDeviceToHost, st));
  AFQ_CUDA(cudaStreamSynchronize(st));
  s->E_T = e0[0];
  if (b.mixed) {
    // the tensor-core operands read their padded columns: clear them once, now
    // that the set-up scratch these buffers alias is no longer needed
    AFQ_CUDA(cudaMemsetAsync(b.acc32, 0, sizeof(float) * (size_t)W * 2 * N * 2 * b.Mp, st));
    AFQ_CUDA(cudaMemsetAsync(b.Tb0, 0, (size_t)W * 2 * N * 2 * b.Mp * b.lo_bytes, st));
    AFQ_CUDA(cudaMemsetAsync(b.Tb1, 0, (size_t)W * 2 * N * 2 * b.Mp * b.lo_bytes, st));
    // autotune the tile width of the force-bias contraction for this shape
    TcGemm gf;
    gf.m = 2 * W;
    gf.n = G;
    gf.k = N * b.Mp;
    gf.A = b.th_lo;
    gf.lda = (long)N * b.Mp;
    gf.B = b.Lh_lo;
    gf.ldb = (long)N * b.Mp;
    gf.tf32 = b.lo_kind == LO_TF32;
    gf.err = b.status;
    AFQ_TRY(tc_tune_store(gf, b.t32, G, 2.0f, st, &s->bn_fb));
    // and of the V contraction (its output, the Taylor operand, is scratch here)
    TcJobDesc dv;
    desc_v(s, &dv);
    AFQ_TRY(tc_tune_v(dv.g, dv.V, dv.lo_kind, dv.W, dv.M, dv.Mp, dv.sdt, st, &s->bn_v));
    s->t_fresh = false;
    AFQ_CUDA(cudaStreamSynchronize(st));
  }
  s->e_shift = std::isnan(p.e_shift) ? s->E_T : p.e_shift;
  s->wmax = std::isnan(p.wmax) ? std::fmax(100.0, W / 10.0) : p.wmax;
  if (p.ecap_C > 0.0) {
    const double half = std::sqrt(p.ecap_C / p.dt);
    s->elo = s->E_T - half;
    s->ehi = s->E_T + half;
  }
  if (!std::isfinite(s->E_T)) {
    set_error("trial energy is not finite");
    return AFQMC_ENONFINITE;
  }
  return AFQMC_OK;
}

}  // namespace afq

static_assert(sizeof(afqmc_params) == 120, "afqmc_params layout");
static_assert(sizeof(afqmc_info) == 64, "afqmc_info layout");

using namespace afq;

// ================================================================= C ABI ====
extern "C" {

void afqmc_default_params(afqmc_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->dt = 0.005;
  p->e_shift = NAN;
  p->H0 = 0.0;
  p->seed = 1;
  p->taylor_order = 6;
  p->qr_period = 5;
  p->pc_period = 0;
  p->energy_period = 1;
  p->precision = AFQMC_FP64;
  p->mode = AFQMC_PHASELESS;
  p->ecap_C = 2.0;
  p->fb_cap = 1.0;
  p->wmax = NAN;
  p->max_records = 4096;
}

int afqmc_workspace_size(const afqmc_params* p, size_t* bytes) {
  AFQ_TRY(check_params(p));
  if (!bytes) {
    set_error("bytes is NULL");
    return AFQMC_EINVAL;
  }
  *bytes = plan(*p, nullptr, nullptr);
  return AFQMC_OK;
}

}  // extern "C"

// Workspace checks, the state, the device set-up and the graph block, for
// afqmc_init (trial) and afqmc_init_multidet (md_*).
static int init_state(const afqmc_params* p, const double* h1, const double* L,
                      const double* trial, const double* trial_dn, const double* md_coef,
                      const double* md_up, const double* md_dn, void* d_workspace,
                      size_t ws_bytes, void* stream, afqmc_state** out) {
  if (reinterpret_cast<uintptr_t>(d_workspace) % 256) {
    set_error("workspace must be 256-byte aligned");
    return AFQMC_EINVAL;
  }
  if (p->use_graph && (stream == nullptr || stream == (void*)cudaStreamLegacy ||
                       stream == (void*)cudaStreamPerThread)) {
    set_error("use_graph needs a stream created by the caller (default streams cannot be captured)");
    return AFQMC_EINVAL;
  }
  const size_t need = plan(*p, nullptr, nullptr);
  if (ws_bytes < need) {
    set_error("workspace %zu bytes < %zu needed", ws_bytes, need);
    return AFQMC_ENOSPC;
  }
  const size_t M = p->M, N = p->N;
  const size_t nd = p->ndet > 0 ? p->ndet : 0;
  AFQ_TRY(all_finite(h1, M * M, "h1"));
  if (nd) {
    AFQ_TRY(all_finite(md_coef, 2 * nd, "coef"));
    AFQ_TRY(all_finite(md_up, nd * M * N, "trial_up"));
    AFQ_TRY(all_finite(md_dn, nd * M * N, "trial_dn"));
  } else {
    AFQ_TRY(all_finite(trial, M * N, "trial_up"));
    if (p->Ndn > 0) AFQ_TRY(all_finite(trial_dn, M * (size_t)p->Ndn, "trial_dn"));
  }
  // L (G M^2 values) is checked on the device after its upload (setup_device)
  afqmc_state* s = new (std::nothrow) afqmc_state();
  if (!s) {
    set_error("out of host memory");
    return AFQMC_EINVAL;
  }
  s->p = *p;
  // internally N counts every orbital column of a walker: with two spin
  // blocks the N_up spin-up columns are followed by the N_dn spin-down ones
  s->nup = p->N;
  if (p->Ndn > 0) {
    s->spin2 = true;
    s->sf = 1.0;
    s->p.N = p->N + p->Ndn;
    s->p.Ndn = 0;
  }
  s->st = static_cast<cudaStream_t>(stream);
  s->ws = static_cast<char*>(d_workspace);
  s->ws_bytes = ws_bytes;
  plan(s->p, &s->b, s->ws);
  s->sdt = std::sqrt(p->dt);
  int r = setup_device(s, h1, L, trial, trial_dn, md_coef, md_up, md_dn);
  if (r != AFQMC_OK) {
    // work enqueued before the failing call still runs in the caller's
    // workspace: let it finish before the caller may free that memory
    cudaStreamSynchronize(s->st);
    delete s;
    return r;
  }
  if (s->b.mixed) {
    // lowest priority: the main stream's blocks are scheduled first
    int lo_pri = 0, hi_pri = 0;
    cudaDeviceGetStreamPriorityRange(&lo_pri, &hi_pri);
    if (cudaStreamCreateWithPriority(&s->side, cudaStreamNonBlocking, lo_pri) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&s->ev_side, cudaEventDisableTiming) != cudaSuccess) {
      if (s->side) cudaStreamDestroy(s->side);
      if (s->ev_fork) cudaEventDestroy(s->ev_fork);
      set_error("side stream or events could not be created");
      delete s;
      return AFQMC_ECUDA;
    }
  }
  // graph block: least common multiple of the non-zero periods (at most 64 steps)
  {
    long blk = 1;
    for (int per : {p->qr_period, p->pc_period, p->energy_period}) {
      if (per <= 0) continue;
      long a = blk, bb = per;
      while (bb) {
        const long t = a % bb;
        a = bb;
        bb = t;
      }
      blk = blk / a * per;
    }
    s->graph_block = blk <= 64 ? (int)blk : 0;
  }
  s->valid = true;
  *out = s;
  return AFQMC_OK;
}

extern "C" {

int afqmc_init(const afqmc_params* p, const double* h1, const double* L, const double* trial_up,
               const double* trial_dn, void* d_workspace, size_t ws_bytes, void* stream,
               afqmc_state** out) {
  if (!out) {
    set_error("out is NULL");
    return AFQMC_EINVAL;
  }
  *out = nullptr;
  AFQ_TRY(check_params(p));
  if (p->ndet != 0) {
    set_error("ndet = %d: a multi-determinant trial is set up by afqmc_init_multidet", p->ndet);
    return AFQMC_EINVAL;
  }
  if (!h1 || !L || !trial_up || !d_workspace) {
    set_error("h1, L, trial_up and d_workspace are required");
    return AFQMC_EINVAL;
  }
  if ((p->Ndn > 0) != (trial_dn != nullptr)) {
    set_error("trial_dn is required with two spin blocks (params.Ndn >= 1) and must be NULL "
              "otherwise");
    return AFQMC_EINVAL;
  }
  return init_state(p, h1, L, trial_up, trial_dn, nullptr, nullptr, nullptr, d_workspace,
                    ws_bytes, stream, out);
}

int afqmc_init_multidet(const afqmc_params* p, const double* h1, const double* L, int32_t ndet,
                        const double* coef, const double* trial_up, const double* trial_dn,
                        void* d_workspace, size_t ws_bytes, void* stream, afqmc_state** out) {
  if (!out) {
    set_error("out is NULL");
    return AFQMC_EINVAL;
  }
  *out = nullptr;
  AFQ_TRY(check_params(p));
  if (ndet < 1 || p->ndet != ndet) {
    set_error("afqmc_init_multidet: ndet = %d must be >= 1 and equal params.ndet = %d", ndet,
              p->ndet);
    return AFQMC_EINVAL;
  }
  if (!h1 || !L || !coef || !trial_up || !trial_dn || !d_workspace) {
    set_error("h1, L, coef, trial_up, trial_dn and d_workspace are required");
    return AFQMC_EINVAL;
  }
  return init_state(p, h1, L, nullptr, nullptr, coef, trial_up, trial_dn, d_workspace, ws_bytes,
                    stream, out);
}

#define AFQ_STATE(s)                       \
  do {                                     \
    if (!(s) || !(s)->valid) {             \
      set_error("invalid state");          \
      return AFQMC_ESTATE;                 \
    }                                      \
  } while (0)

int afqmc_propagate(afqmc_state* s, int32_t nsteps) {
  AFQ_STATE(s);
  if (nsteps < 0) {
    set_error("nsteps < 0");
    return AFQMC_EINVAL;
  }
  if (s->bp_on && s->bp_m + (int64_t)nsteps > s->p.bp_steps) {
    set_error("back-propagation window: %d steps recorded, room for %d", s->bp_m, s->p.bp_steps);
    return AFQMC_ENOSPC;
  }
  const int blk = s->graph_block;
  while (nsteps > 0) {
    // whole blocks that start on a block boundary replay the captured graph;
    // the rest (and every step while profiling) launches kernels one by one
    if (s->p.use_graph && blk > 0 && s->h_step % blk == 0 && nsteps >= blk && !s->prof.on &&
        !s->bp_on) {
      AFQ_TRY(join_side(s));  // the graph starts from a joined stream
      s->t_fresh = false;  // the block recomputes the force-bias traces itself
      if (!s->graph) {
        const int64_t l0 = g_launches;
        const int64_t h0 = s->h_step;
        AFQ_CUDA(cudaStreamBeginCapture(s->st, cudaStreamCaptureModeThreadLocal));
        int r = AFQMC_OK;
        for (int i = 0; i < blk && r == AFQMC_OK; ++i) r = step_once(s);
        if (r == AFQMC_OK) r = join_side(s);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(s->st, &g);
        s->h_step = h0;  // nothing ran yet: the launch below takes the steps
        if (r != AFQMC_OK) {
          if (g) cudaGraphDestroy(g);
          return r;
        }
        if (e != cudaSuccess) {
          set_error("graph capture failed: %s", cudaGetErrorString(e));
          return AFQMC_ECUDA;
        }
        e = cudaGraphInstantiate(&s->graph, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) {
          s->graph = nullptr;
          set_error("graph instantiation failed: %s", cudaGetErrorString(e));
          return AFQMC_ECUDA;
        }
        s->graph_kernels = g_launches - l0;
        g_launches = l0;
      }
      AFQ_CUDA(cudaGraphLaunch(s->graph, s->st));
      g_launches += s->graph_kernels;
      s->h_step += blk;
      // the block ends with an energy evaluation iff the energy period divides blk
      s->t_fresh = s->p.energy_period > 0 && blk % s->p.energy_period == 0;
      nsteps -= blk;
    } else {
      AFQ_TRY(step_once(s));
      --nsteps;
    }
  }
  return join_side(s);
}

int afqmc_energy(afqmc_state* s, double* E, double* wsum) {
  AFQ_STATE(s);
  AFQ_TRY(energy_eval(s, false));
  double last[8];
  AFQ_CUDA(cudaMemcpyAsync(last, s->b.last, sizeof(last), cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  if (E) *E = last[4];
  if (wsum) *wsum = last[1];
  return AFQMC_OK;
}

int afqmc_local_energies(afqmc_state* s, double* eloc) {
  AFQ_STATE(s);
  if (!eloc) {
    set_error("eloc is NULL");
    return AFQMC_EINVAL;
  }
  AFQ_TRY(energy_eval(s, false));
  AFQ_CUDA(cudaMemcpyAsync(eloc, s->b.eloc, sizeof(double) * 2 * s->p.nwalkers,
                           cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  return AFQMC_OK;
}

int afqmc_bp_begin(afqmc_state* s) {
  AFQ_STATE(s);
  if (s->p.bp_steps <= 0) {
    set_error("afqmc_bp_begin: the state has no back-propagation buffers (bp_steps = 0)");
    return AFQMC_EINVAL;
  }
  if (s->bp_on) {
    set_error("afqmc_bp_begin: a window is already open");
    return AFQMC_ESTATE;
  }
  return bp_open(s);
}

int afqmc_bp_end(afqmc_state* s, double* rho, double* rho_phl, double* wsums, int32_t* nsteps) {
  AFQ_STATE(s);
  if (!s->bp_on) {
    set_error("afqmc_bp_end: no open window");
    return AFQMC_ESTATE;
  }
  if (!rho) {
    set_error("afqmc_bp_end: rho is NULL");
    return AFQMC_EINVAL;
  }
  const int m = s->bp_m;
  AFQ_TRY(bp_close(s));
  const size_t MM = (size_t)s->p.M * s->p.M;
  const Bufs& b = s->b;
  AFQ_CUDA(cudaMemcpyAsync(rho, b.bp_out, 2 * MM * sizeof(double), cudaMemcpyDeviceToHost, s->st));
  if (rho_phl)
    AFQ_CUDA(cudaMemcpyAsync(rho_phl, b.bp_out + 2 * MM, 2 * MM * sizeof(double),
                             cudaMemcpyDeviceToHost, s->st));
  if (wsums)
    AFQ_CUDA(cudaMemcpyAsync(wsums, b.bp_out + 4 * MM, 4 * sizeof(double),
                             cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  if (nsteps) *nsteps = m;
  return AFQMC_OK;
}

int afqmc_get_walkers(afqmc_state* s, double* phi, double* weight, double* logov) {
  AFQ_STATE(s);
  const afqmc_params& p = s->p;
  const size_t W = p.nwalkers, N = p.N, M = p.M;
  if (phi) {
    // back to the caller's basis: Phi^T = Phi'^T Q^T
    GemmF64 g;
    g.m = (int)(W * 2 * N);
    g.n = g.k = (int)M;
    g.A = s->b.phiT;
    g.lda = (long)M;
    g.B = s->b.Qb;
    g.ldb = (long)M;
    g.C = s->b.T0;
    g.ldc = (long)M;
    AFQ_TRY(gemm_nt_f64(g, s->st));
    std::vector<double> h(W * 2 * N * M);
    AFQ_CUDA(cudaMemcpyAsync(h.data(), s->b.T0, sizeof(double) * h.size(),
                             cudaMemcpyDeviceToHost, s->st));
    AFQ_CUDA(cudaStreamSynchronize(s->st));
    for (size_t w = 0; w < W; ++w)
      for (size_t c = 0; c < 2; ++c)
        for (size_t i = 0; i < N; ++i)
          for (size_t q = 0; q < M; ++q)
            phi[((w * M + q) * N + i) * 2 + c] = h[((w * 2 + c) * N + i) * M + q];
  }
  if (weight)
    AFQ_CUDA(cudaMemcpyAsync(weight, s->b.wt, sizeof(double) * 2 * W, cudaMemcpyDeviceToHost, s->st));
  if (logov)
    AFQ_CUDA(cudaMemcpyAsync(logov, s->b.ld, sizeof(double) * 2 * W, cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  return AFQMC_OK;
}

int afqmc_set_walkers(afqmc_state* s, const double* phi, const double* weight) {
  AFQ_STATE(s);
  if (!phi || !weight) {
    set_error("phi and weight are required");
    return AFQMC_EINVAL;
  }
  const afqmc_params& p = s->p;
  const size_t W = p.nwalkers, N = p.N, M = p.M;
  AFQ_TRY(all_finite(phi, W * M * N * 2, "phi"));
  AFQ_TRY(all_finite(weight, W * 2, "weight"));
  std::vector<double> h(W * 2 * N * M);
  for (size_t w = 0; w < W; ++w)
    for (size_t c = 0; c < 2; ++c)
      for (size_t i = 0; i < N; ++i)
        for (size_t q = 0; q < M; ++q)
          h[((w * 2 + c) * N + i) * M + q] = phi[((w * M + q) * N + i) * 2 + c];
  AFQ_CUDA(cudaMemcpyAsync(s->b.T0, h.data(), sizeof(double) * h.size(), cudaMemcpyHostToDevice, s->st));
  // into the trial-adapted basis: Phi'^T = Phi^T Q
  GemmF64 g;
  g.m = (int)(W * 2 * N);
  g.n = g.k = (int)M;
  g.A = s->b.T0;
  g.lda = (long)M;
  g.B = s->b.QTb;
  g.ldb = (long)M;
  g.C = s->b.phiT;
  g.ldc = (long)M;
  AFQ_TRY(gemm_nt_f64(g, s->st));
  AFQ_TRY(refresh_phi_lo(s));
  AFQ_CUDA(cudaMemcpyAsync(s->b.wt, weight, sizeof(double) * 2 * W, cudaMemcpyHostToDevice, s->st));
  AFQ_TRY(overlap_update(s, true, false));
  s->t_fresh = false;
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  return AFQMC_OK;
}

int afqmc_get_energy_log(afqmc_state* s, double* rec, int32_t cap, int32_t* n) {
  AFQ_STATE(s);
  if (!n || (cap > 0 && !rec) || cap < 0) {
    set_error("bad arguments");
    return AFQMC_EINVAL;
  }
  unsigned long long count = 0;
  AFQ_CUDA(cudaMemcpyAsync(&count, s->b.counters + CTR_RECORDS, sizeof(count),
                           cudaMemcpyDeviceToHost, s->st));
  std::vector<double> all(4 * (size_t)s->p.max_records);
  AFQ_CUDA(cudaMemcpyAsync(all.data(), s->b.records, sizeof(double) * all.size(),
                           cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  const unsigned long long R = (unsigned long long)s->p.max_records;
  const unsigned long long have = count < R ? count : R;
  const unsigned long long first = count - have;
  const unsigned long long ncopy = have < (unsigned long long)cap ? have : (unsigned long long)cap;
  for (unsigned long long i = 0; i < ncopy; ++i) {
    const unsigned long long slot = (first + i) % R;
    std::memcpy(rec + 4 * i, all.data() + 4 * slot, 4 * sizeof(double));
  }
  *n = (int32_t)ncopy;
  return AFQMC_OK;
}

int afqmc_get_info(afqmc_state* s, afqmc_info* info) {
  AFQ_STATE(s);
  if (!info) {
    set_error("info is NULL");
    return AFQMC_EINVAL;
  }
  unsigned long long ctr[8];
  std::vector<double> wt(2 * (size_t)s->p.nwalkers);
  AFQ_CUDA(cudaMemcpyAsync(ctr, s->b.counters, sizeof(ctr), cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaMemcpyAsync(wt.data(), s->b.wt, sizeof(double) * wt.size(), cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  info->E_T = s->E_T;
  info->H0p = s->H0p;
  info->e_shift = s->e_shift;
  info->wmax = s->wmax;
  info->step = (int64_t)ctr[CTR_STEP];
  info->nonfinite = (int64_t)ctr[CTR_NONFINITE];
  info->launches = g_launches;
  int alive = 0;
  for (int w = 0; w < s->p.nwalkers; ++w) alive += (wt[2 * w] != 0.0 || wt[2 * w + 1] != 0.0);
  info->alive = alive;
  info->status = (int32_t)ctr[CTR_STATUS];
  return AFQMC_OK;
}

namespace {
struct CkptHeader {
  uint64_t magic;
  int32_t M, N, nchol, nwalkers;
  int64_t step;
  uint64_t records, nonfinite;
  uint64_t seed;
  int32_t max_records, nup;  // nup: spin-up columns of a two-block walker, 0 closed shell
};
constexpr uint64_t kMagic = 0x31434D5146414731ull;
}  // namespace

int afqmc_save(afqmc_state* s, void* buf, size_t* bytes) {
  AFQ_STATE(s);
  if (!bytes) {
    set_error("bytes is NULL");
    return AFQMC_EINVAL;
  }
  const afqmc_params& p = s->p;
  const size_t nw = (size_t)p.nwalkers * 2 * p.N * p.M;
  const size_t need = sizeof(CkptHeader) +
                      sizeof(double) * (2 * nw + 4 * (size_t)p.nwalkers + 4 * (size_t)p.max_records);
  if (!buf) {
    *bytes = need;
    return AFQMC_OK;
  }
  if (*bytes < need) {
    set_error("checkpoint buffer %zu < %zu", *bytes, need);
    return AFQMC_ENOSPC;
  }
  unsigned long long ctr[8];
  AFQ_CUDA(cudaMemcpyAsync(ctr, s->b.counters, sizeof(ctr), cudaMemcpyDeviceToHost, s->st));
  char* o = static_cast<char*>(buf) + sizeof(CkptHeader);
  double* d = reinterpret_cast<double*>(o);
  AFQ_CUDA(cudaMemcpyAsync(d, s->b.phiT, sizeof(double) * nw, cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaMemcpyAsync(d + nw, s->b.thetaT, sizeof(double) * nw, cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaMemcpyAsync(d + 2 * nw, s->b.wt, sizeof(double) * 2 * p.nwalkers, cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaMemcpyAsync(d + 2 * nw + 2 * p.nwalkers, s->b.ld, sizeof(double) * 2 * p.nwalkers,
                           cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaMemcpyAsync(d + 2 * nw + 4 * p.nwalkers, s->b.records,
                           sizeof(double) * 4 * p.max_records, cudaMemcpyDeviceToHost, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  CkptHeader h{kMagic, p.M, p.N, p.nchol, p.nwalkers, s->h_step, ctr[CTR_RECORDS],
               ctr[CTR_NONFINITE], p.seed, p.max_records, s->spin2 ? s->nup : 0};
  std::memcpy(buf, &h, sizeof(h));
  *bytes = need;
  return AFQMC_OK;
}

int afqmc_load(afqmc_state* s, const void* buf, size_t bytes) {
  AFQ_STATE(s);
  const afqmc_params& p = s->p;
  if (!buf || bytes < sizeof(CkptHeader)) {
    set_error("checkpoint too small");
    return AFQMC_EINVAL;
  }
  CkptHeader h;
  std::memcpy(&h, buf, sizeof(h));
  const size_t nw = (size_t)p.nwalkers * 2 * p.N * p.M;
  const size_t need = sizeof(CkptHeader) +
                      sizeof(double) * (2 * nw + 4 * (size_t)p.nwalkers + 4 * (size_t)p.max_records);
  if (h.magic != kMagic || h.M != p.M || h.N != p.N || h.nchol != p.nchol ||
      h.nwalkers != p.nwalkers || h.max_records != p.max_records || h.seed != p.seed ||
      h.nup != (s->spin2 ? s->nup : 0) || bytes < need) {
    set_error("checkpoint does not match this state");
    return AFQMC_EINVAL;
  }
  const double* d = reinterpret_cast<const double*>(static_cast<const char*>(buf) + sizeof(CkptHeader));
  AFQ_CUDA(cudaMemcpyAsync(s->b.phiT, d, sizeof(double) * nw, cudaMemcpyHostToDevice, s->st));
  AFQ_TRY(refresh_phi_lo(s));
  AFQ_CUDA(cudaMemcpyAsync(s->b.thetaT, d + nw, sizeof(double) * nw, cudaMemcpyHostToDevice, s->st));
  AFQ_TRY(refresh_theta_lo(s));
  AFQ_CUDA(cudaMemcpyAsync(s->b.wt, d + 2 * nw, sizeof(double) * 2 * p.nwalkers, cudaMemcpyHostToDevice, s->st));
  AFQ_CUDA(cudaMemcpyAsync(s->b.ld, d + 2 * nw + 2 * p.nwalkers, sizeof(double) * 2 * p.nwalkers,
                           cudaMemcpyHostToDevice, s->st));
  AFQ_CUDA(cudaMemcpyAsync(s->b.records, d + 2 * nw + 4 * p.nwalkers, sizeof(double) * 4 * p.max_records,
                           cudaMemcpyHostToDevice, s->st));
  unsigned long long ctr[8] = {0};
  ctr[CTR_STEP] = (unsigned long long)h.step;
  ctr[CTR_RECORDS] = h.records;
  ctr[CTR_NONFINITE] = h.nonfinite;
  AFQ_CUDA(cudaMemcpyAsync(s->b.counters, ctr, sizeof(ctr), cudaMemcpyHostToDevice, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  s->h_step = h.step;
  s->t_fresh = false;
  return AFQMC_OK;
}

int afqmc_destroy(afqmc_state* s) {
  if (!s) return AFQMC_OK;
  s->valid = false;
  if (s->graph) cudaGraphExecDestroy(s->graph);
  if (s->side) {
    cudaStreamSynchronize(s->side);
    cudaStreamDestroy(s->side);
  }
  if (s->ev_fork) cudaEventDestroy(s->ev_fork);
  if (s->ev_side) cudaEventDestroy(s->ev_side);
  for (cudaEvent_t e : s->prof.ev) cudaEventDestroy(e);
  delete s;
  return AFQMC_OK;
}

const char* afqmc_last_error(void) { return g_err; }

int64_t afqmc_launch_count(void) { return g_launches; }

}  // extern "C"

namespace afq {
int launch_philox(uint64_t key, const uint32_t* ctr, long n, uint32_t* out, cudaStream_t st);
int launch_wait_flag(const int* flag, long long max_polls, int* status, cudaStream_t st);
int launch_fields(uint64_t seed, uint32_t step, int w0, int nw, int G, double* out,
                  cudaStream_t st);
int launch_round_f32(const double* src, float* dst, long n, cudaStream_t st);
int launch_widen_f32(const float* src, double* dst, long n, cudaStream_t st);
}  // namespace afq

extern "C" {
int afqmc_wait_flag(const int* d_flag, int64_t max_polls, int* d_status, void* stream) {
  if (!d_flag || !d_status || max_polls < 0 || max_polls > (1ll << 32)) {
    afq::set_error("bad arguments");
    return AFQMC_EINVAL;
  }
  return afq::launch_wait_flag(d_flag, (long long)max_polls, d_status,
                               static_cast<cudaStream_t>(stream));
}

int afqmc_philox4x32_10(uint64_t key, const uint32_t* d_ctr, int64_t n, uint32_t* d_out,
                        void* stream) {
  if (n < 0 || (n > 0 && (!d_ctr || !d_out))) {
    afq::set_error("bad arguments");
    return AFQMC_EINVAL;
  }
  return afq::launch_philox(key, d_ctr, (long)n, d_out, static_cast<cudaStream_t>(stream));
}

int afqmc_round_f32(const double* d_in, float* d_out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!d_in || !d_out))) {
    afq::set_error("bad arguments");
    return AFQMC_EINVAL;
  }
  return afq::launch_round_f32(d_in, d_out, (long)n, static_cast<cudaStream_t>(stream));
}

int afqmc_widen_f32(const float* d_in, double* d_out, int64_t n, void* stream) {
  if (n < 0 || (n > 0 && (!d_in || !d_out))) {
    afq::set_error("bad arguments");
    return AFQMC_EINVAL;
  }
  return afq::launch_widen_f32(d_in, d_out, (long)n, static_cast<cudaStream_t>(stream));
}

int afqmc_gaussian_fields(uint64_t seed, int64_t step, int32_t w0, int32_t nw, int32_t nchol,
                          double* d_out, void* stream) {
  if (step < 0 || step > 0xFFFFFFFFll || w0 < 0 || nw < 0 || nchol < 1 || (nw > 0 && !d_out)) {
    afq::set_error("bad arguments");
    return AFQMC_EINVAL;
  }
  return afq::launch_fields(seed, (uint32_t)step, w0, nw, nchol, d_out,
                            static_cast<cudaStream_t>(stream));
}
}  // extern "C"

extern "C" {
int afqmc_profile_start(afqmc_state* s, int32_t max_steps) {
  AFQ_STATE(s);
  if (max_steps < 1) {
    afq::set_error("max_steps must be positive");
    return AFQMC_EINVAL;
  }
  afq::Profiler& P = s->prof;
  for (cudaEvent_t e : P.ev) cudaEventDestroy(e);
  P = afq::Profiler();
  const int pairs = max_steps * (AFQMC_NPHASE + 2);
  P.ev.resize(2 * (size_t)pairs);
  for (auto& e : P.ev) AFQ_CUDA(cudaEventCreate(&e));
  P.phase.assign(pairs, -1);
  P.kern.assign(pairs, 0);
  P.max_events = pairs;
  P.on = true;
  return AFQMC_OK;
}

int afqmc_profile_stop(afqmc_state* s, double* ms, int64_t* count, int64_t* kernels) {
  AFQ_STATE(s);
  afq::Profiler& P = s->prof;
  if (!P.on) {
    afq::set_error("profiling was not started");
    return AFQMC_ESTATE;
  }
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  for (int i = 0; i < AFQMC_NPHASE; ++i) {
    if (ms) ms[i] = 0.0;
    if (count) count[i] = 0;
    if (kernels) kernels[i] = 0;
  }
  for (int i = 0; i < P.used; ++i) {
    float t = 0.f;
    AFQ_CUDA(cudaEventElapsedTime(&t, P.ev[2 * i], P.ev[2 * i + 1]));
    const int ph = P.phase[i];
    if (ms) ms[ph] += t;
    if (count) count[ph] += 1;
    if (kernels) kernels[ph] += P.kern[i];
  }
  for (cudaEvent_t e : P.ev) cudaEventDestroy(e);
  P = afq::Profiler();
  return AFQMC_OK;
}
}  // extern "C"
