/*
 * afqmc.h -- C ABI of the GB300 phaseless-AFQMC library (libafqmc.so).
 *
 * The library runs the per-walker imaginary-time step of phaseless
 * auxiliary-field quantum Monte Carlo for a closed-shell molecule with a
 * single-determinant (RHF) trial, after M. Motta and S. Zhang, "Ab initio
 * computations of molecular systems by the auxiliary-field quantum Monte
 * Carlo method" (2017):
 *   force bias            Sec. 3.2, Eq. fb; Sec. 3.4.2, Eq. precomputing2
 *   auxiliary fields      Sec. 2.2, Eqs. hs / hs2 (Gaussian p(x))
 *   propagation           Eq. primitive (Trotter split), Sec. 3.4.2
 *                         (A(x), truncated Taylor series), Theorem 1.4
 *   mean-field background Sec. 2.4
 *   weights               Eq. hybrid-wt, Eq. if_rle, Eq. weight_update_2
 *   local energy          Eqs. localenergy, localenergy2, localenergy3
 *   stabilisation         Sec. 3.4.5 (modified Gram-Schmidt), Theorem 1.5
 *   population control    Sec. 3.4.4 (a fixed-size comb)
 *   rare-event caps       Appendix B, Eq. cap
 *
 * Conventions shared by every entry point:
 *   - Return value: AFQMC_OK (0) or a negative afqmc_status.  Nothing aborts,
 *     traps or exits; afqmc_last_error() gives a message for the calling
 *     thread's last failure.
 *   - Host arrays are row-major float64 ("C order") unless stated.  They are
 *     read (and copied) during the call; the caller keeps ownership.
 *   - Device memory is owned by the caller: the library never allocates
 *     device memory.  afqmc_workspace_size() says how many bytes one state
 *     needs; the caller passes a buffer of at least that size (256-byte
 *     aligned) to afqmc_init() and keeps it alive until afqmc_destroy().
 *   - Every kernel of a state runs on the CUDA stream given to afqmc_init()
 *     (a cudaStream_t passed as void*, NULL = legacy default stream).
 *     Calls that return results to the host synchronise that stream.
 *   - One host thread at a time per state.  Different states are
 *     independent.
 *   - Spin: by default the walkers are restricted closed shell
 *     (N_up = N_dn = N); the up and down blocks of every walker are the same
 *     M x N matrix, because the trial is RHF and the propagator B(x) is spin
 *     independent (Sec. 2.3: v_g acts identically on both spins).  With
 *     params.Ndn >= 1 a walker has two spin blocks, N_up = N spin-up and
 *     N_dn = Ndn spin-down orbitals, stored as N + Ndn columns (spin up
 *     first) that B(x) propagates alike; overlaps (the product over spins of
 *     Theorem 1.1), Theta, the exchange and Gram-Schmidt are per block.
 */
#ifndef AFQMC_H
#define AFQMC_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define AFQMC_API __attribute__((visibility("default")))
#else
#define AFQMC_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum afqmc_status {
  AFQMC_OK = 0,
  AFQMC_EINVAL = -1,      /* bad argument, shape or parameter              */
  AFQMC_ENOSPC = -2,      /* workspace smaller than afqmc_workspace_size() */
  AFQMC_ENONFINITE = -3,  /* non-finite value in a host input              */
  AFQMC_ECUDA = -4,       /* a CUDA runtime call failed                    */
  AFQMC_ETIMEOUT = -5,    /* a bounded device-side wait gave up            */
  AFQMC_ESTATE = -6,      /* state not usable (destroyed, wrong phase)     */
  AFQMC_EUNSUPPORTED = -7 /* mode not built into this library              */
} afqmc_status;

/* Arithmetic of the step. */
enum {
  AFQMC_FP64 = 0,       /* every step in float64 / complex128                   */
  AFQMC_MIXED_TF32 = 1, /* contractions on tcgen05 tensor cores, TF32 inputs,   */
                        /* FP32 accumulation; the overlap S = V_T^T Phi, its    */
                        /* LU / inverse S^-1 and log det, the overlap ratios,   */
                        /* weights, Gram-Schmidt and the identity part of the   */
                        /* one-body half steps in FP64 (the rest, B_half - I,   */
                        /* as a high and a low operand part); the product       */
                        /* Theta = Phi S^-1 (an operand of the contractions)    */
                        /* in FP32 from the float64 S^-1                        */
  AFQMC_MIXED_BF16 = 2, /* as MIXED_TF32 with BF16 inputs to the contractions   */
  AFQMC_MIXED_TF32_F32LU = 3, /* as MIXED_TF32 with the elimination (S^-1) and  */
                              /* Gram-Schmidt also in FP32 (log det sums,       */
                              /* overlap ratios and weights stay FP64)          */
  AFQMC_MIXED_BF16_F32LU = 4, /* as MIXED_BF16, the same steps in FP32          */
  AFQMC_MIXED_TF32_F64THETA = 5, /* as MIXED_TF32 with Theta = Phi S^-1 also    */
                                 /* formed in float64                           */
  AFQMC_MIXED_BF16_F64THETA = 6  /* as MIXED_BF16 with Theta in float64         */
};

/* Walker update rule. */
enum {
  AFQMC_PHASELESS = 0, /* Eq. weight_update_2: hybrid weight, cos projection */
  AFQMC_FREE = 1       /* Eq. weight_update: free projection, complex weight */
};

typedef struct afqmc_params {
  int32_t M;             /* orbitals (orthonormal basis)                       */
  int32_t N;             /* spin-up electrons N_up (and N_dn when Ndn = 0),    */
                         /* 1 <= N <= M                                         */
  int32_t nchol;         /* Cholesky vectors N_gamma                           */
  int32_t nwalkers;      /* population size N_w                                */
  double dt;             /* imaginary time step, > 0                           */
  double e_shift;        /* energy shift E_0 in B(x); NaN -> trial energy E_T  */
  double H0;             /* constant (nuclear repulsion) of Eq. bo_ham2        */
  uint64_t seed;         /* Philox key of the auxiliary fields                 */
  int32_t taylor_order;  /* order n of the truncated exp(V) series (>= 1)      */
  int32_t qr_period;     /* steps between Gram-Schmidt passes (0 = never)      */
  int32_t pc_period;     /* steps between comb population controls (0 = off)   */
  int32_t energy_period; /* steps between energy measurements (0 = never)      */
  int32_t precision;     /* AFQMC_FP64, AFQMC_MIXED_* (the enum above)         */
  int32_t mode;          /* AFQMC_PHASELESS / AFQMC_FREE                       */
  double ecap_C;         /* local-energy cap constant C of Eq. cap; <= 0: off  */
  double fb_cap;         /* force-bias magnitude cap v_max; <= 0: off          */
  double wmax;           /* weight cap; NaN -> max(100, nwalkers / 10)         */
  int32_t max_records;   /* capacity of the device energy log (>= 1)           */
  int32_t use_graph;     /* 1: afqmc_propagate captures one block of steps      */
                         /* (the least common multiple of the non-zero periods) */
                         /* as a CUDA graph and replays it; 0: launches kernels */
                         /* one by one.  Results are identical either way.     */
                         /* 1 needs a stream created by the caller (the legacy */
                         /* default stream cannot be captured): else EINVAL.   */
  int32_t bp_steps;      /* capacity (steps) of a back-propagation window,      */
                         /* afqmc_bp_begin / afqmc_bp_end; 0: none              */
  int32_t ndet;          /* determinants of a multi-determinant trial          */
                         /* (afqmc_init_multidet); 0: the single RHF trial of  */
                         /* afqmc_init                                          */
  int32_t Ndn;           /* 0: restricted closed shell (one spin block, the    */
                         /* spin-down orbitals are the spin-up ones, N_dn = N); */
                         /* >= 1: two spin blocks, N_dn = Ndn spin-down         */
                         /* electrons with their own trial orbitals (float64,   */
                         /* N + Ndn <= 64; see afqmc_init)                      */
  int32_t walker0;       /* global index of this state's first walker: walker  */
                         /* w draws the fields of walker walker0 + w (one      */
                         /* population sharded over several states, see        */
                         /* afqmc_comb_plan); 0 for a state on its own         */
} afqmc_params;

/* Fill *p with the defaults: dt 0.005, e_shift NaN, H0 0, seed 1,
 * taylor_order 6, qr_period 5, pc_period 0, energy_period 1, FP64,
 * phaseless, ecap_C 2, fb_cap 1, wmax NaN, max_records 4096, use_graph 0, bp_steps 0,
 * ndet 0, Ndn 0 (closed shell), walker0 0.  The sizes
 * (M, N, nchol, nwalkers) are set to 0 and must be filled in. */
AFQMC_API void afqmc_default_params(afqmc_params* p);

/* Bytes of device workspace one state needs for *p (sizes and precision). */
AFQMC_API int afqmc_workspace_size(const afqmc_params* p, size_t* bytes);

typedef struct afqmc_state afqmc_state; /* opaque */

/*
 * Create a state and run the once-per-run set-up on the device:
 *   h1     [M][M]         one-body matrix h_pq (Eq. bo_ham_matel), symmetric
 *   L      [nchol][M][M]  Cholesky vectors, v_pqrs = sum_g L[g]_pr L[g]_qs
 *                         (Sec. 2.3, Eq. chol), each L[g] symmetric
 *   trial_up [M][N]       occupied orbitals V_T of the trial, orthonormal
 *                         columns (Sec. 3.4.1): the RHF orbitals of both
 *                         spins when params.Ndn = 0, else the spin-up ones
 *   trial_dn [M][Ndn]     spin-down orbitals, orthonormal columns, when
 *                         params.Ndn >= 1 (two spin blocks); NULL when
 *                         params.Ndn = 0
 * all host, row-major float64.  The set-up computes, on the GPU,
 * c_g = Tr(L_g P) with P = sum_sigma V_sigma V_sigma^T (the mean-field
 * background vbar_g = i c_g, Sec. 2.4), v0' = h - 1/2 sum_g L_g^2 +
 * sum_g c_g L_g, H0' = H0 - 1/2 sum_g c_g^2, B_half = exp(-dt v0'/2), the
 * half-rotated vectors V_sigma^T L_g and V_sigma^T h (Eq. precomputing2) and
 * the trial energy E_T, and puts every walker at {V_T, W = 1, theta = 0}
 * (algorithm outline, step 1).  Two spin blocks run on the float64 path
 * only, without back-propagation (else AFQMC_EUNSUPPORTED).
 * d_workspace: device buffer of ws_bytes >= afqmc_workspace_size(p).
 * stream: cudaStream_t (as void*) on which every kernel of the state runs.
 * Synchronises the stream.  On failure *out is NULL.  A NaN or infinity in
 * h1, the trial or L gives AFQMC_ENONFINITE, with the first such index in
 * afqmc_last_error() (L is checked on the device right after its upload).
 * On the mixed precisions (single determinant) the rotation of L to the
 * trial's basis and sum_g L_g^2 use FP32 products (they feed the BF16/TF32
 * operands and B_half, applied as BF16/TF32 parts); V_sigma^T L_g, c_g and
 * H0' stay float64.
 */
AFQMC_API int afqmc_init(const afqmc_params* p, const double* h1, const double* L,
                         const double* trial_up, const double* trial_dn, void* d_workspace,
                         size_t ws_bytes, void* stream, afqmc_state** out);

/*
 * The same with a multi-determinant trial Psi_T = sum_d A_d Psi_d (Sec. 3.4,
 * Eqs. usesherman, precomputing2, localenergy2/3), p->ndet = ndet >= 1:
 *   coef      [ndet][2]     A_d (real, imaginary)
 *   trial_up  [ndet][M][N]  spin-up orbitals of each determinant, and
 *   trial_dn  [ndet][M][N]  spin-down orbitals, orthonormal columns each
 * all host, row-major float64.  Walkers stay closed shell (both spin blocks
 * the same orbitals; the propagator keeps them so) and start at the leading
 * spin-up orbitals trial_up[0]; the overlap is
 * sum_d A_d^* det(V_du^T Phi) det(V_dd^T Phi), the force bias and the local
 * energy are the determinant-weighted sums of Eqs. precomputing2 and
 * localenergy3; the mean-field background comes from determinant 0,
 * c_g = Tr(L_g (P_0u + P_0d)), and E_T is the local energy of the initial
 * walkers.  When ndet >= 2, N <= 32 and every determinant differs from
 * determinant 0 in at most 4 columns per spin (the other columns equal, in
 * the same positions: a CI expansion about determinant 0), the determinants
 * are evaluated relative to determinant 0 by low-rank updates (the
 * Sherman-Morrison-Woodbury remark of Sec. 3.4) in float64 on either
 * precision; that form stays finite where a determinant's overlap with a
 * walker vanishes.  Otherwise each determinant is evaluated in full, the
 * mixed paths running its force-bias traces and exchange on the tensor
 * cores (BF16/TF32 operands) with overlaps, weights and their combinations
 * in float64; a determinant orthogonal to a walker then gets weight 0.
 * Phaseless, population control off, no back-propagation window (else
 * AFQMC_EUNSUPPORTED).  Everything else as afqmc_init.
 */
AFQMC_API int afqmc_init_multidet(const afqmc_params* p, const double* h1, const double* L,
                                  int32_t ndet, const double* coef, const double* trial_up,
                                  const double* trial_dn, void* d_workspace, size_t ws_bytes,
                                  void* stream, afqmc_state** out);

/*
 * Enqueue nsteps steps of the random walk (algorithm outline, steps 2-9):
 * per step and walker with W != 0: force bias, fields, propagation
 * B_half T_n(V) B_half, new overlap / Theta, weight update (phaseless or
 * free); then every qr_period steps modified Gram-Schmidt, every pc_period
 * steps the comb, every energy_period steps one energy record (local
 * energies and the mixed estimator, Eq. localenergy).  Asynchronous: returns
 * once the work is enqueued on the state's stream.
 */
AFQMC_API int afqmc_propagate(afqmc_state* s, int32_t nsteps);

/*
 * Mixed estimator of the energy at the current walkers, Eq. localenergy:
 * *E = sum_w W_w Re E_loc,w / sum_w W_w (phaseless; E_loc capped by Eq. cap)
 * or Re(sum W e^{i theta} E_loc / sum W e^{i theta}) (free projection),
 * *wsum = sum_w W_w (real part).  Synchronises the stream.
 */
AFQMC_API int afqmc_energy(afqmc_state* s, double* E, double* wsum);

/*
 * Local energies of all walkers (Eqs. localenergy2/3), uncapped:
 * eloc [nwalkers][2] host (re, im).  Synchronises the stream.
 */
AFQMC_API int afqmc_local_energies(afqmc_state* s, double* eloc);

/*
 * Copy walkers to the host: phi [nwalkers][M][Nt][2] (re, im, row-major
 * orbital coefficients; Nt = N, or N + Ndn with two spin blocks, spin-up
 * columns first), weight [nwalkers][2] (real and imaginary part of the
 * walker weight W e^{i theta}; theta = 0 for phaseless walks), logov
 * [nwalkers][2] (log <Psi_T|Psi> = 2 log det(V_T^T phi) for both spins, or
 * the sum over the two blocks' log det: real part and phase in (-pi, pi]).
 * Any pointer may be NULL.
 * Synchronises the stream.
 */
AFQMC_API int afqmc_get_walkers(afqmc_state* s, double* phi, double* weight, double* logov);

/*
 * Replace the walkers from host arrays laid out as in afqmc_get_walkers
 * (phi and weight required).  Overlaps and Theta are recomputed on the
 * device.  Synchronises the stream.
 */
AFQMC_API int afqmc_set_walkers(afqmc_state* s, const double* phi, const double* weight);

/*
 * Energy log: up to max_records records (step, mixed estimate E, Re sum W,
 * live walkers) written by afqmc_propagate every energy_period steps, oldest
 * first, to rec [cap][4] host.  *n receives the number of records copied;
 * the log keeps the newest max_records.  Synchronises the stream.
 */
AFQMC_API int afqmc_get_energy_log(afqmc_state* s, double* rec, int32_t cap, int32_t* n);

typedef struct afqmc_info {
  double E_T;            /* trial energy <Psi_T|H|Psi_T>                       */
  double H0p;            /* H0' after the mean-field shift                     */
  double e_shift;        /* shift used in B(x)                                 */
  double wmax;           /* weight cap in use                                  */
  int64_t step;          /* steps taken                                        */
  int64_t nonfinite;     /* walkers zeroed for a non-finite weight             */
  int64_t launches;      /* kernels this state has launched                    */
  int32_t alive;         /* walkers with W != 0 (at the last sync)             */
  int32_t status;        /* sticky device status (afqmc_status)                */
} afqmc_info;

/* State summary; synchronises the stream. */
AFQMC_API int afqmc_get_info(afqmc_state* s, afqmc_info* info);

/*
 * Checkpoint: serialise walkers, weights, overlaps, the step counter and the
 * energy log into host memory.  With buf == NULL, *bytes receives the size
 * needed; otherwise *bytes must be at least that.  The fields are keyed by
 * (seed, step, walker, gamma), so a state restored with afqmc_load() into a
 * state created with the same inputs continues bit-identically.
 */
AFQMC_API int afqmc_save(afqmc_state* s, void* buf, size_t* bytes);
AFQMC_API int afqmc_load(afqmc_state* s, const void* buf, size_t bytes);

/*
 * Groups: many independent runs (different molecules and sizes, each its own
 * state, workspace and stream) advanced together.  Walkers of different
 * states never interact (Sec. 3.5: walkers are independent), so the group's
 * block of steps - one graph block of every state, the least common multiple
 * of its periods - is captured once as ONE CUDA graph whose branches are the
 * states' streams (fork/join on `stream`), and afqmc_group_propagate replays
 * it with one launch per block.  All states need use_graph = 1 and the same
 * graph block length, must be on the current device, and must stay valid
 * while the group exists.  Each state's results are bit-identical to
 * stepping it alone.
 *
 * When every state runs the same mixed precision with the same periods
 * (single-determinant, closed shell, no back-propagation window), the block
 * is captured step by step instead: each of the step's four tensor-core
 * contractions (force bias, V, the two half steps) of ALL states is one
 * persistent launch over a work list of (state, output tile), each state's
 * operands addressed through its own tensor maps in a small device table the
 * group allocates; the per-state kernels between them run on the states'
 * streams.  The tile widths of the force-bias and half-step launches are
 * chosen when the grouped launches are set up, by timing the candidates on
 * the states' own buffers (outputs that are scratch at that point).  By
 * default the group replays its first four blocks two each way, times the
 * second block of each (synchronising the stream then) and keeps the faster
 * capture.  Results stay bit-identical to stepping each state alone either
 * way.
 */
typedef struct afqmc_group afqmc_group; /* opaque */
AFQMC_API int afqmc_group_create(afqmc_state* const* states, int32_t n, void* stream,
                                 afqmc_group** out);
/* nsteps must be a multiple of the block length and every state must sit on
 * a block boundary.  Asynchronous on `stream` (which joins all branches). */
AFQMC_API int afqmc_group_propagate(afqmc_group* g, int32_t nsteps);
/* mode 0: capture each state's own kernel sequence; 1: the grouped
 * contractions where the states allow; 2 (default): choose between the two
 * by timing (restarts the trial).  Takes effect on the next block. */
AFQMC_API int afqmc_group_set_grouped(afqmc_group* g, int32_t mode);
/* 1 when the grouped contractions are in use (after a propagate), else 0;
 * bn[4] receives their tile widths (force bias, V, first and last half step;
 * 0 when not grouped).  Negative on bad arguments. */
AFQMC_API int afqmc_group_tiles(const afqmc_group* g, int32_t* bn);
AFQMC_API int afqmc_group_destroy(afqmc_group* g);

/*
 * One population sharded over several states (typically one per GPU, each in
 * its own process).  Walkers are independent between population controls
 * (Sec. 3.5), so each state steps its own n_s walkers, created with
 * params.walker0 = the global index of its first walker (the fields are keyed
 * by the global index), the same seed, and pc_period = 0; every p steps a
 * host driver runs the comb of Sec. 3.4.4 over the whole population:
 *   1. afqmc_export_weights: the state's n_s real weights into d_weights
 *      (DEVICE float64 [n_s]); the driver gathers every state's weights, in
 *      global walker order, into d_weights_all [n_all] on every state's device;
 *   2. afqmc_comb_plan: on every state the same parents for all n_all new
 *      slots, d_parent_all [n_all] (DEVICE int32 global walker indices; all -1
 *      if no weight is left), with the single-state comb's arithmetic:
 *      sequential float64 cumulative weights (d_cum [n_all], DEVICE scratch),
 *      u from the Philox counter (0, 0xffffffff, step - 1, 0) of the seed,
 *      tooth k = ((k + u) W_tot) / n_all, copies in walker order; W_tot is kept
 *      in the state;
 *   3. afqmc_pack_walkers / afqmc_unpack_walkers: the driver moves the
 *      parents' rows (afqmc_walker_row_bytes each: Phi, Theta and the log
 *      overlap in float64) to the states owning the new slots; unpack writes
 *      them into its slots, sets their weight to W_tot / n_all and refreshes
 *      the mixed path's operand copies.  Every slot of every state must be
 *      written (rows of parents on the same state included), so a state's
 *      own rows are packed before any unpack.
 * With one state holding the whole population this reproduces the
 * state's own comb (pc_period > 0) exactly.  afqmc_energy_sums copies the
 * last estimator evaluation's sums (sum W Re E_loc, sum W, sum W Im E_loc /
 * the imaginary parts for free projection, as afqmc_energy leaves them) to
 * d_sums (DEVICE float64 [4]) for a reduction over states.  All calls are
 * asynchronous on the state's stream; buffers are caller-owned.  Phaseless,
 * single-determinant, no open back-propagation window (else
 * AFQMC_EUNSUPPORTED).
 */
AFQMC_API int afqmc_walker_row_bytes(afqmc_state* s, size_t* bytes);
AFQMC_API int afqmc_export_weights(afqmc_state* s, double* d_weights);
AFQMC_API int afqmc_comb_plan(afqmc_state* s, const double* d_weights_all, int64_t n_all,
                              double* d_cum, int32_t* d_parent_all);
AFQMC_API int afqmc_pack_walkers(afqmc_state* s, const int32_t* d_index, int32_t n,
                                 void* d_rows);
AFQMC_API int afqmc_unpack_walkers(afqmc_state* s, const int32_t* d_slot, int32_t n,
                                   const void* d_rows);
AFQMC_API int afqmc_energy_sums(afqmc_state* s, double* d_sums);

/* Release the host side of a state (the workspace stays the caller's). */
AFQMC_API int afqmc_destroy(afqmc_state* s);

/*
 * Phases of a step, for afqmc_profile_stop():
 *   FORCE_BIAS  t_g = 2 Tr(Lh_g Theta) contraction (Eq. precomputing2)
 *   FIELDS      Philox fields, force bias and its cap, x = xi - xbar
 *   V           sum_g x_g L_g contraction (A(x) of Sec. 3.4.2)
 *   BHALF       the two exp(-dt v0'/2) products (Eq. primitive)
 *   TAYLOR      the truncated exp(V) series
 *   OVERLAP     S = V_T^T Phi, its inverse and log det (Theorem 1.1)
 *   WEIGHT      overlap ratio, phaseless / free weight update
 *   QR          modified Gram-Schmidt (and the log det update it implies)
 *   COMB        population control
 *   ENERGY      local energies (exchange contraction) and the estimator
 *   THETA       Theta = Phi S^-1 (Eq. precomputing), after OVERLAP
 */
enum {
  AFQMC_PH_FORCE_BIAS = 0,
  AFQMC_PH_FIELDS,
  AFQMC_PH_V,
  AFQMC_PH_BHALF,
  AFQMC_PH_TAYLOR,
  AFQMC_PH_OVERLAP,
  AFQMC_PH_WEIGHT,
  AFQMC_PH_QR,
  AFQMC_PH_COMB,
  AFQMC_PH_ENERGY,
  AFQMC_PH_THETA,
  AFQMC_NPHASE
};

/*
 * Time the phases of the next steps with CUDA events recorded on the state's
 * stream around each phase (no host synchronisation while recording).
 * max_steps bounds how many steps are recorded; later steps run untimed.
 */
AFQMC_API int afqmc_profile_start(afqmc_state* s, int32_t max_steps);

/*
 * Stop recording, synchronise the stream and return per phase the summed
 * device time in milliseconds (ms [AFQMC_NPHASE]) and how many times the
 * phase ran (count [AFQMC_NPHASE]); kernels [AFQMC_NPHASE] (may be NULL)
 * receives the kernels each phase launched.  Host arrays.
 */
AFQMC_API int afqmc_profile_stop(afqmc_state* s, double* ms, int64_t* count, int64_t* kernels);

/*
 * The dense contraction of the mixed-precision path on the tcgen05 tensor
 * cores, C[m][n] = alpha * sum_k A[m][k] B[n][k], FP32 accumulation.  The
 * force-bias traces (Eq. precomputing2), V = sum_g x_g L_g (Sec. 3.4.2) and
 * the T_g = Lh_g Theta products of Eq. localenergy3 are all of this form.
 *   dtype   0: A, B are BF16; 1: A, B are FP32 read as TF32
 *   dA, dB  DEVICE row-major operands with row pitches lda, ldb (elements;
 *           pitch * element size a multiple of 16 bytes, bases 16-byte
 *           aligned); entries past column k are not read
 *   dC      DEVICE row-major FP32 output with pitch ldc
 *   d_status DEVICE int: left unchanged on success, set non-zero if a
 *           bounded wait inside the kernel timed out (the result is then
 *           invalid)
 * Asynchronous on `stream`.
 */
AFQMC_API int afqmc_contract(int32_t dtype, int64_t m, int64_t n, int64_t k, const void* dA,
                             int64_t lda, const void* dB, int64_t ldb, float alpha, float* dC,
                             int64_t ldc, int* d_status, void* stream);

/*
 * The truncated Taylor expansion of exp(V) of Sec. 3.4.2 as the mixed path
 * applies it, on the tcgen05 tensor cores: for every walker w
 *     S_w = T_1 + ... + T_order,   T_k = V_w T_{k-1} / k,
 * with T_0 given, so that exp(V_w) T_0 = T_0 + S_w to order `order` (the
 * propagation step then applies exp(-dt v0'/2) to T_0 + S_w).  T_k is rounded
 * to the operand type before it multiplies V; products and S accumulate in
 * FP32.
 *   dtype    0: BF16 operands; 1: FP32 containers holding TF32 values
 *   Mp       padded orbital count, a multiple of 16, Mp >= M
 *   dV       [nwalkers][M][2 Mp]   row p = [Re V[p][0..Mp) | Im V[p][0..Mp)]
 *                                   (columns q >= M zero)
 *   dT0      [nwalkers][2N][2 Mp]  the 0th term as operand rows:
 *                                   row i      = [Re T_i | -Im T_i]
 *                                   row N + i  = [Im T_i |  Re T_i]
 *                                   with T_i[p] = T[p][i] (columns p >= M zero)
 *   dT1      same shape as dT0: scratch of the per-term route (may be NULL
 *            when the whole-series kernel runs); dT0 and dT1 are overwritten
 *   dS       [nwalkers][2N][ldS] FP32 output: row i = Re S_i, row N + i =
 *            Im S_i (S_i[p] = S[p][i]); columns p >= M are not written;
 *            ldS >= Mp, a multiple of 4
 *   per_term 0: one launch for the whole series when the term and the sum fit
 *            in shared and tensor memory (else per term); 1: one launch per term
 *   d_status DEVICE int, set non-zero if a bounded wait timed out
 * All buffers DEVICE, caller-owned, 16-byte aligned.  Requires 2N <= 128.
 * Returns AFQMC_EINVAL on bad sizes or pointers.  Asynchronous on `stream`.
 */
AFQMC_API int afqmc_taylor_series(int32_t dtype, int64_t nwalkers, int64_t N, int64_t M,
                                  int64_t Mp, int32_t order, const void* dV, void* dT0, void* dT1,
                                  float* dS, int64_t ldS, int32_t per_term, int* d_status,
                                  void* stream);

/*
 * The counter-based generator behind the auxiliary fields: Philox4x32 with
 * 10 rounds (J. K. Salmon et al., "Parallel random numbers: as easy as 1, 2,
 * 3", SC'11), key = (key & 0xffffffff, key >> 32).
 * d_ctr [n][4] and d_out [n][4] are DEVICE uint32 arrays owned by the caller;
 * the call is asynchronous on `stream`.
 */
AFQMC_API int afqmc_philox4x32_10(uint64_t key, const uint32_t* d_ctr, int64_t n,
                                  uint32_t* d_out, void* stream);

/*
 * The standard normal fields x ~ p(x) of Eq. hs2 that afqmc_propagate draws
 * for walkers [w0, w0 + nw) at step `step`: d_out [nw][nchol] DEVICE float64.
 * Field pair (2k, 2k+1) of walker w comes from Philox counter
 * (k, w, step, 0) by the Box-Muller transform of u1 (words 0, 1) and u2
 * (words 2, 3), u = fl(fl(a + 0.5) 2^-53), a = (hi >> 5) 2^26 + (lo >> 6).
 * Asynchronous on `stream`.
 */
AFQMC_API int afqmc_gaussian_fields(uint64_t seed, int64_t step, int32_t w0, int32_t nw,
                                    int32_t nchol, double* d_out, void* stream);

/*
 * The IEEE 754 conversions the mixed path's kernels use between the float64
 * orbitals and their FP32 arithmetic (binary64 -> binary32 rounded to
 * nearest, ties to even; binary32 -> binary64 exact), done in integer
 * arithmetic.  d_in / d_out: n DEVICE elements owned by the caller
 * (float64 -> float32 for afqmc_round_f32, float32 -> float64 for
 * afqmc_widen_f32); asynchronous on `stream`.  The results are those of the
 * hardware conversions, bit for bit.
 */
AFQMC_API int afqmc_round_f32(const double* d_in, float* d_out, int64_t n, void* stream);
AFQMC_API int afqmc_widen_f32(const float* d_in, double* d_out, int64_t n, void* stream);

/*
 * Local energies for callers that cannot allocate device memory.
 *
 * The paper has no counterpart: this is the float64 local-energy evaluation
 * of afqmc_local_energies() packaged for callers that own no workspace and may
 * not create one - for example a host program whose device memory all belongs
 * to another framework's pool, or code that must not call cudaMalloc because
 * the allocation would synchronise the device in the middle of its own stream
 * work.  The caller passes only inputs and outputs (all DEVICE float64):
 *   d_Lh     [nchol][N][M]      half-rotated Cholesky vectors V_T^T L_g
 *   d_hh     [N][M]             V_T^T h
 *   d_thetaT [nwalkers][2][N][M] Theta^T = (Phi S^-1)^T, real plane then
 *                               imaginary plane per walker
 *   d_eloc   [nwalkers][2]      output: E_loc (real, imaginary), H0 included
 * The intermediate results (force-bias traces and exchange partial sums,
 * nwalkers * (2 nchol + 2 ceil(nchol / chunk)) float64, chunk = the number of
 * Cholesky vectors one exchange block handles) live in one fixed 16 MiB array
 * inside the library, which every GPU that loads the library reserves until
 * the process exits.  Calls needing more return AFQMC_ENOSPC and launch
 * nothing (split the walkers over several calls); nwalkers above 65535
 * returns AFQMC_EINVAL, also before anything is launched.  Nothing is
 * allocated: no cudaMalloc, no cudaFree, no allocating library routine.
 * Every call made outside stream capture looks up the array's device address
 * on the current device with cudaGetSymbolAddress (the host-side name of the
 * array is not a device address); a call made while `stream` is being
 * captured reuses the address the last uncaptured call on that device found,
 * so make at least one call on a device before capturing one (otherwise
 * AFQMC_ESTATE), and after a cudaDeviceReset() make one again before
 * capturing.  Every call writes all of the array it later
 * reads, so nothing needs clearing, but all calls share the one array: calls
 * that may overlap on the GPU (different streams, or different host threads
 * on the same device) race and must be serialised by the caller.
 * Asynchronous on `stream`.
 */
AFQMC_API int afqmc_local_energies_noalloc(int32_t M, int32_t N, int32_t nchol,
                                           int32_t nwalkers, const double* d_Lh,
                                           const double* d_hh, const double* d_thetaT,
                                           double H0, double* d_eloc, void* stream);

/*
 * Bounded device-side wait, the pattern every wait inside the library follows
 * (the tensor-core pipelines' mbarrier waits): one thread polls the DEVICE
 * int *d_flag up to max_polls times (about 1 us apart); if it never becomes
 * non-zero the kernel writes AFQMC_ETIMEOUT to the DEVICE int *d_status and
 * returns, so the context stays usable and the host reads the status.  Used
 * by the failure-detection tests.  Asynchronous on `stream`.
 */
AFQMC_API int afqmc_wait_flag(const int* d_flag, int64_t max_polls, int* d_status, void* stream);

/*
 * Back-propagation estimator of the one-body density (Sec. "Computing
 * ground-state properties: the backpropagation algorithm", Eqs. bp1, bp,
 * bp_dets), on a state created with bp_steps > 0 (a comb inside the window
 * gives each copy its parent's recorded path).  On the
 * mixed path the fields are recorded as the BF16/TF32 operands the step used
 * and the backward sweep runs on the tensor cores; the densities and weights
 * are formed in float64 on both paths.
 *
 * afqmc_bp_begin opens a window at the current step n: it keeps Psi_n of
 * every walker; each later afqmc_propagate step records the shifted fields
 * x - xbar of B and, for a phaseless walk, the path-restoration factor
 * exp(-i dt Im E_loc(Psi_k)) / max(0, cos dtheta_k) (BP-PRes; the local
 * energies are evaluated every step while the window is open, and the steps
 * launch kernel by kernel).  At most bp_steps steps fit (afqmc_propagate
 * returns AFQMC_ENOSPC beyond).  Enqueued on the state's stream.
 *
 * afqmc_bp_end closes the window after m steps: the trial is propagated
 * backwards, Phi_m = B^+(x_n) ... B^+(x_{n+m-1}) Psi_T with
 * B(x)^+ = B(-conj(x)), and with rho_w,pq = sum_sigma
 * <Phi_m|a+_p,sigma a_q,sigma|Psi_n> / <Phi_m|Psi_n> it returns (HOST,
 * row-major, caller-owned)
 *   rho      [2][M][M]  BP-PRes: sum_w W_w F_w rho_w / sum_w W_w F_w, F_w the
 *                       product of the window's restoration factors (F = 1
 *                       in free projection), real plane then imaginary plane
 *   rho_phl  [2][M][M]  BP-PhL: the same with W_w alone (may be NULL)
 *   wsums    [4]        sum W F (re, im), sum W (re, im) (may be NULL)
 *   nsteps   m (may be NULL)
 * with W_w the weights at step n + m; walkers with W = 0 are left out.  The
 * walk itself is unchanged and continues with its own weights.  Synchronises
 * the stream.  AFQMC_ESTATE if no window is open (end) or one is (begin).
 */
AFQMC_API int afqmc_bp_begin(afqmc_state* s);
AFQMC_API int afqmc_bp_end(afqmc_state* s, double* rho, double* rho_phl, double* wsums,
                           int32_t* nsteps);

/*
 * Modified Cholesky decomposition of the two-electron interaction (Sec. 2.3,
 * Eqs. chol and chol2), the step that produces the Cholesky vectors L that
 * afqmc_init takes.
 *   dim      size of V: M*M for an interaction over M orbitals
 *   d_V      [dim][dim] DEVICE float64, row-major, symmetric positive
 *            semi-definite: V[p*M + r][q*M + s] = v_pqrs.  Read only: its
 *            diagonal, then row nu0 of every pivot nu0 (V is taken to be
 *            symmetric; a non-finite value in a row read stops the call)
 *   delta    threshold: vectors are added until every residual diagonal is
 *            below delta (then every residual element is, by Cauchy-Schwarz)
 *   max_vectors  room in d_L (1 .. 16384)
 *   d_L      [max_vectors][dim] DEVICE float64 output: vector g in row g
 *            (as L[g][p][r] for afqmc_init); rows >= *nvec are not written.
 *            Later iterations read the rows already written back
 *   d_piv    [max_vectors] DEVICE int32 output, may be NULL: the pivot index
 *            nu0 of each vector
 *   nvec     HOST output: number of vectors found
 *   residual HOST output, may be NULL: largest residual diagonal left; the
 *            decomposition converged iff *residual < delta (otherwise
 *            max_vectors vectors were found first)
 *   d_work   DEVICE workspace of afqmc_mcd_workspace_size() bytes, 256-byte
 *            aligned, caller-owned (about 8.8 dim + 8 max_vectors bytes)
 * Each iteration pivots on the largest residual diagonal Delta_max (the
 * smallest index among equal values), zeroes every index whose
 * sqrt(|Delta_mm| Delta_max) <= min(1e-9, delta) (damped prescreening: a
 * zeroed index stays zero in every later vector) and takes
 * L_mu = (V[mu][nu0] - sum_g L[g][mu] L[g][nu0]) / sqrt(Delta_max).
 * Runs on `stream` and returns when the decomposition is done (it reads a
 * few bytes of state back between groups of launches).  Returns
 * AFQMC_EINVAL on bad arguments, AFQMC_ENOSPC if the workspace is too small,
 * AFQMC_ENONFINITE if V's diagonal or a row it read holds a non-finite value.
 */
AFQMC_API int afqmc_mcd_workspace_size(int64_t dim, int32_t max_vectors, size_t* bytes);
AFQMC_API int afqmc_modified_cholesky(int64_t dim, const double* d_V, double delta,
                                      int32_t max_vectors, double* d_L, int32_t* d_piv,
                                      int32_t* nvec, double* residual, void* d_work,
                                      size_t work_bytes, void* stream);

/*
 * The same decomposition for the interaction of real orbitals, whose rows
 * (p, r) and (r, p) of V are equal (v_pqrs = v_rqps), taken over the
 * M (M + 1) / 2 index pairs p <= r: half the arithmetic and a quarter of
 * the matrix.  Pair index P(p, r) = p M - p (p - 1) / 2 + (r - p), p <= r.
 *   M        orbitals (1 .. 2048)
 *   d_Vpair  [npair][npair] DEVICE float64, npair = M (M + 1) / 2:
 *            Vpair[P(p, r)][P(q, s)] = v_pqrs for p <= r, q <= s
 *   d_L      [max_vectors][M][M] DEVICE float64 output: L[g][p][r] =
 *            L[g][r][p]; rows >= *nvec are not written
 *   d_piv    [max_vectors] DEVICE int32 output, may be NULL: pivots as
 *            p M + r with p <= r
 *   d_work   afqmc_mcd_pairs_workspace_size() bytes (about
 *            8 npair (max_vectors + 2) bytes), 256-byte aligned
 * Pivots, vectors and residual are those afqmc_modified_cholesky gives on
 * the full M^2 x M^2 matrix (pivots on the lower index p M + r of a pair,
 * equal rows carrying equal vectors), up to the order of the sums.  Other
 * arguments and the return values as for afqmc_modified_cholesky.
 */
AFQMC_API int afqmc_mcd_pairs_workspace_size(int32_t M, int32_t max_vectors, size_t* bytes);
AFQMC_API int afqmc_modified_cholesky_pairs(int32_t M, const double* d_Vpair, double delta,
                                            int32_t max_vectors, double* d_L, int32_t* d_piv,
                                            int32_t* nvec, double* residual, void* d_work,
                                            size_t work_bytes, void* stream);

/* Message for the calling thread's last failed call (never NULL). */
AFQMC_API const char* afqmc_last_error(void);

/* Number of kernels launched by this library in this process. */
AFQMC_API int64_t afqmc_launch_count(void);

#ifdef __cplusplus
}
#endif
#endif /* AFQMC_H */
