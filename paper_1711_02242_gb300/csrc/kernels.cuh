// Internal launchers of the AFQMC kernels (not part of the C ABI).
#pragma once

#include "common.cuh"

namespace afq {

// Walker weights are stored as [W][2] (re, im); a walker is alive while its
// weight is non-zero (algorithm outline, step 2).
__device__ __forceinline__ bool walker_alive(const double* w2, long w) {
  return w2[2 * w] != 0.0 || w2[2 * w + 1] != 0.0;
}

struct GemmF64 {
  int m = 0, n = 0, k = 0, kb = 1, batch = 1;
  double alpha = 1.0, beta = 0.0;
  const double* A = nullptr;
  long lda = 0, sAk = 0, sAb = 0;
  const double* B = nullptr;
  long ldb = 0, sBk = 0, sBb = 0;
  double* C = nullptr;
  long ldc = 0, sCb = 0;
  const double* mask = nullptr;  // weights [W][2]: skip rows of dead walkers
  int mask_rows = 1;             // rows of C per walker
};
int gemm_nt_f64(const GemmF64& g, cudaStream_t st);

// ---- step kernels (float64) -------------------------------------------------
struct FieldArgs {
  int W, G, mode;
  uint64_t seed;
  double sdt, fb_cap;
  const double* t;   // [W][2][G]  t_g = 2 Tr(Lh_g Theta) (re rows, im rows)
  const double* c;   // [G]
  const double* wt;  // [W][2]
  double* x;         // [W][2][G]  x = xi - xbar
  double* scal;      // [W][8]: sum xi xbar, sum xbar^2, sum x c (complex each)
  const int64_t* dstep;  // device step counter (the step being taken)
};
int launch_field(const FieldArgs& a, cudaStream_t st);

struct TaylorArgs {
  int W, M, N, P, k;  // k: order of the term produced (1..n)
  double scale;       // sqrt(dt) / k
  const double* Y;    // [W][2][P] packed sum_g x_g L_g (re, im)
  const double* tin;  // [W][2][N][M] previous term (transposed orbitals)
  double* tout;       // [W][2][N][M] new term
  double* acc;        // [W][2][N][M] running sum (k == 1: acc = tin + tout)
  const double* wt;
};
int launch_taylor_term(const TaylorArgs& a, cudaStream_t st);

struct LuArgs {
  int W, N;
  const double* S;   // [W][2][N][N]: S_c[i][j] at [w][c][j][i]
  double* Sinv;      // [W][2][N][N]: row-major S^-1
  double* logdet;    // [W][2]: 2 log|det S|, wrapped 2 arg det S
  const double* wt;  // alive mask
};
int launch_lu_inv(const LuArgs& a, cudaStream_t st);

struct ThetaArgs {
  int W, M, N;
  const double* Sinv;  // [W][2][N][N]
  const double* phiT;  // [W][2][N][M]
  double* thetaT;      // [W][2][N][M]
  const double* wt;
};
int launch_theta(const ThetaArgs& a, cudaStream_t st);

struct WeightArgs {
  int W, mode;
  double dt, sdt, H0p, e_shift, wmax;
  const double* ld_new;  // [W][2]
  double* ld;            // [W][2] (updated for live walkers)
  const double* scal;    // [W][8]
  double* wt;            // [W][2]
  unsigned long long* nonfinite;
  int64_t* dstep;  // incremented once per step
};
int launch_weight(const WeightArgs& a, cudaStream_t st);

struct MgsArgs {
  int W, M, N;
  double* phiT;  // [W][2][N][M] in place
  const double* wt;
};
int launch_mgs(const MgsArgs& a, cudaStream_t st);

struct ExchArgs {
  int W, M, N, G, gc, nchunk;
  const double* Lh;      // [G][N][M]
  const double* thetaT;  // [W][2][N][M]
  double* part;          // [W][nchunk][2]
  const double* wt;
};
int exchange_chunk(int N, int G);
int launch_exchange(const ExchArgs& a, cudaStream_t st);

struct ElocArgs {
  int W, M, N, G, nchunk;
  double H0;
  const double* hh;      // [N][M]
  const double* thetaT;  // [W][2][N][M]
  const double* t;       // [W][2][G]
  const double* part;    // [W][nchunk][2]
  double* eloc;          // [W][2]
  const double* wt;
};
int launch_eloc(const ElocArgs& a, cudaStream_t st);

struct RecordArgs {
  int W, mode, max_records;
  double lo, hi;  // clamp of Re E_loc (phaseless)
  const double* eloc;
  const double* wt;
  double* records;  // [max_records][4]
  unsigned long long* rec_count;
  double* last;  // [4]: E num re, den re, num im, den im
  const int64_t* step;
};
int launch_record(const RecordArgs& a, cudaStream_t st);

struct CombArgs {
  int W, M, N;
  uint64_t seed;
  const int64_t* dstep;  // already advanced past the step that ends here
  double* wt;        // [W][2]
  double* cum;       // [W] scratch
  int* parent;       // [W] scratch
  double* phiT;      // [W][2][N][M]
  double* thetaT;    // [W][2][N][M]
  double* ld;        // [W][2]
  double* tmp_phi;   // [W][2][N][M] scratch
  double* tmp_theta; // [W][2][N][M] scratch
  double* tmp_ld;    // [W][2] scratch
  double* wtot;      // [1] scratch
};
int launch_comb(const CombArgs& a, cudaStream_t st);

// ---- set-up kernels -----------------------------------------------------------
int launch_pack_transpose(const double* L, double* LpT, int G, int M, cudaStream_t st);
int launch_rowdot(const double* A, const double* b, double* out, int rows, int len,
                  double scale, cudaStream_t st);
int launch_v0p(const double* h1, const double* L2, const double* cLp, double* X, int M,
               double scale, cudaStream_t st);
int launch_norm1(const double* X, double* out, int M, cudaStream_t st);
int launch_fill_identity(double* X, int M, double scale_diag, cudaStream_t st);
int launch_scale(double* X, long n, double s, cudaStream_t st);
int launch_init_walkers(const double* VTt, double* phiT, double* wt, int W, int N, int M,
                        cudaStream_t st);
int launch_sumsq(const double* v, double* out, int n, cudaStream_t st);

}  // namespace afq
