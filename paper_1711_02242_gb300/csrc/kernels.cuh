// Internal launchers of the AFQMC kernels (not part of the C ABI).
#pragma once

#include <cuda_bf16.h>

#include "common.cuh"

namespace afq {

// Walker weights are stored as [W][2] (re, im); a walker is alive while its
// weight is non-zero (algorithm outline, step 2).
__device__ __forceinline__ bool walker_alive(const double* w2, long w) {
  return w2[2 * w] != 0.0 || w2[2 * w + 1] != 0.0;
}

// Operand copies for the tensor-core contractions of the mixed path.
enum { LO_NONE = 0, LO_BF16 = 1, LO_TF32 = 2 };

// FP32 -> TF32 with round-to-nearest (ties away), kept in an FP32 container.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// IEEE 754 binary64 -> binary32 with round to nearest, ties to even (IEEE
// 754-2008, Secs. 4.3.1 and 5.4.2), in integer arithmetic: this GPU runs F2F
// conversions on its narrow FP64 pipe, the integer pipe is many times wider.
// Results that are normal floats (including a round-up to infinity from the
// top binade) and zeros take the integer path; subnormal, overflowing,
// infinite and NaN inputs take the hardware conversion.
__device__ __forceinline__ float f64_to_f32(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t e = (hi >> 20) & 0x7ffu;
  if (e - 897u < 254u) {
    // sign, exponent re-biased from 1023 to 127, the top 23 of 52 mantissa bits
    uint32_t r = (hi & 0x80000000u) | ((e - 896u) << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
    const uint32_t rest = lo & 0x1fffffffu;  // the 29 bits dropped
    r += (rest > 0x10000000u || (rest == 0x10000000u && (r & 1u))) ? 1u : 0u;
    return __uint_as_float(r);
  }
  if (((hi << 1) | lo) == 0u) return __uint_as_float(hi & 0x80000000u);
  return __double2float_rn(x);
}

// binary32 -> binary64 (exact) in integer arithmetic, as above.
__device__ __forceinline__ double f32_to_f64(float f) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t e = (u >> 23) & 0xffu;
  if (e - 1u < 254u)
    return __hiloint2double((int)((u & 0x80000000u) | ((e + 896u) << 20) | ((u & 0x7fffffu) >> 3)),
                            (int)(u << 29));
  if ((u << 1) == 0u) return __hiloint2double((int)(u & 0x80000000u), 0);
  return (double)f;
}

// FP32 value into a BF16 / TF32 operand copy (no float64 step).
__device__ __forceinline__ void store_lo_f(void* base, int kind, long idx, float v) {
  if (kind == LO_BF16)
    reinterpret_cast<__nv_bfloat16*>(base)[idx] = __float2bfloat16_rn(v);
  else
    reinterpret_cast<float*>(base)[idx] = round_tf32(v);
}

__device__ __forceinline__ void store_lo(void* base, int kind, long idx, double v) {
  if (kind == LO_BF16)
    reinterpret_cast<__nv_bfloat16*>(base)[idx] = __double2bfloat16(v);
  else
    reinterpret_cast<float*>(base)[idx] = round_tf32((float)v);
}

template <typename TA, typename TB, typename TC>
struct GemmNT {
  int m = 0, n = 0, k = 0, kb = 1, batch = 1;
  double alpha = 1.0, beta = 0.0;
  const TA* A = nullptr;
  long lda = 0, sAk = 0, sAb = 0;
  const TB* B = nullptr;
  long ldb = 0, sBk = 0, sBb = 0;
  TC* C = nullptr;
  long ldc = 0, sCb = 0;
  const double* mask = nullptr;  // weights [W][2]: skip rows of dead walkers
  int mask_rows = 1;             // rows of C per walker
};
using GemmF64 = GemmNT<double, double, double>;
int gemm_nt_f64(const GemmF64& g, cudaStream_t st);
// FP32 accumulation: float64 A -> float32 C, and float32 A -> float64 C
int gemm_nt_dff(const GemmNT<double, float, float>& g, cudaStream_t st);
int gemm_nt_ffd(const GemmNT<float, float, double>& g, cudaStream_t st);
int gemm_nt_ddf(const GemmNT<double, double, float>& g, cudaStream_t st);
int gemm_nt_fff(const GemmNT<float, float, float>& g, cudaStream_t st);
// FP32 operands and products, summed in FP32 over each 16-term block of K and
// in float64 across the blocks
int gemm_nt_ffd_split(const GemmNT<float, float, double>& g, cudaStream_t st);
// float64 operands, FP32 products summed in FP32 over each 16-term block of K
// and in float64 across the blocks
int gemm_nt_f32_split(const GemmF64& g, cudaStream_t st);
// float64 -> FP32, round to nearest even
int launch_round_f32(const double* src, float* dst, long n, cudaStream_t st);
// float64 array rounded to FP32 in place, in chunks of c values (tmp: c floats)
int launch_round_f32_inplace(double* buf, long n, long c, float* tmp, cudaStream_t st);
// part[z][i] = sum over the z-th of nz chunks of rows g of c[g] A[g][i]
int launch_wsum_rows(const double* A, const double* c, int G, long n, int nz, double* part,
                     cudaStream_t st);
// dst[g][0 .. len) = src[g * sstride + 0 .. len), FP32 -> float64
int launch_widen_rows(const float* src, long sstride, long len, int G, double* dst,
                      cudaStream_t st);
// smallest index of a non-finite value into *first (which the caller sets to ~0)
int launch_first_nonfinite(const double* v, long n, unsigned long long* first, cudaStream_t st);

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
  // mixed path: t read as float, x written as a BF16/TF32 copy with pitch Gp
  const float* t32 = nullptr;
  void* x_lo = nullptr;
  int lo_kind = LO_NONE, Gp = 0;
  int w0 = 0;  // global index of walker 0 in the Philox counter (sharded populations)
};
int launch_field(const FieldArgs& a, cudaStream_t st);

template <typename T>
struct TaylorArgsT {
  int W, M, N, P, k;  // k: order of the term produced (1..n)
  long ldy;           // pitch of one (walker, re/im) row of Y
  double scale;       // sqrt(dt) / k
  const T* Y;         // [W][2][ldy] packed sum_g x_g L_g (re, im)
  const T* tin;       // [W][2][N][M] previous term (transposed orbitals)
  T* tout;            // [W][2][N][M] new term
  T* acc;             // [W][2][N][M] running sum (k == 1: acc = tin + tout)
};
using TaylorArgs = TaylorArgsT<double>;
int launch_taylor_term(const TaylorArgsT<double>& a, cudaStream_t st);

// Fused overlap: S = V_T^T Phi, Gauss-Jordan S^-1 and log det, Theta = Phi S^-1.
struct OverlapArgs {
  int W, M, N;
  const double* VTt;   // [N][M]
  const double* phiT;  // [W][2][N][M]
  double* thetaT;      // [W][2][N][M] (live walkers)
  double* logdet;      // [W][2] (live walkers)
  const double* wt;    // alive mask (nullptr: all)
  void* th_lo = nullptr;
  int lo_kind = LO_NONE, Mp = 0;
  int unit_trial = 0;  // VTt = [I_N | 0]: S is the top block of Phi, Theta's top rows I
  double2* Sinv = nullptr;  // [W][N][N] scratch: S^-1 of live walkers
  float2* Sinv32 = nullptr;  // _F32LU precisions: FP32 elimination, S^-1 here and FP32 Theta
  int theta32 = 0;  // FP32 product Theta = Phi S^-1 from the float64 S^-1 (Sinv32 unset)
  // spin blocks: columns [0, nup) spin up, [nup, N) spin down (nup = N: one
  // closed-shell block standing for both spins); sf = spins per block (2 or 1)
  int nup = 0;
  double sf = 2.0;
};
// S^-1 and log det (k_overlap), then Theta (k_theta_rows)
int launch_overlap(const OverlapArgs& a, cudaStream_t st);
int launch_theta(const OverlapArgs& a, cudaStream_t st);

struct WeightArgs {
  int W, mode;
  double dt, sdt, H0p, e_shift, wmax;
  const double* ld_new;  // [W][2]
  double* ld;            // [W][2] (updated for live walkers)
  const double* scal;    // [W][8]
  double* wt;            // [W][2]
  unsigned long long* nonfinite;
  int64_t* dstep;  // incremented once per step
  double* cosd = nullptr;  // [W]: cos dtheta of the step (phaseless), when non-null
};
int launch_weight(const WeightArgs& a, cudaStream_t st);

struct MgsArgs {
  int W, M, N;
  double* phiT;  // [W][2][N][M] in place
  const double* wt;
  double* ld;    // [W][2]: log <Psi_T|Psi> of live walkers, lowered by 2 sum_k log r_kk
  int f32 = 0;   // _F32LU precisions: FP32 sweep in shared memory where [N][M] fits
  void* phi_lo = nullptr;  // and, if set, the BF16/TF32 copy of the result (pitch Mp)
  int lo_kind = LO_NONE, Mp = 0;
  int nup = 0;      // spin blocks as in OverlapArgs (0: one block), swept separately
  double sf = 2.0;  // spins per block: log <Psi_T|Psi> drops by sf sum_k log r_kk
};
int launch_mgs(const MgsArgs& a, cudaStream_t st);

struct ExchArgs {
  int W, M, N, G, gc, nchunk;
  const double* Lh;      // [G][N][M]
  const double* thetaT;  // [W][2][N][M]
  double* part;          // [W][nchunk][2]
  const double* wt;
  int nup = 0;  // spin blocks (0: one block): only same-spin pairs (i, j) are summed
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
  const float* t32 = nullptr;  // mixed path: t as float
  double sf = 2.0;  // spins per block: E = H0 + sf e1 + c / 2 - sf x / 2
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
// dst = sum of nparts arrays of n doubles (parts[j][e]), added in the order of j
int launch_sum_parts(const double* parts, int nparts, long n, double* dst, cudaStream_t st);
int launch_init_walkers(const double* VTt, double* phiT, double* wt, int W, int N, int M,
                        cudaStream_t st);
int launch_sumsq(const double* v, double* out, int n, cudaStream_t st);
// dst[r][c] = lo(src[r][c]) for c < cols, 0 for cols <= c < ldd
// dst[r][c] = lo(src[r][c] - (r == c ? minus_diag : 0)), zero for cols <= c < ldd
int launch_convert_lo(const double* src, long rows, long cols, long lds, void* dst, long ldd,
                      int kind, cudaStream_t st, double minus_diag = 0.0);
// src - minus_diag I as nseg K segments of width seg per row (pitch seg nseg),
// segment g the BF16/TF32 high part, or (bit g of lo_mask) the low part.
int launch_split_lo(const double* src, long rows, long cols, long lds, void* dst, long seg,
                    int nseg, unsigned lo_mask, int kind, cudaStream_t st, double minus_diag);
int launch_convert_f32(const double* src, float* dst, long n, cudaStream_t st);
// full Cholesky vectors transposed, rows (p, q) = p * Mp + q, pitch Gp, low precision
int launch_pack_blocks_lo(const double* L, int G, int M, int Mp, int Gp, void* out, int kind,
                          cudaStream_t st);
int launch_pack_blocks_lo(const float* L, int G, int M, int Mp, int Gp, void* out, int kind,
                          cudaStream_t st);

}  // namespace afq
