// Tensor-core (tcgen05) contraction launchers (internal header).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace afq {

// D[m][n] = sum_k A[m][k] * B[n][k]; A, B row-major K-major operands of BF16
// (tf32 = false) or FP32 read as TF32 (tf32 = true); pitches in elements,
// multiples of 16 bytes; base addresses 16-byte aligned.
struct TcGemm {
  int m = 0, n = 0, k = 0;
  const void* A = nullptr;
  long lda = 0;
  const void* B = nullptr;
  long ldb = 0;
  bool tf32 = false;
  int* err = nullptr;  // device status word, set on a timed-out wait
  // A split operand in B ([B_hi | B_lo] along K, each a_wrap wide, a_wrap a
  // multiple of 128 bytes of K): A's K coordinate is taken modulo a_wrap, so
  // that D = A (B_hi + B_lo)^T; ka = A's own K extent (0: k)
  int a_wrap = 0, ka = 0;
};

int tc_gemm_store(const TcGemm& g, float* C, long ldc, float alpha, cudaStream_t st);
// Time the tile-width candidates for this shape on the given buffers (not
// under stream capture) and remember the fastest for tc_gemm_store().
int tc_tune_store(const TcGemm& g, float* C, long ldc, float alpha, cudaStream_t st, int* chosen);

// Exchange energy contraction (rows (g,i) of Lh, columns (w,c,j) of Theta^T)
// with the fused sum_ij T_ij T_ji epilogue; part [W][nchunk][2] (float64).
// Propagation on tcgen05 (mixed path): first half step, Taylor terms, last
// half step (see the epilogues in gemm_tc.cu for the operand layouts).
// (B = D_B = B_half - I; phi_id = the float64 orbitals, pitch M, whose
// identity part the epilogue adds)
int tc_prop_first(const TcGemm& g, float* acc, long ldacc, void* tb, const double* phi_id,
                  int lo_kind, int N, int M, int Mp, cudaStream_t st);
// S = T_k (first) or S += T_k, T_k = scale * (V T_{k-1}); pitch lds
int tc_taylor_term(const TcGemm& g, float* S, long lds, bool first, void* tb_out, int lo_kind,
                   int W, int N, int M, int Mp, float scale, cudaStream_t st);
// also writes the BF16/TF32 copy of the new orbitals (pitch Mp) for live walkers
// (A = [T_0 | S] = acc_id, pitch 2 Mp; B = [D_B | D_B]; the epilogue adds T_0 + S)
int tc_prop_last(const TcGemm& g, double* phiT, const double* wt, int N, int M, void* phi_lo,
                 int lo_kind, int Mp, const float* acc_id, cudaStream_t st);
// V = i sqrt(dt) sum_g x_g L_g from the full transposed vectors (rows p*Mp+q)
// written directly as [Re V | Im V] rows (pitch 2 Mp) of each walker.
int tc_v_full(const TcGemm& g, void* V, int lo_kind, int W, int M, int Mp, double sdt,
              cudaStream_t st);
// Time V's tile-width candidates (128: half blocks, two accumulators; 256:
// whole blocks) on the given buffers and remember the faster for tc_v_full().
int tc_tune_v(const TcGemm& g, void* V, int lo_kind, int W, int M, int Mp, double sdt,
              cudaStream_t st, int* chosen);

// Whole Taylor series per walker in one launch (one CTA per walker at a time):
// the term stays in shared memory and the walker's [Re V | Im V] rows are
// streamed once per term (from L2 after the first).  T0: the 0th term operand
// rows [W][2N][2Mp], V: [W][M][2Mp], S: [W][2N][lds] FP32 receives
// T_1 + ... + T_order (columns p < M).  tc_taylor_series_fits() says whether
// the shape fits the kernel's shared memory and tensor memory.
bool tc_taylor_series_fits(int lo_kind, int N, int M, int Mp);
int tc_taylor_series(const void* V, const void* T0, float* S, long lds, int lo_kind, int W, int N,
                     int M, int Mp, int order, int* err, cudaStream_t st);

// The series by whichever route fits: the whole-series kernel unless per_term
// is set or the shape does not fit, else one launch per term (the operand
// alternates between T0 and T1, so both are overwritten).
int taylor_apply(const void* V, void* T0, void* T1, float* S, long lds, int lo_kind, int W, int N,
                 int M, int Mp, int order, bool per_term, int* err, cudaStream_t st);

// tensor maps (128-byte swizzle, box = 128 bytes x box_rows)
int make_tmap(CUtensorMap* m, const void* base, int elem_bytes, long rows, long cols, long pitch,
              int box_rows);
int make_tmap_3d(CUtensorMap* m, const void* base, int elem_bytes, long planes, long rows,
                 long cols, long pitch, long plane_stride, int box_rows, int box_planes = 1);
int make_tmap_nd(CUtensorMap* m, const void* base, int elem_bytes, int rank, const long* dims,
                 const long* stride_bytes, const int* box);
int tc_sm_count();

// A per-step contraction of the mixed path as a state describes it: run on
// its own (tc_job_launch, the same launches as tc_gemm_store / tc_v_full /
// tc_prop_first / tc_prop_last) or together with other states' contractions
// of the same kind in one persistent launch (TcGrouped: a work list over
// (contraction, tile), each contraction's tensor maps in a device table).
enum TcJobKind { TC_JOB_STORE = 0, TC_JOB_V = 1, TC_JOB_PROP0 = 2, TC_JOB_PHI = 3 };
struct TcJobDesc {
  int kind = TC_JOB_STORE;
  TcGemm g;
  float* C = nullptr;  // store: C = alpha * D, pitch ldc
  long ldc = 0;
  float alpha = 1.f;
  void* V = nullptr;  // V: the [Re V | Im V] operand rows
  int W = 0;
  double sdt = 0.0;
  int lo_kind = 0, N = 0, M = 0, Mp = 0;
  float* acc = nullptr;  // first half step (tc_prop_first's arguments)
  long ldacc = 0;
  void* tb = nullptr;
  const double* phi_id = nullptr;
  double* phiT = nullptr;  // last half step (tc_prop_last's arguments)
  const double* wt = nullptr;
  void* phi_lo = nullptr;
  const float* acc_id = nullptr;
};
int tc_job_launch(const TcJobDesc& d, cudaStream_t st);

struct TcGrouped;  // one grouped launch: its device job table and tile configuration
// Build the grouped launch of n descriptors of one kind and precision with
// tile width bn (0: the kind's default); allocates the device table.
int tc_grouped_create(const TcJobDesc* d, int n, int bn, TcGrouped** out);
// Time the kind's tile-width candidates (not under capture; every candidate
// runs on the descriptors' own buffers, so not for TC_JOB_PHI, whose epilogue
// overwrites the orbitals) and keep the fastest.
int tc_grouped_tune(const TcJobDesc* d, int n, cudaStream_t st, TcGrouped** out);
int tc_grouped_launch(const TcGrouped* g, cudaStream_t st);
int tc_grouped_bn(const TcGrouped* g);
int tc_grouped_tiles(const TcGrouped* g);
void tc_grouped_destroy(TcGrouped* g);

// Exchange blocking: RG Cholesky vectors x CW walkers per 128 x 256 tile, the
// 2N columns of a walker padded to NPAD (a power of two >= 16).
void exchange_tile(int N, int* RG, int* CW, int* NPAD);
int tc_exchange(const TcGemm& g, int G, int W, int N, double* part, int nchunk, cudaStream_t st);

}  // namespace afq
