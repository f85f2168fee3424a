// FP64 "NT" GEMM for the float64 path:
//   C[m][n] = alpha * sum_{b < kb} sum_{k < K} A_b[m][k] * B_b[n][k] + beta * C[m][n]
// batched over blockIdx.z.  Both operands are read along K (contiguous), which
// is how every contraction of the step is laid out (walkers are stored
// orbital-major, Phi^T, so X * Phi becomes Phi^T X^T with symmetric X).
//
// GB300 executes float64 at ~1.2 TFLOP/s (measured DFMA throughput), about
// 1/60 of its FP32 rate, so this kernel is bound by the FP64 pipe whatever the
// tiling: a 64x64 tile with a 4x4 register block per thread keeps it busy
// with a few resident warps per SM.
#include "kernels.cuh"

namespace afq {

namespace {
constexpr int BM = 64, BN = 64, BK = 16, TPB = 256;

__global__ void __launch_bounds__(TPB) k_gemm_nt_f64(GemmF64 g) {
  __shared__ double As[BK][BM + 1];
  __shared__ double Bs[BK][BN + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long z = blockIdx.z;
  const double* A = g.A + z * g.sAb;
  const double* B = g.B + z * g.sBb;
  double* C = g.C + z * g.sCb;
  double acc[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;

  for (int b = 0; b < g.kb; ++b) {
    const double* Ab = A + (long)b * g.sAk;
    const double* Bb = B + (long)b * g.sBk;
    for (int k0 = 0; k0 < g.k; k0 += BK) {
#pragma unroll
      for (int r = 0; r < (BM * BK) / TPB; ++r) {
        int idx = threadIdx.x + r * TPB;
        int row = idx / BK, col = idx % BK;
        int gm = m0 + row, gk = k0 + col;
        As[col][row] = (gm < g.m && gk < g.k) ? Ab[(long)gm * g.lda + gk] : 0.0;
        int gn = n0 + row;
        Bs[col][row] = (gn < g.n && gk < g.k) ? Bb[(long)gn * g.ldb + gk] : 0.0;
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        double a[4], bv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
      }
      __syncthreads();
    }
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    int gm = m0 + ty + 16 * i;
    if (gm >= g.m) continue;
    if (g.mask && !walker_alive(g.mask, gm / g.mask_rows)) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int gn = n0 + tx + 16 * j;
      if (gn >= g.n) continue;
      double* c = C + (long)gm * g.ldc + gn;
      double v = g.alpha * acc[i][j];
      if (g.beta != 0.0) v = fma(g.beta, *c, v);
      *c = v;
    }
  }
}
}  // namespace

int gemm_nt_f64(const GemmF64& g, cudaStream_t st) {
  if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return AFQMC_OK;
  if (g.k < 0 || g.kb < 1) {
    set_error("gemm_nt_f64: bad k=%d kb=%d", g.k, g.kb);
    return AFQMC_EINVAL;
  }
  if (g.mask && g.mask_rows <= 0) {
    set_error("gemm_nt_f64: mask_rows must be positive");
    return AFQMC_EINVAL;
  }
  dim3 grid(cdiv(g.n, BN), cdiv(g.m, BM), g.batch);
  if (grid.y > 65535u || grid.z > 65535u) {
    set_error("gemm_nt_f64: grid too large (m=%d batch=%d)", g.m, g.batch);
    return AFQMC_EINVAL;
  }
  AFQ_LAUNCH(k_gemm_nt_f64, grid, TPB, 0, st, g);
  return AFQMC_OK;
}

}  // namespace afq
