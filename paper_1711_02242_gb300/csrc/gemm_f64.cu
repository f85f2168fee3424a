// SIMT "NT" GEMM on the CUDA cores:
//   C[m][n] = alpha * sum_{b < kb} sum_{k < K} A_b[m][k] * B_b[n][k] + beta * C[m][n]
// batched over blockIdx.z.  Both operands are read along K (contiguous), which
// is how every contraction of the step is laid out (walkers are stored
// orbital-major, Phi^T, so X * Phi becomes Phi^T X^T with symmetric X).
//
// Float64 instance: GB300 executes float64 at ~1.2 TFLOP/s (measured DFMA
// throughput), about 1/60 of its FP32 rate, so the kernel is bound by the
// FP64 pipe whatever the tiling; a 64x64 tile with a 4x4 register block per
// thread keeps it busy with a few resident warps per SM.
// Mixed instances (FP32 accumulation) multiply the exp(-dt v0'/2) factor
// into float64 or float32 walkers and store float32 or float64, and form the
// set-up products of the mixed path that only feed BF16/TF32 operands (the
// basis rotation of the Cholesky vectors, sum_g L_g L_g).
#include <type_traits>

#include "kernels.cuh"

namespace afq {

namespace {
constexpr int BK = 16, TPB = 256, kSplitRun = 16;

// Four consecutive shared-memory values (16- or 32-byte aligned) in one or two
// vector loads.
__device__ __forceinline__ void ld4(const float* p, float* v) {
  const float4 x = *reinterpret_cast<const float4*>(p);
  v[0] = x.x;
  v[1] = x.y;
  v[2] = x.z;
  v[3] = x.w;
}
__device__ __forceinline__ void ld4(const double* p, double* v) {
  const double2 x = reinterpret_cast<const double2*>(p)[0], y = reinterpret_cast<const double2*>(p)[1];
  v[0] = x.x;
  v[1] = x.y;
  v[2] = y.x;
  v[3] = y.y;
}

// SPLIT (FP32 ACC): the products of each run of kSplitRun BK-term blocks of K
// (256 terms) are summed in FP32 and the run sums in float64, so the rounding
// error no longer grows with K (sums over all Cholesky vectors, K = G M); the
// float64 adds, on GB300's slow float64 pipe, stay a small part of the work.
// TM: rows (and columns) per thread; the tile is 16 TM x 16 TM, thread (tx, ty)
// owns rows TM ty .. TM ty + TM - 1 and columns TM tx .. (vector loads of its
// operands from shared memory when TM = 4).  Every output element is summed
// over k in the same order whatever the tile, so results do not depend on it.
template <typename TA, typename TB, typename TC, typename ACC, bool SPLIT = false, int TM = 4>
__global__ void __launch_bounds__(TPB) k_gemm_nt(GemmNT<TA, TB, TC> g) {
  constexpr int BM = 16 * TM, BN = 16 * TM, PAD = TM == 4 ? 4 : 1;
  __shared__ __align__(16) ACC As[BK][BM + PAD];
  __shared__ __align__(16) ACC Bs[BK][BN + PAD];
  using SUM = typename std::conditional<SPLIT, double, ACC>::type;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const long z = blockIdx.z;
  const TA* A = g.A + z * g.sAb;
  const TB* B = g.B + z * g.sBb;
  TC* C = g.C + z * g.sCb;
  SUM acc[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) acc[i][j] = SUM(0);

  ACC blk[TM][TM];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TM; ++j) blk[i][j] = ACC(0);
  int run = 0;  // BK blocks summed in blk since the last float64 add (SPLIT)
  for (int b = 0; b < g.kb; ++b) {
    const TA* Ab = A + (long)b * g.sAk;
    const TB* Bb = B + (long)b * g.sBk;
    for (int k0 = 0; k0 < g.k; k0 += BK) {
#pragma unroll
      for (int r = 0; r < (BM * BK) / TPB; ++r) {
        int idx = threadIdx.x + r * TPB;
        int row = idx / BK, col = idx % BK;
        int gm = m0 + row, gk = k0 + col;
        As[col][row] = (gm < g.m && gk < g.k) ? ACC(Ab[(long)gm * g.lda + gk]) : ACC(0);
        int gn = n0 + row;
        Bs[col][row] = (gn < g.n && gk < g.k) ? ACC(Bb[(long)gn * g.ldb + gk]) : ACC(0);
      }
      __syncthreads();
      if (!SPLIT) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TM; ++j) blk[i][j] = ACC(acc[i][j]);
      }
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        ACC a[TM], bv[TM];
        if constexpr (TM == 4) {
          ld4(&As[kk][TM * ty], a);
          ld4(&Bs[kk][TM * tx], bv);
        } else {
#pragma unroll
          for (int i = 0; i < TM; ++i) a[i] = As[kk][TM * ty + i];
#pragma unroll
          for (int j = 0; j < TM; ++j) bv[j] = Bs[kk][TM * tx + j];
        }
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TM; ++j) blk[i][j] = fma(a[i], bv[j], blk[i][j]);
      }
      if (!SPLIT) {
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TM; ++j) acc[i][j] = SUM(blk[i][j]);
      } else if (++run == kSplitRun) {
        run = 0;
#pragma unroll
        for (int i = 0; i < TM; ++i)
#pragma unroll
          for (int j = 0; j < TM; ++j) {
            acc[i][j] += SUM(blk[i][j]);
            blk[i][j] = ACC(0);
          }
      }
      __syncthreads();
    }
  }
  if (SPLIT && run > 0) {
#pragma unroll
    for (int i = 0; i < TM; ++i)
#pragma unroll
      for (int j = 0; j < TM; ++j) acc[i][j] += SUM(blk[i][j]);
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    int gm = m0 + TM * ty + i;
    if (gm >= g.m) continue;
    if (g.mask && !walker_alive(g.mask, gm / g.mask_rows)) continue;
#pragma unroll
    for (int j = 0; j < TM; ++j) {
      int gn = n0 + TM * tx + j;
      if (gn >= g.n) continue;
      TC* c = C + (long)gm * g.ldc + gn;
      SUM v = SUM(g.alpha) * acc[i][j];
      if (g.beta != 0.0) v = fma(SUM(g.beta), SUM(*c), v);
      *c = TC(v);
    }
  }
}
}  // namespace

template <typename TA, typename TB, typename TC, typename ACC, bool SPLIT = false>
static int launch_gemm(const GemmNT<TA, TB, TC>& g, cudaStream_t st) {
  constexpr int BM = 64, BN = 64;
  if (g.m <= 0 || g.n <= 0 || g.batch <= 0) return AFQMC_OK;
  if (g.k < 0 || g.kb < 1) {
    set_error("gemm_nt: bad k=%d kb=%d", g.k, g.kb);
    return AFQMC_EINVAL;
  }
  if (g.mask && g.mask_rows <= 0) {
    set_error("gemm_nt: mask_rows must be positive");
    return AFQMC_EINVAL;
  }
  dim3 grid(cdiv(g.n, BN), cdiv(g.m, BM), g.batch);
  if (grid.y > 65535u || grid.z > 65535u) {
    set_error("gemm_nt: grid too large (m=%d batch=%d)", g.m, g.batch);
    return AFQMC_EINVAL;
  }
  // a product too small to give every SM a 64 x 64 tile (the M x M steps of
  // the set-up's exp) takes 32 x 32 tiles: four times the CTAs
  if ((long)grid.x * grid.y * grid.z < 152) {
    dim3 g2(cdiv(g.n, 32), cdiv(g.m, 32), g.batch);
    if (g2.y <= 65535u) {
      AFQ_LAUNCH((k_gemm_nt<TA, TB, TC, ACC, SPLIT, 2>), g2, TPB, 0, st, g);
      return AFQMC_OK;
    }
  }
  AFQ_LAUNCH((k_gemm_nt<TA, TB, TC, ACC, SPLIT, 4>), grid, TPB, 0, st, g);
  return AFQMC_OK;
}

int gemm_nt_f64(const GemmF64& g, cudaStream_t st) { return launch_gemm<double, double, double, double>(g, st); }
int gemm_nt_dff(const GemmNT<double, float, float>& g, cudaStream_t st) {
  return launch_gemm<double, float, float, float>(g, st);
}
int gemm_nt_ffd(const GemmNT<float, float, double>& g, cudaStream_t st) {
  return launch_gemm<float, float, double, float>(g, st);
}
int gemm_nt_ddf(const GemmNT<double, double, float>& g, cudaStream_t st) {
  return launch_gemm<double, double, float, float>(g, st);
}
int gemm_nt_fff(const GemmNT<float, float, float>& g, cudaStream_t st) {
  return launch_gemm<float, float, float, float>(g, st);
}
int gemm_nt_ffd_split(const GemmNT<float, float, double>& g, cudaStream_t st) {
  return launch_gemm<float, float, double, float, true>(g, st);
}
int gemm_nt_f32_split(const GemmF64& g, cudaStream_t st) {
  return launch_gemm<double, double, double, float, true>(g, st);
}

}  // namespace afq
