// Tensor-core (tcgen05) contraction launchers (internal header).
#pragma once

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
};

int tc_gemm_store(const TcGemm& g, float* C, long ldc, float alpha, cudaStream_t st);

// Exchange energy contraction (rows (g,i) of Lh, columns (w,c,j) of Theta^T)
// with the fused sum_ij T_ij T_ji epilogue; part [W][nchunk][2] (float64).
void exchange_tile(int N, int* RG, int* CW);
int tc_exchange(const TcGemm& g, int G, int W, int N, double* part, int nchunk, cudaStream_t st);

}  // namespace afq
