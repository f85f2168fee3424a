// Back-propagation estimators of ground-state properties (Sec. "Computing
// ground-state properties: the backpropagation algorithm", Eqs. bp1, bp,
// bp_dets), on the float64 and the mixed path.
//
// A window opened at step n (afqmc_bp_begin) keeps Psi_n of every walker and,
// at each later step, the shifted fields x = xi - xbar that built B(x) and the
// BP-PRes factor exp(-i dt Im E_loc(Psi_k)) / max(0, cos dtheta_k).  At step
// n + m (afqmc_bp_end) the trial is propagated backwards,
//     Phi_m = B^+(x_n) ... B^+(x_{n+m-1}) Psi_T,   B(x)^+ = B(-conj(x)),
// with the forward kernels (V assembly, half steps, Taylor terms, Gram-Schmidt;
// on the mixed path the tensor-core ones, fed the recorded operand-format
// fields with the real plane's sign flipped) fed the conjugated, negated
// fields; then, in float64, per walker
//     rho_w = 2 [Psi_n (Phi_m^H Psi_n)^-1 Phi_m^H]^T  (spin summed)
// and the weighted averages of Eq. bp with W_{n+m} prod_k factor_k (BP-PRes)
// and with W_{n+m} (BP-PhL).  The run's trial-adapted basis is rotated back
// at the end (rho = Q rho' Q^T).
#include "state.cuh"
#include "tc.cuh"

namespace afq {
namespace {

constexpr int kRhoTile = 32;
constexpr int kRhoK = 16;

// C = A B^T for M x M float64 matrices.
int gemm_sq_f64(const double* A, const double* B, double* C, int M, cudaStream_t st) {
  GemmF64 g;
  g.m = g.n = g.k = M;
  g.A = A;
  g.lda = M;
  g.B = B;
  g.ldb = M;
  g.C = C;
  g.ldc = M;
  return gemm_nt_f64(g, st);
}

__global__ void k_bp_fill(int W, double* f) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  f[2 * w] = 1.0;
  f[2 * w + 1] = 0.0;
}

// BP-PRes factor of one step: f *= exp(-i dt Im E_loc) / cos(dtheta); 0 for a
// walker the projection (or a non-finite weight) zeroed.
__global__ void k_bp_factor(int W, double dt, const double* wt, const double* eloc,
                            const double* cosd, double* f) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W) return;
  const double c = cosd[w];
  if (!walker_alive(wt, w) || !(c > 0.0)) {
    f[2 * w] = f[2 * w + 1] = 0.0;
    return;
  }
  double sn, cs;
  sincos(-dt * eloc[2 * w + 1], &sn, &cs);
  const double fr = f[2 * w], fi = f[2 * w + 1];
  f[2 * w] = (fr * cs - fi * sn) / c;
  f[2 * w + 1] = (fr * sn + fi * cs) / c;
}

// Psi_T in the trial-adapted basis: [I_N; 0] for every walker ([W][2][N][M]).
__global__ void k_bp_trial(long n, int N, int M, double* phi) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n;
       t += (long)gridDim.x * blockDim.x) {
    const long p = t % M;
    const long i = (t / M) % N;
    const long c = (t / ((long)M * N)) % 2;
    phi[t] = (c == 0 && p == i) ? 1.0 : 0.0;
  }
}

// Fields of B^+: -conj(x) = (-Re x, Im x), rows [W][2][G].
__global__ void k_bp_fields(long n, int G, const double* hist, double* x) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n;
       t += (long)gridDim.x * blockDim.x) {
    const bool re = ((t / G) & 1) == 0;
    x[t] = re ? -hist[t] : hist[t];
  }
}

// The same in the operand format (BF16, or TF32 in FP32 containers): the
// real plane's sign bit flipped (exact), rows [W][2][Gp].
__global__ void k_bp_fields_lo(long n, int Gp, int bytes, const void* hist, void* x) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n;
       t += (long)gridDim.x * blockDim.x) {
    const bool re = ((t / Gp) & 1) == 0;
    if (bytes == 2) {
      const uint16_t v = static_cast<const uint16_t*>(hist)[t];
      static_cast<uint16_t*>(x)[t] = re ? (uint16_t)(v ^ 0x8000u) : v;
    } else {
      const uint32_t v = static_cast<const uint32_t*>(hist)[t];
      static_cast<uint32_t*>(x)[t] = re ? (v ^ 0x80000000u) : v;
    }
  }
}

// dst row k = src row parent[k] (own row where the comb did nothing), rows
// of `words` 8-byte words.
__global__ void k_bp_gather(int W, long words, const int* parent, const uint64_t* src,
                            uint64_t* dst) {
  const int k = blockIdx.x;
  const int j = parent[k] < 0 ? k : parent[k];
  for (long t = threadIdx.x; t < words; t += blockDim.x) dst[k * words + t] = src[j * words + t];
}

__device__ inline double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Per walker: S = Phi^H Psi, S^-1 by Gauss-Jordan with partial pivoting
// (largest |s_rk|^2, first row on ties), Theta = Psi S^-1 scaled by
// a = 2 W f (thA) and 2 W (thB) as rows [2][N][M]; part = (W f, W).  A dead
// walker leaves zero rows in phi, thA and thB.
__global__ void __launch_bounds__(256)
    k_bp_theta(int W, int M, int N, double* phi, const double* psi, const double* wt,
               const double* f, double* thA, double* thB, double* part) {
  extern __shared__ double2 aug[];  // [N][2N]: [S | I] -> [I | S^-1]
  __shared__ double2 fac[64];
  __shared__ int prow;
  const int w = blockIdx.x;
  const long off = (long)w * 2 * N * M;
  const long NM = (long)N * M;
  double* ph = phi + off;
  const double* ps = psi + off;
  const int tid = threadIdx.x;
  if (!walker_alive(wt, w)) {
    for (long t = tid; t < 2 * NM; t += blockDim.x) ph[t] = thA[off + t] = thB[off + t] = 0.0;
    if (tid < 4) part[4 * w + tid] = 0.0;
    return;
  }
  const int N2 = 2 * N;
  for (int e = tid; e < N * N; e += blockDim.x) {
    const int i = e / N, j = e - (e / N) * N;
    double sr = 0.0, si = 0.0;
    for (int p = 0; p < M; ++p) {
      const double ar = ph[(long)i * M + p], ai = ph[NM + (long)i * M + p];
      const double br = ps[(long)j * M + p], bi = ps[NM + (long)j * M + p];
      sr += ar * br + ai * bi;
      si += ar * bi - ai * br;
    }
    aug[i * N2 + j] = make_double2(sr, si);
    aug[i * N2 + N + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (int k = 0; k < N; ++k) {
    if (tid == 0) {
      int r = k;
      double best = -1.0;
      for (int q = k; q < N; ++q) {
        const double2 v = aug[q * N2 + k];
        const double m2 = v.x * v.x + v.y * v.y;
        if (m2 > best) {
          best = m2;
          r = q;
        }
      }
      prow = r;
    }
    __syncthreads();
    const int r = prow;
    if (r != k) {
      for (int j = tid; j < N2; j += blockDim.x) {
        const double2 t = aug[k * N2 + j];
        aug[k * N2 + j] = aug[r * N2 + j];
        aug[r * N2 + j] = t;
      }
      __syncthreads();
    }
    const double2 pv = aug[k * N2 + k];
    const double den = pv.x * pv.x + pv.y * pv.y;
    const double2 inv = make_double2(pv.x / den, -pv.y / den);
    __syncthreads();
    for (int j = tid; j < N2; j += blockDim.x) aug[k * N2 + j] = cmul(aug[k * N2 + j], inv);
    if (tid < N) fac[tid] = aug[tid * N2 + k];
    __syncthreads();
    for (int e = tid; e < N * N2; e += blockDim.x) {
      const int q = e / N2, j = e - (e / N2) * N2;
      if (q == k) continue;
      const double2 a = fac[q], b = aug[k * N2 + j];
      double2 v = aug[q * N2 + j];
      v.x -= a.x * b.x - a.y * b.y;
      v.y -= a.x * b.y + a.y * b.x;
      aug[q * N2 + j] = v;
    }
    __syncthreads();
  }
  // weights: W (complex in free projection), a = 2 W f and 2 W
  const double2 wc = make_double2(wt[2 * w], wt[2 * w + 1]);
  const double2 wf = cmul(wc, make_double2(f[2 * w], f[2 * w + 1]));
  if (tid == 0) {
    part[4 * w] = wf.x;
    part[4 * w + 1] = wf.y;
    part[4 * w + 2] = wc.x;
    part[4 * w + 3] = wc.y;
  }
  const double2 aA = make_double2(2.0 * wf.x, 2.0 * wf.y), aB = make_double2(2.0 * wc.x, 2.0 * wc.y);
  // Theta[p][j] = sum_i Psi[p][i] S^-1[i][j]
  for (long e = tid; e < NM; e += blockDim.x) {
    const int j = (int)(e / M);
    const long p = e - (long)j * M;
    double tr = 0.0, ti = 0.0;
    for (int i = 0; i < N; ++i) {
      const double br = ps[(long)i * M + p], bi = ps[NM + (long)i * M + p];
      const double2 s = aug[i * N2 + N + j];
      tr += br * s.x - bi * s.y;
      ti += br * s.y + bi * s.x;
    }
    const double2 th = make_double2(tr, ti);
    const double2 ta = cmul(aA, th), tb = cmul(aB, th);
    thA[off + (long)j * M + p] = ta.x;
    thA[off + NM + (long)j * M + p] = ta.y;
    thB[off + (long)j * M + p] = tb.x;
    thB[off + NM + (long)j * M + p] = tb.y;
  }
}

// Partial sums over a slice of the rows k = (w, i) of
//   R[p][q] = sum_k conj(Phi_k[p]) Th_k[q]
// (R_re = sum Phr Thr + Phi Thi, R_im = sum Phr Thi - Phi Thr), one
// kRhoTile^2 tile per block, slice blockIdx.z of gridDim.z, into
// red[z][2][M][M].
__global__ void __launch_bounds__(256)
    k_bp_rho(int M, long K, long NM, int N, const double* __restrict__ phi,
             const double* __restrict__ th, double* __restrict__ red) {
  __shared__ double ar[kRhoK][kRhoTile], ai[kRhoK][kRhoTile];
  __shared__ double br[kRhoK][kRhoTile], bi[kRhoK][kRhoTile];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int p0 = blockIdx.y * kRhoTile, q0 = blockIdx.x * kRhoTile;
  const long k0 = K * blockIdx.z / gridDim.z, k1 = K * (blockIdx.z + 1) / gridDim.z;
  double rr[2][2] = {{0.0, 0.0}, {0.0, 0.0}}, ri[2][2] = {{0.0, 0.0}, {0.0, 0.0}};
  for (long kb = k0; kb < k1; kb += kRhoK) {
    for (int e = threadIdx.x; e < kRhoK * kRhoTile; e += blockDim.x) {
      const int kk = e / kRhoTile, c = e - kk * kRhoTile;
      const long k = kb + kk;
      double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
      if (k < k1) {
        const long w = k / N, i = k - (k / N) * N;
        const long base = w * 2 * NM + i * M;
        if (p0 + c < M) {
          v0 = phi[base + p0 + c];
          v1 = phi[base + NM + p0 + c];
        }
        if (q0 + c < M) {
          v2 = th[base + q0 + c];
          v3 = th[base + NM + q0 + c];
        }
      }
      ar[kk][c] = v0;
      ai[kk][c] = v1;
      br[kk][c] = v2;
      bi[kk][c] = v3;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kRhoK; ++kk) {
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const double a_r = ar[kk][ty * 2 + u], a_i = ai[kk][ty * 2 + u];
#pragma unroll
        for (int v = 0; v < 2; ++v) {
          const double b_r = br[kk][tx * 2 + v], b_i = bi[kk][tx * 2 + v];
          rr[u][v] = fma(a_r, b_r, fma(a_i, b_i, rr[u][v]));
          ri[u][v] = fma(a_r, b_i, fma(-a_i, b_r, ri[u][v]));
        }
      }
    }
    __syncthreads();
  }
  const long MM = (long)M * M;
  double* out = red + (long)blockIdx.z * 2 * MM;
#pragma unroll
  for (int u = 0; u < 2; ++u) {
    const int p = p0 + ty * 2 + u;
#pragma unroll
    for (int v = 0; v < 2; ++v) {
      const int q = q0 + tx * 2 + v;
      if (p < M && q < M) {
        out[(long)p * M + q] = rr[u][v];
        out[MM + (long)p * M + q] = ri[u][v];
      }
    }
  }
}

// Add the slices in order: R[c][p][q] = sum_z red[z][c][p][q].
__global__ void k_bp_reduce(long n, int Z, const double* red, double* R) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n;
       t += (long)gridDim.x * blockDim.x) {
    double s = red[t];
    for (int z = 1; z < Z; ++z) s += red[(long)z * n + t];
    R[t] = s;
  }
}

// Weight sums over the walkers in order: sums = (sum W f, sum W) re/im.
__global__ void k_bp_wsum(int W, const double* part, double* sums) {
  __shared__ double sh[32];
  for (int c = 0; c < 4; ++c) {
    double v = 0.0;
    for (int w = threadIdx.x; w < W; w += blockDim.x) v += part[4 * w + c];
    v = block_sum(v, sh);
    if (threadIdx.x == 0) sums[c] = v;
  }
}

// rho = R / A for the complex weight sum A = sums[off], sums[off + 1].
__global__ void k_bp_scale(long MM, const double* R, const double* sums, int off, double* rho) {
  const double ar = sums[off], ai = sums[off + 1];
  const double den = ar * ar + ai * ai;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < MM;
       t += (long)gridDim.x * blockDim.x) {
    const double xr = R[t], xi = R[MM + t];
    rho[t] = (xr * ar + xi * ai) / den;
    rho[MM + t] = (xi * ar - xr * ai) / den;
  }
}

}  // namespace

// Bytes of one step's recorded fields, and where they come from.
size_t bp_field_bytes(const afqmc_params& p, const Bufs& b) {
  return b.mixed ? (size_t)p.nwalkers * 2 * b.Gp * b.lo_bytes
                 : (size_t)p.nwalkers * 2 * p.nchol * sizeof(double);
}

int bp_record_fields(afqmc_state* s) {
  const Bufs& b = s->b;
  const size_t n = bp_field_bytes(s->p, b);
  char* dst = reinterpret_cast<char*>(b.bp_hist) + (size_t)s->bp_m * n;
  AFQ_CUDA(cudaMemcpyAsync(dst, b.mixed ? b.x_lo : static_cast<const void*>(b.x), n,
                           cudaMemcpyDeviceToDevice, s->st));
  return AFQMC_OK;
}

// After a comb inside the window: every copy takes its parent's Psi_n,
// restoration factor and recorded fields (rows gathered by the comb's parent
// index through a scratch buffer).
int bp_after_comb(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers;
  auto gather = [&](void* buf, size_t row_bytes) -> int {
    const long words = (long)(row_bytes / 8);
    AFQ_LAUNCH(k_bp_gather, W, 256, 0, s->st, W, words, b.parent,
               static_cast<const uint64_t*>(buf), reinterpret_cast<uint64_t*>(b.bp_tmp));
    AFQ_CUDA(cudaMemcpyAsync(buf, b.bp_tmp, row_bytes * W, cudaMemcpyDeviceToDevice, s->st));
    return AFQMC_OK;
  };
  AFQ_TRY(gather(b.bp_psi, sizeof(double) * 2 * (size_t)p.N * p.M));
  AFQ_TRY(gather(b.bp_f, sizeof(double) * 2));
  const size_t fbytes = bp_field_bytes(p, b);
  for (int k = 0; k < s->bp_m; ++k)
    AFQ_TRY(gather(reinterpret_cast<char*>(b.bp_hist) + (size_t)k * fbytes, fbytes / W));
  return AFQMC_OK;
}

int bp_step_factor(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  if (p.mode == AFQMC_PHASELESS)
    AFQ_LAUNCH(k_bp_factor, cdiv(p.nwalkers, 128), 128, 0, s->st, p.nwalkers, p.dt, b.wt, b.eloc,
               b.bp_cos, b.bp_f);
  return AFQMC_OK;
}

int bp_open(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  AFQ_CUDA(cudaMemcpyAsync(b.bp_psi, b.phiT, sizeof(double) * (size_t)p.nwalkers * 2 * p.N * p.M,
                           cudaMemcpyDeviceToDevice, s->st));
  AFQ_LAUNCH(k_bp_fill, cdiv(p.nwalkers, 128), 128, 0, s->st, p.nwalkers, b.bp_f);
  s->bp_on = true;
  s->bp_m = 0;
  return AFQMC_OK;
}

// Backward sweep, estimators and the rotation to the caller's basis; results
// (rho BP-PRes, rho BP-PhL as [2][M][M] re/im planes, weight sums) on the device.
int bp_close(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, N = p.N, M = p.M, G = p.nchol;
  const long NM = (long)N * M, MM = (long)M * M;
  cudaStream_t st = s->st;
  s->bp_on = false;
  AFQ_LAUNCH(k_bp_trial, cdiv((size_t)W * 2 * NM, 256), 256, 0, st, (long)W * 2 * NM, N, M,
             b.bp_phi);
  if (b.mixed)
    AFQ_TRY(launch_convert_lo(b.bp_phi, 2L * N * W, M, M, b.bp_phi_lo, b.Mp, b.lo_kind, st));
  const size_t fbytes = bp_field_bytes(p, b);
  for (int k = s->bp_m - 1, done = 1; k >= 0; --k, ++done) {
    const char* hk = reinterpret_cast<const char*>(b.bp_hist) + (size_t)k * fbytes;
    // the fields of B^+ (-conj x), then Phi <- B_half T_n(V) B_half Phi
    if (b.mixed) {
      const long nx = (long)W * 2 * b.Gp;
      AFQ_LAUNCH(k_bp_fields_lo, cdiv(nx, 256), 256, 0, st, nx, b.Gp, b.lo_bytes, hk, b.x_lo);
      AFQ_TRY(apply_b_mixed(s, b.bp_phi, b.bp_phi_lo, b.bp_phi, b.bp_phi_lo));
    } else {
      const long nx = (long)W * 2 * G;
      AFQ_LAUNCH(k_bp_fields, cdiv(nx, 256), 256, 0, st, nx, G,
                 reinterpret_cast<const double*>(hk), b.x);
      AFQ_TRY(apply_b_f64(s, b.bp_phi, b.bp_phi, nullptr));
    }
    if (p.qr_period && done % p.qr_period == 0) {
      MgsArgs ma{W, M, N, b.bp_phi, b.wt, b.tmp_ld};
      AFQ_TRY(launch_mgs(ma, st));
      if (b.mixed)
        AFQ_TRY(launch_convert_lo(b.bp_phi, 2L * N * W, M, M, b.bp_phi_lo, b.Mp, b.lo_kind, st));
    }
  }
  // per-walker (Phi^H Psi)^-1 and the scaled Theta rows (T0: BP-PRes, T1: BP-PhL)
  const size_t smem = sizeof(double2) * (size_t)N * 2 * N;
  AFQ_CUDA(cudaFuncSetAttribute(k_bp_theta, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  AFQ_LAUNCH(k_bp_theta, W, 256, smem, st, W, M, N, b.bp_phi, b.bp_psi, b.wt, b.bp_f, b.T0, b.T1,
             b.bp_part);
  AFQ_LAUNCH(k_bp_wsum, 1, 256, 0, st, W, b.bp_part, b.bp_out + 4 * MM);
  const long K = (long)W * N;
  const int tiles = (int)cdiv(M, kRhoTile);
  int Z = (int)((4L * tc_sm_count() + tiles * tiles - 1) / (tiles * tiles));
  if (Z > kBpSlices) Z = kBpSlices;
  if (Z > K / kRhoK) Z = (int)(K / kRhoK);
  if (Z < 1) Z = 1;
  for (int e = 0; e < 2; ++e) {
    const double* th = e == 0 ? b.T0 : b.T1;
    AFQ_LAUNCH(k_bp_rho, dim3(tiles, tiles, Z), 256, 0, st, M, K, NM, N, b.bp_phi, th, b.bp_red);
    AFQ_LAUNCH(k_bp_reduce, cdiv(2 * MM, 256), 256, 0, st, 2 * MM, Z, b.bp_red, b.bp_R);
    // rho = Q R Q^T for each plane: Y = Q R^T, then Q Y^T
    for (int c = 0; c < 2; ++c) {
      AFQ_TRY(gemm_sq_f64(b.Qb, b.bp_R + c * MM, b.bp_red, M, st));
      AFQ_TRY(gemm_sq_f64(b.Qb, b.bp_red, b.bp_R + 2 * MM + c * MM, M, st));
    }
    AFQ_LAUNCH(k_bp_scale, cdiv(MM, 256), 256, 0, st, MM, b.bp_R + 2 * MM, b.bp_out + 4 * MM,
               2 * e, b.bp_out + e * 2 * MM);
  }
  return AFQMC_OK;
}

}  // namespace afq
