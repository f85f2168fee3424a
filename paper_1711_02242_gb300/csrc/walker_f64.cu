// Per-walker kernels (float64, and the FP32 variants of the overlap, Theta and
// Gram-Schmidt kernels used by the mixed path's _F32LU precisions) and the
// set-up kernels.
//
// Layouts (W walkers, M orbitals, N electrons per spin, G Cholesky vectors,
// P = M(M+1)/2):
//   phiT, thetaT [W][2][N][M]  orbital-major walkers (re plane, im plane)
//   t, x         [W][2][G]     force-bias traces / shifted fields
//   Y            [W][2][P]     packed sum_g x_g L_g (upper triangle, row-major)
//   weights      [W][2]        (re, im); phaseless walks keep im = 0
#include "kernels.cuh"

namespace afq {

__host__ __device__ inline long packed_index(int p, int q, int M) {
  // p <= q: rows of the upper triangle stored one after another
  return (long)p * M - (long)p * (p - 1) / 2 + (q - p);
}

// ------------------------------------------------------------------ fields --
// Force bias (Eq. fb with the mean-field background of Sec. 2.4):
// xbar_g = -i sqrt(dt) (t_g - c_g), t_g = 2 Tr(Lh_g Theta); magnitude capped
// at fb_cap with the phase kept (Appendix B).  Fields xi_g ~ N(0,1) from
// Philox; x = xi - xbar.  Per-walker sums for the weight: sum xi xbar,
// sum xbar^2 (Eq. hybrid-wt) and sum x c (the scalar of B(x - xbar)).
__global__ void __launch_bounds__(256) k_field(FieldArgs a) {
  __shared__ double sh[32];
  const int w = blockIdx.x;
  const bool alive = walker_alive(a.wt, w);
  double s0 = 0, s1 = 0, s2 = 0, s3 = 0, s4 = 0, s5 = 0;
  const long base = (long)w * 2 * a.G;
  const double* tr = a.t ? a.t + base : nullptr;
  const double* ti = tr ? tr + a.G : nullptr;
  const float* tr32 = a.t32 ? a.t32 + base : nullptr;
  const float* ti32 = tr32 ? tr32 + a.G : nullptr;
  double* xr = a.x ? a.x + base : nullptr;
  double* xim = xr ? xr + a.G : nullptr;
  const long xl = (long)w * 2 * a.Gp;
  const int npair = (a.G + 1) / 2;
  for (int k = threadIdx.x; k < npair; k += blockDim.x) {
    double xa, xb;
    if (a.x_lo)
      field_pair_f32(a.seed, (uint32_t)*a.dstep, (uint32_t)(a.w0 + w), (uint32_t)k, &xa, &xb);
    else
      field_pair(a.seed, (uint32_t)*a.dstep, (uint32_t)(a.w0 + w), (uint32_t)k, &xa, &xb);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = 2 * k + h;
      if (g >= a.G) break;
      const double xi = h ? xb : xa;
      double br = 0.0, bi = 0.0;
      if (a.mode == AFQMC_PHASELESS) {
        const double tre = tr32 ? (double)tr32[g] : tr[g];
        const double tim = ti32 ? (double)ti32[g] : ti[g];
        br = a.sdt * tim;
        bi = -a.sdt * (tre - a.c[g]);
        if (a.fb_cap > 0.0) {
          const double mag = hypot(br, bi);
          if (mag > a.fb_cap) {
            const double f = a.fb_cap / mag;
            br *= f;
            bi *= f;
          }
        }
      }
      double vr = xi - br, vi = -bi;
      if (!alive) vr = vi = 0.0;
      if (xr) {
        xr[g] = vr;
        xim[g] = vi;
      }
      if (a.x_lo) {
        store_lo(a.x_lo, a.lo_kind, xl + g, vr);
        store_lo(a.x_lo, a.lo_kind, xl + a.Gp + g, vi);
      }
      s0 += xi * br;
      s1 += xi * bi;
      s2 += br * br - bi * bi;
      s3 += 2.0 * br * bi;
      s4 += a.c[g] * vr;
      s5 += a.c[g] * vi;
    }
  }
  double r;
  r = block_sum(s0, sh); if (threadIdx.x == 0) a.scal[8L * w + 0] = r;
  r = block_sum(s1, sh); if (threadIdx.x == 0) a.scal[8L * w + 1] = r;
  r = block_sum(s2, sh); if (threadIdx.x == 0) a.scal[8L * w + 2] = r;
  r = block_sum(s3, sh); if (threadIdx.x == 0) a.scal[8L * w + 3] = r;
  r = block_sum(s4, sh); if (threadIdx.x == 0) a.scal[8L * w + 4] = r;
  r = block_sum(s5, sh); if (threadIdx.x == 0) a.scal[8L * w + 5] = r;
}

// Mixed path: the same fields, force bias and sums with the force bias taken
// in FP32 (t comes from an FP32 accumulator and x only feeds the BF16/TF32
// V contraction; float64 hypot and division run on GB300's slow FP64 pipe).
// Each thread sums its fields in FP32; the six per-walker sums are reduced in
// float64 in a fixed order (warps, then the block's warps in turn).
__global__ void __launch_bounds__(256) k_field_lo(FieldArgs a) {
  __shared__ double sh[8][6];
  const int w = blockIdx.x;
  const bool alive = walker_alive(a.wt, w);
  const long base = (long)w * 2 * a.G;
  const float* tr = a.t32 + base;
  const float* ti = tr + a.G;
  const long xl = (long)w * 2 * a.Gp;
  const float sdt = (float)a.sdt, cap = (float)a.fb_cap;
  const bool phaseless = a.mode == AFQMC_PHASELESS;
  const uint32_t step = (uint32_t)*a.dstep;
  float s[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const int npair = (a.G + 1) / 2;
  for (int k = threadIdx.x; k < npair; k += blockDim.x) {
    double xa, xb;
    field_pair_f32(a.seed, step, (uint32_t)(a.w0 + w), (uint32_t)k, &xa, &xb);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int g = 2 * k + h;
      if (g >= a.G) break;
      const float xi = (float)(h ? xb : xa);
      const float cg = (float)a.c[g];
      float br = 0.f, bi = 0.f;
      if (phaseless) {
        br = sdt * ti[g];
        bi = -sdt * (tr[g] - cg);
        if (cap > 0.f) {
          const float mag = hypotf(br, bi);
          if (mag > cap) {
            const float f = cap / mag;
            br *= f;
            bi *= f;
          }
        }
      }
      float vr = xi - br, vi = -bi;
      if (!alive) vr = vi = 0.f;
      store_lo_f(a.x_lo, a.lo_kind, xl + g, vr);
      store_lo_f(a.x_lo, a.lo_kind, xl + a.Gp + g, vi);
      s[0] = fmaf(xi, br, s[0]);
      s[1] = fmaf(xi, bi, s[1]);
      s[2] += br * br - bi * bi;
      s[3] += 2.f * br * bi;
      s[4] = fmaf(cg, vr, s[4]);
      s[5] = fmaf(cg, vi, s[5]);
    }
  }
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    const double d = warp_sum((double)s[i]);
    if (lane == 0) sh[wid][i] = d;
  }
  __syncthreads();
  if (threadIdx.x < 6) {
    double r = 0.0;
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) r += sh[q][threadIdx.x];
    a.scal[8L * w + threadIdx.x] = r;
  }
}

int launch_field(const FieldArgs& a, cudaStream_t st) {
  if (a.x_lo && a.t32 && !a.x && !a.t) {
    AFQ_LAUNCH(k_field_lo, a.W, 256, 0, st, a);
  } else {
    AFQ_LAUNCH(k_field, a.W, 256, 0, st, a);
  }
  return AFQMC_OK;
}

// ------------------------------------------------------------ Taylor term --
// One term of the truncated series T_n(V) Phi = sum_k V^k Phi / k!
// (Sec. 3.4.2): out = V * in / k with V = i sqrt(dt) sum_g x_g L_g complex
// symmetric, read from the packed Y = sum_g x_g L_g as
// V = sqrt(dt) (-Im Y + i Re Y).  In transposed storage out^T = in^T V.
namespace {
constexpr int TT_P = 64, TT_Q = 16, TT_NMAX = 64;
}
template <typename T>
__global__ void __launch_bounds__(256) k_taylor_term(TaylorArgsT<T> a) {
  __shared__ T Ys[2][TT_Q][TT_P];
  __shared__ T Ts[2][TT_NMAX][TT_Q + 1];
  // every walker is computed (the work does not depend on the weights); the
  // result of a dead walker is never stored into its orbitals
  const int w = blockIdx.y;
  const int p0 = blockIdx.x * TT_P;
  const int tx = threadIdx.x % TT_P, ty = threadIdx.x / TT_P;  // 4 rows of i
  const int M = a.M, N = a.N;
  const T* Yr = a.Y + (long)w * 2 * a.ldy;
  const T* Yi = Yr + a.ldy;
  const long wo = (long)w * 2 * N * M;
  const T* tin = a.tin + wo;
  T accR[TT_NMAX / 4], accI[TT_NMAX / 4];
#pragma unroll
  for (int r = 0; r < TT_NMAX / 4; ++r) accR[r] = accI[r] = T(0);
  for (int q0 = 0; q0 < M; q0 += TT_Q) {
    for (int idx = threadIdx.x; idx < TT_Q * TT_P; idx += blockDim.x) {
      const int qq = idx / TT_P, pp = idx % TT_P;
      const int q = q0 + qq, p = p0 + pp;
      T vr = T(0), vi = T(0);
      if (q < M && p < M) {
        const long id = (q <= p) ? packed_index(q, p, M) : packed_index(p, q, M);
        vr = Yr[id];
        vi = Yi[id];
      }
      Ys[0][qq][pp] = vr;
      Ys[1][qq][pp] = vi;
    }
    for (int idx = threadIdx.x; idx < 2 * N * TT_Q; idx += blockDim.x) {
      const int c = idx / (N * TT_Q), rem = idx % (N * TT_Q);
      const int i = rem / TT_Q, qq = rem % TT_Q;
      const int q = q0 + qq;
      Ts[c][i][qq] = (q < M) ? tin[((long)c * N + i) * M + q] : T(0);
    }
    __syncthreads();
#pragma unroll 4
    for (int qq = 0; qq < TT_Q; ++qq) {
      const T yr = Ys[0][qq][tx], yi = Ys[1][qq][tx];
#pragma unroll
      for (int r = 0; r < TT_NMAX / 4; ++r) {
        const int i = ty + 4 * r;
        if (i < N) {
          const T tr = Ts[0][i][qq], ti = Ts[1][i][qq];
          accR[r] = fma(tr, yi, fma(ti, yr, accR[r]));
          accI[r] = fma(tr, yr, fma(-ti, yi, accI[r]));
        }
      }
    }
    __syncthreads();
  }
  const int p = p0 + tx;
  if (p >= M) return;
#pragma unroll
  for (int r = 0; r < TT_NMAX / 4; ++r) {
    const int i = ty + 4 * r;
    if (i >= N) break;
    const T oR = -T(a.scale) * accR[r], oI = T(a.scale) * accI[r];
    const long o0 = wo + (long)i * M + p, o1 = wo + ((long)N + i) * M + p;
    a.tout[o0] = oR;
    a.tout[o1] = oI;
    if (a.k == 1) {
      a.acc[o0] = tin[(long)i * M + p] + oR;
      a.acc[o1] = tin[((long)N + i) * M + p] + oI;
    } else {
      a.acc[o0] += oR;
      a.acc[o1] += oI;
    }
  }
}

template <typename T>
static int launch_taylor(const TaylorArgsT<T>& a, cudaStream_t st) {
  if (a.N > TT_NMAX) {
    set_error("taylor: N=%d above the supported %d", a.N, TT_NMAX);
    return AFQMC_EUNSUPPORTED;
  }
  dim3 grid(cdiv(a.M, TT_P), a.W);
  AFQ_LAUNCH(k_taylor_term<T>, grid, 256, 0, st, a);
  return AFQMC_OK;
}
int launch_taylor_term(const TaylorArgsT<double>& a, cudaStream_t st) { return launch_taylor(a, st); }

// ------------------------------------------------------------- overlap ------
// Theorem 1.1, Eq. precomputing, in the trial-adapted basis where V_T =
// [I_N; 0]; float64 on the float64 path, FP32 with float64 log det sums on
// the _F32LU mixed precisions (k_overlap<float>, k_theta_rows_f32).  k_overlap, one block
// per walker:
//   1. S = V_T^T Phi is the top N x N block of Phi (a gather);
//   2. Gauss-Jordan elimination with partial pivoting (largest |s_rk|^2, the
//      first row on ties, searched by one warp): S^-1 and log det S = sum log
//      p_k (+ i pi per row swap), S^-1 written for k_theta_rows;
// then k_theta_rows forms Theta^T[i][p] = sum_j S^-1[j][i] Phi^T[j][p].
// log <Psi_T|Psi> = 2 log det S (both spins), phase wrapped to (-pi, pi].
// With two spin blocks (a float64 run whose spin-down trial differs from the
// spin-up one) S is the block-diagonal product V_T^T Phi instead of a gather,
// and log <Psi_T|Psi> = log det S_up + log det S_dn.
// Every walker is computed; S^-1 and log det are stored for live walkers.
namespace {
constexpr int OV_T = 256;
}
// Element traits of the overlap kernel: float64; FP32 for the _F32LU mixed
// precisions, whose orbitals carry BF16/TF32 propagation errors far above
// FP32 rounding (the log det sums stay float64).
template <typename T>
struct Vec2;
template <>
struct Vec2<double> {
  using type = double2;
  __device__ static double2 make(double x, double y) { return make_double2(x, y); }
  __device__ static double from_f64(double x) { return x; }
  __device__ static double to_f64(double x) { return x; }
  __device__ static double2* sinv(const OverlapArgs& a) { return a.Sinv; }
};
template <>
struct Vec2<float> {
  using type = float2;
  __device__ static float2 make(float x, float y) { return make_float2(x, y); }
  __device__ static float from_f64(double x) { return f64_to_f32(x); }
  __device__ static double to_f64(float x) { return f32_to_f64(x); }
  __device__ static float2* sinv(const OverlapArgs& a) { return a.Sinv32; }
};

// Steps 1-2 for walker w by the whole block (blockDim >= 64): S into A
// ([N][N] shared), its inverse in place with the columns in the rows' final
// order (pos[c] = the column of A holding column c of S^-1), log det stored
// for live walkers.  Returns true when S is singular (block-uniform).
template <typename T>
__device__ __forceinline__ bool overlap_core(const OverlapArgs& a, int w, bool live,
                                             typename Vec2<T>::type* A, int* pos) {
  using T2 = typename Vec2<T>::type;
  __shared__ __align__(16) unsigned char misc_raw[sizeof(T2) * 129];
  const int N = a.N, M = a.M;
  __shared__ int swaps, singular;
  T2& rpiv = reinterpret_cast<T2*>(misc_raw)[128];
  T2* pivots = reinterpret_cast<T2*>(misc_raw);       // the pivots, for log det afterwards
  T2* fac = reinterpret_cast<T2*>(misc_raw) + 64;     // a_rk / p of the current pivot column
  __shared__ int order[64];
  const double* fr = a.phiT + (long)w * 2 * N * M;
  const double* fi = fr + (long)N * M;
  if (a.unit_trial) {
    // S[i][j] = Phi[i][j], the top block of the orbitals
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int i = idx / N, j = idx % N;
      A[idx] = Vec2<T>::make(Vec2<T>::from_f64(fr[(long)j * M + i]),
                             Vec2<T>::from_f64(fi[(long)j * M + i]));
    }
  } else {
    // two spin blocks: S = blockdiag(V_up^T Phi_up, V_dn^T Phi_dn), zero
    // between the blocks, so that the elimination below never pivots across
    // them and its pivots give det S_up det S_dn (Theorem 1.1)
    const int nup = a.nup > 0 ? a.nup : N;
    for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
      const int i = idx / N, j = idx % N;
      double sr = 0.0, si = 0.0;
      if ((i < nup) == (j < nup)) {
        const double* v = a.VTt + (long)i * M;
        for (int p = 0; p < M; ++p) {
          sr = fma(v[p], fr[(long)j * M + p], sr);
          si = fma(v[p], fi[(long)j * M + p], si);
        }
      }
      A[idx] = Vec2<T>::make(Vec2<T>::from_f64(sr), Vec2<T>::from_f64(si));
    }
  }
  if (threadIdx.x < N) order[threadIdx.x] = threadIdx.x;
  if (threadIdx.x == 0) {
    swaps = 0;
    singular = 0;
  }
  __syncthreads();
  // In-place Gauss-Jordan with partial pivoting: at pivot k (after the row
  // swap), with p = a_kk, a_ij -= a_ik a_kj / p (i, j != k), then
  // a_kj /= p, a_ik = -a_ik / p, a_kk = 1 / p: (N - 1)^2 updates per pivot.
  // Warp 0 picks the pivot, swaps the rows, takes 1 / p once and the factors
  // a_rk / p.  The row interchanges leave the inverse with its columns in the
  // rows' final order, undone when it is stored.
  for (int k = 0; k < N; ++k) {
    if (threadIdx.x < 32) {
      // pivot: the largest |a_rk|^2 over rows r >= k, the first such row on ties
      int best = k;
      T bv = -1;
      for (int r = k + threadIdx.x; r < N; r += 32) {
        const T2 x = A[r * N + k];
        const T v = x.x * x.x + x.y * x.y;
        if (v > bv) {
          bv = v;
          best = r;
        }
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const T ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int ob = __shfl_xor_sync(0xffffffffu, best, o);
        if (ov > bv || (ov == bv && ob < best)) {
          bv = ov;
          best = ob;
        }
      }
      if (bv > 0) {
        if (best != k) {
          for (int j = threadIdx.x; j < N; j += 32) {
            const T2 t = A[k * N + j];
            A[k * N + j] = A[best * N + j];
            A[best * N + j] = t;
          }
          if (threadIdx.x == 0) {
            const int t = order[k];
            order[k] = order[best];
            order[best] = t;
            swaps++;
          }
          __syncwarp();
        }
        // 1 / pivot once per lane (a float64 division runs long on the FP64 pipe)
        const T2 pv = A[k * N + k];
        const T den = pv.x * pv.x + pv.y * pv.y;
        const T2 rp = Vec2<T>::make(pv.x / den, -pv.y / den);
        for (int r = threadIdx.x; r < N; r += 32) {
          const T2 x = A[r * N + k];
          fac[r] = Vec2<T>::make(x.x * rp.x - x.y * rp.y, x.x * rp.y + x.y * rp.x);
        }
        if (threadIdx.x == 0) {
          rpiv = rp;
          pivots[k] = pv;
        }
      } else if (threadIdx.x == 0) {
        singular = 1;
      }
    }
    __syncthreads();
    if (singular) break;
    // a_ij -= (a_ik / p) a_kj for i, j != k
    const int n1 = N - 1;
    for (int idx = threadIdx.x; idx < n1 * n1; idx += blockDim.x) {
      const int ii = idx / n1, jj = idx - (idx / n1) * n1;
      const int i = ii < k ? ii : ii + 1, j = jj < k ? jj : jj + 1;
      const T2 f = fac[i], v = A[k * N + j];
      T2& d = A[i * N + j];
      d.x = fma(-f.x, v.x, fma(f.y, v.y, d.x));
      d.y = fma(-f.x, v.y, fma(-f.y, v.x, d.y));
    }
    __syncthreads();
    // pivot row / p, pivot column -a_ik / p, a_kk = 1 / p
    const T2 rp = rpiv;
    for (int t = threadIdx.x; t < 2 * N - 1; t += blockDim.x) {
      if (t < N) {
        T2& d = A[k * N + t];
        if (t == k) {
          d = rp;
        } else {
          const T2 v = d;
          d = Vec2<T>::make(v.x * rp.x - v.y * rp.y, v.x * rp.y + v.y * rp.x);
        }
      } else {
        const int i = t - N < k ? t - N : t - N + 1;
        A[i * N + k] = Vec2<T>::make(-fac[i].x, -fac[i].y);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < N) pos[order[threadIdx.x]] = threadIdx.x;
  // log det = sum_k log |p_k| + i (sum_k arg p_k + pi swaps), the N logs and
  // phases in parallel, summed in a fixed order (warps 0 and 1: N <= 64)
  // (float64 logs of the pivots also on the FP32 path: N per walker)
  double la = 0.0, ph = 0.0;
  if (!singular && threadIdx.x < N) {
    const double px = Vec2<T>::to_f64(pivots[threadIdx.x].x);
    const double py = Vec2<T>::to_f64(pivots[threadIdx.x].y);
    la = 0.5 * log(px * px + py * py);
    ph = atan2(py, px);
  }
  __shared__ double red[4];
  if (threadIdx.x < 64) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      la += __shfl_xor_sync(0xffffffffu, la, o);
      ph += __shfl_xor_sync(0xffffffffu, ph, o);
    }
    if ((threadIdx.x & 31) == 0) {
      red[2 * (threadIdx.x >> 5)] = la;
      red[2 * (threadIdx.x >> 5) + 1] = ph;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0 && live) {
    if (singular) {
      a.logdet[2L * w] = -INFINITY;
      a.logdet[2L * w + 1] = 0.0;
    } else {
      a.logdet[2L * w] = a.sf * (red[0] + red[2]);
      a.logdet[2L * w + 1] = wrap_pi(a.sf * ((red[1] + red[3]) + 3.141592653589793 * swaps));
    }
  }
  return singular != 0;
}

template <typename T>
__global__ void __launch_bounds__(OV_T) k_overlap(OverlapArgs a) {
  using T2 = typename Vec2<T>::type;
  extern __shared__ __align__(16) unsigned char ov_raw[];
  __shared__ int pos[64];
  const int w = blockIdx.x, N = a.N;
  const bool live = !a.wt || walker_alive(a.wt, w);
  T2* A = reinterpret_cast<T2*>(ov_raw);  // [N][N], inverted in place
  const bool singular = overlap_core<T>(a, w, live, A, pos);
  // S^-1 of live, non-singular walkers for the Theta kernel: column c of the
  // inverse is column pos[c] of A (the row interchanges undone)
  if (singular || !live) return;
  T2* si = Vec2<T>::sinv(a) + (long)w * N * N;
  for (int idx = threadIdx.x; idx < N * N; idx += blockDim.x) {
    const int r = idx / N, c = idx - (idx / N) * N;
    si[idx] = A[r * N + pos[c]];
  }
}

// Theta^T[i][p] = sum_j S^-1[j][i] Phi^T[j][p]: block (x, w) takes rows
// p in [x TH_P, (x + 1) TH_P) of walker w in work items (p, block of IB
// orbitals i), IB the largest divisor of N up to 8 (no padded lanes), so the
// FP64 work of all walkers spreads evenly over the SMs.  With V_T = [I_N; 0]
// rows p < N are rows of S S^-1 = I.  Dead and singular walkers keep Theta.
namespace {
constexpr int TH_P = 64, TH_T = 128;
}
template <int IB>
__global__ void __launch_bounds__(TH_T) k_theta_rows(OverlapArgs a) {
  extern __shared__ double2 th_sinv[];  // [N][N]
  const int w = blockIdx.y, N = a.N, M = a.M;
  if ((a.wt && !walker_alive(a.wt, w)) || !(a.logdet[2L * w] > -INFINITY)) return;
  const double2* si = a.Sinv + (long)w * N * N;
  for (int idx = threadIdx.x; idx < N * N; idx += TH_T) th_sinv[idx] = si[idx];
  __syncthreads();
  const double* fr = a.phiT + (long)w * 2 * N * M;
  const double* fi = fr + (long)N * M;
  double* tr = a.thetaT + (long)w * 2 * N * M;
  double* ti = tr + (long)N * M;
  const int pb = blockIdx.x * TH_P, pe = min(M, pb + TH_P), np = pe - pb, nib = N / IB;
  for (int item = threadIdx.x; item < np * nib; item += TH_T) {
    const int p = pb + item % np, i0 = (item / np) * IB;
    double ar[IB], ai[IB];
#pragma unroll
    for (int u = 0; u < IB; ++u) ar[u] = ai[u] = 0.0;
    if (a.unit_trial && p < N) {
#pragma unroll
      for (int u = 0; u < IB; ++u) ar[u] = (i0 + u == p) ? 1.0 : 0.0;
    } else {
      for (int j = 0; j < N; ++j) {
        const double xr = fr[(long)j * M + p], xi = fi[(long)j * M + p];
#pragma unroll
        for (int u = 0; u < IB; ++u) {
          const double2 sv = th_sinv[j * N + i0 + u];
          ar[u] = fma(xr, sv.x, fma(-xi, sv.y, ar[u]));
          ai[u] = fma(xr, sv.y, fma(xi, sv.x, ai[u]));
        }
      }
    }
#pragma unroll
    for (int u = 0; u < IB; ++u) {
      const int i = i0 + u;
      tr[(long)i * M + p] = ar[u];
      ti[(long)i * M + p] = ai[u];
      if (a.th_lo) {
        store_lo(a.th_lo, a.lo_kind, ((long)w * 2 * N + i) * a.Mp + p, ar[u]);
        store_lo(a.th_lo, a.lo_kind, ((long)w * 2 * N + N + i) * a.Mp + p, ai[u]);
      }
    }
  }
}

// Mixed precisions: the same rows with FP32 arithmetic.  Theta only feeds the
// BF16/TF32 contractions (force bias, exchange) and the one-body energy
// there, so FP32 products (S^-1 and Phi rounded to FP32) lose nothing those do
// not, and this GPU's FP32 pipe is ~60x its FP64 one: the kernel becomes bound
// by the traffic of Phi and Theta.  S^-1 comes from the float64 elimination
// (rounded once to FP32 here), or from the FP32 one of the _F32LU precisions.  The block's TH_P columns of Phi are staged
// in shared memory as FP32 (all loads in flight at once, converted once);
// one work item = row p and IB orbitals i, IB = N / ceil(N / 16) rounded up
// (guarded tail of at most ceil(N / 16) - 1 lanes); S^-1 reads are warp-wide
// broadcasts.  Conversions use the integer-pipe routines.
template <int TF_IB>
__global__ void __launch_bounds__(TH_T) k_theta_rows_f32(OverlapArgs a) {
  extern __shared__ float2 th_sinv32[];  // [N][N], then Phi [2][N][TH_P] (FP32)
  const int w = blockIdx.y, N = a.N, M = a.M;
  if ((a.wt && !walker_alive(a.wt, w)) || !(a.logdet[2L * w] > -INFINITY)) return;
  float* ph = reinterpret_cast<float*>(th_sinv32 + N * N);
  if (a.Sinv32) {
    const float2* si = a.Sinv32 + (long)w * N * N;
    for (int idx = threadIdx.x; idx < N * N; idx += TH_T) th_sinv32[idx] = si[idx];
  } else {
    const double2* si = a.Sinv + (long)w * N * N;
    for (int idx = threadIdx.x; idx < N * N; idx += TH_T) {
      const double2 v = si[idx];
      th_sinv32[idx] = make_float2(f64_to_f32(v.x), f64_to_f32(v.y));
    }
  }
  const double* phw = a.phiT + (long)w * 2 * N * M;
  const int pb = blockIdx.x * TH_P, pe = min(M, pb + TH_P), np = pe - pb;
#pragma unroll 4
  for (int e = threadIdx.x; e < 2 * N * np; e += TH_T) {
    const int row = e / np, pl = e - row * np;  // row = plane * N + j
    ph[row * TH_P + pl] = f64_to_f32(phw[(long)row * M + pb + pl]);
  }
  __syncthreads();
  double* tr = a.thetaT + (long)w * 2 * N * M;
  double* ti = tr + (long)N * M;
  const int nib = (N + TF_IB - 1) / TF_IB;
  for (int item = threadIdx.x; item < np * nib; item += TH_T) {
    const int pl = item % np, p = pb + pl, i0 = (item / np) * TF_IB;
    float ar[TF_IB], ai[TF_IB];
#pragma unroll
    for (int u = 0; u < TF_IB; ++u) ar[u] = ai[u] = 0.f;
    if (a.unit_trial && p < N) {
#pragma unroll
      for (int u = 0; u < TF_IB; ++u) ar[u] = (i0 + u == p) ? 1.f : 0.f;
    } else {
      for (int j = 0; j < N; ++j) {
        const float xr = ph[j * TH_P + pl], xi = ph[(N + j) * TH_P + pl];
        const float2* srow = th_sinv32 + j * N + i0;
#pragma unroll
        for (int u = 0; u < TF_IB; ++u) {
          if (i0 + u < N) {
            const float2 sv = srow[u];
            ar[u] = fmaf(xr, sv.x, fmaf(-xi, sv.y, ar[u]));
            ai[u] = fmaf(xr, sv.y, fmaf(xi, sv.x, ai[u]));
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < TF_IB; ++u) {
      const int i = i0 + u;
      if (i >= N) continue;
      tr[(long)i * M + p] = f32_to_f64(ar[u]);
      ti[(long)i * M + p] = f32_to_f64(ai[u]);
      store_lo_f(a.th_lo, a.lo_kind, ((long)w * 2 * N + i) * a.Mp + p, ar[u]);
      store_lo_f(a.th_lo, a.lo_kind, ((long)w * 2 * N + N + i) * a.Mp + p, ai[u]);
    }
  }
}

template <int IB>
static int launch_theta_f32(const OverlapArgs& a, cudaStream_t st) {
  static std::atomic<unsigned long long> attr{0};
  AFQ_TRY(smem_attr_once(k_theta_rows_f32<IB>, 100 * 1024, attr));
  dim3 grid(cdiv(a.M, TH_P), a.W);
  const size_t smem = sizeof(float2) * (size_t)a.N * a.N + sizeof(float) * 2 * a.N * TH_P;
  AFQ_LAUNCH(k_theta_rows_f32<IB>, grid, TH_T, smem, st, a);
  return AFQMC_OK;
}

template <int IB>
static int launch_theta_rows(const OverlapArgs& a, cudaStream_t st) {
  static std::atomic<unsigned long long> attr{0};
  const size_t smem = sizeof(double2) * (size_t)a.N * a.N;
  AFQ_TRY(smem_attr_once(k_theta_rows<IB>, 100 * 1024, attr));
  dim3 grid(cdiv(a.M, TH_P), a.W);
  AFQ_LAUNCH(k_theta_rows<IB>, grid, TH_T, smem, st, a);
  return AFQMC_OK;
}

int launch_overlap(const OverlapArgs& a, cudaStream_t st) {
  const size_t smem = 2ull * a.N * a.N * sizeof(double2);
  if (!a.Sinv || (!a.unit_trial && (a.Sinv32 || a.nup <= 0 || a.nup > a.N))) {
    set_error("overlap: S^-1 scratch is required, and a trial other than V_T = [I; 0] only "
              "in float64 with two spin blocks");
    return AFQMC_EINVAL;
  }
  if (smem > 200 * 1024) {
    set_error("overlap: N=%d too large", a.N);
    return AFQMC_EUNSUPPORTED;
  }
  static std::atomic<unsigned long long> attr{0};
  AFQ_TRY(smem_attr_once(k_overlap<double>, 200 * 1024, attr));
  if (a.Sinv32) {
    static std::atomic<unsigned long long> attr32{0};
    AFQ_TRY(smem_attr_once(k_overlap<float>, 200 * 1024, attr32));
    AFQ_LAUNCH(k_overlap<float>, a.W, OV_T, smem / 2, st, a);
    return AFQMC_OK;
  }
  AFQ_LAUNCH(k_overlap<double>, a.W, OV_T, smem, st, a);
  return AFQMC_OK;
}

int launch_theta(const OverlapArgs& a, cudaStream_t st) {
  if (a.Sinv32 || a.theta32) {
    if (!a.th_lo) {
      set_error("theta: the FP32 rows need the operand copy");
      return AFQMC_EINVAL;
    }
    const int nib = (a.N + 15) / 16, ib = (a.N + nib - 1) / nib;
    switch (ib) {
#define AFQ_THETA32(n) \
  case n:              \
    return launch_theta_f32<n>(a, st);
      AFQ_THETA32(1) AFQ_THETA32(2) AFQ_THETA32(3) AFQ_THETA32(4) AFQ_THETA32(5)
      AFQ_THETA32(6) AFQ_THETA32(7) AFQ_THETA32(8) AFQ_THETA32(9) AFQ_THETA32(10)
      AFQ_THETA32(11) AFQ_THETA32(12) AFQ_THETA32(13) AFQ_THETA32(14) AFQ_THETA32(15)
      AFQ_THETA32(16)
#undef AFQ_THETA32
      default:
        set_error("theta: IB=%d", ib);
        return AFQMC_EINVAL;
    }
  }
  int ib = 8;
  while (a.N % ib) --ib;
  switch (ib) {
    case 8: return launch_theta_rows<8>(a, st);
    case 7: return launch_theta_rows<7>(a, st);
    case 6: return launch_theta_rows<6>(a, st);
    case 5: return launch_theta_rows<5>(a, st);
    case 4: return launch_theta_rows<4>(a, st);
    case 3: return launch_theta_rows<3>(a, st);
    case 2: return launch_theta_rows<2>(a, st);
    default: return launch_theta_rows<1>(a, st);
  }
}

// ---------------------------------------------------------------- weights --
// Overlap ratio of the step, including the scalar of B(x - xbar):
// log R = l' - l - dt (H0' - E_shift) - i sqrt(dt) sum_g x_g c_g.
// Phaseless (Eqs. hybrid-wt, if_rle, weight_update_2):
//   W <- min(W |I| max(0, cos dtheta), W_max), dtheta = Arg R,
//   |I| = exp(Re log R + Re sum xi xbar - Re sum xbar^2 / 2).
// Free projection (Eq. weight_update): W e^{i theta} <- W e^{i theta} R.
__global__ void k_weight(WeightArgs a) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w == 0 && a.dstep) *a.dstep += 1;
  if (w >= a.W) return;
  if (!walker_alive(a.wt, w)) return;
  const double* s = a.scal + 8L * w;
  const double lr = (a.ld_new[2 * w] - a.ld[2 * w]) - a.dt * (a.H0p - a.e_shift) + a.sdt * s[5];
  const double li = (a.ld_new[2 * w + 1] - a.ld[2 * w + 1]) - a.sdt * s[4];
  double wr, wi;
  if (a.mode == AFQMC_PHASELESS) {
    const double dth = wrap_pi(li);
    const double cd = cos(dth);
    if (a.cosd) a.cosd[w] = cd;
    wr = a.wt[2 * w] * exp(lr + s[0] - 0.5 * s[2]) * fmax(0.0, cd);
    if (!isnan(wr)) wr = fmin(wr, a.wmax);
    wi = 0.0;
  } else {
    const double m = exp(lr);
    double sn, cs;
    sincos(li, &sn, &cs);
    const double rr = m * cs, ri = m * sn;
    const double w0r = a.wt[2 * w], w0i = a.wt[2 * w + 1];
    wr = w0r * rr - w0i * ri;
    wi = w0r * ri + w0i * rr;
  }
  if (!isfinite(wr) || !isfinite(wi)) {
    wr = wi = 0.0;
    atomicAdd(a.nonfinite, 1ull);
  }
  a.wt[2 * w] = wr;
  a.wt[2 * w + 1] = wi;
  a.ld[2 * w] = a.ld_new[2 * w];
  a.ld[2 * w + 1] = a.ld_new[2 * w + 1];
}

int launch_weight(const WeightArgs& a, cudaStream_t st) {
  AFQ_LAUNCH(k_weight, cdiv(a.W, 128), 128, 0, st, a);
  return AFQMC_OK;
}

// -------------------------------------------------- modified Gram-Schmidt --
// Sec. 3.4.5: orbitals k = 1..N in turn; column k is orthogonalised against
// the finished columns one projection at a time (each projection uses the
// partially updated vector), then normalised.  The projections are applied
// as soon as a column is finished ("right-looking"): once q_k is normalised,
// every later column j takes v_j -= <q_k|v_j> q_k, 8 lanes per column, so
// column j sees exactly the projections q_0, q_1, ... in order, as in the
// column-by-column form, with two block barriers per k instead of two block
// reductions per (j, k) pair.
// Phi = Q R with R upper triangular and r_kk = |v_k| > 0, so S = V_T^T Phi
// becomes S R^-1: Theta = Phi S^-1 is unchanged and log det S drops by
// sum_k log r_kk (det R real and positive: the phase is unchanged).  The
// kernel lowers log <Psi_T|Psi> = 2 log det S by 2 sum_k log r_kk; the
// overlap need not be recomputed.
__global__ void __launch_bounds__(256) k_mgs(MgsArgs a) {
  extern __shared__ double2 q_sm[];  // the finished column q_k, [M]
  __shared__ double sh[32];
  __shared__ double inv_sh;
  __shared__ double norms[64];  // |v_k|^2, for log det R after the sweep
  const int w = blockIdx.x;
  if (!walker_alive(a.wt, w)) return;
  const int M = a.M, N = a.N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  double* re = a.phiT + (long)w * 2 * N * M;
  double* im = re + (long)N * M;
  for (int k = 0; k < N; ++k) {
    double* vr = re + (long)k * M;
    double* vi = im + (long)k * M;
    double nn = 0.0;
    for (int p = threadIdx.x; p < M; p += blockDim.x) nn = fma(vr[p], vr[p], fma(vi[p], vi[p], nn));
    nn = block_sum(nn, sh);
    // 1 / |v_k| once (a long FP64 sequence), shared by the block; the logs of
    // the norms are taken after the sweep, all at once
    if (threadIdx.x == 0) {
      inv_sh = 1.0 / sqrt(nn);
      norms[k] = nn;
    }
    __syncthreads();
    const double inv = inv_sh;
    for (int p = threadIdx.x; p < M; p += blockDim.x) {
      const double qr = vr[p] * inv, qi = vi[p] * inv;
      vr[p] = qr;
      vi[p] = qi;
      q_sm[p] = make_double2(qr, qi);
    }
    __syncthreads();
    // one group of 8 lanes per later column (4 columns per warp): the dot
    // product is reduced over 8 lanes (3 shuffle levels) instead of 32, which
    // keeps the FP64 pipe - the bound of this kernel - on the projections
    const int grp = lane >> 3, gl = lane & 7, ngrp = 4 * nwarp;
    // later columns of the same spin block only
    const int jend = (a.nup > 0 && k < a.nup) ? a.nup : N;
    for (int j0 = k + 1; j0 < jend; j0 += ngrp) {
      const int j = j0 + 4 * warp + grp;
      const bool act = j < jend;
      double* ur = re + (long)(act ? j : k) * M;
      double* ui = im + (long)(act ? j : k) * M;
      // <q_k|v_j> and v_j -= <q_k|v_j> q_k as chains of FMAs
      double sr = 0.0, si = 0.0;
      if (act)
        for (int p = gl; p < M; p += 8) {
          const double2 q = q_sm[p];
          const double a_ = ur[p], b_ = ui[p];
          sr = fma(q.x, a_, fma(q.y, b_, sr));
          si = fma(q.x, b_, fma(-q.y, a_, si));
        }
#pragma unroll
      for (int o = 4; o > 0; o >>= 1) {
        sr += __shfl_xor_sync(0xffffffffu, sr, o);
        si += __shfl_xor_sync(0xffffffffu, si, o);
      }
      if (act)
        for (int p = gl; p < M; p += 8) {
          const double2 q = q_sm[p];
          ur[p] = fma(-sr, q.x, fma(si, q.y, ur[p]));
          ui[p] = fma(-sr, q.y, fma(-si, q.x, ui[p]));
        }
    }
    __syncthreads();
  }
  // log det R = sum_k log |v_k|, the N logs in parallel, summed in a fixed order
  double lr = threadIdx.x < N ? 0.5 * log(norms[threadIdx.x]) : 0.0;
  if (threadIdx.x < 64) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lr += __shfl_xor_sync(0xffffffffu, lr, o);
    if (lane == 0) sh[warp] = lr;
  }
  __syncthreads();
  if (threadIdx.x == 0 && a.ld) a.ld[2L * w] -= a.sf * (sh[0] + sh[1]);
}

// Mixed precisions: the same sweep in FP32 with the walker's orbitals resident
// in shared memory ([N][M] complex, read once from and written once to the
// float64 orbitals).  With two spin blocks the blocks are independent sweeps
// and run side by side, one half of the warps each; within a block one warp
// per later column, lanes over p (contiguous, conflict-free).  The orbitals
// only feed the low-precision propagation and the overlap, whose float64 log
// det is lowered by the FP32 norms' sum of logs.
__global__ void __launch_bounds__(256) k_mgs_f32(MgsArgs a) {
  extern __shared__ float2 v_sm[];  // [N][M]
  __shared__ float red[8];
  __shared__ float inv_sh[2];
  __shared__ double norms[64];
  __shared__ double sh[2];
  const int w = blockIdx.x;
  if (!walker_alive(a.wt, w)) return;
  const int M = a.M, N = a.N, NM = M * N;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  // group g of wpg warps sweeps columns [c0, c1): the whole set, or spin block g
  const int ng = a.nup > 0 ? 2 : 1;
  const int wpg = 8 / ng;
  const int g = warp / wpg, gw = warp - g * wpg, gt = gw * 32 + lane;
  const int c0 = g == 0 ? 0 : a.nup;
  const int c1 = (ng == 2 && g == 0) ? a.nup : N;
  const int nk = ng == 2 ? (a.nup > N - a.nup ? a.nup : N - a.nup) : N;
  double* re = a.phiT + (long)w * 2 * NM;
  double* im = re + NM;
  for (int e = threadIdx.x; e < NM; e += blockDim.x)
    v_sm[e] = make_float2(f64_to_f32(re[e]), f64_to_f32(im[e]));
  __syncthreads();
  for (int k = 0; k < nk; ++k) {
    const int col = c0 + k;
    const bool live = col < c1;
    float2* vk = v_sm + (long)(live ? col : c0) * M;
    float nn = 0.f;
    if (live)
      for (int p = gt; p < M; p += 32 * wpg) nn = fmaf(vk[p].x, vk[p].x, fmaf(vk[p].y, vk[p].y, nn));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nn += __shfl_xor_sync(0xffffffffu, nn, o);
    if (lane == 0) red[warp] = nn;
    __syncthreads();
    if (live && gt == 0) {
      float t = 0.f;
      for (int q = 0; q < wpg; ++q) t += red[g * wpg + q];
      norms[col] = (double)t;
      inv_sh[g] = 1.f / sqrtf(t);
    }
    __syncthreads();
    if (live) {
      const float inv = inv_sh[g];
      for (int p = gt; p < M; p += 32 * wpg) vk[p] = make_float2(vk[p].x * inv, vk[p].y * inv);
    }
    __syncthreads();
    // v_j -= <q_k|v_j> q_k for every later column j of the block, one warp per column
    if (live)
      for (int j = col + 1 + gw; j < c1; j += wpg) {
        float2* vj = v_sm + j * M;
        float sr = 0.f, si = 0.f;
        for (int p = lane; p < M; p += 32) {
          const float2 q = vk[p], v = vj[p];
          sr = fmaf(q.x, v.x, fmaf(q.y, v.y, sr));
          si = fmaf(q.x, v.y, fmaf(-q.y, v.x, si));
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
          sr += __shfl_xor_sync(0xffffffffu, sr, o);
          si += __shfl_xor_sync(0xffffffffu, si, o);
        }
        for (int p = lane; p < M; p += 32) {
          const float2 q = vk[p], v = vj[p];
          vj[p] = make_float2(fmaf(-sr, q.x, fmaf(si, q.y, v.x)), fmaf(-sr, q.y, fmaf(-si, q.x, v.y)));
        }
      }
    __syncthreads();
  }
  for (int e = threadIdx.x; e < NM; e += blockDim.x) {
    const float2 v = v_sm[e];
    re[e] = f32_to_f64(v.x);
    im[e] = f32_to_f64(v.y);
    if (a.phi_lo) {
      // rows (w, c, k) of the operand copy, pitch Mp (pad columns stay zero)
      const int k = e / M, p = e - k * M;
      store_lo_f(a.phi_lo, a.lo_kind, ((long)w * 2 * N + k) * a.Mp + p, v.x);
      store_lo_f(a.phi_lo, a.lo_kind, ((long)w * 2 * N + N + k) * a.Mp + p, v.y);
    }
  }
  // log det R = sum_k log |v_k|, as in k_mgs
  double lr = threadIdx.x < N ? 0.5 * log(norms[threadIdx.x]) : 0.0;
  if (threadIdx.x < 64) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) lr += __shfl_xor_sync(0xffffffffu, lr, o);
    if (lane == 0) sh[warp] = lr;
  }
  __syncthreads();
  if (threadIdx.x == 0 && a.ld) a.ld[2L * w] -= a.sf * (sh[0] + sh[1]);
}

int launch_mgs(const MgsArgs& a, cudaStream_t st) {
  const size_t smem32 = sizeof(float2) * (size_t)a.M * a.N;
  if (a.f32 && smem32 <= 200 * 1024) {
    static std::atomic<unsigned long long> attr32{0};
    AFQ_TRY(smem_attr_once(k_mgs_f32, 200 * 1024, attr32));
    AFQ_LAUNCH(k_mgs_f32, a.W, 256, smem32, st, a);
    return AFQMC_OK;
  }
  if (a.phi_lo) {
    // the float64 sweep, then the operand copy of every walker
    MgsArgs b = a;
    b.phi_lo = nullptr;
    AFQ_TRY(launch_mgs(b, st));
    return launch_convert_lo(a.phiT, 2L * a.N * a.W, a.M, a.M, a.phi_lo, a.Mp, a.lo_kind, st);
  }
  const size_t smem = sizeof(double2) * (size_t)a.M;
  if (smem > 200 * 1024) {
    set_error("mgs: M=%d too large", a.M);
    return AFQMC_EUNSUPPORTED;
  }
  static std::atomic<unsigned long long> attr{0};
  AFQ_TRY(smem_attr_once(k_mgs, 200 * 1024, attr));
  AFQ_LAUNCH(k_mgs, a.W, 256, smem, st, a);
  return AFQMC_OK;
}

// --------------------------------------------------------------- exchange --
// Exchange part of Eq. localenergy3: sum_g Tr(Lh_g Theta Lh_g Theta), with
// T_g = Lh_g Theta (N x N) formed in registers for a chunk of g and never
// written to global memory; per-chunk partial sums are reduced later in a
// fixed order.
namespace {
constexpr int EX_T = 256, EX_K = 32, EX_P = 32;
}
int exchange_chunk(int N, int G) {
  // outputs per block <= EX_T * EX_K, and the staged Lh rows
  // (gc * N * EX_P doubles) plus Theta rows fit in 160 KB of shared memory
  int gc = (EX_T * EX_K) / (2 * N * N);
  const int smem_cap = (160 * 1024 / 8 - 2 * N * (EX_P + 1)) / (N * EX_P);
  if (gc > smem_cap) gc = smem_cap;
  if (gc < 1) gc = 1;
  if (gc > G) gc = G;
  return gc;
}

__global__ void __launch_bounds__(EX_T) k_exchange(ExchArgs a) {
  extern __shared__ double ex_sm[];
  const int chunk = blockIdx.x, w = blockIdx.y;  // every walker (dead ones too)
  const int M = a.M, N = a.N;
  const int g0 = chunk * a.gc;
  const int gcount = min(a.gc, a.G - g0);
  double* Ls = ex_sm;                       // [gc][N][EX_P]
  double* Ts = ex_sm + (long)a.gc * N * EX_P;  // [2][N][EX_P + 1]
  const int nout = gcount * 2 * N * N;
  double acc[EX_K];
#pragma unroll
  for (int r = 0; r < EX_K; ++r) acc[r] = 0.0;
  const double* th = a.thetaT + (long)w * 2 * N * M;
  for (int p0 = 0; p0 < M; p0 += EX_P) {
    for (int idx = threadIdx.x; idx < gcount * N * EX_P; idx += blockDim.x) {
      const int gi = idx / EX_P, pp = idx % EX_P;
      const int p = p0 + pp;
      Ls[idx] = (p < M) ? a.Lh[((long)g0 * N + gi) * M + p] : 0.0;
    }
    for (int idx = threadIdx.x; idx < 2 * N * EX_P; idx += blockDim.x) {
      const int cj = idx / EX_P, pp = idx % EX_P;
      const int p = p0 + pp;
      Ts[cj * (EX_P + 1) + pp] = (p < M) ? th[(long)cj * M + p] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < EX_K; ++r) {
      const int o = threadIdx.x + r * EX_T;
      if (o < nout) {
        // o = ((g * 2 + c) * N + i) * N + j
        const int j = o % N, i = (o / N) % N, gc2 = o / (N * N);
        const int c = gc2 & 1, g = gc2 >> 1;
        const double* lrow = Ls + ((long)g * N + i) * EX_P;
        const double* trow = Ts + ((long)c * N + j) * (EX_P + 1);
        double s = acc[r];
#pragma unroll 8
        for (int pp = 0; pp < EX_P; ++pp) s = fma(lrow[pp], trow[pp], s);
        acc[r] = s;
      }
    }
    __syncthreads();
  }
  // T_g[c][i][j] into shared memory, then sum_ij T_ij T_ji (complex)
  double* Tm = ex_sm;
#pragma unroll
  for (int r = 0; r < EX_K; ++r) {
    const int o = threadIdx.x + r * EX_T;
    if (o < nout) Tm[o] = acc[r];
  }
  __syncthreads();
  double er = 0.0, ei = 0.0;
  const int nup = a.nup > 0 ? a.nup : N;
  for (int idx = threadIdx.x; idx < gcount * N * N; idx += blockDim.x) {
    const int g = idx / (N * N), ij = idx % (N * N);
    const int i = ij / N, j = ij % N;
    if ((i < nup) != (j < nup)) continue;  // T_g is taken per spin block
    const double* Tr = Tm + (long)(2 * g) * N * N;
    const double* Ti = Tr + (long)N * N;
    const double ar = Tr[i * N + j], ai = Ti[i * N + j];
    const double br = Tr[j * N + i], bi = Ti[j * N + i];
    er += ar * br - ai * bi;
    ei += ar * bi + ai * br;
  }
  __shared__ double sh[32];
  er = block_sum(er, sh);
  ei = block_sum(ei, sh);
  if (threadIdx.x == 0) {
    double* o = a.part + ((long)w * a.nchunk + chunk) * 2;
    o[0] = er;
    o[1] = ei;
  }
}

int launch_exchange(const ExchArgs& a, cudaStream_t st) {
  if (2 * a.N * a.N > EX_T * EX_K) {
    set_error("exchange: N=%d above the supported 64", a.N);
    return AFQMC_EUNSUPPORTED;
  }
  size_t d1 = (size_t)a.gc * a.N * EX_P + 2ull * a.N * (EX_P + 1);
  size_t d2 = (size_t)a.gc * 2 * a.N * a.N;
  size_t smem = (d1 > d2 ? d1 : d2) * sizeof(double);
  static std::atomic<unsigned long long> attr{0};
  AFQ_TRY(smem_attr_once(k_exchange, 160 * 1024, attr));
  if (smem > 160 * 1024) {
    set_error("exchange: shared memory %zu too large", smem);
    return AFQMC_EUNSUPPORTED;
  }
  dim3 grid(a.nchunk, a.W);
  AFQ_LAUNCH(k_exchange, grid, EX_T, smem, st, a);
  return AFQMC_OK;
}

// ---------------------------------------------------------- local energy --
// E_loc = H0 + 2 Tr(hh Theta) + 1/2 sum_g t_g^2 - sum_g Tr(T_g T_g)
// (Eqs. localenergy2/3; the 1/2 is that of H_2 in Eq. bo_ham2) for the
// closed-shell block; with two spin blocks (sf = 1) the one-body trace and the
// exchange are the sums over the blocks, E_loc = H0 + Tr(hh Theta) +
// 1/2 sum_g [t_g^2 - sum_sigma Tr(T_g,sigma T_g,sigma)].
__global__ void __launch_bounds__(256) k_eloc(ElocArgs a) {
  __shared__ double sh[32];
  const int w = blockIdx.x;
  const int M = a.M, N = a.N, G = a.G;
  const double* th = a.thetaT + (long)w * 2 * N * M;
  double e1r = 0.0, e1i = 0.0;
  for (int idx = threadIdx.x; idx < N * M; idx += blockDim.x) {
    const double hv = a.hh[idx];
    e1r += hv * th[idx];
    e1i += hv * th[(long)N * M + idx];
  }
  double cr = 0.0, ci = 0.0;
  for (int g = threadIdx.x; g < G; g += blockDim.x) {
    double re, imv;
    if (a.t32) {
      re = a.t32[(long)w * 2 * G + g];
      imv = a.t32[(long)w * 2 * G + G + g];
    } else {
      re = a.t[(long)w * 2 * G + g];
      imv = a.t[(long)w * 2 * G + G + g];
    }
    cr += re * re - imv * imv;
    ci += 2.0 * re * imv;
  }
  double xr = 0.0, xi = 0.0;
  const double* pp = a.part + (long)w * a.nchunk * 2;
  for (int c = threadIdx.x; c < a.nchunk; c += blockDim.x) {
    xr += pp[2 * c];
    xi += pp[2 * c + 1];
  }
  e1r = block_sum(e1r, sh);
  e1i = block_sum(e1i, sh);
  cr = block_sum(cr, sh);
  ci = block_sum(ci, sh);
  xr = block_sum(xr, sh);
  xi = block_sum(xi, sh);
  if (threadIdx.x == 0) {
    a.eloc[2 * w] = a.H0 + a.sf * e1r + 0.5 * cr - (0.5 * a.sf) * xr;
    a.eloc[2 * w + 1] = a.sf * e1i + 0.5 * ci - (0.5 * a.sf) * xi;
  }
}

int launch_eloc(const ElocArgs& a, cudaStream_t st) {
  AFQ_LAUNCH(k_eloc, a.W, 256, 0, st, a);
  return AFQMC_OK;
}

// Mixed estimator (Eq. localenergy) over live walkers, Re E_loc clamped to
// [lo, hi] (Eq. cap) for phaseless walks; one record (step, E, sum W, live).
__global__ void __launch_bounds__(256) k_record(RecordArgs a) {
  __shared__ double sh[32];
  double nr = 0.0, ni = 0.0, dr = 0.0, di = 0.0, na = 0.0;
  for (int w = threadIdx.x; w < a.W; w += blockDim.x) {
    if (!walker_alive(a.wt, w)) continue;
    const double wr = a.wt[2 * w], wi = a.wt[2 * w + 1];
    double er = a.eloc[2 * w], ei = a.eloc[2 * w + 1];
    na += 1.0;
    if (a.mode == AFQMC_PHASELESS) {
      er = fmin(fmax(er, a.lo), a.hi);
      nr += wr * er;
      dr += wr;
    } else {
      nr += wr * er - wi * ei;
      ni += wr * ei + wi * er;
      dr += wr;
      di += wi;
    }
  }
  nr = block_sum(nr, sh);
  ni = block_sum(ni, sh);
  dr = block_sum(dr, sh);
  di = block_sum(di, sh);
  na = block_sum(na, sh);
  if (threadIdx.x == 0) {
    double E;
    if (a.mode == AFQMC_PHASELESS) {
      E = nr / dr;
    } else {
      const double den = dr * dr + di * di;
      E = (nr * dr + ni * di) / den;
    }
    a.last[0] = nr;
    a.last[1] = dr;
    a.last[2] = ni;
    a.last[3] = di;
    a.last[4] = E;
    a.last[5] = na;
    if (a.records) {
      const unsigned long long n = *a.rec_count;
      double* r = a.records + 4 * (long)(n % (unsigned long long)a.max_records);
      r[0] = (double)*a.step;
      r[1] = E;
      r[2] = dr;
      r[3] = na;
      *a.rec_count = n + 1;
    }
  }
}

int launch_record(const RecordArgs& a, cudaStream_t st) {
  AFQ_LAUNCH(k_record, 1, 256, 0, st, a);
  return AFQMC_OK;
}

// -------------------------------------------------------------------- comb --
// Fixed-size comb (Sec. 3.4.4 asks for population control but gives no
// scheme): W_tot and the cumulative weights C_j are sequential sums in walker
// order; tooth k sits at ((k + u) W_tot) / N_w with u from Philox counter
// (0, 0xffffffff, step, 0); it goes to the walker j with C_{j-1} <= tooth <
// C_j (the last live walker if rounding puts it past C_{N_w-1}).  Copies land
// in walker-index order and every new weight is W_tot / N_w.
__global__ void __launch_bounds__(256) k_comb_plan(CombArgs a) {
  __shared__ double s_u;
  __shared__ int s_last, s_ok;
  if (threadIdx.x == 0) {
    double s = 0.0;
    int last = -1;
    for (int j = 0; j < a.W; ++j) {
      const double wj = a.wt[2 * j];
      s += wj;
      a.cum[j] = s;
      if (wj > 0.0) last = j;
    }
    a.wtot[0] = s;
    s_last = last;
    s_ok = (s > 0.0 && isfinite(s) && last >= 0) ? 1 : 0;
    u32x4 c = {0u, 0xFFFFFFFFu, (uint32_t)(*a.dstep - 1), 0u};
    u32x4 r = philox4x32_10(c, (uint32_t)a.seed, (uint32_t)(a.seed >> 32));
    s_u = uniform53(r.x, r.y);
  }
  __syncthreads();
  const double wtot = a.wtot[0];
  for (int k = threadIdx.x; k < a.W; k += blockDim.x) {
    if (!s_ok) {
      a.parent[k] = -1;
      continue;
    }
    const double tooth = (((double)k + s_u) * wtot) / (double)a.W;
    int lo = 0, hi = a.W;  // first j with cum[j] > tooth
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (a.cum[mid] > tooth) hi = mid; else lo = mid + 1;
    }
    a.parent[k] = (lo >= a.W) ? s_last : lo;
  }
}

__global__ void __launch_bounds__(256) k_comb_gather(CombArgs a) {
  const int k = blockIdx.x;
  const int j = a.parent[k];
  if (j < 0) return;
  const long n = 2L * a.N * a.M;
  const double* sp = a.phiT + (long)j * n;
  const double* st_ = a.thetaT + (long)j * n;
  double* dp = a.tmp_phi + (long)k * n;
  double* dt_ = a.tmp_theta + (long)k * n;
  for (long i = threadIdx.x; i < n; i += blockDim.x) {
    dp[i] = sp[i];
    dt_[i] = st_[i];
  }
  if (threadIdx.x == 0) {
    a.tmp_ld[2 * k] = a.ld[2 * j];
    a.tmp_ld[2 * k + 1] = a.ld[2 * j + 1];
  }
}

__global__ void __launch_bounds__(256) k_comb_commit(CombArgs a) {
  const int k = blockIdx.x;
  if (a.parent[k] < 0) return;
  const long n = 2L * a.N * a.M;
  for (long i = threadIdx.x; i < n; i += blockDim.x) {
    a.phiT[(long)k * n + i] = a.tmp_phi[(long)k * n + i];
    a.thetaT[(long)k * n + i] = a.tmp_theta[(long)k * n + i];
  }
  if (threadIdx.x == 0) {
    a.ld[2 * k] = a.tmp_ld[2 * k];
    a.ld[2 * k + 1] = a.tmp_ld[2 * k + 1];
    a.wt[2 * k] = a.wtot[0] / (double)a.W;
    a.wt[2 * k + 1] = 0.0;
  }
}

int launch_comb(const CombArgs& a, cudaStream_t st) {
  AFQ_LAUNCH(k_comb_plan, 1, 256, 0, st, a);
  AFQ_LAUNCH(k_comb_gather, a.W, 256, 0, st, a);
  AFQ_LAUNCH(k_comb_commit, a.W, 256, 0, st, a);
  return AFQMC_OK;
}

// ---------------------------------------------------------------- set-up ----
// L[g][p][q] -> LpT[packed(p,q)][g] for p <= q (transposed packed vectors).
__global__ void k_pack_transpose(const double* L, double* LpT, int G, int M) {
  __shared__ double tile[32][33];
  const int g0 = blockIdx.x * 32, p = blockIdx.y, q0 = blockIdx.z * 32;
  if (q0 + 31 < p) return;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int g = g0 + r, q = q0 + threadIdx.x;
    tile[r][threadIdx.x] = (g < G && q < M && q >= p) ? L[((long)g * M + p) * M + q] : 0.0;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int q = q0 + r, g = g0 + threadIdx.x;
    if (q < M && q >= p && g < G) LpT[packed_index(p, q, M) * G + g] = tile[threadIdx.x][r];
  }
}

int launch_pack_transpose(const double* L, double* LpT, int G, int M, cudaStream_t st) {
  dim3 grid(cdiv(G, 32), M, cdiv(M, 32));
  AFQ_LAUNCH(k_pack_transpose, grid, dim3(32, 8), 0, st, L, LpT, G, M);
  return AFQMC_OK;
}

__global__ void __launch_bounds__(256) k_rowdot(const double* A, const double* b, double* out,
                                                int len, double scale) {
  __shared__ double sh[32];
  const double* a = A + (long)blockIdx.x * len;
  double s = 0.0;
  for (int j = threadIdx.x; j < len; j += blockDim.x) s += a[j] * b[j];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[blockIdx.x] = scale * s;
}

int launch_rowdot(const double* A, const double* b, double* out, int rows, int len,
                  double scale, cudaStream_t st) {
  AFQ_LAUNCH(k_rowdot, rows, 256, 0, st, A, b, out, len, scale);
  return AFQMC_OK;
}

// X = scale * (h - 1/2 sum_g L_g^2 + sum_g c_g L_g): the mean-field-shifted
// one-body operator v0' of Sec. 2.4 (Eq. mcd1), times -dt/2.
__global__ void k_v0p(const double* h1, const double* L2, const double* cLp, double* X, int M,
                      double scale) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * M) return;
  const int p = (int)(idx / M), q = (int)(idx % M);
  const long pk = (p <= q) ? packed_index(p, q, M) : packed_index(q, p, M);
  X[idx] = scale * (h1[idx] - 0.5 * L2[idx] + cLp[pk]);
}

int launch_v0p(const double* h1, const double* L2, const double* cLp, double* X, int M,
               double scale, cudaStream_t st) {
  AFQ_LAUNCH(k_v0p, cdiv((size_t)M * M, 256), 256, 0, st, h1, L2, cLp, X, M, scale);
  return AFQMC_OK;
}

__global__ void __launch_bounds__(256) k_norm1(const double* X, double* out, int M) {
  __shared__ double sh[256];
  double best = 0.0;
  for (int q = threadIdx.x; q < M; q += blockDim.x) {
    double s = 0.0;
    for (int p = 0; p < M; ++p) s += fabs(X[(long)p * M + q]);
    best = fmax(best, s);
  }
  sh[threadIdx.x] = best;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) out[0] = sh[0];
}

int launch_norm1(const double* X, double* out, int M, cudaStream_t st) {
  AFQ_LAUNCH(k_norm1, 1, 256, 0, st, X, out, M);
  return AFQMC_OK;
}

__global__ void k_fill_identity(double* X, int M, double d) {
  const long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= (long)M * M) return;
  X[idx] = (idx / M == idx % M) ? d : 0.0;
}

int launch_fill_identity(double* X, int M, double d, cudaStream_t st) {
  AFQ_LAUNCH(k_fill_identity, cdiv((size_t)M * M, 256), 256, 0, st, X, M, d);
  return AFQMC_OK;
}

// dst[e] = sum_{j < nparts} parts[j][e], the parts added in order.
__global__ void k_sum_parts(const double* parts, int nparts, long n, double* dst) {
  for (long e = (long)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int j = 0; j < nparts; ++j) v += parts[(long)j * n + e];
    dst[e] = v;
  }
}

int launch_sum_parts(const double* parts, int nparts, long n, double* dst, cudaStream_t st) {
  if (n <= 0) return AFQMC_OK;
  AFQ_LAUNCH(k_sum_parts, cdiv((size_t)n, 256), 256, 0, st, parts, nparts, n, dst);
  return AFQMC_OK;
}

__global__ void k_scale(double* X, long n, double s) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) X[i] *= s;
}

int launch_scale(double* X, long n, double s, cudaStream_t st) {
  AFQ_LAUNCH(k_scale, cdiv(n, 256), 256, 0, st, X, n, s);
  return AFQMC_OK;
}

// Every walker at {V_T, W = 1} (algorithm outline, step 1).
__global__ void k_init_walkers(const double* VTt, double* phiT, double* wt, int W, int N, int M) {
  const long n = (long)N * M;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  const int w = blockIdx.y;
  if (i < n) {
    phiT[(long)w * 2 * n + i] = VTt[i];
    phiT[(long)w * 2 * n + n + i] = 0.0;
  }
  if (i == 0) {
    wt[2 * w] = 1.0;
    wt[2 * w + 1] = 0.0;
  }
}

int launch_init_walkers(const double* VTt, double* phiT, double* wt, int W, int N, int M,
                        cudaStream_t st) {
  dim3 grid(cdiv((size_t)N * M, 256), W);
  AFQ_LAUNCH(k_init_walkers, grid, 256, 0, st, VTt, phiT, wt, W, N, M);
  return AFQMC_OK;
}

__global__ void __launch_bounds__(256) k_sumsq(const double* v, double* out, int n) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += v[i] * v[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) out[0] = s;
}

int launch_sumsq(const double* v, double* out, int n, cudaStream_t st) {
  AFQ_LAUNCH(k_sumsq, 1, 256, 0, st, v, out, n);
  return AFQMC_OK;
}

}  // namespace afq

// ------------------------------------------------- low-precision copies ----
namespace afq {
__global__ void k_convert_lo(const double* src, long rows, long cols, long lds, void* dst,
                             long ldd, int kind, double minus_diag) {
  const long n = rows * ldd;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const long r = i / ldd, c = i % ldd;
    const double v = c < cols ? src[r * lds + c] - (r == c ? minus_diag : 0.0) : 0.0;
    store_lo(dst, kind, i, v);
  }
}

int launch_convert_lo(const double* src, long rows, long cols, long lds, void* dst, long ldd,
                      int kind, cudaStream_t st, double minus_diag) {
  if (rows <= 0) return AFQMC_OK;
  AFQ_LAUNCH(k_convert_lo, 152 * 8, 256, 0, st, src, rows, cols, lds, dst, ldd, kind, minus_diag);
  return AFQMC_OK;
}

// The value a BF16 / TF32 operand copy holds for v (store_lo's rounding).
__device__ __forceinline__ double lo_value(int kind, double v) {
  if (kind == LO_BF16) return (double)__bfloat162float(__double2bfloat16(v));
  return (double)round_tf32((float)v);
}

// src - minus_diag I as a split operand: row r holds nseg segments of width
// seg (columns c >= cols zero), segment g the high part hi = lo_value(v) or,
// when bit g of lo_mask is set, the low part v - hi rounded again, so that
// hi + lo carries v to about twice the operand precision.
__global__ void k_split_lo(const double* src, long rows, long cols, long lds, void* dst, long seg,
                           int nseg, unsigned lo_mask, int kind, double minus_diag) {
  const long ldd = seg * nseg, n = rows * ldd;
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x) {
    const long r = i / ldd, cc = i % ldd, c = cc % seg;
    const int g = (int)(cc / seg);
    const double v = c < cols ? src[r * lds + c] - (r == c ? minus_diag : 0.0) : 0.0;
    store_lo(dst, kind, i, ((lo_mask >> g) & 1u) ? v - lo_value(kind, v) : v);
  }
}

int launch_split_lo(const double* src, long rows, long cols, long lds, void* dst, long seg,
                    int nseg, unsigned lo_mask, int kind, cudaStream_t st, double minus_diag) {
  if (rows <= 0) return AFQMC_OK;
  AFQ_LAUNCH(k_split_lo, 152 * 8, 256, 0, st, src, rows, cols, lds, dst, seg, nseg, lo_mask, kind,
             minus_diag);
  return AFQMC_OK;
}

__global__ void k_round_f32(const double* src, float* dst, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    dst[i] = f64_to_f32(src[i]);
}

__global__ void k_widen_f32(const float* src, double* dst, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    dst[i] = f32_to_f64(src[i]);
}

// Smallest index i with v[i] not finite (NaN or +-inf) into *first (left
// unchanged when every value is finite): exponent bits all ones.
__global__ void k_first_nonfinite(const double* v, long n, unsigned long long* first) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    if ((__double2hiint(v[i]) & 0x7ff00000) == 0x7ff00000) atomicMin(first, (unsigned long long)i);
}

int launch_first_nonfinite(const double* v, long n, unsigned long long* first, cudaStream_t st) {
  if (n <= 0) return AFQMC_OK;
  AFQ_LAUNCH(k_first_nonfinite, 152 * 8, 256, 0, st, v, n, first);
  return AFQMC_OK;
}

// part[z][i] = sum_{g in chunk z} c[g] A[g][i] over nz equal chunks of the
// G rows (float64; the partials are then added in order by launch_sum_parts).
__global__ void k_wsum_rows(const double* A, const double* c, int G, long n, int nz,
                            double* part) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int z = blockIdx.y, per = (G + nz - 1) / nz, g0 = z * per, g1 = min(G, g0 + per);
  double s = 0.0;
  for (int g = g0; g < g1; ++g) s += c[g] * A[(long)g * n + i];
  part[(long)z * n + i] = s;
}

int launch_wsum_rows(const double* A, const double* c, int G, long n, int nz, double* part,
                     cudaStream_t st) {
  if (n <= 0 || nz < 1) return AFQMC_OK;
  dim3 grid((unsigned)cdiv(n, 256), nz);
  AFQ_LAUNCH(k_wsum_rows, grid, 256, 0, st, A, c, G, n, nz, part);
  return AFQMC_OK;
}

// dst[g][j] = src[g * sstride + j] (FP32 -> float64, exact) for j < len.
__global__ void k_widen_rows(const float* src, long sstride, long len, int G, double* dst) {
  const long j = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= len) return;
  const int g = blockIdx.y;
  dst[(long)g * len + j] = f32_to_f64(src[(long)g * sstride + j]);
}

int launch_widen_rows(const float* src, long sstride, long len, int G, double* dst,
                      cudaStream_t st) {
  if (len <= 0 || G <= 0) return AFQMC_OK;
  dim3 grid((unsigned)cdiv(len, 256), G);
  AFQ_LAUNCH(k_widen_rows, grid, 256, 0, st, src, sstride, len, G, dst);
  return AFQMC_OK;
}

int launch_round_f32(const double* src, float* dst, long n, cudaStream_t st) {
  if (n <= 0) return AFQMC_OK;
  AFQ_LAUNCH(k_round_f32, 152 * 8, 256, 0, st, src, dst, n);
  return AFQMC_OK;
}

// n float64 values at buf rounded to FP32 in place (the FP32 array then starts
// at buf).  Chunk k >= 1 of c values reads bytes [8kc, 8(k+1)c) and writes
// [4kc, 4(k+1)c): disjoint, and below the chunks still to be read.  Chunk 0
// goes through tmp (room for c floats) and is copied to the front last.
int launch_round_f32_inplace(double* buf, long n, long c, float* tmp, cudaStream_t st) {
  if (n <= 0) return AFQMC_OK;
  if (c < 1) {
    set_error("round_f32_inplace: chunk %ld", c);
    return AFQMC_EINVAL;
  }
  float* out = reinterpret_cast<float*>(buf);
  const long c0 = n < c ? n : c;
  AFQ_TRY(launch_round_f32(buf, tmp, c0, st));
  for (long k0 = c; k0 < n; k0 += c)
    AFQ_TRY(launch_round_f32(buf + k0, out + k0, (n - k0 < c ? n - k0 : c), st));
  AFQ_CUDA(cudaMemcpyAsync(out, tmp, sizeof(float) * c0, cudaMemcpyDeviceToDevice, st));
  return AFQMC_OK;
}

int launch_widen_f32(const float* src, double* dst, long n, cudaStream_t st) {
  if (n <= 0) return AFQMC_OK;
  AFQ_LAUNCH(k_widen_f32, 152 * 8, 256, 0, st, src, dst, n);
  return AFQMC_OK;
}

__global__ void k_convert_f32(const double* src, float* dst, long n) {
  for (long i = (long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// Full Cholesky vectors, transposed, in BF16/TF32 for the mixed V contraction:
// row (p, q) = p * Mp + q holds L[g][p][q] over g (pitch Gp); rows with q >= M
// and columns g >= G are zero.  32 x 32 tiles of (q, g) per block, one p.
// The Cholesky operand of the V contraction: the upper 16 x 16 blocks (P, Q),
// P <= Q, of each Mp x Mp vector L[g] (zero beyond M), row-major over the
// blocks; row blk * 256 + pp * 16 + qq of out holds L[g][16 P + pp][16 Q + qq]
// for g < Gp (zero for g >= G).  Block (x, y): 32 vectors, one (blk, pp) row.
template <typename T>
__global__ void k_pack_blocks_lo(const T* L, int G, int M, int Mp, int Gp, void* out,
                                 int kind) {
  __shared__ double tile[32][17];
  const int g0 = blockIdx.x * 32;
  const int blk = blockIdx.y >> 4, pp = blockIdx.y & 15;
  const int nb = Mp / 16;
  int P = 0, rem = blk;
  while (rem >= nb - P) {
    rem -= nb - P;
    ++P;
  }
  const int Q = P + rem;
  const int p = 16 * P + pp, q0 = 16 * Q;
  for (int e = threadIdx.x; e < 32 * 16; e += blockDim.x) {
    const int r = e >> 4, c = e & 15;
    const int g = g0 + r, q = q0 + c;
    tile[r][c] = (g < G && p < M && q < M) ? (double)L[((long)g * M + p) * M + q] : 0.0;
  }
  __syncthreads();
  const long n0 = (long)blk * 256 + pp * 16;
  for (int e = threadIdx.x; e < 32 * 16; e += blockDim.x) {
    const int c = e >> 5, r = e & 31;
    if (g0 + r < Gp) store_lo(out, kind, (n0 + c) * Gp + g0 + r, tile[r][c]);
  }
}

template <typename T>
static int pack_blocks_lo(const T* L, int G, int M, int Mp, int Gp, void* out, int kind,
                          cudaStream_t st) {
  const int nb = Mp / 16;
  dim3 grid(cdiv(Gp, 32), nb * (nb + 1) / 2 * 16);
  AFQ_LAUNCH(k_pack_blocks_lo<T>, grid, 256, 0, st, L, G, M, Mp, Gp, out, kind);
  return AFQMC_OK;
}

int launch_pack_blocks_lo(const double* L, int G, int M, int Mp, int Gp, void* out, int kind,
                          cudaStream_t st) {
  return pack_blocks_lo(L, G, M, Mp, Gp, out, kind, st);
}

int launch_pack_blocks_lo(const float* L, int G, int M, int Mp, int Gp, void* out, int kind,
                          cudaStream_t st) {
  return pack_blocks_lo(L, G, M, Mp, Gp, out, kind, st);
}

int launch_convert_f32(const double* src, float* dst, long n, cudaStream_t st) {
  if (n <= 0) return AFQMC_OK;
  AFQ_LAUNCH(k_convert_f32, 152 * 4, 256, 0, st, src, dst, n);
  return AFQMC_OK;
}
}  // namespace afq

// ------------------------------------------------------------ bounded wait --
namespace afq {
__global__ void k_wait_flag(const int* flag, long long max_polls, int* status) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const volatile int* f = flag;
  for (long long i = 0; i < max_polls; ++i) {
    if (*f) return;
    __nanosleep(1000);
  }
  *status = AFQMC_ETIMEOUT;
}

int launch_wait_flag(const int* flag, long long max_polls, int* status, cudaStream_t st) {
  AFQ_LAUNCH(k_wait_flag, 1, 32, 0, st, flag, max_polls, status);
  return AFQMC_OK;
}
}  // namespace afq

// ------------------------------------------------------- generator access --
namespace afq {
__global__ void k_philox(uint64_t key, const uint32_t* ctr, long n, uint32_t* out) {
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  u32x4 c = {ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]};
  u32x4 r = philox4x32_10(c, (uint32_t)key, (uint32_t)(key >> 32));
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

__global__ void k_fields(uint64_t seed, uint32_t step, int w0, int nw, int G, double* out) {
  const int npair = (G + 1) / 2;
  const long i = (long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long)nw * npair) return;
  const int w = (int)(i / npair), k = (int)(i % npair);
  double a, b;
  field_pair(seed, step, (uint32_t)(w0 + w), (uint32_t)k, &a, &b);
  out[(long)w * G + 2 * k] = a;
  if (2 * k + 1 < G) out[(long)w * G + 2 * k + 1] = b;
}

int launch_philox(uint64_t key, const uint32_t* ctr, long n, uint32_t* out, cudaStream_t st) {
  if (n <= 0) return AFQMC_OK;
  AFQ_LAUNCH(k_philox, cdiv(n, 256), 256, 0, st, key, ctr, n, out);
  return AFQMC_OK;
}

int launch_fields(uint64_t seed, uint32_t step, int w0, int nw, int G, double* out,
                  cudaStream_t st) {
  const long n = (long)nw * ((G + 1) / 2);
  if (n <= 0) return AFQMC_OK;
  AFQ_LAUNCH(k_fields, cdiv(n, 256), 256, 0, st, seed, step, w0, nw, G, out);
  return AFQMC_OK;
}
}  // namespace afq
