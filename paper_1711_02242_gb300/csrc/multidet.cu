// Multi-determinant trial (Sec. 3.4, Eqs. usesherman, precomputing,
// precomputing2, localenergy2, localenergy3).
//
// Psi_T = sum_d A_d Psi_d with per-determinant spin-up and spin-down orbitals
// V_ds; the walkers stay closed shell (both spin blocks phi).  Per walker and
// (d, s): S_ds = V_ds^T phi, its inverse and log det (Gauss-Jordan with
// partial pivoting), Theta_ds = phi S_ds^-1; then
//   <Psi_T|Psi> = sum_d A_d^* det S_du det S_dd   (log-sum-exp over d, fixed order),
//   w_d = A_d^* <Psi_d|Psi> / <Psi_T|Psi>,
//   t_g = sum_d w_d sum_s Tr(Lh_dsg Theta_ds)                    (force bias),
//   E_loc = H0 + sum_d w_d [sum_s Tr(hh_ds Theta_ds)
//           + 1/2 sum_g (sum_s Tr(Lh_dsg Theta_ds))^2 - 1/2 sum_s sum_g Tr(T_dsg T_dsg)],
//   T_dsg = Lh_dsg Theta_ds (the float64 exchange kernel, once per (d, s)).
// On the mixed path the traces and the exchange of each (d, s) run on the
// tensor cores from BF16/TF32 copies of Lh_ds and Theta_ds (written by the
// overlap kernel); overlaps, weights and the combinations stay float64.
// Every determinant is handled in full (the Sherman-Morrison-Woodbury
// shortcut for determinants differing by a few orbitals is not used).  All in
// the run's orthonormal basis, whose first N vectors are the leading spin-up
// determinant's orbitals.
#include "state.cuh"
#include "tc.cuh"

namespace afq {
namespace {

__device__ inline double2 zmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// Block (ds, w): S = V_ds^T phi_w, Gauss-Jordan inverse with log det, and
// Theta_ds = phi S^-1 as rows [2][N][M] of md_theta[ds][w].  A dead walker is
// skipped; a singular S leaves log det = -inf and Theta = 0.
__global__ void __launch_bounds__(256)
    k_md_overlap(int W, int M, int N, const double* __restrict__ Vt, const double* __restrict__ phi,
                 const double* wt, double* theta, double* ldds, void* th_lo, int lo_kind, int Mp) {
  extern __shared__ double2 aug[];  // [N][2N]
  __shared__ double2 fac[64];
  __shared__ int prow, singular, swaps;
  __shared__ double logabs, phase;
  const int ds = blockIdx.x, w = blockIdx.y;
  if (!walker_alive(wt, w)) return;
  const long NM = (long)N * M;
  const double* V = Vt + (long)ds * NM;  // [N][M], row i = column i of V_ds
  const double* fr = phi + (long)w * 2 * NM;
  const double* fi = fr + NM;
  double* th = theta + ((long)ds * W + w) * 2 * NM;
  const int N2 = 2 * N, tid = threadIdx.x;
  for (int e = tid; e < N * N; e += blockDim.x) {
    const int i = e / N, j = e - (e / N) * N;
    double sr = 0.0, si = 0.0;
    for (int p = 0; p < M; ++p) {
      const double v = V[(long)i * M + p];
      sr += v * fr[(long)j * M + p];
      si += v * fi[(long)j * M + p];
    }
    aug[i * N2 + j] = make_double2(sr, si);
    aug[i * N2 + N + j] = make_double2(i == j ? 1.0 : 0.0, 0.0);
  }
  if (tid == 0) {
    singular = 0;
    swaps = 0;
    logabs = 0.0;
    phase = 0.0;
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
      if (!(best > 0.0)) singular = 1;
      if (r != k) swaps++;
    }
    __syncthreads();
    if (singular) break;
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
    if (tid == 0) {
      logabs += 0.5 * log(den);
      phase += atan2(pv.y, pv.x);
    }
    __syncthreads();
    for (int j = tid; j < N2; j += blockDim.x) aug[k * N2 + j] = zmul(aug[k * N2 + j], inv);
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
  double* ld = ldds + ((long)w * gridDim.x + ds) * 2;
  // the operand copy of Theta for the mixed path: rows (c, j) of pitch Mp
  const long lo_row0 = ((long)ds * W + w) * 2 * N;
  if (singular) {
    for (long t = tid; t < 2 * NM; t += blockDim.x) {
      th[t] = 0.0;
      if (th_lo) store_lo(th_lo, lo_kind, (lo_row0 + t / M) * Mp + t % M, 0.0);
    }
    if (tid == 0) {
      ld[0] = -INFINITY;
      ld[1] = 0.0;
    }
    return;
  }
  if (tid == 0) {
    ld[0] = logabs;
    ld[1] = wrap_pi(phase + 3.141592653589793 * swaps);
  }
  // Theta[p][j] = sum_i phi[p][i] S^-1[i][j], stored as row j
  for (long e = tid; e < NM; e += blockDim.x) {
    const int j = (int)(e / M);
    const long p = e - (long)j * M;
    double tr = 0.0, ti = 0.0;
    for (int i = 0; i < N; ++i) {
      const double br = fr[(long)i * M + p], bi = fi[(long)i * M + p];
      const double2 s = aug[i * N2 + N + j];
      tr += br * s.x - bi * s.y;
      ti += br * s.y + bi * s.x;
    }
    th[(long)j * M + p] = tr;
    th[NM + (long)j * M + p] = ti;
    if (th_lo) {
      store_lo(th_lo, lo_kind, (lo_row0 + j) * Mp + p, tr);
      store_lo(th_lo, lo_kind, (lo_row0 + N + j) * Mp + p, ti);
    }
  }
}

// Per walker: log <Psi_T|Psi> = log sum_d exp(log A_d^* + ld_du + ld_dd) in
// the order of d (largest real part factored out), its phase in (-pi, pi],
// and the weights w_d.
__global__ void k_md_combine(int W, int nd, const double* logA, const double* ldds,
                             const double* wt, double* ldout, double* wd) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W || !walker_alive(wt, w)) return;
  const double* l = ldds + (long)w * nd * 4;  // [nd][2 spins][re, im]
  double ref = -INFINITY;
  for (int d = 0; d < nd; ++d) {
    const double re = logA[2 * d] + l[4 * d] + l[4 * d + 2];
    if (re > ref) ref = re;
  }
  double tr = 0.0, ti = 0.0;
  for (int d = 0; d < nd; ++d) {
    const double re = logA[2 * d] + l[4 * d] + l[4 * d + 2];
    if (!(re > -INFINITY)) continue;
    const double m = exp(re - ref);
    double sn, cs;
    sincos(logA[2 * d + 1] + l[4 * d + 1] + l[4 * d + 3], &sn, &cs);
    tr += m * cs;
    ti += m * sn;
  }
  const double den = tr * tr + ti * ti;
  for (int d = 0; d < nd; ++d) {
    const double re = logA[2 * d] + l[4 * d] + l[4 * d + 2];
    double xr = 0.0, xi = 0.0;
    if (re > -INFINITY) {
      const double m = exp(re - ref);
      double sn, cs;
      sincos(logA[2 * d + 1] + l[4 * d + 1] + l[4 * d + 3], &sn, &cs);
      // (m e^{i phi}) / (tr + i ti)
      xr = (m * cs * tr + m * sn * ti) / den;
      xi = (m * sn * tr - m * cs * ti) / den;
    }
    wd[((long)w * nd + d) * 2] = xr;
    wd[((long)w * nd + d) * 2 + 1] = xi;
  }
  ldout[2 * w] = ref + 0.5 * log(den);
  ldout[2 * w + 1] = wrap_pi(atan2(ti, tr));
}

// t[w][c][g] = sum_(d,s) w_d (C_ds[(w,re)][g] + i C_ds[(w,im)][g]) as re/im planes
// (float64 traces and t on the float64 path, FP32 on the mixed path).
template <typename TC>
__global__ void k_md_fb_combine(int W, int nd, int G, const TC* C, const double* wd,
                                const double* wt, TC* t) {
  const long n = (long)W * G;
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n;
       e += (long)gridDim.x * blockDim.x) {
    const int w = (int)(e / G), g = (int)(e - (long)w * G);
    if (!walker_alive(wt, w)) continue;
    double sr = 0.0, si = 0.0;
    for (int d = 0; d < nd; ++d) {
      const double ar = wd[((long)w * nd + d) * 2], ai = wd[((long)w * nd + d) * 2 + 1];
      double cr = 0.0, ci = 0.0;
      for (int s = 0; s < 2; ++s) {
        const TC* Cd = C + (long)(2 * d + s) * 2 * W * G;
        cr += (double)Cd[(2L * w) * G + g];
        ci += (double)Cd[(2L * w + 1) * G + g];
      }
      sr += ar * cr - ai * ci;
      si += ar * ci + ai * cr;
    }
    t[(2L * w) * G + g] = (TC)sr;
    t[(2L * w + 1) * G + g] = (TC)si;
  }
}

// E_loc per walker (one block): sum_d w_d [one-body + Coulomb - exchange / 2] + H0.
template <typename TC>
__global__ void __launch_bounds__(256)
    k_md_eloc(int W, int nd, int M, int N, int G, int nchunk, double H0, const double* hh,
              const double* theta, const TC* C, const double* part, const double* wd,
              const double* wt, double* eloc) {
  __shared__ double sh[32];
  const int w = blockIdx.x;
  if (!walker_alive(wt, w)) return;
  const long NM = (long)N * M;
  double er = 0.0, ei = 0.0;
  for (int d = 0; d < nd; ++d) {
    const double ar = wd[((long)w * nd + d) * 2], ai = wd[((long)w * nd + d) * 2 + 1];
    if (ar == 0.0 && ai == 0.0) continue;
    double e1r = 0.0, e1i = 0.0, cr = 0.0, ci = 0.0, xr = 0.0, xi = 0.0;
    for (int s = 0; s < 2; ++s) {
      const int ds = 2 * d + s;
      const double* h = hh + (long)ds * NM;
      const double* th = theta + ((long)ds * W + w) * 2 * NM;
      for (long e = threadIdx.x; e < NM; e += blockDim.x) {
        e1r += h[e] * th[e];
        e1i += h[e] * th[NM + e];
      }
      const double* pp = part + ((long)ds * W + w) * nchunk * 2;
      for (int c = threadIdx.x; c < nchunk; c += blockDim.x) {
        xr += pp[2 * c];
        xi += pp[2 * c + 1];
      }
    }
    for (int g = threadIdx.x; g < G; g += blockDim.x) {
      double tr = 0.0, ti = 0.0;
      for (int s = 0; s < 2; ++s) {
        const TC* Cd = C + (long)(2 * d + s) * 2 * W * G;
        tr += (double)Cd[(2L * w) * G + g];
        ti += (double)Cd[(2L * w + 1) * G + g];
      }
      cr += tr * tr - ti * ti;
      ci += 2.0 * tr * ti;
    }
    e1r = block_sum(e1r, sh);
    e1i = block_sum(e1i, sh);
    cr = block_sum(cr, sh);
    ci = block_sum(ci, sh);
    xr = block_sum(xr, sh);
    xi = block_sum(xi, sh);
    const double edr = e1r + 0.5 * cr - 0.5 * xr, edi = e1i + 0.5 * ci - 0.5 * xi;
    er += ar * edr - ai * edi;
    ei += ar * edi + ai * edr;
  }
  if (threadIdx.x == 0) {
    eloc[2 * w] = H0 + er;
    eloc[2 * w + 1] = ei;
  }
}

// c_g = sum_s Tr(L_g V_0s V_0s^T) = sum_s sum_(i,p) Lh_0sg[i][p] V_0s[i][p].
__global__ void k_md_meanfield(int G, long NM, const double* Lh, const double* Vt, double* c) {
  __shared__ double sh[32];
  const int g = blockIdx.x;
  double v = 0.0;
  for (int s = 0; s < 2; ++s) {
    const double* a = Lh + ((long)s * G + g) * NM;
    const double* b = Vt + (long)s * NM;
    for (long e = threadIdx.x; e < NM; e += blockDim.x) v += a[e] * b[e];
  }
  v = block_sum(v, sh);
  if (threadIdx.x == 0) c[g] = v;
}

}  // namespace

int md_overlap_update(afqmc_state* s, bool into_ld) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, N = p.N, M = p.M, nd = p.ndet;
  const size_t smem = sizeof(double2) * (size_t)N * 2 * N;
  AFQ_CUDA(cudaFuncSetAttribute(k_md_overlap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  AFQ_LAUNCH(k_md_overlap, dim3(2 * nd, W), 256, smem, s->st, W, M, N, b.md_V, b.phiT, b.wt,
             b.md_theta, b.md_ld, b.mixed ? b.md_theta_lo : nullptr, b.lo_kind, b.Mp);
  AFQ_LAUNCH(k_md_combine, cdiv(W, 128), 128, 0, s->st, W, nd, b.md_logA, b.md_ld, b.wt,
             into_ld ? b.ld : b.ld_new, b.md_w);
  return AFQMC_OK;
}

// Per (d, s): C_ds[(w, c)][g] = Tr(Lh_dsg Theta_ds) for every walker, one
// batched contraction over K = N M.
static int md_traces(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, N = p.N, M = p.M, G = p.nchol, nd = p.ndet;
  GemmF64 g;
  g.m = 2 * W;
  g.n = G;
  g.k = N * M;
  g.batch = 2 * nd;
  g.A = b.md_theta;
  g.lda = (long)N * M;
  g.sAb = (long)W * 2 * N * M;
  g.B = b.md_Lh;
  g.ldb = (long)N * M;
  g.sBb = (long)G * N * M;
  g.C = b.md_C;
  g.ldc = G;
  g.sCb = 2L * W * G;
  return gemm_nt_f64(g, s->st);
}

// Mixed path: the same traces on the tensor cores from the BF16/TF32 copies.
static int md_traces_lo(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, N = p.N, G = p.nchol, nd = p.ndet;
  const long rowA = (long)N * b.Mp;
  for (int ds = 0; ds < 2 * nd; ++ds) {
    TcGemm g;
    g.m = 2 * W;
    g.n = G;
    g.k = N * b.Mp;
    g.A = static_cast<const char*>(b.md_theta_lo) + (size_t)ds * 2 * W * rowA * b.lo_bytes;
    g.lda = rowA;
    g.B = static_cast<const char*>(b.md_Lh_lo) + (size_t)ds * G * rowA * b.lo_bytes;
    g.ldb = rowA;
    g.tf32 = b.lo_kind == LO_TF32;
    g.err = b.status;
    AFQ_TRY(tc_gemm_store(g, b.md_C32 + (size_t)ds * 2 * W * G, G, 1.0f, s->st));
  }
  return AFQMC_OK;
}

int md_force_bias(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const unsigned grid = cdiv((size_t)p.nwalkers * p.nchol, 256);
  if (b.mixed) {
    AFQ_TRY(md_traces_lo(s));
    AFQ_LAUNCH(k_md_fb_combine<float>, grid, 256, 0, s->st, p.nwalkers, p.ndet, p.nchol, b.md_C32,
               b.md_w, b.wt, b.t32);
    return AFQMC_OK;
  }
  AFQ_TRY(md_traces(s));
  AFQ_LAUNCH(k_md_fb_combine<double>, grid, 256, 0, s->st, p.nwalkers, p.ndet, p.nchol, b.md_C,
             b.md_w, b.wt, b.t);
  return AFQMC_OK;
}

// Local energies into b.eloc (the traces md_C are current after md_force_bias).
int md_local_energies(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, N = p.N, M = p.M, G = p.nchol, nd = p.ndet;
  const long NM = (long)N * M;
  for (int ds = 0; ds < 2 * nd; ++ds) {
    double* part = b.md_part + (long)ds * W * b.nchunk * 2;
    if (b.mixed) {
      // T_g = Lh_dsg Theta_ds and sum_ij T_ij T_ji on the tensor cores
      const long rowA = (long)N * b.Mp;
      TcGemm g;
      g.m = G * N;
      g.n = 2 * N * W;
      g.k = M;
      g.A = static_cast<const char*>(b.md_Lh_lo) + (size_t)ds * G * rowA * b.lo_bytes;
      g.lda = b.Mp;
      g.B = static_cast<const char*>(b.md_theta_lo) + (size_t)ds * 2 * W * rowA * b.lo_bytes;
      g.ldb = b.Mp;
      g.tf32 = b.lo_kind == LO_TF32;
      g.err = b.status;
      AFQ_TRY(tc_exchange(g, G, W, N, part, b.nchunk, s->st));
    } else {
      ExchArgs ex{W, M, N, G, b.gc, b.nchunk, b.md_Lh + (long)ds * G * NM,
                  b.md_theta + (long)ds * W * 2 * NM, part, b.wt};
      AFQ_TRY(launch_exchange(ex, s->st));
    }
  }
  if (b.mixed)
    AFQ_LAUNCH(k_md_eloc<float>, W, 256, 0, s->st, W, nd, M, N, G, b.nchunk, p.H0, b.md_hh,
               b.md_theta, b.md_C32, b.md_part, b.md_w, b.wt, b.eloc);
  else
    AFQ_LAUNCH(k_md_eloc<double>, W, 256, 0, s->st, W, nd, M, N, G, b.nchunk, p.H0, b.md_hh,
               b.md_theta, b.md_C, b.md_part, b.md_w, b.wt, b.eloc);
  return AFQMC_OK;
}

// Set-up: the determinants' orbitals (already in the run's basis, [nd][2][N][M]
// in md_V), their half-rotated vectors and one-body matrices, the leading
// determinant's mean field c, and log A_d^*.
int md_setup(afqmc_state* s, const double* coef) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int N = p.N, M = p.M, G = p.nchol, nd = p.ndet;
  const long NM = (long)N * M;
  for (int ds = 0; ds < 2 * nd; ++ds) {
    GemmF64 g;
    g.m = N;
    g.n = M;
    g.k = M;
    g.batch = G;
    g.A = b.md_V + (long)ds * NM;
    g.lda = M;
    g.B = b.Lfull;
    g.ldb = M;
    g.sBb = (long)M * M;
    g.C = b.md_Lh + (long)ds * G * NM;
    g.ldc = M;
    g.sCb = NM;
    AFQ_TRY(gemm_nt_f64(g, s->st));
    GemmF64 h;
    h.m = N;
    h.n = M;
    h.k = M;
    h.A = b.md_V + (long)ds * NM;
    h.lda = M;
    h.B = b.h1;
    h.ldb = M;
    h.C = b.md_hh + (long)ds * NM;
    h.ldc = M;
    AFQ_TRY(gemm_nt_f64(h, s->st));
  }
  AFQ_LAUNCH(k_md_meanfield, G, 256, 0, s->st, G, NM, b.md_Lh, b.md_V, b.c);
  if (b.mixed) {
    // operand copies: the half-rotated vectors (pitch Mp) and Theta's padding
    AFQ_TRY(launch_convert_lo(b.md_Lh, 2L * nd * G * N, M, M, b.md_Lh_lo, b.Mp, b.lo_kind, s->st));
    AFQ_CUDA(cudaMemsetAsync(b.md_theta_lo, 0,
                             (size_t)2 * nd * p.nwalkers * 2 * N * b.Mp * b.lo_bytes, s->st));
  }
  std::vector<double> la(2 * (size_t)nd);
  for (int d = 0; d < nd; ++d) {
    const double ar = coef[2 * d], ai = coef[2 * d + 1];
    la[2 * d] = 0.5 * std::log(ar * ar + ai * ai);  // log |A_d^*|; -inf drops d
    la[2 * d + 1] = -std::atan2(ai, ar);              // arg A_d^*
  }
  AFQ_CUDA(cudaMemcpyAsync(b.md_logA, la.data(), sizeof(double) * 2 * nd, cudaMemcpyHostToDevice,
                           s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  return AFQMC_OK;
}

}  // namespace afq
