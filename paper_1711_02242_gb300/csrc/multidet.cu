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
// All in the run's orthonormal basis, whose first N vectors are the leading
// spin-up determinant's orbitals.
//
// Determinants that differ from determinant 0 in at most kSmwMaxK columns per
// spin (the other columns equal, in place: a CI expansion about a reference)
// are evaluated relative to it in float64 (on either path), as the
// Sherman-Morrison-Woodbury remark of Sec. 3.4 suggests.  With S_0s = V_0s^T phi, Theta_0s =
// phi S_0s^-1 and, for a one-body X, Y = V_ds^T X Theta_0s, determinant d
// enters through the polynomial
//   det(M_ds + e Y) = r_ds + e c1_ds(X) + e^2 c2_ds(X) + ...,  M_ds = V_ds^T Theta_0s,
// r_ds = det(V_ds^T phi) / det S_0s, c1 = r Tr(X G_ds), 2 c2 = r [Tr(X G_ds)^2 -
// Tr(X G_ds X G_ds)] (G_ds determinant d's Green's function), which stay
// finite where det(V_ds^T phi) = 0 (the limits the full evaluation cannot
// take).  M_ds is the identity but for the rows of the holes H (column h_l
// of V_0s replaced by the particle u_l): with Xi = U^T Theta_0s (rows u_l),
// Y0 = V_0s^T X Theta_0s and Yp = U^T X Theta_0s, reordering H first and
// taking the Schur complement of the unit block,
//   det(M + e Y) = det(I + e Z) det(P + e S1 + e^2 S2) + O(e^3),
//   P = Xi[:, H],  Z = Y0[Hc, Hc],
//   S1 = Yp[:, H] - Xi[:, Hc] Y0[Hc, H],
//   S2 = Xi[:, Hc] Z Y0[Hc, H] - Yp[:, Hc] Y0[Hc, H],
// and det(P + e S1 + e^2 S2) = p0 + e p1 + e^2 p2 by multilinearity in the
// k <= kSmwMaxK rows, so that r = p0, c1 = p1 + p0 Tr Z, c2 = p2 + p1 Tr Z +
// p0 (Tr(Z)^2 - Tr(Z^2)) / 2.  Then with A_d^* / Z_T = a_d, Z_T = sum_d A_d^*
// r_du r_dd:  <Psi_T|Psi> = det S_0u det S_0d Z_T,  t_g = sum_d a_d
// [c1_du r_dd + r_du c1_dd](L_g), E_loc = sum_d a_d [H0 r_du r_dd + (c1_du
// r_dd + r_du c1_dd)(h) + sum_g (c2_du r_dd + r_du c2_dd + c1_du c1_dd)(L_g)].
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

// ---------------------------------------- determinants relative to d = 0 --
__device__ inline double2 zadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ inline double2 zsub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ inline double2 zscale(double2 a, double s) { return make_double2(a.x * s, a.y * s); }
__device__ inline double2 zdivd(double2 a, double2 b) {
  const double den = b.x * b.x + b.y * b.y;
  return make_double2((a.x * b.x + a.y * b.y) / den, (a.y * b.x - a.x * b.y) / den);
}
__device__ inline double2 zshfl(double2 v, int src) {
  return make_double2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
}
__device__ inline double2 zwarp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

typedef double2 SmallMat[kSmwMaxK][kSmwMaxK];

// det of the leading k x k block (k <= kSmwMaxK; k = 0 gives 1) by Gaussian
// elimination with partial pivoting; A is overwritten.
__device__ double2 small_det(SmallMat& A, int k) {
  double2 det = make_double2(1.0, 0.0);
  for (int c = 0; c < k; ++c) {
    int piv = c;
    double best = A[c][c].x * A[c][c].x + A[c][c].y * A[c][c].y;
    for (int r = c + 1; r < k; ++r) {
      const double m2 = A[r][c].x * A[r][c].x + A[r][c].y * A[r][c].y;
      if (m2 > best) {
        best = m2;
        piv = r;
      }
    }
    if (!(best > 0.0)) return make_double2(0.0, 0.0);
    if (piv != c) {
      for (int q = 0; q < k; ++q) {
        const double2 t = A[c][q];
        A[c][q] = A[piv][q];
        A[piv][q] = t;
      }
      det = make_double2(-det.x, -det.y);
    }
    det = zmul(det, A[c][c]);
    const double2 inv = zdivd(make_double2(1.0, 0.0), A[c][c]);
    for (int r = c + 1; r < k; ++r) {
      const double2 f = zmul(A[r][c], inv);
      for (int q = c; q < k; ++q) A[r][q] = zsub(A[r][q], zmul(f, A[c][q]));
    }
  }
  return det;
}

// p0, p1, p2 of det(P + e S1 + e^2 S2) by multilinearity in the rows (p2 only
// if `second`).
__device__ void small_poly(const SmallMat& P, const SmallMat& S1, const SmallMat& S2, int k,
                           bool second, double2* p0, double2* p1, double2* p2) {
  SmallMat A;
  auto load = [&](int l1, const SmallMat* R1, int l2, const SmallMat* R2) {
    for (int l = 0; l < k; ++l)
      for (int m = 0; m < k; ++m)
        A[l][m] = l == l1 ? (*R1)[l][m] : (l == l2 ? (*R2)[l][m] : P[l][m]);
  };
  load(-1, nullptr, -1, nullptr);
  *p0 = small_det(A, k);
  *p1 = make_double2(0.0, 0.0);
  *p2 = make_double2(0.0, 0.0);
  for (int l = 0; l < k; ++l) {
    load(l, &S1, -1, nullptr);
    *p1 = zadd(*p1, small_det(A, k));
  }
  if (!second) return;
  for (int l = 0; l < k; ++l) {
    load(l, &S2, -1, nullptr);
    *p2 = zadd(*p2, small_det(A, k));
    for (int m = l + 1; m < k; ++m) {
      load(l, &S1, m, &S1);
      *p2 = zadd(*p2, small_det(A, k));
    }
  }
}

// One block per walker: Xi_s = U_s^T Theta_0s (particle rows of md_V), the
// ratios r_ds = det Xi_s[o_ds + l][h_m], Z_T = sum_d A_d^* r_du r_dd in the
// order of d, log <Psi_T|Psi> = log det S_0u + log det S_0d + log Z_T, and
// a_d = A_d^* / Z_T.  tab[(d, s)] = [k, o, h_0 .. h_3, -, -].
__global__ void __launch_bounds__(128)
    k_smw_ratio(int W, int M, int N, int nd, int ks, int np0, int np1, const int* __restrict__ tab,
                const int* __restrict__ prow, const double* __restrict__ Vt,
                const double* __restrict__ theta, const double* __restrict__ ld0,
                const double* __restrict__ logA, const double* wt, double* xi, double* aw,
                double* ldout) {
  __shared__ double2 zt;
  const int w = blockIdx.x, tid = threadIdx.x;
  if (!walker_alive(wt, w)) return;
  const long NM = (long)N * M;
  double2* aw2 = reinterpret_cast<double2*>(aw) + (long)w * nd;
  for (int s = 0; s < 2; ++s) {
    const int np = s ? np1 : np0;
    const double* th = theta + ((long)s * W + w) * 2 * NM;  // Theta_0s rows [2][N][M]
    double2* xs = reinterpret_cast<double2*>(xi) + ((long)w * 2 + s) * ks * N;
    for (int e = tid; e < np * N; e += blockDim.x) {
      const int pl = e / N, j = e - (e / N) * N;
      const double* u = Vt + (long)prow[s * ks + pl] * M;
      double re = 0.0, im = 0.0;
      for (int q = 0; q < M; ++q) {
        re += u[q] * th[(long)j * M + q];
        im += u[q] * th[NM + (long)j * M + q];
      }
      xs[(long)pl * N + j] = make_double2(re, im);
    }
  }
  __syncthreads();
  for (int d = tid; d < nd; d += blockDim.x) {
    double2 r[2];
    for (int s = 0; s < 2; ++s) {
      const int* tb = tab + (d * 2 + s) * 8;
      const int k = tb[0], o = tb[1];
      const double2* xs = reinterpret_cast<const double2*>(xi) + ((long)w * 2 + s) * ks * N;
      SmallMat P;
      for (int l = 0; l < k; ++l)
        for (int m = 0; m < k; ++m) P[l][m] = xs[(long)(o + l) * N + tb[2 + m]];
      r[s] = small_det(P, k);
    }
    double sn, cs;
    sincos(logA[2 * d + 1], &sn, &cs);
    const double am = exp(logA[2 * d]);
    aw2[d] = zmul(make_double2(am * cs, am * sn), zmul(r[0], r[1]));
  }
  __syncthreads();
  if (tid == 0) {
    double2 z = make_double2(0.0, 0.0);
    for (int d = 0; d < nd; ++d) z = zadd(z, aw2[d]);
    const double* l0 = ld0 + (long)w * 4;  // [spin][re, im] of log det S_0s
    ldout[2 * w] = l0[0] + l0[2] + 0.5 * log(z.x * z.x + z.y * z.y);
    ldout[2 * w + 1] = wrap_pi(l0[1] + l0[3] + atan2(z.y, z.x));
    zt = z;
  }
  __syncthreads();
  for (int d = tid; d < nd; d += blockDim.x) {
    double sn, cs;
    sincos(logA[2 * d + 1], &sn, &cs);
    const double am = exp(logA[2 * d]);
    aw2[d] = zdivd(make_double2(am * cs, am * sn), zt);
  }
}

// p0, p1, p2 of det(P + e S1 + e^2 S2) for k <= KM; KM = 2 in registers
// (closed forms), else the elimination above.
template <int KM>
__device__ __forceinline__ void poly_k(const double2 (&P)[KM][KM], const double2 (&S1)[KM][KM],
                                       const double2 (&S2)[KM][KM], int k, bool second,
                                       double2* p0, double2* p1, double2* p2) {
  if constexpr (KM == 2) {
    const double2 z = make_double2(0.0, 0.0);
    if (k == 0) {
      *p0 = make_double2(1.0, 0.0);
      *p1 = *p2 = z;
    } else if (k == 1) {
      *p0 = P[0][0];
      *p1 = S1[0][0];
      *p2 = second ? S2[0][0] : z;
    } else {
      auto det2 = [](double2 a, double2 b, double2 c, double2 d) { return zsub(zmul(a, d), zmul(b, c)); };
      *p0 = det2(P[0][0], P[0][1], P[1][0], P[1][1]);
      *p1 = zadd(det2(S1[0][0], S1[0][1], P[1][0], P[1][1]), det2(P[0][0], P[0][1], S1[1][0], S1[1][1]));
      *p2 = second ? zadd(det2(S1[0][0], S1[0][1], S1[1][0], S1[1][1]),
                          zadd(det2(S2[0][0], S2[0][1], P[1][0], P[1][1]),
                               det2(P[0][0], P[0][1], S2[1][0], S2[1][1])))
                   : z;
    }
  } else {
    SmallMat A, B, C;
    for (int l = 0; l < k; ++l)
      for (int m = 0; m < k; ++m) {
        A[l][m] = P[l][m];
        B[l][m] = S1[l][m];
        C[l][m] = S2[l][m];
      }
    small_poly(A, B, C, k, second, p0, p1, p2);
  }
}

// Determinant d, spin s, operator rows X (Lh_g or h of (d, s)) for the warp
// of that determinant (lane = column j < N): r, c1 and (second) c2.  KM >= k
// bounds the hole count, so the per-hole arrays are unrolled into registers.
template <int KM, bool SECOND>
__device__ __forceinline__ void det_coeffs(const int* tb, int N, int M, int lane,
                                           const double2* __restrict__ Y,
                                           const double2* __restrict__ X,
                                           const double* __restrict__ th, long NM,
                                           const double* __restrict__ xbase, long xstride_h,
                                           double2 trY, const double2* rjs, double2* rr,
                                           double2* c1, double2* c2) {
  const int k = tb[0], o = tb[1];
  const bool lj = lane < N;
  int h[KM];
#pragma unroll
  for (int l = 0; l < KM; ++l) h[l] = l < k ? tb[2 + l] : 0;
  double2 yp[KM], xy[KM];
#pragma unroll
  for (int l = 0; l < KM; ++l) {
    yp[l] = xy[l] = make_double2(0.0, 0.0);
    if (l >= k || !lj) continue;
    const double* x = xbase + (long)h[l] * xstride_h;
    double re = 0.0, im = 0.0;
    for (int q = 0; q < M; ++q) {
      re += x[q] * th[(long)lane * M + q];
      im += x[q] * th[NM + (long)lane * M + q];
    }
    yp[l] = make_double2(re, im);
    double2 v = make_double2(0.0, 0.0);
    for (int i = 0; i < N; ++i) v = zadd(v, zmul(X[(long)(o + l) * N + i], Y[i * N + lane]));
    xy[l] = v;
  }
  double2 P[KM][KM], S1[KM][KM], S2[KM][KM];
#pragma unroll
  for (int l = 0; l < KM; ++l)
#pragma unroll
    for (int m = 0; m < KM; ++m) {
      P[l][m] = S1[l][m] = S2[l][m] = make_double2(0.0, 0.0);
      if (l >= k || m >= k) continue;
      const double2 ypv = zshfl(yp[l], h[m]), xyv = zshfl(xy[l], h[m]);
      double2 corr = make_double2(0.0, 0.0);
#pragma unroll
      for (int i = 0; i < KM; ++i)
        if (i < k) corr = zadd(corr, zmul(X[(long)(o + l) * N + h[i]], Y[h[i] * N + h[m]]));
      P[l][m] = X[(long)(o + l) * N + h[m]];
      S1[l][m] = zadd(zsub(ypv, xyv), corr);
    }
  double2 tz = trY;
#pragma unroll
  for (int m = 0; m < KM; ++m)
    if (m < k) tz = zsub(tz, Y[h[m] * N + h[m]]);
  double2 e2 = make_double2(0.0, 0.0);
  if constexpr (SECOND) {
    bool hole = false;
#pragma unroll
    for (int m = 0; m < KM; ++m) hole = hole || (m < k && h[m] == lane);
#pragma unroll
    for (int l = 0; l < KM; ++l) {
      if (l >= k) continue;
      double2 F = make_double2(0.0, 0.0);
      if (lj && !hole) {
        F = zsub(xy[l], yp[l]);
#pragma unroll
        for (int i = 0; i < KM; ++i)
          if (i < k) F = zsub(F, zmul(X[(long)(o + l) * N + h[i]], Y[h[i] * N + lane]));
      }
#pragma unroll
      for (int m = 0; m < KM; ++m)
        if (m < k) S2[l][m] = zwarp_sum(lj ? zmul(F, Y[lane * N + h[m]]) : make_double2(0.0, 0.0));
    }
    double2 tz2 = rjs[N];
#pragma unroll
    for (int m = 0; m < KM; ++m) {
      if (m >= k) continue;
      tz2 = zsub(tz2, zscale(rjs[h[m]], 2.0));
#pragma unroll
      for (int m2 = 0; m2 < KM; ++m2)
        if (m2 < k) tz2 = zadd(tz2, zmul(Y[h[m] * N + h[m2]], Y[h[m2] * N + h[m]]));
    }
    e2 = zscale(zsub(zmul(tz, tz), tz2), 0.5);
  }
  double2 p0, p1, p2;
  poly_k<KM>(P, S1, S2, k, SECOND, &p0, &p1, &p2);
  *rr = p0;
  *c1 = zadd(p1, zmul(p0, tz));
  *c2 = zadd(zadd(p2, zmul(p1, tz)), zmul(p0, e2));
}

// Block (chunk c, walker w), 8 warps: for each vector g of the chunk
// (kSmwGC of them; with ENERGY the extra chunk c = nchk takes h instead),
// Y0_s = Lh_0sg Theta_0s in shared memory, then one warp per determinant
// (lane j = column j) forms Yp and Xi Y0 at its holes, the k x k matrices P,
// S1 (and S2) and the coefficients (det_coeffs); the force bias sums a_d
// [c1_du r_dd + r_du c1_dd] over d (per warp in the order of d, then over
// warps in order); the energy keeps per (w, c, d) the sum over the chunk of
// c2_du r_dd + r_du c2_dd + c1_du c1_dd (H0 r_du r_dd + c1_du r_dd + r_du c1_dd
// for h).
template <bool ENERGY>
__global__ void __launch_bounds__(256)
    k_smw_terms(int W, int M, int N, int G, int nd, int ks, int nchk, double H0,
                const int* __restrict__ tab, const double* __restrict__ Lh,
                const double* __restrict__ hh, const double* __restrict__ theta,
                const double* __restrict__ xi, const double* __restrict__ aw, const double* wt,
                double* t, double* part) {
  extern __shared__ double2 y0[];  // [2][N][N]
  __shared__ double2 rj[2][kSmwMaxN + 1];  // Sum_i Y0[j][i] Y0[i][j]; [N]: Tr(Y0^2)
  __shared__ double2 trs[2];
  __shared__ double2 wsum[8];
  const int c = blockIdx.x, w = blockIdx.y, tid = threadIdx.x;
  if (!walker_alive(wt, w)) return;
  const bool onebody = ENERGY && c == nchk;
  const int g0 = onebody ? 0 : c * kSmwGC;
  const int g1 = onebody ? 1 : (G < g0 + kSmwGC ? G : g0 + kSmwGC);
  const long NM = (long)N * M;
  const int lane = tid & 31, warp = tid >> 5, nwarp = blockDim.x >> 5;
  const double2* xw = reinterpret_cast<const double2*>(xi) + (long)w * 2 * ks * N;
  const double2* aw2 = reinterpret_cast<const double2*>(aw) + (long)w * nd;
  // operator rows of (d, s) for vector g (or h): row i at xrow(ds, g) + i M
  auto xrow = [&](int ds, int g) -> const double* {
    return onebody ? hh + (long)ds * NM : Lh + ((long)ds * G + g) * NM;
  };
  for (int g = g0; g < g1; ++g) {
    for (int e = tid; e < 2 * N * N; e += blockDim.x) {
      const int s = e / (N * N), i = (e / N) % N, j = e % N;
      const double* x = xrow(s, g) + (long)i * M;  // determinant 0: ds = s
      const double* th = theta + ((long)s * W + w) * 2 * NM;
      double re = 0.0, im = 0.0;
      for (int q = 0; q < M; ++q) {
        re += x[q] * th[(long)j * M + q];
        im += x[q] * th[NM + (long)j * M + q];
      }
      y0[e] = make_double2(re, im);
    }
    __syncthreads();
    if (tid < 2) {
      double2 tr = make_double2(0.0, 0.0);
      for (int i = 0; i < N; ++i) tr = zadd(tr, y0[tid * N * N + i * N + i]);
      trs[tid] = tr;
    }
    if (ENERGY && !onebody)
      for (int e = tid; e < 2 * N; e += blockDim.x) {
        const int s = e / N, j = e % N;
        const double2* Y = y0 + s * N * N;
        double2 v = make_double2(0.0, 0.0);
        for (int i = 0; i < N; ++i) v = zadd(v, zmul(Y[j * N + i], Y[i * N + j]));
        rj[s][j] = v;
      }
    __syncthreads();
    if (ENERGY && !onebody && tid < 2) {
      double2 v = make_double2(0.0, 0.0);
      for (int j = 0; j < N; ++j) v = zadd(v, rj[tid][j]);
      rj[tid][N] = v;
    }
    __syncthreads();
    double2 fsum = make_double2(0.0, 0.0);
    for (int d = warp; d < nd; d += nwarp) {
      double2 rr[2], c1[2], c2[2];
      const int kmax = tab[(d * 2) * 8] > tab[(d * 2 + 1) * 8] ? tab[(d * 2) * 8] : tab[(d * 2 + 1) * 8];
      for (int s = 0; s < 2; ++s) {
        const int* tb = tab + (d * 2 + s) * 8;
        const double2* Y = y0 + s * N * N;
        const double2* X = xw + (long)s * ks * N;  // Xi_s rows
        const double* th = theta + ((long)s * W + w) * 2 * NM;
        const double* xb = xrow(2 * d + s, g);
        if (ENERGY && !onebody) {
          if (kmax <= 2)
            det_coeffs<2, true>(tb, N, M, lane, Y, X, th, NM, xb, M, trs[s], rj[s], &rr[s], &c1[s], &c2[s]);
          else
            det_coeffs<kSmwMaxK, true>(tb, N, M, lane, Y, X, th, NM, xb, M, trs[s], rj[s], &rr[s],
                                       &c1[s], &c2[s]);
        } else {
          if (kmax <= 2)
            det_coeffs<2, false>(tb, N, M, lane, Y, X, th, NM, xb, M, trs[s], rj[s], &rr[s], &c1[s], &c2[s]);
          else
            det_coeffs<kSmwMaxK, false>(tb, N, M, lane, Y, X, th, NM, xb, M, trs[s], rj[s], &rr[s],
                                        &c1[s], &c2[s]);
        }
      }
      if (lane == 0) {
        if (!ENERGY) {
          fsum = zadd(fsum, zmul(aw2[d], zadd(zmul(c1[0], rr[1]), zmul(rr[0], c1[1]))));
        } else {
          double2 v;
          if (onebody)
            v = zadd(zscale(zmul(rr[0], rr[1]), H0), zadd(zmul(c1[0], rr[1]), zmul(rr[0], c1[1])));
          else
            v = zadd(zadd(zmul(c2[0], rr[1]), zmul(rr[0], c2[1])), zmul(c1[0], c1[1]));
          double2* pp = reinterpret_cast<double2*>(part) + ((long)w * (nchk + 1) + c) * nd + d;
          *pp = g == g0 ? v : zadd(*pp, v);
        }
      }
    }
    if (!ENERGY) {
      if (lane == 0) wsum[warp] = fsum;
      __syncthreads();
      if (tid == 0) {
        double2 tot = make_double2(0.0, 0.0);
        for (int q = 0; q < nwarp; ++q) tot = zadd(tot, wsum[q]);
        t[(2L * w) * G + g] = tot.x;
        t[(2L * w + 1) * G + g] = tot.y;
      }
    }
    __syncthreads();
  }
}

// The mixed path's fields read FP32 traces.
__global__ void k_smw_t32(long n, const double* t, float* t32) {
  for (long e = blockIdx.x * (long)blockDim.x + threadIdx.x; e < n; e += (long)gridDim.x * blockDim.x)
    t32[e] = (float)t[e];
}

// E_loc = sum_d a_d sum_c part[w][c][d] (chunks in order), one thread per walker.
__global__ void k_smw_eloc(int W, int nd, int nchk, const double* aw, const double* part,
                           const double* wt, double* eloc) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= W || !walker_alive(wt, w)) return;
  const double2* a = reinterpret_cast<const double2*>(aw) + (long)w * nd;
  const double2* pw = reinterpret_cast<const double2*>(part) + (long)w * (nchk + 1) * nd;
  double2 e = make_double2(0.0, 0.0);
  for (int d = 0; d < nd; ++d) {
    double2 sd = make_double2(0.0, 0.0);
    for (int c = 0; c <= nchk; ++c) sd = zadd(sd, pw[(long)c * nd + d]);
    e = zadd(e, zmul(a[d], sd));
  }
  eloc[2 * w] = e.x;
  eloc[2 * w + 1] = e.y;
}

}  // namespace

// Holes and particles of every (d, s) relative to determinant 0 from the
// host orbitals ([nd][M][N] row-major): column i of V_ds is a hole when any
// entry differs from column i of V_0s.  The low-rank evaluation is taken on
// float64 (on either path: the mixed path then keeps its low-precision
// propagation and takes the force bias in FP32 from it) when every
// determinant differs in at most kSmwMaxK columns per spin and N <= kSmwMaxN
// (two or more determinants); else each determinant is evaluated in full.
int smw_detect(afqmc_state* s, const double* up, const double* dn) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int nd = p.ndet, N = p.N, M = p.M;
  s->smw = false;
  if (nd < 2 || N > kSmwMaxN) return AFQMC_OK;
  const int ks = kSmwMaxK * nd;
  std::vector<int> tab((size_t)nd * 2 * 8, 0), prow((size_t)2 * ks, 0);
  int np[2] = {0, 0};
  for (int d = 0; d < nd; ++d)
    for (int sp = 0; sp < 2; ++sp) {
      const double* V0 = sp ? dn : up;
      const double* Vd = V0 + (size_t)d * M * N;
      int* tb = tab.data() + (size_t)(d * 2 + sp) * 8;
      int k = 0;
      for (int i = 0; i < N; ++i) {
        bool same = true;
        for (int r = 0; r < M && same; ++r) same = Vd[(size_t)r * N + i] == V0[(size_t)r * N + i];
        if (same) continue;
        if (k == kSmwMaxK) return AFQMC_OK;
        tb[2 + k++] = i;
      }
      tb[0] = k;
      tb[1] = np[sp];
      for (int l = 0; l < k; ++l) prow[(size_t)sp * ks + np[sp]++] = (2 * d + sp) * N + tb[2 + l];
    }
  AFQ_CUDA(cudaMemcpyAsync(b.smw_tab, tab.data(), sizeof(int) * tab.size(), cudaMemcpyHostToDevice,
                           s->st));
  AFQ_CUDA(cudaMemcpyAsync(b.smw_prow, prow.data(), sizeof(int) * prow.size(),
                           cudaMemcpyHostToDevice, s->st));
  AFQ_CUDA(cudaStreamSynchronize(s->st));
  s->smw = true;
  s->smw_np[0] = np[0];
  s->smw_np[1] = np[1];
  return AFQMC_OK;
}

static int smw_chunks(const afqmc_params& p) { return (p.nchol + kSmwGC - 1) / kSmwGC; }

static int smw_overlap_update(afqmc_state* s, bool into_ld) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int W = p.nwalkers, N = p.N, M = p.M, nd = p.ndet;
  const size_t smem = sizeof(double2) * (size_t)N * 2 * N;
  AFQ_CUDA(cudaFuncSetAttribute(k_md_overlap, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem));
  // determinant 0 only: S_0s, log det, Theta_0s (md_ld rows [w][s])
  AFQ_LAUNCH(k_md_overlap, dim3(2, W), 256, smem, s->st, W, M, N, b.md_V, b.phiT, b.wt,
             b.md_theta, b.md_ld, nullptr, b.lo_kind, b.Mp);
  AFQ_LAUNCH(k_smw_ratio, W, 128, 0, s->st, W, M, N, nd, kSmwMaxK * nd, s->smw_np[0],
             s->smw_np[1], b.smw_tab, b.smw_prow, b.md_V, b.md_theta, b.md_ld, b.md_logA, b.wt,
             b.smw_xi, b.md_w, into_ld ? b.ld : b.ld_new);
  return AFQMC_OK;
}

static int smw_force_bias(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int nchk = smw_chunks(p);
  const size_t smem = sizeof(double2) * 2 * (size_t)p.N * p.N;
  AFQ_LAUNCH(k_smw_terms<false>, dim3(nchk, p.nwalkers), 256, smem, s->st, p.nwalkers, p.M, p.N,
             p.nchol, p.ndet, kSmwMaxK * p.ndet, nchk, p.H0, b.smw_tab, b.md_Lh, b.md_hh,
             b.md_theta, b.smw_xi, b.md_w, b.wt, b.t, nullptr);
  if (b.mixed) {
    const long n = 2L * p.nwalkers * p.nchol;
    AFQ_LAUNCH(k_smw_t32, cdiv((size_t)n, 256), 256, 0, s->st, n, b.t, b.t32);
  }
  return AFQMC_OK;
}

static int smw_local_energies(afqmc_state* s) {
  const afqmc_params& p = s->p;
  const Bufs& b = s->b;
  const int nchk = smw_chunks(p);
  const size_t smem = sizeof(double2) * 2 * (size_t)p.N * p.N;
  AFQ_LAUNCH(k_smw_terms<true>, dim3(nchk + 1, p.nwalkers), 256, smem, s->st, p.nwalkers, p.M,
             p.N, p.nchol, p.ndet, kSmwMaxK * p.ndet, nchk, p.H0, b.smw_tab, b.md_Lh, b.md_hh,
             b.md_theta, b.smw_xi, b.md_w, b.wt, nullptr, b.smw_part);
  AFQ_LAUNCH(k_smw_eloc, cdiv(p.nwalkers, 128), 128, 0, s->st, p.nwalkers, p.ndet, nchk, b.md_w,
             b.smw_part, b.wt, b.eloc);
  return AFQMC_OK;
}

int md_overlap_update(afqmc_state* s, bool into_ld) {
  if (s->smw) return smw_overlap_update(s, into_ld);
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
  if (s->smw) return smw_force_bias(s);
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
  if (s->smw) return smw_local_energies(s);
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
