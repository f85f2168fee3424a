// Modified Cholesky decomposition of the two-electron matrix (Sec. 2.3, Eqs.
// chol and chol2) on the GPU.
//
// V is the symmetric positive semi-definite matrix V_{mu nu} = v_pqrs with
// mu = (p, r), nu = (q, s), resident in device memory.  Vectors are found one
// at a time: pivot nu0 on the largest residual diagonal Delta_max, stop when
// Delta_max < delta, zero every index whose sqrt(|Delta_mm| Delta_max) is at
// most min(1e-9, delta) (damped prescreening), and take
//     L_mu = (V_{mu nu0} - sum_g L^g_mu L^g_nu0) / sqrt(Delta_max),
//     Delta_mm -= L_mu^2.
// Only the residual diagonal is kept; each iteration reads row nu0 of V (V is
// symmetric) and the vectors found so far, so one iteration streams
// 8 dim (k + 1) bytes after k vectors: an HBM-bound matrix-vector product.
//
// One launch per iteration.  A block owns 32 consecutive indices mu, one
// per lane, and its 8 warps split the earlier vectors g: warp w reads
// L[g][mu0 .. mu0+31] (256 contiguous bytes of the caller's output) for
// g = w, w+8, ... against the pivot's components L[g][nu0], staged in shared
// memory; the 8 partial sums are added in a fixed order.  The next pivot is
// the (value, index) maximum over the grid: each block writes its maximum
// (with the new vector's value there) and the last block to finish (a ticket
// counter, no waiting) reduces them, gathers the new pivot's components for
// the next launch and writes the state it reads.  Ties go to the smallest
// index, as in the oracle.
#include <climits>
#include <type_traits>

#include "kernels.cuh"

namespace afq {
namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kInitGrid = 1024;
constexpr int kMaxVectors = 16384;
constexpr int kFan = 64;             // arrivals per ticket in the reduction tree
constexpr double kScreen = 1e-9;  // floor of the prescreening threshold

struct McdState {
  double dmax;      // largest residual diagonal
  int32_t piv;      // its index (smallest among equal maxima)
  int32_t n;        // vectors so far
  int32_t done;     // 0 running, 1 converged, 2 max_vectors reached, 3 non-finite
  uint32_t ticket;  // fans of the current launch that have finished
};

struct McdPartial {
  double v;  // largest new residual diagonal of the block
  double l;  // the new vector's component at that index
  int32_t i;
  int32_t bad;
};

// Buffers of the grid-wide maximum: one partial per unit, one per fan of
// kFan units, and a ticket per fan.
struct McdTree {
  McdPartial* part;
  McdPartial* spart;
  uint32_t* sticket;
};

__device__ inline bool ahead(double v, int i, double bv, int bi) {
  return v > bv || (v == bv && i < bi);
}

// (value, index) maximum over a warp, first index among equal values, with a
// payload; every lane returns the result.
__device__ inline void warp_argmax(double& v, int& i, double& l, int& bad) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int oi = __shfl_xor_sync(0xffffffffu, i, o);
    const double ol = __shfl_xor_sync(0xffffffffu, l, o);
    bad |= __shfl_xor_sync(0xffffffffu, bad, o);
    if (ahead(ov, oi, v, i)) {
      v = ov;
      i = oi;
      l = ol;
    }
  }
}

// The same over the block; every thread returns the result.
__device__ inline void block_argmax(double& v, int& i, double& l, int& bad) {
  __shared__ double sv[kWarps], sl[kWarps];
  __shared__ int si[kWarps], sb[kWarps];
  warp_argmax(v, i, l, bad);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
    sv[wid] = v;
    si[wid] = i;
    sl[wid] = l;
    sb[wid] = bad;
  }
  __syncthreads();
  v = sv[0];
  i = si[0];
  l = sl[0];
  bad = sb[0];
  for (int w = 1; w < kWarps; ++w) {
    if (ahead(sv[w], si[w], v, i)) {
      v = sv[w];
      i = si[w];
      l = sl[w];
    }
    bad |= sb[w];
  }
}

// Arrival at one level of the reduction tree: the block publishes its
// (value, index, payload) maximum in parts[slot] and takes a ticket on
// *ticket; the last of the `count` arrivals (parts[first .. first+count))
// gets their maximum in (v, i, l, bad), resets the ticket and returns true.
// At most 64 blocks share a ticket, so the atomics never pile up on one
// address.
__device__ bool arrive(McdPartial* parts, int slot, int first, int count, uint32_t* ticket,
                       double& v, int& i, double& l, int& bad) {
  __shared__ int last;
  if (threadIdx.x == 0) {
    parts[slot] = McdPartial{v, l, i, bad};
    __threadfence();
    last = atomicAdd(ticket, 1u) == (unsigned)count - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  v = -INFINITY;
  l = 0.0;
  i = INT_MAX;
  bad = 0;
  for (int b = threadIdx.x; b < count; b += kThreads) {
    const McdPartial* p = parts + first + b;
    const double pv = __ldcg(&p->v), pl = __ldcg(&p->l);
    const int pi = __ldcg(&p->i);
    bad |= __ldcg(&p->bad);
    if (ahead(pv, pi, v, i)) {
      v = pv;
      i = pi;
      l = pl;
    }
  }
  block_argmax(v, i, l, bad);
  if (threadIdx.x == 0) *ticket = 0;
  return true;
}

// Grid-wide maximum over `nunits` units (unit u = one block's result):
// units arrive in fans of kFan, the last of each fan reduces it and arrives
// at the top level; the last block there holds the grid's maximum.
__device__ bool grid_argmax(McdPartial* part, McdPartial* spart, uint32_t* sticket,
                            uint32_t* top, int unit, int nunits, double& v, int& i, double& l,
                            int& bad) {
  const int fan = unit / kFan;
  const int nfan = (nunits + kFan - 1) / kFan;
  const int first = fan * kFan;
  const int count = nunits - first < kFan ? nunits - first : kFan;
  if (!arrive(part, unit, first, count, &sticket[fan], v, i, l, bad)) return false;
  return arrive(spart, fan, 0, nfan, top, v, i, l, bad);
}

// The grid's last block: record the pivot for the next iteration, gather its
// components L[0..n_next)[piv] into apiv (the last one, from this launch,
// travels in the partial) and write the state the next launch reads.
__device__ void next_pivot(McdState* st, const double* L, int64_t dim, double* apiv, double bv,
                           int bi, double bl, int bb, double delta, int max_vectors, int n_next) {
  const bool ok = !bb && isfinite(bv);
  if (ok && n_next > 0 && n_next < max_vectors) {
    // vectors g < n_next - 1 come from earlier launches
    const int kprev = n_next - 1;  // strided loads, eight in flight per thread
    for (int g0 = threadIdx.x; g0 < kprev; g0 += 8 * kThreads) {
      double x[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = g0 + u * kThreads;
        x[u] = g < kprev ? L[(int64_t)g * dim + bi] : 0.0;
      }
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int g = g0 + u * kThreads;
        if (g < kprev) apiv[g] = x[u];
      }
    }
    if (threadIdx.x == 0) apiv[kprev] = bl;
  }
  if (threadIdx.x == 0) {
    st->dmax = bv;
    st->piv = bi;
    st->n = n_next;
    if (!ok)
      st->done = 3;
    else if (bv < delta)
      st->done = 1;
    else if (n_next >= max_vectors)
      st->done = 2;
  }
}

// Residual diagonal d = diag(V) and the first pivot.
__global__ void __launch_bounds__(kThreads)
    k_mcd_init(const double* __restrict__ V, int64_t dim, double* __restrict__ d, double delta,
               int max_vectors, McdTree tree, McdState* st) {
  double bv = -INFINITY, bl = 0.0;
  int bi = INT_MAX, bad = 0;
  for (int64_t mu = (int64_t)blockIdx.x * kThreads + threadIdx.x; mu < dim;
       mu += (int64_t)gridDim.x * kThreads) {
    const double x = V[mu * dim + mu];
    d[mu] = x;
    if (!isfinite(x)) bad = 1;
    if (ahead(x, (int)mu, bv, bi)) {
      bv = x;
      bi = (int)mu;
    }
  }
  block_argmax(bv, bi, bl, bad);
  if (grid_argmax(tree.part, tree.spart, tree.sticket, &st->ticket, blockIdx.x, gridDim.x, bv, bi,
                  bl, bad))
    next_pivot(st, nullptr, dim, nullptr, bv, bi, bl, bad, delta, max_vectors, 0);
}

// One vector (Eq. chol2) and the residual-diagonal update.  Block b takes
// the 32 VEC indices from mu0 = 32 VEC b, VEC adjacent ones per lane (16-byte
// loads when VEC = 2, which needs an even dim), and its 8 warps split the
// earlier vectors; warp 0 forms the new vector from the 8 partial sums, added
// in a fixed order.
template <int VEC>
__global__ void __launch_bounds__(kThreads, VEC == 2 ? 4 : 5)
    k_mcd_step(const double* __restrict__ V, int64_t dim, double* __restrict__ d, double* L,
               double* apiv, int32_t* __restrict__ pivots, double delta, double tau,
               int max_vectors, McdTree tree, McdState* st) {
  using T = typename std::conditional<VEC == 2, double2, double>::type;
  extern __shared__ __align__(16) double a_sm[];  // L[g][nu0], g < k
  __shared__ double red[kWarps][32 * VEC];
  if (st->done) return;  // uniform: written only by the previous launch
  const int k = st->n;
  const int piv = st->piv;
  const double dmax = st->dmax;
  for (int g = threadIdx.x; g < k; g += kThreads) a_sm[g] = apiv[g];
  if (blockIdx.x == 0 && threadIdx.x == 0 && pivots) pivots[k] = piv;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t mu = ((int64_t)blockIdx.x * 32 + lane) * VEC;
  const bool valid = mu < dim;
  // warp 0 fetches its residual diagonals and pivot-row entries of V early
  double dm[VEC], vv[VEC];
  if (wid == 0 && valid) {
    const T dt = *reinterpret_cast<const T*>(d + mu);
    const T vt = *reinterpret_cast<const T*>(V + (int64_t)piv * dim + mu);
    if constexpr (VEC == 2) {
      dm[0] = dt.x, dm[1] = dt.y, vv[0] = vt.x, vv[1] = vt.y;
    } else {
      dm[0] = dt, vv[0] = vt;
    }
  }
  __syncthreads();
  // sum_g L[g][mu] L[g][nu0] over this warp's g = wid + 8 j, eight loads in flight
  const T* col = reinterpret_cast<const T*>(L + (valid ? mu : 0));
  const int64_t ld = dim / VEC;
  double acc[VEC][4];
#pragma unroll
  for (int c = 0; c < VEC; ++c) acc[c][0] = acc[c][1] = acc[c][2] = acc[c][3] = 0.0;
  int g = wid;
  for (; g + 56 < k; g += 64) {
    T x[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = col[(int64_t)(g + 8 * u) * ld];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const double a = a_sm[g + 8 * u];
      if constexpr (VEC == 2) {
        acc[0][u & 3] = fma(x[u].x, a, acc[0][u & 3]);
        acc[1][u & 3] = fma(x[u].y, a, acc[1][u & 3]);
      } else {
        acc[0][u & 3] = fma(x[u], a, acc[0][u & 3]);
      }
    }
  }
  for (; g < k; g += 8) {
    const T x = col[(int64_t)g * ld];
    if constexpr (VEC == 2) {
      acc[0][0] = fma(x.x, a_sm[g], acc[0][0]);
      acc[1][0] = fma(x.y, a_sm[g], acc[1][0]);
    } else {
      acc[0][0] = fma(x, a_sm[g], acc[0][0]);
    }
  }
#pragma unroll
  for (int c = 0; c < VEC; ++c)
    red[wid][lane * VEC + c] = (acc[c][0] + acc[c][1]) + (acc[c][2] + acc[c][3]);
  __syncthreads();
  double bv = -INFINITY, bl = 0.0;
  int bi = INT_MAX, bad = 0;
  if (wid == 0 && valid) {
    double lv[VEC], nd[VEC];
#pragma unroll
    for (int c = 0; c < VEC; ++c) {
      double s = red[0][lane * VEC + c];
#pragma unroll
      for (int w = 1; w < kWarps; ++w) s += red[w][lane * VEC + c];
      const bool screened = sqrt(__dmul_rn(fabs(dm[c]), dmax)) <= tau;
      lv[c] = screened ? 0.0 : (vv[c] - s) / sqrt(dmax);
      nd[c] = screened ? 0.0 : __dsub_rn(dm[c], __dmul_rn(lv[c], lv[c]));
      if (!isfinite(nd[c])) bad = 1;
      if (ahead(nd[c], (int)(mu + c), bv, bi)) {
        bv = nd[c];
        bi = (int)(mu + c);
        bl = lv[c];
      }
    }
    if constexpr (VEC == 2) {
      *reinterpret_cast<double2*>(L + (int64_t)k * dim + mu) = make_double2(lv[0], lv[1]);
      *reinterpret_cast<double2*>(d + mu) = make_double2(nd[0], nd[1]);
    } else {
      L[(int64_t)k * dim + mu] = lv[0];
      d[mu] = nd[0];
    }
  }
  block_argmax(bv, bi, bl, bad);
  if (grid_argmax(tree.part, tree.spart, tree.sticket, &st->ticket, blockIdx.x, gridDim.x, bv, bi,
                  bl, bad))
    next_pivot(st, L, dim, apiv, bv, bi, bl, bad, delta, max_vectors, k + 1);
}

struct McdLayout {
  size_t state, part, spart, sticket, d, apiv, total;
};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

McdLayout mcd_layout(int64_t dim, int32_t max_vectors) {
  McdLayout l;
  const int64_t groups = (dim + 31) / 32;  // blocks of a step launch, at most
  const int64_t nparts = groups > kInitGrid ? groups : kInitGrid;
  const int64_t nfans = (nparts + kFan - 1) / kFan;
  l.state = 0;
  l.part = align256(sizeof(McdState));
  l.spart = l.part + align256(sizeof(McdPartial) * (size_t)nparts);
  l.sticket = l.spart + align256(sizeof(McdPartial) * (size_t)nfans);
  l.d = l.sticket + align256(sizeof(uint32_t) * (size_t)nfans);
  l.apiv = l.d + align256(sizeof(double) * (size_t)dim);
  l.total = l.apiv + align256(sizeof(double) * (size_t)max_vectors);
  return l;
}

int mcd_check(int64_t dim, int32_t max_vectors) {
  if (dim < 1 || dim > INT_MAX) {
    set_error("modified Cholesky: dimension %lld outside [1, 2^31)", (long long)dim);
    return AFQMC_EINVAL;
  }
  if (max_vectors < 1 || max_vectors > kMaxVectors) {
    set_error("modified Cholesky: max_vectors %d outside [1, %d]", max_vectors, kMaxVectors);
    return AFQMC_EINVAL;
  }
  return AFQMC_OK;
}

// The decomposition of the dim x dim matrix V into the rows of L (pitch
// dim), with the workspace laid out by mcd_layout(dim, max_vectors) at base.
int run_mcd(int64_t dim, const double* d_V, double delta, int32_t max_vectors, double* d_L,
            int32_t* d_piv, int32_t* nvec, double* residual, char* base, const McdLayout& lay,
            cudaStream_t s, const char* who) {
  McdState* st = reinterpret_cast<McdState*>(base + lay.state);
  McdTree tree{reinterpret_cast<McdPartial*>(base + lay.part),
               reinterpret_cast<McdPartial*>(base + lay.spart),
               reinterpret_cast<uint32_t*>(base + lay.sticket)};
  double* d = reinterpret_cast<double*>(base + lay.d);
  double* apiv = reinterpret_cast<double*>(base + lay.apiv);
  const double tau = delta < kScreen ? delta : kScreen;
  // two indices per lane (16-byte accesses) when dim is even and V, L are
  // 16-byte aligned
  const int vec = dim % 2 == 0 && reinterpret_cast<uintptr_t>(d_V) % 16 == 0 &&
                          reinterpret_cast<uintptr_t>(d_L) % 16 == 0
                      ? 2
                      : 1;
  const size_t smem_max = sizeof(double) * (size_t)max_vectors;
  auto step = vec == 2 ? k_mcd_step<2> : k_mcd_step<1>;
  AFQ_CUDA(cudaFuncSetAttribute(step, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)smem_max));
  const unsigned grid = (unsigned)((dim + 32 * vec - 1) / (32 * vec));
  int64_t grid0 = (dim + kThreads - 1) / kThreads;
  if (grid0 > kInitGrid) grid0 = kInitGrid;

  AFQ_CUDA(cudaMemsetAsync(st, 0, sizeof(McdState), s));
  AFQ_CUDA(cudaMemsetAsync(base + lay.sticket, 0, lay.d - lay.sticket, s));
  AFQ_LAUNCH(k_mcd_init, (unsigned)grid0, kThreads, 0, s, d_V, dim, d, delta, max_vectors, tree,
             st);
  // Launch iterations in chunks and read the state between chunks; launches
  // after convergence return at once.  A launch after `launched` others
  // finds k <= launched earlier vectors, which sizes its shared memory.
  McdState hs{};
  int launched = 0;
  for (;;) {
    AFQ_CUDA(cudaMemcpyAsync(&hs, st, sizeof hs, cudaMemcpyDeviceToHost, s));
    AFQ_CUDA(cudaStreamSynchronize(s));
    if (hs.done || launched >= max_vectors) break;
    int chunk = launched < 64 ? 16 : 64;
    if (chunk > max_vectors - launched) chunk = max_vectors - launched;
    for (int c = 0; c < chunk; ++c) {
      const size_t smem = sizeof(double) * (size_t)(launched + 1);
      AFQ_LAUNCH(step, grid, kThreads, smem, s, d_V, dim, d, d_L, apiv, d_piv, delta, tau,
                 max_vectors, tree, st);
      ++launched;
    }
  }
  *nvec = hs.n;
  if (residual) *residual = hs.dmax;
  if (hs.done == 3) {
    set_error("%s: non-finite residual after %d vectors", who, hs.n);
    return AFQMC_ENONFINITE;
  }
  return AFQMC_OK;
}

// Pair index of p <= r: row-major order of the upper triangle.
__host__ __device__ inline int64_t pair_index(int64_t p, int64_t r, int64_t M) {
  return p * M - p * (p - 1) / 2 + (r - p);
}

// L[g][p][r] = L[g][r][p] = Lp[g][pair(min, max)] for the first nvec vectors.
__global__ void k_mcd_expand(const double* __restrict__ Lp, int64_t npair, int M,
                             double* __restrict__ L) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= M * M) return;
  const int p = t / M, r = t - p * M;
  const int a = p < r ? p : r, b = p < r ? r : p;
  const int64_t g = blockIdx.y;
  L[g * M * M + t] = Lp[g * npair + pair_index(a, b, M)];
}

// Pivots from pair index to p M + r (p <= r).
__global__ void k_mcd_pivots_full(int32_t* piv, int n, int M) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t P = piv[i];
  int p = 0;
  while (p + 1 < M && pair_index(p + 1, p + 1, M) <= P) ++p;
  piv[i] = (int32_t)(p * (int64_t)M + p + (P - pair_index(p, p, M)));
}

int64_t npair_of(int64_t M) { return M * (M + 1) / 2; }

size_t mcd_pairs_bytes(int64_t M, int32_t max_vectors) {
  const int64_t np = npair_of(M);
  return mcd_layout(np, max_vectors).total + align256(sizeof(double) * (size_t)np * max_vectors);
}

}  // namespace
}  // namespace afq

extern "C" AFQMC_API int afqmc_mcd_workspace_size(int64_t dim, int32_t max_vectors,
                                                  size_t* bytes) {
  using namespace afq;
  if (!bytes) {
    set_error("afqmc_mcd_workspace_size: bytes is NULL");
    return AFQMC_EINVAL;
  }
  AFQ_TRY(mcd_check(dim, max_vectors));
  *bytes = mcd_layout(dim, max_vectors).total;
  return AFQMC_OK;
}

extern "C" AFQMC_API int afqmc_modified_cholesky(int64_t dim, const double* d_V, double delta,
                                                 int32_t max_vectors, double* d_L,
                                                 int32_t* d_piv, int32_t* nvec, double* residual,
                                                 void* d_work, size_t work_bytes, void* stream) {
  using namespace afq;
  AFQ_TRY(mcd_check(dim, max_vectors));
  if (!d_V || !d_L || !nvec || !d_work || !(delta > 0.0) || !std::isfinite(delta)) {
    set_error("afqmc_modified_cholesky: NULL pointer or delta not a positive finite number");
    return AFQMC_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(d_work) % 256) {
    set_error("afqmc_modified_cholesky: workspace not 256-byte aligned");
    return AFQMC_EINVAL;
  }
  const McdLayout lay = mcd_layout(dim, max_vectors);
  if (work_bytes < lay.total) {
    set_error("afqmc_modified_cholesky: workspace %zu bytes, needs %zu", work_bytes, lay.total);
    return AFQMC_ENOSPC;
  }
  return run_mcd(dim, d_V, delta, max_vectors, d_L, d_piv, nvec, residual,
                 static_cast<char*>(d_work), lay, static_cast<cudaStream_t>(stream),
                 "afqmc_modified_cholesky");
}

extern "C" AFQMC_API int afqmc_mcd_pairs_workspace_size(int32_t M, int32_t max_vectors,
                                                        size_t* bytes) {
  using namespace afq;
  if (!bytes || M < 1 || M > 2048) {
    set_error("afqmc_mcd_pairs_workspace_size: NULL bytes or M outside [1, 2048]");
    return AFQMC_EINVAL;
  }
  AFQ_TRY(mcd_check(npair_of(M), max_vectors));
  *bytes = mcd_pairs_bytes(M, max_vectors);
  return AFQMC_OK;
}

extern "C" AFQMC_API int afqmc_modified_cholesky_pairs(int32_t M, const double* d_Vpair,
                                                       double delta, int32_t max_vectors,
                                                       double* d_L, int32_t* d_piv,
                                                       int32_t* nvec, double* residual,
                                                       void* d_work, size_t work_bytes,
                                                       void* stream) {
  using namespace afq;
  if (M < 1 || M > 2048) {
    set_error("afqmc_modified_cholesky_pairs: M=%d outside [1, 2048]", M);
    return AFQMC_EINVAL;
  }
  const int64_t np = npair_of(M);
  AFQ_TRY(mcd_check(np, max_vectors));
  if (!d_Vpair || !d_L || !nvec || !d_work || !(delta > 0.0) || !std::isfinite(delta)) {
    set_error("afqmc_modified_cholesky_pairs: NULL pointer or delta not a positive finite number");
    return AFQMC_EINVAL;
  }
  if (reinterpret_cast<uintptr_t>(d_work) % 256) {
    set_error("afqmc_modified_cholesky_pairs: workspace not 256-byte aligned");
    return AFQMC_EINVAL;
  }
  if (work_bytes < mcd_pairs_bytes(M, max_vectors)) {
    set_error("afqmc_modified_cholesky_pairs: workspace %zu bytes, needs %zu", work_bytes,
              mcd_pairs_bytes(M, max_vectors));
    return AFQMC_ENOSPC;
  }
  const McdLayout lay = mcd_layout(np, max_vectors);
  char* base = static_cast<char*>(d_work);
  double* Lp = reinterpret_cast<double*>(base + lay.total);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int rc = run_mcd(np, d_Vpair, delta, max_vectors, Lp, d_piv, nvec, residual, base, lay, s,
                         "afqmc_modified_cholesky_pairs");
  if (rc != AFQMC_OK) return rc;
  if (*nvec > 0) {
    AFQ_LAUNCH(k_mcd_expand, dim3(cdiv((size_t)M * M, 256), (unsigned)*nvec), 256, 0, s, Lp, np,
               M, d_L);
    if (d_piv) AFQ_LAUNCH(k_mcd_pivots_full, cdiv(*nvec, 256), 256, 0, s, d_piv, *nvec, M);
  }
  AFQ_CUDA(cudaStreamSynchronize(s));
  return rc;
}
