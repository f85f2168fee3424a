// One walker population split over several states (one per GPU): the pieces a
// host driver needs for the comb of Sec. 3.4.4 and for the mixed estimator
// over the whole population.  Walkers are independent between population
// controls (Sec. 3.5), so each state steps its own walkers (their fields keyed
// by their global index, params.walker0 + w); at a comb every state sees all
// weights, computes the same parents, and the walkers move between states as
// packed rows.
#include "kernels.cuh"
#include "state.cuh"

namespace afq {
int refresh_phi_lo(afqmc_state* s);
int refresh_theta_lo(afqmc_state* s);

namespace {

// The comb over the whole population, as the single-state comb does it:
// W_tot and the cumulative weights C_j are sequential float64 sums in global
// walker order; u from Philox counter (0, 0xffffffff, step - 1, 0) of the
// shared seed; tooth k = ((k + u) W_tot) / n goes to the first j with
// C_j > tooth (the last walker with positive weight if rounding puts it past
// C_{n-1}); parent[k] = -1 for every k when no weight is left.
__global__ void __launch_bounds__(256) k_comb_plan_all(const double* w, long n, double* cum,
                                                       uint64_t seed, const int64_t* dstep,
                                                       int* parent, double* wtot) {
  __shared__ double s_u, s_tot;
  __shared__ long s_last;
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    double s = 0.0;
    long last = -1;
    for (long j = 0; j < n; ++j) {
      const double wj = w[j];
      s += wj;
      cum[j] = s;
      if (wj > 0.0) last = j;
    }
    s_tot = s;
    wtot[0] = s;
    s_last = last;
    s_ok = (s > 0.0 && isfinite(s) && last >= 0) ? 1 : 0;
    u32x4 c = {0u, 0xFFFFFFFFu, (uint32_t)(*dstep - 1), 0u};
    u32x4 r = philox4x32_10(c, (uint32_t)seed, (uint32_t)(seed >> 32));
    s_u = uniform53(r.x, r.y);
  }
  __syncthreads();
  for (long k = threadIdx.x; k < n; k += blockDim.x) {
    if (!s_ok) {
      parent[k] = -1;
      continue;
    }
    const double tooth = (((double)k + s_u) * s_tot) / (double)n;
    long lo = 0, hi = n;  // first j with cum[j] > tooth
    while (lo < hi) {
      const long mid = (lo + hi) >> 1;
      if (cum[mid] > tooth) hi = mid; else lo = mid + 1;
    }
    parent[k] = (int)((lo >= n) ? s_last : lo);
  }
}

// Row r of `rows` = walker idx[r]: Phi^T, Theta^T (2 N M float64 each) and
// log <Psi_T|Psi> (2 float64).
__global__ void __launch_bounds__(256) k_pack_rows(const int* idx, int n, long nm2,
                                                   const double* phiT, const double* thetaT,
                                                   const double* ld, double* rows) {
  const int r = blockIdx.x;
  if (r >= n) return;
  const long j = idx[r];
  double* o = rows + (long)r * (2 * nm2 + 2);
  for (long i = threadIdx.x; i < nm2; i += blockDim.x) {
    o[i] = phiT[j * nm2 + i];
    o[nm2 + i] = thetaT[j * nm2 + i];
  }
  if (threadIdx.x < 2) o[2 * nm2 + threadIdx.x] = ld[2 * j + threadIdx.x];
}

// Walker slot[r] = row r, weight W_tot / n_all (real).
__global__ void __launch_bounds__(256) k_unpack_rows(const int* slot, int n, long nm2,
                                                     const double* rows, const double* wtot,
                                                     double n_all, double* phiT, double* thetaT,
                                                     double* ld, double* wt) {
  const int r = blockIdx.x;
  if (r >= n) return;
  const long k = slot[r];
  const double* src = rows + (long)r * (2 * nm2 + 2);
  for (long i = threadIdx.x; i < nm2; i += blockDim.x) {
    phiT[k * nm2 + i] = src[i];
    thetaT[k * nm2 + i] = src[nm2 + i];
  }
  if (threadIdx.x < 2) ld[2 * k + threadIdx.x] = src[2 * nm2 + threadIdx.x];
  if (threadIdx.x == 0) {
    wt[2 * k] = wtot[0] / n_all;
    wt[2 * k + 1] = 0.0;
  }
}

int check_population_state(afqmc_state* s) {
  if (!s || !s->valid) {
    set_error("invalid state");
    return AFQMC_ESTATE;
  }
  if (s->p.mode != AFQMC_PHASELESS || s->p.ndet > 0 || s->bp_on) {
    set_error("the comb acts on phaseless walks with a single-determinant trial and no open "
              "back-propagation window");
    return AFQMC_EUNSUPPORTED;
  }
  return AFQMC_OK;
}

}  // namespace
}  // namespace afq

using namespace afq;

extern "C" {

int afqmc_walker_row_bytes(afqmc_state* s, size_t* bytes) {
  if (!s || !s->valid || !bytes) {
    set_error("invalid state or NULL bytes");
    return !s || !s->valid ? AFQMC_ESTATE : AFQMC_EINVAL;
  }
  *bytes = sizeof(double) * (4 * (size_t)s->p.N * s->p.M + 2);
  return AFQMC_OK;
}

int afqmc_export_weights(afqmc_state* s, double* d_weights) {
  AFQ_TRY(check_population_state(s));
  if (!d_weights) {
    set_error("d_weights is NULL");
    return AFQMC_EINVAL;
  }
  // the real parts of the [W][2] weights
  AFQ_CUDA(cudaMemcpy2DAsync(d_weights, sizeof(double), s->b.wt, 2 * sizeof(double),
                             sizeof(double), s->p.nwalkers, cudaMemcpyDeviceToDevice, s->st));
  return AFQMC_OK;
}

int afqmc_comb_plan(afqmc_state* s, const double* d_weights_all, int64_t n_all, double* d_cum,
                    int32_t* d_parent_all) {
  AFQ_TRY(check_population_state(s));
  if (n_all < s->p.nwalkers || n_all > 0x7fffffffLL || !d_weights_all || !d_cum ||
      !d_parent_all) {
    set_error("afqmc_comb_plan: n_all = %lld below this state's walkers, or NULL buffers",
              (long long)n_all);
    return AFQMC_EINVAL;
  }
  const Bufs& b = s->b;
  AFQ_LAUNCH(k_comb_plan_all, 1, 256, 0, s->st, d_weights_all, (long)n_all, d_cum, s->p.seed,
             reinterpret_cast<const int64_t*>(b.counters + CTR_STEP), d_parent_all, b.wtot);
  s->comb_nall = n_all;
  return AFQMC_OK;
}

int afqmc_pack_walkers(afqmc_state* s, const int32_t* d_index, int32_t n, void* d_rows) {
  AFQ_TRY(check_population_state(s));
  if (n < 0 || (n > 0 && (!d_index || !d_rows))) {
    set_error("afqmc_pack_walkers: bad arguments");
    return AFQMC_EINVAL;
  }
  if (n == 0) return AFQMC_OK;
  const Bufs& b = s->b;
  const long nm2 = 2L * s->p.N * s->p.M;
  AFQ_LAUNCH(k_pack_rows, n, 256, 0, s->st, d_index, n, nm2, b.phiT, b.thetaT, b.ld,
             static_cast<double*>(d_rows));
  return AFQMC_OK;
}

int afqmc_unpack_walkers(afqmc_state* s, const int32_t* d_slot, int32_t n, const void* d_rows) {
  AFQ_TRY(check_population_state(s));
  if (n < 0 || (n > 0 && (!d_slot || !d_rows))) {
    set_error("afqmc_unpack_walkers: bad arguments");
    return AFQMC_EINVAL;
  }
  if (s->comb_nall <= 0) {
    set_error("afqmc_unpack_walkers: no afqmc_comb_plan on this state");
    return AFQMC_ESTATE;
  }
  const Bufs& b = s->b;
  const long nm2 = 2L * s->p.N * s->p.M;
  if (n > 0)
    AFQ_LAUNCH(k_unpack_rows, n, 256, 0, s->st, d_slot, n, nm2, static_cast<const double*>(d_rows),
               b.wtot, (double)s->comb_nall, b.phiT, b.thetaT, b.ld, b.wt);
  AFQ_TRY(refresh_phi_lo(s));
  AFQ_TRY(refresh_theta_lo(s));
  s->t_fresh = false;  // the walkers moved: their force-bias traces are stale
  return AFQMC_OK;
}

int afqmc_energy_sums(afqmc_state* s, double* d_sums) {
  if (!s || !s->valid || !d_sums) {
    set_error("invalid state or NULL d_sums");
    return !s || !s->valid ? AFQMC_ESTATE : AFQMC_EINVAL;
  }
  AFQ_CUDA(cudaMemcpyAsync(d_sums, s->b.last, 4 * sizeof(double), cudaMemcpyDeviceToDevice,
                           s->st));
  return AFQMC_OK;
}

}  // extern "C"
