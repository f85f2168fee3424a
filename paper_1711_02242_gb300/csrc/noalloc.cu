// Local energies without any device allocation by the library or the caller.
//
// afqmc_local_energies_noalloc() is the float64 local-energy evaluation of
// afqmc_local_energies() (force-bias traces, exchange contraction and the
// combination into E_loc) for callers that cannot allocate device memory: a
// host program whose device memory is all owned by another framework's pool
// and may not grow, or code that must not call cudaMalloc because the
// allocation would synchronise the device in the middle of its own stream
// work.  Such a caller passes only its inputs and outputs; the intermediate
// results live in the fixed array below, which every GPU that loads this
// library reserves (16 MiB) until the process exits.
#include <mutex>

#include "kernels.cuh"

namespace afq {
namespace {

constexpr long kScratchDoubles = 1l << 21;  // 16 MiB of float64 scratch
static __device__ __align__(256) double g_eloc_scratch[kScratchDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double* g_scratch_ptr[kMaxDevices] = {nullptr};

// Device address of the scratch array on the current device.  The host-side
// symbol is only a stand-in, never a device address, so the address comes
// from cudaGetSymbolAddress with the device current.  It is looked up again on
// every call made outside stream capture (a cudaDeviceReset() or a new
// primary context reloads the module at a new address, so a remembered one
// could dangle); during capture the address remembered from the last call
// outside capture on this device is used, and if there is none the call fails.
int scratch_on_current_device(cudaStream_t st, double** out) {
  int dev = -1;
  AFQ_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("device ordinal %d out of range", dev);
    return AFQMC_EINVAL;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  AFQ_CUDA(cudaStreamIsCapturing(st, &cs));
  std::lock_guard<std::mutex> lk(g_mu);
  if (cs == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    AFQ_CUDA(cudaGetSymbolAddress(&p, g_eloc_scratch));
    g_scratch_ptr[dev] = static_cast<double*>(p);
  } else if (!g_scratch_ptr[dev]) {
    set_error("afqmc_local_energies_noalloc: the first call on a device must come before any "
              "stream capture (it looks up the scratch array's device address)");
    return AFQMC_ESTATE;
  }
  *out = g_scratch_ptr[dev];
  return AFQMC_OK;
}

}  // namespace
}  // namespace afq

extern "C" AFQMC_API int afqmc_local_energies_noalloc(int32_t M, int32_t N, int32_t nchol,
                                                      int32_t nwalkers, const double* d_Lh,
                                                      const double* d_hh,
                                                      const double* d_thetaT, double H0,
                                                      double* d_eloc, void* stream) {
  using namespace afq;
  if (M < 1 || N < 1 || N > M || nchol < 1 || nwalkers < 1 || !d_Lh || !d_hh || !d_thetaT ||
      !d_eloc) {
    set_error("afqmc_local_energies_noalloc: bad arguments");
    return AFQMC_EINVAL;
  }
  if (N > 64) {
    set_error("afqmc_local_energies_noalloc: N=%d above 64", N);
    return AFQMC_EUNSUPPORTED;
  }
  if (nwalkers > 65535) {
    // the exchange kernel's grid has one row of blocks per walker
    set_error("afqmc_local_energies_noalloc: nwalkers=%d above 65535 (split the walkers over "
              "several calls)", nwalkers);
    return AFQMC_EINVAL;
  }
  const int gc = exchange_chunk(N, nchol);
  const int nchunk = (nchol + gc - 1) / gc;
  const long need = (long)nwalkers * 2 * nchol + (long)nwalkers * nchunk * 2;
  if (need > kScratchDoubles) {
    set_error("afqmc_local_energies_noalloc: needs %ld float64 of scratch, the fixed array "
              "holds %ld (use fewer walkers per call)",
              need, kScratchDoubles);
    return AFQMC_ENOSPC;
  }
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  double* scratch = nullptr;
  AFQ_TRY(scratch_on_current_device(st, &scratch));
  double* t = scratch;                            // [W][2][G], fully written below
  double* part = scratch + (long)nwalkers * 2 * nchol;  // [W][nchunk][2], fully written
  GemmF64 g;
  g.m = 2 * nwalkers;
  g.n = nchol;
  g.k = N * M;
  g.alpha = 2.0;
  g.A = d_thetaT;
  g.lda = (long)N * M;
  g.B = d_Lh;
  g.ldb = (long)N * M;
  g.C = t;
  g.ldc = nchol;
  AFQ_TRY(gemm_nt_f64(g, st));
  ExchArgs ex{nwalkers, M, N, nchol, gc, nchunk, d_Lh, d_thetaT, part, nullptr};
  AFQ_TRY(launch_exchange(ex, st));
  ElocArgs el{nwalkers, M, N, nchol, nchunk, H0, d_hh, d_thetaT, t, part, d_eloc, nullptr};
  AFQ_TRY(launch_eloc(el, st));
  return AFQMC_OK;
}
