// Whole Taylor series of exp(V) for one walker per CTA (Sec. 3.4.2, the
// truncated expansion of the exponential of the one-body operator) on tcgen05.
//
// For walker w the terms T_k = V T_{k-1} / k, k = 1..n, are formed one after
// another and summed, S = T_1 + ... + T_n (FP32); the last half step then
// applies exp(-dt v0'/2) to T_0 + S.  Per-term launches would stream every
// walker's V from HBM n times and read-modify-write the sum in global memory
// per term; here a CTA keeps the term in shared memory and the sum in tensor
// memory, streams only V (from L2 after the first term) and writes S once.
//
//   A operand  [Re V | Im V] rows p of walker w (128-row tiles, K = 2 Mp),
//              TMA ring whose stage is one 128-byte K block of every p-tile
//              (one 128-row box per tile), so that each stage feeds the MMAs
//              of all p-tiles, interleaved over independent accumulators;
//   B operand  the term T_{k-1} as K-major rows, NH = N rounded up to 16:
//                 row i      = [Re T_i | -Im T_i]   (i < N)
//                 row NH + i = [Im T_i |  Re T_i]
//              (rows i >= N of each half zero), resident in shared memory in
//              the 128-byte-swizzled layout TMA writes, one 1024-byte-aligned
//              block of 2NH x 128 bytes per 128 bytes of K;
//   D          TMEM lane p of p-tile pt, column pt * 2NH + n: (V T_{k-1})[p][n],
//              n = c NH + i (c = 0: real part, 1: imaginary part of row i);
//              the running sum S sits in the same layout PT * 2NH columns on.
//
// The epilogue warps read D, add T_k = D / k to S (tcgen05.ld / st) and,
// unless k = n, write T_k into the B operand in place (every MMA of term k has
// completed by then), then release the MMA thread for term k + 1; after the
// last term S goes to global memory with plain coalesced stores.  With NH a
// multiple of 16 every 16-column chunk of D is one half (real or imaginary)
// and its rows share their position within the 8-row swizzle atoms, so each
// thread computes the swizzled offsets of its two K columns (p and Mp + p)
// once per tile and a store costs one add.  Warp roles: warp 0 TMA producer,
// warp 1 TMEM allocation and the MMA thread, warps 2-17 epilogue (four warps
// per 32-lane quarter of TMEM, splitting the chunks).  Every wait is bounded;
// on time-out the kernel records an error and stops.
#include <cuda_bf16.h>

#include "kernels.cuh"
#include "tc.cuh"
#include "tc_dev.cuh"

namespace afq {
namespace tc {

constexpr int kVBox = BM * BKB;   // one V box: a 128-row p-tile x 128 bytes of K
constexpr int kEpiWarps = 16;     // epilogue warps (4 per TMEM lane quarter)
constexpr int kEpiThreads = 32 * kEpiWarps;
constexpr int kSeriesThreads = 64 + kEpiThreads;

struct SeriesArgs {
  float* S;     // [W][2N][lds]: S = T_1 + ... + T_n, columns p < M
  long lds;
  int W, M, N, Mp, order;
  int nh;       // N rounded up to 16: rows per half of the term operand
  int nb;       // 2 nh = MMA N
  int kblocks;  // 128-byte K blocks covering 2 Mp
  int ptiles;   // 128-row tiles covering p < M
  int stages;   // depth of the V ring (a stage: one K block of every p-tile)
  uint32_t tcols;
};

// Byte offsets, within the term operand, of K column kcol in rows 0..7 of a
// swizzle atom (add 1024 per further 8 rows).
template <bool TF32>
__device__ __forceinline__ void column_offsets(int kcol, uint32_t opk, uint32_t* off) {
  constexpr int ELEM = TF32 ? 4 : 2;
  constexpr int BK = BKB / ELEM;
  const int kb = kcol / BK;
  const uint32_t byte = (uint32_t)(kcol - kb * BK) * ELEM;
#pragma unroll
  for (int j = 0; j < 8; ++j)
    off[j] = (uint32_t)kb * opk + (uint32_t)j * 128u + ((((byte >> 4) ^ (uint32_t)j) << 4) | (byte & 15u));
}

template <bool TF32>
__device__ __forceinline__ void put_op(uint8_t* bop, uint32_t off, float v) {
  if constexpr (TF32)
    *reinterpret_cast<float*>(bop + off) = round_tf32(v);
  else
    *reinterpret_cast<__nv_bfloat16*>(bop + off) = __float2bfloat16_rn(v);
}

// Named barrier over the epilogue threads that also ORs a flag across them,
// so every epilogue warp takes the same branch.
__device__ __forceinline__ bool epi_sync_or(bool flag) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, %2, q;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(out)
      : "r"((uint32_t)flag), "n"(kEpiThreads)
      : "memory");
  return out != 0;
}

template <bool TF32>
__global__ void __launch_bounds__(kSeriesThreads, 1)
    k_taylor_series(const __grid_constant__ CUtensorMap tmV, const __grid_constant__ CUtensorMap tmT,
                    SeriesArgs a, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                             ~uintptr_t(1023));
  const uint32_t opk = (uint32_t)a.nb * BKB;  // bytes of one K block of the term operand
  uint8_t* bop = smem;
  uint8_t* ring = smem + (size_t)a.kblocks * opk;
  const uint32_t stage_bytes = (uint32_t)a.ptiles * kVBox;
  uint64_t* full = reinterpret_cast<uint64_t*>(ring + (size_t)a.stages * stage_bytes);
  uint64_t* empty = full + a.stages;
  uint64_t* bfull = empty + a.stages;  // T_0 of the walker has landed
  uint64_t* bfree = bfull + 1;         // the walker's last MMAs are done: operand space free
  uint64_t* dfull = bfree + 1;         // a term's product is complete in TMEM
  uint64_t* bnext = dfull + 1;         // epilogue done with a term (TMEM read, next term written)
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bnext + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int ELEM = TF32 ? 4 : 2;
  constexpr int BK = BKB / ELEM;
  constexpr int KSTEPS = BKB / 32;

  if (threadIdx.x == 0) {
    for (int s = 0; s < a.stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(bfull, 1);
    mbar_init(bfree, 1);
    mbar_init(dfull, 1);
    mbar_init(bnext, kEpiThreads);  // every epilogue thread arrives
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(a.tcols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    // producer: per walker T_0 once (rows (c, i) -> c NH + i by a 4-D box),
    // then the V tiles of every term
    int it = 0, j = 0, s = 0;
    uint32_t ph = 0;  // ring slot s and its fill round's parity, kept incrementally
    bool stop = false;
    for (int w = blockIdx.x; w < a.W && !stop; w += gridDim.x, ++j) {
      if (j > 0 && !mbar_wait(bfree, (j - 1) & 1, err, 31)) {
        stop = true;
        break;
      }
      mbar_expect_tx(bfull, (uint32_t)a.kblocks * opk);
      for (int kb = 0; kb < a.kblocks; ++kb)
        tma_load_4d(bop + kb * opk, &tmT, bfull, kb * BK, 0, 0, w);
      for (int k = 1; k <= a.order && !stop; ++k)
        for (int kb = 0; kb < a.kblocks; ++kb, ++it) {
          if ((it >= a.stages && !mbar_wait(&empty[s], ph ^ 1u, err, 32)) || *abort_flag) {
            stop = true;
            break;
          }
          mbar_expect_tx(&full[s], stage_bytes);
          for (int pt = 0; pt < a.ptiles; ++pt)
            tma_load_3d(ring + s * stage_bytes + pt * kVBox, &tmV, &full[s], kb * BK, pt * BM, w);
          if (++s == a.stages) {
            s = 0;
            ph ^= 1u;
          }
        }
    }
    if (stop) *abort_flag = 1;
  } else if (warp == 1 && lane == 0) {
    // MMA thread
    const uint32_t idesc = instr_desc(TF32 ? 2u : 1u, (uint32_t)a.nb);
    int g = 0, j = 0, s = 0;
    uint32_t ph = 0;
    bool stop = false;
    for (int w = blockIdx.x; w < a.W && !stop; w += gridDim.x, ++j) {
      for (int k = 1; k <= a.order; ++k, ++g) {
        if ((k == 1 && !mbar_wait(bfull, j & 1, err, 33)) ||
            (g > 0 && !mbar_wait(bnext, (g - 1) & 1, err, 34)) || *abort_flag) {
          stop = true;
          break;
        }
        fence_after();
        // one stage = one K block of every p-tile: the p-tiles' MMAs are
        // interleaved (independent accumulators)
        for (int kb = 0; kb < a.kblocks; ++kb) {
          if (!mbar_wait(&full[s], ph, err, 35)) {
            *abort_flag = 1;
            stop = true;
            break;
          }
          fence_after();
          const uint32_t av = smem_u32(ring + s * stage_bytes);
          const uint32_t bv = smem_u32(bop + kb * opk);
#pragma unroll
          for (int kk = 0; kk < KSTEPS; ++kk)
#pragma unroll
            for (int pt = 0; pt < 4; ++pt)
              if (pt < a.ptiles)
                mma<TF32>(tmem + (uint32_t)(pt * a.nb),
                          sw128_desc(av + (uint32_t)(pt * kVBox) + 32 * kk),
                          sw128_desc(bv + 32 * kk), idesc, (kb > 0 || kk > 0) ? 1u : 0u);
          mma_commit(&empty[s]);
          if (++s == a.stages) {
            s = 0;
            ph ^= 1u;
          }
        }
        mma_commit(dfull);
        if (k == a.order) mma_commit(bfree);
        if (stop) break;
      }
    }
    if (stop) *abort_flag = 1;
  } else if (warp >= 2) {
    // epilogue: warp quarter q holds TMEM lanes (p within the tile) 32q .. 32q + 31;
    // the four warps of a quarter take every fourth 16-column chunk
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t tl = tmem + ((uint32_t)(32 * q) << 16);
    const uint32_t soff = (uint32_t)(a.ptiles * a.nb);  // columns of the running sum
    const int N = a.N, NH = a.nh;
    const int nchunk = a.nb / 16;                      // chunks per p-tile
    int g = 0;
    bool stop = false;
    for (int w = blockIdx.x; w < a.W && !stop; w += gridDim.x) {
      for (int k = 1; k <= a.order; ++k, ++g) {
        bool bad = !mbar_wait_sleep(dfull, g & 1, err, 36) || *abort_flag;
        fence_after();
        if (epi_sync_or(bad)) {
          stop = true;
          break;
        }
        const float scale = 1.0f / (float)k;
        const bool next = k < a.order;
#pragma unroll 1
        for (int pt = 0; pt < a.ptiles; ++pt) {
          const int p = pt * BM + 32 * q + lane;
          const bool pv = p < a.M;
          uint32_t offp[8], offq[8];  // K columns p and Mp + p
          column_offsets<TF32>(p, opk, offp);
          column_offsets<TF32>(a.Mp + p, opk, offq);
#pragma unroll 1
          for (int ch = half; ch < nchunk; ch += kEpiWarps / 4) {
            const int c0 = ch * 16;
            const int cpart = c0 >= NH ? 1 : 0, i0 = c0 - cpart * NH;
            if (i0 >= N) continue;  // a chunk of padding rows only
            const uint32_t col = (uint32_t)(pt * a.nb + c0);
            uint32_t rd[16], rs[16];
            float v[16], sum[16];
            tmem_ld16_async(tl + col, rd);
            if (k > 1) tmem_ld16_async(tl + soff + col, rs);
            tmem_ld_wait();
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              v[u] = __uint_as_float(rd[u]) * scale;
              sum[u] = (k > 1 ? __uint_as_float(rs[u]) : 0.f) + v[u];
            }
            if (next) {
              tmem_st16(tl + soff + col, sum);
            } else if (pv) {
              float* srow = a.S + ((long)w * 2 * N + cpart * N + i0) * a.lds + p;
#pragma unroll
              for (int u = 0; u < 16; ++u)
                if (i0 + u < N) srow[(long)u * a.lds] = sum[u];
            }
            if (!next || !pv) continue;
            // row i gets column p (real half) or Mp + p negated (imaginary
            // half); row NH + i gets the other column
            const uint32_t ra = (uint32_t)(i0 >> 3) * 1024u;
            const uint32_t rb = ra + (uint32_t)(NH >> 3) * 1024u;
            const float sa = cpart ? -1.f : 1.f;
#pragma unroll
            for (int u = 0; u < 16; ++u) {
              if (i0 + u >= N) break;
              const uint32_t blk = (uint32_t)(u >> 3) * 1024u;
              const uint32_t oa = cpart ? offq[u & 7] : offp[u & 7];
              const uint32_t ob = cpart ? offp[u & 7] : offq[u & 7];
              put_op<TF32>(bop, oa + ra + blk, sa * v[u]);
              put_op<TF32>(bop, ob + rb + blk, v[u]);
            }
          }
        }
        tmem_st_wait();
        // generic-proxy writes of the next term -> visible to the MMA (async proxy)
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        fence_before();
        mbar_arrive(bnext);
      }
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tcols));
  }
}

}  // namespace tc

namespace {
constexpr int kSmemMax = 232448;
constexpr int kSmemFixed = 1024 /*align*/ + 256 /*barriers*/;

bool series_plan(int lo_kind, int N, int M, int Mp, tc::SeriesArgs* sa, int* smem) {
  if (N < 1 || M < 1 || Mp < M || Mp % 16) return false;
  const int elem = lo_kind == LO_TF32 ? 4 : 2;
  const int nh = (N + 15) / 16 * 16;
  const int nb = 2 * nh;
  const int kblocks = (2 * Mp * elem + tc::BKB - 1) / tc::BKB;
  const int ptiles = (M + tc::BM - 1) / tc::BM;
  // the product and the running sum side by side in tensor memory
  if (nb > 256 || 2 * ptiles * nb > 512 || ptiles > 4) return false;
  const long op = (long)kblocks * nb * tc::BKB;
  long room = kSmemMax - kSmemFixed - op;
  int stages = (int)(room / ((long)ptiles * tc::kVBox));
  if (stages > 8) stages = 8;
  if (stages < 2) return false;
  uint32_t tcols = 32;
  while (tcols < (uint32_t)(2 * ptiles * nb)) tcols <<= 1;
  if (sa) {
    sa->nh = nh;
    sa->nb = nb;
    sa->kblocks = kblocks;
    sa->ptiles = ptiles;
    sa->stages = stages;
    sa->tcols = tcols;
  }
  if (smem) *smem = (int)(op + (long)stages * ptiles * tc::kVBox + kSmemFixed);
  return true;
}
}  // namespace

bool tc_taylor_series_fits(int lo_kind, int N, int M, int Mp) {
  return series_plan(lo_kind, N, M, Mp, nullptr, nullptr);
}

int tc_taylor_series(const void* V, const void* T0, float* S, long lds, int lo_kind, int W, int N,
                     int M, int Mp, int order, int* err, cudaStream_t st) {
  tc::SeriesArgs sa{};
  int smem = 0;
  if (!series_plan(lo_kind, N, M, Mp, &sa, &smem)) {
    set_error("taylor series kernel: shape N=%d M=%d does not fit", N, M);
    return AFQMC_EUNSUPPORTED;
  }
  if (W <= 0 || order <= 0) return AFQMC_OK;
  sa.S = S;
  sa.lds = lds;
  sa.W = W;
  sa.M = M;
  sa.N = N;
  sa.Mp = Mp;
  sa.order = order;
  const bool tf32 = lo_kind == LO_TF32;
  const int eb = tf32 ? 4 : 2;
  CUtensorMap tv, tt;
  AFQ_TRY(make_tmap_3d(&tv, V, eb, W, M, 2L * Mp, 2L * Mp, (long)M * 2 * Mp, tc::BM));
  // T0 rows (w, c, i) -> operand rows c NH + i: dims (K, i, c, w), box (K block, NH, 2, 1)
  const long tdims[4] = {2L * Mp, N, 2, W};
  const long tstr[3] = {2L * Mp * eb, (long)N * 2 * Mp * eb, 2L * N * 2 * Mp * eb};
  const int tbox[4] = {tc::BKB / eb, sa.nh, 2, 1};
  AFQ_TRY(make_tmap_nd(&tt, T0, eb, 4, tdims, tstr, tbox));
  const int grid = W < tc_sm_count() ? W : tc_sm_count();
  if (tf32) {
    static std::atomic<unsigned long long> attr{0};
    AFQ_TRY(smem_attr_once(tc::k_taylor_series<true>, kSmemMax, attr));
    AFQ_LAUNCH(tc::k_taylor_series<true>, grid, tc::kSeriesThreads, smem, st, tv, tt, sa, err);
  } else {
    static std::atomic<unsigned long long> attr{0};
    AFQ_TRY(smem_attr_once(tc::k_taylor_series<false>, kSmemMax, attr));
    AFQ_LAUNCH(tc::k_taylor_series<false>, grid, tc::kSeriesThreads, smem, st, tv, tt, sa, err);
  }
  return AFQMC_OK;
}

int taylor_apply(const void* V, void* T0, void* T1, float* S, long lds, int lo_kind, int W, int N,
                 int M, int Mp, int order, bool per_term, int* err, cudaStream_t st) {
  if (!per_term && tc_taylor_series_fits(lo_kind, N, M, Mp))
    return tc_taylor_series(V, T0, S, lds, lo_kind, W, N, M, Mp, order, err, st);
  // one launch per term, the term as the A operand (rows (w, c, i)); the
  // operand alternates between T0 and T1
  void* tin = T0;
  void* tout = T1;
  for (int k = 1; k <= order; ++k) {
    TcGemm tg;
    tg.m = W * 2 * N;
    tg.n = W * M;
    tg.k = 2 * Mp;
    tg.A = tin;
    tg.lda = 2L * Mp;
    tg.B = V;
    tg.ldb = 2L * Mp;
    tg.tf32 = lo_kind == LO_TF32;
    tg.err = err;
    AFQ_TRY(tc_taylor_term(tg, S, lds, k == 1, k < order ? tout : nullptr, lo_kind, W, N, M, Mp,
                           1.0f / (float)k, st));
    void* t_ = tin;
    tin = tout;
    tout = t_;
  }
  return AFQMC_OK;
}

}  // namespace afq

extern "C" int afqmc_taylor_series(int32_t dtype, int64_t nwalkers, int64_t N, int64_t M,
                                   int64_t Mp, int32_t order, const void* dV, void* dT0, void* dT1,
                                   float* dS, int64_t ldS, int32_t per_term, int* d_status,
                                   void* stream) {
  using namespace afq;
  const int lo_kind = dtype == 1 ? LO_TF32 : LO_BF16;
  const bool bad_dims = (dtype != 0 && dtype != 1) || nwalkers < 0 || N < 1 || M < 1 || Mp < M ||
                        Mp % 16 || order < 1 || order > 64 || 2 * N > 128 ||
                        nwalkers * 2 * N * 2 * Mp > (1ll << 31) - 1 ||
                        nwalkers * M * 2 * Mp > (1ll << 31) - 1 || ldS < Mp || ldS % 4;
  if (bad_dims || !dV || !dT0 || !dS || !d_status) {
    set_error("afqmc_taylor_series: bad arguments");
    return AFQMC_EINVAL;
  }
  const bool series = !per_term && tc_taylor_series_fits(lo_kind, (int)N, (int)M, (int)Mp);
  if (!series && !dT1) {
    set_error("afqmc_taylor_series: the per-term path needs dT1");
    return AFQMC_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(dV) | reinterpret_cast<uintptr_t>(dT0) |
       reinterpret_cast<uintptr_t>(dT1) | reinterpret_cast<uintptr_t>(dS)) % 16) {
    set_error("afqmc_taylor_series: buffers must be 16-byte aligned");
    return AFQMC_EINVAL;
  }
  return taylor_apply(dV, dT0, dT1, dS, ldS, lo_kind, (int)nwalkers, (int)N, (int)M, (int)Mp,
                      order, !series, d_status, static_cast<cudaStream_t>(stream));
}
