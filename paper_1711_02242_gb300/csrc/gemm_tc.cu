// Tensor-core contraction for the mixed-precision path (sm_103a, tcgen05).
//
//   D[m][n] = alpha * sum_k A[m][k] * B[n][k]     (A, B K-major; FP32 accumulate)
//
// A and B are BF16 (tcgen05.mma kind::f16) or TF32 (kind::tf32) row-major
// matrices with a row pitch that is a multiple of 16 bytes.  One persistent
// CTA per SM walks 128 x BN output tiles:
//   warp 0  one thread issues TMA loads (128-byte swizzle) into a STAGES-deep
//           shared-memory ring, completion tracked by mbarriers;
//   warp 1  allocates two BN-column TMEM accumulators; one thread issues
//           tcgen05.mma (M=128, N=BN, K=32 bytes per instruction) and frees
//           ring slots with tcgen05.commit;
//   warps 2.. read an accumulator with tcgen05.ld (each warp its 32-lane
//           quarter) and run the epilogue while the other one fills.
// Every mbarrier wait is bounded; on time-out the kernel records an error
// in *err and stops issuing work, and TMEM is always freed before exit.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <map>
#include <mutex>
#include <vector>

#include "kernels.cuh"
#include "tc.cuh"
#include "tc_dev.cuh"

namespace afq {
namespace tc {


template <int BN, int STAGES, int MT = 1>
struct Smem {
  static constexpr int A_BYTES = MT * BM * BKB;  // MT 128-row A tiles per stage
  static constexpr int B_BYTES = BN * BKB;
  static constexpr int STAGE = A_BYTES + B_BYTES;
  static constexpr int RING = STAGES * STAGE;
  static constexpr int TOTAL = RING + 1024 /*align*/ + 256 /*barriers*/;
};

// Named barrier 1 over the W epilogue warps, returning the OR of a flag.
template <int W>
__device__ __forceinline__ bool epi_bar_or(bool flag) {
  uint32_t out;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 q, %1, 0;\n\t"
      "bar.red.or.pred p, 1, %2, q;\n\tselp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(out)
      : "r"((uint32_t)flag), "n"(32 * W)
      : "memory");
  return out != 0;
}

// One contraction of a grouped launch: its operands' tensor maps, sizes,
// output tiles (numbered from tile0 in the launch) and epilogue.
template <class Epi>
struct alignas(64) GemmJob {
  CUtensorMap tmA, tmB;
  int M, N, K, gx, ntiles, tile0;
  int a_wrap;  // A's K coordinate taken modulo a_wrap (0: not)
  int* err;
  Epi epi;
};

// What the kernel needs of the contraction that owns tile t.
template <class Epi>
struct JobView {
  const CUtensorMap* tmA;
  const CUtensorMap* tmB;
  int M, N, K, gx, t0, a_wrap;
  int* err;
  const Epi* epi;
};

// The contractions of a launch: one from the kernel parameters, or a table
// in global memory (jobs in order of tile0; a linear search, the tables are short).
template <class Epi, bool GROUPED>
struct JobTable {
  const GemmJob<Epi>* jobs;
  int njobs;
  const CUtensorMap* a;
  const CUtensorMap* b;
  int M, N, K, gx, a_wrap;
  int* err;
  const Epi* epi;
  __device__ __forceinline__ JobView<Epi> at(int t) const {
    if constexpr (!GROUPED) {
      return {a, b, M, N, K, gx, 0, a_wrap, err, epi};
    } else {
      int j = 0;
      while (j + 1 < njobs && jobs[j + 1].tile0 <= t) ++j;
      const GemmJob<Epi>& J = jobs[j];
      return {&J.tmA, &J.tmB, J.M, J.N, J.K, J.gx, J.tile0, J.a_wrap, J.err, &J.epi};
    }
  }
};

// Persistent contraction body for epilogues that need no shared memory: one
// CTA per SM walks the output tiles t = blockIdx.x, blockIdx.x + gridDim.x,
// ... of all contractions of the launch (tile (bx, by) = (lt % gx, lt / gx)
// of its contraction, lt = t - tile0, so CTAs running together share B tiles
// in L2).  Two TMEM accumulators of BN columns: the epilogue warps drain tile j
// while the MMA thread fills tile j + 1 (tfull / tempty mbarriers per
// accumulator).  With Epi::kMT = 2 a tile is 256 rows: one 256-row A box per
// stage feeds two M=128 MMAs against the same B tile (half the B traffic per
// output), and when two such tiles do not fit in tensor memory a single
// accumulator is used.
// MC (one contraction, CTA pairs): the two CTAs of a cluster take tiles 2u and
// 2u + 1 of a row of tiles that share their B tile (gx even), and each loads
// half of that B tile for both (TMA multicast): half the B bytes per CTA.  A
// ring slot is refilled only when both CTAs' MMAs have released it (every
// MMA commit arrives on both CTAs' empty barrier).
template <int BN, int STAGES, bool TF32, class Epi, bool GROUPED, bool MC = false>
__device__ __forceinline__ void gemm_body(const JobTable<Epi, GROUPED>& tab, int ntiles) {
  extern __shared__ uint8_t smem_raw[];
  constexpr int MT = Epi::kMT;
  using S = Smem<BN, STAGES, MT>;
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + S::RING);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;  // [2]
  uint64_t* tempty = tfull + 2;      // [2]
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(tempty + 2);
  int* abort_flag = reinterpret_cast<int*>(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  constexpr int ELEM = TF32 ? 4 : 2;
  constexpr int BK = BKB / ELEM;
  constexpr int KSTEPS = BKB / 32;

  // tiles of this CTA: t0, t0 + tstep, ...
  const uint32_t rank = MC ? cluster_rank() : 0u;
  const int t0 = MC ? (int)(2 * cluster_id_x() + rank) : (int)blockIdx.x;
  const int tstep = MC ? (int)(2 * cluster_count_x()) : (int)gridDim.x;
  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], MC ? 2 : 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&tfull[a], 1);
      mbar_init(&tempty[a], Epi::kWarps);  // one arrival per epilogue warp
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // TMEM columns: a power of two holding NBUF accumulators of MT x BN columns
  constexpr int NBUF = (2 * MT * BN <= 512) ? 2 : 1;
  constexpr int NEED = NBUF * MT * BN;
  constexpr uint32_t TCOLS = (NEED <= 64) ? 64 : (NEED <= 128) ? 128 : (NEED <= 256) ? 256 : 512;
  constexpr uint32_t ASTRIDE = TCOLS / NBUF;
  static_assert(MT * BN <= (int)ASTRIDE && NEED <= 512, "accumulator stride");
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TCOLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  fence_before();
  __syncthreads();
  fence_after();
  // the peer's multicasts and commits target this CTA's barriers: both CTAs
  // have initialised theirs past this point
  if constexpr (MC) cluster_sync();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0 && lane == 0) {
    int it = 0;
    for (int t = t0; t < ntiles && !*(volatile int*)abort_flag; t += tstep) {
      const JobView<Epi> v = tab.at(t);
      const int lt = t - v.t0, bx = lt % v.gx, by = lt / v.gx;
      const int m0 = v.epi->m_origin(bx, by), n0 = v.epi->n_origin(bx, by);
      const int nk = (v.K + BK - 1) / BK;
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = it % STAGES;
        if (it >= STAGES && !mbar_wait(&empty[s], ((it / STAGES) - 1) & 1, v.err, 11)) {
          *(volatile int*)abort_flag = 1;
          break;
        }
        uint8_t* a = smem + s * S::STAGE;
        mbar_expect_tx(&full[s], S::STAGE);
        // A's K coordinate wraps when B carries a split operand ([hi | lo] K halves)
        tma_load_2d(a, v.tmA, &full[s], v.a_wrap ? (kb * BK) % v.a_wrap : kb * BK, m0);
        if constexpr (MC)
          tma_load_2d_mc(a + S::A_BYTES + rank * (BN / 2) * BKB, v.tmB, &full[s], kb * BK,
                         n0 + (int)rank * (BN / 2), (uint16_t)3);
        else if constexpr (Epi::kB3D)
          tma_load_3d(a + S::A_BYTES, v.tmB, &full[s], kb * BK, 0, v.epi->b_plane(bx, by));
        else
          tma_load_2d(a + S::A_BYTES, v.tmB, &full[s], kb * BK, n0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    constexpr uint32_t idesc = instr_desc(TF32 ? 2u : 1u, (uint32_t)BN);
    int it = 0, j = 0;
    for (int t = t0; t < ntiles && !*(volatile int*)abort_flag; t += tstep, ++j) {
      const JobView<Epi> v = tab.at(t);
      const int nk = (v.K + BK - 1) / BK;
      const int acc = NBUF == 2 ? (j & 1) : 0;
      if (j >= NBUF && !mbar_wait(&tempty[acc], ((j / NBUF) - 1) & 1, v.err, 12)) {
        *(volatile int*)abort_flag = 1;
        break;
      }
      fence_after();
      const uint32_t d = tmem + (uint32_t)acc * ASTRIDE;
      bool ok = true;
      for (int kb = 0; kb < nk; ++kb, ++it) {
        const int s = it % STAGES;
        if (!mbar_wait(&full[s], (it / STAGES) & 1, v.err, 13)) {
          ok = false;
          break;
        }
        fence_after();
        const uint32_t a = smem_u32(smem + s * S::STAGE);
        const uint32_t b = a + S::A_BYTES;
#pragma unroll
        for (int k = 0; k < KSTEPS; ++k)
#pragma unroll
          for (int mt = 0; mt < MT; ++mt)
            mma<TF32>(d + (uint32_t)(mt * BN), sw128_desc(a + mt * BM * BKB + 32 * k),
                      sw128_desc(b + 32 * k), idesc, (kb > 0 || k > 0) ? 1u : 0u);
        if constexpr (MC)
          mma_commit_mc(&empty[s], (uint16_t)3);
        else
          mma_commit(&empty[s]);
      }
      mma_commit(&tfull[acc]);
      if (!ok) {
        *(volatile int*)abort_flag = 1;
        break;
      }
    }
  } else if (warp >= 2) {
    const int q = warp & 3;
    float* esm = Epi::kSmemBytes ? reinterpret_cast<float*>(smem + S::RING + 256) : nullptr;
    int j = 0;
    for (int t = t0; t < ntiles; t += tstep, ++j) {
      const JobView<Epi> v = tab.at(t);
      const int acc = NBUF == 2 ? (j & 1) : 0;
      bool bad = !mbar_wait(&tfull[acc], (j / NBUF) & 1, v.err, 14);
      fence_after();
      // one decision for every epilogue warp (barrier 1 with an OR of the flags)
      if (epi_bar_or<Epi::kWarps>(bad || *(volatile int*)abort_flag)) {
        *(volatile int*)abort_flag = 1;
        break;
      }
      const int lt = t - v.t0, bx = lt % v.gx, by = lt / v.gx;
      const Epi& epi = *v.epi;
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
        epi.template run<BN>(tmem + (uint32_t)acc * ASTRIDE + (uint32_t)(mt * BN), q, lane,
                             warp - 2, bx, by, epi.m_origin(bx, by) + mt * BM,
                             epi.n_origin(bx, by), v.M, v.N, esm);
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[acc]);
    }
  }
  fence_before();
  __syncthreads();
  if (warp == 1) {
    fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(TCOLS));
  }
  // the peer's last commits arrive on this CTA's barriers: neither leaves first
  if constexpr (MC) cluster_sync();
}

// One contraction, its tensor maps and epilogue as kernel parameters.
template <int BN, int STAGES, bool TF32, class Epi>
__global__ void __launch_bounds__(64 + 32 * Epi::kWarps, 1)
    k_tc_gemm_persistent(const __grid_constant__ CUtensorMap tmA,
                         const __grid_constant__ CUtensorMap tmB, int M, int N, int K, int gx,
                         int ntiles, int a_wrap, const __grid_constant__ Epi epi, int* err) {
  const JobTable<Epi, false> tab{nullptr, 1, &tmA, &tmB, M, N, K, gx, a_wrap, err, &epi};
  gemm_body<BN, STAGES, TF32, Epi, false>(tab, ntiles);
}

// One contraction on CTA pairs sharing B tiles by multicast (cluster of 2).
template <int BN, int STAGES, bool TF32, class Epi>
__global__ void __launch_bounds__(64 + 32 * Epi::kWarps, 1)
    k_tc_gemm_pairs(const __grid_constant__ CUtensorMap tmA,
                    const __grid_constant__ CUtensorMap tmB, int M, int N, int K, int gx,
                    int ntiles, int a_wrap, const __grid_constant__ Epi epi, int* err) {
  const JobTable<Epi, false> tab{nullptr, 1, &tmA, &tmB, M, N, K, gx, a_wrap, err, &epi};
  gemm_body<BN, STAGES, TF32, Epi, false, true>(tab, ntiles);
}

// Several contractions (of several independent states) in one persistent
// launch: a work list over (contraction, tile).
template <int BN, int STAGES, bool TF32, class Epi>
__global__ void __launch_bounds__(64 + 32 * Epi::kWarps, 1)
    k_tc_gemm_grouped(const GemmJob<Epi>* __restrict__ jobs, int njobs, int ntiles) {
  const JobTable<Epi, true> tab{jobs, njobs, nullptr, nullptr, 0, 0, 0, 0, 0, nullptr, nullptr};
  gemm_body<BN, STAGES, TF32, Epi, true>(tab, ntiles);
}

// ------------------------------------------------------------ epilogues -----
// Plain FP32 store of alpha * D to C[m * ldc + n].
struct EpiStore {
  static constexpr int kSmemBytes = 0;
  static constexpr bool kB3D = false;  // B tile = one 2-D box at row n_origin
  static constexpr int kWarps = 4;      // epilogue warps
  static constexpr int kMT = 1;         // 128-row A tiles per output tile
  float* C;
  long ldc;
  float alpha;
  int bn;  // tile width (the kernel's BN)
  __device__ __forceinline__ int m_origin(int bx, int) const { return bx * BM; }
  __device__ __forceinline__ int n_origin(int, int by) const { return by * bn; }
  template <int BN>
  __device__ __forceinline__ void run(uint32_t tmem, int q, int lane, int, int, int, int m0, int n0,
                                      int M, int N, float*) const {
    const int row = m0 + 32 * q + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
      if (row >= M) continue;
      const int col = n0 + c0;
      float* c = C + (long)row * ldc + col;
      if (col + 16 <= N && (ldc % 4 == 0)) {
#pragma unroll
        for (int i = 0; i < 16; i += 4)
          *reinterpret_cast<float4*>(c + i) =
              make_float4(alpha * v[i], alpha * v[i + 1], alpha * v[i + 2], alpha * v[i + 3]);
      } else {
#pragma unroll
        for (int i = 0; i < 16; ++i)
          if (col + i < N) c[i] = alpha * v[i];
      }
    }
  }
};

// Exchange part of Eq. localenergy3 fused into the T_g = Lh_g Theta
// contraction.  Rows of the product are (g, i) = Lh rows, columns (w, c, j)
// = Theta^T rows (c = re/im plane).  A tile covers RG whole Cholesky vectors
// (RG*N <= 128 rows) and CW whole walkers; the B tile is one 3-D TMA box of
// CW walkers x NPAD rows (the 2N rows of a walker, zero-padded to a power of
// two), so walker wl of the tile owns accumulator columns [wl NPAD, wl NPAD +
// 2N).  The accumulator is copied to this epilogue's own shared memory; the
// thread of row (g, i) then forms its share of sum_ij T_ij T_ji (complex) from
// its own row and column i of the block, the N shares of a vector are summed,
// and part[w][g][2] receives one partial per (g, w) (nchunk = G), summed later
// in a fixed order.  T never reaches global memory.
struct EpiExchange {
  static constexpr int kSmemBytes = 128 * 257 * 4;  // one 128 x 256 FP32 tile
  static constexpr bool kB3D = true;
  static constexpr int kWarps = 8;  // two per TMEM lane quarter, splitting columns / walkers
  static constexpr int kMT = 1;
  static constexpr int kMaxCW = 16;
  double* part;
  int G, W, N, RG, CW, NPAD, nchunk;
  __device__ __forceinline__ int m_origin(int bx, int) const { return bx * RG * N; }
  __device__ __forceinline__ int n_origin(int, int by) const { return by * CW * NPAD; }
  __device__ __forceinline__ int b_plane(int, int by) const { return by * CW; }
  template <int BN>
  __device__ __forceinline__ void run(uint32_t tmem, int q, int lane, int ew, int bx, int by, int,
                                      int, int, int, float* sm) const {
    constexpr int LD = BN + 1;  // odd pitch: row and column walks are conflict-free
    const int r = 32 * q + lane, half = ew >> 2;
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
    // the two warps of a lane quarter take alternate 16-column chunks, two
    // TMEM loads in flight per wait
#pragma unroll 1
    for (int c0 = 16 * half; c0 < BN; c0 += 64) {
      uint32_t ra[16], rb[16];
      tmem_ld16_async(tq + (uint32_t)c0, ra);
      if (c0 + 32 < BN) tmem_ld16_async(tq + (uint32_t)(c0 + 32), rb);
      tmem_ld_wait();
#pragma unroll
      for (int i = 0; i < 16; ++i) sm[r * LD + c0 + i] = __uint_as_float(ra[i]);
      if (c0 + 32 < BN) {
#pragma unroll
        for (int i = 0; i < 16; ++i) sm[r * LD + c0 + 32 + i] = __uint_as_float(rb[i]);
      }
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    const int gl = r / N, i = r - gl * N;
    const bool rv = gl < RG;
    // sum_ij T_ij T_ji of a vector only enters summed over i, so each unordered
    // pair {i, j} is taken once, by the thread of row i with j = i + d (mod N),
    // d = 1 .. (N - 1) / 2, at twice its weight (for even N the pairs d = N / 2
    // are met from both ends, once each); plus T_ii^2.  FP32 sums (the products
    // come from FP32 accumulators; GB300's float64 pipe is ~60x slower than
    // FP32 and would dominate the kernel); the two warps of a row take
    // alternate walkers.
    const int nd = (N - 1) / 2;
    float e[kMaxCW];
#pragma unroll
    for (int h = 0; h < kMaxCW / 2; ++h) {
      const int wl = 2 * h + half;
      float er = 0.f, ei = 0.f;
      if (wl < CW && rv) {
        const float* own = sm + r * LD + wl * NPAD;             // T_ij: [j], [N + j]
        const float* col = sm + (gl * N) * LD + wl * NPAD + i;  // T_ji: [j LD], [j LD + N]
        const float dr = own[i], di = own[N + i];
        float pr = 0.f, pi = 0.f;
#pragma unroll 4
        for (int d = 1; d <= nd; ++d) {
          const int j = i + d < N ? i + d : i + d - N;
          const float ar = own[j], ai = own[N + j];
          const float br = col[j * LD], bi = col[j * LD + N];
          pr = fmaf(ar, br, fmaf(-ai, bi, pr));
          pi = fmaf(ar, bi, fmaf(ai, br, pi));
        }
        er = fmaf(dr, dr, fmaf(-di, di, 2.f * pr));
        ei = fmaf(2.f * dr, di, 2.f * pi);
        if ((N & 1) == 0) {
          const int j = i + N / 2 < N ? i + N / 2 : i - N / 2;
          const float ar = own[j], ai = own[N + j];
          const float br = col[j * LD], bi = col[j * LD + N];
          er = fmaf(ar, br, fmaf(-ai, bi, er));
          ei = fmaf(ar, bi, fmaf(ai, br, ei));
        }
      }
      e[2 * h] = er;
      e[2 * h + 1] = ei;
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");  // every read of the tile is done
#pragma unroll
    for (int h = 0; h < kMaxCW / 2; ++h) {
      const int wl = 2 * h + half;
      if (wl < CW) {
        sm[r * LD + 2 * wl] = e[2 * h];
        sm[r * LD + 2 * wl + 1] = e[2 * h + 1];
      }
    }
    asm volatile("bar.sync 1, 256;" ::: "memory");
    // one thread per (vector, walker, re/im): the N rows' shares added in
    // four interleaved partial sums, combined in a fixed order
    const int g0 = bx * RG, w0 = by * CW;
    for (int item = r + 128 * half; item < 2 * RG * CW; item += 256) {
      const int c = item & 1, gw = item >> 1, g = gw / CW, wl = gw - g * CW;
      if (g0 + g >= G || w0 + wl >= W) continue;
      const float* src = sm + (g * N) * LD + 2 * wl + c;
      float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
      int i2 = 0;
      for (; i2 + 4 <= N; i2 += 4) {
        s0 += src[i2 * LD];
        s1 += src[(i2 + 1) * LD];
        s2 += src[(i2 + 2) * LD];
        s3 += src[(i2 + 3) * LD];
      }
      for (; i2 < N; ++i2) s0 += src[i2 * LD];
      part[((long)(w0 + wl) * nchunk + g0 + g) * 2 + c] = (double)((s0 + s1) + (s2 + s3));
    }
    // the next tile's copy into sm must wait until every warp is done reading
    asm volatile("bar.sync 1, 256;" ::: "memory");
  }
};

// ---- propagation epilogues (Eq. primitive and Sec. 3.4.2 on tcgen05) --------
// A Taylor term T (M x N complex) is kept as the K-major operand
//   Tb = [[Tr^T, -Ti^T], [Ti^T, Tr^T]]  (2N rows x 2Mp columns),
// so that V T = [Vr | Vi] Tb^T: real output columns are rows i of Tb, imaginary
// ones rows N + i.  These helpers write one element of T into Tb.
__device__ __forceinline__ void put_term(void* tb, int kind, long wrow, int N, int Mp, int c,
                                         int i, int p, float v) {
  const long rr = (wrow + i) * 2L * Mp, ri = (wrow + N + i) * 2L * Mp;
  if (c == 0) {
    store_lo_f(tb, kind, rr + p, v);
    store_lo_f(tb, kind, ri + Mp + p, v);
  } else {
    store_lo_f(tb, kind, rr + Mp + p, -v);
    store_lo_f(tb, kind, ri + p, v);
  }
}

// 16 consecutive values (times sign) into a BF16 or TF32 row at element idx
// (idx a multiple of 8 elements, 16-byte aligned): two or four vector stores.
__device__ __forceinline__ void store16_lo(void* base, int kind, long idx, const float* v,
                                           float sign) {
  if (kind == LO_BF16) {
    uint4 w[2];
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(w);
#pragma unroll
    for (int i = 0; i < 8; ++i) h[i] = __floats2bfloat162_rn(sign * v[2 * i], sign * v[2 * i + 1]);
    uint4* d = reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(base) + idx);
    d[0] = w[0];
    d[1] = w[1];
  } else {
    float4* d = reinterpret_cast<float4*>(reinterpret_cast<float*>(base) + idx);
#pragma unroll
    for (int i = 0; i < 4; ++i)
      d[i] = make_float4(round_tf32(sign * v[4 * i]), round_tf32(sign * v[4 * i + 1]),
                         round_tf32(sign * v[4 * i + 2]), round_tf32(sign * v[4 * i + 3]));
  }
}

__device__ __forceinline__ void store8_lo(void* base, int kind, long idx, const float* v,
                                          float sign) {
  if (kind == LO_BF16) {
    uint4 w;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&w);
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(sign * v[2 * i], sign * v[2 * i + 1]);
    *reinterpret_cast<uint4*>(reinterpret_cast<__nv_bfloat16*>(base) + idx) = w;
  } else {
    float4* d = reinterpret_cast<float4*>(reinterpret_cast<float*>(base) + idx);
#pragma unroll
    for (int i = 0; i < 2; ++i)
      d[i] = make_float4(round_tf32(sign * v[4 * i]), round_tf32(sign * v[4 * i + 1]),
                         round_tf32(sign * v[4 * i + 2]), round_tf32(sign * v[4 * i + 3]));
  }
}

// 4 consecutive values (times sign) into a BF16 or TF32 row at element idx
// (idx a multiple of 4 elements): one 8- or 16-byte store.
__device__ __forceinline__ void store4_lo(void* base, int kind, long idx, const float* v,
                                          float sign) {
  if (kind == LO_BF16) {
    uint2 w;
    __nv_bfloat162* h = reinterpret_cast<__nv_bfloat162*>(&w);
    h[0] = __floats2bfloat162_rn(sign * v[0], sign * v[1]);
    h[1] = __floats2bfloat162_rn(sign * v[2], sign * v[3]);
    *reinterpret_cast<uint2*>(reinterpret_cast<__nv_bfloat16*>(base) + idx) = w;
  } else {
    *reinterpret_cast<float4*>(reinterpret_cast<float*>(base) + idx) =
        make_float4(round_tf32(sign * v[0]), round_tf32(sign * v[1]), round_tf32(sign * v[2]),
                    round_tf32(sign * v[3]));
  }
}

// Row-contiguous epilogue access for the half steps.  A TMEM load gives each
// lane one row and 16 consecutive columns; written as such, a warp's global
// accesses touch 32 rows per instruction.  The chunk is passed through 2 KB of
// shared memory per warp instead (16-byte slots, XOR-swizzled by row so that
// both the row-per-lane writes and the reads below are free of bank
// conflicts), and read back as 8 rows x 4 groups of 4 columns per pass: every
// global instruction then covers whole 32-byte sectors of 8 rows.
struct ChunkStage {
  static constexpr int kBytesPerWarp = 32 * 16 * 4;
  float* sm;  // this warp's 32 x 16 floats
  __device__ __forceinline__ static int slot(int r, int s) { return r * 16 + 4 * (s ^ ((r >> 1) & 3)); }
  __device__ __forceinline__ void put(int lane, const float* v) const {
#pragma unroll
    for (int s = 0; s < 4; ++s)
      *reinterpret_cast<float4*>(sm + slot(lane, s)) = make_float4(v[4 * s], v[4 * s + 1], v[4 * s + 2], v[4 * s + 3]);
  }
  // pass k: row 8k + lane / 4, columns 4 (lane % 4) .. + 3
  __device__ __forceinline__ void get(int lane, int k, float* x) const {
    const float4 f = *reinterpret_cast<const float4*>(sm + slot(8 * k + (lane >> 2), lane & 3));
    x[0] = f.x;
    x[1] = f.y;
    x[2] = f.z;
    x[3] = f.w;
  }
};

// First half step: rows (w,c,i) of Phi^T, columns p.  B_half = I + D_B is
// applied as Phi + Phi D_B: the product runs with the BF16/TF32 copies of Phi
// and D_B = B_half - I, and the epilogue adds the float64 orbitals phi_id
// (pitch M, same rows) so that the identity part is exact (rounding B_half's
// diagonal, close to 1, to BF16/TF32 would scale every walker's orbitals by
// the same factor each step).  acc[(w,c,i)][p] = (B_half Phi)^T (FP32, pitch
// ldacc, a multiple of 4) and Tb holds the 0th Taylor term.  Chunks of 16
// columns go through ChunkStage: each lane then reads and writes 4
// consecutive p of one row.
struct EpiProp0 {
  static constexpr int kWarps = 8;      // epilogue warps: two per TMEM lane quarter
  static constexpr int kSmemBytes = kWarps * ChunkStage::kBytesPerWarp;
  static constexpr bool kB3D = false;  // B tile = one 2-D box at row n_origin
  static constexpr int kMT = 1;         // 128-row A tiles per output tile
  float* acc;
  long ldacc;
  void* tb;
  const double* phi_id;
  int lo_kind, N, M, Mp, rows;
  int bn;  // tile width (the kernel's BN)
  __device__ __forceinline__ int m_origin(int bx, int) const { return bx * BM; }
  __device__ __forceinline__ int n_origin(int, int by) const { return by * bn; }
  template <int BN>
  __device__ __forceinline__ void run(uint32_t tmem, int q, int lane, int ew, int, int, int m0,
                                      int n0, int, int, float* esm) const {
    const ChunkStage cs{esm + ew * 512};
    const int cq = 4 * (lane & 3);
    // the four rows this lane writes (row 8k + lane / 4 of the quarter, k < 4):
    // Tb row offsets and the sign of the -Im block, fixed for the whole tile
    long fr[4], t1[4], t2[4];
    float s2[4];
    bool live[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int row = m0 + 32 * q + 8 * k + (lane >> 2);
      live[k] = row < rows;
      const int w = row / (2 * N), rem = row % (2 * N), c = rem / N, i = rem % N;
      const long rr = ((long)w * 2 * N + i) * 2L * Mp, ri = ((long)w * 2 * N + N + i) * 2L * Mp;
      fr[k] = (long)row;
      t1[k] = c == 0 ? rr : ri;            // Re -> rr[p],      Im -> ri[p]
      t2[k] = c == 0 ? ri + Mp : rr + Mp;  // Re -> ri[Mp + p], Im -> -rr[Mp + p]
      s2[k] = c == 0 ? 1.f : -1.f;
    }
    // this lane's float64 orbitals for the chunk at column c0 (zeros outside)
    auto load = [&](double (&f)[4][4], int c0) {
      const int p = n0 + c0 + cq;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const long fi = fr[k] * M + p;
        if (live[k] && p + 4 <= M && (fi & 1) == 0) {
          const double2 d0 = __ldg(reinterpret_cast<const double2*>(phi_id + fi));
          const double2 d1 = __ldg(reinterpret_cast<const double2*>(phi_id + fi + 2));
          f[k][0] = d0.x;
          f[k][1] = d0.y;
          f[k][2] = d1.x;
          f[k][3] = d1.y;
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) f[k][u] = (live[k] && p + u < M) ? __ldg(phi_id + fi + u) : 0.0;
        }
      }
    };
    // the two warps of a lane quarter take alternate 16-column chunks; the
    // next chunk's loads are in flight while this one is written
    double fn[4][4];
    int c0 = 16 * (ew >> 2);
    if (c0 < BN) load(fn, c0);
#pragma unroll 1
    for (; c0 < BN; c0 += 32) {
      double f[4][4];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int u = 0; u < 4; ++u) f[k][u] = fn[k][u];
      if (c0 + 32 < BN) load(fn, c0 + 32);
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
      if (n0 + c0 >= M) continue;  // the same for the whole warp
      const int p = n0 + c0 + cq;
      const bool full4 = p + 4 <= M;
      cs.put(lane, v);
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float x[4];
        cs.get(lane, k, x);
        if (!live[k] || p >= M) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] += (float)f[k][u];
        float* a = acc + fr[k] * ldacc + p;
        if (full4) {
          *reinterpret_cast<float4*>(a) = make_float4(x[0], x[1], x[2], x[3]);
          store4_lo(tb, lo_kind, t1[k] + p, x, 1.f);
          store4_lo(tb, lo_kind, t2[k] + p, x, s2[k]);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (p + u < M) {
              a[u] = x[u];
              store_lo_f(tb, lo_kind, t1[k] + p + u, x[u]);
              store_lo_f(tb, lo_kind, t2[k] + p + u, s2[k] * x[u]);
            }
        }
      }
      __syncwarp();  // the next chunk overwrites this warp's stage
    }
  }
};

// Taylor term k for walker w: T_k = D / k goes to the series sum S (stored
// for k = 1, added after) and, unless it is the last term, is written as the
// next operand.
// The MMA takes the term as A (rows n = (c, i) of Tb_{k-1}: a 128-row tile at
// walker w = by, rows n >= 2N belong to the next walker and are ignored) and
// [Vr | Vi] as B (columns p: tile bx of BN), so D[n][p] = (V T_{k-1})^T and
// each epilogue thread owns one row n and 16 consecutive p per chunk: the
// running sum and the next operand are written with 16-byte vectors.
struct EpiTaylor {
  static constexpr int kSmemBytes = 0;
  static constexpr bool kB3D = false;  // B tile = one 2-D box at row n_origin
  static constexpr int kWarps = 4;      // epilogue warps
  static constexpr int kMT = 1;         // 128-row A tiles per output tile
  static constexpr int kBN = 160;  // two tiles cover p < 320
  float* S;
  long lds;
  int first;
  void* tb_out;
  int lo_kind, N, M, Mp;
  float scale;
  __device__ __forceinline__ int m_origin(int, int by) const { return by * 2 * N; }
  __device__ __forceinline__ int n_origin(int bx, int by) const { return by * M + bx * kBN; }
  template <int BN>
  __device__ __forceinline__ void run(uint32_t tmem, int q, int lane, int, int bx, int by, int, int,
                                      int, int, float*) const {
    const int w = by, n = 32 * q + lane;
    const bool valid = n < 2 * N;
    const int c = valid ? n / N : 0, i = valid ? n % N : 0;
    float* arow = S + ((long)w * 2 * N + n) * lds;
    const long rr = ((long)w * 2 * N + i) * 2L * Mp, ri = ((long)w * 2 * N + N + i) * 2L * Mp;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
      const int pb = bx * BN + c0;
      if (!valid || pb >= M) continue;
#pragma unroll
      for (int u = 0; u < 16; ++u) v[u] *= scale;
      if (pb + 16 <= M) {
        float4* a4 = reinterpret_cast<float4*>(arow + pb);
        float4 o[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) o[k] = first ? make_float4(0.f, 0.f, 0.f, 0.f) : a4[k];
#pragma unroll
        for (int k = 0; k < 4; ++k)
          a4[k] = make_float4(o[k].x + v[4 * k], o[k].y + v[4 * k + 1], o[k].z + v[4 * k + 2],
                              o[k].w + v[4 * k + 3]);
        if (tb_out) {
          if (c == 0) {
            store16_lo(tb_out, lo_kind, rr + pb, v, 1.f);
            store16_lo(tb_out, lo_kind, ri + Mp + pb, v, 1.f);
          } else {
            store16_lo(tb_out, lo_kind, rr + Mp + pb, v, -1.f);
            store16_lo(tb_out, lo_kind, ri + pb, v, 1.f);
          }
        }
      } else {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          if (pb + u >= M) continue;
          arow[pb + u] = (first ? 0.f : arow[pb + u]) + v[u];
          if (tb_out) put_term(tb_out, lo_kind, (long)w * 2 * N, N, Mp, c, i, pb + u, v[u]);
        }
      }
    }
  }
};

// V = i sqrt(dt) sum_g x_g L_g straight into the Taylor operand: rows (w, c)
// of the field matrix (c = 0: Re x, c = 1: Im x), columns (p, q) = p * Mp + q
// of the full Cholesky vectors; Re V = -sqrt(dt) (Im x . L) and Im V =
// sqrt(dt) (Re x . L) land in row (w, p) of [Re V | Im V] at column q or
// Mp + q, 16 consecutive q per thread (pad columns come out zero).
// MT_ = 2: 256-row tiles (each Cholesky tile serves 128 walkers, one
// 512-column accumulator at BN = 256); MT_ = 1: 128-row tiles (two 256-column
// accumulators at BN = 256: the epilogue overlaps the next tile's MMAs).
template <int MT_>
struct EpiVT {
  static constexpr int kSmemBytes = 0;
  static constexpr bool kB3D = false;  // B tile = one 2-D box at row n_origin
  static constexpr int kWarps = 8;      // epilogue warps: two per TMEM lane quarter
  static constexpr int kMT = MT_;
  void* V;
  int lo_kind, W, M, Mp;
  float sdt;
  int bn;  // tile width: 256 (one 16 x 16 block) or 128 (half a block)
  __device__ __forceinline__ int m_origin(int bx, int) const { return bx * BM * kMT; }
  __device__ __forceinline__ int n_origin(int, int by) const { return by * bn; }
  // Output block (P, Q), P <= Q, of the symmetric V (blocks of 256 operand
  // rows in the order of P, then Q): column pp * 16 + qq of the block is
  // V[16 P + pp][16 Q + qq].  BN = 256: the tile is the block and the thread
  // of row (w, c) writes its 16 rows (16 contiguous q each) and, off the
  // diagonal, the mirrored block's 16 rows (V[q][p] = V[p][q]) in two halves
  // of 8 contiguous p, the two warps of a lane quarter one half each.  BN =
  // 128: the tile is half h of the block (pp in [8 h, 8 h + 8)), so two
  // accumulators fit tensor memory and the epilogue overlaps the next tile's
  // MMAs; one warp of the quarter writes the 8 rows, the other the mirror's
  // 16 rows of 8 contiguous p.
  template <int BN>
  __device__ __forceinline__ void run(uint32_t tmem, int q, int lane, int ew, int, int, int m0,
                                      int n0, int, int, float*) const {
    static_assert(BN == 256 || BN == 128, "a 16 x 16 block or half of one per tile");
    const int row = m0 + 32 * q + lane;
    const bool valid = row < 2 * W;
    const int w = row >> 1, c = row & 1;
    const float sign = c ? -sdt : sdt;
    const int nb = Mp / 16;
    int P = 0, rem = n0 / 256;
    while (rem >= nb - P) {
      rem -= nb - P;
      ++P;
    }
    const int Q = P + rem;
    const long vb = (long)w * M * 2L * Mp + (c ? 0 : Mp);
    const uint32_t tq = tmem + ((uint32_t)(32 * q) << 16);
    // half h of the block and whether this warp writes the block's rows or the mirror's
    const int h = BN == 256 ? (ew >> 2) : ((n0 / 128) & 1);
    const bool rows = BN == 256 || (ew >> 2) == 0;
    const bool mirror = BN == 256 || (ew >> 2) == 1;
    uint32_t r[8][16];
#pragma unroll
    for (int u = 0; u < 8; ++u)
      tmem_ld16_async(tq + (uint32_t)(((BN == 256 ? 8 * h : 0) + u) * 16), r[u]);
    tmem_ld_wait();
    if (!valid) return;
    if (rows) {
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int p = 16 * P + 8 * h + u;
        if (p < M) {
          float v[16];
#pragma unroll
          for (int t = 0; t < 16; ++t) v[t] = __uint_as_float(r[u][t]);
          store16_lo(V, lo_kind, vb + (long)p * 2 * Mp + 16 * Q, v, sign);
        }
      }
    }
    if (P == Q || !mirror) return;
#pragma unroll
    for (int t = 0; t < 16; ++t) {
      const int qr = 16 * Q + t;
      if (qr < M) {
        float v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) v[u] = __uint_as_float(r[u][t]);
        store8_lo(V, lo_kind, vb + (long)qr * 2 * Mp + 16 * P + 8 * h, v, sign);
      }
    }
  }
};
using EpiV = EpiVT<2>;
using EpiV1 = EpiVT<1>;

// Last half step: rows (w,c,i) of the series sum, columns p; the product is
// stored as the new float64 orbitals of live walkers.  Chunks of 16 columns go
// through ChunkStage, as in EpiProp0.
struct EpiPhi {
  static constexpr int kWarps = 8;      // epilogue warps: two per TMEM lane quarter
  static constexpr int kSmemBytes = kWarps * ChunkStage::kBytesPerWarp;
  static constexpr bool kB3D = false;  // B tile = one 2-D box at row n_origin
  static constexpr int kMT = 1;         // 128-row A tiles per output tile
  double* phiT;
  const double* wt;
  int N, M, rows;
  int bn;  // tile width (the kernel's BN)
  void* phi_lo;  // BF16/TF32 copy of the orbitals (pitch Mp) for the next first half step
  int lo_kind, Mp;
  // FP32 rows [T_0 | S] (pitch 2 Mp): the product is [T_0 | S] [D_B | D_B]
  // with D_B = B_half - I, and the identity part T_0 + S is added here exactly
  const float* acc_id;
  __device__ __forceinline__ int m_origin(int bx, int) const { return bx * BM; }
  __device__ __forceinline__ int n_origin(int, int by) const { return by * bn; }
  template <int BN>
  __device__ __forceinline__ void run(uint32_t tmem, int q, int lane, int ew, int, int, int m0,
                                      int n0, int, int, float* esm) const {
    const ChunkStage cs{esm + ew * 512};
    const int cq = 4 * (lane & 3);
    // the four rows this lane writes (row 8k + lane / 4 of the quarter, k < 4)
    long fr[4];
    bool live[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const int row = m0 + 32 * q + 8 * k + (lane >> 2);
      fr[k] = (long)row;
      live[k] = row < rows && walker_alive(wt, row / (2 * N));
    }
    // this lane's T_0 and S for the chunk at column c0 (zeros outside); they
    // are summed where used, so that nothing waits on the loads early
    auto load = [&](float (&id)[4][8], int c0) {
      const int p = n0 + c0 + cq;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const float* t0 = acc_id + fr[k] * 2 * Mp + p;
        if (live[k] && p + 4 <= M) {
          const float4 a = __ldg(reinterpret_cast<const float4*>(t0));
          const float4 b = __ldg(reinterpret_cast<const float4*>(t0 + Mp));
          id[k][0] = a.x;
          id[k][1] = a.y;
          id[k][2] = a.z;
          id[k][3] = a.w;
          id[k][4] = b.x;
          id[k][5] = b.y;
          id[k][6] = b.z;
          id[k][7] = b.w;
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const bool in = live[k] && p + u < M;
            id[k][u] = in ? __ldg(t0 + u) : 0.f;
            id[k][4 + u] = in ? __ldg(t0 + Mp + u) : 0.f;
          }
        }
      }
    };
    // the two warps of a lane quarter take alternate 16-column chunks; the
    // next chunk's loads are in flight while this one is written
    float idn[4][8];
    int c0 = 16 * (ew >> 2);
    if (c0 < BN) load(idn, c0);
#pragma unroll 1
    for (; c0 < BN; c0 += 32) {
      float id[4][8];
#pragma unroll
      for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int u = 0; u < 8; ++u) id[k][u] = idn[k][u];
      if (c0 + 32 < BN) load(idn, c0 + 32);
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
      if (n0 + c0 >= M) continue;  // the same for the whole warp
      const int p = n0 + c0 + cq;
      const bool full4 = p + 4 <= M;
      cs.put(lane, v);
      __syncwarp();
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        float x[4];
        cs.get(lane, k, x);
        if (!live[k] || p >= M) continue;
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] += id[k][u] + id[k][4 + u];
        double* o = phiT + fr[k] * M + p;
        if (full4) {
          if (((fr[k] * M + p) & 1) == 0) {
            reinterpret_cast<double2*>(o)[0] = make_double2((double)x[0], (double)x[1]);
            reinterpret_cast<double2*>(o)[1] = make_double2((double)x[2], (double)x[3]);
          } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) o[u] = (double)x[u];
          }
          store4_lo(phi_lo, lo_kind, fr[k] * Mp + p, x, 1.f);
        } else {
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (p + u < M) {
              o[u] = (double)x[u];
              store_lo_f(phi_lo, lo_kind, fr[k] * Mp + p + u, x[u]);
            }
        }
      }
      __syncwarp();  // the next chunk overwrites this warp's stage
    }
  }
};

}  // namespace tc

// ------------------------------------------------------------------- host ----
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  }
  return fn;
}

// 2-D row-major [rows][pitch] operand, box = rows_box x 128 bytes, 128B swizzle.
int make_tmap(CUtensorMap* m, const void* base, int elem_bytes, long rows, long cols, long pitch,
              int box_rows) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available");
    return AFQMC_ECUDA;
  }
  if ((reinterpret_cast<uintptr_t>(base) % 16) || (pitch * elem_bytes) % 16) {
    set_error("tensor map: base or pitch not 16-byte aligned");
    return AFQMC_EINVAL;
  }
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(pitch * elem_bytes)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  2, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled failed (%d)", (int)r);
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

// 3-D operand [planes][rows][pitch] (plane stride in elements), box = 128 bytes
// x box_rows x box_planes, 128B swizzle; rows >= `rows` of a plane and planes
// >= `planes` read as zero, so a box lands as box_planes blocks of box_rows
// (zero-padded) rows.
int make_tmap_3d(CUtensorMap* m, const void* base, int elem_bytes, long planes, long rows,
                 long cols, long pitch, long plane_stride, int box_rows, int box_planes) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available");
    return AFQMC_ECUDA;
  }
  if ((reinterpret_cast<uintptr_t>(base) % 16) || (pitch * elem_bytes) % 16 ||
      (plane_stride * elem_bytes) % 16) {
    set_error("tensor map: base or strides not 16-byte aligned");
    return AFQMC_EINVAL;
  }
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)planes};
  cuuint64_t strides[2] = {(cuuint64_t)(pitch * elem_bytes), (cuuint64_t)(plane_stride * elem_bytes)};
  cuuint32_t box[3] = {(cuuint32_t)(128 / elem_bytes), (cuuint32_t)box_rows,
                       (cuuint32_t)box_planes};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = fn(m, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  3, const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (3-D) failed (%d)", (int)r);
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}


// Tensor map of any rank (2..5): dims innermost first, strides in bytes for
// dims 1.., box sizes per dim; 128-byte swizzle, out-of-range elements read 0.
int make_tmap_nd(CUtensorMap* m, const void* base, int elem_bytes, int rank, const long* dims,
                 const long* stride_bytes, const int* box) {
  auto fn = encode_fn();
  if (!fn) {
    set_error("cuTensorMapEncodeTiled is not available");
    return AFQMC_ECUDA;
  }
  if (rank < 2 || rank > 5 || (reinterpret_cast<uintptr_t>(base) % 16)) {
    set_error("tensor map: bad rank or base");
    return AFQMC_EINVAL;
  }
  cuuint64_t d[5], sb[4];
  cuuint32_t bx[5], es[5];
  for (int i = 0; i < rank; ++i) {
    d[i] = (cuuint64_t)dims[i];
    bx[i] = (cuuint32_t)box[i];
    es[i] = 1;
    if (i > 0) {
      if (stride_bytes[i - 1] % 16) {
        set_error("tensor map: stride not a multiple of 16 bytes");
        return AFQMC_EINVAL;
      }
      sb[i - 1] = (cuuint64_t)stride_bytes[i - 1];
    }
  }
  CUresult r = fn(m, elem_bytes == 2 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                  (cuuint32_t)rank, const_cast<void*>(base), d, sb, bx, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    set_error("cuTensorMapEncodeTiled (rank %d) failed (%d)", rank, (int)r);
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

int tc_sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1)
      n = 148;
  }
  return n;
}

template <int BN, int STAGES, bool TF32, class Epi>
static int launch_tc_persistent(const TcGemm& g, const Epi& epi, int gx, int gy, cudaStream_t st,
                                const CUtensorMap* tb_given = nullptr) {
  constexpr int kTotal = tc::Smem<BN, STAGES, Epi::kMT>::TOTAL + Epi::kSmemBytes;
  static_assert(kTotal <= 232448, "shared memory");
  const int eb = TF32 ? 4 : 2;
  CUtensorMap ta, tb;
  AFQ_TRY(make_tmap(&ta, g.A, eb, g.m, g.ka > 0 ? g.ka : g.k, g.lda, tc::BM * Epi::kMT));
  if (tb_given)
    tb = *tb_given;
  else
    AFQ_TRY(make_tmap(&tb, g.B, eb, g.n, g.k, g.ldb, BN));
  auto kern = tc::k_tc_gemm_persistent<BN, STAGES, TF32, Epi>;
  static std::atomic<unsigned long long> attr{0};
  AFQ_TRY(smem_attr_once(kern, kTotal, attr));
  const long ntiles = (long)gx * gy;
  if (ntiles <= 0) return AFQMC_OK;
  if (ntiles > 0x7fffffffL) {
    set_error("tc gemm: too many tiles");
    return AFQMC_EINVAL;
  }
  const int grid = (int)(ntiles < tc_sm_count() ? ntiles : tc_sm_count());
  AFQ_LAUNCH(kern, grid, 64 + 32 * Epi::kWarps, kTotal, st, ta, tb, g.m, g.n, g.k, gx, (int)ntiles,
             g.a_wrap,
             epi, g.err);
  return AFQMC_OK;
}

// One contraction on CTA pairs (clusters of two, B tiles shared by TMA
// multicast): gx and the tile count must be even; the grid is even.
template <int BN, int STAGES, bool TF32, class Epi>
static int launch_tc_pairs(const TcGemm& g, const Epi& epi, int gx, int gy, cudaStream_t st) {
  constexpr int kTotal = tc::Smem<BN, STAGES, Epi::kMT>::TOTAL + Epi::kSmemBytes;
  static_assert(kTotal <= 232448, "shared memory");
  static_assert(!Epi::kB3D && BN % 16 == 0, "2-D B tiles, halves of whole swizzle atoms");
  const long ntiles = (long)gx * gy;
  if (ntiles <= 0) return AFQMC_OK;
  if ((gx & 1) || ntiles > 0x7fffffffL) {
    set_error("tc gemm (pairs): gx=%d must be even", gx);
    return AFQMC_EINVAL;
  }
  const int eb = TF32 ? 4 : 2;
  CUtensorMap ta, tb;
  AFQ_TRY(make_tmap(&ta, g.A, eb, g.m, g.ka > 0 ? g.ka : g.k, g.lda, tc::BM * Epi::kMT));
  AFQ_TRY(make_tmap(&tb, g.B, eb, g.n, g.k, g.ldb, BN / 2));
  auto kern = tc::k_tc_gemm_pairs<BN, STAGES, TF32, Epi>;
  static std::atomic<unsigned long long> attr{0};
  AFQ_TRY(smem_attr_once(kern, kTotal, attr));
  const int sms = tc_sm_count() & ~1;
  const int grid = (int)(ntiles < sms ? ntiles : sms);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(64 + 32 * Epi::kWarps);
  cfg.dynamicSmemBytes = kTotal;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = 2;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, ta, tb, g.m, g.n, g.k, gx, (int)ntiles,
                                           g.a_wrap, epi, g.err);
  ++g_launches;
  if (e != cudaSuccess) {
    set_error("launch k_tc_gemm_pairs: %s", cudaGetErrorString(e));
    return AFQMC_ECUDA;
  }
  return AFQMC_OK;
}

// ---- plain-store contraction with an autotuned tile width --------------------
// Candidates: BN = 256 (4 stages, one CTA per SM), 128 (3 stages) and 64
// (4 stages), the last two small enough for two CTAs per SM.  tc_tune_store()
// times each once on the caller's buffers and remembers the fastest for the
// shape; tc_gemm_store() uses the remembered choice (256 when untuned).
namespace {
struct ShapeKey {
  int m, n, k;
  bool tf32;
  bool operator<(const ShapeKey& o) const {
    if (m != o.m) return m < o.m;
    if (n != o.n) return n < o.n;
    if (k != o.k) return k < o.k;
    return tf32 < o.tf32;
  }
};
std::mutex g_tune_mu;
std::map<ShapeKey, int> g_tuned_bn, g_tuned_bn_v;
}  // namespace

static int launch_store_bn(const TcGemm& g, float* C, long ldc, float alpha, int bn,
                           cudaStream_t st) {
  tc::EpiStore e{C, ldc, alpha, bn};
  const int gx = cdiv(g.m, tc::BM), gy = cdiv(g.n, bn);
  if (bn == 64) {
    if (g.tf32) return launch_tc_persistent<64, 8, true>(g, e, gx, gy, st);
    return launch_tc_persistent<64, 8, false>(g, e, gx, gy, st);
  }
  if (bn == 128) {
    if (g.tf32) return launch_tc_persistent<128, 6, true>(g, e, gx, gy, st);
    return launch_tc_persistent<128, 6, false>(g, e, gx, gy, st);
  }
  if (g.tf32) return launch_tc_persistent<256, 4, true>(g, e, gx, gy, st);
  return launch_tc_persistent<256, 4, false>(g, e, gx, gy, st);
}

int tc_gemm_store(const TcGemm& g, float* C, long ldc, float alpha, cudaStream_t st) {
  if (g.m <= 0 || g.n <= 0) return AFQMC_OK;
  if (g.k <= 0) {
    set_error("tc gemm: k must be positive");
    return AFQMC_EINVAL;
  }
  int bn = 256;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_bn.find(ShapeKey{g.m, g.n, g.k, g.tf32});
    if (it != g_tuned_bn.end()) bn = it->second;
  }
  return launch_store_bn(g, C, ldc, alpha, bn, st);
}

int tc_tune_store(const TcGemm& g, float* C, long ldc, float alpha, cudaStream_t st, int* chosen) {
  if (g.m <= 0 || g.n <= 0 || g.k <= 0) return AFQMC_OK;
  cudaEvent_t e0, e1;
  AFQ_CUDA(cudaEventCreate(&e0));
  AFQ_CUDA(cudaEventCreate(&e1));
  int best = 256;
  float best_ms = 1e30f;
  for (int bn : {256, 128, 64}) {
    AFQ_TRY(launch_store_bn(g, C, ldc, alpha, bn, st));  // warm-up (and first-use set-up)
    // the fastest of three timings of two launches: one slow timing (another
    // kernel of the device, a clock step) must not decide the tile
    for (int rep = 0; rep < 3; ++rep) {
      AFQ_CUDA(cudaEventRecord(e0, st));
      AFQ_TRY(launch_store_bn(g, C, ldc, alpha, bn, st));
      AFQ_TRY(launch_store_bn(g, C, ldc, alpha, bn, st));
      AFQ_CUDA(cudaEventRecord(e1, st));
      AFQ_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      AFQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = bn;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned_bn[ShapeKey{g.m, g.n, g.k, g.tf32}] = best;
  }
  if (chosen) *chosen = best;
  return AFQMC_OK;
}

// Tile width for an output of n columns: 160 or 256, whichever pads less.
// At 160 the ring keeps five 36 KB stages beside the epilogue's 16 KB stage.
constexpr int kHalfStages160 = 5;
static int half_step_bn(int n) {
  const int pad160 = cdiv(n, 160) * 160 - n, pad256 = cdiv(n, 256) * 256 - n;
  return pad160 < pad256 ? 160 : 256;
}

int tc_prop_first(const TcGemm& g, float* acc, long ldacc, void* tb, const double* phi_id,
                  int lo_kind, int N, int M, int Mp, cudaStream_t st) {
  const int bn = half_step_bn(M);
  tc::EpiProp0 e{acc, ldacc, tb, phi_id, lo_kind, N, M, Mp, g.m, bn};
  const int gx = cdiv(g.m, tc::BM), gy = cdiv(M, bn);
  if (bn == 160) {
    if (g.tf32) return launch_tc_persistent<160, kHalfStages160, true>(g, e, gx, gy, st);
    return launch_tc_persistent<160, kHalfStages160, false>(g, e, gx, gy, st);
  }
  if (g.tf32) return launch_tc_persistent<256, 4, true>(g, e, gx, gy, st);
  return launch_tc_persistent<256, 4, false>(g, e, gx, gy, st);
}

int tc_taylor_term(const TcGemm& g, float* S, long lds, bool first, void* tb_out, int lo_kind,
                   int W, int N, int M, int Mp, float scale, cudaStream_t st) {
  if (2 * N > tc::BM) {
    set_error("tc taylor: 2N=%d above the 128-row tile", 2 * N);
    return AFQMC_EUNSUPPORTED;
  }
  if (lds % 4) {
    set_error("tc taylor: sum pitch %ld not a multiple of 4", lds);
    return AFQMC_EINVAL;
  }
  tc::EpiTaylor e{S, lds, first ? 1 : 0, tb_out, lo_kind, N, M, Mp, scale};
  constexpr int BN = tc::EpiTaylor::kBN;
  if (g.tf32) return launch_tc_persistent<BN, 6, true>(g, e, cdiv(M, BN), W, st);
  return launch_tc_persistent<BN, 6, false>(g, e, cdiv(M, BN), W, st);
}

// V in one of three forms, chosen at set-up by timing: tile width 128 (half
// blocks, double-buffered accumulators, 256-row tiles), 256 on 256-row tiles
// (one accumulator; CTA pairs when the tile rows pair up), or kV256Pairs128:
// 256 on 128-row tiles on CTA pairs (double-buffered accumulators, the
// Cholesky tile shared by the pair).
constexpr int kV256Pairs128 = 257;
static int launch_v_bn(const TcGemm& g, void* V, int lo_kind, int W, int M, int Mp, double sdt,
                       int bn, cudaStream_t st) {
  const int nb = Mp / 16;
  if (bn == kV256Pairs128) {
    tc::EpiV1 e1{V, lo_kind, W, M, Mp, (float)sdt, 256};
    const int gx1 = cdiv(g.m, tc::BM), gy1 = nb * (nb + 1) / 2;
    if (gx1 % 2) {
      set_error("tc V: 128-row tiles on CTA pairs need an even number of them (%d)", gx1);
      return AFQMC_EINVAL;
    }
    if (g.tf32) return launch_tc_pairs<256, 4, true>(g, e1, gx1, gy1, st);
    return launch_tc_pairs<256, 4, false>(g, e1, gx1, gy1, st);
  }
  tc::EpiV e{V, lo_kind, W, M, Mp, (float)sdt, bn};
  const int gx = cdiv(g.m, tc::BM * tc::EpiV::kMT), gy = nb * (nb + 1) / 2 * (256 / bn);
  if (bn == 128) {
    if (g.tf32) return launch_tc_persistent<128, 4, true>(g, e, gx, gy, st);
    return launch_tc_persistent<128, 4, false>(g, e, gx, gy, st);
  }
  // BN = 256: CTA pairs share the Cholesky tile (every output row of tiles
  // is gx = 2W / 256 tiles wide: pairs need gx even)
  if (gx % 2 == 0) {
    if (g.tf32) return launch_tc_pairs<256, 3, true>(g, e, gx, gy, st);
    return launch_tc_pairs<256, 3, false>(g, e, gx, gy, st);
  }
  if (g.tf32) return launch_tc_persistent<256, 3, true>(g, e, gx, gy, st);
  return launch_tc_persistent<256, 3, false>(g, e, gx, gy, st);
}

int tc_v_full(const TcGemm& g, void* V, int lo_kind, int W, int M, int Mp, double sdt,
              cudaStream_t st) {
  if (Mp % 16) {
    set_error("tc V: Mp=%d must be a multiple of 16", Mp);
    return AFQMC_EINVAL;
  }
  const int nb = Mp / 16;
  if (g.n != nb * (nb + 1) / 2 * 256) {
    set_error("tc V: %d operand rows, the %d upper 16 x 16 blocks of Mp=%d need %d", g.n,
              nb * (nb + 1) / 2, Mp, nb * (nb + 1) / 2 * 256);
    return AFQMC_EINVAL;
  }
  int bn = 128;
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tuned_bn_v.find(ShapeKey{g.m, g.n, g.k, g.tf32});
    if (it != g_tuned_bn_v.end()) bn = it->second;
  }
  return launch_v_bn(g, V, lo_kind, W, M, Mp, sdt, bn, st);
}

int tc_tune_v(const TcGemm& g, void* V, int lo_kind, int W, int M, int Mp, double sdt,
              cudaStream_t st, int* chosen) {
  if (g.m <= 0 || g.n <= 0 || g.k <= 0) return AFQMC_OK;
  cudaEvent_t e0, e1;
  AFQ_CUDA(cudaEventCreate(&e0));
  AFQ_CUDA(cudaEventCreate(&e1));
  int best = 128;
  float best_ms = 1e30f;
  std::vector<int> forms = {128, 256};
  if (cdiv(g.m, tc::BM) % 2 == 0) forms.push_back(kV256Pairs128);
  for (int bn : forms) {
    AFQ_TRY(launch_v_bn(g, V, lo_kind, W, M, Mp, sdt, bn, st));  // warm-up
    for (int rep = 0; rep < 3; ++rep) {  // the fastest of three timings
      AFQ_CUDA(cudaEventRecord(e0, st));
      AFQ_TRY(launch_v_bn(g, V, lo_kind, W, M, Mp, sdt, bn, st));
      AFQ_TRY(launch_v_bn(g, V, lo_kind, W, M, Mp, sdt, bn, st));
      AFQ_CUDA(cudaEventRecord(e1, st));
      AFQ_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      AFQ_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (ms < best_ms) {
        best_ms = ms;
        best = bn;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tuned_bn_v[ShapeKey{g.m, g.n, g.k, g.tf32}] = best;
  }
  if (chosen) *chosen = best == kV256Pairs128 ? 256 : best;
  return AFQMC_OK;
}

int tc_prop_last(const TcGemm& g, double* phiT, const double* wt, int N, int M, void* phi_lo,
                 int lo_kind, int Mp, const float* acc_id, cudaStream_t st) {
  if (g.lda != 2L * Mp) {
    set_error("tc last half step: operand pitch %ld, want 2 Mp = %d", g.lda, 2 * Mp);
    return AFQMC_EINVAL;
  }
  const int bn = half_step_bn(M);
  tc::EpiPhi e{phiT, wt, N, M, g.m, bn, phi_lo, lo_kind, Mp, acc_id};
  const int gx = cdiv(g.m, tc::BM), gy = cdiv(M, bn);
  if (bn == 160) {
    if (g.tf32) return launch_tc_persistent<160, kHalfStages160, true>(g, e, gx, gy, st);
    return launch_tc_persistent<160, kHalfStages160, false>(g, e, gx, gy, st);
  }
  if (g.tf32) return launch_tc_persistent<256, 4, true>(g, e, gx, gy, st);
  return launch_tc_persistent<256, 4, false>(g, e, gx, gy, st);
}

// ---- per-step contractions as job descriptors, alone or grouped ------------
int tc_job_launch(const TcJobDesc& d, cudaStream_t st) {
  switch (d.kind) {
    case TC_JOB_STORE:
      return tc_gemm_store(d.g, d.C, d.ldc, d.alpha, st);
    case TC_JOB_V:
      return tc_v_full(d.g, d.V, d.lo_kind, d.W, d.M, d.Mp, d.sdt, st);
    case TC_JOB_PROP0:
      return tc_prop_first(d.g, d.acc, d.ldacc, d.tb, d.phi_id, d.lo_kind, d.N, d.M, d.Mp, st);
    case TC_JOB_PHI:
      return tc_prop_last(d.g, d.phiT, d.wt, d.N, d.M, d.phi_lo, d.lo_kind, d.Mp, d.acc_id, st);
  }
  set_error("tc job: unknown kind %d", d.kind);
  return AFQMC_EINVAL;
}

struct TcGrouped {
  int kind = 0, bn = 0, stages = 0, njobs = 0, ntiles = 0;
  bool tf32 = false;
  void* d_jobs = nullptr;
};

namespace {
// The job of one descriptor with tile width bn: operand maps, grid, epilogue.
template <class Epi>
int fill_job(tc::GemmJob<Epi>* j, const TcGemm& g, int bn, int gx, int gy, const Epi& e) {
  const int eb = g.tf32 ? 4 : 2;
  AFQ_TRY(make_tmap(&j->tmA, g.A, eb, g.m, g.ka > 0 ? g.ka : g.k, g.lda, tc::BM * Epi::kMT));
  AFQ_TRY(make_tmap(&j->tmB, g.B, eb, g.n, g.k, g.ldb, bn));
  j->M = g.m;
  j->N = g.n;
  j->K = g.k;
  j->gx = gx;
  j->ntiles = gx * gy;
  j->tile0 = 0;
  j->a_wrap = g.a_wrap;
  j->err = g.err;
  j->epi = e;
  return AFQMC_OK;
}

int make_job(const TcJobDesc& d, int bn, tc::GemmJob<tc::EpiStore>* j) {
  tc::EpiStore e{d.C, d.ldc, d.alpha, bn};
  return fill_job(j, d.g, bn, cdiv(d.g.m, tc::BM), cdiv(d.g.n, bn), e);
}
int make_job(const TcJobDesc& d, int bn, tc::GemmJob<tc::EpiV>* j) {
  const int nb = d.Mp / 16;
  if (d.Mp % 16 || d.g.n != nb * (nb + 1) / 2 * 256) {
    set_error("grouped V: Mp=%d and %d operand rows do not match", d.Mp, d.g.n);
    return AFQMC_EINVAL;
  }
  tc::EpiV e{d.V, d.lo_kind, d.W, d.M, d.Mp, (float)d.sdt, bn};
  return fill_job(j, d.g, bn, cdiv(d.g.m, tc::BM * tc::EpiV::kMT), nb * (nb + 1) / 2 * (256 / bn),
                  e);
}
int make_job(const TcJobDesc& d, int bn, tc::GemmJob<tc::EpiProp0>* j) {
  tc::EpiProp0 e{d.acc, d.ldacc, d.tb, d.phi_id, d.lo_kind, d.N, d.M, d.Mp, d.g.m, bn};
  return fill_job(j, d.g, bn, cdiv(d.g.m, tc::BM), cdiv(d.M, bn), e);
}
int make_job(const TcJobDesc& d, int bn, tc::GemmJob<tc::EpiPhi>* j) {
  if (d.g.lda != 2L * d.Mp) {
    set_error("grouped last half step: operand pitch %ld, want 2 Mp = %d", d.g.lda, 2 * d.Mp);
    return AFQMC_EINVAL;
  }
  tc::EpiPhi e{d.phiT, d.wt, d.N, d.M, d.g.m, bn, d.phi_lo, d.lo_kind, d.Mp, d.acc_id};
  return fill_job(j, d.g, bn, cdiv(d.g.m, tc::BM), cdiv(d.M, bn), e);
}

// Host table of the n jobs (tile0 = running tile count), copied to the device.
template <class Epi>
int build_table(const TcJobDesc* d, int n, int bn, TcGrouped* gr) {
  std::vector<tc::GemmJob<Epi>> jobs((size_t)n);
  long tiles = 0;
  for (int i = 0; i < n; ++i) {
    AFQ_TRY(make_job(d[i], bn, &jobs[i]));
    jobs[i].tile0 = (int)tiles;
    tiles += jobs[i].ntiles;
  }
  if (tiles > 0x7fffffffL) {
    set_error("grouped contraction: too many tiles");
    return AFQMC_EINVAL;
  }
  AFQ_CUDA(cudaMalloc(&gr->d_jobs, sizeof(tc::GemmJob<Epi>) * (size_t)n));
  AFQ_CUDA(cudaMemcpy(gr->d_jobs, jobs.data(), sizeof(tc::GemmJob<Epi>) * (size_t)n,
                      cudaMemcpyHostToDevice));
  gr->njobs = n;
  gr->ntiles = (int)tiles;
  return AFQMC_OK;
}

template <int BN, int STAGES, bool TF32, class Epi>
int launch_grouped(const TcGrouped& gr, cudaStream_t st) {
  constexpr int kTotal = tc::Smem<BN, STAGES, Epi::kMT>::TOTAL + Epi::kSmemBytes;
  static_assert(kTotal <= 232448, "shared memory");
  auto kern = tc::k_tc_gemm_grouped<BN, STAGES, TF32, Epi>;
  static std::atomic<unsigned long long> attr{0};
  AFQ_TRY(smem_attr_once(kern, kTotal, attr));
  if (gr.ntiles <= 0) return AFQMC_OK;
  const int grid = gr.ntiles < tc_sm_count() ? gr.ntiles : tc_sm_count();
  AFQ_LAUNCH(kern, grid, 64 + 32 * Epi::kWarps, kTotal, st,
             static_cast<const tc::GemmJob<Epi>*>(gr.d_jobs), gr.njobs, gr.ntiles);
  return AFQMC_OK;
}

template <bool TF32>
int dispatch_grouped(const TcGrouped& gr, cudaStream_t st) {
  switch (gr.kind) {
    case TC_JOB_STORE:
      if (gr.bn == 64) return launch_grouped<64, 8, TF32, tc::EpiStore>(gr, st);
      if (gr.bn == 128) return launch_grouped<128, 6, TF32, tc::EpiStore>(gr, st);
      return launch_grouped<256, 4, TF32, tc::EpiStore>(gr, st);
    case TC_JOB_V:
      if (gr.bn == 128) return launch_grouped<128, 4, TF32, tc::EpiV>(gr, st);
      return launch_grouped<256, 3, TF32, tc::EpiV>(gr, st);
    case TC_JOB_PROP0:
      if (gr.bn == 160) return launch_grouped<160, kHalfStages160, TF32, tc::EpiProp0>(gr, st);
      return launch_grouped<256, 4, TF32, tc::EpiProp0>(gr, st);
    case TC_JOB_PHI:
      if (gr.bn == 160) return launch_grouped<160, kHalfStages160, TF32, tc::EpiPhi>(gr, st);
      return launch_grouped<256, 4, TF32, tc::EpiPhi>(gr, st);
  }
  set_error("grouped contraction: unknown kind %d", gr.kind);
  return AFQMC_EINVAL;
}

// Tile-width candidates of each kind (the ones with an instantiated kernel).
std::vector<int> bn_candidates(int kind) {
  switch (kind) {
    case TC_JOB_STORE:
      return {256, 128, 64};
    case TC_JOB_V:
      return {128, 256};
    default:
      return {160, 256};
  }
}
}  // namespace

int tc_grouped_create(const TcJobDesc* d, int n, int bn, TcGrouped** out) {
  *out = nullptr;
  if (n < 1) {
    set_error("grouped contraction: no jobs");
    return AFQMC_EINVAL;
  }
  for (int i = 1; i < n; ++i)
    if (d[i].kind != d[0].kind || d[i].g.tf32 != d[0].g.tf32) {
      set_error("grouped contraction: jobs of different kinds or precisions");
      return AFQMC_EINVAL;
    }
  const int kind = d[0].kind;
  if (bn == 0) bn = kind == TC_JOB_STORE ? 256 : kind == TC_JOB_V ? 128 : half_step_bn(d[0].M);
  bool ok = false;
  for (int c : bn_candidates(kind)) ok = ok || c == bn;
  if (!ok) {
    set_error("grouped contraction: no kernel for tile width %d", bn);
    return AFQMC_EINVAL;
  }
  TcGrouped* gr = new TcGrouped();
  gr->kind = kind;
  gr->bn = bn;
  gr->tf32 = d[0].g.tf32;
  int r = AFQMC_OK;
  switch (kind) {
    case TC_JOB_STORE:
      r = build_table<tc::EpiStore>(d, n, bn, gr);
      break;
    case TC_JOB_V:
      r = build_table<tc::EpiV>(d, n, bn, gr);
      break;
    case TC_JOB_PROP0:
      r = build_table<tc::EpiProp0>(d, n, bn, gr);
      break;
    case TC_JOB_PHI:
      r = build_table<tc::EpiPhi>(d, n, bn, gr);
      break;
    default:
      set_error("grouped contraction: unknown kind %d", kind);
      r = AFQMC_EINVAL;
  }
  if (r != AFQMC_OK) {
    tc_grouped_destroy(gr);
    return r;
  }
  *out = gr;
  return AFQMC_OK;
}

int tc_grouped_launch(const TcGrouped* gr, cudaStream_t st) {
  return gr->tf32 ? dispatch_grouped<true>(*gr, st) : dispatch_grouped<false>(*gr, st);
}

int tc_grouped_tune(const TcJobDesc* d, int n, cudaStream_t st, TcGrouped** out) {
  *out = nullptr;
  if (n < 1 || d[0].kind == TC_JOB_PHI) {
    set_error("grouped tune: no jobs, or a kind whose epilogue overwrites the walkers");
    return AFQMC_EINVAL;
  }
  cudaEvent_t e0, e1;
  AFQ_CUDA(cudaEventCreate(&e0));
  AFQ_CUDA(cudaEventCreate(&e1));
  TcGrouped* best = nullptr;
  float best_ms = 1e30f;
  int r = AFQMC_OK;
  for (int bn : bn_candidates(d[0].kind)) {
    TcGrouped* gr = nullptr;
    r = tc_grouped_create(d, n, bn, &gr);
    if (r != AFQMC_OK) break;
    float ms = 1e30f;
    r = tc_grouped_launch(gr, st);  // warm-up (and first-use set-up)
    // the fastest of three timings of two launches
    for (int trial = 0; trial < 3 && r == AFQMC_OK; ++trial) {
      float t = 0.f;
      if (cudaEventRecord(e0, st) != cudaSuccess) {
        set_error("grouped tune: event timing failed");
        r = AFQMC_ECUDA;
        break;
      }
      for (int rep = 0; rep < 2 && r == AFQMC_OK; ++rep) r = tc_grouped_launch(gr, st);
      if (r == AFQMC_OK && (cudaEventRecord(e1, st) != cudaSuccess ||
                            cudaEventSynchronize(e1) != cudaSuccess ||
                            cudaEventElapsedTime(&t, e0, e1) != cudaSuccess)) {
        set_error("grouped tune: event timing failed");
        r = AFQMC_ECUDA;
      }
      if (t < ms) ms = t;
    }
    if (r != AFQMC_OK) {
      tc_grouped_destroy(gr);
      break;
    }
    if (ms < best_ms) {
      best_ms = ms;
      tc_grouped_destroy(best);
      best = gr;
    } else {
      tc_grouped_destroy(gr);
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (r != AFQMC_OK) {
    tc_grouped_destroy(best);
    return r;
  }
  *out = best;
  return AFQMC_OK;
}

int tc_grouped_bn(const TcGrouped* gr) { return gr ? gr->bn : 0; }
int tc_grouped_tiles(const TcGrouped* gr) { return gr ? gr->ntiles : 0; }

void tc_grouped_destroy(TcGrouped* gr) {
  if (!gr) return;
  if (gr->d_jobs) cudaFree(gr->d_jobs);
  delete gr;
}

// Exchange blocking: RG Cholesky vectors x CW walkers per 128 x 256 tile.
void exchange_tile(int N, int* RG, int* CW, int* NPAD) {
  int npad = 16;
  while (npad < 2 * N) npad <<= 1;
  *NPAD = npad;
  *CW = npad <= 256 ? 256 / npad : 0;
  *RG = N <= 128 ? 128 / N : 0;
}

int tc_exchange(const TcGemm& g, int G, int W, int N, double* part, int nchunk, cudaStream_t st) {
  int RG, CW, NPAD;
  exchange_tile(N, &RG, &CW, &NPAD);
  if (RG < 1 || CW < 1 || CW > tc::EpiExchange::kMaxCW || nchunk != G) {
    set_error("tc exchange: N=%d not supported", N);
    return AFQMC_EUNSUPPORTED;
  }
  // B: Theta^T rows as [W][2N][ldb], one box = CW walkers x NPAD rows
  const int eb = g.tf32 ? 4 : 2;
  CUtensorMap tb;
  AFQ_TRY(make_tmap_3d(&tb, g.B, eb, W, 2L * N, g.k, g.ldb, 2L * N * g.ldb, NPAD, CW));
  tc::EpiExchange e{part, G, W, N, RG, CW, NPAD, nchunk};
  // K = M is a few k-blocks of L2-resident operands: a 2-deep ring leaves room
  // for the epilogue's own 128 KB tile buffer
  if (g.tf32)
    return launch_tc_persistent<256, 2, true>(g, e, cdiv(G, RG), cdiv(W, CW), st, &tb);
  return launch_tc_persistent<256, 2, false>(g, e, cdiv(G, RG), cdiv(W, CW), st, &tb);
}

}  // namespace afq

extern "C" int afqmc_contract(int32_t dtype, int64_t m, int64_t n, int64_t k, const void* dA,
                              int64_t lda, const void* dB, int64_t ldb, float alpha, float* dC,
                              int64_t ldc, int* d_status, void* stream) {
  if ((dtype != 0 && dtype != 1) || m < 0 || n < 0 || k < 1 || !dA || !dB || !dC || !d_status ||
      lda < k || ldb < k || ldc < n || m > (1ll << 31) - 1 || n > (1ll << 31) - 1 ||
      k > (1ll << 31) - 1) {
    afq::set_error("afqmc_contract: bad arguments");
    return AFQMC_EINVAL;
  }
  afq::TcGemm g;
  g.m = (int)m;
  g.n = (int)n;
  g.k = (int)k;
  g.A = dA;
  g.lda = lda;
  g.B = dB;
  g.ldb = ldb;
  g.tf32 = dtype == 1;
  g.err = d_status;
  return afq::tc_gemm_store(g, dC, ldc, alpha, static_cast<cudaStream_t>(stream));
}
