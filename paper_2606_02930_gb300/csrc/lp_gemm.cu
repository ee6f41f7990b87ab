// Low-precision tensor-core GEMM of the mixed-precision H_eff (sm_103a):
//
//   C[b][s] (fp32, M x N) = A[b][M][k-range s] * B[b][N][k-range s]^T
//
// A and B are K-major, either bf16 (tcgen05.mma kind::f16, K = 16 per
// instruction) or fp32 read as tf32 (kind::tf32, K = 8 per instruction);
// accumulation is fp32 in tensor memory.  s indexes an optional split of K
// whose partial products go to separate output slabs (the caller sums them).
//
// Persistent kernel, one CTA per SM, warp-specialised:
//   warp 0   one thread streams 128-byte-wide K tiles of A (128 rows) and B
//            (BN rows) into a ring of STAGES shared-memory buffers with TMA
//            (128-byte swizzle), each stage completing an mbarrier;
//   warp 1   one thread issues tcgen05.mma (M = 128, N = BN) into one of two
//            TMEM accumulators of BN columns and frees ring stages with
//            tcgen05.commit;
//   warps 2-9 read a finished accumulator with tcgen05.ld (two warps per TMEM
//            lane quarter, alternate 32-column chunks), turn the lane-per-row
//            values into row-contiguous stores through shared memory and
//            store fp32 (or bf16) rows, while the MMAs of the next tile fill
//            the other accumulator.
// Work units (batch x split x M tile x N tile) are dealt round-robin to the
// CTAs.  Every mbarrier wait is bounded: a wait that runs out sets the error
// word, the CTA stops issuing work, waits (again bounded) for the copies and
// MMAs it has in flight, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "convert.cuh"
#include "tc_ptx.cuh"

namespace ite {
namespace {

using namespace tc;

constexpr int LP_BM = 128;
constexpr int LP_STAGES = 4;
constexpr int LP_EPI_WARPS = 8;             // two warps per TMEM lane quarter
constexpr int LP_THREADS = 64 + 32 * LP_EPI_WARPS;
constexpr int LP_ROW_BYTES = 128;          // one K tile: 128 bytes per row

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, uint64_t* bar, int x,
                                            int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(bar))
      : "memory");
}

// 128-byte-swizzled K-major operand tile, rows 128 bytes apart, 8-row groups
// 1024 bytes apart (descriptor version 1, leading offset unused)
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// instruction descriptor: fp32 accumulator, A/B format fmt (1 = bf16 for
// kind::f16, 2 = tf32 for kind::tf32), both K-major, M = 128, N = bn
__host__ __device__ constexpr uint32_t lp_idesc(int bn, uint32_t fmt) {
  return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(bn >> 3) << 17) |
         ((uint32_t)(128 >> 4) << 24);
}

template <bool TF32>
__device__ __forceinline__ void mma_lp(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t accumulate) {
  if constexpr (TF32) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
  }
}

struct LpShape {
  int M, N, K;          // per batch entry; K in elements
  int batch, splits;    // batch entries and K splits
  int kb_per_split;     // K tiles per split
  int m_tiles, n_tiles;
  long long ldc, sCb, sCs;   // output (elements): row stride, batch stride, split stride
  int out_bf16;         // output rounded to bf16 instead of fp32
  int out_complex;      // complex FP64 output alpha prod + gamma Z (LpGemmArgs)
  float2 alpha, gamma;
  const cplx* Z;
};

// Per epilogue warp: a 32 x 32 fp32 tile (padded rows) through which the
// warp turns its lane-per-row TMEM reads into row-contiguous stores.
constexpr int LP_TRANS_BYTES = LP_EPI_WARPS * 32 * 33 * 4;

template <int BN, bool TF32>
__global__ void __launch_bounds__(LP_THREADS, 1)
k_lp_gemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
          void* __restrict__ C, LpShape sh, int a_batched, int b_batched, int* err) {
  constexpr uint32_t A_BYTES = LP_BM * LP_ROW_BYTES;    // 16 KB
  constexpr uint32_t B_BYTES = BN * LP_ROW_BYTES;       // 16 or 32 KB
  constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr int KSTEP = TF32 ? 8 : 16;                  // K per MMA instruction
  constexpr int ELEM = TF32 ? 4 : 2;
  constexpr int BK = LP_ROW_BYTES / ELEM;               // K elements per tile
  constexpr int MMAS = BK / KSTEP;                      // 4 per tile
  // two accumulators of BN columns; the allocation is a power of two
  constexpr uint32_t TMEM_COLS = 2 * BN <= 256 ? 256 : 512;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + LP_STAGES * STAGE_BYTES);
  uint64_t* empty = full + LP_STAGES;
  uint64_t* acc_full = empty + LP_STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  float* trans = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(tmem_slot + 4) + 15) & ~uintptr_t(15));
  __shared__ int s_fail;
  __shared__ int s_issued, s_consumed, s_mma_any;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const long long units = (long long)sh.batch * sh.splits * sh.m_tiles * sh.n_tiles;

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    s_mma_any = 0;
    for (int s = 0; s < LP_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], LP_EPI_WARPS);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  auto decode = [&](long long u, int& b, int& sp, int& mt, int& nt) {
    nt = (int)(u % sh.n_tiles);
    u /= sh.n_tiles;
    mt = (int)(u % sh.m_tiles);
    u /= sh.m_tiles;
    sp = (int)(u % sh.splits);
    b = (int)(u / sh.splits);
  };
  const int nkb_total = (sh.K + BK - 1) / BK;

  if (warp == 0) {
    // ---- TMA producer
    if (lane == 0) {
      int it = 0;
      for (long long u = blockIdx.x; u < units && !*((volatile int*)&s_fail); u += gridDim.x) {
        int b, sp, mt, nt;
        decode(u, b, sp, mt, nt);
        const int kb0 = sp * sh.kb_per_split;
        const int kb1 = min(nkb_total, kb0 + sh.kb_per_split);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % LP_STAGES;
          if (it >= LP_STAGES && !mbar_wait(&empty[s], ((it / LP_STAGES) + 1) & 1)) {
            s_fail = 1;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          mbar_expect_tx(&full[s], STAGE_BYTES);
          tma_load_3d(st, &tmA, &full[s], kb * BK, mt * LP_BM, a_batched ? b : 0);
          tma_load_3d(st + A_BYTES, &tmB, &full[s], kb * BK, nt * BN, b_batched ? b : 0);
          s_issued = it + 1;
        }
        if (s_fail) break;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = lp_idesc(BN, TF32 ? 2u : 1u);
      int it = 0, lt = 0;
      for (long long u = blockIdx.x; u < units && !*((volatile int*)&s_fail); u += gridDim.x, ++lt) {
        int b, sp, mt, nt;
        decode(u, b, sp, mt, nt);
        const int kb0 = sp * sh.kb_per_split;
        const int kb1 = min(nkb_total, kb0 + sh.kb_per_split);
        const int buf = lt & 1, use = lt >> 1;
        if (use >= 1 && !mbar_wait(&acc_empty[buf], (use - 1) & 1)) {
          s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + buf * BN;
        bool first = true;
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % LP_STAGES;
          if (!mbar_wait(&full[s], (it / LP_STAGES) & 1)) {
            s_fail = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
          const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < MMAS; ++kk) {
            mma_lp<TF32>(acc, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                         first ? 0u : 1u);
            first = false;
          }
          s_mma_any = 1;
          mma_commit(&empty[s]);
          s_consumed = it + 1;
        }
        if (s_fail) break;
        if (first) {
          // an empty K range (cannot happen for K >= 1): the accumulator was
          // never written, so the epilogue must see zeros; not supported
          s_fail = 1;
          break;
        }
        mma_commit(&acc_full[buf]);
      }
      mma_commit(done);
    }
  } else {
    // ---- epilogue warps 2..9: TMEM lane quarter warp % 4; the two warps of a
    // quarter take alternate 32-column chunks
    const int q = warp & 3, half = (warp - 2) >> 2;
    int lt = 0;
    for (long long u = blockIdx.x; u < units; u += gridDim.x, ++lt) {
      int b, sp, mt, nt;
      decode(u, b, sp, mt, nt);
      const int buf = lt & 1, use = lt >> 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], use & 1) ? 1 : 0) != 0;
      if (!ok) {
        if (lane == 0) s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row0 = mt * LP_BM + q * 32;
      const long long cbase = (long long)b * sh.sCb + (long long)sp * sh.sCs;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + buf * BN;
      float* tp = trans + (warp - 2) * 32 * 33;
#pragma unroll 1
      for (int c = half; c < BN / 32; c += 2) {
        float v[32];
        tmem_ld32(tbase + c * 32, v);
        // lane = row: through shared memory, lane = column
#pragma unroll
        for (int i = 0; i < 32; ++i) tp[lane * 33 + i] = v[i];
        __syncwarp();
        const int col = nt * BN + c * 32 + lane;
        if (sh.out_complex) {
          // lanes 2k, 2k+1 hold (Re, Im) of complex column col / 2: the even
          // lane combines and stores 16 bytes, 16 lanes a 256-byte row segment
          const int rows = min(32, sh.M - row0);
          const long long cc = col >> 1;
          const bool store = (lane & 1) == 0 && col < sh.N;
          for (int r = 0; r < rows; ++r) {
            const float re = tp[r * 33 + lane];
            const float im = __shfl_down_sync(0xffffffffu, re, 1);
            if (store) {
              const long long idx = (long long)(row0 + r) * sh.ldc + cc;
              float ore = sh.alpha.x * re - sh.alpha.y * im;
              float oim = sh.alpha.x * im + sh.alpha.y * re;
              if (sh.Z) {
                const cplx z = __ldcs(sh.Z + idx);
                const float zr = dbl_to_f32(z.x), zi = dbl_to_f32(z.y);
                ore = fmaf(sh.gamma.x, zr, fmaf(-sh.gamma.y, zi, ore));
                oim = fmaf(sh.gamma.x, zi, fmaf(sh.gamma.y, zr, oim));
              }
              __stcs(reinterpret_cast<cplx*>(C) + idx, cmake(f32_to_dbl(ore), f32_to_dbl(oim)));
            }
          }
        } else if (col < sh.N) {
          const int rows = min(32, sh.M - row0);
          if (sh.out_bf16) {
            __nv_bfloat16* cb = reinterpret_cast<__nv_bfloat16*>(C) + cbase + col;
            for (int r = 0; r < rows; ++r)
              cb[(long long)(row0 + r) * sh.ldc] = __float2bfloat16_rn(tp[r * 33 + lane]);
          } else {
            float* cf = reinterpret_cast<float*>(C) + cbase + col;
            for (int r = 0; r < rows; ++r) cf[(long long)(row0 + r) * sh.ldc] = tp[r * 33 + lane];
          }
        }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive1(&acc_empty[buf]);
      if (*((volatile int*)&s_fail)) break;
    }
  }
  __syncthreads();
  // every MMA this CTA issued has completed once `done` fires (bounded); a
  // failed CTA also waits for the copies it issued that no MMA consumed
  if (threadIdx.x == 0) {
    mbar_wait(done, 0);
    if (s_fail) {
      for (int it = s_consumed; it < s_issued; ++it)
        mbar_wait(&full[it % LP_STAGES], (it / LP_STAGES) & 1);
      atomicExch(err, 1);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// ---------------------------------------------------------------- CTA pairs
// The same GEMM on 256 x BN tiles computed by a pair of CTAs (a cluster of
// two, cta_group::2): each CTA stages its 128 rows of A and its BN/2 rows of
// B, the MMAs issued by the even CTA read both CTAs' tiles and write each
// CTA's 128 accumulator rows into its own tensor memory.  Per CTA and K tile
// that moves 16 + BN/4 KB instead of 16 + BN/2 KB for the same MMA work.
//   - Both CTAs' copies complete on the even CTA's `full` barrier, which its
//     producer arms with the bytes of both;
//   - the even CTA's commits arrive on both CTAs' `empty`, `acc_full` and
//     `done` barriers (multicast);
//   - both CTAs' epilogue warps arrive on the even CTA's `acc_empty`.
// Waits are bounded as in the one-CTA kernel; a CTA whose wait ran out stops
// issuing, and before either CTA leaves, the even CTA waits (bounded) for
// every copy either CTA issued that no MMA consumed.
constexpr int LP2_STAGES = 5;

__device__ __forceinline__ uint32_t cluster_rank() {
  uint32_t r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

__device__ __forceinline__ uint32_t map_to_rank(const void* p, uint32_t rank) {
  uint32_t out;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(out) : "r"(smem_u32(p)), "r"(rank));
  return out;
}

__device__ __forceinline__ void cluster_sync() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

__device__ __forceinline__ void tma_load_3d_pair(void* dst, const CUtensorMap* map, uint32_t bar_cluster,
                                                 int x, int y, int z) {
  asm volatile(
      "cp.async.bulk.tensor.3d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
          "r"(smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar_cluster)
      : "memory");
}

template <bool TF32>
__device__ __forceinline__ void mma_lp_pair(uint32_t tmem_d, uint64_t da, uint64_t db,
                                            uint32_t idesc, uint32_t accumulate) {
  if constexpr (TF32) {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::2.kind::tf32 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
  } else {
    asm volatile(
        "{\n"
        ".reg .pred p;\n"
        "setp.ne.b32 p, %4, 0;\n"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n"
        "}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
  }
}

__device__ __forceinline__ void commit_pair(uint64_t* bar) {
  const uint16_t mask = 3;
  asm volatile(
      "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
          smem_u32(bar)),
      "h"(mask)
      : "memory");
}

__device__ __forceinline__ void mbar_arrive_cluster(uint32_t bar_cluster) {
  asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(bar_cluster)
               : "memory");
}

template <int BN, bool TF32>
__global__ void __launch_bounds__(LP_THREADS, 1)
k_lp_gemm_pair(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               void* __restrict__ C, LpShape sh, int a_batched, int b_batched, int* err) {
  constexpr int BMP = 2 * LP_BM;                        // tile rows of the pair
  constexpr int BNH = BN / 2;                           // B rows per CTA
  constexpr uint32_t A_BYTES = LP_BM * LP_ROW_BYTES;    // 16 KB
  constexpr uint32_t B_BYTES = BNH * LP_ROW_BYTES;
  constexpr uint32_t STAGE_BYTES = A_BYTES + B_BYTES;
  constexpr int KSTEP = TF32 ? 8 : 16;
  constexpr int ELEM = TF32 ? 4 : 2;
  constexpr int BK = LP_ROW_BYTES / ELEM;
  constexpr int MMAS = BK / KSTEP;
  constexpr uint32_t TMEM_COLS = 2 * BN <= 256 ? 256 : 512;
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + LP2_STAGES * STAGE_BYTES);
  uint64_t* empty = full + LP2_STAGES;
  uint64_t* acc_full = empty + LP2_STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint64_t* done = acc_empty + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(done + 1);
  int* peer_issued = reinterpret_cast<int*>(tmem_slot + 1);   // written by the odd CTA
  float* trans = reinterpret_cast<float*>(
      (reinterpret_cast<uintptr_t>(tmem_slot + 4) + 15) & ~uintptr_t(15));
  __shared__ int s_fail;
  __shared__ int s_issued, s_consumed;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t rank = cluster_rank();
  const bool leader = rank == 0;
  const int pair = (int)(blockIdx.x >> 1), npairs = (int)(gridDim.x >> 1);
  const long long units = (long long)sh.batch * sh.splits * sh.m_tiles * sh.n_tiles;

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_issued = 0;
    s_consumed = 0;
    *peer_issued = 0;
    for (int s = 0; s < LP2_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 2 * LP_EPI_WARPS);
    }
    mbar_init(done, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(TMEM_COLS));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();                      // barriers and TMEM of both CTAs are set up
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  auto decode = [&](long long u, int& b, int& sp, int& mt, int& nt) {
    nt = (int)(u % sh.n_tiles);
    u /= sh.n_tiles;
    mt = (int)(u % sh.m_tiles);
    u /= sh.m_tiles;
    sp = (int)(u % sh.splits);
    b = (int)(u / sh.splits);
  };
  const int nkb_total = (sh.K + BK - 1) / BK;

  if (warp == 0) {
    // ---- TMA producer of this CTA's halves; copies complete on the even CTA
    if (lane == 0) {
      int it = 0;
      for (long long u = pair; u < units && !*((volatile int*)&s_fail); u += npairs) {
        int b, sp, mt, nt;
        decode(u, b, sp, mt, nt);
        const int kb0 = sp * sh.kb_per_split;
        const int kb1 = min(nkb_total, kb0 + sh.kb_per_split);
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % LP2_STAGES;
          if (it >= LP2_STAGES && !mbar_wait(&empty[s], ((it / LP2_STAGES) + 1) & 1)) {
            s_fail = 1;
            break;
          }
          uint8_t* st = smem + s * STAGE_BYTES;
          if (leader) mbar_expect_tx(&full[s], 2 * STAGE_BYTES);
          const uint32_t fb = map_to_rank(&full[s], 0);
          tma_load_3d_pair(st, &tmA, fb, kb * BK, mt * BMP + (int)rank * LP_BM, a_batched ? b : 0);
          tma_load_3d_pair(st + A_BYTES, &tmB, fb, kb * BK, nt * BN + (int)rank * BNH, b_batched ? b : 0);
          s_issued = it + 1;
        }
        if (s_fail) break;
      }
    }
  } else if (warp == 1) {
    // ---- MMA issuer: the even CTA's one thread drives the pair
    if (lane == 0 && leader) {
      constexpr uint32_t idesc = (1u << 4) | ((TF32 ? 2u : 1u) << 7) | ((TF32 ? 2u : 1u) << 10) |
                                 ((uint32_t)(BN >> 3) << 17) | ((uint32_t)(BMP >> 4) << 24);
      int it = 0, lt = 0;
      for (long long u = pair; u < units && !*((volatile int*)&s_fail); u += npairs, ++lt) {
        int b, sp, mt, nt;
        decode(u, b, sp, mt, nt);
        const int kb0 = sp * sh.kb_per_split;
        const int kb1 = min(nkb_total, kb0 + sh.kb_per_split);
        const int buf = lt & 1, use = lt >> 1;
        if (use >= 1 && !mbar_wait(&acc_empty[buf], (use - 1) & 1)) {
          s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t acc = tmem + buf * BN;
        bool first = true;
        for (int kb = kb0; kb < kb1; ++kb, ++it) {
          const int s = it % LP2_STAGES;
          if (!mbar_wait(&full[s], (it / LP2_STAGES) & 1)) {
            s_fail = 1;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t a0 = smem_u32(smem + s * STAGE_BYTES);
          const uint32_t b0 = a0 + A_BYTES;
#pragma unroll
          for (int kk = 0; kk < MMAS; ++kk) {
            mma_lp_pair<TF32>(acc, sw128_desc(a0 + kk * 32), sw128_desc(b0 + kk * 32), idesc,
                              first ? 0u : 1u);
            first = false;
          }
          commit_pair(&empty[s]);
          s_consumed = it + 1;
        }
        if (s_fail) break;
        if (first) {
          s_fail = 1;
          break;
        }
        commit_pair(&acc_full[buf]);
      }
      commit_pair(done);
    }
  } else {
    // ---- epilogue warps 2..9 of both CTAs: this CTA's 128 rows of the tile
    const int q = warp & 3, half = (warp - 2) >> 2;
    const uint32_t acc_empty_leader[2] = {map_to_rank(&acc_empty[0], 0), map_to_rank(&acc_empty[1], 0)};
    int lt = 0;
    for (long long u = pair; u < units; u += npairs, ++lt) {
      int b, sp, mt, nt;
      decode(u, b, sp, mt, nt);
      const int buf = lt & 1, use = lt >> 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], use & 1) ? 1 : 0) != 0;
      if (!ok) {
        if (lane == 0) s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int row0 = mt * BMP + (int)rank * LP_BM + q * 32;
      const long long cbase = (long long)b * sh.sCb + (long long)sp * sh.sCs;
      const uint32_t tbase = tmem + ((uint32_t)(q * 32) << 16) + buf * BN;
      float* tp = trans + (warp - 2) * 32 * 33;
#pragma unroll 1
      for (int c = half; c < BN / 32; c += 2) {
        float v[32];
        tmem_ld32(tbase + c * 32, v);
#pragma unroll
        for (int i = 0; i < 32; ++i) tp[lane * 33 + i] = v[i];
        __syncwarp();
        const int col = nt * BN + c * 32 + lane;
        const int rows = min(32, sh.M - row0);
        if (sh.out_complex) {
          const long long cc = col >> 1;
          const bool store = (lane & 1) == 0 && col < sh.N;
          for (int r = 0; r < rows; ++r) {
            const float re = tp[r * 33 + lane];
            const float im = __shfl_down_sync(0xffffffffu, re, 1);
            if (store) {
              const long long idx = (long long)(row0 + r) * sh.ldc + cc;
              float ore = sh.alpha.x * re - sh.alpha.y * im;
              float oim = sh.alpha.x * im + sh.alpha.y * re;
              if (sh.Z) {
                const cplx z = __ldcs(sh.Z + idx);
                const float zr = dbl_to_f32(z.x), zi = dbl_to_f32(z.y);
                ore = fmaf(sh.gamma.x, zr, fmaf(-sh.gamma.y, zi, ore));
                oim = fmaf(sh.gamma.x, zi, fmaf(sh.gamma.y, zr, oim));
              }
              __stcs(reinterpret_cast<cplx*>(C) + idx, cmake(f32_to_dbl(ore), f32_to_dbl(oim)));
            }
          }
        } else if (col < sh.N) {
          if (sh.out_bf16) {
            __nv_bfloat16* cb = reinterpret_cast<__nv_bfloat16*>(C) + cbase + col;
            for (int r = 0; r < rows; ++r)
              cb[(long long)(row0 + r) * sh.ldc] = __float2bfloat16_rn(tp[r * 33 + lane]);
          } else {
            float* cf = reinterpret_cast<float*>(C) + cbase + col;
            for (int r = 0; r < rows; ++r) cf[(long long)(row0 + r) * sh.ldc] = tp[r * 33 + lane];
          }
        }
        __syncwarp();
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      __syncwarp();
      if (lane == 0) mbar_arrive_cluster(acc_empty_leader[buf]);
      if (*((volatile int*)&s_fail)) break;
    }
  }
  __syncthreads();
  // every MMA of the pair has completed once `done` fires (bounded)
  if (threadIdx.x == 0) mbar_wait(done, 0);
  // the odd CTA reports the copies it issued; the even CTA then waits for
  // every copy either issued that no MMA consumed, before either leaves
  if (threadIdx.x == 0 && !leader) {
    const uint32_t slot = map_to_rank(peer_issued, 0);
    asm volatile("st.shared::cluster.u32 [%0], %1;" ::"r"(slot), "r"((uint32_t)s_issued) : "memory");
  }
  cluster_sync();
  if (threadIdx.x == 0 && leader) {
    const int issued = max(s_issued, *((volatile int*)peer_issued));
    for (int it = s_consumed; it < issued; ++it)
      if (!mbar_wait(&full[it % LP2_STAGES], (it / LP2_STAGES) & 1)) break;
  }
  if (threadIdx.x == 0 && s_fail) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  cluster_sync();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TMEM_COLS));
  }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 g_enc = nullptr;
std::mutex g_enc_mutex;

cudaError_t encoder() {
  std::lock_guard<std::mutex> lock(g_enc_mutex);
  if (g_enc) return cudaSuccess;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_enc = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return cudaSuccess;
}

// 3-D map over rows x cols (row stride ld elements) x batch (stride sb
// elements; extent 1 when sb == 0), box of box_rows x 128 bytes x 1,
// 128-byte swizzle, zero fill outside.
cudaError_t make_map3(CUtensorMap* map, const void* base, bool tf32, long long rows,
                      long long cols, long long ld, long long batch, long long sb, int box_rows) {
  const int eb = tf32 ? 4 : 2;
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * eb) % 16 || (sb * eb) % 16 || cols < 1 ||
      rows < 1 || batch < 1)
    return cudaErrorInvalidValue;
  const bool batched = sb != 0 && batch > 1;
  cuuint64_t dims[3] = {(cuuint64_t)cols, (cuuint64_t)rows, (cuuint64_t)(batched ? batch : 1)};
  cuuint64_t strides[2] = {(cuuint64_t)(ld * eb), (cuuint64_t)((batched ? sb : rows * ld) * eb)};
  cuuint32_t box[3] = {(cuuint32_t)(LP_ROW_BYTES / eb), (cuuint32_t)box_rows, 1};
  cuuint32_t estr[3] = {1, 1, 1};
  CUresult r = g_enc(map, tf32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                     3, const_cast<void*>(base), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN>
constexpr size_t lp_smem_bytes() {
  return 1024 + LP_STAGES * (LP_BM + BN) * LP_ROW_BYTES + (2 * LP_STAGES + 5) * 8 + 16 + 16 +
         LP_TRANS_BYTES;
}

struct SmCount {
  std::mutex mu;
  int sms[64] = {0};
  int get() {
    int d = 0;
    if (cudaGetDevice(&d) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    if (sms[d & 63] == 0) cudaDeviceGetAttribute(&sms[d & 63], cudaDevAttrMultiProcessorCount, d);
    return sms[d & 63];
  }
};
SmCount g_sms;

template <int BN, bool TF32>
cudaError_t launch_lp(const CUtensorMap& ma, const CUtensorMap& mb, void* C, const LpShape& sh,
                      int a_batched, int b_batched, int* err, cudaStream_t st) {
  static std::atomic<unsigned long long> attr_done{0};
  constexpr size_t smem = lp_smem_bytes<BN>();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_done.load() & bit)) {
    e = cudaFuncSetAttribute(k_lp_gemm<BN, TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    attr_done.fetch_or(bit);
  }
  const long long units = (long long)sh.batch * sh.splits * sh.m_tiles * sh.n_tiles;
  int sms = g_sms.get();
  if (sms <= 0) sms = 148;
  const int grid = (int)(units < sms ? units : sms);
  count_launches(1);
  k_lp_gemm<BN, TF32><<<grid, LP_THREADS, smem, st>>>(ma, mb, C, sh, a_batched, b_batched, err);
  return cudaGetLastError();
}

template <int BN>
constexpr size_t lp2_smem_bytes() {
  return 1024 + LP2_STAGES * (LP_BM + BN / 2) * LP_ROW_BYTES + (2 * LP2_STAGES + 5) * 8 + 16 + 16 +
         LP_TRANS_BYTES;
}

template <int BN, bool TF32>
cudaError_t launch_lp_pair(const CUtensorMap& ma, const CUtensorMap& mb, void* C,
                           const LpShape& sh, int a_batched, int b_batched, int* err,
                           cudaStream_t st) {
  static std::atomic<unsigned long long> attr_done{0};
  constexpr size_t smem = lp2_smem_bytes<BN>();
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const unsigned long long bit = 1ull << (dev & 63);
  if (!(attr_done.load() & bit)) {
    e = cudaFuncSetAttribute(k_lp_gemm_pair<BN, TF32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e != cudaSuccess) return e;
    attr_done.fetch_or(bit);
  }
  const long long units = (long long)sh.batch * sh.splits * sh.m_tiles * sh.n_tiles;
  int sms = g_sms.get();
  if (sms <= 0) sms = 148;
  const int pairs = (int)(units < sms / 2 ? units : sms / 2);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2 * pairs);
  cfg.blockDim = dim3(LP_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  count_launches(1);
  return cudaLaunchKernelEx(&cfg, k_lp_gemm_pair<BN, TF32>, ma, mb, C, sh, a_batched, b_batched,
                            err);
}

}  // namespace

int lp_gemm_sm_count() { return g_sms.get(); }

cudaError_t lp_gemm(const LpGemmArgs& g, int* err, cudaStream_t st) {
  if (g.M < 1 || g.N < 1 || g.K < 1 || g.batch < 1) return cudaSuccess;
  if (g.bn != 128 && g.bn != 192 && g.bn != 256) return cudaErrorInvalidValue;
  cudaError_t e = encoder();
  if (e != cudaSuccess) return e;
  const int eb = g.tf32 ? 4 : 2;
  const int BK = LP_ROW_BYTES / eb;
  const int nkb = (g.K + BK - 1) / BK;
  const int splits = g.splits < 1 ? 1 : (g.splits > nkb ? nkb : g.splits);
  LpShape sh;
  sh.M = g.M;
  sh.N = g.N;
  sh.K = g.K;
  sh.batch = g.batch;
  sh.kb_per_split = (nkb + splits - 1) / splits;
  sh.splits = (nkb + sh.kb_per_split - 1) / sh.kb_per_split;
  const int tile_m = g.pair ? 2 * LP_BM : LP_BM;
  sh.m_tiles = (g.M + tile_m - 1) / tile_m;
  sh.n_tiles = (g.N + g.bn - 1) / g.bn;
  sh.ldc = g.ldc;
  sh.sCb = g.sCb;
  sh.sCs = g.sCs;
  sh.out_bf16 = g.out_bf16 ? 1 : 0;
  sh.out_complex = g.out_complex ? 1 : 0;
  sh.alpha = g.alpha;
  sh.gamma = g.gamma;
  sh.Z = g.Z;
  if (g.out_complex && (splits > 1 || g.batch != 1 || (g.N & 1))) return cudaErrorInvalidValue;
  if (sh.splits > 1 && g.sCs == 0) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  e = make_map3(&ma, g.A, g.tf32, g.M, g.K, g.lda, g.batch, g.sAb, LP_BM);
  if (e != cudaSuccess) return e;
  e = make_map3(&mb, g.B, g.tf32, g.N, g.K, g.ldb, g.batch, g.sBb, g.pair ? g.bn / 2 : g.bn);
  if (e != cudaSuccess) return e;
  const int ab = (g.sAb != 0 && g.batch > 1) ? 1 : 0, bb = (g.sBb != 0 && g.batch > 1) ? 1 : 0;
  if (g.pair) {
    if (g.tf32) {
      if (g.bn == 256) return launch_lp_pair<256, true>(ma, mb, g.C, sh, ab, bb, err, st);
      if (g.bn == 192) return launch_lp_pair<192, true>(ma, mb, g.C, sh, ab, bb, err, st);
      return launch_lp_pair<128, true>(ma, mb, g.C, sh, ab, bb, err, st);
    }
    if (g.bn == 256) return launch_lp_pair<256, false>(ma, mb, g.C, sh, ab, bb, err, st);
    if (g.bn == 192) return launch_lp_pair<192, false>(ma, mb, g.C, sh, ab, bb, err, st);
    return launch_lp_pair<128, false>(ma, mb, g.C, sh, ab, bb, err, st);
  }
  if (g.tf32) {
    if (g.bn == 256) return launch_lp<256, true>(ma, mb, g.C, sh, ab, bb, err, st);
    if (g.bn == 192) return launch_lp<192, true>(ma, mb, g.C, sh, ab, bb, err, st);
    return launch_lp<128, true>(ma, mb, g.C, sh, ab, bb, err, st);
  }
  if (g.bn == 256) return launch_lp<256, false>(ma, mb, g.C, sh, ab, bb, err, st);
  if (g.bn == 192) return launch_lp<192, false>(ma, mb, g.C, sh, ab, bb, err, st);
  return launch_lp<128, false>(ma, mb, g.C, sh, ab, bb, err, st);
}

int lp_gemm_splits_used(const LpGemmArgs& g) {
  const int eb = g.tf32 ? 4 : 2;
  const int BK = LP_ROW_BYTES / eb;
  const int nkb = (g.K + BK - 1) / BK;
  const int splits = g.splits < 1 ? 1 : (g.splits > nkb ? nkb : g.splits);
  const int per = (nkb + splits - 1) / splits;
  return (nkb + per - 1) / per;
}

}  // namespace ite
