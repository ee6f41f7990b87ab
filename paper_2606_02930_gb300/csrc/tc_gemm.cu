// Tensor-core GEMM on sm_103a with the fifth-generation MMA (tcgen05):
//   C[M][N] (fp32) = A[M][K] * B[N][K]^T,  A and B bf16, both K-major.
//
// One CTA computes a 128 x BN tile.  Warp 0 (one thread) streams A and B
// tiles of 64 K-elements into shared memory with TMA (128-byte swizzle) through
// a ring of STAGES buffers; warp 1 (one thread) issues tcgen05.mma (M = 128,
// N = BN, K = 16 per instruction) that accumulate in tensor memory; each MMA
// group's completion frees its ring slot through tcgen05.commit.  After the
// last group, all four warps read the accumulator out of TMEM
// (tcgen05.ld 32x32b: warp w owns rows 32w..32w+31) and store fp32 to C.
//
// Every wait on an mbarrier is bounded.  A wait that runs out sets an error
// word, the block stops issuing work, drains (again bounded) the copies and
// MMAs it already issued, frees its TMEM and returns; the host reports
// ITE_ETIMEOUT.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <atomic>
#include <cstdint>
#include <mutex>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace ite {
namespace {

using namespace tc;

constexpr int TC_THREADS = 128;
constexpr int TC_BM = 128;
constexpr int TC_STAGES = 4;
template <int BN, int TC_BK>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_tc_gemm_bf16(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               float* __restrict__ C, int M, int N, int K, long long ldc, int* err) {
  constexpr uint32_t A_BYTES = TC_BM * TC_BK * 2;
  constexpr uint32_t B_BYTES = BN * TC_BK * 2;
  extern __shared__ uint8_t smem_raw[];
  // 1024-byte alignment for the 128-byte swizzle pattern
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* sA = smem;
  uint8_t* sB = smem + TC_STAGES * A_BYTES;
  uint64_t* full = reinterpret_cast<uint64_t*>(sB + TC_STAGES * B_BYTES);
  uint64_t* empty = full + TC_STAGES;
  uint64_t* accb = empty + TC_STAGES;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(accb + 1);
  __shared__ int s_fail, s_issued_tma, s_issued_mma;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * TC_BM, n0 = blockIdx.x * BN;
  const int nk = (K + TC_BK - 1) / TC_BK;

  if (threadIdx.x == 0) {
    s_fail = 0;
    s_issued_tma = 0;
    s_issued_mma = 0;
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(accb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(BN));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (threadIdx.x == 0) {
    // ---- TMA producer
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % TC_STAGES;
      if (kb >= TC_STAGES && !mbar_wait(&empty[s], ((kb / TC_STAGES) + 1) & 1)) {
        s_fail = 1;
        break;
      }
      mbar_expect_tx(&full[s], A_BYTES + B_BYTES);
      tma_load_2d(sA + s * A_BYTES, &tmA, &full[s], kb * TC_BK, m0);
      tma_load_2d(sB + s * B_BYTES, &tmB, &full[s], kb * TC_BK, n0);
      s_issued_tma = kb + 1;
    }
  } else if (threadIdx.x == 32) {
    // ---- MMA issuer
    constexpr uint32_t idesc = bf16_idesc(BN);
    for (int kb = 0; kb < nk; ++kb) {
      const int s = kb % TC_STAGES;
      if (!mbar_wait(&full[s], (kb / TC_STAGES) & 1)) {
        s_fail = 1;
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t a0 = smem_u32(sA + s * A_BYTES), b0 = smem_u32(sB + s * B_BYTES);
#pragma unroll
      for (int kk = 0; kk < TC_BK / 16; ++kk)
        mma_bf16(tmem, kmajor_desc<TC_BK>(a0 + kk * 32), kmajor_desc<TC_BK>(b0 + kk * 32), idesc,
                 (kb > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
      s_issued_mma = kb + 1;
    }
    mma_commit(accb);
  }
  __syncthreads();
  // ---- epilogue: every warp waits for the accumulator
  const bool ok = __all_sync(0xffffffffu, mbar_wait(accb, 0) ? 1 : 0) != 0;
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const bool failed = s_fail != 0;
  if (ok && !failed) {
    const int row = m0 + warp * 32 + lane;
    const uint32_t tbase = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int c = 0; c < BN / 32; ++c) {
      float v[32];
      tmem_ld32(tbase + c * 32, v);
      if (row < M) {
        float* crow = C + (long long)row * ldc + n0 + c * 32;
        const int lim = N - (n0 + c * 32);
#pragma unroll
        for (int i = 0; i < 32; ++i)
          if (i < lim) crow[i] = v[i];
      }
    }
  } else if (threadIdx.x == 0) {
    atomicExch(err, 1);
  }
  // ---- drain (bounded) copies this block issued that no MMA consumed
  if (threadIdx.x == 0 && (!ok || failed)) {
    for (int kb = s_issued_mma; kb < s_issued_tma; ++kb)
      mbar_wait(&full[kb % TC_STAGES], (kb / TC_STAGES) & 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(BN));
  }
}

// ---------------------------------------------------------------- host side
PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
std::mutex g_encode_mutex;

cudaError_t get_encoder() {
  std::lock_guard<std::mutex> lock(g_encode_mutex);
  if (g_encode) return cudaSuccess;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                   cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  return cudaSuccess;
}

// 2-D bf16 tensor map: `rows` rows of `cols` elements (row stride ld
// elements), box of box_rows x 64 elements, 128-byte swizzle, zero fill.
cudaError_t make_map(CUtensorMap* map, const void* base, long long rows, long long cols,
                     long long ld, int box_rows, int bk) {
  if ((reinterpret_cast<uintptr_t>(base) & 15) || (ld * 2) % 16 || cols < 1 || rows < 1)
    return cudaErrorInvalidValue;
  cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)(ld * 2)};
  cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims,
                        strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                        bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN, int BK>
size_t smem_bytes() {
  return 1024 + TC_STAGES * (TC_BM * BK * 2 + BN * BK * 2) + (2 * TC_STAGES + 1) * 8 + 16;
}

template <int BN, int BK>
cudaError_t launch(const CUtensorMap& ma, const CUtensorMap& mb, float* C, int M, int N, int K,
                   long long ldc, int* err, cudaStream_t st) {
  // the shared-memory attribute is per device; setting it twice from two
  // threads is harmless
  static std::atomic<unsigned long long> attr_done{0};
  const size_t sm = smem_bytes<BN, BK>();
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_done.load() & bit)) {
      e = cudaFuncSetAttribute(k_tc_gemm_bf16<BN, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
      if (e != cudaSuccess) return e;
      attr_done.fetch_or(bit);
    }
  }
  dim3 grid((N + BN - 1) / BN, (M + TC_BM - 1) / TC_BM);
  count_launches(1);
  k_tc_gemm_bf16<BN, BK><<<grid, TC_THREADS, sm, st>>>(ma, mb, C, M, N, K, ldc, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t make_digit_map(CUtensorMap* map, const void* base, long long rows, long long cols,
                           int box_rows) {
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  return make_map(map, base, rows, cols, cols, box_rows, 32);
}

cudaError_t tc_gemm_bf16(const void* A, long long lda, const void* B, long long ldb, float* C,
                         long long ldc, int M, int N, int K, int* err, cudaStream_t st, int bk) {
  if (M < 1 || N < 1 || K < 1) return cudaSuccess;
  if (M > 65535 * TC_BM) return cudaErrorInvalidValue;
  cudaError_t e = get_encoder();
  if (e != cudaSuccess) return e;
  const int bn = (N <= 64) ? 64 : 128;
  if (bk != 64 && bk != 32) return cudaErrorInvalidValue;
  CUtensorMap ma, mb;
  e = make_map(&ma, A, M, K, lda, TC_BM, bk);
  if (e != cudaSuccess) return e;
  e = make_map(&mb, B, N, K, ldb, bn, bk);
  if (e != cudaSuccess) return e;
  if (bk == 32) {
    if (bn == 64) return launch<64, 32>(ma, mb, C, M, N, K, ldc, err, st);
    return launch<128, 32>(ma, mb, C, M, N, K, ldc, err, st);
  }
  if (bn == 64) return launch<64, 64>(ma, mb, C, M, N, K, ldc, err, st);
  return launch<128, 64>(ma, mb, C, M, N, K, ldc, err, st);
}

}  // namespace ite
