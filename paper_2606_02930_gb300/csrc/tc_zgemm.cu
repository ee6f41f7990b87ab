// FP64-accurate complex GEMM on the bf16 tensor cores by exact slicing.
//
// GB300 runs FP64 at about 1.2 TFLOP/s but bf16 MMA at about 2 PFLOP/s, so the
// contractions of the FP64 path are computed as sums of exact bf16 products:
//
//  * complex C = op(A) op(B) becomes the real product of the row-embedded
//    A^ (rows 2r, 2r+1 = [Re, -Im], [Im, Re] interleaved along K) with the
//    K-major B^T (rows = columns of B, (Re, Im) interleaved along K);
//  * every row of A^ and every row of B^T is scaled by its own power of two
//    2^e (largest magnitude < 2^e), rounded to the nearest multiple of
//    2^(e-56) (error <= 2^(e-57)) and cut into S = 8 balanced base-128
//    digits, x = 2^e sum_p a_p 2^(-7p) with a_1 in [-128, 128] and the lower
//    digits in [-64, 64], zero-centred so that the rounding and the dropped
//    products below are unbiased.  Each digit is exact in bf16.  The slicing
//    uses integer operations on the bit patterns only;
//  * digit products a_p b_q of the same weight d = p + q are accumulated by
//    tcgen05.mma in one fp32 TMEM accumulator per d = 2..S+1 over K-chunks of
//    128 real terms: |a_1 b_1| <= 2^14 and every other product is at most
//    2^13, so every partial sum is an integer of magnitude below
//    128 (2 2^13 + (S-2) 2^12) < 2^24 and fp32 accumulation is exact;
//  * after each chunk the epilogue warps convert the accumulators to integers
//    and add them exactly into two int64 registers per output
//    (hi = sum_{d<=4} v_d 2^(7(4-d)), lo = sum_{d>=5} v_d 2^(7(S+1-d))); the
//    result is 2^(eA+eB) (hi 2^-28 + lo 2^-7(S+1)), rounded once to FP64.
//  Products of weight d > S+1 are dropped (both digits are low ones: at most
//  (S-1) 2^12 2^(-7(S+2)) < 2^-55 per term, of either sign); with the
//  rounding this gives an error below about K 2^-54 |A_row| |B_col|
//  (max-norms) in the worst case and about sqrt(K) of that for unrelated
//  terms: FP64-class, at the rounding level of an FP64 product of the same
//  length.
//
// Tiles: 128 real rows x 32 columns, K tiles of 32 (64-byte swizzle); a ring
// of 2 stages each holding the 8 digit tiles of A and of B (80 KB); 8
// accumulators of 32 columns, double-buffered (512 TMEM columns) so the
// epilogue of one chunk overlaps the MMAs of the next.  Warps 0-3: epilogue
// (TMEM lane quarters), warp 4: TMA producer, warp 5: MMA issuer.  All waits
// are bounded.
#include <cuda_bf16.h>

#include <cstdint>

#include <atomic>

#include "common.cuh"
#include "tc_ptx.cuh"

namespace ite {
namespace {

using namespace tc;

constexpr int S = 8;
constexpr int BM = 128, BN = 32, BK = 32;
constexpr int KC = 128;                         // real K terms per exact chunk
constexpr int KB_PER_CHUNK = KC / BK;           // 4
constexpr int STAGES = 2;
constexpr int ACC_COLS = S * BN;                // 256 per buffer
static_assert(S == 8, "the epilogue's lo word is scaled by 2^-7(S+1) = 2^-63");
static_assert(128 * (2 * (1 << 13) + (S - 2) * (1 << 12)) < (1 << 24) && 128 * (1 << 14) < (1 << 24),
              "chunk sums must stay exact in fp32");
constexpr int THREADS = 192;
constexpr uint32_t A_SLICE = BM * BK * 2;       // 8 KB
constexpr uint32_t B_SLICE = BN * BK * 2;       // 2 KB
constexpr uint32_t STAGE_BYTES = S * (A_SLICE + B_SLICE);

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ double pow2(int e) {
  // 2^e for -1022 <= e <= 1023 built from the bit pattern
  if (e < -1022) return 0.0;
  if (e > 1023) e = 1023;
  return __longlong_as_double((long long)(e + 1023) << 52);
}

__global__ void __launch_bounds__(THREADS, 1)
k_zgemm_slices(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
               int Mr, int N, int Kr, const int* __restrict__ eA, const int* __restrict__ eB,
               cplx* __restrict__ C, long long ldc, cplx alpha, cplx beta, const cplx* __restrict__ Z,
               cplx gamma, int* err) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t* stage_base = smem;
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* acc_full = empty + STAGES;
  uint64_t* acc_empty = acc_full + 2;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(acc_empty + 2);
  __shared__ int s_fail;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int nkb = Kr / BK;                      // Kr is a multiple of KC
  const int nchunk = Kr / KC;

  if (threadIdx.x == 0) {
    s_fail = 0;
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&acc_full[b], 1);
      mbar_init(&acc_empty[b], 128);
    }
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  if (warp == 4) {
    // ---- TMA producer: k-block kb brings the 7 digit tiles of A and of B
    if (lane == 0) {
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % STAGES;
        if (kb >= STAGES && !mbar_wait(&empty[s], ((kb / STAGES) + 1) & 1)) {
          s_fail = 1;
          break;
        }
        uint8_t* st = stage_base + s * STAGE_BYTES;
        mbar_expect_tx(&full[s], STAGE_BYTES);
        for (int p = 0; p < S; ++p) {
          tma_load_2d(st + p * A_SLICE, &tmA, &full[s], kb * BK, p * Mr + m0);
          tma_load_2d(st + S * A_SLICE + p * B_SLICE, &tmB, &full[s], kb * BK, p * N + n0);
        }
      }
    }
  } else if (warp == 5) {
    // ---- MMA issuer
    if (lane == 0) {
      constexpr uint32_t idesc = bf16_idesc(BN);
      for (int kb = 0; kb < nkb && !*((volatile int*)&s_fail); ++kb) {
        const int chunk = kb / KB_PER_CHUNK, kin = kb % KB_PER_CHUNK;
        const int buf = chunk & 1, use = chunk >> 1;
        if (kin == 0 && chunk >= 2 && !mbar_wait(&acc_empty[buf], (use - 1) & 1)) {
          s_fail = 1;
          break;
        }
        const int s = kb % STAGES;
        if (!mbar_wait(&full[s], (kb / STAGES) & 1)) {
          s_fail = 1;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t st = smem_u32(stage_base + s * STAGE_BYTES);
        for (int d = 2; d <= S + 1; ++d) {
          const uint32_t acc = tmem + buf * ACC_COLS + (d - 2) * BN;
          const int plo = d - S > 1 ? d - S : 1, phi = d - 1 < S ? d - 1 : S;
          for (int p = plo; p <= phi; ++p) {
            const int q = d - p;
            const uint32_t a0 = st + (p - 1) * A_SLICE;
            const uint32_t b0 = st + S * A_SLICE + (q - 1) * B_SLICE;
#pragma unroll
            for (int kk = 0; kk < BK / 16; ++kk) {
              const uint32_t accum = (kin == 0 && p == plo && kk == 0) ? 0u : 1u;
              mma_bf16(acc, kmajor_desc<BK>(a0 + kk * 32), kmajor_desc<BK>(b0 + kk * 32), idesc, accum);
            }
          }
        }
        mma_commit(&empty[s]);
        if (kin == KB_PER_CHUNK - 1) mma_commit(&acc_full[buf]);
      }
    }
  } else {
    // ---- epilogue warps 0-3: exact integer accumulation of the chunks
    long long hi[BN], lo[BN];
#pragma unroll
    for (int j = 0; j < BN; ++j) { hi[j] = 0; lo[j] = 0; }
    const uint32_t lane_base = tmem + ((uint32_t)(warp * 32) << 16);
    bool ok = true;
    for (int c = 0; c < nchunk; ++c) {
      const int buf = c & 1, use = c >> 1;
      ok = __all_sync(0xffffffffu, mbar_wait(&acc_full[buf], use & 1) ? 1 : 0) != 0;
      if (!ok) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll 1
      for (int dd = 0; dd < S; ++dd) {
        float v[32];
        tmem_ld32(lane_base + buf * ACC_COLS + dd * BN, v);
        const int d = dd + 2;
        if (d <= 4) {
          const int sh = 7 * (4 - d);
#pragma unroll
          for (int j = 0; j < BN; ++j) hi[j] += (long long)__float2int_rn(v[j]) << sh;
        } else {
          const int sh = 7 * (S + 1 - d);
#pragma unroll
          for (int j = 0; j < BN; ++j) lo[j] += (long long)__float2int_rn(v[j]) << sh;
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acc_empty[buf]);
    }
    if (!ok) {
      if (lane == 0) atomicExch(err, 1);
    } else {
      // value of real row rr, column n: 2^(eA+eB) (hi 2^-28 + lo 2^-7(S+1))
      const int rr = m0 + warp * 32 + lane;
      const int ea = (rr < Mr) ? eA[rr >> 1] : 0;
      double val[BN];
#pragma unroll
      for (int j = 0; j < BN; ++j) {
        const int n = n0 + j;
        const int eb = (n < N) ? eB[n] : 0;
        const double base = fma((double)hi[j], 0x1p-28, (double)lo[j] * 0x1p-63);
        val[j] = base * pow2(ea + eb);
      }
      // lanes 2i / 2i+1 hold Re / Im of complex row rr/2: the even lane
      // writes columns 0..15, the odd lane columns 16..31
      const bool odd = lane & 1;
      const int r = rr >> 1;
#pragma unroll
      for (int h = 0; h < BN / 2; ++h) {
        const double a = val[h], b = val[h + BN / 2];
        // the even lane needs Im of column h, the odd lane Re of column h+16
        const double recv = __shfl_xor_sync(0xffffffffu, odd ? a : b, 1);
        const double re = odd ? recv : a;
        const double im = odd ? b : recv;
        const int n = n0 + (odd ? h + BN / 2 : h);
        if (rr < Mr && n < N) {
          const long long idx = (long long)r * ldc + n;
          cplx out = cmul(alpha, cmake(re, im));
          if (beta.x != 0.0 || beta.y != 0.0) out = cadd(out, cmul(beta, C[idx]));
          if (Z) out = cadd(out, cmul(gamma, Z[idx]));
          C[idx] = out;
        }
      }
    }
  }
  __syncthreads();
  if (s_fail && threadIdx.x == 0) atomicExch(err, 1);
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
}

// ------------------------------------------------------------------ slicing
// Magnitude bits of a double (the pattern of |x| orders like |x|).
__device__ __forceinline__ unsigned long long mag_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7FFFFFFFFFFFFFFFull;
}

// exponent e with max magnitude < 2^e, from the largest magnitude pattern
__device__ __forceinline__ int scale_exponent(unsigned long long mb) {
  if (mb == 0) return 0;
  const int E = (int)(mb >> 52);
  if (E == 0) return -1022;                     // subnormal range
  return E - 1023 + 1;
}

// T = |x| 2^(7S - e) rounded to the nearest integer (ties up), from the bit
// pattern.  With max|x| < 2^e the row maximum has a shift of 3 and is exact;
// T < 2^(7S) for every entry of the row.
__device__ __forceinline__ unsigned long long fixed_digits(double x, int e) {
  const unsigned long long b = mag_bits(x);
  const int E = (int)(b >> 52);
  unsigned long long mant = b & 0x000FFFFFFFFFFFFFull;
  int Ee = E;
  if (E == 0) Ee = 1; else mant |= 0x0010000000000000ull;
  const int shift = Ee - 1075 + 7 * S - e;      // |x| = mant 2^(Ee-1075)
  if (shift >= 0) return shift >= 64 ? 0ull : mant << shift;
  const int r = -shift;
  return r >= 64 ? 0ull : (mant + (1ull << (r - 1))) >> r;
}

// Balanced base-128 digits of T: T = sum_p g_p 2^(7(S-p)) with the leading
// g_1 in [0, 128] and g_p in [-64, 63] for p >= 2 (a low digit >= 64 becomes
// g - 128 with a carry into the next one), all negated for x < 0.  The low
// digits are then centred on zero, so neither the dropped low-weight
// products nor the rounding give the sums a bias toward zero.
__device__ __forceinline__ void balanced_digits(unsigned long long T, bool neg, int (&g)[S]) {
  int carry = 0;
#pragma unroll
  for (int p = S; p >= 1; --p) {
    int v = (int)((T >> (7 * (S - p))) & 127ull) + carry;
    carry = 0;
    if (p > 1 && v >= 64) { v -= 128; carry = 1; }
    g[p - 1] = neg ? -v : v;
  }
}

__device__ __forceinline__ __nv_bfloat16 bf(int v) { return __float2bfloat16_rn((float)v); }

// A (M x K complex, element (r,k) at A[r sAm + k sAk], conj) -> digits of the
// real rows 2r (Re, -Im interleaved) and 2r+1 (Im, Re), one warp per row r.
// out: S blocks of (2M) x Kp bf16; eA[r] = row exponent.
__global__ void k_slice_rows_A(const cplx* __restrict__ A, long long sAm, long long sAk, bool conj,
                               int M, int K, int Kp, __nv_bfloat16* __restrict__ out, int* eA) {
  const int r = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (r >= M) return;
  const cplx* row = A + (long long)r * sAm;
  unsigned long long mx = 0;
  for (int k = lane; k < K; k += 32) {
    const cplx v = row[(long long)k * sAk];
    const unsigned long long a = mag_bits(v.x), b = mag_bits(v.y);
    mx = a > mx ? a : mx;
    mx = b > mx ? b : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  const int e = scale_exponent(mx);
  if (lane == 0) eA[r] = e;
  const long long Mr = 2LL * M;
  for (int kk = lane; kk < Kp / 2; kk += 32) {
    double re = 0.0, im = 0.0;
    if (kk < K) {
      const cplx v = row[(long long)kk * sAk];
      re = v.x;
      im = conj ? -v.y : v.y;
    }
    int gr[S], gi[S];
    balanced_digits(fixed_digits(re, e), re < 0.0, gr);
    balanced_digits(fixed_digits(im, e), im < 0.0, gi);
#pragma unroll
    for (int p = 1; p <= S; ++p) {
      __nv_bfloat16* blk = out + (long long)(p - 1) * Mr * Kp;
      const __nv_bfloat16 dr = bf(gr[p - 1]), di = bf(gi[p - 1]), dmi = bf(-gi[p - 1]);
      __nv_bfloat162 even, oddv;
      even.x = dr; even.y = dmi;                 // row 2r:   Re, -Im
      oddv.x = di; oddv.y = dr;                  // row 2r+1: Im,  Re
      *reinterpret_cast<__nv_bfloat162*>(blk + (2LL * r) * Kp + 2 * kk) = even;
      *reinterpret_cast<__nv_bfloat162*>(blk + (2LL * r + 1) * Kp + 2 * kk) = oddv;
    }
  }
}

// B (K x N complex, element (k,n) at B[k sBk + n sBn], conj) -> digits of the
// K-major rows n: (Re, Im) interleaved along K.  One warp per column n.
// out: S blocks of N x Kp bf16; eB[n] = column exponent.
__global__ void k_slice_cols_B(const cplx* __restrict__ B, long long sBk, long long sBn, bool conj,
                               int K, int N, int Kp, __nv_bfloat16* __restrict__ out, int* eB) {
  const int n = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (n >= N) return;
  const cplx* col = B + (long long)n * sBn;
  unsigned long long mx = 0;
  for (int k = lane; k < K; k += 32) {
    const cplx v = col[(long long)k * sBk];
    const unsigned long long a = mag_bits(v.x), b = mag_bits(v.y);
    mx = a > mx ? a : mx;
    mx = b > mx ? b : mx;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long t = __shfl_xor_sync(0xffffffffu, mx, o);
    mx = t > mx ? t : mx;
  }
  const int e = scale_exponent(mx);
  if (lane == 0) eB[n] = e;
  for (int kk = lane; kk < Kp / 2; kk += 32) {
    double re = 0.0, im = 0.0;
    if (kk < K) {
      const cplx v = col[(long long)kk * sBk];
      re = v.x;
      im = conj ? -v.y : v.y;
    }
    int gr[S], gi[S];
    balanced_digits(fixed_digits(re, e), re < 0.0, gr);
    balanced_digits(fixed_digits(im, e), im < 0.0, gi);
#pragma unroll
    for (int p = 1; p <= S; ++p) {
      __nv_bfloat162 pr;
      pr.x = bf(gr[p - 1]);
      pr.y = bf(gi[p - 1]);
      *reinterpret_cast<__nv_bfloat162*>(out + ((long long)(p - 1) * N + n) * Kp + 2 * kk) = pr;
    }
  }
}

}  // namespace

// tensor map over `rows` x `cols` bf16 (row stride cols), box rows x 32, 64-byte swizzle
cudaError_t make_digit_map(CUtensorMap* map, const void* base, long long rows, long long cols,
                           int box_rows);

size_t zgemm_emu_scratch_bytes(int M, int N, int K) {
  const long long Kp = ((2LL * K + KC - 1) / KC) * KC;
  return (size_t)S * (2LL * M + N) * Kp * 2 + (size_t)(M + N) * sizeof(int) + 1024;
}

cudaError_t zgemm_emu(const GemmArgs& g, void* scratch, size_t scratch_bytes, int* err,
                      cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (scratch_bytes < zgemm_emu_scratch_bytes(g.M, g.N, g.K)) return cudaErrorInvalidValue;
  const long long Kp = ((2LL * (g.K > 0 ? g.K : 1) + KC - 1) / KC) * KC;
  const long long Mr = 2LL * g.M;
  if (Mr > 65535LL * BM || (long long)S * Mr > (1LL << 31) || (long long)S * g.N > (1LL << 31))
    return cudaErrorInvalidValue;
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(scratch);
  __nv_bfloat16* Bs = As + (size_t)S * Mr * Kp;
  int* eA = reinterpret_cast<int*>(Bs + (size_t)S * g.N * Kp);
  int* eB = eA + g.M;
  // the shared-memory attribute is per device; setting it twice from two
  // threads is harmless
  static std::atomic<unsigned long long> attr_done{0};
  const size_t smem = 1024 + STAGES * STAGE_BYTES + (2 * STAGES + 4) * 8 + 16;
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (!(attr_done.load() & bit)) {
      e = cudaFuncSetAttribute(k_zgemm_slices, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      attr_done.fetch_or(bit);
    }
  }
  for (int b = 0; b < g.batch; ++b) {
    const cplx* A = g.A + (long long)b * g.sAb;
    const cplx* B = g.B + (long long)b * g.sBb;
    cplx* Cb = g.C + (long long)b * g.sCb;
    const cplx* Zb = g.Z ? g.Z + (long long)b * g.sCb : nullptr;
    if (b == 0 || g.sAb != 0) {
      count_launches(1);
      k_slice_rows_A<<<(g.M + 7) / 8, 256, 0, st>>>(A, g.sAm, g.sAk, g.conjA, g.M, g.K, (int)Kp, As, eA);
    }
    if (b == 0 || g.sBb != 0) {
      count_launches(1);
      k_slice_cols_B<<<(g.N + 7) / 8, 256, 0, st>>>(B, g.sBk, g.sBn, g.conjB, g.K, g.N, (int)Kp, Bs, eB);
    }
    CUtensorMap ma, mb;
    cudaError_t e = make_digit_map(&ma, As, (long long)S * Mr, Kp, BM);
    if (e != cudaSuccess) return e;
    e = make_digit_map(&mb, Bs, (long long)S * g.N, Kp, BN);
    if (e != cudaSuccess) return e;
    dim3 grid((g.N + BN - 1) / BN, (unsigned)((Mr + BM - 1) / BM));
    count_launches(1);
    k_zgemm_slices<<<grid, THREADS, smem, st>>>(ma, mb, (int)Mr, g.N, (int)Kp, eA, eB, Cb, g.ldc,
                                                g.alpha, g.beta, Zb, g.gamma, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace ite
