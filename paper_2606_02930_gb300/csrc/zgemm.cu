// Batched complex FP64 GEMM with arbitrary element strides, used by every
// tensor contraction of the FP64 path (two-site H_eff, environments, local
// right-hand sides, two-site merges).
//
// On GB300 the FP64 pipe issues about two DFMA per clock per SM (measured
// 1.19 TFLOP/s for the whole GPU), so this kernel is bound by that pipe; the
// tile shape only has to keep the pipe busy, and shared-memory and DRAM
// traffic are far below their limits.
#include "common.cuh"

namespace ite {
namespace {

constexpr int BM = 32, BN = 32, BK = 8, THREADS = 256;

template <bool CONJ_A, bool CONJ_B>
__global__ void __launch_bounds__(THREADS)
zgemm_kernel(GemmArgs g, bool a_kfast, bool b_nfast) {
  __shared__ cplx As[BK][BM + 1];
  __shared__ cplx Bs[BK][BN + 1];
  const int t = threadIdx.x;
  const int tx = t % 16, ty = t / 16;
  const int row0 = blockIdx.y * BM, col0 = blockIdx.x * BN;
  const int b = blockIdx.z;
  const cplx* A = g.A + (long long)b * g.sAb;
  const cplx* B = g.B + (long long)b * g.sBb;

  // load mapping: A tile is BM x BK (256 elements), B tile is BK x BN
  const int ai = a_kfast ? t / BK : t % BM;
  const int ak = a_kfast ? t % BK : t / BM;
  const int bk = b_nfast ? t / BN : t % BK;
  const int bj = b_nfast ? t % BN : t / BK;

  cplx acc[2][2];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j) acc[i][j] = cmake(0.0, 0.0);

  for (int k0 = 0; k0 < g.K; k0 += BK) {
    {
      const int gi = row0 + ai, gk = k0 + ak;
      cplx v = cmake(0.0, 0.0);
      if (gi < g.M && gk < g.K) {
        v = A[(long long)gi * g.sAm + (long long)gk * g.sAk];
        if (CONJ_A) v = cconj(v);
      }
      As[ak][ai] = v;
    }
    {
      const int gk = k0 + bk, gj = col0 + bj;
      cplx v = cmake(0.0, 0.0);
      if (gk < g.K && gj < g.N) {
        v = B[(long long)gk * g.sBk + (long long)gj * g.sBn];
        if (CONJ_B) v = cconj(v);
      }
      Bs[bk][bj] = v;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < BK; ++k) {
      const cplx a0 = As[k][ty * 2], a1 = As[k][ty * 2 + 1];
      const cplx b0 = Bs[k][tx * 2], b1 = Bs[k][tx * 2 + 1];
      cfma(acc[0][0], a0, b0);
      cfma(acc[0][1], a0, b1);
      cfma(acc[1][0], a1, b0);
      cfma(acc[1][1], a1, b1);
    }
    __syncthreads();
  }

  cplx* C = g.C + (long long)b * g.sCb;
  const cplx* Z = g.Z ? g.Z + (long long)b * g.sCb : nullptr;
  const bool use_beta = (g.beta.x != 0.0 || g.beta.y != 0.0);
#pragma unroll
  for (int i = 0; i < 2; ++i) {
    const int r = row0 + ty * 2 + i;
    if (r >= g.M) continue;
#pragma unroll
    for (int j = 0; j < 2; ++j) {
      const int c = col0 + tx * 2 + j;
      if (c >= g.N) continue;
      const long long idx = (long long)r * g.ldc + c;
      cplx v = cmul(g.alpha, acc[i][j]);
      if (use_beta) v = cadd(v, cmul(g.beta, C[idx]));
      if (Z) v = cadd(v, cmul(g.gamma, Z[idx]));
      C[idx] = v;
    }
  }
}

}  // namespace

cudaError_t zgemm(const GemmArgs& g, cudaStream_t st) {
  if (g.M <= 0 || g.N <= 0 || g.batch <= 0) return cudaSuccess;
  if (g.batch > 65535 || (g.M + BM - 1) / BM > 65535) return cudaErrorInvalidValue;
  dim3 grid((g.N + BN - 1) / BN, (g.M + BM - 1) / BM, g.batch);
  const bool a_kfast = (g.sAk == 1);
  const bool b_nfast = (g.sBn == 1) || (g.sBk != 1);
  count_launches(1);
  if (g.conjA && g.conjB)
    zgemm_kernel<true, true><<<grid, THREADS, 0, st>>>(g, a_kfast, b_nfast);
  else if (g.conjA)
    zgemm_kernel<true, false><<<grid, THREADS, 0, st>>>(g, a_kfast, b_nfast);
  else if (g.conjB)
    zgemm_kernel<false, true><<<grid, THREADS, 0, st>>>(g, a_kfast, b_nfast);
  else
    zgemm_kernel<false, false><<<grid, THREADS, 0, st>>>(g, a_kfast, b_nfast);
  return cudaGetLastError();
}

}  // namespace ite
