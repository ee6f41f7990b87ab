// Kernels of the mixed-precision truncated SVD of the tensor-core mode (the
// engine sequences them with FP64-class GEMMs and the FP64 Jacobi kernel):
// fp32 copies of the split matrix, the fp32 rotations turned into an FP64
// matrix of vectors, and the gathers that pick the kept vectors.
#include "common.cuh"

namespace ite {
namespace {

constexpr int T = 256;

int blocks_for(long long n) {
  long long g = (n + T - 1) / T;
  if (g > 1216) g = 1216;
  if (g < 1) g = 1;
  return (int)g;
}

// out (p x q fp32) = X (m x n) or X^H, cast to fp32
__global__ void k_to_f32(const cplx* X, int m, int n, bool ct, float2* out) {
  const long long tot = (long long)m * n;
  for (long long e = blockIdx.x * (long long)T + threadIdx.x; e < tot; e += (long long)gridDim.x * T) {
    if (!ct) {
      out[e] = make_float2((float)X[e].x, (float)X[e].y);
    } else {
      // out is n x m: out[j][i] = conj(X[i][j]); e indexes out
      const long long j = e / m, i = e - j * m;
      const cplx v = X[i * n + j];
      out[e] = make_float2((float)v.x, (float)-v.y);
    }
  }
}

// W (p x p complex128) = Q32^H
__global__ void k_q32_to_w(const float2* Q, int p, cplx* W) {
  const long long tot = (long long)p * p;
  for (long long e = blockIdx.x * (long long)T + threadIdx.x; e < tot; e += (long long)gridDim.x * T) {
    const long long i = e / p, j = e - i * p;
    const float2 v = Q[j * p + i];
    W[e] = cmake((double)v.x, -(double)v.y);
  }
}

// isometry columns: out = W[:, perm[0..r)] as (p x r), or its conjugate
// transpose (r x p) when ct
__global__ void k_gather_cols(const cplx* W, const int* perm, int p, int r, bool ct, cplx* out) {
  const long long tot = (long long)p * r;
  for (long long e = blockIdx.x * (long long)T + threadIdx.x; e < tot; e += (long long)gridDim.x * T) {
    if (!ct) {
      const long long i = e / r;
      const int k = (int)(e - i * r);
      out[e] = W[i * p + perm[k]];
    } else {
      const int k = (int)(e / p);
      const long long j = e - (long long)k * p;
      out[e] = cconj(W[j * p + perm[k]]);
    }
  }
}

// rows of B picked by perm: out[k][j] = B[perm[k]][j] (r x q), or, when ct,
// out[i][k] = conj(B[perm[k]][i]) (q x r)
__global__ void k_gather_rows(const cplx* B, const int* perm, int q, int r, bool ct, cplx* out) {
  const long long tot = (long long)q * r;
  for (long long e = blockIdx.x * (long long)T + threadIdx.x; e < tot; e += (long long)gridDim.x * T) {
    if (!ct) {
      const int k = (int)(e / q);
      const long long j = e - (long long)k * q;
      out[e] = B[(long long)perm[k] * q + j];
    } else {
      const long long i = e / r;
      const int k = (int)(e - i * r);
      out[e] = cconj(B[(long long)perm[k] * q + i]);
    }
  }
}

}  // namespace

cudaError_t mixsvd_gather_rows(const cplx* B, const int* perm, int q, int r, bool ct, cplx* out,
                               cudaStream_t st) {
  count_launches(1);
  k_gather_rows<<<blocks_for((long long)q * r), T, 0, st>>>(B, perm, q, r, ct, out);
  return cudaGetLastError();
}

cudaError_t mixsvd_to_f32(const cplx* X, int m, int n, bool ct, float2* out, cudaStream_t st) {
  count_launches(1);
  k_to_f32<<<blocks_for((long long)m * n), T, 0, st>>>(X, m, n, ct, out);
  return cudaGetLastError();
}

cudaError_t mixsvd_q32_to_w(const float2* Q, int p, cplx* W, cudaStream_t st) {
  count_launches(1);
  k_q32_to_w<<<blocks_for((long long)p * p), T, 0, st>>>(Q, p, W);
  return cudaGetLastError();
}

cudaError_t mixsvd_gather(const cplx* W, const int* perm, int p, int r, bool ct, cplx* out,
                          cudaStream_t st) {
  count_launches(1);
  k_gather_cols<<<blocks_for((long long)p * r), T, 0, st>>>(W, perm, p, r, ct, out);
  return cudaGetLastError();
}

}  // namespace ite
