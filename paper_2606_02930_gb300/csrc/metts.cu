// METTS collapse: one site of the sequential Born-rule draw from an MPS in
// right-canonical form (orthogonality centre on the first site).  Given the
// normalised row vector v of the earlier choices, the site's candidate rows
// are M_s = <b_s| v A_i (s < d, b_s the columns of the collapse basis, or
// the computational basis), their weights w_s = |M_s|^2 give the conditional
// probabilities p_s = w_s / sum w, the choice is the smallest s whose
// cumulative probability exceeds the uniform u (the last s of nonzero weight
// when rounding leaves the total at or below u), and the next vector is
// M_s / |M_s|.
#include "common.cuh"

namespace ite {
namespace {

constexpr int ST = 256;

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// one block; dynamic shared memory holds M (d x chr complex)
__global__ void __launch_bounds__(ST)
k_sample_site(const cplx* A, int chl, int d, int chr, const cplx* v, double u, const cplx* basis,
              cplx* v_out, int* choice, double* prob) {
  extern __shared__ cplx M[];
  __shared__ double red[ST / 32][4];
  __shared__ double sel[2];
  const int tid = threadIdx.x;
  // M[s][b] = sum_a v[a] A[a][s][b]
  for (int e = tid; e < d * chr; e += ST) {
    const int s = e / chr, b = e - s * chr;
    cplx acc = cmake(0.0, 0.0);
    for (int a = 0; a < chl; ++a) cfma(acc, v[a], A[((long long)a * d + s) * chr + b]);
    M[e] = acc;
  }
  __syncthreads();
  if (basis) {
    // <b_s| components: M'[s][b] = sum_t conj(B[t][s]) M[t][b]; at most 4 per column
    for (int b = tid; b < chr; b += ST) {
      cplx col[4];
      for (int t = 0; t < d; ++t) col[t] = M[t * chr + b];
      for (int s = 0; s < d; ++s) {
        cplx acc = cmake(0.0, 0.0);
        for (int t = 0; t < d; ++t) cfma(acc, cconj(basis[t * d + s]), col[t]);
        M[s * chr + b] = acc;
      }
    }
    __syncthreads();
  }
  double w[4] = {0.0, 0.0, 0.0, 0.0};
  for (int s = 0; s < d; ++s)
    for (int b = tid; b < chr; b += ST) {
      const cplx m = M[s * chr + b];
      w[s] = fma(m.x, m.x, fma(m.y, m.y, w[s]));
    }
  for (int s = 0; s < d; ++s) {
    w[s] = warp_sum_d(w[s]);
    if ((tid & 31) == 0) red[tid >> 5][s] = w[s];
  }
  __syncthreads();
  if (tid == 0) {
    double ws[4], tot = 0.0;
    for (int s = 0; s < d; ++s) {
      ws[s] = 0.0;
      for (int k = 0; k < ST / 32; ++k) ws[s] += red[k][s];
      tot += ws[s];
    }
    int pick = -1, last = d - 1;
    double cum = 0.0;
    for (int s = 0; s < d; ++s) {
      if (ws[s] > 0.0) last = s;
      cum += ws[s] / tot;
      if (pick < 0 && cum > u) pick = s;
    }
    if (pick < 0) pick = last;
    *choice = pick;
    *prob *= ws[pick] / tot;
    sel[0] = (double)pick;
    sel[1] = ws[pick] > 0.0 ? 1.0 / sqrt(ws[pick]) : 0.0;
  }
  __syncthreads();
  const int pick = (int)sel[0];
  const double inv = sel[1];
  for (int b = tid; b < chr; b += ST) v_out[b] = cscale(M[pick * chr + b], inv);
}

}  // namespace

cudaError_t sample_site(const cplx* A, int chl, int d, int chr, const cplx* v, double u,
                        const cplx* basis, cplx* v_out, int* choice, double* prob, cudaStream_t st) {
  if (d < 1 || d > 4 || chl < 1 || chr < 1) return cudaErrorInvalidValue;
  const size_t smem = sizeof(cplx) * (size_t)d * chr;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_sample_site, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(1);
  k_sample_site<<<1, ST, smem, st>>>(A, chl, d, chr, v, u, basis, v_out, choice, prob);
  return cudaGetLastError();
}

}  // namespace ite
