// Krylov vector kernels (block dot, block axpy, norms, scaling), the MPO
// mixing kernel, small trace/site-operator kernels and the device-side GMRES
// control (Givens QR of the Hessenberg matrix) of the local solves.
//
// All reductions are two-stage with a grid size fixed by the vector length,
// and the second stage sums the partials in block order, so results are
// bitwise reproducible run to run.
#include "common.cuh"

namespace ite {
namespace {

constexpr int VT = 256;          // threads per block of the vector kernels
constexpr int MAXV = 32;         // largest Krylov basis handled

int grid_for(long long n) {
  long long g = (n + VT - 1) / VT;
  if (g > 608) g = 608;          // 4 blocks per SM on 152 SMs
  if (g < 1) g = 1;
  return (int)g;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// block-wide sum of one double; result valid in thread 0
__device__ double block_sum(double v, double* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  v = warp_sum(v);
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  double r = 0.0;
  if (wid == 0) {
    r = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0.0;
    r = warp_sum(r);
  }
  __syncthreads();
  return r;
}

__global__ void k_copy(cplx* y, const cplx* x, long long n) {
  for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < n; e += (long long)gridDim.x * VT)
    y[e] = x[e];
}

__global__ void k_zero(cplx* y, long long n) {
  for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < n; e += (long long)gridDim.x * VT)
    y[e] = cmake(0.0, 0.0);
}

__global__ void k_axpby(cplx* y, const cplx* x, cplx a, cplx b, long long n) {
  for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < n; e += (long long)gridDim.x * VT)
    y[e] = cadd(cmul(a, x[e]), cmul(b, y[e]));
}

// partial[blk*nv + i] = block's share of sum_e conj(V_i[e]) w[e]
__global__ void k_block_dot(const cplx* V, long long ldv, int nv, const cplx* w, long long n,
                            cplx* partial, const int* active) {
  if (active && *active == 0) return;
  __shared__ double sh[32];
  for (int i0 = 0; i0 < nv; i0 += 4) {
    cplx acc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) acc[u] = cmake(0.0, 0.0);
    for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < n; e += (long long)gridDim.x * VT) {
      const cplx we = w[e];
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (i0 + u < nv) cfma_conj(acc[u], V[(long long)(i0 + u) * ldv + e], we);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      if (i0 + u >= nv) break;
      const double re = block_sum(acc[u].x, sh);
      const double im = block_sum(acc[u].y, sh);
      if (threadIdx.x == 0) partial[(long long)blockIdx.x * nv + i0 + u] = cmake(re, im);
    }
  }
}

// out[i] = sum over the nblk partial rows of column i: warp i takes column
// i, its lanes sum rows lane, lane + 32, ... in order and a fixed shuffle tree
// adds the lanes, so the order of the sum is fixed and each lane issues its
// loads together (a single thread summing the rows one by one waited on each
// L2 load in turn, tens of microseconds per call).
__global__ void k_reduce_cplx(const cplx* partial, int nblk, int nv, cplx* out, const int* active) {
  if (active && *active == 0) return;
  const int i = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (i >= nv) return;
  double sr = 0.0, si = 0.0;
  for (int b = lane; b < nblk; b += 32) {
    const cplx v = partial[(long long)b * nv + i];
    sr += v.x;
    si += v.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sr += __shfl_xor_sync(0xffffffffu, sr, o);
    si += __shfl_xor_sync(0xffffffffu, si, o);
  }
  if (lane == 0) out[i] = cmake(sr, si);
}

__global__ void k_block_axpy(const cplx* V, long long ldv, int nv, const int* nv_dev,
                             const cplx* h, double sign, cplx* w, long long n, const int* active) {
  if (active && *active == 0) return;
  __shared__ cplx hs[MAXV];
  int m = nv;
  if (nv_dev && *nv_dev < m) m = *nv_dev;
  if (threadIdx.x < m) hs[threadIdx.x] = cscale(h[threadIdx.x], sign);
  __syncthreads();
  for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < n; e += (long long)gridDim.x * VT) {
    cplx acc = w[e];
    for (int i = 0; i < m; ++i) cfma(acc, hs[i], V[(long long)i * ldv + e]);
    w[e] = acc;
  }
}

__global__ void k_norm2_partial(const cplx* x, long long n, double* partial, const int* active) {
  if (active && *active == 0) return;
  __shared__ double sh[32];
  double acc = 0.0;
  for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < n; e += (long long)gridDim.x * VT) {
    const cplx v = x[e];
    acc = fma(v.x, v.x, acc);
    acc = fma(v.y, v.y, acc);
  }
  const double s = block_sum(acc, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// *out = sum of the nblk partials, by one warp in the fixed order of
// k_reduce_cplx
__global__ void k_reduce_real(const double* partial, int nblk, double* out, const int* active) {
  if (active && *active == 0) return;
  const int lane = threadIdx.x & 31;
  if (threadIdx.x >= 32) return;
  double s = 0.0;
  for (int b = lane; b < nblk; b += 32) s += partial[b];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) *out = s;
}

__global__ void k_scale_dev(cplx* y, const double* scale, long long n, const int* active) {
  if (active && *active == 0) return;
  const double s = *scale;
  for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < n; e += (long long)gridDim.x * VT)
    y[e] = cscale(y[e], s);
}

// L is D x m x n, R is D x n x m; sum_{w,b,c} L[w][b][c] R[w][c][b]
__global__ void k_env_trace(const cplx* L, const cplx* R, int D, int m, int n, cplx* partial) {
  __shared__ double sh[32];
  const long long tot = (long long)D * m * n;
  cplx acc = cmake(0.0, 0.0);
  for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < tot; e += (long long)gridDim.x * VT) {
    const long long w = e / ((long long)m * n);
    const long long rem = e - w * (long long)m * n;
    const long long b = rem / n, c = rem - b * n;
    cfma(acc, L[e], R[(w * n + c) * m + b]);
  }
  const double re = block_sum(acc.x, sh);
  const double im = block_sum(acc.y, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = cmake(re, im);
}

__global__ void k_site_op(const cplx* O, const cplx* K, cplx* Kout, int chl, int d, int chr) {
  const long long tot = (long long)chl * d * chr;
  for (long long e = blockIdx.x * (long long)VT + threadIdx.x; e < tot; e += (long long)gridDim.x * VT) {
    const long long a = e / ((long long)d * chr);
    const long long rem = e - a * d * chr;
    const int sp = (int)(rem / chr);
    const long long b = rem - (long long)sp * chr;
    cplx acc = cmake(0.0, 0.0);
    for (int s = 0; s < d; ++s) cfma(acc, O[sp * d + s], K[(a * d + s) * chr + b]);
    Kout[e] = acc;
  }
}

// ------------------------------------------------------------------ mixing
constexpr int MIX_MAX = 128;   // largest row/column count of a mixing matrix

__global__ void k_mix(MixPlan pl, MixStrides s, int P, int Q, const cplx* in, long long iP,
                      long long iQ, cplx* out, long long oP, long long oQ) {
  __shared__ long long ioff[MIX_MAX], ooff[MIX_MAX];
  for (int j = threadIdx.x; j < pl.ncols; j += blockDim.x) {
    const int j2 = j % pl.cdim[2], j1 = (j / pl.cdim[2]) % pl.cdim[1], j0 = j / (pl.cdim[2] * pl.cdim[1]);
    ioff[j] = j0 * s.ic[0] + j1 * s.ic[1] + j2 * s.ic[2];
  }
  for (int k = threadIdx.x; k < pl.nrows; k += blockDim.x) {
    const int k2 = k % pl.rdim[2], k1 = (k / pl.rdim[2]) % pl.rdim[1], k0 = k / (pl.rdim[2] * pl.rdim[1]);
    ooff[k] = k0 * s.oc[0] + k1 * s.oc[1] + k2 * s.oc[2];
  }
  __syncthreads();
  const long long tot = (long long)P * Q;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long p = e / Q, q = e - p * Q;
    const cplx* ib = in + p * iP + q * iQ;
    cplx* ob = out + p * oP + q * oQ;
    for (int k = 0; k < pl.nrows; ++k) {
      cplx acc = cmake(0.0, 0.0);
      for (int t = __ldg(pl.row_ptr + k); t < __ldg(pl.row_ptr + k + 1); ++t)
        cfma(acc, pl.val[t], ib[ioff[__ldg(pl.col + t)]]);
      ob[ooff[k]] = acc;
    }
  }
}

// ------------------------------------------------------------------ GMRES control
__device__ __forceinline__ cplx& Hc(GmresState* s, int i, int j) { return s->H[j * (32 + 1) + i]; }

__global__ void k_gmres_start(GmresState* s, const double* r0n2, const double* bn2) {
  const double beta = sqrt(*r0n2);
  s->beta = beta;
  s->bnorm = sqrt(*bn2);
  s->steps = 0;
  s->breakdown = 0;
  s->res = beta;
  for (int i = 0; i < 33; ++i) s->g[i] = cmake(0.0, 0.0);
  for (int i = 0; i < 32; ++i) s->y[i] = cmake(0.0, 0.0);
  for (int i = 0; i < 33 * 32; ++i) s->H[i] = cmake(0.0, 0.0);
  if (beta > 0.0 && isfinite(beta)) {
    s->active = 1;
    s->inv_h = 1.0 / beta;
    s->g[0] = cmake(beta, 0.0);
  } else {
    s->active = 0;
    s->inv_h = 0.0;
  }
}

__global__ void k_gmres_collect(GmresState* s, int j, const cplx* h1, const cplx* h2) {
  if (!s->active) return;
  const int i = threadIdx.x;
  if (i <= j) Hc(s, i, j) = cadd(h1[i], h2[i]);
}

__global__ void k_gmres_step(GmresState* s, int j, int m, double brel, double ltol) {
  if (!s->active) return;
  const double hj1 = sqrt(s->wnorm2);
  // |A v_j|^2 = sum_i |h_ij|^2 + h_{j+1,j}^2 (Arnoldi relation), read before
  // the rotations touch column j; a happy breakdown is a new direction that
  // is negligible against it
  double col2 = s->wnorm2;
  for (int i = 0; i <= j; ++i) {
    const cplx h = Hc(s, i, j);
    col2 = fma(h.x, h.x, fma(h.y, h.y, col2));
  }
  // earlier rotations on column j
  for (int i = 0; i < j; ++i) {
    const cplx a = Hc(s, i, j), b = Hc(s, i + 1, j);
    const cplx c = s->cs[i], sn = s->sn[i];
    Hc(s, i, j) = cadd(cmul(c, a), cmul(sn, b));
    Hc(s, i + 1, j) = csub(cmul(c, b), cmul(cconj(sn), a));
  }
  // new rotation zeroing h_{j+1,j}
  const cplx a = Hc(s, j, j);
  const double an = hypot(a.x, a.y);
  const double r = hypot(an, hj1);
  cplx c, sn;
  if (r == 0.0) {
    c = cmake(1.0, 0.0); sn = cmake(0.0, 0.0);
  } else if (an == 0.0) {
    c = cmake(0.0, 0.0); sn = cmake(1.0, 0.0);
  } else {
    c = cmake(an / r, 0.0);
    sn = cscale(a, hj1 / (an * r));
  }
  s->cs[j] = c;
  s->sn[j] = sn;
  Hc(s, j, j) = (an == 0.0) ? cmake(hj1, 0.0) : cscale(a, r / an);
  Hc(s, j + 1, j) = cmake(0.0, 0.0);
  const cplx gj = s->g[j];
  s->g[j] = cmul(c, gj);
  s->g[j + 1] = cscale(cmul(cconj(sn), gj), -1.0);
  s->res = hypot(s->g[j + 1].x, s->g[j + 1].y);
  s->steps = j + 1;
  if (!(hj1 > brel * sqrt(col2)) || !isfinite(hj1)) {
    s->breakdown = 1;
    s->active = 0;
  } else if (ltol > 0.0 && s->res <= ltol * s->bnorm) {
    s->active = 0;
  } else if (j + 1 >= m) {
    s->active = 0;
  } else {
    s->inv_h = 1.0 / hj1;
  }
}

__global__ void k_gmres_finish(GmresState* s) {
  const int k = s->steps;
  for (int i = k - 1; i >= 0; --i) {
    cplx acc = s->g[i];
    for (int l = i + 1; l < k; ++l) acc = csub(acc, cmul(Hc(s, i, l), s->y[l]));
    const cplx d = Hc(s, i, i);
    const double dn = d.x * d.x + d.y * d.y;
    s->y[i] = (dn > 0.0) ? cscale(cmul(acc, cconj(d)), 1.0 / dn) : cmake(0.0, 0.0);
  }
}

}  // namespace

cudaError_t vec_copy(cplx* y, const cplx* x, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launches(1);
  k_copy<<<grid_for(n), VT, 0, st>>>(y, x, n);
  return cudaGetLastError();
}
cudaError_t vec_zero(cplx* y, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launches(1);
  k_zero<<<grid_for(n), VT, 0, st>>>(y, n);
  return cudaGetLastError();
}
cudaError_t vec_axpby(cplx* y, const cplx* x, cplx a, cplx b, long long n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launches(1);
  k_axpby<<<grid_for(n), VT, 0, st>>>(y, x, a, b, n);
  return cudaGetLastError();
}
cudaError_t vec_block_dot(const cplx* V, long long ldv, int nv, const cplx* w, long long n,
                          cplx* out, cplx* partial, const int* active, cudaStream_t st) {
  if (nv <= 0) return cudaSuccess;
  if (nv > MAXV) return cudaErrorInvalidValue;
  const int g = grid_for(n);
  count_launches(1);
  k_block_dot<<<g, VT, 0, st>>>(V, ldv, nv, w, n, partial, active);
  count_launches(1);
  k_reduce_cplx<<<1, 32 * nv, 0, st>>>(partial, g, nv, out, active);
  return cudaGetLastError();
}
cudaError_t vec_block_axpy(const cplx* V, long long ldv, int nv, const int* nv_dev,
                           const cplx* h, double sign, cplx* w, long long n, const int* active,
                           cudaStream_t st) {
  if (nv <= 0 || n <= 0) return cudaSuccess;
  if (nv > MAXV) return cudaErrorInvalidValue;
  count_launches(1);
  k_block_axpy<<<grid_for(n), VT, 0, st>>>(V, ldv, nv, nv_dev, h, sign, w, n, active);
  return cudaGetLastError();
}
cudaError_t vec_norm2(const cplx* x, long long n, double* out, double* partial,
                      const int* active, cudaStream_t st) {
  const int g = grid_for(n);
  count_launches(1);
  k_norm2_partial<<<g, VT, 0, st>>>(x, n, partial, active);
  count_launches(1);
  k_reduce_real<<<1, 32, 0, st>>>(partial, g, out, active);
  return cudaGetLastError();
}
namespace {
__global__ void k_scale_scalar(double* v, double s) {
  if (threadIdx.x == 0) *v *= s;
}
}  // namespace

cudaError_t scaled_norm2(const cplx* x, long long n, double scale, double* out, double* partial,
                         cudaStream_t st) {
  cudaError_t e = vec_norm2(x, n, out, partial, nullptr, st);
  if (e != cudaSuccess) return e;
  count_launches(1);
  k_scale_scalar<<<1, 32, 0, st>>>(out, scale);
  return cudaGetLastError();
}

cudaError_t vec_scale_dev(cplx* y, const double* scale, long long n, const int* active,
                          cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  count_launches(1);
  k_scale_dev<<<grid_for(n), VT, 0, st>>>(y, scale, n, active);
  return cudaGetLastError();
}
cudaError_t env_trace(const cplx* L, const cplx* R, int D, int m, int n, cplx* out,
                      cplx* partial, cudaStream_t st) {
  const long long tot = (long long)D * m * n;
  const int g = grid_for(tot);
  count_launches(1);
  k_env_trace<<<g, VT, 0, st>>>(L, R, D, m, n, partial);
  count_launches(1);
  k_reduce_cplx<<<1, 32, 0, st>>>(partial, g, 1, out, nullptr);
  return cudaGetLastError();
}
cudaError_t apply_site_op(const cplx* O, const cplx* K, cplx* Kout, int chl, int d, int chr,
                          cudaStream_t st) {
  const long long tot = (long long)chl * d * chr;
  if (tot <= 0) return cudaSuccess;
  count_launches(1);
  k_site_op<<<grid_for(tot), VT, 0, st>>>(O, K, Kout, chl, d, chr);
  return cudaGetLastError();
}
cudaError_t mix_apply(const MixPlan& plan, const MixStrides& s, int P, int Q, const cplx* in,
                      long long iP, long long iQ, cplx* out, long long oP, long long oQ,
                      cudaStream_t st) {
  if (plan.nrows > MIX_MAX || plan.ncols > MIX_MAX) return cudaErrorInvalidValue;
  const long long tot = (long long)P * Q;
  if (tot <= 0) return cudaSuccess;
  long long g = (tot + 127) / 128;
  if (g > 1216) g = 1216;
  count_launches(1);
  k_mix<<<(int)g, 128, 0, st>>>(plan, s, P, Q, in, iP, iQ, out, oP, oQ);
  return cudaGetLastError();
}
cudaError_t gmres_start(GmresState* s, const double* r0norm2, const double* bnorm2,
                        cudaStream_t st) {
  count_launches(1);
  k_gmres_start<<<1, 1, 0, st>>>(s, r0norm2, bnorm2);
  return cudaGetLastError();
}
cudaError_t gmres_collect(GmresState* s, int j, int m, const cplx* h1, const cplx* h2,
                          cudaStream_t st) {
  (void)m;
  count_launches(1);
  k_gmres_collect<<<1, 32, 0, st>>>(s, j, h1, h2);
  return cudaGetLastError();
}
cudaError_t gmres_step(GmresState* s, int j, int m, double breakdown_rel, double local_tol,
                       cudaStream_t st) {
  count_launches(1);
  k_gmres_step<<<1, 1, 0, st>>>(s, j, m, breakdown_rel, local_tol);
  return cudaGetLastError();
}
cudaError_t gmres_finish(GmresState* s, cudaStream_t st) {
  count_launches(1);
  k_gmres_finish<<<1, 1, 0, st>>>(s);
  return cudaGetLastError();
}

}  // namespace ite
