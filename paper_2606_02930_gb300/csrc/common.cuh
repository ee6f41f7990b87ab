// Shared device/host helpers of the CUDA library: complex arithmetic on
// double2 (interleaved re, im), launch checks and the internal API between the
// translation units.
#pragma once

#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>

typedef double2 cplx;

__host__ __device__ __forceinline__ cplx cmake(double r, double i) { return make_double2(r, i); }
__host__ __device__ __forceinline__ cplx cadd(cplx a, cplx b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ cplx csub(cplx a, cplx b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ cplx cmul(cplx a, cplx b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ cplx cconj(cplx a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ cplx cscale(cplx a, double s) { return make_double2(a.x * s, a.y * s); }
// acc += a * b
__host__ __device__ __forceinline__ void cfma(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(-a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(a.y, b.x, acc.y);
}
// acc += conj(a) * b
__host__ __device__ __forceinline__ void cfma_conj(cplx& acc, cplx a, cplx b) {
  acc.x = fma(a.x, b.x, acc.x);
  acc.x = fma(a.y, b.y, acc.x);
  acc.y = fma(a.x, b.y, acc.y);
  acc.y = fma(-a.y, b.x, acc.y);
}

namespace ite {

// Number of kernels this library has launched (process-wide, all contexts).
void count_launches(unsigned long long n);
unsigned long long launches();

// ---------------------------------------------------------------- GEMM (FP64)
// C[b] = alpha * op(A[b]) * op(B[b]) + beta * C[b] (+ gamma * Z[b] if Z), complex.
// Element (i, k) of A is at A[b*sAb + i*sAm + k*sAk] (conjugated if conjA);
// element (k, j) of B at B[b*sBb + k*sBk + j*sBn]; C and Z are row-major with
// leading dimension ldc and batch stride sCb.  Strides are in complex units.
struct GemmArgs {
  int M, N, K, batch;
  const cplx* A; long long sAm, sAk, sAb; bool conjA;
  const cplx* B; long long sBk, sBn, sBb; bool conjB;
  cplx* C; long long ldc, sCb;
  cplx alpha, beta;
  const cplx* Z; cplx gamma;   // optional: C = alpha*AB + beta*C + gamma*Z
};
cudaError_t zgemm(const GemmArgs& g, cudaStream_t st);

// ---------------------------------------------------------------- tensor cores
// C[M][N] (fp32, leading dimension ldc) = A[M][K] B[N][K]^T with A, B bf16
// row-major (K contiguous, leading dimensions lda, ldb: multiples of 8).
// tcgen05 MMA with TMA-staged tiles; *err is set if a bounded wait ran out.
// bk = 64 (128-byte swizzle tiles) or 32 (64-byte swizzle tiles).
cudaError_t tc_gemm_bf16(const void* A, long long lda, const void* B, long long ldb, float* C,
                         long long ldc, int M, int N, int K, int* err, cudaStream_t st,
                         int bk = 64);

// Low-precision GEMM (lp_gemm.cu): C[b][split] (fp32 or bf16) = A[b] B[b]^T over the
// split's K range, A (M x K) and B (N x K) K-major in bf16 or, with tf32, fp32
// read as tf32 by kind::tf32 MMAs; fp32 accumulation in TMEM.  Leading
// dimensions and batch strides in elements, multiples of 16 bytes; a batch
// stride of 0 shares the operand across the batch.  bn = 128 or 256 (N tile);
// splits > 1 needs sCs (the output stride between K splits).  *err is set if
// a bounded wait ran out.
struct LpGemmArgs {
  int M, N, K, batch, splits, bn;
  bool tf32;
  const void* A; long long lda, sAb;
  const void* B; long long ldb, sBb;
  void* C; long long ldc, sCb, sCs;   // fp32, or bf16 with out_bf16 (elements)
  bool out_bf16;
  // complex output (splits 1, batch 1, N even): columns 2b, 2b+1 of the
  // product are (Re, Im) of complex column b, and the epilogue stores
  // C[m][b] (complex double, ldc in complex units) = alpha prod + gamma Z[m][b]
  // (fp32 arithmetic, Z may be NULL; Z has the leading dimension of C)
  bool out_complex;
  float2 alpha, gamma;
  const cplx* Z;
  // 256 x bn tiles on CTA pairs (cluster of two, cta_group::2 MMAs)
  bool pair;
};
cudaError_t lp_gemm(const LpGemmArgs& g, int* err, cudaStream_t st);
int lp_gemm_splits_used(const LpGemmArgs& g);
int lp_gemm_sm_count();

// Two-site H_eff with low-precision operands (heff_lp.cu): prepare embeds L
// and R once into `ops` (heff_lp_operand_bytes); apply computes
// Y = alpha H_eff X + gamma Z with bf16 (or tf32) tensor-core contractions and
// fp32 accumulation, using `scratch` (heff_lp_scratch_bytes).  Layouts as in
// the FP64 heff: L[w][a_bra][a_ket], R[w][b_ket][b_bra], X/Y/Z [a][s][t][b].
size_t heff_lp_operand_bytes(int D0, int D2, int chlB, int chlK, int chrK, int chrB, bool tf32);
size_t heff_lp_scratch_bytes(int d, int D0, int D2, int chlB, int chlK, int chrK, int chrB,
                             bool tf32);
cudaError_t heff_lp_prepare(const cplx* L, const cplx* R, int D0, int D2, int chlB, int chlK,
                            int chrK, int chrB, bool tf32, void* ops, size_t ops_bytes,
                            cudaStream_t st);
struct MixPlan;
cudaError_t heff_lp_apply(const void* ops, const MixPlan& plan2, int d, int D0, int D2, int chlB,
                          int chlK, int chrK, int chrB, bool tf32, const cplx* X, cplx* Y,
                          cplx alpha, const cplx* Z, cplx gamma, void* scratch,
                          size_t scratch_bytes, int* err, cudaStream_t st);

// FP64-accurate complex GEMM on the bf16 tensor cores (exact 7-bit slicing,
// see tc_zgemm.cu): same contract as zgemm; scratch of at least
// zgemm_emu_scratch_bytes(M, N, K) bytes; *err set if a bounded wait ran out.
size_t zgemm_emu_scratch_bytes(int M, int N, int K);
cudaError_t zgemm_emu(const GemmArgs& g, void* scratch, size_t scratch_bytes, int* err,
                      cudaStream_t st);

// ---------------------------------------------------------------- MPO mixing
// Sparse "gather - small matrix - scatter" along the MPO channel and physical
// indices.  Row k and column j of the small matrix decompose into up to three
// digits (k0,k1,k2) / (j0,j1,j2) with sizes rdim / cdim (row-major digit
// order).  For every outer pair (p, q), p < P, q < Q:
//   out[p*oP + q*oQ + sum_i k_i*oc[i]] = sum_e val[e] * in[p*iP + q*iQ + sum_i j_i*ic[i]]
// over the CSR entries e of row k (rows without entries write zero).
struct MixPlan {
  int nrows, ncols, nnz;
  int rdim[3], cdim[3];
  int* row_ptr;  // device, nrows+1
  int* col;      // device, nnz
  cplx* val;     // device, nnz
  float2* val32; // device, nnz: val rounded to fp32 (the low-precision contractions)
};
struct MixStrides {
  long long ic[3], oc[3];
};
cudaError_t mix_apply(const MixPlan& plan, const MixStrides& s, int P, int Q, const cplx* in,
                      long long iP, long long iQ, cplx* out, long long oP, long long oQ,
                      cudaStream_t st);

// ---------------------------------------------------------------- vectors
// Krylov and reduction kernels.  Partial sums are reduced in a fixed order,
// so every reduction is deterministic for a given launch shape.
cudaError_t vec_copy(cplx* y, const cplx* x, long long n, cudaStream_t st);
cudaError_t vec_zero(cplx* y, long long n, cudaStream_t st);
// y = a*x + b*y  (a, b complex scalars given on the host)
cudaError_t vec_axpby(cplx* y, const cplx* x, cplx a, cplx b, long long n, cudaStream_t st);
// out[i] = sum_e conj(V[i*ldv + e]) * w[e], i < nv  (device output); skips if *active == 0
cudaError_t vec_block_dot(const cplx* V, long long ldv, int nv, const cplx* w, long long n,
                          cplx* out, cplx* partial, const int* active, cudaStream_t st);
// w += sign * sum_i h[i] * V[i*ldv + .]  (h on device); skips if *active == 0
// (if nv_dev is given, only the first min(nv, *nv_dev) vectors are used)
cudaError_t vec_block_axpy(const cplx* V, long long ldv, int nv, const int* nv_dev,
                           const cplx* h, double sign, cplx* w, long long n, const int* active,
                           cudaStream_t st);
// out = sum |x|^2 (device double); skips if *active == 0
cudaError_t vec_norm2(const cplx* x, long long n, double* out, double* partial,
                      const int* active, cudaStream_t st);
// y *= *scale (device double); skips if *active == 0
cudaError_t vec_scale_dev(cplx* y, const double* scale, long long n, const int* active,
                          cudaStream_t st);
// out = sum_{w,b,b'} L[w][b][b'] * R[w][b'][b]  (device complex)
cudaError_t env_trace(const cplx* L, const cplx* R, int D, int m, int n, cplx* out,
                      cplx* partial, cudaStream_t st);
// K'[a][s'][b] = sum_s O[s'][s] K[a][s][b] (O on device, d x d)
cudaError_t apply_site_op(const cplx* O, const cplx* K, cplx* Kout, int chl, int d, int chr,
                          cudaStream_t st);

// ---------------------------------------------------------------- GMRES control
// Device-side state of one GMRES cycle (Givens QR of the Hessenberg matrix).
struct GmresState {
  cplx H[(32 + 1) * 32];  // column-major (m+1) x m, m <= 32
  cplx cs[32], sn[32];
  cplx g[33];
  cplx y[32];
  cplx h[64];             // scratch: this step's projections (two passes)
  double beta, bnorm, wnorm2, inv_h, res;
  int steps, active, breakdown;
};
// r0 = B - AX0 is in V0 with |r0|^2 in *norm2: set beta, scale factor, g.
cudaError_t gmres_start(GmresState* s, const double* r0norm2, const double* bnorm2,
                        cudaStream_t st);
// after Arnoldi step j (h1, h2 in s->h, |w|^2 in s->wnorm2): Givens update,
// breakdown/convergence test, 1/h_{j+1,j} for the next basis vector.
cudaError_t gmres_step(GmresState* s, int j, int m, double breakdown_rel, double local_tol,
                       cudaStream_t st);
// solve the triangular system for y (k = s->steps) and write y into s->y
cudaError_t gmres_finish(GmresState* s, cudaStream_t st);
// add the projections of the two Gram-Schmidt passes into column j of H
cudaError_t gmres_collect(GmresState* s, int j, int m, const cplx* h1, const cplx* h2,
                          cudaStream_t st);

// ---------------------------------------------------------------- SVD (FP64)
// Householder LQ of the rows of W (p x q, row-major), in place: row j keeps
// its part left of the diagonal as L[j][0..j) and beta[j] receives L[j][j].
// One cooperative launch; dev_state (8 device words) gets a nonzero word 4 if
// a grid-barrier wait ran out.
// refl (device, 3 k doubles, may be NULL) receives each reflector's
// (Re u_0, Im u_0, c) for lq_formq.
cudaError_t svd_lq(cplx* W, int p, int q, cplx* beta, double* refl, unsigned int* dev_state,
                   cudaStream_t st);
// L (p x k, row-major) with Xr = L Q^H from the output of svd_lq
cudaError_t lq_left(const cplx* W, const cplx* beta, int p, int q, cplx* Lout, cudaStream_t st);
// *out = |L1^{-1}|_F^2 for the leading k x k triangle L1 of svd_lq's L (+inf
// if a pivot is zero); colnorm2 (k doubles) is scratch.  sigma_min(Xr)^2 >=
// 1 / *out.
cudaError_t lq_inv_fnorm2(const cplx* W, const cplx* beta, int q, int k, double* colnorm2,
                          double* out, cudaStream_t st);
// Qh (k x q) = Q^H, the orthonormal rows with Xr = L Q^H, from svd_lq's
// output and refl.  One cooperative launch; dev_state (8 words) as svd_lq.
cudaError_t lq_formq(const cplx* W, const double* refl, int q, int k, cplx* Qh,
                     unsigned int* dev_state, cudaStream_t st);
// R (k x p, k = min(p, q)) = L^H from the output of svd_lq
cudaError_t svd_lq_r(const cplx* W, const cplx* beta, int p, int q, cplx* R, cudaStream_t st);
// One-sided Jacobi on the rows (length len) of A until they are mutually
// orthogonal; no rotation is accumulated.  One cooperative launch;
// dev_state (24 device words) returns the sweeps done in word 5, the pairs
// examined and rotated in words 6 and 7, and a nonzero word 4 if a bounded
// wait ran out; stamps (rows ints), wts and nref (rows doubles each: tracked
// and last computed squared row norms) are device scratch.  *anorm2 (device) is |A|_F^2: pairs of
// rows whose squared norms are both <= skip_rel |A|_F^2 are left as they are.
// keep_rank is the most rows the caller will keep: the sweeps stop once only
// rows that cannot be among them are still rotating (keep_rank >= rows
// disables this).
cudaError_t jacobi_rows(cplx* A, int rows, int len, int max_sweeps, double tol,
                        const double* anorm2, double skip_rel, int keep_rank,
                        unsigned int* dev_state, int* stamps, double* wts, double* nref,
                        cudaStream_t st);
// Several jacobi_rows problems in one cooperative launch (the truncated
// splits of concurrent evolutions).  Each item is one matrix with its own
// dev_state, stamps, wts and nref as jacobi_rows takes them, cleared
// beforehand by jacobi_prepare on the item's stream; every item ends exactly as
// jacobi_rows would leave it.  Items need at least 3 rows; n <= kJacobiGroupMax.
// group_state (24 device words) holds the group's grid barrier.
struct JacobiItem {
  cplx* A;
  const double* anorm2;
  unsigned int* st;
  int* stamps;
  double* wts;
  double* nref;
  double tol, skip_rel;
  int rows, len, max_sweeps, keep_rank;
};
constexpr int kJacobiGroupMax = 32;
struct JacobiGroup {
  int n;
  JacobiItem it[kJacobiGroupMax];
};
cudaError_t jacobi_prepare(int rows, unsigned int* dev_state, int* stamps, cudaStream_t st);
cudaError_t jacobi_rows_grouped(const JacobiItem* items, int n, unsigned int* group_state,
                                cudaStream_t st);
// blocks the grouped kernel can hold co-resident on the current device, and
// the blocks jacobi_rows_grouped launches for these items
cudaError_t jacobi_grouped_capacity(int* blocks);
int jacobi_grouped_blocks(const JacobiItem* items, int n);
// Grouped Jacobi launches across concurrent evolutions (group.cu): members
// post their split's Jacobi with group_jacobi; posts collected within the
// window, or once `expected` members have posted, run as one launch.
struct SplitGroup;
cudaError_t group_create(int device, double window_ms, SplitGroup** out);
void group_destroy(SplitGroup* g);
void group_set_expected(SplitGroup* g, int expected);
void group_set_policy(SplitGroup* g, int mode, double window_ms);
void group_stats(SplitGroup* g, long long* launches, long long* items);
cudaError_t group_jacobi(SplitGroup* g, const JacobiItem& item, cudaEvent_t ready, cudaEvent_t done,
                         unsigned int* gstate, cudaStream_t st);
// one cooperative launch of `blocks` blocks meeting at the grid barrier, the
// first `absent` of them never arriving; word 4 of dev_state ends nonzero
// when the wait ran out (blocks must be co-resident: at most the SM count)
cudaError_t barrier_selftest(unsigned int* dev_state, int blocks, int absent, cudaStream_t st);
// row norms sigma[i] = |A row i|, the permutation sorting them descending (ties
// by index), and the kept rank by the truncation rule (see engine).
cudaError_t svd_rank(const cplx* A, int p, int q, double* sigma, int* perm, double* sorted_sigma,
                     int chi_max, double cutoff, double weight_floor, double tie_rel,
                     int* rank_out, double* discarded_out, cudaStream_t st);
// sort given singular values descending and apply the truncation rule
cudaError_t sort_rank(const double* sigma, int p, int* perm, double* sorted_sigma, int chi_max,
                      double cutoff, double weight_floor, double tie_rel, int* rank_out,
                      double* discarded_out, cudaStream_t st);
// Uh (r x len) = rows perm[0..r) of D divided by sorted_sigma (unit vectors
// for zero rows)
cudaError_t svd_gather_uh(const cplx* D, int len, const int* perm, const double* sorted_sigma,
                          int r, cplx* Uh, cudaStream_t st);
// *out = scale * sum |x|^2 (device), deterministic
cudaError_t scaled_norm2(const cplx* x, long long n, double scale, double* out, double* partial,
                         cudaStream_t st);
// METTS collapse, one site (metts.cu): from the unit row vector v (chl) and
// the site tensor A (chl x d x chr), draws the site's state with the uniform
// u in the collapse basis (d x d device matrix, NULL: computational), writes
// it to *choice, multiplies *prob by its conditional probability and writes
// the next unit vector to v_out (chr).  d <= 4.
cudaError_t sample_site(const cplx* A, int chl, int d, int chr, const cplx* v, double u,
                        const cplx* basis, cplx* v_out, int* choice, double* prob, cudaStream_t st);
// out = A^H for a row-major m x n matrix A (out is n x m)
cudaError_t conj_transpose(const cplx* A, int m, int n, cplx* out, cudaStream_t st);

}  // namespace ite
