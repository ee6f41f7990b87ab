/*
 * ite_kernels.h -- kernel-level entry points of the GB300 library, one per
 * step of the two-site linear-solve sweep (Method, "two operations"; App. B).
 * They exist so that each step can be driven and checked on its own; the
 * sweep in ite_implicit_step runs exactly these kernels.
 *
 * All array arguments are DEVICE pointers to interleaved complex doubles,
 * owned by the caller, row-major, not aliasing each other unless stated.
 * Work is enqueued on the context stream; entry points that return host
 * values synchronise it.  Errors: ITE_EINVAL for bad sizes or an MPO bond /
 * site out of range, ITE_ECUDA for a failed launch (message in ite_last_error).
 */
#ifndef ITE_KERNELS_H
#define ITE_KERNELS_H

#include "ite.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Precision of the contractions inside the kernel-level calls below
 * (ite_k_heff, ite_k_env_left/right, ite_k_local_solve): ITE_FP64 (default)
 * or ITE_FP64_TC (FP64-class products on the tensor cores, as in the step's
 * tensor-core mode), or ITE_MIXED_BF16 / ITE_MIXED_TF32: ite_k_heff and the
 * environment updates then run as ITE_FP64_TC, and ite_k_local_solve runs the
 * mixed modes' refinement (ite.h, ite_precision) with refine_tol = local_tol
 * (1e-10 when 0) and at most 20 corrections.  ITE_EINVAL for any other
 * value. */
ite_status ite_ctx_set_kernel_precision(ite_ctx ctx, int precision);

/* Low-precision two-site H_eff of the mixed modes (the inner matvec of their
 * refinement; App. B's effective Hamiltonian), in two calls.  prepare copies
 * the environments L (D_i, chl_bra, chl_ket) and R (D_{i+2}, chr_ket, chr_bra),
 * laid out as for ite_k_heff, into the context's operand buffer as embedded
 * real matrices in bf16 (precision ITE_MIXED_BF16) or tf32 (ITE_MIXED_TF32);
 * apply then computes, for any number of X,
 *   Y = alpha * H_eff X + gamma * Z
 * with X, Y, Z as in ite_k_heff, the three contractions on the tensor cores
 * with fp32 accumulation and the alpha/gamma combination in FP64.  apply
 * uses the last prepare on this context and returns ITE_EINVAL if that was
 * for another MPO, bond or shape.  The relative error of Y - gamma Z is of
 * the order of the operand unit roundoff (2^-8 bf16, 2^-11 tf32) times the
 * conditioning of the sums. */
ite_status ite_k_heff_lp_prepare(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket,
                                 int chr_ket, int chr_bra, const double* L, const double* R,
                                 int precision);
ite_status ite_k_heff_lp_apply(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket,
                               int chr_ket, int chr_bra, const double* X, double* Y,
                               const double alpha[2], const double* Z, const double gamma[2]);
/* The same matvec `reps` times back to back on the context stream, with one
 * host synchronisation at the end, as the matvecs of a Krylov cycle run (App.
 * B's local solve issues them without host round trips); Y ends as one apply
 * leaves it.  For timing the matvec as the solve sees it.  ITE_EINVAL for
 * reps < 1 or Y equal to X or Z. */
ite_status ite_k_heff_lp_apply_n(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket,
                                 int chr_ket, int chr_bra, const double* X, double* Y,
                                 const double alpha[2], const double* Z, const double gamma[2],
                                 int reps);

/* Two-site effective Hamiltonian on sites (i, i+1) of the MPO (the dominant
 * operation of the local solves, App. B):
 *   Y[a,s',t',b] = alpha * sum L[w,a,a'] W_i[w,s',s,v] W_{i+1}[v,t',t,w'']
 *                              R[w'',b',b] X[a',s,t,b']  +  gamma * Z[a,s',t',b]
 * L: (D_i, chl_bra, chl_ket); R: (D_{i+2}, chr_ket, chr_bra) (ket index before
 * bra index); X: (chl_ket, d, d, chr_ket); Y, Z: (chl_bra, d, d, chr_bra).
 * Z may be NULL; Z may equal X when the bra and ket dimensions agree.
 * alpha and gamma are complex (re, im). */
ite_status ite_k_heff(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket, int chr_ket,
                      int chr_bra, const double* L, const double* R, const double* X, double* Y,
                      const double alpha[2], const double* Z, const double gamma[2]);

/* Environment updates (App. B: the projected operator of the two-site solve).
 * Left:  Lout[w',b,b'] = sum conj(bra[a,s',b]) Lin[w,a,a'] W_i[w,s',s,w'] ket[a',s,b']
 *        Lin (D_i, chl_bra, chl_ket), bra (chl_bra, d, chr_bra), ket (chl_ket, d, chr_ket),
 *        Lout (D_{i+1}, chr_bra, chr_ket).
 * Right: Rout[w,a',a] = sum ket[a',s,b'] Rin[w',b',b] W_i[w,s',s,w'] conj(bra[a,s',b])
 *        Rin (D_{i+1}, chr_ket, chr_bra), Rout (D_i, chl_ket, chl_bra). */
ite_status ite_k_env_left(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket, int chr_bra,
                          int chr_ket, const double* Lin, const double* bra, const double* ket,
                          double* Lout);
ite_status ite_k_env_right(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket, int chr_bra,
                           int chr_ket, const double* Rin, const double* bra, const double* ket,
                           double* Rout);

/* Local solve of one bond (App. B, App. D): one GMRES cycle of at most
 * krylov_dim Arnoldi steps on  (alpha I + c H_eff) X = B,  starting from the X
 * passed in, which is overwritten with the result.  L, R as in ite_k_heff with
 * bra = ket dimensions (chl, chr).  steps / rel_res (host, may be NULL) receive
 * the Arnoldi steps taken and the residual estimate |r|/|B|. */
ite_status ite_k_local_solve(ite_ctx ctx, ite_mpo H, int i, int chl, int chr, const double* L,
                             const double* R, const double* B, double* X, double alpha, double c,
                             int krylov_dim, double local_tol, int* steps, double* rel_res);

/* Truncated SVD split of X viewed as an m x n matrix (Heisenberg section: the
 * truncation keeps the discarded squared Schmidt weight below cutoff):
 * X = U S V^dag, kept rank r by the library's truncation rule (chi_max, cutoff,
 * weight floor 1e-24, near-degenerate groups kept whole).  centre_right != 0
 * writes left = U_r (m x r) and right = S_r V_r^dag = U_r^dag X (r x n);
 * otherwise left = U_r S_r = X V_r and right = V_r^dag.  left needs m*min(m,n)
 * and right min(m,n)*n complex entries of room; the output that receives the
 * projection (right when centre_right, else left) must not overlap X.
 * sigma (device, may be NULL) receives min(m,n) values in descending order:
 * singular values for the first chi_max entries down to a squared weight of
 * 1e-3 max(cutoff, 1e-25) of the total.  Rows that cannot be kept (below that
 * weight, or far below the chi_max-th) are not resolved among themselves, so
 * beyond those entries only the sum of squares is exact.  Algorithm: Householder LQ of the rows on the isometry side, one-sided
 * Jacobi on the triangular factor, projection GEMM.  flags bit 0 runs the
 * projection GEMM on the tensor cores with FP64-class accuracy (the emulation
 * of ite_k_zgemm mode 1). */
ite_status ite_k_split(ite_ctx ctx, const double* X, int m, int n, int chi_max, double cutoff,
                       int centre_right, double* left, double* right, double* sigma, int* rank,
                       double* discarded, int flags);

/* Self-test of the bounded grid-wide wait that the cooperative kernels of the
 * SVD (LQ and Jacobi sweeps) meet at after each step or round; the paper has
 * no counterpart.  Launches `blocks` co-resident blocks (2 <= blocks <= the
 * SM count) at one grid barrier, of which the first `absent` (0 <= absent <
 * blocks) never arrive.  absent == 0: the barrier completes, ITE_OK.
 * absent > 0: the waiting blocks give up at the barrier's iteration limit
 * (about a second), record the failure and return, and the call returns
 * ITE_ETIMEOUT with the context still usable.  ITE_EINVAL for other
 * arguments. */
ite_status ite_k_barrier_selftest(ite_ctx ctx, int blocks, int absent);

/* Tensor-core GEMM (the contraction engine of the library on sm_103a):
 * C[M][N] = A[M][K] B[N][K]^T, A and B bf16 row-major with K contiguous
 * (leading dimensions lda, ldb in elements, multiples of 8, pointers 16-byte
 * aligned), C fp32 row-major with leading dimension ldc.  Products are exact
 * in fp32 and accumulated in fp32 in tensor memory.  Serves the dense
 * contractions of the two-site effective Hamiltonian (App. B).  flags bit 0
 * selects 32-wide K tiles (64-byte swizzle) instead of 64-wide (128-byte).
 * ITE_ETIMEOUT if a bounded wait inside the kernel ran out. */
/* The persistent tensor-core GEMM of the low-precision H_eff (mixed modes):
 * for every batch entry b and K split s,
 *   C[b*sCb + s*sCs + m*ldc + n] = sum_{k in split s} A[b*sAb + m*lda + k] B[b*sBb + n*ldb + k]
 * with A, B K-major bf16 (tf32 == 0) or fp32 read as tf32 (tf32 != 0), fp32
 * accumulation in tensor memory, C fp32.  bn (128, 192 or 256) is the N tile; K
 * is cut into `splits` nearly equal ranges of 128-byte tiles (splits > 1 needs
 * sCs > 0).  Leading dimensions and batch strides are in elements and must be
 * multiples of 16 bytes; pointers 16-byte aligned; a batch stride of 0 shares
 * that operand across the batch.  flags bit 0 computes 256-row tiles on pairs
 * of CTAs (a cluster of two sharing each MMA, cta_group::2).  ITE_ETIMEOUT if
 * a bounded wait ran out. */
ite_status ite_k_gemm_lp(ite_ctx ctx, int M, int N, int K, int batch, const void* A, long long lda,
                         long long sAb, const void* B, long long ldb, long long sBb, float* C,
                         long long ldc, long long sCb, long long sCs, int tf32, int bn, int splits,
                         int flags);

ite_status ite_k_gemm_bf16(ite_ctx ctx, int M, int N, int K, const void* A, long long lda,
                           const void* B, long long ldb, float* C, long long ldc, int flags);

/* Complex GEMM C = alpha op(A) op(B) + beta C in FP64, the contraction
 * primitive of every environment and two-site product.  Element (i,k) of A
 * is A[i sAm + k sAk] (conjugated if conjA), element (k,j) of B is
 * B[k sBk + j sBn]; C is row-major with leading dimension ldc (complex
 * units).  mode 0: native FP64 arithmetic.  mode 1: FP64-class accuracy from
 * the bf16 tensor cores by exact 7-bit slicing of A and B (error below about
 * K 2^-52 max|A row| max|B column|).  alpha, beta may be NULL (1, 0). */
ite_status ite_k_zgemm(ite_ctx ctx, int mode, int M, int N, int K, const double* A, long long sAm,
                       long long sAk, int conjA, const double* B, long long sBk, long long sBn,
                       int conjB, double* C, long long ldc, const double alpha[2],
                       const double beta[2]);

/* Same result as ite_k_heff in FP64 mode, for callers that cannot allocate device memory
 * at call time (cudaMalloc can synchronise the whole device, the process may
 * have given all device memory to another pool, or allocation calls may be
 * forbidden where the caller runs).  This call allocates nothing: its two
 * intermediates live in one static device array of 2 x 524288 complex doubles
 * (16 MiB), held by every GPU that loads the library until the process exits.
 * The paper has no counterpart; it is a property of this library.
 * Sizes: D_i*chl_bra*d^2*chr_ket and D_{i+2}*chl_bra*d^2*chr_ket must each be
 * <= 524288, otherwise ITE_EINVAL (message in ite_last_error) and nothing runs.
 * All calls share the array: calls whose GPU work overlaps (other streams or
 * host threads) race and must be ordered by the caller.  Nothing in the array
 * needs to start at zero.  The first call on a device looks up the array's
 * device address, so make it before any stream capture.  Synchronises the
 * context stream before returning.  Always computes on the FP64 pipe, whatever
 * ite_ctx_set_kernel_precision selected (the tensor-core path needs slice
 * buffers sized per call).  Makes the context's device current for the call
 * and gives the calling thread its previous current device back. */
ite_status ite_k_heff_noalloc(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket,
                              int chr_ket, int chr_bra, const double* L, const double* R,
                              const double* X, double* Y, const double alpha[2],
                              const double* Z, const double gamma[2]);

#ifdef __cplusplus
}
#endif

#endif /* ITE_KERNELS_H */
