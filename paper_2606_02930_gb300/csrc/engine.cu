// Host orchestration and the C ABI (include/ite.h, include/ite_kernels.h).
//
// One implicit step (Eq. 4 or backward Euler) runs, in this order:
//   1. right-hand side MPS b: psi itself (backward Euler) or a two-site fit of
//      (I - c (H - s)) psi (trapezoid rule, Method operation (i));
//   2. x <- b (trapezoid) or psi (backward Euler) as the initial guess (App. B);
//   3. gauge move: x right-canonical by SVDs from the last site to the second;
//   4. right environments of <x|H|x> and <x|b>;
//   5. two-site sweep L->R then R->L (App. B, App. D): at each bond the local
//      right-hand side (projection of b), GMRES on (1 - c s) X + c H_eff X = B,
//      truncated SVD split, environment update;
//   6. normalisation of the centre tensor and the energy.
// Every numerical step is a CUDA kernel of this library; the host only
// sequences launches and reads back the kept rank of each split.
#include "common.cuh"
#include "ite.h"
#include "ite_kernels.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

using namespace ite;

namespace ite {
static std::atomic<unsigned long long> g_launches{0};
void count_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace ite

namespace {

constexpr double kWeightFloor = 1e-24;   // relative squared weight treated as zero
constexpr double kTieRel = 1e-10;        // near-degenerate singular values
constexpr double kBreakdownRel = 1e-14;  // GMRES happy breakdown: h_{j+1,j} <= this * |A v_j|
// one-sided Jacobi: rows count as orthogonal once |a_u^H a_v| <= q eps |a_u||a_v|
// (the rounding floor of a length-q inner product); sweeps are capped
constexpr double kEps = 2.220446049250313e-16;
constexpr int kJacobiSweeps = 30;
constexpr int kMaxKrylov = 32;
constexpr double kEmuMinWork = 2.0e6;    // complex MACs below which GEMMs stay native
// Algorithmic FP64 work of a truncated SVD of a p x q complex block, as the
// reference count that roofline figures divide by: the 22 n^3-class estimate
// of 8.7 GFLOP for a 512 x 512 block, scaled by p q min(p, q).
constexpr double kSvdAlgFlopsPerPQK = 8.7e9 / (512.0 * 512.0 * 512.0);
// Rows whose squared norm is below skip_weight(cutoff) |A|^2 can never be
// kept by the truncation rule, so the Jacobi sweeps do not orthogonalise two
// such rows against each other (their total weight is exact regardless).
double skip_weight(double cutoff) { return 1e-3 * std::max(cutoff, kWeightFloor * 0.1); }
// small SVD workspace for k rows: sigma, sorted (double), beta (complex),
// wts, nref (double), perm, stamps, done (int)
size_t small_bytes(long long k) { return (size_t)k * (4 * sizeof(double) + sizeof(cplx) + 3 * sizeof(int)) + 256; }
constexpr int kPartialSlots = 608 * kMaxKrylov;

struct HostRead {
  int rank;
  int steps;
  int counter;
  int pad;
  int lq_err;
  int pad2;
  unsigned int pairs[2];
  double disc;
  double res;
  double d[4];
  cplx z[4];
};

struct Buf {
  void* p = nullptr;
  size_t n = 0;
};

}  // namespace

struct ite_ctx_s {
  int device = 0;
  cudaStream_t stream = nullptr;
  ite_alloc_fn alloc = nullptr;
  ite_free_fn release = nullptr;
  void* user = nullptr;
  std::string err;
  size_t bytes = 0;
  // workspace
  Buf ws_X, ws_B, ws_X2, ws_V, ws_T1, ws_T2, ws_svdA, ws_svdQ, ws_left, ws_small, ws_env, ws_emu,
      ws_ovm, ws_lpops, ws_lpscr, ws_R, ws_D, ws_R2, ws_Xt;
  // mixed modes: precision of the inner matvecs while a refinement correction
  // runs (-1: none, 0: bf16, 1: tf32), and what the operand buffer holds
  int lp_level = -1;
  struct LpPrepared {
    const void* H = nullptr;
    int i = -1, dims[4] = {0, 0, 0, 0}, level = -1;
  } lp_prep;
  long long refinements = 0, lp_matvecs = 0;
  GmresState* gm = nullptr;
  double* dscal = nullptr;     // device scalars
  cplx* dcplx = nullptr;       // device complex scalars
  cplx* partial = nullptr;     // reduction partials
  int* dcounter = nullptr;
  HostRead* hr = nullptr;      // pinned
  int gemm_mode = 0;           // 0 native FP64, 1 tensor-core FP64 emulation
  int kernel_precision = 0;    // precision of the kernel-level entry points (ite_precision)
  long long jacobi_sweeps_total = 0, jacobi_splits = 0;
  double jacobi_flops = 0.0, lq_flops = 0.0, svd_alg_flops = 0.0;
  int jacobi_sweeps_max = 0;
  // event profiling of the sweep's stages (off unless started)
  bool prof = false;
  std::vector<cudaEvent_t> evpool;
  size_t evused = 0;
  struct Rec { int cat; size_t e0, e1; double flops; };
  std::vector<Rec> recs;
  // child contexts, each on its own stream, for solves that run concurrently
  // (the Gauss-Legendre step's shifted solves)
  std::vector<ite_ctx> children;
  std::vector<cudaStream_t> child_streams;
  // grouped Jacobi launches with other contexts (served runtime), and the
  // events that order this context's stream around them
  SplitGroup* group = nullptr;
  cudaEvent_t group_ready = nullptr, group_done = nullptr;
  unsigned int* group_state = nullptr;     // 24 words: barrier of a grouped launch it leads
};

struct ite_mpo_s {
  ite_ctx ctx = nullptr;
  int N = 0, d = 0;
  std::vector<int> D;                      // N+1
  std::vector<std::vector<cplx>> Wh;       // host copies, W_i[w][s'][s][w']
  Buf Wdev;
  std::vector<cplx*> W;                    // device pointers per site
  Buf plan_mem;
  std::vector<MixPlan> planL, planR, plan2;
  int Dmax = 1;
};

struct ite_mps_s {
  ite_ctx ctx = nullptr;
  int N = 0, d = 0, chi_cap = 0;
  std::vector<int> chi, cap;               // N+1
  Buf mem;
  std::vector<cplx*> site;
  ite_mps work_x = nullptr, work_b = nullptr, work_p = nullptr;  // internal copies for the step
  std::vector<ite_mps> work_gl;            // Gauss-Legendre partial-fraction solutions
};

// ------------------------------------------------------------------ memory
namespace {

ite_status fail(ite_ctx ctx, ite_status st, const std::string& msg) {
  if (ctx) ctx->err = msg;
  return st;
}

#define CK(call)                                                                  \
  do {                                                                            \
    cudaError_t e_ = (call);                                                      \
    if (e_ != cudaSuccess)                                                        \
      return fail(ctx, ITE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CS(call)                          \
  do {                                    \
    ite_status s_ = (call);               \
    if (s_ != ITE_OK) return s_;          \
  } while (0)

void* dev_alloc(ite_ctx ctx, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (ctx->alloc) {
    p = ctx->alloc(bytes, ctx->user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) ctx->bytes += bytes;
  return p;
}

void dev_free(ite_ctx ctx, void* p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  if (ctx->release) ctx->release(p, bytes, ctx->user);
  else cudaFree(p);
  ctx->bytes -= bytes;
}

void buf_free(ite_ctx ctx, Buf& b) {
  dev_free(ctx, b.p, b.n);
  b.p = nullptr;
  b.n = 0;
}

ite_status buf_ensure(ite_ctx ctx, Buf& b, size_t bytes) {
  if (b.n >= bytes && b.p) return ITE_OK;
  buf_free(ctx, b);
  b.p = dev_alloc(ctx, bytes);
  if (!b.p) return fail(ctx, ITE_ENOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  b.n = bytes;
  return ITE_OK;
}

template <typename T>
T* P(Buf& b) { return reinterpret_cast<T*>(b.p); }

cplx C(double r, double i = 0.0) { return cmake(r, i); }

ite_status sync(ite_ctx ctx) {
  CK(cudaStreamSynchronize(ctx->stream));
  return ITE_OK;
}

// ------------------------------------------------------------------ profiling
enum { P_HEFF = 0, P_ENV, P_SOLVE, P_SVD, P_GAUGE, P_PROJ, P_STEP, P_LQ, P_JACOBI, P_HEFF_LP, P_NCAT };
static_assert(P_NCAT <= ITE_PROFILE_SLOTS, "profile categories exceed the ABI's slots");

size_t prof_event(ite_ctx ctx) {
  if (ctx->evused == ctx->evpool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return (size_t)-1;
    ctx->evpool.push_back(e);
  }
  const size_t k = ctx->evused++;
  cudaEventRecord(ctx->evpool[k], ctx->stream);
  return k;
}

// Records an event pair around a stage when profiling is on.
struct Scope {
  ite_ctx ctx;
  int cat;
  size_t e0;
  double flops;
  Scope(ite_ctx c, int k, double f = 0.0) : ctx(c), cat(k), e0((size_t)-1), flops(f) {
    if (ctx->prof) e0 = prof_event(ctx);
  }
  ~Scope() {
    if (ctx->prof && e0 != (size_t)-1) {
      const size_t e1 = prof_event(ctx);
      if (e1 != (size_t)-1) ctx->recs.push_back({cat, e0, e1, flops});
    }
  }
};

// Kernel-level entry points run their contractions in the precision set by
// ite_ctx_set_kernel_precision; the emulated GEMMs' wait-error word is
// cleared on entry and checked by kernel_finish.
struct KernelMode {
  ite_ctx c;
  explicit KernelMode(ite_ctx ctx) : c(ctx) {
    c->gemm_mode = c->kernel_precision == ITE_FP64 ? 0 : 1;
    cudaMemsetAsync(reinterpret_cast<int*>(c->dcounter) + 10, 0, sizeof(int), c->stream);
  }
  ~KernelMode() { c->gemm_mode = 0; }
};

ite_status kernel_finish(ite_ctx ctx) {
  CK(cudaMemcpyAsync(&ctx->hr->steps, reinterpret_cast<int*>(ctx->dcounter) + 10, sizeof(int),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  if (ctx->hr->steps != 0) return fail(ctx, ITE_ETIMEOUT, "tensor-core GEMM wait ran out");
  return ITE_OK;
}

// ------------------------------------------------------------------ contractions
// Plain GEMM helpers.  Row-major matrices; strides in complex units.
ite_status gemm(ite_ctx ctx, int M, int N, int K, const cplx* A, long long sAm, long long sAk,
                bool conjA, const cplx* B, long long sBk, long long sBn, bool conjB, cplx* Cm,
                long long ldc, cplx alpha = C(1), cplx beta = C(0), const cplx* Z = nullptr,
                cplx gamma = C(0), int batch = 1, long long sAb = 0, long long sBb = 0,
                long long sCb = 0) {
  GemmArgs g;
  g.M = M; g.N = N; g.K = K; g.batch = batch;
  g.A = A; g.sAm = sAm; g.sAk = sAk; g.sAb = sAb; g.conjA = conjA;
  g.B = B; g.sBk = sBk; g.sBn = sBn; g.sBb = sBb; g.conjB = conjB;
  g.C = Cm; g.ldc = ldc; g.sCb = sCb;
  g.alpha = alpha; g.beta = beta; g.Z = Z; g.gamma = gamma;
  // large contractions on the tensor cores when the step asks for it; small
  // ones (edge bonds) stay on the FP64 pipe where launch latency dominates
  if (ctx->gemm_mode == 1 && (double)M * N * K >= kEmuMinWork && K >= 16) {
    CS(buf_ensure(ctx, ctx->ws_emu, zgemm_emu_scratch_bytes(M, N, K)));
    CK(zgemm_emu(g, ctx->ws_emu.p, ctx->ws_emu.n, reinterpret_cast<int*>(ctx->dcounter) + 10,
                 ctx->stream));
    return ITE_OK;
  }
  CK(zgemm(g, ctx->stream));
  return ITE_OK;
}

// Y = alpha * H_eff X + gamma * Z on sites (i, i+1)
ite_status heff(ite_ctx ctx, ite_mpo H, int i, int chlB, int chlK, int chrK, int chrB,
                const cplx* L, const cplx* R, const cplx* X, cplx* Y, cplx alpha, const cplx* Z,
                cplx gamma) {
  const int d = H->d, D0 = H->D[i], D1 = H->D[i + 1], D2 = H->D[i + 2];
  const long long d2 = (long long)d * d;
  // algorithmic real FLOPs of the dense two-site contraction (complex MACs x 8)
  const double flops = 8.0 * ((double)D0 * d2 * chlB * chlK * chrK + (double)D2 * d2 * chlB * chrK * chrB +
                              2.0 * D1 * D1 * d2 * d * chlB * chrK);
  Scope sc(ctx, P_HEFF, flops);
  cplx* T1 = P<cplx>(ctx->ws_T1);
  cplx* T2 = P<cplx>(ctx->ws_T2);
  // T1[(w a), (s t b')] = L[(w a), a'] X[a', (s t b')]
  CS(gemm(ctx, D0 * chlB, (int)(d2 * chrK), chlK, L, chlK, 1, false, X, d2 * chrK, 1, false, T1,
          d2 * chrK));
  // T2[a, s', t', w'', b'] = sum W2[(s' t' w''), (w s t)] T1[w, a, s, t, b']
  MixStrides ms;
  ms.ic[0] = (long long)chlB * d2 * chrK; ms.ic[1] = (long long)d * chrK; ms.ic[2] = chrK;
  ms.oc[0] = (long long)d * D2 * chrK; ms.oc[1] = (long long)D2 * chrK; ms.oc[2] = chrK;
  CK(mix_apply(H->plan2[i], ms, chlB, chrK, T1, d2 * chrK, 1, T2, d2 * D2 * chrK, 1, ctx->stream));
  // Y[(a s' t'), b] = alpha * T2[(a s' t'), (w'' b')] R[(w'' b'), b] + gamma Z
  CS(gemm(ctx, (int)(chlB * d2), chrB, D2 * chrK, T2, (long long)D2 * chrK, 1, false, R, chrB, 1,
          false, Y, chrB, alpha, C(0), Z, gamma));
  return ITE_OK;
}

// Low-precision H_eff from the operands prepared for (H, i, dims) at
// ctx->lp_level (bf16 or tf32): Y = alpha H_eff X + gamma Z.
ite_status heff_lp(ite_ctx ctx, ite_mpo H, int i, int chlB, int chlK, int chrK, int chrB,
                   const cplx* X, cplx* Y, cplx alpha, const cplx* Z, cplx gamma) {
  const int d = H->d, D0 = H->D[i], D1 = H->D[i + 1], D2 = H->D[i + 2];
  const auto& pp = ctx->lp_prep;
  if (pp.H != H || pp.i != i || pp.dims[0] != chlB || pp.dims[1] != chlK || pp.dims[2] != chrK ||
      pp.dims[3] != chrB || pp.level != ctx->lp_level)
    return fail(ctx, ITE_EINVAL, "low-precision H_eff: operands prepared for another bond or shape");
  const long long d2 = (long long)d * d;
  const double flops = 8.0 * ((double)D0 * d2 * chlB * chlK * chrK + (double)D2 * d2 * chlB * chrK * chrB +
                              2.0 * D1 * D1 * d2 * d * chlB * chrK);
  Scope sc(ctx, P_HEFF_LP, flops);
  const bool tf32 = ctx->lp_level == 1;
  CS(buf_ensure(ctx, ctx->ws_lpscr, heff_lp_scratch_bytes(d, D0, D2, chlB, chlK, chrK, chrB, tf32)));
  CK(heff_lp_apply(ctx->ws_lpops.p, H->plan2[i], d, D0, D2, chlB, chlK, chrK, chrB, tf32, X, Y,
                   alpha, Z, gamma, ctx->ws_lpscr.p, ctx->ws_lpscr.n,
                   reinterpret_cast<int*>(ctx->dcounter) + 10, ctx->stream));
  ctx->lp_matvecs += 1;
  return ITE_OK;
}

// Embeds L and R for heff_lp at precision level (0 bf16, 1 tf32).
ite_status heff_lp_setup(ite_ctx ctx, ite_mpo H, int i, int chlB, int chlK, int chrK, int chrB,
                         const cplx* L, const cplx* R, int level) {
  const int D0 = H->D[i], D2 = H->D[i + 2];
  const bool tf32 = level == 1;
  CS(buf_ensure(ctx, ctx->ws_lpops, heff_lp_operand_bytes(D0, D2, chlB, chlK, chrK, chrB, tf32)));
  CK(heff_lp_prepare(L, R, D0, D2, chlB, chlK, chrK, chrB, tf32, ctx->ws_lpops.p, ctx->ws_lpops.n,
                     ctx->stream));
  auto& pp = ctx->lp_prep;
  pp.H = H;
  pp.i = i;
  pp.dims[0] = chlB; pp.dims[1] = chlK; pp.dims[2] = chrK; pp.dims[3] = chrB;
  pp.level = level;
  return ITE_OK;
}

// The local operator's H_eff: low precision inside a refinement correction,
// else the FP64 (or FP64-class) contraction.
ite_status apply_heff(ite_ctx ctx, ite_mpo H, int i, int chl, int chr, const cplx* L,
                      const cplx* R, const cplx* X, cplx* Y, cplx alpha, const cplx* Z, cplx gamma) {
  if (ctx->lp_level >= 0) return heff_lp(ctx, H, i, chl, chl, chr, chr, X, Y, alpha, Z, gamma);
  return heff(ctx, H, i, chl, chl, chr, chr, L, R, X, Y, alpha, Z, gamma);
}

ite_status env_left(ite_ctx ctx, ite_mpo H, int i, int chlB, int chlK, int chrB, int chrK,
                    const cplx* Lin, const cplx* bra, const cplx* ket, cplx* Lout) {
  const int d = H->d, D0 = H->D[i], D1 = H->D[i + 1];
  Scope sc(ctx, P_ENV);
  cplx* T1 = P<cplx>(ctx->ws_T1);
  cplx* T2 = P<cplx>(ctx->ws_T2);
  const long long ld = (long long)d * chrK;
  CS(gemm(ctx, D0 * chlB, (int)ld, chlK, Lin, chlK, 1, false, ket, ld, 1, false, T1, ld));
  MixStrides ms;
  ms.ic[0] = (long long)chlB * ld; ms.ic[1] = chrK; ms.ic[2] = 0;
  ms.oc[0] = (long long)chlB * ld; ms.oc[1] = chrK; ms.oc[2] = 0;
  CK(mix_apply(H->planL[i], ms, chlB, chrK, T1, ld, 1, T2, ld, 1, ctx->stream));
  // Lout[w'] (chrB x chrK) = bra^H ((chrB) x (chlB d)) T2[w'] ((chlB d) x chrK)
  CS(gemm(ctx, chrB, chrK, chlB * d, bra, 1, chrB, true, T2, chrK, 1, false, Lout, chrK, C(1),
          C(0), nullptr, C(0), D1, 0, (long long)chlB * ld, (long long)chrB * chrK));
  return ITE_OK;
}

ite_status env_right(ite_ctx ctx, ite_mpo H, int i, int chlB, int chlK, int chrB, int chrK,
                     const cplx* Rin, const cplx* bra, const cplx* ket, cplx* Rout) {
  const int d = H->d, D0 = H->D[i], D1 = H->D[i + 1];
  Scope sc(ctx, P_ENV);
  cplx* T1 = P<cplx>(ctx->ws_T1);
  cplx* T2 = P<cplx>(ctx->ws_T2);
  const long long blk = (long long)chlK * d * chrB;
  // T1[w'][(a' s)][b] = ket[(a' s), b'] Rin[w'][b'][b]
  CS(gemm(ctx, chlK * d, chrB, chrK, ket, chrK, 1, false, Rin, chrB, 1, false, T1, chrB, C(1),
          C(0), nullptr, C(0), D1, 0, (long long)chrK * chrB, blk));
  MixStrides ms;
  ms.ic[0] = blk; ms.ic[1] = chrB; ms.ic[2] = 0;
  ms.oc[0] = blk; ms.oc[1] = chrB; ms.oc[2] = 0;
  CK(mix_apply(H->planR[i], ms, chlK, chrB, T1, (long long)d * chrB, 1, T2, (long long)d * chrB, 1,
               ctx->stream));
  // Rout[w] (chlK x chlB) = T2[w] (chlK x (d chrB)) conj(bra)^T ((d chrB) x chlB)
  CS(gemm(ctx, chlK, chlB, d * chrB, T2, (long long)d * chrB, 1, false, bra, 1, (long long)d * chrB,
          true, Rout, chlB, C(1), C(0), nullptr, C(0), D0, blk, 0, (long long)chlK * chlB));
  return ITE_OK;
}

ite_status ov_left(ite_ctx ctx, int d, int chlB, int chlK, int chrB, int chrK, const cplx* Lin,
                   const cplx* bra, const cplx* ket, cplx* Lout) {
  Scope sc(ctx, P_ENV);
  cplx* T1 = P<cplx>(ctx->ws_T1);
  const long long ld = (long long)d * chrK;
  CS(gemm(ctx, chlB, (int)ld, chlK, Lin, chlK, 1, false, ket, ld, 1, false, T1, ld));
  CS(gemm(ctx, chrB, chrK, chlB * d, bra, 1, chrB, true, T1, chrK, 1, false, Lout, chrK));
  return ITE_OK;
}

ite_status ov_right(ite_ctx ctx, int d, int chlB, int chlK, int chrB, int chrK, const cplx* Rin,
                    const cplx* bra, const cplx* ket, cplx* Rout) {
  Scope sc(ctx, P_ENV);
  cplx* T1 = P<cplx>(ctx->ws_T1);
  CS(gemm(ctx, chlK * d, chrB, chrK, ket, chrK, 1, false, Rin, chrB, 1, false, T1, chrB));
  CS(gemm(ctx, chlK, chlB, d * chrB, T1, (long long)d * chrB, 1, false, bra, 1, (long long)d * chrB,
          true, Rout, chlB));
  return ITE_OK;
}

// out[a,s,t,b] = alpha * sum LO[a][a''] K1[a'',s,c] K2[c,t,b''] RO[b''][b]
ite_status project(ite_ctx ctx, int d, int chlB, int chlK, int chm, int chrK, int chrB,
                   const cplx* LO, const cplx* K1, const cplx* K2, const cplx* RO, cplx* out) {
  Scope sc(ctx, P_PROJ);
  cplx* T1 = P<cplx>(ctx->ws_T1);
  cplx* T2 = P<cplx>(ctx->ws_T2);
  CS(gemm(ctx, chlB, d * chm, chlK, LO, chlK, 1, false, K1, (long long)d * chm, 1, false, T1,
          (long long)d * chm));
  CS(gemm(ctx, chlB * d, d * chrK, chm, T1, chm, 1, false, K2, (long long)d * chrK, 1, false, T2,
          (long long)d * chrK));
  CS(gemm(ctx, chlB * d * d, chrB, chrK, T2, chrK, 1, false, RO, chrB, 1, false, out, chrB));
  return ITE_OK;
}

ite_status merge(ite_ctx ctx, int d, int chl, int chm, int chr, const cplx* K1, const cplx* K2,
                 cplx* out) {
  Scope sc(ctx, P_PROJ);
  return gemm(ctx, chl * d, d * chr, chm, K1, chm, 1, false, K2, (long long)d * chr, 1, false, out,
              (long long)d * chr);
}

// Truncated SVD of X (m x n) into left (m x r) and right (r x n); returns r.
// The rows of Xr are indexed by the side whose isometry is wanted: Xr = X
// when centre_right (left = U_r), Xr = X^H otherwise (right = V_r^H).  The
// LQ-preconditioned Jacobi gives sigma and U_r^H; the other factor is the
// projection U_r^H Xr (one GEMM, on the tensor cores in the tensor-core mode).
ite_status split(ite_ctx ctx, const cplx* X, int m, int n, int chi_max, double cutoff,
                 bool centre_right, cplx* left, cplx* right, int* r_out, double* disc_out,
                 double* sigma_out = nullptr) {
  Scope sc(ctx, P_SVD);
  const bool tr = !centre_right;
  const int p = tr ? n : m, q = tr ? m : n;
  const int k = std::min(p, q);
  CS(buf_ensure(ctx, ctx->ws_svdA, (size_t)m * n * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_svdQ, (size_t)k * p * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_small, small_bytes(k)));
  cplx* W = P<cplx>(ctx->ws_svdA);
  cplx* R = P<cplx>(ctx->ws_svdQ);
  char* sm = P<char>(ctx->ws_small);
  double* sigma = reinterpret_cast<double*>(sm);
  double* sorted = sigma + k;
  cplx* beta = reinterpret_cast<cplx*>(sorted + k);
  double* wts = reinterpret_cast<double*>(beta + k);
  double* nref = wts + k;
  int* perm = reinterpret_cast<int*>(nref + k);
  int* stamps = perm + k;
  // dcounter words: 8-10 GEMM error flags, 16-39 Jacobi state, 40-47 LQ state
  unsigned int* jstate = reinterpret_cast<unsigned int*>(ctx->dcounter) + 16;
  unsigned int* lqstate = reinterpret_cast<unsigned int*>(ctx->dcounter) + 40;
  double* anorm2 = ctx->dscal + 8;
  if (tr) CK(conj_transpose(X, m, n, W, ctx->stream));
  else CK(vec_copy(W, X, (long long)m * n, ctx->stream));
  CK(scaled_norm2(W, (long long)p * q, 1.0, anorm2, ctx->dscal + 16, ctx->stream));
  // 1-2. R = L^H from the Householder LQ of the rows of Xr
  {
    // algorithmic FP64 flops: per step j the norm of the tail (4 (q-j)) and,
    // per later row, the product with the reflector and the update (16 (q-j))
    double f = 0.0;
    for (int j = 0; j < k; ++j) f += 4.0 * (q - j) + 16.0 * (q - j) * (p - j - 1);
    ctx->lq_flops += f;
    Scope lq_scope(ctx, P_LQ, f);
    CK(svd_lq(W, p, q, beta, nullptr, lqstate, ctx->stream));
  }
  CK(svd_lq_r(W, beta, p, q, R, ctx->stream));
  // 3. one-sided Jacobi on the k rows (length p) of R
  {
    Scope jacobi_scope(ctx, P_JACOBI);
    const double tol = std::max(1e-15, p * kEps);
    if (ctx->group && k >= 3) {
      // the same Jacobi, launched together with other contexts' splits
      CK(jacobi_prepare(k, jstate, stamps, ctx->stream));
      const JacobiItem item{R, anorm2, jstate, stamps, wts, nref, tol, skip_weight(cutoff),
                            k, p, kJacobiSweeps, chi_max};
      CK(group_jacobi(ctx->group, item, ctx->group_ready, ctx->group_done, ctx->group_state,
                      ctx->stream));
    } else {
      CK(jacobi_rows(R, k, p, kJacobiSweeps, tol, anorm2, skip_weight(cutoff), chi_max, jstate,
                     stamps, wts, nref, ctx->stream));
    }
  }
  // 4. singular values, order and rank
  int* rank_dev = reinterpret_cast<int*>(ctx->dscal + 6);
  double* disc_dev = ctx->dscal + 7;
  CK(svd_rank(R, k, p, sigma, perm, sorted, chi_max, cutoff, kWeightFloor, kTieRel, rank_dev,
              disc_dev, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->rank, rank_dev, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->disc, disc_dev, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->counter, jstate + 4, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->pad, jstate + 5, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->lq_err, lqstate + 4, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(ctx->hr->pairs, jstate + 6, 2 * sizeof(unsigned int), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->steps, reinterpret_cast<int*>(ctx->dcounter) + 10, sizeof(int),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  if (ctx->hr->counter != 0 || ctx->hr->lq_err != 0)
    return fail(ctx, ITE_ETIMEOUT, "SVD grid barrier wait ran out");
  if (ctx->hr->steps != 0) return fail(ctx, ITE_ETIMEOUT, "tensor-core GEMM wait ran out");
  ctx->jacobi_sweeps_total += ctx->hr->pad;
  ctx->jacobi_splits += 1;
  ctx->jacobi_sweeps_max = std::max(ctx->jacobi_sweeps_max, ctx->hr->pad);
  // FP64 flops of the Jacobi as the device ran it: 8 per element and examined
  // pair (one inner product; the row norms are tracked), 20 per element and
  // rotated pair (the rotation)
  ctx->jacobi_flops += (8.0 * ctx->hr->pairs[0] + 20.0 * ctx->hr->pairs[1]) * p;
  ctx->svd_alg_flops += kSvdAlgFlopsPerPQK * (double)p * q * k;
  const int r = ctx->hr->rank;
  if (r < 1 || r > k) return fail(ctx, ITE_ESINGULAR, "invalid rank from SVD");
  if (!std::isfinite(ctx->hr->disc)) return fail(ctx, ITE_ESINGULAR, "non-finite singular values");
  if (sigma_out) {
    CK(cudaMemsetAsync(sigma_out, 0, sizeof(double) * std::min(m, n), ctx->stream));
    CK(cudaMemcpyAsync(sigma_out, sorted, sizeof(double) * k, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  // 5. factors: Uh = U_r^H (r x p) in the LQ workspace (free again), then
  // the projection.  X is read in full before the isometry side is written,
  // so X may share memory with that side (the gauge moves do).
  cplx* Uh = W;
  CK(svd_gather_uh(R, p, perm, sorted, r, Uh, ctx->stream));
  if (!centre_right) {
    // left = X V_r (m x r), right = V_r^H (r x n)
    CS(gemm(ctx, m, r, n, X, n, 1, false, Uh, 1, n, true, left, r));
    CK(vec_copy(right, Uh, (long long)r * n, ctx->stream));
  } else {
    // right = U_r^H X (r x n), left = U_r (m x r)
    CS(gemm(ctx, r, n, m, Uh, m, 1, false, X, n, 1, false, right, n));
    CK(conj_transpose(Uh, r, m, left, ctx->stream));
  }
  *r_out = r;
  *disc_out = ctx->hr->disc;
  return ITE_OK;
}

// One GMRES cycle on (alpha I + c H_eff) X = B; X updated in place.
ite_status gmres_cycle(ite_ctx ctx, ite_mpo H, int i, int chl, int chr, const cplx* L,
                       const cplx* R, const cplx* B, cplx* X, cplx alpha, cplx c, int m,
                       double local_tol, int* steps, double* res) {
  Scope sc(ctx, P_SOLVE);
  const long long n = (long long)chl * H->d * H->d * chr;
  cplx* V = P<cplx>(ctx->ws_V);
  GmresState* gs = ctx->gm;
  int* active = &gs->active;
  double* r0n2 = ctx->dscal + 0;
  double* bn2 = ctx->dscal + 1;
  const cplx ca = alpha, cc = c;
  // r0 = B - A X0
  CS(apply_heff(ctx, H, i, chl, chr, L, R, X, V, cc, X, ca));
  CK(vec_axpby(V, B, C(1), C(-1), n, ctx->stream));
  CK(vec_norm2(V, n, r0n2, ctx->dscal + 16, nullptr, ctx->stream));
  CK(vec_norm2(B, n, bn2, ctx->dscal + 16, nullptr, ctx->stream));
  CK(gmres_start(gs, r0n2, bn2, ctx->stream));
  CK(vec_scale_dev(V, &gs->inv_h, n, active, ctx->stream));
  for (int j = 0; j < m; ++j) {
    cplx* vj = V + j * n;
    cplx* w = V + (j + 1) * n;
    CS(apply_heff(ctx, H, i, chl, chr, L, R, vj, w, cc, vj, ca));
    CK(vec_block_dot(V, n, j + 1, w, n, gs->h, ctx->partial, active, ctx->stream));
    CK(vec_block_axpy(V, n, j + 1, nullptr, gs->h, -1.0, w, n, active, ctx->stream));
    CK(vec_block_dot(V, n, j + 1, w, n, gs->h + 32, ctx->partial, active, ctx->stream));
    CK(vec_block_axpy(V, n, j + 1, nullptr, gs->h + 32, -1.0, w, n, active, ctx->stream));
    CK(gmres_collect(gs, j, m, gs->h, gs->h + 32, ctx->stream));
    CK(vec_norm2(w, n, &gs->wnorm2, ctx->dscal + 16, active, ctx->stream));
    CK(gmres_step(gs, j, m, kBreakdownRel, local_tol, ctx->stream));
    CK(vec_scale_dev(w, &gs->inv_h, n, active, ctx->stream));
  }
  CK(gmres_finish(gs, ctx->stream));
  CK(vec_block_axpy(V, n, m, &gs->steps, gs->y, 1.0, X, n, nullptr, ctx->stream));
  if (steps || res) {
    CK(cudaMemcpyAsync(&ctx->hr->steps, &gs->steps, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&ctx->hr->res, &gs->res, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(&ctx->hr->d[0], &gs->bnorm, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    CS(sync(ctx));
    if (steps) *steps = ctx->hr->steps;
    if (res) *res = ctx->hr->d[0] > 0 ? ctx->hr->res / ctx->hr->d[0] : 0.0;
  }
  return ITE_OK;
}

// ------------------------------------------------------------------ MPO setup
void build_plan(std::vector<int>& rp, std::vector<int>& cols, std::vector<cplx>& vals,
                const std::vector<cplx>& dense, int nrows, int ncols) {
  rp.assign(nrows + 1, 0);
  cols.clear();
  vals.clear();
  for (int k = 0; k < nrows; ++k) {
    for (int j = 0; j < ncols; ++j) {
      const cplx v = dense[(size_t)k * ncols + j];
      if (v.x != 0.0 || v.y != 0.0) {
        cols.push_back(j);
        vals.push_back(v);
      }
    }
    rp[k + 1] = (int)cols.size();
  }
}

ite_status mpo_finish(ite_mpo H) {
  ite_ctx ctx = H->ctx;
  const int N = H->N, d = H->d;
  H->Dmax = *std::max_element(H->D.begin(), H->D.end());
  size_t total = 0;
  std::vector<size_t> off(N);
  for (int i = 0; i < N; ++i) {
    off[i] = total;
    total += H->Wh[i].size();
  }
  CS(buf_ensure(ctx, H->Wdev, total * sizeof(cplx)));
  H->W.resize(N);
  for (int i = 0; i < N; ++i) {
    H->W[i] = P<cplx>(H->Wdev) + off[i];
    CK(cudaMemcpy(H->W[i], H->Wh[i].data(), H->Wh[i].size() * sizeof(cplx), cudaMemcpyHostToDevice));
  }
  // mixing matrices on the host (MPO setup), then one device block for all
  struct Host { std::vector<int> rp, col; std::vector<cplx> val; int nr, nc, rd[3], cd[3]; };
  std::vector<Host> hs;
  auto Wat = [&](int i, int w, int sp, int s, int w2) -> cplx {
    const int Dr = H->D[i + 1];
    return H->Wh[i][(((size_t)w * d + sp) * d + s) * Dr + w2];
  };
  for (int i = 0; i < N; ++i) {
    const int Dl = H->D[i], Dr = H->D[i + 1];
    // left update: rows (w', s'), cols (w, s)
    Host hl; hl.nr = Dr * d; hl.nc = Dl * d;
    hl.rd[0] = Dr; hl.rd[1] = d; hl.rd[2] = 1; hl.cd[0] = Dl; hl.cd[1] = d; hl.cd[2] = 1;
    std::vector<cplx> dl((size_t)hl.nr * hl.nc, C(0));
    for (int w = 0; w < Dl; ++w)
      for (int sp = 0; sp < d; ++sp)
        for (int s = 0; s < d; ++s)
          for (int w2 = 0; w2 < Dr; ++w2) dl[(size_t)(w2 * d + sp) * hl.nc + (w * d + s)] = Wat(i, w, sp, s, w2);
    build_plan(hl.rp, hl.col, hl.val, dl, hl.nr, hl.nc);
    hs.push_back(hl);
    // right update: rows (w, s'), cols (w', s)
    Host hr; hr.nr = Dl * d; hr.nc = Dr * d;
    hr.rd[0] = Dl; hr.rd[1] = d; hr.rd[2] = 1; hr.cd[0] = Dr; hr.cd[1] = d; hr.cd[2] = 1;
    std::vector<cplx> dr((size_t)hr.nr * hr.nc, C(0));
    for (int w = 0; w < Dl; ++w)
      for (int sp = 0; sp < d; ++sp)
        for (int s = 0; s < d; ++s)
          for (int w2 = 0; w2 < Dr; ++w2) dr[(size_t)(w * d + sp) * hr.nc + (w2 * d + s)] = Wat(i, w, sp, s, w2);
    build_plan(hr.rp, hr.col, hr.val, dr, hr.nr, hr.nc);
    hs.push_back(hr);
  }
  for (int i = 0; i + 1 < N; ++i) {
    const int D0 = H->D[i], D1 = H->D[i + 1], D2 = H->D[i + 2];
    Host h2; h2.nr = d * d * D2; h2.nc = D0 * d * d;
    h2.rd[0] = d; h2.rd[1] = d; h2.rd[2] = D2; h2.cd[0] = D0; h2.cd[1] = d; h2.cd[2] = d;
    std::vector<cplx> dd((size_t)h2.nr * h2.nc, C(0));
    for (int w = 0; w < D0; ++w)
      for (int sp = 0; sp < d; ++sp)
        for (int s = 0; s < d; ++s)
          for (int v = 0; v < D1; ++v) {
            const cplx a = Wat(i, w, sp, s, v);
            if (a.x == 0.0 && a.y == 0.0) continue;
            for (int tp = 0; tp < d; ++tp)
              for (int t = 0; t < d; ++t)
                for (int w2 = 0; w2 < D2; ++w2) {
                  const cplx b = Wat(i + 1, v, tp, t, w2);
                  cplx& dst = dd[(size_t)((sp * d + tp) * D2 + w2) * h2.nc + ((w * d + s) * d + t)];
                  dst = cadd(dst, cmul(a, b));
                }
          }
    build_plan(h2.rp, h2.col, h2.val, dd, h2.nr, h2.nc);
    hs.push_back(h2);
  }
  size_t bytes = 0;
  for (auto& h : hs)
    bytes += (h.rp.size() + h.col.size()) * sizeof(int) + h.val.size() * (sizeof(cplx) + sizeof(float2)) + 80;
  CS(buf_ensure(ctx, H->plan_mem, bytes));
  char* base = P<char>(H->plan_mem);
  size_t pos = 0;
  std::vector<MixPlan> plans;
  for (auto& h : hs) {
    MixPlan pl;
    pl.nrows = h.nr; pl.ncols = h.nc; pl.nnz = (int)h.val.size();
    for (int t = 0; t < 3; ++t) { pl.rdim[t] = h.rd[t]; pl.cdim[t] = h.cd[t]; }
    pos = (pos + 15) & ~size_t(15);
    pl.val = reinterpret_cast<cplx*>(base + pos);
    CK(cudaMemcpy(pl.val, h.val.data(), h.val.size() * sizeof(cplx), cudaMemcpyHostToDevice));
    pos += h.val.size() * sizeof(cplx);
    pl.row_ptr = reinterpret_cast<int*>(base + pos);
    CK(cudaMemcpy(pl.row_ptr, h.rp.data(), h.rp.size() * sizeof(int), cudaMemcpyHostToDevice));
    pos += h.rp.size() * sizeof(int);
    pl.col = reinterpret_cast<int*>(base + pos);
    CK(cudaMemcpy(pl.col, h.col.data(), h.col.size() * sizeof(int), cudaMemcpyHostToDevice));
    pos += h.col.size() * sizeof(int);
    pos = (pos + 15) & ~size_t(15);
    pl.val32 = reinterpret_cast<float2*>(base + pos);
    {
      std::vector<float2> v32(h.val.size());
      for (size_t e = 0; e < h.val.size(); ++e) v32[e] = make_float2((float)h.val[e].x, (float)h.val[e].y);
      CK(cudaMemcpy(pl.val32, v32.data(), v32.size() * sizeof(float2), cudaMemcpyHostToDevice));
    }
    pos += h.val.size() * sizeof(float2);
    plans.push_back(pl);
  }
  H->planL.resize(N);
  H->planR.resize(N);
  for (int i = 0; i < N; ++i) {
    H->planL[i] = plans[2 * i];
    H->planR[i] = plans[2 * i + 1];
  }
  H->plan2.clear();
  for (int i = 0; i + 1 < N; ++i) H->plan2.push_back(plans[2 * N + i]);
  return ITE_OK;
}

// ------------------------------------------------------------------ MPS setup
std::vector<int> capacities(int N, int d, int chi_cap) {
  std::vector<int> cap(N + 1, 1);
  for (int b = 1; b < N; ++b) {
    long long c = chi_cap;
    long long l = 1, r = 1;
    for (int k = 0; k < b && l < c; ++k) l *= d;
    for (int k = 0; k < N - b && r < c; ++k) r *= d;
    c = std::min(c, std::min(l, r));
    cap[b] = (int)c;
  }
  return cap;
}

ite_status mps_alloc(ite_ctx ctx, int N, int d, int chi_cap, ite_mps* out) {
  ite_mps m = new ite_mps_s();
  m->ctx = ctx;
  m->N = N;
  m->d = d;
  m->chi_cap = chi_cap;
  m->cap = capacities(N, d, chi_cap);
  m->chi.assign(N + 1, 1);
  size_t total = 0;
  std::vector<size_t> off(N);
  bool overflow = false;
  for (int i = 0; i < N && !overflow; ++i) {
    off[i] = total;
    size_t t = 0;
    overflow = __builtin_mul_overflow((size_t)m->cap[i], (size_t)d, &t) ||
               __builtin_mul_overflow(t, (size_t)m->cap[i + 1], &t) ||
               __builtin_add_overflow(total, t, &total);
  }
  if (overflow || total > SIZE_MAX / sizeof(cplx)) {
    delete m;
    return fail(ctx, ITE_ENOMEM, "MPS of this length and capacity exceeds the address space");
  }
  ite_status st = buf_ensure(ctx, m->mem, total * sizeof(cplx));
  if (st != ITE_OK) {
    delete m;
    return st;
  }
  m->site.resize(N);
  for (int i = 0; i < N; ++i) m->site[i] = P<cplx>(m->mem) + off[i];
  *out = m;
  return ITE_OK;
}

void mps_free(ite_mps m) {
  if (!m) return;
  if (m->work_x) mps_free(m->work_x);
  if (m->work_b) mps_free(m->work_b);
  if (m->work_p) mps_free(m->work_p);
  for (ite_mps w : m->work_gl) mps_free(w);
  buf_free(m->ctx, m->mem);
  delete m;
}

ite_status mps_copy_into(ite_ctx ctx, ite_mps src, ite_mps dst) {
  for (int i = 0; i < src->N; ++i)
    CK(vec_copy(dst->site[i], src->site[i], (long long)src->chi[i] * src->d * src->chi[i + 1], ctx->stream));
  dst->chi = src->chi;
  return ITE_OK;
}

void mps_swap(ite_mps a, ite_mps b) {
  std::swap(a->mem, b->mem);
  std::swap(a->site, b->site);
  std::swap(a->chi, b->chi);
}

ite_status ensure_work(ite_ctx ctx, ite_mps psi) {
  if (!psi->work_x) CS(mps_alloc(ctx, psi->N, psi->d, psi->chi_cap, &psi->work_x));
  if (!psi->work_b) CS(mps_alloc(ctx, psi->N, psi->d, psi->chi_cap, &psi->work_b));
  return ITE_OK;
}

// workspace for sweeps over an MPS of these capacities with this MPO
ite_status ensure_workspace(ite_ctx ctx, ite_mpo H, const std::vector<int>& cap, int d, int krylov) {
  const int N = H->N;
  long long nmax = 1, pmax = 1, envs = 0, ovs = 0, site_max = 1;
  for (int i = 0; i + 1 < N; ++i) {
    const long long m = (long long)cap[i] * d, n = (long long)d * cap[i + 2];
    nmax = std::max(nmax, m * n);
    pmax = std::max(pmax, std::min(m, n));
  }
  for (int i = 0; i < N; ++i) {
    site_max = std::max(site_max, (long long)cap[i] * d * cap[i + 1]);
    pmax = std::max(pmax, std::min((long long)cap[i], (long long)d * cap[i + 1]));
  }
  nmax = std::max(nmax, site_max);
  for (int b = 0; b <= N; ++b) {
    envs += (long long)H->D[b] * cap[b] * cap[b];
    ovs += (long long)cap[b] * cap[b];
  }
  const size_t cs = sizeof(cplx);
  const long long tmax = (long long)H->Dmax * nmax;
  CS(buf_ensure(ctx, ctx->ws_X, nmax * cs));
  CS(buf_ensure(ctx, ctx->ws_B, nmax * cs));
  CS(buf_ensure(ctx, ctx->ws_X2, nmax * cs));
  CS(buf_ensure(ctx, ctx->ws_V, (size_t)(krylov + 1) * nmax * cs));
  CS(buf_ensure(ctx, ctx->ws_T1, tmax * cs));
  CS(buf_ensure(ctx, ctx->ws_T2, tmax * cs));
  CS(buf_ensure(ctx, ctx->ws_svdA, nmax * cs));
  CS(buf_ensure(ctx, ctx->ws_svdQ, nmax * cs));
  CS(buf_ensure(ctx, ctx->ws_left, nmax * cs));
  CS(buf_ensure(ctx, ctx->ws_small, small_bytes(pmax)));
  CS(buf_ensure(ctx, ctx->ws_env, (size_t)(2 * envs + 2 * ovs + 16) * cs));
  return ITE_OK;
}

struct EnvSet {
  std::vector<cplx*> LE, RE, LO, RO;
};

// carve the env workspace: operator envs sized D[b] cap_bra[b] cap_ket[b], overlaps cap^2
EnvSet carve_envs(ite_ctx ctx, ite_mpo H, const std::vector<int>& cap) {
  EnvSet e;
  const int N = H->N;
  cplx* p = P<cplx>(ctx->ws_env);
  e.LE.resize(N + 1); e.RE.resize(N + 1); e.LO.resize(N + 1); e.RO.resize(N + 1);
  for (int b = 0; b <= N; ++b) {
    const long long op = (long long)H->D[b] * cap[b] * cap[b], ov = (long long)cap[b] * cap[b];
    e.LE[b] = p; p += op;
    e.RE[b] = p; p += op;
    e.LO[b] = p; p += ov;
    e.RO[b] = p; p += ov;
  }
  return e;
}

ite_status set_one(ite_ctx ctx, cplx* p) {
  const cplx one = C(1);
  CK(cudaMemcpyAsync(p, &one, sizeof(cplx), cudaMemcpyHostToDevice, ctx->stream));
  return ITE_OK;
}

// gauge move: sites N-1..1 right-orthonormal by SVD (weight floor only)
// Gauge move of one site tensor X (m x n, rows = left bond) when it has full
// rank: X = L Q^H by the Householder LQ, right = Q^H (orthonormal rows),
// left = L.  The SVD split that the gauge move is defined by keeps every
// singular value above the weight floor; when sigma_min(X)^2 is certified
// above 1e-20 |X|^2 (four decades over the floor) it keeps all min(m, n) of
// them, and its factors (V^dag, U S) differ from (Q^H, L) only by a unitary on
// the new bond, under which the sweep that follows is covariant.  The
// certificate is 1 / |L1^{-1}|_F^2 <= sigma_min(L1)^2 <= sigma_min(X)^2 for
// the leading triangle L1.  *ok = false (nothing written) when it fails.
constexpr double kGaugeCertRel = 1e-20;
ite_status gauge_lq(ite_ctx ctx, const cplx* X, int m, int n, cplx* left, cplx* right, bool* ok) {
  *ok = false;
  const int k = std::min(m, n);
  CS(buf_ensure(ctx, ctx->ws_svdA, (size_t)m * n * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_small, small_bytes(k)));
  cplx* W = P<cplx>(ctx->ws_svdA);
  cplx* beta = P<cplx>(ctx->ws_small);
  double* refl = reinterpret_cast<double*>(beta + k);
  double* colnorm = refl + 3 * k;
  unsigned int* lqstate = reinterpret_cast<unsigned int*>(ctx->dcounter) + 40;
  double* anorm2 = ctx->dscal + 8;
  double* inv2 = ctx->dscal + 10;
  CK(vec_copy(W, X, (long long)m * n, ctx->stream));
  CK(scaled_norm2(W, (long long)m * n, 1.0, anorm2, ctx->dscal + 16, ctx->stream));
  CK(svd_lq(W, m, n, beta, refl, lqstate, ctx->stream));
  CK(lq_inv_fnorm2(W, beta, n, k, colnorm, inv2, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->d[2], anorm2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->d[3], inv2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->lq_err, lqstate + 4, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  if (ctx->hr->lq_err != 0) return fail(ctx, ITE_ETIMEOUT, "LQ grid barrier wait ran out");
  const double total = ctx->hr->d[2], inv = ctx->hr->d[3];
  if (!(total > 0.0) || !std::isfinite(inv) || !(inv > 0.0) || 1.0 / inv <= kGaugeCertRel * total)
    return ITE_OK;
  CK(lq_left(W, beta, m, n, left, ctx->stream));
  CK(lq_formq(W, refl, n, k, right, lqstate, ctx->stream));
  *ok = true;
  return ITE_OK;
}

ite_status right_canonicalize(ite_ctx ctx, ite_mps x) {
  Scope sc(ctx, P_GAUGE);
  const int d = x->d;
  for (int i = x->N - 1; i >= 1; --i) {
    const int chl = x->chi[i], chr = x->chi[i + 1];
    int r = 0;
    double disc = 0.0;
    cplx* left = P<cplx>(ctx->ws_left);
    bool done = false;
    CS(gauge_lq(ctx, x->site[i], chl, d * chr, left, x->site[i], &done));
    if (done) r = std::min(chl, d * chr);
    else CS(split(ctx, x->site[i], chl, d * chr, 1 << 30, 0.0, false, left, x->site[i], &r, &disc));
    // x_{i-1} <- x_{i-1} (U S)
    const int chll = x->chi[i - 1];
    cplx* T = P<cplx>(ctx->ws_X2);
    CS(gemm(ctx, chll * d, r, chl, x->site[i - 1], chl, 1, false, left, r, 1, false, T, r));
    CK(vec_copy(x->site[i - 1], T, (long long)chll * d * r, ctx->stream));
    x->chi[i] = r;
  }
  return ITE_OK;
}

struct SweepStats {
  double max_disc = 0.0, max_res = 0.0;
  int steps = 0;
};

// Up to `cycles` GMRES(m) cycles, each restarted from the last iterate; a
// cycle that ends before m steps (breakdown, or the relative residual at
// local_tol) ends the solve.  steps: all cycles' Arnoldi steps; res: the
// last relative residual.
ite_status local_solve(ite_ctx ctx, ite_mpo H, int i, int chl, int chr, const cplx* L,
                       const cplx* R, const cplx* B, cplx* X, cplx alpha, cplx c, int m,
                       int cycles, double local_tol, int* steps, double* res) {
  int total = 0;
  double r = 0.0;
  for (int cy = 0; cy < std::max(1, cycles); ++cy) {
    int k = 0;
    CS(gmres_cycle(ctx, H, i, chl, chr, L, R, B, X, alpha, c, m, local_tol, &k, &r));
    total += k;
    if (k < m || (local_tol > 0.0 && r <= local_tol)) break;
  }
  if (steps) *steps = total;
  if (res) *res = r;
  return ITE_OK;
}

// Mixed modes (reading c13 of the local solve): iterative refinement.  The
// residual r = B - (alpha X + c H_eff X) comes from the FP64-class
// contraction; each correction solves (alpha + c H_eff) D = r by one
// GMRES(m) cycle from D = 0 whose matvecs use low-precision operands, then
// X += D.  Stops when |r| <= refine_tol |B| or after refine_max corrections.
// A correction that leaves |r| above half its previous value moves the inner
// matvecs up one precision (bf16 -> tf32 -> FP64-class); blocks too small for
// the tensor-core tiles use the FP64-class matvec throughout.
ite_status local_solve_mixed(ite_ctx ctx, ite_mpo H, int i, int chl, int chr, const cplx* L,
                             const cplx* R, const cplx* B, cplx* X, cplx alpha, cplx c, int m,
                             int precision, int refine_max, double refine_tol, int* steps,
                             double* res) {
  const int d = H->d;
  const long long n = (long long)chl * d * d * chr;
  CS(buf_ensure(ctx, ctx->ws_R, (size_t)n * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_R2, (size_t)n * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_D, (size_t)n * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_Xt, (size_t)n * sizeof(cplx)));
  cplx* r = P<cplx>(ctx->ws_R);        // residual of X
  cplx* rt = P<cplx>(ctx->ws_R2);      // residual of the trial X + D
  cplx* D = P<cplx>(ctx->ws_D);
  cplx* Xt = P<cplx>(ctx->ws_Xt);
  struct LevelGuard {
    ite_ctx c;
    ~LevelGuard() { c->lp_level = -1; }
  } guard{ctx};
  ctx->lp_level = -1;
  const double work = (double)H->D[i] * d * d * chl * (double)chl * chr;
  int level = precision == ITE_MIXED_TF32 ? 1 : 0;
  if (work < kEmuMinWork || chl < 16 || chr < 16) level = 2;
  int prepared = -1, total = 0;
  // out = B - alpha Y - c H_eff Y (FP64-class); its squared norm to slot
  auto residual = [&](const cplx* Y, cplx* out, int slot) -> ite_status {
    ctx->lp_level = -1;
    CS(heff(ctx, H, i, chl, chl, chr, chr, L, R, Y, out, csub(C(0), c), Y, csub(C(0), alpha)));
    CK(vec_axpby(out, B, C(1), C(1), n, ctx->stream));
    CK(vec_norm2(out, n, ctx->dscal + slot, ctx->dscal + 16, nullptr, ctx->stream));
    return ITE_OK;
  };
  CS(residual(X, r, 3));
  CK(vec_norm2(B, n, ctx->dscal + 4, ctx->dscal + 16, nullptr, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->d[0], ctx->dscal + 3, 2 * sizeof(double), cudaMemcpyDeviceToHost,
                     ctx->stream));
  CS(sync(ctx));
  double rho = std::sqrt(ctx->hr->d[0]);
  const double bnorm = std::sqrt(ctx->hr->d[1]);
  if (!std::isfinite(rho) || !std::isfinite(bnorm))
    return fail(ctx, ITE_ESINGULAR, "non-finite residual in the refinement");
  // Each correction solves (alpha + c H_eff) D = r with the inner matvecs at
  // the current level and is kept only if the FP64-class residual of X + D is
  // smaller than that of X: a correction that went astray (an inner solve whose
  // low-precision operator is too far from the true one) is dropped, and the
  // inner matvecs move up one level, as they do when the residual falls by
  // less than half.  At level 2 the inner and outer operators agree, so GMRES
  // cannot raise the residual beyond rounding; a rejection there ends the loop.
  for (int it = 0; it < refine_max && bnorm > 0.0 && rho > refine_tol * bnorm; ++it) {
    if (level < 2 && prepared != level) {
      CS(heff_lp_setup(ctx, H, i, chl, chl, chr, chr, L, R, level));
      prepared = level;
    }
    CK(vec_zero(D, n, ctx->stream));
    ctx->lp_level = level < 2 ? level : -1;
    int k = 0;
    double rr = 0.0;
    CS(gmres_cycle(ctx, H, i, chl, chr, L, R, r, D, alpha, c, m, 0.0, &k, &rr));
    ctx->lp_level = -1;
    total += k;
    ctx->refinements += 1;
    CK(vec_copy(Xt, X, n, ctx->stream));
    CK(vec_axpby(Xt, D, C(1), C(1), n, ctx->stream));
    CS(residual(Xt, rt, 5));
    CK(cudaMemcpyAsync(&ctx->hr->d[2], ctx->dscal + 5, sizeof(double), cudaMemcpyDeviceToHost,
                       ctx->stream));
    CS(sync(ctx));
    const double rho_t = std::sqrt(ctx->hr->d[2]);
    if (!(rho_t < rho)) {
      if (level == 2) break;
      ++level;
      continue;
    }
    if (rho_t > 0.5 * rho && level < 2) ++level;
    CK(vec_copy(X, Xt, n, ctx->stream));
    std::swap(r, rt);
    rho = rho_t;
  }
  if (steps) *steps = total;
  if (res) *res = bnorm > 0.0 ? rho / bnorm : 0.0;
  return ITE_OK;
}

bool mixed_precision(int p) { return p == ITE_MIXED_BF16 || p == ITE_MIXED_TF32; }

// Two-site sweep solving (alpha I + c H) x = b, or (fit mode) x ~ alpha b + beta H b.
ite_status sweep(ite_ctx ctx, ite_mpo H, ite_mps x, ite_mps b, bool fit, cplx alpha, cplx cbeta,
                 int chi_max, double cutoff, const ite_solver_opts& o, SweepStats& stats) {
  const int N = x->N, d = x->d;
  EnvSet e = carve_envs(ctx, H, x->cap);
  // operator envs: bra x, ket (fit ? b : x); overlap envs: bra x, ket b
  ite_mps kop = fit ? b : x;
  CS(set_one(ctx, e.RE[N]));
  CS(set_one(ctx, e.RO[N]));
  for (int i = N - 1; i >= 2; --i) {
    CS(env_right(ctx, H, i, x->chi[i], kop->chi[i], x->chi[i + 1], kop->chi[i + 1], e.RE[i + 1],
                 x->site[i], kop->site[i], e.RE[i]));
    CS(ov_right(ctx, d, x->chi[i], b->chi[i], x->chi[i + 1], b->chi[i + 1], e.RO[i + 1], x->site[i],
                b->site[i], e.RO[i]));
  }
  CS(set_one(ctx, e.LE[0]));
  CS(set_one(ctx, e.LO[0]));
  cplx* X = P<cplx>(ctx->ws_X);
  cplx* B = P<cplx>(ctx->ws_B);
  for (int pass = 0; pass < 2; ++pass) {
    const bool lr = pass == 0;
    for (int k = 0; k < N - 1; ++k) {
      const int i = lr ? k : N - 2 - k;
      const int chl = x->chi[i], chr = x->chi[i + 2];
      const int bl = b->chi[i], bm = b->chi[i + 1], br = b->chi[i + 2];
      if (!fit) {
        CS(merge(ctx, d, chl, x->chi[i + 1], chr, x->site[i], x->site[i + 1], X));
        CS(project(ctx, d, chl, bl, bm, br, chr, e.LO[i], b->site[i], b->site[i + 1], e.RO[i + 2], B));
        int steps = 0;
        double res = 0.0;
        if (mixed_precision(o.precision))
          CS(local_solve_mixed(ctx, H, i, chl, chr, e.LE[i], e.RE[i + 2], B, X, alpha, cbeta,
                               o.krylov_dim, o.precision, o.refine_max, o.refine_tol, &steps, &res));
        else
          CS(local_solve(ctx, H, i, chl, chr, e.LE[i], e.RE[i + 2], B, X, alpha, cbeta, o.krylov_dim,
                         o.max_cycles, o.local_tol, &steps, &res));
        stats.steps += steps;
        stats.max_res = std::max(stats.max_res, res);
      } else {
        // X = alpha * P b + beta * H_eff^{mixed} (b_i b_{i+1})
        CS(project(ctx, d, chl, bl, bm, br, chr, e.LO[i], b->site[i], b->site[i + 1], e.RO[i + 2], B));
        cplx* theta = P<cplx>(ctx->ws_X2);
        CS(merge(ctx, d, bl, bm, br, b->site[i], b->site[i + 1], theta));
        CS(heff(ctx, H, i, chl, bl, br, chr, e.LE[i], e.RE[i + 2], theta, X, cbeta, B, alpha));
      }
      int r = 0;
      double disc = 0.0;
      CS(split(ctx, X, chl * d, d * chr, chi_max, cutoff, lr, x->site[i], x->site[i + 1], &r, &disc));
      x->chi[i + 1] = r;
      stats.max_disc = std::max(stats.max_disc, disc);
      if (lr) {
        CS(env_left(ctx, H, i, x->chi[i], kop->chi[i], x->chi[i + 1], kop->chi[i + 1], e.LE[i],
                    x->site[i], kop->site[i], e.LE[i + 1]));
        CS(ov_left(ctx, d, x->chi[i], b->chi[i], x->chi[i + 1], b->chi[i + 1], e.LO[i], x->site[i],
                   b->site[i], e.LO[i + 1]));
      } else {
        CS(env_right(ctx, H, i + 1, x->chi[i + 1], kop->chi[i + 1], x->chi[i + 2], kop->chi[i + 2],
                     e.RE[i + 2], x->site[i + 1], kop->site[i + 1], e.RE[i + 1]));
        CS(ov_right(ctx, d, x->chi[i + 1], b->chi[i + 1], x->chi[i + 2], b->chi[i + 2], e.RO[i + 2],
                    x->site[i + 1], b->site[i + 1], e.RO[i + 1]));
      }
    }
  }
  return ITE_OK;
}

// Two-site variational fit y ~ sum_t coef[t] targets[t], starting from y
// as given (right-canonical): each local block is the exact projection of
// the combination onto y's current environments, i.e. the sum of the
// targets' two-site blocks, each contracted with its own pair of overlap
// environments.  Forms the Gauss-Legendre step from its partial-fraction
// solutions.
ite_status fit_combination(ite_ctx ctx, ite_mps y, const std::vector<ite_mps>& tg,
                           const std::vector<cplx>& coef, int chi_max, double cutoff, int sweeps,
                           SweepStats& stats) {
  const int N = y->N, d = y->d, T = (int)tg.size();
  long long ovs = 0;
  for (int b = 0; b <= N; ++b) ovs += (long long)y->cap[b] * y->cap[b];
  CS(buf_ensure(ctx, ctx->ws_ovm, (size_t)2 * T * ovs * sizeof(cplx)));
  std::vector<std::vector<cplx*>> LO(T, std::vector<cplx*>(N + 1)), RO(T, std::vector<cplx*>(N + 1));
  {
    cplx* p = P<cplx>(ctx->ws_ovm);
    for (int t = 0; t < T; ++t)
      for (int b = 0; b <= N; ++b) {
        const long long ov = (long long)y->cap[b] * y->cap[b];
        LO[t][b] = p; p += ov;
        RO[t][b] = p; p += ov;
      }
  }
  cplx* X = P<cplx>(ctx->ws_X);
  cplx* B = P<cplx>(ctx->ws_B);
  for (int sw = 0; sw < std::max(1, sweeps); ++sw) {
    for (int t = 0; t < T; ++t) {
      const ite_mps k = tg[t];
      CS(set_one(ctx, RO[t][N]));
      CS(set_one(ctx, LO[t][0]));
      for (int i = N - 1; i >= 2; --i)
        CS(ov_right(ctx, d, y->chi[i], k->chi[i], y->chi[i + 1], k->chi[i + 1], RO[t][i + 1],
                    y->site[i], k->site[i], RO[t][i]));
    }
    for (int pass = 0; pass < 2; ++pass) {
      const bool lr = pass == 0;
      for (int kk = 0; kk < N - 1; ++kk) {
        const int i = lr ? kk : N - 2 - kk;
        const int chl = y->chi[i], chr = y->chi[i + 2];
        const long long n = (long long)chl * d * d * chr;
        CK(vec_zero(X, n, ctx->stream));
        for (int t = 0; t < T; ++t) {
          const ite_mps k = tg[t];
          CS(project(ctx, d, chl, k->chi[i], k->chi[i + 1], k->chi[i + 2], chr, LO[t][i],
                     k->site[i], k->site[i + 1], RO[t][i + 2], B));
          CK(vec_axpby(X, B, coef[t], C(1), n, ctx->stream));
        }
        int r = 0;
        double disc = 0.0;
        CS(split(ctx, X, chl * d, d * chr, chi_max, cutoff, lr, y->site[i], y->site[i + 1], &r, &disc));
        y->chi[i + 1] = r;
        stats.max_disc = std::max(stats.max_disc, disc);
        for (int t = 0; t < T; ++t) {
          const ite_mps k = tg[t];
          if (lr)
            CS(ov_left(ctx, d, y->chi[i], k->chi[i], y->chi[i + 1], k->chi[i + 1], LO[t][i],
                       y->site[i], k->site[i], LO[t][i + 1]));
          else
            CS(ov_right(ctx, d, y->chi[i + 1], k->chi[i + 1], y->chi[i + 2], k->chi[i + 2],
                        RO[t][i + 2], y->site[i + 1], k->site[i + 1], RO[t][i + 1]));
        }
      }
    }
  }
  return ITE_OK;
}

// R_q(z) = P_q(-z) / P_q(z), the (q, q) Pade approximant of e^{-z} (the
// Gauss-Legendre collocation step of the linear ODE), in partial fractions:
// r_inf + sum_j a_j / (z - z_j).  P_q(z) = sum_k (2q-k)! q! / ((2q)! k! (q-k)!)
// z^k; its roots by the Durand-Kerner (Weierstrass) iteration polished by
// Newton steps; a_j = P_q(-z_j) / P_q'(z_j); r_inf = (-1)^q.
struct Cd {
  double re, im;
};
Cd cd_add(Cd a, Cd b) { return {a.re + b.re, a.im + b.im}; }
Cd cd_sub(Cd a, Cd b) { return {a.re - b.re, a.im - b.im}; }
Cd cd_mul(Cd a, Cd b) { return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re}; }
Cd cd_div(Cd a, Cd b) {
  const double den = b.re * b.re + b.im * b.im;
  return {(a.re * b.re + a.im * b.im) / den, (a.im * b.re - a.re * b.im) / den};
}
Cd cd_poly(const std::vector<double>& p, Cd z) {   // p[k] z^k, Horner
  Cd acc{0.0, 0.0};
  for (int k = (int)p.size() - 1; k >= 0; --k) acc = cd_add(cd_mul(acc, z), Cd{p[k], 0.0});
  return acc;
}
bool gl_partial_fractions(int q, std::vector<Cd>& z, std::vector<Cd>& a, double* r_inf) {
  if (q < 1 || q > 8) return false;
  std::vector<double> p(q + 1), pm(q + 1), dp(q);
  auto fact = [](int n) {
    double f = 1.0;
    for (int k = 2; k <= n; ++k) f *= k;
    return f;
  };
  for (int k = 0; k <= q; ++k) {
    p[k] = fact(2 * q - k) * fact(q) / (fact(2 * q) * fact(k) * fact(q - k));
    pm[k] = (k % 2 ? -1.0 : 1.0) * p[k];
  }
  for (int k = 1; k <= q; ++k) dp[k - 1] = k * p[k];
  // monic form for Durand-Kerner
  std::vector<double> mon(q + 1);
  for (int k = 0; k <= q; ++k) mon[k] = p[k] / p[q];
  z.assign(q, Cd{0.0, 0.0});
  Cd seed{0.4, 0.9};
  Cd w{1.0, 0.0};
  for (int j = 0; j < q; ++j) {
    z[j] = cd_mul(w, Cd{4.0, 0.0});
    w = cd_mul(w, seed);
  }
  for (int it = 0; it < 500; ++it) {
    double change = 0.0;
    for (int j = 0; j < q; ++j) {
      Cd den{1.0, 0.0};
      for (int k = 0; k < q; ++k)
        if (k != j) den = cd_mul(den, cd_sub(z[j], z[k]));
      const Cd step = cd_div(cd_poly(mon, z[j]), den);
      z[j] = cd_sub(z[j], step);
      change = std::max(change, std::hypot(step.re, step.im));
    }
    if (change < 1e-15) break;
  }
  for (int j = 0; j < q; ++j)
    for (int it = 0; it < 3; ++it) z[j] = cd_sub(z[j], cd_div(cd_poly(p, z[j]), cd_poly(dp, z[j])));
  a.resize(q);
  for (int j = 0; j < q; ++j) a[j] = cd_div(cd_poly(pm, z[j]), cd_poly(dp, z[j]));
  *r_inf = q % 2 ? -1.0 : 1.0;
  for (int j = 0; j < q; ++j)
    if (!std::isfinite(z[j].re) || !std::isfinite(z[j].im)) return false;
  return true;
}

}  // namespace

// ================================================================== C ABI
extern "C" {

void ite_solver_opts_default(ite_solver_opts* o) {
  if (!o) return;
  o->krylov_dim = 10;
  o->max_cycles = 1;
  o->sweeps = 1;
  o->local_tol = 0.0;
  o->sweep_tol = 0.0;
  o->fit_sweeps = 1;
  o->precision = ITE_FP64;
  o->refine_max = 10;
  o->refine_tol = 1e-10;
}

ite_status ite_ctx_create(int device, void* stream, ite_alloc_fn alloc, ite_free_fn release,
                          void* alloc_user, ite_ctx* out) {
  if (!out) return ITE_EINVAL;
  *out = nullptr;
  if ((alloc == nullptr) != (release == nullptr)) return ITE_EINVAL;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return ITE_ECUDA;
  }
  if (cudaSetDevice(device) != cudaSuccess) return ITE_ECUDA;
  ite_ctx ctx = new ite_ctx_s();
  ctx->device = device;
  ctx->stream = (cudaStream_t)stream;
  ctx->alloc = alloc;
  ctx->release = release;
  ctx->user = alloc_user;
  ctx->gm = (GmresState*)dev_alloc(ctx, sizeof(GmresState));
  ctx->dscal = (double*)dev_alloc(ctx, 64 * sizeof(double) + kPartialSlots * sizeof(double));
  ctx->dcplx = (cplx*)dev_alloc(ctx, 512 * sizeof(cplx));
  ctx->partial = (cplx*)dev_alloc(ctx, (size_t)kPartialSlots * sizeof(cplx));
  ctx->dcounter = (int*)dev_alloc(ctx, 64 * sizeof(int));
  if (cudaMallocHost((void**)&ctx->hr, sizeof(HostRead)) != cudaSuccess) ctx->hr = nullptr;
  if (!ctx->gm || !ctx->dscal || !ctx->dcplx || !ctx->partial || !ctx->dcounter || !ctx->hr) {
    ite_ctx_destroy(ctx);
    return ITE_ENOMEM;
  }
  // error words and device states start cleared
  if (cudaMemsetAsync(ctx->dcounter, 0, 64 * sizeof(int), ctx->stream) != cudaSuccess) {
    ite_ctx_destroy(ctx);
    return ITE_ECUDA;
  }
  *out = ctx;
  return ITE_OK;
}

ite_status ite_ctx_set_stream(ite_ctx ctx, void* stream) {
  if (!ctx) return ITE_EINVAL;
  ctx->stream = (cudaStream_t)stream;
  return ITE_OK;
}

void ite_ctx_destroy(ite_ctx ctx) {
  if (!ctx) return;
  for (size_t k = 0; k < ctx->children.size(); ++k) {
    ite_ctx_destroy(ctx->children[k]);
    cudaStreamDestroy(ctx->child_streams[k]);
  }
  cudaStreamSynchronize(ctx->stream);
  Buf* bufs[] = {&ctx->ws_X, &ctx->ws_B, &ctx->ws_X2, &ctx->ws_V, &ctx->ws_T1, &ctx->ws_T2,
                 &ctx->ws_svdA, &ctx->ws_svdQ, &ctx->ws_left, &ctx->ws_small, &ctx->ws_env,
                 &ctx->ws_emu, &ctx->ws_ovm, &ctx->ws_lpops, &ctx->ws_lpscr, &ctx->ws_R,
                 &ctx->ws_D, &ctx->ws_R2, &ctx->ws_Xt};
  for (Buf* b : bufs) buf_free(ctx, *b);
  dev_free(ctx, ctx->gm, sizeof(GmresState));
  dev_free(ctx, ctx->dscal, 64 * sizeof(double) + kPartialSlots * sizeof(double));
  dev_free(ctx, ctx->dcplx, 512 * sizeof(cplx));
  dev_free(ctx, ctx->partial, (size_t)kPartialSlots * sizeof(cplx));
  dev_free(ctx, ctx->dcounter, 64 * sizeof(int));
  if (ctx->hr) cudaFreeHost(ctx->hr);
  for (cudaEvent_t e : ctx->evpool) cudaEventDestroy(e);
  if (ctx->group_state) dev_free(ctx, ctx->group_state, 24 * sizeof(unsigned int));
  if (ctx->group_ready) cudaEventDestroy(ctx->group_ready);
  if (ctx->group_done) cudaEventDestroy(ctx->group_done);
  delete ctx;
}

const char* ite_last_error(ite_ctx ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t ite_ctx_device_bytes(ite_ctx ctx) { return ctx ? ctx->bytes : 0; }

unsigned long long ite_kernel_launches(void) { return ite::launches(); }

ite_status ite_svd_stats(ite_ctx ctx, long long* splits, long long* sweeps_total, int* sweeps_max,
                         double fp64_flops[2]) {
  if (!ctx) return ITE_EINVAL;
  if (splits) *splits = ctx->jacobi_splits;
  if (sweeps_total) *sweeps_total = ctx->jacobi_sweeps_total;
  if (sweeps_max) *sweeps_max = ctx->jacobi_sweeps_max;
  if (fp64_flops) {
    fp64_flops[0] = ctx->lq_flops;
    fp64_flops[1] = ctx->jacobi_flops;
    fp64_flops[2] = ctx->svd_alg_flops;
  }
  ctx->jacobi_splits = ctx->jacobi_sweeps_total = 0;
  ctx->jacobi_sweeps_max = 0;
  ctx->jacobi_flops = ctx->lq_flops = ctx->svd_alg_flops = 0.0;
  return ITE_OK;
}

ite_status ite_profile_start(ite_ctx ctx) {
  if (!ctx) return ITE_EINVAL;
  ctx->prof = true;
  ctx->evused = 0;
  ctx->recs.clear();
  return ITE_OK;
}

ite_status ite_profile_stop(ite_ctx ctx, double ms[ITE_PROFILE_SLOTS],
                            double flops[ITE_PROFILE_SLOTS], long long counts[ITE_PROFILE_SLOTS]) {
  if (!ctx) return ITE_EINVAL;
  ctx->prof = false;
  CK(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < ITE_PROFILE_SLOTS; ++k) {
    if (ms) ms[k] = 0.0;
    if (flops) flops[k] = 0.0;
    if (counts) counts[k] = 0;
  }
  for (const auto& r : ctx->recs) {
    float t = 0.0f;
    CK(cudaEventElapsedTime(&t, ctx->evpool[r.e0], ctx->evpool[r.e1]));
    if (r.cat < 0 || r.cat >= ITE_PROFILE_SLOTS) continue;
    if (ms) ms[r.cat] += t;
    if (flops) flops[r.cat] += r.flops;
    if (counts) counts[r.cat] += 1;
  }
  ctx->recs.clear();
  ctx->evused = 0;
  return ITE_OK;
}

}  // extern "C"

// ================================================================== step, measurements
namespace {

ite_status validate_pair(ite_ctx ctx, ite_mpo H, ite_mps psi) {
  if (!ctx || !H || !psi) return ITE_EINVAL;
  if (H->N != psi->N || H->d != psi->d) return fail(ctx, ITE_EINVAL, "MPO and MPS do not match");
  return ITE_OK;
}

ite_status read_cplx(ite_ctx ctx, const cplx* dev, cplx* host) {
  CK(cudaMemcpyAsync(&ctx->hr->z[0], dev, sizeof(cplx), cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  *host = ctx->hr->z[0];
  return ITE_OK;
}

std::vector<int> max_caps(ite_mps a, ite_mps b) {
  std::vector<int> c(a->cap);
  for (size_t k = 0; k < c.size(); ++k) c[k] = std::max(c[k], b->cap[k]);
  return c;
}

// <bra|ket> through the overlap-environment chain; optional one-site operators
// on the ket sites (ops[i] device d x d or nullptr)
ite_status overlap_impl(ite_ctx ctx, ite_mps bra, ite_mps ket, const std::vector<const cplx*>* ops,
                        cplx* out) {
  const int N = bra->N, d = bra->d;
  std::vector<int> cap = max_caps(bra, ket);
  // workspace: envs of cap^2, T1 of cap*d*cap, a temp site
  long long site_max = 1, ovs = 0;
  for (int i = 0; i < N; ++i) site_max = std::max(site_max, (long long)cap[i] * d * cap[i + 1]);
  for (int b = 0; b <= N; ++b) ovs += (long long)cap[b] * cap[b];
  CS(buf_ensure(ctx, ctx->ws_T1, site_max * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_X2, site_max * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_B, (size_t)(2 * ovs + 4) * sizeof(cplx)));
  cplx* envp = P<cplx>(ctx->ws_B);
  std::vector<cplx*> LO(N + 1);
  for (int b = 0; b <= N; ++b) {
    LO[b] = envp;
    envp += (long long)cap[b] * cap[b];
  }
  CS(set_one(ctx, LO[0]));
  for (int i = 0; i < N; ++i) {
    const cplx* k = ket->site[i];
    if (ops && (*ops)[i]) {
      CK(apply_site_op((*ops)[i], k, P<cplx>(ctx->ws_X2), ket->chi[i], d, ket->chi[i + 1], ctx->stream));
      k = P<cplx>(ctx->ws_X2);
    }
    CS(ov_left(ctx, d, bra->chi[i], ket->chi[i], bra->chi[i + 1], ket->chi[i + 1], LO[i],
               bra->site[i], k, LO[i + 1]));
  }
  return read_cplx(ctx, LO[N], out);
}

ite_status energy_impl(ite_ctx ctx, ite_mpo H, ite_mps psi, double* E) {
  const int N = psi->N;
  CS(ensure_workspace(ctx, H, psi->cap, psi->d, 1));
  EnvSet e = carve_envs(ctx, H, psi->cap);
  CS(set_one(ctx, e.LE[0]));
  for (int i = 0; i < N; ++i)
    CS(env_left(ctx, H, i, psi->chi[i], psi->chi[i], psi->chi[i + 1], psi->chi[i + 1], e.LE[i],
                psi->site[i], psi->site[i], e.LE[i + 1]));
  cplx num;
  CS(read_cplx(ctx, e.LE[N], &num));
  cplx den;
  CS(overlap_impl(ctx, psi, psi, nullptr, &den));
  if (!(den.x > 0.0)) return fail(ctx, ITE_ESINGULAR, "zero-norm state");
  *E = num.x / den.x;
  if (!std::isfinite(*E)) return fail(ctx, ITE_ESINGULAR, "non-finite energy");
  return ITE_OK;
}

ite_status normalize_impl(ite_ctx ctx, ite_mps psi) {
  cplx nn;
  CS(overlap_impl(ctx, psi, psi, nullptr, &nn));
  if (!(nn.x > 0.0) || !std::isfinite(nn.x)) return fail(ctx, ITE_ESINGULAR, "zero or non-finite norm");
  CK(vec_axpby(psi->site[0], psi->site[0], C(0), C(1.0 / std::sqrt(nn.x)),
               (long long)psi->chi[0] * psi->d * psi->chi[1], ctx->stream));
  return ITE_OK;
}

// Stream-ordered allocation on a child context's own stream.
void* child_alloc(size_t bytes, void* user) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, static_cast<cudaStream_t>(user)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void child_free(void* p, size_t, void* user) { cudaFreeAsync(p, static_cast<cudaStream_t>(user)); }

ite_status ensure_children(ite_ctx ctx, int n) {
  while ((int)ctx->children.size() < n) {
    cudaStream_t st = nullptr;
    CK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
    ite_ctx c = nullptr;
    const ite_status r = ite_ctx_create(ctx->device, st, child_alloc, child_free, st, &c);
    if (r != ITE_OK) {
      cudaStreamDestroy(st);
      return fail(ctx, r, "cannot create a child context");
    }
    ctx->children.push_back(c);
    ctx->child_streams.push_back(st);
  }
  return ITE_OK;
}

ite_status step_impl(ite_ctx ctx, ite_mpo H, ite_mps psi, double dtau, int scheme, double shift,
                     int chi_max, double cutoff, const ite_solver_opts& o, ite_step_info* info) {
  CS(validate_pair(ctx, H, psi));
  if (!(dtau > 0.0) || !std::isfinite(dtau) || !std::isfinite(shift) || !(cutoff >= 0.0) ||
      chi_max < 1 || chi_max > psi->chi_cap || o.krylov_dim < 1 || o.krylov_dim > kMaxKrylov ||
      o.sweeps < 1 || o.fit_sweeps < 1 ||
      (scheme != ITE_BACKWARD_EULER && scheme != ITE_TRAPEZOID &&
       scheme != ITE_GAUSS_LEGENDRE_2 && scheme != ITE_GAUSS_LEGENDRE_3 &&
       scheme != ITE_FORWARD_EULER && scheme != ITE_HEUN) ||
      (o.precision != ITE_FP64 && o.precision != ITE_FP64_TC && !mixed_precision(o.precision)) ||
      (mixed_precision(o.precision) && (o.refine_max < 0 || !(o.refine_tol >= 0.0))) || psi->N < 2)
    return fail(ctx, ITE_EINVAL, "invalid step arguments");
  CS(ensure_work(ctx, psi));
  CS(ensure_workspace(ctx, H, psi->cap, psi->d, o.krylov_dim));
  Scope step_scope(ctx, P_STEP);
  struct ModeGuard {
    ite_ctx c;
    ~ModeGuard() { c->gemm_mode = 0; }
  } mode_guard{ctx};
  ctx->gemm_mode = o.precision == ITE_FP64 ? 0 : 1;
  CK(cudaMemsetAsync(reinterpret_cast<int*>(ctx->dcounter) + 10, 0, sizeof(int), ctx->stream));
  SweepStats st;
  ite_mps x = psi->work_x;
  if (o.sweep_tol > 0.0 && !psi->work_p) CS(mps_alloc(ctx, psi->N, psi->d, psi->chi_cap, &psi->work_p));
  // sweeps of the linear solve (1 - c s) xx + c H xx = b from the guess in xx
  auto solve = [&](ite_mps xx, ite_mps b, cplx c) -> ite_status {
    const cplx alpha = csub(C(1), cscale(c, shift));
    for (int s = 0; s < o.sweeps; ++s) {
      const bool check = o.sweep_tol > 0.0 && s > 0;
      if (check) CS(mps_copy_into(ctx, xx, psi->work_p));
      CS(sweep(ctx, H, xx, b, false, alpha, c, chi_max, cutoff, o, st));
      if (check) {
        cplx ab, aa, bb;
        CS(overlap_impl(ctx, psi->work_p, xx, nullptr, &ab));
        CS(overlap_impl(ctx, psi->work_p, psi->work_p, nullptr, &aa));
        CS(overlap_impl(ctx, xx, xx, nullptr, &bb));
        const double ov = std::hypot(ab.x, ab.y) / std::sqrt(aa.x * bb.x);
        if (1.0 - ov < o.sweep_tol) break;
      }
    }
    return ITE_OK;
  };
  // right operator environments of x, for the energy below (the fits keep
  // only overlap or mixed environments)
  auto right_envs_of_x = [&]() -> ite_status {
    EnvSet e = carve_envs(ctx, H, x->cap);
    const int N = x->N;
    CS(set_one(ctx, e.RE[N]));
    for (int i = N - 1; i >= 1; --i)
      CS(env_right(ctx, H, i, x->chi[i], x->chi[i], x->chi[i + 1], x->chi[i + 1], e.RE[i + 1],
                   x->site[i], x->site[i], e.RE[i]));
    return ITE_OK;
  };
  if (scheme == ITE_FORWARD_EULER || scheme == ITE_HEUN) {
    // explicit steps: y = (I - dtau H') psi by a two-site fit (forward
    // Euler); Heun then fits y2 = (I - dtau H') y and the corrector
    // psi_k = psi / 2 + y2 / 2
    const cplx a = C(1.0 + dtau * shift), b = C(-dtau);
    ite_mps y = scheme == ITE_HEUN ? psi->work_b : x;
    CS(mps_copy_into(ctx, psi, y));
    CS(right_canonicalize(ctx, y));
    for (int f = 0; f < o.fit_sweeps; ++f) CS(sweep(ctx, H, y, psi, true, a, b, chi_max, cutoff, o, st));
    if (scheme == ITE_HEUN) {
      if (psi->work_gl.empty()) {
        ite_mps w = nullptr;
        CS(mps_alloc(ctx, psi->N, psi->d, psi->chi_cap, &w));
        psi->work_gl.push_back(w);
      }
      ite_mps y2 = psi->work_gl[0];
      CS(mps_copy_into(ctx, y, y2));
      CS(right_canonicalize(ctx, y2));
      for (int f = 0; f < o.fit_sweeps; ++f) CS(sweep(ctx, H, y2, y, true, a, b, chi_max, cutoff, o, st));
      CS(mps_copy_into(ctx, psi, x));
      CS(right_canonicalize(ctx, x));
      CS(fit_combination(ctx, x, {psi, y2}, {C(0.5), C(0.5)}, chi_max, cutoff, o.fit_sweeps, st));
    }
    CS(right_envs_of_x());
  } else if (scheme == ITE_GAUSS_LEGENDRE_2 || scheme == ITE_GAUSS_LEGENDRE_3) {
    // psi_k = r_inf psi + sum_j w_j x_j, (I + c_j H') x_j = psi, c_j = -dtau / z_j,
    // w_j = -a_j / z_j, from R_q(z) = r_inf + sum_j a_j / (z - z_j)
    const int q = scheme == ITE_GAUSS_LEGENDRE_2 ? 2 : 3;
    std::vector<Cd> zp, ap;
    double r_inf = 0.0;
    if (!gl_partial_fractions(q, zp, ap, &r_inf)) return fail(ctx, ITE_EINVAL, "no Pade poles");
    while ((int)psi->work_gl.size() < q) {
      ite_mps w = nullptr;
      CS(mps_alloc(ctx, psi->N, psi->d, psi->chi_cap, &w));
      psi->work_gl.push_back(w);
    }
    std::vector<ite_mps> targets{psi};
    std::vector<cplx> coefs{C(r_inf)};
    std::vector<cplx> cs(q);
    for (int j = 0; j < q; ++j) {
      ite_mps xj = psi->work_gl[j];
      CS(mps_copy_into(ctx, psi, xj));
      CS(right_canonicalize(ctx, xj));
      const Cd cj = cd_div(Cd{-dtau, 0.0}, zp[j]);
      cs[j] = C(cj.re, cj.im);
      const Cd wj = cd_div(Cd{-ap[j].re, -ap[j].im}, zp[j]);
      targets.push_back(xj);
      coefs.push_back(C(wj.re, wj.im));
    }
    if (o.sweep_tol > 0.0) {
      // the convergence check shares one scratch MPS: solve one at a time
      for (int j = 0; j < q; ++j) CS(solve(psi->work_gl[j], psi, cs[j]));
    } else {
      // The q solves are independent: each runs in a child context (own
      // stream, own workspaces) from its own host thread, so that their
      // kernels overlap on the GPU; they only read psi and the MPO.
      CS(ensure_children(ctx, q));
      CS(sync(ctx));
      std::vector<SweepStats> cst(q);
      std::vector<ite_status> cres(q, ITE_OK);
      std::vector<std::thread> th;
      for (int j = 0; j < q; ++j) {
        th.emplace_back([&, j] {
          ite_ctx cc = ctx->children[j];
          ite_status r = cudaSetDevice(ctx->device) == cudaSuccess ? ITE_OK : ITE_ECUDA;
          cc->gemm_mode = ctx->gemm_mode;
          if (r == ITE_OK &&
              cudaMemsetAsync(reinterpret_cast<int*>(cc->dcounter) + 10, 0, sizeof(int), cc->stream) !=
                  cudaSuccess)
            r = ITE_ECUDA;
          if (r == ITE_OK) r = ensure_workspace(cc, H, psi->cap, psi->d, o.krylov_dim);
          const cplx alpha = csub(C(1), cscale(cs[j], shift));
          for (int sw = 0; sw < o.sweeps && r == ITE_OK; ++sw)
            r = sweep(cc, H, psi->work_gl[j], psi, false, alpha, cs[j], chi_max, cutoff, o, cst[j]);
          if (r == ITE_OK) r = sync(cc);
          cc->gemm_mode = 0;
          cres[j] = r;
        });
      }
      for (auto& t : th) t.join();
      for (int j = 0; j < q; ++j) {
        ite_ctx cc = ctx->children[j];
        if (cres[j] != ITE_OK) return fail(ctx, cres[j], cc->err);
        st.steps += cst[j].steps;
        st.max_res = std::max(st.max_res, cst[j].max_res);
        st.max_disc = std::max(st.max_disc, cst[j].max_disc);
        ctx->jacobi_sweeps_total += cc->jacobi_sweeps_total;
        ctx->jacobi_splits += cc->jacobi_splits;
        ctx->jacobi_sweeps_max = std::max(ctx->jacobi_sweeps_max, cc->jacobi_sweeps_max);
        ctx->jacobi_flops += cc->jacobi_flops;
        ctx->lq_flops += cc->lq_flops;
        ctx->svd_alg_flops += cc->svd_alg_flops;
        cc->jacobi_sweeps_total = cc->jacobi_splits = 0;
        cc->jacobi_sweeps_max = 0;
        cc->jacobi_flops = cc->lq_flops = cc->svd_alg_flops = 0.0;
      }
    }
    CS(mps_copy_into(ctx, psi, x));
    CS(right_canonicalize(ctx, x));
    CS(fit_combination(ctx, x, targets, coefs, chi_max, cutoff, o.fit_sweeps, st));
    CS(right_envs_of_x());
  } else {
    ite_mps bm = psi;
    double c;
    if (scheme == ITE_BACKWARD_EULER) {
      c = dtau;
    } else {
      c = 0.5 * dtau;
      bm = psi->work_b;
      CS(mps_copy_into(ctx, psi, bm));
      CS(right_canonicalize(ctx, bm));
      for (int f = 0; f < o.fit_sweeps; ++f)
        CS(sweep(ctx, H, bm, psi, true, C(1.0 + c * shift), C(-c), chi_max, cutoff, o, st));
    }
    CS(mps_copy_into(ctx, bm, x));
    CS(right_canonicalize(ctx, x));
    CS(solve(x, bm, C(c)));
  }
  // normalise the centre tensor (site 0; the rest is right-orthonormal)
  const long long n0 = (long long)x->chi[0] * x->d * x->chi[1];
  CK(vec_norm2(x->site[0], n0, ctx->dscal + 2, ctx->dscal + 16, nullptr, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->d[1], ctx->dscal + 2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->steps, reinterpret_cast<int*>(ctx->dcounter) + 10, sizeof(int),
                     cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  if (ctx->hr->steps != 0) return fail(ctx, ITE_ETIMEOUT, "tensor-core GEMM wait ran out");
  const double nrm = std::sqrt(ctx->hr->d[1]);
  if (!(nrm > 0.0) || !std::isfinite(nrm)) return fail(ctx, ITE_ESINGULAR, "solution has zero or non-finite norm");
  CK(vec_axpby(x->site[0], x->site[0], C(0), C(1.0 / nrm), n0, ctx->stream));
  // energy from the centre: L_1 from site 0, then tr(L_1 R_1)
  EnvSet e = carve_envs(ctx, H, x->cap);
  CS(set_one(ctx, e.LE[0]));
  CS(env_left(ctx, H, 0, 1, 1, x->chi[1], x->chi[1], e.LE[0], x->site[0], x->site[0], e.LE[1]));
  CK(env_trace(e.LE[1], e.RE[1], H->D[1], x->chi[1], x->chi[1], ctx->dcplx, ctx->partial, ctx->stream));
  cplx E;
  CS(read_cplx(ctx, ctx->dcplx, &E));
  if (!std::isfinite(E.x)) return fail(ctx, ITE_ESINGULAR, "non-finite energy");
  mps_swap(psi, x);
  if (info) {
    info->energy = E.x;
    info->norm_before = nrm;
    info->max_discarded_weight = st.max_disc;
    info->max_local_residual = st.max_res;
    info->shift = shift;
    info->max_chi = *std::max_element(psi->chi.begin(), psi->chi.end());
    info->gmres_steps = st.steps;
    info->status = ITE_OK;
  }
  return ITE_OK;
}

void grid_geometric_impl(double a, double b, int K, double* nodes) {
  nodes[0] = 0.0;
  if (K == 1) {
    nodes[1] = b;
    return;
  }
  for (int k = 1; k <= K; ++k) nodes[k] = a * std::pow(b / a, (double)(k - 1) / (K - 1));
}

void grid_panels_impl(double tau_max, int Pn, int n, double* nodes) {
  std::vector<double> ends(Pn + 1);
  ends[0] = 0.0;
  for (int j = 1; j <= Pn; ++j) ends[j] = tau_max / std::ldexp(1.0, Pn - j);
  int k = 0;
  nodes[k++] = 0.0;
  for (int p = 0; p < Pn; ++p)
    for (int i = 1; i <= n; ++i) nodes[k++] = ends[p] + (ends[p + 1] - ends[p]) * i / n;
}

ite_status evolve_impl(ite_ctx ctx, ite_mpo H, ite_mps psi, const std::vector<double>& nodes,
                       int scheme, int shift_mode, double shift0, int chi_max, double cutoff,
                       const ite_solver_opts& o, ite_step_info* per_step) {
  CS(validate_pair(ctx, H, psi));
  if (shift_mode != ITE_SHIFT_FIXED && shift_mode != ITE_SHIFT_CURRENT_ENERGY)
    return fail(ctx, ITE_EINVAL, "invalid shift mode");
  CS(normalize_impl(ctx, psi));
  double s = shift0;
  if (shift_mode == ITE_SHIFT_CURRENT_ENERGY) CS(energy_impl(ctx, H, psi, &s));
  for (size_t k = 1; k < nodes.size(); ++k) {
    ite_step_info info;
    std::memset(&info, 0, sizeof(info));
    ite_status st = step_impl(ctx, H, psi, nodes[k] - nodes[k - 1], scheme, s, chi_max, cutoff, o, &info);
    info.status = st;
    if (per_step) per_step[k - 1] = info;
    if (st != ITE_OK) return st;
    if (shift_mode == ITE_SHIFT_CURRENT_ENERGY) s = info.energy;
  }
  return ITE_OK;
}

ite_status upload_ops(ite_ctx ctx, int d, const double* host, int slot, const cplx** dev) {
  if (!host) {
    *dev = nullptr;
    return ITE_OK;
  }
  cplx* p = ctx->dcplx + 16 + slot * 64;
  CK(cudaMemcpyAsync(p, host, sizeof(cplx) * d * d, cudaMemcpyHostToDevice, ctx->stream));
  *dev = p;
  return ITE_OK;
}

}  // namespace

// ================================================================== C ABI (objects, steps)
extern "C" {

ite_status ite_mpo_create(ite_ctx ctx, int N, const int* d, const int* D, const double* W,
                          ite_mpo* out) {
  if (!ctx || !out || !d || !D || !W || N < 1) return ITE_EINVAL;
  *out = nullptr;
  for (int i = 0; i < N; ++i)
    if (d[i] != d[0] || d[i] < 1 || d[i] > 16) return fail(ctx, ITE_EINVAL, "site dimensions must be equal and <= 16");
  if (D[0] != 1 || D[N] != 1) return fail(ctx, ITE_EINVAL, "MPO boundary bond dimensions must be 1");
  for (int b = 0; b <= N; ++b)
    if (D[b] < 1 || D[b] > 32) return fail(ctx, ITE_EINVAL, "MPO bond dimension out of range");
  ite_mpo H = new ite_mpo_s();
  H->ctx = ctx;
  H->N = N;
  H->d = d[0];
  H->D.assign(D, D + N + 1);
  for (int i = 0; i < N; ++i)
    if ((long long)H->D[i] * H->d * H->d > 128 || (long long)H->D[i + 1] * H->d * H->d > 128) {
      delete H;
      return fail(ctx, ITE_EINVAL, "D*d^2 above 128 is not supported");
    }
  const double* p = W;
  H->Wh.resize(N);
  for (int i = 0; i < N; ++i) {
    const size_t cnt = (size_t)H->D[i] * H->d * H->d * H->D[i + 1];
    H->Wh[i].resize(cnt);
    for (size_t k = 0; k < cnt; ++k) H->Wh[i][k] = cmake(p[2 * k], p[2 * k + 1]);
    p += 2 * cnt;
  }
  ite_status st = mpo_finish(H);
  if (st != ITE_OK) {
    ite_mpo_destroy(H);
    return st;
  }
  *out = H;
  return ITE_OK;
}

// Heisenberg chain as a finite-state machine: channel 0 = nothing placed,
// 1/2/3 = S+ / S- / Sz placed on the previous site, 4 = term complete.
ite_status ite_mpo_create_heisenberg(ite_ctx ctx, int N, double J, double Jz, ite_mpo* out) {
  if (!ctx || !out || N < 2) return ITE_EINVAL;
  const int d = 2, Db = 5;
  // local operators [s'][s], index 0 = up
  const double Id[2][2] = {{1, 0}, {0, 1}};
  const double Sp[2][2] = {{0, 1}, {0, 0}};
  const double Sm[2][2] = {{0, 0}, {1, 0}};
  const double Sz[2][2] = {{0.5, 0}, {0, -0.5}};
  std::vector<double> bulk((size_t)Db * d * d * Db * 2, 0.0);
  auto put = [&](int w, int w2, const double (*op)[2], double f) {
    for (int sp = 0; sp < 2; ++sp)
      for (int s = 0; s < 2; ++s) bulk[((((size_t)w * d + sp) * d + s) * Db + w2) * 2] += f * op[sp][s];
  };
  put(0, 0, Id, 1.0);
  put(0, 1, Sp, 1.0);
  put(0, 2, Sm, 1.0);
  put(0, 3, Sz, 1.0);
  put(1, 4, Sm, 0.5 * J);
  put(2, 4, Sp, 0.5 * J);
  put(3, 4, Sz, Jz);
  put(4, 4, Id, 1.0);
  std::vector<int> dv(N, d), Dv(N + 1, Db);
  Dv[0] = Dv[N] = 1;
  std::vector<double> W;
  for (int i = 0; i < N; ++i) {
    const int w0 = (i == 0) ? 0 : 0, wn = (i == 0) ? 1 : Db;
    const int v0 = (i == N - 1) ? Db - 1 : 0, vn = (i == N - 1) ? Db : Db;
    for (int w = w0; w < wn; ++w)
      for (int sp = 0; sp < d; ++sp)
        for (int s = 0; s < d; ++s)
          for (int w2 = v0; w2 < vn; ++w2) {
            const size_t k = (((size_t)w * d + sp) * d + s) * Db + w2;
            W.push_back(bulk[2 * k]);
            W.push_back(bulk[2 * k + 1]);
          }
  }
  return ite_mpo_create(ctx, N, dv.data(), Dv.data(), W.data(), out);
}

// Anderson impurity, star geometry.  Local basis index n_up + 2 n_down.
// Channels: 0 start, 1 d^dag_up F, 2 d^dag_down F, 3 F d_up, 4 F d_down, 5 done.
ite_status ite_mpo_create_anderson(ite_ctx ctx, int n_bath, const double* eps, const double* V,
                                   double U, double eps_d, ite_mpo* out) {
  if (!ctx || !out || n_bath < 1 || !eps || !V) return ITE_EINVAL;
  const int d = 4, Db = 6, N = n_bath + 1;
  typedef std::vector<double> M4;  // 4x4 real, [s'][s]
  auto zero = []() { return M4(16, 0.0); };
  M4 I = zero(), F = zero(), cu = zero(), cd = zero(), nu = zero(), nd = zero();
  for (int k = 0; k < 4; ++k) I[k * 4 + k] = 1.0;
  F[0] = 1; F[5] = -1; F[10] = -1; F[15] = 1;
  cu[0 * 4 + 1] = 1.0; cu[2 * 4 + 3] = 1.0;      // c_up |up> = |0>, c_up |ud> = |dn>
  cd[0 * 4 + 2] = 1.0; cd[1 * 4 + 3] = -1.0;     // c_dn |dn> = |0>, c_dn |ud> = -|up>
  nu[5] = 1; nu[15] = 1;
  nd[10] = 1; nd[15] = 1;
  auto mul = [](const M4& a, const M4& b) {
    M4 r(16, 0.0);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j)
        for (int k = 0; k < 4; ++k) r[i * 4 + j] += a[i * 4 + k] * b[k * 4 + j];
    return r;
  };
  auto tr = [](const M4& a) {
    M4 r(16, 0.0);
    for (int i = 0; i < 4; ++i)
      for (int j = 0; j < 4; ++j) r[i * 4 + j] = a[j * 4 + i];
    return r;
  };
  std::vector<int> dv(N, d), Dv(N + 1, Db);
  Dv[0] = Dv[N] = 1;
  std::vector<double> W;
  for (int i = 0; i < N; ++i) {
    std::vector<double> bulk((size_t)Db * 16 * Db, 0.0);
    auto put = [&](int w, int w2, const M4& op, double f) {
      for (int sp = 0; sp < 4; ++sp)
        for (int s = 0; s < 4; ++s) bulk[(((size_t)w * 4 + sp) * 4 + s) * Db + w2] += f * op[sp * 4 + s];
    };
    if (i == 0) {
      put(0, 0, I, 1.0);
      put(0, 1, mul(tr(cu), F), 1.0);
      put(0, 2, mul(tr(cd), F), 1.0);
      put(0, 3, mul(F, cu), 1.0);
      put(0, 4, mul(F, cd), 1.0);
      M4 onsite = zero();
      for (int k = 0; k < 16; ++k) onsite[k] = eps_d * (nu[k] + nd[k]);
      M4 nn = mul(nu, nd);
      for (int k = 0; k < 16; ++k) onsite[k] += U * nn[k];
      put(0, 5, onsite, 1.0);
    } else {
      const double e = eps[i - 1], v = V[i - 1];
      put(0, 0, I, 1.0);
      M4 n = zero();
      for (int k = 0; k < 16; ++k) n[k] = nu[k] + nd[k];
      put(0, 5, n, e);
      for (int ch = 1; ch <= 4; ++ch) put(ch, ch, F, 1.0);
      put(1, 5, cu, v);
      put(2, 5, cd, v);
      put(3, 5, tr(cu), v);
      put(4, 5, tr(cd), v);
      put(5, 5, I, 1.0);
    }
    const int w0 = 0, wn = (i == 0) ? 1 : Db;
    const int v0 = (i == N - 1) ? Db - 1 : 0, vn = Db;
    for (int w = w0; w < wn; ++w)
      for (int sp = 0; sp < d; ++sp)
        for (int s = 0; s < d; ++s)
          for (int w2 = v0; w2 < vn; ++w2) {
            W.push_back(bulk[(((size_t)w * d + sp) * d + s) * Db + w2]);
            W.push_back(0.0);
          }
  }
  return ite_mpo_create(ctx, N, dv.data(), Dv.data(), W.data(), out);
}

int ite_mpo_length(ite_mpo H) { return H ? H->N : 0; }

void ite_mpo_destroy(ite_mpo H) {
  if (!H) return;
  buf_free(H->ctx, H->Wdev);
  buf_free(H->ctx, H->plan_mem);
  delete H;
}

ite_status ite_mps_create(ite_ctx ctx, int N, int d, const int* chi, const double* A, int chi_cap,
                          ite_mps* out) {
  if (!ctx || !out || N < 1 || d < 1 || d > 16 || chi_cap < 1 || !chi || !A) return ITE_EINVAL;
  *out = nullptr;
  ite_mps m = nullptr;
  CS(mps_alloc(ctx, N, d, chi_cap, &m));
  ite_status st = ite_mps_set(ctx, m, chi, A);
  if (st != ITE_OK) {
    mps_free(m);
    return st;
  }
  *out = m;
  return ITE_OK;
}

ite_status ite_mps_create_product(ite_ctx ctx, int N, int d, const double* site_vecs, int chi_cap,
                                  ite_mps* out) {
  if (!site_vecs) return ITE_EINVAL;
  std::vector<int> chi(N + 1, 1);
  return ite_mps_create(ctx, N, d, chi.data(), site_vecs, chi_cap, out);
}

ite_status ite_mps_set(ite_ctx ctx, ite_mps m, const int* chi, const double* A) {
  if (!ctx || !m || !chi || !A) return ITE_EINVAL;
  if (chi[0] != 1 || chi[m->N] != 1) return fail(ctx, ITE_EINVAL, "boundary bond dimensions must be 1");
  for (int b = 0; b <= m->N; ++b)
    if (chi[b] < 1 || chi[b] > m->cap[b]) return fail(ctx, ITE_EINVAL, "bond dimension above capacity");
  const double* p = A;
  for (int i = 0; i < m->N; ++i) {
    const size_t cnt = (size_t)chi[i] * m->d * chi[i + 1];
    CK(cudaMemcpyAsync(m->site[i], p, cnt * sizeof(cplx), cudaMemcpyHostToDevice, ctx->stream));
    p += 2 * cnt;
  }
  m->chi.assign(chi, chi + m->N + 1);
  return sync(ctx);
}

namespace {
constexpr char kMpsMagic[8] = {'I', 'T', 'E', 'M', 'P', 'S', '0', '1'};
}

ite_status ite_mps_bytes(ite_mps m, size_t* bytes) {
  if (!m || !bytes) return ITE_EINVAL;
  size_t nd = 0;
  ite_mps_bond_dims(m, nullptr, &nd);
  *bytes = 8 + 8 * (3 + (size_t)m->N + 1) + nd * sizeof(double);
  return ITE_OK;
}

ite_status ite_mps_save(ite_mps m, void* buf, size_t cap) {
  size_t need = 0;
  if (!m || !buf || ite_mps_bytes(m, &need) != ITE_OK) return ITE_EINVAL;
  if (cap < need) return fail(m->ctx, ITE_EINVAL, "checkpoint buffer too small");
  char* p = static_cast<char*>(buf);
  std::memcpy(p, kMpsMagic, 8);
  std::vector<long long> head = {m->N, m->d, m->chi_cap};
  for (int b = 0; b <= m->N; ++b) head.push_back(m->chi[b]);
  std::memcpy(p + 8, head.data(), head.size() * 8);
  const size_t off = 8 + head.size() * 8;
  return ite_mps_get(m->ctx, m, reinterpret_cast<double*>(p + off), (cap - off) / sizeof(double));
}

ite_status ite_mps_checkpoint_info(const void* buf, size_t len, int* N_out, int* d_out,
                                   int* chi_cap_out, int* chi_out, size_t chi_len,
                                   size_t* n_doubles) {
  if (!buf) return ITE_EINVAL;
  const char* p = static_cast<const char*>(buf);
  if (len < 8 + 3 * 8 || std::memcmp(p, kMpsMagic, 8) != 0) return ITE_EINVAL;
  long long N = 0, d = 0, cap = 0;
  std::memcpy(&N, p + 8, 8);
  std::memcpy(&d, p + 16, 8);
  std::memcpy(&cap, p + 24, 8);
  if (N < 1 || N > (1 << 20) || d < 1 || d > 16 || cap < 1 || cap > (1 << 20)) return ITE_EINVAL;
  const size_t off = 8 + 8 * (3 + (size_t)N + 1);
  if (len < off) return ITE_EINVAL;
  std::vector<int> chi(N + 1);
  size_t nd = 0;
  for (long long b = 0; b <= N; ++b) {
    long long c = 0;
    std::memcpy(&c, p + 32 + 8 * b, 8);
    if (c < 1 || c > cap) return ITE_EINVAL;
    chi[b] = (int)c;
  }
  if (chi[0] != 1 || chi[N] != 1) return ITE_EINVAL;
  // Each site's share is compared with the doubles that remain in the buffer
  // before it is added, so the running sum never exceeds len / 8 and cannot
  // wrap (a term is at most 2 * 2^20 * 16 * 2^20 = 2^45, but 2^19 of them
  // would overflow a 64-bit sum).
  size_t remaining = (len - off) / sizeof(double);
  for (long long i = 0; i < N; ++i) {
    const size_t term = 2 * (size_t)chi[i] * (size_t)d * (size_t)chi[i + 1];
    if (term > remaining) return ITE_EINVAL;
    remaining -= term;
    nd += term;
  }
  if (chi_out && chi_len < (size_t)N + 1) return ITE_EINVAL;
  if (N_out) *N_out = (int)N;
  if (d_out) *d_out = (int)d;
  if (chi_cap_out) *chi_cap_out = (int)cap;
  if (chi_out) std::copy(chi.begin(), chi.end(), chi_out);
  if (n_doubles) *n_doubles = nd;
  return ITE_OK;
}

ite_status ite_mps_load(ite_ctx ctx, const void* buf, size_t len, ite_mps* out) {
  if (!ctx || !buf || !out) return ITE_EINVAL;
  *out = nullptr;
  int N = 0, d = 0, cap = 0;
  size_t nd = 0;
  if (ite_mps_checkpoint_info(buf, len, &N, &d, &cap, nullptr, 0, &nd) != ITE_OK)
    return fail(ctx, ITE_EINVAL, "not a valid MPS checkpoint (magic, header or length)");
  std::vector<int> chi(N + 1);
  ite_mps_checkpoint_info(buf, len, nullptr, nullptr, nullptr, chi.data(), chi.size(), nullptr);
  const size_t off = 8 + 8 * (3 + (size_t)N + 1);
  // the tensors may sit at any alignment in the caller's buffer
  std::vector<double> A(nd);
  std::memcpy(A.data(), static_cast<const char*>(buf) + off, nd * sizeof(double));
  return ite_mps_create(ctx, N, d, chi.data(), A.data(), cap, out);
}

ite_status ite_mps_to_dense(ite_ctx ctx, ite_mps m, double* out, size_t cap_doubles) {
  if (!ctx || !m || !out) return ITE_EINVAL;
  double logsz = m->N * std::log2((double)m->d);
  if (logsz > 24.0) return fail(ctx, ITE_EINVAL, "state too large for a dense vector");
  size_t dim = 1;
  for (int i = 0; i < m->N; ++i) dim *= (size_t)m->d;
  if (cap_doubles < 2 * dim) return fail(ctx, ITE_EINVAL, "output buffer too small");
  size_t nd = 0;
  ite_mps_bond_dims(m, nullptr, &nd);
  std::vector<double> A(nd);
  CS(ite_mps_get(ctx, m, A.data(), nd));
  // v[prefix][bond] grows one site at a time: v' = v . A_i (prefix x d)
  typedef std::complex<double> z;
  std::vector<z> v(1, z(1.0, 0.0)), w;
  size_t rows = 1, pos = 0;
  for (int i = 0; i < m->N; ++i) {
    const int cl = m->chi[i], cr = m->chi[i + 1], d = m->d;
    const z* Ai = reinterpret_cast<const z*>(A.data()) + pos;
    // a minimal MPS keeps every intermediate within d^N <= 2^24 entries
    if ((double)rows * d * cr > (double)(1u << 26)) return fail(ctx, ITE_EINVAL, "intermediate too large");
    w.assign(rows * d * cr, z(0.0, 0.0));
    for (size_t r = 0; r < rows; ++r)
      for (int a = 0; a < cl; ++a) {
        const z va = v[r * cl + a];
        if (va == z(0.0, 0.0)) continue;
        for (int s = 0; s < d; ++s)
          for (int b = 0; b < cr; ++b) w[(r * d + s) * cr + b] += va * Ai[((size_t)a * d + s) * cr + b];
      }
    v.swap(w);
    rows *= d;
    pos += (size_t)cl * d * cr;
  }
  std::memcpy(out, v.data(), 2 * dim * sizeof(double));
  return ITE_OK;
}

ite_status ite_mps_copy(ite_ctx ctx, ite_mps src, ite_mps dst) {
  if (!ctx || !src || !dst || src->N != dst->N || src->d != dst->d) return ITE_EINVAL;
  for (int b = 0; b <= src->N; ++b)
    if (src->chi[b] > dst->cap[b]) return fail(ctx, ITE_EINVAL, "destination capacity too small");
  CS(mps_copy_into(ctx, src, dst));
  return sync(ctx);
}

ite_status ite_mps_bond_dims(ite_mps m, int* chi, size_t* n_doubles) {
  if (!m) return ITE_EINVAL;
  size_t tot = 0;
  for (int i = 0; i < m->N; ++i) tot += (size_t)m->chi[i] * m->d * m->chi[i + 1];
  if (chi) std::copy(m->chi.begin(), m->chi.end(), chi);
  if (n_doubles) *n_doubles = 2 * tot;
  return ITE_OK;
}

ite_status ite_mps_get(ite_ctx ctx, ite_mps m, double* A, size_t cap_doubles) {
  if (!ctx || !m || !A) return ITE_EINVAL;
  size_t need = 0;
  ite_mps_bond_dims(m, nullptr, &need);
  if (cap_doubles < need) return fail(ctx, ITE_EINVAL, "output buffer too small");
  double* p = A;
  for (int i = 0; i < m->N; ++i) {
    const size_t cnt = (size_t)m->chi[i] * m->d * m->chi[i + 1];
    CK(cudaMemcpyAsync(p, m->site[i], cnt * sizeof(cplx), cudaMemcpyDeviceToHost, ctx->stream));
    p += 2 * cnt;
  }
  return sync(ctx);
}

void ite_mps_destroy(ite_mps m) { mps_free(m); }

ite_status ite_implicit_step(ite_ctx ctx, ite_mpo H, ite_mps psi, double dtau, int scheme,
                             double shift, int chi_max, double cutoff, const ite_solver_opts* opts,
                             ite_step_info* info) {
  ite_solver_opts o;
  ite_solver_opts_default(&o);
  if (opts) o = *opts;
  return step_impl(ctx, H, psi, dtau, scheme, shift, chi_max, cutoff, o, info);
}

ite_status ite_mps_sample(ite_ctx ctx, ite_mps psi, const double* u, const double* basis,
                          int* config, double* prob) {
  if (!ctx || !psi || !u || !config || psi->ctx != ctx || psi->d < 1 || psi->d > 4)
    return ITE_EINVAL;
  for (int i = 0; i < psi->N; ++i)
    if (!(u[i] >= 0.0 && u[i] < 1.0)) return fail(ctx, ITE_EINVAL, "uniform numbers must lie in [0, 1)");
  const int N = psi->N, d = psi->d;
  // the draw reads the state in right-canonical form; the state is unchanged.
  // The gauge move writes its left factor (chl x min(chl, d chr)) and the
  // product into the neighbouring site (chl_{i-1} d x chl_i): both fit in
  // the largest site capacity.
  long long site_max = 1;
  for (int i = 0; i < N; ++i)
    site_max = std::max(site_max, (long long)psi->cap[i] * d * psi->cap[i + 1]);
  CS(buf_ensure(ctx, ctx->ws_left, (size_t)site_max * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_X2, (size_t)site_max * sizeof(cplx)));
  CS(right_canonicalize(ctx, psi));
  CS(buf_ensure(ctx, ctx->ws_X, (size_t)2 * psi->chi_cap * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_small, std::max<size_t>(small_bytes(1), (size_t)N * sizeof(int) + 256)));
  cplx* va = P<cplx>(ctx->ws_X);
  cplx* vb = va + psi->chi_cap;
  int* cfg = P<int>(ctx->ws_small);
  double* pr = ctx->dscal + 11;
  cplx* bdev = nullptr;
  if (basis) {
    bdev = ctx->dcplx + 256;
    CK(cudaMemcpyAsync(bdev, basis, sizeof(cplx) * d * d, cudaMemcpyHostToDevice, ctx->stream));
  }
  const double one = 1.0;
  CK(cudaMemcpyAsync(pr, &one, sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  CS(set_one(ctx, va));
  for (int i = 0; i < N; ++i) {
    CK(sample_site(psi->site[i], psi->chi[i], d, psi->chi[i + 1], va, u[i], bdev, vb, cfg + i, pr,
                   ctx->stream));
    std::swap(va, vb);
  }
  CK(cudaMemcpyAsync(config, cfg, sizeof(int) * N, cudaMemcpyDeviceToHost, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->d[0], pr, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  if (prob) *prob = ctx->hr->d[0];
  if (!(ctx->hr->d[0] > 0.0)) return fail(ctx, ITE_ESINGULAR, "zero or non-finite state in the draw");
  return ITE_OK;
}

ite_status ite_metts(ite_ctx ctx, ite_mpo H, const int* config0, const double* nodes, int n_steps,
                     int scheme, int shift_mode, double shift0, int chi_max, double cutoff,
                     const ite_solver_opts* opts, const double* alt_basis, const double* obs,
                     int obs_site, int n_samples, const double* uniforms, double* energies,
                     double* obs_values, int* configs) {
  if (!ctx || !H || !config0 || !nodes || !uniforms || !energies || n_samples < 1 || n_steps < 1 ||
      chi_max < 1 || H->ctx != ctx || H->d > 4 ||
      (obs && (obs_site < 0 || obs_site >= H->N || !obs_values)))
    return ITE_EINVAL;
  std::vector<double> grid(nodes, nodes + n_steps + 1);
  if (grid[0] != 0.0) return fail(ctx, ITE_EINVAL, "the tau grid must start at 0");
  for (int k = 1; k <= n_steps; ++k)
    if (!(grid[k] > grid[k - 1]) || !std::isfinite(grid[k]))
      return fail(ctx, ITE_EINVAL, "the tau grid must increase strictly");
  ite_solver_opts o;
  ite_solver_opts_default(&o);
  if (opts) o = *opts;
  const int N = H->N, d = H->d;
  for (int i = 0; i < N; ++i)
    if (config0[i] < 0 || config0[i] >= d) return fail(ctx, ITE_EINVAL, "start configuration out of range");
  ite_mps psi = nullptr;
  CS(mps_alloc(ctx, N, d, chi_max, &psi));
  struct Free {
    ite_mps m;
    ~Free() { mps_free(m); }
  } free_psi{psi};
  std::vector<double> A((size_t)2 * N * d), ident((size_t)2 * d * d, 0.0), out(2);
  for (int k = 0; k < d; ++k) ident[2 * (k * d + k)] = 1.0;
  std::vector<int> ones(N + 1, 1), config(config0, config0 + N);
  std::vector<ite_step_info> info(n_steps);
  const double* cur_basis = nullptr;      // the product state's basis (NULL: computational)
  for (int k = 0; k < n_samples; ++k) {
    // product state: site i is column config[i] of the current basis
    for (int i = 0; i < N; ++i)
      for (int t = 0; t < d; ++t) {
        const int e = 2 * (t * d + config[i]);
        A[2 * (i * d + t)] = cur_basis ? cur_basis[e] : (t == config[i] ? 1.0 : 0.0);
        A[2 * (i * d + t) + 1] = cur_basis ? cur_basis[e + 1] : 0.0;
      }
    CS(ite_mps_set(ctx, psi, ones.data(), A.data()));
    CS(evolve_impl(ctx, H, psi, grid, scheme, shift_mode, shift0, chi_max, cutoff, o, info.data()));
    energies[k] = info[n_steps - 1].energy;
    if (obs) {
      CS(ite_correlator(ctx, psi, obs, obs_site, ident.data(), obs_site, nullptr, out.data()));
      obs_values[k] = out[0];
    }
    const double* basis_k = (alt_basis && k % 2 == 0) ? alt_basis : nullptr;
    double p = 0.0;
    CS(ite_mps_sample(ctx, psi, uniforms + (size_t)k * N, basis_k, config.data(), &p));
    if (configs) std::copy(config.begin(), config.end(), configs + (size_t)k * N);
    cur_basis = basis_k;
  }
  return ITE_OK;
}

ite_status ite_gl_partial_fractions(int q, double* poles, double* residues, double* r_inf) {
  if (!poles || !residues || !r_inf) return ITE_EINVAL;
  std::vector<Cd> z, a;
  if (!gl_partial_fractions(q, z, a, r_inf)) return ITE_EINVAL;
  for (int j = 0; j < q; ++j) {
    poles[2 * j] = z[j].re;
    poles[2 * j + 1] = z[j].im;
    residues[2 * j] = a[j].re;
    residues[2 * j + 1] = a[j].im;
  }
  return ITE_OK;
}

ite_status ite_grid_geometric(double tau0, double tau_max, int n_steps, double* nodes) {
  if (!nodes || n_steps < 1 || !(tau0 > 0.0) || !(tau_max >= tau0)) return ITE_EINVAL;
  grid_geometric_impl(tau0, tau_max, n_steps, nodes);
  return ITE_OK;
}

ite_status ite_grid_panels(double tau_max, int Pn, int n, double* nodes) {
  if (!nodes || Pn < 1 || n < 1 || !(tau_max > 0.0) || Pn > 1000) return ITE_EINVAL;
  grid_panels_impl(tau_max, Pn, n, nodes);
  return ITE_OK;
}

ite_status ite_evolve_loggrid(ite_ctx ctx, ite_mpo H, ite_mps psi, double tau0, double tau_max,
                              int n_steps, int scheme, int shift_mode, double shift0, int chi_max,
                              double cutoff, const ite_solver_opts* opts, ite_step_info* per_step,
                              double* nodes_out) {
  std::vector<double> nodes(std::max(n_steps, 1) + 1);
  if (ite_grid_geometric(tau0, tau_max, n_steps, nodes.data()) != ITE_OK)
    return fail(ctx, ITE_EINVAL, "invalid grid");
  if (nodes_out) std::copy(nodes.begin(), nodes.end(), nodes_out);
  ite_solver_opts o;
  ite_solver_opts_default(&o);
  if (opts) o = *opts;
  return evolve_impl(ctx, H, psi, nodes, scheme, shift_mode, shift0, chi_max, cutoff, o, per_step);
}

ite_status ite_evolve_panels(ite_ctx ctx, ite_mpo H, ite_mps psi, double tau_max, int Pn, int n,
                             int scheme, int shift_mode, double shift0, int chi_max, double cutoff,
                             const ite_solver_opts* opts, ite_step_info* per_step, double* nodes_out) {
  if (Pn < 1 || n < 1 || Pn > 1000) return fail(ctx, ITE_EINVAL, "invalid grid");
  std::vector<double> nodes((size_t)Pn * n + 1);
  if (ite_grid_panels(tau_max, Pn, n, nodes.data()) != ITE_OK) return fail(ctx, ITE_EINVAL, "invalid grid");
  if (nodes_out) std::copy(nodes.begin(), nodes.end(), nodes_out);
  ite_solver_opts o;
  ite_solver_opts_default(&o);
  if (opts) o = *opts;
  return evolve_impl(ctx, H, psi, nodes, scheme, shift_mode, shift0, chi_max, cutoff, o, per_step);
}

ite_status ite_energy(ite_ctx ctx, ite_mpo H, ite_mps psi, double* E) {
  CS(validate_pair(ctx, H, psi));
  if (!E) return ITE_EINVAL;
  return energy_impl(ctx, H, psi, E);
}

ite_status ite_overlap(ite_ctx ctx, ite_mps bra, ite_mps ket, double out[2]) {
  if (!ctx || !bra || !ket || !out) return ITE_EINVAL;
  if (bra->N != ket->N || bra->d != ket->d) return fail(ctx, ITE_EINVAL, "MPS shapes differ");
  cplx z;
  CS(overlap_impl(ctx, bra, ket, nullptr, &z));
  out[0] = z.x;
  out[1] = z.y;
  return ITE_OK;
}

ite_status ite_correlator(ite_ctx ctx, ite_mps psi, const double* O, int i, const double* Pm,
                          int j, const double* string_op, double out[2]) {
  if (!ctx || !psi || !O || !Pm || !out || i < 0 || j >= psi->N || i > j) return ITE_EINVAL;
  const int d = psi->d;
  std::vector<const cplx*> ops(psi->N, nullptr);
  const cplx *o, *p, *s;
  CS(upload_ops(ctx, d, O, 0, &o));
  CS(upload_ops(ctx, d, Pm, 1, &p));
  CS(upload_ops(ctx, d, string_op, 2, &s));
  if (i == j) {
    // O P on one site: form the product on the host
    std::vector<double> op(2 * d * d, 0.0);
    for (int a = 0; a < d; ++a)
      for (int b = 0; b < d; ++b)
        for (int k = 0; k < d; ++k) {
          const double ar = O[2 * (a * d + k)], ai = O[2 * (a * d + k) + 1];
          const double br = Pm[2 * (k * d + b)], bi = Pm[2 * (k * d + b) + 1];
          op[2 * (a * d + b)] += ar * br - ai * bi;
          op[2 * (a * d + b) + 1] += ar * bi + ai * br;
        }
    CS(upload_ops(ctx, d, op.data(), 3, &o));
    CS(sync(ctx));
    ops[i] = o;
  } else {
    ops[i] = o;
    ops[j] = p;
    if (s)
      for (int k = i + 1; k < j; ++k) ops[k] = s;
  }
  cplx num, den;
  CS(overlap_impl(ctx, psi, psi, &ops, &num));
  CS(overlap_impl(ctx, psi, psi, nullptr, &den));
  if (!(den.x > 0.0)) return fail(ctx, ITE_ESINGULAR, "zero-norm state");
  out[0] = num.x / den.x;
  out[1] = num.y / den.x;
  return ITE_OK;
}

// ------------------------------------------------------------------ kernel-level entry points
ite_status ite_ctx_set_kernel_precision(ite_ctx ctx, int precision) {
  if (!ctx || (precision != ITE_FP64 && precision != ITE_FP64_TC && !mixed_precision(precision)))
    return ITE_EINVAL;
  ctx->kernel_precision = precision;
  return ITE_OK;
}

ite_status ite_k_heff_lp_prepare(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket,
                                 int chr_ket, int chr_bra, const double* L, const double* R,
                                 int precision) {
  if (!ctx || !H || !L || !R || i < 0 || i + 1 >= H->N || chl_bra < 1 || chl_ket < 1 ||
      chr_ket < 1 || chr_bra < 1 || !mixed_precision(precision))
    return ITE_EINVAL;
  CK(cudaMemsetAsync(reinterpret_cast<int*>(ctx->dcounter) + 10, 0, sizeof(int), ctx->stream));
  CS(heff_lp_setup(ctx, H, i, chl_bra, chl_ket, chr_ket, chr_bra, (const cplx*)L, (const cplx*)R,
                   precision == ITE_MIXED_TF32 ? 1 : 0));
  return kernel_finish(ctx);
}

ite_status ite_k_heff_lp_apply(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket,
                               int chr_ket, int chr_bra, const double* X, double* Y,
                               const double alpha[2], const double* Z, const double gamma[2]) {
  if (!ctx || !H || !X || !Y || !alpha || i < 0 || i + 1 >= H->N || chl_bra < 1 || chl_ket < 1 ||
      chr_ket < 1 || chr_bra < 1)
    return ITE_EINVAL;
  CK(cudaMemsetAsync(reinterpret_cast<int*>(ctx->dcounter) + 10, 0, sizeof(int), ctx->stream));
  struct LevelGuard {
    ite_ctx c;
    ~LevelGuard() { c->lp_level = -1; }
  } guard{ctx};
  ctx->lp_level = ctx->lp_prep.level;
  const cplx g = gamma ? C(gamma[0], gamma[1]) : C(0);
  CS(heff_lp(ctx, H, i, chl_bra, chl_ket, chr_ket, chr_bra, (const cplx*)X, (cplx*)Y,
             C(alpha[0], alpha[1]), (const cplx*)Z, g));
  return kernel_finish(ctx);
}

ite_status ite_k_heff_lp_apply_n(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket,
                                 int chr_ket, int chr_bra, const double* X, double* Y,
                                 const double alpha[2], const double* Z, const double gamma[2],
                                 int reps) {
  if (!ctx || !H || !X || !Y || !alpha || i < 0 || i + 1 >= H->N || chl_bra < 1 || chl_ket < 1 ||
      chr_ket < 1 || chr_bra < 1 || reps < 1 || Y == X || Y == Z)
    return ITE_EINVAL;
  CK(cudaMemsetAsync(reinterpret_cast<int*>(ctx->dcounter) + 10, 0, sizeof(int), ctx->stream));
  struct LevelGuard {
    ite_ctx c;
    ~LevelGuard() { c->lp_level = -1; }
  } guard{ctx};
  ctx->lp_level = ctx->lp_prep.level;
  const cplx g = gamma ? C(gamma[0], gamma[1]) : C(0);
  for (int r = 0; r < reps; ++r)
    CS(heff_lp(ctx, H, i, chl_bra, chl_ket, chr_ket, chr_bra, (const cplx*)X, (cplx*)Y,
               C(alpha[0], alpha[1]), (const cplx*)Z, g));
  return kernel_finish(ctx);
}

ite_status ite_k_heff(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket, int chr_ket,
                      int chr_bra, const double* L, const double* R, const double* X, double* Y,
                      const double alpha[2], const double* Z, const double gamma[2]) {
  if (!ctx || !H || !L || !R || !X || !Y || !alpha || i < 0 || i + 1 >= H->N || chl_bra < 1 ||
      chl_ket < 1 || chr_ket < 1 || chr_bra < 1)
    return ITE_EINVAL;
  KernelMode km(ctx);
  const long long d2 = (long long)H->d * H->d;
  const long long t = (long long)H->Dmax * std::max(chl_bra, chl_ket) * d2 * std::max(chr_ket, chr_bra);
  CS(buf_ensure(ctx, ctx->ws_T1, t * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_T2, t * sizeof(cplx)));
  const cplx g = gamma ? C(gamma[0], gamma[1]) : C(0);
  CS(heff(ctx, H, i, chl_bra, chl_ket, chr_ket, chr_bra, (const cplx*)L, (const cplx*)R,
          (const cplx*)X, (cplx*)Y, C(alpha[0], alpha[1]), (const cplx*)Z, g));
  return kernel_finish(ctx);
}

ite_status ite_k_env_left(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket, int chr_bra,
                          int chr_ket, const double* Lin, const double* bra, const double* ket,
                          double* Lout) {
  if (!ctx || !H || !Lin || !bra || !ket || !Lout || i < 0 || i >= H->N || chl_bra < 1 ||
      chl_ket < 1 || chr_bra < 1 || chr_ket < 1)
    return ITE_EINVAL;
  KernelMode km(ctx);
  const long long t = (long long)H->Dmax * std::max(chl_bra, chl_ket) * H->d * std::max(chr_bra, chr_ket);
  CS(buf_ensure(ctx, ctx->ws_T1, t * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_T2, t * sizeof(cplx)));
  CS(env_left(ctx, H, i, chl_bra, chl_ket, chr_bra, chr_ket, (const cplx*)Lin, (const cplx*)bra,
              (const cplx*)ket, (cplx*)Lout));
  return kernel_finish(ctx);
}

ite_status ite_k_env_right(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket, int chr_bra,
                           int chr_ket, const double* Rin, const double* bra, const double* ket,
                           double* Rout) {
  if (!ctx || !H || !Rin || !bra || !ket || !Rout || i < 0 || i >= H->N || chl_bra < 1 ||
      chl_ket < 1 || chr_bra < 1 || chr_ket < 1)
    return ITE_EINVAL;
  KernelMode km(ctx);
  const long long t = (long long)H->Dmax * std::max(chl_bra, chl_ket) * H->d * std::max(chr_bra, chr_ket);
  CS(buf_ensure(ctx, ctx->ws_T1, t * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_T2, t * sizeof(cplx)));
  CS(env_right(ctx, H, i, chl_bra, chl_ket, chr_bra, chr_ket, (const cplx*)Rin, (const cplx*)bra,
               (const cplx*)ket, (cplx*)Rout));
  return kernel_finish(ctx);
}

ite_status ite_k_local_solve(ite_ctx ctx, ite_mpo H, int i, int chl, int chr, const double* L,
                             const double* R, const double* B, double* X, double alpha, double c,
                             int krylov_dim, double local_tol, int* steps, double* rel_res) {
  if (!ctx || !H || !L || !R || !B || !X || i < 0 || i + 1 >= H->N || chl < 1 || chr < 1 ||
      krylov_dim < 1 || krylov_dim > kMaxKrylov)
    return ITE_EINVAL;
  KernelMode km(ctx);
  const long long n = (long long)chl * H->d * H->d * chr;
  CS(buf_ensure(ctx, ctx->ws_V, (size_t)(krylov_dim + 1) * n * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_T1, (size_t)H->Dmax * n * sizeof(cplx)));
  CS(buf_ensure(ctx, ctx->ws_T2, (size_t)H->Dmax * n * sizeof(cplx)));
  int s = 0;
  double r = 0.0;
  if (mixed_precision(ctx->kernel_precision))
    CS(local_solve_mixed(ctx, H, i, chl, chr, (const cplx*)L, (const cplx*)R, (const cplx*)B,
                         (cplx*)X, C(alpha), C(c), krylov_dim, ctx->kernel_precision, 20,
                         local_tol > 0.0 ? local_tol : 1e-10, &s, &r));
  else
    CS(local_solve(ctx, H, i, chl, chr, (const cplx*)L, (const cplx*)R, (const cplx*)B, (cplx*)X,
                   C(alpha), C(c), krylov_dim, 1, local_tol, &s, &r));
  if (steps) *steps = s;
  if (rel_res) *rel_res = r;
  return kernel_finish(ctx);
}

ite_status ite_k_gemm_lp(ite_ctx ctx, int M, int N, int K, int batch, const void* A, long long lda,
                         long long sAb, const void* B, long long ldb, long long sBb, float* Cm,
                         long long ldc, long long sCb, long long sCs, int tf32, int bn, int splits,
                         int flags) {
  const int eb = tf32 ? 4 : 2;
  if (!ctx || !A || !B || !Cm || M < 1 || N < 1 || K < 1 || batch < 1 || lda < K || ldb < K ||
      ldc < N || (lda * eb) % 16 || (ldb * eb) % 16 || (sAb * eb) % 16 || (sBb * eb) % 16 ||
      sAb < 0 || sBb < 0 || sCb < 0 || sCs < 0 || (bn != 128 && bn != 192 && bn != 256) || splits < 1 ||
      (splits > 1 && sCs == 0))
    return ITE_EINVAL;
  int* err = reinterpret_cast<int*>(ctx->dcounter) + 8;
  CK(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  LpGemmArgs g = {};
  g.M = M; g.N = N; g.K = K; g.batch = batch; g.splits = splits; g.bn = bn; g.tf32 = tf32 != 0;
  g.A = A; g.lda = lda; g.sAb = sAb;
  g.B = B; g.ldb = ldb; g.sBb = sBb;
  g.C = Cm; g.ldc = ldc; g.sCb = sCb; g.sCs = sCs;
  g.pair = (flags & 1) != 0;
  CK(lp_gemm(g, err, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->counter, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  if (ctx->hr->counter != 0) return fail(ctx, ITE_ETIMEOUT, "tensor-core GEMM wait ran out");
  return ITE_OK;
}

ite_status ite_k_gemm_bf16(ite_ctx ctx, int M, int N, int K, const void* A, long long lda,
                           const void* B, long long ldb, float* Cm, long long ldc, int flags) {
  if (!ctx || !A || !B || !Cm || M < 1 || N < 1 || K < 1 || lda < K || ldb < K || ldc < N ||
      lda % 8 || ldb % 8)
    return ITE_EINVAL;
  int* err = reinterpret_cast<int*>(ctx->dcounter) + 8;
  CK(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  CK(tc_gemm_bf16(A, lda, B, ldb, Cm, ldc, M, N, K, err, ctx->stream, (flags & 1) ? 32 : 64));
  CK(cudaMemcpyAsync(&ctx->hr->counter, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  if (ctx->hr->counter != 0) return fail(ctx, ITE_ETIMEOUT, "tensor-core GEMM wait ran out");
  return ITE_OK;
}

ite_status ite_k_zgemm(ite_ctx ctx, int mode, int M, int N, int K, const double* A, long long sAm,
                       long long sAk, int conjA, const double* B, long long sBk, long long sBn,
                       int conjB, double* Cm, long long ldc, const double alpha[2],
                       const double beta[2]) {
  if (!ctx || !A || !B || !Cm || M < 1 || N < 1 || K < 1 || (mode != 0 && mode != 1))
    return ITE_EINVAL;
  GemmArgs g;
  g.M = M; g.N = N; g.K = K; g.batch = 1;
  g.A = (const cplx*)A; g.sAm = sAm; g.sAk = sAk; g.sAb = 0; g.conjA = conjA != 0;
  g.B = (const cplx*)B; g.sBk = sBk; g.sBn = sBn; g.sBb = 0; g.conjB = conjB != 0;
  g.C = (cplx*)Cm; g.ldc = ldc; g.sCb = 0;
  g.alpha = alpha ? C(alpha[0], alpha[1]) : C(1);
  g.beta = beta ? C(beta[0], beta[1]) : C(0);
  g.Z = nullptr; g.gamma = C(0);
  if (mode == 0) {
    CK(zgemm(g, ctx->stream));
    return sync(ctx);
  }
  const size_t need = zgemm_emu_scratch_bytes(M, N, K);
  CS(buf_ensure(ctx, ctx->ws_emu, need));
  int* err = reinterpret_cast<int*>(ctx->dcounter) + 9;
  CK(cudaMemsetAsync(err, 0, sizeof(int), ctx->stream));
  CK(zgemm_emu(g, ctx->ws_emu.p, ctx->ws_emu.n, err, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->counter, err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  if (ctx->hr->counter != 0) return fail(ctx, ITE_ETIMEOUT, "emulated GEMM wait ran out");
  return ITE_OK;
}

ite_status ite_k_barrier_selftest(ite_ctx ctx, int blocks, int absent) {
  if (!ctx || blocks < 2 || absent < 0 || absent >= blocks) return ITE_EINVAL;
  int sms = 0;
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ctx->device));
  if (blocks > sms) return ITE_EINVAL;
  unsigned int* st = reinterpret_cast<unsigned int*>(ctx->dcounter) + 16;
  CK(barrier_selftest(st, blocks, absent, ctx->stream));
  CK(cudaMemcpyAsync(&ctx->hr->counter, st + 4, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CS(sync(ctx));
  if (ctx->hr->counter != 0) return fail(ctx, ITE_ETIMEOUT, "grid barrier wait ran out");
  return ITE_OK;
}

ite_status ite_k_split(ite_ctx ctx, const double* X, int m, int n, int chi_max, double cutoff,
                       int centre_right, double* left, double* right, double* sigma, int* rank,
                       double* discarded, int flags) {
  if (!ctx || !X || !left || !right || m < 1 || n < 1 || chi_max < 1 || !(cutoff >= 0.0))
    return ITE_EINVAL;
  struct ModeGuard {
    ite_ctx c;
    ~ModeGuard() { c->gemm_mode = 0; }
  } mode_guard{ctx};
  ctx->gemm_mode = (flags & 1) ? 1 : 0;
  CK(cudaMemsetAsync(reinterpret_cast<int*>(ctx->dcounter) + 10, 0, sizeof(int), ctx->stream));
  int r = 0;
  double disc = 0.0;
  CS(split(ctx, (const cplx*)X, m, n, chi_max, cutoff, centre_right != 0, (cplx*)left, (cplx*)right,
           &r, &disc, sigma));
  CS(sync(ctx));
  if (rank) *rank = r;
  if (discarded) *discarded = disc;
  return ITE_OK;
}

}  // extern "C"

// ================================================================== accessors
// Read-only views of context and MPO internals for the allocation-free
// variant in heff_static.cu.
namespace ite {

bool internal_ctx_info(ite_ctx ctx, int* device, cudaStream_t* stream) {
  if (!ctx) return false;
  *device = ctx->device;
  *stream = ctx->stream;
  return true;
}

bool internal_bond_info(ite_mpo H, int i, int* d, int* D0, int* D1, int* D2, const MixPlan** plan) {
  if (!H || i < 0 || i + 1 >= H->N) return false;
  *d = H->d;
  *D0 = H->D[i];
  *D1 = H->D[i + 1];
  *D2 = H->D[i + 2];
  *plan = &H->plan2[i];
  return true;
}

ite_status internal_fail(ite_ctx ctx, ite_status st, const char* msg) { return fail(ctx, st, msg); }

// Attaches ctx to a group of grouped Jacobi launches (nullptr detaches).
ite_status internal_set_group(ite_ctx ctx, SplitGroup* g) {
  if (g && !ctx->group_ready) {
    CK(cudaEventCreateWithFlags(&ctx->group_ready, cudaEventDisableTiming));
    CK(cudaEventCreateWithFlags(&ctx->group_done, cudaEventDisableTiming));
  }
  if (g && !ctx->group_state) {
    ctx->group_state = static_cast<unsigned int*>(dev_alloc(ctx, 24 * sizeof(unsigned int)));
    if (!ctx->group_state) return fail(ctx, ITE_ENOMEM, "group state allocation failed");
  }
  ctx->group = g;
  return ITE_OK;
}

// Frees the context's reusable workspaces (they grow again on demand), so
// that a long-lived context holds only its small fixed state between jobs.
void internal_release_workspace(ite_ctx ctx) {
  if (!ctx) return;
  cudaStreamSynchronize(ctx->stream);
  Buf* bufs[] = {&ctx->ws_X, &ctx->ws_B, &ctx->ws_X2, &ctx->ws_V, &ctx->ws_T1, &ctx->ws_T2,
                 &ctx->ws_svdA, &ctx->ws_svdQ, &ctx->ws_left, &ctx->ws_small, &ctx->ws_env,
                 &ctx->ws_emu, &ctx->ws_ovm, &ctx->ws_lpops, &ctx->ws_lpscr, &ctx->ws_R,
                 &ctx->ws_D, &ctx->ws_R2, &ctx->ws_Xt};
  for (Buf* b : bufs) buf_free(ctx, *b);
  ctx->lp_prep = ite_ctx_s::LpPrepared();
}

}  // namespace ite
