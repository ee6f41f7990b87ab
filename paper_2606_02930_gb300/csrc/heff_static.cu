// Two-site H_eff matvec that allocates nothing: the two intermediates of the
// contraction live in one fixed device array defined in this file instead of
// in the context workspace.
//
// Some callers cannot allocate device memory at the moment they need a
// matvec: cudaMalloc may synchronise the whole device (stalling other streams
// of a latency-critical serving loop), the process may have handed all device
// memory to another pool, or the caller runs where the CUDA runtime forbids
// allocation calls.  For them this entry point computes the matvec that
// ite_k_heff computes in FP64 mode, with the same FP64 kernels, using a scratch
// array that is part of the loaded library image.  It always runs on the FP64
// pipe: the context's kernel precision (ite_ctx_set_kernel_precision) does not
// apply, because the tensor-core path needs slice buffers sized per call.
//
// The array is 2 x kScratchComplex complex doubles (2 x 8 MiB = 16 MiB) and is
// held by every GPU that loads this library until the process exits.  Every
// call shares it: two calls whose work overlaps on the GPU (different streams,
// or different host threads) race on it, so the caller must order them.  The
// contents left by the previous call do not matter here: both intermediates
// are fully overwritten before they are read, so nothing needs clearing.
//
// Its device address is looked up once per device with cudaGetSymbolAddress
// (host code cannot use the array's name as a device pointer).  The first
// call on each device performs that lookup, so that first call should be made
// before any stream capture begins.
#include <mutex>

#include "common.cuh"
#include "ite.h"
#include "ite_kernels.h"

namespace ite {
bool internal_ctx_info(ite_ctx ctx, int* device, cudaStream_t* stream);
bool internal_bond_info(ite_mpo H, int i, int* d, int* D0, int* D1, int* D2, const MixPlan** plan);
ite_status internal_fail(ite_ctx ctx, ite_status st, const char* msg);
}  // namespace ite

using namespace ite;

namespace {

constexpr long long kScratchComplex = 1LL << 19;   // per intermediate: 512 Ki complex = 8 MiB
constexpr int kMaxDevices = 64;

static __device__ __align__(256) cplx g_heff_scratch[2 * kScratchComplex];

std::mutex g_setup_mutex;
cplx* g_scratch_addr[kMaxDevices] = {nullptr};

// Device address of the scratch array on `device` (made current by the caller).
cudaError_t scratch_address(int device, cplx** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_heff_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[device] = static_cast<cplx*>(p);
  }
  *out = g_scratch_addr[device];
  return cudaSuccess;
}

// Makes `dev` current for the lifetime of the guard and gives the calling
// thread its previous current device back on every return path.
struct DeviceGuard {
  int prev = -1;
  bool ok = false;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) {
      prev = -1;
      return;
    }
    ok = prev == dev || cudaSetDevice(dev) == cudaSuccess;
  }
  ~DeviceGuard() {
    int cur = -1;
    if (prev >= 0 && cudaGetDevice(&cur) == cudaSuccess && cur != prev) cudaSetDevice(prev);
  }
};

}  // namespace

extern "C" ite_status ite_k_heff_noalloc(ite_ctx ctx, ite_mpo H, int i, int chl_bra, int chl_ket,
                                         int chr_ket, int chr_bra, const double* L,
                                         const double* R, const double* X, double* Y,
                                         const double alpha[2], const double* Z,
                                         const double gamma[2]) {
  int dev = 0;
  cudaStream_t st = nullptr;
  int d = 0, D0 = 0, D1 = 0, D2 = 0;
  const MixPlan* plan = nullptr;
  if (!internal_ctx_info(ctx, &dev, &st) || !internal_bond_info(H, i, &d, &D0, &D1, &D2, &plan) ||
      !L || !R || !X || !Y || !alpha || chl_bra < 1 || chl_ket < 1 || chr_ket < 1 || chr_bra < 1)
    return ITE_EINVAL;
  if (dev < 0 || dev >= kMaxDevices) return internal_fail(ctx, ITE_EINVAL, "device index out of range");
  const long long d2 = (long long)d * d;
  const long long t1 = (long long)D0 * chl_bra * d2 * chr_ket;
  const long long t2 = (long long)D2 * chl_bra * d2 * chr_ket;
  if (t1 > kScratchComplex || t2 > kScratchComplex)
    return internal_fail(ctx, ITE_EINVAL,
                         "ite_k_heff_noalloc: D*chl_bra*d^2*chr_ket exceeds the static scratch of "
                         "524288 complex numbers per intermediate");
  DeviceGuard guard(dev);
  if (!guard.ok) return internal_fail(ctx, ITE_ECUDA, "cannot make the context's device current");
  cplx* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess)
    return internal_fail(ctx, ITE_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
  cplx* T1 = base;
  cplx* T2 = base + kScratchComplex;

  // T1[(w a), (s t b')] = L[(w a), a'] X[a', (s t b')]
  GemmArgs g1 = {};
  g1.M = (int)(D0 * chl_bra); g1.N = (int)(d2 * chr_ket); g1.K = chl_ket; g1.batch = 1;
  g1.A = (const cplx*)L; g1.sAm = chl_ket; g1.sAk = 1; g1.sAb = 0; g1.conjA = false;
  g1.B = (const cplx*)X; g1.sBk = d2 * chr_ket; g1.sBn = 1; g1.sBb = 0; g1.conjB = false;
  g1.C = T1; g1.ldc = d2 * chr_ket; g1.sCb = 0;
  g1.alpha = cmake(1.0, 0.0); g1.beta = cmake(0.0, 0.0); g1.Z = nullptr; g1.gamma = cmake(0.0, 0.0);
  if (zgemm(g1, st) != cudaSuccess) return internal_fail(ctx, ITE_ECUDA, "zgemm launch failed");
  // T2[a, s', t', w'', b'] = sum W2[(s' t' w''), (w s t)] T1[w, a, s, t, b']
  MixStrides ms;
  ms.ic[0] = (long long)chl_bra * d2 * chr_ket; ms.ic[1] = (long long)d * chr_ket; ms.ic[2] = chr_ket;
  ms.oc[0] = (long long)d * D2 * chr_ket; ms.oc[1] = (long long)D2 * chr_ket; ms.oc[2] = chr_ket;
  if (mix_apply(*plan, ms, chl_bra, chr_ket, T1, d2 * chr_ket, 1, T2, d2 * D2 * chr_ket, 1, st) !=
      cudaSuccess)
    return internal_fail(ctx, ITE_ECUDA, "mix launch failed");
  // Y[(a s' t'), b] = alpha * T2[(a s' t'), (w'' b')] R[(w'' b'), b] + gamma Z
  GemmArgs g2 = {};
  g2.M = (int)(chl_bra * d2); g2.N = chr_bra; g2.K = D2 * chr_ket; g2.batch = 1;
  g2.A = T2; g2.sAm = (long long)D2 * chr_ket; g2.sAk = 1; g2.sAb = 0; g2.conjA = false;
  g2.B = (const cplx*)R; g2.sBk = chr_bra; g2.sBn = 1; g2.sBb = 0; g2.conjB = false;
  g2.C = (cplx*)Y; g2.ldc = chr_bra; g2.sCb = 0;
  g2.alpha = cmake(alpha[0], alpha[1]); g2.beta = cmake(0.0, 0.0);
  g2.Z = (const cplx*)Z; g2.gamma = gamma ? cmake(gamma[0], gamma[1]) : cmake(0.0, 0.0);
  if (zgemm(g2, st) != cudaSuccess) return internal_fail(ctx, ITE_ECUDA, "zgemm launch failed");
  if (cudaStreamSynchronize(st) != cudaSuccess) return internal_fail(ctx, ITE_ECUDA, "stream sync failed");
  return ITE_OK;
}
