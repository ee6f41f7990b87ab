// Two-site H_eff in low precision (bf16 or tf32 operands, fp32 accumulation on
// the tensor cores) for the inner solves of the mixed-precision mode:
//
//   Y[a,s',t',b] = alpha sum L[w][a][a'] W2[w s t -> w'' s' t'] R[w''][b'][b]
//                        X[a',s,t,b'] + gamma Z[a,s',t',b]
//
// in three contractions, the same order as the FP64 path (App. B's two-site
// effective Hamiltonian):
//   1. T1_w = L_w X for every MPO channel w: one batched real GEMM of the
//      row-embedded L (rows 2a, 2a+1 = [Re, -Im], [Im, Re] along a') with the
//      K-major X^T ((Re, Im) interleaved along a'), giving Re and Im rows;
//   2. T2[(a s' t')][(w'' b')] = sum over the non-zero two-site MPO entries of
//      T1[w][a][(s t b')]: the channel/physical mix, written as the K-major
//      complex-interleaved A operand of step 3;
//   3. Y32 = T2 R~ with the column-embedded R~ (rows 2b, 2b+1 = [Re, -Im],
//      [Im, Re] along (w'' b')), whose fp32 output is complex-interleaved;
//   then Y = alpha Y32 + gamma Z, stored as complex FP64.
// The embedded L and R depend only on the environments, so a local solve
// prepares them once (heff_lp_prepare) and reuses them for every matvec.
#include <cuda_bf16.h>

#include <map>
#include <mutex>
#include <tuple>

#include "common.cuh"
#include "convert.cuh"

namespace ite {
namespace {

template <bool TF32>
struct Lp;
template <>
struct Lp<false> {
  typedef __nv_bfloat16 T;
  typedef __nv_bfloat162 T2;
  static __device__ __forceinline__ T from(double x) {
    return __ushort_as_bfloat16((unsigned short)dbl_to_e8<7>(x));
  }
  static __device__ __forceinline__ T fromf(float x) { return __float2bfloat16_rn(x); }
  static __device__ __forceinline__ T2 pair(T a, T b) { return __halves2bfloat162(a, b); }
};
template <>
struct Lp<true> {
  typedef float T;
  typedef float2 T2;
  static __device__ __forceinline__ float fromf(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
  }
  static __device__ __forceinline__ float from(double x) { return fromf(dbl_to_f32(x)); }
  static __device__ __forceinline__ T2 pair(float a, float b) { return make_float2(a, b); }
};

// Lemb[w][2a + co][2a' + ci] from L[w][a][a'] (chlB x chlK per channel)
template <bool TF32>
__global__ void k_lp_embed_L(const cplx* __restrict__ L, int D0, int chlB, int chlK,
                             typename Lp<TF32>::T* __restrict__ out, long long ld) {
  typedef typename Lp<TF32>::T T;
  const long long tot = (long long)D0 * chlB * chlK;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e % chlK);
    const long long wa = e / chlK;
    const int a = (int)(wa % chlB), w = (int)(wa / chlB);
    const cplx v = L[e];
    const T re = Lp<TF32>::from(v.x), im = Lp<TF32>::from(v.y), mim = Lp<TF32>::from(-v.y);
    T* r0 = out + ((long long)w * 2 * chlB + 2 * a) * ld + 2 * k;
    T* r1 = r0 + ld;
    *reinterpret_cast<typename Lp<TF32>::T2*>(r0) = Lp<TF32>::pair(re, mim);
    *reinterpret_cast<typename Lp<TF32>::T2*>(r1) = Lp<TF32>::pair(im, re);
  }
}

// Remb[2b + co][2(w chrK + b') + ci] from R[w][b'][b] (chrK x chrB per channel);
// consecutive threads take consecutive k = w chrK + b', so the embedded rows
// are written contiguously
template <bool TF32>
__global__ void k_lp_embed_R(const cplx* __restrict__ R, int D2, int chrK, int chrB,
                             typename Lp<TF32>::T* __restrict__ out, long long ld) {
  typedef typename Lp<TF32>::T T;
  const long long nk = (long long)D2 * chrK;
  const long long tot = nk * chrB;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long k = e % nk;                        // w chrK + b'
    const int b = (int)(e / nk);
    const cplx v = R[k * chrB + b];
    const T re = Lp<TF32>::from(v.x), im = Lp<TF32>::from(v.y), mim = Lp<TF32>::from(-v.y);
    T* r0 = out + (long long)(2 * b) * ld + 2 * k;
    T* r1 = r0 + ld;
    *reinterpret_cast<typename Lp<TF32>::T2*>(r0) = Lp<TF32>::pair(re, mim);
    *reinterpret_cast<typename Lp<TF32>::T2*>(r1) = Lp<TF32>::pair(im, re);
  }
}

// XT[n][2a' + c] = X[a'][n] (re, im), a 32 x 32 tile transpose through
// shared memory: coalesced reads along n, paired writes along a'
template <bool TF32>
__global__ void k_lp_xt(const cplx* __restrict__ X, int rows, long long n_cols,
                        typename Lp<TF32>::T* __restrict__ XT, long long ld) {
  typedef typename Lp<TF32>::T T;
  __shared__ cplx tile[32][33];
  const long long n0 = (long long)blockIdx.x * 32;
  const int a0 = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int a = a0 + y;
    const long long n = n0 + threadIdx.x;
    if (a < rows && n < n_cols) tile[y][threadIdx.x] = X[(long long)a * n_cols + n];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const long long n = n0 + y;
    const int a = a0 + threadIdx.x;
    if (a < rows && n < n_cols) {
      const cplx v = tile[threadIdx.x][y];
      T* dst = XT + n * ld + 2 * a;
      *reinterpret_cast<typename Lp<TF32>::T2*>(dst) = Lp<TF32>::pair(Lp<TF32>::from(v.x),
                                                                     Lp<TF32>::from(v.y));
    }
  }
}

// T2[(a s' t')][2 (w'' chrK + b') + c] = sum_e val_e T1[w_e][a][(s_e t_e) chrK + b']
// with T1[w][2a + c][n] (bf16, n = (s t) chrK + b'); the plan's rows are
// (s', t', w''), its columns (w, s, t).  One block per (a, MIX_B values of
// b'): the block stages the bf16 rows T1[w][2a + c][(s t) chrK + b0 ..] it
// needs in shared memory with 16-byte loads, and the plan (fp32 values,
// column indices) beside them; then thread (pair p, group g) forms the
// outputs k = g, g + groups, ... of the two values b' = b0 + 2p, b0 + 2p + 1
// (paired loads and stores halve the instructions per output).
// MIX_B (64, 128 or 256 values of b' per block) is chosen per shape so that a
// block stages about 24 KB: enough bytes in flight per SM to stream the
// L2-resident intermediates at a high rate.
template <bool TF32, int MIX_B>
__global__ void __launch_bounds__(256)
k_lp_mix(MixPlan pl, const __nv_bfloat16* __restrict__ T1, int chlB, int chrK, int d, int D0,
         int D2, long long N1, typename Lp<TF32>::T* __restrict__ T2, long long ld2) {
  typedef typename Lp<TF32>::T T;
  constexpr int MIX_P = MIX_B / 2;    // threads per group
  extern __shared__ uint4 smem_u4[];
  const int dd = d * d;
  const int ncol = D0 * dd;                              // (w, s t)
  const int nrow = 2 * ncol;                             // (w, s t, c) rows of MIX_B bf16
  __nv_bfloat16* st1 = reinterpret_cast<__nv_bfloat16*>(smem_u4);
  float2* sval = reinterpret_cast<float2*>(st1 + (size_t)nrow * MIX_B);
  int* scol = reinterpret_cast<int*>(sval + pl.nnz);
  int* srp = scol + pl.nnz;
  long long* roff = reinterpret_cast<long long*>(((uintptr_t)(srp + pl.nrows + 1) + 7) & ~uintptr_t(7));
  const int a = blockIdx.y;
  const int b0 = blockIdx.x * MIX_B;
  const int nthr = blockDim.x, tid = threadIdx.x;
  const int p = tid % MIX_P, g = tid / MIX_P, groups = nthr / MIX_P;
  for (int e = tid; e < pl.nnz; e += nthr) {
    sval[e] = pl.val32[e];
    scol[e] = pl.col[e];
  }
  for (int k = tid; k <= pl.nrows; k += nthr) srp[k] = pl.row_ptr[k];
  for (int j = tid; j < ncol; j += nthr) {
    const int w = j / dd, stt = j - w * dd;
    roff[j] = ((long long)w * 2 * chlB + 2 * a) * N1 + (long long)stt * chrK + b0;
  }
  __syncthreads();
  // staging: row r = 2 j + c; MIX_B / 8 chunks of 8 bf16 per row
  const bool vec = (chrK % 8 == 0) && (N1 % 8 == 0);
  constexpr int CH = MIX_B / 8;
  const int lim0 = chrK - b0;
  for (int item = tid; item < nrow * CH; item += nthr) {
    const int r = item / CH, ch = item - r * CH;
    const __nv_bfloat16* src = T1 + roff[r >> 1] + (r & 1) * N1 + ch * 8;
    __nv_bfloat16* dst = st1 + (size_t)r * MIX_B + ch * 8;
    const int lim = lim0 - ch * 8;
    if (vec && lim >= 8) {
      *reinterpret_cast<uint4*>(dst) = __ldcs(reinterpret_cast<const uint4*>(src));
    } else {
      for (int q = 0; q < 8; ++q) dst[q] = q < lim ? src[q] : __float2bfloat16_rn(0.f);
    }
  }
  __syncthreads();
  const int bp = b0 + 2 * p;
  if (bp >= chrK) return;
  const __nv_bfloat162* s2 = reinterpret_cast<const __nv_bfloat162*>(st1);
  for (int k = g; k < pl.nrows; k += groups) {
    float2 re = make_float2(0.f, 0.f), im = make_float2(0.f, 0.f);
    const int e1 = srp[k + 1];
    for (int e = srp[k]; e < e1; ++e) {
      const int j = scol[e];                            // (w d + s) d + t
      const float2 xr = __bfloat1622float2(s2[(size_t)(2 * j) * MIX_P + p]);
      const float2 xi = __bfloat1622float2(s2[(size_t)(2 * j + 1) * MIX_P + p]);
      const float2 v = sval[e];
      re.x = fmaf(v.x, xr.x, fmaf(-v.y, xi.x, re.x));
      re.y = fmaf(v.x, xr.y, fmaf(-v.y, xi.y, re.y));
      im.x = fmaf(v.x, xi.x, fmaf(v.y, xr.x, im.x));
      im.y = fmaf(v.x, xi.y, fmaf(v.y, xr.y, im.y));
    }
    const int wpp = k % D2, spt = k / D2;               // k = (s' d + t') D2 + w''
    T* dst = T2 + ((long long)a * dd + spt) * ld2 + 2LL * ((long long)wpp * chrK + bp);
    *reinterpret_cast<typename Lp<TF32>::T2*>(dst) =
        Lp<TF32>::pair(Lp<TF32>::fromf(re.x), Lp<TF32>::fromf(im.x));
    if (bp + 1 < chrK)
      *reinterpret_cast<typename Lp<TF32>::T2*>(dst + 2) =
          Lp<TF32>::pair(Lp<TF32>::fromf(re.y), Lp<TF32>::fromf(im.y));
  }
}

// Y[m][b] = alpha sum_sp (Y32[sp][m][2b], Y32[sp][m][2b+1]) + gamma Z[m][b],
// formed in fp32 (the product is good to the operand precision only, and
// GB300's FP64 pipe is 1/64 of its fp32 rate) and stored as FP64.  A
// separate pass: folded into the GEMM's epilogue, the dependent loads of Z
// row by row made that epilogue the bottleneck.
__global__ void k_lp_combine(const float* __restrict__ Y32, int splits, long long slab, long long M,
                             int ncols, float2 alpha, const cplx* __restrict__ Z, float2 gamma,
                             cplx* __restrict__ Y) {
  const long long tot = M * ncols;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    float re = 0.f, im = 0.f;
    for (int sp = 0; sp < splits; ++sp) {
      const float2 v = __ldcs(reinterpret_cast<const float2*>(Y32 + sp * slab) + e);
      re += v.x;
      im += v.y;
    }
    float ore = alpha.x * re - alpha.y * im, oim = alpha.x * im + alpha.y * re;
    if (Z) {
      const cplx z = __ldcs(Z + e);
      const float zr = dbl_to_f32(z.x), zi = dbl_to_f32(z.y);
      ore = fmaf(gamma.x, zr, fmaf(-gamma.y, zi, ore));
      oim = fmaf(gamma.x, zi, fmaf(gamma.y, zr, oim));
    }
    __stcs(Y + e, cmake(f32_to_dbl(ore), f32_to_dbl(oim)));
  }
}

int grid_of(long long tot, int threads) {
  long long g = (tot + threads - 1) / threads;
  if (g > 4096) g = 4096;
  if (g < 1) g = 1;
  return (int)g;
}

long long round_up(long long x, long long m) { return (x + m - 1) / m * m; }

// The N tile and K split of one GEMM, from a model of its time on `sms` SMs:
// the busiest SM runs ceil(units / sms) units, each costing its MMA work
// (columns x K tiles, the full tile width even where it overhangs N; a
// 128-wide tile runs at about 0.8 of the rate of a wider one) plus a fixed
// epilogue share; K splits add the pass that sums the partial slabs.
void pick_tiles(int M, int N, int K, int batch, bool tf32, int sms, int* bn, int* splits,
                int max_splits) {
  const int BK = tf32 ? 32 : 64;
  const int nkb = (K + BK - 1) / BK;
  double best = 1e300;
  *bn = 256;
  *splits = 1;
  for (int b : {256, 192, 128}) {
    const long long tiles = (long long)batch * ((M + 127) / 128) * ((N + b - 1) / b);
    for (int s = 1; s <= max_splits; ++s) {
      if (s > 1 && nkb / s < 4) break;
      const long long per = (nkb + s - 1) / s;
      const long long units = tiles * s;
      const long long waves = (units + sms - 1) / sms;
      const double t = waves * (b * per * (b == 128 ? 1.25 : 1.0) + 6.0 * b) +
                       (s > 1 ? 0.5 * s * (double)M * N / (128.0 * sms) : 0.0);
      if (t < best * 0.999) {
        best = t;
        *bn = b;
        *splits = s;
      }
    }
  }
}

// Tile autotuner: the first time a GEMM shape is seen on a device, every
// candidate (N tile 128/192/256, one CTA or a CTA pair per tile, K split up
// to max_splits) is timed on the caller's stream with CUDA events (three
// runs, the first discarded, the faster of the others) and the fastest kept
// for that shape; each candidate writes C, which the real
// launch then overwrites.
// While the stream is being captured into a graph, or if timing fails, the
// model of pick_tiles decides instead.
struct TileKey {
  int dev, M, N, K, batch, tf32, mode, max_splits;
  bool operator<(const TileKey& o) const {
    return std::tie(dev, M, N, K, batch, tf32, mode, max_splits) <
           std::tie(o.dev, o.M, o.N, o.K, o.batch, o.tf32, o.mode, o.max_splits);
  }
};
std::mutex g_tune_mu;
struct TileChoice {
  int bn, splits;
  bool pair;
};
std::map<TileKey, TileChoice> g_tuned;

cudaError_t tune_tiles(LpGemmArgs& g, int max_splits, int sms, int* err, cudaStream_t st) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  const TileKey key{dev, g.M, g.N, g.K, g.batch, g.tf32 ? 1 : 0,
                     g.out_complex ? 2 : (g.out_bf16 ? 1 : 0), max_splits};
  {
    std::lock_guard<std::mutex> lock(g_tune_mu);
    auto it = g_tuned.find(key);
    if (it != g_tuned.end()) {
      g.bn = it->second.bn;
      g.splits = it->second.splits;
      g.pair = it->second.pair;
      return cudaSuccess;
    }
  }
  pick_tiles(g.M, g.N, g.K, g.batch, g.tf32, sms, &g.bn, &g.splits, max_splits);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cap) != cudaSuccess || cap != cudaStreamCaptureStatusNone)
    return cudaSuccess;
  const int BK = g.tf32 ? 32 : 64;
  const int nkb = (g.K + BK - 1) / BK;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    cudaGetLastError();
    return cudaSuccess;
  }
  float best = 1e30f;
  int bbn = g.bn, bsp = g.splits;
  bool bpair = false;
  for (int pr = 0; pr < (g.M >= 256 ? 2 : 1); ++pr)
  for (int bn : {256, 192, 128}) {
    for (int sp : {1, 2, 3, 4, 6, 8}) {
      if (sp > max_splits || (sp > 1 && nkb / sp < 4)) continue;
      LpGemmArgs c = g;
      c.bn = bn;
      c.splits = sp;
      c.pair = pr == 1;
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {
        if (cudaEventRecord(e0, st) != cudaSuccess || lp_gemm(c, err, st) != cudaSuccess ||
            cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess) {
          ms = 1e30f;
          cudaGetLastError();
          break;
        }
        float t = 0.f;
        cudaEventElapsedTime(&t, e0, e1);
        if (rep > 0 && t < ms) ms = t;      // the first run pays one-time costs
      }
      if (ms < best) {
        best = ms;
        bbn = bn;
        bsp = sp;
        bpair = c.pair;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best < 1e29f) {
    g.bn = bbn;
    g.splits = bsp;
    g.pair = bpair;
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = {bbn, bsp, bpair};
  }
  return cudaSuccess;
}

}  // namespace

size_t heff_lp_operand_bytes(int D0, int D2, int chlB, int chlK, int chrK, int chrB, bool tf32) {
  const int eb = tf32 ? 4 : 2, al = 16 / eb;
  const long long ldl = round_up(2LL * chlK, al), ldr = round_up(2LL * D2 * chrK, al);
  return (size_t)(D0 * 2LL * chlB * ldl + 2LL * chrB * ldr) * eb + 512;
}

size_t heff_lp_scratch_bytes(int d, int D0, int D2, int chlB, int chlK, int chrK, int chrB,
                             bool tf32) {
  const int eb = tf32 ? 4 : 2, al = 16 / eb;
  const long long N1 = (long long)d * d * chrK, M3 = (long long)chlB * d * d;
  const long long ldx = round_up(2LL * chlK, al), ld2 = round_up(2LL * D2 * chrK, al);
  const size_t xt = (size_t)N1 * ldx * eb;
  const size_t t1 = (size_t)D0 * 2 * chlB * N1 * 2;
  const size_t t2 = (size_t)M3 * ld2 * eb;
  const size_t y32 = (size_t)8 * M3 * 2 * chrB * 4;
  return xt + t1 + t2 + y32 + 4 * 256;
}

cudaError_t heff_lp_prepare(const cplx* L, const cplx* R, int D0, int D2, int chlB, int chlK,
                            int chrK, int chrB, bool tf32, void* ops, size_t ops_bytes,
                            cudaStream_t st) {
  if (ops_bytes < heff_lp_operand_bytes(D0, D2, chlB, chlK, chrK, chrB, tf32))
    return cudaErrorInvalidValue;
  const int eb = tf32 ? 4 : 2, al = 16 / eb;
  const long long ldl = round_up(2LL * chlK, al), ldr = round_up(2LL * D2 * chrK, al);
  char* p = static_cast<char*>(ops);
  void* Lemb = p;
  void* Remb = p + round_up((long long)D0 * 2 * chlB * ldl * eb, 256);
  const long long nl = (long long)D0 * chlB * chlK, nr = (long long)D2 * chrK * chrB;
  count_launches(2);
  if (tf32) {
    k_lp_embed_L<true><<<grid_of(nl, 256), 256, 0, st>>>(L, D0, chlB, chlK, (float*)Lemb, ldl);
    k_lp_embed_R<true><<<grid_of(nr, 256), 256, 0, st>>>(R, D2, chrK, chrB, (float*)Remb, ldr);
  } else {
    k_lp_embed_L<false><<<grid_of(nl, 256), 256, 0, st>>>(L, D0, chlB, chlK, (__nv_bfloat16*)Lemb, ldl);
    k_lp_embed_R<false><<<grid_of(nr, 256), 256, 0, st>>>(R, D2, chrK, chrB, (__nv_bfloat16*)Remb, ldr);
  }
  return cudaGetLastError();
}

cudaError_t heff_lp_apply(const void* ops, const MixPlan& plan2, int d, int D0, int D2, int chlB,
                          int chlK, int chrK, int chrB, bool tf32, const cplx* X, cplx* Y,
                          cplx alpha, const cplx* Z, cplx gamma, void* scratch,
                          size_t scratch_bytes, int* err, cudaStream_t st) {
  if (scratch_bytes < heff_lp_scratch_bytes(d, D0, D2, chlB, chlK, chrK, chrB, tf32))
    return cudaErrorInvalidValue;
  const int eb = tf32 ? 4 : 2, al = 16 / eb;
  const long long N1 = (long long)d * d * chrK, M3 = (long long)chlB * d * d;
  const long long ldl = round_up(2LL * chlK, al), ldr = round_up(2LL * D2 * chrK, al);
  const long long ldx = round_up(2LL * chlK, al), ld2 = round_up(2LL * D2 * chrK, al);
  const char* po = static_cast<const char*>(ops);
  const void* Lemb = po;
  const void* Remb = po + round_up((long long)D0 * 2 * chlB * ldl * eb, 256);
  char* p = static_cast<char*>(scratch);
  void* XT = p;
  p += round_up(N1 * ldx * eb, 256);
  __nv_bfloat16* T1 = reinterpret_cast<__nv_bfloat16*>(p);
  p += round_up((long long)D0 * 2 * chlB * N1 * 2, 256);
  void* T2 = p;
  p += round_up(M3 * ld2 * eb, 256);
  float* Y32 = reinterpret_cast<float*>(p);
  const int sms = lp_gemm_sm_count() > 0 ? lp_gemm_sm_count() : 148;
  cudaError_t e;
  // 0. X^T in the operand precision
  {
    dim3 grid((unsigned)((N1 + 31) / 32), (unsigned)((chlK + 31) / 32));
    count_launches(1);
    if (tf32) k_lp_xt<true><<<grid, dim3(32, 8), 0, st>>>(X, chlK, N1, (float*)XT, ldx);
    else k_lp_xt<false><<<grid, dim3(32, 8), 0, st>>>(X, chlK, N1, (__nv_bfloat16*)XT, ldx);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  // 1. T1[w] = Lemb[w] XT^T: (2 chlB) x N1 per channel, K = 2 chlK
  {
    LpGemmArgs g = {};
    g.M = 2 * chlB; g.N = (int)N1; g.K = 2 * chlK; g.batch = D0; g.tf32 = tf32;
    g.A = Lemb; g.lda = ldl; g.sAb = 2LL * chlB * ldl;
    g.B = XT; g.ldb = ldx; g.sBb = 0;
    g.C = T1; g.ldc = N1; g.sCb = 2LL * chlB * N1; g.sCs = 0; g.out_bf16 = true;
    if ((e = tune_tiles(g, 1, sms, err, st)) != cudaSuccess) return e;
    if ((e = lp_gemm(g, err, st)) != cudaSuccess) return e;
  }
  // 2. mix into the K-major complex-interleaved T2
  {
    const int stage_row = 4 * D0 * d * d;        // bytes staged per value of b'
    const int mixb = stage_row * 256 <= 24 * 1024 ? 256 : (stage_row * 128 <= 24 * 1024 ? 128 : 64);
    dim3 grid((unsigned)((chrK + mixb - 1) / mixb), (unsigned)chlB);
    const size_t smem = (size_t)stage_row * mixb +
                        (size_t)plan2.nnz * (sizeof(float2) + sizeof(int)) +
                        (size_t)(plan2.nrows + 1) * sizeof(int) + 16 +
                        (size_t)D0 * d * d * sizeof(long long);
    if (smem > 200 * 1024) return cudaErrorInvalidValue;
    const void* fn = tf32 ? (mixb == 256 ? (const void*)k_lp_mix<true, 256>
                             : mixb == 128 ? (const void*)k_lp_mix<true, 128> : (const void*)k_lp_mix<true, 64>)
                          : (mixb == 256 ? (const void*)k_lp_mix<false, 256>
                             : mixb == 128 ? (const void*)k_lp_mix<false, 128> : (const void*)k_lp_mix<false, 64>);
    if (smem > 48 * 1024) {
      cudaError_t ea = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (ea != cudaSuccess) return ea;
    }
    // thread groups of mixb / 2 threads, each group taking every groups-th
    // output row; at most 256 threads, and no more groups than row pairs
    const int mixp = mixb / 2;
    int groups = plan2.nrows / 2;
    groups = groups < 1 ? 1 : (groups > 256 / mixp ? 256 / mixp : groups);
    count_launches(1);
    void* T2p = T2;
    MixPlan pl = plan2;
    int a_chlB = chlB, a_chrK = chrK, a_d = d, a_D0 = D0, a_D2 = D2;
    long long a_N1 = N1, a_ld2 = ld2;
    const __nv_bfloat16* T1c = T1;
    void* args[] = {&pl, &T1c, &a_chlB, &a_chrK, &a_d, &a_D0, &a_D2, &a_N1, &T2p, &a_ld2};
    if ((e = cudaLaunchKernel(fn, grid, dim3(mixp * groups), args, smem, st)) != cudaSuccess) return e;
  }
  // 3. Y32[sp] = T2 Remb^T: M3 x (2 chrB), K = 2 D2 chrK, split over K
  int splits = 1;
  {
    LpGemmArgs g = {};
    g.M = (int)M3; g.N = 2 * chrB; g.K = (int)(2LL * D2 * chrK); g.batch = 1; g.tf32 = tf32;
    g.A = T2; g.lda = ld2; g.sAb = 0;
    g.B = Remb; g.ldb = ldr; g.sBb = 0;
    g.C = Y32; g.ldc = 2LL * chrB; g.sCb = 0; g.sCs = M3 * 2LL * chrB;
    if ((e = tune_tiles(g, 8, sms, err, st)) != cudaSuccess) return e;
    splits = lp_gemm_splits_used(g);
    if (splits > 8) return cudaErrorInvalidValue;
    if ((e = lp_gemm(g, err, st)) != cudaSuccess) return e;
  }
  // 4. Y = alpha Y32 + gamma Z
  count_launches(1);
  k_lp_combine<<<grid_of(M3 * chrB, 256), 256, 0, st>>>(
      Y32, splits, M3 * 2LL * chrB, M3, chrB, make_float2((float)alpha.x, (float)alpha.y), Z,
      make_float2((float)gamma.x, (float)gamma.y), Y);
  return cudaGetLastError();
}

}  // namespace ite
