// FP64 truncated SVD of the two-site blocks and of the gauge moves.
//
// For a p x q complex matrix Xr (row-major), whose rows are indexed by the
// side whose isometry is wanted, the split runs
//   1. a Householder LQ of the rows, Xr H_0 H_1 ... H_{k-1} = L (p x k lower
//      trapezoidal, k = min(p, q)), all k reflector steps in one cooperative
//      launch;
//   2. R = L^H (k x p, upper trapezoidal), so that R^H R = Xr Xr^H: the rows
//      of R carry the left singular structure of Xr and are graded like its
//      singular values, which is what lets the Jacobi below converge in few
//      sweeps (QR preconditioning of the one-sided Jacobi method);
//   3. one-sided (Hestenes) Jacobi on the rows of R until they are mutually
//      orthogonal: R_out = Sigma U^H, U the left singular vectors of Xr;
//   4. row norms, the descending order and the truncation rule; the kept
//      rows of U^H are the rows of R_out divided by their norms.
// No rotation is accumulated: the engine forms the other factor as the
// projection U_r^H Xr with one GEMM.
#include <mutex>

#include "common.cuh"

namespace ite {
namespace {

constexpr int JT = 128;   // threads of the LQ and row-norm blocks

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// Sums of a and b over the JT threads of the block, returned to every thread
// (fixed order, so deterministic).  sh holds JT/32 doubles per value.
__device__ __forceinline__ void block_sum2(double& a, double& b, double (*sh)[JT / 32]) {
  a = warp_sum(a);
  b = warp_sum(b);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();                 // sh may still be read from its previous use
  if (lane == 0) {
    sh[0][wid] = a;
    sh[1][wid] = b;
  }
  __syncthreads();
  a = 0.0;
  b = 0.0;
#pragma unroll
  for (int w = 0; w < JT / 32; ++w) {
    a += sh[0][w];
    b += sh[1][w];
  }
}

__device__ __forceinline__ int player(int pos, int round, int pp) {
  return pos == 0 ? 0 : ((pos - 1 + round) % (pp - 1)) + 1;
}

// Grid-wide barrier for a cooperative launch.  st[0] arrivals, st[1]
// generation, st[4] error flag.  Waits are bounded: after ~2^24 polls the
// error flag is set and the block leaves (the caller then exits); a wait also
// gives up as soon as another block has set the flag.
__device__ bool grid_barrier(unsigned int* st, unsigned int nblocks) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* gen = st + 1;
    const unsigned int g = *gen;
    __threadfence();
    const unsigned int ticket = atomicAdd(st, 1u);
    if (ticket == nblocks - 1) {
      atomicExch(st, 0u);
      __threadfence();
      atomicAdd(st + 1, 1u);
    } else {
      unsigned long long spins = 0;
      while (*gen == g) {
        if (*((volatile unsigned int*)(st + 4)) != 0u) break;
        if (++spins > (1ull << 24)) {
          atomicExch(st + 4, 1u);
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *((volatile unsigned int*)(st + 4)) == 0u;
}

// ------------------------------------------------------------ Householder LQ
// Step j takes the tail x = W[j][j..q) of row j and the reflector
// H = I - c u^H u (u a row vector) with x H = beta e_0:
//   beta = -e^{i phi} |x|,  u_0 = e^{i phi} (|x_0| + |x|),  u_e = x_e (e > 0),
//   c = 1 / (|x| (|x| + |x_0|)),  phi = arg x_0,
// and applies it to every later row: y <- y - c (y u^H) u.  Row j itself is
// left as it is (it holds u beyond position j); beta goes to beta[j].  Every
// block recomputes the reflector of step j from row j, which no block writes
// during step j; one grid barrier separates the steps.
__global__ void __launch_bounds__(JT)
k_lq_persistent(cplx* W, int p, int q, cplx* beta, double* refl, unsigned int* st) {
  __shared__ double sh[2][JT / 32];
  __shared__ double hs[3];
  const int k = p < q ? p : q;
  const unsigned int nb = gridDim.x;
  for (int j = 0; j < k; ++j) {
    const cplx* x = W + (long long)j * q;
    double s = 0.0, unused = 0.0;
    for (int e = j + threadIdx.x; e < q; e += JT) s = fma(x[e].x, x[e].x, fma(x[e].y, x[e].y, s));
    block_sum2(s, unused, sh);
    if (threadIdx.x == 0) {
      const cplx x0 = x[j];
      const double nx = sqrt(s), a0 = hypot(x0.x, x0.y);
      const double phr = a0 > 0.0 ? x0.x / a0 : 1.0, phi = a0 > 0.0 ? x0.y / a0 : 0.0;
      hs[0] = phr * (a0 + nx);
      hs[1] = phi * (a0 + nx);
      hs[2] = nx > 0.0 ? 1.0 / (nx * (nx + a0)) : 0.0;
      if (blockIdx.x == 0) {
        beta[j] = cmake(-phr * nx, -phi * nx);
        if (refl) {
          refl[3 * j] = hs[0];
          refl[3 * j + 1] = hs[1];
          refl[3 * j + 2] = hs[2];
        }
      }
    }
    __syncthreads();
    const double c = hs[2];
    const cplx u0 = cmake(hs[0], hs[1]);
    if (c != 0.0) {
      for (int i = j + 1 + (int)blockIdx.x; i < p; i += (int)nb) {
        cplx* y = W + (long long)i * q;
        double dr = 0.0, di = 0.0;     // y u^H
        for (int e = j + threadIdx.x; e < q; e += JT) {
          const cplx u = e == j ? u0 : x[e];
          const cplx v = y[e];
          dr = fma(v.x, u.x, fma(v.y, u.y, dr));
          di = fma(v.y, u.x, fma(-v.x, u.y, di));
        }
        block_sum2(dr, di, sh);
        const double fr = c * dr, fi = c * di;
        for (int e = j + threadIdx.x; e < q; e += JT) {
          const cplx u = e == j ? u0 : x[e];
          cplx v = y[e];
          v.x -= fr * u.x - fi * u.y;
          v.y -= fr * u.y + fi * u.x;
          y[e] = v;
        }
      }
    }
    if (!grid_barrier(st, nb)) return;
  }
}

// R (k x p) = L^H: R[j][i] = conj(L[i][j]); L[i][j] = W[i][j] below the
// diagonal, beta[j] on it, zero above.
__global__ void k_lq_r(const cplx* W, const cplx* beta, int p, int q, int k, cplx* R) {
  const long long tot = (long long)k * p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int j = (int)(e / p), i = (int)(e - (long long)j * p);
    cplx v = cmake(0.0, 0.0);
    if (i > j) v = cconj(W[(long long)i * q + j]);
    else if (i == j) v = cconj(beta[j]);
    R[e] = v;
  }
}

// L (p x k, row-major, lower trapezoidal) from the output of the LQ
__global__ void k_lq_left(const cplx* W, const cplx* beta, int p, int q, int k, cplx* Lout) {
  const long long tot = (long long)p * k;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / k), j = (int)(e - (long long)i * k);
    cplx v = cmake(0.0, 0.0);
    if (j < i) v = W[(long long)i * q + j];
    else if (j == i) v = beta[i];
    Lout[e] = v;
  }
}

// |column c of L1^{-1}|^2 for the leading k x k triangle L1 of the LQ, by
// forward substitution (one warp per column, the solution in shared memory):
// z_c = 1 / L_cc, z_i = -(sum_{c <= j < i} L_ij z_j) / L_ii.  A zero pivot
// gives +inf.
__global__ void __launch_bounds__(32)
k_tri_inv_colnorm(const cplx* W, const cplx* beta, int q, int k, double* colnorm2) {
  extern __shared__ cplx zs[];
  const int c = blockIdx.x, lane = threadIdx.x;
  double acc = 0.0;
  bool singular = false;
  for (int i = c; i < k && !singular; ++i) {
    double sr = 0.0, si = 0.0;
    if (i > c) {
      const cplx* row = W + (long long)i * q;
      for (int j = c + lane; j < i; j += 32) {
        const cplx l = row[j], z = zs[j];
        sr = fma(l.x, z.x, fma(-l.y, z.y, sr));
        si = fma(l.x, z.y, fma(l.y, z.x, si));
      }
      sr = warp_sum(sr);
      si = warp_sum(si);
    }
    if (lane == 0) {
      const cplx b = beta[i];
      const double bb = b.x * b.x + b.y * b.y;
      cplx z;
      if (bb == 0.0) {
        z = cmake(0.0, 0.0);
      } else if (i == c) {
        z = cmake(b.x / bb, -b.y / bb);                    // 1 / b
      } else {
        // -(s / b) = -s conj(b) / |b|^2
        z = cmake(-(sr * b.x + si * b.y) / bb, -(si * b.x - sr * b.y) / bb);
      }
      zs[i] = z;
      acc += z.x * z.x + z.y * z.y;
      if (bb == 0.0) acc = INFINITY;
    }
    singular = __shfl_sync(0xffffffffu, isinf(acc) ? 1 : 0, 0) != 0;
    __syncwarp();
  }
  if (lane == 0) colnorm2[c] = acc;
}

// *out = sum of x[0..n) in a fixed order (one block)
__global__ void k_sum_small(const double* x, int n, double* out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
    *out = t;
  }
}

// rows of the k x q identity
__global__ void k_eye_rows(cplx* Q, int k, int q) {
  const long long tot = (long long)k * q;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int i = (int)(e / q), j = (int)(e - (long long)i * q);
    Q[e] = cmake(i == j ? 1.0 : 0.0, 0.0);
  }
}

// Q^H (k x q, orthonormal rows) with X = L Q^H, from the reflectors of the
// LQ: the reflectors are Hermitian, so Q^H is the first k rows of
// H_{k-1} ... H_0, accumulated backwards: starting from identity rows, step
// j = k-1, ..., 0 applies y <- y - c_j (y u_j^H) u_j to rows j..k-1 (rows
// above j are still unit vectors that H_j leaves alone).  One grid barrier
// separates the steps.
__global__ void __launch_bounds__(JT)
k_lq_formq(const cplx* W, const double* refl, int q, int k, cplx* Qh, unsigned int* st) {
  __shared__ double sh[2][JT / 32];
  const unsigned int nb = gridDim.x;
  for (int j = k - 1; j >= 0; --j) {
    const double c = refl[3 * j + 2];
    const cplx u0 = cmake(refl[3 * j], refl[3 * j + 1]);
    const cplx* x = W + (long long)j * q;
    if (c != 0.0) {
      for (int i = j + (int)blockIdx.x; i < k; i += (int)nb) {
        cplx* y = Qh + (long long)i * q;
        double dr = 0.0, di = 0.0;     // y u^H
        for (int e = j + threadIdx.x; e < q; e += JT) {
          const cplx u = e == j ? u0 : x[e];
          const cplx v = y[e];
          dr = fma(v.x, u.x, fma(v.y, u.y, dr));
          di = fma(v.y, u.x, fma(-v.x, u.y, di));
        }
        block_sum2(dr, di, sh);
        const double fr = c * dr, fi = c * di;
        for (int e = j + threadIdx.x; e < q; e += JT) {
          const cplx u = e == j ? u0 : x[e];
          cplx v = y[e];
          v.x -= fr * u.x - fi * u.y;
          v.y -= fr * u.y + fi * u.x;
          y[e] = v;
        }
      }
    }
    if (!grid_barrier(st, nb)) return;
  }
}

// ---------------------------------------------------------- one-sided Jacobi
// GB300 runs FP64 on a narrow pipe (2 DFMA per clock per SM), so the Jacobi
// is arranged to issue little besides the inner products and the rotation
// itself, with enough independent FP64 work in flight to hide the pipe's
// latency: one team of TPP threads (two warps) per pair of rows, each thread
// holding its len/TPP elements of both rows in registers (one load, one
// store), four independent partial sums per quantity, warp shuffles plus one
// shared-memory exchange, and the rotation parameters formed by thread 0.

// words of the Jacobi state (dev_state, 24 words): grid barrier (0, 1), error
// flag, sweeps done, pairs examined and rotated, two per-sweep rotation
// counters and two per-sweep maxw values (64-bit, 8-byte aligned)
constexpr int S_ARRIVE = 0, S_GEN = 1, S_ERR = 4, S_SWEEPS = 5, S_EXAMINED = 6, S_ROTATED = 7,
              S_CNT = 8, S_MAXW = 12, S_WORDS = 24;
static_assert(S_ERR == 4, "grid_barrier uses word 4 as its error flag");

constexpr int TPP = 64;                 // threads per pair (one block)
constexpr int TPW = TPP / 32;           // warps per pair

__device__ __forceinline__ double warp_allsum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

struct PairOut {
  bool rotated, counted;
  double al, be;       // squared norms before the rotation (every thread)
};

// Row norms are tracked (Hestenes): a rotation that makes rows u, v orthogonal
// moves t|gamma| of squared norm from one to the other, alpha' = alpha - t|g|,
// beta' = beta + t|g|, so examining a pair needs only the inner product
// gamma = a_u^H a_v.  A tracked norm that falls below a tenth of the value last
// computed from the row itself is recomputed from the rotated row (the
// subtraction loses digits as it shrinks).  wts[row] holds the tracked squared
// norm, nref[row] the last computed one.
//
// Rotation parameters with one square root and one division: with
// Delta = beta - alpha and g2 = |gamma|^2,
//   u = 2 / (|Delta| + sqrt(Delta^2 + 4 g2)),  t = sign(Delta) u |gamma|,
//   c = 1 / sqrt(1 + u^2 g2),  s e^{i theta} = c u sign(Delta) gamma,
// (sign(0) = +1), the same rotation as t = sign(zeta) / (|zeta| +
// sqrt(1 + zeta^2)) with zeta = Delta / (2 |gamma|).  Squaring Delta limits
// this form to rows of norm above about 1e-77.
constexpr int F_ROT = 1, F_COUNT = 2, F_RECOMP_U = 4, F_RECOMP_V = 8;
constexpr double kRecomputeFrac = 0.1;

// Team-wide sums of the two inner-product partials, then the rotation of the
// pair formed by thread 0 and shared with the team.  Two block barriers;
// every read of the shared scratch precedes the barrier before its next write.
__device__ __forceinline__ void pair_decide(double gr, double gi, double al, double be,
                                            double ref_u, double ref_v, double tol, double skip,
                                            double& c, double& sr, double& si, int& flags,
                                            double& al2, double& be2) {
  __shared__ double red[TPW][2];
  __shared__ double par[6];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  gr = warp_allsum(gr);
  gi = warp_allsum(gi);
  if (lane == 0) {
    red[w][0] = gr;
    red[w][1] = gi;
  }
  __syncthreads();
  gr = gi = 0.0;
#pragma unroll
  for (int k = 0; k < TPW; ++k) {
    gr += red[k][0];
    gi += red[k][1];
  }
  if (tid == 0) {
    double cc = 1.0, r0 = 0.0, i0 = 0.0, a2 = al, b2 = be;
    int f = 0;
    const double g2 = fma(gr, gr, gi * gi);
    // A pair of rows both below the skip weight can never be kept: their
    // mutual orthogonality does not matter (their total weight does, and
    // rotations preserve it).
    if (g2 > tol * tol * al * be && g2 > 0.0 && (al > skip || be > skip)) {
      const double D = be - al;
      const double u = 2.0 / (fabs(D) + sqrt(fma(D, D, 4.0 * g2)));
      const double ug2 = u * u * g2;
      cc = rsqrt(1.0 + ug2);
      const double cu = D >= 0.0 ? cc * u : -cc * u;
      r0 = cu * gr;
      i0 = cu * gi;                            // s e^{i theta}
      const double tg = D >= 0.0 ? u * g2 : -u * g2;   // t |gamma|
      a2 = al - tg;
      b2 = be + tg;
      f = F_ROT;
      // A rotation counts towards another sweep when it changes the heavier
      // row by more than tol (relative): |t| sqrt(min / max) > tol, i.e. the
      // angle itself for rows of similar weight, less against a much lighter
      // row, whose leftover overlap moves the heavier row by only that much.
      // Rotations against rows below the skip weight never count: those rows
      // are never rotated among themselves, so they stay a non-orthogonal
      // set, and orthogonalising a kept row against all of them one pair at a
      // time converges only slowly; its overlap with them changes the kept
      // product at second order.
      const double lo = fmin(al, be), hi = fmax(al, be);
      if (ug2 * lo > tol * tol * hi && al > skip && be > skip) f |= F_COUNT;
      if (a2 < kRecomputeFrac * ref_u) f |= F_RECOMP_U;
      if (b2 < kRecomputeFrac * ref_v) f |= F_RECOMP_V;
    }
    par[0] = cc;
    par[1] = r0;
    par[2] = i0;
    par[3] = (double)f;
    par[4] = a2;
    par[5] = b2;
  }
  __syncthreads();
  c = par[0];
  sr = par[1];
  si = par[2];
  flags = (int)par[3];
  al2 = par[4];
  be2 = par[5];
}

// team-wide sum (every thread gets it); the scratch is read before the next
// barrier of pair_decide writes its own
__device__ __forceinline__ double team_sum(double v) {
  __shared__ double red1[TPW];
  const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
  v = warp_allsum(v);
  __syncthreads();
  if (lane == 0) red1[w] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < TPW; ++k) s += red1[k];
  return s;
}

// a_u' = c a_u - s e^{-i theta} a_v ;  a_v' = s e^{i theta} a_u + c a_v
__device__ __forceinline__ void rotate(cplx& x, cplx& y, double c, double sr, double si) {
  const cplx x0 = x, y0 = y;
  x = cmake(c * x0.x - (sr * y0.x + si * y0.y), c * x0.y - (sr * y0.y - si * y0.x));
  y = cmake((sr * x0.x - si * x0.y) + c * y0.x, (sr * x0.y + si * x0.x) + c * y0.y);
}

// Finishes a pair after its rotation: recomputed norms where flagged, tracked
// norms written back by thread 0.
__device__ __forceinline__ void pair_norms_out(int u, int v, int flags, double al2, double be2,
                                               double su, double sv, double* wts, double* nref) {
  if (flags & F_RECOMP_U) al2 = team_sum(su);
  if (flags & F_RECOMP_V) be2 = team_sum(sv);
  if (threadIdx.x == 0) {
    wts[u] = al2;
    wts[v] = be2;
    if (flags & F_RECOMP_U) nref[u] = al2;
    if (flags & F_RECOMP_V) nref[v] = be2;
  }
}

// One Jacobi rotation on rows u < v (length len <= TPP EPL) of A by the team,
// the rows held in registers.  With last >= 0 the pair is skipped (*skipped
// set, nothing written) when neither row has been rotated since global round
// `last` (stamps); the stamps are loaded together with the rows, so a round
// costs one L2 round trip before the arithmetic instead of two.
template <int EPL>
__device__ PairOut pair_regs(cplx* A, int len, int u, int v, double tol, double skip, double* wts,
                             double* nref, const int* stamps, int last, bool* skipped) {
  const int tid = threadIdx.x;
  cplx* au = A + (long long)u * len;
  cplx* av = A + (long long)v * len;
  cplx x[EPL], y[EPL];
  // rows, norms and stamps come from other SMs' rotations: read through L2, so
  // that every thread sees the same stamps and the block takes one branch
  const int stu = last >= 0 ? __ldcg(stamps + u) : 0, stv = last >= 0 ? __ldcg(stamps + v) : 0;
  const double al = __ldcg(wts + u), be = __ldcg(wts + v);
  const double ru = __ldcg(nref + u), rv = __ldcg(nref + v);
#pragma unroll
  for (int i = 0; i < EPL; ++i) {
    const int e = tid + TPP * i;
    x[i] = e < len ? __ldcg(au + e) : cmake(0.0, 0.0);
    y[i] = e < len ? __ldcg(av + e) : cmake(0.0, 0.0);
  }
  PairOut out;
  if (last >= 0 && stu <= last && stv <= last) {
    *skipped = true;
    out.rotated = out.counted = false;
    out.al = al;
    out.be = be;
    return out;
  }
  // independent partial sums keep the dependent FP64 chains short
  constexpr int NP = EPL < 4 ? EPL : 4;
  double pr[NP], pi[NP];
#pragma unroll
  for (int a = 0; a < NP; ++a) pr[a] = pi[a] = 0.0;
#pragma unroll
  for (int i = 0; i < EPL; ++i) {
    const int a = i % NP;
    pr[a] = fma(x[i].x, y[i].x, fma(x[i].y, y[i].y, pr[a]));     // Re(conj(x) y)
    pi[a] = fma(x[i].x, y[i].y, fma(-x[i].y, y[i].x, pi[a]));    // Im(conj(x) y)
  }
  double gr = 0.0, gi = 0.0;
#pragma unroll
  for (int a = 0; a < NP; ++a) {
    gr += pr[a];
    gi += pi[a];
  }
  double c, sr, si, al2, be2;
  int flags;
  pair_decide(gr, gi, al, be, ru, rv, tol, skip, c, sr, si, flags, al2, be2);
  out.rotated = (flags & F_ROT) != 0;
  out.counted = (flags & F_COUNT) != 0;
  out.al = al;
  out.be = be;
  if (out.rotated) {
    double su = 0.0, sv = 0.0;
#pragma unroll
    for (int i = 0; i < EPL; ++i) {
      const int e = tid + TPP * i;
      rotate(x[i], y[i], c, sr, si);
      if (e < len) {
        au[e] = x[i];
        av[e] = y[i];
      }
    }
    if (flags & (F_RECOMP_U | F_RECOMP_V)) {
#pragma unroll
      for (int i = 0; i < EPL; ++i) {
        su = fma(x[i].x, x[i].x, fma(x[i].y, x[i].y, su));
        sv = fma(y[i].x, y[i].x, fma(y[i].y, y[i].y, sv));
      }
    }
    pair_norms_out(u, v, flags, al2, be2, su, sv, wts, nref);
  }
  return out;
}

// The same for rows of any length, streamed from memory twice.
__device__ PairOut pair_stream(cplx* A, int len, int u, int v, double tol, double skip,
                               double* wts, double* nref) {
  const int tid = threadIdx.x;
  cplx* au = A + (long long)u * len;
  cplx* av = A + (long long)v * len;
  const double al = __ldcg(wts + u), be = __ldcg(wts + v);
  const double ru = __ldcg(nref + u), rv = __ldcg(nref + v);
  double gr = 0, gi = 0;
#pragma unroll 4
  for (int e = tid; e < len; e += TPP) {
    const cplx x = __ldcg(au + e), y = __ldcg(av + e);
    gr = fma(x.x, y.x, fma(x.y, y.y, gr));
    gi = fma(x.x, y.y, fma(-x.y, y.x, gi));
  }
  PairOut out;
  double c, sr, si, al2, be2;
  int flags;
  pair_decide(gr, gi, al, be, ru, rv, tol, skip, c, sr, si, flags, al2, be2);
  out.rotated = (flags & F_ROT) != 0;
  out.counted = (flags & F_COUNT) != 0;
  out.al = al;
  out.be = be;
  if (out.rotated) {
    double su = 0.0, sv = 0.0;
#pragma unroll 4
    for (int e = tid; e < len; e += TPP) {
      cplx x = __ldcg(au + e), y = __ldcg(av + e);
      rotate(x, y, c, sr, si);
      au[e] = x;
      av[e] = y;
      su = fma(x.x, x.x, fma(x.y, x.y, su));
      sv = fma(y.x, y.x, fma(y.y, y.y, sv));
    }
    pair_norms_out(u, v, flags, al2, be2, su, sv, wts, nref);
  }
  return out;
}

// The pair (u, v) of A; with last >= 0 it is skipped (*skipped set) when
// neither row has been rotated since global round `last`.
__device__ __forceinline__ PairOut jacobi_pair(cplx* A, int len, int u, int v, double tol,
                                               double skip, double* wts, double* nref,
                                               const int* stamps, int last, bool* skipped) {
  if (u > v) { const int t = u; u = v; v = t; }
  *skipped = false;
  if (len <= 2 * TPP) return pair_regs<2>(A, len, u, v, tol, skip, wts, nref, stamps, last, skipped);
  if (len <= 4 * TPP) return pair_regs<4>(A, len, u, v, tol, skip, wts, nref, stamps, last, skipped);
  if (len <= 8 * TPP) return pair_regs<8>(A, len, u, v, tol, skip, wts, nref, stamps, last, skipped);
  if (len <= 16 * TPP)
    return pair_regs<16>(A, len, u, v, tol, skip, wts, nref, stamps, last, skipped);
  if (last >= 0 && __ldcg(stamps + u) <= last && __ldcg(stamps + v) <= last) {
    *skipped = true;
    PairOut out;
    out.rotated = out.counted = false;
    out.al = out.be = 0.0;
    return out;
  }
  return pair_stream(A, len, u, v, tol, skip, wts, nref);
}

// Squared norms of rows [r0, r1) by one team, written to wts and nref.
__device__ void team_row_norms(const cplx* A, int len, int r0, int r1, int step, double* wts,
                               double* nref) {
  for (int r = r0; r < r1; r += step) {
    const cplx* a = A + (long long)r * len;
    double s = 0.0;
    for (int e = threadIdx.x; e < len; e += TPP) s = fma(a[e].x, a[e].x, fma(a[e].y, a[e].y, s));
    s = team_sum(s);
    if (threadIdx.x == 0) {
      wts[r] = s;
      nref[r] = s;
    }
  }
}

// A single pair (rows == 2), one team.
__global__ void __launch_bounds__(TPP)
k_jacobi_round(cplx* A, int len, double tol, const double* anorm2, double skip_rel,
               unsigned int* st, double* wts, double* nref) {
  const double a2 = anorm2 ? *anorm2 : 0.0;
  team_row_norms(A, len, 0, 2, 1, wts, nref);
  __syncthreads();
  bool skipped;
  const PairOut o = jacobi_pair(A, len, 0, 1, tol, skip_rel * a2, wts, nref, nullptr, -1, &skipped);
  if (threadIdx.x == 0) {
    if (o.counted) atomicAdd(st + S_CNT, 1u);
    atomicAdd(st + S_EXAMINED, 1u);
    if (o.rotated) atomicAdd(st + S_ROTATED, 1u);
  }
}

// All sweeps of the round-robin one-sided Jacobi in one cooperative launch;
// pair slot k of every round goes to block k of the grid (and k + blocks,
// ...), one grid barrier after every round.  (Tracking each row's completed round
// instead, so that a pair waits only for its own two rows, measured slower on
// GB300: the per-pair fence and flag round trip cost more than the barrier.)
//
// Termination.  A sweep with no counted rotation (every rotation changed the
// heavier of its rows by at most tol) ends the iteration.  So does a sweep in
// which every counted rotation was between two rows too light to be kept:
// with maxw the largest max(alpha, beta) over the counted rotations of the
// sweep, if at least keep_rank rows weigh more than maxw / kKeepMargin, the
// truncation, which keeps at most keep_rank rows, keeps none of the rows that
// still rotate, and their rotations leave every kept row as it is.
// wts[row] holds the row's tracked squared norm.
//
// The counters and maxw of sweep sw live in slot sw % 2.  A sweep's slot is
// read by every block after the sweep's last barrier; the slot of the
// following sweep is cleared by block 0 in round 1 of the current sweep,
// after every block has passed round 0 (and so has finished reading it two
// sweeps ago).
// stamps[row] holds the global round at which the row was last rotated.  The
// tournament repeats every sweep, so a pair was last examined pp-1 rounds ago;
// if neither row has been rotated since then (a rotation at that very round
// left the pair orthogonal), examining it again cannot fire and is skipped.
constexpr double kKeepMargin = 1e-2;
__global__ void __launch_bounds__(TPP)
k_jacobi_persistent(cplx* A, int rows, int len, int pp, double tol, const double* anorm2,
                    double skip_rel, int max_sweeps, int keep_rank, unsigned int* st, int* stamps,
                    double* wts, double* nref) {
  const unsigned int nb = gridDim.x;
  const int tid = threadIdx.x;
  const double skip = skip_rel * (anorm2 ? *anorm2 : 0.0);
  int* counters = reinterpret_cast<int*>(st + S_CNT);
  unsigned long long* maxws = reinterpret_cast<unsigned long long*>(st + S_MAXW);
  unsigned int examined = 0, rotations_done = 0;
  // the tracked squared norms start from the rows themselves
  team_row_norms(A, len, blockIdx.x, rows, (int)nb, wts, nref);
  if (!grid_barrier(st, nb)) return;
  for (int sw = 0; sw < max_sweeps; ++sw) {
    int* cnt = counters + (sw & 1);
    unsigned long long* maxw = maxws + (sw & 1);
    for (int r = 0; r < pp - 1; ++r) {
      if (r == 1 && blockIdx.x == 0 && threadIdx.x == 0) {
        counters[(sw + 1) & 1] = 0;
        maxws[(sw + 1) & 1] = 0ull;
      }
      const int g = sw * (pp - 1) + r;
      for (int k = blockIdx.x; k < pp / 2; k += (int)nb) {
        int u = player(k, r, pp), v = player(pp - 1 - k, r, pp);
        if (u >= rows || v >= rows) continue;
        if (u > v) { const int t = u; u = v; v = t; }
        // from the second sweep on, a pair neither of whose rows has been
        // rotated since it was last examined is skipped
        bool skipped;
        const PairOut o = jacobi_pair(A, len, u, v, tol, skip, wts, nref, stamps,
                                      sw > 0 ? g - (pp - 1) : -1, &skipped);
        if (skipped) continue;
        ++examined;
        if (o.rotated) {
          ++rotations_done;
          if (tid == 0) {
            stamps[u] = g;
            stamps[v] = g;
            if (o.counted) {
              atomicAdd(cnt, 1);
              // squared norms are non-negative: their bit patterns order like them
              atomicMax(maxw, (unsigned long long)__double_as_longlong(fmax(o.al, o.be)));
            }
          }
        }
      }
      if (!grid_barrier(st, nb)) break;
    }
    if (*((volatile unsigned int*)(st + S_ERR)) != 0u) break;
    if (blockIdx.x == 0 && threadIdx.x == 0) st[S_SWEEPS] = (unsigned int)(sw + 1);
    const int rotations = *((volatile int*)cnt);
    if (rotations == 0) break;
    if (keep_rank < rows) {
      // same data and order in every block, so every block decides alike
      const double thr = __longlong_as_double((long long)__ldcg(maxw)) / kKeepMargin;
      int heavy = 0;
      for (int i0 = 0; i0 < rows; i0 += blockDim.x) {
        const int i = i0 + threadIdx.x;
        heavy += __syncthreads_count(i < rows && __ldcg(wts + i) > thr);
      }
      if (heavy >= keep_rank) break;
    }
  }
  if (tid == 0) {
    atomicAdd(st + S_EXAMINED, examined);
    atomicAdd(st + S_ROTATED, rotations_done);
  }
}

// The same Jacobi for several independent matrices in one cooperative launch
// (the splits of concurrent evolutions).  Every matrix runs its own
// round-robin tournament from global round 0, one round per global round, so
// that its round G is round G % (pp - 1) of sweep G / (pp - 1); the pairs of
// all matrices still sweeping are spread over the blocks, and one grid
// barrier follows every global round.  Each matrix's pairs, stamps, counters
// and stopping rule are those of k_jacobi_persistent, and a pair's arithmetic
// does not depend on the block that takes it, so each matrix ends bit for bit
// as it would alone.  Matrices need pp >= 4 (at least 3 rows).  gst holds the
// group's barrier (words 0, 1) and error flag (word 4); on a failed wait every
// matrix's error word is set.
__global__ void __launch_bounds__(TPP)
k_jacobi_grouped(const __grid_constant__ JacobiGroup g, unsigned int* gst) {
  const unsigned int nb = gridDim.x;
  const int tid = threadIdx.x;
  __shared__ unsigned int s_ex[kJacobiGroupMax], s_rot[kJacobiGroupMax];
  __shared__ int s_done[kJacobiGroupMax], s_act[kJacobiGroupMax];
  __shared__ double s_skip[kJacobiGroupMax];
  const int n = g.n;
  for (int j = tid; j < n; j += TPP) {
    s_ex[j] = s_rot[j] = 0u;
    s_done[j] = 0;
    s_skip[j] = g.it[j].skip_rel * (g.it[j].anorm2 ? *g.it[j].anorm2 : 0.0);
  }
  __syncthreads();
  // the tracked squared norms start from the rows themselves
  int total_rows = 0;
  for (int j = 0; j < n; ++j) total_rows += g.it[j].rows;
  for (int f = blockIdx.x; f < total_rows; f += (int)nb) {
    int j = 0, r = f;
    while (r >= g.it[j].rows) r -= g.it[j++].rows;
    team_row_norms(g.it[j].A, g.it[j].len, r, r + 1, 1, g.it[j].wts, g.it[j].nref);
  }
  bool ok = grid_barrier(gst, nb);
  for (int G = 0; ok; ++G) {
    // matrices still sweeping (every block decides alike)
    int total = 0;
    for (int j = 0; j < n; ++j) {
      const int pp = g.it[j].rows + (g.it[j].rows & 1);
      const bool act = !s_done[j] && G / (pp - 1) < g.it[j].max_sweeps;
      if (tid == 0) s_act[j] = act;
      if (act) total += pp / 2;
    }
    if (total == 0) break;
    if (blockIdx.x == 0 && tid == 0) {
      for (int j = 0; j < n; ++j) {
        const int pp = g.it[j].rows + (g.it[j].rows & 1);
        const int sw = G / (pp - 1);
        if (s_act[j] && G % (pp - 1) == 1) {
          reinterpret_cast<int*>(g.it[j].st + S_CNT)[(sw + 1) & 1] = 0;
          reinterpret_cast<unsigned long long*>(g.it[j].st + S_MAXW)[(sw + 1) & 1] = 0ull;
        }
      }
    }
    __syncthreads();
    for (int f = blockIdx.x; f < total; f += (int)nb) {
      int j = 0, k = f;
      for (;; ++j) {
        if (!s_act[j]) continue;
        const int half = (g.it[j].rows + (g.it[j].rows & 1)) / 2;
        if (k < half) break;
        k -= half;
      }
      const JacobiItem& it = g.it[j];
      const int rows = it.rows, pp = rows + (rows & 1);
      const int sw = G / (pp - 1), r = G % (pp - 1);
      int u = player(k, r, pp), v = player(pp - 1 - k, r, pp);
      if (u >= rows || v >= rows) continue;
      if (u > v) { const int t = u; u = v; v = t; }
      bool skipped;
      const PairOut o = jacobi_pair(it.A, it.len, u, v, it.tol, s_skip[j], it.wts, it.nref,
                                    it.stamps, sw > 0 ? G - (pp - 1) : -1, &skipped);
      if (skipped) continue;
      if (tid == 0) {
        ++s_ex[j];
        if (o.rotated) {
          ++s_rot[j];
          it.stamps[u] = G;
          it.stamps[v] = G;
          if (o.counted) {
            atomicAdd(reinterpret_cast<int*>(it.st + S_CNT) + (sw & 1), 1);
            atomicMax(reinterpret_cast<unsigned long long*>(it.st + S_MAXW) + (sw & 1),
                      (unsigned long long)__double_as_longlong(fmax(o.al, o.be)));
          }
        }
      }
    }
    ok = grid_barrier(gst, nb);
    if (!ok) break;
    // the matrices whose sweep ended with this round decide whether to go on
    for (int j = 0; j < n; ++j) {
      if (!s_act[j]) continue;
      const JacobiItem& it = g.it[j];
      const int rows = it.rows, pp = rows + (rows & 1);
      if (G % (pp - 1) != pp - 2) continue;
      const int sw = G / (pp - 1);
      if (blockIdx.x == 0 && tid == 0) it.st[S_SWEEPS] = (unsigned int)(sw + 1);
      bool stop = *((volatile int*)(reinterpret_cast<int*>(it.st + S_CNT) + (sw & 1))) == 0;
      if (!stop && it.keep_rank < rows) {
        const double thr = __longlong_as_double((long long)__ldcg(
                               reinterpret_cast<unsigned long long*>(it.st + S_MAXW) + (sw & 1))) /
                           kKeepMargin;
        int heavy = 0;
        for (int i0 = 0; i0 < rows; i0 += blockDim.x) {
          const int i = i0 + tid;
          heavy += __syncthreads_count(i < rows && __ldcg(it.wts + i) > thr);
        }
        stop = heavy >= it.keep_rank;
      }
      __syncthreads();
      if (stop && tid == 0) s_done[j] = 1;
    }
    __syncthreads();
  }
  __syncthreads();
  const bool failed = *((volatile unsigned int*)(gst + S_ERR)) != 0u;
  for (int j = tid; j < n; j += TPP) {
    atomicAdd(g.it[j].st + S_EXAMINED, s_ex[j]);
    atomicAdd(g.it[j].st + S_ROTATED, s_rot[j]);
    if (failed) atomicExch(g.it[j].st + S_ERR, 1u);
  }
}

// ------------------------------------------------------- ranks and factors
__global__ void k_row_norms(const cplx* A, int p, int q, double* sigma) {
  const int i = blockIdx.x;
  const cplx* a = A + (long long)i * q;
  double s = 0.0;
  for (int e = threadIdx.x; e < q; e += JT) s = fma(a[e].x, a[e].x, fma(a[e].y, a[e].y, s));
  __shared__ double sh[JT / 32];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < JT / 32; ++w) t += sh[w];
    sigma[i] = sqrt(t);
  }
}

// sort descending (ties by index) by counting, then the truncation rule
__global__ void k_sort_rank(const double* sigma, int p, int* perm, double* sorted, int chi_max,
                            double cutoff, double floor_w, double tie_rel, int* rank_out,
                            double* disc_out) {
  // a non-finite value leaves no valid ordering: report rank -1 and stop
  __shared__ int bad;
  if (threadIdx.x == 0) bad = 0;
  __syncthreads();
  for (int i = threadIdx.x; i < p; i += blockDim.x)
    if (!isfinite(sigma[i])) bad = 1;
  __syncthreads();
  if (bad) {
    if (threadIdx.x == 0) {
      *rank_out = -1;
      *disc_out = 0.0;
    }
    return;
  }
  for (int i = threadIdx.x; i < p; i += blockDim.x) {
    const double si = sigma[i];
    int pos = 0;
    for (int j = 0; j < p; ++j) {
      const double sj = sigma[j];
      pos += (sj > si) || (sj == si && j < i);
    }
    perm[pos] = i;
    sorted[pos] = si;
  }
  __syncthreads();
  if (threadIdx.x != 0) return;
  // tail[r] = sum_{k >= r} sigma_k^2, accumulated from the smallest value up
  double total = 0.0;
  for (int k = p - 1; k >= 0; --k) total += sorted[k] * sorted[k];
  int r = p;
  if (total == 0.0) {
    *rank_out = 1;
    *disc_out = 0.0;
    return;
  }
  const double tol = (cutoff > floor_w ? cutoff : floor_w) * total;
  // find the smallest r >= 1 with tail[r] <= tol: walk up from the end
  {
    double tail = 0.0;     // tail[p] = 0
    int best = p;
    for (int cand = p; cand >= 1; --cand) {
      // tail currently = tail[cand]
      if (tail <= tol) best = cand; else break;
      tail += sorted[cand - 1] * sorted[cand - 1];
    }
    r = best;
  }
  if (r > chi_max) r = chi_max;
  if (r < p && sorted[r] >= sorted[r - 1] * (1.0 - tie_rel)) {
    int g = r - 1;
    while (g > 0 && sorted[g] >= sorted[g - 1] * (1.0 - tie_rel)) --g;
    if (g >= 1) r = g;
  }
  double tail = 0.0;
  for (int k = p - 1; k >= r; --k) tail += sorted[k] * sorted[k];
  *rank_out = r;
  *disc_out = tail / total;
}

// Uh[k][i] = D[perm[k]][i] / sorted[k]; a zero row (only for X = 0, rank 1)
// becomes the unit vector e_k, so that Uh keeps orthonormal rows.
__global__ void k_gather_uh(const cplx* D, int len, const int* perm, const double* sorted, int r,
                            cplx* Uh) {
  const long long tot = (long long)r * len;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const int k = (int)(e / len), i = (int)(e - (long long)k * len);
    const double s = sorted[k];
    Uh[e] = s > 0.0 ? cscale(D[(long long)perm[k] * len + i], 1.0 / s)
                    : cmake(i == k ? 1.0 : 0.0, 0.0);
  }
}

__global__ void k_conj_transpose(const cplx* A, int m, int n, cplx* out) {
  __shared__ cplx tile[32][33];
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int i = by + y, j = bx + threadIdx.x;
    if (i < m && j < n) tile[y][threadIdx.x] = A[(long long)i * n + j];
  }
  __syncthreads();
  for (int y = threadIdx.y; y < 32; y += blockDim.y) {
    const int j = bx + y, i = by + threadIdx.x;
    if (i < m && j < n) out[(long long)j * m + i] = cconj(tile[threadIdx.x][y]);
  }
}

int grid_for(long long tot) {
  long long g = (tot + 255) / 256;
  if (g > 1216) g = 1216;
  if (g < 1) g = 1;
  return (int)g;
}

// Blocks of a kernel that can be co-resident on the current device (the grid
// of a cooperative launch), cached per kernel and device; several host
// threads may ask at once.
struct Coresident {
  std::mutex mu;
  int blocks[64] = {0};
  cudaError_t get(const void* kernel, int threads, int* out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(mu);
    int& b = blocks[d & 63];
    if (b == 0) {
      int per_sm = 0, sms = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
      if (e != cudaSuccess) return e;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
      if (e != cudaSuccess) return e;
      b = per_sm * sms;
    }
    *out = b;
    return b > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
  }
};
Coresident g_lq_blocks, g_jacobi_blocks, g_formq_blocks, g_jgroup_blocks;

// The grid barrier of the cooperative kernels with `absent` blocks that never
// arrive: the others wait until the barrier's iteration limit, set the error
// word and return.
__global__ void k_barrier_selftest(unsigned int* st, int absent) {
  if ((int)blockIdx.x < absent) return;
  grid_barrier(st, gridDim.x);
}

}  // namespace

cudaError_t barrier_selftest(unsigned int* dev_state, int blocks, int absent, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(dev_state, 0, S_WORDS * sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  void* args[] = {&dev_state, &absent};
  count_launches(1);
  return cudaLaunchCooperativeKernel((void*)k_barrier_selftest, dim3(blocks), dim3(32), args, 0, st);
}

cudaError_t svd_lq(cplx* W, int p, int q, cplx* beta, double* refl, unsigned int* dev_state,
                   cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(dev_state, 0, 8 * sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  if (p < 1 || q < 1) return cudaSuccess;
  int max_blocks = 0;
  err = g_lq_blocks.get((const void*)k_lq_persistent, JT, &max_blocks);
  if (err != cudaSuccess) return err;
  int nblk = p - 1;
  if (nblk > max_blocks) nblk = max_blocks;
  if (nblk < 1) nblk = 1;
  void* args[] = {&W, &p, &q, &beta, &refl, &dev_state};
  count_launches(1);
  return cudaLaunchCooperativeKernel((void*)k_lq_persistent, dim3(nblk), dim3(JT), args, 0, st);
}

cudaError_t lq_left(const cplx* W, const cplx* beta, int p, int q, cplx* Lout, cudaStream_t st) {
  const int k = p < q ? p : q;
  if (k < 1) return cudaSuccess;
  count_launches(1);
  k_lq_left<<<grid_for((long long)p * k), 256, 0, st>>>(W, beta, p, q, k, Lout);
  return cudaGetLastError();
}

cudaError_t lq_inv_fnorm2(const cplx* W, const cplx* beta, int q, int k, double* colnorm2,
                          double* out, cudaStream_t st) {
  if (k < 1) return cudaSuccess;
  const size_t smem = sizeof(cplx) * (size_t)k;
  if (smem > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(k_tri_inv_colnorm, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
  }
  count_launches(2);
  k_tri_inv_colnorm<<<k, 32, smem, st>>>(W, beta, q, k, colnorm2);
  k_sum_small<<<1, 1024, 0, st>>>(colnorm2, k, out);
  return cudaGetLastError();
}

cudaError_t lq_formq(const cplx* W, const double* refl, int q, int k, cplx* Qh,
                     unsigned int* dev_state, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(dev_state, 0, 8 * sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  if (k < 1) return cudaSuccess;
  count_launches(1);
  k_eye_rows<<<grid_for((long long)k * q), 256, 0, st>>>(Qh, k, q);
  int max_blocks = 0;
  err = g_formq_blocks.get((const void*)k_lq_formq, JT, &max_blocks);
  if (err != cudaSuccess) return err;
  int nblk = k;
  if (nblk > max_blocks) nblk = max_blocks;
  void* args[] = {&W, &refl, &q, &k, &Qh, &dev_state};
  count_launches(1);
  return cudaLaunchCooperativeKernel((void*)k_lq_formq, dim3(nblk), dim3(JT), args, 0, st);
}

cudaError_t svd_lq_r(const cplx* W, const cplx* beta, int p, int q, cplx* R, cudaStream_t st) {
  const int k = p < q ? p : q;
  if (k < 1) return cudaSuccess;
  count_launches(1);
  k_lq_r<<<grid_for((long long)k * p), 256, 0, st>>>(W, beta, p, q, k, R);
  return cudaGetLastError();
}

cudaError_t jacobi_rows(cplx* A, int rows, int len, int max_sweeps, double tol,
                        const double* anorm2, double skip_rel, int keep_rank,
                        unsigned int* dev_state, int* stamps, double* wts, double* nref,
                        cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(dev_state, 0, S_WORDS * sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  if (rows < 2) return cudaSuccess;
  err = cudaMemsetAsync(stamps, 0, sizeof(int) * rows, st);
  if (err != cudaSuccess) return err;
  const int pp = rows + (rows & 1);
  if (pp == 2) {
    // a single pair: one rotation makes it orthogonal; a second launch confirms
    for (int sw = 0; sw < 2; ++sw) {
      count_launches(1);
      k_jacobi_round<<<1, TPP, 0, st>>>(A, len, tol, anorm2, skip_rel, dev_state, wts, nref);
    }
    return cudaGetLastError();
  }
  int max_blocks = 0;
  err = g_jacobi_blocks.get((const void*)k_jacobi_persistent, TPP, &max_blocks);
  if (err != cudaSuccess) return err;
  int nblk = pp / 2;
  if (nblk > max_blocks) nblk = max_blocks;
  void* args[] = {&A, &rows, &len, (void*)&pp, &tol, &anorm2, &skip_rel, &max_sweeps, &keep_rank,
                  &dev_state, &stamps, &wts, &nref};
  count_launches(1);
  return cudaLaunchCooperativeKernel((void*)k_jacobi_persistent, dim3(nblk), dim3(TPP), args, 0,
                                     st);
}

cudaError_t jacobi_prepare(int rows, unsigned int* dev_state, int* stamps, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(dev_state, 0, S_WORDS * sizeof(unsigned int), st);
  if (err != cudaSuccess || rows < 2) return err;
  return cudaMemsetAsync(stamps, 0, sizeof(int) * rows, st);
}

namespace {
// co-resident blocks of k_jacobi_grouped on the current device (cached)
int g_jgroup_capacity[64] = {0};
int jgroup_cap_cached() {
  int d = 0;
  if (cudaGetDevice(&d) != cudaSuccess) return 0;
  return g_jgroup_capacity[d & 63];
}
}  // namespace

cudaError_t jacobi_grouped_capacity(int* blocks) {
  int max_blocks = 0;
  cudaError_t err = g_jgroup_blocks.get((const void*)k_jacobi_grouped, TPP, &max_blocks);
  if (err != cudaSuccess) return err;
  int d = 0;
  err = cudaGetDevice(&d);
  if (err != cudaSuccess) return err;
  g_jgroup_capacity[d & 63] = max_blocks;
  *blocks = max_blocks;
  return cudaSuccess;
}

// one block per pair of a round, up to every block the SMs can hold at once
int jacobi_grouped_blocks(const JacobiItem* items, int n) {
  int total = 0;
  for (int j = 0; j < n; ++j) total += (items[j].rows + (items[j].rows & 1)) / 2;
  int cap = jgroup_cap_cached();
  if (cap < 1) cap = 152;
  return total < cap ? total : cap;
}

cudaError_t jacobi_rows_grouped(const JacobiItem* items, int n, unsigned int* group_state,
                                cudaStream_t st) {
  if (n < 1 || n > kJacobiGroupMax) return cudaErrorInvalidValue;
  JacobiGroup g;
  g.n = n;
  for (int j = 0; j < n; ++j) {
    if (items[j].rows < 3) return cudaErrorInvalidValue;
    g.it[j] = items[j];
  }
  cudaError_t err = cudaMemsetAsync(group_state, 0, S_WORDS * sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  int cap = 0;
  err = jacobi_grouped_capacity(&cap);
  if (err != cudaSuccess) return err;
  const int nblk = jacobi_grouped_blocks(items, n);
  void* args[] = {&g, &group_state};
  count_launches(1);
  return cudaLaunchCooperativeKernel((void*)k_jacobi_grouped, dim3(nblk), dim3(TPP), args, 0, st);
}

cudaError_t svd_rank(const cplx* A, int p, int q, double* sigma, int* perm, double* sorted_sigma,
                     int chi_max, double cutoff, double weight_floor, double tie_rel,
                     int* rank_out, double* discarded_out, cudaStream_t st) {
  if (p <= 0) return cudaErrorInvalidValue;
  count_launches(1);
  k_row_norms<<<p, JT, 0, st>>>(A, p, q, sigma);
  count_launches(1);
  k_sort_rank<<<1, 1024, 0, st>>>(sigma, p, perm, sorted_sigma, chi_max, cutoff, weight_floor,
                                  tie_rel, rank_out, discarded_out);
  return cudaGetLastError();
}

cudaError_t sort_rank(const double* sigma, int p, int* perm, double* sorted_sigma, int chi_max,
                      double cutoff, double weight_floor, double tie_rel, int* rank_out,
                      double* discarded_out, cudaStream_t st) {
  if (p <= 0) return cudaErrorInvalidValue;
  count_launches(1);
  k_sort_rank<<<1, 1024, 0, st>>>(sigma, p, perm, sorted_sigma, chi_max, cutoff, weight_floor,
                                  tie_rel, rank_out, discarded_out);
  return cudaGetLastError();
}

cudaError_t svd_gather_uh(const cplx* D, int len, const int* perm, const double* sorted_sigma,
                          int r, cplx* Uh, cudaStream_t st) {
  if (r < 1) return cudaSuccess;
  count_launches(1);
  k_gather_uh<<<grid_for((long long)r * len), 256, 0, st>>>(D, len, perm, sorted_sigma, r, Uh);
  return cudaGetLastError();
}

cudaError_t conj_transpose(const cplx* A, int m, int n, cplx* out, cudaStream_t st) {
  dim3 grid((n + 31) / 32, (m + 31) / 32);
  count_launches(1);
  k_conj_transpose<<<grid, dim3(32, 8), 0, st>>>(A, m, n, out);
  return cudaGetLastError();
}

}  // namespace ite
