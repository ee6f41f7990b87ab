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
#include "common.cuh"

namespace ite {
namespace {

constexpr int JT = 128;

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
// error flag is set and the block leaves (the caller then exits).
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
k_lq_persistent(cplx* W, int p, int q, cplx* beta, unsigned int* st) {
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
      if (blockIdx.x == 0) beta[j] = cmake(-phr * nx, -phi * nx);
      hs[0] = phr * (a0 + nx);
      hs[1] = phi * (a0 + nx);
      hs[2] = nx > 0.0 ? 1.0 / (nx * (nx + a0)) : 0.0;
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

// ---------------------------------------------------------- one-sided Jacobi
// One Jacobi rotation on rows u, v (length len) of A: make the pair orthogonal
// if |gamma| > tol sqrt(alpha beta).  Called by all JT threads of a block;
// returns (to every thread) whether the rows were rotated.
__device__ bool jacobi_pair(cplx* A, int len, int u, int v, double tol, double skip, int* counter) {
  __shared__ double sh[2][2][JT / 32];
  if (u > v) { const int t = u; u = v; v = t; }
  cplx* au = A + (long long)u * len;
  cplx* av = A + (long long)v * len;
  double sa = 0, sb = 0, gr = 0, gi = 0;
  for (int e = threadIdx.x; e < len; e += JT) {
    const cplx x = au[e], y = av[e];
    sa = fma(x.x, x.x, fma(x.y, x.y, sa));
    sb = fma(y.x, y.x, fma(y.y, y.y, sb));
    gr = fma(x.x, y.x, fma(x.y, y.y, gr));     // Re(conj(x) y)
    gi = fma(x.x, y.y, fma(-x.y, y.x, gi));    // Im(conj(x) y)
  }
  block_sum2(sa, sb, sh[0]);
  block_sum2(gr, gi, sh[1]);
  const double al = sa, be = sb;
  const double gabs = hypot(gr, gi);
  // A pair of rows both below the skip weight can never be kept: their
  // mutual orthogonality does not matter (their total weight does, and
  // rotations preserve it).
  if (!(gabs > tol * sqrt(al * be) && gabs > 0.0 && (al > skip || be > skip))) return false;
  const double zeta = (be - al) / (2.0 * gabs);
  const double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
  const double c = 1.0 / sqrt(1.0 + t * t);
  const double sn = c * t;
  const double sr = sn * gr / gabs, si = sn * gi / gabs;   // s e^{i theta}
  // Only rotations by an angle above tol between two rows that can be kept
  // keep the sweeps going.  Rotations against rows below the skip weight are
  // still applied, but those rows are never rotated among themselves, so they
  // stay a non-orthogonal set, and orthogonalising a kept row against all of
  // them one pair at a time converges only slowly; its overlap with them
  // changes the kept product at second order.
  if (threadIdx.x == 0 && fabs(t) > tol && al > skip && be > skip) atomicAdd(counter, 1);
  // a_u' = c a_u - s e^{-i theta} a_v ;  a_v' = s e^{i theta} a_u + c a_v
  for (int e = threadIdx.x; e < len; e += JT) {
    const cplx x = au[e], y = av[e];
    au[e] = cmake(c * x.x - (sr * y.x + si * y.y), c * x.y - (sr * y.y - si * y.x));
    av[e] = cmake((sr * x.x - si * x.y) + c * y.x, (sr * x.y + si * x.x) + c * y.y);
  }
  return true;
}

__global__ void __launch_bounds__(JT)
k_jacobi_round(cplx* A, int rows, int len, int round, int pp, double tol, const double* anorm2,
               double skip_rel, int* counter) {
  const int k = blockIdx.x;
  const int u = player(k, round, pp), v = player(pp - 1 - k, round, pp);
  if (u >= rows || v >= rows) return;
  const double a2 = anorm2 ? *anorm2 : 0.0;
  jacobi_pair(A, len, u, v, tol, skip_rel * a2, counter);
}

// All sweeps of the round-robin one-sided Jacobi in one cooperative launch.
// st[2], st[3]: rotation counters of even / odd sweeps; st[5]: sweeps done.
// A sweep's counter is read by every block after the sweep's last barrier;
// the counter of the following sweep is cleared by block 0 in round 1 of the
// current sweep, after every block has passed round 0 (and so has finished
// reading it two sweeps ago).
// stamps[row] holds the global round at which the row was last rotated.  The
// tournament repeats every sweep, so a pair was last examined pp-1 rounds ago;
// if neither row has been rotated since then (a rotation at that very round
// left the pair orthogonal), examining it again cannot fire and is skipped.
__global__ void __launch_bounds__(JT)
k_jacobi_persistent(cplx* A, int rows, int len, int pp, double tol, const double* anorm2,
                    double skip_rel, int max_sweeps, unsigned int* st, int* stamps) {
  const unsigned int nb = gridDim.x;
  const double skip = skip_rel * (anorm2 ? *anorm2 : 0.0);
  int* counters = reinterpret_cast<int*>(st + 2);
  for (int sw = 0; sw < max_sweeps; ++sw) {
    int* cnt = counters + (sw & 1);
    for (int r = 0; r < pp - 1; ++r) {
      if (r == 1 && blockIdx.x == 0 && threadIdx.x == 0) counters[(sw + 1) & 1] = 0;
      const int g = sw * (pp - 1) + r;
      for (int k = blockIdx.x; k < pp / 2; k += nb) {
        const int u = player(k, r, pp), v = player(pp - 1 - k, r, pp);
        if (u >= rows || v >= rows) continue;
        if (sw > 0) {
          const int last = g - (pp - 1);
          // read through L2 so that every thread of the block sees the same
          // stamps and takes the same branch
          if (__ldcg(stamps + u) <= last && __ldcg(stamps + v) <= last) continue;
        }
        const bool rotated = jacobi_pair(A, len, u, v, tol, skip, cnt);
        if (rotated && threadIdx.x == 0) {
          stamps[u] = g;
          stamps[v] = g;
        }
      }
      if (!grid_barrier(st, nb)) return;
    }
    const int rotations = *((volatile int*)cnt);
    if (blockIdx.x == 0 && threadIdx.x == 0) st[5] = (unsigned int)(sw + 1);
    if (rotations == 0) break;
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

// Blocks of JT threads of a kernel that can be co-resident on the current
// device (the grid of a cooperative launch), cached per kernel and device.
struct Coresident {
  int dev = -1, blocks = 0;
  cudaError_t get(const void* kernel, int* out) {
    int d = 0;
    cudaError_t e = cudaGetDevice(&d);
    if (e != cudaSuccess) return e;
    if (d != dev) {
      int per_sm = 0, sms = 0;
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, JT, 0);
      if (e != cudaSuccess) return e;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, d);
      if (e != cudaSuccess) return e;
      blocks = per_sm * sms;
      dev = d;
    }
    *out = blocks;
    return blocks > 0 ? cudaSuccess : cudaErrorInvalidConfiguration;
  }
};
Coresident g_lq_blocks, g_jacobi_blocks;

}  // namespace

cudaError_t svd_lq(cplx* W, int p, int q, cplx* beta, unsigned int* dev_state, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(dev_state, 0, 8 * sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  if (p < 1 || q < 1) return cudaSuccess;
  int max_blocks = 0;
  err = g_lq_blocks.get((const void*)k_lq_persistent, &max_blocks);
  if (err != cudaSuccess) return err;
  int nblk = p - 1;
  if (nblk > max_blocks) nblk = max_blocks;
  if (nblk < 1) nblk = 1;
  void* args[] = {&W, &p, &q, &beta, &dev_state};
  count_launches(1);
  return cudaLaunchCooperativeKernel((void*)k_lq_persistent, dim3(nblk), dim3(JT), args, 0, st);
}

cudaError_t svd_lq_r(const cplx* W, const cplx* beta, int p, int q, cplx* R, cudaStream_t st) {
  const int k = p < q ? p : q;
  if (k < 1) return cudaSuccess;
  count_launches(1);
  k_lq_r<<<grid_for((long long)k * p), 256, 0, st>>>(W, beta, p, q, k, R);
  return cudaGetLastError();
}

cudaError_t jacobi_rows(cplx* A, int rows, int len, int max_sweeps, double tol,
                        const double* anorm2, double skip_rel, unsigned int* dev_state,
                        int* stamps, cudaStream_t st) {
  cudaError_t err = cudaMemsetAsync(dev_state, 0, 8 * sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  if (rows < 2) return cudaSuccess;
  err = cudaMemsetAsync(stamps, 0, sizeof(int) * rows, st);
  if (err != cudaSuccess) return err;
  const int pp = rows + (rows & 1);
  if (pp == 2) {
    // a single pair: one rotation makes it orthogonal; a second launch confirms
    int* cnt = reinterpret_cast<int*>(dev_state + 2);
    for (int sw = 0; sw < 2; ++sw) {
      count_launches(1);
      k_jacobi_round<<<1, JT, 0, st>>>(A, rows, len, 0, pp, tol, anorm2, skip_rel, cnt);
    }
    return cudaGetLastError();
  }
  int max_blocks = 0;
  err = g_jacobi_blocks.get((const void*)k_jacobi_persistent, &max_blocks);
  if (err != cudaSuccess) return err;
  int nblk = pp / 2;
  if (nblk > max_blocks) nblk = max_blocks;
  void* args[] = {&A, &rows, &len, (void*)&pp, &tol, &anorm2, &skip_rel, &max_sweeps, &dev_state,
                  &stamps};
  count_launches(1);
  return cudaLaunchCooperativeKernel((void*)k_jacobi_persistent, dim3(nblk), dim3(JT), args, 0, st);
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
