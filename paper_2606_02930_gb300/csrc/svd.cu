// FP64 truncated SVD of the two-site blocks and the gauge moves: parallel
// one-sided (Hestenes) Jacobi on the rows of a p x q complex matrix.
//
// Each launch performs one round of a round-robin tournament: the p rows form
// p/2 disjoint pairs, one CTA per pair.  The CTA forms alpha = |a_u|^2,
// beta = |a_v|^2 and gamma = a_u^H a_v, and if |gamma| > tol sqrt(alpha beta)
// applies the complex Jacobi rotation that makes the pair orthogonal to both
// the pair of rows and to the matching rows of the accumulated unitary Q.  A
// sweep is p-1 rounds; sweeps repeat until no rotation fires.  On exit
// Q A_in = A_out, the rows of A_out are orthogonal with norms sigma_i, so
// A_in = Q^H diag(sigma) V^H with V^H the normalised rows.
#include "common.cuh"

namespace ite {
namespace {

constexpr int JT = 128;

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ int player(int pos, int round, int pp) {
  return pos == 0 ? 0 : ((pos - 1 + round) % (pp - 1)) + 1;
}

// complex helpers over the real type R (double: FP64 path, float: the
// approximate FP32 stage of the mixed-precision SVD)
template <typename R> struct Cx;
template <> struct Cx<double> { typedef double2 T; };
template <> struct Cx<float> { typedef float2 T; };

template <typename R>
__device__ __forceinline__ typename Cx<R>::T cx(R a, R b) {
  typename Cx<R>::T z;
  z.x = a;
  z.y = b;
  return z;
}

template <typename R>
__device__ __forceinline__ R warp_sum_t(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// One Jacobi rotation on rows u, v of A (and of Q): make the pair orthogonal
// if |gamma| > tol sqrt(alpha beta).  Called by all JT threads of a block.
template <typename R>
__device__ void jacobi_pair(typename Cx<R>::T* A, int p, int q, typename Cx<R>::T* Q, int u, int v,
                            R tol, R skip, int* counter) {
  typedef typename Cx<R>::T T;
  if (u > v) { const int t = u; u = v; v = t; }
  T* au = A + (long long)u * q;
  T* av = A + (long long)v * q;
  R sa = 0, sb = 0, gr = 0, gi = 0;
  for (int e = threadIdx.x; e < q; e += JT) {
    const T x = au[e], y = av[e];
    sa = fma(x.x, x.x, fma(x.y, x.y, sa));
    sb = fma(y.x, y.x, fma(y.y, y.y, sb));
    gr = fma(x.x, y.x, fma(x.y, y.y, gr));     // Re(conj(x) y)
    gi = fma(x.x, y.y, fma(-x.y, y.x, gi));    // Im(conj(x) y)
  }
  __shared__ R sh[4][JT / 32];
  __shared__ R rot[4];
  sa = warp_sum_t(sa); sb = warp_sum_t(sb); gr = warp_sum_t(gr); gi = warp_sum_t(gi);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) { sh[0][wid] = sa; sh[1][wid] = sb; sh[2][wid] = gr; sh[3][wid] = gi; }
  __syncthreads();
  if (threadIdx.x == 0) {
    R al = 0, be = 0, Gr = 0, Gi = 0;
    for (int w = 0; w < JT / 32; ++w) { al += sh[0][w]; be += sh[1][w]; Gr += sh[2][w]; Gi += sh[3][w]; }
    const R gabs = hypot(Gr, Gi);
    R c = 1, sr = 0, si = 0;   // rotation: c, and s*e^{i theta}
    // A pair of rows both below the skip weight can never be kept: their
    // mutual orthogonality does not matter (their total weight does, and
    // rotations preserve it).
    if (gabs > tol * sqrt(al * be) && gabs > R(0) && (al > skip || be > skip)) {
      const R zeta = (be - al) / (R(2) * gabs);
      const R t = (zeta >= R(0) ? R(1) : R(-1)) / (fabs(zeta) + sqrt(R(1) + zeta * zeta));
      c = R(1) / sqrt(R(1) + t * t);
      const R sn = c * t;
      sr = sn * Gr / gabs;
      si = sn * Gi / gabs;
      // Only rotations by an angle above tol between two rows that can be
      // kept keep the sweeps going.  Rotations against rows below the skip
      // weight are still applied, but those rows are never rotated among
      // themselves, so they stay a non-orthogonal set, and orthogonalising a
      // kept row against all of them one pair at a time converges only
      // slowly; its overlap with them changes the kept product at second order.
      if (fabs(t) > tol && al > skip && be > skip) atomicAdd(counter, 1);
    }
    rot[0] = c; rot[1] = sr; rot[2] = si; rot[3] = (sr != R(0) || si != R(0)) ? R(1) : R(0);
  }
  __syncthreads();
  const R c = rot[0], sr = rot[1], si = rot[2];   // se = s e^{i theta}
  const bool apply = rot[3] != R(0);
  __syncthreads();                             // rot[] is reused by the next pair
  if (!apply) return;
  // a_u' = c a_u - s e^{-i theta} a_v ;  a_v' = s e^{i theta} a_u + c a_v
  for (int e = threadIdx.x; e < q; e += JT) {
    const T x = au[e], y = av[e];
    au[e] = cx<R>(c * x.x - (sr * y.x + si * y.y), c * x.y - (sr * y.y - si * y.x));
    av[e] = cx<R>((sr * x.x - si * x.y) + c * y.x, (sr * x.y + si * x.x) + c * y.y);
  }
  T* qu = Q + (long long)u * p;
  T* qv = Q + (long long)v * p;
  for (int e = threadIdx.x; e < p; e += JT) {
    const T x = qu[e], y = qv[e];
    qu[e] = cx<R>(c * x.x - (sr * y.x + si * y.y), c * x.y - (sr * y.y - si * y.x));
    qv[e] = cx<R>((sr * x.x - si * x.y) + c * y.x, (sr * x.y + si * x.x) + c * y.y);
  }
}

template <typename R>
__global__ void __launch_bounds__(JT)
k_jacobi_round(typename Cx<R>::T* A, int p, int q, typename Cx<R>::T* Q, int round, int pp, R tol,
               const double* anorm2, double skip_rel, int* counter) {
  const int k = blockIdx.x;
  const int u = player(k, round, pp), v = player(pp - 1 - k, round, pp);
  if (u >= p || v >= p) return;
  const double a2 = anorm2 ? *anorm2 : 0.0;
  jacobi_pair<R>(A, p, q, Q, u, v, tol, (R)(skip_rel * a2), counter);
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

// All sweeps of the round-robin one-sided Jacobi in one cooperative launch.
// st[2], st[3]: rotation counters of even / odd sweeps; st[5]: sweeps done.
// A sweep's counter is read by every block after the sweep's last barrier;
// the counter of the following sweep is cleared by block 0 in round 1 of the
// current sweep, after every block has passed round 0 (and so has finished
// reading it two sweeps ago).
template <typename R>
__global__ void __launch_bounds__(JT)
k_jacobi_persistent(typename Cx<R>::T* A, int p, int q, typename Cx<R>::T* Q, int pp, R tol,
                    const double* anorm2, double skip_rel, int max_sweeps, unsigned int* st) {
  const unsigned int nb = gridDim.x;
  const double a2 = anorm2 ? *anorm2 : 0.0;
  const R skip = (R)(skip_rel * a2);
  int* counters = reinterpret_cast<int*>(st + 2);
  for (int sw = 0; sw < max_sweeps; ++sw) {
    int* cnt = counters + (sw & 1);
    for (int r = 0; r < pp - 1; ++r) {
      if (r == 1 && blockIdx.x == 0 && threadIdx.x == 0) counters[(sw + 1) & 1] = 0;
      for (int k = blockIdx.x; k < pp / 2; k += nb) {
        const int u = player(k, r, pp), v = player(pp - 1 - k, r, pp);
        if (u < p && v < p) jacobi_pair<R>(A, p, q, Q, u, v, tol, skip, cnt);
      }
      if (!grid_barrier(st, nb)) return;
    }
    const int rotations = *((volatile int*)cnt);
    if (blockIdx.x == 0 && threadIdx.x == 0) st[5] = (unsigned int)(sw + 1);
    if (rotations == 0) break;
  }
}

template <typename R>
__global__ void k_identity_t(typename Cx<R>::T* Q, int p) {
  const long long tot = (long long)p * p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / p, j = e - i * p;
    Q[e] = cx<R>(i == j ? R(1) : R(0), R(0));
  }
}

__global__ void k_identity(cplx* Q, int p) {
  const long long tot = (long long)p * p;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot;
       e += (long long)gridDim.x * blockDim.x) {
    const long long i = e / p, j = e - i * p;
    Q[e] = cmake(i == j ? 1.0 : 0.0, 0.0);
  }
}

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

// transposed == false: A = M (m x n, m <= n), Q is m x m, u_k = conj(Q row), s_k v_k^H = A row
// transposed == true : A = M^H (n x m),     Q is n x n, s_k u_k = conj(A row), v_k^H = Q row
__global__ void k_emit(const cplx* Arot, const cplx* Q, const double* sorted, const int* perm,
                       int r, int p, int q, bool transposed, bool centre_right, cplx* left,
                       cplx* right) {
  // left: (m x r), right: (r x n); m = transposed ? q : p; n = transposed ? p : q
  const int m = transposed ? q : p, n = transposed ? p : q;
  const long long totL = (long long)m * r, totR = (long long)r * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < totL + totR;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < totL) {
      const long long i = e / r;
      const int k = (int)(e - i * r);
      const int src = perm[k];
      const double s = sorted[k];
      cplx v;
      if (!transposed) {
        v = cconj(Q[(long long)src * p + i]);
        if (!centre_right) v = cscale(v, s);
      } else {
        v = cconj(Arot[(long long)src * q + i]);
        if (centre_right) v = cscale(v, 1.0 / s);
      }
      left[e] = v;
    } else {
      const long long f = e - totL;
      const int k = (int)(f / n);
      const long long j = f - (long long)k * n;
      const int src = perm[k];
      const double s = sorted[k];
      cplx v;
      if (!transposed) {
        v = Arot[(long long)src * q + j];
        if (!centre_right) v = cscale(v, 1.0 / s);
      } else {
        v = Q[(long long)src * p + j];
        if (centre_right) v = cscale(v, s);
      }
      right[f] = v;
    }
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

}  // namespace

cudaError_t set_identity(cplx* Q, int p, cudaStream_t st) {
  long long tot = (long long)p * p;
  long long g = (tot + 255) / 256;
  if (g > 1216) g = 1216;
  if (g < 1) g = 1;
  count_launches(1);
  k_identity<<<(int)g, 256, 0, st>>>(Q, p);
  return cudaGetLastError();
}

template <typename R>
cudaError_t jacobi_rows_t(typename Cx<R>::T* A, int p, int q, typename Cx<R>::T* Q, int max_sweeps,
                          R tol, const double* anorm2, double skip_rel, unsigned int* dev_state,
                          cudaStream_t st) {
  {
    long long tot = (long long)p * p;
    long long g = (tot + 255) / 256;
    if (g > 1216) g = 1216;
    if (g < 1) g = 1;
    count_launches(1);
    k_identity_t<R><<<(int)g, 256, 0, st>>>(Q, p);
  }
  cudaError_t err = cudaMemsetAsync(dev_state, 0, 8 * sizeof(unsigned int), st);
  if (err != cudaSuccess) return err;
  if (p < 2) return cudaSuccess;
  const int pp = p + (p & 1);
  if (pp == 2) {
    // a single pair: one rotation makes it orthogonal; a second launch confirms
    int* cnt = reinterpret_cast<int*>(dev_state + 2);
    for (int sw = 0; sw < 2; ++sw) {
      count_launches(1);
      k_jacobi_round<R><<<1, JT, 0, st>>>(A, p, q, Q, 0, pp, tol, anorm2, skip_rel, cnt);
    }
    return cudaGetLastError();
  }
  // co-resident grid for the cooperative launch (cached per device and type)
  static int cached_dev = -1, max_blocks = 0;
  int dev = 0;
  err = cudaGetDevice(&dev);
  if (err != cudaSuccess) return err;
  if (dev != cached_dev) {
    int per_sm = 0, sms = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_jacobi_persistent<R>, JT, 0);
    if (err != cudaSuccess) return err;
    err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (err != cudaSuccess) return err;
    max_blocks = per_sm * sms;
    cached_dev = dev;
  }
  int nblk = pp / 2;
  if (nblk > max_blocks) nblk = max_blocks;
  if (nblk < 1) return cudaErrorInvalidConfiguration;
  void* args[] = {&A, &p, &q, &Q, (void*)&pp, &tol, &anorm2, &skip_rel, &max_sweeps, &dev_state};
  count_launches(1);
  return cudaLaunchCooperativeKernel((void*)k_jacobi_persistent<R>, dim3(nblk), dim3(JT), args, 0, st);
}

cudaError_t jacobi_rows(cplx* A, int p, int q, cplx* Q, int max_sweeps, double tol,
                        const double* anorm2, double skip_rel, unsigned int* dev_state,
                        cudaStream_t st) {
  return jacobi_rows_t<double>(A, p, q, Q, max_sweeps, tol, anorm2, skip_rel, dev_state, st);
}

cudaError_t jacobi_rows_f32(float2* A, int p, int q, float2* Q, int max_sweeps, float tol,
                            const double* anorm2, double skip_rel, unsigned int* dev_state,
                            cudaStream_t st) {
  return jacobi_rows_t<float>(A, p, q, Q, max_sweeps, tol, anorm2, skip_rel, dev_state, st);
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

cudaError_t svd_emit(const cplx* Arot, const cplx* Q, const double* sorted_sigma,
                     const int* perm, int r, int p, int q, bool transposed, bool centre_right,
                     cplx* left, cplx* right, cudaStream_t st) {
  const long long tot = (long long)r * (p + q);
  long long g = (tot + 255) / 256;
  if (g > 1216) g = 1216;
  if (g < 1) g = 1;
  count_launches(1);
  k_emit<<<(int)g, 256, 0, st>>>(Arot, Q, sorted_sigma, perm, r, p, q, transposed, centre_right,
                                  left, right);
  return cudaGetLastError();
}

cudaError_t conj_transpose(const cplx* A, int m, int n, cplx* out, cudaStream_t st) {
  dim3 grid((n + 31) / 32, (m + 31) / 32);
  count_launches(1);
  k_conj_transpose<<<grid, dim3(32, 8), 0, st>>>(A, m, n, out);
  return cudaGetLastError();
}

}  // namespace ite
