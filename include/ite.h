/*
 * ite.h -- C ABI of the GB300 (sm_103a) library for imaginary-time evolution
 * of matrix product states by A-stable implicit steps on logarithmic tau grids.
 *
 * The method (arXiv 2606.02930): evolve |psi(tau)> = e^{-H tau}|psi(0)>
 * (Method, Eq. 1) on a grid whose steps grow geometrically (Method, log-grid
 * and panel paragraphs), each step being the implicit linear solve
 *
 *     (I + c (H - s)) |psi_k> = |b>                                   (Eq. 4)
 *
 * with c = dtau/2, b = (I - c (H - s)) psi_{k-1} for the trapezoid rule
 * (Eq. 4, App. A), or c = dtau, b = psi_{k-1} for backward Euler.  The solve is
 * an MPO-MPS linear system done by a two-site DMRG-style sweep with GMRES
 * local solves (Method, "two operations"; App. B, App. D).
 *
 * Conventions
 *   - Complex numbers are interleaved (re, im) doubles, i.e. the memory layout
 *     of C99 double complex / numpy complex128.
 *   - MPS site tensor i: A_i[a][s][b], shape (chi_i, d, chi_{i+1}), row-major,
 *     chi_0 = chi_N = 1.  Bond index b = 0..N (bond b sits left of site b).
 *   - MPO site tensor i: W_i[w][s'][s][w'], shape (D_i, d, d, D_{i+1}),
 *     D_0 = D_N = 1; s' is the output (bra) index.  The operator is the
 *     product of the W_i over the channel indices.
 *   - Heisenberg local basis: 0 = spin up.  Anderson local basis:
 *     {|0>, |up>, |down>, |up down>} (index n_up + 2 n_down), impurity on site
 *     0, bath j on site j (star geometry), Jordan-Wigner order up before down.
 *
 * Ownership and memory
 *   - Handles are library-owned and released by the matching *_destroy.
 *   - Host arrays passed in are copied before the call returns; outputs go to
 *     caller buffers whose capacity is passed alongside.
 *   - Every device allocation goes through the allocator given to
 *     ite_ctx_create (NULL = cudaMalloc/cudaFree).  All device work is
 *     enqueued on the context stream; calls that return host values
 *     synchronise that stream before returning.
 *
 * Errors
 *   - Every call returns an ite_status; ite_last_error(ctx) gives a message.
 *     No call aborts the process.  ITE_ESINGULAR flags non-finite values;
 *     ITE_ENOTCONV is informational (a fixed-effort GMRES is not an error).
 *   - A handle of NULL, a negative size or a bond dimension above the
 *     object's capacity gives ITE_EINVAL and leaves all state unchanged.
 */
#ifndef ITE_H
#define ITE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ite_ctx_s* ite_ctx;
typedef struct ite_mpo_s* ite_mpo;
typedef struct ite_mps_s* ite_mps;

typedef enum {
  ITE_OK = 0,
  ITE_EINVAL = 1,
  ITE_ENOMEM = 2,
  ITE_ESINGULAR = 3,
  ITE_ENOTCONV = 4,   /* reserved: fixed-effort solves (the paper's one sweep, one
                         GMRES cycle) are not failures and return ITE_OK, with
                         their residuals in ite_step_info                       */
  ITE_ETIMEOUT = 5,
  ITE_ECUDA = 6,
  ITE_PENDING = 7     /* a served job has not finished yet (ite_server.h) */
} ite_status;

/* Time stepper.  Trapezoid: Eq. 4 (A-stable, App. A).  Backward Euler: the
 * first-order A-stable (and L-stable) implicit step, R(z) = 1/(1+z).
 * Gauss-Legendre q = 2, 3: the paper's Gauss-Legendre collocation (Method,
 * spectral panel scheme); for this linear ODE the q-stage collocation step is
 * R_q(z) = P_q(-z)/P_q(z), the (q, q) Pade approximant of e^{-z} (order 2q,
 * A-stable), evaluated as q complex-shifted solves (I + c_j (H - s)) x_j = psi
 * and a two-site fit of r_inf psi + sum_j w_j x_j (see
 * ite_gl_partial_fractions); opts.fit_sweeps sweeps of that fit. */
typedef enum {
  ITE_BACKWARD_EULER = 0,
  ITE_TRAPEZOID = 1,
  ITE_GAUSS_LEGENDRE_2 = 2,
  ITE_GAUSS_LEGENDRE_3 = 3,
  ITE_FORWARD_EULER = 4,   /* explicit, R(z) = 1 - z (stability counter-example) */
  ITE_HEUN = 5             /* explicit predictor-corrector, R(z) = 1 - z + z^2/2:
                              unstable once dtau (E - s) > 2 for an eigenvalue E
                              (the explicit counter-example of the stability
                              section); both products formed by two-site fits */
} ite_scheme;

/* Arithmetic of the contractions.  ITE_FP64: complex128 everywhere on the
 * FP64 pipes.  ITE_FP64_TC: the same algorithm, with every large contraction
 * computed to FP64-class accuracy on the bf16 tensor cores by exact slicing
 * (ite_k_zgemm mode 1); everything else stays FP64.
 * ITE_MIXED_BF16 / ITE_MIXED_TF32: each local solve of the sweep (App. B) is
 * converged by iterative refinement: the residual B - A X is formed with the
 * FP64-class contraction of ITE_FP64_TC, and each correction solves A D = r by
 * one GMRES(krylov_dim) cycle whose H_eff matvecs use bf16 (or tf32) operands
 * with fp32 accumulation on the tensor cores; X += D, until |r| <= refine_tol
 * |B| or refine_max corrections.  A correction that does not halve |r| moves
 * the inner matvecs up one precision (bf16 -> tf32 -> FP64-class).  Krylov
 * vectors, the Hessenberg solve, environments, SVDs, norms and energies stay
 * FP64 (environments FP64-class), so the converged local solution carries the
 * FP64-class residual.  local_tol and max_cycles do not apply in these modes. */
typedef enum { ITE_FP64 = 0, ITE_FP64_TC = 1, ITE_MIXED_BF16 = 2, ITE_MIXED_TF32 = 3 } ite_precision;

/* Spectrum shift s of each step.  FIXED: the caller's value.  CURRENT_ENERGY:
 * s_k = <psi_{k-1}|H|psi_{k-1}> (App. D shifts H by the energy of the state
 * each step produced, which keeps the norm of the next step near one). */
typedef enum { ITE_SHIFT_FIXED = 0, ITE_SHIFT_CURRENT_ENERGY = 1 } ite_shift_mode;

/* Device allocator hooks: alloc returns a device pointer (NULL on failure). */
typedef void* (*ite_alloc_fn)(size_t bytes, void* user);
typedef void (*ite_free_fn)(void* ptr, size_t bytes, void* user);

/* Solver effort (App. D: one sweep, one GMRES cycle of Krylov dimension 10). */
typedef struct {
  int krylov_dim;     /* Arnoldi steps per local solve (default 10)            */
  int sweeps;         /* maximum sweeps per solve (default 1)                  */
  double local_tol;   /* stop GMRES at |r|/|B| <= local_tol (0: fixed effort)  */
  double sweep_tol;   /* stop sweeping at 1-|<x_s|x_{s-1}>| < tol (0: fixed)   */
  int fit_sweeps;     /* sweeps of the trapezoid right-hand-side fit (1)       */
  int precision;      /* ite_precision (ITE_FP64 or ITE_FP64_TC)               */
  int max_cycles;     /* GMRES(krylov_dim) cycles per local solve, each
                         restarted from the last iterate (default 1, as App. D;
                         <= 0 counts as 1); a cycle that ends early (breakdown
                         or local_tol reached) ends the solve                  */
  int refine_max;     /* mixed modes: most refinement corrections per local
                         solve (default 10)                                    */
  double refine_tol;  /* mixed modes: stop at |B - A X| <= refine_tol |B|
                         (default 1e-10)                                       */
} ite_solver_opts;

/* Per-step report. */
typedef struct {
  double energy;               /* <psi_k|H|psi_k> after normalisation          */
  double norm_before;          /* |x| before normalisation                     */
  double max_discarded_weight; /* largest relative discarded weight of a bond  */
  double max_local_residual;   /* largest GMRES relative residual estimate     */
  double shift;                /* shift s used by this step                    */
  int max_chi;                 /* largest bond dimension after the step        */
  int gmres_steps;             /* Arnoldi steps summed over all local solves   */
  int status;                  /* ite_status of this step                      */
} ite_step_info;

void ite_solver_opts_default(ite_solver_opts* opts);

/* Context: one device, one stream (cudaStream_t or NULL for the legacy
 * default stream), optional allocator hooks with a user pointer. */
ite_status ite_ctx_create(int device, void* stream, ite_alloc_fn alloc, ite_free_fn release,
                          void* alloc_user, ite_ctx* out);
ite_status ite_ctx_set_stream(ite_ctx ctx, void* stream);
void ite_ctx_destroy(ite_ctx ctx);
const char* ite_last_error(ite_ctx ctx);
/* Bytes currently held through the allocator by this context and its objects. */
size_t ite_ctx_device_bytes(ite_ctx ctx);
/* Number of CUDA kernels the library has launched so far in this process. */
unsigned long long ite_kernel_launches(void);
/* Stage timers (CUDA events on the context stream).  Between start and stop
 * every stage of the sweep records an event pair; stop synchronises and
 * returns, per category, the summed milliseconds, the summed algorithmic FLOPs
 * and the number of stages: 0 two-site H_eff, 1 environment updates, 2 local
 * solves (GMRES, H_eff included), 3 truncated SVD splits, 4 gauge moves (SVDs
 * included), 5 local right-hand sides and two-site merges, 6 whole steps,
 * 7 the Householder LQ launches of the splits, 8 the Jacobi launches of the
 * splits (7 and 8 are inside 3 and 4).  The arrays have ITE_PROFILE_SLOTS
 * entries; unused ones are zero. */
#define ITE_PROFILE_SLOTS 16
ite_status ite_profile_start(ite_ctx ctx);
/* Category 9: the low-precision H_eff matvecs of the mixed modes (FLOPs by
 * the same algorithmic count as category 0, which they are not part of). */
ite_status ite_profile_stop(ite_ctx ctx, double ms[ITE_PROFILE_SLOTS],
                            double flops[ITE_PROFILE_SLOTS], long long counts[ITE_PROFILE_SLOTS]);
/* SVD statistics since the last call (then reset): splits performed, total
 * and largest number of Jacobi sweeps, and (fp64_flops, may be NULL; three
 * entries) the algorithmic FP64 flops of the Householder LQ ([0]), of the
 * Jacobi rotations and inner products actually executed ([1]), and the
 * reference algorithmic work of the truncated SVDs ([2]: 8.7 GFLOP for a
 * 512 x 512 complex block, the 22 n^3-class count, scaled by p q min(p, q)). */
ite_status ite_svd_stats(ite_ctx ctx, long long* splits, long long* sweeps_total, int* sweeps_max,
                         double fp64_flops[3]);

/* MPO from explicit site tensors: d[N] site dimensions (all equal), D[N+1]
 * bond dimensions with D[0] = D[N] = 1, W the concatenated W_i (interleaved
 * complex), sum_i D_i d^2 D_{i+1} complex numbers. */
ite_status ite_mpo_create(ite_ctx ctx, int N, const int* d, const int* D, const double* W,
                          ite_mpo* out);
/* Heisenberg chain J sum (SxSx + SySy) + Jz sum SzSz, open boundaries, D = 5
 * (Heisenberg-chain section; Jz = J is the isotropic chain). */
ite_status ite_mpo_create_heisenberg(ite_ctx ctx, int N, double J, double Jz, ite_mpo* out);
/* Single-impurity Anderson model (Anderson-impurity section):
 * eps_d n_d + U n_up n_down + sum_j eps_j n_j + sum_{j,s} V_j (d^dag_s c_js + h.c.),
 * star geometry, d = 4, D = 6. */
ite_status ite_mpo_create_anderson(ite_ctx ctx, int n_bath, const double* eps, const double* V,
                                   double U, double eps_d, ite_mpo* out);
int ite_mpo_length(ite_mpo mpo);
void ite_mpo_destroy(ite_mpo mpo);

/* MPS with bond-dimension capacity chi_cap (bond b holds at most
 * min(d^b, d^(N-b), chi_cap)).  chi[N+1] are the initial bond dimensions and
 * A the concatenated site tensors (interleaved complex). */
ite_status ite_mps_create(ite_ctx ctx, int N, int d, const int* chi, const double* A,
                          int chi_cap, ite_mps* out);
/* Product state from site_vecs[N][d] (interleaved complex). */
ite_status ite_mps_create_product(ite_ctx ctx, int N, int d, const double* site_vecs,
                                  int chi_cap, ite_mps* out);
/* Replace the tensors of an existing MPS (same N, d; chi within capacity). */
ite_status ite_mps_set(ite_ctx ctx, ite_mps mps, const int* chi, const double* A);
ite_status ite_mps_copy(ite_ctx ctx, ite_mps src, ite_mps dst);
/* Bond dimensions chi[N+1] and the number of doubles ite_mps_get writes. */
ite_status ite_mps_bond_dims(ite_mps mps, int* chi, size_t* n_doubles);
ite_status ite_mps_get(ite_ctx ctx, ite_mps mps, double* A, size_t cap_doubles);
void ite_mps_destroy(ite_mps mps);

/* Checkpoint of an MPS, to resume an evolution later or in another process
 * (library addition; the paper has no counterpart).  The byte image is
 * the magic "ITEMPS01", then the 8-byte integers N, d, chi_cap and
 * chi[0..N], then the site tensors as ite_mps_get writes them (interleaved
 * complex doubles), all in the host's byte order (little-endian on the
 * supported hosts).  ite_mps_bytes gives its size; ite_mps_save writes it to
 * host memory buf of cap bytes (ITE_EINVAL if too small); ite_mps_load
 * creates a new MPS in ctx from len bytes at buf, and returns ITE_EINVAL for
 * a wrong magic, truncated or inconsistent image without creating one. */
ite_status ite_mps_bytes(ite_mps mps, size_t* bytes);
ite_status ite_mps_save(ite_mps mps, void* buf, size_t cap);
ite_status ite_mps_load(ite_ctx ctx, const void* buf, size_t len, ite_mps* out);
/* Reads a checkpoint's header without a device: N, d, chi_cap, the bond
 * dimensions (chi_out[chi_len >= N+1]) and the number of doubles of its
 * tensors; each output may be NULL.  ITE_EINVAL for a wrong magic, a header
 * out of range (1 <= N, chi_cap <= 2^20, 1 <= d <= 16, 1 <= chi[b] <=
 * chi_cap, chi[0] = chi[N] = 1) or a buffer shorter than the image. */
ite_status ite_mps_checkpoint_info(const void* buf, size_t len, int* N, int* d, int* chi_cap,
                                   int* chi_out, size_t chi_len, size_t* n_doubles);
/* The state as a dense vector psi[s_0 ... s_{N-1}] (s_0 most significant;
 * interleaved complex; cap_doubles >= 2 d^N), contracted on the host from
 * the tensors: a check for small systems (d^N <= 2^24), ITE_EINVAL above. */
ite_status ite_mps_to_dense(ite_ctx ctx, ite_mps mps, double* out, size_t cap_doubles);

/* One implicit step of size dtau with shift s (Eq. 4 / backward Euler), in
 * place.  The state is normalised afterwards (Heisenberg section, App. D). */
ite_status ite_implicit_step(ite_ctx ctx, ite_mpo H, ite_mps psi, double dtau, int scheme,
                             double shift, int chi_max, double cutoff,
                             const ite_solver_opts* opts, ite_step_info* info);

/* Geometric grid t_0 = 0, t_k = tau0 (tau_max/tau0)^((k-1)/(n_steps-1)),
 * k = 1..n_steps, and evolution over it.  per_step[n_steps], nodes[n_steps+1]
 * may be NULL. */
ite_status ite_grid_geometric(double tau0, double tau_max, int n_steps, double* nodes);
/* METTS collapse (Anderson-impurity section: METTS on top of the implicit
 * steps): draws a product configuration sigma with probability
 * |<sigma|psi>|^2 / <psi|psi> by sequential conditional draws, site i taking
 * the smallest state s whose cumulative conditional probability exceeds
 * u[i] (u: N host numbers in [0, 1)).  basis (host, d x d interleaved
 * complex unitary, may be NULL) gives the collapse basis: sigma is a product
 * of its columns; NULL is the computational basis.  Brings psi to
 * right-canonical form first (the state is unchanged).  config[N] (host)
 * receives the states, *prob (may be NULL) the probability.  d <= 4. */
ite_status ite_mps_sample(ite_ctx ctx, ite_mps psi, const double* u, const double* basis,
                          int* config, double* prob);
/* METTS chain (Anderson-impurity section): from the product configuration
 * config0 (computational basis), n_samples times: evolve the product state
 * over the tau grid nodes[0..n_steps] (host; nodes[0] = 0, strictly
 * increasing; nodes[n_steps] = beta/2), with scheme, shift_mode and shift0
 * as ite_evolve_loggrid, record its energy in energies[k] and, if obs (d x d
 * interleaved complex) is given, <obs at obs_site> in obs_values[k], then
 * collapse it with uniforms[k N .. k N + N) into the next configuration
 * (written to configs[k N ..], may be NULL) in the computational basis, or on
 * even k in alt_basis when given (alternating bases let the chain leave a
 * conserved sector of its start state).  Averages over the chain estimate
 * thermal averages at inverse temperature beta.  The paper's grid is the
 * panel grid (ite_grid_panels: first panel about [0, 0.01], 4 steps per
 * panel) with the trapezoid rule and the current-energy shift; its steps stay
 * small against tau, so dtau (s - E0) stays below 1 and every solve is well
 * conditioned.  A few long steps from a high-energy product state with the
 * current-energy shift make (I + c (H - s)) indefinite instead. */
ite_status ite_metts(ite_ctx ctx, ite_mpo H, const int* config0, const double* nodes, int n_steps,
                     int scheme, int shift_mode, double shift0, int chi_max, double cutoff,
                     const ite_solver_opts* opts, const double* alt_basis, const double* obs,
                     int obs_site, int n_samples, const double* uniforms, double* energies,
                     double* obs_values, int* configs);
/* Partial fractions of the q-stage Gauss-Legendre step (host only, q = 1..8):
 * R_q(z) = r_inf + sum_j a_j / (z - z_j); poles[2q] and residues[2q] receive
 * z_j and a_j (interleaved complex).  The step with dtau uses the shifts
 * c_j = -dtau / z_j and the weights w_j = -a_j / z_j. */
ite_status ite_gl_partial_fractions(int q, double* poles, double* residues, double* r_inf);
ite_status ite_evolve_loggrid(ite_ctx ctx, ite_mpo H, ite_mps psi, double tau0, double tau_max,
                              int n_steps, int scheme, int shift_mode, double shift0,
                              int chi_max, double cutoff, const ite_solver_opts* opts,
                              ite_step_info* per_step, double* nodes);

/* The paper's panel grid (Method): P panels with endpoints
 * {0, tau_max/2^(P-j), j = 1..P} and n uniform steps per panel; P*n steps. */
ite_status ite_grid_panels(double tau_max, int P, int n, double* nodes);
ite_status ite_evolve_panels(ite_ctx ctx, ite_mpo H, ite_mps psi, double tau_max, int P, int n,
                             int scheme, int shift_mode, double shift0, int chi_max,
                             double cutoff, const ite_solver_opts* opts,
                             ite_step_info* per_step, double* nodes);

/* Measurements (Heisenberg section: overlaps; Anderson section: double
 * occupancy <n_up n_down> as a one-site correlator). */
ite_status ite_energy(ite_ctx ctx, ite_mpo H, ite_mps psi, double* energy);
ite_status ite_overlap(ite_ctx ctx, ite_mps bra, ite_mps ket, double out[2]);
/* <psi| O_i S_{i+1}..S_{j-1} P_j |psi> / <psi|psi>, i <= j, O, P, S d x d
 * interleaved complex (S may be NULL: identity; for i == j the operator is
 * O P on site i). */
ite_status ite_correlator(ite_ctx ctx, ite_mps psi, const double* O, int i, const double* P,
                          int j, const double* string_op, double out[2]);

#ifdef __cplusplus
}
#endif

#endif /* ITE_H */
