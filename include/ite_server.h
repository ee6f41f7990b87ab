/*
 * ite_server.h -- many imaginary-time evolutions at once on one GPU.
 *
 * The paper evolves one state at a time (Method; App. B, App. D).  Its
 * Anderson-impurity study needs many independent evolutions (METTS samples,
 * parameter scans: Anderson-impurity section), and one evolution's kernels
 * leave most of a GB300 idle: the sweep is a chain of small dependent steps
 * whose largest cost, the truncated SVD, is bound by FP64 latency.  This
 * server runs independent evolutions side by side.  Each worker owns a
 * library context on its own CUDA stream, so the kernels of different jobs
 * overlap on the device.  The paper has no counterpart; it is this library's
 * addition.
 *
 *   - Admission: a job is started only when its device-memory estimate
 *     (ite_job_device_bytes) fits the server's budget next to the jobs
 *     already running.  Jobs start in submission order, so a large job at the
 *     head of the queue waits rather than being overtaken.  A job whose
 *     estimate alone exceeds the budget is refused at submission
 *     (ITE_ENOMEM).
 *   - Memory: workers allocate stream-ordered (cudaMallocAsync on their own
 *     stream), so no job's allocation waits for the whole device, and release
 *     a job's workspaces when it ends.
 *   - Each job is the same computation as ite_evolve_loggrid (or
 *     ite_evolve_panels) on a product start state, or as ite_metts for a
 *     METTS job: its results do not depend on what else runs (the kernels
 *     are deterministic and jobs share no data).
 *   - Host arrays in ite_job are copied by ite_server_submit; the output
 *     buffers (energies, state) must stay valid until the job has finished.
 *   - All calls are thread-safe.  Errors: ITE_EINVAL for invalid arguments,
 *     ITE_ENOMEM as above, ITE_ECUDA if a worker cannot set up its device.
 */
#ifndef ITE_SERVER_H
#define ITE_SERVER_H

#include "ite.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef enum { ITE_MODEL_HEISENBERG = 0, ITE_MODEL_ANDERSON = 1 } ite_model;
typedef enum { ITE_JOB_GRID_GEOMETRIC = 0, ITE_JOB_GRID_PANELS = 1 } ite_job_grid;

/* One job: model, truncation, tau grid, and either one evolution of a product
 * start state or a METTS chain.
 *   grid ITE_JOB_GRID_GEOMETRIC: tau0 -> tau_max in n_steps steps (as
 *     ite_evolve_loggrid); ITE_JOB_GRID_PANELS: `panels` panels of n_steps
 *     uniform steps each up to tau_max (as ite_grid_panels; tau0 unused).
 *   metts_samples == 0: one evolution of site_vecs over the grid.
 *   metts_samples > 0: a METTS chain (as ite_metts) from metts_config0 over
 *     the grid (tau_max = beta/2) with metts_uniforms[samples][N], the optional
 *     collapse basis and observable (d x d interleaved complex), all copied at
 *     submit; writes metts_energies[samples], metts_obs_values[samples] (when
 *     metts_obs is given) and metts_configs[samples][N] (may be NULL).
 *     site_vecs, energies and state are not used.
 * A zero-initialised tail (grid, panels, metts_*) gives one evolution on the
 * geometric grid. */
typedef struct {
  int model;                  /* ite_model                                          */
  int n;                      /* Heisenberg: sites N; Anderson: bath sites (N = n+1) */
  double J, Jz;               /* Heisenberg couplings                               */
  double U, eps_d;            /* Anderson impurity                                  */
  const double* eps;          /* Anderson bath energies [n] (copied at submit)      */
  const double* V;            /* Anderson hybridisations [n] (copied at submit)     */
  const double* site_vecs;    /* start state [N][d], interleaved complex (copied)   */
  int chi_max;
  double cutoff;
  int scheme;                 /* ite_scheme                                         */
  int shift_mode;             /* ite_shift_mode                                     */
  double shift0;
  double tau0, tau_max;
  int n_steps;
  ite_solver_opts opts;
  double* energies;           /* optional out [n_steps]: energy after each step     */
  double* state;              /* optional out: final tensors as ite_mps_get writes  */
  size_t state_cap;           /* capacity of state in doubles                       */
  int* state_chi;             /* optional out [N+1]: final bond dimensions          */
  int grid;                   /* ite_job_grid                                       */
  int panels;                 /* panel count for ITE_JOB_GRID_PANELS                */
  int metts_samples;          /* 0: one evolution; > 0: METTS chain of this length  */
  const int* metts_config0;   /* [N] start configuration (copied)                   */
  const double* metts_uniforms;  /* [samples][N] in [0, 1) (copied)                 */
  const double* metts_alt_basis; /* optional d x d collapse basis (copied)          */
  const double* metts_obs;    /* optional d x d observable (copied)                 */
  int metts_obs_site;
  double* metts_energies;     /* out [samples]                                      */
  double* metts_obs_values;   /* out [samples], needed with metts_obs               */
  int* metts_configs;         /* optional out [samples][N]                          */
} ite_job;

/* For a METTS job, steps_done counts the steps of all samples, energy is the
 * last sample's, and max_discarded_weight and max_chi are 0. */
typedef struct {
  int status;                 /* ite_status of the evolution                         */
  int steps_done;
  double energy;              /* energy after the last step                          */
  double max_discarded_weight;
  int max_chi;
  double queue_ms;            /* submission -> start                                 */
  double run_ms;              /* start -> finish                                     */
  double latency_ms;          /* submission -> finish                                */
  size_t device_bytes;        /* the admission estimate                              */
} ite_job_result;

typedef struct {
  long long submitted, completed, failed;
  int peak_running;           /* most jobs ever running at once                      */
  double p50_latency_ms, p99_latency_ms;   /* over completed jobs                    */
  double wall_ms;             /* first submission -> last completion                 */
  double tau_steps;           /* steps completed over all jobs                       */
  double tau_steps_per_s;     /* tau_steps / wall                                    */
  long long group_launches;   /* grouped Jacobi launches (see ite_server_set_grouping) */
  long long group_items;      /* splits those launches carried                       */
} ite_server_stats;

typedef struct ite_server_s* ite_server;

/* Device-memory estimate of one job (host arithmetic, no device needed): the
 * MPS and its two work copies at the capacity set by chi_max, the
 * environments, the Krylov basis and the sweep's workspaces, and the
 * tensor-core scratch in ITE_FP64_TC mode.  0 for an invalid job. */
size_t ite_job_device_bytes(const ite_job* job);

/* n_slots workers (1..64) on `device`, admitting jobs while their estimates
 * sum to at most mem_budget bytes (0: 90% of the device's free memory). */
ite_status ite_server_create(int device, int n_slots, size_t mem_budget, ite_server* out);
/* Queue a job; *ticket identifies it. */
ite_status ite_server_submit(ite_server s, const ite_job* job, long long* ticket);
/* ITE_OK and *out when the job has finished, ITE_PENDING before. */
ite_status ite_server_poll(ite_server s, long long ticket, ite_job_result* out);
/* Grouped launches across jobs.  The one-sided Jacobi of a truncated split
 * (the SVD that follows every two-site solve, App. B) is a chain of dependent
 * rounds that leaves most of the GPU idle, and two large ones already take
 * every block the SMs hold at once.  With grouping, a running job posts the
 * Jacobi of each split to the server instead of launching it, and posts go to
 * the device together as one cooperative launch (k_jacobi_grouped).
 *   mode 0 (default): off (each job launches its own Jacobi on its stream);
 *   mode 1: continuous batching: a post goes out at once if it fits
 *     next to the grouped launches still running, else as soon as every
 *     running job outside a running launch has posted, a running launch has
 *     made room, or the first post has waited window_ms (default 20);
 *   mode 2: gather: posts wait for every running job's post, or window_ms.
 * A post waits on the host only, never on the GPU.  Each split ends bit for
 * bit as it would alone, so results do not depend on the mode.  On GB300 the
 * Jacobis of concurrent jobs already overlap from their own streams, and the
 * grouped modes measured 2-4% below that, hence off by default.  Applies to
 * jobs that start after the call.  ITE_EINVAL for a mode outside 0..2 or
 * window_ms outside [0, 1e4]. */
ite_status ite_server_set_grouping(ite_server s, int mode, double window_ms);
/* Block until the job has finished. */
ite_status ite_server_wait(ite_server s, long long ticket, ite_job_result* out);
/* Block until every submitted job has finished. */
ite_status ite_server_drain(ite_server s);
ite_status ite_server_stats_get(ite_server s, ite_server_stats* out);
/* Drains, then stops the workers. */
void ite_server_destroy(ite_server s);

/* n jobs through a temporary server: create, submit all, drain, destroy.
 * out[n] receives the results in job order; stats may be NULL. */
ite_status ite_evolve_batch(int device, int n_slots, size_t mem_budget, int n, const ite_job* jobs,
                            ite_job_result* out, ite_server_stats* stats);
/* The same with the grouping mode and window of ite_server_set_grouping
 * (ite_evolve_batch uses mode 0). */
ite_status ite_evolve_batch_grouped(int device, int n_slots, size_t mem_budget, int grouping,
                                    double window_ms, int n, const ite_job* jobs,
                                    ite_job_result* out, ite_server_stats* stats);

#ifdef __cplusplus
}
#endif

#endif
