// Served / batched execution: independent evolutions side by side on one GPU
// (see ite_server.h).  Host-side runtime: a FIFO queue with admission by the
// jobs' device-memory estimates, worker threads that each own a library
// context on their own non-blocking stream with stream-ordered allocation,
// and per-job latency records.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include <cuda_runtime.h>

#include "common.cuh"
#include "ite.h"
#include "ite_server.h"

namespace ite {
void internal_release_workspace(ite_ctx ctx);
ite_status internal_set_group(ite_ctx ctx, SplitGroup* g);
}

namespace {

using Clock = std::chrono::steady_clock;
// longest a posted Jacobi waits for the other running jobs' posts while the
// device is busy with grouped launches
constexpr double kDefaultGroupWindowMs = 20.0;

double ms_between(Clock::time_point a, Clock::time_point b) {
  return std::chrono::duration<double, std::milli>(b - a).count();
}

// largest bond dimensions the MPS can use: min(d^b, d^(N-b), chi_max)
std::vector<long long> bond_caps(int N, int d, int chi_max) {
  std::vector<long long> cap(N + 1, 1);
  for (int b = 0; b <= N; ++b) {
    long long left = 1, right = 1;
    for (int k = 0; k < b && left < chi_max; ++k) left *= d;
    for (int k = 0; k < N - b && right < chi_max; ++k) right *= d;
    cap[b] = std::min<long long>(std::min(left, right), chi_max);
  }
  return cap;
}

int job_sites(const ite_job* j) { return j->model == ITE_MODEL_HEISENBERG ? j->n : j->n + 1; }
int job_d(const ite_job* j) { return j->model == ITE_MODEL_HEISENBERG ? 2 : 4; }

bool job_valid(const ite_job* j) {
  if (!j || j->n < 1 || j->chi_max < 1 || !(j->cutoff >= 0.0) || j->n_steps < 1) return false;
  if (j->grid == ITE_JOB_GRID_GEOMETRIC) {
    if (!(j->tau0 > 0.0) || !(j->tau_max > j->tau0)) return false;
  } else if (j->grid == ITE_JOB_GRID_PANELS) {
    if (j->panels < 1 || j->panels > 1000 || !(j->tau_max > 0.0)) return false;
  } else {
    return false;
  }
  if (j->model == ITE_MODEL_HEISENBERG) {
    if (j->n < 2) return false;
  } else if (j->model == ITE_MODEL_ANDERSON) {
    if (!j->eps || !j->V) return false;
  } else {
    return false;
  }
  if (j->metts_samples < 0) return false;
  if (j->metts_samples == 0) return j->site_vecs != nullptr;
  const int N = job_sites(j), d = job_d(j);
  if (!j->metts_config0 || !j->metts_uniforms || !j->metts_energies) return false;
  if (j->metts_obs && (!j->metts_obs_values || j->metts_obs_site < 0 || j->metts_obs_site >= N))
    return false;
  for (int i = 0; i < N; ++i)
    if (j->metts_config0[i] < 0 || j->metts_config0[i] >= d) return false;
  return true;
}

// steps of one evolution on the job's grid
int job_steps(const ite_job* j) {
  return j->grid == ITE_JOB_GRID_PANELS ? j->panels * j->n_steps : j->n_steps;
}
int job_D(const ite_job* j) { return j->model == ITE_MODEL_HEISENBERG ? 5 : 6; }

size_t estimate_bytes(const ite_job* j) {
  if (!job_valid(j)) return 0;
  const int N = job_sites(j), d = job_d(j), D = job_D(j);
  const std::vector<long long> cap = bond_caps(N, d, j->chi_max);
  long long mps = 0, nmax = 1, envs = 0, ovs = 0;
  for (int i = 0; i < N; ++i) {
    mps += cap[i] * d * cap[i + 1];
    nmax = std::max(nmax, cap[i] * d * cap[i + 1]);
    if (i + 1 < N) nmax = std::max(nmax, cap[i] * d * d * cap[i + 2]);
  }
  for (int b = 0; b <= N; ++b) {
    envs += (long long)D * cap[b] * cap[b];
    ovs += cap[b] * cap[b];
  }
  const int krylov = j->opts.krylov_dim > 0 ? j->opts.krylov_dim : 10;
  // the MPS and its three work copies, left/right environments of x and of
  // the right-hand side, Krylov basis, two contraction intermediates and the
  // sweep's other two-site buffers
  long long elems = 4 * mps + 2 * envs + 2 * ovs + (long long)(krylov + 1) * nmax +
                    2LL * D * nmax + 6 * nmax;
  // Gauss-Legendre: q more MPS copies and overlap environments per fit target
  const int q = j->scheme == ITE_GAUSS_LEGENDRE_2 ? 2
                : j->scheme == ITE_GAUSS_LEGENDRE_3 ? 3
                : j->scheme == ITE_HEUN ? 1 : 0;
  elems += q * mps + 2LL * (q + 1) * ovs;
  size_t bytes = (size_t)elems * 16;
  if (j->opts.precision == ITE_FP64_TC) bytes += (size_t)128 * D * nmax;   // slice scratch
  if (j->opts.precision == ITE_MIXED_BF16 || j->opts.precision == ITE_MIXED_TF32)
    // slice scratch of the FP64-class residuals, the refinement's four vectors,
    // and the low-precision operands and intermediates
    bytes += (size_t)(128 + 16) * D * nmax + (size_t)64 * nmax;
  return bytes + ((size_t)8 << 20);                                         // fixed state
}

struct Job {
  long long id = 0;
  ite_job spec{};
  std::vector<double> eps, V, site_vecs, uniforms, alt_basis, obs;
  std::vector<int> config0;
  size_t bytes = 0;
  Clock::time_point t_submit, t_start, t_end;
  bool done = false;
  ite_job_result result{};
};

// Stream-ordered allocation on the worker's stream.
void* worker_alloc(size_t bytes, void* user) {
  void* p = nullptr;
  if (cudaMallocAsync(&p, bytes, static_cast<cudaStream_t>(user)) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return p;
}
void worker_free(void* p, size_t, void* user) { cudaFreeAsync(p, static_cast<cudaStream_t>(user)); }

}  // namespace

struct ite_server_s {
  int device = 0;
  size_t budget = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> queue;
  std::map<long long, std::shared_ptr<Job>> jobs;
  std::vector<std::thread> workers;
  size_t reserved = 0;
  int running = 0, peak_running = 0;
  long long next_id = 1, submitted = 0, completed = 0, failed = 0;
  bool stop = false, any_submitted = false;
  Clock::time_point t_first, t_last;
  std::vector<double> latencies;
  double tau_steps = 0.0;
  ite_status setup_status = ITE_OK;
  // grouped Jacobi launches across the running jobs (off unless switched on)
  ite::SplitGroup* group = nullptr;
  bool grouping = false;

  void worker_main();
  void run_job(ite_ctx ctx, cudaStream_t st, Job& job);
};

void ite_server_s::run_job(ite_ctx ctx, cudaStream_t st, Job& job) {
  ite_job& j = job.spec;
  const int N = job_sites(&j), d = job_d(&j), K = job_steps(&j);
  ite_mpo H = nullptr;
  ite_mps psi = nullptr;
  ite_status s = ITE_OK;
  ite_job_result& r = job.result;
  r.steps_done = 0;
  r.max_discarded_weight = 0.0;
  r.max_chi = 0;
  if (j.model == ITE_MODEL_HEISENBERG)
    s = ite_mpo_create_heisenberg(ctx, N, j.J, j.Jz, &H);
  else
    s = ite_mpo_create_anderson(ctx, j.n, job.eps.data(), job.V.data(), j.U, j.eps_d, &H);
  if (j.metts_samples > 0) {
    std::vector<double> nodes((size_t)K + 1);
    if (s == ITE_OK)
      s = j.grid == ITE_JOB_GRID_PANELS ? ite_grid_panels(j.tau_max, j.panels, j.n_steps, nodes.data())
                                        : ite_grid_geometric(j.tau0, j.tau_max, j.n_steps, nodes.data());
    if (s == ITE_OK)
      s = ite_metts(ctx, H, job.config0.data(), nodes.data(), K, j.scheme, j.shift_mode, j.shift0,
                    j.chi_max, j.cutoff, &j.opts, job.alt_basis.empty() ? nullptr : job.alt_basis.data(),
                    job.obs.empty() ? nullptr : job.obs.data(), j.metts_obs_site, j.metts_samples,
                    job.uniforms.data(), j.metts_energies, j.metts_obs_values, j.metts_configs);
    r.status = s;
    if (s == ITE_OK) {
      r.steps_done = j.metts_samples * K;
      r.energy = j.metts_energies[j.metts_samples - 1];
    }
  } else {
    if (s == ITE_OK) s = ite_mps_create_product(ctx, N, d, job.site_vecs.data(), j.chi_max, &psi);
    std::vector<ite_step_info> info(K);
    if (s == ITE_OK)
      s = j.grid == ITE_JOB_GRID_PANELS
              ? ite_evolve_panels(ctx, H, psi, j.tau_max, j.panels, j.n_steps, j.scheme, j.shift_mode,
                                  j.shift0, j.chi_max, j.cutoff, &j.opts, info.data(), nullptr)
              : ite_evolve_loggrid(ctx, H, psi, j.tau0, j.tau_max, j.n_steps, j.scheme, j.shift_mode,
                                   j.shift0, j.chi_max, j.cutoff, &j.opts, info.data(), nullptr);
    r.status = s;
    // steps that ran have filled their record (max_chi >= 1)
    for (int k = 0; k < K && info[k].max_chi > 0; ++k) {
      ++r.steps_done;
      r.energy = info[k].energy;
      r.max_discarded_weight = std::max(r.max_discarded_weight, info[k].max_discarded_weight);
      r.max_chi = std::max(r.max_chi, info[k].max_chi);
      if (j.energies) j.energies[k] = info[k].energy;
    }
    if (s == ITE_OK && (j.state || j.state_chi)) {
      std::vector<int> chi(N + 1);
      size_t nd = 0;
      s = ite_mps_bond_dims(psi, chi.data(), &nd);
      if (s == ITE_OK && j.state_chi) std::copy(chi.begin(), chi.end(), j.state_chi);
      if (s == ITE_OK && j.state) s = nd <= j.state_cap ? ite_mps_get(ctx, psi, j.state, j.state_cap)
                                                        : ITE_EINVAL;
      r.status = s;
    }
  }
  if (psi) ite_mps_destroy(psi);
  if (H) ite_mpo_destroy(H);
  ite::internal_release_workspace(ctx);
  cudaStreamSynchronize(st);
}

void ite_server_s::worker_main() {
  cudaStream_t st = nullptr;
  ite_ctx ctx = nullptr;
  bool ok = cudaSetDevice(device) == cudaSuccess &&
            cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess;
  if (ok) ok = ite_ctx_create(device, st, worker_alloc, worker_free, st, &ctx) == ITE_OK;
  if (!ok) {
    std::lock_guard<std::mutex> lock(mu);
    setup_status = ITE_ECUDA;
  }
  for (;;) {
    std::shared_ptr<Job> job;
    {
      std::unique_lock<std::mutex> lock(mu);
      // FIFO: the head starts when it fits next to the running jobs (or when
      // nothing runs)
      cv_work.wait(lock, [&] {
        return stop || (!queue.empty() &&
                        (running == 0 || reserved + queue.front()->bytes <= budget));
      });
      if (queue.empty()) {
        if (stop) break;
        continue;
      }
      job = queue.front();
      queue.pop_front();
      reserved += job->bytes;
      ++running;
      peak_running = std::max(peak_running, running);
      job->t_start = Clock::now();
      if (group) ite::group_set_expected(group, running);
      if (ctx) ite::internal_set_group(ctx, grouping ? group : nullptr);
    }
    if (ctx) {
      run_job(ctx, st, *job);
    } else {
      job->result.status = ITE_ECUDA;
    }
    {
      std::lock_guard<std::mutex> lock(mu);
      job->t_end = Clock::now();
      ite_job_result& r = job->result;
      r.queue_ms = ms_between(job->t_submit, job->t_start);
      r.run_ms = ms_between(job->t_start, job->t_end);
      r.latency_ms = ms_between(job->t_submit, job->t_end);
      r.device_bytes = job->bytes;
      job->done = true;
      reserved -= job->bytes;
      --running;
      if (group) ite::group_set_expected(group, running);
      if (r.status == ITE_OK) {
        ++completed;
        latencies.push_back(r.latency_ms);
        tau_steps += r.steps_done;
      } else {
        ++failed;
      }
      t_last = job->t_end;
    }
    cv_work.notify_all();
    cv_done.notify_all();
  }
  if (ctx) ite_ctx_destroy(ctx);
  if (st) cudaStreamDestroy(st);
}

extern "C" {

size_t ite_job_device_bytes(const ite_job* job) { return estimate_bytes(job); }

ite_status ite_server_create(int device, int n_slots, size_t mem_budget, ite_server* out) {
  if (!out || n_slots < 1 || n_slots > 64 || device < 0) return ITE_EINVAL;
  *out = nullptr;
  int count = 0;
  if (cudaGetDeviceCount(&count) != cudaSuccess || device >= count) {
    cudaGetLastError();
    return ITE_ECUDA;
  }
  if (mem_budget == 0) {
    size_t free_b = 0, total_b = 0;
    if (cudaSetDevice(device) != cudaSuccess || cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
      cudaGetLastError();
      return ITE_ECUDA;
    }
    mem_budget = free_b / 10 * 9;
  }
  ite_server s = new ite_server_s;
  s->device = device;
  s->budget = mem_budget;
  if (ite::group_create(device, kDefaultGroupWindowMs, &s->group) != cudaSuccess) {
    delete s;
    return ITE_ECUDA;
  }
  for (int w = 0; w < n_slots; ++w) s->workers.emplace_back([s] { s->worker_main(); });
  *out = s;
  return ITE_OK;
}

ite_status ite_server_submit(ite_server s, const ite_job* job, long long* ticket) {
  if (!s || !ticket || !job_valid(job)) return ITE_EINVAL;
  auto j = std::make_shared<Job>();
  j->spec = *job;
  const int N = job_sites(job), d = job_d(job);
  if (job->metts_samples == 0) {
    j->site_vecs.assign(job->site_vecs, job->site_vecs + (size_t)2 * N * d);
  } else {
    j->config0.assign(job->metts_config0, job->metts_config0 + N);
    j->uniforms.assign(job->metts_uniforms, job->metts_uniforms + (size_t)job->metts_samples * N);
    if (job->metts_alt_basis) j->alt_basis.assign(job->metts_alt_basis, job->metts_alt_basis + 2 * d * d);
    if (job->metts_obs) j->obs.assign(job->metts_obs, job->metts_obs + 2 * d * d);
  }
  if (job->model == ITE_MODEL_ANDERSON) {
    j->eps.assign(job->eps, job->eps + job->n);
    j->V.assign(job->V, job->V + job->n);
  }
  j->spec.site_vecs = nullptr;
  j->spec.eps = j->spec.V = nullptr;
  j->spec.metts_config0 = nullptr;
  j->spec.metts_uniforms = j->spec.metts_alt_basis = j->spec.metts_obs = nullptr;
  j->bytes = estimate_bytes(job);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    if (s->setup_status != ITE_OK) return s->setup_status;
    if (j->bytes > s->budget) return ITE_ENOMEM;
    j->id = s->next_id++;
    j->t_submit = Clock::now();
    if (!s->any_submitted) {
      s->t_first = j->t_submit;
      s->any_submitted = true;
    }
    ++s->submitted;
    s->jobs[j->id] = j;
    s->queue.push_back(j);
    *ticket = j->id;
  }
  s->cv_work.notify_all();
  return ITE_OK;
}

ite_status ite_server_poll(ite_server s, long long ticket, ite_job_result* out) {
  if (!s || !out) return ITE_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return ITE_EINVAL;
  if (!it->second->done) return ITE_PENDING;
  *out = it->second->result;
  return ITE_OK;
}

ite_status ite_server_wait(ite_server s, long long ticket, ite_job_result* out) {
  if (!s || !out) return ITE_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  auto it = s->jobs.find(ticket);
  if (it == s->jobs.end()) return ITE_EINVAL;
  std::shared_ptr<Job> j = it->second;
  s->cv_done.wait(lock, [&] { return j->done; });
  *out = j->result;
  return ITE_OK;
}

ite_status ite_server_drain(ite_server s) {
  if (!s) return ITE_EINVAL;
  std::unique_lock<std::mutex> lock(s->mu);
  s->cv_done.wait(lock, [&] { return s->completed + s->failed == s->submitted; });
  return ITE_OK;
}

ite_status ite_server_stats_get(ite_server s, ite_server_stats* out) {
  if (!s || !out) return ITE_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  std::memset(out, 0, sizeof(*out));
  out->submitted = s->submitted;
  out->completed = s->completed;
  out->failed = s->failed;
  out->peak_running = s->peak_running;
  std::vector<double> lat = s->latencies;
  std::sort(lat.begin(), lat.end());
  auto pct = [&](double q) {
    if (lat.empty()) return 0.0;
    // nearest rank
    size_t k = (size_t)std::ceil(q * lat.size());
    k = std::min(std::max<size_t>(k, 1), lat.size());
    return lat[k - 1];
  };
  out->p50_latency_ms = pct(0.50);
  out->p99_latency_ms = pct(0.99);
  out->wall_ms = s->any_submitted && s->completed + s->failed > 0 ? ms_between(s->t_first, s->t_last) : 0.0;
  out->tau_steps = s->tau_steps;
  out->tau_steps_per_s = out->wall_ms > 0.0 ? s->tau_steps / (out->wall_ms * 1e-3) : 0.0;
  if (s->group) ite::group_stats(s->group, &out->group_launches, &out->group_items);
  return ITE_OK;
}

ite_status ite_server_set_grouping(ite_server s, int mode, double window_ms) {
  if (!s || mode < 0 || mode > 2 || !(window_ms >= 0.0) || window_ms > 1e4) return ITE_EINVAL;
  std::lock_guard<std::mutex> lock(s->mu);
  s->grouping = mode != 0;
  ite::group_set_policy(s->group, mode == 0 ? 1 : mode, window_ms);
  return ITE_OK;
}

void ite_server_destroy(ite_server s) {
  if (!s) return;
  ite_server_drain(s);
  {
    std::lock_guard<std::mutex> lock(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  for (auto& t : s->workers) t.join();
  ite::group_destroy(s->group);
  delete s;
}

ite_status ite_evolve_batch(int device, int n_slots, size_t mem_budget, int n, const ite_job* jobs,
                            ite_job_result* out, ite_server_stats* stats) {
  return ite_evolve_batch_grouped(device, n_slots, mem_budget, 0, kDefaultGroupWindowMs, n, jobs,
                                  out, stats);
}

ite_status ite_evolve_batch_grouped(int device, int n_slots, size_t mem_budget, int grouping,
                                    double window_ms, int n, const ite_job* jobs,
                                    ite_job_result* out, ite_server_stats* stats) {
  if (n < 0 || (n > 0 && (!jobs || !out))) return ITE_EINVAL;
  for (int i = 0; i < n; ++i)
    if (!job_valid(&jobs[i])) return ITE_EINVAL;
  ite_server s = nullptr;
  ite_status st = ite_server_create(device, n_slots, mem_budget, &s);
  if (st != ITE_OK) return st;
  st = ite_server_set_grouping(s, grouping, window_ms);
  if (st != ITE_OK) {
    ite_server_destroy(s);
    return st;
  }
  std::vector<long long> tickets(n, 0);
  for (int i = 0; i < n && st == ITE_OK; ++i) st = ite_server_submit(s, &jobs[i], &tickets[i]);
  if (st == ITE_OK) {
    for (int i = 0; i < n; ++i) ite_server_wait(s, tickets[i], &out[i]);
    if (stats) ite_server_stats_get(s, stats);
  }
  ite_server_destroy(s);
  return st;
}

}  // extern "C"
