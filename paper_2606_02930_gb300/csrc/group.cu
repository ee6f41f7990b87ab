// Grouped launches across concurrent evolutions (the served runtime).
//
// The one-sided Jacobi of a truncated split is a chain of dependent rounds,
// one grid barrier each, with at most rows/2 pairs per round: one evolution's
// split keeps the FP64 units of a GB300 mostly idle, and two such cooperative
// launches already take all the blocks the SMs can hold at once, so further
// jobs' Jacobis queue behind them.  With grouping, each worker context posts
// the Jacobi of its split here instead of launching it, and the posts go to
// the device together as one cooperative launch of k_jacobi_grouped: one grid
// barrier per round serves all of them, and the pairs of all matrices fill
// the SMs.
//
// When a batch goes out (continuous batching, mode 1): at once if its blocks
// fit next to the grouped launches still running (the cooperative launch
// could start now), else as soon as every running job that is not inside a
// running launch has posted, a running launch has finished and made room, or
// the first post has waited the window (a safety net).  Posts that arrive
// while the device is full thus accumulate into the next launch, and small
// Jacobis go out at once.  Mode 2 (gather) always waits for every running
// job's post, or the window: it makes grouping certain, for tests.
//
// Ordering is by CUDA events: a post records an event on the member's stream
// after the member's own work up to the Jacobi; the launch goes on the stream
// of the batch's first member (whose thread is waiting here), after waiting
// for the events of all its items, and records each member's completion event
// after the kernel; each member's stream waits for its event.  Host threads
// block only until their item has been launched, never on the GPU beyond
// polling event status.  Each item ends bit for bit as the ungrouped Jacobi
// would leave it, so grouping never changes a result.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace ite {

namespace {
using Clock = std::chrono::steady_clock;
constexpr auto kPoll = std::chrono::microseconds(50);
}  // namespace

struct SplitGroup {
  std::mutex mu;
  std::condition_variable cv;
  int device = 0;
  double window_ms = 20.0;
  int mode = 1;                           // 1 continuous batching, 2 gather every post
  int capacity = 0;                       // co-resident blocks of k_jacobi_grouped
  int expected = 0;                       // members that will post (running jobs)
  struct Post {
    JacobiItem item;
    cudaEvent_t ready, done;
    cudaStream_t stream;
    unsigned int* gstate;
    cudaError_t* status;
    long long ticket;
  };
  std::vector<Post> pending;
  struct Flight {
    cudaEvent_t ev;
    int items, blocks;
  };
  std::vector<Flight> flights;            // launches not yet seen complete
  std::vector<cudaEvent_t> spare;         // completion events for reuse
  int in_flight_items = 0, in_flight_blocks = 0;
  long long next_ticket = 1, launched_upto = 0;
  long long launches = 0, items = 0;
};

namespace {

// Drops the launches whose completion event has fired (lock held).
void retire_locked(SplitGroup* g) {
  for (size_t k = 0; k < g->flights.size();) {
    const cudaError_t q = cudaEventQuery(g->flights[k].ev);
    if (q == cudaErrorNotReady) {
      ++k;
      continue;
    }
    if (q != cudaSuccess) cudaGetLastError();
    g->in_flight_items -= g->flights[k].items;
    g->in_flight_blocks -= g->flights[k].blocks;
    g->spare.push_back(g->flights[k].ev);
    g->flights.erase(g->flights.begin() + k);
  }
}

// Launches every pending post (in batches of at most kJacobiGroupMax), with
// the group's lock held.  A batch runs on its first member's stream with that
// member's barrier words.
void launch_locked(SplitGroup* g) {
  while (!g->pending.empty()) {
    const int n = std::min<int>((int)g->pending.size(), kJacobiGroupMax);
    const SplitGroup::Post& lead = g->pending[0];
    cudaStream_t st = lead.stream;
    JacobiItem items[kJacobiGroupMax];
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < n && e == cudaSuccess; ++k) {
      items[k] = g->pending[k].item;
      if (k > 0) e = cudaStreamWaitEvent(st, g->pending[k].ready, 0);
    }
    if (e == cudaSuccess) e = jacobi_rows_grouped(items, n, lead.gstate, st);
    cudaEvent_t fev = nullptr;
    if (e == cudaSuccess) {
      if (!g->spare.empty()) {
        fev = g->spare.back();
        g->spare.pop_back();
      } else {
        e = cudaEventCreateWithFlags(&fev, cudaEventDisableTiming);
      }
    }
    if (e == cudaSuccess) e = cudaEventRecord(fev, st);
    for (int k = 0; k < n; ++k) {
      cudaError_t ek = e;
      if (ek == cudaSuccess) ek = cudaEventRecord(g->pending[k].done, st);
      *g->pending[k].status = ek;
    }
    if (e == cudaSuccess) {
      const int blocks = jacobi_grouped_blocks(items, n);
      g->flights.push_back({fev, n, blocks});
      g->in_flight_items += n;
      g->in_flight_blocks += blocks;
    } else if (fev) {
      g->spare.push_back(fev);
    }
    g->launched_upto = g->pending[n - 1].ticket;
    g->pending.erase(g->pending.begin(), g->pending.begin() + n);
    g->launches += 1;
    g->items += n;
  }
  g->cv.notify_all();
}

// Whether the pending posts should go out now (lock held, flights retired).
bool due_locked(SplitGroup* g, Clock::time_point deadline) {
  if (g->pending.empty()) return false;
  if ((int)g->pending.size() >= std::max(1, g->expected - g->in_flight_items)) return true;
  if (Clock::now() >= deadline) return true;
  if (g->mode != 1) return false;
  if (g->flights.empty()) return true;
  JacobiItem items[kJacobiGroupMax];
  const int n = std::min<int>((int)g->pending.size(), kJacobiGroupMax);
  for (int k = 0; k < n; ++k) items[k] = g->pending[k].item;
  return g->in_flight_blocks + jacobi_grouped_blocks(items, n) <= g->capacity;
}

}  // namespace

cudaError_t group_create(int device, double window_ms, SplitGroup** out) {
  *out = nullptr;
  int prev = 0, cap = 0;
  cudaError_t e = cudaGetDevice(&prev);
  if (e == cudaSuccess) e = cudaSetDevice(device);
  if (e == cudaSuccess) {
    e = jacobi_grouped_capacity(&cap);
    cudaSetDevice(prev);
  }
  if (e != cudaSuccess) return e;
  *out = new SplitGroup();
  (*out)->device = device;
  (*out)->window_ms = window_ms;
  (*out)->capacity = cap;
  return cudaSuccess;
}

void group_destroy(SplitGroup* g) {
  if (!g) return;
  for (auto& f : g->flights) {
    cudaEventSynchronize(f.ev);
    cudaEventDestroy(f.ev);
  }
  for (cudaEvent_t e : g->spare) cudaEventDestroy(e);
  delete g;
}

void group_set_expected(SplitGroup* g, int expected) {
  std::lock_guard<std::mutex> lock(g->mu);
  g->expected = expected;
  g->cv.notify_all();
}

void group_set_policy(SplitGroup* g, int mode, double window_ms) {
  std::lock_guard<std::mutex> lock(g->mu);
  g->mode = mode;
  g->window_ms = window_ms;
}

void group_stats(SplitGroup* g, long long* launches, long long* items) {
  std::lock_guard<std::mutex> lock(g->mu);
  *launches = g->launches;
  *items = g->items;
}

// The member's Jacobi through the group: posts it after the work already on
// `st`, waits until it has been launched, and makes `st` wait for its
// completion.  ready and done are the member's own events, gstate its own 24
// device words (the barrier of a batch it leads).
cudaError_t group_jacobi(SplitGroup* g, const JacobiItem& item, cudaEvent_t ready, cudaEvent_t done,
                         unsigned int* gstate, cudaStream_t st) {
  cudaError_t status = cudaSuccess;
  cudaError_t e = cudaEventRecord(ready, st);
  if (e != cudaSuccess) return e;
  {
    std::unique_lock<std::mutex> lock(g->mu);
    const long long ticket = g->next_ticket++;
    g->pending.push_back({item, ready, done, st, gstate, &status, ticket});
    const auto deadline = Clock::now() + std::chrono::microseconds((long long)(g->window_ms * 1e3));
    for (;;) {
      retire_locked(g);
      if (g->launched_upto >= ticket) break;
      if (due_locked(g, deadline)) {
        launch_locked(g);
        continue;
      }
      g->cv.wait_for(lock, kPoll);
    }
  }
  if (status != cudaSuccess) return status;
  return cudaStreamWaitEvent(st, done, 0);
}

}  // namespace ite
