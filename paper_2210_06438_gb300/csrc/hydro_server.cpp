// hydro_server.cpp -- the serving loop: continuous batching of sub-grid tasks
// over the aggregated tile kernel.
//
// This is strategy 3 of Sec. V-D with several parent executors (strategy 2
// on top): tasks arrive at any time; while a launch stream is busy, newly
// arrived tasks wait; as soon as a stream is idle, every queued task that fits
// the memory budget (in arrival order, up to max_batch sub-grids) enters one
// aggregated launch on it.  A task's state (its ghosted input blocks) is
// already resident on the device; the budget bounds the bytes of admitted and
// unfinished tasks (their read blocks plus outputs), the analogue of the
// pre-allocated buffer pool of Sec. V-C.
//
// One scheduler thread owns the CUDA work: it polls the streams' completion
// events, admits, builds the work list in the stream's pinned staging buffer,
// copies it and launches.  Callers only touch the queue and the task table
// under the server mutex.  In dry-run mode no CUDA call is made and a launch
// completes a fixed time after it starts, so the host logic can be tested on
// machines without a GPU.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "hydro.h"
#include "hydro_internal.h"
#include "hydro_kernels.cuh"

using hydro_dev::Status;
using hydro_dev::Tile;

namespace hydro_host {
int ctx_status_ptr(Status** st, int* n_sm, int* smem_optin);
void fill_tile(Tile& t, const hydro_subgrid_t& d, int ghost, int64_t out_off, int64_t amax_off,
               int sub, int tx, int ty, int tz, bool multi);
}  // namespace hydro_host
using namespace hydro_host;

static int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

namespace {

enum TaskState { QUEUED = 0, LAUNCHED = 1, DONE = 2, FAILED = 3 };

struct Task {
  int64_t ticket = 0;
  std::vector<hydro_subgrid_t> sg;
  double* out = nullptr;
  double* amax = nullptr;
  int64_t bytes = 0;
  int64_t tiles = 0;
  int64_t t_submit = 0, t_launch = 0, t_done = 0;
  int state = QUEUED;
};

struct Slot {
  cudaStream_t stream = nullptr;
  cudaEvent_t done = nullptr;
  Tile* dev_tiles = nullptr;
  Tile* host_tiles = nullptr;
  size_t cap = 0;
  bool busy = false;
  int64_t t_start = 0;  // dry run: launch start
  std::vector<int64_t> tickets;
  int64_t bytes = 0;
};

}  // namespace

struct hydro_server {
  hydro_server_cfg_t cfg;
  int device = 0;
  int n_sm = 1, smem_optin = 0;
  Status* status = nullptr;
  std::vector<Slot> slots;
  std::mutex mu;
  std::condition_variable cv;       // task completions
  std::condition_variable work_cv;  // new submissions
  std::deque<int64_t> queue;
  std::unordered_map<int64_t, Task> tasks;
  int64_t next_ticket = 1;
  hydro_server_stats_t st;
  bool stop = false;
  std::thread thr;
  std::vector<Tile> scratch;
};

static int64_t task_bytes(const hydro_subgrid_t* sg, int32_t n, int ghost, int64_t* tiles) {
  int64_t b = 0, t = 0;
  for (int32_t i = 0; i < n; i++) {
    int64_t N = sg[i].N, F = sg[i].n_fields, G = N + 2 * ghost;
    b += (G * G * G + N * N * N) * F * 8 + 8;
    int64_t nt = (N + hydro_dev::TE - 1) / hydro_dev::TE;
    t += nt * nt * nt;
  }
  *tiles = t;
  return b;
}

// Build and launch one aggregated work list for the tasks in `ids` on slot s.
// Called by the scheduler thread with the mutex held.
static int launch_batch(hydro_server* S, Slot& s, const std::vector<int64_t>& ids) {
  const int ghost = S->cfg.ghost;
  int64_t ntiles = 0;
  int Fmax = 6;
  for (int64_t id : ids) {
    const Task& T = S->tasks[id];
    ntiles += T.tiles;
    for (auto& d : T.sg) Fmax = std::max(Fmax, (int)d.n_fields);
  }
  s.tickets = ids;
  s.bytes = 0;
  int64_t now = now_ns();
  for (int64_t id : ids) {
    Task& T = S->tasks[id];
    T.state = LAUNCHED;
    T.t_launch = now;
    s.bytes += T.bytes;
  }
  s.busy = true;
  s.t_start = now;
  if (S->cfg.dry_run_ns > 0) return HYDRO_OK;

  cudaError_t e;
  if ((size_t)ntiles > s.cap) {  // grow this stream's work-list buffers
    if ((e = cudaStreamSynchronize(s.stream)) != cudaSuccess) return cuda_fail(e, "sync");
    if (s.dev_tiles) cudaFree(s.dev_tiles);
    if (s.host_tiles) cudaFreeHost(s.host_tiles);
    s.dev_tiles = nullptr;
    s.host_tiles = nullptr;
    size_t cap = std::max<size_t>((size_t)ntiles, 2 * s.cap);
    if (cudaMalloc(&s.dev_tiles, cap * sizeof(Tile)) != cudaSuccess) return HYDRO_ENOMEM;
    if (cudaMallocHost(&s.host_tiles, cap * sizeof(Tile)) != cudaSuccess) return HYDRO_ENOMEM;
    s.cap = cap;
  }
  // outputs of all tasks are addressed relative to the first task's pointers
  double* obase = S->tasks[ids[0]].out;
  double* abase = S->tasks[ids[0]].amax;
  size_t k = 0;
  for (int64_t id : ids) {
    Task& T = S->tasks[id];
    int64_t off = (T.out - obase);
    for (size_t i = 0; i < T.sg.size(); i++) {
      const hydro_subgrid_t& d = T.sg[i];
      int nt = (d.N + hydro_dev::TE - 1) / hydro_dev::TE;
      bool multi = nt > 1;
      if (multi && (e = cudaMemsetAsync(T.amax + i, 0, sizeof(double), s.stream)) != cudaSuccess)
        return cuda_fail(e, "cudaMemsetAsync(amax)");
      for (int tz = 0; tz < nt; tz++)
        for (int ty = 0; ty < nt; ty++)
          for (int tx = 0; tx < nt; tx++)
            fill_tile(s.host_tiles[k++], d, ghost, off, (T.amax + i) - abase, (int)i, tx, ty, tz,
                      multi);
      off += (int64_t)d.n_fields * d.N * d.N * d.N;
    }
  }
  if ((e = cudaMemcpyAsync(s.dev_tiles, s.host_tiles, k * sizeof(Tile), cudaMemcpyHostToDevice,
                           s.stream)) != cudaSuccess)
    return cuda_fail(e, "cudaMemcpyAsync(work list)");
  LaunchCfg c = default_cfg(S->cfg.prec, Fmax, S->n_sm, S->smem_optin, (int64_t)k, true,
                            (S->cfg.flags & HYDRO_F_QUAD26) != 0);
  if ((e = launch_tiles(c, S->cfg.prec, s.dev_tiles, (int)k, Fmax, obase, abase, S->status,
                        S->cfg.gamma, 1, s.stream, (S->cfg.flags & HYDRO_F_KNP) ? 1 : 0)) != cudaSuccess)
    return cuda_fail(e, "launch");
  if ((e = cudaEventRecord(s.done, s.stream)) != cudaSuccess) return cuda_fail(e, "cudaEventRecord");
  return HYDRO_OK;
}

static void finish_slot(hydro_server* S, Slot& s, int state) {
  int64_t now = now_ns();
  for (int64_t id : s.tickets) {
    Task& T = S->tasks[id];
    T.state = state;
    T.t_done = now;
    T.sg.clear();
    T.sg.shrink_to_fit();
    S->st.completed++;
  }
  S->st.bytes_in_flight -= s.bytes;
  s.tickets.clear();
  s.bytes = 0;
  s.busy = false;
}

static void scheduler(hydro_server* S) {
  if (S->cfg.dry_run_ns <= 0) cudaSetDevice(S->device);
  std::unique_lock<std::mutex> lk(S->mu);
  while (true) {
    bool progressed = false;
    // completions
    for (Slot& s : S->slots) {
      if (!s.busy) continue;
      bool done;
      if (S->cfg.dry_run_ns > 0) {
        done = now_ns() - s.t_start >= S->cfg.dry_run_ns;
      } else {
        cudaError_t q = cudaEventQuery(s.done);
        done = q == cudaSuccess;
        if (q != cudaSuccess && q != cudaErrorNotReady) {
          cuda_fail(q, "launch failed");
          finish_slot(S, s, FAILED);
          progressed = true;
          continue;
        }
      }
      if (done) {
        finish_slot(S, s, DONE);
        progressed = true;
      }
    }
    if (progressed) S->cv.notify_all();
    // admission: every idle stream takes the queued tasks that fit
    for (Slot& s : S->slots) {
      if (s.busy || S->queue.empty()) continue;
      std::vector<int64_t> ids;
      int64_t nsub = 0, bytes = 0;
      while (!S->queue.empty()) {
        Task& T = S->tasks[S->queue.front()];
        int64_t n = (int64_t)T.sg.size();
        if (!ids.empty() && (S->cfg.per_task || nsub + n > S->cfg.max_batch)) break;
        if (S->st.bytes_in_flight + bytes + T.bytes > S->cfg.budget_bytes) break;
        ids.push_back(T.ticket);
        nsub += n;
        bytes += T.bytes;
        S->queue.pop_front();
        if (S->cfg.per_task) break;
      }
      if (ids.empty()) break;  // the head task waits for budget
      S->st.bytes_in_flight += bytes;
      S->st.peak_bytes_in_flight = std::max(S->st.peak_bytes_in_flight, S->st.bytes_in_flight);
      S->st.launches++;
      S->st.subgrids_launched += nsub;
      S->st.max_subgrids_per_launch = std::max(S->st.max_subgrids_per_launch, nsub);
      int rc = launch_batch(S, s, ids);
      if (rc != HYDRO_OK) finish_slot(S, s, FAILED);
      progressed = true;
    }
    S->st.queued = (int64_t)S->queue.size();
    bool any_busy = false;
    for (Slot& s : S->slots) any_busy |= s.busy;
    if (S->stop && S->queue.empty() && !any_busy) break;
    if (!progressed) {
      if (any_busy) {
        // launches in flight: poll their events again shortly
        lk.unlock();
        std::this_thread::sleep_for(std::chrono::microseconds(5));
        lk.lock();
      } else {
        S->work_cv.wait_for(lk, std::chrono::milliseconds(50));
      }
    }
  }
}

extern "C" {

int64_t hydro_now_ns(void) { return now_ns(); }

int hydro_server_create(const hydro_server_cfg_t* cfg, hydro_server_t** out) {
  if (!cfg || !out) return HYDRO_EINVAL;
  *out = nullptr;
  if (cfg->budget_bytes <= 0 || cfg->max_batch < 1 || cfg->n_streams < 1 || cfg->n_streams > 1024 ||
      cfg->ghost < 3 || cfg->queue_capacity < 1 || !(cfg->gamma > 1.0) ||
      (cfg->prec != HYDRO_FP64 && cfg->prec != HYDRO_FP32_FLUX_FP64_ACC) ||
      (cfg->flags & ~(uint32_t)(HYDRO_F_KNP | HYDRO_F_QUAD26)))
    return HYDRO_EINVAL;
  hydro_server* S = new hydro_server();
  S->cfg = *cfg;
  memset(&S->st, 0, sizeof S->st);
  S->slots.resize(cfg->n_streams);
  if (cfg->dry_run_ns <= 0) {
    int rc = ctx_status_ptr(&S->status, &S->n_sm, &S->smem_optin);
    if (rc) {
      delete S;
      return rc;
    }
    cudaGetDevice(&S->device);
    for (Slot& s : S->slots) {
      cudaError_t e;
      size_t cap = (size_t)std::max(64, cfg->max_batch);  // one 8^3 tile per sub-grid
      if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess ||
          (e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess ||
          (e = cudaMalloc(&s.dev_tiles, cap * sizeof(Tile))) != cudaSuccess ||
          (e = cudaMallocHost(&s.host_tiles, cap * sizeof(Tile))) != cudaSuccess) {
        int r = cuda_fail(e, "server streams");
        for (Slot& t : S->slots) {
          if (t.stream) cudaStreamDestroy(t.stream);
          if (t.done) cudaEventDestroy(t.done);
          if (t.dev_tiles) cudaFree(t.dev_tiles);
          if (t.host_tiles) cudaFreeHost(t.host_tiles);
        }
        delete S;
        return r;
      }
      s.cap = cap;
    }
  }
  S->thr = std::thread(scheduler, S);
  *out = S;
  return HYDRO_OK;
}

int hydro_server_submit(hydro_server_t* S, const hydro_subgrid_t* sg, int32_t n, double* out_dUdt,
                        double* out_amax, int64_t* ticket) {
  if (!S || !sg || n < 1 || !out_dUdt || !out_amax || !ticket) return HYDRO_EINVAL;
  for (int32_t i = 0; i < n; i++) {
    const hydro_subgrid_t& d = sg[i];
    if (!d.U || d.N < 2 || d.N > HYDRO_MAX_N || d.n_fields < 6 || d.n_fields > HYDRO_MAX_FIELDS ||
        !(d.dx > 0.0))
      return HYDRO_EINVAL;
  }
  int64_t tiles;
  int64_t bytes = task_bytes(sg, n, S->cfg.ghost, &tiles);
  std::lock_guard<std::mutex> g(S->mu);
  if (bytes > S->cfg.budget_bytes) {
    S->st.rejected++;
    return HYDRO_EBUDGET;
  }
  if ((int64_t)S->queue.size() >= S->cfg.queue_capacity) {
    S->st.rejected++;
    return HYDRO_EBUSY;
  }
  Task T;
  T.ticket = S->next_ticket++;
  T.sg.assign(sg, sg + n);
  T.out = out_dUdt;
  T.amax = out_amax;
  T.bytes = bytes;
  T.tiles = tiles;
  T.t_submit = now_ns();
  S->queue.push_back(T.ticket);
  *ticket = T.ticket;
  S->tasks.emplace(T.ticket, std::move(T));
  S->st.submitted++;
  S->work_cv.notify_one();
  return HYDRO_OK;
}

static int state_rc(const Task& T) {
  if (T.state == DONE) return HYDRO_OK;
  if (T.state == FAILED) return HYDRO_ECUDA;
  return HYDRO_EBUSY;
}

int hydro_server_poll(hydro_server_t* S, int64_t ticket) {
  if (!S) return HYDRO_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->tasks.find(ticket);
  if (it == S->tasks.end()) return HYDRO_EINVAL;
  return state_rc(it->second);
}

int hydro_server_wait(hydro_server_t* S, int64_t ticket, int64_t timeout_ns) {
  if (!S) return HYDRO_EINVAL;
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->tasks.find(ticket);
  if (it == S->tasks.end()) return HYDRO_EINVAL;
  auto pred = [&] { return it->second.state >= DONE; };
  if (timeout_ns < 0) {
    S->cv.wait(lk, pred);
  } else if (!S->cv.wait_for(lk, std::chrono::nanoseconds(timeout_ns), pred)) {
    return HYDRO_ETIMEDOUT;
  }
  return state_rc(it->second);
}

int hydro_server_times(hydro_server_t* S, int64_t ticket, int64_t* ts, int64_t* tl, int64_t* td) {
  if (!S) return HYDRO_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  auto it = S->tasks.find(ticket);
  if (it == S->tasks.end()) return HYDRO_EINVAL;
  if (ts) *ts = it->second.t_submit;
  if (tl) *tl = it->second.t_launch;
  if (td) *td = it->second.t_done;
  return HYDRO_OK;
}

int hydro_server_stats(hydro_server_t* S, hydro_server_stats_t* out) {
  if (!S || !out) return HYDRO_EINVAL;
  std::lock_guard<std::mutex> g(S->mu);
  *out = S->st;
  out->queued = (int64_t)S->queue.size();
  return HYDRO_OK;
}

int hydro_server_destroy(hydro_server_t* S) {
  if (!S) return HYDRO_EINVAL;
  {
    std::lock_guard<std::mutex> g(S->mu);
    S->stop = true;
    S->work_cv.notify_all();
  }
  S->thr.join();
  if (S->cfg.dry_run_ns <= 0) {
    for (Slot& s : S->slots) {
      if (s.stream) cudaStreamSynchronize(s.stream);
      if (s.dev_tiles) cudaFree(s.dev_tiles);
      if (s.host_tiles) cudaFreeHost(s.host_tiles);
      if (s.done) cudaEventDestroy(s.done);
      if (s.stream) cudaStreamDestroy(s.stream);
    }
  }
  delete S;
  return HYDRO_OK;
}

}  // extern "C"
