// Serving loop: continuous batching of Montgomery-multiplication and sweep
// jobs on one GPU.
//
// A server owns a device arena of a fixed byte budget and `slots` worker
// threads, each with its own CUDA stream.  Submitted jobs wait in one FIFO
// queue.  An idle worker admits the job at the head of the queue as soon as
// the job's device buffers fit in the arena (first fit; jobs larger than the
// whole budget are refused at submission), so jobs that arrive while others
// run are admitted as slots and memory free up, and the work of up to
// `slots` jobs overlaps on the device.  A modmul job copies its host operands
// into its arena buffers, runs mont_mul on the worker's stream and copies the
// products back; a sweep job runs mont_verify_sweep on that stream.  Every
// wait for the device is bounded: the worker polls an event and gives up
// after the server's job timeout, reporting MONT_ETIMEOUT (the job's arena
// region is then retired, never reused, since the device may still write it).
// Each job records its submission, admission and completion times on a
// steady clock, from which callers compute latency percentiles.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"

namespace montgb {
namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// First-fit allocator over [0, capacity), kAlign granularity.
class Arena {
 public:
  explicit Arena(size_t cap) : cap_(cap) {
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second >= bytes) {
        *off = it->first;
        const size_t rest = it->second - bytes;
        const size_t at = it->first + bytes;
        free_.erase(it);
        if (rest) free_[at] = rest;
        return true;
      }
    }
    return false;
  }
  void release(size_t off, size_t bytes) {
    bytes = align_up(bytes);
    auto it = free_.emplace(off, bytes).first;
    auto next = std::next(it);
    if (next != free_.end() && it->first + it->second == next->first) {
      it->second += next->second;
      free_.erase(next);
    }
    if (it != free_.begin()) {
      auto prev = std::prev(it);
      if (prev->first + prev->second == it->first) {
        prev->second += it->second;
        free_.erase(it);
      }
    }
  }
  size_t free_bytes() const {
    size_t s = 0;
    for (const auto& kv : free_) s += kv.second;
    return s;
  }
  size_t capacity() const { return cap_; }

 private:
  size_t cap_;
  std::map<size_t, size_t> free_;
};

struct Job {
  uint64_t id = 0;
  mont_job desc{};
  mont_bounds claimed{};
  bool has_claimed = false;
  size_t bytes = 0;       // arena bytes reserved while the job runs
  double t_submit = 0, t_admit = 0, t_done = 0;
  int status = MONT_OK;
};

}  // namespace
}  // namespace montgb

using namespace montgb;

struct mont_server {
  int device = 0;
  char* base = nullptr;
  Arena arena{0};
  int timeout_ms = 60000;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Job*> queue;
  std::map<uint64_t, Job*> done;
  std::map<uint64_t, Job*> pending;  // submitted, not yet retrieved
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> streams;
  bool stopping = false;
  uint64_t next_id = 1;
  size_t running = 0;
  size_t retired_bytes = 0;
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

size_t job_bytes(const mont_job& j) {
  if (j.kind == MONT_JOB_MODMUL) {
    const size_t nb = align_up(j.n * 4u * static_cast<size_t>(j.ctx->n_limbs));
    return 3 * nb;
  }
  // a sweep's own scratch: its table, counters and example buffer
  const size_t n_odd = j.N_hi >= j.N_lo ? (j.N_hi - j.N_lo) / 2 + 1 : 0;
  return align_up(n_odd * 64 + j.cex_cap * sizeof(mont_cex) + 4096);
}

// Wait for all work enqueued so far on s, at most timeout_ms.
int bounded_sync(cudaStream_t s, int timeout_ms) {
  cudaEvent_t ev;
  cudaError_t e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaEventRecord(ev, s);
  if (e != cudaSuccess) {
    cudaEventDestroy(ev);
    return cuda_status(e);
  }
  const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
  int st = MONT_OK;
  auto pause = std::chrono::microseconds(2);
  for (;;) {
    e = cudaEventQuery(ev);
    if (e == cudaSuccess) break;
    if (e != cudaErrorNotReady) {
      st = cuda_status(e);
      break;
    }
    if (std::chrono::steady_clock::now() >= deadline) {
      st = MONT_ETIMEOUT;
      break;
    }
    std::this_thread::sleep_for(pause);
    if (pause < std::chrono::microseconds(200)) pause *= 2;
  }
  cudaEventDestroy(ev);
  return st;
}

int run_modmul(mont_server* sv, Job* j, char* dev, cudaStream_t s) {
  const mont_job& d = j->desc;
  if (d.n == 0) return MONT_OK;
  const size_t nb = d.n * 4u * static_cast<size_t>(d.ctx->n_limbs);
  char* da = dev;
  char* db = dev + align_up(nb);
  char* dout = db + align_up(nb);
  int st = MONT_OK;
  cudaError_t e = cudaMemcpyAsync(da, d.a, nb, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(db, d.b, nb, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) st = cuda_status(e);
  if (st == MONT_OK) st = mont_mul(d.ctx, da, db, dout, d.n, s);
  if (st == MONT_OK) {
    e = cudaMemcpyAsync(d.out, dout, nb, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) st = cuda_status(e);
  }
  // whatever was enqueued must finish before the region is released
  const int w = bounded_sync(s, sv->timeout_ms);
  return w == MONT_ETIMEOUT ? w : (st != MONT_OK ? st : w);
}

int run_sweep(Job* j, cudaStream_t s) {
  const mont_job& d = j->desc;
  return mont_verify_sweep(d.variant, d.log2R, d.alpha, d.N_lo, d.N_hi,
                           j->has_claimed ? &j->claimed : nullptr, d.flags, d.per_N_counts,
                           d.per_N_checked, d.cex, d.cex_cap, d.n_cex_total, s);
}

void worker(mont_server* sv, int slot) {
  cudaSetDevice(sv->device);
  cudaStream_t s = sv->streams[static_cast<size_t>(slot)];
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    Job* j = nullptr;
    size_t off = 0;
    for (;;) {
      if (!sv->queue.empty()) {
        Job* head = sv->queue.front();
        if (head->bytes > sv->arena.capacity() - sv->retired_bytes) {
          // regions retired by timeouts left too little memory for this job
          sv->queue.pop_front();
          head->t_admit = head->t_done = sv->now();
          head->status = MONT_ENOMEM;
          sv->done[head->id] = head;
          sv->cv_done.notify_all();
          continue;
        }
        if (sv->arena.alloc(head->bytes, &off)) {
          j = head;
          sv->queue.pop_front();
          break;
        }
      } else if (sv->stopping) {
        return;
      }
      sv->cv_work.wait(lk);
    }
    j->t_admit = sv->now();
    ++sv->running;
    lk.unlock();

    int st;
    if (j->desc.kind == MONT_JOB_MODMUL) {
      st = run_modmul(sv, j, sv->base + off, s);
    } else {
      st = run_sweep(j, s);
      if (st == MONT_EOVERFLOW) st = MONT_OK;  // counts are exact; the caller sees n_cex_total
    }

    lk.lock();
    if (st == MONT_ETIMEOUT) {
      sv->retired_bytes += align_up(j->bytes);  // the device may still write it: never reuse
    } else {
      sv->arena.release(off, j->bytes);
    }
    --sv->running;
    j->status = st;
    j->t_done = sv->now();
    sv->done[j->id] = j;
    sv->cv_work.notify_all();
    sv->cv_done.notify_all();
  }
}

}  // namespace

extern "C" int mont_server_create(mont_server_t* out, size_t mem_budget_bytes, int slots,
                                  int job_timeout_ms) {
  if (!out || slots < 1 || slots > 64 || mem_budget_bytes < kAlign) return MONT_EINVAL;
  mont_server* sv = new (std::nothrow) mont_server;
  if (!sv) return MONT_ENOMEM;
  cudaError_t e = cudaGetDevice(&sv->device);
  if (e == cudaSuccess) e = cudaMalloc(&sv->base, align_up(mem_budget_bytes));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete sv;
    return e == cudaErrorMemoryAllocation ? MONT_ENOMEM : cuda_status(e);
  }
  sv->arena = Arena(align_up(mem_budget_bytes));
  sv->timeout_ms = job_timeout_ms > 0 ? job_timeout_ms : 60000;
  for (int i = 0; i < slots; ++i) {
    cudaStream_t s;
    e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      for (auto st : sv->streams) cudaStreamDestroy(st);
      cudaFree(sv->base);
      delete sv;
      return cuda_status(e);
    }
    sv->streams.push_back(s);
  }
  for (int i = 0; i < slots; ++i) sv->workers.emplace_back(worker, sv, i);
  *out = sv;
  return MONT_OK;
}

extern "C" int mont_server_submit(mont_server_t sv, const mont_job* job, uint64_t* id) {
  if (!sv || !job || !id) return MONT_EINVAL;
  if (job->kind == MONT_JOB_MODMUL) {
    if (!job->ctx) return MONT_EINVAL;
    if (job->n > 0 && (!job->a || !job->b || !job->out)) return MONT_EINVAL;
  } else if (job->kind == MONT_JOB_SWEEP) {
    if (!job->per_N_counts || !job->n_cex_total || (job->cex_cap > 0 && !job->cex))
      return MONT_EINVAL;
  } else {
    return MONT_EINVAL;
  }
  Job* j = new (std::nothrow) Job;
  if (!j) return MONT_ENOMEM;
  j->desc = *job;
  if (job->kind == MONT_JOB_SWEEP && job->claimed) {
    j->claimed = *job->claimed;
    j->has_claimed = true;
  }
  j->desc.claimed = nullptr;
  j->bytes = job_bytes(*job);
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    if (j->bytes > sv->arena.capacity()) {
      delete j;
      return MONT_ENOMEM;
    }
    if (sv->stopping) {
      delete j;
      return MONT_EINVAL;
    }
    j->id = sv->next_id++;
    j->t_submit = sv->now();
    sv->pending[j->id] = j;
    sv->queue.push_back(j);
    *id = j->id;
  }
  sv->cv_work.notify_one();
  return MONT_OK;
}

extern "C" int mont_server_wait(mont_server_t sv, uint64_t id, int timeout_ms,
                                mont_job_result* res) {
  if (!sv) return MONT_EINVAL;
  std::unique_lock<std::mutex> lk(sv->mu);
  if (!sv->pending.count(id)) return MONT_EINVAL;
  const auto ready = [&] { return sv->done.count(id) > 0; };
  if (timeout_ms < 0) {
    sv->cv_done.wait(lk, ready);
  } else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready)) {
    return MONT_ETIMEOUT;
  }
  Job* j = sv->done[id];
  sv->done.erase(id);
  sv->pending.erase(id);
  if (res) {
    res->status = j->status;
    res->t_submit = j->t_submit;
    res->t_admit = j->t_admit;
    res->t_done = j->t_done;
  }
  delete j;
  return MONT_OK;
}

extern "C" int mont_server_query(mont_server_t sv, size_t* queued, size_t* running,
                                 size_t* arena_free, double* now_s) {
  if (!sv) return MONT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (queued) *queued = sv->queue.size();
  if (running) *running = sv->running;
  if (arena_free) *arena_free = sv->arena.free_bytes();
  if (now_s) *now_s = sv->now();
  return MONT_OK;
}

extern "C" int mont_server_destroy(mont_server_t sv) {
  if (!sv) return MONT_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stopping = true;
  }
  sv->cv_work.notify_all();
  for (auto& t : sv->workers) t.join();
  for (auto& kv : sv->pending) delete kv.second;
  for (auto s : sv->streams) cudaStreamDestroy(s);
  // a region retired after a timeout may still be written by the device:
  // wait for the device before freeing the arena
  if (sv->retired_bytes) cudaDeviceSynchronize();
  cudaFree(sv->base);
  delete sv;
  return MONT_OK;
}
