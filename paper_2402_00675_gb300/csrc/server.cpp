// Serving loop: continuous batching of Montgomery-multiplication and sweep
// jobs on one GPU.
//
// A server owns a device arena of a fixed byte budget and `slots` worker
// threads.  Submitted jobs wait in two FIFO queues, one for modmul jobs and
// one for sweep jobs.  An idle worker admits the job at the head of a queue
// as soon as the job's device memory fits in the arena (first fit; jobs
// larger than the whole budget are refused at submission), so jobs that
// arrive while others run are admitted as slots and memory free up, and the
// work of up to `slots` jobs overlaps on the device.  The first
// max(1, slots / 4) workers take the sweep queue's head first and otherwise a
// modmul job; the others take modmul jobs only.  One sweep launch already
// fills the GPU, so this caps concurrent sweeps without costing throughput,
// and a modmul job never waits in the queue behind a sweep.
//
// A modmul job copies its host operands into its arena buffers, runs mont_mul
// and copies the products back, on its worker's high-priority stream, in
// pieces of 16 MiB per operand, at most two in flight, so that the copies of
// concurrent jobs interleave.  A
// sweep job takes its table, counters and example buffer from the arena too
// and runs on its worker's low-priority stream in launches of about 2^31
// checks (a millisecond or two of the whole GPU), at most two in flight, so
// that the kernels of modmul jobs on other streams are scheduled between them
// instead of waiting for the whole sweep.
//
// Every wait for the device is bounded by the job's deadline (its own timeout,
// or the server's).  A job past its deadline completes with MONT_ETIMEOUT and
// becomes a straggler: its device work may still be running, so its arena
// region and (for a modmul job) its host buffers stay in use until an event
// recorded behind that work completes.  Stragglers are polled; a finished one
// gives its region back.  mont_server_job_busy tells a caller when a
// timed-out job's buffers are free.  Each job records its submission,
// admission and completion times on a steady clock, from which callers
// compute latency percentiles.
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "internal.h"
#include "sweep.h"

namespace montgb {
namespace {

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }

// Checks per sweep launch: about 1 ms of the whole GPU at 2 T checks/s.
constexpr uint64_t kSweepChecksPerLaunch = uint64_t{1} << 31;

// First-fit allocator over [0, capacity), kAlign granularity.
class Arena {
 public:
  explicit Arena(size_t cap) : cap_(cap) {
    if (cap) free_[0] = cap;
  }
  bool alloc(size_t bytes, size_t* off) {
    bytes = align_up(bytes);
    if (!bytes) {
      *off = 0;
      return true;
    }
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
    if (!bytes) return;
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

using Clock = std::chrono::steady_clock;

struct Job {
  uint64_t id = 0;
  mont_job desc{};
  mont_bounds claimed{};
  bool has_claimed = false;
  std::unique_ptr<SweepPlan> plan;   // sweep jobs: built and checked at submission
  size_t bytes = 0;                  // arena bytes reserved while the job runs
  int timeout_ms = 0;
  double t_submit = 0, t_admit = 0, t_done = 0;
  double t_blocked = -1;             // first time the job could not be admitted with nothing running
  int status = MONT_OK;
};

// A timed-out job whose device work may still be running.
struct Straggler {
  uint64_t id;
  cudaEvent_t ev;     // recorded behind every piece of the job's device work
  size_t off, bytes;  // its arena region
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
  std::deque<Job*> modmul_q;          // queued modmul jobs
  std::deque<Job*> sweep_q;           // queued sweep jobs
  int sweep_workers = 1;              // workers 0 .. sweep_workers-1 also run sweeps
  std::map<uint64_t, Job*> done;
  std::map<uint64_t, Job*> pending;  // submitted, not yet retrieved
  std::vector<Straggler> stragglers;
  std::vector<std::thread> workers;
  std::vector<cudaStream_t> hi_streams;  // per slot: modmul jobs (highest priority)
  std::vector<cudaStream_t> lo_streams;  // per slot: sweep jobs (lowest priority)
  bool stopping = false;
  uint64_t next_id = 1;
  size_t running = 0;
  Clock::time_point t0 = Clock::now();

  double now() const { return std::chrono::duration<double>(Clock::now() - t0).count(); }
};

namespace {

size_t modmul_bytes(const mont_job& j) {
  return 3 * align_up(j.n * 4u * static_cast<size_t>(j.ctx->n_limbs));
}

// Give back the regions of stragglers whose device work has finished (a
// failed query also ends the wait: the context no longer runs that work).
// Called with sv->mu held; returns true if a region was given back.
bool reap_locked(mont_server* sv) {
  bool freed = false;
  for (size_t i = 0; i < sv->stragglers.size();) {
    const cudaError_t e = cudaEventQuery(sv->stragglers[i].ev);
    if (e == cudaErrorNotReady) {
      ++i;
      continue;
    }
    if (e != cudaSuccess) cudaGetLastError();
    sv->arena.release(sv->stragglers[i].off, sv->stragglers[i].bytes);
    cudaEventDestroy(sv->stragglers[i].ev);
    sv->stragglers.erase(sv->stragglers.begin() + static_cast<std::ptrdiff_t>(i));
    freed = true;
  }
  return freed;
}

// Poll ev until it completes or the deadline passes (MONT_ETIMEOUT).
int wait_event(cudaEvent_t ev, Clock::time_point deadline, int max_pause_us) {
  auto pause = std::chrono::microseconds(2);
  for (;;) {
    const cudaError_t e = cudaEventQuery(ev);
    if (e == cudaSuccess) return MONT_OK;
    if (e != cudaErrorNotReady) return cuda_status(e);
    if (Clock::now() >= deadline) return MONT_ETIMEOUT;
    std::this_thread::sleep_for(pause);
    if (pause < std::chrono::microseconds(max_pause_us)) pause *= 2;
  }
}

// Record an event behind everything enqueued on s so far.
int record(cudaStream_t s, cudaEvent_t* ev) {
  cudaError_t e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaEventRecord(*ev, s);
  if (e != cudaSuccess) {
    cudaEventDestroy(*ev);
    *ev = nullptr;
    return cuda_status(e);
  }
  return MONT_OK;
}

// Outcome of a job's device work: a status and, when it timed out, the event
// behind its work (the caller makes it a straggler).
struct Run {
  int status = MONT_OK;
  cudaEvent_t pending = nullptr;
};

// Wait (bounded) for everything enqueued on s; on timeout keep the event.
Run finish(cudaStream_t s, Clock::time_point deadline, int enqueue_status) {
  Run r;
  cudaEvent_t ev = nullptr;
  const int st = record(s, &ev);
  if (st != MONT_OK) {
    // nothing to wait on: fall back to an unbounded synchronisation
    const cudaError_t e = cudaStreamSynchronize(s);
    r.status = enqueue_status != MONT_OK ? enqueue_status : (e == cudaSuccess ? st : cuda_status(e));
    return r;
  }
  const int w = wait_event(ev, deadline, 200);
  if (w == MONT_ETIMEOUT) {
    r.status = MONT_ETIMEOUT;
    r.pending = ev;
    return r;
  }
  cudaEventDestroy(ev);
  r.status = enqueue_status != MONT_OK ? enqueue_status : w;
  return r;
}

// Bytes of one operand piece of a modmul job.  A job's transfers are issued
// in pieces, at most two in flight: the streams of the server share the
// device's few hardware queues, and a job that enqueued all of its copies at
// once would put a small job's commands behind all of them.  With bounded
// pieces a small job waits behind at most a few pieces of a large one, and a
// large job's own copies overlap its kernels.
constexpr size_t kCopyPieceBytes = size_t{16} << 20;

Run run_modmul(Job* j, char* dev, cudaStream_t s, Clock::time_point deadline) {
  const mont_job& d = j->desc;
  if (d.n == 0) return Run{};
  const size_t eb = 4u * static_cast<size_t>(d.ctx->n_limbs);
  const size_t nb = d.n * eb;
  char* da = dev;
  char* db = dev + align_up(nb);
  char* dout = db + align_up(nb);
  const size_t piece = kCopyPieceBytes / eb > 0 ? kCopyPieceBytes / eb : 1;   // elements
  const auto* ha = static_cast<const char*>(d.a);
  const auto* hb = static_cast<const char*>(d.b);
  auto* hout = static_cast<char*>(d.out);
  cudaEvent_t inflight[2] = {nullptr, nullptr};
  int st = MONT_OK;
  size_t k = 0;
  for (size_t e0 = 0; st == MONT_OK && e0 < d.n; e0 += piece, ++k) {
    cudaEvent_t& slot = inflight[k % 2];
    if (slot) {  // two pieces back: wait for it before queueing another
      st = wait_event(slot, deadline, 50);
      cudaEventDestroy(slot);
      slot = nullptr;
      if (st != MONT_OK) break;
    }
    const size_t cnt = d.n - e0 < piece ? d.n - e0 : piece;
    const size_t off = e0 * eb, bytes = cnt * eb;
    cudaError_t e = cudaMemcpyAsync(da + off, ha + off, bytes, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(db + off, hb + off, bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) {
      st = cuda_status(e);
      break;
    }
    st = mont_mul(d.ctx, da + off, db + off, dout + off, cnt, s);
    if (st != MONT_OK) break;
    e = cudaMemcpyAsync(hout + off, dout + off, bytes, cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) {
      st = cuda_status(e);
      break;
    }
    if (d.n - e0 > piece) st = record(s, &slot);   // no event after the last piece
  }
  for (auto& ev : inflight)
    if (ev) cudaEventDestroy(ev);
  // whatever was enqueued must finish before the region and buffers are free
  return finish(s, deadline, st);
}

// The sweep in launches of about kSweepChecksPerLaunch checks, at most two in
// flight; the deadline is checked between launches, and the results are read
// back only once every launch has completed.
Run run_sweep(Job* j, char* dev, cudaStream_t s, Clock::time_point deadline) {
  const SweepPlan& plan = *j->plan;
  const mont_job& d = j->desc;
  Run r;
  if (plan.tab.empty()) {
    *d.n_cex_total = 0;
    return r;
  }
  cudaError_t e = sweep_upload(plan, dev, s);
  const uint64_t step = sweep_items_for_checks(plan, kSweepChecksPerLaunch);
  cudaEvent_t inflight[2] = {nullptr, nullptr};
  int st = e == cudaSuccess ? MONT_OK : cuda_status(e);
  uint64_t launch = 0;
  for (uint64_t lo = 0; st == MONT_OK && lo < plan.items; lo += step, ++launch) {
    cudaEvent_t& slot = inflight[launch % 2];
    if (slot) {  // two launches back: wait for it before queueing another
      const int w = wait_event(slot, deadline, 50);
      cudaEventDestroy(slot);
      slot = nullptr;
      if (w != MONT_OK) {
        st = w;
        break;
      }
    }
    e = sweep_launch(plan, dev, lo, lo + step, s);
    if (e != cudaSuccess) {
      st = cuda_status(e);
      break;
    }
    st = record(s, &slot);
  }
  for (auto& ev : inflight)
    if (ev) cudaEventDestroy(ev);
  r = finish(s, deadline, st);
  if (r.status != MONT_OK) return r;
  r.status = sweep_collect(plan, dev, s, d.per_N_counts, d.cex, d.n_cex_total);
  if (r.status == MONT_EOVERFLOW) r.status = MONT_OK;  // counts are exact; the caller sees n_cex_total
  return r;
}

void complete_locked(mont_server* sv, Job* j, int status) {
  j->status = status;
  j->t_done = sv->now();
  sv->done[j->id] = j;
  sv->cv_done.notify_all();
}

// Admit the head of q if it fits; complete it with MONT_ENOMEM when it never
// can (nothing running, and no memory held by timed-out jobs comes back
// within its timeout).  Returns the admitted job or nullptr.
Job* admit_head_locked(mont_server* sv, std::deque<Job*>& q, size_t* off) {
  while (!q.empty()) {
    Job* head = q.front();
    if (sv->arena.alloc(head->bytes, off)) {
      q.pop_front();
      return head;
    }
    if (sv->running != 0) return nullptr;
    const double now = sv->now();
    if (head->t_blocked < 0) head->t_blocked = now;
    if (!sv->stragglers.empty() && (now - head->t_blocked) * 1e3 <= head->timeout_ms) return nullptr;
    q.pop_front();
    head->t_admit = now;
    complete_locked(sv, head, MONT_ENOMEM);
  }
  return nullptr;
}

void worker(mont_server* sv, int slot) {
  cudaSetDevice(sv->device);
  const bool runs_sweeps = slot < sv->sweep_workers;
  std::unique_lock<std::mutex> lk(sv->mu);
  for (;;) {
    Job* j = nullptr;
    size_t off = 0;
    for (;;) {
      reap_locked(sv);
      if (runs_sweeps) j = admit_head_locked(sv, sv->sweep_q, &off);
      if (!j) j = admit_head_locked(sv, sv->modmul_q, &off);
      if (j) break;
      if (sv->stopping && sv->modmul_q.empty() && (!runs_sweeps || sv->sweep_q.empty())) return;
      if (sv->stragglers.empty()) {
        sv->cv_work.wait(lk);
      } else {
        sv->cv_work.wait_for(lk, std::chrono::milliseconds(1));
      }
    }
    j->t_admit = sv->now();
    ++sv->running;
    lk.unlock();

    const auto deadline = Clock::now() + std::chrono::milliseconds(j->timeout_ms);
    const Run r = j->desc.kind == MONT_JOB_MODMUL
                      ? run_modmul(j, sv->base + off, sv->hi_streams[static_cast<size_t>(slot)], deadline)
                      : run_sweep(j, sv->base + off, sv->lo_streams[static_cast<size_t>(slot)], deadline);

    lk.lock();
    if (r.pending) {
      sv->stragglers.push_back(Straggler{j->id, r.pending, off, j->bytes});
    } else {
      sv->arena.release(off, j->bytes);
    }
    --sv->running;
    complete_locked(sv, j, r.status);
    sv->cv_work.notify_all();
  }
}

}  // namespace

extern "C" int mont_server_create(mont_server_t* out, size_t mem_budget_bytes, int slots,
                                  int job_timeout_ms) {
  if (!out || slots < 1 || slots > 64 || mem_budget_bytes < kAlign) return MONT_EINVAL;
  mont_server* sv = new (std::nothrow) mont_server;
  if (!sv) return MONT_ENOMEM;
  int least = 0, greatest = 0;
  cudaError_t e = cudaGetDevice(&sv->device);
  if (e == cudaSuccess) e = cudaDeviceGetStreamPriorityRange(&least, &greatest);
  if (e == cudaSuccess) e = cudaMalloc(&sv->base, align_up(mem_budget_bytes));
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete sv;
    return e == cudaErrorMemoryAllocation ? MONT_ENOMEM : cuda_status(e);
  }
  sv->arena = Arena(align_up(mem_budget_bytes));
  sv->timeout_ms = job_timeout_ms > 0 ? job_timeout_ms : 60000;
  sv->sweep_workers = slots / 4 > 1 ? slots / 4 : 1;
  for (int i = 0; i < slots && e == cudaSuccess; ++i) {
    cudaStream_t hi = nullptr, lo = nullptr;
    e = cudaStreamCreateWithPriority(&hi, cudaStreamNonBlocking, greatest);
    if (e == cudaSuccess) {
      sv->hi_streams.push_back(hi);
      e = cudaStreamCreateWithPriority(&lo, cudaStreamNonBlocking, least);
      if (e == cudaSuccess) sv->lo_streams.push_back(lo);
    }
  }
  if (e != cudaSuccess) {
    for (auto s : sv->hi_streams) cudaStreamDestroy(s);
    for (auto s : sv->lo_streams) cudaStreamDestroy(s);
    cudaFree(sv->base);
    delete sv;
    return cuda_status(e);
  }
  for (int i = 0; i < slots; ++i) sv->workers.emplace_back(worker, sv, i);
  *out = sv;
  return MONT_OK;
}

extern "C" int mont_server_submit(mont_server_t sv, const mont_job* job, uint64_t* id) {
  if (!sv || !job || !id) return MONT_EINVAL;
  Job* j = new (std::nothrow) Job;
  if (!j) return MONT_ENOMEM;
  j->desc = *job;
  j->timeout_ms = job->timeout_ms > 0 ? job->timeout_ms : sv->timeout_ms;
  if (job->kind == MONT_JOB_MODMUL) {
    if (!job->ctx || (job->n > 0 && (!job->a || !job->b || !job->out))) {
      delete j;
      return MONT_EINVAL;
    }
    j->bytes = modmul_bytes(*job);
  } else if (job->kind == MONT_JOB_SWEEP) {
    if (!job->per_N_counts || !job->n_cex_total || (job->cex_cap > 0 && !job->cex)) {
      delete j;
      return MONT_EINVAL;
    }
    if (job->claimed) {
      j->claimed = *job->claimed;
      j->has_claimed = true;
    }
    j->plan.reset(new (std::nothrow) SweepPlan);
    if (!j->plan) {
      delete j;
      return MONT_ENOMEM;
    }
    const int st = sweep_plan(job->variant, job->log2R, job->alpha, job->N_lo, job->N_hi,
                              j->has_claimed ? &j->claimed : nullptr, job->flags, job->cex_cap,
                              job->per_N_counts, job->per_N_checked, j->plan.get());
    if (st != MONT_OK) {
      delete j;
      return st;
    }
    j->bytes = j->plan->tab.empty() ? 0 : sweep_scratch_bytes(j->plan->tab.size(), job->cex_cap);
  } else {
    delete j;
    return MONT_EINVAL;
  }
  j->desc.claimed = nullptr;
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
    (j->desc.kind == MONT_JOB_SWEEP ? sv->sweep_q : sv->modmul_q).push_back(j);
    *id = j->id;
  }
  sv->cv_work.notify_all();   // only some workers take sweeps
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

extern "C" int mont_server_job_busy(mont_server_t sv, uint64_t id, int* busy) {
  if (!sv || !busy) return MONT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (reap_locked(sv)) sv->cv_work.notify_all();
  *busy = 0;
  for (const auto& st : sv->stragglers)
    if (st.id == id) *busy = 1;
  return MONT_OK;
}

extern "C" int mont_server_query(mont_server_t sv, size_t* queued, size_t* running,
                                 size_t* arena_free, double* now_s) {
  if (!sv) return MONT_EINVAL;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (reap_locked(sv)) sv->cv_work.notify_all();
  if (queued) *queued = sv->modmul_q.size() + sv->sweep_q.size();
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
  // The workers have waited for every job but the stragglers; wait for those
  // (bounded by twice the server's timeout), stream by stream, never for the
  // whole device.
  const auto deadline = Clock::now() + std::chrono::milliseconds(2 * static_cast<int64_t>(sv->timeout_ms));
  bool idle = true;
  for (auto& st : sv->stragglers) {
    if (wait_event(st.ev, deadline, 1000) != MONT_OK) idle = false;
  }
  for (auto* streams : {&sv->hi_streams, &sv->lo_streams}) {
    for (auto s : *streams) {
      cudaEvent_t ev = nullptr;
      if (record(s, &ev) == MONT_OK) {
        if (wait_event(ev, deadline, 1000) != MONT_OK) idle = false;
        cudaEventDestroy(ev);
      } else if (cudaStreamSynchronize(s) != cudaSuccess) {
        idle = false;
      }
    }
  }
  for (auto& st : sv->stragglers) cudaEventDestroy(st.ev);
  for (auto s : sv->hi_streams) cudaStreamDestroy(s);
  for (auto s : sv->lo_streams) cudaStreamDestroy(s);
  // memory the device may still write is never freed
  if (idle) cudaFree(sv->base);
  delete sv;
  return idle ? MONT_OK : MONT_ETIMEOUT;
}
