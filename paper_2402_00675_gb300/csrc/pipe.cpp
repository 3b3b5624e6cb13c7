// Host-buffer pipeline: the element-wise operations on vectors in host memory.
//
// A pipe owns one device staging buffer cut into MONT_PIPE_SLOTS fixed
// slots, and three non-blocking streams: s_in (host-to-device copies),
// s_run (kernels) and s_out (device-to-host copies).  Chunk c of a run uses
// slot c mod MONT_PIPE_SLOTS:
//
//   s_in : wait out_done[slot]; copy the chunk of every distinct input;
//          record in_done[slot]
//   s_run: wait in_done[slot];  launch every operation on the slot;
//          record run_done[slot]
//   s_out: wait run_done[slot]; copy every result chunk to the host;
//          record out_done[slot]
//
// so the copies of chunk c+1 in, the kernels of chunk c and the copies of
// chunk c-1 out run at once (the host link carries both directions).  A
// slot is reused only after its previous results left it (out_done, which
// follows that chunk's kernels, which follow its input copies); since slots
// are fixed regions of the staging buffer, this also holds between runs
// whose operations lay a slot out differently.  An event that was never
// recorded satisfies a wait at once, so the first use of a slot waits for
// nothing.
//
// Chunk size: every copy costs a few microseconds of fixed device time, so
// chunks are large, up to 16 MiB of the widest vector (on GB300, 8 inputs
// and 8 outputs of 32-bit words moved 31.5, 35.6 and 37.5 G elements/s
// through chunks of 4, 8 and 16 MiB).
#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "internal.h"

namespace {

constexpr size_t kSlotAlign = 256;
constexpr size_t kMaxChunkBytes = size_t{16} << 20;   // one chunk of the widest vector

struct Input {
  const void* host;
  size_t bytes_per_elem;
  size_t n;
};

struct Plan {
  std::vector<Input> inputs;   // distinct inputs
  std::vector<int> a_idx, b_idx;
  std::vector<size_t> out_bytes;   // element size of each op's output
  size_t chunk = 0;
};

size_t elem_bytes(mont_ctx_t ctx) { return 4u * static_cast<size_t>(ctx->n_limbs); }

bool ranges_overlap(const void* p, size_t bp, const void* q, size_t bq) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p), b = reinterpret_cast<uintptr_t>(q);
  return bp && bq && a < b + bq && b < a + bp;
}

int find_or_add(std::vector<Input>& v, const void* host, size_t eb, size_t n) {
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i].host == host && v[i].bytes_per_elem == eb && v[i].n == n) return static_cast<int>(i);
  v.push_back({host, eb, n});
  return static_cast<int>(v.size()) - 1;
}

}  // namespace

struct mont_pipe {
  int device = 0;
  void* staging = nullptr;
  size_t slot_bytes = 0;
  cudaStream_t s_in = nullptr, s_run = nullptr, s_out = nullptr;
  cudaEvent_t start = nullptr;
  cudaEvent_t tail[3] = {};   // ends of the three streams after a failure part-way
  cudaEvent_t in_done[MONT_PIPE_SLOTS] = {};
  cudaEvent_t run_done[MONT_PIPE_SLOTS] = {};
  cudaEvent_t out_done[MONT_PIPE_SLOTS] = {};
  std::mutex lock;
};

namespace {

void release(mont_pipe* p) {
  for (cudaStream_t s : {p->s_in, p->s_run, p->s_out})
    if (s) cudaStreamSynchronize(s);
  for (int i = 0; i < MONT_PIPE_SLOTS; ++i)
    for (cudaEvent_t e : {p->in_done[i], p->run_done[i], p->out_done[i]})
      if (e) cudaEventDestroy(e);
  if (p->start) cudaEventDestroy(p->start);
  for (cudaEvent_t e : p->tail)
    if (e) cudaEventDestroy(e);
  for (cudaStream_t s : {p->s_in, p->s_run, p->s_out})
    if (s) cudaStreamDestroy(s);
  if (p->staging) cudaFree(p->staging);
  delete p;
}

// Argument checks and the run's layout.  Nothing touches the device.
int make_plan(const mont_pipe* p, const mont_host_op* ops, int count, Plan* plan) {
  if (!p || count < 0 || count > MONT_PIPE_MAX_OPS || (count > 0 && !ops)) return MONT_EINVAL;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev != p->device) return MONT_EINVAL;
  plan->a_idx.assign(count, -1);
  plan->b_idx.assign(count, -1);
  plan->out_bytes.assign(count, 0);
  size_t per_elem = 0, widest = 0;
  for (int i = 0; i < count; ++i) {
    const mont_host_op& o = ops[i];
    if (!o.ctx || o.op < MONT_OP_MUL || o.op > MONT_OP_FROM_DOMAIN) return MONT_EINVAL;
    const size_t e = elem_bytes(o.ctx);
    if (o.n == 0) continue;
    if (!o.a || !o.out || (o.op == MONT_OP_MUL && !o.b)) return MONT_EINVAL;
    const size_t ea = o.op == MONT_OP_REDC ? 2 * e : e;
    if (o.n > SIZE_MAX / ea) return MONT_EINVAL;
    const size_t na = plan->inputs.size();
    plan->a_idx[i] = find_or_add(plan->inputs, o.a, ea, o.n);
    if (plan->inputs.size() > na) per_elem += ea;
    if (o.op == MONT_OP_MUL) {
      const size_t nb = plan->inputs.size();
      plan->b_idx[i] = find_or_add(plan->inputs, o.b, e, o.n);
      if (plan->inputs.size() > nb) per_elem += e;
    }
    plan->out_bytes[i] = e;
    per_elem += e;
    widest = std::max(widest, ea);
  }
  // outputs overlap neither inputs nor each other (host ranges)
  for (int i = 0; i < count; ++i) {
    const mont_host_op& o = ops[i];
    if (o.n == 0) continue;
    const size_t ob = o.n * plan->out_bytes[i];
    for (const Input& in : plan->inputs)
      if (ranges_overlap(o.out, ob, in.host, in.n * in.bytes_per_elem)) return MONT_EINVAL;
    for (int j = i + 1; j < count; ++j)
      if (ops[j].n && ranges_overlap(o.out, ob, ops[j].out, ops[j].n * plan->out_bytes[j]))
        return MONT_EINVAL;
  }
  if (per_elem == 0) {   // every operation empty
    plan->chunk = 0;
    return MONT_OK;
  }
  // one slot holds a chunk of every vector, each region kSlotAlign-aligned
  const size_t nvec = plan->inputs.size() + static_cast<size_t>(count);
  const size_t usable = p->slot_bytes > nvec * kSlotAlign ? p->slot_bytes - nvec * kSlotAlign : 0;
  size_t chunk = usable / per_elem;
  chunk = std::min(chunk, kMaxChunkBytes / widest);
  chunk = chunk / MONT_PIPE_MIN_CHUNK * MONT_PIPE_MIN_CHUNK;
  if (chunk < MONT_PIPE_MIN_CHUNK) return MONT_ENOMEM;
  plan->chunk = chunk;
  return MONT_OK;
}

size_t align_up(size_t x) { return (x + kSlotAlign - 1) / kSlotAlign * kSlotAlign; }


int run_op(const mont_host_op& o, const void* a, const void* b, void* out, size_t n,
           cudaStream_t s) {
  switch (o.op) {
    case MONT_OP_MUL: return mont_mul(o.ctx, a, b, out, n, s);
    case MONT_OP_REDC: return mont_redc(o.ctx, a, out, n, s);
    case MONT_OP_TO_DOMAIN: return mont_to_domain(o.ctx, a, out, n, s);
    default: return mont_from_domain(o.ctx, a, out, n, s);
  }
}

}  // namespace

extern "C" int mont_pipe_create(mont_pipe_t* out, size_t staging_bytes) {
  if (!out || staging_bytes < static_cast<size_t>(MONT_PIPE_SLOTS) * (64u << 10)) return MONT_EINVAL;
  mont_pipe* p = new (std::nothrow) mont_pipe;
  if (!p) return MONT_ENOMEM;
  cudaError_t e = cudaGetDevice(&p->device);
  if (e != cudaSuccess) {
    delete p;
    return montgb::cuda_status(e);
  }
  p->slot_bytes = staging_bytes / MONT_PIPE_SLOTS / kSlotAlign * kSlotAlign;
  e = cudaMalloc(&p->staging, p->slot_bytes * MONT_PIPE_SLOTS);
  if (e != cudaSuccess) {
    p->staging = nullptr;
    cudaGetLastError();
    release(p);
    return MONT_ENOMEM;
  }
  for (cudaStream_t* s : {&p->s_in, &p->s_run, &p->s_out})
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(s, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&p->start, cudaEventDisableTiming);
  for (cudaEvent_t& ev : p->tail)
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
  for (int i = 0; i < MONT_PIPE_SLOTS && e == cudaSuccess; ++i)
    for (cudaEvent_t* ev : {&p->in_done[i], &p->run_done[i], &p->out_done[i]})
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(ev, cudaEventDisableTiming);
  if (e != cudaSuccess) {
    const int st = montgb::cuda_status(e);
    release(p);
    return st;
  }
  *out = p;
  return MONT_OK;
}

extern "C" int mont_pipe_plan(mont_pipe_t pipe, const mont_host_op* ops, int count, size_t* chunk,
                              int* distinct_inputs) {
  Plan plan;
  const int st = make_plan(pipe, ops, count, &plan);
  if (st != MONT_OK) return st;
  if (chunk) *chunk = plan.chunk;
  if (distinct_inputs) *distinct_inputs = static_cast<int>(plan.inputs.size());
  return MONT_OK;
}

extern "C" int mont_pipe_run(mont_pipe_t pipe, const mont_host_op* ops, int count, void* stream) {
  if (!pipe) return MONT_EINVAL;
  std::lock_guard<std::mutex> g(pipe->lock);
  Plan plan;
  int st = make_plan(pipe, ops, count, &plan);
  if (st != MONT_OK || plan.chunk == 0) return st;
  const size_t C = plan.chunk;
  size_t n_max = 0;
  for (int i = 0; i < count; ++i) n_max = std::max(n_max, ops[i].n);
  const size_t n_chunks = (n_max + C - 1) / C;

  // slot layout: distinct inputs, then one output region per operation
  std::vector<size_t> in_off(plan.inputs.size()), out_off(count, 0);
  size_t off = 0;
  for (size_t u = 0; u < plan.inputs.size(); ++u) {
    in_off[u] = off;
    off += align_up(C * plan.inputs[u].bytes_per_elem);
  }
  for (int i = 0; i < count; ++i) {
    out_off[i] = off;
    off += align_up(C * plan.out_bytes[i]);
  }

  cudaStream_t user = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaEventRecord(pipe->start, user);
  for (cudaStream_t s : {pipe->s_in, pipe->s_run, pipe->s_out})
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, pipe->start, 0);
  int last_slot = -1;
  for (size_t c = 0; c < n_chunks && e == cudaSuccess && st == MONT_OK; ++c) {
    const int slot = static_cast<int>(c % MONT_PIPE_SLOTS);
    char* base = static_cast<char*>(pipe->staging) + static_cast<size_t>(slot) * pipe->slot_bytes;
    const size_t lo = c * C;
    // inputs in
    e = cudaStreamWaitEvent(pipe->s_in, pipe->out_done[slot], 0);
    for (size_t u = 0; u < plan.inputs.size() && e == cudaSuccess; ++u) {
      const Input& in = plan.inputs[u];
      if (in.n <= lo) continue;
      const size_t len = std::min(C, in.n - lo);
      e = cudaMemcpyAsync(base + in_off[u], static_cast<const char*>(in.host) + lo * in.bytes_per_elem,
                          len * in.bytes_per_elem, cudaMemcpyHostToDevice, pipe->s_in);
    }
    if (e == cudaSuccess) e = cudaEventRecord(pipe->in_done[slot], pipe->s_in);
    // kernels
    if (e == cudaSuccess) e = cudaStreamWaitEvent(pipe->s_run, pipe->in_done[slot], 0);
    for (int i = 0; i < count && e == cudaSuccess && st == MONT_OK; ++i) {
      const mont_host_op& o = ops[i];
      if (o.n <= lo) continue;
      const size_t len = std::min(C, o.n - lo);
      const void* a = base + in_off[plan.a_idx[i]];
      const void* b = plan.b_idx[i] >= 0 ? base + in_off[plan.b_idx[i]] : nullptr;
      st = run_op(o, a, b, base + out_off[i], len, pipe->s_run);
    }
    if (e == cudaSuccess) e = cudaEventRecord(pipe->run_done[slot], pipe->s_run);
    // results out
    if (e == cudaSuccess) e = cudaStreamWaitEvent(pipe->s_out, pipe->run_done[slot], 0);
    for (int i = 0; i < count && e == cudaSuccess; ++i) {
      const mont_host_op& o = ops[i];
      if (o.n <= lo) continue;
      const size_t len = std::min(C, o.n - lo);
      e = cudaMemcpyAsync(static_cast<char*>(o.out) + lo * plan.out_bytes[i], base + out_off[i],
                          len * plan.out_bytes[i], cudaMemcpyDeviceToHost, pipe->s_out);
    }
    if (e == cudaSuccess) e = cudaEventRecord(pipe->out_done[slot], pipe->s_out);
    if (e == cudaSuccess) last_slot = slot;
  }
  // The caller's stream waits for everything enqueued: on success the last
  // result copy (s_out follows s_run follows s_in, chunk by chunk); after a
  // failure part-way, the current end of each of the three streams.
  cudaError_t e2 = cudaSuccess;
  if (e == cudaSuccess && st == MONT_OK) {
    e2 = cudaStreamWaitEvent(user, pipe->out_done[last_slot], 0);
  } else {
    const cudaStream_t ss[3] = {pipe->s_in, pipe->s_run, pipe->s_out};
    for (int k = 0; k < 3; ++k)
      if (cudaEventRecord(pipe->tail[k], ss[k]) == cudaSuccess && e2 == cudaSuccess)
        e2 = cudaStreamWaitEvent(user, pipe->tail[k], 0);
  }
  if (st != MONT_OK) return st;
  if (e != cudaSuccess) return montgb::cuda_status(e);
  return e2 == cudaSuccess ? MONT_OK : montgb::cuda_status(e2);
}

extern "C" int mont_pipe_destroy(mont_pipe_t pipe) {
  if (!pipe) return MONT_OK;
  release(pipe);
  return MONT_OK;
}
