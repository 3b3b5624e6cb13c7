// Batched Montgomery multiplication over many moduli and uneven lengths.
//
// One persistent launch covers up to kMaxDesc vectors.  Their descriptors
// (operand pointers, length, the modulus's constants, the variant) travel by
// value in the kernel's parameter space (up to 32 KB on sm_90 and later), so
// the call needs no device memory and no upload; each CTA stages the
// descriptors in shared memory once.
//
// Load balance: the vectors are laid end to end in one flat element index
// space of total length L, and CTA c owns the contiguous slice
// [c S, (c + 1) S) with S = ceil(L / grid), rounded to whole 256-bit vectors.
// A slice may span several vectors; the CTA finds the first by binary search
// over the descriptors' flat offsets and walks forward.  Every CTA therefore
// moves the same number of bytes, whatever the length mix.  Inside a slice
// the CTA streams the operands like the element-wise kernel (256-bit loads, U
// vectors in flight per thread), with scalar heads and tails where a slice
// boundary cuts a 256-bit vector.
//
// A batch whose vectors all use one variant runs a kernel specialised for
// it; a mixed batch runs a kernel that switches per vector (uniform across
// the CTA) into out-of-line per-variant bodies.
//
// mont_batch_* wrap the launches of one batch in a CUDA graph built once and
// replayed; new operand pointers for the same shapes update the graph's
// kernel nodes in place.
#include <algorithm>
#include <cstring>
#include <new>
#include <type_traits>
#include <vector>

#include "tune.h"
#include "word_kernel.cuh"

namespace montgb {
namespace {

constexpr int kMaxDesc = 128;

template <class C>
struct BatchDesc {
  const void* a;
  const void* b;
  void* out;
  uint64_t len;
  uint64_t elem0;   // offset of this vector in the flat element space
  C c;              // constants of the modulus
  int32_t variant;
  int32_t vec_ok;   // all three pointers 32-byte aligned
};

template <class C>
struct BatchParams {
  int32_t count;
  int32_t uniform_variant;  // the variant of every vector, or -1 for a mix
  uint64_t total;           // sum of the lengths
  uint64_t per_cta;         // slice length S
  BatchDesc<C> d[kMaxDesc];
};

// Elements [o0, o1) of one vector.
template <class Op, int VB, int U>
__device__ __forceinline__ void segment(const BatchDesc<typename Op::C>& d, uint64_t o0,
                                        uint64_t o1) {
  using E = typename Op::E;
  using TT = typename Op::TT;
  constexpr int EPV = VB / static_cast<int>(sizeof(E));
  uint64_t v_lo = 0, v_hi = 0;  // whole 256-bit vectors [v_lo, v_hi) inside [o0, o1)
  if (d.vec_ok) {
    v_lo = (o0 + EPV - 1) / EPV;
    v_hi = o1 / EPV;
    if (v_hi < v_lo) v_hi = v_lo;
  }
  const uint64_t h_end = v_hi > v_lo ? v_lo * EPV : o1;   // scalar head [o0, h_end)
  for (uint64_t i = o0 + threadIdx.x; i < h_end; i += blockDim.x)
    scalar_element<Op, Mode::kMul>(d.a, d.b, d.out, i, d.c);
  if (v_hi > v_lo) {
    const char* a = static_cast<const char*>(d.a);
    const char* b = static_cast<const char*>(d.b);
    char* o = static_cast<char*>(d.out);
    for (uint64_t base = v_lo; base < v_hi; base += static_cast<uint64_t>(blockDim.x) * U) {
      Vec<VB> va[U], vb[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const uint64_t v = base + threadIdx.x + static_cast<uint64_t>(j) * blockDim.x;
        if (v < v_hi) {
          vld(va[j], a + v * VB);
          vld(vb[j], b + v * VB);
        }
      }
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const uint64_t v = base + threadIdx.x + static_cast<uint64_t>(j) * blockDim.x;
        if (v < v_hi) {
          Vec<VB> vo;
#pragma unroll
          for (int e = 0; e < EPV; ++e)
            vset<E, VB>(vo, e, apply<Op, Mode::kMul>(vget<E, VB>(va[j], e), vget<E, VB>(vb[j], e),
                                                     TT{}, d.c));
          vst(o + v * VB, vo);
        }
      }
    }
    for (uint64_t i = v_hi * EPV + threadIdx.x; i < o1; i += blockDim.x)   // scalar tail
      scalar_element<Op, Mode::kMul>(d.a, d.b, d.out, i, d.c);
  }
}

template <class Op, int VB, int U>
__device__ __noinline__ void segment_outlined(const BatchDesc<typename Op::C>& d, uint64_t o0,
                                              uint64_t o1) {
  segment<Op, VB, U>(d, o0, o1);
}

template <class C, int VB, int U>
__device__ __forceinline__ void segment_mixed(const BatchDesc<C>& d, uint64_t o0, uint64_t o1) {
  if constexpr (sizeof(C) == sizeof(WordConst64)) {
    switch (d.variant) {
      case MONT_REDC: segment_outlined<Redc64, VB, U>(d, o0, o1); break;
      case MONT_SIGNED: segment_outlined<Signed64, VB, U>(d, o0, o1); break;
      case MONT_PLANTARD: segment_outlined<Plantard64, VB, U>(d, o0, o1); break;
      case MONT_SIGNED_PLANTARD: segment_outlined<SignedPlantard64, VB, U>(d, o0, o1); break;
      default: segment_outlined<SignedPlantard2_64, VB, U>(d, o0, o1); break;
    }
  } else {
    switch (d.variant) {
      case MONT_REDC: segment_outlined<Redc32, VB, U>(d, o0, o1); break;
      case MONT_SIGNED: segment_outlined<Signed32, VB, U>(d, o0, o1); break;
      case MONT_PLANTARD: segment_outlined<Plantard32, VB, U>(d, o0, o1); break;
      case MONT_SIGNED_PLANTARD: segment_outlined<SignedPlantard32, VB, U>(d, o0, o1); break;
      default: segment_outlined<SignedPlantard2_32, VB, U>(d, o0, o1); break;
    }
  }
}

// Op = void: mixed variants.
template <class C, class Op, int VB, int U>
__global__ void __launch_bounds__(256, (U >= 4 ? 2 : 4)) batched_kernel(const __grid_constant__ BatchParams<C> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto* sd = reinterpret_cast<BatchDesc<C>*>(smem);
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(p.d);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sd);
    const int words = p.count * static_cast<int>(sizeof(BatchDesc<C>) / 4);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  const uint64_t g0 = static_cast<uint64_t>(blockIdx.x) * p.per_cta;
  if (g0 >= p.total) return;
  const uint64_t g1 = g0 + p.per_cta < p.total ? g0 + p.per_cta : p.total;
  int lo = 0, hi = p.count - 1;   // last vector with elem0 <= g0
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (sd[mid].elem0 <= g0) lo = mid; else hi = mid - 1;
  }
  for (int j = lo; j < p.count && sd[j].elem0 < g1; ++j) {
    const BatchDesc<C>& d = sd[j];
    const uint64_t s0 = g0 > d.elem0 ? g0 : d.elem0;
    const uint64_t e = d.elem0 + d.len;
    const uint64_t s1 = g1 < e ? g1 : e;
    if (s1 <= s0) continue;
    if constexpr (std::is_void_v<Op>) {
      segment_mixed<C, VB, U>(d, s0 - d.elem0, s1 - d.elem0);
    } else {
      segment<Op, VB, U>(d, s0 - d.elem0, s1 - d.elem0);
    }
  }
}

static_assert(sizeof(BatchParams<WordConst64>) <= 32000, "descriptors exceed parameter space");

// One group of at most kMaxDesc vectors, ready to launch.
struct Group {
  int width = 0;
  BatchParams<WordConst32> p32;
  BatchParams<WordConst64> p64;
  unsigned grid = 0;
  int threads = 256;
  size_t smem = 0;
  const void* kernel = nullptr;
  uint64_t total() const { return width == 32 ? p32.total : p64.total; }
  void* params() { return width == 32 ? static_cast<void*>(&p32) : static_cast<void*>(&p64); }
};

template <class C, class Op>
const void* kernel_u(int unroll) {
  switch (unroll) {
    case 1: return reinterpret_cast<const void*>(batched_kernel<C, Op, 32, 1>);
    case 4: return reinterpret_cast<const void*>(batched_kernel<C, Op, 32, 4>);
    default: return reinterpret_cast<const void*>(batched_kernel<C, Op, 32, 2>);
  }
}

template <class C>
const void* kernel_for(int variant, int unroll) {
  constexpr bool w64 = sizeof(C) == sizeof(WordConst64);
  using R = std::conditional_t<w64, Redc64, Redc32>;
  using S = std::conditional_t<w64, Signed64, Signed32>;
  using P = std::conditional_t<w64, Plantard64, Plantard32>;
  using S1 = std::conditional_t<w64, SignedPlantard64, SignedPlantard32>;
  using S2 = std::conditional_t<w64, SignedPlantard2_64, SignedPlantard2_32>;
  switch (variant) {
    case MONT_REDC: return kernel_u<C, R>(unroll);
    case MONT_SIGNED: return kernel_u<C, S>(unroll);
    case MONT_PLANTARD: return kernel_u<C, P>(unroll);
    case MONT_SIGNED_PLANTARD: return kernel_u<C, S1>(unroll);
    case MONT_SIGNED_PLANTARD2: return kernel_u<C, S2>(unroll);
    default: return kernel_u<C, void>(unroll);
  }
}

template <class C>
void fill(BatchParams<C>& p, const C& c, int variant, const void* a, const void* b, void* o,
          uint64_t len, int slot) {
  BatchDesc<C>& d = p.d[slot];
  d.a = a;
  d.b = b;
  d.out = o;
  d.len = len;
  d.c = c;
  d.variant = variant;
  const auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 31u) == 0; };
  d.vec_ok = al(a) && al(b) && al(o) ? 1 : 0;
}

// Flat offsets, the common variant and the slice length for `grid` CTAs.
template <class C>
void finish(BatchParams<C>& p, int count) {
  p.count = count;
  uint64_t t = 0;
  int uv = -2;
  for (int i = 0; i < count; ++i) {
    p.d[i].elem0 = t;
    t += p.d[i].len;
    if (p.d[i].len == 0) continue;
    uv = (uv == -2 || uv == p.d[i].variant) ? p.d[i].variant : -1;
  }
  p.total = t;
  p.uniform_variant = uv < 0 ? -1 : uv;
}

template <class C>
void slice(BatchParams<C>& p, unsigned grid, uint64_t quantum) {
  uint64_t s = (p.total + grid - 1) / grid;
  s = (s + quantum - 1) / quantum * quantum;
  p.per_cta = s > 0 ? s : quantum;
}

// Validate the batch and cut it into launch groups.
int plan_groups(const mont_ctx_t* ctxs, const void* const* a, const void* const* b,
                void* const* out, const size_t* lens, int count, std::vector<Group>* groups) {
  if (count < 0 || (count > 0 && (!ctxs || !a || !b || !out || !lens))) return MONT_EINVAL;
  if (count == 0) return MONT_OK;
  const int width = ctxs[0] ? ctxs[0]->width : 0;
  if (width != 32 && width != 64) return MONT_EINVAL;
  const size_t esize = width / 8;
  for (int i = 0; i < count; ++i) {
    if (!ctxs[i] || ctxs[i]->width != width) return MONT_EINVAL;
    if (lens[i] == 0) continue;
    if (!a[i] || !b[i] || !out[i]) return MONT_EINVAL;
    for (const void* q : {a[i], b[i], static_cast<const void*>(out[i])})
      if (reinterpret_cast<uintptr_t>(q) % esize) return MONT_EINVAL;
  }
  const LaunchShape shape = tuned_batched_shape(width);
  // slices are whole multiples of one CTA iteration when possible
  const uint64_t epv = 32 / esize;
  for (int start = 0; start < count; start += kMaxDesc) {
    const int n = std::min(kMaxDesc, count - start);
    Group g;
    g.width = width;
    g.threads = shape.threads;
    for (int i = 0; i < n; ++i) {
      const int k = start + i;
      if (width == 32)
        fill(g.p32, ctxs[k]->w32, ctxs[k]->variant, a[k], b[k], out[k], lens[k], i);
      else
        fill(g.p64, ctxs[k]->w64, ctxs[k]->variant, a[k], b[k], out[k], lens[k], i);
    }
    int uv;
    if (width == 32) {
      finish(g.p32, n);
      uv = g.p32.uniform_variant;
      g.smem = n * sizeof(BatchDesc<WordConst32>);
      g.kernel = kernel_for<WordConst32>(uv, shape.unroll);
    } else {
      finish(g.p64, n);
      uv = g.p64.uniform_variant;
      g.smem = n * sizeof(BatchDesc<WordConst64>);
      g.kernel = kernel_for<WordConst64>(uv, shape.unroll);
    }
    if (g.total() == 0) continue;
    const int per_sm = shape.blocks_per_sm > 0 ? shape.blocks_per_sm
                                               : resident_blocks(g.kernel, g.threads);
    const uint64_t cap = static_cast<uint64_t>(device_sm_count()) * per_sm;
    // at least one CTA iteration of work per CTA
    const uint64_t min_slice = static_cast<uint64_t>(g.threads) * shape.unroll * epv;
    const uint64_t want = (g.total() + min_slice - 1) / min_slice;
    g.grid = static_cast<unsigned>(std::max<uint64_t>(1, std::min<uint64_t>(cap, want)));
    if (width == 32) slice(g.p32, g.grid, epv); else slice(g.p64, g.grid, epv);
    groups->push_back(g);
  }
  return MONT_OK;
}

cudaError_t launch_group(Group& g, cudaStream_t s) {
  void* args[] = {g.params()};
  return cudaLaunchKernel(g.kernel, dim3(g.grid), dim3(g.threads), args, g.smem, s);
}

}  // namespace
}  // namespace montgb

using namespace montgb;

struct mont_batch {
  std::vector<Group> groups;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<cudaGraphNode_t> nodes;
  int count = 0;
  int device = 0;
  std::vector<size_t> lens;
  std::vector<int> widths;
};

extern "C" int mont_mul_batched(const mont_ctx_t* ctxs, const void* const* a,
                                const void* const* b, void* const* out, const size_t* lens,
                                int count, void* stream) {
  std::vector<Group> groups;
  const int st = plan_groups(ctxs, a, b, out, lens, count, &groups);
  if (st != MONT_OK) return st;
  for (auto& g : groups) {
    const cudaError_t e = launch_group(g, static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_status(e);
  }
  return MONT_OK;
}

namespace {
int build_graph(mont_batch* bt) {
  cudaError_t e = cudaGraphCreate(&bt->graph, 0);
  if (e != cudaSuccess) return cuda_status(e);
  cudaGraphNode_t prev = nullptr;
  for (auto& g : bt->groups) {
    cudaKernelNodeParams kp{};
    void* args[] = {g.params()};
    kp.func = const_cast<void*>(g.kernel);
    kp.gridDim = dim3(g.grid);
    kp.blockDim = dim3(g.threads);
    kp.sharedMemBytes = static_cast<unsigned>(g.smem);
    kp.kernelParams = args;
    cudaGraphNode_t node;
    e = cudaGraphAddKernelNode(&node, bt->graph, prev ? &prev : nullptr, prev ? 1 : 0, &kp);
    if (e != cudaSuccess) return cuda_status(e);
    bt->nodes.push_back(node);
    prev = node;
  }
  e = cudaGraphInstantiate(&bt->exec, bt->graph, 0);
  return cuda_status(e);
}
}  // namespace

extern "C" int mont_batch_create(mont_batch_t* out_batch, const mont_ctx_t* ctxs,
                                 const void* const* a, const void* const* b, void* const* out,
                                 const size_t* lens, int count) {
  if (!out_batch) return MONT_EINVAL;
  mont_batch* bt = new (std::nothrow) mont_batch;
  if (!bt) return MONT_ENOMEM;
  int st = plan_groups(ctxs, a, b, out, lens, count, &bt->groups);
  if (st == MONT_OK) {
    bt->count = count;
    bt->lens.assign(lens, lens + count);
    cudaGetDevice(&bt->device);
    st = build_graph(bt);
  }
  if (st != MONT_OK) {
    mont_batch_destroy(bt);
    return st;
  }
  *out_batch = bt;
  return MONT_OK;
}

extern "C" int mont_batch_launch(mont_batch_t batch, void* stream) {
  if (!batch || !batch->exec) return MONT_EINVAL;
  return cuda_status(cudaGraphLaunch(batch->exec, static_cast<cudaStream_t>(stream)));
}

extern "C" int mont_batch_update(mont_batch_t batch, const void* const* a, const void* const* b,
                                 void* const* out) {
  if (!batch || !batch->exec || !a || !b || !out) return MONT_EINVAL;
  size_t gi = 0;
  int k = 0;
  // Walk the groups in the order plan_groups made them (groups whose vectors
  // are all empty were dropped; their vectors keep length 0).
  for (int start = 0; start < batch->count; start += kMaxDesc) {
    const int n = std::min(kMaxDesc, batch->count - start);
    bool any = false;
    for (int i = 0; i < n; ++i) any = any || batch->lens[start + i] > 0;
    if (!any) continue;
    Group& g = batch->groups[gi++];
    for (int i = 0; i < n; ++i) {
      k = start + i;
      if (batch->lens[k] == 0) continue;
      if (!a[k] || !b[k] || !out[k]) return MONT_EINVAL;
      const size_t esize = g.width / 8;
      for (const void* q : {a[k], b[k], static_cast<const void*>(out[k])})
        if (reinterpret_cast<uintptr_t>(q) % esize) return MONT_EINVAL;
      auto upd = [&](auto& p) {
        auto& d = p.d[i];
        d.a = a[k];
        d.b = b[k];
        d.out = out[k];
        const auto al = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) & 31u) == 0; };
        d.vec_ok = al(a[k]) && al(b[k]) && al(out[k]) ? 1 : 0;
      };
      if (g.width == 32) upd(g.p32); else upd(g.p64);
    }
    cudaKernelNodeParams kp{};
    void* args[] = {g.params()};
    kp.func = const_cast<void*>(g.kernel);
    kp.gridDim = dim3(g.grid);
    kp.blockDim = dim3(g.threads);
    kp.sharedMemBytes = static_cast<unsigned>(g.smem);
    kp.kernelParams = args;
    const cudaError_t e = cudaGraphExecKernelNodeSetParams(batch->exec, batch->nodes[gi - 1], &kp);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return MONT_OK;
}

extern "C" int mont_batch_destroy(mont_batch_t batch) {
  if (!batch) return MONT_OK;
  if (batch->exec) cudaGraphExecDestroy(batch->exec);
  if (batch->graph) cudaGraphDestroy(batch->graph);
  delete batch;
  return MONT_OK;
}
