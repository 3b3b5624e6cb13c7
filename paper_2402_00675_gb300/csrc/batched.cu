// Batched Montgomery multiplication over many moduli and uneven lengths.
//
// One persistent launch covers up to kMaxDesc vectors.  Their descriptors
// (operand pointers, length, the modulus's constants, the variant) travel by
// value in the kernel's parameter space (up to 32 KB on sm_90 and later), so
// the call needs no device memory and no upload; each CTA stages the
// descriptors in shared memory once and then walks "tiles" round-robin: tile
// t is `tile_elems` consecutive elements of one vector, found by a binary
// search over the descriptors' first-tile indices.  Inside a tile the CTA
// streams the operands exactly like the element-wise kernel (256-bit loads,
// U vectors in flight per thread) and applies that vector's variant; the
// variant switch is uniform across the CTA.
//
// mont_batch_* wrap the launches of one batch in a CUDA graph built once and
// replayed; new operand pointers for the same shapes update the graph's
// kernel nodes in place.
#include <algorithm>
#include <cstring>
#include <new>
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
  uint64_t tile0;   // index of this vector's first tile
  C c;              // constants of the modulus
  int32_t variant;
  int32_t vec_ok;   // all three pointers 32-byte aligned
};

template <class C>
struct BatchParams {
  int32_t count;
  uint32_t tile_elems;
  uint64_t total_tiles;
  BatchDesc<C> d[kMaxDesc];
};

// Elements [off, off + cnt) of one vector; off is a multiple of the tile size.
template <class Op, int VB, int U>
__device__ __forceinline__ void tile_body(const BatchDesc<typename Op::C>& d, uint64_t off,
                                          uint64_t cnt) {
  using E = typename Op::E;
  using TT = typename Op::TT;
  constexpr int EPV = VB / static_cast<int>(sizeof(E));
  uint64_t done = 0;
  if (d.vec_ok) {
    const char* a = static_cast<const char*>(d.a) + off * sizeof(E);
    const char* b = static_cast<const char*>(d.b) + off * sizeof(E);
    char* o = static_cast<char*>(d.out) + off * sizeof(E);
    const uint64_t nv = cnt / EPV;
    for (uint64_t base = 0; base < nv; base += static_cast<uint64_t>(blockDim.x) * U) {
      Vec<VB> va[U], vb[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const uint64_t v = base + threadIdx.x + static_cast<uint64_t>(j) * blockDim.x;
        if (v < nv) {
          vld(va[j], a + v * VB);
          vld(vb[j], b + v * VB);
        }
      }
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const uint64_t v = base + threadIdx.x + static_cast<uint64_t>(j) * blockDim.x;
        if (v < nv) {
          Vec<VB> vo;
#pragma unroll
          for (int e = 0; e < EPV; ++e)
            vset<E, VB>(vo, e, apply<Op, Mode::kMul>(vget<E, VB>(va[j], e), vget<E, VB>(vb[j], e),
                                                     TT{}, d.c));
          vst(o + v * VB, vo);
        }
      }
    }
    done = nv * EPV;
  }
  for (uint64_t i = done + threadIdx.x; i < cnt; i += blockDim.x)
    scalar_element<Op, Mode::kMul>(d.a, d.b, d.out, off + i, d.c);
}

template <class C, int VB, int U>
__global__ void __launch_bounds__(512) batched_kernel(const __grid_constant__ BatchParams<C> p) {
  extern __shared__ __align__(16) unsigned char smem[];
  auto* sd = reinterpret_cast<BatchDesc<C>*>(smem);
  {
    const uint32_t* src = reinterpret_cast<const uint32_t*>(p.d);
    uint32_t* dst = reinterpret_cast<uint32_t*>(sd);
    const int words = p.count * static_cast<int>(sizeof(BatchDesc<C>) / 4);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
  }
  __syncthreads();
  for (uint64_t tile = blockIdx.x; tile < p.total_tiles; tile += gridDim.x) {
    int lo = 0, hi = p.count - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (sd[mid].tile0 <= tile) lo = mid; else hi = mid - 1;
    }
    const BatchDesc<C>& d = sd[lo];
    const uint64_t off = (tile - d.tile0) * p.tile_elems;
    const uint64_t rest = d.len - off;
    const uint64_t cnt = rest < p.tile_elems ? rest : p.tile_elems;
    if constexpr (sizeof(C) == sizeof(WordConst64)) {
      switch (d.variant) {
        case MONT_REDC: tile_body<Redc64, VB, U>(d, off, cnt); break;
        case MONT_SIGNED: tile_body<Signed64, VB, U>(d, off, cnt); break;
        case MONT_PLANTARD: tile_body<Plantard64, VB, U>(d, off, cnt); break;
        case MONT_SIGNED_PLANTARD: tile_body<SignedPlantard64, VB, U>(d, off, cnt); break;
        default: tile_body<SignedPlantard2_64, VB, U>(d, off, cnt); break;
      }
    } else {
      switch (d.variant) {
        case MONT_REDC: tile_body<Redc32, VB, U>(d, off, cnt); break;
        case MONT_SIGNED: tile_body<Signed32, VB, U>(d, off, cnt); break;
        case MONT_PLANTARD: tile_body<Plantard32, VB, U>(d, off, cnt); break;
        case MONT_SIGNED_PLANTARD: tile_body<SignedPlantard32, VB, U>(d, off, cnt); break;
        default: tile_body<SignedPlantard2_32, VB, U>(d, off, cnt); break;
      }
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
  uint64_t tiles() const { return width == 32 ? p32.total_tiles : p64.total_tiles; }
  void* params() { return width == 32 ? static_cast<void*>(&p32) : static_cast<void*>(&p64); }
};

template <class C>
const void* kernel_for(int unroll) {
  switch (unroll) {
    case 1: return reinterpret_cast<const void*>(batched_kernel<C, 32, 1>);
    case 4: return reinterpret_cast<const void*>(batched_kernel<C, 32, 4>);
    default: return reinterpret_cast<const void*>(batched_kernel<C, 32, 2>);
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

template <class C>
void finish(BatchParams<C>& p, int count, uint32_t tile_elems) {
  p.count = count;
  p.tile_elems = tile_elems;
  uint64_t t = 0;
  for (int i = 0; i < count; ++i) {
    p.d[i].tile0 = t;
    t += (p.d[i].len + tile_elems - 1) / tile_elems;
  }
  p.total_tiles = t;
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
  // one tile = tile_iters CTA iterations of `unroll` 256-bit vectors per thread
  const uint32_t tile_elems = static_cast<uint32_t>(shape.threads) * shape.unroll *
                              static_cast<uint32_t>(32 / esize) *
                              static_cast<uint32_t>(shape.tile_iters > 0 ? shape.tile_iters : 1);
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
    if (width == 32) {
      finish(g.p32, n, tile_elems);
      g.smem = n * sizeof(BatchDesc<WordConst32>);
      g.kernel = kernel_for<WordConst32>(shape.unroll);
    } else {
      finish(g.p64, n, tile_elems);
      g.smem = n * sizeof(BatchDesc<WordConst64>);
      g.kernel = kernel_for<WordConst64>(shape.unroll);
    }
    if (g.tiles() == 0) continue;
    const int per_sm = resident_blocks(g.kernel, g.threads);
    const uint64_t cap = static_cast<uint64_t>(device_sm_count()) * per_sm;
    g.grid = static_cast<unsigned>(std::min<uint64_t>(cap, g.tiles()));
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
