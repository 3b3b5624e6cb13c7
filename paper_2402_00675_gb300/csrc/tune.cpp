// Launch-shape table and the autotuner.
//
// The element-wise word kernels, the batched kernel and the multi-limb
// kernels each have a few launch knobs (block size, vectors in flight per
// thread, vector width, lanes per element).  The table maps (device, word
// width, variant, mode) to a shape; missing entries use the built-in
// defaults.  mont_autotune fills the table by timing every candidate shape
// on scratch buffers with CUDA events and keeping the fastest;
// mont_tune_save / mont_tune_load persist it as a small text file keyed by
// device name and SM count, so a tuned process can hand its choices to the
// next one.
#include "tune.h"

#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

namespace montgb {

namespace {
std::mutex g_mu;
std::map<std::tuple<int, int, int, int>, LaunchShape> g_table;  // (device, width, variant, mode)

int current_device() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return dev;
}
}  // namespace

LaunchShape tuned_shape(int width, int variant, int mode) {
  const auto key = std::make_tuple(current_device(), width, variant, mode);
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(key);
  if (it != g_table.end()) return it->second;
  LaunchShape d{};
  // multi-limb Algorithms 1-4 (one thread per element): 128-thread blocks at
  // the occupancy limit measured best (1024 bits: 0.39 against 0.36 Gmodmul/s)
  if (width > 64 && variant != MONT_REDC) d.threads = 128;
  // multi-limb REDC and Algorithm 1 (both on the CIOS schedule): 0 = the block
  // size follows the limb count (cios.cu)
  if (width > 64 && (variant == MONT_REDC || variant == MONT_SIGNED)) d.threads = 0;
  return d;
}

void set_tuned_shape(int width, int variant, int mode, const LaunchShape& shape) {
  const auto key = std::make_tuple(current_device(), width, variant, mode);
  std::lock_guard<std::mutex> lock(g_mu);
  g_table[key] = shape;
}

static void erase_tuned_shape(int width, int variant, int mode) {
  const auto key = std::make_tuple(current_device(), width, variant, mode);
  std::lock_guard<std::mutex> lock(g_mu);
  g_table.erase(key);
}

LaunchShape tuned_batched_shape(int width) {
  // default when untuned: 256 threads, one 256-bit vector in flight per
  // operand (measured fastest for the 32-prime RNS batch on GB300)
  const auto key = std::make_tuple(current_device(), width, -1, -1);
  std::lock_guard<std::mutex> lock(g_mu);
  auto it = g_table.find(key);
  if (it != g_table.end()) return it->second;
  LaunchShape s;
  s.unroll = 1;
  return s;
}

void set_tuned_batched_shape(int width, const LaunchShape& shape) {
  set_tuned_shape(width, -1, -1, shape);
}

namespace {

LaunchShape from_public(const mont_launch_shape& p) {
  LaunchShape s;
  if (p.threads > 0) s.threads = p.threads;
  if (p.unroll > 0) s.unroll = p.unroll;
  s.vec_bytes = p.vec_bytes;
  s.blocks_per_sm = p.blocks_per_sm;
  if (p.tile_iters > 0) s.tile_iters = p.tile_iters;
  s.team = p.team;
  return s;
}

mont_launch_shape to_public(const LaunchShape& s) {
  mont_launch_shape p{};
  p.threads = s.threads;
  p.unroll = s.unroll;
  p.vec_bytes = s.vec_bytes;
  p.blocks_per_sm = s.blocks_per_sm;
  p.tile_iters = s.tile_iters;
  p.team = s.team;
  return p;
}

bool shape_valid(int width, int mode, const LaunchShape& s) {
  if (mode == MONT_TUNE_MODE_BATCHED) {
    return (s.threads == 128 || s.threads == 256) && (s.unroll == 1 || s.unroll == 2 || s.unroll == 4);
  }
  if (width > 64) {
    return (s.threads == 32 || s.threads == 64 || s.threads == 128 || s.threads == 256) &&
           s.blocks_per_sm >= 0;
  }
  return (s.threads == 64 || s.threads == 128 || s.threads == 256 || s.threads == 512) &&
         (s.unroll == 1 || s.unroll == 2 || s.unroll == 4) &&
         (s.vec_bytes == 0 || s.vec_bytes == 16 || s.vec_bytes == 32) && s.blocks_per_sm >= 0;
}

// Average milliseconds of `reps` calls of fn on stream s (after one warm-up call).
template <class F>
int time_ms(F fn, cudaStream_t s, int reps, float* ms) {
  if (int st = fn(); st != MONT_OK) return st;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return cuda_status(cudaGetLastError());
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_status(cudaGetLastError());
  }
  int st = MONT_OK;
  cudaEventRecord(e0, s);
  for (int r = 0; r < reps && st == MONT_OK; ++r) st = fn();
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  if (st == MONT_OK && e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != MONT_OK) return st;
  if (e != cudaSuccess) return cuda_status(e);
  *ms /= reps;
  return MONT_OK;
}

}  // namespace
}  // namespace montgb

using namespace montgb;

extern "C" int mont_tune_set(int width_bits, int variant, int mode, const mont_launch_shape* shape) {
  if (mode < MONT_TUNE_MODE_BATCHED || mode > 3) return MONT_EINVAL;
  const int v = mode == MONT_TUNE_MODE_BATCHED ? -1 : variant;
  if (!shape) {
    erase_tuned_shape(width_bits, v, mode);
    return MONT_OK;
  }
  const LaunchShape s = from_public(*shape);
  if (!shape_valid(width_bits, mode, s)) return MONT_EINVAL;
  set_tuned_shape(width_bits, v, mode, s);
  return MONT_OK;
}

extern "C" int mont_tune_get(int width_bits, int variant, int mode, mont_launch_shape* shape) {
  if (!shape || mode < MONT_TUNE_MODE_BATCHED || mode > 3) return MONT_EINVAL;
  *shape = to_public(mode == MONT_TUNE_MODE_BATCHED ? tuned_batched_shape(width_bits)
                                                    : tuned_shape(width_bits, variant, mode));
  return MONT_OK;
}

extern "C" int mont_autotune(mont_ctx_t ctx, size_t n, int flags, void* stream) {
  if (!ctx || n == 0) return MONT_EINVAL;
  if (flags == 0) flags = MONT_TUNE_ELEMENTWISE;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t esize = 4u * static_cast<size_t>(ctx->n_limbs);
  const size_t bytes = 3 * n * esize + 256;
  void* buf = nullptr;
  cudaError_t e = cudaMallocAsync(&buf, bytes, s);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MONT_ENOMEM : cuda_status(e);
  }
  // Operand values do not change the kernels' timing (no data-dependent
  // branches beyond selects); any bit pattern is a valid input to time.
  e = cudaMemsetAsync(buf, 0x11, bytes, s);
  char* base = static_cast<char*>(buf);
  void* a = base;
  void* b = base + n * esize;
  void* o = base + 2 * n * esize;
  int st = e == cudaSuccess ? MONT_OK : cuda_status(e);
  const int reps = 5;

  if (st == MONT_OK && (flags & MONT_TUNE_ELEMENTWISE)) {
    std::vector<LaunchShape> cands;
    if (ctx->n_limbs <= 2) {
      for (int th : {128, 256, 512})
        for (int u : {1, 2, 4})
          for (int vb : {32, 16}) {
            LaunchShape c;
            c.threads = th; c.unroll = u; c.vec_bytes = vb;
            cands.push_back(c);
          }
    } else if (ctx->variant != MONT_REDC && ctx->variant != MONT_SIGNED) {
      // Algorithms 2-4 at multi-limb widths: one thread per element, so the
      // block size is the only choice; small blocks spread a launch of a few
      // warps per SM evenly over the SMs
      for (int th : {32, 64, 128, 256}) {
        LaunchShape c;
        c.threads = th;
        cands.push_back(c);
      }
    } else {
      // lanes per element, block size, and how many blocks per SM the grid
      // fills: a launch of one to three waves of elements can run faster on
      // fewer resident warps than the occupancy maximum (2048 bits, 2^15
      // elements: 57.5 us at three 128-thread blocks per SM, 62.3 us at five)
      for (int team : {1, 2, 4, 8, 16}) {
        if (!multilimb_team_supported(ctx->n_limbs, team)) continue;
        for (int th : {64, 128, 256})
          for (int bps : {0, 2, 3, 4}) {
            LaunchShape c;
            c.threads = th; c.team = team; c.blocks_per_sm = bps;
            cands.push_back(c);
          }
      }
    }
    float best = 1e30f;
    LaunchShape best_shape;
    bool found = false;
    for (const auto& c : cands) {
      for (int mode = 0; mode < 4; ++mode) set_tuned_shape(ctx->width, ctx->variant, mode, c);
      float ms = 0;
      const int r = time_ms([&] { return mont_mul(ctx, a, b, o, n, stream); }, s, reps, &ms);
      if (r != MONT_OK) {
        cudaGetLastError();
        continue;
      }
      if (ms < best) {
        best = ms;
        best_shape = c;
        found = true;
      }
    }
    for (int mode = 0; mode < 4; ++mode) {
      if (found) set_tuned_shape(ctx->width, ctx->variant, mode, best_shape);
      else erase_tuned_shape(ctx->width, ctx->variant, mode);
    }
  }

  if (st == MONT_OK && (flags & MONT_TUNE_BATCHED) && ctx->n_limbs <= 2) {
    // a synthetic batch of 32 vectors of uneven lengths covering the scratch
    const int count = 32;
    std::vector<mont_ctx_t> cs(count, ctx);
    std::vector<const void*> pa(count), pb(count);
    std::vector<void*> po(count);
    std::vector<size_t> lens(count);
    size_t off = 0;
    uint32_t lcg = 12345u;
    std::vector<double> w(count);
    double wsum = 0;
    for (int i = 0; i < count; ++i) {
      lcg = lcg * 1664525u + 1013904223u;
      w[i] = 1.0 + static_cast<double>(lcg >> 8) / (1u << 24) * 15.0;
      wsum += w[i];
    }
    for (int i = 0; i < count; ++i) {
      lens[i] = static_cast<size_t>(static_cast<double>(n) * w[i] / wsum);
      if (off + lens[i] > n) lens[i] = n - off;
      pa[i] = static_cast<const char*>(a) + off * esize;
      pb[i] = static_cast<const char*>(b) + off * esize;
      po[i] = static_cast<char*>(o) + off * esize;
      off += lens[i];
    }
    float best = 1e30f;
    LaunchShape best_shape;
    bool found = false;
    for (int th : {128, 256})
      for (int u : {1, 2, 4}) {
        LaunchShape c;
        c.threads = th; c.unroll = u;
        set_tuned_batched_shape(ctx->width, c);
        float ms = 0;
        const int r = time_ms([&] {
          return mont_mul_batched(cs.data(), pa.data(), pb.data(), po.data(), lens.data(), count,
                                  stream);
        }, s, reps, &ms);
        if (r != MONT_OK) {
          cudaGetLastError();
          continue;
        }
        if (ms < best) {
          best = ms;
          best_shape = c;
          found = true;
        }
      }
    if (found) set_tuned_batched_shape(ctx->width, best_shape);
    else erase_tuned_shape(ctx->width, -1, -1);
  }

  cudaError_t fe = cudaFreeAsync(buf, s);
  cudaError_t se = cudaStreamSynchronize(s);
  if (st == MONT_OK && fe != cudaSuccess) st = cuda_status(fe);
  if (st == MONT_OK && se != cudaSuccess) st = cuda_status(se);
  return st;
}

namespace {
bool device_key(std::string* name, int* sms) {
  int dev = 0;
  cudaDeviceProp prop;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  *name = prop.name;
  for (auto& ch : *name)
    if (ch == ' ') ch = '_';
  *sms = prop.multiProcessorCount;
  return true;
}
}  // namespace

extern "C" int mont_tune_save(const char* path) {
  if (!path) return MONT_EINVAL;
  std::string name;
  int sms = 0;
  if (!device_key(&name, &sms)) return MONT_ECUDA;
  const int dev = current_device();
  FILE* f = std::fopen(path, "w");
  if (!f) return MONT_EINVAL;
  std::fprintf(f, "montgb-tune 1\n");
  {
    std::lock_guard<std::mutex> lock(g_mu);
    for (const auto& kv : g_table) {
      if (std::get<0>(kv.first) != dev) continue;
      const LaunchShape& s = kv.second;
      std::fprintf(f, "%s %d %d %d %d %d %d %d %d %d %d\n", name.c_str(), sms,
                   std::get<1>(kv.first), std::get<2>(kv.first), std::get<3>(kv.first), s.threads,
                   s.unroll, s.vec_bytes, s.blocks_per_sm, s.tile_iters, s.team);
    }
  }
  std::fclose(f);
  return MONT_OK;
}

extern "C" int mont_tune_load(const char* path) {
  if (!path) return MONT_EINVAL;
  std::string name;
  int sms = 0;
  if (!device_key(&name, &sms)) return MONT_ECUDA;
  FILE* f = std::fopen(path, "r");
  if (!f) return MONT_EINVAL;
  char header[64] = {0};
  int version = 0;
  if (std::fscanf(f, "%63s %d", header, &version) != 2 || std::strcmp(header, "montgb-tune") ||
      version != 1) {
    std::fclose(f);
    return MONT_EINVAL;
  }
  char dname[256];
  int dsms, width, variant, mode;
  LaunchShape s;
  while (std::fscanf(f, "%255s %d %d %d %d %d %d %d %d %d %d", dname, &dsms, &width, &variant,
                     &mode, &s.threads, &s.unroll, &s.vec_bytes, &s.blocks_per_sm, &s.tile_iters,
                     &s.team) == 11) {
    if (name == dname && dsms == sms) set_tuned_shape(width, variant, mode, s);
  }
  std::fclose(f);
  return MONT_OK;
}
