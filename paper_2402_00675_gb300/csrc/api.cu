// C-ABI entry points of the element-wise operations and the utilities.
#include <cstdint>
#include <map>
#include <mutex>
#include <utility>

#include "internal.h"
#include "tune.h"

namespace montgb {

namespace {
thread_local int g_last_cuda_error = 0;
}

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return MONT_OK;
  g_last_cuda_error = static_cast<int>(e);
  return MONT_ECUDA;
}

int device_sm_count() {
  static std::mutex mu;
  static std::map<int, int> cache;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(dev);
  if (it != cache.end()) return it->second;
  int sms = 0;
  if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    cudaGetLastError();
    sms = 1;
  }
  cache[dev] = sms;
  return sms;
}

int resident_blocks(const void* kernel, int threads) {
  static std::mutex mu;
  static std::map<std::pair<std::pair<const void*, int>, int>, int> cache;
  int dev = 0;
  cudaGetDevice(&dev);
  const auto key = std::make_pair(std::make_pair(kernel, threads), dev);
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(key);
  if (it != cache.end()) return it->second;
  int blocks = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, kernel, threads, 0) != cudaSuccess ||
      blocks < 1) {
    cudaGetLastError();
    blocks = 1;
  }
  cache[key] = blocks;
  return blocks;
}

namespace {

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

// [p, p+bytes) and [q, q+bytes2) overlap without being the same range
bool partial_overlap(const void* p, size_t bp, const void* q, size_t bq) {
  const uintptr_t a = reinterpret_cast<uintptr_t>(p), b = reinterpret_cast<uintptr_t>(q);
  if (a == b && bp == bq) return false;
  return a < b + bq && b < a + bp;
}

int elementwise(mont_ctx_t ctx, Mode mode, const void* x, const void* y, void* out, size_t n,
                void* stream) {
  if (!ctx) return MONT_EINVAL;
  if (n == 0) return MONT_OK;
  if (!x || !out || (mode == Mode::kMul && !y)) return MONT_EINVAL;
  if (ctx->n_limbs > 2) return launch_multilimb_op(ctx, mode, x, y, out, n, stream);
  const size_t esize = 4u * static_cast<size_t>(ctx->n_limbs);
  const size_t in_size = mode == Mode::kRedc ? 2 * esize : esize;
  if (!aligned(x, in_size) || !aligned(out, esize) || (y && !aligned(y, esize)))
    return MONT_EINVAL;
  if (n > (SIZE_MAX / in_size)) return MONT_EINVAL;
  if (partial_overlap(x, n * in_size, out, n * esize)) return MONT_EINVAL;
  if (mode == Mode::kMul && partial_overlap(y, n * esize, out, n * esize)) return MONT_EINVAL;
  if (mode == Mode::kRedc && x == out) return MONT_EINVAL;  // widths differ: no in-place

  LaunchShape shape = tuned_shape(ctx->width, ctx->variant, static_cast<int>(mode));
  // Largest vector width every operand is aligned to.
  const void* ptrs[3] = {x, mode == Mode::kMul ? y : x, out};
  while (shape.vec_bytes > 0) {
    bool ok = true;
    for (const void* p : ptrs) ok = ok && aligned(p, static_cast<size_t>(shape.vec_bytes));
    if (ok) break;
    shape.vec_bytes = shape.vec_bytes == 32 ? 16 : 0;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e = ctx->n_limbs == 1
                      ? launch_word32(ctx->variant, mode, ctx->w32, x, y, out, n, s, shape)
                      : launch_word64(ctx->variant, mode, ctx->w64, x, y, out, n, s, shape);
  return cuda_status(e);
}

}  // namespace
}  // namespace montgb

using montgb::Mode;

extern "C" int mont_mul(mont_ctx_t ctx, const void* a, const void* b, void* out, size_t n,
                        void* stream) {
  return montgb::elementwise(ctx, Mode::kMul, a, b, out, n, stream);
}

extern "C" int mont_redc(mont_ctx_t ctx, const void* T, void* out, size_t n, void* stream) {
  return montgb::elementwise(ctx, Mode::kRedc, T, nullptr, out, n, stream);
}

extern "C" int mont_to_domain(mont_ctx_t ctx, const void* x, void* out, size_t n, void* stream) {
  return montgb::elementwise(ctx, Mode::kToDomain, x, nullptr, out, n, stream);
}

extern "C" int mont_from_domain(mont_ctx_t ctx, const void* y, void* out, size_t n, void* stream) {
  return montgb::elementwise(ctx, Mode::kFromDomain, y, nullptr, out, n, stream);
}

extern "C" const char* mont_strerror(int status) {
  switch (status) {
    case MONT_OK: return "success";
    case MONT_EINVAL: return "invalid argument or unsupported parameters";
    case MONT_ENOMEM: return "out of memory";
    case MONT_ECUDA: return "CUDA runtime error";
    case MONT_ETIMEOUT: return "bounded wait timed out";
    case MONT_EOVERFLOW: return "output buffer too small";
  }
  return "unknown status";
}

extern "C" int mont_last_cuda_error(void) { return montgb::g_last_cuda_error; }

extern "C" int mont_sync(void* stream) {
  return montgb::cuda_status(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
}

extern "C" int mont_version(void) { return 1 * 10000 + 0 * 100 + 0; }
