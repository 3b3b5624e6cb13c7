// Integer-pipe throughput probe (mont_probe_int_rate).
//
// The multi-limb kernels and the verify sweep are bound by integer
// instruction throughput, not by memory.  This probe measures the rate the
// GPU sustains for the instruction mixes they use, with many independent
// chains per thread so that latency is hidden:
//   kind 0  mad.lo.u32                      (IMAD)
//   kind 1  mad.hi.u32                      (IMAD.HI)
//   kind 2  mad.lo.cc / madc.hi.cc pairs    (the carry chains of a CIOS row)
//   kind 3  add.u32                         (plain ALU)
//   kind 4  mad.wide.u32                    (IMAD.WIDE, a full 32x32->64 product + 64-bit addend)
//   kind 5  mad.lo.u32 and mad.hi.u32 on independent accumulators (the
//           low and high halves of different limb products, as product
//           scanning issues them)
// Each thread runs 8 independent accumulators for `iters` iterations; the
// rate is instructions per second over the whole grid, timed with CUDA events
// on the caller's stream.  Results go to a file-scope device sink so the work
// cannot be optimised away.
#include "internal.h"

namespace montgb {
namespace {

__device__ uint32_t g_probe_sink;

template <int KIND>
__global__ void __launch_bounds__(256) int_rate_kernel(uint32_t seed, int iters) {
  uint32_t x[8], y[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    x[j] = seed + threadIdx.x * 8 + j;
    y[j] = x[j] ^ 0x5bd1e995u;
  }
  const uint32_t m = seed | 1u, c = seed ^ 0x9E3779B9u;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      if constexpr (KIND == 0) {
        asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[j]) : "r"(m), "r"(c));
      } else if constexpr (KIND == 1) {
        asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(x[j]) : "r"(m), "r"(c));
      } else if constexpr (KIND == 2) {
        // two instructions: the low and the high product of one limb
        asm volatile("mad.lo.cc.u32 %0, %0, %1, %0;\n\tmadc.hi.u32 %0, %0, %1, %2;"
                     : "+r"(x[j]) : "r"(m), "r"(c));
      } else if constexpr (KIND == 3) {
        asm volatile("add.u32 %0, %0, %1;" : "+r"(x[j]) : "r"(c));
      } else if constexpr (KIND == 5) {
        asm volatile("mad.lo.u32 %0, %0, %2, %3;\n\tmad.hi.u32 %1, %1, %2, %3;"
                     : "+r"(x[j]), "+r"(y[j]) : "r"(m), "r"(c));
      } else {
        // both halves feed the chain, so the full 64-bit product is needed
        asm volatile(
            "{\n\t.reg .u64 w;\n\t.reg .u32 lo, hi;\n\tmad.wide.u32 w, %0, %1, %2;\n\t"
            "mov.b64 {lo, hi}, w;\n\txor.b32 %0, lo, hi;\n\t}"
            : "+r"(x[j]) : "r"(m), "l"(static_cast<uint64_t>(c)));
      }
    }
  }
  uint32_t acc = 0;
#pragma unroll
  for (int j = 0; j < 8; ++j) acc ^= x[j] ^ y[j];
  if (acc == 0x12345678u) g_probe_sink = acc;  // keeps the loop live
}

template <int KIND>
cudaError_t launch_rate(cudaStream_t s, int iters, unsigned* grid) {
  const void* k = reinterpret_cast<const void*>(int_rate_kernel<KIND>);
  *grid = static_cast<unsigned>(device_sm_count() * resident_blocks(k, 256));
  int_rate_kernel<KIND><<<*grid, 256, 0, s>>>(0x2545F491u, iters);
  return cudaGetLastError();
}

}  // namespace
}  // namespace montgb

using namespace montgb;

extern "C" int mont_probe_int_rate(int kind, int iters, void* stream, double* ops_per_s) {
  if (kind < 0 || kind > 5 || iters < 1 || !ops_per_s) return MONT_EINVAL;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned grid = 0;
  auto launch = [&]() {
    switch (kind) {
      case 0: return launch_rate<0>(s, iters, &grid);
      case 1: return launch_rate<1>(s, iters, &grid);
      case 2: return launch_rate<2>(s, iters, &grid);
      case 3: return launch_rate<3>(s, iters, &grid);
      case 4: return launch_rate<4>(s, iters, &grid);
      default: return launch_rate<5>(s, iters, &grid);
    }
  };
  cudaError_t e = launch();  // warm-up
  if (e != cudaSuccess) return cuda_status(e);
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess) return cuda_status(e);
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_status(e);
  }
  cudaEventRecord(e0, s);
  e = launch();
  cudaEventRecord(e1, s);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  float ms = 0;
  if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (e != cudaSuccess) return cuda_status(e);
  const double per_thread = 8.0 * iters * (kind == 2 || kind == 5 ? 2.0 : 1.0);
  *ops_per_s = per_thread * grid * 256.0 / (ms * 1e-3);
  return MONT_OK;
}
