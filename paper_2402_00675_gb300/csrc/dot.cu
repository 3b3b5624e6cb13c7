// Lazy reduction with Algorithm 4 (mont_dot_lazy).
//
// Section 3.3: Algorithm 4 (SigPRedc2) is correct for every |T| <= 2^{2 alpha}
// N^2 when alpha >= 1.  A product of two centred residues has |a b| <= N^2/4,
// so a sum of k <= 4^{alpha + 1} such products can be accumulated exactly in a
// double word and reduced once: out[j] = SigPRedc2(sum_i a[j,i] b[j,i]) =
// -(sum_i a b) R^{-1} mods N, one reduction per row instead of one per product.
//
// One thread per row; the row's elements are read with L1-cached loads
// (16-byte vectors when the row is aligned), products accumulated in int64
// (32-bit words: |T| <= 4^alpha N^2 < 2^62 because N < 2^{31-alpha}) or in a
// 128-bit integer (64-bit words).
#include "word_kernel.cuh"

namespace montgb {
namespace {

template <class Op>
__global__ void __launch_bounds__(256) dot_kernel(const typename Op::E* __restrict__ a,
                                                  const typename Op::E* __restrict__ b,
                                                  typename Op::E* __restrict__ out, size_t rows,
                                                  uint32_t k, int vec16,
                                                  const typename Op::C c) {
  using E = typename Op::E;
  using TT = typename Op::TT;
  constexpr int V = 16 / static_cast<int>(sizeof(E));   // elements per 16-byte vector
  const size_t nthreads = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t j = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < rows;
       j += nthreads) {
    const E* ra = a + j * k;
    const E* rb = b + j * k;
    TT T = 0;
    uint32_t i = 0;
    if (vec16) {
      for (; i + V <= k; i += V) {
        const uint4 va = *reinterpret_cast<const uint4*>(ra + i);
        const uint4 vb = *reinterpret_cast<const uint4*>(rb + i);
        const E* xa = reinterpret_cast<const E*>(&va);
        const E* xb = reinterpret_cast<const E*>(&vb);
#pragma unroll
        for (int e = 0; e < V; ++e) T += Op::mul(xa[e], xb[e]);
      }
    }
    for (; i < k; ++i) T += Op::mul(ra[i], rb[i]);
    out[j] = Op::reduce(T, c);
  }
}

template <class Op>
cudaError_t launch_dot(const typename Op::C& c, const void* a, const void* b, void* out,
                       size_t rows, uint32_t k, int vec16, cudaStream_t s) {
  const void* kern = reinterpret_cast<const void*>(dot_kernel<Op>);
  const size_t want = (rows + 255) / 256;
  const size_t cap = static_cast<size_t>(device_sm_count()) * resident_blocks(kern, 256);
  dot_kernel<Op><<<static_cast<unsigned>(want < cap ? want : cap), 256, 0, s>>>(
      static_cast<const typename Op::E*>(a), static_cast<const typename Op::E*>(b),
      static_cast<typename Op::E*>(out), rows, k, vec16, c);
  return cudaGetLastError();
}

}  // namespace
}  // namespace montgb

using namespace montgb;

extern "C" int mont_dot_lazy(mont_ctx_t ctx, const void* a, const void* b, void* out, size_t rows,
                             uint32_t k, void* stream) {
  if (!ctx || ctx->variant != MONT_SIGNED_PLANTARD2 || ctx->n_limbs > 2) return MONT_EINVAL;
  // k <= 4^{alpha + 1}: keeps |sum a b| <= k N^2 / 4 <= 4^alpha N^2
  if (k == 0 || (ctx->alpha + 1 < 16 && k > (1u << (2 * (ctx->alpha + 1))))) return MONT_EINVAL;
  if (rows == 0) return MONT_OK;
  if (!a || !b || !out) return MONT_EINVAL;
  const size_t es = 4u * static_cast<size_t>(ctx->n_limbs);
  const auto al = [](const void* p, size_t x) { return (reinterpret_cast<uintptr_t>(p) % x) == 0; };
  if (!al(a, es) || !al(b, es) || !al(out, es)) return MONT_EINVAL;
  if (rows > SIZE_MAX / (es * k)) return MONT_EINVAL;
  const uintptr_t o = reinterpret_cast<uintptr_t>(out);
  for (const void* p : {a, b}) {
    const uintptr_t q = reinterpret_cast<uintptr_t>(p);
    if (q < o + rows * es && o < q + rows * k * es) return MONT_EINVAL;   // out must not overlap inputs
  }
  const int vec16 = al(a, 16) && al(b, 16) && ((k * es) % 16 == 0) ? 1 : 0;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const cudaError_t e = ctx->n_limbs == 1
                            ? launch_dot<SignedPlantard2_32>(ctx->w32, a, b, out, rows, k, vec16, s)
                            : launch_dot<SignedPlantard2_64>(ctx->w64, a, b, out, rows, k, vec16, s);
  return cuda_status(e);
}
