// Plantard's fixed-multiplier form (Section 3.2): mont_const_prepare and
// mont_mul_pre.
//
// For a multiplier b used many times (a twiddle factor, a key), the Plantard
// family can precompute b' = b N^{-1} mod R once.  The reduction of a b then
// needs m = a b' mod R -- a word-by-double-word low product, of which only
// the high word is used -- and no double-width T = a b at all.  The results
// are identical to mont_mul's.  The kernels stream like the element-wise
// word kernels: 256-bit loads of a and of the double-word b', U vectors in
// flight per thread, scalar tails.
#include "word_kernel.cuh"

namespace montgb {
namespace {

enum class PreMode : int { kPrepare = 0, kMul = 1 };

// b' for element i (kPrepare), or a[i] times prepared b'[i] (kMul).
template <class Op, PreMode M>
__device__ __forceinline__ void pre_scalar(const void* xp, const void* yp, void* op, size_t i,
                                           const typename Op::C& c) {
  using E = typename Op::E;
  using TT = typename Op::TT;
  if constexpr (M == PreMode::kPrepare) {
    static_cast<TT*>(op)[i] = Op::prepare(static_cast<const E*>(xp)[i], c);
  } else {
    static_cast<E*>(op)[i] = Op::mul_pre(static_cast<const E*>(xp)[i], static_cast<const TT*>(yp)[i], c);
  }
}

template <class Op, PreMode M, int VB, int U>
__global__ void __launch_bounds__(512) pre_kernel(const void* __restrict__ xp,
                                                  const void* __restrict__ yp,
                                                  void* __restrict__ op, size_t n,
                                                  const typename Op::C c) {
  using E = typename Op::E;
  using TT = typename Op::TT;
  const size_t nthreads = static_cast<size_t>(gridDim.x) * blockDim.x;
  const size_t tid = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  size_t done = 0;
  if constexpr (VB > 0) {
    constexpr int EPV = VB / static_cast<int>(sizeof(E));   // E elements per vector; TT needs 2 vectors
    const size_t nv = n / EPV;
    const char* x = static_cast<const char*>(xp);
    const char* y = static_cast<const char*>(yp);
    char* o = static_cast<char*>(op);
    for (size_t base = static_cast<size_t>(blockIdx.x) * blockDim.x * U; base < nv;
         base += nthreads * U) {
      Vec<VB> vx[U], vy0[U], vy1[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const size_t v = base + threadIdx.x + static_cast<size_t>(j) * blockDim.x;
        if (v < nv) {
          vld(vx[j], x + v * VB);
          if constexpr (M == PreMode::kMul) {
            vld(vy0[j], y + 2 * v * VB);
            vld(vy1[j], y + 2 * v * VB + VB);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const size_t v = base + threadIdx.x + static_cast<size_t>(j) * blockDim.x;
        if (v < nv) {
          if constexpr (M == PreMode::kMul) {
            Vec<VB> vo;
#pragma unroll
            for (int e = 0; e < EPV; ++e)
              vset<E, VB>(vo, e, Op::mul_pre(vget<E, VB>(vx[j], e), vget_tt<TT, VB>(vy0[j], vy1[j], e), c));
            vst(o + v * VB, vo);
          } else {
            Vec<VB> w0, w1;   // EPV prepared values over two vectors
            constexpr int W = static_cast<int>(sizeof(TT) / 4);
            constexpr int PER = (VB / 4) / W;
#pragma unroll
            for (int e = 0; e < EPV; ++e) {
              const TT t = Op::prepare(vget<E, VB>(vx[j], e), c);
              Vec<VB>& w = e < PER ? w0 : w1;
              const int b0 = (e % PER) * W;
              if constexpr (W == 2) {
                const uint64_t u = static_cast<uint64_t>(t);
                w.w[b0] = static_cast<uint32_t>(u);
                w.w[b0 + 1] = static_cast<uint32_t>(u >> 32);
              } else {
                const u128 u = static_cast<u128>(t);
                w.w[b0] = static_cast<uint32_t>(u);
                w.w[b0 + 1] = static_cast<uint32_t>(u >> 32);
                w.w[b0 + 2] = static_cast<uint32_t>(u >> 64);
                w.w[b0 + 3] = static_cast<uint32_t>(u >> 96);
              }
            }
            vst(o + 2 * v * VB, w0);
            vst(o + 2 * v * VB + VB, w1);
          }
        }
      }
    }
    done = nv * EPV;
  }
  for (size_t i = done + tid; i < n; i += nthreads) pre_scalar<Op, M>(xp, yp, op, i, c);
}

template <class Op, PreMode M, int VB, int U>
cudaError_t launch_pre_one(const typename Op::C& c, const void* x, const void* y, void* out,
                           size_t n, cudaStream_t s, int threads) {
  auto kernel = pre_kernel<Op, M, VB, U>;
  const size_t epv = VB > 0 ? VB / sizeof(typename Op::E) : 1;
  const size_t units = VB > 0 ? n / epv : n;
  const size_t per_block = static_cast<size_t>(threads) * (VB > 0 ? U : 1);
  const size_t want = units / per_block + 1;
  const int per_sm = resident_blocks(reinterpret_cast<const void*>(kernel), threads);
  const size_t cap = static_cast<size_t>(device_sm_count()) * per_sm;
  kernel<<<static_cast<unsigned>(want < cap ? want : cap), threads, 0, s>>>(x, y, out, n, c);
  return cudaGetLastError();
}

template <class Op>
cudaError_t launch_pre(PreMode m, const typename Op::C& c, const void* x, const void* y, void* out,
                       size_t n, cudaStream_t s, bool vec) {
  if (m == PreMode::kPrepare) {
    return vec ? launch_pre_one<Op, PreMode::kPrepare, 32, 2>(c, x, y, out, n, s, 256)
               : launch_pre_one<Op, PreMode::kPrepare, 0, 1>(c, x, y, out, n, s, 256);
  }
  return vec ? launch_pre_one<Op, PreMode::kMul, 32, 2>(c, x, y, out, n, s, 256)
             : launch_pre_one<Op, PreMode::kMul, 0, 1>(c, x, y, out, n, s, 256);
}

int pre_entry(mont_ctx_t ctx, PreMode m, const void* x, const void* y, void* out, size_t n,
              void* stream) {
  if (!ctx) return MONT_EINVAL;
  if (ctx->variant < MONT_PLANTARD || ctx->n_limbs > 2) return MONT_EINVAL;  // Plantard family, words
  if (n == 0) return MONT_OK;
  if (!x || !out || (m == PreMode::kMul && !y)) return MONT_EINVAL;
  const size_t es = 4u * static_cast<size_t>(ctx->n_limbs);
  const auto al = [](const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; };
  // prepared values are double words: 8-byte aligned at 32 bits, 16-byte at 64 bits
  const void* pre = m == PreMode::kMul ? y : out;
  if (!al(x, es) || !al(pre, 2 * es) || !al(out, es)) return MONT_EINVAL;
  if (n > SIZE_MAX / (2 * es)) return MONT_EINVAL;
  // no overlap between the prepared array and the element arrays
  const uintptr_t pp = reinterpret_cast<uintptr_t>(pre);
  const uintptr_t xx = reinterpret_cast<uintptr_t>(x);
  if (pp < xx + n * es && xx < pp + 2 * n * es) return MONT_EINVAL;
  if (m == PreMode::kMul) {
    const uintptr_t oo = reinterpret_cast<uintptr_t>(out);
    if (pp < oo + n * es && oo < pp + 2 * n * es) return MONT_EINVAL;
    if (oo != xx && oo < xx + n * es && xx < oo + n * es) return MONT_EINVAL;
  }
  const bool vec = al(x, 32) && al(y ? y : out, 32) && al(out, 32);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  if (ctx->n_limbs == 1) {
    switch (ctx->variant) {
      case MONT_PLANTARD: e = launch_pre<Plantard32>(m, ctx->w32, x, y, out, n, s, vec); break;
      case MONT_SIGNED_PLANTARD: e = launch_pre<SignedPlantard32>(m, ctx->w32, x, y, out, n, s, vec); break;
      default: e = launch_pre<SignedPlantard2_32>(m, ctx->w32, x, y, out, n, s, vec); break;
    }
  } else {
    switch (ctx->variant) {
      case MONT_PLANTARD: e = launch_pre<Plantard64>(m, ctx->w64, x, y, out, n, s, vec); break;
      case MONT_SIGNED_PLANTARD: e = launch_pre<SignedPlantard64>(m, ctx->w64, x, y, out, n, s, vec); break;
      default: e = launch_pre<SignedPlantard2_64>(m, ctx->w64, x, y, out, n, s, vec); break;
    }
  }
  return cuda_status(e);
}

}  // namespace
}  // namespace montgb

using montgb::PreMode;

extern "C" int mont_const_prepare(mont_ctx_t ctx, const void* b, void* b_pre, size_t n,
                                  void* stream) {
  return montgb::pre_entry(ctx, PreMode::kPrepare, b, nullptr, b_pre, n, stream);
}

extern "C" int mont_mul_pre(mont_ctx_t ctx, const void* a, const void* b_pre, void* out, size_t n,
                            void* stream) {
  return montgb::pre_entry(ctx, PreMode::kMul, a, b_pre, out, n, stream);
}
