// Element-wise word kernels: one launch streams the operands from HBM with
// 256-bit (or 128-bit) vector loads, applies one of the word reductions of
// word_ops.cuh, and streams the result back.  Nothing else touches memory, so
// the kernels are bound by HBM bandwidth: per element they move
// 2 E in + 1 E out (mont_mul), 1 E in + 1 E out (domain maps) or
// 1 TT in + 1 E out (mont_redc).
//
// Work distribution: a grid-stride loop over "units" of one vector of output
// elements; each thread keeps `U` units in flight (all loads issued before
// any arithmetic) so that enough bytes are outstanding per SM to cover HBM
// latency.  The ragged tail (fewer elements than one vector) runs on the
// scalar path at the end.
#pragma once

#include <cstdint>

#include "word_ops.cuh"

namespace montgb {

template <int VB>
struct Vec {
  uint32_t w[VB / 4];
};

__device__ __forceinline__ void vld(Vec<32>& v, const void* p) {
  asm volatile(
      "ld.global.L1::no_allocate.v8.u32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3]), "=r"(v.w[4]), "=r"(v.w[5]),
        "=r"(v.w[6]), "=r"(v.w[7])
      : "l"(p));
}
__device__ __forceinline__ void vld(Vec<16>& v, const void* p) {
  asm volatile("ld.global.L1::no_allocate.v4.u32 {%0,%1,%2,%3}, [%4];"
               : "=r"(v.w[0]), "=r"(v.w[1]), "=r"(v.w[2]), "=r"(v.w[3])
               : "l"(p));
}
__device__ __forceinline__ void vst(void* p, const Vec<32>& v) {
  asm volatile("st.global.cs.v8.u32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"l"(p), "r"(v.w[0]),
               "r"(v.w[1]), "r"(v.w[2]), "r"(v.w[3]), "r"(v.w[4]), "r"(v.w[5]), "r"(v.w[6]),
               "r"(v.w[7])
               : "memory");
}
__device__ __forceinline__ void vst(void* p, const Vec<16>& v) {
  asm volatile("st.global.cs.v4.u32 [%0], {%1,%2,%3,%4};" ::"l"(p), "r"(v.w[0]), "r"(v.w[1]),
               "r"(v.w[2]), "r"(v.w[3])
               : "memory");
}

// Element e of a vector, for 32-bit and 64-bit element types.
template <class E, int VB>
__device__ __forceinline__ E vget(const Vec<VB>& v, int e) {
  if constexpr (sizeof(E) == 4) {
    return static_cast<E>(v.w[e]);
  } else {
    return static_cast<E>(static_cast<uint64_t>(v.w[2 * e]) |
                          (static_cast<uint64_t>(v.w[2 * e + 1]) << 32));
  }
}
template <class E, int VB>
__device__ __forceinline__ void vset(Vec<VB>& v, int e, E x) {
  if constexpr (sizeof(E) == 4) {
    v.w[e] = static_cast<uint32_t>(x);
  } else {
    const uint64_t u = static_cast<uint64_t>(x);
    v.w[2 * e] = static_cast<uint32_t>(u);
    v.w[2 * e + 1] = static_cast<uint32_t>(u >> 32);
  }
}
// Double-width element e of the pair of vectors (lo, hi) holding consecutive T.
template <class TT, int VB>
__device__ __forceinline__ TT vget_tt(const Vec<VB>& a, const Vec<VB>& b, int e) {
  constexpr int W = sizeof(TT) / 4;       // 32-bit words per TT
  constexpr int PER = (VB / 4) / W;       // TT per vector
  const Vec<VB>& v = e < PER ? a : b;
  const int base = (e % PER) * W;
  if constexpr (W == 2) {
    return static_cast<TT>(static_cast<uint64_t>(v.w[base]) |
                           (static_cast<uint64_t>(v.w[base + 1]) << 32));
  } else {
    const uint64_t lo = static_cast<uint64_t>(v.w[base]) | (static_cast<uint64_t>(v.w[base + 1]) << 32);
    const uint64_t hi =
        static_cast<uint64_t>(v.w[base + 2]) | (static_cast<uint64_t>(v.w[base + 3]) << 32);
    return static_cast<TT>((static_cast<u128>(hi) << 64) | lo);
  }
}

template <class Op, Mode M>
__device__ __forceinline__ typename Op::E apply(typename Op::E x, typename Op::E y,
                                                typename Op::TT t, const typename Op::C& c) {
  using E = typename Op::E;
  if constexpr (M == Mode::kMul) {
    return Op::reduce(Op::mul(x, y), c);
  } else if constexpr (M == Mode::kToDomain) {
    return Op::reduce(Op::mul(x, static_cast<E>(c.r2)), c);
  } else if constexpr (M == Mode::kFromDomain) {
    return Op::canon(Op::reduce(Op::widen(x), c), c);
  } else {
    return Op::reduce(t, c);
  }
}

// One scalar element (the tail, and every element on the scalar path).
template <class Op, Mode M>
__device__ __forceinline__ void scalar_element(const void* xp, const void* yp, void* op, size_t i,
                                               const typename Op::C& c) {
  using E = typename Op::E;
  using TT = typename Op::TT;
  E x{}, y{};
  TT t{};
  if constexpr (M == Mode::kRedc) {
    t = static_cast<const TT*>(xp)[i];
  } else {
    x = static_cast<const E*>(xp)[i];
    if constexpr (M == Mode::kMul) y = static_cast<const E*>(yp)[i];
  }
  static_cast<E*>(op)[i] = apply<Op, M>(x, y, t, c);
}

template <class Op, Mode M, int VB, int U>
__global__ void __launch_bounds__(512) word_kernel(const void* __restrict__ xp,
                                                   const void* __restrict__ yp,
                                                   void* __restrict__ op, size_t n,
                                                   const typename Op::C c) {
  using E = typename Op::E;
  using TT = typename Op::TT;
  pdl_enter();   // launched by launch_pdl (without its attribute, a no-op)
  const size_t nthreads = static_cast<size_t>(gridDim.x) * blockDim.x;
  const size_t tid = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  size_t done = 0;
  if constexpr (VB > 0) {
    constexpr int EPV = VB / static_cast<int>(sizeof(E));  // elements per vector
    const size_t nv = n / EPV;
    const char* x = static_cast<const char*>(xp);
    const char* y = static_cast<const char*>(yp);
    char* o = static_cast<char*>(op);
    for (size_t base = static_cast<size_t>(blockIdx.x) * blockDim.x * U; base < nv;
         base += nthreads * U) {
      Vec<VB> vx[U], vy[U];
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const size_t v = base + threadIdx.x + static_cast<size_t>(j) * blockDim.x;
        if (v < nv) {
          if constexpr (M == Mode::kRedc) {
            vld(vx[j], x + 2 * v * VB);
            vld(vy[j], x + 2 * v * VB + VB);
          } else {
            vld(vx[j], x + v * VB);
            if constexpr (M == Mode::kMul) vld(vy[j], y + v * VB);
          }
        }
      }
#pragma unroll
      for (int j = 0; j < U; ++j) {
        const size_t v = base + threadIdx.x + static_cast<size_t>(j) * blockDim.x;
        if (v < nv) {
          Vec<VB> vo;
#pragma unroll
          for (int e = 0; e < EPV; ++e) {
            E xe{}, ye{};
            TT te{};
            if constexpr (M == Mode::kRedc) {
              te = vget_tt<TT, VB>(vx[j], vy[j], e);
            } else {
              xe = vget<E, VB>(vx[j], e);
              if constexpr (M == Mode::kMul) ye = vget<E, VB>(vy[j], e);
            }
            vset<E, VB>(vo, e, apply<Op, M>(xe, ye, te, c));
          }
          vst(o + v * VB, vo);
        }
      }
    }
    done = nv * EPV;
  }
  for (size_t i = done + tid; i < n; i += nthreads) scalar_element<Op, M>(xp, yp, op, i, c);
}

template <class Op, Mode M, int VB, int U>
cudaError_t launch_one(const typename Op::C& c, const void* x, const void* y, void* out, size_t n,
                       cudaStream_t s, const LaunchShape& shape) {
  auto kernel = word_kernel<Op, M, VB, U>;
  const int threads = shape.threads;
  const size_t epv = VB > 0 ? VB / sizeof(typename Op::E) : 1;
  const size_t units = VB > 0 ? n / epv : n;
  const size_t per_block = static_cast<size_t>(threads) * (VB > 0 ? U : 1);
  size_t want = units / per_block + 1;  // +1 also covers the ragged tail
  const int per_sm = shape.blocks_per_sm > 0 ? shape.blocks_per_sm : resident_blocks(reinterpret_cast<const void*>(kernel), threads);
  const size_t cap = static_cast<size_t>(device_sm_count()) * per_sm;
  const unsigned grid = static_cast<unsigned>(want < cap ? want : cap);
  return launch_pdl(kernel, grid, static_cast<unsigned>(threads), 0, s, x, y, out, n, c);
}

template <class Op, Mode M>
cudaError_t launch_shape(const typename Op::C& c, const void* x, const void* y, void* out, size_t n,
                         cudaStream_t s, const LaunchShape& shape) {
  if (shape.vec_bytes == 32) {
    switch (shape.unroll) {
      case 1: return launch_one<Op, M, 32, 1>(c, x, y, out, n, s, shape);
      case 4: return launch_one<Op, M, 32, 4>(c, x, y, out, n, s, shape);
      default: return launch_one<Op, M, 32, 2>(c, x, y, out, n, s, shape);
    }
  }
  if (shape.vec_bytes == 16) {
    switch (shape.unroll) {
      case 1: return launch_one<Op, M, 16, 1>(c, x, y, out, n, s, shape);
      case 4: return launch_one<Op, M, 16, 4>(c, x, y, out, n, s, shape);
      default: return launch_one<Op, M, 16, 2>(c, x, y, out, n, s, shape);
    }
  }
  return launch_one<Op, M, 0, 1>(c, x, y, out, n, s, shape);
}

template <class Op>
cudaError_t launch_mode(Mode mode, const typename Op::C& c, const void* x, const void* y, void* out,
                        size_t n, cudaStream_t s, const LaunchShape& shape) {
  switch (mode) {
    case Mode::kMul: return launch_shape<Op, Mode::kMul>(c, x, y, out, n, s, shape);
    case Mode::kToDomain: return launch_shape<Op, Mode::kToDomain>(c, x, y, out, n, s, shape);
    case Mode::kFromDomain: return launch_shape<Op, Mode::kFromDomain>(c, x, y, out, n, s, shape);
    case Mode::kRedc: return launch_shape<Op, Mode::kRedc>(c, x, y, out, n, s, shape);
  }
  return cudaErrorInvalidValue;
}

}  // namespace montgb
