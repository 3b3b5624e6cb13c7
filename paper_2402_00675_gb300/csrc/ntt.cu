// Batched negacyclic number-theoretic transform (mont_ntt_*).
//
// The paper names the NTT of lattice and homomorphic-encryption schemes as
// the reason word-size Montgomery-type reductions matter (Section 1) and
// Plantard's fixed-multiplier form as what makes his reduction attractive
// there (Section 3.2); the transform itself is textbook:
//   forward  A[i] = sum_j a[j] psi^{(2 brv(i) + 1) j}  (mod N), bit-reversed output,
//   inverse  a[j] = n^{-1} sum_i A[i] psi^{-(2 brv(i) + 1) j},
// for a primitive 2n-th root of unity psi.  Forward layers are Cooley-Tukey
// butterflies (x, y) -> (x + w y, x - w y) with w = psi^{brv(k)}, k = n/(2 len)
// + group, for len = n/2 down to 1; the inverse undoes them in reverse order,
// (X, Y) -> (X + Y, (X - Y) w^{-1}), and scales by n^{-1} at the end.
//
// Mapping: for n = 32 a warp owns a polynomial, one coefficient per lane,
// and every layer pairs lane t with lane t ^ len through one shuffle, both
// lanes computing the same product w y; for n >= 64 groups of lanes own a
// polynomial with several coefficients per lane in registers (the phased
// kernel below).  Twiddles live in shared memory in multiplier form: w R mod
// N for REDC (so REDC(y * wR) = y w), and Plantard's prepared b' = (-w R mod
// N) N^{-1} mod R for the Plantard reduction (so the product -y (-wR) R^{-1}
// = y w); the data stays in the plain representation [0, N).
//
// Lazy butterflies (4N <= 2^w).  Algorithm 2 returns the exact residue for
// every 0 <= T <= N 2^w once N <= 2^{w-1} (with m = m1 2^w + m0 its output is
// floor(k + d), k = (mN - T)/R the residue, d = (N 2^w + m0 N - T)/R in
// [0, 1) on that domain), and REDC without its final subtraction returns
// (T + mN)/R < 2N for every T < RN.  So a twiddle product t of any y < 4N is
// below B N (B = 1 for Plantard, 2 for REDC), and the coefficients may stay
// unreduced: forward inputs below (2 + B) N, x -> min(x, x - 2N) below 2N,
// then (x + t, x + B N - t); inverse inputs below 2N, (X, Y) -> (min(s, s -
// 2N), w (X + 2N - Y)) with s = X + Y.  Unsigned min picks the reduced value
// because the other one wraps past 2^w.  One min step pair at the end of the
// forward transform, and the final (canonical) product by n^{-1} in the
// inverse, return [0, N).
#include <cstring>
#include <new>
#include <vector>

#include "word_kernel.cuh"

namespace montgb {
namespace {

template <class Op>
struct Tw;
template <>
struct Tw<Redc32> {
  using T = uint32_t;
  static constexpr uint32_t kB = 2;   // mul_lazy < kB N
  static __device__ __forceinline__ uint32_t mul(uint32_t y, T w, const WordConst32& c) {
    return Redc32::reduce(Redc32::mul(y, w), c);
  }
  // REDC without its final subtraction: (T + mN)/R < 2N for T < RN.  The low
  // words of T and mN cancel, so the carry out of their sum is (T mod R != 0).
  static __device__ __forceinline__ uint32_t mul_lazy(uint32_t y, T w, const WordConst32& c) {
    const uint64_t t = static_cast<uint64_t>(y) * w;
    const uint32_t lo = static_cast<uint32_t>(t);
    const uint32_t m = lo * c.nprime;
    return static_cast<uint32_t>(t >> 32) + __umulhi(m, c.N) + (lo != 0u ? 1u : 0u);
  }
};
template <>
struct Tw<Plantard32> {
  using T = uint64_t;
  static constexpr uint32_t kB = 1;   // exact: below N
  static __device__ __forceinline__ uint32_t mul(uint32_t y, T w, const WordConst32& c) {
    return Plantard32::mul_pre(y, w, c);
  }
  static __device__ __forceinline__ uint32_t mul_lazy(uint32_t y, T w, const WordConst32& c) {
    return Plantard32::mul_pre(y, w, c);
  }
};
template <>
struct Tw<Redc64> {
  using T = uint64_t;
  static constexpr uint64_t kB = 2;
  static __device__ __forceinline__ uint64_t mul(uint64_t y, T w, const WordConst64& c) {
    return Redc64::reduce(Redc64::mul(y, w), c);
  }
  static __device__ __forceinline__ uint64_t mul_lazy(uint64_t y, T w, const WordConst64& c) {
    const uint64_t lo = y * w;
    const uint64_t m = lo * c.nprime;
    return __umul64hi(y, w) + __umul64hi(m, c.N) + (lo != 0u ? 1u : 0u);
  }
};
template <>
struct Tw<Plantard64> {
  using T = u128;
  static constexpr uint64_t kB = 1;
  static __device__ __forceinline__ uint64_t mul(uint64_t y, T w, const WordConst64& c) {
    return Plantard64::mul_pre(y, w, c);
  }
  static __device__ __forceinline__ uint64_t mul_lazy(uint64_t y, T w, const WordConst64& c) {
    return Plantard64::mul_pre(y, w, c);
  }
};

template <class E>
__device__ __forceinline__ E add_n(E x, E t, E N) {  // x, t in [0, N)
  const E s = x + t;
  return (s < x || s >= N) ? s - N : s;
}
template <class E>
__device__ __forceinline__ E sub_n(E x, E t, E N) {
  return x >= t ? x - t : x - t + N;
}

// x - c if x >= c else x, for x < c + 2^w - c: the wrapped difference is larger
template <class E>
__device__ __forceinline__ E sub_if_ge(E x, E c) { return min(x, static_cast<E>(x - c)); }

// One butterfly on a register pair: forward (a, b) -> (a + w b, a - w b),
// inverse (a, b) -> (a + b, (a - b) w); canonical or lazy (see above).
template <class Op, bool INV, bool LAZY>
__device__ __forceinline__ void butterfly(typename Op::E& a, typename Op::E& b,
                                          const typename Tw<Op>::T w, const typename Op::C& c) {
  using E = typename Op::E;
  const E N = static_cast<E>(c.N);
  if constexpr (!INV) {
    if constexpr (LAZY) {
      const E x = sub_if_ge<E>(a, 2 * N);
      const E t = Tw<Op>::mul_lazy(b, w, c);   // below kB N
      a = x + t;
      b = x + Tw<Op>::kB * N - t;
    } else {
      const E t = Tw<Op>::mul(b, w, c);
      const E x = a;
      a = add_n<E>(x, t, N);
      b = sub_n<E>(x, t, N);
    }
  } else {
    if constexpr (LAZY) {
      const E s = a + b;
      const E d = a + 2 * N - b;
      a = sub_if_ge<E>(s, 2 * N);
      b = Tw<Op>::mul_lazy(d, w, c);
    } else {
      const E x = a, y = b;
      a = add_n<E>(x, y, N);
      b = Tw<Op>::mul(sub_n<E>(x, y, N), w, c);
    }
  }
}

// One layer of the n = 32 transform (one coefficient per lane): lane t
// pairs with lane t ^ len through one shuffle.
template <class Op, int LOG2N, int L, bool INV, bool LAZY>
__device__ __forceinline__ void layer(typename Op::E (&v)[(1 << LOG2N) / 32],
                                      const typename Tw<Op>::T* stw, int lane,
                                      const typename Op::C& c) {
  static_assert(LOG2N == 5, "the shuffle layers serve n = 32 only");
  using E = typename Op::E;
  constexpr int n = 1 << LOG2N;
  constexpr int len = 1 << L;
  const bool upper = (lane & len) != 0;
  const typename Tw<Op>::T w = stw[(n >> (L + 1)) + (lane >> (L + 1))];
  const E other = __shfl_xor_sync(0xFFFFFFFFu, v[0], len);
  E x = upper ? other : v[0];
  E y = upper ? v[0] : other;
  butterfly<Op, INV, LAZY>(x, y, w, c);   // both lanes, each keeps its half
  v[0] = upper ? y : x;
}

template <class Op, int LOG2N, bool LAZY, int L>
__device__ __forceinline__ void layers_fwd(typename Op::E (&v)[(1 << LOG2N) / 32],
                                           const typename Tw<Op>::T* stw, int lane,
                                           const typename Op::C& c) {
  layer<Op, LOG2N, L, false, LAZY>(v, stw, lane, c);
  if constexpr (L > 0) layers_fwd<Op, LOG2N, LAZY, L - 1>(v, stw, lane, c);
}

template <class Op, int LOG2N, bool LAZY, int L>
__device__ __forceinline__ void layers_inv(typename Op::E (&v)[(1 << LOG2N) / 32],
                                           const typename Tw<Op>::T* stw, int lane,
                                           const typename Op::C& c) {
  layer<Op, LOG2N, L, true, LAZY>(v, stw, lane, c);
  if constexpr (L + 1 < LOG2N) layers_inv<Op, LOG2N, LAZY, L + 1>(v, stw, lane, c);
}

// [0, 3N) -> [0, N) after a lazy forward transform
template <class E>
__device__ __forceinline__ E canon3(E x, E N) { return sub_if_ge<E>(sub_if_ge<E>(x, 2 * N), N); }

template <class Op, int LOG2N, bool INV, bool LAZY>
__global__ void __launch_bounds__(256) ntt_kernel(const typename Op::E* __restrict__ in,
                                                  typename Op::E* __restrict__ out, size_t batch,
                                                  const typename Tw<Op>::T* __restrict__ tw,
                                                  const typename Tw<Op>::T scale,
                                                  const typename Op::C c) {
  using E = typename Op::E;
  using T = typename Tw<Op>::T;
  constexpr int n = 1 << LOG2N;
  constexpr int EPT = n / 32;
  __shared__ T stw[n];
  for (int i = threadIdx.x; i < n; i += blockDim.x) stw[i] = tw[i];
  __syncthreads();
  const int lane = threadIdx.x & 31;
  const size_t warp = (static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = (static_cast<size_t>(gridDim.x) * blockDim.x) >> 5;
  for (size_t p = warp; p < batch; p += nwarps) {
    const E* src = in + p * n;
    E v[EPT];
#pragma unroll
    for (int e = 0; e < EPT; ++e) v[e] = src[lane + 32 * e];
    if constexpr (!INV) {
      layers_fwd<Op, LOG2N, LAZY, LOG2N - 1>(v, stw, lane, c);
      if constexpr (LAZY) {
#pragma unroll
        for (int e = 0; e < EPT; ++e) v[e] = canon3<E>(v[e], static_cast<E>(c.N));
      }
    } else {
      layers_inv<Op, LOG2N, LAZY, 0>(v, stw, lane, c);
#pragma unroll
      for (int e = 0; e < EPT; ++e) v[e] = Tw<Op>::mul(v[e], scale, c);
    }
    E* dst = out + p * n;
#pragma unroll
    for (int e = 0; e < EPT; ++e) dst[lane + 32 * e] = v[e];
  }
}

// ------------------------------------------------------------ phased kernel
//
// For n >= 64 a group of 2^LB lanes owns one polynomial, each lane holding
// EPT = 2^K coefficients, K = max(log2 n - 5, 4): a whole warp per polynomial
// from n = 512, a half-warp at n = 256, 8 lanes at 128, 4 at 64 (fewer
// phases, hence fewer shared-memory transposes, than one coefficient row per
// lane); with 64-bit words at n = 1024, K = 4 and two warps per polynomial
// (32 coefficients of 64 bits per lane overflowed the registers and the
// instruction cache), their transposes separated by block barriers.  The transform runs in phases; phase ph puts the index bits [lo,
// lo + K), lo = max(0, m - (ph + 1) K), inside the lane (element e supplies
// them) and the other LB bits in the lane's number t within its group:
//     i(ph, t, e) = ((t >> lo) << (lo + K)) | (e << lo) | (t & (2^lo - 1)),
// so every butterfly of the phase's layers pairs two registers of one lane.
// Between phases the group rewrites its coefficients through its own region
// of shared memory (one plane of 32-bit words per word of the element;
// address i + 4 (i >> 5) spreads a phase's accesses over the banks, and the
// groups of a warp sit 2^LB words apart modulo 32 so that they use different
// banks).  Phase 0 is i = 2^LB e + t (coalesced element loads), the last
// phase is i = EPT t + e (each lane owns EPT consecutive coefficients:
// vector accesses).

template <int LOG2N, int W>
struct Phases {
  static constexpr int m = LOG2N;
  // coefficient bits per lane: at most 16 64-bit words (two warps per polynomial
  // at n = 1024), else max(log2 n - 5, 4)
  static constexpr int K = (W == 2 && LOG2N >= 10) ? 4 : (LOG2N - 5 > 4 ? LOG2N - 5 : 4);
  static constexpr int LB = m - K;                           // lane bits of a group
  static constexpr bool kBlock = LB > 5;                     // a group spans several warps
  static constexpr int GPB = 256 >> LB;                      // polynomials per 256-thread block
  static constexpr int EPT = 1 << K;
  static constexpr int count = (m + K - 1) / K;
  __host__ __device__ static constexpr int lo(int ph) { return m - (ph + 1) * K > 0 ? m - (ph + 1) * K : 0; }
  __host__ __device__ static constexpr int top(int ph) { return m - ph * K; }   // bits [bottom, top) butterflied in ph
  __host__ __device__ static constexpr int bottom(int ph) { return lo(ph); }
  __host__ __device__ static constexpr int pad(int n) { return n + (n >> 3); }
  static constexpr int plane = pad(1 << m);                  // words of one plane
  // words of one group's region with `planes` planes, 2^LB (mod 32) apart
  __host__ __device__ static constexpr int group_words(int planes) {
    return (planes * plane + 31) / 32 * 32 + (LB < 5 ? (1 << LB) : 0);
  }
};

__device__ __forceinline__ int swz(int i) { return i + ((i >> 5) << 2); }

template <int LOG2N, int W>
__device__ __forceinline__ int index_of(int lo, int lane, int e) {
  constexpr int K = Phases<LOG2N, W>::K;
  return ((lane >> lo) << (lo + K)) | (e << lo) | (lane & ((1 << lo) - 1));
}

template <class E>
struct Planes;
template <>
struct Planes<uint32_t> {
  static constexpr int count = 1;
  static __device__ __forceinline__ void put(uint32_t* b, int stride, int a, uint32_t v) { b[a] = v; }
  static __device__ __forceinline__ uint32_t get(const uint32_t* b, int stride, int a) { return b[a]; }
};
template <>
struct Planes<uint64_t> {
  static constexpr int count = 2;
  static __device__ __forceinline__ void put(uint32_t* b, int stride, int a, uint64_t v) {
    b[a] = static_cast<uint32_t>(v);
    b[stride + a] = static_cast<uint32_t>(v >> 32);
  }
  static __device__ __forceinline__ uint64_t get(const uint32_t* b, int stride, int a) {
    return static_cast<uint64_t>(b[a]) | (static_cast<uint64_t>(b[stride + a]) << 32);
  }
};

// Move the lane's coefficients from phase layout `from` to layout `to` (buf:
// the group's region, lane: the lane's number in its group).  In the last
// layout (lo = 0) a lane's EPT coefficients are consecutive and stay inside
// one 32-word row of the padded buffer (starting at a multiple of four
// words), so that side moves as 128-bit accesses.
template <class E, int LOG2N>
__device__ __forceinline__ void transpose(E (&v)[Phases<LOG2N, Planes<E>::count>::EPT],
                                          uint32_t* buf, int lane, int lo_from, int lo_to) {
  using P = Phases<LOG2N, Planes<E>::count>;
  constexpr int W = Planes<E>::count;
  constexpr int EPT = P::EPT;
  constexpr int stride = P::plane;
  constexpr bool kVec = EPT % 4 == 0;
  const int row = swz(lane * EPT);
  if (kVec && lo_from == 0) {
#pragma unroll
    for (int q = 0; q < Planes<E>::count; ++q)
#pragma unroll
      for (int j = 0; j < EPT / 4; ++j)
        *reinterpret_cast<uint4*>(buf + q * stride + row + 4 * j) =
            make_uint4(static_cast<uint32_t>(static_cast<uint64_t>(v[4 * j]) >> (32 * q)),
                       static_cast<uint32_t>(static_cast<uint64_t>(v[4 * j + 1]) >> (32 * q)),
                       static_cast<uint32_t>(static_cast<uint64_t>(v[4 * j + 2]) >> (32 * q)),
                       static_cast<uint32_t>(static_cast<uint64_t>(v[4 * j + 3]) >> (32 * q)));
  } else {
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      Planes<E>::put(buf, stride, swz(index_of<LOG2N, W>(lo_from, lane, e)), v[e]);
  }
  if constexpr (P::kBlock) __syncthreads(); else __syncwarp();
  if (kVec && lo_to == 0) {
#pragma unroll
    for (int e = 0; e < EPT; ++e) v[e] = 0;
#pragma unroll
    for (int q = 0; q < Planes<E>::count; ++q)
#pragma unroll
      for (int j = 0; j < EPT / 4; ++j) {
        const uint4 w = *reinterpret_cast<const uint4*>(buf + q * stride + row + 4 * j);
        v[4 * j] |= static_cast<E>(static_cast<uint64_t>(w.x) << (32 * q));
        v[4 * j + 1] |= static_cast<E>(static_cast<uint64_t>(w.y) << (32 * q));
        v[4 * j + 2] |= static_cast<E>(static_cast<uint64_t>(w.z) << (32 * q));
        v[4 * j + 3] |= static_cast<E>(static_cast<uint64_t>(w.w) << (32 * q));
      }
  } else {
#pragma unroll
    for (int e = 0; e < EPT; ++e)
      v[e] = Planes<E>::get(buf, stride, swz(index_of<LOG2N, W>(lo_to, lane, e)));
  }
  if constexpr (P::kBlock) __syncthreads(); else __syncwarp();
}

// Shared-memory slot of twiddle i (layer L holds entries [n >> (L+1), n >> L)).
// The layers of the last phase (lo = 0) are read by group lane t at natural
// index (t << s) | g, s = K - L - 1: stored instead at g 2^LB + t, so a
// group's reads are consecutive (and the groups of a warp read the same
// words).  The other layers keep the natural order.
template <int LOG2N, int W>
__device__ __forceinline__ int twiddle_slot(int i) {
  using P = Phases<LOG2N, W>;
  constexpr int K = P::K;
  constexpr int top_last = P::top(P::count - 1);   // layers [0, top_last) run at lo = 0
  if (i == 0) return 0;
  const int lead = 31 - __clz(i);                  // n >> (L + 1) = 2^lead
  const int L = LOG2N - 1 - lead;
  if (L >= top_last) return i;
  const int s = K - L - 1;
  const int j = i - (1 << lead);
  return (1 << lead) + ((j & ((1 << s) - 1)) << P::LB) + (j >> s);
}

// All layers of bits [bottom, top) in phase layout lo; descending for the
// forward transform, ascending for the inverse.
template <class Op, int LOG2N, bool INV, bool LAZY>
__device__ __forceinline__ void phase_layers(
    typename Op::E (&v)[Phases<LOG2N, Planes<typename Op::E>::count>::EPT],
    const typename Tw<Op>::T* stw, int lane, int lo, int bottom, int top,
    const typename Op::C& c) {
  using E = typename Op::E;
  constexpr int W = Planes<E>::count;
  constexpr int n = 1 << LOG2N;
  constexpr int EPT = Phases<LOG2N, W>::EPT;
  constexpr int LB = Phases<LOG2N, W>::LB;
  const E N = static_cast<E>(c.N);
#pragma unroll
  for (int step = 0; step < LOG2N; ++step) {
    const int L = INV ? bottom + step : top - 1 - step;
    if (L < bottom || L >= top) continue;
    const int h = 1 << (L - lo);   // partner register distance
#pragma unroll
    for (int e = 0; e < EPT; ++e) {
      if ((e & h) == 0) {
        const int i = index_of<LOG2N, W>(lo, lane, e);
        const int k = lo == 0 ? (n >> (L + 1)) + ((e >> (L + 1)) << LB) + lane   // permuted layers
                              : (n >> (L + 1)) + (i >> (L + 1));
        butterfly<Op, INV, LAZY>(v[e], v[e + h], stw[k], c);
      }
    }
  }
}

template <class Op, int LOG2N, bool INV, bool LAZY>
__global__ void __launch_bounds__(256) ntt_phased_kernel(const typename Op::E* __restrict__ in,
                                                         typename Op::E* __restrict__ out,
                                                         size_t batch,
                                                         const typename Tw<Op>::T* __restrict__ tw,
                                                         const typename Tw<Op>::T scale,
                                                         const typename Op::C c) {
  using E = typename Op::E;
  using T = typename Tw<Op>::T;
  using P = Phases<LOG2N, Planes<E>::count>;
  constexpr int n = 1 << LOG2N;
  constexpr int EPT = P::EPT;
  constexpr int LB = P::LB;
  constexpr int group_words = P::group_words(Planes<E>::count);
  __shared__ T stw[n];
  extern __shared__ __align__(16) uint32_t dyn_buf[];
  for (int i = threadIdx.x; i < n; i += blockDim.x)
    stw[twiddle_slot<LOG2N, Planes<E>::count>(i)] = tw[i];
  __syncthreads();
  // blockDim.x = 256: the block holds 256 >> LB groups, group g = threads
  // [g 2^LB, (g + 1) 2^LB); the block walks its polynomials in lock step, so
  // block barriers between phases are reached by every thread alike
  const int grp = threadIdx.x >> LB;               // group (polynomial) within the block
  const int lane = threadIdx.x & ((1 << LB) - 1);  // lane within the group
  uint32_t* buf = dyn_buf + grp * group_words;
  const size_t first = static_cast<size_t>(blockIdx.x) * P::GPB;
  const size_t step = static_cast<size_t>(gridDim.x) * P::GPB;
  constexpr int last = P::count - 1;
  // When a lane's coefficients take at most 64 bytes, the group's next
  // polynomial loads while this one is transformed (measured 0-9% faster at
  // n = 256, 32 bits; at n = 1024, 64 bits the doubled registers cost 25%).
  // Every lane of the warp runs every round (the
  // transposes synchronise the warp); a group without a polynomial in the last
  // round computes on zeros and stores nothing.  Polynomials are private to
  // one group, so in-place calls are safe.
  constexpr bool kPrefetch = EPT * sizeof(E) <= 64;
  E nxt[EPT];
  // The lane-contiguous side (forward stores, inverse loads: EPT consecutive
  // elements per lane) moves as 128-bit accesses when the buffers allow it,
  // so each 32-byte sector is completed by one lane in at most two accesses.
  constexpr int VPE = 16 / static_cast<int>(sizeof(E));   // elements per 16-byte vector
  const bool vec = (EPT % VPE == 0) && ((reinterpret_cast<uintptr_t>(in) |
                                         reinterpret_cast<uintptr_t>(out)) % 16 == 0);
  auto load = [&](size_t p) {   // first layout: 2^LB e + lane (forward), EPT lane + e (inverse)
    const E* src = in + p * n;
    if (p >= batch) {
#pragma unroll
      for (int e = 0; e < EPT; ++e) nxt[e] = E{0};
    } else if (INV && vec) {
#pragma unroll
      for (int j = 0; j < EPT / VPE; ++j) {
        const uint4 w = reinterpret_cast<const uint4*>(src + lane * EPT)[j];
        const E* we = reinterpret_cast<const E*>(&w);
#pragma unroll
        for (int t = 0; t < VPE; ++t) nxt[j * VPE + t] = we[t];
      }
    } else {
#pragma unroll
      for (int e = 0; e < EPT; ++e) nxt[e] = INV ? src[lane * EPT + e] : src[(e << LB) + lane];
    }
  };
  if (kPrefetch && first < batch) load(first + grp);
  for (size_t base = first; base < batch; base += step) {
    const size_t p = base + grp;
    E v[EPT];
    if (!kPrefetch) load(p);
#pragma unroll
    for (int e = 0; e < EPT; ++e) v[e] = nxt[e];
    if (kPrefetch && base + step < batch) load(p + step);
    if constexpr (!INV) {
#pragma unroll
      for (int ph = 0; ph < P::count; ++ph) {
        if (ph > 0) transpose<E, LOG2N>(v, buf, lane, P::lo(ph - 1), P::lo(ph));
        phase_layers<Op, LOG2N, false, LAZY>(v, stw, lane, P::lo(ph), P::bottom(ph), P::top(ph), c);
      }
      if (p < batch) {
        E* dst = out + p * n + lane * EPT;                        // last layout: contiguous
#pragma unroll
        for (int e = 0; e < EPT; ++e) v[e] = LAZY ? canon3<E>(v[e], static_cast<E>(c.N)) : v[e];
        if (vec) {
#pragma unroll
          for (int j = 0; j < EPT / VPE; ++j) {
            uint4 w;
            E* we = reinterpret_cast<E*>(&w);
#pragma unroll
            for (int t = 0; t < VPE; ++t) we[t] = v[j * VPE + t];
            reinterpret_cast<uint4*>(dst)[j] = w;
          }
        } else {
#pragma unroll
          for (int e = 0; e < EPT; ++e) dst[e] = v[e];
        }
      }
    } else {
#pragma unroll
      for (int ph = last; ph >= 0; --ph) {
        if (ph < last) transpose<E, LOG2N>(v, buf, lane, P::lo(ph + 1), P::lo(ph));
        phase_layers<Op, LOG2N, true, LAZY>(v, stw, lane, P::lo(ph), P::bottom(ph), P::top(ph), c);
      }
      if (p < batch) {
        E* dst = out + p * n;
#pragma unroll
        for (int e = 0; e < EPT; ++e) dst[(e << LB) + lane] = Tw<Op>::mul(v[e], scale, c);
      }
    }
  }
}

// ------------------------------------------------------------ host tables

using u128h = unsigned __int128;

uint64_t mulmod(uint64_t a, uint64_t b, uint64_t N) {
  return static_cast<uint64_t>((static_cast<u128h>(a) * b) % N);
}
uint64_t powmod(uint64_t a, uint64_t e, uint64_t N) {
  uint64_t r = 1 % N;
  a %= N;
  while (e) {
    if (e & 1) r = mulmod(r, a, N);
    a = mulmod(a, a, N);
    e >>= 1;
  }
  return r;
}
uint32_t bitrev(uint32_t k, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) r = (r << 1) | ((k >> i) & 1u);
  return r;
}

template <class Op, int LOG2N, bool INV, bool LAZY>
cudaError_t launch_ntt(const void* in, void* out, size_t batch, const void* tw, const void* scale,
                       const typename Op::C& c, cudaStream_t s) {
  using T = typename Tw<Op>::T;
  using E = typename Op::E;
  const size_t warps_per_block = 8;
  const size_t want = (batch + warps_per_block - 1) / warps_per_block;
  if constexpr (LOG2N == 5) {   // one coefficient per lane: the shuffle kernel
    const void* k = reinterpret_cast<const void*>(ntt_kernel<Op, LOG2N, INV, LAZY>);
    const size_t cap = static_cast<size_t>(device_sm_count()) * resident_blocks(k, 256);
    ntt_kernel<Op, LOG2N, INV, LAZY><<<static_cast<unsigned>(want < cap ? want : cap), 256, 0, s>>>(
        static_cast<const E*>(in), static_cast<E*>(out), batch, static_cast<const T*>(tw),
        *static_cast<const T*>(scale), c);
  } else {
    auto kernel = ntt_phased_kernel<Op, LOG2N, INV, LAZY>;
    using P = Phases<LOG2N, Planes<E>::count>;
    const size_t want_blocks = (batch + P::GPB - 1) / P::GPB;
    const size_t smem = static_cast<size_t>(P::GPB) *
                        static_cast<size_t>(P::group_words(Planes<E>::count)) * sizeof(uint32_t);
    static bool attr_set = false;   // opt in above 48 KB once per process
    if (!attr_set) {
      cudaFuncSetAttribute(reinterpret_cast<const void*>(kernel),
                           cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
      attr_set = true;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
    const size_t cap = static_cast<size_t>(device_sm_count()) * per_sm;
    kernel<<<static_cast<unsigned>(want_blocks < cap ? want_blocks : cap), 256, smem, s>>>(
        static_cast<const E*>(in), static_cast<E*>(out), batch, static_cast<const T*>(tw),
        *static_cast<const T*>(scale), c);
  }
  return cudaGetLastError();
}

template <class Op, bool INV, bool LAZY = false>
cudaError_t launch_ntt_n(int log2n, const void* in, void* out, size_t batch, const void* tw,
                         const void* scale, const typename Op::C& c, cudaStream_t s) {
  switch (log2n) {
    case 5: return launch_ntt<Op, 5, INV, LAZY>(in, out, batch, tw, scale, c, s);
    case 6: return launch_ntt<Op, 6, INV, LAZY>(in, out, batch, tw, scale, c, s);
    case 7: return launch_ntt<Op, 7, INV, LAZY>(in, out, batch, tw, scale, c, s);
    case 8: return launch_ntt<Op, 8, INV, LAZY>(in, out, batch, tw, scale, c, s);
    case 9: return launch_ntt<Op, 9, INV, LAZY>(in, out, batch, tw, scale, c, s);
    default: return launch_ntt<Op, 10, INV, LAZY>(in, out, batch, tw, scale, c, s);
  }
}

// Lazy butterflies when the plan allows them (4N <= 2^w)
template <class Op, bool INV>
cudaError_t launch_lazy(bool lazy, int log2n, const void* in, void* out, size_t batch,
                        const void* tw, const void* scale, const typename Op::C& c,
                        cudaStream_t s) {
  return lazy ? launch_ntt_n<Op, INV, true>(log2n, in, out, batch, tw, scale, c, s)
              : launch_ntt_n<Op, INV, false>(log2n, in, out, batch, tw, scale, c, s);
}

}  // namespace
}  // namespace montgb

using namespace montgb;

struct mont_ntt {
  int variant = 0, width = 0, log2n = 0;
  WordConst32 w32{};
  WordConst64 w64{};
  void* d_tables = nullptr;   // forward table, inverse table
  size_t tw_bytes = 0;        // bytes of one table entry
  std::vector<unsigned char> scale;  // multiplier form of n^{-1}
  bool lazy = false;                 // 4N <= 2^w: lazy butterflies
};

extern "C" int mont_ntt_create(mont_ntt_t* out, mont_ctx_t ctx, int log2n, const uint32_t* psi_limbs) {
  if (!out || !ctx || !psi_limbs) return MONT_EINVAL;
  if (log2n < 5 || log2n > 10) return MONT_EINVAL;
  if (ctx->n_limbs > 2 || (ctx->variant != MONT_REDC && ctx->variant != MONT_PLANTARD))
    return MONT_EINVAL;
  const int n = 1 << log2n;
  const uint64_t N = ctx->n_limbs == 1 ? ctx->w32.N : ctx->w64.N;
  const uint64_t psi = ctx->n_limbs == 1 ? psi_limbs[0]
                                         : (static_cast<uint64_t>(psi_limbs[1]) << 32) | psi_limbs[0];
  if (psi == 0 || psi >= N) return MONT_EINVAL;
  if (powmod(psi, static_cast<uint64_t>(n), N) != N - 1) return MONT_EINVAL;  // psi^n = -1
  mont_ntt* p = new (std::nothrow) mont_ntt;
  if (!p) return MONT_ENOMEM;
  p->variant = ctx->variant;
  p->width = ctx->width;
  p->log2n = log2n;
  p->w32 = ctx->w32;
  p->w64 = ctx->w64;
  const bool plantard = ctx->variant == MONT_PLANTARD;
  p->lazy = static_cast<u128h>(4) * N <= (u128h{1} << ctx->width);
  const int w = ctx->width;
  p->tw_bytes = (plantard ? 2 : 1) * static_cast<size_t>(w / 8);
  // R mod N for R = 2^w (REDC) or 2^{2w} (Plantard)
  const uint64_t r1 = static_cast<uint64_t>((u128h{1} << w) % N);  // 2^w mod N
  const uint64_t Rmod = plantard ? mulmod(r1, r1, N) : r1;
  const u128h ninv2 = w == 32 ? static_cast<u128h>(ctx->w32.ninv2)
                              : (static_cast<u128h>(ctx->w64.ninv2_hi) << 64) | ctx->w64.ninv2_lo;
  // multiplier form of a residue x: x R mod N (REDC), or (-x R mod N) N^{-1} mod R (Plantard)
  auto form = [&](uint64_t x, unsigned char* dst) {
    uint64_t m = mulmod(x, Rmod, N);
    if (!plantard) {
      if (w == 32) { const uint32_t v = static_cast<uint32_t>(m); std::memcpy(dst, &v, 4); }
      else std::memcpy(dst, &m, 8);
      return;
    }
    m = m ? N - m : 0;
    if (w == 32) {
      const uint64_t b = m * static_cast<uint64_t>(ninv2);   // mod 2^64
      std::memcpy(dst, &b, 8);
    } else {
      const u128h b = static_cast<u128h>(m) * ninv2;         // mod 2^128
      std::memcpy(dst, &b, 16);
    }
  };
  std::vector<unsigned char> host(2 * n * p->tw_bytes);
  const uint64_t psi_inv = powmod(psi, 2 * static_cast<uint64_t>(n) - 1, N);   // psi^{2n-1} = psi^{-1}
  for (int k = 0; k < n; ++k) {
    const uint64_t e = bitrev(static_cast<uint32_t>(k), log2n);
    form(powmod(psi, e, N), &host[k * p->tw_bytes]);
    form(powmod(psi_inv, e, N), &host[(n + k) * p->tw_bytes]);
  }
  p->scale.resize(p->tw_bytes);
  // n^{-1} mod N (N odd): invert n = 2^log2n by halving 1 repeatedly
  uint64_t ninv_n = 1;
  for (int i = 0; i < log2n; ++i) ninv_n = (ninv_n & 1) ? static_cast<uint64_t>((static_cast<u128h>(ninv_n) + N) >> 1) : ninv_n >> 1;
  form(ninv_n, p->scale.data());
  cudaError_t e = cudaMalloc(&p->d_tables, host.size());
  if (e == cudaSuccess) e = cudaMemcpy(p->d_tables, host.data(), host.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    if (p->d_tables) cudaFree(p->d_tables);
    delete p;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MONT_ENOMEM : cuda_status(e);
  }
  *out = p;
  return MONT_OK;
}

extern "C" int mont_ntt_destroy(mont_ntt_t p) {
  if (!p) return MONT_OK;
  if (p->d_tables) cudaFree(p->d_tables);
  delete p;
  return MONT_OK;
}

static int ntt_run(mont_ntt_t p, const void* in, void* out, size_t batch, void* stream, bool inv) {
  if (!p) return MONT_EINVAL;
  if (batch == 0) return MONT_OK;
  if (!in || !out) return MONT_EINVAL;
  const size_t es = static_cast<size_t>(p->width / 8);
  const size_t bytes = batch << p->log2n;
  if (reinterpret_cast<uintptr_t>(in) % es || reinterpret_cast<uintptr_t>(out) % es) return MONT_EINVAL;
  const uintptr_t a = reinterpret_cast<uintptr_t>(in), b = reinterpret_cast<uintptr_t>(out);
  if (a != b && a < b + bytes * es && b < a + bytes * es) return MONT_EINVAL;
  const char* tw = static_cast<const char*>(p->d_tables) + (inv ? (size_t{1} << p->log2n) * p->tw_bytes : 0);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  const void* sc = p->scale.data();
  if (p->width == 32) {
    if (p->variant == MONT_REDC)
      e = inv ? launch_lazy<Redc32, true>(p->lazy, p->log2n, in, out, batch, tw, sc, p->w32, s)
              : launch_lazy<Redc32, false>(p->lazy, p->log2n, in, out, batch, tw, sc, p->w32, s);
    else
      e = inv ? launch_lazy<Plantard32, true>(p->lazy, p->log2n, in, out, batch, tw, sc, p->w32, s)
              : launch_lazy<Plantard32, false>(p->lazy, p->log2n, in, out, batch, tw, sc, p->w32, s);
  } else {
    if (p->variant == MONT_REDC)
      e = inv ? launch_lazy<Redc64, true>(p->lazy, p->log2n, in, out, batch, tw, sc, p->w64, s)
              : launch_lazy<Redc64, false>(p->lazy, p->log2n, in, out, batch, tw, sc, p->w64, s);
    else
      e = inv ? launch_lazy<Plantard64, true>(p->lazy, p->log2n, in, out, batch, tw, sc, p->w64, s)
              : launch_lazy<Plantard64, false>(p->lazy, p->log2n, in, out, batch, tw, sc, p->w64, s);
  }
  return cuda_status(e);
}

extern "C" int mont_ntt_forward(mont_ntt_t p, const void* in, void* out, size_t batch, void* stream) {
  return ntt_run(p, in, out, batch, stream, false);
}

extern "C" int mont_ntt_inverse(mont_ntt_t p, const void* in, void* out, size_t batch, void* stream) {
  return ntt_run(p, in, out, batch, stream, true);
}
