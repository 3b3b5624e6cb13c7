// Algorithms 1-4 at multi-limb widths.
//
// The paper states Algorithm 1 for R = 2^n and the Plantard family
// (Algorithms 2-4) for R = 2^{2n}, for any word size n.  For a modulus of k
// 32-bit limbs the library takes n = 32k: Algorithm 1 works modulo
// R = 2^{32k}, Algorithms 2-4 modulo R = 2^{64k}.  Signed elements are k-limb
// two's complement integers.  Every step is exact limb arithmetic:
//
//   Algorithm 1  m = (T mod R) N^{-1} mods R                 (low k limbs)
//                r = (T >> n) - ((m N) >> n)                  in (-N, N)
//   Algorithm 2  m = T N^{-1} mod 2^{2n}                      (low 2k limbs)
//                r = (((m >> n) + 1) N) >> n                  in [0, N)
//   Algorithm 3  m = (int_{2n})(T N^{-1}),  q = (m + 2^{n-1}) >> n,
//                r = (q N + 2^{n-1}) >> n                     mods N
//   Algorithm 4  m = (int_{2n})(T N^{-1}),
//                r = (((m >> n) + 2^alpha) N) >> n            mods N (alpha >= 1)
//
// Shifts of signed values are arithmetic.  A product with a signed factor
// is formed as the unsigned product of the two's complement limbs, then
// corrected: a factor x < 0 stands for x + 2^{32j} (j its limbs), so the
// other factor times 2^{32j} is subtracted from the limbs it reaches.
//
// One thread per element, grid-stride.  Up to k = 16 the loops are fully
// unrolled and an element's state lives in registers; at k = 32 and 64 it
// lives in local memory and the products run over 16 x 16-limb register
// blocks.  The variant and the operation are uniform run-time branches: one
// kernel per limb count.
#include "internal.h"

namespace montgb {
namespace {

constexpr int unroll_for(int k) { return k <= 16 ? 128 : 1; }

// (a0, a1, a2) += x y: a 96-bit column accumulator, in one asm statement so
// that nothing can clobber the carry flag between the steps.
__device__ __forceinline__ void mac96(uint32_t (&acc)[3], uint32_t x, uint32_t y) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2])
      : "r"(x), "r"(y));
}

// (a0, a1, a2) += (x0, x1) 96-bit.
__device__ __forceinline__ void add64_96(uint32_t (&acc)[3], uint32_t x0, uint32_t x1) {
  asm("add.cc.u32 %0, %0, %3;\n\t"
      "addc.cc.u32 %1, %1, %4;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2])
      : "r"(x0), "r"(x1));
}

// (a0, a1, a2) += x, x one word.
__device__ __forceinline__ void add32_96(uint32_t (&acc)[3], uint32_t x) {
  asm("add.cc.u32 %0, %0, %3;\n\t"
      "addc.cc.u32 %1, %1, 0;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(acc[0]), "+r"(acc[1]), "+r"(acc[2])
      : "r"(x));
}

constexpr int kBlk = 16;   // limbs per register block of the local-memory products

// One 16 x 16-limb block product, accumulated: with
//   v = o[0, 16) (0 unless has_old) + hi + 2^512 (tc1:tc0) + ra rb,
// o[0, 16) <- v mod 2^512, hi <- (v >> 512) mod 2^512, (tc1:tc0) <- v >> 1024.
// Columns are summed in 96-bit accumulators (even and odd limbs of ra apart).
// LOW_ONLY: only the low 16 columns (a truncated product's top block).
template <bool LOW_ONLY>
__device__ __forceinline__ void block_mac(const uint32_t (&ra)[kBlk], const uint32_t (&rb)[kBlk],
                                          uint32_t* o, bool has_old, uint32_t (&hi)[kBlk],
                                          uint32_t& tc0, uint32_t& tc1) {
  uint32_t carry0 = 0, carry1 = 0;
#pragma unroll
  for (int col = 0; col < (LOW_ONLY ? kBlk : 2 * kBlk); ++col) {
    uint32_t s0[3] = {carry0, carry1, 0u}, s1[3] = {0u, 0u, 0u};
    if (col < kBlk) {
      s1[0] = hi[col];
      if (has_old) add32_96(s0, o[col]);
    } else if (col == kBlk) {
      s1[0] = tc0;
      s1[1] = tc1;
    }
#pragma unroll
    for (int i = 0; i < kBlk; ++i) {
      const int j = col - i;
      if (j >= 0 && j < kBlk) {
        if (i & 1) mac96(s1, ra[i], rb[j]);
        else mac96(s0, ra[i], rb[j]);
      }
    }
    add64_96(s0, s1[0], s1[1]);
    if (col < kBlk) o[col] = s0[0];
    else hi[col - kBlk] = s0[0];
    carry0 = s0[1];
    carry1 = s0[2] + s1[2];   // a column total stays below 2^69: no overflow
  }
  if (!LOW_ONLY) {
    tc0 = carry0;
    tc1 = carry1;
  }
}

// out[0, M) = (a[0, KA) * b[0, KB)) mod 2^{32M} for the limb counts whose
// arrays live in local memory (k >= 32): schoolbook over 16 x 16-limb
// blocks, each block product formed by product scanning in registers.  Row I
// of blocks (a's block I against every block of b) carries the high half of
// each block product into the next block in registers, so a block costs 16
// operand loads and 16 loads and stores of the result for 256 limb products.
// Row I accumulates into blocks I .. I+NB-1, which row I-1 has written, and
// writes block I+NB first; the row's running sum is below 2^{512(I+1+NB)},
// so nothing carries past that block.
template <int KA, int KB, int M>
__device__ __noinline__ void mul_blocked(const uint32_t* a, const uint32_t* b, uint32_t* out) {
  static_assert(KA % kBlk == 0 && KB % kBlk == 0 && M % kBlk == 0 && M <= KA + KB,
                "block shapes");
  constexpr int NA = KA / kBlk, NB = KB / kBlk, NM = M / kBlk;
  for (int I = 0; I < NA && I < NM; ++I) {
    uint32_t ra[kBlk], hi[kBlk];
#pragma unroll
    for (int t = 0; t < kBlk; ++t) {
      ra[t] = a[kBlk * I + t];
      hi[t] = 0u;
    }
    uint32_t tc0 = 0, tc1 = 0;
    const bool has_old = I > 0;
    for (int J = 0; J < NB && I + J < NM; ++J) {
      uint32_t rb[kBlk];
#pragma unroll
      for (int t = 0; t < kBlk; ++t) rb[t] = b[kBlk * J + t];
      uint32_t* o = out + kBlk * (I + J);
      if (I + J == NM - 1) block_mac<true>(ra, rb, o, has_old, hi, tc0, tc1);
      else block_mac<false>(ra, rb, o, has_old, hi, tc0, tc1);
    }
    if (I + NB < NM) {
#pragma unroll
      for (int t = 0; t < kBlk; ++t) out[kBlk * (I + NB) + t] = hi[t];
    }
  }
}

// The same product scanning fully unrolled, for operands in registers
// (k <= 16): two accumulators per column (even and odd a-limbs) so that the
// carry chains of a column can interleave.
template <int KA, int KB, int M>
__device__ __forceinline__ void mul_scan_reg(const uint32_t* a, const uint32_t* b, uint32_t* out) {
  uint32_t carry0 = 0, carry1 = 0;
#pragma unroll
  for (int c = 0; c < M; ++c) {
    uint32_t s0[3] = {carry0, carry1, 0u}, s1[3] = {0u, 0u, 0u};
#pragma unroll
    for (int i = 0; i < KA; ++i) {
      const int j = c - i;
      if (j >= 0 && j < KB) {
        if (i & 1) mac96(s1, a[i], b[j]);
        else mac96(s0, a[i], b[j]);
      }
    }
    add64_96(s0, s1[0], s1[1]);
    out[c] = s0[0];
    carry0 = s0[1];
    carry1 = s0[2] + s1[2];   // the column total stays below 2^64 + its carry: no overflow
  }
}

// out[0, KA+KB) = a[0, KA) * b[0, KB), unsigned.
template <int K, int KA, int KB>
__device__ __forceinline__ void mul_full(const uint32_t* a, const uint32_t* b, uint32_t* out) {
  if constexpr (K > 16) {
    mul_blocked<KA, KB, KA + KB>(a, b, out);
  } else {
    mul_scan_reg<KA, KB, KA + KB>(a, b, out);
  }
}

// out[0, M) = (a[0, KA) * b[0, KB)) mod 2^{32M}, unsigned.
template <int K, int KA, int KB, int M>
__device__ __forceinline__ void mul_low(const uint32_t* a, const uint32_t* b, uint32_t* out) {
  if constexpr (K > 16) {
    mul_blocked<KA, KB, M>(a, b, out);
  } else {
    mul_scan_reg<KA, KB, M>(a, b, out);
  }
}

// x[0, L) -= (y[0, L) & mask), modulo 2^{32L}.
template <int K, int L>
__device__ __forceinline__ void sub_masked(uint32_t* x, const uint32_t* y, uint32_t mask) {
  constexpr int U = unroll_for(K);
  uint32_t borrow = 0;
#pragma unroll U
  for (int i = 0; i < L; ++i) {
    const uint64_t d = static_cast<uint64_t>(x[i]) - (y[i] & mask) - borrow;
    x[i] = static_cast<uint32_t>(d);
    borrow = static_cast<uint32_t>(d >> 32) & 1u;
  }
}

// x[0, L) += (y[0, L) & mask), modulo 2^{32L}.
template <int K, int L>
__device__ __forceinline__ void add_masked(uint32_t* x, const uint32_t* y, uint32_t mask) {
  constexpr int U = unroll_for(K);
  uint32_t carry = 0;
#pragma unroll U
  for (int i = 0; i < L; ++i) {
    const uint64_t s = static_cast<uint64_t>(x[i]) + (y[i] & mask) + carry;
    x[i] = static_cast<uint32_t>(s);
    carry = static_cast<uint32_t>(s >> 32);
  }
}

// x[0, L) -= (y[0, L) & my) + (z[0, L) & mz), modulo 2^{32L}.
template <int K, int L>
__device__ __forceinline__ void sub2_masked(uint32_t* x, const uint32_t* y, uint32_t my,
                                            const uint32_t* z, uint32_t mz) {
  constexpr int U = unroll_for(K);
  uint32_t borrow = 0;   // 0, 1 or 2
#pragma unroll U
  for (int i = 0; i < L; ++i) {
    const int64_t d = static_cast<int64_t>(x[i]) - (y[i] & my) - (z[i] & mz) - borrow;
    x[i] = static_cast<uint32_t>(d);
    borrow = static_cast<uint32_t>(-(d >> 32));   // d >= -2^33: d >> 32 in {-2, -1, 0}
  }
}

// x[0, L) += 2^bit, modulo 2^{32L} (bit < 32 L).
template <int K, int L>
__device__ __forceinline__ void add_pow2(uint32_t* x, int bit) {
  constexpr int U = unroll_for(K);
  const int limb = bit >> 5;
  uint32_t carry = 0;
#pragma unroll U
  for (int i = 0; i < L; ++i) {
    const uint32_t add = (i == limb ? (1u << (bit & 31)) : 0u) + carry;
    const uint32_t s = x[i] + add;
    carry = s < add ? 1u : 0u;
    x[i] = s;
  }
}

__device__ __forceinline__ uint32_t sign_mask(uint32_t top) { return 0u - (top >> 31); }

// The steps of one element use two buffers of local state, reused in turn:
//   X (2K+1 limbs): T, then the product whose high half is r
//   Y (3K+1 limbs): the operands a | b, then m (and Algorithm 1's m N)
// so an element holds 5K+2 limbs whatever the algorithm.  No product below
// writes a buffer it reads.

// Algorithm 1 at R = 2^{32K}: T in X (2K limbs, two's complement) -> r in
// X[K, 2K).
template <int K>
__device__ __forceinline__ void sig_redc(uint32_t* X, uint32_t* Y, const LimbVarConst& c) {
  uint32_t* m = Y;                              // K limbs
  uint32_t* P = Y + K;                          // 2K limbs
  mul_low<K, K, K, K>(X, c.ninv, m);            // m = (T mod R) N^{-1} mod R; signed view = mods R
  mul_full<K, K, K>(m, c.N, P);                 // (m mod R) N
  const uint32_t m_neg = sign_mask(m[K - 1]);
  sub_masked<K, K>(X + K, P + K, 0xFFFFFFFFu);  // (T >> n) - ((m mod R) N >> n)
  add_masked<K, K>(X + K, c.N, m_neg);          // m < 0: (m N) >> n = ((m mod R) N >> n) - N
}

// m = T N^{-1} mod 2^{64K} (low 2K limbs) for the Plantard family: T in X,
// m in Y[0, 2K).
template <int K>
__device__ __forceinline__ void plantard_m(const uint32_t* X, const LimbVarConst& c, uint32_t* Y) {
  mul_low<K, 2 * K, 2 * K, 2 * K>(X, c.ninv, Y);
}

// r = (q N) >> n with q signed of K+1 limbs (Y[K, 2K]), plus 2^{n-1} before
// the shift when round_half is set.  The product is formed in X (2K+1 limbs;
// T is no longer needed) and r is X[K, 2K).
template <int K>
__device__ __forceinline__ void shifted_product(const uint32_t* q, const LimbVarConst& c,
                                                bool round_half, uint32_t* X) {
  uint32_t* P = X;
  if constexpr (K > 16) {
    // the blocked product takes whole blocks: q's low K limbs times N, then
    // the row q_K N 2^{32K} (q_K is 0, 1 or 2^32 - 1)
    mul_full<K, K, K>(q, c.N, P);
    uint32_t carry = 0;
#pragma unroll 1
    for (int j = 0; j < K; ++j) {
      const uint64_t t = static_cast<uint64_t>(q[K]) * c.N[j] + P[K + j] + carry;
      P[K + j] = static_cast<uint32_t>(t);
      carry = static_cast<uint32_t>(t >> 32);
    }
    P[2 * K] = carry;
  } else {
    mul_full<K, K + 1, K>(q, c.N, P);
  }
  // q < 0 stands for q + 2^{32(K+1)}: remove N 2^{32(K+1)} from limbs K+1..2K
  sub_masked<K, K>(P + K + 1, c.N, sign_mask(q[K]));
  if (round_half) add_pow2<K, K + 2>(P + K - 1, 31);   // + 2^{32K-1}: limbs K-1 .. 2K
}

// Algorithm 2 at R = 2^{64K}: T in X -> r in X[K, 2K).
template <int K>
__device__ __forceinline__ void p_redc(uint32_t* X, uint32_t* Y, const LimbVarConst& c) {
  constexpr int U = unroll_for(K);
  plantard_m<K>(X, c, Y);
  uint32_t* q = Y + K;                          // (m >> n) + 1, unsigned, in place over m's high half
  uint32_t carry = 1;
#pragma unroll U
  for (int i = 0; i < K; ++i) {
    const uint32_t s = q[i] + carry;
    carry = s < carry ? 1u : 0u;
    q[i] = s;
  }
  q[K] = carry;
  shifted_product<K>(q, c, false, X);           // q >= 0: no sign correction applies
}

// Algorithms 3 and 4 at R = 2^{64K}: T in X -> r in X[K, 2K).
template <int K>
__device__ __forceinline__ void sig_p_redc(uint32_t* X, uint32_t* Y, const LimbVarConst& c) {
  constexpr int U = unroll_for(K);
  plantard_m<K>(X, c, Y);                       // two's complement view = (int_{2n})(T N^{-1})
  uint32_t* q = Y + K;                          // in place over m's high half, one limb above
  const uint32_t m_sign = sign_mask(Y[2 * K - 1]);
  if (c.variant == MONT_SIGNED_PLANTARD) {
    // q = (m + 2^{n-1}) >> n on 2K+1 limbs: add 2^31 to limb K-1, carry upward
    uint32_t carry = (Y[K - 1] + 0x80000000u) < Y[K - 1] ? 1u : 0u;
#pragma unroll U
    for (int i = 0; i < K; ++i) {
      const uint32_t s = q[i] + carry;
      carry = s < carry ? 1u : 0u;
      q[i] = s;
    }
    q[K] = m_sign + carry;
    shifted_product<K>(q, c, true, X);
  } else {
    // q = (m >> n) + 2^alpha on K+1 limbs
    q[K] = m_sign;
    add_pow2<K, K + 1>(q, c.alpha);
    shifted_product<K>(q, c, false, X);
  }
}

template <int C>
__device__ __forceinline__ void load_limbs(const uint32_t* p, uint32_t* v, int vec16) {
  constexpr int U = unroll_for(C / 2);
  if (C % 4 == 0 && vec16) {
#pragma unroll U
    for (int q = 0; q < C / 4; ++q) {
      const uint4 u = reinterpret_cast<const uint4*>(p)[q];
      v[4 * q] = u.x;
      v[4 * q + 1] = u.y;
      v[4 * q + 2] = u.z;
      v[4 * q + 3] = u.w;
    }
  } else {
#pragma unroll U
    for (int i = 0; i < C; ++i) v[i] = p[i];
  }
}

template <int K>
__device__ __forceinline__ void store_limbs(uint32_t* p, const uint32_t* v, int vec16) {
  constexpr int U = unroll_for(K);
  if (K % 4 == 0 && vec16) {
#pragma unroll U
    for (int q = 0; q < K / 4; ++q)
      reinterpret_cast<uint4*>(p)[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
  } else {
#pragma unroll U
    for (int i = 0; i < K; ++i) p[i] = v[i];
  }
}

template <int K>
__global__ void __launch_bounds__(256) limb_variant_kernel(const uint32_t* __restrict__ x,
                                                           const uint32_t* __restrict__ y,
                                                           uint32_t* __restrict__ out, size_t n,
                                                           int mode, int vec16,
                                                           const LimbVarConst c) {
  constexpr int U = unroll_for(K);
  const bool is_signed = c.variant != MONT_PLANTARD;
  const size_t stride = static_cast<size_t>(gridDim.x) * blockDim.x;
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n; e += stride) {
    uint32_t X[2 * K + 1], Y[3 * K + 1];
    if (mode == static_cast<int>(Mode::kRedc)) {
      load_limbs<2 * K>(x + e * 2 * K, X, vec16);
    } else {
      uint32_t* a = Y;
      uint32_t* b = Y + K;
      load_limbs<K>(x + e * K, a, vec16);
      if (mode == static_cast<int>(Mode::kFromDomain)) {
        const uint32_t ext = is_signed ? sign_mask(a[K - 1]) : 0u;
#pragma unroll U
        for (int i = 0; i < K; ++i) {
          X[i] = a[i];
          X[K + i] = ext;
        }
      } else {
        if (mode == static_cast<int>(Mode::kMul)) {
          load_limbs<K>(y + e * K, b, vec16);
        } else {
#pragma unroll U
          for (int i = 0; i < K; ++i) b[i] = c.dom[i];
        }
        mul_full<K, K, K>(a, b, X);
        if (is_signed)                          // T mod 2^{64K} of the signed product
          sub2_masked<K, K>(X + K, b, sign_mask(a[K - 1]), a, sign_mask(b[K - 1]));
      }
    }
    uint32_t* r = X + K;
    if (c.variant == MONT_SIGNED) {
      sig_redc<K>(X, Y, c);
      if (mode == static_cast<int>(Mode::kFromDomain)) {
        // (-N, N) -> mods N: r > (N-1)/2 gives r - N, r < -(N-1)/2 gives r + N
        uint32_t* t = Y;                        // m and m N are no longer needed
#pragma unroll U
        for (int i = 0; i < K; ++i) t[i] = c.half[i];
        sub_masked<K, K>(t, r, 0xFFFFFFFFu);    // (N-1)/2 - r
        const uint32_t above = sign_mask(t[K - 1]);
#pragma unroll U
        for (int i = 0; i < K; ++i) t[i] = r[i];
        add_masked<K, K>(t, c.half, 0xFFFFFFFFu);   // r + (N-1)/2
        const uint32_t below = sign_mask(t[K - 1]);
        sub_masked<K, K>(r, c.N, above);
        add_masked<K, K>(r, c.N, below);
      }
    } else if (c.variant == MONT_PLANTARD) {
      p_redc<K>(X, Y, c);
    } else {
      sig_p_redc<K>(X, Y, c);
    }
    store_limbs<K>(out + e * K, r, vec16);
  }
}

// Launch shape from the tuning table (threads 128 or 256, resident blocks
// per SM; 0 = the occupancy limit).  At k >= 32 fewer resident blocks, to keep
// the local-memory arrays in L1, measured slower at every setting.
template <int K>
cudaError_t launch_k(Mode mode, const LimbVarConst& c, const uint32_t* x, const uint32_t* y,
                     uint32_t* o, size_t n, cudaStream_t s, int vec16, const LaunchShape& shape) {
  const void* kern = reinterpret_cast<const void*>(limb_variant_kernel<K>);
  const int threads =
      shape.threads == 32 || shape.threads == 64 || shape.threads == 256 ? shape.threads : 128;
  int per_sm = resident_blocks(kern, threads);
  if (shape.blocks_per_sm > 0 && shape.blocks_per_sm < per_sm) per_sm = shape.blocks_per_sm;
  const size_t want = (n + threads - 1) / threads;
  const size_t grid = static_cast<size_t>(device_sm_count()) * (per_sm > 0 ? per_sm : 1);
  limb_variant_kernel<K><<<static_cast<unsigned>(want < grid ? want : grid), threads, 0, s>>>(
      x, y, o, n, static_cast<int>(mode), vec16, c);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_limb_variant(int k, Mode mode, const LimbVarConst& c, const uint32_t* x,
                                const uint32_t* y, uint32_t* o, size_t n, cudaStream_t s,
                                int vec16, const LaunchShape& shape) {
  switch (k) {
    case 4: return launch_k<4>(mode, c, x, y, o, n, s, vec16, shape);
    case 8: return launch_k<8>(mode, c, x, y, o, n, s, vec16, shape);
    case 12: return launch_k<12>(mode, c, x, y, o, n, s, vec16, shape);
    case 16: return launch_k<16>(mode, c, x, y, o, n, s, vec16, shape);
    case 32: return launch_k<32>(mode, c, x, y, o, n, s, vec16, shape);
    case 64: return launch_k<64>(mode, c, x, y, o, n, s, vec16, shape);
  }
  return cudaErrorInvalidConfiguration;
}

}  // namespace montgb
