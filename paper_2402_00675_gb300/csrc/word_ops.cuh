// Word-size Montgomery-type reductions as device functions, one struct per
// (word width, variant).  Each struct gives
//   E        the element type (unsigned for REDC/Plantard, signed otherwise),
//   TT       the double-width product type,
//   mul      T = a b in TT,
//   widen    T = y (sign- or zero-extension),
//   reduce   the paper's reduction of T, in word arithmetic,
//   canon    the canonical residue of a reduction output (mont_from_domain).
//
// The word-level steps evaluate exactly the paper's formulas for every T in
// the algorithm's input domain; the comments give the bound that keeps each
// intermediate inside its register.
#pragma once

#include <cstdint>
#include <type_traits>

#include "internal.h"

namespace montgb {

// Every variant without a prepared form (REDC, Algorithm 1: the fixed-
// multiplier trick of Section 3.2 is Plantard's) reports kHasPre = false.
template <class Op, class = void>
struct HasPre { static constexpr bool value = false; };
template <class Op>
struct HasPre<Op, std::void_t<decltype(Op::kHasPre)>> { static constexpr bool value = Op::kHasPre; };

// (a sign-extended to 64 bits) * b' mod 2^64 from 32-bit products: the low
// word of a times b' plus the correction -b'_lo 2^32 when a < 0.
__device__ __forceinline__ uint64_t signed_times_prepared32(int32_t a, uint64_t bp) {
  const uint32_t ua = static_cast<uint32_t>(a);
  const uint32_t blo = static_cast<uint32_t>(bp), bhi = static_cast<uint32_t>(bp >> 32);
  const uint32_t lo = ua * blo;
  const uint32_t hi = __umulhi(ua, blo) + ua * bhi - (a < 0 ? blo : 0u);
  return (static_cast<uint64_t>(hi) << 32) | lo;
}

// ---------------------------------------------------------------------------
// 32-bit words.  REDC and Algorithm 1 use R = 2^32; the Plantard family uses
// R = 2^64 = 2^{2n} with n = 32.
// ---------------------------------------------------------------------------

// REDC (Section 1): m = (T mod R) N' mod R; t = (T + mN)/R; one subtraction.
struct Redc32 {
  using E = uint32_t;
  using TT = uint64_t;
  using C = WordConst32;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<uint64_t>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint32_t lo = static_cast<uint32_t>(T);
    const uint32_t hi = static_cast<uint32_t>(T >> 32);
    const uint32_t m = lo * c.nprime;                 // (T mod R) N' mod R
    const uint32_t mn_hi = __umulhi(m, c.N);
    // lo(T) + lo(mN) = 0 mod 2^32, so it carries exactly when lo(T) != 0.
    // t = (T + mN) / R < 2N may need 33 bits when N > 2^31.
    const uint64_t t = static_cast<uint64_t>(hi) + mn_hi + (lo != 0u);
    return static_cast<uint32_t>(t >= c.N ? t - c.N : t);
  }
  static __device__ __forceinline__ E canon(E r, const C&) { return r; }
};

// Algorithm 1 (SigRedc): T = a1 R + a0, m0 = a0 N^{-1} mods R,
// t = floor(m0 N / R), r = a1 - t.
struct Signed32 {
  using E = int32_t;
  using TT = int64_t;
  using C = WordConst32;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<int64_t>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint32_t a0 = static_cast<uint32_t>(T);             // 0 <= a0 < R
    const int32_t a1 = static_cast<int32_t>(T >> 32);          // floor(T / R)
    const int32_t m0 = static_cast<int32_t>(a0 * c.ninv);      // two's complement = mods R
    const int32_t t = __mulhi(m0, static_cast<int32_t>(c.N)); // floor(m0 N / 2^32); 2N < R
    return a1 - t;
  }
  static __device__ __forceinline__ E canon(E r, const C& c) {
    const int32_t h = static_cast<int32_t>(c.half);
    const int32_t N = static_cast<int32_t>(c.N);
    return r > h ? r - N : (r < -h ? r + N : r);
  }
};

// Algorithm 2 (PRedc), R = 2^64: r = floor((floor((T N^{-1} mod R)/2^32) + 1) N / 2^32).
// The paper's final "if r = N" test is omitted: the Remark after Algorithm 2
// shows r < N whenever N < 2^32/phi and 0 <= T <= N^2.
struct Plantard32 {
  using E = uint32_t;
  using TT = uint64_t;
  using C = WordConst32;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<uint64_t>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint64_t m = T * c.ninv2;                       // T N^{-1} mod 2^64
    const uint32_t q = static_cast<uint32_t>(m >> 32);    // floor(m / 2^n)
    // (q + 1) N <= 2^32 N < 2^64
    const uint64_t p = static_cast<uint64_t>(q) * c.N + c.N;
    return static_cast<uint32_t>(p >> 32);
  }
  static __device__ __forceinline__ E canon(E r, const C&) { return r; }
  // Section 3.2's fixed multiplier: b' = b N^{-1} mod 2^64, then only
  // floor((a b' mod 2^64) / 2^32) is needed, two 32-bit products.
  static constexpr bool kHasPre = true;
  static __device__ __forceinline__ TT prepare(E b, const C& c) { return static_cast<uint64_t>(b) * c.ninv2; }
  static __device__ __forceinline__ E mul_pre(E a, TT bp, const C& c) {
    const uint32_t q = __umulhi(a, static_cast<uint32_t>(bp)) + a * static_cast<uint32_t>(bp >> 32);
    const uint64_t p = static_cast<uint64_t>(q) * c.N + c.N;
    return static_cast<uint32_t>(p >> 32);
  }
};

// Algorithm 3 (SigPRedc1), R = 2^64:
// r = round(round((T Ñ^{-1} mods R)/2^32) N / 2^32), rounding half up.
struct SignedPlantard32 {
  using E = int32_t;
  using TT = int64_t;
  using C = WordConst32;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<int64_t>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint64_t m = static_cast<uint64_t>(T) * c.ninv2;   // bits of T Ñ^{-1} mods 2^64
    // floor(m/2^32 + 1/2) = floor(m/2^32) + bit 31 of m; may equal 2^31, so 64-bit.
    const int64_t q = static_cast<int64_t>(static_cast<int32_t>(m >> 32)) +
                      static_cast<int64_t>((m >> 31) & 1u);
    // |q N| <= 2^31 * 2^31
    const int64_t p = q * static_cast<int64_t>(c.N) + (int64_t{1} << 31);
    return static_cast<int32_t>(p >> 32);
  }
  static __device__ __forceinline__ E canon(E r, const C&) { return r; }
  static constexpr bool kHasPre = true;
  static __device__ __forceinline__ TT prepare(E b, const C& c) {
    return static_cast<int64_t>(static_cast<uint64_t>(static_cast<int64_t>(b)) * c.ninv2);
  }
  static __device__ __forceinline__ E mul_pre(E a, TT bp, const C& c) {
    const uint64_t m = signed_times_prepared32(a, static_cast<uint64_t>(bp));
    const int64_t q = static_cast<int64_t>(static_cast<int32_t>(m >> 32)) +
                      static_cast<int64_t>((m >> 31) & 1u);
    const int64_t p = q * static_cast<int64_t>(c.N) + (int64_t{1} << 31);
    return static_cast<int32_t>(p >> 32);
  }
};

// Algorithm 4 (SigPRedc2), R = 2^64: r = floor((floor((T Ñ^{-1} mods R)/2^32) + 2^alpha) N / 2^32).
struct SignedPlantard2_32 {
  using E = int32_t;
  using TT = int64_t;
  using C = WordConst32;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<int64_t>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint64_t m = static_cast<uint64_t>(T) * c.ninv2;
    const int64_t q = static_cast<int64_t>(static_cast<int32_t>(m >> 32)) +
                      (int64_t{1} << c.alpha);
    // N < 2^{31-alpha}, |q| <= 2^31 + 2^alpha
    return static_cast<int32_t>((q * static_cast<int64_t>(c.N)) >> 32);
  }
  static __device__ __forceinline__ E canon(E r, const C&) { return r; }
  static constexpr bool kHasPre = true;
  static __device__ __forceinline__ TT prepare(E b, const C& c) {
    return static_cast<int64_t>(static_cast<uint64_t>(static_cast<int64_t>(b)) * c.ninv2);
  }
  static __device__ __forceinline__ E mul_pre(E a, TT bp, const C& c) {
    const uint64_t m = signed_times_prepared32(a, static_cast<uint64_t>(bp));
    const int64_t q = static_cast<int64_t>(static_cast<int32_t>(m >> 32)) + (int64_t{1} << c.alpha);
    return static_cast<int32_t>((q * static_cast<int64_t>(c.N)) >> 32);
  }
};

// ---------------------------------------------------------------------------
// 64-bit words.  REDC and Algorithm 1 use R = 2^64; the Plantard family uses
// R = 2^128 (n = 64).
// ---------------------------------------------------------------------------

using u128 = unsigned __int128;
using i128 = __int128;

struct Redc64 {
  using E = uint64_t;
  using TT = u128;
  using C = WordConst64;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<u128>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint64_t lo = static_cast<uint64_t>(T);
    const uint64_t hi = static_cast<uint64_t>(T >> 64);
    const uint64_t m = lo * c.nprime;
    const uint64_t mn_hi = __umul64hi(m, c.N);
    const u128 t = static_cast<u128>(hi) + mn_hi + (lo != 0u);   // < 2N, up to 65 bits
    return static_cast<uint64_t>(t >= c.N ? t - c.N : t);
  }
  static __device__ __forceinline__ E canon(E r, const C&) { return r; }
};

struct Signed64 {
  using E = int64_t;
  using TT = i128;
  using C = WordConst64;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<i128>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint64_t a0 = static_cast<uint64_t>(T);
    const int64_t a1 = static_cast<int64_t>(T >> 64);
    const int64_t m0 = static_cast<int64_t>(a0 * c.ninv);
    const int64_t t = __mul64hi(m0, static_cast<int64_t>(c.N));
    return a1 - t;
  }
  static __device__ __forceinline__ E canon(E r, const C& c) {
    const int64_t h = static_cast<int64_t>(c.half);
    const int64_t N = static_cast<int64_t>(c.N);
    return r > h ? r - N : (r < -h ? r + N : r);
  }
};

// High word (bits 64..127) of T N^{-1} mod 2^128.
__device__ __forceinline__ uint64_t plantard_m_hi(uint64_t Tl, uint64_t Th, const WordConst64& c) {
  return __umul64hi(Tl, c.ninv2_lo) + Tl * c.ninv2_hi + Th * c.ninv2_lo;
}

struct Plantard64 {
  using E = uint64_t;
  using TT = u128;
  using C = WordConst64;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<u128>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint64_t q = plantard_m_hi(static_cast<uint64_t>(T), static_cast<uint64_t>(T >> 64), c);
    const u128 p = static_cast<u128>(q) * c.N + c.N;      // (q + 1) N < 2^128
    return static_cast<uint64_t>(p >> 64);
  }
  static __device__ __forceinline__ E canon(E r, const C&) { return r; }
  static constexpr bool kHasPre = true;
  static __device__ __forceinline__ TT prepare(E b, const C& c) {   // b N^{-1} mod 2^128
    const u128 ninv = (static_cast<u128>(c.ninv2_hi) << 64) | c.ninv2_lo;
    return static_cast<u128>(b) * ninv;
  }
  static __device__ __forceinline__ E mul_pre(E a, TT bp, const C& c) {
    const uint64_t blo = static_cast<uint64_t>(bp), bhi = static_cast<uint64_t>(bp >> 64);
    const uint64_t q = __umul64hi(a, blo) + a * bhi;
    const u128 p = static_cast<u128>(q) * c.N + c.N;
    return static_cast<uint64_t>(p >> 64);
  }
};

struct SignedPlantard64 {
  using E = int64_t;
  using TT = i128;
  using C = WordConst64;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<i128>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint64_t Tl = static_cast<uint64_t>(T);
    const uint64_t Th = static_cast<uint64_t>(static_cast<u128>(T) >> 64);
    const uint64_t ml = Tl * c.ninv2_lo;                       // bits 0..63 of m
    const int64_t mh = static_cast<int64_t>(plantard_m_hi(Tl, Th, c));  // floor(m / 2^64)
    // q = mh + bit 63 of m may be 2^63: keep the extra N in 128-bit arithmetic
    const i128 p = static_cast<i128>(mh) * static_cast<int64_t>(c.N) +
                   ((ml >> 63) ? static_cast<i128>(c.N) : i128{0}) + (i128{1} << 63);
    return static_cast<int64_t>(p >> 64);
  }
  static __device__ __forceinline__ E canon(E r, const C&) { return r; }
  static constexpr bool kHasPre = true;
  static __device__ __forceinline__ TT prepare(E b, const C& c) {
    const u128 ninv = (static_cast<u128>(c.ninv2_hi) << 64) | c.ninv2_lo;
    return static_cast<i128>(static_cast<u128>(static_cast<i128>(b)) * ninv);
  }
  static __device__ __forceinline__ E mul_pre(E a, TT bp, const C& c) {
    const uint64_t ua = static_cast<uint64_t>(a);
    const uint64_t blo = static_cast<uint64_t>(bp);
    const uint64_t bhi = static_cast<uint64_t>(static_cast<u128>(bp) >> 64);
    const uint64_t ml = ua * blo;
    const int64_t mh = static_cast<int64_t>(__umul64hi(ua, blo) + ua * bhi - (a < 0 ? blo : 0u));
    const i128 p = static_cast<i128>(mh) * static_cast<int64_t>(c.N) +
                   ((ml >> 63) ? static_cast<i128>(c.N) : i128{0}) + (i128{1} << 63);
    return static_cast<int64_t>(p >> 64);
  }
};

struct SignedPlantard2_64 {
  using E = int64_t;
  using TT = i128;
  using C = WordConst64;
  static __device__ __forceinline__ TT mul(E a, E b) { return static_cast<i128>(a) * b; }
  static __device__ __forceinline__ TT widen(E y) { return y; }
  static __device__ __forceinline__ E reduce(TT T, const C& c) {
    const uint64_t Tl = static_cast<uint64_t>(T);
    const uint64_t Th = static_cast<uint64_t>(static_cast<u128>(T) >> 64);
    const int64_t mh = static_cast<int64_t>(plantard_m_hi(Tl, Th, c));
    const i128 p = static_cast<i128>(mh) * static_cast<int64_t>(c.N) +
                   (static_cast<i128>(c.N) << c.alpha);
    return static_cast<int64_t>(p >> 64);
  }
  static __device__ __forceinline__ E canon(E r, const C&) { return r; }
  static constexpr bool kHasPre = true;
  static __device__ __forceinline__ TT prepare(E b, const C& c) {
    const u128 ninv = (static_cast<u128>(c.ninv2_hi) << 64) | c.ninv2_lo;
    return static_cast<i128>(static_cast<u128>(static_cast<i128>(b)) * ninv);
  }
  static __device__ __forceinline__ E mul_pre(E a, TT bp, const C& c) {
    const uint64_t ua = static_cast<uint64_t>(a);
    const uint64_t blo = static_cast<uint64_t>(bp);
    const uint64_t bhi = static_cast<uint64_t>(static_cast<u128>(bp) >> 64);
    const int64_t mh = static_cast<int64_t>(__umul64hi(ua, blo) + ua * bhi - (a < 0 ? blo : 0u));
    const i128 p = static_cast<i128>(mh) * static_cast<int64_t>(c.N) +
                   (static_cast<i128>(c.N) << c.alpha);
    return static_cast<int64_t>(p >> 64);
  }
};

}  // namespace montgb
