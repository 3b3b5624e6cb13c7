// Exhaustive verify sweep (mont_verify_sweep): the CRT check of Section 3.
//
// Work decomposition.  The host lists the swept moduli in a table (one entry
// per odd N with its constants, its T interval and its claimed output range)
// and cuts each N's T interval into chunks of C consecutive T; chunk i of the
// whole sweep belongs to the entry whose first chunk index is the largest one
// <= i.  A grid of resident threads walks the chunk indices grid-stride.
//
// Per chunk, a thread evaluates the algorithm on every T exactly as the paper
// writes it (REDC of Section 1, Algorithms 1-4), in 32/64-bit registers, and
// compares with the reference value c(T) = s T R^{-1} mod N.  c is computed
// with one modulo at the chunk start and then stepped, c(T+1) = c(T) + s R^{-1}
// mod N with one conditional subtraction, so no check divides.  The congruence
// test r = c (mod N) takes a fast path for r - c in {0, -N, +N} and divides
// only otherwise.  The kernel reads nothing but the table: it is bound by the
// integer pipes, not by memory.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <vector>

#include "internal.h"
#include "sweep.h"

namespace montgb {
namespace {

// NONNEG: every T of the chunk is >= 0 (REDC's own domain), so REDC's sum
// T + mN is formed in one unsigned word without testing T's sign.
template <int V, bool NONNEG>
__device__ __forceinline__ int32_t candidate(int32_t T, const SweepN& e, const SweepParams& p) {
  const uint32_t mask = (1u << p.log2R) - 1u;
  const int32_t N = e.N;
  const int up = 32 - p.log2R;   // sign extension of the low log2R bits: x mods R
  if constexpr (V == MONT_REDC) {
    // m <- (T mod R) N' mod R;  t <- (T + mN) / R;  if t >= N: t - N
    const uint32_t m = (static_cast<uint32_t>(T) * e.nprime) & mask;
    if (NONNEG || T >= 0) {
      // T < 2^31 and m N < 2^16 * 2^15: the sum fits an unsigned word
      const uint32_t t = (static_cast<uint32_t>(T) + m * static_cast<uint32_t>(N)) >> p.log2R;
      return static_cast<int32_t>(t >= static_cast<uint32_t>(N) ? t - static_cast<uint32_t>(N) : t);
    }
    const int64_t t = (static_cast<int64_t>(T) + static_cast<int64_t>(m) * N) >> p.log2R;
    return static_cast<int32_t>(t >= N ? t - N : t);
  } else if constexpr (V == MONT_SIGNED) {
    // T = a1 R + a0;  m0 <- a0 N^{-1} mods R;  t <- floor(m0 N / R);  r <- a1 - t
    const int32_t a1 = T >> p.log2R;
    const int32_t m0 = static_cast<int32_t>((static_cast<uint32_t>(T) * e.ninv) << up) >> up;
    return a1 - ((m0 * N) >> p.log2R);
  } else if constexpr (V == MONT_PLANTARD) {
    // r <- floor((floor((T N^{-1} mod R) / 2^n) + 1) N / 2^n);  if r = N: 0
    const uint32_t m = (static_cast<uint32_t>(T) * e.ninv) & mask;
    const int32_t r = static_cast<int32_t>((((m >> p.n) + 1u) * static_cast<uint32_t>(N)) >> p.n);
    return r == N ? 0 : r;
  } else {
    // m <- T Ñ^{-1} mods R
    const int32_t m = static_cast<int32_t>((static_cast<uint32_t>(T) * e.ninv) << up) >> up;
    if constexpr (V == MONT_SIGNED_PLANTARD) {
      // r <- round(round(m / 2^n) N / 2^n), halves rounded up
      const int32_t half = 1 << (p.n - 1);
      const int32_t q = (m + half) >> p.n;
      return (q * N + half) >> p.n;
    } else {
      // r <- floor((floor(m / 2^n) + 2^alpha) N / 2^n)
      return (((m >> p.n) + (1 << p.alpha)) * N) >> p.n;
    }
  }
}

// How the claimed range is tested.  The reference c = s T R^{-1} mod N is
// kept in [0, N) (kept centred in [-(N-1)/2, (N-1)/2] for kCentred), and:
//   kUnsigned  range [0, N-1]:            the only congruent value in range is c
//   kCentred   range [-(N-1)/2, (N-1)/2]: the only congruent value in range is c
//   kWide      range [-(N-1), N-1]:       c, and c - N when c != 0
//   kGeneric   any explicit range:        c or c - N inside the range
// A check that fails these goes through exact_bad, so the verdict is exact.
enum RangeKind : int { kUnsigned = 0, kCentred = 1, kWide = 2, kGeneric = 3 };

template <int RK>
__device__ __forceinline__ bool fast_good(int32_t r, uint32_t c, const SweepN& e) {
  const int32_t ci = static_cast<int32_t>(c);
  if constexpr (RK == kUnsigned || RK == kCentred) {
    return r == ci;
  } else if constexpr (RK == kWide) {
    return r == ci || (r == ci - e.N && ci != 0);
  } else {
    return (r == ci || r == ci - e.N) && r >= e.r_lo && r <= e.r_hi;
  }
}

// The exact test: counterexample unless r = c (mod N) and r in range.
__device__ __forceinline__ bool exact_bad(int32_t r, uint32_t c, const SweepN& e) {
  if (r < e.r_lo || r > e.r_hi) return true;   // out of range: no congruence needed
  const int64_t d = static_cast<int64_t>(r) - static_cast<int64_t>(static_cast<int32_t>(c));
  const int64_t N = e.N;
  if (d == 0 || d == N || d == -N) return false;
  return (d % N) != 0;
}

__device__ __forceinline__ uint32_t add_mod(uint32_t c, uint32_t s, uint32_t N) {
  const uint32_t x = c + s;            // c, s < N < 2^15
  return min(x, x - N);                // x - N wraps above x when x < N
}

// c + s for a centred c in [-(N-1)/2, (N-1)/2] and 0 <= s < N, kept centred.
__device__ __forceinline__ uint32_t add_mod_centred(uint32_t c, uint32_t s, uint32_t N) {
  const int32_t x = static_cast<int32_t>(c) + static_cast<int32_t>(s);
  const int32_t h = static_cast<int32_t>((N - 1u) / 2u);
  return static_cast<uint32_t>(x > h ? x - static_cast<int32_t>(N) : x);
}

template <int RK>
__device__ __forceinline__ uint32_t step_ref(uint32_t c, uint32_t s, uint32_t N) {
  if constexpr (RK == kCentred) return add_mod_centred(c, s, N);
  else return add_mod(c, s, N);
}

// Append one counterexample; returns true once the buffer is seen full, after
// which the caller stops calling (so a sweep with many failures pays only for
// counting them).
template <bool kUnsignedTarget>
__device__ __noinline__ bool record(int32_t T, int32_t r, uint32_t c, uint32_t N,
                                    mont_cex* __restrict__ cex,
                                    unsigned long long* __restrict__ cex_n,
                                    unsigned long long cap) {
  if (*reinterpret_cast<volatile unsigned long long*>(cex_n) >= cap) return true;
  const unsigned long long slot = atomicAdd(cex_n, 1ull);
  if (slot >= cap) return true;
  // c is in [0, N) or, for a centred chain, already in [-(N-1)/2, (N-1)/2]
  int64_t expect = static_cast<int32_t>(c);
  if (expect < 0) expect += N;
  if (!kUnsignedTarget && expect > static_cast<int64_t>((N - 1u) / 2u)) expect -= N;
  mont_cex rec;
  rec.N = N;
  rec.reserved = 0;
  rec.T = T;
  rec.r = r;
  rec.expected = expect;
  cex[slot] = rec;
  return false;
}

// The checks of one chunk: T0 .. T0 + cnt - 1 against the four reference
// chains c0..c3 (stepped by s4, the tail by s1); returns the counterexamples.
template <int V, int RK, bool NONNEG>
__device__ __forceinline__ uint32_t check_chunk(int64_t T0, uint32_t cnt, const SweepN& e,
                                                const SweepParams& p, uint32_t c0, uint32_t c1,
                                                uint32_t c2, uint32_t c3, uint32_t s1, uint32_t s4,
                                                mont_cex* __restrict__ cex,
                                                unsigned long long* __restrict__ cex_n,
                                                unsigned long long cap, bool& full) {
  constexpr bool kUnsignedTarget = (V == MONT_REDC || V == MONT_PLANTARD);
  const uint32_t N = static_cast<uint32_t>(e.N);
  uint32_t local = 0;
  uint32_t Tu = static_cast<uint32_t>(static_cast<int32_t>(T0));
  uint32_t i = 0;
  for (; i + 4 <= cnt; i += 4, Tu += 4) {
    const int32_t Ta = static_cast<int32_t>(Tu), Tb = static_cast<int32_t>(Tu + 1u);
    const int32_t Tc = static_cast<int32_t>(Tu + 2u), Td = static_cast<int32_t>(Tu + 3u);
    const int32_t ra = candidate<V, NONNEG>(Ta, e, p), rb = candidate<V, NONNEG>(Tb, e, p);
    const int32_t rc = candidate<V, NONNEG>(Tc, e, p), rd = candidate<V, NONNEG>(Td, e, p);
    const bool ga = fast_good<RK>(ra, c0, e), gb = fast_good<RK>(rb, c1, e);
    const bool gc = fast_good<RK>(rc, c2, e), gd = fast_good<RK>(rd, c3, e);
    if (!(ga && gb && gc && gd)) {
      const bool ba = !ga && exact_bad(ra, c0, e), bb = !gb && exact_bad(rb, c1, e);
      const bool bc = !gc && exact_bad(rc, c2, e), bd = !gd && exact_bad(rd, c3, e);
      local += static_cast<uint32_t>(ba) + static_cast<uint32_t>(bb) + static_cast<uint32_t>(bc) +
               static_cast<uint32_t>(bd);
      if (!full && (ba || bb || bc || bd)) {
        if (ba && !full) full = record<kUnsignedTarget>(Ta, ra, c0, N, cex, cex_n, cap);
        if (bb && !full) full = record<kUnsignedTarget>(Tb, rb, c1, N, cex, cex_n, cap);
        if (bc && !full) full = record<kUnsignedTarget>(Tc, rc, c2, N, cex, cex_n, cap);
        if (bd && !full) full = record<kUnsignedTarget>(Td, rd, c3, N, cex, cex_n, cap);
      }
    }
    c0 = step_ref<RK>(c0, s4, N);
    c1 = step_ref<RK>(c1, s4, N);
    c2 = step_ref<RK>(c2, s4, N);
    c3 = step_ref<RK>(c3, s4, N);
  }
  for (; i < cnt; ++i, ++Tu) {
    const int32_t T = static_cast<int32_t>(Tu);
    const int32_t r = candidate<V, NONNEG>(T, e, p);
    if (!fast_good<RK>(r, c0, e) && exact_bad(r, c0, e)) {
      ++local;
      if (!full) full = record<kUnsignedTarget>(T, r, c0, N, cex, cex_n, cap);
    }
    c0 = step_ref<RK>(c0, s1, N);
  }
  return local;
}

// The low word of a b + c, written as PTX so that products of the loop index
// stay multiply-adds instead of becoming induction additions.  With b = 1
// held in a register (a kernel parameter the compiler cannot see through) it
// is an addition issued to the multiply-add pipe, which the sweep otherwise
// leaves half idle while the ALU pipe runs the compares and minima.
__device__ __forceinline__ uint32_t mad_lo(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// The same chunk as check_chunk for REDC on non-negative T and for Algorithm
// 1, with the work spread over both integer pipes.  T = T0 + j + i for chain
// j at loop offset i.
//  REDC:   m = (T N') mod R as the low log2R bits of i N' + T_j N' (one
//          multiply-add), t = (T + mN) >> log2R, r = min(t, t - N) (unsigned:
//          t - N wraps above t when t < N, so this is "if t >= N: t - N").
//  Alg. 1: u = T (N^{-1} << sh) mod 2^32 (sh = 32 - log2R) read as a signed
//          word is m0 << sh, m0 = T N^{-1} mods R (the sign extension of the
//          low log2R bits), so floor(m0 N / R) is the signed high word of u N;
//          a1 = T >> log2R; r = a1 - floor(m0 N / R).
// The reference chains step with two multiply-adds and one minimum.
template <int V, int RK>
__device__ __forceinline__ uint32_t check_chunk_fast(int64_t T0, uint32_t cnt, const SweepN& e,
                                                     const SweepParams& p, uint32_t c0,
                                                     uint32_t c1, uint32_t c2, uint32_t c3,
                                                     uint32_t s1, uint32_t s4,
                                                     mont_cex* __restrict__ cex,
                                                     unsigned long long* __restrict__ cex_n,
                                                     unsigned long long cap, bool& full) {
  constexpr bool kUnsignedTarget = (V == MONT_REDC);
  const uint32_t N = static_cast<uint32_t>(e.N);
  const uint32_t one = p.one;
  const uint32_t negN = 0u - N;
  const int L = p.log2R;
  const uint32_t mask = (1u << L) - 1u;
  const uint32_t k = V == MONT_REDC ? e.nprime : e.ninv << (32 - L);
  const uint32_t T0w = static_cast<uint32_t>(static_cast<int32_t>(T0));
  // With the unsigned range (REDC) or the centred one (Algorithm 1) the only
  // good value is the chain's c itself, so the checks of a step fold into
  // one word: the OR of (r + off) ^ c (one three-input logic operation per
  // check), tested once per step.  The folded chains are kept in [0, N):
  // off = (N - 1) / 2 moves the centred range there.  Algorithm 1's own
  // range (-N, N) has two good values, c and c - N (the latter for c > 0):
  // with t = r + N, min(r, t) (unsigned) is r for r in [0, N) and r + N for
  // r in [-N, 0), so it equals c exactly for the good values and for r = -N
  // at c = 0, which the running minimum of t (zero only at r = -N) rules out.
  constexpr bool kFoldWide = (V == MONT_SIGNED && RK == kWide);
  constexpr bool kFold = (V == MONT_REDC && RK == kUnsigned) ||
                         (V == MONT_SIGNED && RK == kCentred) || kFoldWide;
  constexpr int kChainRK = kFold ? kUnsigned : RK;
  const uint32_t off = (kFold && RK == kCentred) ? (N - 1u) / 2u : 0u;
  // W chains per step: the step's fixed cost (loop test, mismatch test,
  // branches) is shared by W checks.  Chain j >= 4 starts four steps of s
  // after chain j - 4; every chain steps by sW = W s mod N.  (Eight chains
  // for the folded checks; the other range kinds run four, as eight cost
  // them more registers than the shared step saves.)
  constexpr int W = kFold ? 8 : 4;
  uint32_t Tb[W], kb[W];
#pragma unroll
  for (int j = 0; j < W; ++j) {
    Tb[j] = T0w + static_cast<uint32_t>(j);
    kb[j] = Tb[j] * k;
  }
  uint32_t c[W];
  c[0] = c0 + off; c[1] = c1 + off; c[2] = c2 + off; c[3] = c3 + off;
#pragma unroll
  for (int j = 4; j < W; ++j) c[j] = step_ref<kChainRK>(c[j - 4], s4, N);
  uint32_t sW = s4;                                    // W s mod N, in [0, N)
#pragma unroll
  for (int w = 4; w < W; w *= 2) sW = step_ref<kUnsigned>(sW, sW, N);
  const uint32_t sWm = sW - N;
  uint32_t local = 0;
  uint32_t i = 0;
  for (; i + W <= cnt; i += W) {
    int32_t r[W];
    bool g[W];
    uint32_t diff = 0, tmin = 0xFFFFFFFFu;
#pragma unroll
    for (int j = 0; j < W; ++j) {
      // Algorithm 1's signed high product is a half-rate multiply, which
      // leaves the multiply pipe the busier one: its loop index and chain
      // steps stay plain additions (ALU), only r + N goes to the multiply
      // pipe; REDC's additions all go there
      const uint32_t T = kFoldWide ? i + Tb[j] : mad_lo(i, one, Tb[j]);
      const uint32_t u = mad_lo(i, k, kb[j]);            // T k mod 2^32
      if constexpr (V == MONT_REDC) {
        const uint32_t t = mad_lo(u & mask, N, T) >> L;  // (T + mN) / R, below 2^32
        r[j] = static_cast<int32_t>(min(t, mad_lo(t, one, negN)));
      } else {
        r[j] = (static_cast<int32_t>(T) >> L) -
               __mulhi(static_cast<int32_t>(u), static_cast<int32_t>(N));
      }
      if constexpr (kFoldWide) {
        const uint32_t ru = static_cast<uint32_t>(r[j]), t = mad_lo(N, one, ru);
        diff |= min(ru, t) ^ c[j];
        tmin = min(tmin, t);
      } else if constexpr (kFold) {
        diff |= (static_cast<uint32_t>(r[j]) + off) ^ c[j];
      } else {
        g[j] = fast_good<RK>(r[j], c[j], e);
      }
    }
    bool all_good = true;
    if constexpr (!kFold) {
#pragma unroll
      for (int j = 0; j < W; ++j) all_good = all_good && g[j];
    }
    if (kFold ? (diff != 0u || tmin == 0u) : !all_good) {
      if constexpr (kFold) {   // the rare step with a mismatch: which checks
#pragma unroll
        for (int j = 0; j < W; ++j) g[j] = fast_good<RK>(r[j], c[j] - off, e);
      }
#pragma unroll
      for (int j = 0; j < W; ++j) {
        if (!g[j] && exact_bad(r[j], c[j] - off, e)) {
          ++local;
          if (!full)
            full = record<kUnsignedTarget>(static_cast<int32_t>(T0w + i + static_cast<uint32_t>(j)),
                                           r[j], c[j] - off, N, cex, cex_n, cap);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < W; ++j) {
      if constexpr (kChainRK == kCentred) {
        c[j] = step_ref<kChainRK>(c[j], sW, N);
      } else if constexpr (kFoldWide) {
        c[j] = min(c[j] + sW, c[j] + sWm);
      } else {
        c[j] = min(mad_lo(c[j], one, sW), mad_lo(c[j], one, sWm));
      }
    }
  }
  for (; i < cnt; ++i) {
    const int32_t T = static_cast<int32_t>(T0w + i);
    const int32_t r = candidate<V, true>(T, e, p);
    const uint32_t ct = c[0] - off;   // the chain in RK's representation
    if (!fast_good<RK>(r, ct, e) && exact_bad(r, ct, e)) {
      ++local;
      if (!full) full = record<kUnsignedTarget>(T, r, ct, N, cex, cex_n, cap);
    }
    c[0] = step_ref<kChainRK>(c[0], s1, N);
  }
  return local;
}

// Chunks item_lo .. item_hi - 1 of the sweep, grid-stride.
template <int V, int RK>
__global__ void __launch_bounds__(256) sweep_kernel(const SweepN* __restrict__ tab, int n_tab,
                                                    uint64_t item_lo, uint64_t item_hi,
                                                    SweepParams p,
                                                    unsigned long long* __restrict__ counts,
                                                    mont_cex* __restrict__ cex,
                                                    unsigned long long* __restrict__ cex_n,
                                                    unsigned long long cap) {
  const uint64_t nthreads = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  bool full = false;  // the example buffer was seen full: stop touching it
  for (uint64_t item = item_lo + static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
       item < item_hi; item += nthreads) {
    int lo = 0, hi = n_tab - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (tab[mid].item0 <= item) lo = mid; else hi = mid - 1;
    }
    const SweepN e = tab[lo];
    const int64_t T0 = e.t_lo + static_cast<int64_t>(item - e.item0) * p.chunk;
    const int64_t T1 = T0 + p.chunk - 1 < e.t_hi ? T0 + p.chunk - 1 : e.t_hi;
    const uint32_t cnt = static_cast<uint32_t>(T1 - T0 + 1);
    const uint32_t N = static_cast<uint32_t>(e.N);
    int64_t tm = T0 % e.N;
    if (tm < 0) tm += e.N;
    // four reference chains: c_j = s (T0 + j + 4i) R^{-1} mod N
    const uint32_t s1 = e.step;
    const uint32_t s2 = add_mod(s1, s1, N), s3 = add_mod(s2, s1, N), s4 = add_mod(s3, s1, N);
    uint32_t c0 = static_cast<uint32_t>((static_cast<uint64_t>(tm) * e.step) % N);
    uint32_t c1 = add_mod(c0, s1, N), c2 = add_mod(c0, s2, N), c3 = add_mod(c0, s3, N);
    if constexpr (RK == kCentred) {  // move the chains to the centred representatives
      const uint32_t h = (N - 1u) / 2u;
      c0 = c0 > h ? c0 - N : c0;
      c1 = c1 > h ? c1 - N : c1;
      c2 = c2 > h ? c2 - N : c2;
      c3 = c3 > h ? c3 - N : c3;
    }
    uint32_t local;
    if constexpr (V == MONT_SIGNED) {
      local = check_chunk_fast<V, RK>(T0, cnt, e, p, c0, c1, c2, c3, s1, s4, cex, cex_n, cap, full);
    } else if constexpr (V == MONT_REDC) {
      local = T0 >= 0
                  ? check_chunk_fast<V, RK>(T0, cnt, e, p, c0, c1, c2, c3, s1, s4, cex, cex_n, cap, full)
                  : check_chunk<V, RK, false>(T0, cnt, e, p, c0, c1, c2, c3, s1, s4, cex, cex_n, cap, full);
    } else {
      local = check_chunk<V, RK, false>(T0, cnt, e, p, c0, c1, c2, c3, s1, s4, cex, cex_n, cap, full);
    }
    if (local) atomicAdd(counts + lo, static_cast<unsigned long long>(local));
  }
}

// ---------------------------------------------------------------- host side

uint32_t inv_pow2_u32(uint32_t N, uint32_t mask) {  // N^{-1} mod 2^k, Newton-Hensel
  uint32_t x = N;
  for (int i = 0; i < 5; ++i) x *= 2u - N * x;
  return x & mask;
}

int64_t inv_mod(int64_t a, int64_t m) {  // a^{-1} mod m, extended Euclid; gcd(a, m) = 1
  int64_t r0 = m, r1 = ((a % m) + m) % m, s0 = 0, s1 = 1;
  while (r1 != 0) {
    const int64_t q = r0 / r1;
    int64_t t = r0 - q * r1; r0 = r1; r1 = t;
    t = s0 - q * s1; s0 = s1; s1 = t;
  }
  return ((s0 % m) + m) % m;
}

bool precondition(int variant, int64_t N, int log2R, int alpha) {
  const int64_t R = int64_t{1} << log2R;
  const int n = log2R / 2;
  switch (variant) {
    case MONT_REDC: return N < R;
    case MONT_SIGNED: return 2 * N < R;
    case MONT_PLANTARD: {  // 5 N^2 < (2^{n+1} - N)^2, N < 2^15 so this fits in 64 bits
      const int64_t d = (int64_t{1} << (n + 1)) - N;
      return d > 0 && 5 * N * N < d * d;
    }
    case MONT_SIGNED_PLANTARD: return N < (int64_t{1} << (n - 1));
    case MONT_SIGNED_PLANTARD2:
      return n - alpha - 1 >= 0 && N < (int64_t{1} << (n - alpha - 1));
  }
  return false;
}

void default_domain(int variant, int64_t N, int log2R, int alpha, int64_t* lo, int64_t* hi) {
  const int64_t R = int64_t{1} << log2R;
  const int n = log2R / 2;
  switch (variant) {
    case MONT_REDC: *lo = 0; *hi = R * N - 1; return;
    case MONT_SIGNED: *lo = -(N * R / 2) + 1; *hi = N * R / 2 - 1; return;
    case MONT_PLANTARD: *lo = 0; *hi = N * N; return;
    case MONT_SIGNED_PLANTARD: *hi = int64_t{1} << (2 * n - 2); *lo = -*hi; return;
    default: *hi = (int64_t{1} << (2 * alpha)) * N * N; *lo = -*hi; return;
  }
}

void default_range(int variant, int64_t N, int64_t* lo, int64_t* hi) {
  switch (variant) {
    case MONT_REDC:
    case MONT_PLANTARD: *lo = 0; *hi = N - 1; return;
    case MONT_SIGNED: *lo = -(N - 1); *hi = N - 1; return;
    default: *lo = -((N - 1) / 2); *hi = (N - 1) / 2; return;
  }
}

template <int V, int RK>
cudaError_t launch_sweep_rk(const SweepN* tab, int n_tab, uint64_t item_lo, uint64_t item_hi,
                            const SweepParams& p, unsigned long long* counts, mont_cex* cex,
                            unsigned long long* cex_n, unsigned long long cap, cudaStream_t s) {
  if (item_hi <= item_lo) return cudaSuccess;
  const int threads = 256;
  const int per_sm = resident_blocks(reinterpret_cast<const void*>(sweep_kernel<V, RK>), threads);
  const uint64_t cap_blocks = static_cast<uint64_t>(device_sm_count()) * per_sm;
  const uint64_t want = (item_hi - item_lo + threads - 1) / threads;
  const unsigned grid = static_cast<unsigned>(want < cap_blocks ? want : cap_blocks);
  sweep_kernel<V, RK><<<grid, threads, 0, s>>>(tab, n_tab, item_lo, item_hi, p, counts, cex, cex_n,
                                               cap);
  return cudaGetLastError();
}

// The range kind of a call: the claimed range rule resolved for the variant.
int range_kind(int variant, int range_rule) {
  switch (range_rule) {
    case MONT_RANGE_UNSIGNED: return kUnsigned;
    case MONT_RANGE_WIDE: return kWide;
    case MONT_RANGE_CENTRED: return kCentred;
    case MONT_RANGE_DEFAULT:
      if (variant == MONT_REDC || variant == MONT_PLANTARD) return kUnsigned;
      if (variant == MONT_SIGNED) return kWide;
      return kCentred;
  }
  return kGeneric;
}

template <int V>
cudaError_t launch_sweep_v(const SweepN* tab, int n_tab, uint64_t lo, uint64_t hi,
                           const SweepParams& p, unsigned long long* counts, mont_cex* cex,
                           unsigned long long* cex_n, unsigned long long cap, cudaStream_t s) {
  switch (p.range_kind) {
    case kUnsigned: return launch_sweep_rk<V, kUnsigned>(tab, n_tab, lo, hi, p, counts, cex, cex_n, cap, s);
    case kCentred: return launch_sweep_rk<V, kCentred>(tab, n_tab, lo, hi, p, counts, cex, cex_n, cap, s);
    case kWide: return launch_sweep_rk<V, kWide>(tab, n_tab, lo, hi, p, counts, cex, cex_n, cap, s);
    default: return launch_sweep_rk<V, kGeneric>(tab, n_tab, lo, hi, p, counts, cex, cex_n, cap, s);
  }
}

// Chunks [lo, hi) of a sweep whose table, counters and example buffer are in
// device memory.
cudaError_t launch_sweep(int variant, const SweepN* tab, int n_tab, uint64_t lo, uint64_t hi,
                         const SweepParams& p, unsigned long long* counts, mont_cex* cex,
                         unsigned long long* cex_n, unsigned long long cap, cudaStream_t s) {
  switch (variant) {
    case MONT_REDC: return launch_sweep_v<MONT_REDC>(tab, n_tab, lo, hi, p, counts, cex, cex_n, cap, s);
    case MONT_SIGNED: return launch_sweep_v<MONT_SIGNED>(tab, n_tab, lo, hi, p, counts, cex, cex_n, cap, s);
    case MONT_PLANTARD: return launch_sweep_v<MONT_PLANTARD>(tab, n_tab, lo, hi, p, counts, cex, cex_n, cap, s);
    case MONT_SIGNED_PLANTARD: return launch_sweep_v<MONT_SIGNED_PLANTARD>(tab, n_tab, lo, hi, p, counts, cex, cex_n, cap, s);
    default: return launch_sweep_v<MONT_SIGNED_PLANTARD2>(tab, n_tab, lo, hi, p, counts, cex, cex_n, cap, s);
  }
}

// Where the parts of a sweep's scratch sit, from its 256-byte aligned start.
struct ScratchLayout {
  size_t counts, cex_n, cex, total;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

ScratchLayout scratch_layout(size_t n_tab, size_t cex_cap) {
  ScratchLayout l;
  l.counts = align256(n_tab * sizeof(SweepN));
  l.cex_n = l.counts + align256(n_tab * sizeof(unsigned long long));
  l.cex = l.cex_n + 256;
  l.total = l.cex + cex_cap * sizeof(mont_cex);
  return l;
}

// The checked domain and claimed range of modulus N under the call's rules.
// Returns false when N is skipped (too small, or outside the variant's
// condition unless out-of-spec moduli are asked for).
bool resolve_rules(int variant, int log2R, int alpha, int64_t N, int flags, const mont_bounds& rules,
                   int64_t* tlo, int64_t* thi, int64_t* rlo, int64_t* rhi) {
  if (N < 3) return false;
  if (!(flags & MONT_SWEEP_INCLUDE_OUT_OF_SPEC) && !precondition(variant, N, log2R, alpha)) return false;
  const int64_t R = int64_t{1} << log2R;
  if (rules.domain_rule == MONT_DOMAIN_DEFAULT) {
    default_domain(variant, N, log2R, alpha, tlo, thi);
  } else if (rules.domain_rule == MONT_DOMAIN_REDC) {
    *tlo = 0;
    *thi = R * N - 1;
  } else {
    *tlo = rules.t_lo;
    *thi = rules.t_hi;
  }
  switch (rules.range_rule) {
    case MONT_RANGE_DEFAULT: default_range(variant, N, rlo, rhi); break;
    case MONT_RANGE_UNSIGNED: *rlo = 0; *rhi = N - 1; break;
    case MONT_RANGE_WIDE: *rlo = -(N - 1); *rhi = N - 1; break;
    case MONT_RANGE_CENTRED: *rlo = -((N - 1) / 2); *rhi = (N - 1) / 2; break;
    default: *rlo = rules.r_lo; *rhi = rules.r_hi; break;
  }
  return true;
}

// The constants of a table entry for N (its T interval and range set by the caller).
void fill_constants(int variant, int log2R, int64_t N, SweepN* e) {
  const uint32_t mask = (1u << log2R) - 1u;
  const int64_t R = int64_t{1} << log2R;
  e->N = static_cast<int32_t>(N);
  e->ninv = inv_pow2_u32(static_cast<uint32_t>(N), mask);
  e->nprime = (0u - e->ninv) & mask;
  const int64_t rinv = inv_mod(R % N, N);
  e->step = static_cast<uint32_t>(variant >= MONT_PLANTARD ? (N - rinv) % N : rinv);
}

// The argument checks every sweep entry point shares.
int check_args(int variant, int log2R, int alpha, uint32_t N_lo, uint32_t N_hi,
               const mont_bounds& rules) {
  if (variant < MONT_REDC || variant > MONT_SIGNED_PLANTARD2) return MONT_EINVAL;
  if (log2R < 2 || log2R > MONT_SWEEP_MAX_LOG2R) return MONT_EINVAL;
  if (variant >= MONT_PLANTARD && (log2R % 2)) return MONT_EINVAL;
  if (variant == MONT_SIGNED_PLANTARD2 && (alpha < 0 || alpha > 14)) return MONT_EINVAL;
  if (N_lo > N_hi || N_hi > MONT_SWEEP_MAX_N || N_hi < 3) return MONT_EINVAL;
  if (rules.domain_rule < MONT_DOMAIN_DEFAULT || rules.domain_rule > MONT_DOMAIN_EXPLICIT) return MONT_EINVAL;
  if (rules.range_rule < MONT_RANGE_DEFAULT || rules.range_rule > MONT_RANGE_EXPLICIT) return MONT_EINVAL;
  return MONT_OK;
}

// Chunk size: a power of two in [32, 4096] giving >= 8 chunks per resident
// thread of a full-occupancy grid.
uint64_t chunk_for(uint64_t total_T) {
  const uint64_t resident = static_cast<uint64_t>(device_sm_count()) * 2048u;
  uint64_t chunk = 4096;
  while (chunk > 32 && total_T / chunk < 8 * resident) chunk >>= 1;
  return chunk;
}

}  // namespace

int sweep_plan(int variant, int log2R, int alpha, uint32_t N_lo, uint32_t N_hi,
               const mont_bounds* claimed, int flags, size_t cex_cap, uint64_t* per_N_counts,
               uint64_t* per_N_checked, SweepPlan* plan) {
  mont_bounds rules{MONT_DOMAIN_DEFAULT, MONT_RANGE_DEFAULT, 0, 0, 0, 0};
  if (claimed) rules = *claimed;
  const int st = check_args(variant, log2R, alpha, N_lo, N_hi, rules);
  if (st != MONT_OK) return st;
  if (!per_N_counts) return MONT_EINVAL;
  const uint32_t first = (N_lo % 2) ? N_lo : N_lo + 1;
  plan->variant = variant;
  plan->cex_cap = cex_cap;
  plan->n_odd = first > N_hi ? 0 : (N_hi - first) / 2 + 1;
  plan->tab.clear();
  plan->tab_index.clear();
  plan->total_T = 0;
  for (size_t i = 0; i < plan->n_odd; ++i) {
    per_N_counts[i] = 0;
    if (per_N_checked) per_N_checked[i] = 0;
  }
  for (size_t i = 0; i < plan->n_odd; ++i) {
    const int64_t N = first + 2 * static_cast<int64_t>(i);
    int64_t tlo, thi, rlo, rhi;
    if (!resolve_rules(variant, log2R, alpha, N, flags, rules, &tlo, &thi, &rlo, &rhi)) continue;
    if (tlo > thi) continue;  // empty domain: nothing checked
    if (tlo < INT32_MIN || thi > INT32_MAX || rlo < INT32_MIN || rhi > INT32_MAX || rlo > rhi)
      return MONT_EINVAL;
    SweepN e{};
    fill_constants(variant, log2R, N, &e);
    e.t_lo = tlo;
    e.t_hi = thi;
    e.r_lo = static_cast<int32_t>(rlo);
    e.r_hi = static_cast<int32_t>(rhi);
    plan->tab.push_back(e);
    plan->tab_index.push_back(i);
    plan->total_T += static_cast<uint64_t>(thi - tlo + 1);
    if (per_N_checked) per_N_checked[i] = static_cast<uint64_t>(thi - tlo + 1);
  }
  const uint64_t chunk = plan->tab.empty() ? 32 : chunk_for(plan->total_T);
  plan->items = 0;
  for (auto& e : plan->tab) {
    e.item0 = plan->items;
    plan->items += (static_cast<uint64_t>(e.t_hi - e.t_lo) + chunk) / chunk;
  }
  plan->p = SweepParams{log2R, log2R / 2, alpha, static_cast<uint32_t>(chunk),
                        range_kind(variant, rules.range_rule), 1u};
  return MONT_OK;
}

size_t sweep_scratch_bytes(size_t n_tab, size_t cex_cap) {
  return scratch_layout(n_tab, cex_cap).total;
}

cudaError_t sweep_upload(const SweepPlan& plan, void* scratch, cudaStream_t s) {
  const ScratchLayout l = scratch_layout(plan.tab.size(), plan.cex_cap);
  char* base = static_cast<char*>(scratch);
  cudaError_t e = cudaMemcpyAsync(base, plan.tab.data(), plan.tab.size() * sizeof(SweepN),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemsetAsync(base + l.counts, 0, plan.tab.size() * sizeof(unsigned long long), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(base + l.cex_n, 0, sizeof(unsigned long long), s);
  return e;
}

cudaError_t sweep_launch(const SweepPlan& plan, void* scratch, uint64_t item_lo, uint64_t item_hi,
                         cudaStream_t s) {
  if (plan.tab.empty()) return cudaSuccess;
  const ScratchLayout l = scratch_layout(plan.tab.size(), plan.cex_cap);
  char* base = static_cast<char*>(scratch);
  if (item_hi > plan.items) item_hi = plan.items;
  return launch_sweep(plan.variant, reinterpret_cast<const SweepN*>(base),
                      static_cast<int>(plan.tab.size()), item_lo, item_hi, plan.p,
                      reinterpret_cast<unsigned long long*>(base + l.counts),
                      reinterpret_cast<mont_cex*>(base + l.cex),
                      reinterpret_cast<unsigned long long*>(base + l.cex_n), plan.cex_cap, s);
}

uint64_t sweep_items_for_checks(const SweepPlan& plan, uint64_t checks) {
  const uint64_t per = checks / (plan.p.chunk ? plan.p.chunk : 1);
  return per ? per : 1;
}

int sweep_collect(const SweepPlan& plan, void* scratch, cudaStream_t s, uint64_t* per_N_counts,
                  mont_cex* cex, size_t* n_cex_total) {
  *n_cex_total = 0;
  const size_t n_tab = plan.tab.size();
  if (n_tab == 0) return MONT_OK;
  const ScratchLayout l = scratch_layout(n_tab, plan.cex_cap);
  char* base = static_cast<char*>(scratch);
  std::vector<unsigned long long> h_counts(n_tab);
  unsigned long long h_cex_n = 0;
  cudaError_t err = cudaMemcpyAsync(h_counts.data(), base + l.counts,
                                    n_tab * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(&h_cex_n, base + l.cex_n, sizeof(h_cex_n), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  size_t n_rec = 0;
  if (err == cudaSuccess) {
    n_rec = static_cast<size_t>(h_cex_n < plan.cex_cap ? h_cex_n : plan.cex_cap);
    if (n_rec)
      err = cudaMemcpyAsync(cex, base + l.cex, n_rec * sizeof(mont_cex), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  }
  if (err != cudaSuccess) return cuda_status(err);
  uint64_t total = 0;
  for (size_t j = 0; j < n_tab; ++j) {
    per_N_counts[plan.tab_index[j]] = h_counts[j];
    total += h_counts[j];
  }
  std::sort(cex, cex + n_rec, [](const mont_cex& a, const mont_cex& b) {
    return a.N != b.N ? a.N < b.N : a.T < b.T;
  });
  *n_cex_total = static_cast<size_t>(total);
  return total > plan.cex_cap ? MONT_EOVERFLOW : MONT_OK;
}

}  // namespace montgb

using namespace montgb;

extern "C" int mont_verify_sweep(int variant, int log2R, int alpha, uint32_t N_lo, uint32_t N_hi,
                                 const mont_bounds* claimed, int flags, uint64_t* per_N_counts,
                                 uint64_t* per_N_checked, mont_cex* cex, size_t cex_cap,
                                 size_t* n_cex_total, void* stream) {
  if (!per_N_counts || !n_cex_total || (cex_cap > 0 && !cex)) return MONT_EINVAL;
  SweepPlan plan;
  const int st = sweep_plan(variant, log2R, alpha, N_lo, N_hi, claimed, flags, cex_cap,
                            per_N_counts, per_N_checked, &plan);
  if (st != MONT_OK) return st;
  *n_cex_total = 0;
  if (plan.tab.empty()) return MONT_OK;

  cudaStream_t s = static_cast<cudaStream_t>(stream);
  void* scratch = nullptr;
  cudaError_t err = cudaMallocAsync(&scratch, sweep_scratch_bytes(plan.tab.size(), cex_cap), s);
  if (err != cudaSuccess) {
    cudaGetLastError();
    return err == cudaErrorMemoryAllocation ? MONT_ENOMEM : cuda_status(err);
  }
  err = sweep_upload(plan, scratch, s);
  if (err == cudaSuccess) err = sweep_launch(plan, scratch, 0, plan.items, s);
  int status = err == cudaSuccess ? sweep_collect(plan, scratch, s, per_N_counts, cex, n_cex_total)
                                  : cuda_status(err);
  const cudaError_t ferr = cudaFreeAsync(scratch, s);
  const cudaError_t serr = cudaStreamSynchronize(s);
  if (status == MONT_OK || status == MONT_EOVERFLOW) {
    if (ferr != cudaSuccess) return cuda_status(ferr);
    if (serr != cudaSuccess) return cuda_status(serr);
  }
  return status;
}

// ---------------------------------------------------------------------------
// mont_verify_sweep_noalloc: the same sweep for callers that must not
// allocate.  Its device scratch (moduli table, per-N counters, example
// buffer) lives in one fixed file-scope device array instead of memory
// allocated per call, and its host side builds the table in one fixed
// file-scope host array and otherwise uses only the caller's buffers.
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kNoAllocModuli = MONT_SWEEP_NOALLOC_MAX_MODULI;
constexpr size_t kNoAllocCex = MONT_SWEEP_NOALLOC_MAX_CEX;
constexpr size_t kNoAllocBytes =
    (kNoAllocModuli * sizeof(SweepN) + 255) / 256 * 256 +
    (kNoAllocModuli * sizeof(unsigned long long) + 255) / 256 * 256 + 256 +
    kNoAllocCex * sizeof(mont_cex);
}  // namespace

// Shared by every call on a device and held until the process exits.  Host
// code must not take this symbol's address directly (it is a host-side
// stand-in); it uses the device address from noalloc_scratch().
static __device__ __align__(256) unsigned char g_sweep_noalloc_scratch[kNoAllocBytes];

// The table of one call, built on the host and uploaded in one copy.  Like the
// device array it is shared by every call (the call returns only after the
// copy has consumed it, so one call never sees another's half-built table).
static SweepN g_noalloc_table[kNoAllocModuli];

namespace {
// Device address of the scratch array in the current device's context,
// looked up on every call (a lookup allocates nothing, and a cached address
// would go stale if the context were torn down and created again).
int noalloc_scratch(char** out) {
  void* p = nullptr;
  const cudaError_t e = cudaGetSymbolAddress(&p, g_sweep_noalloc_scratch);
  if (e != cudaSuccess) return cuda_status(e);
  *out = static_cast<char*>(p);
  return MONT_OK;
}

// One table entry for modulus N under the call's rules; *checked receives the
// number of T swept (0 when N is skipped or its domain is empty).  Returns
// MONT_EINVAL when a bound leaves the 32-bit range.
int noalloc_entry(int variant, int log2R, int alpha, int64_t N, int flags, const mont_bounds& rules,
                  SweepN* e, uint64_t* checked) {
  *e = SweepN{};
  e->N = static_cast<int32_t>(N);
  e->t_lo = 0;
  e->t_hi = -1;
  *checked = 0;
  int64_t tlo, thi, rlo, rhi;
  if (!resolve_rules(variant, log2R, alpha, N, flags, rules, &tlo, &thi, &rlo, &rhi)) return MONT_OK;
  if (tlo > thi) return MONT_OK;
  if (tlo < INT32_MIN || thi > INT32_MAX || rlo < INT32_MIN || rhi > INT32_MAX || rlo > rhi)
    return MONT_EINVAL;
  fill_constants(variant, log2R, N, e);
  e->t_lo = tlo;
  e->t_hi = thi;
  e->r_lo = static_cast<int32_t>(rlo);
  e->r_hi = static_cast<int32_t>(rhi);
  *checked = static_cast<uint64_t>(thi - tlo + 1);
  return MONT_OK;
}
}  // namespace

extern "C" int mont_verify_sweep_noalloc(int variant, int log2R, int alpha, uint32_t N_lo,
                                         uint32_t N_hi, const mont_bounds* claimed, int flags,
                                         uint64_t* per_N_counts, uint64_t* per_N_checked,
                                         mont_cex* cex, size_t cex_cap, size_t* n_cex_total,
                                         void* stream) {
  mont_bounds rules{MONT_DOMAIN_DEFAULT, MONT_RANGE_DEFAULT, 0, 0, 0, 0};
  if (claimed) rules = *claimed;
  const int ast = check_args(variant, log2R, alpha, N_lo, N_hi, rules);
  if (ast != MONT_OK) return ast;
  if (!per_N_counts || !n_cex_total || (cex_cap > 0 && !cex)) return MONT_EINVAL;
  const uint32_t first = (N_lo % 2) ? N_lo : N_lo + 1;
  const size_t n_odd = first > N_hi ? 0 : (N_hi - first) / 2 + 1;
  // the fixed scratch bounds the request
  if (n_odd > kNoAllocModuli || cex_cap > kNoAllocCex) return MONT_EINVAL;

  // pass 1: validate every modulus, count the T to sweep
  uint64_t total_T = 0;
  for (size_t i = 0; i < n_odd; ++i) {
    SweepN e;
    uint64_t checked = 0;
    const int st = noalloc_entry(variant, log2R, alpha, first + 2 * static_cast<int64_t>(i), flags,
                                 rules, &e, &checked);
    if (st != MONT_OK) return st;
    per_N_counts[i] = 0;
    if (per_N_checked) per_N_checked[i] = checked;
    total_T += checked;
  }
  *n_cex_total = 0;
  if (total_T == 0) return MONT_OK;

  char* scratch = nullptr;
  const int sst = noalloc_scratch(&scratch);
  if (sst != MONT_OK) return sst;
  const ScratchLayout l = scratch_layout(n_odd, cex_cap);
  SweepN* d_tab = reinterpret_cast<SweepN*>(scratch);
  auto* d_counts = reinterpret_cast<unsigned long long*>(scratch + l.counts);
  auto* d_cex_n = reinterpret_cast<unsigned long long*>(scratch + l.cex_n);
  auto* d_cex = reinterpret_cast<mont_cex*>(scratch + l.cex);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const uint64_t chunk = chunk_for(total_T);

  // pass 2: the table (every odd N; skipped ones get no chunks), in one copy
  uint64_t items = 0;
  for (size_t i = 0; i < n_odd; ++i) {
    uint64_t checked = 0;
    noalloc_entry(variant, log2R, alpha, first + 2 * static_cast<int64_t>(i), flags, rules,
                  &g_noalloc_table[i], &checked);
    g_noalloc_table[i].item0 = items;
    items += (checked + chunk - 1) / chunk;
  }
  cudaError_t err = cudaMemcpyAsync(d_tab, g_noalloc_table, n_odd * sizeof(SweepN),
                                    cudaMemcpyHostToDevice, s);
  // counters start at zero on every call (the array keeps the last call's values)
  if (err == cudaSuccess) err = cudaMemsetAsync(d_counts, 0, n_odd * sizeof(unsigned long long), s);
  if (err == cudaSuccess) err = cudaMemsetAsync(d_cex_n, 0, sizeof(unsigned long long), s);
  SweepParams p{log2R, log2R / 2, alpha, static_cast<uint32_t>(chunk),
                range_kind(variant, rules.range_rule), 1u};
  if (err == cudaSuccess)
    err = launch_sweep(variant, d_tab, static_cast<int>(n_odd), 0, items, p, d_counts, d_cex,
                       d_cex_n, cex_cap, s);
  unsigned long long h_cex_n = 0;
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(per_N_counts, d_counts, n_odd * sizeof(uint64_t), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess)
    err = cudaMemcpyAsync(&h_cex_n, d_cex_n, sizeof(h_cex_n), cudaMemcpyDeviceToHost, s);
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  size_t n_rec = 0;
  if (err == cudaSuccess) {
    n_rec = static_cast<size_t>(h_cex_n < cex_cap ? h_cex_n : cex_cap);
    if (n_rec) err = cudaMemcpyAsync(cex, d_cex, n_rec * sizeof(mont_cex), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  }
  if (err != cudaSuccess) return cuda_status(err);
  uint64_t total = 0;
  for (size_t i = 0; i < n_odd; ++i) total += per_N_counts[i];
  std::sort(cex, cex + n_rec, [](const mont_cex& a, const mont_cex& b) {
    return a.N != b.N ? a.N < b.N : a.T < b.T;
  });
  *n_cex_total = static_cast<size_t>(total);
  return total > cex_cap ? MONT_EOVERFLOW : MONT_OK;
}
