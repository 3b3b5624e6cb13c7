// Multi-limb Montgomery multiplication: REDC (Section 1) at R = 2^{32k},
// scheduled as CIOS (coarsely integrated operand scanning; Koc, Acar and
// Kaliski, IEEE Micro 1996), which interleaves the product a b with the
// reduction one 32-bit word of b at a time:
//
//   t = 0
//   for i in 0..k-1:
//     t += a * b_i                  (k+1 limbs)
//     m  = t_0 * N'_0 mod 2^32      (N'_0 = -N^{-1} mod 2^32, the low word of N')
//     t  = (t + m N) / 2^32         (exact: the low word becomes 0)
//   if t >= N: t -= N               (t < 2N, as in Section 1)
//
// The result equals REDC's (T + mN)/R with T = a b, because the word-serial
// m's together form m = T N' mod R.
//
// Mapping to the GPU.  A team of L lanes of one warp owns one element (L = 1:
// one thread per element).  Lane l holds S = k/L limbs of a, b, N and of the
// running t, plus two overflow words h0, h1 at positions S, S+1 above its
// slice: t is kept in carry-save form across lanes, so that the k row
// updates need no inter-lane carry propagation.  Per iteration: b_i is
// fetched from its owning lane with one shuffle, the team's lane 0 computes m
// and broadcasts it with one shuffle, and the division by 2^32 moves every
// lane's lowest limb to the lane below with one shuffle-down, folding h0 into
// the vacated top limb.  Each row update is one generated inline-PTX carry
// chain (mad.lo.cc / madc.hi.cc, see cios_chains.cuh).  At the end the
// deferred inter-lane carries are resolved with one carry-lookahead step
// computed from warp ballots (carry into lane l = bit l of
// ((G << 1) + P) ^ P for generate mask G and propagate mask P), and the final
// subtraction of N resolves its borrows the same way.
//
// Algorithm 1 (the signed Montgomery reduction) runs on the same schedule.
// Its m = T N^{-1} mods R and CIOS's m' = -T N^{-1} mod R (the word-serial
// digits m_i above) are congruent up to sign: m = -m' when m' <= R/2, else
// m = R - m'.  So Algorithm 1's r = (T - mN)/R is (T + m'N)/R, less N when
// m' > R/2.  Signed elements are k-limb two's complement integers A, B, read
// as unsigned by the rows; for T = a b, A B = T + R (a [b < 0] + b [a < 0]) +
// R^2 [a, b < 0], so modulo R (r lies in (-N, N), which k limbs hold)
//   r = (A B + m'N)/R - [b < 0] A - [a < 0] B - [m' > R/2] N   (mod R),
// three conditional subtractions with the same inter-lane borrow lookahead.
// For a given 2k-limb T (mont_redc) the rows see T + R^2 [T < 0], which
// changes nothing modulo R.
#include <algorithm>

#include "cios_chains.cuh"
#include "tune.h"

namespace montgb {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <int S>
__device__ __forceinline__ void load_limbs(uint32_t (&d)[S], const uint32_t* p, bool vec16) {
  if constexpr (S % 4 == 0) {
    if (vec16) {
#pragma unroll
      for (int j = 0; j < S; j += 4) {
        const uint4 v = *reinterpret_cast<const uint4*>(p + j);
        d[j] = v.x; d[j + 1] = v.y; d[j + 2] = v.z; d[j + 3] = v.w;
      }
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < S; ++j) d[j] = p[j];
}

template <int S>
__device__ __forceinline__ void store_limbs(uint32_t* p, const uint32_t (&d)[S], bool vec16) {
  if constexpr (S % 4 == 0) {
    if (vec16) {
#pragma unroll
      for (int j = 0; j < S; j += 4)
        *reinterpret_cast<uint4*>(p + j) = make_uint4(d[j], d[j + 1], d[j + 2], d[j + 3]);
      return;
    }
  }
#pragma unroll
  for (int j = 0; j < S; ++j) p[j] = d[j];
}

template <int S>
__device__ __forceinline__ bool all_ones(const uint32_t (&t)[S]) {
  uint32_t x = 0xFFFFFFFFu;
#pragma unroll
  for (int j = 0; j < S; ++j) x &= t[j];
  return x == 0xFFFFFFFFu;
}

template <int S>
__device__ __forceinline__ bool all_zero(const uint32_t (&t)[S]) {
  uint32_t x = 0;
#pragma unroll
  for (int j = 0; j < S; ++j) x |= t[j];
  return x == 0;
}

// Lanes of the team (bits 0..L-1) that receive a carry, from generate and
// propagate masks: carry into l = g_{l-1} | (p_{l-1} & carry into l-1).
template <int L>
__device__ __forceinline__ unsigned lookahead(unsigned G, unsigned P) {
  constexpr unsigned mask = L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1u);
  return (((G << 1) + P) ^ P) & mask;
}

template <int L>
__device__ __forceinline__ unsigned team_bits(bool x, unsigned team_base) {
  constexpr unsigned mask = L == 32 ? 0xFFFFFFFFu : ((1u << L) - 1u);
  return (__ballot_sync(kFull, x) >> team_base) & mask;
}

// d <- d - (y & mask) modulo 2^{32k} over the team's slices: each lane
// subtracts its slice, and the borrows between lanes resolve by lookahead.
template <int S, int L>
__device__ __forceinline__ void team_sub_masked(uint32_t (&d)[S], const uint32_t (&y)[S],
                                                uint32_t mask, unsigned team_base, unsigned tl) {
  uint32_t ym[S], r[S];
#pragma unroll
  for (int j = 0; j < S; ++j) ym[j] = y[j] & mask;
  const uint32_t gb = sub_rows<S>(r, d, ym);
  if constexpr (L > 1) {
    const unsigned G = team_bits<L>(gb != 0, team_base);
    const unsigned P = team_bits<L>(all_zero<S>(r), team_base);
    const unsigned B = lookahead<L>(G, P);
    if ((B >> tl) & 1u) sub_word<S>(r, 1u);
  }
#pragma unroll
  for (int j = 0; j < S; ++j) d[j] = r[j];
}

// One element per team.  M: kMul (x*y), kToDomain (x * R^2 mod N),
// kFromDomain (reduce x), kRedc (reduce the 2k-limb x).  SIG: Algorithm 1
// (signed elements; kMul, kToDomain and kRedc), else REDC.
template <int K, int L, Mode M, bool SIG>
__global__ void __launch_bounds__(256) cios_kernel(const uint32_t* __restrict__ x,
                                                   const uint32_t* __restrict__ y,
                                                   uint32_t* __restrict__ out, size_t n,
                                                   const __grid_constant__ LimbConst c, int vec16) {
  constexpr int S = K / L;
  constexpr int TPW = 32 / L;  // teams per warp
  constexpr bool kProduct = (M == Mode::kMul || M == Mode::kToDomain);
  const unsigned lane = threadIdx.x & 31u;
  const unsigned tl = lane % L;            // lane within the team
  const unsigned team_base = lane - tl;    // first lane of the team
  const size_t warp = (static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
  const size_t nwarps = (static_cast<size_t>(gridDim.x) * blockDim.x) >> 5;

  uint32_t nl[S], bconst[S];
#pragma unroll
  for (int j = 0; j < S; ++j) {
    nl[j] = c.N[tl * S + j];
    bconst[j] = SIG ? c.dom[tl * S + j] : c.r2[tl * S + j];
  }

  for (size_t e0 = warp * TPW; e0 < n; e0 += nwarps * TPW) {
    const size_t e = e0 + lane / L;
    const bool valid = e < n;
    uint32_t al[S], bl[S], t[S], hi_in[S];
    uint32_t h0 = 0, h1 = 0;
    uint32_t m_low = 0, m_top = 0;   // Algorithm 1: digits of m
#pragma unroll
    for (int j = 0; j < S; ++j) { al[j] = 0; bl[j] = 0; t[j] = 0; hi_in[j] = 0; }
    if (valid) {
      if constexpr (M == Mode::kRedc) {
        load_limbs<S>(t, x + e * (2 * K) + tl * S, vec16);        // T mod R
        load_limbs<S>(hi_in, x + e * (2 * K) + K + tl * S, vec16); // floor(T / R)
      } else if constexpr (M == Mode::kFromDomain) {
        load_limbs<S>(t, x + e * K + tl * S, vec16);
      } else {
        load_limbs<S>(al, x + e * K + tl * S, vec16);
        if constexpr (M == Mode::kMul) {
          load_limbs<S>(bl, y + e * K + tl * S, vec16);
        }
      }
    }
    if constexpr (M == Mode::kToDomain) {
#pragma unroll
      for (int j = 0; j < S; ++j) bl[j] = bconst[j];
    }

    // K iterations, as L rounds of S: round I takes b's limbs from the
    // team's lane I.  Only a round is unrolled, so that the body stays in the
    // instruction cache at 1024 and 2048 bits.
#pragma unroll 1
    for (int I = 0; I < L; ++I) {
#pragma unroll
    for (int s = 0; s < S; ++s) {
      if constexpr (kProduct) {  // t += a * b_i, i = I S + s
        uint32_t bi;
        if constexpr (L == 1) {
          bi = bl[s];
        } else {
          bi = __shfl_sync(kFull, bl[s], static_cast<int>(team_base) + I);
        }
        mac_row<S>(t, h0, h1, al, bi);
      }
      uint32_t m = t[0] * c.n0prime;                     // exact on the team's lane 0
      if constexpr (L > 1) m = __shfl_sync(kFull, m, static_cast<int>(team_base));
      if constexpr (SIG) {   // m' > R/2: its top digit, and whether any lower one is nonzero
        if (I * S + s < K - 1) m_low |= m;
        else m_top = m;
      }
      mac_row<S>(t, h0, h1, nl, m);                      // t += m N; the low word is now 0
      uint32_t next0 = 0;                                // lowest limb of the lane above
      if constexpr (L > 1) {
        next0 = __shfl_down_sync(kFull, t[0], 1);
        if (tl == L - 1) next0 = 0;
      }
#pragma unroll
      for (int j = 0; j + 1 < S; ++j) t[j] = t[j + 1];
      const uint32_t top = next0 + h0;
      t[S - 1] = top;
      h0 = h1 + (top < h0 ? 1u : 0u);
      h1 = 0;
    }
    }

    // t = sum over lanes of (slice + h0 at position S).  REDC of a given T
    // adds floor(T / R) now (the reduction loop only consumed T mod R).
    if constexpr (M == Mode::kRedc) h0 += add_rows<S>(t, hi_in);

    uint32_t top_word;  // the element's word at position k (0 or 1 at the end)
    if constexpr (L == 1) {
      top_word = h0;
    } else {
      // resolve the deferred inter-lane carries: lane l's h0 belongs to lane l+1
      uint32_t cin = __shfl_up_sync(kFull, h0, 1);
      if (tl == 0) cin = 0;
      const uint32_t g = add_word<S>(t, cin);
      const unsigned G = team_bits<L>(g != 0, team_base);
      const unsigned P = team_bits<L>(all_ones<S>(t), team_base);
      const unsigned C = lookahead<L>(G, P);
      if ((C >> tl) & 1u) add_word<S>(t, 1u);
      const unsigned carry_out = ((G >> (L - 1)) | ((P >> (L - 1)) & (C >> (L - 1)))) & 1u;
      top_word = __shfl_sync(kFull, h0, static_cast<int>(team_base + L - 1)) + carry_out;
    }

    if constexpr (SIG) {
      uint32_t d[S];
#pragma unroll
      for (int j = 0; j < S; ++j) d[j] = t[j];
      (void)top_word;   // r is taken modulo R
      if constexpr (kProduct) {
        const uint32_t a_neg = (L == 1 ? al[S - 1] : __shfl_sync(kFull, al[S - 1], static_cast<int>(team_base + L - 1))) >> 31;
        const uint32_t b_neg = (L == 1 ? bl[S - 1] : __shfl_sync(kFull, bl[S - 1], static_cast<int>(team_base + L - 1))) >> 31;
        team_sub_masked<S, L>(d, al, 0u - b_neg, team_base, tl);   // - A if b < 0
        team_sub_masked<S, L>(d, bl, 0u - a_neg, team_base, tl);   // - B if a < 0
      }
      const bool gt = m_top > 0x80000000u || (m_top == 0x80000000u && m_low != 0u);
      team_sub_masked<S, L>(d, nl, gt ? 0xFFFFFFFFu : 0u, team_base, tl);   // - N if m' > R/2
      if (valid) store_limbs<S>(out + e * K + tl * S, d, vec16);
      continue;
    }

    // one conditional subtraction of N (t < 2N)
    uint32_t d[S];
    const uint32_t gb = sub_rows<S>(d, t, nl);
    unsigned borrow_out;
    if constexpr (L == 1) {
      borrow_out = gb;
    } else {
      const unsigned G = team_bits<L>(gb != 0, team_base);
      const unsigned P = team_bits<L>(all_zero<S>(d), team_base);
      const unsigned B = lookahead<L>(G, P);
      if ((B >> tl) & 1u) sub_word<S>(d, 1u);
      borrow_out = ((G >> (L - 1)) | ((P >> (L - 1)) & (B >> (L - 1)))) & 1u;
    }
    const bool take_d = top_word != 0 || borrow_out == 0;
    if (valid) {
      uint32_t* o = out + e * K + tl * S;
      if (take_d) store_limbs<S>(o, d, vec16); else store_limbs<S>(o, t, vec16);
    }
  }
}

template <int K, int L, Mode M, bool SIG>
cudaError_t launch_kl(const LimbConst& c, const uint32_t* x, const uint32_t* y, uint32_t* o,
                      size_t n, cudaStream_t s, int vec16, int threads, int bps) {
  const void* k = reinterpret_cast<const void*>(cios_kernel<K, L, M, SIG>);
  const int resident = resident_blocks(k, threads);
  const int per_sm = bps > 0 ? std::min(bps, resident) : resident;
  const size_t teams_per_block = static_cast<size_t>(threads) / L;
  const size_t want = (n + teams_per_block - 1) / teams_per_block;
  const size_t cap = static_cast<size_t>(device_sm_count()) * per_sm;
  const unsigned grid = static_cast<unsigned>(std::max<size_t>(1, std::min(want, cap)));
  cios_kernel<K, L, M, SIG><<<grid, threads, 0, s>>>(x, y, o, n, c, vec16);
  return cudaGetLastError();
}

template <int K, int L>
cudaError_t launch_mode_kl(Mode mode, bool sig, const LimbConst& c, const uint32_t* x,
                           const uint32_t* y, uint32_t* o, size_t n, cudaStream_t s, int vec16,
                           int threads, int bps) {
  if (sig) {
    switch (mode) {
      case Mode::kMul: return launch_kl<K, L, Mode::kMul, true>(c, x, y, o, n, s, vec16, threads, bps);
      case Mode::kToDomain: return launch_kl<K, L, Mode::kToDomain, true>(c, x, y, o, n, s, vec16, threads, bps);
      case Mode::kRedc: return launch_kl<K, L, Mode::kRedc, true>(c, x, y, o, n, s, vec16, threads, bps);
      default: return cudaErrorInvalidValue;
    }
  }
  switch (mode) {
    case Mode::kMul: return launch_kl<K, L, Mode::kMul, false>(c, x, y, o, n, s, vec16, threads, bps);
    case Mode::kToDomain: return launch_kl<K, L, Mode::kToDomain, false>(c, x, y, o, n, s, vec16, threads, bps);
    case Mode::kFromDomain:
      return launch_kl<K, L, Mode::kFromDomain, false>(c, x, y, o, n, s, vec16, threads, bps);
    case Mode::kRedc: return launch_kl<K, L, Mode::kRedc, false>(c, x, y, o, n, s, vec16, threads, bps);
  }
  return cudaErrorInvalidValue;
}

// Team size for a limb count: the tuned one if valid, else the default
// (measured: 1024 bits at 2^17 elements, 2 lanes 57.4 us against 61.5 for 4;
// 2048 bits at 2^15, 4 lanes 62.8 us against 64.6 for 8 and 73.8 for 16).
int default_team(int k) { return k <= 16 ? 1 : (k == 32 ? 2 : 4); }

cudaError_t dispatch(int k, int team, Mode mode, bool sig, const LimbConst& c, const uint32_t* x,
                     const uint32_t* y, uint32_t* o, size_t n, cudaStream_t s, int vec16,
                     int threads, int bps) {
#define MONTGB_KL(K_, L_) \
  if (k == K_ && team == L_) return launch_mode_kl<K_, L_>(mode, sig, c, x, y, o, n, s, vec16, threads, bps);
  MONTGB_KL(4, 1)
  MONTGB_KL(8, 1)
  MONTGB_KL(8, 2)
  MONTGB_KL(12, 1)
  MONTGB_KL(12, 4)
  MONTGB_KL(16, 1)
  MONTGB_KL(16, 2)
  MONTGB_KL(16, 4)
  MONTGB_KL(32, 2)
  MONTGB_KL(32, 4)
  MONTGB_KL(32, 8)
  MONTGB_KL(64, 4)
  MONTGB_KL(64, 8)
  MONTGB_KL(64, 16)
#undef MONTGB_KL
  return cudaErrorInvalidConfiguration;
}

bool team_supported(int k, int team) {
  switch (k) {
    case 4: return team == 1;
    case 8: return team == 1 || team == 2;
    case 12: return team == 1 || team == 4;
    case 16: return team == 1 || team == 2 || team == 4;
    case 32: return team == 2 || team == 4 || team == 8;
    case 64: return team == 4 || team == 8 || team == 16;
  }
  return false;
}

// Block size when none is tuned: 256 threads, 128 for 2048 bits (measured at
// 2^15 elements, four lanes each: 128 threads 62.8 us, 256 threads 63.5 us,
// 64 threads 70.0 us).
int default_threads(int k, int, size_t) { return k == 64 ? 128 : 256; }

bool aligned(const void* p, size_t a) { return (reinterpret_cast<uintptr_t>(p) % a) == 0; }

}  // namespace

bool multilimb_team_supported(int k, int team) { return team_supported(k, team); }

int launch_multilimb_op(mont_ctx_t ctx, Mode mode, const void* x, const void* y, void* out,
                        size_t n, void* stream) {
  const int k = ctx->n_limbs;
  const size_t esize = 4u * static_cast<size_t>(k);
  const size_t in_size = mode == Mode::kRedc ? 2 * esize : esize;
  if (!aligned(x, 4) || !aligned(out, 4) || (y && !aligned(y, 4))) return MONT_EINVAL;
  if (n > SIZE_MAX / in_size) return MONT_EINVAL;
  const uintptr_t xo = reinterpret_cast<uintptr_t>(x), oo = reinterpret_cast<uintptr_t>(out);
  const bool same = xo == oo;
  if (!same && xo < oo + n * esize && oo < xo + n * in_size) return MONT_EINVAL;
  if (mode == Mode::kRedc && same) return MONT_EINVAL;
  if (mode == Mode::kMul) {
    const uintptr_t yo = reinterpret_cast<uintptr_t>(y);
    if (yo != oo && yo < oo + n * esize && oo < yo + n * esize) return MONT_EINVAL;
  }
  // Algorithm 1's products and reductions run on the CIOS schedule (see the
  // top of this file); its from_domain, which also canonicalises, and
  // Algorithms 2-4 run in limb_variants.cu
  const bool sig = ctx->variant == MONT_SIGNED && mode != Mode::kFromDomain;
  if (ctx->variant != MONT_REDC && !sig) {   // limb_variants.cu
    const int v16 = aligned(x, 16) && aligned(out, 16) && (!y || aligned(y, 16)) ? 1 : 0;
    return cuda_status(launch_limb_variant(k, mode, ctx->limbv, static_cast<const uint32_t*>(x),
                                           static_cast<const uint32_t*>(y),
                                           static_cast<uint32_t*>(out), n,
                                           static_cast<cudaStream_t>(stream), v16,
                                           tuned_shape(ctx->width, ctx->variant,
                                                       static_cast<int>(mode))));
  }
  LaunchShape shape = tuned_shape(ctx->width, ctx->variant, static_cast<int>(mode));
  int team = shape.team > 0 ? shape.team : default_team(k);
  if (!team_supported(k, team)) team = default_team(k);
  int threads = shape.threads;
  if (threads != 32 && threads != 64 && threads != 128 && threads != 256) {
    threads = default_threads(k, team, n);
  }
  const int vec16 = aligned(x, 16) && aligned(out, 16) && (!y || aligned(y, 16)) ? 1 : 0;
  const cudaError_t e = dispatch(k, team, mode, sig, ctx->limb, static_cast<const uint32_t*>(x),
                                 static_cast<const uint32_t*>(y), static_cast<uint32_t*>(out), n,
                                 static_cast<cudaStream_t>(stream), vec16, threads,
                                 shape.blocks_per_sm);
  return cuda_status(e);
}

}  // namespace montgb
