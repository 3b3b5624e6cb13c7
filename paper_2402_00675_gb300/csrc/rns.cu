// Residue-number-system conversions (mont_rns_*): the multi-modulus CRT that
// Section 2 derives in the two-modulus case from Qin's identity.
//
// Big integer -> residues.  X mod p = sum_j X_j 2^{32 j} mod p over the 32-bit
// limbs X_j.  With c_j = 2^{32 j} R mod p (R = 2^64), REDC(sum_j X_j c_j) =
// X mod p: the sum of k products of a limb and a word stays below k 2^32 p <
// p R, so it is accumulated exactly in 128 bits and reduced once.  The sums
// form a product of an (elements x limbs) matrix and a (limbs x moduli)
// matrix, so the kernel is tiled like one: a block converts 64 elements for
// a group of up to 32 moduli, with the tile's limbs staged in shared memory
// transposed ([limb][element], rows padded to 65 words, so that both the
// coalesced staging writes and the per-limb reads are free of bank
// conflicts) and the group's c_j as [limb][modulus].  Warp w takes moduli
// 4w..4w+3 of the group and lane l elements l and l+32 of the tile: every
// thread keeps 2 x 4 sums of four 32-bit words and spends one carry chain
// (two mad.lo, two mad.hi, three addc) per limb product, reading one limb
// per element and one broadcast 32-byte row of constants per limb.
//
// Residues -> big integer: the CRT formula itself.  With M_i = P / p_i and
// xh_i = x_i M_i^{-1} mod p_i, S = sum_i xh_i M_i is congruent to X modulo
// every p_i and S / P = sum_i xh_i / p_i, so X = S - qP with q = floor(S/P).
// q comes from 64-bit fractions f_i = floor(xh_i floor(2^128 / p_i) / 2^64)
// <= xh_i 2^64 / p_i, each at most 2 below it: q' = floor(sum_i f_i / 2^64)
// is q or q - 1, so S - q'P lies in [0, 2P) and one conditional subtraction
// of P finishes.  S - q'P is formed in the same product as S, by one more
// row q' (2^{32K} - P): its extra q' 2^{32K} falls above the K limbs kept.
// The product is an (elements x moduli) by (moduli x limbs) matrix product,
// tiled like the conversion above: a block takes 64 elements; warp w owns
// limbs K/8 w .. K/8 (w+1) - 1 and lane l elements l and l + 32, each output
// a 128-bit sum, with xh staged in shared memory as [modulus][element] and
// M as [modulus][limb] (read as broadcasts).  Each thread then folds its
// limbs into words plus a carry out of its group; one thread per element
// adds the groups' carries in order and subtracts P if needed.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "word_kernel.cuh"

namespace montgb {
namespace {

constexpr int kRnsMaxModuli = 64;

// a[0..3] += v c  (a 32-bit limb times a 64-bit word into a 128-bit sum)
__device__ __forceinline__ void mac_limb_word(uint32_t (&a)[4], uint32_t v, uint64_t c) {
  const uint32_t c0 = static_cast<uint32_t>(c), c1 = static_cast<uint32_t>(c >> 32);
  asm("mad.lo.cc.u32 %0, %4, %5, %0;\n\t"
      "madc.hi.cc.u32 %1, %4, %5, %1;\n\t"
      "madc.hi.cc.u32 %2, %4, %6, %2;\n\t"
      "addc.u32 %3, %3, 0;\n\t"
      "mad.lo.cc.u32 %1, %4, %6, %1;\n\t"
      "addc.cc.u32 %2, %2, 0;\n\t"
      "addc.u32 %3, %3, 0;"
      : "+r"(a[0]), "+r"(a[1]), "+r"(a[2]), "+r"(a[3])
      : "r"(v), "r"(c0), "r"(c1));
}

constexpr int kToTile = 64;    // elements per tile
constexpr int kToGroup = 32;   // moduli per block

template <int K>
__global__ void __launch_bounds__(256) rns_to_kernel(const uint32_t* __restrict__ X,
                                                     uint64_t* __restrict__ res, size_t n,
                                                     int count,
                                                     const WordConst64* __restrict__ mods,
                                                     const uint64_t* __restrict__ c) {
  __shared__ uint32_t xs[K][kToTile + 1];
  __shared__ __align__(16) uint64_t cs[K][kToGroup];
  const int m0 = static_cast<int>(blockIdx.y) * kToGroup;   // first modulus of the group
  const int mc = min(kToGroup, count - m0);
  for (int w = threadIdx.x; w < kToGroup * K; w += blockDim.x) {
    const int m = w / K, j = w % K;
    cs[j][m] = m < mc ? c[static_cast<size_t>(m0 + m) * K + j] : 0;
  }
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t tiles = (n + kToTile - 1) / kToTile;
  for (size_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const size_t e0 = tile * kToTile;
    __syncthreads();   // the previous tile's reads are done (and cs is staged)
    for (int w = threadIdx.x; w < kToTile * K; w += blockDim.x) {
      const int e = w / K, j = w % K;
      xs[j][e] = e0 + e < n ? X[e0 * K + w] : 0u;
    }
    __syncthreads();
    if (4 * warp >= mc) continue;
    uint32_t acc[2][4][4];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int q = 0; q < 4; ++q)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[h][q][t] = 0;
#pragma unroll 8
    for (int j = 0; j < K; ++j) {
      const uint32_t v0 = xs[j][lane], v1 = xs[j][lane + 32];
      const ulonglong2 ca = *reinterpret_cast<const ulonglong2*>(&cs[j][4 * warp]);
      const ulonglong2 cb = *reinterpret_cast<const ulonglong2*>(&cs[j][4 * warp + 2]);
      mac_limb_word(acc[0][0], v0, ca.x);
      mac_limb_word(acc[0][1], v0, ca.y);
      mac_limb_word(acc[0][2], v0, cb.x);
      mac_limb_word(acc[0][3], v0, cb.y);
      mac_limb_word(acc[1][0], v1, ca.x);
      mac_limb_word(acc[1][1], v1, ca.y);
      mac_limb_word(acc[1][2], v1, cb.x);
      mac_limb_word(acc[1][3], v1, cb.y);
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int i = m0 + 4 * warp + q;
      if (i >= count) break;
      const WordConst64 m = mods[i];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const size_t e = e0 + lane + 32 * h;
        if (e >= n) continue;
        const uint32_t* a4 = acc[h][q];
        const u128 T = (static_cast<u128>((static_cast<uint64_t>(a4[3]) << 32) | a4[2]) << 64) |
                       ((static_cast<uint64_t>(a4[1]) << 32) | a4[0]);
        res[static_cast<size_t>(i) * n + e] = Redc64::reduce(T, m);
      }
    }
  }
}

// The 128-bit value of four little-endian words.
__device__ __forceinline__ u128 sum128(const uint32_t (&a)[4]) {
  return (static_cast<u128>((static_cast<uint64_t>(a[3]) << 32) | a[2]) << 64) |
         ((static_cast<uint64_t>(a[1]) << 32) | a[0]);
}

constexpr int kCrtGroups = 8;  // limb groups (one per warp)
constexpr int kCrtEpt = 1;     // elements per thread: a block tile is 32 kCrtEpt elements

// Dynamic shared memory of the reconstruction for K limbs and count moduli
// (rows = count + 1, the last row being q' and 2^{32K} - P):
//   ms [rows][K] uint32, xh [rows][T] uint64, st [T][K+1] uint32,
//   ov [8 groups][4 words][T] uint32, fr [256 / T parts][2 words][T] uint64, P [K] uint32
// for a tile of T = 32 kCrtEpt elements.
size_t crt_smem_bytes(int K, int count) {
  const size_t rows = static_cast<size_t>(count) + 1, T = 32 * kCrtEpt;
  return rows * K * 4 + rows * T * 8 + T * (K + 1) * 4 + kCrtGroups * 4 * T * 4 + 256 * 2 * 8 +
         static_cast<size_t>(K) * 4;
}

template <int K>
__global__ void __launch_bounds__(256) rns_crt_kernel(const uint64_t* __restrict__ res,
                                                      uint32_t* __restrict__ X, size_t n,
                                                      int count,
                                                      const WordConst64* __restrict__ mods,
                                                      const uint64_t* __restrict__ cinv,
                                                      const uint64_t* __restrict__ recip,
                                                      const uint32_t* __restrict__ Mt,
                                                      const uint32_t* __restrict__ Pl) {
  constexpr int LPW = K / kCrtGroups;   // limbs of one warp
  constexpr int kCrtTile = 32 * kCrtEpt;
  constexpr int kParts = 256 / kCrtTile;
  extern __shared__ __align__(16) unsigned char smem[];
  const int rows = count + 1;
  uint32_t* ms = reinterpret_cast<uint32_t*>(smem);                   // [rows][K]
  uint64_t* xh = reinterpret_cast<uint64_t*>(ms + rows * K);          // [rows][64]
  uint32_t* st = reinterpret_cast<uint32_t*>(xh + rows * kCrtTile);   // [64][K+1]
  uint32_t* ov = st + kCrtTile * (K + 1);                             // [8][4][64]
  uint64_t* fr = reinterpret_cast<uint64_t*>(ov + kCrtGroups * 4 * kCrtTile);   // [parts][2][T]
  uint32_t* ps = reinterpret_cast<uint32_t*>(fr + kParts * 2 * kCrtTile);  // [K]
  for (int w = threadIdx.x; w < rows * K; w += blockDim.x) ms[w] = Mt[w];
  for (int w = threadIdx.x; w < K; w += blockDim.x) ps[w] = Pl[w];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const size_t tiles = (n + kCrtTile - 1) / kCrtTile;
  for (size_t tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const size_t e0 = tile * kCrtTile;
    __syncthreads();   // the previous tile is written out (and ms, ps are staged)
    {  // xh_i = REDC(x_i (M_i^{-1} R mod p_i)) and the fractions, in parts of the moduli
      const int e = threadIdx.x & (kCrtTile - 1), part = threadIdx.x / kCrtTile;
      const bool valid = e0 + e < n;
      u128 f = 0;
      for (int i = part; i < count; i += kParts) {
        const uint64_t x = valid ? res[static_cast<size_t>(i) * n + e0 + e] : 0u;
        const uint64_t h = Redc64::reduce(static_cast<u128>(x) * cinv[i], mods[i]);
        xh[i * kCrtTile + e] = h;
        f += h * recip[2 * i + 1] + __umul64hi(h, recip[2 * i]);   // floor(h recip / 2^64) < 2^64
      }
      fr[(part * 2) * kCrtTile + e] = static_cast<uint64_t>(f);
      fr[(part * 2 + 1) * kCrtTile + e] = static_cast<uint64_t>(f >> 64);
    }
    __syncthreads();
    if (threadIdx.x < kCrtTile) {   // q' = floor(sum of the fractions / 2^64): the last row
      const int e = threadIdx.x;
      u128 f = 0;
      for (int part = 0; part < kParts; ++part)
        f += (static_cast<u128>(fr[(part * 2 + 1) * kCrtTile + e]) << 64) | fr[(part * 2) * kCrtTile + e];
      xh[count * kCrtTile + e] = static_cast<uint64_t>(f >> 64);
    }
    __syncthreads();
    // S - q'P + q' 2^{32K} = sum over the rows of xh M: this warp's limbs,
    // elements lane + 32 h
    uint32_t acc[kCrtEpt][LPW][4];
#pragma unroll
    for (int h = 0; h < kCrtEpt; ++h)
#pragma unroll
      for (int jj = 0; jj < LPW; ++jj)
#pragma unroll
        for (int t = 0; t < 4; ++t) acc[h][jj][t] = 0u;
#pragma unroll 4
    for (int i = 0; i < rows; ++i) {
      uint64_t v[kCrtEpt];
#pragma unroll
      for (int h = 0; h < kCrtEpt; ++h) v[h] = xh[i * kCrtTile + lane + 32 * h];
      const uint32_t* mrow = ms + i * K + warp * LPW;
#pragma unroll
      for (int jj = 0; jj < LPW; ++jj) {
        const uint32_t m = mrow[jj];
#pragma unroll
        for (int h = 0; h < kCrtEpt; ++h) mac_limb_word(acc[h][jj], m, v[h]);
      }
    }
    // the group's limbs with the carries inside the group, and its carry out (< 2^72)
    uint32_t lim[kCrtEpt][LPW];
#pragma unroll
    for (int h = 0; h < kCrtEpt; ++h) {
      const int e = lane + 32 * h;
      u128 pend = 0;
#pragma unroll
      for (int jj = 0; jj < LPW; ++jj) {
        const u128 sum = sum128(acc[h][jj]) + pend;
        lim[h][jj] = static_cast<uint32_t>(sum);
        pend = sum >> 32;
      }
      ov[(warp * 4 + 0) * kCrtTile + e] = static_cast<uint32_t>(pend);
      ov[(warp * 4 + 1) * kCrtTile + e] = static_cast<uint32_t>(pend >> 32);
      ov[(warp * 4 + 2) * kCrtTile + e] = static_cast<uint32_t>(pend >> 64);
    }
    __syncthreads();
    if constexpr (LPW >= 4) {
      // Groups of at least 128 bits: a carry out below 2^72 added to a group
      // leaves it at most one bit, so the groups settle in parallel with
      // generate / propagate bits (a word of flags per group and element).
      uint32_t* fl = st;   // [8 groups][64 elements] flags (st is free in this path)
#pragma unroll
      for (int h = 0; h < kCrtEpt; ++h) {
        const int e = lane + 32 * h;
        uint32_t gen = 0, all1 = 0xFFFFFFFFu;
        if (warp > 0) {
          u128 cin = (static_cast<u128>(ov[((warp - 1) * 4 + 2) * kCrtTile + e]) << 64) |
                     (static_cast<u128>(ov[((warp - 1) * 4 + 1) * kCrtTile + e]) << 32) |
                     ov[((warp - 1) * 4) * kCrtTile + e];
#pragma unroll
          for (int jj = 0; jj < LPW; ++jj) {
            const u128 sum = static_cast<u128>(lim[h][jj]) + cin;
            lim[h][jj] = static_cast<uint32_t>(sum);
            cin = sum >> 32;
          }
          gen = static_cast<uint32_t>(cin);   // 0 or 1
        }
#pragma unroll
        for (int jj = 0; jj < LPW; ++jj) all1 &= lim[h][jj];
        fl[warp * kCrtTile + e] = gen | (all1 == 0xFFFFFFFFu ? 2u : 0u);
      }
      __syncthreads();
      // the carry bit into this group, then X' >= P: compare the groups with P's
      uint32_t take[kCrtEpt];
#pragma unroll
      for (int h = 0; h < kCrtEpt; ++h) {
        const int e = lane + 32 * h;
        uint32_t c = 0;
        for (int g = 0; g < warp; ++g) {
          const uint32_t f = fl[g * kCrtTile + e];
          c = (f & 1u) | ((f >> 1) & c);
        }
        if (c) {
#pragma unroll
          for (int jj = 0; jj < LPW; ++jj) {   // + 1; the carry out was counted above
            lim[h][jj] += c;
            c = lim[h][jj] == 0u ? c : 0u;
          }
        }
        // borrow of this group's limbs minus P's (generate) and equality (propagate)
        uint32_t borrow = 0, eq = 1;
#pragma unroll
        for (int jj = 0; jj < LPW; ++jj) {
          const uint32_t pj = ps[warp * LPW + jj];
          const uint64_t d = static_cast<uint64_t>(lim[h][jj]) - pj - borrow;
          borrow = static_cast<uint32_t>(d >> 63);
          eq &= lim[h][jj] == pj ? 1u : 0u;
        }
        take[h] = borrow | (eq << 1);
      }
      __syncthreads();   // every group has read the carry flags
#pragma unroll
      for (int h = 0; h < kCrtEpt; ++h) fl[warp * kCrtTile + lane + 32 * h] = take[h];
      __syncthreads();
#pragma unroll
      for (int h = 0; h < kCrtEpt; ++h) {
        const int e = lane + 32 * h;
        if (e0 + e >= n) continue;
        uint32_t b = 0, bin = 0;   // borrow into the top of every group; into this one
        for (int g = 0; g < kCrtGroups; ++g) {
          if (g == warp) bin = b;
          const uint32_t f = fl[g * kCrtTile + e];
          b = (f & 1u) | ((f >> 1) & b);
        }
        const uint32_t mask = b ? 0u : 0xFFFFFFFFu;   // no borrow out of the top: X' >= P
        uint32_t borrow = bin & (mask & 1u);
#pragma unroll
        for (int jj = 0; jj < LPW; ++jj) {
          const uint64_t d = static_cast<uint64_t>(lim[h][jj]) - (ps[warp * LPW + jj] & mask) - borrow;
          lim[h][jj] = static_cast<uint32_t>(d);
          borrow = static_cast<uint32_t>(d >> 63);
        }
        uint4* o = reinterpret_cast<uint4*>(X + (e0 + e) * K + warp * LPW);
#pragma unroll
        for (int q = 0; q < LPW / 4; ++q)
          o[q] = make_uint4(lim[h][4 * q], lim[h][4 * q + 1], lim[h][4 * q + 2], lim[h][4 * q + 3]);
      }
    } else {
      // narrow groups: one thread per element settles the carries in order
#pragma unroll
      for (int h = 0; h < kCrtEpt; ++h)
#pragma unroll
        for (int jj = 0; jj < LPW; ++jj) st[(lane + 32 * h) * (K + 1) + warp * LPW + jj] = lim[h][jj];
      __syncthreads();
      if (threadIdx.x < kCrtTile && e0 + threadIdx.x < n) {
        const int e = threadIdx.x;
        uint32_t* sv = st + e * (K + 1);
        // carry each group's carry out into the groups above; what passes limb
        // K - 1 is q' 2^{32K} (and nothing else, since S - q'P < 2P <= 2^{32K})
        u128 pend = 0;
        for (int g = 1; g < kCrtGroups; ++g) {
          pend += (static_cast<u128>(ov[((g - 1) * 4 + 2) * kCrtTile + e]) << 64) |
                  (static_cast<u128>(ov[((g - 1) * 4 + 1) * kCrtTile + e]) << 32) |
                  ov[((g - 1) * 4) * kCrtTile + e];
#pragma unroll
          for (int jj = 0; jj < LPW; ++jj) {
            const u128 sum = static_cast<u128>(sv[g * LPW + jj]) + pend;
            sv[g * LPW + jj] = static_cast<uint32_t>(sum);
            pend = sum >> 32;
          }
        }
        // X' in [0, 2P): subtract P once if X' >= P
        uint32_t borrow = 0;
        for (int j = 0; j < K; ++j) {
          const uint64_t d = static_cast<uint64_t>(sv[j]) - ps[j] - borrow;
          borrow = static_cast<uint32_t>(d >> 63);
        }
        const uint32_t take = borrow ? 0u : 0xFFFFFFFFu;
        borrow = 0;
        for (int j = 0; j < K; ++j) {
          const uint64_t d = static_cast<uint64_t>(sv[j]) - (ps[j] & take) - borrow;
          sv[j] = static_cast<uint32_t>(d);
          borrow = static_cast<uint32_t>(d >> 63);
        }
      }
      __syncthreads();
      for (int w = threadIdx.x; w < kCrtTile * K; w += blockDim.x) {
        const int e = w / K, j = w % K;
        if (e0 + e < n) X[(e0 + e) * K + j] = st[e * (K + 1) + j];
      }
    }
  }
}

// ------------------------------------------------------------- host helpers

using u128h = unsigned __int128;

uint64_t gcd64(uint64_t a, uint64_t b) {
  while (b) {
    const uint64_t t = a % b;
    a = b;
    b = t;
  }
  return a;
}
uint64_t mulmod64(uint64_t a, uint64_t b, uint64_t p) {
  return static_cast<uint64_t>(static_cast<u128h>(a) * b % p);
}
uint64_t invmod64(uint64_t a, uint64_t p) {   // a^{-1} mod p, gcd(a, p) = 1
  __int128 r0 = p, r1 = a % p, s0 = 0, s1 = 1;
  while (r1 != 0) {
    const __int128 q = r0 / r1;
    __int128 t = r0 - q * r1; r0 = r1; r1 = t;
    t = s0 - q * s1; s0 = s1; s1 = t;
  }
  __int128 s = s0 % static_cast<__int128>(p);
  if (s < 0) s += p;
  return static_cast<uint64_t>(s);
}

template <int K>
cudaError_t launch_to(const uint32_t* X, uint64_t* res, size_t n, int count, const WordConst64* mods,
                      const uint64_t* c, cudaStream_t s) {
  const void* k = reinterpret_cast<const void*>(rns_to_kernel<K>);
  const unsigned groups = static_cast<unsigned>((count + kToGroup - 1) / kToGroup);
  const size_t tiles = (n + kToTile - 1) / kToTile;
  const size_t cap = static_cast<size_t>(device_sm_count()) * resident_blocks(k, 256) / groups;
  const dim3 grid(static_cast<unsigned>(std::max<size_t>(1, std::min(tiles, cap))), groups);
  rns_to_kernel<K><<<grid, 256, 0, s>>>(X, res, n, count, mods, c);
  return cudaGetLastError();
}

template <int K>
cudaError_t launch_crt(const uint64_t* res, uint32_t* X, size_t n, int count,
                       const WordConst64* mods, const uint64_t* cinv, const uint64_t* recip,
                       const uint32_t* Mt, const uint32_t* Pl, cudaStream_t s) {
  const void* k = reinterpret_cast<const void*>(rns_crt_kernel<K>);
  const size_t smem = crt_smem_bytes(K, count);
  if (smem > 48u * 1024u) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);
  if (e != cudaSuccess) return e;
  const size_t tiles = (n + 32 * kCrtEpt - 1) / (32 * kCrtEpt);
  const size_t cap = static_cast<size_t>(device_sm_count()) * static_cast<size_t>(std::max(per_sm, 1));
  rns_crt_kernel<K><<<static_cast<unsigned>(std::min(tiles, cap)), 256, smem, s>>>(
      res, X, n, count, mods, cinv, recip, Mt, Pl);
  return cudaGetLastError();
}

}  // namespace
}  // namespace montgb

using namespace montgb;

struct mont_rns {
  int count = 0;
  int limbs = 0;                 // K: limbs of every big integer (32 K > bits of P)
  void* dev = nullptr;           // one allocation for every table below
  WordConst64* d_mods = nullptr; // Montgomery constants of each p_i (R = 2^64)
  uint64_t* d_c = nullptr;       // [count][K]: 2^{32 j} R mod p_i
  uint64_t* d_cinv = nullptr;    // [count]: M_i^{-1} R mod p_i, M_i = P / p_i
  uint64_t* d_recip = nullptr;   // [count][2]: floor(2^128 / p_i), low and high word
  uint32_t* d_Mt = nullptr;      // [count + 1][K]: M_i, then 2^{32K} - P
  uint32_t* d_P = nullptr;       // [K]: P
};

extern "C" int mont_rns_create(mont_rns_t* out, const uint64_t* moduli, int count) {
  if (!out || !moduli || count < 1 || count > kRnsMaxModuli) return MONT_EINVAL;
  for (int i = 0; i < count; ++i) {
    const uint64_t p = moduli[i];
    if (p < 3 || !(p & 1) || (p >> 63)) return MONT_EINVAL;
    for (int j = 0; j < i; ++j)
      if (gcd64(p, moduli[j]) != 1) return MONT_EINVAL;
  }
  // Pi_i = p_0 ... p_{i-1} as 32-bit limbs, and P = Pi_count
  std::vector<std::vector<uint32_t>> Pi(count + 1);
  Pi[0] = {1u};
  for (int i = 0; i < count; ++i) {
    const std::vector<uint32_t>& a = Pi[i];
    std::vector<uint32_t> r(a.size() + 2, 0u);
    const uint64_t p = moduli[i];
    u128h carry = 0;
    for (size_t j = 0; j < r.size(); ++j) {
      const u128h t = (j < a.size() ? static_cast<u128h>(a[j]) * p : 0) + carry;
      r[j] = static_cast<uint32_t>(t);
      carry = t >> 32;
    }
    while (r.size() > 1 && r.back() == 0) r.pop_back();
    Pi[i + 1] = r;
  }
  const std::vector<uint32_t>& P = Pi[count];
  int bitsP = 32 * static_cast<int>(P.size());
  for (uint32_t top = P.back(); !(top >> 31); top <<= 1) --bitsP;
  int K = 8;
  while (32 * K <= bitsP) K *= 2;   // one spare bit: the reconstruction needs 2P < 2^{32K}
  if (K > 64) return MONT_EINVAL;    // P of 2048 bits or more

  std::vector<WordConst64> mods(count);
  std::vector<uint64_t> c(static_cast<size_t>(count) * K);
  std::vector<uint64_t> cinv(count);
  std::vector<uint64_t> recip(2 * static_cast<size_t>(count));
  std::vector<uint32_t> Mt(static_cast<size_t>(count + 1) * K, 0u);
  std::vector<uint32_t> Pl(K, 0u);
  for (size_t j = 0; j < P.size(); ++j) Pl[j] = P[j];
  for (int i = 0; i < count; ++i) {
    const uint64_t p = moduli[i];
    WordConst64 m{};
    m.N = p;
    uint64_t x = p;   // N^{-1} mod 2^64 by Newton-Hensel
    for (int it = 0; it < 6; ++it) x *= 2 - p * x;
    m.ninv = x;
    m.nprime = 0 - x;
    m.half = (p - 1) / 2;
    mods[i] = m;
    const uint64_t r64 = static_cast<uint64_t>((static_cast<u128h>(1) << 64) % p);   // R mod p
    const uint64_t two32 = static_cast<uint64_t>((static_cast<u128h>(1) << 32) % p);
    uint64_t cj = r64;   // 2^{32 j} R mod p
    for (int j = 0; j < K; ++j) {
      c[static_cast<size_t>(i) * K + j] = cj;
      cj = mulmod64(cj, two32, p);
    }
    // M_i = P / p_i by long division over the limbs of P
    u128h rem = 0;
    for (int j = K - 1; j >= 0; --j) {
      const u128h cur = (rem << 32) | Pl[j];
      Mt[static_cast<size_t>(i) * K + j] = static_cast<uint32_t>(cur / p);
      rem = cur % p;
    }
    uint64_t mm = 1 % p;   // M_i mod p_i = prod_{j != i} p_j mod p_i
    for (int j = 0; j < count; ++j)
      if (j != i) mm = mulmod64(mm, moduli[j] % p, p);
    cinv[i] = mulmod64(invmod64(mm, p), r64, p);
    const u128h rc = ~static_cast<u128h>(0) / p;   // floor((2^128 - 1) / p) = floor(2^128 / p)
    recip[2 * static_cast<size_t>(i)] = static_cast<uint64_t>(rc);
    recip[2 * static_cast<size_t>(i) + 1] = static_cast<uint64_t>(rc >> 64);
  }
  {  // the last row: 2^{32K} - P, two's complement of P over K limbs
    uint64_t borrow = 0;
    for (int j = 0; j < K; ++j) {
      const uint64_t d = 0 - static_cast<uint64_t>(Pl[j]) - borrow;
      Mt[static_cast<size_t>(count) * K + j] = static_cast<uint32_t>(d);
      borrow = (d >> 32) & 1u;
    }
  }
  mont_rns* r = new (std::nothrow) mont_rns;
  if (!r) return MONT_ENOMEM;
  r->count = count;
  r->limbs = K;
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  const size_t b_mods = count * sizeof(WordConst64), b_c = c.size() * 8, b_cinv = cinv.size() * 8,
               b_recip = recip.size() * 8, b_Mt = Mt.size() * 4, b_P = Pl.size() * 4;
  const size_t off_c = up(b_mods), off_cinv = off_c + up(b_c), off_recip = off_cinv + up(b_cinv),
               off_Mt = off_recip + up(b_recip), off_P = off_Mt + up(b_Mt);
  cudaError_t e = cudaMalloc(&r->dev, off_P + b_P);
  if (e == cudaSuccess) {
    char* base = static_cast<char*>(r->dev);
    r->d_mods = reinterpret_cast<WordConst64*>(base);
    r->d_c = reinterpret_cast<uint64_t*>(base + off_c);
    r->d_cinv = reinterpret_cast<uint64_t*>(base + off_cinv);
    r->d_recip = reinterpret_cast<uint64_t*>(base + off_recip);
    r->d_Mt = reinterpret_cast<uint32_t*>(base + off_Mt);
    r->d_P = reinterpret_cast<uint32_t*>(base + off_P);
    e = cudaMemcpy(r->d_mods, mods.data(), b_mods, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_c, c.data(), b_c, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_cinv, cinv.data(), b_cinv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_recip, recip.data(), b_recip, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_Mt, Mt.data(), b_Mt, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_P, Pl.data(), b_P, cudaMemcpyHostToDevice);
  }
  if (e != cudaSuccess) {
    if (r->dev) cudaFree(r->dev);
    delete r;
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? MONT_ENOMEM : cuda_status(e);
  }
  *out = r;
  return MONT_OK;
}

extern "C" int mont_rns_query(mont_rns_t r, int* count, int* limbs) {
  if (!r) return MONT_EINVAL;
  if (count) *count = r->count;
  if (limbs) *limbs = r->limbs;
  return MONT_OK;
}

extern "C" int mont_rns_destroy(mont_rns_t r) {
  if (!r) return MONT_OK;
  if (r->dev) cudaFree(r->dev);
  delete r;
  return MONT_OK;
}

static int rns_check(mont_rns_t r, const void* big, const void* res, size_t n) {
  if (!r) return MONT_EINVAL;
  if (n == 0) return 1;
  if (!big || !res) return MONT_EINVAL;
  if (reinterpret_cast<uintptr_t>(big) % 16 || reinterpret_cast<uintptr_t>(res) % 8) return MONT_EINVAL;
  const size_t bb = n * 4u * static_cast<size_t>(r->limbs);
  const size_t rb = n * 8u * static_cast<size_t>(r->count);
  const uintptr_t a = reinterpret_cast<uintptr_t>(big), b = reinterpret_cast<uintptr_t>(res);
  if (a < b + rb && b < a + bb) return MONT_EINVAL;
  return 0;
}

extern "C" int mont_rns_to_residues(mont_rns_t r, const uint32_t* X, uint64_t* residues, size_t n,
                                    void* stream) {
  const int chk = rns_check(r, X, residues, n);
  if (chk) return chk == 1 ? MONT_OK : chk;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (r->limbs) {
    case 8: e = launch_to<8>(X, residues, n, r->count, r->d_mods, r->d_c, s); break;
    case 16: e = launch_to<16>(X, residues, n, r->count, r->d_mods, r->d_c, s); break;
    case 32: e = launch_to<32>(X, residues, n, r->count, r->d_mods, r->d_c, s); break;
    default: e = launch_to<64>(X, residues, n, r->count, r->d_mods, r->d_c, s); break;
  }
  return cuda_status(e);
}

extern "C" int mont_rns_from_residues(mont_rns_t r, const uint64_t* residues, uint32_t* X, size_t n,
                                      void* stream) {
  const int chk = rns_check(r, X, residues, n);
  if (chk) return chk == 1 ? MONT_OK : chk;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaError_t e;
  switch (r->limbs) {
    case 8: e = launch_crt<8>(residues, X, n, r->count, r->d_mods, r->d_cinv, r->d_recip, r->d_Mt, r->d_P, s); break;
    case 16: e = launch_crt<16>(residues, X, n, r->count, r->d_mods, r->d_cinv, r->d_recip, r->d_Mt, r->d_P, s); break;
    case 32: e = launch_crt<32>(residues, X, n, r->count, r->d_mods, r->d_cinv, r->d_recip, r->d_Mt, r->d_P, s); break;
    default: e = launch_crt<64>(residues, X, n, r->count, r->d_mods, r->d_cinv, r->d_recip, r->d_Mt, r->d_P, s); break;
  }
  return cuda_status(e);
}
