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
// Residues -> big integer.  Mixed radix (Garner): X = sum_i v_i Pi_i with
// Pi_i = p_0 ... p_{i-1} and v_i = (x_i - X_{<i}) Pi_i^{-1} mod p_i, where
// X_{<i} = sum_{j<i} v_j Pi_j is the partial value already built.  One thread
// per element keeps X in registers as 32-bit limbs; each step reduces X_{<i}
// modulo p_i with the lazy accumulation above, forms v_i with one REDC
// (Pi_i^{-1} kept in Montgomery form), and adds v_i Pi_i limb by limb.  Since
// X_{<i} < Pi_i, both passes of step i run only over the limbs of Pi_i and
// Pi_{i+1} (in blocks of four, a warp-uniform skip), about half of all.  The
// result is the unique X in [0, P), P = prod p_i, with no quotient estimate
// and no correction step.
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

// Dynamic shared memory of the residues -> big kernel: the constants of
// every step, staged once per block (the steps read them in lock step, so
// every read is a broadcast).
size_t from_smem_bytes(int K, int count) {
  return static_cast<size_t>(count) * K * (sizeof(uint64_t) + sizeof(uint32_t)) +
         static_cast<size_t>(count) * (sizeof(uint64_t) + sizeof(WordConst64)) +
         static_cast<size_t>(count + 1) * sizeof(int);
}

template <int K>
__global__ void __launch_bounds__(256) rns_from_kernel(const uint64_t* __restrict__ res,
                                                       uint32_t* __restrict__ X, size_t n,
                                                       int count,
                                                       const WordConst64* __restrict__ mods,
                                                       const uint64_t* __restrict__ c,
                                                       const uint32_t* __restrict__ pi,
                                                       const uint64_t* __restrict__ inv,
                                                       const int* __restrict__ live) {
  extern __shared__ __align__(16) unsigned char smem[];
  uint64_t* cs = reinterpret_cast<uint64_t*>(smem);                      // count x K
  WordConst64* ms = reinterpret_cast<WordConst64*>(cs + count * K);      // count
  uint64_t* is = reinterpret_cast<uint64_t*>(ms + count);                // count
  uint32_t* ps = reinterpret_cast<uint32_t*>(is + count);                // count x K
  int* ls = reinterpret_cast<int*>(ps + count * K);                      // count + 1
  for (int w = threadIdx.x; w < count * K; w += blockDim.x) {
    cs[w] = c[w];
    ps[w] = pi[w];
  }
  for (int w = threadIdx.x; w < count; w += blockDim.x) {
    ms[w] = mods[w];
    is[w] = inv[w];
  }
  for (int w = threadIdx.x; w <= count; w += blockDim.x) ls[w] = live[w];
  __syncthreads();
  for (size_t e = static_cast<size_t>(blockIdx.x) * blockDim.x + threadIdx.x; e < n;
       e += static_cast<size_t>(gridDim.x) * blockDim.x) {
    uint32_t x[K];
#pragma unroll
    for (int j = 0; j < K; ++j) x[j] = 0;
    uint64_t xi_next = res[e];
    for (int i = 0; i < count; ++i) {
      const uint64_t xi = xi_next;
      if (i + 1 < count) xi_next = res[static_cast<size_t>(i + 1) * n + e];   // one step ahead
      const WordConst64 m = ms[i];
      const uint64_t* ci = cs + i * K;
      const uint32_t* pii = ps + i * K;
      // X_{<i} < Pi_i and X_{<i+1} < Pi_{i+1}: only their limbs can be non-zero
      const int li = ls[i], ln = ls[i + 1];
      // r = X_{<i} mod p_i, over the live limbs (blocks of 4; the skip is warp-uniform)
      uint32_t a[4] = {0u, 0u, 0u, 0u};
#pragma unroll
      for (int q = 0; q < K / 4; ++q) {
        if (4 * q < li) {
#pragma unroll
          for (int t = 0; t < 4; ++t) mac_limb_word(a, x[4 * q + t], ci[4 * q + t]);
        }
      }
      const u128 T = (static_cast<u128>((static_cast<uint64_t>(a[3]) << 32) | a[2]) << 64) |
                     ((static_cast<uint64_t>(a[1]) << 32) | a[0]);
      const uint64_t r = Redc64::reduce(T, m);
      const uint64_t d = xi >= r ? xi - r : xi + (m.N - r);
      // v_i = (x_i - r) Pi_i^{-1} mod p_i   (is holds Pi_i^{-1} R mod p_i)
      const uint64_t v = Redc64::reduce(static_cast<u128>(d) * is[i], m);
      const uint32_t v0 = static_cast<uint32_t>(v), v1 = static_cast<uint32_t>(v >> 32);
      // X += v Pi_i as two rows, v0 Pi_i and v1 Pi_i 2^32, in one pass over the
      // limbs of Pi_{i+1} (row two lags one limb); each step is a 32x32 product
      // plus two words, below 2^64, so the carries are single words
      uint32_t ca = 0, cb = 0, p_prev = 0;
#pragma unroll
      for (int q = 0; q < K / 4; ++q) {
        if (4 * q < ln) {
#pragma unroll
          for (int t = 0; t < 4; ++t) {
            const int j = 4 * q + t;
            const uint32_t p = pii[j];
            const uint64_t s0 = static_cast<uint64_t>(v0) * p + x[j] + ca;
            ca = static_cast<uint32_t>(s0 >> 32);
            const uint64_t s1 = static_cast<uint64_t>(v1) * p_prev + static_cast<uint32_t>(s0) + cb;
            cb = static_cast<uint32_t>(s1 >> 32);
            x[j] = static_cast<uint32_t>(s1);
            p_prev = p;
          }
        }
      }
    }
    uint4* out = reinterpret_cast<uint4*>(X + e * K);
#pragma unroll
    for (int j = 0; j < K / 4; ++j) out[j] = make_uint4(x[4 * j], x[4 * j + 1], x[4 * j + 2], x[4 * j + 3]);
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
cudaError_t launch_from(const uint64_t* res, uint32_t* X, size_t n, int count,
                        const WordConst64* mods, const uint64_t* c, const uint32_t* pi,
                        const uint64_t* inv, const int* live, cudaStream_t s) {
  const void* k = reinterpret_cast<const void*>(rns_from_kernel<K>);
  const size_t smem = from_smem_bytes(K, count);
  if (smem > 48u * 1024u) {
    const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               static_cast<int>(smem));
    if (e != cudaSuccess) return e;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, 256, smem);
  if (e != cudaSuccess) return e;
  const size_t want = (n + 255) / 256;
  const size_t cap = static_cast<size_t>(device_sm_count()) * static_cast<size_t>(std::max(per_sm, 1));
  rns_from_kernel<K><<<static_cast<unsigned>(std::min(want, cap)), 256, smem, s>>>(
      res, X, n, count, mods, c, pi, inv, live);
  return cudaGetLastError();
}

}  // namespace
}  // namespace montgb

using namespace montgb;

struct mont_rns {
  int count = 0;
  int limbs = 0;                 // K: limbs of every big integer (>= those of P)
  void* dev = nullptr;           // one allocation: mods, c, pi, inv
  WordConst64* d_mods = nullptr;
  uint64_t* d_c = nullptr;
  uint32_t* d_pi = nullptr;
  uint64_t* d_inv = nullptr;
  int* d_live = nullptr;         // live[i] = limbs of Pi_i, i = 0..count
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
  const int needed = static_cast<int>(Pi[count].size());
  int K = 8;
  while (K < needed) K *= 2;
  if (K > 64) return MONT_EINVAL;   // P above 2^2048

  std::vector<WordConst64> mods(count);
  std::vector<uint64_t> c(static_cast<size_t>(count) * K);
  std::vector<uint32_t> pi(static_cast<size_t>(count) * K, 0u);
  std::vector<uint64_t> inv(count);
  std::vector<int> live(count + 1);
  for (int i = 0; i <= count; ++i) live[i] = static_cast<int>(Pi[i].size());
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
    for (size_t j = 0; j < Pi[i].size(); ++j) pi[static_cast<size_t>(i) * K + j] = Pi[i][j];
    uint64_t pim = 1 % p;   // Pi_i mod p
    for (int j = 0; j < i; ++j) pim = mulmod64(pim, moduli[j] % p, p);
    inv[i] = mulmod64(invmod64(pim, p), r64, p);   // Montgomery form of Pi_i^{-1}
  }
  mont_rns* r = new (std::nothrow) mont_rns;
  if (!r) return MONT_ENOMEM;
  r->count = count;
  r->limbs = K;
  const size_t b_mods = count * sizeof(WordConst64);
  const size_t b_c = c.size() * sizeof(uint64_t);
  const size_t b_pi = pi.size() * sizeof(uint32_t);
  const size_t b_inv = inv.size() * sizeof(uint64_t);
  const size_t b_live = live.size() * sizeof(int);
  const size_t off_c = (b_mods + 255) / 256 * 256;
  const size_t off_pi = off_c + (b_c + 255) / 256 * 256;
  const size_t off_inv = off_pi + (b_pi + 255) / 256 * 256;
  const size_t off_live = off_inv + (b_inv + 255) / 256 * 256;
  cudaError_t e = cudaMalloc(&r->dev, off_live + b_live);
  if (e == cudaSuccess) {
    char* base = static_cast<char*>(r->dev);
    r->d_mods = reinterpret_cast<WordConst64*>(base);
    r->d_c = reinterpret_cast<uint64_t*>(base + off_c);
    r->d_pi = reinterpret_cast<uint32_t*>(base + off_pi);
    r->d_inv = reinterpret_cast<uint64_t*>(base + off_inv);
    r->d_live = reinterpret_cast<int*>(base + off_live);
    e = cudaMemcpy(r->d_mods, mods.data(), b_mods, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_c, c.data(), b_c, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_pi, pi.data(), b_pi, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_inv, inv.data(), b_inv, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(r->d_live, live.data(), b_live, cudaMemcpyHostToDevice);
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
    case 8: e = launch_from<8>(residues, X, n, r->count, r->d_mods, r->d_c, r->d_pi, r->d_inv, r->d_live, s); break;
    case 16: e = launch_from<16>(residues, X, n, r->count, r->d_mods, r->d_c, r->d_pi, r->d_inv, r->d_live, s); break;
    case 32: e = launch_from<32>(residues, X, n, r->count, r->d_mods, r->d_c, r->d_pi, r->d_inv, r->d_live, s); break;
    default: e = launch_from<64>(residues, X, n, r->count, r->d_mods, r->d_c, r->d_pi, r->d_inv, r->d_live, s); break;
  }
  return cuda_status(e);
}
