// Host-side per-modulus precomputation and validation (mont_ctx_create).
//
// Constants (Section 1 and Theorem 2.1 of the paper):
//   N^{-1} mod R   by Newton-Hensel lifting x <- x (2 - N x) mod 2^w, which
//                  doubles the number of correct low bits each step and starts
//                  from x = N (correct mod 8 for every odd N);
//   N' = R - N^{-1};
//   R mod N, R^2 mod N by repeated doubling modulo N.
// Everything runs on little-endian 32-bit limb vectors so that 32-bit, 64-bit
// and multi-limb moduli share one code path.
#include <cstring>
#include <new>

#include "internal.h"

namespace {

using Limbs = std::vector<uint32_t>;

Limbs resized(const Limbs& a, size_t L) {
  Limbs r(L, 0u);
  for (size_t i = 0; i < L && i < a.size(); ++i) r[i] = a[i];
  return r;
}

// a * b mod 2^{32L}
Limbs mul_lo(const Limbs& a, const Limbs& b, size_t L) {
  Limbs r(L, 0u);
  for (size_t i = 0; i < L; ++i) {
    uint64_t carry = 0;
    const uint64_t ai = i < a.size() ? a[i] : 0u;
    for (size_t j = 0; i + j < L; ++j) {
      const uint64_t bj = j < b.size() ? b[j] : 0u;
      const uint64_t cur = r[i + j] + ai * bj + carry;
      r[i + j] = static_cast<uint32_t>(cur);
      carry = cur >> 32;
    }
  }
  return r;
}

// a * b, full product (a.size() + b.size() limbs)
Limbs mul_full(const Limbs& a, const Limbs& b) {
  Limbs r(a.size() + b.size(), 0u);
  for (size_t i = 0; i < a.size(); ++i) {
    uint64_t carry = 0;
    for (size_t j = 0; j < b.size(); ++j) {
      const uint64_t cur = r[i + j] + static_cast<uint64_t>(a[i]) * b[j] + carry;
      r[i + j] = static_cast<uint32_t>(cur);
      carry = cur >> 32;
    }
    r[i + b.size()] = static_cast<uint32_t>(carry);
  }
  return r;
}

// a - b mod 2^{32L} (both read as L limbs)
Limbs sub_lo(const Limbs& a, const Limbs& b, size_t L) {
  Limbs r(L, 0u);
  int64_t borrow = 0;
  for (size_t i = 0; i < L; ++i) {
    const int64_t cur = static_cast<int64_t>(i < a.size() ? a[i] : 0u) -
                        static_cast<int64_t>(i < b.size() ? b[i] : 0u) - borrow;
    r[i] = static_cast<uint32_t>(cur);
    borrow = cur < 0 ? 1 : 0;
  }
  return r;
}

// -1, 0, +1 for a <, =, > b (any lengths)
int cmp(const Limbs& a, const Limbs& b) {
  const size_t L = a.size() > b.size() ? a.size() : b.size();
  for (size_t i = L; i-- > 0;) {
    const uint32_t x = i < a.size() ? a[i] : 0u;
    const uint32_t y = i < b.size() ? b[i] : 0u;
    if (x != y) return x < y ? -1 : 1;
  }
  return 0;
}

// x <- 2x mod N for 0 <= x < N (x and N have the same length)
void double_mod(Limbs& x, const Limbs& N) {
  uint32_t carry = 0;
  for (auto& w : x) {
    const uint32_t nc = w >> 31;
    w = (w << 1) | carry;
    carry = nc;
  }
  if (carry || cmp(x, N) >= 0) x = sub_lo(x, N, x.size());
}

// N^{-1} mod 2^{32L} for odd N (Newton-Hensel lifting)
Limbs inverse_pow2(const Limbs& N, size_t L) {
  const Limbs n = resized(N, L);
  Limbs x = n;  // correct modulo 2^3
  Limbs two(L, 0u);
  two[0] = 2;
  for (size_t bits = 3; bits < 32 * L; bits *= 2) {
    x = mul_lo(x, sub_lo(two, mul_lo(n, x, L), L), L);
  }
  return x;
}

int top_bit_index(const Limbs& a) {  // -1 for zero
  for (size_t i = a.size(); i-- > 0;) {
    if (a[i]) {
      int b = 31;
      while (!((a[i] >> b) & 1u)) --b;
      return static_cast<int>(32 * i) + b;
    }
  }
  return -1;
}

Limbs pow2(int e, size_t L) {
  Limbs r(L, 0u);
  r[static_cast<size_t>(e) / 32] = 1u << (e % 32);
  return r;
}

bool is_supported_multilimb(int k) {
  return k == 4 || k == 8 || k == 12 || k == 16 || k == 32 || k == 64;
}

// N < 2^n / phi  <=>  5 N^2 < (2^{n+1} - N)^2   (exact, Section 3.2)
bool plantard_bound_ok(const Limbs& N, int n) {
  const size_t L = static_cast<size_t>(n) / 32 + 2;
  const Limbs lim = pow2(n + 1, L);
  const Limbs nn = resized(N, L);
  if (cmp(nn, lim) >= 0) return false;
  const Limbs d = sub_lo(lim, nn, L);
  Limbs five(1, 5u);
  const Limbs lhs = mul_full(five, mul_full(nn, nn));
  const Limbs rhs = mul_full(d, d);
  return cmp(lhs, rhs) < 0;
}

uint64_t u64_of(const Limbs& a, size_t off) {
  const uint64_t lo = off < a.size() ? a[off] : 0u;
  const uint64_t hi = off + 1 < a.size() ? a[off + 1] : 0u;
  return lo | (hi << 32);
}

}  // namespace

extern "C" int mont_ctx_create(mont_ctx_t* out, const uint32_t* N_limbs, int n_limbs,
                               int log2R, int variant, int alpha) {
  if (!out || !N_limbs) return MONT_EINVAL;
  if (variant < MONT_REDC || variant > MONT_SIGNED_PLANTARD2) return MONT_EINVAL;
  const bool word = (n_limbs == 1 || n_limbs == 2);
  if (!word && !is_supported_multilimb(n_limbs)) return MONT_EINVAL;
  const bool plantard = variant >= MONT_PLANTARD;
  const int want_log2R = plantard ? 64 * n_limbs : 32 * n_limbs;
  if (log2R != want_log2R) return MONT_EINVAL;

  Limbs N(N_limbs, N_limbs + n_limbs);
  const int top = top_bit_index(N);
  if ((N[0] & 1u) == 0 || top < 1) return MONT_EINVAL;  // even, or N = 1
  const int w = 32 * n_limbs;
  const int n = w;  // Plantard family: R = 2^{2n} with n the word size
  switch (variant) {
    case MONT_REDC:  // N < R holds: N fits in log2R bits
      break;
    case MONT_SIGNED:  // 2N < R
      if (top >= w - 1) return MONT_EINVAL;
      break;
    case MONT_PLANTARD:  // N < 2^n / phi
      if (!plantard_bound_ok(N, n)) return MONT_EINVAL;
      break;
    case MONT_SIGNED_PLANTARD:  // N < 2^{n-1}
      if (top >= n - 1) return MONT_EINVAL;
      break;
    case MONT_SIGNED_PLANTARD2:  // alpha >= 1 (Section 3.3) and N < 2^{n-alpha-1}
      if (alpha < 1 || alpha > n - 3) return MONT_EINVAL;
      if (top >= n - alpha - 1) return MONT_EINVAL;
      break;
  }

  mont_ctx* c = new (std::nothrow) mont_ctx;
  if (!c) return MONT_ENOMEM;
  c->variant = variant;
  c->alpha = (variant == MONT_SIGNED_PLANTARD2) ? alpha : 0;
  c->log2R = log2R;
  c->n_limbs = n_limbs;
  c->width = w;
  c->N = N;

  const size_t LR = static_cast<size_t>(log2R) / 32;
  c->ninv = inverse_pow2(N, LR);
  c->nprime = sub_lo(Limbs(LR, 0u), c->ninv, LR);  // R - N^{-1} (N^{-1} != 0)

  Limbs x(N.size(), 0u);
  x[0] = 1;
  for (int i = 0; i < log2R; ++i) double_mod(x, N);
  c->r_mod_n = x;
  for (int i = 0; i < log2R; ++i) double_mod(x, N);
  c->r2_mod_n = x;

  // Domain constant: signed variants use the mods-N form of R^2 mod N.
  c->domain_r2 = c->r2_mod_n;
  if (variant == MONT_SIGNED || variant == MONT_SIGNED_PLANTARD ||
      variant == MONT_SIGNED_PLANTARD2) {
    Limbs twice = c->r2_mod_n;
    twice.push_back(0u);
    uint32_t carry = 0;
    for (auto& wd : twice) {
      const uint32_t nc = wd >> 31;
      wd = (wd << 1) | carry;
      carry = nc;
    }
    if (cmp(twice, N) >= 0) c->domain_r2 = sub_lo(c->r2_mod_n, N, N.size());  // r2 - N < 0
  }

  if (n_limbs == 1) {
    auto& k = c->w32;
    k.N = N[0];
    k.nprime = c->nprime[0];
    k.ninv = c->ninv[0];
    k.half = (N[0] - 1u) / 2u;
    k.ninv2 = plantard ? u64_of(c->ninv, 0) : 0u;
    k.r2 = c->domain_r2[0];
    k.alpha = c->alpha;
  } else if (n_limbs == 2) {
    auto& k = c->w64;
    k.N = u64_of(N, 0);
    k.nprime = u64_of(c->nprime, 0);
    k.ninv = u64_of(c->ninv, 0);
    k.half = (k.N - 1u) / 2u;
    k.ninv2_lo = plantard ? u64_of(c->ninv, 0) : 0u;
    k.ninv2_hi = plantard ? u64_of(c->ninv, 2) : 0u;
    k.r2 = u64_of(c->domain_r2, 0);
    k.alpha = c->alpha;
  } else {
    auto& k = c->limb;
    k.n0prime = c->nprime[0];
    for (int i = 0; i < n_limbs; ++i) {
      k.N[i] = N[i];
      k.r2[i] = c->r2_mod_n[i];
      k.dom[i] = c->domain_r2[i];
    }
    auto& v = c->limbv;
    v.variant = variant;
    v.alpha = c->alpha;
    // half = (N - 1) / 2 = N >> 1 (N odd), shifted limb by limb
    for (int i = 0; i < n_limbs; ++i) {
      v.N[i] = N[i];
      v.dom[i] = c->domain_r2[i];
      v.half[i] = (N[i] >> 1) | (i + 1 < n_limbs ? (N[i + 1] << 31) : 0u);
    }
    for (size_t i = 0; i < LR; ++i) v.ninv[i] = c->ninv[i];
  }
  *out = c;
  return MONT_OK;
}

extern "C" int mont_ctx_destroy(mont_ctx_t ctx) {
  delete ctx;
  return MONT_OK;
}

extern "C" int mont_ctx_constant(mont_ctx_t ctx, int which, uint32_t* limbs, int cap,
                                 int* n_out) {
  if (!ctx || !limbs || !n_out) return MONT_EINVAL;
  const Limbs* src = nullptr;
  switch (which) {
    case MONT_CONST_N: src = &ctx->N; break;
    case MONT_CONST_NINV: src = &ctx->ninv; break;
    case MONT_CONST_NPRIME: src = &ctx->nprime; break;
    case MONT_CONST_R_MOD_N: src = &ctx->r_mod_n; break;
    case MONT_CONST_R2_MOD_N: src = &ctx->r2_mod_n; break;
    case MONT_CONST_DOMAIN_R2: src = &ctx->domain_r2; break;
    default: return MONT_EINVAL;
  }
  if (cap < static_cast<int>(src->size())) return MONT_EOVERFLOW;
  std::memcpy(limbs, src->data(), src->size() * sizeof(uint32_t));
  *n_out = static_cast<int>(src->size());
  return MONT_OK;
}

extern "C" int mont_ctx_query(mont_ctx_t ctx, int* width_bits, int* n_limbs, int* elem_bytes,
                              int* variant, int* log2R, int* alpha) {
  if (!ctx) return MONT_EINVAL;
  if (width_bits) *width_bits = ctx->width;
  if (n_limbs) *n_limbs = ctx->n_limbs;
  if (elem_bytes) *elem_bytes = 4 * ctx->n_limbs;
  if (variant) *variant = ctx->variant;
  if (log2R) *log2R = ctx->log2R;
  if (alpha) *alpha = ctx->alpha;
  return MONT_OK;
}
