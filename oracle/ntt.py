"""Plantard's constant-multiplicand form and the negacyclic number-theoretic
transform built on it.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 3.2 notes that Plantard's reduction turns the product of a 2n-bit
and an n-bit integer into a product of two n-bit integers: when one factor
b is fixed, b N^{-1} mod R can be computed once, and then
T N^{-1} mod R = a (b N^{-1} mod R) mod R needs no double-width T.  The
motivating application the paper names (Section 1) is the number-theoretic
transform of lattice and homomorphic-encryption schemes, whose twiddle
factors are exactly such fixed multipliers; the paper itself does not treat
it, so the transform below is the textbook definition.

Definitions used here:
* the prepared multiplier of b: b' = b N^{-1} mod R (Plantard family);
* psi: a primitive 2n-th root of unity mod N (psi^n = -1);
* forward negacyclic NTT, output in bit-reversed order:
      A[i] = sum_j a[j] psi^{(2 brv(i) + 1) j}  mod N,
  i.e. A[i] is a(x) evaluated at the root psi^{2 brv(i) + 1} of x^n + 1;
* inverse: a[j] = n^{-1} sum_i A[i] psi^{-(2 brv(i) + 1) j}  mod N.
"""

from __future__ import annotations

from .montgomery import constants, mods


def prepared_multiplier(b: int, N: int, log2R: int) -> int:
    """b' = b N^{-1} mod R, the fixed-multiplier form of Section 3.2."""
    c = constants(N, log2R)
    return (b * c.Ninv) % c.R


def predc_prepared_alg(a: int, b_pre: int, N: int, log2R: int) -> int:
    """Algorithm 2 with the multiplier prepared: m = a b' mod R replaces
    T N^{-1} mod R, then r = floor((floor(m / 2^n) + 1) N / 2^n)."""
    n = log2R // 2
    R = 1 << log2R
    m = (a * b_pre) % R
    return ((m >> n) + 1) * N >> n


def sigpredc1_prepared_alg(a: int, b_pre: int, N: int, log2R: int) -> int:
    """Algorithm 3 with the multiplier prepared: m = a b' mods R."""
    n = log2R // 2
    R = 1 << log2R
    m = mods(a * b_pre, R)
    half = 1 << (n - 1)
    q = (m + half) >> n
    return (q * N + half) >> n


def brv(i: int, bits: int) -> int:
    """Bit reversal of i over `bits` bits."""
    r = 0
    for _ in range(bits):
        r = (r << 1) | (i & 1)
        i >>= 1
    return r


def is_primitive_2n_root(psi: int, N: int, n: int) -> bool:
    """psi has order exactly 2n mod N (n a power of two): psi^n = -1."""
    return pow(psi, n, N) == N - 1


def ntt_forward(a, N: int, psi: int):
    """The definition, O(n^2): A[i] = sum_j a[j] psi^{(2 brv(i) + 1) j} mod N."""
    n = len(a)
    bits = n.bit_length() - 1
    out = []
    for i in range(n):
        e = 2 * brv(i, bits) + 1
        w = pow(psi, e, N)
        acc, wj = 0, 1
        for j in range(n):
            acc += a[j] * wj
            wj = wj * w % N
        out.append(acc % N)
    return out


def ntt_inverse(A, N: int, psi: int):
    """a[j] = n^{-1} sum_i A[i] psi^{-(2 brv(i) + 1) j} mod N."""
    n = len(A)
    bits = n.bit_length() - 1
    psi_inv = pow(psi, -1, N)
    n_inv = pow(n, -1, N)
    out = []
    for j in range(n):
        acc = 0
        for i in range(n):
            e = (2 * brv(i, bits) + 1) * j
            acc += A[i] * pow(psi_inv, e, N)
        out.append(acc * n_inv % N)
    return out


def negacyclic_product(a, b, N: int):
    """Schoolbook a(x) b(x) mod (x^n + 1, N)."""
    n = len(a)
    out = [0] * n
    for i in range(n):
        for j in range(n):
            k = i + j
            if k < n:
                out[k] += a[i] * b[j]
            else:
                out[k - n] -= a[i] * b[j]
    return [x % N for x in out]
