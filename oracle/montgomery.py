"""Plain, slow, obviously correct definitions of Montgomery-type reduction.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): the library never
imports this module.

Notation follows the paper (Xu, Jia, Yang, "Chinese Remainder Theorem
Approach to Montgomery-Type Algorithms"):

* ``N`` odd modulus, ``R = 2^log2R`` (for the Plantard family ``R = 2^{2n}``,
  so ``n = log2R / 2``).
* ``N^{-1} = N^{-1} mod R`` and ``R^{-1} = R^{-1} mod N`` (Theorem 2.1).
* ``N' = R - (N^{-1} mod R)`` (Section 1, REDC).
* ``x mods n`` is the least absolute remainder in ``[-n/2, n/2)`` (Section 2).
* ``Ñ^{-1} = N^{-1} mods R`` (Sections 3.2, 3.3).

Two kinds of function live here:

``*_value``  the plain definition of what a reduction returns, computed with a
             modular inverse (``pow(x, -1, m)``) and ``%``.  These are the
             parity targets for every GPU output.
``*_alg``    the paper's algorithm evaluated step by step, in exact integers,
             in the order and notation of the paper (REDC of Section 1,
             Algorithms 1-4 of Section 3).  These are what the exhaustive
             sweep checks against the definitions, and what a word-level
             implementation must reproduce bit for bit inside the stated
             input domain.
"""

from __future__ import annotations

from dataclasses import dataclass

# Variant codes.  The numbering is this project's own; the names follow the
# paper's function names.
REDC = 0               # Section 1, REDC(T)
SIGNED = 1             # Algorithm 1, SigRedc (Seiler's signed Montgomery)
PLANTARD = 2           # Algorithm 2, PRedc (Plantard)
SIGNED_PLANTARD = 3    # Algorithm 3, SigPRedc1 (signed Plantard)
SIGNED_PLANTARD2 = 4   # Algorithm 4, SigPRedc2 (signed Plantard with alpha)
VARIANTS = (REDC, SIGNED, PLANTARD, SIGNED_PLANTARD, SIGNED_PLANTARD2)
VARIANT_NAMES = {
    REDC: "redc",
    SIGNED: "sigredc",
    PLANTARD: "predc",
    SIGNED_PLANTARD: "sigpredc1",
    SIGNED_PLANTARD2: "sigpredc2",
}
_PLANTARD_FAMILY = (PLANTARD, SIGNED_PLANTARD, SIGNED_PLANTARD2)
_SIGNED_OUTPUT = (SIGNED, SIGNED_PLANTARD, SIGNED_PLANTARD2)


def mods(x: int, n: int) -> int:
    """Least absolute remainder of ``x`` by ``n > 0``, in ``[-n/2, n/2)``.

    Section 2 fixes the interval as half-open on the right, so for even ``n``
    the value ``-n/2`` is allowed and ``+n/2`` is not.
    """
    if n <= 0:
        raise ValueError("mods needs a positive modulus")
    r = x % n                 # Python: r in [0, n)
    if 2 * r >= n:            # r >= n/2  ->  move to the negative side
        r -= n
    return r


def _check_modulus(N: int) -> None:
    if N < 3 or N % 2 == 0:
        raise ValueError(f"N must be an odd integer >= 3, got {N}")


@dataclass(frozen=True)
class Constants:
    """Per-modulus constants of Sections 1-3 for ``R = 2^log2R``."""

    N: int
    log2R: int
    R: int
    Ninv: int      # N^{-1} mod R, in [1, R)             (Theorem 2.1)
    Nprime: int    # N' = R - N^{-1}, in [1, R)          (Section 1, REDC)
    Ninv_s: int    # Ñ^{-1} = N^{-1} mods R              (Sections 3.1-3.3)
    Rinv: int      # R^{-1} mod N, in [1, N)             (Theorem 2.1)
    Rinv_s: int    # R̃^{-1} = R^{-1} mods N              (Sections 3.2-3.3)
    R_mod_N: int   # R mod N                             (Section 1, map Φ)
    R2_mod_N: int  # R^2 mod N


def constants(N: int, log2R: int) -> Constants:
    """All constants the reductions use, from the definitions directly."""
    _check_modulus(N)
    if log2R < 1:
        raise ValueError("log2R must be >= 1")
    R = 1 << log2R
    Ninv = pow(N, -1, R)
    Rinv = pow(R, -1, N)
    return Constants(
        N=N, log2R=log2R, R=R, Ninv=Ninv, Nprime=R - Ninv, Ninv_s=mods(Ninv, R),
        Rinv=Rinv, Rinv_s=mods(Rinv, N), R_mod_N=R % N, R2_mod_N=(R * R) % N,
    )


def plantard_bound_ok(N: int, n: int) -> bool:
    """Exact test of ``N < 2^n / phi`` with ``phi = (1 + sqrt 5) / 2`` (Section 3.2).

    ``N < 2^n/phi``  <=>  ``N (1 + sqrt 5) < 2^{n+1}``  <=>  ``N sqrt 5 < 2^{n+1} - N``,
    and with both sides positive this is ``5 N^2 < (2^{n+1} - N)^2``.
    """
    rhs = (1 << (n + 1)) - N
    return rhs > 0 and 5 * N * N < rhs * rhs


def precondition_ok(variant: int, N: int, log2R: int, alpha: int = 0) -> bool:
    """The modulus conditions each algorithm states before its Require line."""
    if N < 3 or N % 2 == 0 or log2R < 2:
        return False
    R = 1 << log2R
    if variant == REDC:                      # Section 1: R > N
        return N < R
    if variant == SIGNED:                    # Section 3.1: 2N < R
        return 2 * N < R
    if log2R % 2:                            # Plantard family: R = 2^{2n}
        return False
    n = log2R // 2
    if variant == PLANTARD:                  # Section 3.2: N < 2^n / phi
        return plantard_bound_ok(N, n)
    if variant == SIGNED_PLANTARD:           # Section 3.2, signed: N < 2^{n-1}
        return N < (1 << (n - 1))
    if variant == SIGNED_PLANTARD2:          # Section 3.3: N < 2^{n-alpha-1}
        return alpha >= 0 and n - alpha - 1 >= 0 and N < (1 << (n - alpha - 1))
    raise ValueError(f"unknown variant {variant}")


def input_domain(variant: int, N: int, log2R: int, alpha: int = 0) -> tuple[int, int]:
    """Inclusive range of T that each algorithm's Require line admits.

    Where the paper states a bound once with ``<`` and once with ``<=``
    (Algorithms 2-4 against their proofs) the inclusive reading is used.
    """
    R = 1 << log2R
    if variant == REDC:                      # 0 <= T < RN
        return 0, R * N - 1
    if variant == SIGNED:                    # -NR/2 < T < NR/2
        half = N * R // 2
        return -half + 1, half - 1
    n = log2R // 2
    if variant == PLANTARD:                  # 0 <= T <= N^2
        return 0, N * N
    if variant == SIGNED_PLANTARD:           # |T| <= 2^{2n-2}
        b = 1 << (2 * n - 2)
        return -b, b
    if variant == SIGNED_PLANTARD2:          # |T| <= 2^{2 alpha} N^2
        b = (1 << (2 * alpha)) * N * N
        return -b, b
    raise ValueError(f"unknown variant {variant}")


def claimed_range(variant: int, N: int) -> tuple[int, int]:
    """Inclusive integer range each algorithm's Ensure line claims for r."""
    if variant in (REDC, PLANTARD):          # r in [0, N)
        return 0, N - 1
    if variant == SIGNED:                    # -N < r < N
        return -(N - 1), N - 1
    if variant == SIGNED_PLANTARD:           # r = (...) mods N, i.e. in [-N/2, N/2)
        return -(N // 2), (N - 1) // 2
    if variant == SIGNED_PLANTARD2:          # -N/2 < r < N/2
        return -((N - 1) // 2), (N - 1) // 2
    raise ValueError(f"unknown variant {variant}")


def sign_of(variant: int) -> int:
    """+1 when r is congruent to T R^{-1}; -1 when it is congruent to -T R^{-1}."""
    return -1 if variant in _PLANTARD_FAMILY else 1


# ---------------------------------------------------------------------------
# Definitions (parity targets)
# ---------------------------------------------------------------------------

def redc_value(T: int, N: int, R: int) -> int:
    """``T R^{-1} mod N`` in ``[0, N)`` -- what REDC returns (Section 1)."""
    return (T * pow(R, -1, N)) % N


def sigredc_value(T: int, N: int, R: int) -> int:
    """The representative Algorithm 1 returns: ``(T - m N) / R`` with
    ``m = T N^{-1} mods R`` (Eq. (5), Section 2, with the mods choice of m).

    The quotient is exact because ``T - mN`` is divisible by R (Section 2).
    """
    m = mods(T * pow(N, -1, R), R)
    q, rem = divmod(T - m * N, R)
    if rem != 0:
        raise AssertionError("T - mN not divisible by R")
    return q


def predc_value(T: int, N: int, R: int) -> int:
    """``-T R^{-1} mod N`` in ``[0, N)`` -- Algorithm 2's Ensure line."""
    return (-T * pow(R, -1, N)) % N


def sigpredc_value(T: int, N: int, R: int) -> int:
    """``-T R̃^{-1} mods N`` -- the Ensure line of Algorithms 3 and 4."""
    return mods(-T * pow(R, -1, N), N)


def reduce_value(variant: int, T: int, N: int, log2R: int, alpha: int = 0) -> int:
    """Definition of the reduction of T for the given variant."""
    R = 1 << log2R
    if variant == REDC:
        return redc_value(T, N, R)
    if variant == SIGNED:
        return sigredc_value(T, N, R)
    if variant == PLANTARD:
        return predc_value(T, N, R)
    if variant in (SIGNED_PLANTARD, SIGNED_PLANTARD2):
        return sigpredc_value(T, N, R)
    raise ValueError(f"unknown variant {variant}")


def mul_value(variant: int, a: int, b: int, N: int, log2R: int, alpha: int = 0) -> int:
    """Montgomery-type product: the reduction of ``T = a b``."""
    return reduce_value(variant, a * b, N, log2R, alpha)


def _r2_constant(variant: int, N: int, log2R: int) -> int:
    """The ``R^2 mod N`` constant the domain map multiplies by: the canonical
    residue in ``[0, N)`` for unsigned variants, its mods-N form for signed ones."""
    r2 = pow(2, 2 * log2R, N)
    return mods(r2, N) if variant in _SIGNED_OUTPUT else r2


def to_domain_value(variant: int, x: int, N: int, log2R: int, alpha: int = 0) -> int:
    """Map into the representation of Section 1's map Φ: reduce ``x (R^2 mod N)``.

    For REDC and Algorithm 1 this is ``x R mod N`` (up to Algorithm 1's choice
    of representative); for the Plantard family, whose reductions return
    ``-T R^{-1}``, it is ``-x R mod N``, which keeps the product closed.
    """
    return reduce_value(variant, x * _r2_constant(variant, N, log2R), N, log2R, alpha)


def from_domain_value(variant: int, y: int, N: int, log2R: int, alpha: int = 0) -> int:
    """Leave the representation: reduce ``y`` (i.e. ``y * 1``) and return the
    canonical residue -- ``[0, N)`` for unsigned variants, ``mods N`` for
    signed ones."""
    r = reduce_value(variant, y, N, log2R, alpha)
    return mods(r, N) if variant in _SIGNED_OUTPUT else r % N


# ---------------------------------------------------------------------------
# The algorithms, step by step in exact integers
# ---------------------------------------------------------------------------

def redc_alg(T: int, N: int, log2R: int) -> int:
    """REDC (Section 1): m <- (T mod R) N' mod R; t <- (T + mN)/R; one
    conditional subtraction of N."""
    c = constants(N, log2R)
    R = c.R
    m = ((T % R) * c.Nprime) % R
    t, rem = divmod(T + m * N, R)
    if rem != 0:
        raise AssertionError("T + mN not divisible by R")
    return t - N if t >= N else t


def sigredc_alg(T: int, N: int, log2R: int) -> int:
    """Algorithm 1 (SigRedc): write T = a1 R + a0 with 0 <= a0 < R;
    m0 <- a0 N^{-1} mods R; t <- floor(m0 N / R); r <- a1 - t."""
    c = constants(N, log2R)
    R = c.R
    a0 = T % R
    a1 = (T - a0) // R
    m0 = mods(a0 * c.Ninv, R)
    t = (m0 * N) // R
    return a1 - t


def predc_alg(T: int, N: int, log2R: int) -> int:
    """Algorithm 2 (PRedc), R = 2^{2n}:
    r <- floor((floor((T N^{-1} mod R) / 2^n) + 1) N / 2^n); if r = N return 0."""
    if log2R % 2:
        raise ValueError("Plantard reduction needs R = 2^{2n}")
    c = constants(N, log2R)
    n = log2R // 2
    m = (T * c.Ninv) % c.R
    r = ((m >> n) + 1) * N >> n
    if r == N:
        return 0
    return r


def _round_half_up(x_num: int, shift: int) -> int:
    """``floor(x + 1/2)`` for ``x = x_num / 2^shift`` (the paper's rounding)."""
    return (x_num + (1 << (shift - 1))) >> shift


def sigpredc1_alg(T: int, N: int, log2R: int) -> int:
    """Algorithm 3 (SigPRedc1), R = 2^{2n}:
    r <- round( round((T Ñ^{-1} mods R) / 2^n) N / 2^n ), rounding half up."""
    if log2R % 2:
        raise ValueError("Plantard reduction needs R = 2^{2n}")
    c = constants(N, log2R)
    n = log2R // 2
    m = mods(T * c.Ninv_s, c.R)
    q = _round_half_up(m, n)
    return _round_half_up(q * N, n)


def sigpredc2_alg(T: int, N: int, log2R: int, alpha: int) -> int:
    """Algorithm 4 (SigPRedc2), R = 2^{2n}:
    r <- floor((floor((T Ñ^{-1} mods R) / 2^n) + 2^alpha) N / 2^n)."""
    if log2R % 2:
        raise ValueError("Plantard reduction needs R = 2^{2n}")
    if alpha < 0:
        raise ValueError("alpha must be >= 0")
    c = constants(N, log2R)
    n = log2R // 2
    m = mods(T * c.Ninv_s, c.R)
    return ((m >> n) + (1 << alpha)) * N >> n


def candidate(variant: int, T: int, N: int, log2R: int, alpha: int = 0) -> int:
    """The algorithm's own output for T (what the sweep tests)."""
    if variant == REDC:
        return redc_alg(T, N, log2R)
    if variant == SIGNED:
        return sigredc_alg(T, N, log2R)
    if variant == PLANTARD:
        return predc_alg(T, N, log2R)
    if variant == SIGNED_PLANTARD:
        return sigpredc1_alg(T, N, log2R)
    if variant == SIGNED_PLANTARD2:
        return sigpredc2_alg(T, N, log2R, alpha)
    raise ValueError(f"unknown variant {variant}")


# ---------------------------------------------------------------------------
# Multi-limb values: 32-bit limbs, least significant first
# ---------------------------------------------------------------------------

def from_limbs(limbs) -> int:
    """Integer from little-endian 32-bit limbs."""
    x = 0
    for i, limb in enumerate(limbs):
        x |= int(limb) << (32 * i)
    return x


def to_limbs(x: int, k: int) -> list[int]:
    """``k`` little-endian 32-bit limbs of ``0 <= x < 2^{32k}``."""
    if x < 0 or x >> (32 * k):
        raise ValueError("value does not fit in k limbs")
    return [(x >> (32 * i)) & 0xFFFFFFFF for i in range(k)]
