"""Exhaustive counterexample search of Section 3 (the CRT validation).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 2 reduces every Montgomery-type algorithm to the question whether its
output r satisfies ``r = +-T R^{-1} (mod N)`` and lies in the range its Ensure
line claims; Section 3.3 finds Huang et al.'s algorithm (Algorithm 4 with
alpha = 0) wrong by exhibiting one T that breaks both (Example 3.1).  This
module performs that check for every odd N in a range and every T in a domain:

    counterexample  <=>  (r - s T R^{-1}) mod N != 0   or   r outside [lo, hi]

with ``s = +1`` for REDC / Algorithm 1 and ``s = -1`` for the Plantard family,
``r`` the algorithm's own output (``oracle.montgomery.candidate``) and
``R^{-1}`` the inverse of R modulo N.

``sweep`` walks T one at a time with Python integers.  It is meant for tiny
moduli.  ``count_candidate_failures_np`` restates the same test on numpy
``int64`` vectors for one N at a time and is used for larger N; it refuses
parameters for which an intermediate could reach 2^62.
"""

from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from .montgomery import (
    REDC, SIGNED, PLANTARD, SIGNED_PLANTARD, SIGNED_PLANTARD2, candidate,
    claimed_range, constants, input_domain, mods, precondition_ok, sign_of,
)

# Domain rules ("which T are swept")
DOMAIN_DEFAULT = "default"   # each algorithm's own Require line
DOMAIN_REDC = "redc"         # 0 <= T < RN for every variant (Section 1's domain)
# Range rules ("which r are claimed")
RANGE_DEFAULT = "default"    # each algorithm's own Ensure line
RANGE_UNSIGNED = "unsigned"  # [0, N-1]
RANGE_WIDE = "wide"          # [-(N-1), N-1]
RANGE_CENTRED = "centred"    # [-(N-1)/2, (N-1)/2] for odd N


def resolve_domain(rule, variant, N, log2R, alpha):
    """Inclusive T range for one modulus under a domain rule."""
    if rule == DOMAIN_DEFAULT:
        return input_domain(variant, N, log2R, alpha)
    if rule == DOMAIN_REDC:
        return 0, (1 << log2R) * N - 1
    lo, hi = rule
    return int(lo), int(hi)


def resolve_range(rule, variant, N):
    """Inclusive claimed r range for one modulus under a range rule."""
    if rule == RANGE_DEFAULT:
        return claimed_range(variant, N)
    if rule == RANGE_UNSIGNED:
        return 0, N - 1
    if rule == RANGE_WIDE:
        return -(N - 1), N - 1
    if rule == RANGE_CENTRED:
        return -((N - 1) // 2), (N - 1) // 2
    lo, hi = rule
    return int(lo), int(hi)


def expected_value(variant: int, T: int, N: int, log2R: int) -> int:
    """The canonical target the Ensure line names: ``T R^{-1}`` (mod N, or mods N
    for Algorithm 1) and ``-T R^{-1}`` (mod N for Algorithm 2, mods N for 3, 4)."""
    Rinv = pow(1 << log2R, -1, N)
    if variant == REDC:
        return (T * Rinv) % N
    if variant == SIGNED:
        return mods(T * Rinv, N)
    if variant == PLANTARD:
        return (-T * Rinv) % N
    return mods(-T * Rinv, N)


@dataclass
class SweepResult:
    """Per-modulus counterexample counts and the counterexamples themselves."""

    counts: dict = field(default_factory=dict)     # N -> number of failing T
    checked: dict = field(default_factory=dict)    # N -> number of T checked
    skipped: list = field(default_factory=list)    # N that violate the precondition
    examples: list = field(default_factory=list)   # (N, T, r, expected), sorted

    @property
    def total(self) -> int:
        return sum(self.counts.values())


def _odd_moduli(N_lo: int, N_hi: int):
    start = N_lo if N_lo % 2 else N_lo + 1
    return range(max(start, 3), N_hi + 1, 2)


def sweep(variant: int, log2R: int, alpha: int, N_lo: int, N_hi: int,
          domain=DOMAIN_DEFAULT, claimed=RANGE_DEFAULT,
          include_out_of_spec: bool = False, vectorised: bool = False) -> SweepResult:
    """Check the algorithm on every odd N in ``[N_lo, N_hi]`` and every T of
    the domain rule; moduli outside the algorithm's precondition are skipped
    unless ``include_out_of_spec``.  Examples are sorted by (N, T)."""
    res = SweepResult()
    for N in _odd_moduli(N_lo, N_hi):
        if not precondition_ok(variant, N, log2R, alpha) and not include_out_of_spec:
            res.skipped.append(N)
            continue
        t_lo, t_hi = resolve_domain(domain, variant, N, log2R, alpha)
        r_lo, r_hi = resolve_range(claimed, variant, N)
        if vectorised:
            cnt, ex = count_candidate_failures_np(variant, N, log2R, alpha,
                                                  t_lo, t_hi, r_lo, r_hi)
        else:
            cnt, ex = _count_failures_python(variant, N, log2R, alpha,
                                             t_lo, t_hi, r_lo, r_hi)
        res.counts[N] = cnt
        res.checked[N] = max(0, t_hi - t_lo + 1)
        res.examples.extend((N, T, r, e) for (T, r, e) in ex)
    res.examples.sort()
    return res


def _count_failures_python(variant, N, log2R, alpha, t_lo, t_hi, r_lo, r_hi):
    s = sign_of(variant)
    Rinv = pow(1 << log2R, -1, N)
    count = 0
    examples = []
    for T in range(t_lo, t_hi + 1):
        r = candidate(variant, T, N, log2R, alpha)
        if (r - s * T * Rinv) % N != 0 or not (r_lo <= r <= r_hi):
            count += 1
            examples.append((T, r, expected_value(variant, T, N, log2R)))
    return count, examples


# ---------------------------------------------------------------------------
# numpy restatement for one modulus (same formulas, int64 vectors)
# ---------------------------------------------------------------------------

def _np_mods(x: np.ndarray, n: int) -> np.ndarray:
    r = x % n                                  # numpy %: result in [0, n) for n > 0
    return np.where(2 * r >= n, r - n, r)


def _np_candidate(variant, T, N, log2R, alpha, c):
    """The algorithms of Section 1 and 3 on an int64 vector of T."""
    R = 1 << log2R
    n = log2R // 2
    if variant == REDC:
        m = ((T % R) * c.Nprime) % R
        num = T + m * N
        t = num // R
        return np.where(t >= N, t - N, t), num % R
    if variant == SIGNED:
        a0 = T % R
        a1 = (T - a0) // R
        m0 = _np_mods(a0 * c.Ninv, R)
        return a1 - (m0 * N) // R, None
    if variant == PLANTARD:
        m = (T * c.Ninv) % R
        r = (((m >> n) + 1) * N) >> n
        return np.where(r == N, 0, r), None
    if variant == SIGNED_PLANTARD:
        m = _np_mods(T * c.Ninv_s, R)
        half = 1 << (n - 1)
        q = (m + half) >> n
        return (q * N + half) >> n, None
    if variant == SIGNED_PLANTARD2:
        m = _np_mods(T * c.Ninv_s, R)
        return (((m >> n) + (1 << alpha)) * N) >> n, None
    raise ValueError(f"unknown variant {variant}")


def count_candidate_failures_np(variant: int, N: int, log2R: int, alpha: int,
                                t_lo: int, t_hi: int, r_lo: int, r_hi: int,
                                chunk: int = 1 << 22, max_examples: int = 1 << 16):
    """Number of T in ``[t_lo, t_hi]`` for which the algorithm's output fails
    the congruence or the range test, plus up to ``max_examples`` of them as
    ``(T, r, expected)``.  Exact for ``log2R <= 24``, ``N < 2^16``,
    ``|T| < 2^38`` (every product stays below 2^62)."""
    if log2R > 24 or N >= (1 << 16) or max(abs(t_lo), abs(t_hi)) >= (1 << 38):
        raise ValueError("parameters too large for the int64 restatement")
    if alpha > 8:
        raise ValueError("alpha too large for the int64 restatement")
    c = constants(N, log2R)
    s = sign_of(variant)
    Rinv = c.Rinv
    count = 0
    examples = []
    T0 = t_lo
    while T0 <= t_hi:
        T1 = min(t_hi, T0 + chunk - 1)
        T = np.arange(T0, T1 + 1, dtype=np.int64)
        r, rem = _np_candidate(variant, T, N, log2R, alpha, c)
        if rem is not None and np.any(rem != 0):
            raise AssertionError("T + mN not divisible by R")
        target = (s * (T % N) * Rinv) % N       # s T R^{-1} mod N, in [0, N)
        bad = ((r - target) % N != 0) | (r < r_lo) | (r > r_hi)
        nbad = int(np.count_nonzero(bad))
        if nbad:
            count += nbad
            if len(examples) < max_examples:
                idx = np.nonzero(bad)[0][: max_examples - len(examples)]
                for i in idx:
                    Ti = int(T[i])
                    examples.append((Ti, int(r[i]), expected_value(variant, Ti, N, log2R)))
        T0 = T1 + 1
    return count, examples


__all__ = [
    "sweep", "SweepResult", "count_candidate_failures_np", "expected_value",
    "resolve_domain", "resolve_range", "DOMAIN_DEFAULT", "DOMAIN_REDC",
    "RANGE_DEFAULT", "RANGE_UNSIGNED", "RANGE_WIDE", "RANGE_CENTRED",
    "REDC", "SIGNED", "PLANTARD", "SIGNED_PLANTARD", "SIGNED_PLANTARD2",
]
