"""Seeded generators for the synthetic workloads.

Every generator takes an explicit seed and uses numpy's PCG64, so the same
call yields the same arrays on every machine.  Shapes and distributions:

* word modmul   -- odd modulus N, operands uniform in [0, N) (unsigned
                   variants) or in the centred range (-N/2, N/2] (signed
                   variants), stored as uint32/int32 or uint64/int64 vectors.
* RNS moduli    -- distinct primes p with 2^59 <= p < 2^62 and p = 1 mod 2^17,
                   found by drawing c uniformly and testing p = c 2^17 + 1 with
                   Miller-Rabin over the first twelve prime bases (deterministic
                   below 3.3e24, far above 2^62).
* lengths       -- floor(2^U) with U uniform on [lo, hi].
* multi-limb    -- odd N of exactly ``bits`` bits (top and bottom bit set,
                   the rest uniform); operands uniform in [0, N) by rejection;
                   little-endian 32-bit limbs, element-major (element i occupies
                   limbs [i k, (i+1) k)).
* serving jobs  -- Poisson arrivals with a mix of variants, widths, lengths and
                   sweep jobs.
"""

from __future__ import annotations

from dataclasses import dataclass

import numpy as np

__all__ = [
    "rng", "uniform_residues", "centred_residues", "lift_unsigned", "is_probable_prime",
    "rns_primes", "log_uniform_lengths", "random_odd_modulus", "limbs_of",
    "int_of_limbs", "uniform_limb_residues", "bounded_limb_residues", "centred_limb_residues",
    "Job", "serving_jobs",
    "REDC32_N", "WORD32_MODULI", "ntt_prime", "primitive_2n_root",
]

# Moduli of the 32-bit workloads: Kyber's q = 3329 and Dilithium's q = 8380417.
REDC32_N = 3329
WORD32_MODULI = (3329, 8380417)


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def uniform_residues(N: int, count: int, seed: int, dtype=np.uint32) -> np.ndarray:
    """``count`` integers uniform in [0, N)."""
    g = rng(seed)
    if N <= (1 << 63):
        return g.integers(0, N, size=count, dtype=np.uint64).astype(dtype)
    # N above 2^63: draw 64-bit words and reject those >= N (acceptance > 1/2)
    out = np.empty(count, dtype=np.uint64)
    filled = 0
    while filled < count:
        x = g.integers(0, 1 << 64, size=2 * (count - filled) + 16, dtype=np.uint64)
        x = x[x < np.uint64(N)]
        take = min(len(x), count - filled)
        out[filled:filled + take] = x[:take]
        filled += take
    return out.astype(dtype)


def centred_residues(N: int, count: int, seed: int, dtype=np.int32) -> np.ndarray:
    """``count`` integers uniform in the centred range (-N/2, N/2]."""
    g = rng(seed)
    lo = -((N - 1) // 2) if N % 2 else -(N // 2) + 1
    hi = N // 2
    return g.integers(lo, hi + 1, size=count, dtype=np.int64).astype(dtype)


def lift_unsigned(x: np.ndarray, N: int, dtype=np.uint32) -> np.ndarray:
    """Representation change of centred residues to [0, N): x + N where x < 0."""
    x64 = x.astype(np.int64)
    return np.where(x64 < 0, x64 + N, x64).astype(dtype)


_MR_BASES = (2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37)


def is_probable_prime(p: int) -> bool:
    """Miller-Rabin over the first twelve prime bases; exact for p < 3.3e24."""
    if p < 2:
        return False
    for q in _MR_BASES:
        if p % q == 0:
            return p == q
    d, s = p - 1, 0
    while d % 2 == 0:
        d //= 2
        s += 1
    for a in _MR_BASES:
        x = pow(a, d, p)
        if x in (1, p - 1):
            continue
        for _ in range(s - 1):
            x = x * x % p
            if x == p - 1:
                break
        else:
            return False
    return True


def rns_primes(count: int = 32, seed: int = 3, lo_bits: int = 59, hi_bits: int = 62,
               two_adicity: int = 17) -> list[int]:
    """``count`` distinct primes p, 2^lo_bits <= p < 2^hi_bits, p = 1 mod 2^two_adicity."""
    g = rng(seed)
    step = 1 << two_adicity
    c_lo = ((1 << lo_bits) - 1) // step + 1
    c_hi = ((1 << hi_bits) - 1) // step
    out: list[int] = []
    seen = set()
    while len(out) < count:
        c = int(g.integers(c_lo, c_hi, dtype=np.int64, endpoint=True))
        p = c * step + 1
        if (1 << lo_bits) <= p < (1 << hi_bits) and p not in seen and is_probable_prime(p):
            seen.add(p)
            out.append(p)
    return out


def log_uniform_lengths(count: int, lo: float, hi: float, seed: int) -> list[int]:
    """``floor(2^U)`` with ``U`` uniform on ``[lo, hi]``."""
    g = rng(seed)
    u = g.uniform(lo, hi, size=count)
    return [int(np.floor(2.0 ** x)) for x in u]


def random_odd_modulus(bits: int, seed: int) -> int:
    """Odd integer of exactly ``bits`` bits, uniform in its other bits."""
    g = rng(seed)
    words = g.integers(0, 1 << 32, size=(bits + 31) // 32, dtype=np.uint64)
    x = 0
    for i, w in enumerate(words):
        x |= int(w) << (32 * i)
    x &= (1 << bits) - 1
    return x | (1 << (bits - 1)) | 1


def limbs_of(x: int, k: int) -> np.ndarray:
    """``k`` little-endian 32-bit limbs of a non-negative integer."""
    if x < 0 or x >> (32 * k):
        raise ValueError("value does not fit in k limbs")
    return np.array([(x >> (32 * i)) & 0xFFFFFFFF for i in range(k)], dtype=np.uint32)


def int_of_limbs(limbs) -> int:
    x = 0
    for i, w in enumerate(limbs):
        x |= int(w) << (32 * i)
    return x


def _less_than_limbs(x: np.ndarray, n: np.ndarray) -> np.ndarray:
    """Row-wise ``x < n`` for little-endian limb rows ``x`` (count, k) and ``n`` (k,)."""
    k = n.shape[0]
    lt = np.zeros(x.shape[0], dtype=bool)
    decided = np.zeros(x.shape[0], dtype=bool)
    for j in range(k - 1, -1, -1):
        xj = x[:, j]
        nj = n[j]
        lt |= (~decided) & (xj < nj)
        decided |= xj != nj
    return lt


def uniform_limb_residues(N: int, k: int, count: int, seed: int) -> np.ndarray:
    """``count`` residues uniform in [0, N) as a (count, k) uint32 limb array.

    Draws the limbs N occupies, the top one uniform in [0, top limb of N] and
    the others uniform, rejects values >= N (at least half are kept), and pads
    with zero limbs up to k."""
    g = rng(seed)
    kk = max(1, (N.bit_length() + 31) // 32)
    if kk > k:
        raise ValueError("N does not fit in k limbs")
    n = limbs_of(N, kk)
    top = int(n[kk - 1])
    out = np.zeros((count, k), dtype=np.uint32)
    filled = 0
    while filled < count:
        want = 2 * (count - filled) + 64
        x = g.integers(0, 1 << 32, size=(want, kk), dtype=np.uint64).astype(np.uint32)
        x[:, kk - 1] = g.integers(0, top + 1, size=want, dtype=np.uint64).astype(np.uint32)
        x = x[_less_than_limbs(x, n)]
        take = min(len(x), count - filled)
        out[filled:filled + take, :kk] = x[:take]
        filled += take
    return out


def centred_limb_residues(N: int, x: np.ndarray) -> np.ndarray:
    """Residues ``x`` in [0, N) (a (count, k) limb array) moved to the centred
    interval [-(N-1)/2, (N-1)/2], each stored as k-limb two's complement:
    the rows above (N-1)/2 become x - N (mod 2^{32k})."""
    count, k = x.shape
    above = ~_less_than_limbs(x, limbs_of((N - 1) // 2 + 1, k))
    n = limbs_of(N, k).astype(np.int64)
    rows = x[above].astype(np.int64)
    borrow = np.zeros(rows.shape[0], dtype=np.int64)
    for j in range(k):
        d = rows[:, j] - n[j] - borrow
        borrow = (d < 0).astype(np.int64)
        rows[:, j] = d + (borrow << 32)
    out = x.copy()
    out[above] = rows.astype(np.uint32)
    return out


def bounded_limb_residues(N: int, k: int, count: int, seed: int) -> np.ndarray:
    """``count`` residues below N as a (count, k) limb array, drawn fast: the
    top limb uniform in [0, top limb of N), the others uniform.  Every value is
    in [0, N), though not uniform over it (used for large serving pools)."""
    g = rng(seed)
    n = limbs_of(N, k)
    out = g.integers(0, 1 << 32, size=(count, k), dtype=np.uint64).astype(np.uint32)
    top = int(n[k - 1])
    if top == 0:
        raise ValueError("N must fill its top limb")
    out[:, k - 1] = g.integers(0, top, size=count, dtype=np.uint64).astype(np.uint32)
    return out


def ntt_prime(bits_lo: int, bits_hi: int, two_adicity: int, seed: int) -> int:
    """A prime 2^bits_lo <= p < 2^bits_hi with p = 1 mod 2^two_adicity."""
    g = rng(seed)
    step = 1 << two_adicity
    c_lo = ((1 << bits_lo) - 1) // step + 1
    c_hi = ((1 << bits_hi) - 2) // step
    while True:
        c = int(g.integers(c_lo, c_hi, dtype=np.int64, endpoint=True))
        p = c * step + 1
        if is_probable_prime(p):
            return p


def primitive_2n_root(N: int, n: int, seed: int) -> int:
    """psi with psi^n = -1 mod N (a primitive 2n-th root of unity for a power
    of two n), found as g^((N-1)/2n) for random g; N prime, 2n | N - 1."""
    if (N - 1) % (2 * n):
        raise ValueError("2n must divide N - 1")
    g = rng(seed)
    while True:
        x = int(g.integers(2, N - 1, dtype=np.uint64)) if N < (1 << 63) else \
            int(g.integers(2, 1 << 62, dtype=np.int64))
        psi = pow(x, (N - 1) // (2 * n), N)
        if pow(psi, n, N) == N - 1:
            return psi


@dataclass
class Job:
    """One request of the serving workload."""

    arrival_s: float      # arrival time from the start of the stream
    kind: str             # "modmul" or "sweep"
    variant: int          # 0 REDC, 1 signed, 2 Plantard (modmul); sweep variant
    width: int            # 32, 64 or 256 (modmul)
    length: int           # elements (modmul) or odd moduli (sweep)
    n_lo: int = 0         # sweep: first odd modulus
    seed: int = 0         # operand seed


def serving_jobs(count: int, rate_per_s: float, seed: int = 5, sweep_frac: float = 0.05,
                 len_lo: float = 10.0, len_hi: float = 24.0, sweep_moduli: int = 512,
                 sweep_n_max: int = 4095) -> list[Job]:
    """Poisson stream: exponential inter-arrival times at ``rate_per_s``;
    modmul jobs pick variant from {REDC, signed, Plantard} and width from
    {32, 64, 256} (256-bit is REDC only, so other draws are redrawn); a
    ``sweep_frac`` share are sweep jobs over ``sweep_moduli`` consecutive odd N
    at R = 2^16, with the algorithm drawn from {REDC, signed, Plantard}."""
    g = rng(seed)
    t = 0.0
    jobs = []
    for i in range(count):
        t += float(g.exponential(1.0 / rate_per_s))
        if g.uniform() < sweep_frac:
            last_start = sweep_n_max - 2 * (sweep_moduli - 1)
            start = int(g.integers(1, (last_start - 1) // 2 + 1)) * 2 + 1
            variant = int(g.integers(0, 3))
            jobs.append(Job(t, "sweep", variant, 16, sweep_moduli, n_lo=start,
                            seed=seed * 1000003 + i))
            continue
        while True:
            variant = int(g.integers(0, 3))
            width = int((32, 64, 256)[int(g.integers(0, 3))])
            if width != 256 or variant == 0:
                break
        length = int(np.floor(2.0 ** g.uniform(len_lo, len_hi)))
        jobs.append(Job(t, "modmul", variant, width, length, seed=seed * 1000003 + i))
    return jobs
