"""Pins of the whole-array oracle (``oracle.bulk``) against the scalar
definitions of ``oracle.montgomery`` (themselves pinned against the paper by
``test_oracle_pins.py``): every variant, random and edge operands, the
smallest, the benchmark's and the largest admissible moduli, at 32-bit,
64-bit and multi-limb widths."""

import random

import numpy as np
import pytest

import oracle as o
from oracle import bulk

VARIANTS = (0, 1, 2, 3, 4)


def log2R_of(variant, width):
    return 2 * width if variant in (2, 3, 4) else width


def largest_modulus(variant, width, alpha=1):
    """Largest odd N the variant admits at this word width (search down)."""
    l = log2R_of(variant, width)
    if variant == 2:   # N < 2^n / phi: bisect the exact test, then step to odd
        lo, hi = 1, 1 << width
        while hi - lo > 1:
            mid = (lo + hi) // 2
            lo, hi = (mid, hi) if o.plantard_bound_ok(mid, width) else (lo, mid)
        N = lo | 1
    else:              # N < R, 2N < R, N < 2^{n-1}, N < 2^{n-alpha-1}
        N = (1 << {0: width, 1: width - 1, 3: width - 1, 4: width - alpha - 1}[variant]) - 1
    for _ in range(1 << 16):
        if o.precondition_ok(variant, N, l, alpha):
            return N
        N -= 2
    raise AssertionError("no admissible modulus found near the bound")


def operand_range(variant, N):
    """mont_mul's input range: the variant's own output range."""
    if variant in (0, 2):
        return 0, N - 1
    if variant == 1:
        return -(N - 1), N - 1
    return -((N - 1) // 2), (N - 1) // 2


def operands(variant, N, n, rnd):
    lo, hi = operand_range(variant, N)
    xs = [rnd.randint(lo, hi) for _ in range(n)]
    edges = [lo, hi, 0, 1, hi - 1, lo + 1, -1 if lo < 0 else 2]
    xs[:len(edges)] = edges
    return xs


def moduli(variant, width, rnd):
    l = log2R_of(variant, width)
    out = [3, 3329, largest_modulus(variant, width)]
    if o.precondition_ok(variant, 8380417, l, 1):
        out.append(8380417)
    while len(out) < 6:
        N = rnd.randrange(3, largest_modulus(variant, width) + 1) | 1
        if o.precondition_ok(variant, N, l, 1):
            out.append(N)
    return out


@pytest.mark.parametrize("variant", VARIANTS)
def test_u32_path_equals_scalar_definition(variant):
    rnd = random.Random(11 + variant)
    l = log2R_of(variant, 32)
    for N in moduli(variant, 32, rnd):
        a = operands(variant, N, 3000, rnd)
        b = operands(variant, N, 3000, rnd)
        b[:7] = list(reversed(b[:7]))
        dt = np.int32 if variant != 0 and variant != 2 else np.uint32
        got = bulk.mul_value_u32(variant, np.array(a, dtype=np.int64).astype(dt),
                                 np.array(b, dtype=np.int64).astype(dt), N, l, 1)
        want = [o.mul_value(variant, x, y, N, l, 1) for x, y in zip(a, b)]
        assert got.dtype == np.int64
        assert got.tolist() == want, (variant, N)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("width", [32, 64])
def test_object_path_equals_scalar_definition(variant, width):
    rnd = random.Random(100 * width + variant)
    l = log2R_of(variant, width)
    for N in moduli(variant, width, rnd):
        a = operands(variant, N, 1500, rnd)
        b = operands(variant, N, 1500, rnd)
        got = bulk.mul_value_obj(variant, np.array(a, dtype=object), np.array(b, dtype=object),
                                 N, l, 1)
        want = [o.mul_value(variant, x, y, N, l, 1) for x, y in zip(a, b)]
        assert list(got) == want, (variant, width, N)


@pytest.mark.parametrize("variant", VARIANTS)
def test_paths_agree_on_large_arrays(variant):
    """The uint64 and the Python-integer evaluations agree on 2^17 elements of
    the benchmark's moduli (the u32 path is the one full-size tests use)."""
    rng = np.random.default_rng(7 + variant)
    l = log2R_of(variant, 32)
    for N in (3329, 8380417):
        lo, hi = operand_range(variant, N)
        a = rng.integers(lo, hi + 1, size=1 << 17, dtype=np.int64)
        b = rng.integers(lo, hi + 1, size=1 << 17, dtype=np.int64)
        fast = bulk.mul_value_u32(variant, a, b, N, l, 1)
        slow = bulk.mul_value_obj(variant, a, b, N, l, 1)
        assert fast.tolist() == list(slow)


@pytest.mark.parametrize("variant", VARIANTS)
@pytest.mark.parametrize("k", [8, 32])
def test_limb_widths_equal_scalar_definition(variant, k):
    rnd = random.Random(1000 * k + variant)
    bits = 32 * k
    l = 2 * bits if variant in (2, 3, 4) else bits
    top = {0: bits, 1: bits - 1, 2: bits - 1, 3: bits - 1, 4: bits - 2}[variant]
    for N in (rnd.randrange(1 << (top - 1), 1 << top) | 1, (1 << top) - 1 if variant != 2 else
              (rnd.randrange(1 << (top - 2), 1 << (top - 1)) | 1)):
        assert o.precondition_ok(variant, N, l, 1)
        a = operands(variant, N, 300, rnd)
        b = operands(variant, N, 300, rnd)
        signed = variant in (1, 3, 4)
        la, lb = bulk.limbs_from_ints(a, k), bulk.limbs_from_ints(b, k)
        A = bulk.ints_from_limbs(la.reshape(-1), k, signed=signed)
        B = bulk.ints_from_limbs(lb.reshape(-1), k, signed=signed)
        assert list(A) == a and list(B) == b
        got = bulk.mul_value_obj(variant, A, B, N, l, 1)
        assert list(got) == [o.mul_value(variant, x, y, N, l, 1) for x, y in zip(a, b)]


def test_limb_conversions_match_scalar_helpers():
    rnd = random.Random(3)
    for k in (1, 2, 8, 64):
        xs = [0, 1, (1 << (32 * k)) - 1] + [rnd.randrange(1 << (32 * k)) for _ in range(50)]
        limbs = bulk.limbs_from_ints(xs, k)
        assert [o.to_limbs(x, k) for x in xs] == limbs.tolist()
        assert list(bulk.ints_from_limbs(limbs, k)) == [o.from_limbs(r) for r in limbs.tolist()]
        # two's complement reading: the top bit carries weight -2^{32k-1}
        signed = bulk.ints_from_limbs(limbs, k, signed=True)
        assert list(signed) == [x - (1 << (32 * k)) if x >> (32 * k - 1) else x for x in xs]


def test_u32_path_refuses_what_it_cannot_compute_exactly():
    with pytest.raises(ValueError):
        bulk.mul_value_u32(0, np.array([1]), np.array([1]), 1 << 33 | 1, 64)
    with pytest.raises(ValueError):
        bulk.mul_value_u32(1, np.array([1 << 31], dtype=np.int64), np.array([1]), 3329, 32)
    with pytest.raises(ValueError):
        bulk.mul_value_u32(1, np.array([1]), np.array([1]), 3329, 64)
