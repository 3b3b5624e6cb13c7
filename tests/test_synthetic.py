"""The seeded input generators: deterministic, in range, right shapes."""

import numpy as np
import pytest

import synthetic as sy


def test_residues_deterministic_and_in_range():
    a = sy.uniform_residues(3329, 10000, 1)
    b = sy.uniform_residues(3329, 10000, 1)
    assert a.dtype == np.uint32 and np.array_equal(a, b)
    assert a.max() < 3329
    c = sy.centred_residues(8380417, 10000, 2)
    assert c.dtype == np.int32 and c.min() >= -4190208 and c.max() <= 4190208
    u = sy.lift_unsigned(c, 8380417)
    assert u.dtype == np.uint32 and u.max() < 8380417
    assert np.array_equal((u.astype(np.int64) - c) % 8380417, np.zeros(10000, dtype=np.int64))
    big = sy.uniform_residues((1 << 64) - 59, 1000, 3, dtype=np.uint64)
    assert big.dtype == np.uint64


def test_rns_primes():
    ps = sy.rns_primes(32, seed=3)
    assert len(set(ps)) == 32
    for p in ps:
        assert (1 << 59) <= p < (1 << 62) and p % (1 << 17) == 1
    assert ps == sy.rns_primes(32, seed=3)
    sympy = pytest.importorskip("sympy")
    assert all(sympy.isprime(p) for p in ps)


def test_miller_rabin_small_numbers():
    sieve = [True] * 5000
    sieve[0] = sieve[1] = False
    for i in range(2, 5000):
        if sieve[i]:
            for j in range(i * i, 5000, i):
                sieve[j] = False
    assert [sy.is_probable_prime(i) for i in range(5000)] == sieve


def test_lengths_and_moduli():
    ls = sy.log_uniform_lengths(1000, 12, 22, 3)
    assert min(ls) >= 1 << 12 and max(ls) <= 1 << 22
    for bits in (256, 384, 1024, 2048):
        N = sy.random_odd_modulus(bits, 4)
        assert N.bit_length() == bits and N % 2 == 1


def test_limb_residues_below_modulus():
    N = sy.random_odd_modulus(256, 4)
    x = sy.uniform_limb_residues(N, 8, 2000, 5)
    assert x.shape == (2000, 8) and x.dtype == np.uint32
    vals = [sy.int_of_limbs(row) for row in x]
    assert all(0 <= v < N for v in vals)
    assert sy.int_of_limbs(sy.limbs_of(N, 8)) == N


def test_serving_jobs_mix():
    jobs = sy.serving_jobs(2000, 100.0, seed=5)
    assert all(j2.arrival_s >= j1.arrival_s for j1, j2 in zip(jobs, jobs[1:]))
    sweeps = [j for j in jobs if j.kind == "sweep"]
    assert 0.02 < len(sweeps) / len(jobs) < 0.09
    for j in jobs:
        if j.kind == "modmul":
            assert j.variant in (0, 1, 2) and j.width in (32, 64, 256)
            assert j.width != 256 or j.variant == 0
            assert (1 << 10) <= j.length <= (1 << 24)
        else:
            assert j.n_lo % 2 == 1 and j.n_lo >= 3 and j.n_lo + 2 * 511 <= 4095


def test_bounded_limb_residues():
    N = sy.random_odd_modulus(256, 11)
    x = sy.bounded_limb_residues(N, 8, 5000, 3)
    assert x.shape == (5000, 8)
    assert all(sy.int_of_limbs(r) < N for r in x)


def test_centred_limb_residues():
    N = sy.random_odd_modulus(255, seed=5)
    x = sy.uniform_limb_residues(N, 8, 4000, seed=3)
    c = sy.centred_limb_residues(N, x)
    half = (N - 1) // 2
    signed = []
    for xr, cr in zip(x, c):
        v = sy.int_of_limbs(cr)
        v = v - (1 << 256) if v >> 255 else v
        assert (v - sy.int_of_limbs(xr)) % N == 0 and -half <= v <= half
        signed.append(v)
    assert 0.4 < sum(v < 0 for v in signed) / len(signed) < 0.6
    # the ends of the interval map as specified
    ends = np.stack([sy.limbs_of(half, 8), sy.limbs_of(half + 1, 8), sy.limbs_of(0, 8)])
    got = sy.centred_limb_residues(N, ends)
    assert sy.int_of_limbs(got[0]) == half
    assert sy.int_of_limbs(got[1]) == (half + 1 - N) % (1 << 256)
    assert sy.int_of_limbs(got[2]) == 0
