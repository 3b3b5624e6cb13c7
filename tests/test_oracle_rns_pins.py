"""Pins of the oracle's CRT conversions: brute-force search on tiny moduli,
the two-modulus case written as Eq. (2) of Section 2, and round trips."""

import random

import oracle as o
from oracle import rns


def test_reconstruction_by_search():
    for moduli in ([3, 5], [3, 5, 7], [5, 7, 9, 11], [13, 17], [3, 7, 11, 13]):
        P = rns.product(moduli)
        for X in range(P):
            xs = [X % p for p in moduli]
            found = [y for y in range(P) if all(y % p == x for p, x in zip(moduli, xs))]
            assert found == [X]
            assert rns.from_residues(xs, moduli) == X


def test_two_moduli_is_qins_crt_formula():
    # Eq. (2): T = r1 R^{-1} R + r2 N^{-1} N (mod N R), with R^{-1} mod N and N^{-1} mod R
    rnd = random.Random(3)
    for _ in range(300):
        N = rnd.randrange(3, 1 << 40) | 1
        R = rnd.randrange(3, 1 << 40) | 1
        if not rns.pairwise_coprime([N, R]):
            continue
        T = rnd.randrange(N * R)
        r1, r2 = T % N, T % R
        via_qin = (r1 * pow(R, -1, N) * R + r2 * pow(N, -1, R) * N) % (N * R)
        assert via_qin == T
        assert rns.from_residues([r1, r2], [N, R]) == T


def test_round_trips_on_rns_primes():
    import synthetic as sy
    ps = sy.rns_primes(32, seed=3)
    assert rns.pairwise_coprime(ps)
    P = rns.product(ps)
    rnd = random.Random(5)
    for _ in range(50):
        X = rnd.randrange(P)
        assert rns.from_residues(rns.to_residues(X, ps), ps) == X
