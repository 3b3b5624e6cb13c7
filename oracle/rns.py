"""Residue-number-system conversions through the Chinese remainder theorem.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Section 2 derives the two-modulus CRT from Qin's identity (Eq. (2): T is
congruent to r1 R^{-1} R + r2 N^{-1} N modulo NR) and says the multi-modulus
case follows in the same manner without stating it.  The definition used
here is the textbook one: for pairwise coprime moduli p_i with product P and
M_i = P / p_i, the integer X in [0, P) with X = x_i (mod p_i) for every i is

    X = sum_i x_i M_i (M_i^{-1} mod p_i)  mod P.
"""

from __future__ import annotations

from math import gcd


def product(moduli) -> int:
    P = 1
    for p in moduli:
        P *= p
    return P


def pairwise_coprime(moduli) -> bool:
    return all(gcd(a, b) == 1 for i, a in enumerate(moduli) for b in moduli[i + 1:])


def to_residues(X: int, moduli):
    """[X mod p_i]."""
    return [X % p for p in moduli]


def from_residues(xs, moduli) -> int:
    """The unique X in [0, P) with X = x_i (mod p_i): the CRT formula above."""
    P = product(moduli)
    X = 0
    for x, p in zip(xs, moduli):
        M = P // p
        X += x * M * pow(M, -1, p)
    return X % P
