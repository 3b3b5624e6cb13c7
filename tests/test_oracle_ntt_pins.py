"""Pins of the oracle's prepared-multiplier products and NTT definitions.

* The prepared form (Section 3.2's fixed-multiplier trick) must give exactly
  the definition's value for every in-domain a, b: checked exhaustively on
  small R against predc_value / sigpredc_value, which use a modular inverse.
* The transform: a hand-derived 4-point example fixes the output order; the
  negacyclic convolution theorem (pointwise product of transforms equals the
  transform of the schoolbook product modulo x^n + 1) and the round trip pin
  the forward and inverse definitions against each other and against plain
  polynomial arithmetic.
"""

import random

import pytest

import oracle as o
from oracle import ntt


@pytest.mark.parametrize("n", [3, 4, 5, 6])
def test_prepared_plantard_equals_definition(n):
    l = 2 * n
    R = 1 << l
    for N in range(3, 1 << n, 2):
        if o.plantard_bound_ok(N, n):
            for b in range(N):
                bp = ntt.prepared_multiplier(b, N, l)
                assert (bp * N - b) % R == 0          # b' N = b (mod R)
                for a in range(N):
                    assert ntt.predc_prepared_alg(a, bp, N, l) == o.predc_value(a * b, N, R)
        if N < (1 << (n - 1)):
            h = (N - 1) // 2
            for b in range(-h, h + 1):
                bp = ntt.prepared_multiplier(b, N, l)
                for a in range(-h, h + 1):
                    assert ntt.sigpredc1_prepared_alg(a, bp, N, l) == o.sigpredc_value(a * b, N, R)


def test_four_point_transform_by_hand():
    # N = 17, n = 4, psi = 2 (2^4 = 16 = -1 mod 17).  For a(x) = x the outputs are
    # psi^(2 brv(i) + 1) with brv over 2 bits = (0, 2, 1, 3): exponents 1, 5, 3, 7,
    # i.e. 2, 32 = 15, 8, 128 = 9 (mod 17).
    assert ntt.is_primitive_2n_root(2, 17, 4)
    assert ntt.ntt_forward([0, 1, 0, 0], 17, 2) == [2, 15, 8, 9]
    assert ntt.ntt_forward([1, 0, 0, 0], 17, 2) == [1, 1, 1, 1]
    assert ntt.ntt_forward([1, 1, 0, 0], 17, 2) == [3, 16, 9, 10]


@pytest.mark.parametrize("N,n", [(17, 8), (97, 16), (7681, 64), (8380417, 64), (12289, 128)])
def test_convolution_theorem_and_round_trip(N, n):
    rnd = random.Random(N + n)
    psi = next(g for g in range(2, N) if ntt.is_primitive_2n_root(pow(g, (N - 1) // (2 * n), N), N, n))
    psi = pow(psi, (N - 1) // (2 * n), N)
    assert ntt.is_primitive_2n_root(psi, N, n)
    for _ in range(3):
        a = [rnd.randrange(N) for _ in range(n)]
        b = [rnd.randrange(N) for _ in range(n)]
        A, B = ntt.ntt_forward(a, N, psi), ntt.ntt_forward(b, N, psi)
        C = [x * y % N for x, y in zip(A, B)]
        assert ntt.ntt_inverse(C, N, psi) == ntt.negacyclic_product(a, b, N)
        assert ntt.ntt_inverse(A, N, psi) == a


def test_planted_natural_order_is_caught():
    def forward_natural(a, N, psi):
        n = len(a)
        return [sum(a[j] * pow(psi, (2 * i + 1) * j, N) for j in range(n)) % N for i in range(n)]
    assert forward_natural([0, 1, 0, 0], 17, 2) != [2, 15, 8, 9]
