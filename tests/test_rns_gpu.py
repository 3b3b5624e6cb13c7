"""GPU parity of the RNS conversions against the oracle's CRT definition."""

import random

import numpy as np
import pytest
import torch

from oracle import rns as orns
import paper_2402_00675_gb300 as mg
import synthetic as sy
from gpu_helpers import sync

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


def limbs_tensor(vals, k):
    arr = np.zeros((len(vals), k), dtype=np.uint32)
    for i, v in enumerate(vals):
        arr[i] = sy.limbs_of(v, k)
    return torch.from_numpy(arr.reshape(-1)).cuda()


def bigs(t, k):
    return [sy.int_of_limbs(r) for r in t.cpu().numpy().reshape(-1, k)]


def moduli_sets():
    rnd = random.Random(9)
    odd_small = [3, 5, 7, 11, 13]
    mixed = []
    while len(mixed) < 6:
        c = rnd.randrange(1 << 40, 1 << 63) | 1
        if orns.pairwise_coprime(mixed + [c]):
            mixed.append(c)
    return [odd_small, sy.rns_primes(4, seed=3), sy.rns_primes(32, seed=3), mixed,
            [(1 << 63) - 25, (1 << 63) - 259]]


@pytest.mark.parametrize("idx", range(5))
def test_round_trip_and_definitions(idx):
    ps = moduli_sets()[idx]
    r = mg.Rns(ps)
    P = orns.product(ps)
    k = r.limbs
    assert P < 1 << (32 * k)
    rnd = random.Random(idx)
    n = 1000
    X = [rnd.randrange(P) for _ in range(n)]
    # small values (and 0, 1, P - 1): their CRT sums lie just above a multiple
    # of P, where the quotient estimate is one short and P is subtracted
    X[:10] = [0, 1, P - 1, 2, 3, (1 << 32) - 1, 1 << 32, (1 << 64) - 1, P - 2, P // 2]
    X[:10] = [x % P for x in X[:10]]
    tX = limbs_tensor(X, k)
    res = torch.zeros(len(ps) * n, dtype=torch.uint64, device="cuda")
    r.to_residues(tX, res, n)
    back = torch.zeros_like(tX)
    r.from_residues(res, back, n)
    sync()
    got_res = res.cpu().numpy().reshape(len(ps), n)
    for e in range(n):
        assert [int(got_res[i][e]) for i in range(len(ps))] == orns.to_residues(X[e], ps)
    assert bigs(back, k) == X
    # from_residues on arbitrary residue vectors against the CRT formula
    xs = [[rnd.randrange(p) for p in ps] for _ in range(n)]
    rr = torch.from_numpy(np.array([[x[i] for x in xs] for i in range(len(ps))],
                                   dtype=np.uint64).reshape(-1)).cuda()
    out = torch.zeros_like(tX)
    r.from_residues(rr, out, n)
    sync()
    assert bigs(out, k) == [orns.from_residues(x, ps) for x in xs]


def test_to_residues_above_P():
    ps = sy.rns_primes(4, seed=3)
    r = mg.Rns(ps)
    k = r.limbs
    rnd = random.Random(2)
    X = [rnd.randrange(1 << (32 * k)) for _ in range(257)]
    res = torch.zeros(len(ps) * len(X), dtype=torch.uint64, device="cuda")
    r.to_residues(limbs_tensor(X, k), res, len(X))
    sync()
    got = res.cpu().numpy().reshape(len(ps), len(X))
    for e, x in enumerate(X):
        assert [int(got[i][e]) for i in range(len(ps))] == orns.to_residues(x, ps)


def test_rns_rejects_bad_moduli():
    for bad in ([4, 7], [9, 15], [3, 1 << 63], [], [3] * 65):
        with pytest.raises((mg.MontError, ValueError, OverflowError)):
            mg.Rns(bad)
    big = sy.rns_primes(34, seed=3)                 # product above 2^2048
    with pytest.raises(mg.MontError):
        mg.Rns(big)
