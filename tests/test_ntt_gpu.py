"""GPU parity of Plantard's prepared-multiplier products and of the batched
negacyclic NTT against the oracle's definitions."""

import random

import numpy as np
import pytest
import torch

import oracle as o
from oracle import ntt as on
import paper_2402_00675_gb300 as mg
import synthetic as sy
from gpu_helpers import dev, empty_like_elems, host, input_range, log2R_of, max_modulus, np_dtype, sync

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


@pytest.mark.parametrize("width", [32, 64])
@pytest.mark.parametrize("variant", [2, 3, 4])
def test_prepared_multipliers(variant, width):
    rnd = random.Random(10 * variant + width)
    l = log2R_of(variant, width)
    dt = np_dtype(variant, width)
    for N in (3329, 8380417 if width == 32 else (1 << 61) - 1, max_modulus(variant, width)):
        if not o.precondition_ok(variant, N, l, 1):
            continue
        ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
        for n, pad in ((4099, 0), (37, 1), (1, 0), (300, 2)):
            lo, hi = input_range(variant, N)
            a = [rnd.randint(lo, hi) for _ in range(n)]
            b = [rnd.randint(lo, hi) for _ in range(n)]
            a[:2] = [lo, hi][:n]
            da, db = dev(a, dt, pad), dev(b, dt, pad)
            pre = torch.zeros((n + pad) * (2 if width == 32 else 4), dtype=torch.int32 if width == 32 else torch.int32, device="cuda")
            pre = pre[pad * (2 if width == 32 else 4):]
            mg.mont_const_prepare(ctx, db, pre, n=n)
            out = empty_like_elems(n, dt, pad)
            mg.mont_mul_pre(ctx, da, pre, out, n=n)
            sync()
            words = pre.cpu().numpy().view(np.uint32).reshape(n, -1)
            got_pre = [sum(int(w) << (32 * i) for i, w in enumerate(row)) for row in words]
            assert got_pre == [on.prepared_multiplier(x, N, l) for x in b], (variant, width, N)
            assert host(out) == [o.mul_value(variant, x, y, N, l, 1) for x, y in zip(a, b)]
            ref = empty_like_elems(n, dt)
            mg.mont_mul(ctx, da, db, ref)
            sync()
            assert host(ref) == host(out)


def test_prepared_refused_for_montgomery_family():
    ctx = mg.mont_ctx_create(3329, 32, 0)
    x = torch.zeros(8, dtype=torch.uint32, device="cuda")
    with pytest.raises(mg.MontError):
        mg.mont_const_prepare(ctx, x, torch.zeros(8, dtype=torch.uint64, device="cuda"))


def ntt_cases():
    p32_big = sy.ntt_prime(31, 32, 12, seed=21)          # above 2^31: exercises carries
    p_plant = sy.ntt_prime(30, 31, 12, seed=22)          # inside Plantard's 2^32/phi bound
    rns = sy.rns_primes(1, seed=3)[0]
    p_lazy_top = sy.ntt_prime(29, 30, 12, seed=24)      # 4N <= 2^32: lazy butterflies, largest values
    return [
        (p_lazy_top, 32, 2, 10), (p_lazy_top, 32, 2, 5), (p_lazy_top, 32, 0, 10),
        (8380417, 32, 0, 8), (8380417, 32, 2, 8), (3329, 32, 0, 7), (3329, 32, 2, 7),
        (7681, 32, 2, 5), (p32_big, 32, 0, 10), (p_plant, 32, 2, 9), (p_plant, 32, 2, 6),
        (rns, 64, 0, 8), (rns, 64, 2, 10), (rns, 64, 2, 5), (rns, 64, 0, 9),
    ]


@pytest.mark.parametrize("N,width,variant,log2n", ntt_cases())
def test_ntt_forward_inverse_against_definition(N, width, variant, log2n):
    n = 1 << log2n
    l = log2R_of(variant, width)
    ctx = mg.mont_ctx_create(N, l, variant)
    psi = sy.primitive_2n_root(N, n, seed=log2n)
    plan = mg.Ntt(ctx, log2n, psi)
    batch = 37
    rnd = random.Random(N + log2n)
    polys = [[rnd.randrange(N) for _ in range(n)] for _ in range(batch)]
    polys[0] = [N - 1] * n
    dt = np.uint32 if width == 32 else np.uint64
    x = dev([c for p in polys for c in p], dt)
    y = torch.empty_like(x)
    plan.forward(x, y)
    z = torch.empty_like(x)
    plan.inverse(y, z)
    sync()
    assert torch.equal(z, x)                                # round trip, every polynomial
    got = host(y)
    check = [0, 1, batch - 1] if n <= 256 else [0, batch - 1]
    for p in check:
        assert got[p * n:(p + 1) * n] == on.ntt_forward(polys[p], N, psi), p
    # inverse against the definition on arbitrary transform-domain input
    A = [rnd.randrange(N) for _ in range(n)]
    xa = dev(A, dt)
    ya = torch.empty_like(xa)
    plan.inverse(xa, ya, batch=1)
    sync()
    if n <= 256:
        assert host(ya) == on.ntt_inverse(A, N, psi)
    # in place
    plan.forward(x, x)
    sync()
    assert torch.equal(x, y)


def test_ntt_rejects_bad_parameters():
    ctx = mg.mont_ctx_create(8380417, 32, 0)
    with pytest.raises(mg.MontError):
        mg.Ntt(ctx, 8, 5)                                   # 5^256 != -1 mod N
    with pytest.raises(mg.MontError):
        mg.Ntt(ctx, 11, sy.primitive_2n_root(8380417, 2048, 1))
    s1 = mg.mont_ctx_create(8380417, 32, 1)
    with pytest.raises(mg.MontError):
        mg.Ntt(s1, 8, sy.primitive_2n_root(8380417, 256, 1))


@pytest.mark.parametrize("variant", [0, 2])
def test_ntt_full_size_2p18_polynomials(variant):
    """The benchmark's transform: 2^18 polynomials of length 256 mod 8380417;
    round trip of every coefficient, sampled polynomials against the oracle."""
    N, log2n, batch = 8380417, 8, 1 << 18
    n = 1 << log2n
    psi = sy.primitive_2n_root(N, n, seed=1)
    ctx = mg.mont_ctx_create(N, 32 if variant == 0 else 64, variant)
    plan = mg.Ntt(ctx, log2n, psi)
    x = torch.from_numpy(sy.uniform_residues(N, batch * n, seed=7)).cuda()
    y = torch.empty_like(x)
    plan.forward(x, y)
    z = torch.empty_like(x)
    plan.inverse(y, z)
    sync()
    assert torch.equal(z, x)
    xs = x.view(torch.int32).cpu().numpy()
    ys = y.view(torch.int32).cpu().numpy()
    rnd = random.Random(variant)
    for p in [0, batch - 1] + [rnd.randrange(batch) for _ in range(3)]:
        poly = [int(v) for v in xs[p * n:(p + 1) * n]]
        assert [int(v) for v in ys[p * n:(p + 1) * n]] == on.ntt_forward(poly, N, psi), p
