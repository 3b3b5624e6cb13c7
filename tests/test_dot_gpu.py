"""GPU parity of the lazy-reduction dot products (Algorithm 4 applied once to
sums of up to 4^(alpha+1) products) against the definition."""

import random

import numpy as np
import pytest
import torch

import oracle as o
import paper_2402_00675_gb300 as mg
import synthetic as sy
from gpu_helpers import dev, host, sync

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


def cases():
    rns = sy.rns_primes(1, seed=3)[0]      # < 2^62: alpha = 1 admissible at 64 bits
    return [(8380417, 32, 1), (3329, 32, 1), (3329, 32, 2), ((1 << 29) - 3, 32, 1),
            (3329, 32, 8), (rns, 64, 1), (12289, 64, 3)]


@pytest.mark.parametrize("N,width,alpha", cases())
def test_dot_lazy_matches_definition(N, width, alpha):
    l = 2 * width
    if not o.precondition_ok(o.SIGNED_PLANTARD2, N, l, alpha):
        pytest.skip("modulus outside Algorithm 4's bound for this alpha")
    ctx = mg.mont_ctx_create(N, l, o.SIGNED_PLANTARD2, alpha=alpha)
    rnd = random.Random(N + alpha)
    h = (N - 1) // 2
    dt = np.int32 if width == 32 else np.int64
    kmax = 4 ** (alpha + 1)
    for k in sorted({1, 3, 4, 7, min(kmax, 16), min(kmax, 1024), kmax}):
        rows = 513 if k <= 64 else (31 if k <= 1024 else 2)
        a = [rnd.randint(-h, h) for _ in range(rows * k)]
        b = [rnd.randint(-h, h) for _ in range(rows * k)]
        # the extreme row: every product at +N^2/4 / -N^2/4
        a[:k] = [-h] * k
        b[:k] = [-h] * k
        a[k:2 * k] = [h] * k
        b[k:2 * k] = [-h] * k
        out = torch.zeros(rows, dtype=torch.int32 if width == 32 else torch.int64, device="cuda")
        mg.mont_dot_lazy(ctx, dev(a, dt), dev(b, dt), out, k)
        sync()
        want = [o.sigpredc_value(sum(x * y for x, y in zip(a[j * k:(j + 1) * k], b[j * k:(j + 1) * k])),
                                 N, 1 << l) for j in range(rows)]
        assert host(out) == want, (N, width, alpha, k)
    with pytest.raises(mg.MontError):
        mg.mont_dot_lazy(ctx, dev([0] * (kmax + 1), dt), dev([0] * (kmax + 1), dt),
                         torch.zeros(1, dtype=out.dtype, device="cuda"), kmax + 1)


def test_dot_lazy_refuses_other_variants():
    ctx = mg.mont_ctx_create(3329, 64, o.SIGNED_PLANTARD)
    z = torch.zeros(4, dtype=torch.int32, device="cuda")
    with pytest.raises(mg.MontError):
        mg.mont_dot_lazy(ctx, z, z, z[:1], 4)
