"""GPU parity of the batched RNS path (mont_mul_batched and the graph plan).

Each vector of a batch must equal the oracle element by element, and equal
what mont_mul gives for the same vector alone."""

import random

import numpy as np
import pytest
import torch

import oracle as o
from oracle import bulk
import paper_2402_00675_gb300 as mg
import synthetic as sy
from gpu_helpers import dev, empty_like_elems, host, input_range, log2R_of, np_dtype, sync

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


def make_batch(width, count, len_lo, len_hi, seed, variants=(0,), moduli=None, pad=False):
    rnd = random.Random(seed)
    if moduli is None:
        moduli = sy.rns_primes(count, seed=seed) if width == 64 else \
            [p for p in (3329, 8380417, 12289, 7681, 65537, 40961, 786433, 5767169) * 40][:count]
    entries = []
    for j in range(count):
        N = moduli[j % len(moduli)]
        variant = variants[j % len(variants)]
        l = log2R_of(variant, width)
        if not o.precondition_ok(variant, N, l, 1):
            variant, l = 0, width
        n = int(2 ** rnd.uniform(len_lo, len_hi)) if len_hi > 0 else 0
        if j % 7 == 3:
            n = 0
        lo, hi = input_range(variant, N)
        a = [rnd.randint(lo, hi) for _ in range(n)]
        b = [rnd.randint(lo, hi) for _ in range(n)]
        dt = np_dtype(variant, width)
        p = (j % 3) if pad else 0
        entries.append(dict(N=N, variant=variant, l=l, a=a, b=b, dt=dt,
                            da=dev(a, dt, p), db=dev(b, dt, p), out=empty_like_elems(n, dt, p),
                            ctx=mg.mont_ctx_create(N, l, variant, alpha=1)))
    return entries


def check(entries):
    for e in entries:
        want = [o.mul_value(e["variant"], x, y, e["N"], e["l"], 1) for x, y in zip(e["a"], e["b"])]
        assert host(e["out"]) == want, (e["N"], e["variant"])


def run_batched(entries):
    mg.mont_mul_batched([e["ctx"] for e in entries], [e["da"] for e in entries],
                        [e["db"] for e in entries], [e["out"] for e in entries],
                        [len(e["a"]) for e in entries])
    sync()


@pytest.mark.parametrize("width", [32, 64])
def test_batched_mixed_variants_match_oracle(width):
    entries = make_batch(width, 40, 0, 14, seed=width, variants=(0, 1, 2, 3, 4))
    run_batched(entries)
    check(entries)


@pytest.mark.parametrize("width", [32, 64])
def test_batched_misaligned_and_empty(width):
    entries = make_batch(width, 17, 0, 11, seed=100 + width, variants=(0, 1, 3), pad=True)
    run_batched(entries)
    check(entries)


def test_batched_more_than_one_launch_group():
    entries = make_batch(64, 300, 0, 8, seed=7, variants=(0, 2))
    run_batched(entries)
    check(entries)


def test_batched_equals_alone():
    entries = make_batch(64, 32, 4, 12, seed=11, variants=(0, 1, 2, 3, 4))
    run_batched(entries)
    for e in entries:
        alone = torch.empty_like(e["out"])
        if len(e["a"]):
            mg.mont_mul(e["ctx"], e["da"], e["db"], alone)
        sync()
        assert torch.equal(alone, e["out"])


def test_batch_plan_graph_launch_and_update():
    entries = make_batch(64, 33, 0, 12, seed=13, variants=(0, 1, 2))
    plan = mg.Batch([e["ctx"] for e in entries], [e["da"] for e in entries],
                    [e["db"] for e in entries], [e["out"] for e in entries],
                    [len(e["a"]) for e in entries])
    plan.launch()
    sync()
    check(entries)
    # new buffers with the same shapes: swap a and b, write to fresh outputs
    outs2 = [torch.zeros_like(e["out"]) for e in entries]
    plan.update([e["db"] for e in entries], [e["da"] for e in entries], outs2)
    plan.launch()
    plan.launch()
    sync()
    for e, o2 in zip(entries, outs2):
        want = [o.mul_value(e["variant"], y, x, e["N"], e["l"], 1) for x, y in zip(e["a"], e["b"])]
        assert host(o2) == want
    plan.close()


def test_batched_argument_errors():
    e64 = make_batch(64, 2, 3, 4, seed=17)
    e32 = make_batch(32, 1, 3, 4, seed=18)
    mixed = e64 + e32
    with pytest.raises(mg.MontError):
        run_batched(mixed)
    ctx_big = mg.mont_ctx_create((1 << 255) + 1, 256, 0)
    with pytest.raises(mg.MontError):
        mg.mont_mul_batched([ctx_big], [e64[0]["da"]], [e64[0]["db"]], [e64[0]["out"]], [3])
    mg.mont_mul_batched([], [], [], [], [])


def test_full_size_rns64_batch():
    """32 primes of 60-62 bits, p = 1 mod 2^17, log-uniform lengths 2^12..2^22,
    one graph-launched batch: every element of every vector against the
    definition T R^{-1} mod p (Python integers)."""
    primes = sy.rns_primes(32, seed=3)
    lens = sy.log_uniform_lengths(32, 12, 22, seed=3)
    ctxs, da, db, outs, hs = [], [], [], [], []
    for j, (p, n) in enumerate(zip(primes, lens)):
        a = sy.uniform_residues(p, n, seed=1000 + j, dtype=np.uint64)
        b = sy.uniform_residues(p, n, seed=2000 + j, dtype=np.uint64)
        ctxs.append(mg.mont_ctx_create(p, 64, 0))
        da.append(torch.from_numpy(a).cuda())
        db.append(torch.from_numpy(b).cuda())
        outs.append(torch.empty(n, dtype=torch.uint64, device="cuda"))
        hs.append((a, b))
    plan = mg.Batch(ctxs, da, db, outs, lens)
    plan.launch()
    sync()
    for j, (p, n) in enumerate(zip(primes, lens)):
        got = bulk.as_ints(outs[j].cpu().numpy())
        a, b = hs[j]
        want = bulk.mul_value_obj(0, a, b, p, 64)
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, (j, bad[:5])
        assert int(want[0]) == o.mul_value(0, int(a[0]), int(b[0]), p, 64)
