"""GPU parity of the 32- and 64-bit word kernels against the oracle.

Every comparison is exact (integer results, bit for bit).  Sizes span many
vectors and blocks plus a ragged tail; edge cases cover n in {1, 3, ...}
(shorter than one vector), misaligned buffers (scalar and 128-bit paths),
in-place operation, the extreme operands 0, 1, N-1 and the largest modulus
each variant admits."""

import random

import numpy as np
import pytest
import torch

import oracle as o
from oracle import bulk
import paper_2402_00675_gb300 as mg
from gpu_helpers import (dev, dev_wide, empty_like_elems, host, input_range, log2R_of,
                         max_modulus, np_dtype, sync)

pytestmark = pytest.mark.gpu

VARIANTS = [0, 1, 2, 3, 4]
WIDTHS = [32, 64]


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


def moduli_for(variant, width, rnd):
    l = log2R_of(variant, width)
    top = max_modulus(variant, width)
    out = [3, 3329, top]
    if width == 32:
        out.append(8380417 if o.precondition_ok(variant, 8380417, l, 1) else 12289)
    while len(out) < 6:
        N = rnd.randrange(3, top + 1) | 1
        if o.precondition_ok(variant, N, l, 1):
            out.append(N)
    return out


def operands(variant, N, n, rnd):
    lo, hi = input_range(variant, N)
    edges = [lo, hi, 0, 1 if hi >= 1 else 0, hi - 1 if hi > lo else hi]
    xs = [rnd.randint(lo, hi) for _ in range(n)]
    for i, e in enumerate(edges[: min(len(edges), n)]):
        xs[i] = e
    return xs


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_mul_parity(variant, width):
    rnd = random.Random(1000 * variant + width)
    l = log2R_of(variant, width)
    dt = np_dtype(variant, width)
    for idx, N in enumerate(moduli_for(variant, width, rnd)):
        n = 100_003 if idx == 1 else 4099
        ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
        a = operands(variant, N, n, rnd)
        b = operands(variant, N, n, rnd)
        b[:5] = list(reversed(b[:5]))
        out = empty_like_elems(n, dt)
        mg.mont_mul(ctx, dev(a, dt), dev(b, dt), out)
        sync()
        got = host(out)
        want = [o.mul_value(variant, x, y, N, l, 1) for x, y in zip(a, b)]
        assert got == want, (variant, width, N)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_domain_maps_parity(variant, width):
    rnd = random.Random(2000 * variant + width)
    l = log2R_of(variant, width)
    dt = np_dtype(variant, width)
    for N in moduli_for(variant, width, rnd)[:4]:
        ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
        n = 5003
        x = operands(variant, N, n, rnd)
        if variant in (3, 4):
            pass
        elif variant == 1:
            x = [o.mods(v, N) for v in x]     # canonical inputs for the round trip
        y = empty_like_elems(n, dt)
        mg.mont_to_domain(ctx, dev(x, dt), y)
        back = empty_like_elems(n, dt)
        mg.mont_from_domain(ctx, y, back)
        sync()
        gy = host(y)
        assert gy == [o.to_domain_value(variant, v, N, l, 1) for v in x]
        assert host(back) == [o.from_domain_value(variant, v, N, l, 1) for v in gy]
        assert host(back) == x
        # from_domain on arbitrary outputs of the variant's range
        z = operands(variant, N, n, rnd)
        zo = empty_like_elems(n, dt)
        mg.mont_from_domain(ctx, dev(z, dt), zo)
        sync()
        assert host(zo) == [o.from_domain_value(variant, v, N, l, 1) for v in z]


def redc_inputs(variant, N, l, n, rnd, alpha=1):
    lo, hi = o.input_domain(variant, N, l, alpha)
    T = [rnd.randint(lo, hi) for _ in range(n)]
    edges = [lo, hi, 0, lo + 1, hi - 1]
    T[: len(edges)] = edges
    return T


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_redc_parity(variant, width):
    rnd = random.Random(3000 * variant + width)
    l = log2R_of(variant, width)
    dt = np_dtype(variant, width)
    for N in moduli_for(variant, width, rnd):
        ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
        n = 6007
        T = redc_inputs(variant, N, l, n, rnd)
        out = empty_like_elems(n, dt)
        mg.mont_redc(ctx, dev_wide(T, width), out)
        sync()
        assert host(out) == [o.reduce_value(variant, t, N, l, 1) for t in T], (variant, N)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_ragged_sizes_alignment_and_in_place(variant, width):
    rnd = random.Random(4000 * variant + width)
    l = log2R_of(variant, width)
    dt = np_dtype(variant, width)
    N = moduli_for(variant, width, rnd)[2]
    ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
    for n in (1, 2, 3, 5, 7, 8, 9, 15, 16, 17, 31, 33, 63, 65, 257, 1023, 2049):
        for pad in (0, 1, 2, 4):
            a = operands(variant, N, n, rnd)
            b = operands(variant, N, n, rnd)
            want = [o.mul_value(variant, x, y, N, l, 1) for x, y in zip(a, b)]
            da, db = dev(a, dt, pad), dev(b, dt, pad)
            out = empty_like_elems(n, dt, pad)
            mg.mont_mul(ctx, da, db, out)
            sync()
            assert host(out) == want, (n, pad)
            mg.mont_mul(ctx, da, db, da)          # in place over a
            sync()
            assert host(da) == want, (n, pad, "in place")
    # n = 0 touches nothing
    z = empty_like_elems(4, dt)
    mg.mont_mul(ctx, z, z, z, n=0)
    sync()


def test_full_size_redc32_2p20():
    """REDC, R = 2^32, N = 3329, 2^20 pairs uniform in [0, N): every element
    against the definition T R^{-1} mod N."""
    import synthetic as sy
    N, n = sy.REDC32_N, 1 << 20
    a = sy.uniform_residues(N, n, seed=1)
    b = sy.uniform_residues(N, n, seed=101)
    ctx = mg.mont_ctx_create(N, 32, 0)
    out = torch.empty(n, dtype=torch.uint32, device="cuda")
    mg.mont_mul(ctx, torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), out)
    sync()
    got = out.cpu().numpy().astype(np.int64)
    want = bulk.mul_value_u32(0, a, b, N, 32)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (bad[:10], got[bad[:10]], want[bad[:10]])
    # the whole-array oracle agrees with the scalar definition where it is cheap
    for i in (0, 1, n // 2, n - 1):
        assert int(want[i]) == o.mul_value(0, int(a[i]), int(b[i]), N, 32)


@pytest.mark.parametrize("N", [3329, 8380417])
def test_full_size_word32_variants_2p26(N):
    """The 2^26-pair workload of the signed and Plantard variants, as the
    benchmark launches it: every element of every output against the
    definition (Algorithm 1: its representative (T - mN)/R; Algorithms 2-4:
    -T R^{-1} mod N, mods N for the signed ones)."""
    import synthetic as sy
    n = 1 << 26
    a = sy.centred_residues(N, n, seed=2 * N + 1)
    b = sy.centred_residues(N, n, seed=2 * N + 2)
    au, bu = sy.lift_unsigned(a, N), sy.lift_unsigned(b, N)
    da, db = torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda()
    dau, dbu = torch.from_numpy(au).cuda(), torch.from_numpy(bu).cuda()
    for variant, l in ((1, 32), (2, 64), (3, 64), (4, 64)):
        ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
        signed = variant != 2
        out = torch.empty(n, dtype=torch.int32 if signed else torch.uint32, device="cuda")
        if signed:
            mg.mont_mul(ctx, da, db, out)
        else:
            mg.mont_mul(ctx, dau, dbu, out)
        sync()
        got = out.cpu().numpy().astype(np.int64)
        xa, xb = (a, b) if signed else (au, bu)
        want = bulk.mul_value_u32(variant, xa, xb, N, l, 1)
        bad = np.flatnonzero(got != want)
        assert bad.size == 0, (variant, bad[:10], got[bad[:10]], want[bad[:10]])
        lo, hi = o.claimed_range(variant, N)
        assert got.min() >= lo and got.max() <= hi
        for i in (0, n - 1):
            assert int(want[i]) == o.mul_value(variant, int(xa[i]), int(xb[i]), N, l, 1)


@pytest.mark.parametrize("width", WIDTHS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_dependent_launch_chain(variant, width):
    """Word kernels start while the kernel before them drains (programmatic
    launch) and wait for it before touching memory.  A chain of 8 dependent
    products x <- x b, ping-ponging between two buffers (each launch reads
    what the previous one wrote and overwrites what it read), run directly
    and replayed from a captured CUDA graph, equals the oracle's chain."""
    rnd = random.Random(4000 + 10 * variant + width)
    l = log2R_of(variant, width)
    dt = np_dtype(variant, width)
    N = moduli_for(variant, width, rnd)[-1]
    ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
    n = (1 << 18) + 3
    a = operands(variant, N, n, rnd)
    b = operands(variant, N, n, rnd)
    want = np.array(a, dtype=object)
    B = np.array(b, dtype=object)
    for _ in range(8):
        want = bulk.mul_value_obj(variant, want, B, N, l, 1)
    db = dev(b, dt)
    bufs = [dev(a, dt), empty_like_elems(n, dt)]

    def chain():
        for i in range(8):
            mg.mont_mul(ctx, bufs[i % 2], db, bufs[(i + 1) % 2], n=n)

    chain()
    sync()
    assert host(bufs[0]) == [int(x) for x in want]
    bufs[0].copy_(dev(a, dt))
    bufs[1].zero_()
    sync()
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=side):
        chain()
    torch.cuda.current_stream().wait_stream(side)
    bufs[0].copy_(dev(a, dt))   # capture does not run the kernels; start again
    g.replay()
    sync()
    assert host(bufs[0]) == [int(x) for x in want]
