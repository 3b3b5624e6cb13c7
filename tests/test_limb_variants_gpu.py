"""GPU parity of Algorithms 1-4 at multi-limb widths against the oracle.

For k limbs the word size is n = 32k: Algorithm 1 reduces modulo
R = 2^{32k}, Algorithms 2-4 modulo R = 2^{64k}.  Every result is compared bit
for bit with the oracle's definition (the unique value in the variant's
output range; for Algorithm 1 the representative (T - mN)/R its choice of m
fixes).  Cases: every supported limb count; moduli at the variant's largest
admissible size, random ones and ones with leading zero limbs; products,
caller-supplied double-width T across the whole input domain, domain maps
and their round trip; operands at the ends of their ranges; alpha on both
sides of a limb boundary; in-place operation and misaligned buffers; the
benchmark's stated-size workloads, every element, at the built-in and the
autotuned launch shape."""

import random

import numpy as np
import pytest
import torch

import oracle as o
import paper_2402_00675_gb300 as mg
import synthetic as sy

pytestmark = pytest.mark.gpu

KS = [4, 8, 12, 16, 32, 64]
VARIANTS = [mg.MONT_SIGNED, mg.MONT_PLANTARD, mg.MONT_SIGNED_PLANTARD, mg.MONT_SIGNED_PLANTARD2]


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


def log2R_of(variant, k):
    return 64 * k if variant in mg.PLANTARD_VARIANTS else 32 * k


def largest_modulus(variant, k, alpha):
    n = 32 * k
    if variant == mg.MONT_PLANTARD:
        import math
        N = (math.isqrt(5 << (2 * n - 2)) - (1 << (n - 1))) | 1
        while o.plantard_bound_ok(N + 2, n):
            N += 2
        while not o.plantard_bound_ok(N, n):
            N -= 2
        return N
    if variant == mg.MONT_SIGNED_PLANTARD2:
        return (1 << (n - alpha - 1)) - 1
    return (1 << (n - 1)) - 1


def moduli(variant, k, alpha, rnd):
    top = largest_modulus(variant, k, alpha)
    return [top,
            rnd.randrange(top // 2, top) | 1,
            rnd.randrange(top >> 45, top >> 40) | 1]   # leading zero limbs


def input_range(variant, N):
    if variant == mg.MONT_PLANTARD:
        return 0, N - 1
    if variant == mg.MONT_SIGNED:
        return -(N - 1), N - 1
    return -((N - 1) // 2), (N - 1) // 2


def operands(variant, N, count, rnd):
    lo, hi = input_range(variant, N)
    xs = [rnd.randint(lo, hi) for _ in range(count)]
    xs[:6] = [lo, hi, 0, min(1, hi), max(-1, lo), hi - 1]
    return xs


def to_dev(vals, limbs, pad=0):
    """Two's complement limbs of each value; with pad > 0 the view starts
    pad limbs into a larger buffer (not 16-byte aligned for odd pad)."""
    arr = np.zeros(len(vals) * limbs + pad, dtype=np.uint32)
    for i, v in enumerate(vals):
        arr[pad + i * limbs: pad + (i + 1) * limbs] = sy.limbs_of(v % (1 << (32 * limbs)), limbs)
    return torch.from_numpy(arr).cuda()[pad:]


def from_dev(t, limbs, signed):
    arr = t.cpu().numpy().reshape(-1, limbs)
    out = []
    for row in arr:
        v = sy.int_of_limbs(row)
        if signed and v >> (32 * limbs - 1):
            v -= 1 << (32 * limbs)
        out.append(v)
    return out


def count_for(k):
    return {4: 3001, 8: 2003, 12: 1201, 16: 1001, 32: 401, 64: 203}[k]


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_mul_parity(variant, k):
    rnd = random.Random(100 * variant + k)
    alpha = 1
    l = log2R_of(variant, k)
    signed = variant != mg.MONT_PLANTARD
    for N in moduli(variant, k, alpha, rnd):
        ctx = mg.mont_ctx_create(N, l, variant, alpha=alpha, n_limbs=k)
        cnt = count_for(k)
        a, b = operands(variant, N, cnt, rnd), operands(variant, N, cnt, rnd)
        b[:6] = list(reversed(b[:6]))
        out = torch.zeros(cnt * k, dtype=torch.uint32, device="cuda")
        mg.mont_mul(ctx, to_dev(a, k), to_dev(b, k), out, n=cnt)
        torch.cuda.synchronize()
        want = [o.mul_value(variant, x, y, N, l, alpha) for x, y in zip(a, b)]
        assert from_dev(out, k, signed) == want, (variant, k, N)


@pytest.mark.parametrize("k", KS)
@pytest.mark.parametrize("variant", VARIANTS)
def test_redc_parity_whole_domain(variant, k):
    """Caller-supplied T spread over the whole input domain, ends included."""
    rnd = random.Random(200 * variant + k)
    alpha = 1
    l = log2R_of(variant, k)
    signed = variant != mg.MONT_PLANTARD
    for N in moduli(variant, k, alpha, rnd)[:2]:
        ctx = mg.mont_ctx_create(N, l, variant, alpha=alpha, n_limbs=k)
        lo, hi = o.input_domain(variant, N, l, alpha)
        cnt = count_for(k)
        T = [rnd.randint(lo, hi) for _ in range(cnt)]
        T[:4] = [lo, hi, 0, lo + 1]
        out = torch.zeros(cnt * k, dtype=torch.uint32, device="cuda")
        mg.mont_redc(ctx, to_dev(T, 2 * k), out, n=cnt)
        torch.cuda.synchronize()
        want = [o.reduce_value(variant, t, N, l, alpha) for t in T]
        assert from_dev(out, k, signed) == want, (variant, k, N)
        # the candidate formulas of the algorithms give the same values
        assert want[:50] == [o.candidate(variant, t, N, l, alpha) for t in T[:50]]


@pytest.mark.parametrize("k", [4, 8, 16, 64])
@pytest.mark.parametrize("variant", VARIANTS)
def test_domain_maps_round_trip(variant, k):
    rnd = random.Random(300 * variant + k)
    l = log2R_of(variant, k)
    signed = variant != mg.MONT_PLANTARD
    for N in moduli(variant, k, 1, rnd)[:2]:
        ctx = mg.mont_ctx_create(N, l, variant, alpha=1, n_limbs=k)
        cnt = count_for(k)
        x = [o.mods(v, N) if signed else v for v in operands(variant, N, cnt, rnd)]
        y = torch.zeros(cnt * k, dtype=torch.uint32, device="cuda")
        mg.mont_to_domain(ctx, to_dev(x, k), y, n=cnt)
        torch.cuda.synchronize()
        gy = from_dev(y, k, signed)
        assert gy == [o.to_domain_value(variant, v, N, l, 1) for v in x], (variant, k)
        back = torch.zeros_like(y)
        mg.mont_from_domain(ctx, y, back, n=cnt)
        torch.cuda.synchronize()
        assert from_dev(back, k, signed) == x, (variant, k)
        # from_domain of values outside the canonical range (Algorithm 1 outputs)
        z = [rnd.randint(*input_range(variant, N)) for _ in range(cnt)]
        zo = torch.zeros_like(y)
        mg.mont_from_domain(ctx, to_dev(z, k), zo, n=cnt)
        torch.cuda.synchronize()
        assert from_dev(zo, k, signed) == [o.from_domain_value(variant, v, N, l, 1) for v in z]


@pytest.mark.parametrize("alpha", [2, 31, 32, 33, 100])
def test_algorithm4_alpha_across_limbs(alpha):
    k = 8
    rnd = random.Random(alpha)
    l = 64 * k
    for N in moduli(mg.MONT_SIGNED_PLANTARD2, k, alpha, rnd):
        ctx = mg.mont_ctx_create(N, l, mg.MONT_SIGNED_PLANTARD2, alpha=alpha, n_limbs=k)
        lo, hi = o.input_domain(mg.MONT_SIGNED_PLANTARD2, N, l, alpha)
        cnt = 1500
        T = [rnd.randint(lo, hi) for _ in range(cnt)]
        T[:2] = [lo, hi]
        out = torch.zeros(cnt * k, dtype=torch.uint32, device="cuda")
        mg.mont_redc(ctx, to_dev(T, 2 * k), out, n=cnt)
        torch.cuda.synchronize()
        want = [o.reduce_value(mg.MONT_SIGNED_PLANTARD2, t, N, l, alpha) for t in T]
        assert from_dev(out, k, True) == want, (alpha, N)


@pytest.mark.parametrize("variant", VARIANTS)
def test_in_place_and_misaligned(variant):
    k = 8
    rnd = random.Random(400 + variant)
    l = log2R_of(variant, k)
    signed = variant != mg.MONT_PLANTARD
    N = moduli(variant, k, 1, rnd)[1]
    ctx = mg.mont_ctx_create(N, l, variant, alpha=1, n_limbs=k)
    cnt = 777
    a, b = operands(variant, N, cnt, rnd), operands(variant, N, cnt, rnd)
    want = [o.mul_value(variant, x, y, N, l, 1) for x, y in zip(a, b)]
    da = to_dev(a, k)
    mg.mont_mul(ctx, da, to_dev(b, k), da, n=cnt)            # out aliases a
    torch.cuda.synchronize()
    assert from_dev(da, k, signed) == want
    ma, mb = to_dev(a, k, pad=1), to_dev(b, k, pad=3)        # 4-byte aligned only
    mo = torch.zeros(cnt * k + 1, dtype=torch.uint32, device="cuda")[1:]
    mg.mont_mul(ctx, ma, mb, mo, n=cnt)
    torch.cuda.synchronize()
    assert from_dev(mo, k, signed) == want


def test_pipe_runs_multilimb_variants():
    """The host-buffer pipeline takes any ctx: 256-bit Algorithm 3 products."""
    k = 8
    rnd = random.Random(9)
    N = moduli(mg.MONT_SIGNED_PLANTARD, k, 1, rnd)[1]
    l = 64 * k
    ctx = mg.mont_ctx_create(N, l, mg.MONT_SIGNED_PLANTARD, n_limbs=k)
    cnt = 5000
    a, b = operands(3, N, cnt, rnd), operands(3, N, cnt, rnd)
    ha = to_dev(a, k).cpu().pin_memory()
    hb = to_dev(b, k).cpu().pin_memory()
    out = torch.zeros(cnt * k, dtype=torch.uint32).pin_memory()
    pipe = mg.mont_pipe_create(3 * (256 << 10))
    pipe.run([(ctx, mg.MONT_OP_MUL, ha, hb, out, cnt)])
    torch.cuda.synchronize()
    assert from_dev(out, k, True) == [o.mul_value(3, x, y, N, l) for x, y in zip(a, b)]
    pipe.close()


@pytest.mark.parametrize("k", [8, 32])
def test_launch_shapes_do_not_change_results(k):
    """Tuned launch shapes (threads, resident blocks per SM) change speed only."""
    rnd = random.Random(500 + k)
    variant = mg.MONT_SIGNED_PLANTARD2
    l = 64 * k
    N = moduli(variant, k, 1, rnd)[1]
    ctx = mg.mont_ctx_create(N, l, variant, alpha=1, n_limbs=k)
    cnt = 3000 if k == 8 else 700
    a, b = operands(variant, N, cnt, rnd), operands(variant, N, cnt, rnd)
    want = [o.mul_value(variant, x, y, N, l, 1) for x, y in zip(a, b)]
    da, db = to_dev(a, k), to_dev(b, k)
    try:
        for shape in ({"threads": 128, "blocks_per_sm": 1}, {"threads": 256, "blocks_per_sm": 0},
                      {"threads": 256, "blocks_per_sm": 3}, {"threads": 32, "blocks_per_sm": 0},
                      {"threads": 64, "blocks_per_sm": 2}, None):
            mg.mont_tune_set(32 * k, variant, 0, shape)
            out = torch.zeros(cnt * k, dtype=torch.uint32, device="cuda")
            mg.mont_mul(ctx, da, db, out, n=cnt)
            torch.cuda.synchronize()
            assert from_dev(out, k, True) == want, shape
    finally:
        mg.mont_tune_set(32 * k, variant, 0, None)


def test_autotune_picks_a_block_size_and_keeps_results():
    """mont_autotune on an Algorithm 2 context chooses a block size (the
    kernel runs one thread per element: no lane teams); products after tuning
    still equal the oracle's."""
    k, variant = 8, mg.MONT_PLANTARD
    rnd = random.Random(600)
    l = 64 * k
    N = moduli(variant, k, 1, rnd)[1]
    ctx = mg.mont_ctx_create(N, l, variant, n_limbs=k)
    try:
        mg.mont_autotune(ctx, 1 << 14)
        shape = mg.mont_tune_get(32 * k, variant, 0)
        assert shape["threads"] in (32, 64, 128, 256) and shape["team"] == 0
        cnt = 2000
        a, b = operands(variant, N, cnt, rnd), operands(variant, N, cnt, rnd)
        out = torch.zeros(cnt * k, dtype=torch.uint32, device="cuda")
        mg.mont_mul(ctx, to_dev(a, k), to_dev(b, k), out, n=cnt)
        torch.cuda.synchronize()
        assert from_dev(out, k, False) == [o.mul_value(variant, x, y, N, l) for x, y in zip(a, b)]
    finally:
        for mode in range(4):
            mg.mont_tune_set(32 * k, variant, mode, None)


@pytest.mark.parametrize("bits,count", [(256, 1 << 21), (1024, 1 << 17), (2048, 1 << 15)])
def test_full_size_workloads(bits, count):
    """The benchmark's Algorithm 1-4 workloads at their stated sizes (the same
    seeded moduli and operands), at the built-in launch shape and at the one
    the autotuner picks for that size: every element against the whole-array
    definition (Python integers)."""
    from oracle import bulk
    k = bits // 32
    for variant in VARIANTS:
        top_bits = {1: bits - 1, 2: bits - 1, 3: bits - 1, 4: bits - 2}[variant]
        N = sy.random_odd_modulus(top_bits, seed=4 + variant)
        l = log2R_of(variant, k)
        ctx = mg.mont_ctx_create(N, l, variant, alpha=1, n_limbs=k)
        a = sy.uniform_limb_residues(N, k, count, seed=40 + variant)
        b = sy.uniform_limb_residues(N, k, count, seed=80 + variant)
        signed = variant != mg.MONT_PLANTARD
        if signed:
            a, b = (sy.centred_limb_residues(N, x) for x in (a, b))
        da, db = torch.from_numpy(a.reshape(-1)).cuda(), torch.from_numpy(b.reshape(-1)).cuda()
        outs = []
        try:
            for tuned in (False, True):
                if tuned:
                    mg.mont_autotune(ctx, count)
                out = torch.empty(count * k, dtype=torch.uint32, device="cuda")
                mg.mont_mul(ctx, da, db, out, n=count)
                torch.cuda.synchronize()
                outs.append(out.cpu().numpy())
        finally:
            for mode in range(4):
                mg.mont_tune_set(32 * k, variant, mode, None)
        A, B = bulk.ints_from_limbs(a, k, signed), bulk.ints_from_limbs(b, k, signed)
        want = bulk.mul_value_obj(variant, A, B, N, l, 1)
        assert int(want[7]) == o.mul_value(variant, int(A[7]), int(B[7]), N, l, 1)
        for tuned, got in zip((False, True), outs):
            bad = np.flatnonzero(bulk.ints_from_limbs(got, k, signed) != want)
            assert bad.size == 0, (bits, variant, tuned, bad[:5])
