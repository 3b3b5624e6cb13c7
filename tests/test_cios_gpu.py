"""GPU parity of the multi-limb (CIOS) kernels against the oracle's
T R^{-1} mod N at R = 2^{32k}, for every limb count and every team size
(lanes per element), every mode, ragged sizes and the 2^22/2^21/2^17/2^15-pair
workloads of 256/384/1024/2048-bit moduli (sampled)."""

import random

import numpy as np
import pytest
import torch

import oracle as o
from oracle import bulk
import paper_2402_00675_gb300 as mg
import synthetic as sy
from gpu_helpers import sync

pytestmark = pytest.mark.gpu

TEAMS = {4: [1], 8: [1, 2], 12: [1, 4], 16: [1, 2, 4], 32: [2, 4, 8], 64: [4, 8, 16]}


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


@pytest.fixture(autouse=True)
def reset_shapes():
    yield
    for k in TEAMS:
        for mode in range(4):
            mg.mont_tune_set(32 * k, 0, mode, None)


def limbs_tensor(vals, k, pad=0):
    arr = np.zeros((len(vals) + pad, k), dtype=np.uint32)
    for i, v in enumerate(vals):
        arr[pad + i] = sy.limbs_of(v, k)
    t = torch.from_numpy(arr.reshape(-1)).cuda()
    return t[pad * k:]


def ints_of(t, k):
    arr = t.cpu().numpy().reshape(-1, k)
    return [sy.int_of_limbs(r) for r in arr]


def moduli(k, rnd):
    b = 32 * k
    return [rnd.randrange(1 << (b - 1), 1 << b) | 1,     # top bit set
            (1 << b) - 1,                                 # all ones
            (1 << (b - 1)) + 1,                           # smallest with top bit
            rnd.randrange(1 << (b - 45), 1 << (b - 40)) | 1]  # leading zero limbs


def set_team(k, team):
    for mode in range(4):
        mg.mont_tune_set(32 * k, 0, mode, {"threads": 256, "team": team})


@pytest.mark.parametrize("k", sorted(TEAMS))
def test_cios_mul_every_team(k):
    rnd = random.Random(k)
    for team in TEAMS[k]:
        set_team(k, team)
        for N in moduli(k, rnd):
            ctx = mg.mont_ctx_create(N, 32 * k, 0)
            n = 333
            a = [rnd.randrange(N) for _ in range(n)]
            b = [rnd.randrange(N) for _ in range(n)]
            a[:4] = [0, 1, N - 1, N - 1]
            b[:4] = [N - 1, N - 1, N - 1, 1]
            out = torch.zeros(n * k, dtype=torch.uint32, device="cuda")
            mg.mont_mul(ctx, limbs_tensor(a, k), limbs_tensor(b, k), out, n=n)
            sync()
            want = [o.mul_value(0, x, y, N, 32 * k) for x, y in zip(a, b)]
            assert ints_of(out, k) == want, (k, team, hex(N))


@pytest.mark.parametrize("k", sorted(TEAMS))
def test_cios_redc_and_domain_maps(k):
    rnd = random.Random(100 + k)
    R = 1 << (32 * k)
    for team in TEAMS[k]:
        set_team(k, team)
        N = moduli(k, rnd)[0]
        ctx = mg.mont_ctx_create(N, 32 * k, 0)
        n = 130
        # mont_redc on T in [0, RN)
        T = [rnd.randrange(R * N) for _ in range(n)]
        T[:3] = [0, R * N - 1, N * N]
        Tt = limbs_tensor(T, 2 * k)
        out = torch.zeros(n * k, dtype=torch.uint32, device="cuda")
        mg.mont_redc(ctx, Tt, out, n=n)
        sync()
        assert ints_of(out, k) == [o.redc_value(t, N, R) for t in T], (k, team)
        # to / from the Montgomery representation
        x = [rnd.randrange(N) for _ in range(n)]
        y = torch.zeros(n * k, dtype=torch.uint32, device="cuda")
        mg.mont_to_domain(ctx, limbs_tensor(x, k), y, n=n)
        back = torch.zeros(n * k, dtype=torch.uint32, device="cuda")
        mg.mont_from_domain(ctx, y, back, n=n)
        sync()
        assert ints_of(y, k) == [o.to_domain_value(0, v, N, 32 * k) for v in x]
        assert ints_of(back, k) == x


@pytest.mark.parametrize("k", [8, 32])
def test_cios_ragged_misaligned_in_place(k):
    rnd = random.Random(200 + k)
    N = moduli(k, rnd)[0]
    ctx = mg.mont_ctx_create(N, 32 * k, 0)
    for team in TEAMS[k]:
        set_team(k, team)
        for n in (1, 2, 3, 7, 31, 33, 257):
            for pad in (0, 1):
                a = [rnd.randrange(N) for _ in range(n)]
                b = [rnd.randrange(N) for _ in range(n)]
                want = [o.mul_value(0, x, y, N, 32 * k) for x, y in zip(a, b)]
                da, db = limbs_tensor(a, k, pad), limbs_tensor(b, k, pad)
                out = torch.zeros((n + pad) * k, dtype=torch.uint32, device="cuda")[pad * k:]
                mg.mont_mul(ctx, da, db, out, n=n)
                sync()
                assert ints_of(out, k) == want, (k, team, n, pad)
                mg.mont_mul(ctx, da, db, da, n=n)     # in place
                sync()
                assert ints_of(da, k) == want


@pytest.mark.parametrize("k", [8, 32, 64])
def test_cios_block_sizes_and_default_shape(k):
    """32-, 64-, 128- and 256-thread blocks and the untuned size-dependent
    default give the same products (several blocks and a ragged tail)."""
    rnd = random.Random(700 + k)
    N = moduli(k, rnd)[0]
    ctx = mg.mont_ctx_create(N, 32 * k, 0)
    n = 5 * 64 + 7
    a = [rnd.randrange(N) for _ in range(n)]
    b = [rnd.randrange(N) for _ in range(n)]
    want = [o.mul_value(0, x, y, N, 32 * k) for x, y in zip(a, b)]
    da, db = limbs_tensor(a, k), limbs_tensor(b, k)
    for team in TEAMS[k]:
        for threads in (32, 64, 128, 256):
            for mode in range(4):
                mg.mont_tune_set(32 * k, 0, mode, {"threads": threads, "team": team})
            out = torch.zeros(n * k, dtype=torch.uint32, device="cuda")
            mg.mont_mul(ctx, da, db, out, n=n)
            sync()
            assert ints_of(out, k) == want, (k, team, threads)
    for mode in range(4):
        mg.mont_tune_set(32 * k, 0, mode, None)
    assert mg.mont_tune_get(32 * k, 0, 0)["threads"] == 0
    out = torch.zeros(n * k, dtype=torch.uint32, device="cuda")
    mg.mont_mul(ctx, da, db, out, n=n)
    sync()
    assert ints_of(out, k) == want


@pytest.mark.parametrize("k", [32, 64])
def test_cios_grid_capped_by_blocks_per_sm(k):
    """A grid capped at 1, 2 or 3 blocks per SM walks the elements in more
    rounds per warp and gives the same products (every element checked)."""
    count = (1 << 16) // k * 8 + 5
    N = sy.random_odd_modulus(32 * k, seed=12)
    a = sy.uniform_limb_residues(N, k, count, seed=13)
    b = sy.uniform_limb_residues(N, k, count, seed=14)
    ctx = mg.mont_ctx_create(N, 32 * k, 0)
    want = bulk.mul_value_obj(0, bulk.ints_from_limbs(a, k), bulk.ints_from_limbs(b, k), N, 32 * k)
    da, db = torch.from_numpy(a.reshape(-1)).cuda(), torch.from_numpy(b.reshape(-1)).cuda()
    for team in TEAMS[k]:
        for bps in (1, 2, 3):
            mg.mont_tune_set(32 * k, 0, 0, {"threads": 128, "team": team, "blocks_per_sm": bps})
            out = torch.zeros(count * k, dtype=torch.uint32, device="cuda")
            mg.mont_mul(ctx, da, db, out, n=count)
            sync()
            bad = np.flatnonzero(bulk.ints_from_limbs(out.cpu().numpy(), k) != want)
            assert bad.size == 0, (k, team, bps, bad[:5])


@pytest.mark.parametrize("tuned", [False, True], ids=["default_shape", "autotuned"])
@pytest.mark.parametrize("bits,count", [(256, 1 << 22), (384, 1 << 21), (1024, 1 << 17),
                                        (2048, 1 << 15)])
def test_cios_full_size_workloads(bits, count, tuned):
    """The multi-limb benchmark sizes, at the built-in launch shape and at the
    shape the autotuner picks for that size (the one the benchmark times):
    every element against the definition T R^{-1} mod N (Python integers)."""
    k = bits // 32
    N = sy.random_odd_modulus(bits, seed=4)
    a = sy.uniform_limb_residues(N, k, count, seed=40 + k)
    b = sy.uniform_limb_residues(N, k, count, seed=80 + k)
    ctx = mg.mont_ctx_create(N, 32 * k, 0)
    if tuned:
        mg.mont_autotune(ctx, count)
        assert mg.mont_tune_get(bits, 0, 0)["team"] in TEAMS[k]
    out = torch.empty(count * k, dtype=torch.uint32, device="cuda")
    mg.mont_mul(ctx, torch.from_numpy(a.reshape(-1)).cuda(), torch.from_numpy(b.reshape(-1)).cuda(),
                out, n=count)
    sync()
    got = bulk.ints_from_limbs(out.cpu().numpy(), k)
    A, B = bulk.ints_from_limbs(a, k), bulk.ints_from_limbs(b, k)
    want = bulk.mul_value_obj(0, A, B, N, 32 * k)
    bad = np.flatnonzero(got != want)
    assert bad.size == 0, (bits, bad[:5])
    assert int(want[0]) == o.mul_value(0, sy.int_of_limbs(a[0]), sy.int_of_limbs(b[0]), N, 32 * k)


def test_autotune_and_persist(tmp_path):
    N = sy.random_odd_modulus(1024, seed=9)
    ctx = mg.mont_ctx_create(N, 1024, 0)
    mg.mont_autotune(ctx, 1 << 14)
    sh = mg.mont_tune_get(1024, 0, 0)
    assert sh["team"] in (0, 1, 2, 4, 8, 16)
    w = mg.mont_ctx_create(3329, 32, 1)
    mg.mont_autotune(w, 1 << 22, mg.MONT_TUNE_ELEMENTWISE | mg.MONT_TUNE_BATCHED)
    s32 = mg.mont_tune_get(32, 1, 0)
    sb = mg.mont_tune_get(32, 0, mg.MONT_TUNE_MODE_BATCHED)
    path = str(tmp_path / "tune.txt")
    mg.mont_tune_save(path)
    mg.mont_tune_set(32, 1, 0, None)
    mg.mont_tune_set(32, 0, mg.MONT_TUNE_MODE_BATCHED, None)
    mg.mont_tune_load(path)
    assert mg.mont_tune_get(32, 1, 0) == s32
    assert mg.mont_tune_get(32, 0, mg.MONT_TUNE_MODE_BATCHED) == sb
    # tuned shapes still give exact results
    a = torch.randint(-1664, 1665, (100_001,), dtype=torch.int32, device="cuda")
    b = torch.randint(-1664, 1665, (100_001,), dtype=torch.int32, device="cuda")
    out = torch.empty_like(a)
    mg.mont_mul(w, a, b, out)
    sync()
    aa, bb, oo = a.cpu().tolist(), b.cpu().tolist(), out.cpu().tolist()
    assert oo == [o.mul_value(1, x, y, 3329, 32) for x, y in zip(aa, bb)]
    mg.mont_tune_set(32, 1, 0, None)
    mg.mont_tune_set(32, 0, mg.MONT_TUNE_MODE_BATCHED, None)
    mg.mont_tune_set(1024, 0, 0, None)
