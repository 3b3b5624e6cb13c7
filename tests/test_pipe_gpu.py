"""GPU parity of the host-buffer pipeline (mont_pipe_*) against the oracle.

Results of operations on host vectors are compared bit for bit with the
oracle's definitions (Section 1 REDC, Algorithms 1-4) and with the
device-pointer entry points on the same inputs.  Small staging buffers force
many chunks, every slot reuse and a ragged last chunk; the cases cover every
operation code, word and multi-limb contexts, inputs shared by several
operations, mixed and empty lengths, back-to-back runs whose outputs feed the
next run with no synchronisation between them, pageable host memory and the
argument checks."""

import ctypes
import random

import numpy as np
import pytest
import torch

import oracle as o
import paper_2402_00675_gb300 as mg
import synthetic as sy
from gpu_helpers import input_range, log2R_of, np_dtype

pytestmark = pytest.mark.gpu

SMALL = 3 * (64 << 10)     # the smallest staging: slots of 64 KiB


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


def pinned(arr):
    return torch.from_numpy(np.ascontiguousarray(arr)).pin_memory()


def host_empty(n, dtype, pin=True):
    t = torch.from_numpy(np.zeros(n, dtype=dtype))
    return t.pin_memory() if pin else t


def ints(t):
    return [int(x) for x in t.numpy().tolist()]


def operands(variant, N, n, rnd):
    lo, hi = input_range(variant, N)
    xs = [rnd.randint(lo, hi) for _ in range(n)]
    xs[:3] = [lo, hi, 0]
    return xs


@pytest.mark.parametrize("width", [32, 64])
@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
def test_pipe_mul_parity(variant, width):
    rnd = random.Random(31 * variant + width)
    l = log2R_of(variant, width)
    N = {32: 8380417 if variant != 2 else 3329, 64: (1 << 61) - 1}[width]
    if not o.precondition_ok(variant, N, l, 1):
        N = 12289
    dt = np_dtype(variant, width)
    ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
    n = 20_011
    a, b = operands(variant, N, n, rnd), operands(variant, N, n, rnd)
    ha, hb = pinned(np.array(a, dtype=dt)), pinned(np.array(b, dtype=dt))
    out = host_empty(n, dt)
    pipe = mg.mont_pipe_create(SMALL)
    chunk, distinct = pipe.plan([(ctx, mg.MONT_OP_MUL, ha, hb, out)])
    assert distinct == 2 and chunk % mg.MONT_PIPE_MIN_CHUNK == 0 and n > 3 * chunk
    pipe.run([(ctx, mg.MONT_OP_MUL, ha, hb, out)])
    torch.cuda.synchronize()
    assert ints(out) == [o.mul_value(variant, x, y, N, l, 1) for x, y in zip(a, b)]
    pipe.close()


@pytest.mark.parametrize("width", [32, 64])
def test_pipe_redc_and_domain_maps(width):
    rnd = random.Random(7 + width)
    pipe = mg.mont_pipe_create(SMALL)
    for variant in (0, 1, 2, 3, 4):
        l = log2R_of(variant, width)
        N = 3329 if width == 32 else (1 << 59) + 27
        while not (o.precondition_ok(variant, N, l, 1) and N % 2):
            N -= 2
        dt = np_dtype(variant, width)
        ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
        n = 9_001
        lo, hi = o.input_domain(variant, N, l, 1)
        T = [rnd.randint(lo, hi) for _ in range(n)]
        T[:2] = [lo, hi]
        if width == 32:
            hT = pinned(np.array(T, dtype=np.int64 if lo < 0 else np.uint64))
        else:
            words = []
            for t in T:
                words += [t & (2**64 - 1), (t >> 64) & (2**64 - 1)]
            hT = pinned(np.array(words, dtype=np.uint64))
        x = [o.mods(v, N) if variant in (1, 3, 4) else v % N for v in operands(variant, N, n, rnd)]
        hx = pinned(np.array(x, dtype=dt))
        r, y, back = host_empty(n, dt), host_empty(n, dt), host_empty(n, dt)
        pipe.run([(ctx, mg.MONT_OP_REDC, hT, None, r),
                  (ctx, mg.MONT_OP_TO_DOMAIN, hx, None, y)])
        pipe.run([(ctx, mg.MONT_OP_FROM_DOMAIN, y, None, back)])   # y produced by the run before
        torch.cuda.synchronize()
        assert ints(r) == [o.reduce_value(variant, t, N, l, 1) for t in T], (variant, N)
        assert ints(y) == [o.to_domain_value(variant, v, N, l, 1) for v in x], (variant, N)
        assert ints(back) == x, (variant, N)
    pipe.close()


@pytest.mark.parametrize("k", [8, 32])
def test_pipe_multilimb(k):
    rnd = random.Random(k)
    N = rnd.randrange(1 << (32 * k - 1), 1 << (32 * k)) | 1
    ctx = mg.mont_ctx_create(N, 32 * k, 0, n_limbs=k)
    n = 1_500 if k == 8 else 700
    a = sy.uniform_limb_residues(N, k, n, seed=k)
    b = sy.uniform_limb_residues(N, k, n, seed=k + 1)
    T = [sy.int_of_limbs(x) * sy.int_of_limbs(y) for x, y in zip(a, b)]
    hT = pinned(np.stack([sy.limbs_of(t, 2 * k) for t in T]).reshape(-1))
    ha, hb = pinned(a.reshape(-1)), pinned(b.reshape(-1))
    prod = host_empty(n * k, np.uint32)
    red = host_empty(n * k, np.uint32)
    pipe = mg.mont_pipe_create({8: 512 << 10, 32: 1 << 20}[k])   # 2-7 chunks
    ops = [(ctx, mg.MONT_OP_MUL, ha, hb, prod, n), (ctx, mg.MONT_OP_REDC, hT, None, red, n)]
    chunk, distinct = pipe.plan(ops)
    assert chunk < n and distinct == 3
    pipe.run(ops)
    torch.cuda.synchronize()
    R = 1 << (32 * k)
    want = [t * pow(R, -1, N) % N for t in T]
    got = [sy.int_of_limbs(r) for r in prod.numpy().reshape(-1, k)]
    assert got == want
    got = [sy.int_of_limbs(r) for r in red.numpy().reshape(-1, k)]
    assert got == want
    pipe.close()


def test_pipe_shared_inputs_match_device_path():
    """Eight operations on two moduli sharing four inputs each, as in the
    Gmodmul/s workload (Algorithm 1 at R = 2^32, Algorithms 2-4 at R = 2^64),
    against the device-pointer products, and the oracle on a sample."""
    n = 3 * (1 << 20) + 12_345
    pipe = mg.mont_pipe_create(64 << 20)
    ops, expect = [], []
    for N, seed in ((3329, 2), (8380417, 3)):
        g = np.random.default_rng(seed)
        a = g.integers(-(N // 2), N // 2 + 1, n, dtype=np.int64).astype(np.int32)
        b = g.integers(-(N // 2), N // 2 + 1, n, dtype=np.int64).astype(np.int32)
        au = np.where(a < 0, a + N, a).astype(np.uint32)
        bu = np.where(b < 0, b + N, b).astype(np.uint32)
        ha, hb, hau, hbu = pinned(a), pinned(b), pinned(au), pinned(bu)
        for variant, l in ((1, 32), (2, 64), (3, 64), (4, 64)):
            ctx = mg.mont_ctx_create(N, l, variant, alpha=1)
            x, y = (hau, hbu) if variant == 2 else (ha, hb)
            dt = np.uint32 if variant == 2 else np.int32
            out = host_empty(n, dt)
            ops.append((ctx, mg.MONT_OP_MUL, x, y, out))
            d = torch.empty(n, dtype=torch.int32, device="cuda")
            mg.mont_mul(ctx, x.cuda(), y.cuda(), d)
            xs, ys = (au, bu) if variant == 2 else (a, b)
            expect.append((variant, N, l, xs, ys, d))
    chunk, distinct = pipe.plan(ops)
    assert distinct == 8 and chunk < n
    pipe.run(ops)
    torch.cuda.synchronize()
    idx = np.random.default_rng(9).integers(0, n, 200)
    for (ctx, _, x, y, out), (variant, N, l, xx, yy, d) in zip(ops, expect):
        assert torch.equal(out.view(torch.int32), d.cpu()), (variant, N)
        got = out.numpy()
        for i in idx:
            assert int(got[i]) == o.mul_value(variant, int(xx[i]), int(yy[i]), N, l, 1)
    pipe.close()


def test_pipe_mixed_and_empty_lengths():
    rnd = random.Random(5)
    N = 8380417
    ctx = mg.mont_ctx_create(N, 32, 0)
    pipe = mg.mont_pipe_create(SMALL)
    lengths = [0, 1, 255, 256, 257, 7_000, 23_456]
    ops, data = [], []
    for n in lengths:
        a = [rnd.randrange(N) for _ in range(n)]
        b = [rnd.randrange(N) for _ in range(n)]
        ha = pinned(np.array(a, dtype=np.uint32))
        hb = pinned(np.array(b, dtype=np.uint32))
        out = host_empty(max(n, 1), np.uint32)
        ops.append((ctx, mg.MONT_OP_MUL, ha, hb, out, n))
        data.append((a, b, out))
    pipe.run(ops)
    pipe.run([])                                      # count = 0: nothing
    pipe.run([(ctx, mg.MONT_OP_MUL, None, None, None, 0)])   # every op empty
    torch.cuda.synchronize()
    for (a, b, out), n in zip(data, lengths):
        assert ints(out)[:n] == [o.mul_value(0, x, y, N, 32) for x, y in zip(a, b)], n
    pipe.close()


def test_pipe_back_to_back_chained_runs():
    """Runs with different slot layouts follow one another without a
    synchronisation; each run's inputs are the previous run's outputs."""
    rnd = random.Random(11)
    N = 3329
    ctx = mg.mont_ctx_create(N, 32, 0)
    ctx64 = mg.mont_ctx_create((1 << 61) - 1, 64, 0)
    n = 50_000
    pipe = mg.mont_pipe_create(SMALL)
    x = [rnd.randrange(N) for _ in range(n)]
    c = [rnd.randrange(N) for _ in range(n)]
    hx = pinned(np.array(x, dtype=np.uint32))
    hc = pinned(np.array(c, dtype=np.uint32))
    w = [rnd.randrange((1 << 61) - 1) for _ in range(n)]
    hw = pinned(np.array(w, dtype=np.uint64))
    cur, want = hx, x
    R = 1 << 32
    outs = []
    for step in range(6):
        nxt = host_empty(n, np.uint32)
        ops = [(ctx, mg.MONT_OP_MUL, cur, hc, nxt)]
        if step % 2:   # a wider layout in odd runs
            w_out = host_empty(n, np.uint64)
            ops.append((ctx64, mg.MONT_OP_MUL, hw, hw, w_out))
            outs.append(w_out)
        pipe.run(ops)
        want = [v * y * pow(R, -1, N) % N for v, y in zip(want, c)]
        cur = nxt
    torch.cuda.synchronize()
    assert ints(cur) == want
    P = (1 << 61) - 1
    ww = [v * v * pow(1 << 64, -1, P) % P for v in w]
    for w_out in outs:
        assert ints(w_out) == ww
    pipe.close()


def test_pipe_pageable_memory():
    rnd = random.Random(13)
    N = 8380417
    ctx = mg.mont_ctx_create(N, 64, 3)
    n = 30_000
    a, b = operands(3, N, n, rnd), operands(3, N, n, rnd)
    ha = torch.from_numpy(np.array(a, dtype=np.int32))     # not pinned
    hb = torch.from_numpy(np.array(b, dtype=np.int32))
    out = host_empty(n, np.int32, pin=False)
    pipe = mg.mont_pipe_create(SMALL)
    pipe.run([(ctx, mg.MONT_OP_MUL, ha, hb, out)])
    torch.cuda.synchronize()
    assert ints(out) == [o.mul_value(3, x, y, N, 64, 1) for x, y in zip(a, b)]
    pipe.close()


def test_pipe_argument_checks():
    L = mg.lib()
    ctx = mg.mont_ctx_create(3329, 32, 0)
    pipe = mg.mont_pipe_create(SMALL)
    a = host_empty(1000, np.uint32)
    b = host_empty(1000, np.uint32)
    out = host_empty(1000, np.uint32)

    def st(ops, count=None):
        arr = mg.Pipe._ops(ops)
        return L.mont_pipe_run(pipe.handle, arr, len(ops) if count is None else count, None)

    assert st([(ctx, mg.MONT_OP_MUL, a, b, out)]) == mg.MONT_OK
    torch.cuda.synchronize()
    assert st([(ctx, mg.MONT_OP_MUL, a, b, a)]) == mg.MONT_EINVAL          # out is an input
    half = out[500:]
    assert st([(ctx, mg.MONT_OP_MUL, a, b, out), (ctx, mg.MONT_OP_MUL, a, b, half)]) == mg.MONT_EINVAL
    assert st([(ctx, 9, a, b, out)]) == mg.MONT_EINVAL                       # unknown op
    assert st([(ctx, mg.MONT_OP_MUL, a, None, out)]) == mg.MONT_EINVAL       # MUL without b
    assert st([(ctx, mg.MONT_OP_MUL, a, b, out)], count=mg.MONT_PIPE_MAX_OPS + 1) == mg.MONT_EINVAL
    assert st([(ctx, mg.MONT_OP_MUL, a, b, out)], count=-1) == mg.MONT_EINVAL
    assert L.mont_pipe_run(None, None, 0, None) == mg.MONT_EINVAL
    # one slot of 64 KiB cannot hold 256 elements of three 2048-bit vectors
    big = mg.mont_ctx_create((1 << 2047) + 1, 2048, 0, n_limbs=64)
    x = host_empty(64 * 300, np.uint32)
    y = host_empty(64 * 300, np.uint32)
    z = host_empty(64 * 300, np.uint32)
    assert st([(big, mg.MONT_OP_MUL, x, y, z)]) == mg.MONT_ENOMEM
    h = ctypes.c_void_p()
    assert L.mont_pipe_create(ctypes.byref(h), 1000) == mg.MONT_EINVAL
    assert L.mont_pipe_destroy(None) == mg.MONT_OK
    pipe.close()
