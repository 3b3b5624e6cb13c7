"""The serving loop on the GPU: results in a concurrent mix equal the results
of the same jobs alone and the oracle; admission by device memory; refusal of
oversized jobs; bounded waits."""

import random
import time

import numpy as np
import pytest
import torch

import oracle as o
import paper_2402_00675_gb300 as mg
import synthetic as sy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


def make_ctxs():
    N64 = sy.rns_primes(1, seed=31)[0]
    N256 = sy.random_odd_modulus(256, seed=32)
    return {
        (0, 32): (3329, mg.mont_ctx_create(3329, 32, 0)),
        (1, 32): (3329, mg.mont_ctx_create(3329, 32, 1)),
        (2, 32): (3329, mg.mont_ctx_create(3329, 64, 2)),
        (0, 64): (N64, mg.mont_ctx_create(N64, 64, 0)),
        (1, 64): (N64, mg.mont_ctx_create(N64, 64, 1)),
        (2, 64): (N64, mg.mont_ctx_create(N64, 128, 2)),
        (0, 256): (N256, mg.mont_ctx_create(N256, 256, 0)),
    }


def host_operands(variant, width, N, n, rnd):
    if width == 256:
        vals = [rnd.randrange(N) for _ in range(n)]
        arr = np.zeros((n, 8), dtype=np.uint32)
        for i, v in enumerate(vals):
            arr[i] = sy.limbs_of(v, 8)
        return vals, torch.from_numpy(arr.reshape(-1)).pin_memory()
    if variant == 1:
        lo, hi = -((N - 1) // 2), (N - 1) // 2
        vals = [rnd.randint(lo, hi) for _ in range(n)]
        dt = np.int32 if width == 32 else np.int64
        return vals, torch.from_numpy(np.array(vals, dtype=np.int64).astype(dt)).pin_memory()
    vals = [rnd.randrange(N) for _ in range(n)]
    dt = np.uint32 if width == 32 else np.uint64
    return vals, torch.from_numpy(np.array(vals, dtype=np.uint64).astype(dt)).pin_memory()


def values_of(t, width, n):
    if width == 256:
        arr = t.numpy().reshape(n, 8)
        return [sy.int_of_limbs(r) for r in arr]
    return [int(x) for x in t.numpy().tolist()]


def build_jobs(ctxs, count, seed, len_hi=14):
    rnd = random.Random(seed)
    keys = sorted(ctxs)
    jobs = []
    for i in range(count):
        variant, width = keys[rnd.randrange(len(keys))]
        N, ctx = ctxs[(variant, width)]
        n = int(2 ** rnd.uniform(4, len_hi))
        a_vals, a = host_operands(variant, width, N, n, rnd)
        b_vals, b = host_operands(variant, width, N, n, rnd)
        out = torch.zeros_like(a).pin_memory()
        log2R = width * 2 if variant == 2 else width
        jobs.append(dict(variant=variant, width=width, N=N, ctx=ctx, n=n, a=a, b=b, out=out,
                         a_vals=a_vals, b_vals=b_vals, log2R=log2R))
    return jobs


def test_mix_equals_alone_and_oracle():
    ctxs = make_ctxs()
    jobs = build_jobs(ctxs, 60, seed=5)
    sweeps = [(o.SIGNED_PLANTARD2, 12, 0, 3, 31), (o.REDC, 12, 0, 101, 163)]
    srv = mg.Server(64 << 20, slots=4)
    ids = []
    for k, j in enumerate(jobs):
        ids.append(srv.submit_modmul(j["ctx"], j["a"], j["b"], j["out"], n=j["n"]))
        if k in (10, 40):
            s = sweeps[k // 40]
            ids.append(srv.submit_sweep(*s, cex_cap=4096))
    results = [srv.wait(i, timeout_ms=120000) for i in ids]
    assert all(r["status"] == 0 for r in results)
    assert all(r["t_submit"] <= r["t_admit"] <= r["t_done"] for r in results)
    sweep_results = [r["sweep"] for r in results if "sweep" in r]
    srv.close()
    # alone: each job through mont_mul on the device, one at a time
    for j in jobs:
        da, db = j["a"].cuda(), j["b"].cuda()
        alone = torch.empty_like(da)
        mg.mont_mul(j["ctx"], da, db, alone, n=j["n"])
        torch.cuda.synchronize()
        assert torch.equal(alone.cpu(), j["out"]), (j["variant"], j["width"], j["n"])
        got = values_of(j["out"], j["width"], j["n"])
        want = [o.mul_value(j["variant"], x, y, j["N"], j["log2R"]) for x, y in
                zip(j["a_vals"], j["b_vals"])]
        assert got == want
    for s, r in zip(sweeps, sweep_results):
        want = o.sweep(*s)
        alone = mg.mont_verify_sweep(*s, cex_cap=4096)
        assert r.counts == alone.counts and r.examples == alone.examples
        assert r.total == want.total and r.examples == want.examples


def test_admission_by_memory_serialises_when_budget_is_tight():
    ctxs = make_ctxs()
    jobs = [j for j in build_jobs(ctxs, 40, seed=6, len_hi=12) if j["width"] == 64][:12]
    biggest = max(3 * j["n"] * 8 for j in jobs)
    srv = mg.Server(biggest + 4096, slots=4)     # room for about one job at a time
    ids = [srv.submit_modmul(j["ctx"], j["a"], j["b"], j["out"], n=j["n"]) for j in jobs]
    results = [srv.wait(i, timeout_ms=60000) for i in ids]
    srv.close()
    assert all(r["status"] == 0 for r in results)
    for j in jobs:
        want = [o.mul_value(j["variant"], x, y, j["N"], j["log2R"]) for x, y in
                zip(j["a_vals"], j["b_vals"])]
        assert values_of(j["out"], 64, j["n"]) == want


def test_oversized_job_refused_and_bounded_waits():
    ctxs = make_ctxs()
    N, ctx = ctxs[(0, 32)]
    srv = mg.Server(1 << 20, slots=2)
    big = torch.zeros(1 << 20, dtype=torch.uint32)
    with pytest.raises(mg.MontError) as ei:
        srv.submit_modmul(ctx, big, big, big)
    assert ei.value.status == mg.MONT_ENOMEM
    with pytest.raises(mg.MontError):
        srv.wait(12345, 0)                       # unknown id
    small = torch.ones(1000, dtype=torch.uint32).pin_memory()
    out = torch.zeros(1000, dtype=torch.uint32).pin_memory()
    jid = srv.submit_modmul(ctx, small, small, out)
    r = srv.wait(jid, 30000)
    assert r["status"] == 0
    assert out.tolist() == [o.mul_value(0, 1, 1, 3329, 32)] * 1000
    srv.close()


def test_job_timeout_reports_and_server_recovers():
    """A job that runs longer than its timeout completes with MONT_ETIMEOUT
    (no GPU fault is involved: the host stops waiting, and stops issuing the
    job's remaining pieces).  Its buffers stay busy until the device work
    already issued ends; then a prefix of whole pieces holds correct products,
    the arena region is given back and the server keeps serving."""
    N = sy.random_odd_modulus(2048, seed=8)
    ctx = mg.mont_ctx_create(N, 2048, 0)
    n = 1 << 21          # 512 MiB per operand: copies and compute of well over 1 ms
    one = np.zeros((n, 64), dtype=np.uint32)
    one[:, 0] = 1
    a = torch.from_numpy(one.reshape(-1)).pin_memory()
    out = torch.zeros_like(a).pin_memory()
    budget = 3 * n * 64 * 4 + (1 << 20)
    srv = mg.Server(budget, slots=1, job_timeout_ms=1)
    jid = srv.submit_modmul(ctx, a, a, out, n=n)
    r = srv.wait(jid, 60000)
    assert r["status"] == mg.MONT_ETIMEOUT
    assert srv.job_busy(jid)                   # the copies and the kernel still run
    for _ in range(30000):
        if not srv.job_busy(jid):
            break
        time.sleep(0.001)
    assert not srv.job_busy(jid)
    assert srv.query()["arena_free"] >= 3 * n * 64 * 4   # the region came back
    want = np.array(sy.limbs_of(o.mul_value(0, 1, 1, N, 2048), 64), dtype=np.uint32)
    rows = out.numpy().reshape(n, 64)
    done = (rows == want).all(axis=1)
    untouched = (rows == 0).all(axis=1)
    assert (done | untouched).all()
    k = int(np.argmin(done)) if not done.all() else n          # written prefix
    assert k > 0 and done[:k].all() and untouched[k:].all()
    piece = (16 << 20) // (64 * 4)
    assert k % piece == 0 or k == n
    # the same server runs the next job (with a timeout of its own)
    small = torch.from_numpy(one[:8].reshape(-1).copy()).pin_memory()
    o2 = torch.zeros_like(small).pin_memory()
    jid = srv.submit_modmul(ctx, small, small, o2, n=8, timeout_ms=30000)
    assert srv.wait(jid, 30000)["status"] == 0
    assert (o2.numpy().reshape(8, 64) == want).all()
    assert srv.close() == mg.MONT_OK


def test_straggler_region_is_reused_not_stalled():
    """A timed-out job holds its arena region only while its device work runs:
    a later job larger than every free piece waits for that region and then
    runs, instead of stalling the queue."""
    N = sy.random_odd_modulus(2048, seed=9)
    ctx = mg.mont_ctx_create(N, 2048, 0)
    unit = 1 << 19                                 # elements per job unit
    nb = unit * 64 * 4                             # bytes per operand of one unit
    srv = mg.Server(3 * (3 * nb) + 4096, slots=2)  # room for three units
    one = np.zeros((2 * unit, 64), dtype=np.uint32)
    one[:, 0] = 1
    a = torch.from_numpy(one.reshape(-1)).pin_memory()
    outs = [torch.zeros(2 * unit * 64, dtype=torch.uint32).pin_memory() for _ in range(3)]
    x = srv.submit_modmul(ctx, a, a, outs[0], n=unit)
    y = srv.submit_modmul(ctx, a, a, outs[1], n=unit, timeout_ms=1)
    z = srv.submit_modmul(ctx, a, a, outs[2], n=2 * unit)
    rx, ry, rz = srv.wait(x, 60000), srv.wait(y, 60000), srv.wait(z, 60000)
    assert rx["status"] == 0 and rz["status"] == 0
    assert ry["status"] in (0, mg.MONT_ETIMEOUT)
    want = np.array(sy.limbs_of(o.mul_value(0, 1, 1, N, 2048), 64), dtype=np.uint32)
    assert (outs[2].numpy().reshape(2 * unit, 64) == want).all()
    assert srv.close() == mg.MONT_OK


def test_sweep_jobs_bounded_and_scratch_from_arena():
    """A sweep job's scratch counts against the arena (refused when larger
    than the budget); a sweep past its timeout completes with MONT_ETIMEOUT
    between its launches and its region comes back; an untimed sweep in the
    same server equals mont_verify_sweep."""
    tiny = mg.Server(4096, slots=1)
    with pytest.raises(mg.MontError) as ei:
        tiny.submit_sweep(o.REDC, 16, 0, 3, 4095, cex_cap=16)
    assert ei.value.status == mg.MONT_ENOMEM
    tiny.close()
    srv = mg.Server(64 << 20, slots=2)
    slow = srv.submit_sweep(o.REDC, 16, 0, 3073, 4095, cex_cap=16, timeout_ms=1)
    r = srv.wait(slow, 60000)
    assert r["status"] == mg.MONT_ETIMEOUT and "sweep" not in r
    for _ in range(30000):
        if not srv.job_busy(slow):
            break
        time.sleep(0.001)
    assert not srv.job_busy(slow)
    ok = srv.submit_sweep(o.SIGNED_PLANTARD2, 12, 0, 3, 63, cex_cap=4096)
    got = srv.wait(ok, 60000)
    assert got["status"] == 0
    alone = mg.mont_verify_sweep(o.SIGNED_PLANTARD2, 12, 0, 3, 63, cex_cap=4096)
    assert got["sweep"].counts == alone.counts and got["sweep"].examples == alone.examples
    assert srv.query()["arena_free"] == 64 << 20      # every region came back
    assert srv.close() == mg.MONT_OK
