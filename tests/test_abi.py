"""The C-ABI library: it builds, loads, exports every declared symbol, and its
host-side precomputation (the per-modulus constants) matches the oracle.
No test here launches a kernel; all run without a GPU."""

import ctypes
import glob
import math
import os
import random
import re

import pytest

import oracle as o
import paper_2402_00675_gb300 as mg
from paper_2402_00675_gb300.build import build, INCLUDE

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build()
    return mg.lib()


def declared_functions():
    names = []
    for h in glob.glob(os.path.join(INCLUDE, "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        text = re.sub(r"//[^\n]*", "", text)
        names += re.findall(r"\b(mont_\w+)\s*\(", text)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(L):
    names = declared_functions()
    assert len(names) >= 12
    for name in names:
        assert hasattr(L, name), name


def test_version_and_strerror(L):
    assert mg.mont_version() >= 10000
    for s in range(0, 7):
        assert isinstance(mg.mont_strerror(s), str) and mg.mont_strerror(s)


def _const(ctx, which):
    return mg.mont_ctx_constant(ctx, which)


@pytest.mark.parametrize("variant", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("width", [32, 64])
def test_host_precompute_matches_oracle(L, variant, width):
    rnd = random.Random(100 * variant + width)
    log2R = width if variant < 2 else 2 * width
    n = width
    moduli = [3, 5, 3329, 8380417]
    while len(moduli) < 40:
        N = rnd.randrange(3, 1 << width) | 1
        moduli.append(N)
    for N in moduli:
        ok = o.precondition_ok(variant, N, log2R, 1)
        if not ok:
            with pytest.raises(mg.MontError) as ei:
                mg.mont_ctx_create(N, log2R, variant, alpha=1)
            assert ei.value.status == mg.MONT_EINVAL
            continue
        ctx = mg.mont_ctx_create(N, log2R, variant, alpha=1)
        c = o.constants(N, log2R)
        assert _const(ctx, mg.MONT_CONST_N) == N
        assert _const(ctx, mg.MONT_CONST_NINV) == c.Ninv
        assert _const(ctx, mg.MONT_CONST_NPRIME) == c.Nprime
        assert _const(ctx, mg.MONT_CONST_R_MOD_N) == c.R_mod_N
        assert _const(ctx, mg.MONT_CONST_R2_MOD_N) == c.R2_mod_N
        dr2 = _const(ctx, mg.MONT_CONST_DOMAIN_R2)
        if variant in (1, 3, 4):
            want = o.mods(c.R2_mod_N, N) % (1 << width)  # two's complement word
        else:
            want = c.R2_mod_N
        assert dr2 == want
        q = mg.mont_ctx_query(ctx)
        assert q["width_bits"] == width and q["log2R"] == log2R and q["variant"] == variant


@pytest.mark.parametrize("k", [4, 8, 12, 16, 32, 64])
def test_multilimb_precompute_matches_oracle(L, k):
    rnd = random.Random(k)
    for _ in range(5):
        N = rnd.randrange(1 << (32 * k - 1), 1 << (32 * k)) | 1
        ctx = mg.mont_ctx_create(N, 32 * k, 0)
        c = o.constants(N, 32 * k)
        assert _const(ctx, mg.MONT_CONST_NPRIME) == c.Nprime
        assert _const(ctx, mg.MONT_CONST_R2_MOD_N) == c.R2_mod_N
        assert _const(ctx, mg.MONT_CONST_R_MOD_N) == c.R_mod_N
    # Algorithms 1-4 at k limbs: N^{-1} mod R at R = 2^{32k} or 2^{64k}, domain constant
    for variant in (mg.MONT_SIGNED, mg.MONT_PLANTARD, mg.MONT_SIGNED_PLANTARD,
                    mg.MONT_SIGNED_PLANTARD2):
        log2R = 64 * k if variant in mg.PLANTARD_VARIANTS else 32 * k
        N = rnd.randrange(1 << (32 * k - 3), 1 << (32 * k - 2)) | 1
        ctx = mg.mont_ctx_create(N, log2R, variant, alpha=1, n_limbs=k)
        assert _const(ctx, mg.MONT_CONST_NINV) == pow(N, -1, 1 << log2R)
        r2 = pow(2, 2 * log2R, N)
        dom = _const(ctx, mg.MONT_CONST_DOMAIN_R2)
        if variant == mg.MONT_PLANTARD:
            assert dom == r2
        else:
            assert dom == o.mods(r2, N) % (1 << (32 * k))    # two's complement in k limbs
    # a modulus with leading zero limbs is accepted too
    N = (1 << 100) + 3
    ctx = mg.mont_ctx_create(N, 32 * 8, 0, n_limbs=8)
    assert _const(ctx, mg.MONT_CONST_R2_MOD_N) == o.constants(N, 256).R2_mod_N


def test_precondition_boundaries(L):
    # Plantard, n = 32: N < 2^32/phi = 2654435769.49...
    assert o.plantard_bound_ok(2654435769, 32) and not o.plantard_bound_ok(2654435771, 32)
    mg.mont_ctx_create(2654435769, 64, mg.MONT_PLANTARD)
    with pytest.raises(mg.MontError):
        mg.mont_ctx_create(2654435771, 64, mg.MONT_PLANTARD)
    # Algorithm 1: 2N < R
    mg.mont_ctx_create((1 << 31) - 1, 32, mg.MONT_SIGNED)
    with pytest.raises(mg.MontError):
        mg.mont_ctx_create((1 << 31) + 1, 32, mg.MONT_SIGNED)
    # Algorithm 3: N < 2^{n-1}
    mg.mont_ctx_create((1 << 31) - 1, 64, mg.MONT_SIGNED_PLANTARD)
    with pytest.raises(mg.MontError):
        mg.mont_ctx_create((1 << 31) + 1, 64, mg.MONT_SIGNED_PLANTARD)
    # Algorithm 4: alpha >= 1 and N < 2^{n-alpha-1}
    with pytest.raises(mg.MontError):
        mg.mont_ctx_create(3329, 64, mg.MONT_SIGNED_PLANTARD2, alpha=0)
    mg.mont_ctx_create((1 << 30) - 1, 64, mg.MONT_SIGNED_PLANTARD2, alpha=1)
    with pytest.raises(mg.MontError):
        mg.mont_ctx_create((1 << 30) + 1, 64, mg.MONT_SIGNED_PLANTARD2, alpha=1)
    # even and tiny moduli, wrong log2R, Plantard on multi-limb
    for bad in ((3328, 32, 0), (1, 32, 0), (3329, 32, 2)):
        with pytest.raises(mg.MontError):
            mg.mont_ctx_create(*bad)
    with pytest.raises(mg.MontError):
        mg.mont_ctx_create(3329, 64, 0, n_limbs=1)          # log2R must be 32 n_limbs
    # multi-limb moduli: each variant's condition on N at n = 32k (here n = 256)
    # 2^n / phi = 2^{n-1} (sqrt(5) - 1): start from the integer square root
    top = (math.isqrt(5 << 510) - (1 << 255)) | 1
    while o.plantard_bound_ok(top + 2, 256):
        top += 2
    while not o.plantard_bound_ok(top, 256):
        top -= 2
    mg.mont_ctx_create(top, 512, mg.MONT_PLANTARD, n_limbs=8)
    with pytest.raises(mg.MontError):
        mg.mont_ctx_create(top + 2, 512, mg.MONT_PLANTARD, n_limbs=8)
    for variant, log2R, bound in ((mg.MONT_SIGNED, 256, 1 << 255),
                                  (mg.MONT_SIGNED_PLANTARD, 512, 1 << 255),
                                  (mg.MONT_SIGNED_PLANTARD2, 512, 1 << 254)):
        mg.mont_ctx_create(bound - 1, log2R, variant, alpha=1, n_limbs=8)
        with pytest.raises(mg.MontError):
            mg.mont_ctx_create(bound + 1, log2R, variant, alpha=1, n_limbs=8)
    # REDC accepts N up to R - 1
    mg.mont_ctx_create((1 << 32) - 1, 32, 0)
    mg.mont_ctx_create((1 << 64) - 59, 64, 0)


def test_argument_errors_need_no_gpu(L):
    ctx = mg.mont_ctx_create(3329, 32, 0)
    # n = 0 is a no-op; NULL ctx and NULL pointers are refused before any launch
    assert L.mont_mul(ctx.handle, None, None, None, 0, None) == mg.MONT_OK
    assert L.mont_mul(None, 16, 16, 16, 4, None) == mg.MONT_EINVAL
    assert L.mont_mul(ctx.handle, None, 16, 16, 4, None) == mg.MONT_EINVAL
    # misaligned element pointers and partial overlap
    assert L.mont_mul(ctx.handle, 4096 + 1, 8192, 12288, 4, None) == mg.MONT_EINVAL
    assert L.mont_mul(ctx.handle, 4096, 8192, 4096 + 4, 4, None) == mg.MONT_EINVAL
    assert L.mont_redc(ctx.handle, 4096 + 4, 8192, 4, None) == mg.MONT_EINVAL
    buf = (ctypes.c_uint32 * 1)()
    n = ctypes.c_int()
    assert L.mont_ctx_constant(ctx.handle, mg.MONT_CONST_R2_MOD_N, buf, 0, ctypes.byref(n)) == \
        mg.MONT_EOVERFLOW
    assert L.mont_ctx_constant(ctx.handle, 99, buf, 1, ctypes.byref(n)) == mg.MONT_EINVAL
    assert L.mont_ctx_destroy(None) == mg.MONT_OK


def test_product_path_has_no_fallback(monkeypatch, tmp_path):
    """With the library missing the binding raises instead of computing."""
    import gc
    # Finalizers of earlier tests' contexts call lib(); run them now, and point
    # the path at the missing file before dropping the loaded handle, so that
    # none can reload the real library in between.
    gc.collect()
    monkeypatch.setattr(mg, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mg, "_lib", None)
    with pytest.raises(RuntimeError):
        mg.lib()


def test_sweep_argument_checks_need_no_gpu(L):
    import ctypes as C
    counts = (C.c_uint64 * 4096)()
    total = C.c_size_t()
    bad = [(0, 17, 0, 3, 31), (2, 15, 0, 3, 31), (0, 16, 0, 40, 30), (0, 16, 0, 3, 40000),
           (7, 16, 0, 3, 31), (4, 16, 15, 3, 31)]
    for v, l, a, lo, hi in bad:
        assert L.mont_verify_sweep(v, l, a, lo, hi, None, 0, counts, None, None, 0,
                                   C.byref(total), None) == mg.MONT_EINVAL
    # every N out of spec and skipped: nothing to launch, all counts zero
    assert L.mont_verify_sweep(2, 8, 0, 21, 31, None, 0, counts, None, None, 0,
                               C.byref(total), None) == mg.MONT_OK
    assert total.value == 0 and all(counts[i] == 0 for i in range(6))
    # an explicit domain outside 32-bit T is refused
    b = mg.MontBounds(mg.MONT_DOMAIN_EXPLICIT, mg.MONT_RANGE_DEFAULT, 0, 1 << 40, 0, 0)
    assert L.mont_verify_sweep(0, 16, 0, 3, 31, C.byref(b), 0, counts, None, None, 0,
                               C.byref(total), None) == mg.MONT_EINVAL


def test_tune_table_set_get_without_gpu(L):
    mg.mont_tune_set(32, 1, 0, {"threads": 128, "unroll": 4, "vec_bytes": 16})
    got = mg.mont_tune_get(32, 1, 0)
    assert (got["threads"], got["unroll"], got["vec_bytes"]) == (128, 4, 16)
    with pytest.raises(mg.MontError):
        mg.mont_tune_set(32, 1, 0, {"threads": 100, "unroll": 2, "vec_bytes": 32})
    with pytest.raises(mg.MontError):
        mg.mont_tune_set(32, 1, 7, {"threads": 128})
    mg.mont_tune_set(32, 1, 0, None)
    assert mg.mont_tune_get(32, 1, 0)["threads"] == 256
    # multi-limb widths: 32- to 256-thread blocks, blocks per SM >= 0
    mg.mont_tune_set(1024, 0, 0, {"threads": 32, "team": 4, "blocks_per_sm": 3})
    got = mg.mont_tune_get(1024, 0, 0)
    assert (got["threads"], got["team"], got["blocks_per_sm"]) == (32, 4, 3)
    for bad in ({"threads": 512}, {"threads": 128, "blocks_per_sm": -1}):
        with pytest.raises(mg.MontError):
            mg.mont_tune_set(1024, 0, 0, bad)
    mg.mont_tune_set(1024, 0, 0, None)
    assert mg.mont_tune_get(1024, 0, 0)["threads"] == 0


def test_server_and_device_calls_fail_cleanly_without_gpu(L):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    st = L.mont_server_create(ctypes.byref(h), 1 << 20, 2, 0)
    assert st in (mg.MONT_ECUDA, mg.MONT_ENOMEM)
    assert L.mont_server_create(ctypes.byref(h), 1 << 20, 0, 0) == mg.MONT_EINVAL
    assert L.mont_server_destroy(None) == mg.MONT_OK
    assert L.mont_pipe_create(ctypes.byref(h), 1 << 20) in (mg.MONT_ECUDA, mg.MONT_ENOMEM)
    assert L.mont_pipe_create(ctypes.byref(h), 1000) == mg.MONT_EINVAL
    assert L.mont_pipe_create(None, 1 << 20) == mg.MONT_EINVAL
    assert L.mont_pipe_run(None, None, 0, None) == mg.MONT_EINVAL
    assert L.mont_pipe_plan(None, None, 0, None, None) == mg.MONT_EINVAL
    assert L.mont_pipe_destroy(None) == mg.MONT_OK
