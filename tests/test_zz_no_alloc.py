"""The allocation-free sweep entry point (mont_verify_sweep_noalloc).

Callers that must not allocate -- a fixed device-memory budget, a device
owned by another allocator, a loop that cannot take cudaMalloc's implicit
synchronisation -- use this entry point; it keeps its device scratch in one
fixed array inside the library.  Its results must equal those of
mont_verify_sweep, call after call: the shared array keeps the previous
call's contents, so each test makes at least two calls in a row, on
different workloads, and compares both with the allocating entry point.

This file is named to be collected last, so that a run stopping at the
first failure has already run every other test.
"""

import ctypes

import pytest
import torch

import paper_2402_00675_gb300 as mg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


def same(a, b):
    assert a.moduli == b.moduli
    assert a.counts == b.counts
    assert a.checked == b.checked
    assert a.total == b.total
    assert a.overflow == b.overflow
    if not a.overflow:
        assert a.examples == b.examples
    else:
        assert len(a.examples) == len(b.examples) and a.examples == sorted(a.examples)


CASES = [
    # (variant, log2R, alpha, N_lo, N_hi, bounds, flags, cap)
    (mg.MONT_SIGNED_PLANTARD2, 12, 0, 3, 31, None, 0, 4096),          # Example 3.1's sweep
    (mg.MONT_SIGNED_PLANTARD2, 16, 1, 3, 127, None, 0, 4096),          # no counterexample
    (mg.MONT_PLANTARD, 16, 0, 141, 171, None, mg.MONT_SWEEP_INCLUDE_OUT_OF_SPEC, 4096),
    (mg.MONT_SIGNED_PLANTARD2, 16, 0, 3, 127, None, 0, 100),           # overflowing cap
    (mg.MONT_REDC, 16, 0, 3, 4095, None, 0, 16),                       # the full R = 2^16 range
    (mg.MONT_SIGNED, 10, 0, 3, 255,
     mg.MontBounds(mg.MONT_DOMAIN_REDC, mg.MONT_RANGE_DEFAULT, 0, 0, 0, 0), 0, 4096),
]


def test_noalloc_matches_allocating_entry_on_consecutive_calls():
    for rep in range(2):
        for v, l, a, lo, hi, b, f, cap in CASES:
            want = mg.mont_verify_sweep(v, l, a, lo, hi, b, f, cex_cap=cap)
            got = mg.mont_verify_sweep_noalloc(v, l, a, lo, hi, b, f, cex_cap=cap)
            same(got, want)
            again = mg.mont_verify_sweep_noalloc(v, l, a, lo, hi, b, f, cex_cap=cap)
            same(again, want)


def test_noalloc_rejects_requests_beyond_its_fixed_scratch():
    L = mg.lib()
    counts = (ctypes.c_uint64 * 16384)()
    total = ctypes.c_size_t()
    cex = (mg.MontCex * (mg.MONT_SWEEP_NOALLOC_MAX_CEX + 1))()
    # more odd moduli than the table holds
    st = L.mont_verify_sweep_noalloc(0, 16, 0, 3, 3 + 2 * mg.MONT_SWEEP_NOALLOC_MAX_MODULI, None,
                                     0, counts, None, None, 0, ctypes.byref(total), None)
    assert st == mg.MONT_EINVAL
    # a larger example buffer than the scratch holds
    st = L.mont_verify_sweep_noalloc(0, 12, 0, 3, 31, None, 0, counts, None, cex,
                                     mg.MONT_SWEEP_NOALLOC_MAX_CEX + 1, ctypes.byref(total), None)
    assert st == mg.MONT_EINVAL
    # the largest admitted request still works and matches
    hi = 3 + 2 * (mg.MONT_SWEEP_NOALLOC_MAX_MODULI - 1)
    got = mg.mont_verify_sweep_noalloc(mg.MONT_SIGNED_PLANTARD2, 16, 1, 3, hi,
                                       cex_cap=mg.MONT_SWEEP_NOALLOC_MAX_CEX)
    want = mg.mont_verify_sweep(mg.MONT_SIGNED_PLANTARD2, 16, 1, 3, hi,
                                cex_cap=mg.MONT_SWEEP_NOALLOC_MAX_CEX)
    same(got, want)
