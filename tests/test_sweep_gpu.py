"""GPU verify sweep against the oracle's exhaustive sweep.

Counts per modulus and the sorted counterexample lists must agree exactly.
The full-size run (R = 2^16, every odd N in [3, 4095]) is checked by the
theorems (no counterexample for any in-spec algorithm; the number of T
checked per N equals the domain size) and against the oracle on sampled N."""

import pytest
import torch

import oracle as o
from oracle import exhaustive as ex
import paper_2402_00675_gb300 as mg
from conftest import read_golden

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    mg.build()
    assert torch.cuda.is_available()


def oracle_rules(bounds):
    if bounds is None:
        return ex.DOMAIN_DEFAULT, ex.RANGE_DEFAULT
    dom = {mg.MONT_DOMAIN_DEFAULT: ex.DOMAIN_DEFAULT, mg.MONT_DOMAIN_REDC: ex.DOMAIN_REDC}.get(
        bounds.domain_rule, (bounds.t_lo, bounds.t_hi))
    rng = {mg.MONT_RANGE_DEFAULT: ex.RANGE_DEFAULT, mg.MONT_RANGE_UNSIGNED: ex.RANGE_UNSIGNED,
           mg.MONT_RANGE_WIDE: ex.RANGE_WIDE, mg.MONT_RANGE_CENTRED: ex.RANGE_CENTRED}.get(
        bounds.range_rule, (bounds.r_lo, bounds.r_hi))
    return dom, rng


def compare(variant, log2R, alpha, lo, hi, bounds=None, flags=0, vectorised=False, cap=1 << 17):
    got = mg.mont_verify_sweep(variant, log2R, alpha, lo, hi, bounds, flags, cex_cap=cap)
    dom, rng = oracle_rules(bounds)
    want = o.sweep(variant, log2R, alpha, lo, hi, domain=dom, claimed=rng,
                   include_out_of_spec=bool(flags & mg.MONT_SWEEP_INCLUDE_OUT_OF_SPEC),
                   vectorised=vectorised)
    for N in got.moduli:
        assert got.counts[N] == want.counts.get(N, 0), (variant, log2R, alpha, N)
        assert got.checked[N] == want.checked.get(N, 0), (variant, N)
    assert got.total == want.total
    if want.total <= cap:
        assert not got.overflow
        assert got.examples == want.examples
    else:   # the counts stay exact; the examples are cap of them, sorted
        assert got.overflow and len(got.examples) == cap
        assert got.examples == sorted(got.examples) and set(got.examples) <= set(want.examples)
    return got


def test_example_3_1_on_gpu():
    g = read_golden("example_3_1.txt")
    got = compare(mg.MONT_SIGNED_PLANTARD2, 2 * g["n"], g["alpha"], g["N"], g["N"])
    assert (g["N"], g["T"], g["algorithm_output"], g["correct"]) in got.examples


@pytest.mark.parametrize("variant,alpha", [(0, 0), (1, 0), (2, 0), (3, 0), (4, 0), (4, 1), (4, 2)])
@pytest.mark.parametrize("log2R", [8, 12])
def test_small_sweeps_match_oracle(variant, alpha, log2R):
    hi = 63 if log2R == 8 else 95
    compare(variant, log2R, alpha, 3, hi)
    compare(variant, log2R, alpha, 3, hi, flags=mg.MONT_SWEEP_INCLUDE_OUT_OF_SPEC)
    compare(variant, log2R, alpha, 3, 41,
            bounds=mg.MontBounds(mg.MONT_DOMAIN_REDC, mg.MONT_RANGE_DEFAULT, 0, 0, 0, 0),
            flags=mg.MONT_SWEEP_INCLUDE_OUT_OF_SPEC)


def test_alpha0_at_n8_matches_oracle():
    got = compare(mg.MONT_SIGNED_PLANTARD2, 16, 0, 3, 127, vectorised=True)
    assert got.total > 0


def test_plantard_bound_tightness_on_gpu():
    got = compare(mg.MONT_PLANTARD, 16, 0, 141, 171, flags=mg.MONT_SWEEP_INCLUDE_OUT_OF_SPEC,
                  vectorised=True)
    assert all(got.counts[N] == 0 for N in got.moduli if o.plantard_bound_ok(N, 8))
    assert got.counts[159] > 0


def test_explicit_rules():
    b = mg.MontBounds(mg.MONT_DOMAIN_EXPLICIT, mg.MONT_RANGE_EXPLICIT, -5000, 7000, -3, 40)
    for variant in range(5):
        compare(variant, 12, 1, 3, 45, bounds=b, flags=mg.MONT_SWEEP_INCLUDE_OUT_OF_SPEC)
    b = mg.MontBounds(mg.MONT_DOMAIN_DEFAULT, mg.MONT_RANGE_CENTRED, 0, 0, 0, 0)
    compare(mg.MONT_SIGNED, 10, 0, 3, 255, bounds=b)
    b = mg.MontBounds(mg.MONT_DOMAIN_DEFAULT, mg.MONT_RANGE_UNSIGNED, 0, 0, 0, 0)
    compare(mg.MONT_SIGNED, 10, 0, 3, 255, bounds=b)


def test_overflow_keeps_counts_exact():
    got = mg.mont_verify_sweep(mg.MONT_SIGNED_PLANTARD2, 12, 0, 3, 31, cex_cap=10)
    want = o.sweep(o.SIGNED_PLANTARD2, 12, 0, 3, 31)
    assert got.overflow and got.total == want.total
    assert len(got.examples) == 10 and set(got.examples) <= set(want.examples)
    assert got.examples == sorted(got.examples)
    assert all(got.counts[N] == want.counts.get(N, 0) for N in got.moduli)


@pytest.mark.parametrize("variant,alpha", [(0, 0), (1, 0), (2, 0), (3, 0), (4, 1)])
def test_full_sweep_r16_all_odd_N_to_4095(variant, alpha):
    """Every odd N in [3, 4095] at R = 2^16, each algorithm on its own domain:
    no counterexample (Sections 1 and 3), every T of every domain checked,
    and the oracle agrees on sampled moduli."""
    got = mg.mont_verify_sweep(variant, 16, alpha, 3, 4095, cex_cap=1024)
    assert got.total == 0 and not got.overflow
    for N in got.moduli:
        if o.precondition_ok(variant, N, 16, alpha):
            lo, hi = o.input_domain(variant, N, 16, alpha)
            assert got.checked[N] == hi - lo + 1
        else:
            assert got.checked[N] == 0
    for N in (3, 5, 101, 127, 157, 1001):
        if o.precondition_ok(variant, N, 16, alpha):
            want = o.sweep(variant, 16, alpha, N, N, vectorised=True)
            assert got.counts[N] == want.counts[N] == 0


def test_full_sweep_redc_domain_for_every_variant():
    """The literal rule 'every T in [0, RN)' applied to every variant: REDC
    passes; the others leave their claimed ranges.  Counts match the oracle on
    sampled moduli."""
    b = mg.MontBounds(mg.MONT_DOMAIN_REDC, mg.MONT_RANGE_DEFAULT, 0, 0, 0, 0)
    for variant, alpha in ((0, 0), (1, 0), (2, 0), (3, 0), (4, 1)):
        got = mg.mont_verify_sweep(variant, 16, alpha, 3, 4095, b, cex_cap=4096)
        if variant == 0:
            assert got.total == 0
        for N in (3, 7, 45, 63, 101):
            if got.checked[N] == 0:
                continue
            want = o.sweep(variant, 16, alpha, N, N, domain=ex.DOMAIN_REDC, vectorised=True)
            assert got.counts[N] == want.counts[N], (variant, N)


def test_redc_sweep_r16_moduli_to_1023():
    """REDC at R = 2^16 over every odd N <= 1023 (1.7e10 checks): no
    counterexample, full domains checked, oracle agreement on sampled N."""
    got = mg.mont_verify_sweep(mg.MONT_REDC, 16, 0, 3, 1023, cex_cap=64)
    assert got.total == 0
    assert all(got.checked[N] == (1 << 16) * N for N in got.moduli)
    for N in (3, 255, 1023):
        assert o.sweep(o.REDC, 16, 0, N, N, vectorised=True).counts[N] == got.counts[N] == 0
