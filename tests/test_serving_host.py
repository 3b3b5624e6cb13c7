"""Host-side logic of the serving measurement and of the CPU baseline, on CPU:
the checks a sweep job performs (against the oracle's input domains), the
stream bound's arithmetic, and the all-core oracle timing of bench.py on a
small sample."""

import pytest

import oracle as o
from paper_2402_00675_gb300 import serving

import synthetic as sy


@pytest.mark.parametrize("variant", [o.REDC, o.SIGNED, o.PLANTARD])
def test_sweep_checks_equal_the_domains(variant):
    """serving.sweep_checks counts exactly the T of every in-spec modulus's
    own domain (the oracle's Require lines), skipping out-of-spec moduli."""
    for n_lo, count in ((3, 40), (101, 17), (3073, 12)):
        want = 0
        for i in range(count):
            N = n_lo + 2 * i
            if o.precondition_ok(variant, N, 16, 0):
                lo, hi = o.input_domain(variant, N, 16, 0)
                want += hi - lo + 1
        assert serving.sweep_checks(variant, 16, n_lo, count) == want, (variant, n_lo)


def test_stream_bound_arithmetic():
    jobs = [sy.Job(0.0, "modmul", 0, 32, 1000, seed=1),
            sy.Job(0.1, "modmul", 1, 64, 1 << 20, seed=2),
            sy.Job(0.2, "modmul", 0, 256, 1 << 30, seed=3),      # capped at max_len
            sy.Job(0.3, "sweep", o.REDC, 16, 3, n_lo=3, seed=4)]
    rates = {o.REDC: 1e12, o.SIGNED: 1e12, o.PLANTARD: 1e12}
    b = serving.stream_bound(jobs, rates, link_gbs=100.0, hbm_gbs=1000.0, max_len=1 << 24)
    checks = serving.sweep_checks(o.REDC, 16, 3, 3)
    assert checks == (1 << 16) * (3 + 5 + 7)
    by = [1000 * 4, (1 << 20) * 8, (1 << 24) * 32]
    assert b["sweep_device_s"] == round(checks / 1e12, 3)
    assert b["modmul_kernel_s"] == round(sum(3 * x for x in by) / 1e12, 4)
    assert b["link_s"] == round(2 * sum(by) / 100e9, 3)        # operands in: twice the products out
    bound = max(checks / 1e12 + sum(3 * x for x in by) / 1e12, 2 * sum(by) / 100e9)
    assert b["bound_s"] == round(bound, 3)
    assert b["jobs_per_s_bound"] == round(len(jobs) / bound, 1)


def test_oracle_baseline_uses_every_core_on_disjoint_pairs(monkeypatch):
    """bench.oracle_baseline: one spawned process per core, each on its own
    slice of every vector, products counted over all of them."""
    import bench
    monkeypatch.setattr(bench, "N_PAIRS", 1 << 12)
    monkeypatch.setattr(bench, "SLICE_PAIRS", 1 << 8)
    inputs = bench.make_inputs()
    slices = [bench._oracle_slices(inputs, w) for w in range(3)]
    # disjoint: worker w holds pairs [w S, (w + 1) S) of every vector
    for w in range(3):
        for (_, _, _, xs, _), (N, vec) in zip(slices[w], [(N, v) for N in bench.MODULI
                                                          for v in bench.COMBOS]):
            a, b, au, bu = inputs[N]
            src = au if vec[0] == 2 else a
            assert xs == src[w * 256:(w + 1) * 256].tolist()
    monkeypatch.setattr(bench, "host_cpu", lambda: (2, "test cpu"))
    res = bench.oracle_baseline(inputs, 0.3)
    assert res["cores"] == 2 and res["kind"] == "oracle" and res["value"] > 0
    assert "2 spawned processes" in res["sample"]
