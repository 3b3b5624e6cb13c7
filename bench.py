#!/usr/bin/env python3
"""Throughput of Montgomery-type modular multiplication on one or more GPUs.

Workload (one "step"): the 32-bit signed and Plantard-style variants on the
moduli N = 3329 and N = 8380417, 2^26 operand pairs per modulus drawn
uniformly from the centred range (-N/2, N/2] (the Plantard reduction gets the
same residues lifted to [0, N)), R = 2^32 for the signed Montgomery reduction
(Algorithm 1) and R = 2^64 for the Plantard reduction (Algorithm 2) and the
two signed Plantard reductions (Algorithm 3; Algorithm 4 with alpha = 1).
One step is 8 mont_mul launches of 2^26 elements: 5.4e8 modular products,
6.4 GB of operand traffic.  Every operand array is 256 MiB, larger than the
129 MB L2, so no flush is needed between steps.

Output: one JSON line (rank 0).  ``value`` is Gmodmul/s with the operands
resident in HBM; ``e2e`` is the same metric through the same C-ABI calls
with the operands copied from pinned host memory and the products copied
back inside the timed region.  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synthetic as sy  # noqa: E402

METRIC = "Gmodmul/s"
WORKLOAD = ("word32 mont_mul: Alg.1 SigRedc R=2^32, Alg.2 PRedc, Alg.3 SigPRedc1, "
            "Alg.4 SigPRedc2(alpha=1) R=2^64; N in {3329, 8380417}; 2^26 pairs per modulus")
N_PAIRS = 1 << 26
MODULI = sy.WORD32_MODULI
# (variant, log2R): Algorithm 1, 2, 3, 4
COMBOS = ((1, 32), (2, 64), (3, 64), (4, 64))
VARIANT_NAMES = {1: "sigredc", 2: "predc", 3: "sigpredc1", 4: "sigpredc2_a1"}
BYTES_PER_MODMUL = 12          # two 4-byte operands in, one 4-byte product out
# device staging of the end-to-end leg's pipe: three slots, each holding a
# chunk of 2^22 elements (16 MiB) of the 8 distinct inputs and the 8 outputs
E2E_STAGING_BYTES = 800 << 20
ALPHA = 1

# DRAM bytes per launch of the word kernel on this workload (read + write,
# mean of the 8 launches of one step), from a one-pass ncu capture of the
# full-size launch.  Reads equal the algorithmic 536.9 MB; writes (228.1 MB of
# 268.4 MB) exclude the output tail still dirty in L2 when the kernel ends,
# which the next launch writes back.
NCU_TRAFFIC_BYTES_PER_LAUNCH = 764626656


def parse_args():
    p = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=2000)
    p.add_argument("--warmup", type=int, default=20)
    p.add_argument("--impl", choices=("ours", "reference"), default="ours")
    p.add_argument("--e2e-steps", type=int, default=0, help="0: min(steps, 10)")
    p.add_argument("--cpu-work-s", type=float, default=24.0,
                   help="CPU seconds (summed over cores) the oracle baseline runs")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-extras", action="store_true",
                   help="skip the per-config measurements after the main step")
    p.add_argument("--serving-jobs", type=int, default=10000)
    p.add_argument("--extra", action="append", default=[], metavar="NAME",
                   help="run only this per-config measurement (repeatable; e.g. rns_convert, "
                        "sweep_r16, cios) and print {\"extras\": {...}}; for profiling")
    p.add_argument("--log2-pairs", type=int, default=26,
                   help="pairs per modulus = 2^this (26 is the benchmark workload)")
    a = p.parse_args()
    global N_PAIRS
    N_PAIRS = 1 << a.log2_pairs
    return a


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", str(rank)))
    return rank, world, local


# ---------------------------------------------------------------- ranks

def max_over_ranks(elapsed_ms: float, world: int, device: str = "cuda") -> float:
    """The job's time: the largest of the ranks' times (all ranks call this)."""
    if world == 1:
        return elapsed_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([elapsed_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, elapsed_ms: float) -> float:
    """Units of every rank (each rank runs the same replica) per second, in 1e9."""
    return world * units_per_rank / (elapsed_ms * 1e-3) / 1e9


# ---------------------------------------------------------------- inputs

def make_inputs():
    """Seeded operands per modulus: centred int32 and their [0, N) lift."""
    out = {}
    for N in MODULI:
        a = sy.centred_residues(N, N_PAIRS, seed=2 * N + 1)
        b = sy.centred_residues(N, N_PAIRS, seed=2 * N + 2)
        out[N] = (a, b, sy.lift_unsigned(a, N), sy.lift_unsigned(b, N))
    return out


# ---------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100", "-i", str(self.dev)],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.25)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        rows = [r.split(",") for r in out.strip().splitlines() if r.strip()]
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except ValueError:
                continue
            for name, val in zip(names, r[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        if not sm:
            return None
        # samples under load: the top of the distribution (idle gaps read low)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- cpu oracle

SLICE_PAIRS = 1 << 15   # pairs of each of the 8 vectors a worker cycles over


def _oracle_slices(inputs, worker: int):
    """Worker `worker`'s own disjoint pairs of each (modulus, variant) vector."""
    lo = worker * SLICE_PAIRS
    hi = min(lo + SLICE_PAIRS, N_PAIRS)
    out = []
    for N in MODULI:
        a, b, au, bu = inputs[N]
        for variant, l in COMBOS:
            x, y = (au, bu) if variant == 2 else (a, b)
            out.append((variant, N, l, x[lo:hi].tolist(), y[lo:hi].tolist()))
    return out


def _oracle_work(task):
    """Runs in a spawned process: the oracle, as it stands, over this worker's
    slices.  ("budget", s): round-robin blocks of 256 pairs per vector until s
    seconds pass; ("count", c): exactly c pairs of each vector.  Returns
    (products, seconds)."""
    import oracle as o
    mode, amount, slices = task
    pos = 0
    done = 0
    t0 = time.perf_counter()
    while True:
        blk = 256 if mode == "budget" else amount
        for variant, N, l, xs, ys in slices:
            m = len(xs)
            for j in range(pos, pos + blk):
                i = j % m
                o.mul_value(variant, xs[i], ys[i], N, l, ALPHA)
        done += blk * len(slices)
        pos += blk
        if mode == "count" or time.perf_counter() - t0 >= amount:
            break
    return done, time.perf_counter() - t0


def host_cpu():
    """(logical cores, CPU model) of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return os.cpu_count() or 1, model or "unknown"


class OraclePool:
    """One spawned process per host core, each holding its own disjoint
    slice of the workload (SLICE_PAIRS pairs of each of the 8 vectors)."""

    def __init__(self, inputs, cores: int):
        import multiprocessing as mp
        self.cores = max(1, min(cores, N_PAIRS // SLICE_PAIRS))
        self.slices = [_oracle_slices(inputs, w) for w in range(self.cores)]
        self.pool = mp.get_context("spawn").Pool(self.cores)
        self.pool.map(_oracle_work, [("count", 1, sl) for sl in self.slices])   # imports

    def budget(self, seconds: float):
        """Products per second over all cores, each running `seconds`."""
        t0 = time.perf_counter()
        res = self.pool.map(_oracle_work, [("budget", seconds, sl) for sl in self.slices])
        wall = time.perf_counter() - t0
        done = sum(r[0] for r in res)
        return done / wall, done, wall

    def count(self, per: int):
        """Every core evaluates `per` pairs of each of its 8 vectors."""
        res = self.pool.map(_oracle_work, [("count", per, sl) for sl in self.slices])
        return sum(r[0] for r in res)

    def close(self):
        self.pool.close()
        self.pool.join()


def oracle_baseline(inputs, budget_s: float):
    """The oracle timed on every host core (one process each) for about
    budget_s seconds of wall time."""
    cores, model = host_cpu()
    pool = OraclePool(inputs, cores)
    rate, done, wall = pool.budget(budget_s)
    pool.close()
    return {"value": rate / 1e9, "unit": METRIC, "cores": pool.cores, "kind": "oracle",
            "cpu": model,
            "sample": f"{pool.cores} spawned processes (one per host core), each cycling over its "
                      f"own disjoint {SLICE_PAIRS} pairs of each of the 8 (modulus, variant) vectors: "
                      f"{done} oracle products in {wall:.1f} s wall, Python big-int"}


# ---------------------------------------------------------------- extras
# Each extra measures one other workload of the library outside the main
# timed region, with CUDA events on the launching stream, and carries its own
# roofline.  Peaks: HBM from MEASURED_PEAKS.json; integer peaks derived from
# unit counts per SM and clock (4 schedulers x 32 lanes = 128 issued thread
# instructions; 64 mad.lo; 32 mad.hi, so a 32x32->64 limb product, lo + hi,
# takes 3/64 of an SM-cycle) times the SM count queried from the device and
# its maximum SM clock; the sweep's peak is the mad.lo rate measured live.

PEAKS = {"sms": 152, "sm_mhz_max": 2070.0}


def set_int_peaks(sms: int, sm_mhz_max: float) -> None:
    """Integer peaks of the device the benchmark runs on."""
    hz = sm_mhz_max * 1e6
    PEAKS.update(sms=sms, sm_mhz_max=sm_mhz_max,
                 issue=128.0 * sms * hz,                 # thread-instructions / s
                 limb=64.0 / 3.0 * sms * hz,             # lo + hi limb products / s
                 mad_lo=64.0 * sms * hz)                 # mad.lo.u32 / s


set_int_peaks(152, 2070.0)


def read_measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def device_int_peaks(peaks_file: dict) -> None:
    import torch
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    set_int_peaks(props.multi_processor_count, float(peaks_file.get("sm_max_mhz") or 2070.0))


# Integer operations per sweep check of each algorithm's formula as issued
# (the formula's own operations, the reference step c += s R^-1 mod N, the
# congruence and range tests and the loop step): an issue-slot figure only.
SWEEP_OPS = {0: 16, 1: 17, 2: 16, 3: 17, 4: 16}
# The survey's algorithmic unit for the sweep: a check costs about 3 IMAD
# slots (T N' low product, m N, and the reference step), so the roofline is
# the measured mad.lo rate / 3 checks per second.
SWEEP_IMAD_PER_CHECK = 3.0


def _events_ms(fn, reps, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_link(h_in, d_in, h_out, d_out, stream):
    """Host link of this machine, measured on the end-to-end leg's own pinned
    buffers (256 MiB each): one copy in, one copy out, and both at once, each
    direction on its own stream (GB/s each way)."""
    import torch
    nb = h_in.numel() * h_in.element_size()
    s_in, s_out = torch.cuda.Stream(), torch.cuda.Stream()

    def run(do_in, do_out):
        ev = torch.cuda.Event()
        ev.record(stream)
        for s_, do, fn in ((s_in, do_in, lambda: d_in.copy_(h_in, non_blocking=True)),
                           (s_out, do_out, lambda: h_out.copy_(d_out, non_blocking=True))):
            if do:
                s_.wait_event(ev)
                with torch.cuda.stream(s_):
                    fn()
                stream.wait_stream(s_)
    ms_in = _events_ms(lambda: run(True, False), 5, stream)
    ms_out = _events_ms(lambda: run(False, True), 5, stream)
    ms_both = _events_ms(lambda: run(True, True), 5, stream)
    return {"h2d_gbs": round(nb / (ms_in * 1e-3) / 1e9, 1),
            "d2h_gbs": round(nb / (ms_out * 1e-3) / 1e9, 1),
            "both_each_gbs": round(nb / (ms_both * 1e-3) / 1e9, 1)}


def extra_redc32(mg, stream, peak):
    """REDC, R = 2^32, N = 3329, 2^20 pairs: hot (same buffers, L2-resident)
    and cold (16 rotating buffer sets, 201 MB > L2), each as calls through
    the C ABI and as the same launches replayed from a CUDA graph."""
    import torch
    N, n = sy.REDC32_N, 1 << 20
    ctx = mg.mont_ctx_create(N, 32, 0)
    sets = []
    for r in range(16):
        a = torch.from_numpy(sy.uniform_residues(N, n, seed=1 + 100 * r)).cuda()
        b = torch.from_numpy(sy.uniform_residues(N, n, seed=101 + 100 * r)).cuda()
        sets.append((a, b, torch.empty_like(a)))
    L = mg.lib()
    sp = stream.cuda_stream
    calls = [(x.data_ptr(), y.data_ptr(), z.data_ptr()) for x, y, z in sets]
    for _ in range(20):
        L.mont_mul(ctx.handle, *calls[0], n, sp)
    hot = _events_ms(lambda: L.mont_mul(ctx.handle, *calls[0], n, sp), 400, stream)
    k = [0]

    def rot():
        L.mont_mul(ctx.handle, *calls[k[0] % 16], n, sp)
        k[0] += 1
    cold = _events_ms(rot, 400, stream)
    gb = 12 * n / (cold * 1e-3) / 1e9
    # The same launches replayed from a CUDA graph (16 per replay: the 16
    # buffer sets in turn, or one set 16 times), so that the host's call and
    # launch cost per kernel is out of the timing: the device's own rate.
    graph = {}
    try:
        side = torch.cuda.Stream()
        side.wait_stream(stream)
        for name, order in (("cold_l2", list(range(16))), ("hot_l2", [0] * 16)):
            g = torch.cuda.CUDAGraph()
            with torch.cuda.stream(side):
                with torch.cuda.graph(g, stream=side):
                    for j in order:
                        L.mont_mul(ctx.handle, *calls[j], n, side.cuda_stream)
            stream.wait_stream(side)
            for _ in range(3):
                g.replay()
            ms = _events_ms(g.replay, 50, torch.cuda.current_stream()) / 16
            graph[name] = round(n / (ms * 1e-3) / 1e9, 1)
            graph[f"us_per_launch_{name.split('_')[0]}"] = round(ms * 1e3, 2)
            graph[f"frac_hbm_{name.split('_')[0]}"] = round(12 * n / (ms * 1e-3) / 1e9 / peak, 3)
        torch.cuda.synchronize()
    except Exception as exc:   # capture unavailable: report why, keep the rest
        graph = {"unavailable": str(exc)[:200]}
    return {"workload": "REDC R=2^32 N=3329, 2^20 pairs", "unit": "Gmodmul/s",
            "hot_l2": round(n / (hot * 1e-3) / 1e9, 1), "cold_l2": round(n / (cold * 1e-3) / 1e9, 1),
            "us_per_launch_hot": round(hot * 1e3, 2), "us_per_launch_cold": round(cold * 1e3, 2),
            "graph_replay": graph,
            "roofline": {"bound": "hbm", "achieved": round(gb, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gb / peak, 3), "note": "cold-L2 rotation; a 12.6 MB launch "
                         "is dominated by launch and ramp time"}}


def extra_rns64(mg, stream, peak):
    """32 primes of 60-62 bits, p = 1 mod 2^17, log-uniform lengths 2^12..2^22:
    one graph-launched persistent batch, its launch shape picked by the
    autotuner for 64-bit words, against 32 plain launches."""
    import torch
    primes = sy.rns_primes(32, seed=3)
    lens = sy.log_uniform_lengths(32, 12, 22, seed=3)
    ctxs, da, db, outs = [], [], [], []
    for j, (p_, n) in enumerate(zip(primes, lens)):
        ctxs.append(mg.mont_ctx_create(p_, 64, 0))
        da.append(torch.from_numpy(sy.uniform_residues(p_, n, seed=1000 + j, dtype=np.uint64)).cuda())
        db.append(torch.from_numpy(sy.uniform_residues(p_, n, seed=2000 + j, dtype=np.uint64)).cuda())
        outs.append(torch.empty(n, dtype=torch.uint64, device="cuda"))
    default_shape = mg.mont_tune_get(64, 0, mg.MONT_TUNE_MODE_BATCHED)
    mg.mont_autotune(ctxs[0], 1 << 22, mg.MONT_TUNE_BATCHED, stream)
    tuned = mg.mont_tune_get(64, 0, mg.MONT_TUNE_MODE_BATCHED)
    plan = mg.Batch(ctxs, da, db, outs, lens)
    L = mg.lib()
    sp = stream.cuda_stream
    calls = [(c.handle, x.data_ptr(), y.data_ptr(), z.data_ptr(), n)
             for c, x, y, z, n in zip(ctxs, da, db, outs, lens)]

    def plain():
        for h, x, y, z, n in calls:
            L.mont_mul(h, x, y, z, n, sp)
    for _ in range(10):
        plan.launch(stream)
        plain()
    t_batch = _events_ms(lambda: plan.launch(stream), 300, stream)
    t_plain = _events_ms(plain, 300, stream)
    tot = sum(lens)
    gb = 24 * tot / (t_batch * 1e-3) / 1e9
    plan.close()
    shape = lambda d: f"{d['threads']}t/u{d['unroll']}/{d['blocks_per_sm'] or 'occ'}"
    return {"workload": f"RNS REDC R=2^64, 32 primes, sum(len)={tot}", "unit": "Gmodmul/s",
            "batched_graph": round(tot / (t_batch * 1e-3) / 1e9, 1),
            "plain_32_launches": round(tot / (t_plain * 1e-3) / 1e9, 1),
            "speedup": round(t_plain / t_batch, 2),
            "us_batched": round(t_batch * 1e3, 2), "us_plain": round(t_plain * 1e3, 2),
            "shape_tuned": shape(tuned), "shape_default": shape(default_shape),
            "roofline": {"bound": "hbm", "achieved": round(gb, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gb / peak, 3)}}


def extra_cios(mg, stream, peak):
    """Multi-limb REDC (CIOS) at the stated sizes: random odd N of
    256/384/1024/2048 bits, 2^22/2^21/2^17/2^15 pairs uniform in [0, N).
    Each width is timed at the built-in launch shape, then autotuned at its
    stated size (lanes per element, block size, blocks per SM) and timed
    again; the tuned time is the reported one."""
    import torch
    out = {}
    for bits, count in ((256, 1 << 22), (384, 1 << 21), (1024, 1 << 17), (2048, 1 << 15)):
        k = bits // 32
        N = sy.random_odd_modulus(bits, seed=4)
        ctx = mg.mont_ctx_create(N, bits, 0)
        a = torch.from_numpy(sy.uniform_limb_residues(N, k, count, seed=40 + k).reshape(-1)).cuda()
        b = torch.from_numpy(sy.uniform_limb_residues(N, k, count, seed=80 + k).reshape(-1)).cuda()
        o = torch.empty_like(a)
        L = mg.lib()
        sp = stream.cuda_stream
        f = lambda: L.mont_mul(ctx.handle, a.data_ptr(), b.data_ptr(), o.data_ptr(), count, sp)
        for _ in range(5):
            f()
        ms_default = _events_ms(f, 50, stream)
        mg.mont_autotune(ctx, count, mg.MONT_TUNE_ELEMENTWISE, stream)
        t = mg.mont_tune_get(bits, 0, mg.MONT_TUNE_MODE_MUL)
        for _ in range(5):
            f()
        ms = _events_ms(f, 50, stream)
        for mode in range(4):      # later workloads start from the built-in shapes
            mg.mont_tune_set(bits, 0, mode, None)
        prods = (2 * k * k + k) * count
        ach = prods / (ms * 1e-3)
        gb = 12 * k * count / (ms * 1e-3) / 1e9
        out[f"{bits}b"] = {
            "pairs": count, "gmodmul_s": round(count / (ms * 1e-3) / 1e9, 3),
            "us": round(ms * 1e3, 2), "us_default_shape": round(ms_default * 1e3, 2),
            "shape_tuned": f"team{t['team']}/{t['threads']}t/{t['blocks_per_sm'] or 'occ'}",
            "roofline": {"bound": "alu", "achieved": round(ach / 1e12, 3),
                         "peak": round(PEAKS["limb"] / 1e12, 3),
                         "unit": "T limb-products/s (32x32->64, lo+hi)",
                         "frac": round(ach / PEAKS["limb"], 3),
                         "hbm_frac": round(gb / peak, 3)}}
    return out


def extra_limb_variants(mg, stream, peak):
    """Algorithms 1-4 at 256, 1024 and 2048 bits (n = 32k: R = 2^{32k} for
    Algorithm 1, 2^{64k} for Algorithms 2-4), random odd N at each variant's
    largest size class, operands uniform in the variant's output range;
    2^21 / 2^17 / 2^15 pairs.  Each is timed at the built-in launch shape,
    then autotuned at its size and timed again; the tuned time is reported."""
    import torch
    out = {}
    names = {1: "sigredc", 2: "predc", 3: "sigpredc1", 4: "sigpredc2_a1"}
    for bits, count in ((256, 1 << 21), (1024, 1 << 17), (2048, 1 << 15)):
        k = bits // 32
        L = mg.lib()
        sp = stream.cuda_stream
        for variant in (1, 2, 3, 4):
            top_bits = {1: bits - 1, 2: bits - 1, 3: bits - 1, 4: bits - 2}[variant]
            N = sy.random_odd_modulus(top_bits, seed=4 + variant)
            log2R = 2 * bits if variant >= 2 else bits
            ctx = mg.mont_ctx_create(N, log2R, variant, alpha=1, n_limbs=k)
            a = sy.uniform_limb_residues(N, k, count, seed=40 + variant)
            b = sy.uniform_limb_residues(N, k, count, seed=80 + variant)
            if variant != 2:   # signed variants: centre the residues (x - N for x > N/2)
                a, b = (sy.centred_limb_residues(N, x) for x in (a, b))
            da = torch.from_numpy(a.reshape(-1)).cuda()
            db = torch.from_numpy(b.reshape(-1)).cuda()
            o = torch.empty_like(da)
            f = lambda: L.mont_mul(ctx.handle, da.data_ptr(), db.data_ptr(), o.data_ptr(), count, sp)
            for _ in range(5):
                f()
            ms_default = _events_ms(f, 20, stream)
            mg.mont_autotune(ctx, count, mg.MONT_TUNE_ELEMENTWISE, stream)
            t = mg.mont_tune_get(bits, variant, mg.MONT_TUNE_MODE_MUL)
            for _ in range(5):
                f()
            ms = _events_ms(f, 20, stream)
            for mode in range(4):   # later workloads start from the built-in shapes
                mg.mont_tune_set(bits, variant, mode, None)
            # limb products as the kernels form them: Algorithm 1 on the CIOS
            # schedule, 2k^2 + k (a b and m'N row by row, the k digits of m');
            # Algorithms 2-4: T = a b (k^2), m = T N^{-1} mod 2^{64k} (k(2k+1))
            # and q N ((k+1) k)
            per = 2 * k * k + k if variant == 1 else 4 * k * k + 2 * k
            ach = per * count / (ms * 1e-3)
            out[f"{bits}b_{names[variant]}"] = {
                "pairs": count, "gmodmul_s": round(count / (ms * 1e-3) / 1e9, 3),
                "us": round(ms * 1e3, 2), "us_default_shape": round(ms_default * 1e3, 2),
                "shape_tuned": f"team{t['team']}/{t['threads']}t/{t['blocks_per_sm'] or 'occ'}",
                "roofline": {"bound": "alu", "achieved": round(ach / 1e12, 3),
                             "peak": round(PEAKS["limb"] / 1e12, 3),
                             "unit": "T limb-products/s (32x32->64, lo+hi)",
                             "frac": round(ach / PEAKS["limb"], 3),
                             "hbm_frac": round(12 * k * count / (ms * 1e-3) / 1e9 / peak, 3)}}
    return out


def extra_sweep(mg, stream):
    """R = 2^16, every odd N in [3, 4095]; each algorithm on its own domain,
    and on REDC's domain 0 <= T < RN.  Roofline: the measured mad.lo rate / 3
    checks per second; the issue-slot fraction of the formula's own operation
    count is kept beside it."""
    import torch
    out = {}
    names = {0: "redc", 1: "sigredc", 2: "predc", 3: "sigpredc1", 4: "sigpredc2_a1"}
    mad_lo = mg.mont_probe_int_rate(0, 4096, stream)
    peak_checks = mad_lo / SWEEP_IMAD_PER_CHECK
    out["peak"] = {"mad_lo_t_s": round(mad_lo / 1e12, 2), "checks_t_s": round(peak_checks / 1e12, 3),
                   "unit": "T checks/s = measured mad.lo rate / 3"}
    redc_dom = mg.MontBounds(mg.MONT_DOMAIN_REDC, mg.MONT_RANGE_DEFAULT, 0, 0, 0, 0)
    for v, alpha in ((0, 0), (1, 0), (2, 0), (3, 0), (4, 1)):
        for dom_name, dom in (("own_domain", None), ("redc_domain", redc_dom)):
            mg.mont_verify_sweep(v, 16, alpha, 3, 255, dom, cex_cap=16, stream=stream)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            r = mg.mont_verify_sweep(v, 16, alpha, 3, 4095, dom, cex_cap=64, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            checks = sum(r.checked.values())
            rate = checks / (ms * 1e-3)
            out[f"{names[v]}_{dom_name}"] = {
                "checks": checks, "counterexamples": r.total,
                "ms": round(ms, 3), "gchecks_s": round(rate / 1e9, 2),
                "roofline": {"bound": "alu", "achieved": round(rate / 1e12, 3),
                             "peak": round(peak_checks / 1e12, 3), "unit": "T checks/s",
                             "frac": round(rate / peak_checks, 3),
                             "issue_frac": round(rate * SWEEP_OPS[v] / PEAKS["issue"], 3)}}
    return out


# 32-bit integer operations per butterfly of the algorithm each plan runs; the
# benchmark's moduli have 4N <= 2^w, so both kinds of twiddle run lazy
# butterflies (coefficients kept below 4N, reduced below N once at the end).
# REDC twiddles: REDC without its final subtraction (the product, m, the high
# product with N, the carry and the add, 6), x reduced below 2N (2), x + t and
# x + 2N - t (2), the final reduction amortised over the butterflies (1): 11.
# Plantard's prepared twiddles: the product (two products and one product with
# N, 3), then 2 + 2 + 1 as above: 8.  64-bit words, counting every 64-bit
# product in 32-bit multiply-adds (4 for a full or high product, 3 for a low
# one) and 64-bit adds as 2: REDC 30, Plantard 26.
NTT_BUTTERFLY_OPS = {(0, 32): 11, (2, 32): 8, (0, 64): 30, (2, 64): 26}
# Limb products (32x32 -> 64, lo + hi = 1; a low or a high half alone = 1/3 or
# 2/3, at the multiply pipe's rates) of one butterfly's twiddle product.
# 32-bit: REDC y w (1), m = lo N' (1/3), hi(m N) (2/3); Plantard hi(a b'lo) (2/3),
# lo(a b'hi) (1/3), (q + 1) N (1).  64-bit: REDC y w (4), m low 64 bits (5/3),
# hi64(m N) (11/3); Plantard hi64(a b'lo) (11/3), lo64(a b'hi) (5/3), (q+1) N (4).
NTT_BUTTERFLY_LIMB_PRODUCTS = {(0, 32): 2.0, (2, 32): 2.0, (0, 64): 28 / 3, (2, 64): 28 / 3}


def extra_ntt(mg, stream, peak):
    """Batched negacyclic NTTs: 2^18 polynomials of length 256 mod 8380417
    (32-bit words) and 2^15 of length 1024 mod a 62-bit RNS prime (64-bit
    words), with REDC (Montgomery-form twiddles) and Plantard (prepared
    twiddles) butterflies; plus mont_mul_pre against mont_mul."""
    import torch
    out = {}
    L = mg.lib()
    sp = stream.cuda_stream
    rns = sy.rns_primes(1, seed=3)[0]
    for N, w, log2n, batch in ((8380417, 32, 8, 1 << 18), (rns, 64, 10, 1 << 15)):
        n = 1 << log2n
        psi = sy.primitive_2n_root(N, n, seed=1)
        dt = torch.uint32 if w == 32 else torch.uint64
        x = torch.from_numpy(sy.uniform_residues(N, batch * n, seed=7,
                                                 dtype=np.uint32 if w == 32 else np.uint64)).cuda()
        y = torch.empty_like(x)
        for v in (0, 2):
            ctx = mg.mont_ctx_create(N, w if v == 0 else 2 * w, v)
            plan = mg.Ntt(ctx, log2n, psi)
            f = lambda: L.mont_ntt_forward(plan.handle, x.data_ptr(), y.data_ptr(), batch, sp)
            g = lambda: L.mont_ntt_inverse(plan.handle, y.data_ptr(), y.data_ptr(), batch, sp)
            for _ in range(3):
                f()
            ms_f = _events_ms(f, 20, stream)
            ms_i = _events_ms(g, 20, stream)
            bfly = batch * (n // 2) * log2n
            ops = bfly * NTT_BUTTERFLY_OPS[(v, w)] / (ms_f * 1e-3)
            lp = bfly * NTT_BUTTERFLY_LIMB_PRODUCTS[(v, w)] / (ms_f * 1e-3)
            gb = 2 * batch * n * (w // 8) / (ms_f * 1e-3) / 1e9
            out[f"n{n}_w{w}_{'redc' if v == 0 else 'plantard'}"] = {
                "polys": batch, "forward_us": round(ms_f * 1e3, 1), "inverse_us": round(ms_i * 1e3, 1),
                "gcoeff_s": round(batch * n / (ms_f * 1e-3) / 1e9, 1),
                "roofline": {"bound": "alu", "achieved": round(lp / 1e12, 3),
                             "peak": round(PEAKS["limb"] / 1e12, 3),
                             "unit": "T limb-products/s (the twiddle products on the multiply pipe)",
                             "frac": round(lp / PEAKS["limb"], 3),
                             "issue_frac": round(ops / PEAKS["issue"], 3),
                             "hbm_frac": round(gb / peak, 3)}}
            plan.close()
    for tag in ("n256_w32", "n1024_w64"):
        out[f"{tag}_plantard_speedup_over_redc"] = round(
            out[f"{tag}_redc"]["forward_us"] / out[f"{tag}_plantard"]["forward_us"], 2)
    # prepared multipliers on the 32-bit workload size
    N, n = 8380417, 1 << 26
    ctx = mg.mont_ctx_create(N, 64, 2)
    a = torch.from_numpy(sy.uniform_residues(N, n, seed=8)).cuda()
    b = torch.from_numpy(sy.uniform_residues(N, n, seed=9)).cuda()
    bp = torch.empty(n, dtype=torch.uint64, device="cuda")
    o = torch.empty_like(a)
    mg.mont_const_prepare(ctx, b, bp)
    fp = lambda: L.mont_mul_pre(ctx.handle, a.data_ptr(), bp.data_ptr(), o.data_ptr(), n, sp)
    fm = lambda: L.mont_mul(ctx.handle, a.data_ptr(), b.data_ptr(), o.data_ptr(), n, sp)
    for _ in range(3):
        fp()
        fm()
    ms_p = _events_ms(fp, 50, stream)
    ms_m = _events_ms(fm, 50, stream)
    out["mul_pre_2p26"] = {"us": round(ms_p * 1e3, 1), "gmodmul_s": round(n / (ms_p * 1e-3) / 1e9, 1),
                           "mont_mul_us": round(ms_m * 1e3, 1),
                           "roofline": {"bound": "hbm", "achieved": round(16 * n / (ms_p * 1e-3) / 1e9, 1),
                                        "peak": peak, "unit": "GB/s",
                                        "frac": round(16 * n / (ms_p * 1e-3) / 1e9 / peak, 3),
                                        "note": "16 B per product: a (4), b' (8), out (4)"}}
    return out


def extra_dot(mg, stream, peak):
    """Row dot products of 16 centred residues mod 8380417 reduced once with
    Algorithm 4 (alpha = 1), 2^22 rows: against 16 separate reductions per
    row (mont_mul with the same algorithm, 2^26 products)."""
    import torch
    N, k, rows = 8380417, 16, 1 << 22
    ctx = mg.mont_ctx_create(N, 64, 4, alpha=1)
    a = torch.from_numpy(sy.centred_residues(N, rows * k, seed=11)).cuda()
    b = torch.from_numpy(sy.centred_residues(N, rows * k, seed=12)).cuda()
    o = torch.empty(rows, dtype=torch.int32, device="cuda")
    prod = torch.empty_like(a)
    L = mg.lib()
    sp = stream.cuda_stream
    f = lambda: L.mont_dot_lazy(ctx.handle, a.data_ptr(), b.data_ptr(), o.data_ptr(), rows, k, sp)
    g = lambda: L.mont_mul(ctx.handle, a.data_ptr(), b.data_ptr(), prod.data_ptr(), rows * k, sp)
    for _ in range(3):
        f()
        g()
    ms = _events_ms(f, 50, stream)
    ms_mul = _events_ms(g, 50, stream)
    gb = (8 * rows * k + 4 * rows) / (ms * 1e-3) / 1e9
    return {"workload": "2^22 rows x 16 products mod 8380417, Algorithm 4 alpha = 1",
            "us": round(ms * 1e3, 1), "gproducts_s": round(rows * k / (ms * 1e-3) / 1e9, 1),
            "reductions_per_row": 1, "mont_mul_all_products_us": round(ms_mul * 1e3, 1),
            "roofline": {"bound": "hbm", "achieved": round(gb, 1), "peak": peak, "unit": "GB/s",
                         "frac": round(gb / peak, 3)}}


def extra_rns(mg, stream):
    """Conversions between 2^17 big integers uniform below P and their
    residues modulo the 32 RNS primes (product of 1950 bits, 64 limbs)."""
    import torch
    ps = sy.rns_primes(32, seed=3)
    r = mg.Rns(ps)
    n, k = 1 << 17, r.limbs
    X = torch.from_numpy(sy.uniform_limb_residues(_product(ps), k, n, seed=13).reshape(-1)).cuda()
    res = torch.empty(32 * n, dtype=torch.uint64, device="cuda")
    Y = torch.empty_like(X)
    f = lambda: r.to_residues(X, res, n, stream)
    g = lambda: r.from_residues(res, Y, n, stream)
    for _ in range(3):
        f()
        g()
    ms_to = _events_ms(f, 20, stream)
    ms_from = _events_ms(g, 20, stream)
    assert torch.equal(X, Y)
    # 32x32 -> 64-bit limb products (lo + hi) the algorithms need per element.
    # to_residues: each of the 32 residues sums limbs(X) limb-by-word products
    # (2 limb products each) and ends in one 64-bit REDC (about 12).
    # from_residues (the CRT formula): xh_i M_i for every i (2 per limb of
    # M_i = P / p_i), q' P (1 per limb of P), and per modulus xh_i by one
    # 64-bit REDC of x_i times a constant (28/3) and the 64-bit fraction
    # xh_i floor(2^128 / p_i) / 2^64 (16/3).
    P = _product(ps)
    lx = -(-P.bit_length() // 32)
    prods_to = 32 * (2 * lx + 12)
    prods_from = round(sum(2 * -(-(P // p).bit_length() // 32) for p in ps) + lx
                       + len(ps) * (28 / 3 + 16 / 3))
    r.close()
    a_to = n * prods_to / (ms_to * 1e-3)
    a_from = n * prods_from / (ms_from * 1e-3)
    return {"workload": "2^17 integers below P, 32 primes of 60-62 bits",
            "to_residues_us": round(ms_to * 1e3, 1), "from_residues_us": round(ms_from * 1e3, 1),
            "to_melem_s": round(n / (ms_to * 1e-3) / 1e6, 1),
            "from_melem_s": round(n / (ms_from * 1e-3) / 1e6, 1),
            "roofline": {"bound": "alu", "unit": "T limb-products/s (32x32->64, lo+hi)",
                         "peak": round(PEAKS["limb"] / 1e12, 3),
                         "limb_products_per_element": {"to": prods_to, "from": prods_from},
                         "achieved_to": round(a_to / 1e12, 3),
                         "achieved_from": round(a_from / 1e12, 3),
                         "frac_to": round(a_to / PEAKS["limb"], 3),
                         "frac_from": round(a_from / PEAKS["limb"], 3)}}


def _product(xs):
    p = 1
    for x in xs:
        p *= x
    return p


def extra_serving(mg, jobs_count, stream, peak):
    """Poisson stream of mixed jobs through the serving loop at full rate
    (capacity) and at 0.5x and 0.8x of the measured capacity, with the
    stream's lower-bound time (sweep checks at the measured sweep rates, the
    host link at its measured rate) beside it."""
    import torch
    from paper_2402_00675_gb300 import serving
    ctxs = serving.Contexts.create(3329, sy.rns_primes(1, seed=31)[0],
                                   sy.random_odd_modulus(256, seed=32))
    pools = serving.Pools(ctxs, 1 << 24)
    ring = serving.OutputRing(3 << 30)
    server = mg.Server(8 << 30, slots=8)
    out = {"jobs_per_run": jobs_count, "slots": 8, "arena_gb": 8}
    jobs = sy.serving_jobs(jobs_count, 1.0, seed=5)
    # the link as the serving copies see it: pinned pool in, pinned ring out
    h_in = pools.pools[(0, 256)][0]
    d_buf = torch.empty_like(h_in, device="cuda")
    h_out = ring.buf[: h_in.numel() * h_in.element_size()].view(h_in.dtype)
    link = measure_link(h_in, d_buf, h_out, d_buf, stream)
    del d_buf
    # sweep rates as the jobs see them: one 512-moduli window per algorithm,
    # alone (REDC and Algorithm 1 at the top of the range, where their
    # windows spend most of their time; Algorithm 2 where its moduli are)
    rates = {}
    for v, lo in ((0, 3073), (1, 3073), (2, 3)):
        mg.mont_verify_sweep(v, 16, 0, lo, lo + 1022, cex_cap=16, stream=stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = mg.mont_verify_sweep(v, 16, 0, lo, lo + 1022, cex_cap=16, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        rates[v] = sum(r.checked.values()) / (e0.elapsed_time(e1) * 1e-3)
    bound = serving.stream_bound(jobs, rates, link["both_each_gbs"], peak, pools.max_len)
    bound["link"] = link
    bound["sweep_gchecks_s"] = {k: round(v / 1e9, 1) for k, v in rates.items()}
    out["bound"] = bound
    cap = serving.summarise(serving.run_stream(server, jobs, ctxs, pools, ring, rate_scale=0.0))
    out["capacity"] = cap
    out["capacity_frac_of_bound"] = round(cap["makespan_s"] and bound["bound_s"] / cap["makespan_s"], 3)
    for lam in (0.5, 0.8):
        rate = lam * cap["jobs_per_s"]
        jobs = sy.serving_jobs(jobs_count, rate, seed=5)
        out[f"load_{lam}"] = serving.summarise(
            serving.run_stream(server, jobs, ctxs, pools, ring, rate_scale=1.0))
    server.close()
    return out


# ---------------------------------------------------------------- our arm

def run_ours(args):
    import torch
    import torch.distributed as dist

    import paper_2402_00675_gb300 as mg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    mg.build()
    L = mg.lib()
    device_int_peaks(read_measured_peaks())

    inputs = make_inputs()
    dev_in = {}
    for N in MODULI:
        dev_in[N] = tuple(torch.from_numpy(x).cuda() for x in inputs[N])
    ctxs, outs, calls = {}, {}, []
    stream = torch.cuda.current_stream()
    sptr = stream.cuda_stream
    for N in MODULI:
        da, db, dau, dbu = dev_in[N]
        for variant, l in COMBOS:
            ctx = mg.mont_ctx_create(N, l, variant, alpha=ALPHA)
            ctxs[(N, variant)] = ctx
            out = torch.empty(N_PAIRS, dtype=torch.uint32 if variant == 2 else torch.int32,
                              device="cuda")
            outs[(N, variant)] = out
            x, y = (dau, dbu) if variant == 2 else (da, db)
            calls.append(((N, variant), ctx.handle, x.data_ptr(), y.data_ptr(), out.data_ptr()))

    def step(evs=None, k=0):
        for j, (_, h, xp, yp, op) in enumerate(calls):
            if evs is not None:
                evs[k][j][0].record(stream)
            st = L.mont_mul(h, xp, yp, op, N_PAIRS, sptr)
            if st:
                raise mg.MontError(st, "mont_mul")
            if evs is not None:
                evs[k][j][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    K = args.steps
    evs = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            for _ in calls] for _ in range(K)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start.record(stream)
    for k in range(K):
        step(evs, k)
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    elapsed_ms = max_over_ranks(t_start.elapsed_time(t_end), world)

    per_launch = [[evs[k][j][0].elapsed_time(evs[k][j][1]) for k in range(K)]
                  for j in range(len(calls))]
    all_launch_ms = [x for row in per_launch for x in row]
    avg_launch_ms = sum(all_launch_ms) / len(all_launch_ms)
    per_variant = {}
    for j, ((N, variant), *_rest) in enumerate(calls):
        ms = sum(per_launch[j]) / K
        per_variant[f"{VARIANT_NAMES[variant]}_N{N}"] = round(N_PAIRS / (ms * 1e-3) / 1e9, 2)

    modmuls_per_step = N_PAIRS * len(calls)
    value = whole_job_rate(modmuls_per_step * K, world, elapsed_ms)

    # ---------------- end to end: pinned host operands in, products out
    e2e_steps = args.e2e_steps or min(K, 10)
    host_in = {N: tuple(torch.from_numpy(x).pin_memory() for x in inputs[N]) for N in MODULI}
    host_out = {key: torch.empty(N_PAIRS, dtype=outs[key].dtype).pin_memory() for key in outs}
    h2d = sum(t.numel() * t.element_size() for N in MODULI for t in host_in[N])
    d2h = sum(t.numel() * t.element_size() for t in host_out.values())

    # The e2e step is one call of the library's host-buffer entry point
    # (mont_pipe_run): the 8 products of the device-resident step on the
    # pinned host operands.  The pipe copies each distinct input chunk in
    # once, runs the 8 mont_mul launches on the chunk and copies the 8 result
    # chunks out, overlapping both copy directions and the kernels.
    keys = list(outs.keys())
    pipe = mg.mont_pipe_create(E2E_STAGING_BYTES)
    e2e_ops = []
    for (N, variant) in keys:
        ha, hb, hau, hbu = host_in[N]
        x, y = (hau, hbu) if variant == 2 else (ha, hb)
        e2e_ops.append((ctxs[(N, variant)], mg.MONT_OP_MUL, x, y, host_out[(N, variant)]))
    e2e_chunk, e2e_distinct = pipe.plan(e2e_ops)

    def e2e_step():
        pipe.run(e2e_ops, stream)

    def link_now():
        lk = measure_link(host_in[MODULI[0]][0], dev_in[MODULI[0]][0],
                          host_out[keys[0]], outs[keys[0]], stream)
        # each product moves 4 bytes in and 4 bytes out: the link's two-way rate / 4
        lk["ceiling_gmodmul_s"] = round(lk["both_each_gbs"] / 4, 2)
        return lk

    # the host link is shared with other jobs on this host: measured right
    # before and right after the leg
    link_before = link_now()
    host_out[keys[0]].zero_()   # the leg's own copies must write it again
    e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(stream)
    torch.cuda.synchronize()
    # the results arrived: check a sample of every output against the
    # device-resident step's products
    for key in keys:
        idx = torch.randint(0, N_PAIRS, (4096,))
        h = host_out[key].view(torch.int32)
        d = outs[key].view(torch.int32)
        assert torch.equal(h[idx], d[idx.cuda()].cpu()), key
    pipe.close()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), world)
    e2e_value = whole_job_rate(modmuls_per_step * e2e_steps, world, e2e_ms)
    link = {"before": link_before, "after": link_now()}

    # ---------------- roofline of the dominant kernel (the word kernel)
    peaks = read_measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    achieved = BYTES_PER_MODMUL * N_PAIRS / (avg_launch_ms * 1e-3) / 1e9

    extras = None
    if world == 1 and not args.no_extras:
        extras = {
            "redc32_2p20": extra_redc32(mg, stream, peak),
            "rns64_batched": extra_rns64(mg, stream, peak),
            "cios": extra_cios(mg, stream, peak),
            "limb_variants": extra_limb_variants(mg, stream, peak),
            "sweep_r16": extra_sweep(mg, stream),
            "ntt": extra_ntt(mg, stream, peak),
            "dot_lazy": extra_dot(mg, stream, peak),
            "rns_convert": extra_rns(mg, stream),
        }
        extras["serving"] = extra_serving(mg, args.serving_jobs, stream, peak)

    result = None
    if rank == 0:
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            cores = os.cpu_count() or 1
            cpu = oracle_baseline(inputs, max(1.5, args.cpu_work_s / cores))
        roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak,
                "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": NCU_TRAFFIC_BYTES_PER_LAUNCH,
                "peak_source": f"{peak_src} hbm_gbs (copy bandwidth)",
                "kernel": "word_kernel (mont_mul, 32-bit words)",
                "avg_launch_us": round(avg_launch_ms * 1e3, 2),
                "algorithmic_bytes_per_launch": BYTES_PER_MODMUL * N_PAIRS}
        result = {
            "metric": METRIC, "value": round(value, 3), "unit": METRIC, "n_gpus": world,
            "steps": K, "warmup": args.warmup, "ms_per_step": round(elapsed_ms / K, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/i32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "pairs_per_modulus": N_PAIRS, "moduli": list(MODULI),
                       "launches_per_step": len(calls), "parallelism": f"replicas x{world}",
                       "l2": "no flush: every operand array is 256 MiB, larger than the 129 MB L2"},
            "e2e": {"value": round(e2e_value, 3), "unit": METRIC, "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "steps": e2e_steps, "link": link,
                    "path": f"mont_pipe_run, one call per step: {e2e_distinct} distinct pinned "
                            f"inputs copied in once, 8 outputs copied out, chunks of "
                            f"{e2e_chunk} elements"},
            "gpu_launches": len(calls) * K,
            "roofline": roof,
            "per_variant_gmodmul_s": per_variant,
            "clocks": clk,
            "cpu_baseline": cpu,
            "int_peaks": {"sms": PEAKS["sms"], "sm_mhz_max": PEAKS["sm_mhz_max"],
                          "limb_t_s": round(PEAKS["limb"] / 1e12, 3),
                          "issue_t_s": round(PEAKS["issue"] / 1e12, 2)},
            "extras": extras,
        }
        # last key, so that it survives a reader that keeps only the tail
        result["configs"] = config_summary(round(value, 1), roof, extras)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return result


def config_summary(value, roof, ex):
    """One compact entry per workload at its stated size: throughput and
    roofline fraction (of measured HBM, of the derived limb-product peak, or
    of the measured mad.lo rate / 3 for the sweep)."""
    c = {"2_word32_2p26": {"gmodmul_s": value, "frac_hbm": roof["frac"]}}
    if not ex:
        return c
    r = ex["redc32_2p20"]
    c["1_redc32_2p20"] = {"gmodmul_s_hot": r["hot_l2"], "gmodmul_s_cold": r["cold_l2"],
                          "graph_hot_cold": [r["graph_replay"].get("hot_l2"),
                                             r["graph_replay"].get("cold_l2")],
                          "frac_hbm_cold_graph": r["graph_replay"].get("frac_hbm_cold"),
                          "frac_hbm_cold": r["roofline"]["frac"]}
    b = ex["rns64_batched"]
    c["3_rns64_batch"] = {"gmodmul_s": b["batched_graph"], "frac_hbm": b["roofline"]["frac"],
                          "plain_gmodmul_s": b["plain_32_launches"], "speedup": b["speedup"],
                          "tuned": b["shape_tuned"]}
    c["4a_cios"] = {k.rstrip("b"): [v["gmodmul_s"], v["roofline"]["frac"]]
                    for k, v in ex["cios"].items()}
    sw = ex["sweep_r16"]
    c["4b_sweep_r16"] = {k.replace("_own_domain", ""): [v["gchecks_s"], v["roofline"]["frac"]]
                         for k, v in sw.items() if k.endswith("_own_domain")}
    sv = ex["serving"]
    c["5_serving"] = {"cap_jobs_s": round(sv["capacity"]["jobs_per_s"], 1),
                      "cap_frac_of_bound": sv.get("capacity_frac_of_bound"),
                      "gmodmul_s": round(sv["capacity"]["gmodmul_s"], 2),
                      "p50_p99_ms_0.5": [round(sv["load_0.5"]["p50_ms"], 1),
                                         round(sv["load_0.5"]["p99_ms"], 1)],
                      "modmul_p50_p99_ms_0.5": [round(sv["load_0.5"]["modmul_p50_ms"], 1),
                                                round(sv["load_0.5"]["modmul_p99_ms"], 1)],
                      "p50_p99_ms_0.8": [round(sv["load_0.8"]["p50_ms"], 1),
                                         round(sv["load_0.8"]["p99_ms"], 1)]}
    lv = ex["limb_variants"]
    nt = ex["ntt"]
    rc = ex["rns_convert"]["roofline"]
    c["next"] = {
        "ntt256_w32_plantard_mul_issue_hbm": [nt["n256_w32_plantard"]["roofline"][k]
                                              for k in ("frac", "issue_frac", "hbm_frac")],
        "ntt1024_w64_plantard_mul_issue_hbm": [nt["n1024_w64_plantard"]["roofline"][k]
                                               for k in ("frac", "issue_frac", "hbm_frac")],
        "dot_lazy_hbm": ex["dot_lazy"]["roofline"]["frac"],
        "rns_to_from": [rc["frac_to"], rc["frac_from"]],
        "alg1to4": {w: [min(v["roofline"]["frac"] for k, v in lv.items() if k.startswith(w)),
                        max(v["roofline"]["frac"] for k, v in lv.items() if k.startswith(w))]
                    for w in ("256b", "1024b", "2048b")}}
    return c


# ---------------------------------------------------------------- reference arm

def run_reference(args):
    """The CPU oracle as the reference arm, on every host core (one spawned
    process each, each over its own disjoint pairs of the 8 vectors): each
    step evaluates a bounded sample of the same workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return None
    inputs = make_inputs()
    cores, model = host_cpu()
    pool = OraclePool(inputs, cores)
    # size a step so that warmup + steps take about a minute in total
    probe_rate, _, _ = pool.budget(0.5)
    per_step_s = 60.0 / max(1, args.steps + args.warmup)
    per = max(1, int(per_step_s * probe_rate / (8 * pool.cores)))
    for _ in range(args.warmup):
        pool.count(per)
    t0 = time.perf_counter()
    done = 0
    for _ in range(args.steps):
        done += pool.count(per)
    secs = time.perf_counter() - t0
    pool.close()
    value = done / secs / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": secs / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32/i32",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "pairs_per_modulus": N_PAIRS, "moduli": list(MODULI),
                   "sample_pairs_per_vector_per_step_per_core": per},
        "cpu_baseline": {"value": value, "unit": METRIC, "cores": pool.cores, "kind": "oracle",
                         "cpu": model,
                         "sample": f"{pool.cores} spawned processes (one per host core), each "
                                   f"evaluating {per} of its own disjoint pairs of each of the 8 "
                                   "(modulus, variant) vectors per step, Python big-int"},
        "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def run_extras_only(names):
    import torch
    import paper_2402_00675_gb300 as mg
    mg.build()
    peaks = read_measured_peaks()
    device_int_peaks(peaks)
    peak = peaks.get("hbm_gbs") or 6800.0
    stream = torch.cuda.current_stream()
    table = {"redc32_2p20": extra_redc32, "rns64_batched": extra_rns64, "cios": extra_cios,
             "limb_variants": extra_limb_variants, "sweep_r16": extra_sweep, "ntt": extra_ntt,
             "dot_lazy": extra_dot, "rns_convert": extra_rns}
    out = {}
    for name in names:
        if name == "serving":
            out[name] = extra_serving(mg, 10000, stream, peak)
            continue
        fn = table[name]
        out[name] = fn(mg, stream, peak) if fn.__code__.co_argcount == 3 else fn(mg, stream)
    return {"extras": out}


def main():
    args = parse_args()
    if args.extra:
        print(json.dumps(run_extras_only(args.extra)), flush=True)
        return
    res = run_reference(args) if args.impl == "reference" else run_ours(args)
    if res is not None:
        print(json.dumps(res), flush=True)


if __name__ == "__main__":
    main()
