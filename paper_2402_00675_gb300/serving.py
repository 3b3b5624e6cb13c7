"""Driver for the serving loop (mont_server_*): a request stream with Poisson
arrivals replayed against a Server, with per-job latency and aggregate
throughput.

The native server does the scheduling (admission by device memory, worker
slots, bounded waits); this module only feeds it: it keeps one pinned host
operand pool per (variant, word width) large enough for the longest job,
gives every job a slice of its pool as operands and a region of a pinned
output ring, submits each job at its arrival time, and reads the server's
own timestamps back.  Operand pools hold valid residues (uniform in the
variant's input range); a job's operands are the first `length` elements of
its pool.
"""

from __future__ import annotations

import time
from dataclasses import dataclass

import numpy as np
import torch

from . import (MONT_ETIMEOUT, MONT_PLANTARD, MONT_REDC, MONT_SIGNED, Server, mont_ctx_create)

_ELEM_BYTES = {32: 4, 64: 8, 256: 32}


@dataclass
class Contexts:
    """Resident contexts of the serving workload, one per (variant, width)."""

    by_key: dict
    moduli: dict

    @staticmethod
    def create(N32: int, N64: int, N256: int) -> "Contexts":
        by, mod = {}, {}
        for v in (MONT_REDC, MONT_SIGNED, MONT_PLANTARD):
            by[(v, 32)] = mont_ctx_create(N32, 64 if v == MONT_PLANTARD else 32, v)
            by[(v, 64)] = mont_ctx_create(N64, 128 if v == MONT_PLANTARD else 64, v)
            mod[(v, 32)], mod[(v, 64)] = N32, N64
        by[(MONT_REDC, 256)] = mont_ctx_create(N256, 256, MONT_REDC)
        mod[(MONT_REDC, 256)] = N256
        return Contexts(by, mod)


class Pools:
    """Pinned host operand pools (a and b) per (variant, width)."""

    def __init__(self, ctxs: Contexts, max_len: int, seed: int = 5):
        import synthetic as sy
        self.max_len = max_len
        self.pools = {}
        for (v, w), N in ctxs.moduli.items():
            s = seed * 100 + v * 10 + w
            if w == 256:
                a = sy.bounded_limb_residues(N, 8, max_len, s).reshape(-1)
                b = sy.bounded_limb_residues(N, 8, max_len, s + 1).reshape(-1)
            elif v == MONT_SIGNED:
                dt = np.int32 if w == 32 else np.int64
                a = sy.centred_residues(N, max_len, s, dtype=dt)
                b = sy.centred_residues(N, max_len, s + 1, dtype=dt)
            else:
                dt = np.uint32 if w == 32 else np.uint64
                a = sy.uniform_residues(N, max_len, s, dtype=dt)
                b = sy.uniform_residues(N, max_len, s + 1, dtype=dt)
            self.pools[(v, w)] = (torch.from_numpy(a).pin_memory(),
                                  torch.from_numpy(b).pin_memory())


class OutputRing:
    """Pinned byte ring handing out contiguous output regions in order."""

    def __init__(self, nbytes: int):
        self.buf = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
        self.size = nbytes
        self.head = 0
        self.live = []  # (job id, start, end) in allocation order

    def take(self, nbytes: int, retire):
        """A region of nbytes; `retire(job_id)` is called on the oldest live
        jobs until the region is free."""
        if nbytes > self.size:
            raise ValueError("output larger than the ring")
        start = self.head if self.head + nbytes <= self.size else 0
        end = start + nbytes
        while self.live and self._overlaps(start, end):
            retire(self.live[0][0])
        self.head = end
        return start, self.buf[start:end]

    def _overlaps(self, start, end):
        return any(s < end and start < e for _, s, e in self.live)

    def add(self, jid, start, nbytes):
        self.live.append((jid, start, start + nbytes))

    def drop(self, jid):
        self.live = [x for x in self.live if x[0] != jid]


def run_stream(server: Server, jobs, ctxs: Contexts, pools: Pools, ring: OutputRing,
               rate_scale: float = 1.0, sweep_cex_cap: int = 64):
    """Replay `jobs` (synthetic.Job list; arrival times multiplied by
    rate_scale, 0 = all at once) and return per-job records and totals."""
    results = {}
    ids = []
    info = {}
    ring.live = []   # every job of an earlier stream has been waited for

    def retire(jid):
        r = server.wait(jid)
        results[jid] = r
        if r["status"] == MONT_ETIMEOUT:   # the device may still write its region
            while server.job_busy(jid):
                time.sleep(0.001)
        ring.drop(jid)

    t0 = time.perf_counter()
    for job in jobs:
        target = t0 + job.arrival_s * rate_scale
        now = time.perf_counter()
        if target > now:
            time.sleep(target - now)
        if job.kind == "sweep":
            jid = server.submit_sweep(job.variant, 16, 0, job.n_lo, job.n_lo + 2 * (job.length - 1),
                                      cex_cap=sweep_cex_cap)
            info[jid] = ("sweep", 0)
        else:
            key = (job.variant, job.width)
            n = min(job.length, pools.max_len)
            a, b = pools.pools[key]
            eb = _ELEM_BYTES[job.width]
            start, region = ring.take(n * eb, retire)
            jid = server.submit_modmul(ctxs.by_key[key], a[: n * (eb // a.element_size())],
                                       b[: n * (eb // b.element_size())], region, n=n)
            ring.add(jid, start, n * eb)
            info[jid] = ("modmul", n)
        ids.append(jid)
    for jid in ids:
        if jid not in results:
            retire(jid)
    recs = []
    for jid in ids:
        r = results[jid]
        kind, n = info[jid]
        recs.append(dict(kind=kind, n=n, status=r["status"], t_submit=r["t_submit"],
                         t_admit=r["t_admit"], t_done=r["t_done"]))
    return recs


def _percentiles(lat_ms):
    if len(lat_ms) == 0:
        return None, None
    return float(np.percentile(lat_ms, 50)), float(np.percentile(lat_ms, 99))


def summarise(recs) -> dict:
    """p50 / p99 latency (submission to results in host memory), for all jobs
    and for modmul and sweep jobs apart, and throughput."""
    lat = np.array([r["t_done"] - r["t_submit"] for r in recs]) * 1e3
    kinds = np.array([r["kind"] for r in recs])
    t_first = min(r["t_submit"] for r in recs)
    t_last = max(r["t_done"] for r in recs)
    modmuls = sum(r["n"] for r in recs if r["kind"] == "modmul")
    ok = sum(1 for r in recs if r["status"] == 0)
    p50, p99 = _percentiles(lat)
    m50, m99 = _percentiles(lat[kinds == "modmul"])
    s50, s99 = _percentiles(lat[kinds == "sweep"])
    return {
        "jobs": len(recs), "ok": ok,
        "sweep_jobs": int((kinds == "sweep").sum()),
        "p50_ms": p50, "p99_ms": p99,
        "modmul_p50_ms": m50, "modmul_p99_ms": m99,
        "sweep_p50_ms": s50, "sweep_p99_ms": s99,
        "mean_ms": float(lat.mean()), "makespan_s": t_last - t_first,
        "gmodmul_s": modmuls / (t_last - t_first) / 1e9,
        "jobs_per_s": len(recs) / (t_last - t_first),
    }


def sweep_checks(variant: int, log2R: int, n_lo: int, count: int) -> int:
    """(N, T) checks of a sweep job over `count` consecutive odd N from n_lo,
    each algorithm on its own domain (moduli outside its condition skipped):
    REDC R N; Algorithm 1 N R - 1 (|T| < N R / 2); Algorithm 2 N^2 + 1 for
    N < 2^n / phi, n = log2R / 2."""
    R = 1 << log2R
    n = log2R // 2
    total = 0
    for i in range(count):
        N = n_lo + 2 * i
        if variant == MONT_REDC and N < R:
            total += R * N
        elif variant == MONT_SIGNED and 2 * N < R:
            total += N * R - 1
        elif variant == MONT_PLANTARD:
            d = (1 << (n + 1)) - N
            if d > 0 and 5 * N * N < d * d:
                total += N * N + 1
    return total


def stream_bound(jobs, sweep_rate: dict, link_gbs: float, hbm_gbs: float,
                 max_len: int) -> dict:
    """A lower bound on the time the device needs for a job stream: the sweep
    jobs' checks at the sweep's measured rates (checks/s per variant) plus the
    modmul kernels' bytes at the HBM rate, against the host link moving every
    modmul operand in and every product out (link_gbs each way, both
    directions at once).  The copies overlap the kernels, so the bound is the
    larger of the two."""
    sweep_s = 0.0
    kernel_s = 0.0
    bytes_in = bytes_out = 0
    for j in jobs:
        if j.kind == "sweep":
            sweep_s += sweep_checks(j.variant, 16, j.n_lo, j.length) / sweep_rate[j.variant]
        else:
            n = min(j.length, max_len)
            eb = _ELEM_BYTES[j.width]
            bytes_in += 2 * n * eb
            bytes_out += n * eb
            kernel_s += 3 * n * eb / (hbm_gbs * 1e9)
    link_s = max(bytes_in, bytes_out) / (link_gbs * 1e9)
    device_s = sweep_s + kernel_s
    bound_s = max(device_s, link_s)
    return {"sweep_device_s": round(sweep_s, 3), "modmul_kernel_s": round(kernel_s, 4),
            "link_s": round(link_s, 3), "bound_s": round(bound_s, 3),
            "jobs_per_s_bound": round(len(jobs) / bound_s, 1)}
