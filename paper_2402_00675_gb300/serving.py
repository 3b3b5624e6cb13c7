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

from . import (MONT_PLANTARD, MONT_REDC, MONT_SIGNED, Server, mont_ctx_create)

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
            results[jid] = server.wait(jid)
            ring.drop(jid)
    recs = []
    for jid in ids:
        r = results[jid]
        kind, n = info[jid]
        recs.append(dict(kind=kind, n=n, status=r["status"], t_submit=r["t_submit"],
                         t_admit=r["t_admit"], t_done=r["t_done"]))
    return recs


def summarise(recs) -> dict:
    """p50 / p99 latency (submission to results in host memory) and throughput."""
    lat = np.array([r["t_done"] - r["t_submit"] for r in recs]) * 1e3
    t_first = min(r["t_submit"] for r in recs)
    t_last = max(r["t_done"] for r in recs)
    modmuls = sum(r["n"] for r in recs if r["kind"] == "modmul")
    ok = sum(1 for r in recs if r["status"] == 0)
    return {
        "jobs": len(recs), "ok": ok,
        "sweep_jobs": sum(1 for r in recs if r["kind"] == "sweep"),
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "mean_ms": float(lat.mean()), "makespan_s": t_last - t_first,
        "gmodmul_s": modmuls / (t_last - t_first) / 1e9,
        "jobs_per_s": len(recs) / (t_last - t_first),
    }
