"""Open-loop load generator for the serving loop (``Server``).

Requests arrive at the times of a Poisson stream (``inputs.serving_stream``);
each is submitted when its arrival time comes, whatever is still running, and
results are collected as they finish.  Latency is the server's own
submission-to-result time of each request.  Sources are drawn from a small
pool per (cells, rule) that stays on the device, and each request writes its
own output buffer, recycled once the request is done, so that memory stays
bounded at any arrival rate; requests the server refuses because its queue is
full are counted, not retried.
"""
from __future__ import annotations

import time

import numpy as np

from . import MGError, Server, inputs

BUSY = 7


class SourcePool:
    """``per_key`` device sources for every (n, bc) of the stream."""

    def __init__(self, sizes=inputs.SERVE_SIZES, bcs=inputs.SERVE_BCS, per_key=2, seed=20230227,
                 device="cuda"):
        self.src = {}
        for n in sizes:
            for bc in bcs:
                self.src[(n, bc)] = [
                    inputs.serving_source(dict(n=n, bc=bc, seed=seed + 7919 * k + 31 * n + bc,
                                               n_blobs=1 + (k * 3 + n) % 8), device)
                    for k in range(per_key)]
        self.free = {}
        self.device = device

    def rho(self, req):
        lst = self.src[(req["n"], req["bc"])]
        return lst[req["seed"] % len(lst)]

    def take_phi(self, n):
        import torch
        lst = self.free.setdefault(n, [])
        if lst:
            return lst.pop()
        return torch.empty((n, n, n), dtype=torch.float64, device=self.device)

    def give_phi(self, phi):
        self.free.setdefault(phi.shape[0], []).append(phi)


def run_stream(server: Server, stream, pool: SourcePool, four_pi_G: float = 1.0):
    """Submit ``stream`` (list of request dicts with arrival time ``t``) in real
    time; return per-request records and the wall time of the whole run."""
    outstanding = {}  # ticket -> (request, phi)
    records, busy = [], 0
    t0 = time.perf_counter()

    def collect(block=False):
        for tk in list(outstanding):
            res, hist = server.wait(tk, 600.0) if block else server.poll(tk)
            if res.done:
                req, phi = outstanding.pop(tk)
                pool.give_phi(phi)
                records.append(dict(n=req["n"], bc=req["bc"], tol=req["tol"], status=res.status,
                                    total_ms=res.total_ms, queue_ms=res.queue_ms,
                                    solve_ms=res.solve_ms, cycles=len(hist),
                                    final=float(hist[-1]) if len(hist) else float("nan")))

    for req in stream:
        while True:
            now = time.perf_counter() - t0
            if now >= req["t"]:
                break
            collect()
            if req["t"] - (time.perf_counter() - t0) > 2e-4:
                time.sleep(1e-4)
        phi = pool.take_phi(req["n"])
        try:
            tk = server.submit(pool.rho(req), phi, bc=req["bc"], four_pi_G=four_pi_G,
                               tol=req["tol"], lmax=req["lmax"])
        except MGError as e:
            pool.give_phi(phi)
            if e.status != BUSY:
                raise
            busy += 1
            continue
        outstanding[tk] = (req, phi)
    collect(block=True)
    wall = time.perf_counter() - t0
    return records, busy, wall


def summarize(records, busy, wall, rate, duration):
    lat = np.array([r["total_ms"] for r in records]) if records else np.zeros(1)
    cells = sum(r["n"] ** 3 for r in records)
    ok = sum(1 for r in records if r["status"] == 0)
    return dict(rate=rate, duration_s=duration, offered=len(records) + busy,
                completed=len(records), converged=ok, rejected_busy=busy,
                p50_ms=float(np.percentile(lat, 50)), p99_ms=float(np.percentile(lat, 99)),
                mean_ms=float(lat.mean()), cells_per_s=cells / wall, wall_s=wall)
