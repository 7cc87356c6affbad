"""Benchmark: cells solved per second to ||d||/||f|| < 1e-10 on the 512^3
periodic Gaussian-blob workload (FMG + V(1,1) cycles; FP32 multigrid inside
FP64 defect correction), one solve per step, on one GB300 per rank.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  Under torchrun each rank solves its own grid (the solve
does not shard: replicas), and value is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "cells solved/s to ||r||/||f||<1e-10 (512^3)"
UNIT = "cells/s"
TOL = 1e-10
SEED = 20230227

# Algorithmic bytes per finest cell of one launch of each kernel class, by
# the width w of the level precision: the least data
# that launch must move.
def algorithmic_bytes_per_cell(kernel: str, w: int, fixed_point: bool = True) -> float:
    return {
        "sor": 2.0 * w,                 # read u, read f (own colour), write u (own colour)
        "defect_restrict": 2.0 * w + w / 8.0,
        "prolong": 2.0 * w + w / 8.0,   # read u, coarse e; write u
        "fmg_prolong": w + w / 8.0,
        "defect_norm": 16.0,            # FP64 u, f
        # fixed-point outer step: int64 phi, F and FP32 e in; int64 phi, FP32 r out;
        # the plain FP64 residual: FP64 u, f in, FP32 r out
        "outer_residual": 32.0 if fixed_point else 20.0,
        "correct": 20.0,                # FP64 u, FP32 e -> FP64 u
        # FP64 rho -> FP64 f; on the mixed path's fixed-point start only the
        # pass over rho for its sum and maximum (read rho)
        "source": 8.0 if fixed_point else 16.0,
        "fused_down": 3.0 * w + w / 8.0,  # read u, f; write u, coarse f
        "fused_down0": 2.0 * w + w / 8.0,  # from a zero start: read f; write u, coarse f
        "fused_up": 3.0 * w + w / 8.0,    # read u, coarse e, f; write u
        # the up leg of one V-cycle and the down leg of the next in one pass:
        # read u, f, coarse e; write u, coarse f
        "fused_updown": 3.0 * w + w / 4.0,
        "gravity": 32.0,                  # int64 phi in; FP64 phi and 3 FP64 g out (fixed point)
    }[kernel]


FP32_CLASSES = {"sor", "defect_restrict", "prolong", "fmg_prolong", "fused_down", "fused_down0",
                "fused_up", "fused_updown"}


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# Sources that define each kernel class (its device program and launcher, and
# the headers they include); a traffic figure applies while these are unchanged.
KERNEL_SOURCES = {
    "fused_up": ["mg_fused.cuh", "mg_fused_launch.cuh", "mg_fused.cu", "mg_internal.h"],
    "fused_down": ["mg_fused.cuh", "mg_fused_launch.cuh", "mg_fused.cu", "mg_internal.h"],
    "fused_down0": ["mg_fused.cuh", "mg_fused_launch.cuh", "mg_fused.cu", "mg_internal.h"],
    # the down legs with tensor copies
    "fused_down_tma": ["mg_fused.cuh", "mg_fused_tma.cu", "mg_internal.h"],
    "fused_down0_tma": ["mg_fused.cuh", "mg_fused_tma.cu", "mg_internal.h"],
    "fused_up_tma": ["mg_fused.cuh", "mg_fused_tma.cu", "mg_internal.h"],
    "outer_residual": ["mg_fixed.cu", "mg_convert.cuh", "mg_device.cuh", "mg_internal.h"],
}


NOMINAL_HBM_GBS = 7900.0  # nominal HBM3e bandwidth of the part, for context


def mixed_solve_bytes_per_cell(outer: int, inner: int, paired: bool = True) -> float:
    """Algorithmic bytes per finest cell of one mixed solve: per outer iteration
    `inner` FP32 V(1,1) cycles (the first from a zero correction: its down leg
    reads f only, 2w + w/8; the others 3w + w/8; every up leg 3w + w/8; coarse
    levels add 1/7 of the zero-start legs' bytes) and one fixed-point outer step
    (32 B: int64 phi, F and FP32 e in, int64 phi and FP32 r out; the first, from
    phi = 0, 24 B); plus the passes around the loop: rho read three times (mean
    and maximum, first residual, integer h^2 f), r32 and the integer f written, e
    read once for its maximum, phi converted back (read and write): 56 B.
    paired: on the finest level the up leg of each cycle but the last and the
    down leg of the next are one pass (3w + w/4)."""
    w = 4.0
    leg0, leg, ud = 2 * w + w / 8, 3 * w + w / 8, 3 * w + w / 4
    if paired:
        finest = leg0 + (inner - 1) * ud + leg
    else:
        finest = (leg0 + leg) + (inner - 1) * (2 * leg)
    coarse = inner * (leg0 + leg) / 7.0
    steps = 24.0 + 32.0 * (outer - 1)
    return outer * (finest + coarse) + steps + 56.0


def src_sha(kernel: str = None) -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_2302_13903_gb300", "csrc")
    names = KERNEL_SOURCES.get(kernel) or sorted(os.listdir(d))
    for fn in names:
        h.update(open(os.path.join(d, fn), "rb").read())
    return h.hexdigest()[:12]


def ncu_traffic(kernel: str, prec: str, n: int):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    sha = src_sha(kernel)
    best = None
    for line in open(p):
        f = line.split()
        if len(f) != 6 or f[0].startswith("#"):
            continue
        k, pr, nn, cells_captured, bytes_per_launch, s = f
        if k == kernel and pr == prec and s == sha:
            scale = n ** 3 / float(cells_captured)  # traffic grows with the cells of a launch
            best = float(bytes_per_launch) * scale
    return best


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    def __init__(self, gpu_index: int):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            if len(r) < 9:
                continue
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
            except ValueError:
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def near_cpus(gpu_index: int) -> dict:
    """The GPU's PCI address, its local CPUs and NUMA node (sysfs), for placing
    page-locked host buffers next to it."""
    out = {}
    try:
        bus = subprocess.run(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=pci.bus_id",
                              "--format=csv,noheader"], capture_output=True, text=True,
                             timeout=30).stdout.strip()
        dom, rest = bus.lower().split(":", 1)
        path = f"/sys/bus/pci/devices/{dom[-4:]}:{rest}"
        out["pci"] = f"{dom[-4:]}:{rest}"
        out["numa_node"] = int(open(os.path.join(path, "numa_node")).read().strip())
        cpus = set()
        for part in open(os.path.join(path, "local_cpulist")).read().strip().split(","):
            a, _, b = part.partition("-")
            cpus.update(range(int(a), int(b or a) + 1))
        out["local_cpus"] = sorted(cpus)
        out["local_cpus_text"] = open(os.path.join(path, "local_cpulist")).read().strip()
    except Exception as e:  # not fatal: the buffers are then placed by the default policy
        out["error"] = str(e)[:200]
    return out


def pages_by_node(ptr: int) -> dict:
    """Pages per NUMA node of the mapping that holds address ptr
    (/proc/self/numa_maps)."""
    best, line_best = -1, None
    try:
        for line in open("/proc/self/numa_maps"):
            start = int(line.split()[0], 16)
            if start <= ptr and start > best:
                best, line_best = start, line
    except Exception:
        return {}
    if line_best is None:
        return {}
    return {f[1:].split("=")[0]: int(f.split("=")[1]) for f in line_best.split()
            if f.startswith("N") and "=" in f}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def oracle_solve_timed(n: int, threads: int):
    import oracle
    from paper_2302_13903_gb300 import inputs
    oracle.build()
    oracle.set_num_threads(threads)
    rho = inputs.gaussian_blobs(n, 64, seed=SEED)
    t = time.perf_counter()
    r = oracle.solve(rho, 1.0 / n, oracle.PERIODIC, tol=TOL, four_pi_G=1.0)
    dt = time.perf_counter() - t
    assert r.ok, r.hist
    return dt, len(r.hist)


def cpu_baseline(n_sample: int):
    threads = os.cpu_count() or 1
    dt, cycles = oracle_solve_timed(n_sample, threads)
    # the same recipe on one core, at half the size (an eighth of the cells)
    n1 = max(n_sample // 2, 8)
    dt1, cycles1 = oracle_solve_timed(n1, 1)
    oracle_threads(threads)
    return {"value": n_sample ** 3 / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"one oracle solve of the same recipe at {n_sample}^3 (64 blobs, seed {SEED}), "
                      f"FMG + V(1,1) to 1e-10 ({cycles} residual checks), {dt:.2f} s wall",
            "single_core": {"value": n1 ** 3 / dt1, "unit": UNIT, "cores": 1,
                            "sample": f"one oracle solve at {n1}^3 ({cycles1} residual checks), "
                                      f"{dt1:.2f} s"}}


def oracle_threads(threads: int):
    import oracle
    oracle.set_num_threads(threads)


def run_reference(args, ws, rank):
    if rank != 0:
        return
    n_sample = args.cpu_n
    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle_solve_timed(n_sample, threads)
    times = []
    for _ in range(args.steps):
        dt, cycles = oracle_solve_timed(n_sample, threads)
        times.append(dt)
    tot = sum(times)
    value = n_sample ** 3 * len(times) / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{n_sample}^3 periodic Gaussian blobs (64, seed {SEED}), FP64 "
                               f"FMG + V(1,1) to 1e-10 on the host cores (bounded sample of the "
                               f"512^3 workload)", "n": n_sample, "bc": "periodic", "tol": TOL},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": f"{n_sample}^3 instance of the same recipe, one solve per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_open_sphere(args, stream):
    """256^3 uniform sphere (R = 0.25, 10^3 sub-cells) on [-0.5, 0.5]^3 with open
    boundaries (multipoles to l = 4 about the centre of mass), 4 pi G = 4 pi, to
    1e-10 in FP64 and in mixed precision; error against the analytic potential."""
    import numpy as np
    import torch

    import paper_2302_13903_gb300 as mg
    from paper_2302_13903_gb300 import inputs
    n = 256
    rho_h = inputs.uniform_sphere(n, 0.25, 10)
    exact = inputs.sphere_potential(n, 0.25, G=1.0)
    rho = torch.from_numpy(rho_h).cuda()
    phi = torch.zeros_like(rho)
    out = {"workload": "256^3 uniform sphere R = 0.25 (cell-averaged, 10^3 sub-cells), open "
                       "boundaries from multipoles to l = 4, 4 pi G = 4 pi, tol 1e-10"}
    for name, prec in (("fp64", mg.FP64), ("mixed", mg.MIXED)):
        with mg.Solver(n, 1.0 / n, mg.OPEN, prec=prec, lmax=4) as s:
            for _ in range(2):
                _, hist, st = s.solve(rho, 4 * math.pi, TOL, phi=phi, stream=stream)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.open_steps):
                _, hist, st = s.solve(rho, 4 * math.pi, TOL, phi=phi, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / args.open_steps
        p = phi.cpu().numpy()
        out[name] = {"ms_per_solve": ms, "value": n ** 3 / (ms * 1e-3), "unit": UNIT,
                     "status": st, "residual_checks": len(hist), "final_ratio": float(hist[-1]),
                     "max_rel_error_vs_analytic": float(np.abs(p - exact).max() /
                                                        np.abs(exact).max())}
    return out


def run_sinusoid(args, stream):
    """The 64^3 periodic sinusoid rho = sin 2 pi x sin 2 pi y sin 2 pi z with
    4 pi G = 1 (Sec. 4.1.1 test), FMG + V(1,1) to 1e-10, FP64 and mixed:
    latency of one solve, and the error against the exact discrete solution
    f / lambda, lambda = -(12 / h^2) sin^2(pi h)."""
    import numpy as np
    import torch

    import paper_2302_13903_gb300 as mg
    from paper_2302_13903_gb300 import inputs
    n = 64
    h = 1.0 / n
    rho_h = inputs.sinusoid(n)
    exact = rho_h / (-(12.0 / h ** 2) * math.sin(math.pi * h) ** 2)
    rho = torch.from_numpy(rho_h).cuda()
    phi = torch.zeros_like(rho)
    out = {"workload": "64^3 periodic sinusoid, 4 pi G = 1, FMG + V(1,1) to 1e-10"}
    for name, prec in (("fp64", mg.FP64), ("mixed", mg.MIXED)):
        with mg.Solver(n, h, mg.PERIODIC, prec=prec) as s:
            for _ in range(3):
                _, hist, st = s.solve(rho, 1.0, TOL, phi=phi, stream=stream)
            torch.cuda.synchronize()
            ts = []
            for _ in range(args.sin_steps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                _, hist, st = s.solve(rho, 1.0, TOL, phi=phi, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
        p = phi.cpu().numpy()
        ms = statistics.median(ts)
        out[name] = {"ms_per_solve_median": ms, "ms_p99": sorted(ts)[int(0.99 * (len(ts) - 1))],
                     "value": n ** 3 / (ms * 1e-3), "unit": UNIT, "status": st,
                     "residual_checks": len(hist), "final_ratio": float(hist[-1]),
                     "max_rel_error_vs_exact_discrete":
                         float(np.abs(p - exact).max() / np.abs(exact).max())}
    return out


def batch_roofline(specs, hists, phase_ms, inner_cycles, peak):
    """Algorithmic bytes of the batched solve's fused down and up phases (every
    level of 32^3 and up; levels below run in the single-CTA bottom phase),
    from each grid's own count of outer iterations, against their device
    time.  FP32 levels (w = 4): down leg 3w + w/8 (2w + w/8 from a zero
    start), up leg 3w + w/8."""
    w = 4.0
    down = up = 0.0
    for spec, hist in zip(specs, hists):
        n, outer = spec["n"], len(hist)
        levels = []
        m = n
        while m >= 32:
            levels.append(m)
            m //= 2
        if not levels:
            continue
        cycles = outer * (1 + inner_cycles)
        fin = levels[0] ** 3
        down += outer * ((2 * w + w / 8) + inner_cycles * (3 * w + w / 8)) * fin
        up += cycles * (3 * w + w / 8) * fin
        for m in levels[1:]:
            down += cycles * (2 * w + w / 8) * m ** 3
            up += cycles * (3 * w + w / 8) * m ** 3
    out = {}
    for name, b in (("down", down), ("up", up)):
        ms = phase_ms.get(name, 0.0)
        if ms > 0:
            gbs = b / (ms * 1e-3) / 1e9
            out[name] = {"algorithmic_bytes": b, "ms": ms, "achieved_gbs": gbs, "frac": gbs / peak}
    return out


def run_per_face(args, stream):
    """512^3 slab: periodic in x and y, phi = 0 on both z faces (a rule per
    face, Sec. 2.3.6), the headline's 64 blobs, to 1e-10 in FP64 and in mixed
    precision.  These grids run the per-level kernels with the face rules in
    their ghost synthesis and the FP64 outer residual."""
    import torch

    import paper_2302_13903_gb300 as mg
    from paper_2302_13903_gb300 import inputs
    n = args.n
    P, F = mg.PERIODIC, mg.FIXED
    kinds = [P, P, P, P, F, F]
    rho = inputs.gaussian_blobs(n, 64, seed=SEED, device="cuda")
    phi = torch.zeros_like(rho)
    out = {"workload": f"{n}^3 slab, periodic in x and y, phi = 0 on the z faces, 64 Gaussian "
                       f"blobs (seed {SEED}), tol 1e-10"}
    for name, prec in (("fp64", mg.FP64), ("mixed", mg.MIXED)):
        with mg.Solver(n, 1.0 / n, kinds, prec=prec) as s:
            for _ in range(2):
                _, hist, st = s.solve(rho, 1.0, TOL, phi=phi, stream=stream)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.face_steps):
                _, hist, st = s.solve(rho, 1.0, TOL, phi=phi, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / args.face_steps
        out[name] = {"ms_per_solve": ms, "value": n ** 3 / (ms * 1e-3), "unit": UNIT,
                     "status": st, "residual_checks": len(hist), "final_ratio": float(hist[-1])}
    return out


def run_batched(args, ws, rank, stream):
    """512 grids of {16,32,64,128}^3 (Zipf weights), mixed rules, one persistent
    graph-captured launch per solve; under torchrun each rank takes its LPT share."""
    import torch

    import paper_2302_13903_gb300 as mg
    from paper_2302_13903_gb300 import inputs
    from paper_2302_13903_gb300.sharding import max_over_ranks, partition_lpt
    specs = inputs.batch_specs(512)
    share = partition_lpt([s["n"] ** 3 for s in specs], ws)[rank]
    mine = [specs[i] for i in share]
    sizes = [s["n"] for s in mine]
    rhos = [inputs.batch_source(s, device="cuda") for s in mine]
    phis = [torch.zeros_like(r) for r in rhos]
    with mg.Batch(sizes, [1.0 / n for n in sizes], [s["bc"] for s in mine]) as b:
        for _ in range(max(args.warmup, 3)):
            st, hists, sts = b.solve(rhos, phis, 1.0, TOL, stream=stream)
        torch.cuda.synchronize()
        a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.batch_steps):
            st, hists, sts = b.solve(rhos, phis, 1.0, TOL, stream=stream)
        e.record(stream)
        torch.cuda.synchronize()
        ms = max_over_ranks(a.elapsed_time(e) / args.batch_steps)
        cells = b.cells
        graph = b.graph
        phases = {k: round(v, 3) for k, v in b.phase_ms().items() if v > 0}
        inner_cycles = b.opts.inner_cycles
    total = sum(s["n"] ** 3 for s in specs)
    peak, _ = peaks()
    roof = batch_roofline(mine, hists, phases, inner_cycles, peak)
    return {"grids": len(specs), "cells": total, "ms_per_solve": ms, "roofline": roof,
            "value": total / (ms * 1e-3), "unit": UNIT, "graph": graph,
            "converged": int(sum(1 for x in sts if x == 0)), "of": len(sts),
            "max_outer_iterations": max(len(h) for h in hists), "rank_cells": cells,
            "phase_ms": phases,
            "workload": "512 grids, sizes {16,32,64,128}^3 with Zipf 1/rank weights, rules "
                        "periodic / fixed 0 / zero gradient, 1-8 Gaussian blobs each; FP32 "
                        "multigrid inside FP64 defect correction to 1e-10; one persistent "
                        "cooperative launch captured as a CUDA graph"}


def run_serving(args):
    """Poisson arrivals of 32^3-256^3 requests with mixed rules (open with
    lmax 0-4), tol log-uniform in [1e-10, 1e-6], HBM budget half of free memory."""
    import torch

    import paper_2302_13903_gb300 as mg
    from paper_2302_13903_gb300 import inputs, serving
    free, _ = torch.cuda.mem_get_info()
    pool = serving.SourcePool()
    out = []
    with mg.Server(free // 2, slots=8, max_queue=128) as srv:
        serving.run_stream(srv, inputs.serving_stream(200, 0.5, seed=1), pool)  # warm hierarchies
        for rate in (100, 300, 1000, 3000, 5000):
            stream = inputs.serving_stream(rate, args.serve_seconds)
            rec, busy, wall = serving.run_stream(srv, stream, pool)
            out.append(serving.summarize(rec, busy, wall, rate, args.serve_seconds))
        stats = srv.stats()
    # the same streams at two rates with the small requests merged into batched
    # launches (opts.batch_small = 1)
    batched = []
    with mg.Server(free // 2, slots=8, max_queue=128, batch_small=1) as srv:
        serving.run_stream(srv, inputs.serving_stream(200, 0.5, seed=1), pool)
        for rate in (300, 3000):
            stream = inputs.serving_stream(rate, args.serve_seconds)
            rec, busy, wall = serving.run_stream(srv, stream, pool)
            batched.append(serving.summarize(rec, busy, wall, rate, args.serve_seconds))
        bstats = srv.stats()
    return {"rates": out, "slots": 8, "max_queue": 128, "budget_bytes": stats["budget_bytes"],
            "peak_resident_bytes": stats["peak_bytes"], "evictions": stats["evictions"],
            "latency": "submission to result in the caller's phi (server clock)",
            "with_batch_small": {"rates": batched, "batched_requests": bstats["batched"],
                                 "what": "requests of at most 64^3 cells merged into "
                                         "persistent batched launches (opts.batch_small = 1)"}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=512)
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--fp64-steps", type=int, default=2, help="timed FP64-path solves (0: skip)")
    ap.add_argument("--e2e-steps", type=int, default=16)
    ap.add_argument("--e2e-inflight", type=int, default=3,
                    help="requests in flight in the served end-to-end measurement")
    ap.add_argument("--cpu-n", type=int, default=256, help="oracle sample size")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the built-in launch shapes")
    ap.add_argument("--legs-steps", type=int, default=3,
                    help="timed solves with separate finest-level legs (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=3, help="timed batched solves (0: skip)")
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="seconds of arrivals per serving rate (0: skip)")
    ap.add_argument("--face-steps", type=int, default=3,
                    help="timed solves of the per-face slab (0: skip)")
    ap.add_argument("--sin-steps", type=int, default=20,
                    help="timed solves of the 64^3 sinusoid per precision (0: skip)")
    ap.add_argument("--open-steps", type=int, default=3,
                    help="timed solves of the 256^3 open-boundary sphere per precision (0: skip)")
    args = ap.parse_args()
    ws, rank, local = dist_env()

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import numpy as np
    import torch

    import paper_2302_13903_gb300 as mg
    from paper_2302_13903_gb300 import inputs

    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    n = args.n
    prec = mg.MIXED if args.prec == "mixed" else mg.FP64
    stream = torch.cuda.Stream()
    rho = inputs.gaussian_blobs(n, 64, seed=SEED, device="cuda")
    phi = torch.zeros_like(rho)
    torch.cuda.synchronize()

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    solver = mg.Solver(n, 1.0 / n, mg.PERIODIC, prec=prec)
    if not args.no_tune:
        solver.autotune(stream)
    tiles = solver.tile_configs()
    tcopies = solver.tensor_copies()
    hist = None
    with torch.cuda.stream(stream):
        for _ in range(max(args.warmup, 3)):
            _, hist, st = solver.solve(rho, 1.0, TOL, phi=phi, stream=stream)
            assert st == 0, (st, hist)
    cycles = len(hist)
    # the headline: K solves with no instrumentation (the inner FP32 solves
    # replay as CUDA graphs)
    barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    launches = 0
    evs[0].record(stream)
    for q in range(args.steps):
        _, hist, st = solver.solve(rho, 1.0, TOL, phi=phi, stream=stream)
        assert st == 0, (st, hist)
        launches += solver.last_launches
        evs[q + 1].record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    ms = evs[0].elapsed_time(evs[-1])
    step_ms = [evs[q].elapsed_time(evs[q + 1]) for q in range(args.steps)]
    # the same K solves again with CUDA events around every finest-level
    # launch (kernel durations for the roofline; the launches go one by one)
    solver.set_timing(True)
    for _ in range(args.steps):
        _, hist, st = solver.solve(rho, 1.0, TOL, phi=phi, stream=stream)
        assert st == 0, (st, hist)
    torch.cuda.synchronize()
    if ws > 1:
        t = torch.tensor([ms], device="cuda")
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        ms = float(t.item())
    ms_per_step = ms / args.steps
    value = ws * n ** 3 / (ms_per_step * 1e-3)
    ktimes = solver.kernel_times()
    solver.set_timing(False)

    # roofline of every finest-level launch class, each credited with its own
    # algorithmic bytes per launch; the dominant class (by device time) is the
    # headline roofline
    peak, peak_kind = peaks()
    fin = n.bit_length() - 1

    def variant(k):  # the finest legs' kernel: tensor copies or per-thread copies
        which = {"fused_down": 0, "fused_down0": 1, "fused_up": 2}.get(k)
        if which is not None and tcopies.get(fin, (0, 0, 0))[which]:
            return k + "_tma"
        return k

    by_class = {}
    for k, (tot_ms, nl) in ktimes.items():
        if nl == 0:
            continue
        w = 4 if (prec == mg.MIXED and k in FP32_CLASSES) else 8
        alg = algorithmic_bytes_per_cell(k, w, fixed_point=(prec == mg.MIXED)) * n ** 3
        if k == "outer_residual" and prec == mg.MIXED:
            # the first step of a solve starts from phi = 0 and does not read it
            per_solve = nl / args.steps
            alg *= (per_solve - 0.25) / per_solve
        ach = alg / (tot_ms / nl * 1e-3) / 1e9
        by_class[k] = {"launches_per_solve": nl / args.steps, "ms_per_launch": tot_ms / nl,
                       "algorithmic_bytes_per_launch": alg, "achieved_gbs": ach,
                       "frac": ach / peak, "dtype": "f32" if w == 4 else "f64",
                       "kernel": variant(k),
                       "traffic": ncu_traffic(variant(k), "f32" if w == 4 else "f64", n)}
    dom = max(ktimes, key=lambda k: ktimes[k][0])
    d = by_class[dom]
    prec_tag = d["dtype"]
    traffic = d["traffic"]
    roofline = {"bound": "hbm", "achieved": d["achieved_gbs"], "peak": peak, "unit": "GB/s",
                "frac": d["frac"], "traffic": traffic, "kernel": f"{variant(dom)}_{prec_tag}",
                "peak_source": peak_kind,
                "algorithmic_bytes_per_launch": d["algorithmic_bytes_per_launch"],
                "frac_of_nominal": d["achieved_gbs"] / NOMINAL_HBM_GBS,
                "by_class": by_class}
    # the whole solve against the same roofline, and its V-cycle rate
    whole = None
    if prec == mg.MIXED:
        inner = 1 + solver.opts.inner_cycles
        paired = ktimes.get("fused_updown", (0, 0))[1] > 0
        b_cell = mixed_solve_bytes_per_cell(cycles, inner, paired)
        whole = {"algorithmic_bytes_per_cell": b_cell, "paired_legs": paired,
                 "achieved_gbs": b_cell * n ** 3 / (ms_per_step * 1e-3) / 1e9,
                 "v_cycles": cycles * inner,
                 "cell_v_cycles_per_s": n ** 3 * cycles * inner / (ms_per_step * 1e-3)}
        whole["frac"] = whole["achieved_gbs"] / peak
        whole["frac_of_nominal"] = whole["achieved_gbs"] / NOMINAL_HBM_GBS

    # the same solve with every finest-level leg as its own pass (no fused
    # up-down pass): what the temporal blocking saves
    legs = None
    if args.legs_steps > 0 and prec == mg.MIXED:
        with mg.Solver(n, 1.0 / n, mg.PERIODIC, prec=prec, leg_pairs=2) as s2:
            if not args.no_tune:
                s2.autotune(stream)
            for _ in range(2):
                s2.solve(rho, 1.0, TOL, phi=phi, stream=stream)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            for _ in range(args.legs_steps):
                _, h2, st2 = s2.solve(rho, 1.0, TOL, phi=phi, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            tl = a.elapsed_time(b) / args.legs_steps
        legs = {"ms_per_solve": tl, "value": n ** 3 / (tl * 1e-3), "unit": UNIT, "status": st2,
                "what": "the same solve with the up and down legs of consecutive finest-level "
                        "V-cycles as separate passes (opts.leg_pairs = 2)"}

    # end to end through the host API: pinned host rho/phi, copies inside the timed region
    e2e = None
    if args.e2e_steps > 0:
        # page-locked buffers on the memory node next to this GPU: allocate them
        # from a thread bound to the GPU's local CPUs (first touch places pages)
        numa = near_cpus(local)
        saved_aff = None
        if numa.get("local_cpus"):
            try:
                saved_aff = os.sched_getaffinity(0)
                os.sched_setaffinity(0, numa["local_cpus"])
            except OSError:
                saved_aff = None
        rho_h = rho.cpu().pin_memory()
        phi_h = torch.zeros_like(rho_h).pin_memory()
        solver.solve_host(rho_h, 1.0, TOL, phi=phi_h, stream=stream)
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            _, _, st = solver.solve_host(rho_h, 1.0, TOL, phi=phi_h, stream=stream)
            assert st == 0
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        if ws > 1:
            t = torch.tensor([dt], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            dt = float(t.item())
        nbytes = n ** 3 * 8
        sequential = {"value": ws * n ** 3 * args.e2e_steps / dt, "unit": UNIT,
                      "via": "mg_solve_host, one solve at a time (its first pass reads the "
                             "pinned rho, its last writes the pinned phi)"}
        # the same solves through the serving loop with host buffers: each slot
        # copies its request's rho in and phi out on its own stream, so the
        # transfers of one request overlap the solves of the others
        inflight = args.e2e_inflight
        k_req = inflight * args.e2e_steps
        phis_h = [torch.zeros_like(rho_h).pin_memory() for _ in range(inflight)]
        numa["rho_pages_by_node"] = pages_by_node(rho_h.data_ptr())
        numa["phi_pages_by_node"] = pages_by_node(phis_h[0].data_ptr())
        copies = []  # (h2d ms, d2h ms, solve ms) of every timed request
        free, _ = torch.cuda.mem_get_info()
        with mg.Server(free // 2, slots=inflight, max_queue=4 * inflight, prec=mg.MIXED) as srv:
            for tk in [srv.submit(rho_h, p, tol=TOL) for p in phis_h]:  # hierarchies, shapes
                assert srv.wait(tk, 600)[0].status == 0
            barrier()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            # keep `inflight` requests outstanding: as soon as any one is done
            # (polled in turn), the next is submitted with its phi buffer
            outstanding = {srv.submit(rho_h, phis_h[q], tol=TOL): q for q in range(inflight)}
            submitted = inflight
            while outstanding:
                done = []
                for tk, q in outstanding.items():
                    res, _ = srv.poll(tk)
                    if res.done:
                        assert res.status == 0
                        copies.append((res.h2d_ms, res.d2h_ms, res.solve_ms, res.queue_ms,
                                       res.total_ms))
                        done.append((tk, q))
                for tk, q in done:
                    del outstanding[tk]
                    if submitted < k_req:
                        outstanding[srv.submit(rho_h, phis_h[q], tol=TOL)] = q
                        submitted += 1
                if not done:
                    time.sleep(2e-4)
            dt2 = time.perf_counter() - t0
        if saved_aff is not None:
            os.sched_setaffinity(0, saved_aff)
        if ws > 1:
            t = torch.tensor([dt2], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            dt2 = float(t.item())
        h2d = statistics.median(c[0] for c in copies)
        d2h = statistics.median(c[1] for c in copies)
        e2e = {"value": ws * n ** 3 * k_req / dt2, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
               "via": f"mg_server with pinned host rho / phi, {inflight} requests in flight "
                      f"({k_req} solves timed, copies on the slots' streams)",
               "copies": {"h2d_ms_median": h2d, "d2h_ms_median": d2h,
                          "h2d_gbs": nbytes / (h2d * 1e-3) / 1e9,
                          "d2h_gbs": nbytes / (d2h * 1e-3) / 1e9,
                          "solve_ms_median": statistics.median(c[2] for c in copies),
                          "queue_ms_median": statistics.median(c[3] for c in copies),
                          "total_ms_median": statistics.median(c[4] for c in copies),
                          "slot_busy_fraction": sum(c[2] for c in copies) / (inflight * dt2 * 1e3),
                          "what": "per request, device time of the slot's copies (events on its "
                                  "stream; concurrent with other slots' solves and copies)"},
               "numa": numa,
               "sequential": sequential}
        del rho_h, phi_h, phis_h

    # the same solve with the acceleration g = -grad phi fused into its last pass
    grav = None
    if args.e2e_steps > 0:
        g = torch.empty((3, n, n, n), dtype=torch.float64, device="cuda")
        solver.solve_gravity(rho, 1.0, TOL, phi=phi, g=g, stream=stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.e2e_steps):
            _, _, _, st = solver.solve_gravity(rho, 1.0, TOL, phi=phi, g=g, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        tg = a.elapsed_time(b) / args.e2e_steps
        grav = {"ms_per_solve_with_g": tg, "ms_epilogue": tg - ms_per_step,
                "value": n ** 3 / (tg * 1e-3), "unit": UNIT, "status": st,
                "what": "mg_solve_gravity: the same solve, with g = -grad phi (Sec. 3.2.3) "
                        "written in the pass that converts the fixed-point phi"}
        del g

    # the plain FP64 GPU path on the same workload, for comparison
    fp64 = None
    if args.fp64_steps > 0 and prec == mg.MIXED:
        solver.close()
        s64 = mg.Solver(n, 1.0 / n, mg.PERIODIC, prec=mg.FP64)
        _, h64, st = s64.solve(rho, 1.0, TOL, phi=phi, stream=stream)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.fp64_steps):
            _, h64, st = s64.solve(rho, 1.0, TOL, phi=phi, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        t64 = a.elapsed_time(b) / args.fp64_steps
        fp64 = {"value": n ** 3 / (t64 * 1e-3), "unit": UNIT, "ms_per_step": t64,
                "cycles": len(h64), "status": st,
                "cell_v_cycles_per_s_after_fmg": n ** 3 * (len(h64) - 1) / (t64 * 1e-3)}
        s64.close()
    else:
        solver.close()

    open_sphere = run_open_sphere(args, stream) if args.open_steps > 0 else None
    sinusoid = run_sinusoid(args, stream) if args.sin_steps > 0 else None
    per_face = run_per_face(args, stream) if args.face_steps > 0 else None
    batched = run_batched(args, ws, rank, stream) if args.batch_steps > 0 else None
    serving = run_serving(args) if args.serve_seconds > 0 and ws == 1 else None

    cpu = None
    if rank == 0 and not args.no_cpu and ws == 1:
        cpu = cpu_baseline(args.cpu_n)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == mg.MIXED else "f64", "data": "synthetic",
            "config": {"workload": f"{n}^3 periodic unit cube, 64 Gaussian blobs (seed {SEED}, "
                                   f"sigma 0.02-0.08, lognormal amplitudes), mean removed; "
                                   f"FMG + V(1,1) RB-SOR to ||d||/||f|| < 1e-10; "
                                   + ("FP32 multigrid inside FP64 defect correction"
                                      if prec == mg.MIXED else "FP64"),
                       "n": n, "bc": "periodic", "prec": args.prec, "tol": TOL,
                       "parallelism": f"replicas x{ws}",
                       "tile_configs": {k: {str(l): list(v) for l, v in d.items()}
                                        for k, d in tiles.items() if d},
                       # levels whose down leg (nonzero start, zero start) and
                       # up leg take their planes by tensor copies
                       "tensor_copies": {str(l): list(v) for l, v in tcopies.items()},
                       "l2": "inputs larger than L2 (1 GiB per FP64 field), no flush"},
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "ms_per_step_median": statistics.median(step_ms),
            "whole_solve_roofline": whole,
            "gpu_launches": launches,
            "clocks": clk,
            "residual_checks_per_solve": cycles,
            "final_ratio": float(hist[-1]),
            "kernel_ms_per_step": {k: v[0] / args.steps for k, v in ktimes.items() if v[1]},
            "fp64_path": fp64,
            "separate_legs": legs,
            "with_gravity": grav,
            "open_sphere": open_sphere,
            "sinusoid_64": sinusoid,
            "per_face": per_face,
            "batched": batched,
            "serving": serving,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
