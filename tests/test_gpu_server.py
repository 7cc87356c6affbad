"""Serving loop: requests of different sizes and rules run concurrently on
resident hierarchies under an HBM budget, and every result equals the same
request solved alone (bit for bit: each solve is deterministic and a
hierarchy serves one request at a time)."""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_2302_13903_gb300 as mg
from paper_2302_13903_gb300 import inputs

pytestmark = pytest.mark.gpu

MIX = [(64, mg.PERIODIC, 0, 1e-10), (32, mg.OPEN, 4, 1e-8), (128, mg.FIXED, 0, 1e-9),
       (32, mg.ZEROGRAD, 0, 1e-10), (128, mg.OPEN, 2, 1e-10), (64, mg.FIXED, 0, 1e-6),
       (16, mg.PERIODIC, 0, 1e-10), (128, mg.PERIODIC, 0, 1e-7), (64, mg.ZEROGRAD, 0, 1e-10),
       (64, mg.OPEN, 0, 1e-9), (32, mg.FIXED, 0, 1e-10), (128, mg.ZEROGRAD, 0, 1e-8)]


def sources(mix, seed=11):
    return [inputs.serving_source(dict(n=n, bc=bc, seed=seed + k, n_blobs=1 + k % 8), "cuda")
            for k, (n, bc, _, _) in enumerate(mix)]


def solve_alone(rho, n, bc, lmax, tol, **opts):
    with mg.Server(1 << 34, slots=1, max_queue=4, **opts) as s:
        phi = torch.zeros_like(rho)
        res, hist = s.wait(s.submit(rho, phi, bc=bc, tol=tol, lmax=lmax), 120)
        assert res.done and res.status in (0, 4)
    return phi, hist


def test_server_mix_equals_alone():
    rhos = sources(MIX)
    alone = [solve_alone(r, n, bc, lmax, tol) for r, (n, bc, lmax, tol) in zip(rhos, MIX)]
    with mg.Server(1 << 34, slots=4, max_queue=64) as s:
        phis = [torch.full_like(r, float("nan")) for r in rhos]
        tickets = [s.submit(r, p, bc=bc, tol=tol, lmax=lmax)
                   for r, p, (n, bc, lmax, tol) in zip(rhos, phis, MIX)]
        results = [s.wait(t, 120) for t in tickets]
        st = s.stats()
    assert st["completed"] == len(MIX) and st["rejected"] == 0
    for k, ((res, hist), (pa, ha)) in enumerate(zip(results, alone)):
        assert res.done and res.status == 0, (k, res.status)
        assert hist[-1] < MIX[k][3]
        assert 0.0 <= res.queue_ms <= res.total_ms and res.solve_ms > 0.0
        assert torch.equal(phis[k], pa), k
        assert np.array_equal(hist, ha), k


def test_server_mix_with_batching_equals_alone():
    """The same mix with small requests served by batched hierarchies
    (batch_small = 1): every result still equals the request alone."""
    rhos = sources(MIX, seed=13)
    alone = [solve_alone(r, n, bc, lmax, tol, batch_small=1)
             for r, (n, bc, lmax, tol) in zip(rhos, MIX)]
    with mg.Server(1 << 34, slots=4, max_queue=64, batch_small=1) as s:
        phis = [torch.full_like(r, float("nan")) for r in rhos]
        tickets = [s.submit(r, p, bc=bc, tol=tol, lmax=lmax)
                   for r, p, (n, bc, lmax, tol) in zip(rhos, phis, MIX)]
        results = [s.wait(t, 120) for t in tickets]
    for k, ((res, hist), (pa, ha)) in enumerate(zip(results, alone)):
        assert res.done and res.status == 0, (k, res.status)
        assert torch.equal(phis[k], pa), k
        assert np.array_equal(hist, ha), k


def test_server_open_request_matches_oracle():
    n, bc, lmax, tol = 32, mg.OPEN, 4, 1e-10
    rho = inputs.serving_source(dict(n=n, bc=bc, seed=5, n_blobs=3))
    ref = orc.solve(rho, 1.0 / n, bc, lmax=lmax, tol=0.0, max_cycles=80)
    with mg.Server(1 << 32, slots=2) as s:
        rd = torch.from_numpy(rho).cuda()
        phi = torch.zeros_like(rd)
        res, hist = s.wait(s.submit(rd, phi, bc=bc, tol=tol, lmax=lmax), 120)
    assert res.status == 0 and hist[-1] < tol
    err = float(np.abs(phi.cpu().numpy() - ref.phi).max() / np.abs(ref.phi).max())
    assert err <= 1e-9, err


def test_server_budget_evicts_and_results_stay_equal():
    mix = [(128, mg.PERIODIC, 0, 1e-10), (64, mg.FIXED, 0, 1e-10), (128, mg.ZEROGRAD, 0, 1e-10),
           (32, mg.OPEN, 3, 1e-10), (64, mg.PERIODIC, 0, 1e-10), (128, mg.FIXED, 0, 1e-10),
           (64, mg.FIXED, 0, 1e-10), (128, mg.PERIODIC, 0, 1e-10)]
    need = {(n, bc, lmax): mg.required_bytes(n, bc, prec=mg.MIXED, lmax=lmax)
            for n, bc, lmax, _ in mix}
    budget = int(1.2 * max(need.values()) + need[(64, mg.FIXED, 0)])
    rhos = sources(mix, seed=40)
    alone = [solve_alone(r, n, bc, lmax, tol)[0] for r, (n, bc, lmax, tol) in zip(rhos, mix)]
    with mg.Server(budget, slots=3, max_queue=64) as s:
        phis = [torch.zeros_like(r) for r in rhos]
        tickets = [s.submit(r, p, bc=bc, tol=tol, lmax=lmax)
                   for r, p, (n, bc, lmax, tol) in zip(rhos, phis, mix)]
        results = [s.wait(t, 120)[0] for t in tickets]
        st = s.stats()
    assert all(r.done and r.status == 0 for r in results)
    assert st["peak_bytes"] <= budget and st["evictions"] > 0
    for k in range(len(mix)):
        assert torch.equal(phis[k], alone[k]), k


def test_server_refusals_and_ticket_lifecycle():
    rho = inputs.serving_source(dict(n=128, bc=mg.PERIODIC, seed=1, n_blobs=2), "cuda")
    small = mg.required_bytes(32, mg.PERIODIC, prec=mg.MIXED)
    with mg.Server(small + 1, slots=1, max_queue=2) as s:
        with pytest.raises(mg.MGError) as e:  # its hierarchy alone exceeds the budget
            s.submit(rho, torch.zeros_like(rho), tol=1e-10)
        assert e.value.status == 2
        assert s.stats()["rejected"] == 1
    with mg.Server(1 << 33, slots=1, max_queue=1) as s:
        phis = [torch.zeros_like(rho) for _ in range(6)]
        taken, busy = [], 0
        for p in phis:  # one runs, one waits, the rest find the queue full
            try:
                taken.append((s.submit(rho, p, tol=1e-10), p))
            except mg.MGError as err:
                assert err.status == 7
                busy += 1
        assert busy >= 1 and len(taken) >= 1
        assert s.stats()["rejected"] == busy
        done = [s.wait(t, 120)[0] for t, _ in taken]
        assert all(r.done and r.status == 0 for r in done)
        with pytest.raises(mg.MGError):  # retired once reported done
            s.poll(taken[0][0])
        for _, p in taken[1:]:
            assert torch.equal(p, taken[0][1])


@pytest.mark.parametrize("pinned", [True, False])
def test_server_host_buffers_equal_device_buffers(pinned):
    """Requests with host rho and phi (copied in and out by the slot's stream)
    give the bits of the same requests on device arrays, several at once."""
    mix = [(64, mg.PERIODIC, 0, 1e-10), (32, mg.OPEN, 4, 1e-9), (64, mg.FIXED, 0, 1e-10),
           (32, mg.ZEROGRAD, 0, 1e-10)]
    rhos = sources(mix, seed=31)
    dev = [solve_alone(r, n, bc, lmax, tol) for r, (n, bc, lmax, tol) in zip(rhos, mix)]
    host_rho = [r.cpu() for r in rhos]
    if pinned:
        host_rho = [r.pin_memory() for r in host_rho]
    phis = [torch.full_like(r, float("nan")) for r in host_rho]
    if pinned:
        phis = [p.pin_memory() for p in phis]
    with mg.Server(1 << 34, slots=3, max_queue=16) as s:
        tickets = [s.submit(r, p, bc=bc, tol=tol, lmax=lmax)
                   for r, p, (n, bc, lmax, tol) in zip(host_rho, phis, mix)]
        results = [s.wait(t, 120) for t in tickets]
    for k, ((res, hist), (pd, hd)) in enumerate(zip(results, dev)):
        assert res.done and res.status == 0, (k, res.status)
        assert torch.equal(phis[k], pd.cpu()), k
        assert np.array_equal(hist, hd), k


def test_server_refuses_mixed_memory():
    rho = torch.zeros((16, 16, 16), dtype=torch.float64, device="cuda")
    phi = torch.zeros((16, 16, 16), dtype=torch.float64)
    with mg.Server(1 << 30, slots=1) as s:
        with pytest.raises(mg.MGError):
            s.submit(rho, phi)


def test_server_requests_overlap_on_the_device():
    """Requests on different slots run at the same time: by the server's own
    timestamps, eight 128^3 solves on four slots finish in less time than the
    sum of the same solves' lone solve times (each on a warm one-slot
    server), and some of them ran at once."""
    import time
    mix = [(128, bc, 0, 1e-10) for bc in (mg.PERIODIC, mg.FIXED, mg.ZEROGRAD) * 3][:8]
    rhos = sources(mix, seed=50)
    phis = [torch.zeros_like(r) for r in rhos]

    def run(server, order):
        return [server.wait(server.submit(rhos[k], phis[k], bc=mix[k][1], tol=mix[k][3]), 120)[0]
                for k in order]

    with mg.Server(1 << 34, slots=1, max_queue=16) as s1:
        run(s1, range(len(mix)))  # hierarchies created and tuned
        lone = [r.solve_ms for r in run(s1, range(len(mix)))]
    with mg.Server(1 << 34, slots=4, max_queue=16) as s4:
        warm = [s4.submit(r, p, bc=m[1], tol=m[3]) for r, p, m in zip(rhos, phis, mix)]
        assert all(s4.wait(t, 120)[0].status == 0 for t in warm)
        t0 = time.perf_counter()
        tickets = [s4.submit(r, p, bc=m[1], tol=m[3]) for r, p, m in zip(rhos, phis, mix)]
        spread_ms = (time.perf_counter() - t0) * 1e3  # submissions, one after the other
        results = [s4.wait(t, 120)[0] for t in tickets]
    assert all(r.done and r.status == 0 for r in results)
    wall_ms = spread_ms + max(r.total_ms for r in results)
    assert wall_ms < 0.8 * sum(lone), (wall_ms, sum(lone))
    # run intervals [queue_ms, total_ms] from (nearly) one submission instant
    spans = sorted((r.queue_ms, r.total_ms) for r in results)
    assert any(b[0] + spread_ms < a[1] for a, b in zip(spans, spans[1:]))


def test_small_requests_are_batched_and_match_alone_and_oracle():
    """Continuous batching: a burst of small requests of one shape and rule
    queued behind a busy slot runs as one batched launch (the server counts
    them); each result equals the same request alone, and a fixed-rule one
    the oracle's converged solution within 1e-9."""
    n = 32
    mix = [(n, mg.FIXED, 0, tol) for tol in (1e-10, 1e-8, 1e-6, 1e-10, 1e-9, 1e-10)]
    rhos = sources(mix, seed=70)
    alone = [solve_alone(r, nn, bc, lmax, tol, batch_small=1)
             for r, (nn, bc, lmax, tol) in zip(rhos, mix)]
    big = inputs.serving_source(dict(n=128, bc=mg.PERIODIC, seed=3, n_blobs=2), "cuda")
    with mg.Server(1 << 34, slots=1, max_queue=64, batch_small=1) as s:
        s.wait(s.submit(rhos[0], torch.zeros_like(rhos[0]), bc=mg.FIXED, tol=1e-10), 120)
        hold = s.submit(big, torch.zeros_like(big), tol=1e-10)  # keeps the one slot busy
        phis = [torch.full_like(r, float("nan")) for r in rhos]
        tickets = [s.submit(r, p, bc=bc, tol=tol) for r, p, (_, bc, _, tol) in zip(rhos, phis, mix)]
        results = [s.wait(t, 120) for t in tickets]
        assert s.wait(hold, 120)[0].status == 0
        st = s.stats()
    assert st["batched"] >= 2
    for k, ((res, hist), (pa, ha)) in enumerate(zip(results, alone)):
        assert res.done and res.status == 0, (k, res.status)
        assert hist[-1] < mix[k][3]
        assert torch.equal(phis[k], pa), k
        assert np.array_equal(hist, ha), k
    rho = rhos[0].cpu().numpy()
    ref = orc.solve(rho, 1.0 / n, orc.FIXED, tol=0.0, max_cycles=80)
    err = float(np.abs(phis[0].cpu().numpy() - ref.phi).max() / np.abs(ref.phi).max())
    assert err <= 1e-9, err


def test_server_rule_per_face_requests():
    """Requests with a rule per face (Sec. 2.3.6) next to uniform ones: each
    gives the bits of mg_create_faces' solve of the same grid, and the oracle's
    converged solution within 1e-9."""
    P, F, Z = mg.PERIODIC, mg.FIXED, mg.ZEROGRAD
    faces = [((P, P, P, P, F, F), (0, 0, 0, 0, 0.3, -0.2)), ((Z, F, F, Z, P, P), (0, 0.4, 0.1, 0, 0, 0))]
    n = 64
    rhos = [torch.from_numpy(inputs.gaussian_blobs(n, 6, seed=80 + k, periodic=False,
                                                   remove_mean=False)).cuda() for k in range(2)]
    ref = []
    for rho, (kinds, vals) in zip(rhos, faces):
        with mg.Solver(n, 1.0 / n, list(kinds), face_values=list(vals), prec=mg.MIXED) as s:
            s.autotune()
            phi, hist, st = s.solve(rho, 1.0, 1e-10)
            ref.append((phi, hist))
    uni = inputs.serving_source(dict(n=n, bc=P, seed=9, n_blobs=3), "cuda")
    with mg.Server(1 << 34, slots=3, max_queue=16) as srv:
        phis = [torch.zeros_like(r) for r in rhos]
        tickets = [srv.submit(r, p, bc=list(k), face_values=list(v), tol=1e-10)
                   for r, p, (k, v) in zip(rhos, phis, faces)]
        t_uni = srv.submit(uni, torch.zeros_like(uni), tol=1e-10)
        results = [srv.wait(t, 120) for t in tickets]
        assert srv.wait(t_uni, 120)[0].status == 0
        with pytest.raises(mg.MGError):  # periodic faces come in pairs
            srv.submit(uni, torch.zeros_like(uni), bc=[P, F, P, P, P, P])
    for k, ((res, hist), (pr, hr)) in enumerate(zip(results, ref)):
        assert res.done and res.status == 0, (k, res.status)
        assert torch.equal(phis[k], pr) and np.array_equal(hist, hr), k
        kinds, vals = faces[k]
        o = orc.solve(rhos[k].cpu().numpy(), 1.0 / n, orc.PER_FACE,
                      faces=orc.mixed_rule(kinds, vals), tol=0.0, max_cycles=80)
        err = float(np.abs(phis[k].cpu().numpy() - o.phi).max() / np.abs(o.phi).max())
        assert err <= 1e-9, (k, err)
