"""Batched solve: many independent grids of uneven size and mixed rules in one
persistent launch, each against the oracle's converged solution (the mixed
path's tolerance, 1e-9) and against the same grid solved alone."""
import math

import numpy as np
import pytest
import torch

import oracle as orc
import paper_2302_13903_gb300 as mg
from paper_2302_13903_gb300 import inputs

pytestmark = pytest.mark.gpu


def emax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def make_case(specs, seed=0):
    rhos, fixed = [], []
    for k, (n, bc) in enumerate(specs):
        spec = dict(n=n, bc=bc, seed=seed * 100 + k, n_blobs=3)
        rhos.append(inputs.batch_source(spec))
        fixed.append(0.2 if bc == mg.FIXED and k % 2 else 0.0)
    return rhos, fixed


SPECS = [(8, mg.PERIODIC), (16, mg.FIXED), (32, mg.ZEROGRAD), (64, mg.PERIODIC),
         (128, mg.FIXED), (64, mg.ZEROGRAD), (32, mg.FIXED), (128, mg.PERIODIC),
         (16, mg.ZEROGRAD), (64, mg.FIXED), (2, mg.PERIODIC), (4, mg.FIXED)]


def test_batch_matches_oracle_per_grid():
    rhos, fixed = make_case(SPECS)
    sizes = [n for n, _ in SPECS]
    with mg.Batch(sizes, [1.0 / n for n in sizes], [bc for _, bc in SPECS], fixed) as b:
        assert b.cells == sum(n ** 3 for n in sizes)
        rd = [torch.from_numpy(r).cuda() for r in rhos]
        pd = [torch.zeros_like(r) for r in rd]
        st, hists, sts = b.solve(rd, pd, 1.0, 1e-10)
    assert st == 0, (st, sts)
    for k, ((n, bc), rho) in enumerate(zip(SPECS, rhos)):
        ref = orc.solve(rho, 1.0 / n, bc, bc_value=fixed[k], tol=0.0, max_cycles=80)
        assert hists[k][-1] < 1e-10, (k, hists[k])
        err = emax(pd[k].cpu().numpy(), ref.phi)
        assert err <= 1e-9, (k, n, bc, err)


def test_batch_repeat_is_deterministic_and_matches_alone():
    specs = SPECS[:8]
    rhos, fixed = make_case(specs, seed=3)
    sizes = [n for n, _ in specs]
    with mg.Batch(sizes, [1.0 / n for n in sizes], [bc for _, bc in specs], fixed) as b:
        rd = [torch.from_numpy(r).cuda() for r in rhos]
        p1 = [torch.zeros_like(r) for r in rd]
        p2 = [torch.zeros_like(r) for r in rd]
        st1, h1, _ = b.solve(rd, p1, 1.0, 1e-10)
        st2, h2, _ = b.solve(rd, p2, 1.0, 1e-10)  # replays the captured graph
        assert b.graph
    assert st1 == st2 == 0
    for k in range(len(specs)):
        assert torch.equal(p1[k], p2[k]) and np.array_equal(h1[k], h2[k])
    # the same grid alone in a batch of one gives the same bits
    k = 4
    with mg.Batch([sizes[k]], [1.0 / sizes[k]], [specs[k][1]], [fixed[k]]) as b1:
        alone = torch.zeros_like(rd[k])
        st, ha, _ = b1.solve([rd[k]], [alone], 1.0, 1e-10)
    assert st == 0 and torch.equal(alone, p1[k]) and np.array_equal(ha[0], h1[k])


def test_batch_rejects_unsupported_options():
    with pytest.raises(mg.MGError):
        mg.Batch([8], [0.1], [mg.OPEN])
    with pytest.raises(mg.MGError):
        mg.Batch([8], [0.1], [mg.PERIODIC], prec=mg.FP64)
    with pytest.raises(mg.MGError):
        mg.Batch([12], [0.1], [mg.PERIODIC])


def test_barrier_limit_runs_out_and_the_batch_recovers():
    """A grid-wide barrier wait of at most one clock cycle cannot see every
    block arrive: the waiting blocks give up, set the error flag and return,
    so the solve ends with MG_ERR_TIMEOUT instead of hanging.  With the
    default limit back, the same batch solves again and gives the bits of a
    batch that never timed out."""
    specs = [(16, mg.PERIODIC), (32, mg.FIXED), (16, mg.ZEROGRAD), (32, mg.PERIODIC)]
    rhos, fixed = make_case(specs, seed=7)
    sizes = [n for n, _ in specs]
    rd = [torch.from_numpy(r).cuda() for r in rhos]
    args = (sizes, [1.0 / n for n in sizes], [bc for _, bc in specs], fixed)
    with mg.Batch(*args) as ref_b:
        ref_phi = [torch.zeros_like(r) for r in rd]
        st, ref_h, _ = ref_b.solve(rd, ref_phi, 1.0, 1e-10)
        assert st == 0
    with mg.Batch(*args) as b:
        phis = [torch.zeros_like(r) for r in rd]
        b.set_barrier_limit(1)
        timeouts = 0
        for _ in range(3):
            try:
                b.solve(rd, phis, 1.0, 1e-10)
            except mg.MGError as e:
                assert e.status == 6, e  # MG_ERR_TIMEOUT, never a CUDA error
                timeouts += 1
        assert timeouts >= 1
        with pytest.raises(mg.MGError):
            b.set_barrier_limit(-1)
        b.set_barrier_limit(4_000_000_000)
        st, h, _ = b.solve(rd, phis, 1.0, 1e-10)
        assert st == 0 and b.graph
        for p, q, ha, hb in zip(phis, ref_phi, h, ref_h):
            assert torch.equal(p, q) and np.array_equal(ha, hb)


def test_batch_slots_left_out_and_fewer_ctas():
    """Slots without a grid in a solve (rho = None) are passed by: the other
    grids give the bits they give with every slot used, also on fewer CTAs,
    and the empty slots' phi stays untouched."""
    specs = [(32, mg.PERIODIC), (64, mg.FIXED), (32, mg.ZEROGRAD), (16, mg.PERIODIC)]
    rhos, fixed = make_case(specs, seed=9)
    sizes = [n for n, _ in specs]
    rd = [torch.from_numpy(r).cuda() for r in rhos]
    with mg.Batch(sizes, [1.0 / n for n in sizes], [bc for _, bc in specs], fixed) as b:
        full = [torch.zeros_like(r) for r in rd]
        st, hf, _ = b.solve(rd, full, 1.0, 1e-10)
        assert st == 0
        part = [torch.full_like(r, 7.0) for r in rd]
        use = [True, False, True, False]
        st, hp, sts = b.solve([r if u else None for r, u in zip(rd, use)],
                              [p if u else None for p, u in zip(part, use)], 1.0, 1e-10)
        assert st == 0 and list(sts) == [0, 0, 0, 0]
        for g, u in enumerate(use):
            if u:
                assert torch.equal(part[g], full[g]) and np.array_equal(hp[g], hf[g])
            else:
                assert len(hp[g]) == 0
        b.set_blocks(8)
        few = [torch.zeros_like(r) for r in rd]
        st, h8, _ = b.solve(rd, few, 1.0, 1e-10)
        assert st == 0 and b.graph
        for g in range(len(specs)):
            assert torch.equal(few[g], full[g]) and np.array_equal(h8[g], hf[g])
        st, _, _ = b.solve([None] * 4, [None] * 4, 1.0, 1e-10)
        assert st == 1  # MG_ERR_ARG: no grid to solve
