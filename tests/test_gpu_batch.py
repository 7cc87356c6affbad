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
