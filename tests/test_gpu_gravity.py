"""Gravitational acceleration g = -grad phi at cell centres (Sec. 3.2.3): the
standalone kernel against the oracle's, and the acceleration that
mg_solve_gravity forms with the solve (in the fixed-point mixed solve from the
exact integer potential) against the oracle applied to the returned phi."""
import math

import numpy as np
import pytest
import torch

import oracle as orc
import paper_2302_13903_gb300 as mg
from paper_2302_13903_gb300 import inputs

pytestmark = pytest.mark.gpu

BCS = [mg.PERIODIC, mg.FIXED, mg.ZEROGRAD, mg.OPEN]


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", [8, 32])
def test_op_gravity_matches_oracle(bc, n):
    rng = np.random.default_rng(n + 10 * bc)
    phi = rng.standard_normal((n, n, n))
    h = 1.0 / n
    faces = rng.standard_normal(orc.faces_size(n, n, n)) if bc == mg.OPEN else None
    b = 0.4 if bc == mg.FIXED else 0.0
    ref = orc.gravity(phi, h, bc, bc_value=b, faces=faces)
    got = mg.op_gravity(torch.from_numpy(phi).cuda(), h, bc, bc_value=b,
                        faces=None if faces is None else torch.from_numpy(faces).cuda())
    assert rel(got.cpu().numpy(), ref) <= 1e-13


def test_gravity_of_the_sinusoid_solution_closed_form():
    """64^3 periodic sinusoid (the discrete solution is exact, Sec. 4.1): the
    acceleration of the FP64 solution is the closed-form central difference
    of the eigenmode."""
    n = 64
    h = 1.0 / n
    rho = inputs.sinusoid(n)
    with mg.Solver(n, h, mg.PERIODIC, prec=mg.FP64) as s:
        phi, g, hist, st = s.solve_gravity(torch.from_numpy(rho).cuda(), 1.0, 1e-12)
    assert st == 0
    x = (np.arange(n) + 0.5) * h
    sn, cs = np.sin(2 * np.pi * x), np.cos(2 * np.pi * x)
    amp = h * h / (-12.0 * np.sin(np.pi * h) ** 2)  # phi = amp * rho exactly
    k = amp * np.sin(2 * np.pi * h) / h
    want = [-k * sn[:, None, None] * sn[None, :, None] * cs[None, None, :],
            -k * sn[:, None, None] * cs[None, :, None] * sn[None, None, :],
            -k * cs[:, None, None] * sn[None, :, None] * sn[None, None, :]]
    for comp, w in zip(g.cpu().numpy(), want):
        assert rel(comp, w) <= 1e-9


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
@pytest.mark.parametrize("bc", BCS)
def test_solve_gravity_matches_oracle_on_its_phi(prec, bc):
    n = 64
    h = 1.0 / n
    if bc == mg.OPEN:
        rho, fpg = inputs.uniform_sphere(n, 0.25, 4), 4 * math.pi
    else:
        rho, fpg = inputs.gaussian_blobs(n, 6, seed=9, periodic=(bc == mg.PERIODIC)), 1.0
    b = 0.25 if bc == mg.FIXED else 0.0
    rd = torch.from_numpy(rho).cuda()
    with mg.Solver(n, h, bc, prec=prec, fixed_value=b) as s:
        phi_g, g, hist, st = s.solve_gravity(rd, fpg, 1e-10)
        phi_p, hist_p, st_p = s.solve(rd, fpg, 1e-10)
    assert st == st_p == 0
    assert torch.equal(phi_g, phi_p) and np.array_equal(hist, hist_p)
    p = phi_g.cpu().numpy()
    faces = None
    if bc == mg.OPEN:  # the oracle's own multipole faces for this source
        Q, org = orc.multipole_moments(rho, h, 4)
        faces = orc.open_faces(n, n, n, h, Q, 4, fpg / (4 * math.pi), org)
    ref = orc.gravity(p, h, bc, bc_value=b, faces=faces)
    assert rel(g.cpu().numpy(), ref) <= 1e-12
