"""Per-kernel parity: each CUDA operator, called through the C ABI, against the
oracle's operator on the same seeded inputs, element by element.

Tolerances: FP64 kernels differ from the oracle only in rounding order (FMA
contraction, x-then-y-then-z sums), so they agree to a few ulp of the largest
term: 1e-13 relative to the largest output.  FP32 kernels are compared with the
oracle run on the same FP32 inputs widened to FP64: 2e-6 relative (a few FP32
ulp over at most 27 terms).
"""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_2302_13903_gb300 as mg

pytestmark = pytest.mark.gpu

BCS = [mg.PERIODIC, mg.FIXED, mg.ZEROGRAD, mg.OPEN]
DT = {mg.FP64: torch.float64, mg.MIXED: torch.float32}
TOL = {mg.FP64: 1e-13, mg.MIXED: 2e-6}


def dev(a, dtype=torch.float64):
    return torch.from_numpy(np.ascontiguousarray(a)).to("cuda", dtype)


def host(t):
    return t.double().cpu().numpy()


def rel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


def orc_bc(bc):
    """The oracle's kind for a level with given face values."""
    return orc.FACES if bc == mg.OPEN else bc


def make(n, bc, prec, seed):
    rng = np.random.default_rng(seed)
    u = rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    faces = rng.standard_normal(orc.faces_size(n, n, n)) if bc == mg.OPEN else None
    if prec == mg.MIXED:  # both sides see the same FP32 values
        u, f = u.astype(np.float32).astype(np.float64), f.astype(np.float32).astype(np.float64)
    return u, f, faces


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("colours", [0, 1, 2])
def test_smooth(prec, bc, colours):
    n, h, b = 16, 1.0 / 16, 0.3
    u, f, faces = make(n, bc, prec, 1 + bc)
    steps = 2 if colours == 0 else 1
    ref = orc.smooth(u, f, h, orc_bc(bc), bc_value=b, faces=faces, omega=1.15, steps=steps,
                     colours=colours)
    ug = dev(u, DT[prec])
    mg.op_smooth(ug, dev(f, DT[prec]), h, bc, b, None if faces is None else dev(faces),
                 omega=1.15, steps=steps, colours=colours)
    assert rel(host(ug), ref) < TOL[prec] * (10 if prec == mg.MIXED else 1)


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", [2, 16, 32])
def test_defect_and_fused_restrict(prec, bc, n):
    h, b = 1.0 / n, -0.4
    u, f, faces = make(n, bc, prec, 10 + n + bc)
    ref = orc.defect(u, f, h, orc_bc(bc), bc_value=b, faces=faces)
    fd = None if faces is None else dev(faces)
    d = mg.op_defect(dev(u, DT[prec]), dev(f, DT[prec]), h, bc, b, fd)
    assert rel(host(d), ref) < TOL[prec]
    fc = mg.op_defect_restrict(dev(u, DT[prec]), dev(f, DT[prec]), h, bc, b, fd)
    # the mean of eight defects can cancel: measure against the summands' size
    err = np.abs(host(fc) - orc.restrict(ref)).max() / np.abs(ref).max()
    assert err < TOL[prec]


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
@pytest.mark.parametrize("shape", [(2, 2, 2), (8, 16, 32)])
def test_restrict(prec, shape):
    rng = np.random.default_rng(4)
    u = rng.standard_normal(shape)
    if prec == mg.MIXED:
        u = u.astype(np.float32).astype(np.float64)
    uc = mg.op_restrict(dev(u, DT[prec]))
    assert rel(host(uc), orc.restrict(u)) < TOL[prec]


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("high", [False, True])
@pytest.mark.parametrize("add", [False, True])
@pytest.mark.parametrize("nc", [1, 2, 8])
def test_prolong(prec, bc, high, add, nc):
    rng = np.random.default_rng(20 + nc + bc)
    uc = rng.standard_normal((nc, nc, nc))
    uf = rng.standard_normal((2 * nc,) * 3)
    faces = rng.standard_normal(orc.faces_size(nc, nc, nc)) if bc == mg.OPEN else None
    if prec == mg.MIXED:
        uc, uf = uc.astype(np.float32).astype(np.float64), uf.astype(np.float32).astype(np.float64)
    ref = orc.prolong(uc, orc_bc(bc), bc_value=0.7, coarse_faces=faces, high_order=high, add=add,
                      uf=uf)
    out = mg.op_prolong(dev(uc, DT[prec]), bc, 0.7, None if faces is None else dev(faces),
                        high_order=high, add=add, uf=dev(uf, DT[prec]))
    assert rel(host(out), ref) < TOL[prec]


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
@pytest.mark.parametrize("bc", BCS)
def test_coarsest(prec, bc):
    rng = np.random.default_rng(30 + bc)
    f = np.array([[[1.25]]])
    faces = rng.standard_normal(orc.faces_size(1, 1, 1)) if bc == mg.OPEN else None
    ref = orc.coarsest(f, 0.5, orc_bc(bc), bc_value=0.2, faces=faces)
    u = mg.op_coarsest(dev(f, DT[prec]), 0.5, bc, 0.2, None if faces is None else dev(faces))
    assert rel(host(u), ref) < TOL[prec] if np.abs(ref).max() > 0 else host(u)[0, 0, 0] == 0.0


@pytest.mark.parametrize("use_com", [True, False])
def test_multipole_moments_and_faces(use_com):
    from paper_2302_13903_gb300 import inputs
    n, h = 32, 1.0 / 32
    rho = inputs.uniform_sphere(n, 0.2, 4)
    rng = np.random.default_rng(6)
    rho = rho * (1.0 + 0.3 * rng.random(rho.shape))  # break the symmetry
    origin = (0.01, -0.02, 0.015)
    Qo, oo = orc.multipole_moments(rho, h, 4, use_com, origin)
    Qg, og = mg.op_multipole_moments(dev(rho), h, 4, use_com, origin)
    assert np.abs(og - oo).max() < 1e-15
    assert np.abs(Qg - Qo).max() < 1e-13 * np.abs(Qo).max()
    for lmax in (0, 2, 4):
        for nl, hl in ((n, h), (4, 8 * h), (1, 32 * h)):
            fo = orc.open_faces(nl, nl, nl, hl, Qo, lmax, 0.9, oo)
            fg = mg.op_open_faces(nl, hl, Qg, lmax, 0.9, og)
            assert rel(host(fg), fo) < 1e-13


@pytest.mark.parametrize("bc", [mg.PERIODIC, mg.FIXED, mg.ZEROGRAD])
@pytest.mark.parametrize("n", [16, 32, 64, 128])
@pytest.mark.parametrize("zero_guess", [False, True])
def test_fused_down_leg(bc, n, zero_guess):
    """One SMOOTH step then the restricted defect (Algorithm 1, steps 1-3),
    against the oracle's smoother, defect and restriction in turn.  Sizes span
    several tiles and z-chunks of the fused kernel (16 runs the per-step
    kernels)."""
    h = 1.0 / n
    u, f, _ = make(n, bc, mg.MIXED, 40 + n + bc)
    u0 = np.zeros_like(u) if zero_guess else u
    ref_u = orc.smooth(u0, f, h, bc, bc_value=0.0, omega=1.15, steps=1, colours=0)
    ref_d = orc.defect(ref_u, f, h, bc, bc_value=0.0)
    uo, fc = mg.op_vcycle_down(dev(u, torch.float32), dev(f, torch.float32), h, bc,
                               zero_guess=zero_guess)
    assert rel(host(uo), ref_u) < 2e-6
    err = np.abs(host(fc) - orc.restrict(ref_d)).max() / np.abs(ref_d).max()
    assert err < 2e-6


@pytest.mark.parametrize("bc", [mg.PERIODIC, mg.FIXED, mg.ZEROGRAD])
@pytest.mark.parametrize("n", [16, 32, 64, 128])
def test_fused_up_leg(bc, n):
    """u + trilinear(e_coarse), then one SMOOTH step (Algorithm 1, steps 5-7)."""
    h = 1.0 / n
    u, f, _ = make(n, bc, mg.MIXED, 50 + n + bc)
    ec = np.random.default_rng(60 + n).standard_normal((n // 2,) * 3)
    ec = ec.astype(np.float32).astype(np.float64)
    ref = orc.prolong(ec, bc, bc_value=0.0, add=True, uf=u)
    ref = orc.smooth(ref, f, h, bc, bc_value=0.0, omega=1.15, steps=1, colours=0)
    uo = mg.op_vcycle_up(dev(u, torch.float32), dev(f, torch.float32), dev(ec, torch.float32), h, bc)
    assert rel(host(uo), ref) < 2e-6
