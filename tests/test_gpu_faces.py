"""A rule per face (Sec. 2.3.6: the boundaries may carry different rules; a
fixed value on any face sets the zero point of the potential, otherwise the
means of f and phi are removed) through mg_create_faces, against the oracle's
per-face rule.

FP64 path: the same schedule gives e_max <= 1e-11 (rounding order only), in
the correction scheme and in FAS, on cubes and on a box.  Mixed path: at
||d||/||f|| < 1e-10 within 1e-9 of the oracle's converged solution.  Six equal
rules give the bits of the uniform rule's own context.
"""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_2302_13903_gb300 as mg
from paper_2302_13903_gb300 import inputs

pytestmark = pytest.mark.gpu

P, F, Z = mg.PERIODIC, mg.FIXED, mg.ZEROGRAD
NO_STALL = 1e300

# (kinds x-, x+, y-, y+, z-, z+; values on the fixed faces)
CASES = {
    "slab": ((P, P, P, P, F, F), (0, 0, 0, 0, 0.3, -0.2)),  # periodic in x, y; fixed in z
    "wall": ((F, Z, P, P, Z, Z), (0.5, 0, 0, 0, 0, 0)),  # one fixed face
    "box": ((Z, F, F, Z, F, Z), (0, -0.4, 0.1, 0, 0.7, 0)),
    "channel": ((P, P, Z, Z, Z, Z), (0,) * 6),  # no zero point: means removed
    "zero_walls": ((P, P, F, F, F, F), (0,) * 6),  # homogeneous: fast source path off too
    # z periodic with walls across x or y: periodic-axis masks 4, 5 and 6
    "z_pipe": ((F, F, Z, Z, P, P), (0.2, -0.1, 0, 0, 0, 0)),  # periodic in z only
    "xz_sheet": ((P, P, F, Z, P, P), (0, 0, 0.4, 0, 0, 0)),  # periodic in x and z
    "yz_sheet": ((Z, F, P, P, P, P), (0, -0.3, 0, 0, 0, 0)),  # periodic in y and z
}


def emax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def source(shape, case, seed):
    nz, ny, nx = shape
    kinds = CASES[case][0]
    # with a fixed face the mean of f stays (it is not removed by the solve)
    rho = inputs.gaussian_blobs(nx, 8, seed=seed, periodic=False, remove_mean=F not in kinds)
    if (nz, ny) != (nx, nx):
        rho = rho[:nz, :ny, :]
    return np.ascontiguousarray(rho)


def oracle_solve(rho, case, **kw):
    kinds, values = CASES[case]
    nx = rho.shape[2]
    return orc.solve(rho, 1.0 / nx, orc.PER_FACE, faces=orc.mixed_rule(kinds, values), **kw)


def gpu_solve(rho, case, tol, **opts):
    kinds, values = CASES[case]
    nz, ny, nx = rho.shape
    with mg.Solver((nx, ny, nz), 1.0 / nx, list(kinds), face_values=list(values), **opts) as s:
        phi, hist, st = s.solve(torch.from_numpy(rho).cuda(), 1.0, tol)
        return phi.cpu().numpy(), hist, st


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("n", [8, 32])
def test_fp64_same_schedule_matches_oracle(case, n):
    rho = source((n, n, n), case, seed=n + len(case))
    for k in (0, 2):
        ref = oracle_solve(rho, case, tol=0.0, max_cycles=k, stall_ratio=NO_STALL)
        phi, hist, st = gpu_solve(rho, case, 0.0, prec=mg.FP64, max_cycles=k, stall_ratio=NO_STALL)
        assert len(hist) == len(ref.hist) == k + 1
        assert st == ref.status
        assert emax(phi, ref.phi) <= 1e-11, (k, emax(phi, ref.phi))
        assert np.allclose(hist, ref.hist, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("case", ["slab", "box"])
def test_fas_same_schedule_matches_oracle(case):
    n = 32
    rho = source((n, n, n), case, seed=41)
    ref = oracle_solve(rho, case, tol=0.0, max_cycles=2, stall_ratio=NO_STALL, cycle=orc.FAS)
    phi, hist, st = gpu_solve(rho, case, 0.0, prec=mg.FP64, max_cycles=2, stall_ratio=NO_STALL,
                              fas=1)
    assert emax(phi, ref.phi) <= 1e-11
    assert np.allclose(hist, ref.hist, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("case", ["slab", "wall", "channel"])
@pytest.mark.parametrize("shape", [(8, 8, 16), (16, 32, 64)])
def test_box_fp64_same_schedule_matches_oracle(case, shape):
    """(nz, ny, nx) boxes: the coarsest level has several cells (Gauss-Seidel
    sweeps, Sec. 2.3.2) and its ghosts come from the face rules too."""
    rho = source(shape, case, seed=sum(shape))
    for k in (0, 2):
        ref = oracle_solve(rho, case, tol=0.0, max_cycles=k, stall_ratio=NO_STALL)
        phi, hist, st = gpu_solve(rho, case, 0.0, prec=mg.FP64, max_cycles=k, stall_ratio=NO_STALL)
        assert emax(phi, ref.phi) <= 1e-11, (k, emax(phi, ref.phi))


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("n", [16, 64])
def test_mixed_matches_converged_oracle(case, n):
    rho = source((n, n, n), case, seed=3 * n + len(case))
    ref = oracle_solve(rho, case, tol=0.0, max_cycles=80)
    assert ref.ok
    phi, hist, st = gpu_solve(rho, case, 1e-10, prec=mg.MIXED)
    assert st == 0 and hist[-1] < 1e-10, (st, hist)
    assert emax(phi, ref.phi) <= 1e-9


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
def test_literal_coarse_rule_with_face_rules(prec):
    """coarse_literal gives the zero-gradient faces zero fixed values on the
    coarse correction levels: the FP64 cycles are the oracle's literal ones and
    the mixed solve still reaches the converged solution (at 16^3: the literal
    rule contracts about 0.96 per V-cycle there, 0.98 at 32^3)."""
    case = "wall"
    n = 32 if prec == mg.FP64 else 16
    rho = source((n, n, n), case, seed=77)
    if prec == mg.FP64:
        ref = oracle_solve(rho, case, tol=0.0, max_cycles=3, stall_ratio=NO_STALL,
                           coarse_literal=True)
        phi, hist, st = gpu_solve(rho, case, 0.0, prec=prec, max_cycles=3, stall_ratio=NO_STALL,
                                  coarse_literal=1)
        assert emax(phi, ref.phi) <= 1e-11
        assert np.allclose(hist, ref.hist, rtol=1e-6, atol=1e-14)
    else:
        ref = oracle_solve(rho, case, tol=0.0, max_cycles=80)
        phi, hist, st = gpu_solve(rho, case, 1e-10, prec=prec, coarse_literal=1, stall_ratio=1.0,
                                  max_cycles=250)
        assert st == 0, (st, hist[-3:])
        assert emax(phi, ref.phi) <= 1e-9


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
@pytest.mark.parametrize("kind,value", [(P, 0.0), (F, 0.3), (Z, 0.0)])
def test_six_equal_rules_are_the_uniform_rule(prec, kind, value):
    n = 32
    rho = inputs.gaussian_blobs(n, 8, seed=5, periodic=(kind == P))
    with mg.Solver(n, 1.0 / n, kind, prec=prec, fixed_value=value) as s:
        a, ha, _ = s.solve(torch.from_numpy(rho).cuda(), 1.0, 1e-10)
    with mg.Solver(n, 1.0 / n, [kind] * 6, face_values=[value] * 6, prec=prec) as s:
        b, hb, _ = s.solve(torch.from_numpy(rho).cuda(), 1.0, 1e-10)
    assert torch.equal(a, b) and np.array_equal(ha, hb)


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
def test_gravity_with_face_rules(prec):
    """g = -grad phi with each face's ghosts (Sec. 3.2.3), against the oracle's
    gravity of the returned phi."""
    n, case = 32, "box"
    kinds, values = CASES[case]
    rho = source((n, n, n), case, seed=12)
    with mg.Solver(n, 1.0 / n, list(kinds), face_values=list(values), prec=prec) as s:
        phi, g, hist, st = s.solve_gravity(torch.from_numpy(rho).cuda(), 1.0, 1e-10)
    assert st == 0
    ref = orc.gravity(phi.cpu().numpy(), 1.0 / n, orc.PER_FACE, faces=orc.mixed_rule(kinds, values))
    assert emax(g.cpu().numpy(), ref) <= 1e-13


def test_host_buffers_with_face_rules():
    n, case = 32, "slab"
    kinds, values = CASES[case]
    rho = source((n, n, n), case, seed=13)
    with mg.Solver(n, 1.0 / n, list(kinds), face_values=list(values), prec=mg.MIXED) as s:
        dev, hd, _ = s.solve(torch.from_numpy(rho).cuda(), 1.0, 1e-10)
        host, hh, st = s.solve_host(rho.copy(), 1.0, 1e-10)
    assert st == 0
    assert np.array_equal(np.asarray(host), dev.cpu().numpy()) and np.array_equal(hd, hh)


@pytest.mark.parametrize("case", ["slab", "box"])
@pytest.mark.parametrize("pre,post", [(2, 2), (0, 2), (2, 0)])
def test_mixed_smoothing_counts_with_face_rules(case, pre, post):
    """V(M,N) variants run the fused legs' extra smoothing kernel (and the
    per-level kernels where a leg has no smoothing step) with the face rules;
    the outer loop still reaches the oracle's converged solution."""
    n = 64
    rho = source((n, n, n), case, seed=5 + pre + 3 * post)
    ref = oracle_solve(rho, case, tol=0.0, max_cycles=80)
    phi, hist, st = gpu_solve(rho, case, 1e-10, prec=mg.MIXED, pre=pre, post=post,
                              max_cycles=60)
    assert st == 0 and hist[-1] < 1e-10, (st, hist)
    assert emax(phi, ref.phi) <= 1e-9


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
def test_initial_guess_with_face_rules(prec):
    """MGI mode (Sec. 2.3.7): phi_dev holds the initial guess; a perturbed
    converged solution converges back to it."""
    n, case = 64, "slab"
    kinds, values = CASES[case]
    rho = source((n, n, n), case, seed=61)
    ref = oracle_solve(rho, case, tol=0.0, max_cycles=80)
    guess = ref.phi + 1e-3 * np.sin(np.arange(n ** 3).reshape(n, n, n))
    with mg.Solver(n, 1.0 / n, list(kinds), face_values=list(values), prec=prec,
                   mode_fmg=0) as s:
        phi = torch.from_numpy(np.ascontiguousarray(guess)).cuda()
        phi, hist, st = s.solve(torch.from_numpy(rho).cuda(), 1.0, 1e-10, phi=phi)
    assert st == 0 and hist[-1] < 1e-10, (st, hist)
    assert emax(phi.cpu().numpy(), ref.phi) <= 1e-9


@pytest.mark.parametrize("case", ["slab", "box", "wall"])
def test_mixed_box_with_face_rules(case):
    """A 64 x 64 x 32 box (x, y, z): its finest level runs the fused legs with
    the face rules on a grid shorter in z; the coarsest level has several cells."""
    shape = (32, 64, 64)  # (nz, ny, nx)
    rho = source(shape, case, seed=91)
    ref = oracle_solve(rho, case, tol=0.0, max_cycles=80)
    assert ref.ok
    phi, hist, st = gpu_solve(rho, case, 1e-10, prec=mg.MIXED, max_cycles=60)
    assert st == 0 and hist[-1] < 1e-10, (st, hist)
    assert emax(phi, ref.phi) <= 1e-9
