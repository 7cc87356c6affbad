"""Pins for the CPU oracle: every check here compares it with something other
than itself -- closed-form discrete solutions, a dense direct solve, values the
paper prints, operator invariants, quadrature and library special functions.

None of these tests needs a GPU.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import eval_legendre

from paper_2302_13903_gb300 import inputs

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))
PERIODIC, FIXED, ZEROGRAD, OPEN, FACES = 0, 1, 2, 3, 4


def emax(a, b):
    """Max error relative to the max of the reference."""
    return float(np.abs(a - b).max() / np.abs(b).max())


def grid(n, lo=0.0, hi=1.0):
    x = inputs.cell_centres(n, lo, hi)
    return x[None, None, :], x[None, :, None], x[:, None, None]  # x, y, z broadcastable


# --------------------------------------------------------------------------
# Closed-form discrete solutions (Eq. discretized2 with each boundary rule).

@pytest.mark.parametrize("n,k", [(16, (1, 1, 1)), (32, (1, 2, 3)), (16, (3, 1, 2))])
def test_periodic_sine_mode_is_exact(orc, n, k):
    """sin(2 pi k x) modes are eigenvectors of the periodic 7-point Laplacian:
    lambda = -(4/h^2) sum_d sin^2(pi k_d h)."""
    h = 1.0 / n
    x, y, z = grid(n)
    f = np.sin(2 * np.pi * k[0] * x) * np.sin(2 * np.pi * k[1] * y) * np.sin(2 * np.pi * k[2] * z)
    lam = -(4 / h ** 2) * sum(math.sin(math.pi * kd * h) ** 2 for kd in k)
    r = orc.solve(f, h, PERIODIC, tol=0.0, max_cycles=40)
    assert r.ok, r.hist
    assert emax(r.phi, f / lam) < 1e-12


@pytest.mark.parametrize("b", [0.0, 0.7])
def test_fixed_sine_mode_is_exact(orc, b):
    """With ghost = 2b - active, sin(pi k x) (which vanishes on the faces) plus
    the constant b solves L phi = f exactly for f = lambda sin sin sin."""
    n, k = 16, (1, 2, 3)
    h = 1.0 / n
    x, y, z = grid(n)
    s = np.sin(np.pi * k[0] * x) * np.sin(np.pi * k[1] * y) * np.sin(np.pi * k[2] * z)
    lam = -(4 / h ** 2) * sum(math.sin(math.pi * kd * h / 2) ** 2 for kd in k)
    r = orc.solve(s, h, FIXED, bc_value=b, tol=0.0, max_cycles=40)
    assert r.ok
    ref = b + s / lam
    assert np.abs(r.phi - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_zero_gradient_cosine_mode_is_exact(orc):
    """Zero-gradient ghosts copy the adjacent cell: cos(pi k x) modes are
    eigenvectors; a constant added to rho is removed (Sec. 2.3.6)."""
    n, k = 16, (2, 1, 3)
    h = 1.0 / n
    x, y, z = grid(n)
    c = np.cos(np.pi * k[0] * x) * np.cos(np.pi * k[1] * y) * np.cos(np.pi * k[2] * z)
    lam = -(4 / h ** 2) * sum(math.sin(math.pi * kd * h / 2) ** 2 for kd in k)
    r = orc.solve(c + 3.0, h, ZEROGRAD, tol=0.0, max_cycles=40)
    assert r.ok
    assert emax(r.phi, c / lam) < 1e-12
    assert abs(r.phi.mean()) < 1e-14 * np.abs(r.phi).max()


# --------------------------------------------------------------------------
# Dense direct solve of the same discrete system on small grids.

def dense_system(n, h, bc, b=0.0, faces=None):
    """Matrix of (sum nb - 6u)/h^2 with the ghost eliminated, and the part of
    the operator that the boundary values contribute."""
    N = n ** 3
    A = np.zeros((N, N))
    g = np.zeros(N)
    idx = lambda i, j, k: (k * n + j) * n + i
    if faces is not None:
        sizes = [(n + 2) ** 2] * 6
        offs = np.cumsum([0] + sizes)
        fa = [faces[offs[q]:offs[q + 1]].reshape(n + 2, n + 2) for q in range(6)]
    for k in range(n):
        for j in range(n):
            for i in range(n):
                c = idx(i, j, k)
                A[c, c] -= 6 / h ** 2
                for axis in range(3):
                    for side in (-1, 1):
                        p = [i, j, k]
                        p[axis] += side
                        if 0 <= p[axis] < n:
                            A[c, idx(*p)] += 1 / h ** 2
                        elif bc == PERIODIC:
                            p[axis] %= n
                            A[c, idx(*p)] += 1 / h ** 2
                        elif bc == ZEROGRAD:
                            A[c, c] += 1 / h ** 2
                        else:
                            A[c, c] -= 1 / h ** 2
                            if bc == FIXED:
                                bv = b
                            else:
                                face = 2 * axis + (0 if side < 0 else 1)
                                t = [q + 1 for q in (i, j, k)]
                                del t[axis]
                                bv = fa[face][t[1], t[0]]
                            g[c] += 2 * bv / h ** 2
    return A, g


@pytest.mark.parametrize("bc", [PERIODIC, FIXED, ZEROGRAD, FACES])
@pytest.mark.parametrize("n", [4, 8])
def test_converged_multigrid_equals_dense_solve(orc, bc, n):
    rng = np.random.default_rng(7 + n + bc)
    h = 1.0 / n
    rho = rng.standard_normal((n, n, n))
    faces = rng.standard_normal(orc.faces_size(n, n, n)) if bc == FACES else None
    b = 0.3 if bc == FIXED else 0.0
    A, g = dense_system(n, h, bc, b, faces)
    f = rho.ravel().copy()
    if bc in (PERIODIC, ZEROGRAD):
        f -= f.mean()
        # bordered system: mean of phi is zero
        M = np.zeros((n ** 3 + 1, n ** 3 + 1))
        M[:-1, :-1] = A
        M[:-1, -1] = 1.0
        M[-1, :-1] = 1.0
        ref = np.linalg.solve(M, np.append(f - g, 0.0))[:-1]
    else:
        ref = np.linalg.solve(A, f - g)
    r = orc.solve(rho, h, bc, bc_value=b, faces=faces, fmg=(bc != FACES), tol=0.0, max_cycles=80)
    assert r.ok, (r.status, r.hist)
    assert emax(r.phi.ravel(), ref) < 1e-12


def test_open_boundary_solve_equals_dense_solve_with_multipole_faces(orc):
    n = 8
    h = 1.0 / n
    rho = inputs.uniform_sphere(n, 0.25, 4)
    four_pi_G = 4 * math.pi
    r = orc.solve(rho, h, OPEN, four_pi_G=four_pi_G, tol=0.0, max_cycles=80)
    assert r.ok
    faces = orc.open_faces(n, n, n, h, r.Q, 4, 1.0, r.origin)
    A, g = dense_system(n, h, FACES, faces=faces)
    ref = np.linalg.solve(A, four_pi_G * rho.ravel() - g)
    assert emax(r.phi.ravel(), ref) < 1e-12


# --------------------------------------------------------------------------
# A rule per face (Sec. 2.3.6: the rules may differ between boundaries; a
# fixed value on any face sets the zero point, otherwise the means of f and
# phi are removed).

def dense_system_per_face(n, h, kinds, values):
    """The 7-point operator with each face's own ghost elimination: periodic
    wraps, zero gradient adds the cell itself, fixed b adds 2b - u."""
    N = n ** 3
    A = np.zeros((N, N))
    g = np.zeros(N)
    idx = lambda i, j, k: (k * n + j) * n + i
    for k in range(n):
        for j in range(n):
            for i in range(n):
                c = idx(i, j, k)
                A[c, c] -= 6 / h ** 2
                for axis in range(3):
                    for side in (-1, 1):
                        p = [i, j, k]
                        p[axis] += side
                        face = 2 * axis + (0 if side < 0 else 1)
                        if 0 <= p[axis] < n:
                            A[c, idx(*p)] += 1 / h ** 2
                        elif kinds[face] == PERIODIC:
                            p[axis] %= n
                            A[c, idx(*p)] += 1 / h ** 2
                        elif kinds[face] == ZEROGRAD:
                            A[c, c] += 1 / h ** 2
                        else:
                            A[c, c] -= 1 / h ** 2
                            g[c] += 2 * values[face] / h ** 2
    return A, g


MIXED_CASES = [
    ((PERIODIC, PERIODIC, ZEROGRAD, ZEROGRAD, FIXED, FIXED), (0, 0, 0, 0, 0.3, -0.2)),
    ((FIXED, ZEROGRAD, PERIODIC, PERIODIC, ZEROGRAD, ZEROGRAD), (0.5, 0, 0, 0, 0, 0)),
    ((ZEROGRAD, FIXED, FIXED, ZEROGRAD, FIXED, ZEROGRAD), (0, -0.4, 0.1, 0, 0.7, 0)),
    ((PERIODIC, PERIODIC, ZEROGRAD, ZEROGRAD, ZEROGRAD, ZEROGRAD), (0,) * 6),  # no zero point
]


@pytest.mark.parametrize("case", range(len(MIXED_CASES)))
@pytest.mark.parametrize("n", [4, 8])
def test_per_face_rules_converge_to_the_dense_solve(orc, case, n):
    kinds, values = MIXED_CASES[case]
    rng = np.random.default_rng(60 + 7 * case + n)
    h = 1.0 / n
    rho = rng.standard_normal((n, n, n))
    A, g = dense_system_per_face(n, h, kinds, values)
    f = rho.ravel().copy()
    if FIXED not in kinds:
        f -= f.mean()
        M = np.zeros((n ** 3 + 1, n ** 3 + 1))
        M[:-1, :-1] = A
        M[:-1, -1] = 1.0
        M[-1, :-1] = 1.0
        ref = np.linalg.solve(M, np.append(f - g, 0.0))[:-1]
    else:
        ref = np.linalg.solve(A, f - g)
    for cycle in (orc.CORRECTION, orc.FAS):
        r = orc.solve(rho, h, orc.PER_FACE, faces=orc.mixed_rule(kinds, values), tol=0.0,
                      max_cycles=80, cycle=cycle)
        assert r.ok, (cycle, r.status, r.hist)
        assert emax(r.phi.ravel(), ref) < 1e-12, cycle


@pytest.mark.parametrize("n", [1, 2])
def test_per_face_coarsest_is_exact(orc, n):
    """COARSEST on one or eight cells with the ghosts eliminated face by face
    (a periodic or zero-gradient ghost is the cell itself) equals the dense
    solve; without a fixed face the one-cell system is singular and stays 0."""
    h = 0.5
    kinds, values = MIXED_CASES[2]
    f = np.random.default_rng(3).standard_normal((n, n, n))
    A, g = dense_system_per_face(n, h, kinds, values)
    ref = np.linalg.solve(A, f.ravel() - g)
    if n == 1:
        u = orc.coarsest(f, h, orc.PER_FACE, faces=orc.mixed_rule(kinds, values))
    else:  # N_0,max Gauss-Seidel sweeps do not solve exactly: iterate V-cycles instead
        u = np.zeros_like(f)
        for _ in range(60):
            u = orc.vcycle(u, f, h, orc.PER_FACE, faces=orc.mixed_rule(kinds, values))
    assert emax(u.ravel(), ref) < 1e-12
    kinds0, values0 = MIXED_CASES[3]
    u0 = orc.coarsest(np.ones((1, 1, 1)), h, orc.PER_FACE, faces=orc.mixed_rule(kinds0, values0))
    assert u0[0, 0, 0] == 0.0


def test_per_face_mixed_eigenmode_is_exact(orc):
    """sin(2 pi x) cos(pi y) sin(pi z) with x periodic, y zero gradient and z
    zero fixed is an eigenvector of that operator: lambda is the sum of the
    one-dimensional eigenvalues -(4/h^2) sin^2(pi h), -(4/h^2) sin^2(pi h / 2)
    and -(4/h^2) sin^2(pi h / 2)."""
    n = 32
    h = 1.0 / n
    x, y, z = grid(n)
    f = np.sin(2 * np.pi * x) * np.cos(np.pi * y) * np.sin(np.pi * z)
    lam = -(4 / h ** 2) * (np.sin(np.pi * h) ** 2 + 2 * np.sin(np.pi * h / 2) ** 2)
    kinds = (PERIODIC, PERIODIC, ZEROGRAD, ZEROGRAD, FIXED, FIXED)
    r = orc.solve(f, h, orc.PER_FACE, faces=orc.mixed_rule(kinds), tol=1e-12, max_cycles=60)
    assert r.ok
    assert emax(r.phi, f / lam) < 1e-10


def test_per_face_linear_potential_is_exact(orc):
    """With no source, fixed values a and b on the x faces and zero gradient
    elsewhere the discrete solution is the straight line between them: the
    7-point operator and the ghost 2b - u are exact for linear functions."""
    n = 16
    h = 1.0 / n
    a, b = 0.25, -1.5
    x, _, _ = grid(n)
    kinds = (FIXED, FIXED, ZEROGRAD, ZEROGRAD, ZEROGRAD, ZEROGRAD)
    r = orc.solve(np.zeros((n, n, n)), h, orc.PER_FACE, faces=orc.mixed_rule(kinds, (a, b, 0, 0, 0, 0)),
                  tol=1e-13, max_cycles=80)
    assert r.ok, r.hist
    want = np.broadcast_to(a + (b - a) * x, (n, n, n))
    assert np.abs(r.phi - want).max() < 1e-12


def test_per_face_uniform_descriptor_is_the_uniform_rule(orc):
    n = 16
    rho = inputs.gaussian_blobs(n, 4, seed=8, periodic=False)
    for kind, val in ((PERIODIC, 0.0), (FIXED, 0.3), (ZEROGRAD, 0.0)):
        a = orc.solve(rho, 1.0 / n, kind, bc_value=val, tol=1e-10)
        b = orc.solve(rho, 1.0 / n, orc.PER_FACE, faces=orc.mixed_rule([kind] * 6, [val] * 6),
                      tol=1e-10)
        assert np.array_equal(a.phi, b.phi) and np.array_equal(a.hist, b.hist)


def test_per_face_descriptor_is_checked(orc):
    n = 4
    bad = [(PERIODIC, FIXED, ZEROGRAD, ZEROGRAD, FIXED, FIXED),  # periodic needs its pair
           (OPEN, OPEN, ZEROGRAD, ZEROGRAD, FIXED, FIXED)]  # open faces are all-or-nothing
    for kinds in bad:
        r = orc.solve(np.ones((n, n, n)), 0.25, orc.PER_FACE, faces=orc.mixed_rule(kinds))
        assert r.status == 1


# --------------------------------------------------------------------------
# Convergence behaviour the paper prints (Sec. 4.1.1).

@pytest.mark.parametrize("bc", [PERIODIC, FIXED, ZEROGRAD])
def test_convergence_factor_band(orc, bc):
    """Periodic V(1,1): CF ~ 0.125 and 10-15 cycles (Sec. 4.1.1).  The paper
    prints no factor for the other rules; for them the cell-centred boundary
    treatment slows the slowest mode, so the pin is a bound plus independence
    of N (Sec. 3.4: the iteration count does not grow with N)."""
    cf_paper = GOLDEN["convergence_factor_V11"]["value"]
    lo, hi = GOLDEN["cycles_to_full_convergence"]["value"]
    cfs = []
    for n in (32, 64):
        rho = inputs.gaussian_blobs(n, 16, seed=3, periodic=(bc == PERIODIC))
        r = orc.solve(rho, 1.0 / n, bc, tol=1e-11, omega=GOLDEN["omega"]["value"])
        assert r.ok
        hst = r.hist
        cf = (hst[-1] / hst[-5]) ** 0.25  # asymptotic factor over the last 4 cycles
        cfs.append(cf)
        if bc == PERIODIC:
            assert 0.4 * cf_paper < cf < 1.6 * cf_paper, (n, cf, hst)
            assert len(hst) - 1 <= hi
        else:
            assert cf < 0.35, (n, cf, hst)
            assert len(hst) - 1 <= 20
    assert abs(cfs[0] - cfs[1]) < 0.03


def test_second_order_against_continuum(orc):
    """Converged solutions reach second order against the analytic potential
    phi = -4 pi G A / (3 (2 pi)^2) sin sin sin (Sec. 4.1, Fig. 6d)."""
    s = GOLDEN["sinusoid_test"]
    errs = []
    for n in (16, 32, 64):
        rho = s["rho0"] + s["A"] * inputs.sinusoid(n)
        four_pi_G = 4 * math.pi * s["G"]
        r = orc.solve(rho, 1.0 / n, PERIODIC, four_pi_G=four_pi_G, tol=1e-12)
        assert r.ok
        exact = -four_pi_G * s["A"] / (3 * (2 * math.pi) ** 2) * inputs.sinusoid(n)
        errs.append(np.abs(r.phi - exact).max())
    for a, b in zip(errs, errs[1:]):
        assert 3.8 < a / b < 4.2


def test_single_fmg_sweep_reaches_truncation_error(orc):
    """After one FMG sweep the error against the analytic potential is already
    of the order of the truncation error (Sec. 4.1.1)."""
    n = 64
    rho = inputs.sinusoid(n)
    exact = -1.0 / (12 * math.pi ** 2) * rho
    one = orc.solve(rho, 1.0 / n, PERIODIC, tol=1e-12, max_cycles=0)
    conv = orc.solve(rho, 1.0 / n, PERIODIC, tol=1e-12)
    assert len(one.hist) == 1
    e1, ec = np.abs(one.phi - exact).max(), np.abs(conv.phi - exact).max()
    assert e1 < 2.0 * ec


def test_mgi_and_fmg_reach_the_same_solution(orc):
    n = 32
    rho = inputs.gaussian_blobs(n, 8, seed=11)
    a = orc.solve(rho, 1.0 / n, PERIODIC, tol=1e-12)
    b = orc.solve(rho, 1.0 / n, PERIODIC, tol=1e-12, fmg=False, max_cycles=60)
    assert a.ok and b.ok
    assert len(b.hist) > len(a.hist)  # FMG needs fewer cycles (Sec. 4.1.1)
    assert emax(a.phi, b.phi) < 1e-10


def test_fas_equals_correction_scheme_on_uniform_grid(orc):
    """Algorithm 3 is equivalent to Algorithm 1 for a linear problem on a
    uniform grid (Sec. 2.3.5)."""
    rng = np.random.default_rng(5)
    n = 16
    for bc in (PERIODIC, FIXED, ZEROGRAD):
        u0 = rng.standard_normal((n, n, n))
        f = rng.standard_normal((n, n, n))
        if bc != FIXED:
            f -= f.mean()
        a = orc.vcycle(u0, f, 1.0 / n, bc, bc_value=0.4 if bc == FIXED else 0.0, cycle=0)
        b = orc.vcycle(u0, f, 1.0 / n, bc, bc_value=0.4 if bc == FIXED else 0.0, cycle=1)
        assert np.abs(a - b).max() < 1e-12 * np.abs(a).max()


def test_stall_stops_with_zero_tolerance(orc):
    """A threshold of zero iterates until the reduction stalls (Sec. 2.3.7)."""
    n = 16
    r = orc.solve(inputs.sinusoid(n), 1.0 / n, PERIODIC, tol=0.0, max_cycles=60)
    assert r.ok and len(r.hist) < 60
    assert r.hist[-1] < 1e-13


# --------------------------------------------------------------------------
# The coarse-level rule read word for word (Sec. 2.3.6: zero fixed values on
# the coarse levels of the correction scheme unless the grid is periodic).  By
# default a zero-gradient grid's corrections keep the zero-gradient rule; the
# literal option gives them zero fixed values.

def _vcycle_by_hand(orc, u, f, h, top, coarse):
    """Algorithm 1 on a 4^3 grid (levels 4, 2, 1) from the oracle's pinned
    single operators, rule `top` on the finest level and `coarse` below."""
    u = orc.smooth(u, f, h, top)
    fc = orc.restrict(orc.defect(u, f, h, top))
    uc = orc.smooth(np.zeros_like(fc), fc, 2 * h, coarse)
    fcc = orc.restrict(orc.defect(uc, fc, 2 * h, coarse))
    uc = orc.prolong(orc.coarsest(fcc, 4 * h, coarse), coarse, add=True, uf=uc)
    uc = orc.smooth(uc, fc, 2 * h, coarse)
    u = orc.prolong(uc, coarse, add=True, uf=u)
    return orc.smooth(u, f, h, top)


def test_literal_coarse_rule_vcycle_is_algorithm_1_with_zero_fixed_corrections(orc):
    rng = np.random.default_rng(31)
    n, h = 4, 0.25
    u0 = rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    f -= f.mean()
    lit = orc.vcycle(u0, f, h, ZEROGRAD, coarse_literal=True)
    assert np.array_equal(lit, _vcycle_by_hand(orc, u0, f, h, ZEROGRAD, FIXED))
    hom = orc.vcycle(u0, f, h, ZEROGRAD)
    assert np.array_equal(hom, _vcycle_by_hand(orc, u0, f, h, ZEROGRAD, ZEROGRAD))
    assert np.abs(lit - hom).max() > 1e-3  # the option changes the zero-gradient cycle


@pytest.mark.parametrize("bc", [PERIODIC, FIXED])
def test_literal_coarse_rule_leaves_other_rules_alone(orc, bc):
    n = 16
    rho = inputs.gaussian_blobs(n, 4, seed=2, periodic=(bc == PERIODIC))
    a = orc.solve(rho, 1.0 / n, bc, bc_value=0.2 if bc == FIXED else 0.0, tol=1e-10)
    b = orc.solve(rho, 1.0 / n, bc, bc_value=0.2 if bc == FIXED else 0.0, tol=1e-10,
                  coarse_literal=True)
    assert np.array_equal(a.phi, b.phi) and np.array_equal(a.hist, b.hist)


@pytest.mark.parametrize("n", [4, 8])
def test_literal_coarse_rule_converges_to_the_dense_solution(orc, n):
    """The coarse rule changes only how fast the cycle converges, not the
    discrete problem of the finest level: iterated to the rounding floor, the
    literal reading reaches the same zero-mean solution as a dense solve."""
    rng = np.random.default_rng(40 + n)
    h = 1.0 / n
    rho = rng.standard_normal((n, n, n))
    A, _ = dense_system(n, h, ZEROGRAD)
    f = rho.ravel() - rho.mean()
    M = np.zeros((n ** 3 + 1, n ** 3 + 1))
    M[:-1, :-1] = A
    M[:-1, -1] = 1.0
    M[-1, :-1] = 1.0
    ref = np.linalg.solve(M, np.append(f, 0.0))[:-1]
    r = orc.solve(rho, h, ZEROGRAD, tol=0.0, stall_ratio=1.0, max_cycles=400, hist_cap=512,
                  coarse_literal=True)
    assert r.ok, (r.status, r.hist[-5:])
    assert emax(r.phi.ravel(), ref) < 1e-12


def test_literal_coarse_rule_converges_slowly(orc):
    """Zero fixed corrections cannot represent the smooth modes of a
    zero-gradient defect near the walls, so the factor per V(1,1) cycle is far
    above the homogeneous rule's and grows with N; it stays below 1."""
    cfs = []
    for n in (16, 32):
        rho = inputs.gaussian_blobs(n, 8, seed=5, periodic=False)
        r = orc.solve(rho, 1.0 / n, ZEROGRAD, tol=1e-8, stall_ratio=1.0, max_cycles=600,
                      hist_cap=700, coarse_literal=True)
        assert r.ok, (n, r.status, r.hist[-3:])
        hst = r.hist
        cfs.append((hst[-1] / hst[-11]) ** 0.1)
        hom = orc.solve(rho, 1.0 / n, ZEROGRAD, tol=1e-8)
        assert hom.ok and len(hom.hist) < len(hst) // 4
    assert 0.5 < cfs[0] < cfs[1] < 1.0, cfs


# --------------------------------------------------------------------------
# Operators (Sec. 2.3.1 and 2.3.2).

def test_restriction_preserves_sum_and_constants(orc):
    rng = np.random.default_rng(1)
    u = rng.standard_normal((8, 16, 32))
    c = orc.restrict(u)
    assert c.shape == (4, 8, 16)
    assert abs(c.sum() * 8 - u.sum()) < 1e-12
    assert np.allclose(orc.restrict(np.full((8, 8, 8), 2.5)), 2.5, rtol=0, atol=0)
    # each coarse value is the mean of its own 2x2x2 children
    assert abs(c[1, 2, 3] - u[2:4, 4:6, 6:8].mean()) < 1e-15


def test_prolongation_weights_match_paper(orc):
    """A single coarse delta shows the 1-D weights of Eq. (trilinear) and I'."""
    nc = 8
    uc = np.zeros((nc, nc, nc))
    uc[4, 4, 4] = 1.0
    for high, key, scale in ((False, "trilinear_weights", 1.0), (True, "fmg_weights_32nds", 32.0)):
        uf = orc.prolong(uc, PERIODIC, high_order=high)
        w = GOLDEN[key]
        # fine cells along x at fixed (z, y) = (8, 8) (even, even: w0 = 3/4 or 30/32)
        line = uf[8, 8, :] / (uf[8, 8, 8] / (w["even"][1] / scale))
        # fine cell 10 (even) has the delta as its I-1 neighbour, 7 (odd) as I+1
        assert abs(line[10] - w["even"][0] / scale) < 1e-14
        assert abs(line[9] - w["odd"][1] / scale) < 1e-14
        assert abs(line[7] - w["odd"][2] / scale) < 1e-14
        assert abs(line[6] - w["even"][2] / scale) < 1e-14


def test_prolongation_reproduces_polynomials_in_interior(orc):
    nc = 8
    X = (np.arange(nc) + 0.5) / nc
    xc, yc, zc = X[None, None, :], X[None, :, None], X[:, None, None]
    Xf = (np.arange(2 * nc) + 0.5) / (2 * nc)
    xf, yf, zf = Xf[None, None, :], Xf[None, :, None], Xf[:, None, None]
    inner = (slice(2, -2),) * 3
    lin = lambda x, y, z: 1.0 + 2 * x - 3 * y + 0.5 * z
    quad = lambda x, y, z: 1.0 + x * x - 2 * y * z + 3 * z * z + x * y
    uf = orc.prolong(lin(xc, yc, zc), PERIODIC)
    assert np.abs(uf[inner] - lin(xf, yf, zf)[inner]).max() < 1e-13
    uf = orc.prolong(quad(xc, yc, zc), PERIODIC, high_order=True)
    assert np.abs(uf[inner] - quad(xf, yf, zf)[inner]).max() < 1e-13
    # trilinear is not exact for the quadratic: the test can tell the two apart
    uf = orc.prolong(quad(xc, yc, zc), PERIODIC)
    assert np.abs(uf[inner] - quad(xf, yf, zf)[inner]).max() > 1e-4


def test_prolongation_boundary_ghosts(orc):
    """Constant coarse field: periodic and zero-gradient ghosts keep it; the
    zero-fixed rule (ghost = -active) gives 3/4 - 1/4 = 1/2 per boundary axis."""
    uc = np.full((4, 4, 4), 2.0)
    assert np.allclose(orc.prolong(uc, PERIODIC), 2.0, atol=1e-15)
    assert np.allclose(orc.prolong(uc, ZEROGRAD), 2.0, atol=1e-15)
    uf = orc.prolong(uc, FIXED, bc_value=0.0)
    assert abs(uf[0, 0, 0] - 2.0 / 8) < 1e-15     # corner: three boundary axes
    assert abs(uf[4, 4, 0] - 2.0 / 2) < 1e-15     # face: one boundary axis
    assert abs(uf[4, 4, 4] - 2.0) < 1e-15         # interior


def test_red_then_black_sor_update(orc):
    """A red half-sweep changes only (i+j+k)-even cells and scales their
    defect by (1 - omega); the black half-sweep does the same for odd cells."""
    rng = np.random.default_rng(3)
    n, h, om = 8, 1.0 / 8, GOLDEN["omega"]["value"]
    u = rng.standard_normal((n, n, n))
    f = rng.standard_normal((n, n, n))
    k, j, i = np.meshgrid(range(n), range(n), range(n), indexing="ij")
    red = (i + j + k) % 2 == 0
    inner = np.zeros_like(red)
    inner[1:-1, 1:-1, 1:-1] = True
    for bc in (PERIODIC, FIXED, ZEROGRAD):
        # Away from non-periodic faces a cell's ghosts do not depend on itself,
        # so the relation is exact there.
        sel = np.ones_like(red) if bc == PERIODIC else inner
        d0 = orc.defect(u, f, h, bc, bc_value=0.2)
        ur = orc.smooth(u, f, h, bc, bc_value=0.2, omega=om, colours=1)
        assert np.array_equal(ur[~red], u[~red])
        d1 = orc.defect(ur, f, h, bc, bc_value=0.2)
        m = red & sel
        assert np.abs(d1[m] - (1 - om) * d0[m]).max() < 1e-10 * np.abs(d0).max()
        ub = orc.smooth(ur, f, h, bc, bc_value=0.2, omega=om, colours=2)
        assert np.array_equal(ub[red], ur[red])
        d2 = orc.defect(ub, f, h, bc, bc_value=0.2)
        m = ~red & sel
        assert np.abs(d2[m] - (1 - om) * d1[m]).max() < 1e-10 * np.abs(d0).max()
        both = orc.smooth(u, f, h, bc, bc_value=0.2, omega=om, colours=0)
        assert np.array_equal(both, ub)


@pytest.mark.parametrize("bc", [FIXED, FACES])
def test_one_cell_coarsest_is_exact(orc, bc):
    rng = np.random.default_rng(9)
    f = np.array([[[1.7]]])
    faces = rng.standard_normal(orc.faces_size(1, 1, 1)) if bc == FACES else None
    u = orc.coarsest(f, 2.0, bc, bc_value=0.4, faces=faces)
    d = orc.defect(u, f, 2.0, bc, bc_value=0.4, faces=faces)
    assert abs(d[0, 0, 0]) < 1e-14
    assert orc.coarsest(np.zeros((1, 1, 1)), 2.0, PERIODIC)[0, 0, 0] == 0.0


# --------------------------------------------------------------------------
# Multipole expansion (App. A).

def test_ylm_orthonormal_by_quadrature(orc):
    mu, wmu = np.polynomial.legendre.leggauss(24)
    nphi = 24
    phis = 2 * np.pi * np.arange(nphi) / nphi
    pts, wts = [], []
    for m_, w_ in zip(mu, wmu):
        s = math.sqrt(1 - m_ * m_)
        for p in phis:
            pts.append((s * math.cos(p), s * math.sin(p), m_))
            wts.append(w_ * 2 * np.pi / nphi)
    lm = [(l, m) for l in range(5) for m in range(-l, l + 1)]
    Y = np.array([[orc.ylm(l, m, *p) for p in pts] for l, m in lm])
    G = (Y * np.array(wts)) @ Y.T
    assert np.abs(G - np.eye(len(lm))).max() < 1e-12


def test_ylm_addition_theorem(orc):
    rng = np.random.default_rng(2)
    for _ in range(20):
        a = rng.standard_normal(3); a /= np.linalg.norm(a)
        b = rng.standard_normal(3); b /= np.linalg.norm(b)
        for l in range(5):
            s = sum(orc.ylm(l, m, *a) * orc.ylm(l, m, *b) for m in range(-l, l + 1))
            assert abs(s - (2 * l + 1) / (4 * np.pi) * eval_legendre(l, a @ b)) < 1e-13


def test_ylm_normalisation_constants_from_table(orc):
    """At a generic direction, each Y_lm divided by its printed constant
    sqrt(c/pi) * prefactor must be a polynomial that the Legendre addition
    theorem already fixes; here we check the printed constants give unit norm
    (the quadrature test) *and* that the table's l = 0 and l = 1 entries take
    their printed values on the axes."""
    t = GOLDEN["ylm_normalisation_squared_times_pi"]
    assert abs(orc.ylm(0, 0, 0, 0, 1) - math.sqrt(t["0,0"][0] / math.pi)) < 1e-15
    assert abs(orc.ylm(1, 1, 1, 0, 0) - math.sqrt(t["1,1"][0] / math.pi)) < 1e-15
    assert abs(orc.ylm(1, -1, 0, 1, 0) - math.sqrt(t["1,-1"][0] / math.pi)) < 1e-15
    assert abs(orc.ylm(1, 0, 0, 0, 1) - math.sqrt(t["1,0"][0] / math.pi)) < 1e-15
    assert abs(orc.ylm(2, 0, 0, 0, 1) - 2 * math.sqrt(t["2,0"][0] / math.pi)) < 1e-15


def test_multipole_point_masses(orc):
    """Q_00 is the mass; about the centre of mass the dipole vanishes; far away
    the truncated expansion matches -G sum m / |r - r'| to O((r'/r)^5), and the
    l = 0 term has the attractive sign (-G M / r)."""
    n, h = 16, 1.0 / 16
    rho = np.zeros((n, n, n))
    rho[8, 8, 9] = 3.0
    rho[7, 6, 8] = 1.0
    rho[9, 8, 5] = 2.0
    Q, org = orc.multipole_moments(rho, h, 4, use_com=True)
    M = rho.sum() * h ** 3
    assert abs(Q[0] - M) < 1e-15
    assert np.abs(Q[1:4]).max() < 1e-15
    c = inputs.cell_centres(n, -0.5, 0.5)
    pts = [(c[i], c[j], c[k], rho[k, j, i] * h ** 3) for k, j, i in np.argwhere(rho != 0)]
    com = sum(np.array(p[:3]) * p[3] for p in pts) / M
    assert np.abs(org - com).max() < 1e-15
    G = 0.7
    for R in (1.5, 3.0):
        for d in ([1, 0, 0], [0.3, -0.5, 0.8], [0, 0, -1]):
            d = np.array(d) / np.linalg.norm(d)
            x = com + R * d
            exact = -G * sum(p[3] / np.linalg.norm(x - np.array(p[:3])) for p in pts)
            approx = orc.multipole_potential(Q, 4, G, org, *x)
            rmax = max(np.linalg.norm(np.array(p[:3]) - com) for p in pts)
            assert abs(approx - exact) <= 2 * abs(exact) * (rmax / R) ** 5
            l0 = orc.multipole_potential(Q, 0, G, org, *x)
            assert abs(l0 + G * M / R) < 1e-14


def test_uniform_sphere_open_boundary_second_order(orc):
    """Open boundaries from the multipole expansion: the converged potential of
    a cell-averaged uniform sphere approaches the analytic one at O(h^2)
    (Sec. 4.2.1 test with the uniform-sphere workload)."""
    s = GOLDEN["sphere_test"]
    errs = []
    for n in (32, 64):
        rho = inputs.uniform_sphere(n, s["R"], s["subcells_per_axis"])
        r = orc.solve(rho, 1.0 / n, OPEN, four_pi_G=4 * math.pi, tol=1e-11)
        assert r.ok
        exact = inputs.sphere_potential(n, s["R"], G=1.0)
        errs.append(np.abs(r.phi - exact).max() / np.abs(exact).max())
    assert errs[0] < 5e-3
    assert 2.5 < errs[0] / errs[1] < 6.0


# ---------------------------------------------------------------------------
# Cell-centred gravitational acceleration (Sec. 3.2.3): the average of the two
# face accelerations along each axis.

def test_gravity_periodic_sinusoid_closed_form(orc):
    """For phi = sin 2pi x sin 2pi y sin 2pi z at cell centres the average of the
    two face differences is the central difference, whose value on a sine is
    known in closed form: g_x = -(sin(2 pi h) / h) cos 2pi x sin 2pi y sin 2pi z."""
    n = 16
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    s, c = np.sin(2 * np.pi * x), np.cos(2 * np.pi * x)
    phi = s[:, None, None] * s[None, :, None] * s[None, None, :]
    g = orc.gravity(phi, h, PERIODIC)
    k = np.sin(2 * np.pi * h) / h
    gx = -k * s[:, None, None] * s[None, :, None] * c[None, None, :]
    gy = -k * s[:, None, None] * c[None, :, None] * s[None, None, :]
    gz = -k * c[:, None, None] * s[None, :, None] * s[None, None, :]
    for got, want in zip(g, (gx, gy, gz)):
        assert np.abs(got - want).max() <= 1e-13 * k


def test_gravity_zero_gradient_cosine_closed_form(orc):
    """phi = cos(pi x) (x only): the zero-gradient ghost equals the mirrored
    cosine, so g_x = sin(pi x) sin(pi h) / h holds up to the boundary cells;
    g_y = g_z = 0."""
    n = 8
    h = 1.0 / n
    x = (np.arange(n) + 0.5) * h
    phi = np.broadcast_to(np.cos(np.pi * x)[None, None, :], (n, n, n)).copy()
    g = orc.gravity(phi, h, ZEROGRAD)
    want = np.sin(np.pi * x) * np.sin(np.pi * h) / h
    assert np.abs(g[0] - want[None, None, :]).max() <= 1e-13
    assert np.abs(g[1]).max() == 0.0 and np.abs(g[2]).max() == 0.0


def test_gravity_given_faces_linear_potential(orc):
    """A linear potential with its own values on the faces (ghost = 2 b - cell,
    applied x, then y, then z) is continued linearly into every ghost, so g is
    the constant -(a, b, c) in every cell including edges and corners."""
    n = 4
    h = 1.0 / n
    a, b, c, d = 0.7, -1.3, 2.1, 0.4
    lin = lambda x, y, z: a * x + b * y + c * z + d
    p = (np.arange(n + 2) - 0.5) * h  # padded index -> coordinate
    faces = []
    for face in range(6):
        axis, hi = divmod(face, 2)
        wall = 1.0 if hi else 0.0
        if axis == 0:
            A, B = np.meshgrid(p, p, indexing="xy")  # (k, j) grid, j fastest
            vals = lin(wall, A, B)
        elif axis == 1:
            A, B = np.meshgrid(p, p, indexing="xy")  # (k, i)
            vals = lin(A, wall, B)
        else:
            A, B = np.meshgrid(p, p, indexing="xy")  # (j, i)
            vals = lin(A, B, wall)
        faces.append(vals.ravel())
    faces = np.concatenate(faces)
    assert faces.size == orc.faces_size(n, n, n)
    xc = (np.arange(n) + 0.5) * h
    phi = lin(xc[None, None, :], xc[None, :, None], xc[:, None, None])
    g = orc.gravity(phi, h, FACES, faces=faces)
    for comp, want in zip(g, (-a, -b, -c)):
        assert np.abs(comp - want).max() <= 1e-12


def test_gravity_fixed_rule_boundary_cells(orc):
    """Fixed value b: the ghost is 2 b - phi, so in the first cell the
    left face acceleration is -(phi_0 - b) / (h / 2); check one cell by hand."""
    n = 4
    h = 1.0 / n
    rng = np.random.default_rng(3)
    phi = rng.standard_normal((n, n, n))
    bval = 0.3
    g = orc.gravity(phi, h, FIXED, bc_value=bval)
    k, j = 2, 1
    ghost = 2 * bval - phi[k, j, 0]
    want = 0.5 * (-(phi[k, j, 0] - ghost) / h - (phi[k, j, 1] - phi[k, j, 0]) / h)
    assert abs(g[0, k, j, 0] - want) <= 1e-14 * max(1.0, abs(want))


# ---------------------------------------------------------------------------
# Non-cubic grids (the Jeans-wave box 1 x 0.5 x 0.5 of Sec. 4.3): levels are
# halved until the shortest side has one cell, so the coarsest level has more
# than one cell and COARSEST is N_0,max Gauss-Seidel sweeps (Sec. 2.3.2).

def dense_system_box(nx, ny, nz, h, bc, b=0.0):
    """(sum nb - 6u)/h^2 on an nx*ny*nz box with the ghost eliminated."""
    N = nx * ny * nz
    A = np.zeros((N, N))
    g = np.zeros(N)
    dims = (nx, ny, nz)
    idx = lambda i, j, k: (k * ny + j) * nx + i
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                c = idx(i, j, k)
                A[c, c] -= 6 / h ** 2
                for axis in range(3):
                    for side in (-1, 1):
                        p = [i, j, k]
                        p[axis] += side
                        if 0 <= p[axis] < dims[axis]:
                            A[c, idx(*p)] += 1 / h ** 2
                        elif bc == PERIODIC:
                            p[axis] %= dims[axis]
                            A[c, idx(*p)] += 1 / h ** 2
                        elif bc == ZEROGRAD:
                            A[c, c] += 1 / h ** 2
                        else:
                            A[c, c] -= 1 / h ** 2
                            g[c] += 2 * b / h ** 2
    return A, g


@pytest.mark.parametrize("bc", [PERIODIC, FIXED, ZEROGRAD])
@pytest.mark.parametrize("shape", [(8, 4, 4), (8, 8, 2), (4, 2, 2)])
def test_non_cubic_converged_multigrid_equals_dense_solve(orc, bc, shape):
    nx, ny, nz = shape
    rng = np.random.default_rng(nx * 100 + ny * 10 + nz + bc)
    h = 1.0 / nx
    rho = rng.standard_normal((nz, ny, nx))
    b = 0.3 if bc == FIXED else 0.0
    A, g = dense_system_box(nx, ny, nz, h, bc, b)
    f = rho.ravel().copy()
    if bc in (PERIODIC, ZEROGRAD):
        f -= f.mean()
        M = np.zeros((f.size + 1, f.size + 1))
        M[:-1, :-1] = A
        M[:-1, -1] = 1.0
        M[-1, :-1] = 1.0
        ref = np.linalg.solve(M, np.append(f - g, 0.0))[:-1]
    else:
        ref = np.linalg.solve(A, f - g)
    r = orc.solve(rho, h, bc, bc_value=b, tol=0.0, max_cycles=80)
    assert r.ok, (r.status, r.hist)
    assert emax(r.phi.ravel(), ref) < 1e-12


def test_jeans_box_periodic_mode_is_exact(orc):
    """Periodic 1 x 0.5 x 0.5 box (32 x 16 x 16 cells): the mode
    sin 2pi x sin 4pi y sin 4pi z is an eigenvector of the 7-point operator,
    eigenvalue -(4/h^2)(sin^2(pi h) + 2 sin^2(2 pi h)); the converged solve
    returns rho / lambda.  The coarsest level is 2 x 1 x 1."""
    nx, ny, nz = 32, 16, 16
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    rho = (np.sin(4 * np.pi * y)[:, None, None] * np.sin(4 * np.pi * y)[None, :, None] *
           np.sin(2 * np.pi * x)[None, None, :])
    lam = -(4 / h ** 2) * (math.sin(math.pi * h) ** 2 + 2 * math.sin(2 * math.pi * h) ** 2)
    r = orc.solve(rho, h, PERIODIC, tol=0.0, max_cycles=60)
    assert r.ok and len(r.hist) < 60
    assert emax(r.phi, rho / lam) < 1e-12


# ---------------------------------------------------------------------------
# The FMG ladder under non-periodic rules (Algorithm 2 with the physical rule
# on every level, Sec. 2.3.6): one sweep must already be near the truncation
# error, which a rule applied wrongly on the coarse FMG levels (a dropped
# boundary value, the wrong rule, open-boundary values at the wrong points)
# would spoil.

def test_fmg_sweep_fixed_rule_with_boundary_value(orc):
    """Fixed b = 0.7: phi = b + s / lambda_c for f = s = sin(pi x) sin(2 pi y)
    sin(3 pi z), the continuum solution.  One FMG sweep is within 2x of the
    converged error against it (which is the truncation error), at 32^3 and
    64^3."""
    k, b = (1, 2, 3), 0.7
    for n in (32, 64):
        h = 1.0 / n
        x, y, z = grid(n)
        s = np.sin(np.pi * k[0] * x) * np.sin(np.pi * k[1] * y) * np.sin(np.pi * k[2] * z)
        exact = b + s / (-(math.pi ** 2) * sum(kk * kk for kk in k))
        one = orc.solve(s, h, FIXED, bc_value=b, tol=0.0, max_cycles=0)
        conv = orc.solve(s, h, FIXED, bc_value=b, tol=0.0, max_cycles=60)
        assert len(one.hist) == 1 and conv.ok
        e1, ec = np.abs(one.phi - exact).max(), np.abs(conv.phi - exact).max()
        assert ec < 2e-4 / (n / 32) ** 2  # second order
        assert e1 < 2.0 * ec, (n, e1, ec)


def test_fmg_sweep_zero_gradient_rule(orc):
    """Zero gradient, f = cos(2 pi x) cos(pi y) cos(3 pi z): the continuum
    solution is f / lambda_c.  The zero-gradient cycle contracts by about 0.29
    (against 0.1 for periodic), so one FMG sweep lands a few times above the
    truncation error (2.5x at 32^3, 3.7x at 64^3) and FMG plus one V-cycle
    within 1.1x of it."""
    for n, bound in ((32, 3.0), (64, 4.5)):
        h = 1.0 / n
        x, y, z = grid(n)
        c = np.cos(2 * np.pi * x) * np.cos(np.pi * y) * np.cos(3 * np.pi * z)
        exact = c / (-(math.pi ** 2) * (4 + 1 + 9))
        one = orc.solve(c, h, ZEROGRAD, tol=0.0, max_cycles=0)
        two = orc.solve(c, h, ZEROGRAD, tol=0.0, max_cycles=1, stall_ratio=1e300)
        conv = orc.solve(c, h, ZEROGRAD, tol=0.0, max_cycles=60)
        e1, e2, ec = (np.abs(r.phi - exact).max() for r in (one, two, conv))
        assert e1 < bound * ec, (n, e1, ec)
        assert e2 < 1.1 * ec, (n, e2, ec)


def test_fmg_sweep_open_uniform_sphere(orc):
    """Open boundaries, the uniform sphere of the golden values against its
    analytic potential: one FMG sweep within 2x of the converged error."""
    s = GOLDEN["sphere_test"]
    for n in (32, 64):
        rho = inputs.uniform_sphere(n, s["R"], s["subcells_per_axis"])
        exact = inputs.sphere_potential(n, s["R"], G=1.0)
        one = orc.solve(rho, 1.0 / n, OPEN, four_pi_G=4 * math.pi, tol=0.0, max_cycles=0)
        conv = orc.solve(rho, 1.0 / n, OPEN, four_pi_G=4 * math.pi, tol=1e-12)
        e1, ec = np.abs(one.phi - exact).max(), np.abs(conv.phi - exact).max()
        assert e1 < 2.0 * ec, (n, e1, ec)


def _face_points(nx, ny, nz, H):
    """Positions of every point of a faces array (x-, x+, y-, y+, z-, z+; the
    documented layout, index 0 and n+1 the extended points) of a level of
    nx*ny*nz cells of width H, centred on the origin."""
    def centre(a, m):  # padded index a in 0..m+1 -> cell-centre coordinate
        return (a - 0.5 - m / 2.0) * H
    pts = []
    for face in range(6):
        axis, hi = divmod(face, 2)
        n = (nx, ny, nz)
        wall = (0.5 if hi else -0.5) * n[axis] * H
        others = [a for a in range(3) if a != axis]  # (first, second) index axes
        ma, mb = n[others[0]], n[others[1]]
        for bidx in range(mb + 2):
            for aidx in range(ma + 2):
                p = [0.0, 0.0, 0.0]
                p[axis] = wall
                p[others[0]] = centre(aidx, ma)
                p[others[1]] = centre(bidx, mb)
                pts.append(p)
    return np.array(pts)


def test_open_faces_of_every_level_at_its_own_face_points(orc):
    """A single massive cell: its expansion about the centre of mass is the
    monopole alone, so the boundary value at any point p is -G M / |p - c|
    (App. A at l = 0; G = 1 here).  Each level of the FMG hierarchy carries
    that value at its own face points, which move between levels (Sec.
    2.3.6); computed here from the geometry, not from the oracle's faces."""
    n, h = 32, 1.0 / 32
    rho = np.zeros((n, n, n))
    i, j, k = 5, 20, 9
    rho[k, j, i] = 3.0
    M = 3.0 * h ** 3
    c = np.array([(i + 0.5 - n / 2) * h, (j + 0.5 - n / 2) * h, (k + 0.5 - n / 2) * h])
    for level in range(6):
        m = n >> (5 - level)
        got = orc.open_level_faces(rho, h, level, lmax=4, four_pi_G=4 * math.pi)
        p = _face_points(m, m, m, h * (n // m))
        want = -M / np.linalg.norm(p - c, axis=1)
        assert np.abs(got - want).max() < 1e-12 * np.abs(want).max(), level


def test_fx_step_integer_defect(orc):
    """The exact integer defect of the mixed outer loop against the FP64 defect
    of Eq. (defect) (orc.defect, pinned above) on values where FP64 is exact:
    with 2^S = 1 and h = 1, R = F - (sum_nb P' - 6 P') is f - L u for u = P',
    f = F, fixed faces b_q = B_q / 2."""
    rng = np.random.default_rng(3)
    shape = (8, 16, 32)
    kinds = [orc.FIXED, orc.ZEROGRAD, orc.PERIODIC, orc.PERIODIC, orc.ZEROGRAD, orc.FIXED]
    b = [1.5, 0.0, 0.0, 0.0, 0.0, -2.5]
    phi = rng.integers(-1000, 1000, size=shape)
    F = rng.integers(-1000, 1000, size=shape)
    e = rng.integers(-50, 50, size=shape).astype(np.float32) * np.float32(0.25)
    out, r = orc.fx_step(phi, e, 4.0, F, kinds, b, 1.0, 1.0)
    assert np.array_equal(out, phi + (e * np.float32(4.0)).astype(np.int64))
    d = orc.defect(out.astype(np.float64), F.astype(np.float64), 1.0, orc.PER_FACE,
                   faces=orc.mixed_rule(kinds, b))
    assert np.array_equal(r.astype(np.float64), d)


def test_fx_step_rounding(orc):
    """round(e c) rounds half to even (2.5 -> 2, 3.5 -> 4, -2.5 -> -2); with
    P = 0 and no correction the residual is F itself, scaled in FP32."""
    F = np.zeros((2, 2, 2), dtype=np.int64)
    e = np.array([2.5, 3.5, -2.5, -3.5, 0.49999997, 1.5, 0.5, -0.5], np.float32).reshape(2, 2, 2)
    out, _ = orc.fx_step(None, e, 1.0, F, [orc.PERIODIC] * 6, [0.0] * 6, 1.0, 1.0)
    assert out.ravel().tolist() == [2, 4, -2, -4, 0, 2, 0, 0]
    F = np.arange(8, dtype=np.int64).reshape(2, 2, 2) * (2 ** 40 + 3)
    _, r = orc.fx_step(None, None, 1.0, F, [orc.ZEROGRAD] * 6, [0.0] * 6, 1.0, 0.5)
    assert np.array_equal(r, F.astype(np.float32) * np.float32(0.5))
