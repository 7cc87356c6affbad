"""Whole-solve parity through the C ABI against the oracle.

FP64 path: the same schedule (FMG + k V-cycles) on both sides agrees to
e_max = max|phi_gpu - phi_ref| / max|phi_ref| <= 1e-11 at every k, and the
solve to tolerance agrees with the oracle's converged solution to 1e-11.
Mixed path (FP32 multigrid inside an FP64-accurate defect correction, with
the outer residual in FP64 or exact 64-bit fixed point): the solution at
||d||/||f|| < 1e-10 agrees with the oracle's converged FP64 solution to 1e-9.
"""
import math

import numpy as np
import pytest
import torch

import oracle as orc
import paper_2302_13903_gb300 as mg
from paper_2302_13903_gb300 import inputs

pytestmark = pytest.mark.gpu

BCS = [mg.PERIODIC, mg.FIXED, mg.ZEROGRAD, mg.OPEN]
NO_STALL = 1e300


def emax(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def source(n, bc, seed=5):
    if bc == mg.OPEN:
        rho = inputs.uniform_sphere(n, 0.25, 4)
        return rho * (1.0 + 0.2 * np.random.default_rng(seed).random(rho.shape)), 4 * math.pi
    return inputs.gaussian_blobs(n, 8, seed=seed, periodic=(bc == mg.PERIODIC)), 1.0


def gpu_solve(rho, bc, four_pi_G, tol, prec=mg.FP64, **opts):
    n = rho.shape[0]
    with mg.Solver(n, 1.0 / n, bc, prec=prec, fixed_value=0.25 if bc == mg.FIXED else 0.0,
                   **opts) as s:
        phi, hist, st = s.solve(torch.from_numpy(rho).cuda(), four_pi_G, tol)
        return phi.cpu().numpy(), hist, st, s.last_launches


@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", [8, 32])
def test_fp64_same_schedule_matches_oracle(bc, n):
    rho, fpg = source(n, bc)
    for k in (0, 1, 3):
        ref = orc.solve(rho, 1.0 / n, bc, bc_value=0.25 if bc == mg.FIXED else 0.0, four_pi_G=fpg,
                        tol=0.0, max_cycles=k, stall_ratio=NO_STALL)
        phi, hist, st, _ = gpu_solve(rho, bc, fpg, 0.0, max_cycles=k, stall_ratio=NO_STALL)
        assert len(hist) == len(ref.hist) == k + 1
        assert st == ref.status
        assert emax(phi, ref.phi) <= 1e-11, (k, emax(phi, ref.phi))
        assert np.allclose(hist, ref.hist, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("bc", BCS)
def test_fp64_to_tolerance_matches_oracle(bc):
    """Same stopping rule on both sides: the same cycles and the same phi."""
    n = 32
    rho, fpg = source(n, bc, seed=8)
    ref = orc.solve(rho, 1.0 / n, bc, bc_value=0.25 if bc == mg.FIXED else 0.0, four_pi_G=fpg,
                    tol=1e-10)
    phi, hist, st, launches = gpu_solve(rho, bc, fpg, 1e-10)
    assert st == 0 and hist[-1] < 1e-10 and launches > 0
    assert len(hist) == len(ref.hist)
    assert emax(phi, ref.phi) <= 1e-11


@pytest.mark.parametrize("bc", BCS)
def test_fp64_converged_matches_converged_oracle(bc):
    """Iterating until the reduction stalls (tol = 0) on both sides reaches the
    discrete solution: the two agree to 1e-11 whatever the cycle counts."""
    n = 32
    rho, fpg = source(n, bc, seed=8)
    ref = orc.solve(rho, 1.0 / n, bc, bc_value=0.25 if bc == mg.FIXED else 0.0, four_pi_G=fpg,
                    tol=0.0, max_cycles=80)
    phi, hist, st, _ = gpu_solve(rho, bc, fpg, 0.0, max_cycles=80)
    assert st == 0 and ref.ok
    assert emax(phi, ref.phi) <= 1e-11


def test_fp64_sinusoid_64_exact_discrete_solution():
    """The 64^3 periodic sinusoid: FMG + V(1,1) to 1e-10 reaches the exact
    discrete solution phi*_h = -h^2 f / (12 sin^2(pi h))."""
    n = 64
    h = 1.0 / n
    rho = inputs.sinusoid(n)
    phi, hist, st, _ = gpu_solve(rho, mg.PERIODIC, 1.0, 1e-10)
    exact = -h * h * rho / (12 * math.sin(math.pi * h) ** 2)
    assert st == 0 and len(hist) <= 16
    assert emax(phi, exact) < 1e-9
    ref = orc.solve(rho, h, mg.PERIODIC, tol=1e-10)
    assert len(ref.hist) == len(hist)
    assert emax(phi, ref.phi) <= 1e-11


@pytest.mark.parametrize("outer_fixed", [1, 0])
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("n", [16, 64])
def test_mixed_matches_converged_oracle(bc, n, outer_fixed):
    """Both outer loops -- the exact 64-bit fixed-point residual (default) and
    the FP64 one -- reach the oracle's converged FP64 solution."""
    rho, fpg = source(n, bc, seed=9)
    ref = orc.solve(rho, 1.0 / n, bc, bc_value=0.25 if bc == mg.FIXED else 0.0, four_pi_G=fpg,
                    tol=0.0, max_cycles=80)
    phi, hist, st, _ = gpu_solve(rho, bc, fpg, 1e-10, prec=mg.MIXED, outer_fixed=outer_fixed)
    assert st == 0, (st, hist)
    assert hist[-1] < 1e-10
    assert emax(phi, ref.phi) <= 1e-9


@pytest.mark.parametrize("b", [-3.0, 10.0])
@pytest.mark.parametrize("gravity", [False, True])
def test_mixed_fixed_value_offset(b, gravity):
    """A fixed value b on every face (Sec. 2.3.6): the mixed path solves for
    phi - b, whose faces are zero-fixed, and adds b back.  Against the oracle's
    converged solution with the same b, also where b dwarfs the potential the
    source makes (10) -- the offset takes no bits of the fixed-point scale --
    and through the solve that also writes g = -grad phi."""
    n = 64
    rho, fpg = source(n, mg.FIXED, seed=13)
    ref = orc.solve(rho, 1.0 / n, mg.FIXED, bc_value=b, four_pi_G=fpg, tol=0.0, max_cycles=80)
    with mg.Solver(n, 1.0 / n, mg.FIXED, prec=mg.MIXED, fixed_value=b) as s:
        rd = torch.from_numpy(rho).cuda()
        if gravity:
            phi, g, hist, st = s.solve_gravity(rd, fpg, 1e-10)
            g0 = s.solve_gravity(rd, fpg, 1e-10)[1]  # the same again: deterministic
            assert torch.equal(g, g0)
        else:
            phi, hist, st = s.solve(rd, fpg, 1e-10)
    assert st == 0 and hist[-1] < 1e-10, (st, hist)
    assert emax(phi.cpu().numpy(), ref.phi) <= 1e-9


@pytest.mark.parametrize("inner_fmg,inner_cycles", [(1, 1), (1, 3), (0, 1), (0, 5)])
@pytest.mark.parametrize("bc", [mg.PERIODIC, mg.ZEROGRAD])
def test_mixed_inner_schedules(inner_fmg, inner_cycles, bc):
    """Every inner schedule of the FP32 solves converges to the same FP64
    solution (the outer FP64 loop decides the accuracy)."""
    n = 64
    rho, fpg = source(n, bc, seed=21)
    ref = orc.solve(rho, 1.0 / n, bc, four_pi_G=fpg, tol=0.0, max_cycles=80)
    phi, hist, st, _ = gpu_solve(rho, bc, fpg, 1e-10, prec=mg.MIXED, inner_fmg=inner_fmg,
                                 inner_cycles=inner_cycles)
    assert st == 0 and hist[-1] < 1e-10
    assert emax(phi, ref.phi) <= 1e-9


@pytest.mark.parametrize("bc", [mg.PERIODIC, mg.ZEROGRAD, mg.OPEN])
def test_first_outer_iteration_cycles(bc):
    """first_cycles changes only the first outer iteration's inner solve: one
    V-cycle there leaves a larger first residual, the later iterations keep
    1 + inner_cycles, and the solve still reaches the oracle's converged
    solution; first_cycles = 1 + inner_cycles is the default schedule, bit for
    bit, through both inner-solve graphs (a second solve replays them)."""
    n = 64 if bc != mg.OPEN else 32
    rho, fpg = source(n, bc, seed=41)
    ref = orc.solve(rho, 1.0 / n, bc, four_pi_G=fpg, tol=0.0, max_cycles=80)
    rd = torch.from_numpy(rho).cuda()
    runs = {}
    for first in (0, 4, 1):
        with mg.Solver(n, 1.0 / n, bc, prec=mg.MIXED, first_cycles=first) as s:
            s.solve(rd, fpg, 1e-10)
            phi, hist, st = s.solve(rd, fpg, 1e-10)
        assert st == 0 and hist[-1] < 1e-10, (first, hist)
        assert emax(phi.cpu().numpy(), ref.phi) <= 1e-9
        runs[first] = (phi, hist)
    assert torch.equal(runs[4][0], runs[0][0]) and np.array_equal(runs[4][1], runs[0][1])
    assert runs[1][1][0] > 10 * runs[0][1][0]
    with pytest.raises(mg.MGError):
        mg.Solver(8, 1.0 / 8, bc, prec=mg.MIXED, first_cycles=66)


def test_batch_first_outer_iteration_cycles():
    """The batched solve takes first_cycles for its first outer iteration as
    mg_solve does (the first residual grows with one V-cycle there) and still
    converges; more than 17 is refused."""
    n = 32
    rho = inputs.gaussian_blobs(n, 4, seed=43)
    ref = orc.solve(rho, 1.0 / n, mg.PERIODIC, tol=0.0, max_cycles=80)
    rd = torch.from_numpy(rho).cuda()
    hists = {}
    for first in (0, 1):
        with mg.Batch([n], [1.0 / n], [mg.PERIODIC], first_cycles=first) as b:
            pd = torch.zeros_like(rd)
            st, h, _ = b.solve([rd], [pd], 1.0, 1e-10)
        assert st == 0 and h[0][-1] < 1e-10, (first, h)
        assert emax(pd.cpu().numpy(), ref.phi) <= 1e-9
        hists[first] = h[0]
    assert hists[1][0] > 10 * hists[0][0]
    with pytest.raises(mg.MGError):
        mg.Batch([n], [1.0 / n], [mg.PERIODIC], first_cycles=18)


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
def test_mgi_initial_guess(prec):
    n = 16
    rho, _ = source(n, mg.PERIODIC, seed=2)
    ref = orc.solve(rho, 1.0 / n, mg.PERIODIC, tol=0.0, max_cycles=80)
    guess = ref.phi + 1e-3 * np.random.default_rng(1).standard_normal(ref.phi.shape)
    tol = 0.0 if prec == mg.FP64 else 1e-10
    with mg.Solver(n, 1.0 / n, mg.PERIODIC, prec=prec, mode_fmg=0, max_cycles=80) as s:
        phi, hist, st = s.solve(torch.from_numpy(rho).cuda(), 1.0, tol,
                                phi=torch.from_numpy(guess).cuda())
    assert st == 0
    assert emax(phi.cpu().numpy(), ref.phi) <= (1e-11 if prec == mg.FP64 else 1e-9)
    if prec == mg.FP64:  # same schedule as the oracle from the same guess
        ref2 = orc.solve(rho, 1.0 / n, mg.PERIODIC, tol=1e-10, fmg=False, phi0=guess)
        with mg.Solver(n, 1.0 / n, mg.PERIODIC, prec=prec, mode_fmg=0) as s:
            phi2, hist2, st2 = s.solve(torch.from_numpy(rho).cuda(), 1.0, 1e-10,
                                       phi=torch.from_numpy(guess).cuda())
        assert len(hist2) == len(ref2.hist)
        assert emax(phi2.cpu().numpy(), ref2.phi) <= 1e-11


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
@pytest.mark.parametrize("n", [2, 4])
def test_smallest_grids(prec, n):
    for bc in BCS:
        rho, fpg = source(n, bc, seed=3) if bc != mg.OPEN else (np.ones((n, n, n)), 4 * math.pi)
        ref = orc.solve(rho, 1.0 / n, bc, bc_value=0.25 if bc == mg.FIXED else 0.0,
                        four_pi_G=fpg, tol=0.0, max_cycles=80)
        phi, hist, st, _ = gpu_solve(rho, bc, fpg, 0.0 if prec == mg.FP64 else 1e-12, prec=prec,
                                     max_cycles=80)
        assert st == 0, (bc, st, hist)
        assert emax(phi, ref.phi) <= (1e-11 if prec == mg.FP64 else 1e-9)


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
def test_zero_source(prec):
    n = 8
    for bc in (mg.PERIODIC, mg.ZEROGRAD, mg.FIXED):
        phi, hist, st, _ = gpu_solve(np.zeros((n, n, n)), bc, 1.0, 1e-10, prec=prec)
        assert st == 0
        if bc == mg.FIXED:  # phi = b everywhere (to the tolerance of the solve)
            assert np.abs(phi - 0.25).max() < 1e-9 * 0.25
        else:
            assert np.abs(phi).max() == 0.0


@pytest.mark.parametrize("bc,prec", [(mg.PERIODIC, mg.MIXED), (mg.FIXED, mg.MIXED),
                                     (mg.OPEN, mg.MIXED), (mg.PERIODIC, mg.FP64)])
def test_solve_host_matches_device(bc, prec):
    """Host buffers give the device solve's bits: pageable ones through copies,
    pinned ones read by the first pass over rho and written by the last pass
    (the mixed path's fixed-point conversion)."""
    n = 32
    rho, fpg = source(n, bc, seed=4)
    with mg.Solver(n, 1.0 / n, bc, prec=prec) as s:
        pd, hd, _ = s.solve(torch.from_numpy(rho).cuda(), fpg, 1e-10)
        ph, hh, st = s.solve_host(rho.copy(), fpg, 1e-10)
        rp = torch.from_numpy(rho.copy()).pin_memory()
        pp = torch.full_like(rp, float("nan")).pin_memory()
        _, hp, st2 = s.solve_host(rp, fpg, 1e-10, phi=pp)
    assert st == st2 == 0
    assert np.array_equal(pd.cpu().numpy(), ph)
    assert np.array_equal(hd, hh)
    assert np.array_equal(pd.cpu().numpy(), pp.numpy())
    assert np.array_equal(hd, hp)


def test_deterministic_repeat():
    n = 32
    rho, _ = source(n, mg.FIXED, seed=12)
    a = gpu_solve(rho, mg.FIXED, 1.0, 1e-10)
    b = gpu_solve(rho, mg.FIXED, 1.0, 1e-10)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


@pytest.mark.parametrize("bc,n", [(mg.PERIODIC, 64), (mg.ZEROGRAD, 32), (mg.OPEN, 32)])
def test_inner_solve_graph_replay_gives_the_same_bits(bc, n):
    """From its second run on the inner FP32 solve replays as a captured CUDA
    graph; per-kernel timing keeps the launches one by one.  Both are the same
    kernels on the same buffers, so phi, the history and the kernel count
    agree exactly (and again after the tuner has dropped the graph)."""
    rho, fpg = source(n, bc, seed=33)
    rd = torch.from_numpy(rho).cuda()
    stream = torch.cuda.Stream()
    with mg.Solver(n, 1.0 / n, bc, prec=mg.MIXED) as s:
        with torch.cuda.stream(stream):
            s.solve(rd, fpg, 1e-10, stream=stream)  # first run: plain launches, graph captured
            p_graph, h_graph, st = s.solve(rd, fpg, 1e-10, stream=stream)
            n_graph = s.last_launches
            s.set_timing(True)
            p_plain, h_plain, st2 = s.solve(rd, fpg, 1e-10, stream=stream)
            n_plain = s.last_launches
            s.set_timing(False)
            s.autotune(stream)
            p_again, h_again, st3 = s.solve(rd, fpg, 1e-10, stream=stream)
        stream.synchronize()
    assert st == st2 == st3 == 0
    assert torch.equal(p_graph, p_plain) and np.array_equal(h_graph, h_plain)
    assert n_graph == n_plain > 0
    assert len(h_again) == len(h_plain) and np.allclose(h_again, h_plain, rtol=64 * 2.0 ** -24)
    assert torch.equal(p_again, p_plain)


def test_invalid_arguments_on_gpu():
    with mg.Solver(8, 1.0 / 8) as s:
        rho = torch.zeros((8, 8, 8), dtype=torch.float64, device="cuda")
        L = mg.lib()
        import ctypes
        nh = ctypes.c_int(0)
        hist = np.zeros(4)
        assert L.mg_solve(s.ctx, rho.data_ptr(), 1.0, -1.0, rho.data_ptr(),
                          hist.ctypes.data, 4, ctypes.byref(nh), None) == 1
        assert L.mg_solve(s.ctx, None, 1.0, 1e-10, rho.data_ptr(), hist.ctypes.data, 4,
                          ctypes.byref(nh), None) == 1


@pytest.mark.parametrize("bc,n", [(mg.PERIODIC, 128), (mg.FIXED, 64), (mg.ZEROGRAD, 32)])
def test_autotuned_shapes_keep_the_result(bc, n):
    """The tuner only changes launch shapes: the same phi bits (the fixed-point
    outer loop is exact), the residual history up to its summation order (each
    thread of the outer step sums at most 64 squares in FP32 before the FP64
    block sum, so a relative 64 * 2^-24 bounds the change), and a second
    context of the same shape takes the same shapes."""
    rho, fpg = source(n, bc, seed=21)
    rd = torch.from_numpy(rho).cuda()
    with mg.Solver(n, 1.0 / n, bc, prec=mg.MIXED) as s:
        p0, h0, st0 = s.solve(rd, fpg, 1e-10)
        s.autotune()
        cfg = s.tile_configs()
        p1, h1, st1 = s.solve(rd, fpg, 1e-10)
    assert st0 == st1 == 0
    fused_levels = [l for l in range(n.bit_length()) if (n >> (n.bit_length() - 1 - l)) >= 32]
    assert sorted(cfg["fused_down"]) == sorted(cfg["fused_up"]) == fused_levels
    for l, (tx, ty, cz) in list(cfg["fused_down"].items()) + list(cfg["fused_up"].items()):
        width = n >> (n.bit_length() - 1 - l)
        assert tx in (32, 64) and width % tx == 0 and cz in [4] + list(range(8, 65, 8))
        assert cz <= width
        assert ty in (16, 32) and width % ty == 0
    for l, (tx, ty, cz) in cfg["fused_updown"].items():  # the finest level's paired cycles
        assert l == n.bit_length() - 1 and tx == 64 and ty in (16, 32) and cz in (16, 32, 64, 128)
    assert list(cfg["outer_residual"]) == [n.bit_length() - 1]
    assert cfg["outer_residual"][n.bit_length() - 1][2] in (4, 8, 16, 32, 64)
    assert torch.equal(p0, p1)
    assert len(h0) == len(h1) and np.allclose(h0, h1, rtol=64 * 2.0 ** -24, atol=0)
    with mg.Solver(n, 1.0 / n, bc, prec=mg.MIXED) as s2:
        s2.autotune()
        assert s2.tile_configs() == cfg


@pytest.mark.parametrize("prec", [mg.FP64, mg.MIXED])
def test_open_sphere_256_full_size(prec):
    """The open-boundary workload at full size: a cell-averaged uniform sphere
    (R = 0.25, 10^3 sub-cells) on [-0.5, 0.5]^3 at 256^3, multipoles to l = 4,
    4 pi G = 4 pi, solved to 1e-10.  Against the oracle's converged solution
    (FP64: 1e-11, mixed: 1e-9) and against the analytic potential, whose
    error falls at second order from 128^3 (Sec. 4.2.1)."""
    errs = {}
    for n in (128, 256):
        rho = inputs.uniform_sphere(n, 0.25, 10)
        phi, hist, st, _ = gpu_solve(rho, mg.OPEN, 4 * math.pi, 1e-10, prec=prec)
        assert st == 0 and hist[-1] < 1e-10
        exact = inputs.sphere_potential(n, 0.25, G=1.0)
        errs[n] = emax(phi, exact)
        if n == 256:
            ref = orc.solve(rho, 1.0 / n, mg.OPEN, four_pi_G=4 * math.pi, tol=0.0, max_cycles=40)
            assert emax(phi, ref.phi) <= (1e-11 if prec == mg.FP64 else 1e-9)
    assert errs[256] < 1e-3
    assert 2.5 < errs[128] / errs[256] < 6.0


@pytest.mark.parametrize("bc", BCS)
def test_fas_same_schedule_matches_oracle(bc):
    """Algorithm 3 (FAS, with FMG built on it) on the FP64 path: the same phi
    as the oracle's FAS after the same number of cycles."""
    n = 32
    rho, fpg = source(n, bc, seed=14)
    for k in (0, 2):
        ref = orc.solve(rho, 1.0 / n, bc, bc_value=0.25 if bc == mg.FIXED else 0.0, four_pi_G=fpg,
                        tol=0.0, max_cycles=k, stall_ratio=NO_STALL, cycle=orc.FAS)
        phi, hist, st, _ = gpu_solve(rho, bc, fpg, 0.0, max_cycles=k, stall_ratio=NO_STALL, fas=1)
        assert len(hist) == len(ref.hist) == k + 1
        assert emax(phi, ref.phi) <= 1e-11, (k, emax(phi, ref.phi))
        assert np.allclose(hist, ref.hist, rtol=1e-6, atol=1e-14)


@pytest.mark.parametrize("bc", BCS)
def test_fas_equals_correction_scheme(bc):
    """On a uniform grid the two schemes are the same iteration (Sec. 2.3.5):
    after the same cycles the potentials agree to rounding."""
    n = 64
    rho, fpg = source(n, bc, seed=15)
    a = gpu_solve(rho, bc, fpg, 0.0, max_cycles=3, stall_ratio=NO_STALL, fas=1)
    b = gpu_solve(rho, bc, fpg, 0.0, max_cycles=3, stall_ratio=NO_STALL, fas=0)
    assert emax(a[0], b[0]) <= 1e-12
    assert np.allclose(a[1], b[1], rtol=1e-8, atol=1e-15)


@pytest.mark.parametrize("fas", [0, 1])
@pytest.mark.parametrize("n", [8, 32])
def test_literal_coarse_rule_same_schedule_matches_oracle(n, fas):
    """Zero fixed values on the coarse correction levels of a zero-gradient
    grid (Sec. 2.3.6 taken word for word): the FP64 path, in the correction
    scheme and in FAS, gives the oracle's phi after the same cycles."""
    bc = mg.ZEROGRAD
    rho, fpg = source(n, bc, seed=17)
    for k in (0, 3):
        ref = orc.solve(rho, 1.0 / n, bc, four_pi_G=fpg, tol=0.0, max_cycles=k,
                        stall_ratio=NO_STALL, cycle=orc.FAS if fas else orc.CORRECTION,
                        coarse_literal=True)
        phi, hist, st, _ = gpu_solve(rho, bc, fpg, 0.0, max_cycles=k, stall_ratio=NO_STALL,
                                     fas=fas, coarse_literal=1)
        assert len(hist) == len(ref.hist) == k + 1
        assert emax(phi, ref.phi) <= 1e-11, (k, emax(phi, ref.phi))
        assert np.allclose(hist, ref.hist, rtol=1e-6, atol=1e-14)
    hom = orc.solve(rho, 1.0 / n, bc, four_pi_G=fpg, tol=0.0, max_cycles=3, stall_ratio=NO_STALL,
                    cycle=orc.FAS if fas else orc.CORRECTION)
    assert emax(phi, hom.phi) > 1e-6  # the option took effect


@pytest.mark.parametrize("outer_fixed", [1, 0])
def test_mixed_literal_coarse_rule_reaches_the_converged_solution(outer_fixed):
    """With zero fixed coarse corrections the FP32 inner solves contract
    slowly, but the FP64-accurate outer loop still reaches the oracle's
    converged solution (the coarse rule does not change the finest level's
    discrete problem)."""
    n, bc = 32, mg.ZEROGRAD
    rho, fpg = source(n, bc, seed=18)
    ref = orc.solve(rho, 1.0 / n, bc, four_pi_G=fpg, tol=0.0, max_cycles=80)
    phi, hist, st, _ = gpu_solve(rho, bc, fpg, 1e-10, prec=mg.MIXED, outer_fixed=outer_fixed,
                                 coarse_literal=1, stall_ratio=1.0, max_cycles=250)
    assert st == 0, (st, hist[-3:])
    assert hist[-1] < 1e-10
    assert emax(phi, ref.phi) <= 1e-9
    default = gpu_solve(rho, bc, fpg, 1e-10, prec=mg.MIXED, outer_fixed=outer_fixed)
    assert len(default[1]) * 3 < len(hist)


def test_fas_needs_the_fp64_path():
    with pytest.raises(mg.MGError):
        mg.Solver(16, 1.0 / 16, mg.PERIODIC, prec=mg.MIXED, fas=1)


def box_source(shape, bc, seed):
    nx, ny, nz = shape
    rng = np.random.default_rng(seed)
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    z = (np.arange(nz) + 0.5) * h
    rho = np.zeros((nz, ny, nx))
    for _ in range(4):
        c = rng.random(3) * np.array([nx, ny, nz]) * h
        sig = 0.05 + 0.05 * rng.random()
        rho += (np.exp(-((z - c[2]) ** 2) / (2 * sig ** 2))[:, None, None] *
                np.exp(-((y - c[1]) ** 2) / (2 * sig ** 2))[None, :, None] *
                np.exp(-((x - c[0]) ** 2) / (2 * sig ** 2))[None, None, :])
    if bc in (mg.PERIODIC, mg.ZEROGRAD):
        rho -= rho.mean()
    return rho


@pytest.mark.parametrize("bc", [mg.PERIODIC, mg.FIXED, mg.ZEROGRAD, mg.OPEN])
@pytest.mark.parametrize("shape", [(16, 8, 8), (64, 32, 16), (32, 32, 8)])
def test_non_cubic_fp64_same_schedule_matches_oracle(bc, shape):
    """Boxes whose shortest side reaches one cell first: the coarsest level
    has several cells and gets N_0,max Gauss-Seidel sweeps (Sec. 2.3.2)."""
    nx, ny, nz = shape
    rho = box_source(shape, bc, seed=nx + ny + nz + bc)
    fpg = 1.0
    b = 0.25 if bc == mg.FIXED else 0.0
    for k in (0, 2):
        ref = orc.solve(rho, 1.0 / nx, bc, bc_value=b, four_pi_G=fpg, tol=0.0, max_cycles=k,
                        stall_ratio=NO_STALL)
        with mg.Solver(shape, 1.0 / nx, bc, prec=mg.FP64, fixed_value=b, max_cycles=k,
                       stall_ratio=NO_STALL) as s:
            phi, hist, st = s.solve(torch.from_numpy(rho).cuda(), fpg, 0.0)
        assert len(hist) == len(ref.hist) == k + 1
        assert emax(phi.cpu().numpy(), ref.phi) <= 1e-11, (k, emax(phi.cpu().numpy(), ref.phi))


@pytest.mark.parametrize("bc", [mg.PERIODIC, mg.FIXED, mg.ZEROGRAD, mg.OPEN])
def test_non_cubic_mixed_matches_converged_oracle(bc):
    """The Jeans-wave box shape 1 x 0.5 x 0.5 at 128 x 64 x 64 (fused kernels on
    the levels that allow them), mixed precision to 1e-10."""
    shape = (128, 64, 64)
    rho = box_source(shape, bc, seed=3 + bc)
    b = 0.25 if bc == mg.FIXED else 0.0
    ref = orc.solve(rho, 1.0 / 128, bc, bc_value=b, tol=0.0, max_cycles=60)
    with mg.Solver(shape, 1.0 / 128, bc, prec=mg.MIXED, fixed_value=b) as s:
        phi, hist, st = s.solve(torch.from_numpy(rho).cuda(), 1.0, 1e-10)
    assert st == 0 and hist[-1] < 1e-10
    assert emax(phi.cpu().numpy(), ref.phi) <= 1e-9


def test_jeans_box_mode_exact_on_gpu():
    """64 x 32 x 32 periodic box: sin 2pi x sin 4pi y sin 4pi z is an exact
    eigenvector; the FP64 solve to 1e-12 returns rho / lambda."""
    nx, ny, nz = 64, 32, 32
    h = 1.0 / nx
    x = (np.arange(nx) + 0.5) * h
    y = (np.arange(ny) + 0.5) * h
    rho = (np.sin(4 * np.pi * y)[:, None, None] * np.sin(4 * np.pi * y)[None, :, None] *
           np.sin(2 * np.pi * x)[None, None, :])
    lam = -(4 / h ** 2) * (math.sin(math.pi * h) ** 2 + 2 * math.sin(2 * math.pi * h) ** 2)
    with mg.Solver((nx, ny, nz), h, mg.PERIODIC, prec=mg.FP64) as s:
        phi, hist, st = s.solve(torch.from_numpy(rho).cuda(), 1.0, 1e-12)
    assert st == 0
    assert emax(phi.cpu().numpy(), rho / lam) <= 1e-11


def test_non_cubic_shape_rules():
    with pytest.raises(mg.MGError):  # x must be a longest side
        mg.Solver((8, 16, 16), 0.1, mg.PERIODIC)
    with pytest.raises(mg.MGError):
        mg.Solver((12, 8, 8), 0.1, mg.PERIODIC)


@pytest.mark.parametrize("bc,n", [(mg.PERIODIC, 64), (mg.FIXED, 128), (mg.ZEROGRAD, 64),
                                  (mg.OPEN, 64)])
def test_paired_legs_give_the_same_bits(bc, n):
    """The finest level's inner V-cycles with each up leg fused to the next
    cycle's down leg (one pass, two SMOOTH steps) run the same per-cell
    arithmetic as the two legs apart: the same phi and residual history, bit
    for bit."""
    rho, fpg = source(n, bc, seed=31)
    a = gpu_solve(rho, bc, fpg, 1e-10, prec=mg.MIXED, leg_pairs=1)
    b = gpu_solve(rho, bc, fpg, 1e-10, prec=mg.MIXED, leg_pairs=2)
    assert a[2] == b[2] == 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    assert a[3] < b[3]  # fewer launches: one pass per pair of legs


def test_tensor_copies_give_the_same_bits():
    """The fused legs with their planes brought in by tensor copies
    (opts.tensor_copies = 1) run the same per-cell arithmetic as with
    per-thread copies (2), and so does whatever the autotuner picks (0): the
    same phi and residual history, bit for bit (the tuned run's history up
    to the summation order of its norm).  Tensor copies apply to the
    periodic levels at least 64 cells wide (the down leg's with rows in
    32s)."""
    n = 128
    rho, fpg = source(n, mg.PERIODIC, seed=37)
    a = gpu_solve(rho, mg.PERIODIC, fpg, 1e-10, prec=mg.MIXED, tensor_copies=1)
    b = gpu_solve(rho, mg.PERIODIC, fpg, 1e-10, prec=mg.MIXED, tensor_copies=2)
    assert a[2] == b[2] == 0
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    with mg.Solver(n, 1.0 / n, mg.PERIODIC, prec=mg.MIXED, tensor_copies=1) as s:
        assert s.tensor_copies() == {6: (1, 1, 1), 7: (1, 1, 1)}  # the 64^3 and 128^3 levels
    with mg.Solver(n, 1.0 / n, mg.PERIODIC, prec=mg.MIXED, tensor_copies=2) as s:
        assert s.tensor_copies() == {}
    with mg.Solver(n, 1.0 / n, mg.FIXED, prec=mg.MIXED, tensor_copies=1) as s:
        assert s.tensor_copies() == {}  # periodic levels only
    with mg.Solver(n, 1.0 / n, mg.PERIODIC, prec=mg.MIXED) as s:
        s.autotune()
        assert set(s.tensor_copies()) <= {6, 7}
        phi, hist, st = s.solve(torch.from_numpy(rho).cuda(), fpg, 1e-10)
        assert st == 0
        # the tuned shapes sum the residual norm's FP32 partials in another order
        assert np.array_equal(phi.cpu().numpy(), b[0])
        assert np.allclose(hist, b[1], rtol=64 * 2.0 ** -24, atol=0.0)


def test_tensor_copies_on_a_box():
    """A 256 x 128 x 64 periodic box: the same bits with and without tensor
    copies, on every level they apply to."""
    rng = np.random.default_rng(41)
    rho = rng.standard_normal((64, 128, 256))
    rho -= rho.mean()
    out = []
    for tc in (1, 2):
        with mg.Solver((256, 128, 64), 1.0 / 256, mg.PERIODIC, prec=mg.MIXED,
                       tensor_copies=tc) as s:
            if tc == 1:
                assert 6 in s.tensor_copies() and 5 in s.tensor_copies()
            phi, hist, st = s.solve(torch.from_numpy(rho).cuda(), 1.0, 1e-9)
            assert st == 0
            out.append((phi.cpu().numpy(), hist))
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.fixture(scope="module")
def headline_reference():
    """The oracle's converged solution of the 512^3 periodic workload (64
    Gaussian blobs, seed 20230227): the FP64 solve iterated to its rounding
    floor on the host cores."""
    n = 512
    rho = inputs.gaussian_blobs(n, 64, seed=20230227)
    ref = orc.solve(rho, 1.0 / n, mg.PERIODIC, tol=0.0, max_cycles=40)
    assert ref.ok, ref.hist
    return rho, ref


def test_headline_512_mixed_after_autotune_matches_converged_oracle(headline_reference):
    """The configuration the throughput is quoted on, in the launch shapes the
    bench times: 512^3 periodic blobs, mixed precision to 1e-10 after
    autotune(), element by element against the converged FP64 oracle."""
    rho, ref = headline_reference
    n = rho.shape[0]
    rd = torch.from_numpy(rho).cuda()
    with mg.Solver(n, 1.0 / n, mg.PERIODIC, prec=mg.MIXED) as s:
        s.autotune()
        phi, hist, st = s.solve(rd, 1.0, 1e-10)
        tiles = s.tile_configs()
    assert st == 0 and hist[-1] < 1e-10, (st, hist)
    assert n.bit_length() - 1 in tiles["fused_down"]  # tuned shapes on the finest level
    assert emax(phi.cpu().numpy(), ref.phi) <= 1e-9
