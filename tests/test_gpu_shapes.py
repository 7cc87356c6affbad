"""Every compiled variant of the fused FP32 legs and of the fixed-point outer
step, called directly through the C ABI (mg_op_fused_leg, mg_op_fx_step),
against the oracle's operators: each periodic-axis mask 0-7 (a rule per face,
Sec. 2.3.6) times each launch shape the autotuner may choose (tiles of 32 or
64 cells by 16 or 32 rows, z-chunks of 4 to 64 planes, including chunks that
leave a ragged last one), on a 128^3 cube and a 256 x 128 x 128 box.

Tolerance of the FP32 legs: 2e-6 of the largest output (a few FP32 ulp of at
most 27 terms; the oracle runs in FP64 on the same FP32 inputs).  The
fixed-point step is integer arithmetic up to two FP32 roundings that both
sides take the same way: bit for bit.
"""
import numpy as np
import pytest
import torch

import oracle as orc
import paper_2302_13903_gb300 as mg

pytestmark = pytest.mark.gpu

P, F, Z = mg.PERIODIC, mg.FIXED, mg.ZEROGRAD
# non-periodic faces of each axis get two different rules (per-face signs)
WALLS = [(F, Z), (Z, F), (F, Z)]
GRIDS = {"cube128": (128, 128, 128), "box256": (128, 128, 256)}  # (nz, ny, nx)
SHAPES = [(tx, ty, cz) for tx in (32, 64) for ty in (16, 32) for cz in (4, 8, 12, 24, 64)]
SHAPES += [(0, 0, 0)]
_REF = {}


def kinds_of(mask):
    k = []
    for a in range(3):
        k += [P, P] if mask >> a & 1 else list(WALLS[a])
    return k


def rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def inputs(grid, mask, leg):
    nz, ny, nx = GRIDS[grid]
    rng = np.random.default_rng(1000 * mask + 10 * leg + nx // 64)
    u = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    f = rng.standard_normal((nz, ny, nx)).astype(np.float32)
    ec = rng.standard_normal((nz // 2, ny // 2, nx // 2)).astype(np.float32)
    return u, f, ec


def reference(grid, mask, leg):
    """The oracle's operators in FP64 on the FP32 inputs, once per case (the
    result does not depend on the launch shape)."""
    key = (grid, mask, leg)
    if key not in _REF:
        u, f, ec = (a.astype(np.float64) for a in inputs(grid, mask, leg))
        h = 1.0 / GRIDS[grid][2]
        rule = dict(faces=orc.mixed_rule(kinds_of(mask)))
        if leg == 1:
            v = orc.prolong(ec, orc.PER_FACE, add=True, uf=u, coarse_faces=rule["faces"])
            _REF[key] = (orc.smooth(v, f, h, orc.PER_FACE, omega=1.15, steps=1, **rule), None)
        elif leg == 3:  # steps 5-7 of one cycle, then 1-3 of the next
            v = orc.prolong(ec, orc.PER_FACE, add=True, uf=u, coarse_faces=rule["faces"])
            v = orc.smooth(v, f, h, orc.PER_FACE, omega=1.15, steps=1, **rule)
            v = orc.smooth(v, f, h, orc.PER_FACE, omega=1.15, steps=1, **rule)
            d = orc.defect(v, f, h, orc.PER_FACE, **rule)
            _REF[key] = (v, (orc.restrict(d), np.abs(d).max()))
        else:
            u0 = np.zeros_like(u) if leg == 2 else u
            v = orc.smooth(u0, f, h, orc.PER_FACE, omega=1.15, steps=1, **rule)
            d = orc.defect(v, f, h, orc.PER_FACE, **rule)
            _REF[key] = (v, (orc.restrict(d), np.abs(d).max()))
    return _REF[key]


@pytest.mark.parametrize("grid", sorted(GRIDS))
@pytest.mark.parametrize("mask", range(8))
@pytest.mark.parametrize("leg", [0, 1, 2], ids=["down", "up", "down_from_zero"])
def test_fused_legs_every_shape_and_mask(grid, mask, leg):
    u, f, ec = inputs(grid, mask, leg)
    h = 1.0 / GRIDS[grid][2]
    ref_u, ref_d = reference(grid, mask, leg)
    ud, fd, ecd = (torch.from_numpy(a).cuda() for a in (u, f, ec))
    for tile in SHAPES:
        if leg == 1:
            uo = mg.op_fused_leg(1, ud, fd, h, kinds_of(mask), ec=ecd, tile=tile)
        else:
            uo, fc = mg.op_fused_leg(0, ud, fd, h, kinds_of(mask), zero_guess=(leg == 2),
                                     tile=tile)
            # the mean of eight defects can cancel: measured against the summands
            err = np.abs(fc.double().cpu().numpy() - ref_d[0]).max() / ref_d[1]
            assert err < 2e-6, (tile, err)
        assert rel(uo.double().cpu().numpy(), ref_u) < 2e-6, tile


UD_SHAPES = [(64, ty, cz) for ty in (16, 32) for cz in (8, 24, 64)] + [(0, 0, 0)]


@pytest.mark.parametrize("grid", sorted(GRIDS))
@pytest.mark.parametrize("mask", range(8))
def test_fused_up_then_down_every_shape_and_mask(grid, mask):
    """The up leg of one V-cycle and the down leg of the next in one pass
    (temporal blocking: two SMOOTH steps per pass), against the oracle's
    prolongation, two smoother steps, defect and restriction in turn."""
    u, f, ec = inputs(grid, mask, 3)
    h = 1.0 / GRIDS[grid][2]
    ref_u, ref_d = reference(grid, mask, 3)
    ud, fd, ecd = (torch.from_numpy(a).cuda() for a in (u, f, ec))
    for tile in UD_SHAPES:
        uo, fc = mg.op_fused_leg(2, ud, fd, h, kinds_of(mask), ec=ecd, tile=tile)
        assert rel(uo.double().cpu().numpy(), ref_u) < 2e-6, tile
        err = np.abs(fc.double().cpu().numpy() - ref_d[0]).max() / ref_d[1]
        assert err < 2e-6, (tile, err)


@pytest.mark.parametrize("zero", [False, True], ids=["down", "down_from_zero"])
def test_fused_down_with_tensor_copies_matches_plain_down_leg(zero):
    """Leg 3: the periodic down leg whose tiles inside the level take their
    planes by tensor copies; the tiles at the level's edges keep per-thread
    copies.  Same arithmetic: bit for bit the plain down leg's results."""
    rng = np.random.default_rng(33)
    nz, ny, nx = 48, 128, 256  # 2 x 2 of the 4 x 4 tiles lie inside the level
    u, f = (torch.from_numpy(rng.standard_normal((nz, ny, nx)).astype(np.float32)).cuda()
            for _ in range(2))
    for cz in (4, 8, 16, 0):
        a = mg.op_fused_leg(0, u, f, 1.0 / nx, [P] * 6, zero_guess=zero, tile=(64, 32, cz))
        b = mg.op_fused_leg(3, u, f, 1.0 / nx, [P] * 6, zero_guess=zero, tile=(64, 32, cz))
        torch.cuda.synchronize()
        assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]), cz


def test_fused_up_with_tensor_copies_matches_plain_up_leg():
    """Leg 4: the periodic up leg whose tiles inside the level take their
    planes of u and f by tensor copies: bit for bit leg 1's results."""
    rng = np.random.default_rng(34)
    nz, ny, nx = 48, 64, 256  # 2 x 2 of the 4 x 4 tiles lie inside the level
    u, f = (torch.from_numpy(rng.standard_normal((nz, ny, nx)).astype(np.float32)).cuda()
            for _ in range(2))
    ec = torch.from_numpy(rng.standard_normal((nz // 2, ny // 2, nx // 2)).astype(np.float32))
    ec = ec.cuda()
    for cz in (4, 8, 16, 0):
        a = mg.op_fused_leg(1, u, f, 1.0 / nx, [P] * 6, ec=ec, tile=(64, 16, cz))
        b = mg.op_fused_leg(4, u, f, 1.0 / nx, [P] * 6, ec=ec, tile=(64, 16, cz))
        torch.cuda.synchronize()
        assert torch.equal(a, b), cz


def test_fused_leg_rejects_shapes_it_does_not_take():
    f = torch.zeros((64, 48, 64), device="cuda")  # 48 rows: 16-row tiles only
    mg.op_fused_leg(0, f, f, 1.0, [P] * 6, tile=(64, 16, 8))  # taken
    for tile in [(32, 32, 0), (48, 16, 0), (32, 16, 6), (32, 16, 2)]:
        with pytest.raises(mg.MGError):
            mg.op_fused_leg(0, f, f, 1.0, [P] * 6, tile=tile)
    with pytest.raises(mg.MGError):  # periodic faces come in pairs
        mg.op_fused_leg(0, f, f, 1.0, [P, F, P, P, P, P])
    with pytest.raises(mg.MGError):  # below 32 cells the fused kernels do not run
        g = torch.zeros((16, 16, 16), device="cuda")
        mg.op_fused_leg(0, g, g, 1.0, [P] * 6)
    e = torch.zeros((32, 24, 32), device="cuda")
    with pytest.raises(mg.MGError):  # up then down: 64-cell tiles only
        mg.op_fused_leg(2, f, f, 1.0, [P] * 6, ec=e, tile=(32, 16, 8))
    with pytest.raises(mg.MGError):  # ... and 32-row tiles need rows in 32s
        mg.op_fused_leg(2, f, f, 1.0, [P] * 6, ec=e, tile=(64, 32, 8))
    with pytest.raises(mg.MGError):  # ... and z-chunks in 8s
        mg.op_fused_leg(2, f, f, 1.0, [P] * 6, ec=e, tile=(64, 16, 4))
    u2, fc2 = mg.op_fused_leg(2, f, f, 1.0, [P] * 6, ec=e, tile=(64, 16, 16))  # taken


def fx_inputs(shape, mask, seed):
    rng = np.random.default_rng(seed)
    S = 40
    phi = rng.integers(-2 ** 50, 2 ** 50, size=shape, dtype=np.int64)
    F = rng.integers(-2 ** 53, 2 ** 53, size=shape, dtype=np.int64)
    e = rng.standard_normal(shape).astype(np.float32)
    # exact ties of e * c decide by round-half-even on both sides
    e.flat[::97] = np.float32(2.5)
    e.flat[1::97] = np.float32(-3.5)
    return phi, F, e, S


@pytest.mark.parametrize("grid", sorted(GRIDS))
@pytest.mark.parametrize("mask", range(8))
@pytest.mark.parametrize("values", [False, True], ids=["zero_faces", "valued_faces"])
def test_fx_step_every_mask_and_chunk(grid, mask, values):
    shape = GRIDS[grid]
    nz, ny, nx = shape
    phi, Fx, e, S = fx_inputs(shape, mask, 7 * mask + values)
    kinds = kinds_of(mask)
    b = [0.37 * (q + 1) * (-1) ** q if (values and kinds[q] == F) else 0.0 for q in range(6)]
    c, factor, two_S = np.float32(2.0 ** 20), np.float32(2.0 ** -45), 2.0 ** S
    ref_p, ref_r = orc.fx_step(phi, e, c, Fx, kinds, b, two_S, factor)
    faces = None
    if values:
        fa = np.zeros(orc.faces_size(nx, ny, nz))
        o = 0
        for q, (m1, m2) in enumerate([(ny, nz), (ny, nz), (nx, nz), (nx, nz), (nx, ny), (nx, ny)]):
            cnt = (m1 + 2) * (m2 + 2)
            fa[o:o + cnt] = b[q]
            o += cnt
        faces = torch.from_numpy(fa).cuda()
    pd, Fd, ed = (torch.from_numpy(a).cuda() for a in (phi, Fx, e))
    for cz in (0, 4, 12, 64):
        out, r = mg.op_fx_step(pd, ed, c, Fd, kinds, two_S, factor, faces=faces, cz=cz)
        assert np.array_equal(out.cpu().numpy(), ref_p), cz
        assert np.array_equal(r.cpu().numpy().view(np.int32), ref_r.view(np.int32)), cz
    # zero start (P = 0, the integer phi is not read) with the same correction
    out, r = mg.op_fx_step(None, ed, c, Fd, kinds, two_S, factor, faces=faces)
    ref_p, ref_r = orc.fx_step(None, e, c, Fx, kinds, b, two_S, factor)
    assert np.array_equal(out.cpu().numpy(), ref_p)
    assert np.array_equal(r.cpu().numpy().view(np.int32), ref_r.view(np.int32))
    with pytest.raises(mg.MGError):  # the correction is required
        mg.op_fx_step(pd, None, c, Fd, kinds, two_S, factor, faces=faces)
