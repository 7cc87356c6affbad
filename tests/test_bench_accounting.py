"""The bench's algorithmic-byte accounting, by hand: the bytes each launch
class must move per finest cell, and the whole mixed solve's count.  These
figures are the numerators of every roofline fraction the bench reports."""
import bench


def test_bytes_per_cell_of_each_launch_class():
    w = 4  # FP32 levels
    # down leg: read u and f, write u and the coarse f (1/8 of a cell)
    assert bench.algorithmic_bytes_per_cell("fused_down", w) == 3 * 4 + 0.5
    # from a zero start u is not read
    assert bench.algorithmic_bytes_per_cell("fused_down0", w) == 2 * 4 + 0.5
    # up leg: read u, f and the coarse e, write u
    assert bench.algorithmic_bytes_per_cell("fused_up", w) == 3 * 4 + 0.5
    # up then down in one pass: read u, f, coarse e; write u, coarse f
    assert bench.algorithmic_bytes_per_cell("fused_updown", w) == 3 * 4 + 1.0
    # fixed-point step: int64 phi, F and FP32 e in, int64 phi and FP32 r out
    assert bench.algorithmic_bytes_per_cell("outer_residual", w) == 8 + 8 + 4 + 8 + 4
    # the fixed-point start reads rho once for its sum and maximum; FP64: rho -> f
    assert bench.algorithmic_bytes_per_cell("source", w, fixed_point=True) == 8
    assert bench.algorithmic_bytes_per_cell("source", 8, fixed_point=False) == 16


def test_whole_mixed_solve_bytes():
    # 3 outer iterations of 4 V(1,1) cycles, the legs apart:
    # finest level per outer iteration: one zero-start cycle (8.5 + 12.5) and
    # three more (2 x 12.5 each); coarse levels 1/7 of four zero-start cycles
    finest = (8.5 + 12.5) + 3 * 25.0
    coarse = 4 * 21.0 / 7
    steps = 24.0 + 32.0 + 32.0  # the first step starts from phi = 0
    passes = 3 * 8 + 4 + 8 + 4 + 16  # rho x3; r32, integer f, e max, phi back
    assert passes == 56
    total = 3 * (finest + coarse) + steps + passes
    assert total == 468
    assert bench.mixed_solve_bytes_per_cell(3, 4, paired=False) == total
    # pairing the up leg with the next down leg saves 25 - 13 B per pair
    assert bench.mixed_solve_bytes_per_cell(3, 4, paired=True) == total - 3 * 3 * 12.0
