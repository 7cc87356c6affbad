"""Launch the fused FP32 V-cycle legs on one box larger than L2 and time them:
the command the per-kernel profiles of the legs are taken with.

python -m paper_2302_13903_gb300.legs_timing LEGS [REPS] [NZ NY NX]

LEGS is a comma-separated list of down (SMOOTH + defect + restriction, 64 x 32
tiles, 64 planes per CTA), down0 (the same from a zero start), tma / tma0 (down
/ down0 with the planes brought in by tensor copies), upt (up, the same way), up
(prolongation + correction + SMOOTH, 64 x 16 tiles), ud16 / ud32 (the up leg
of one V-cycle fused with the down leg of the next, 16- or 32-row tiles), fx
(the fixed-point outer step, 64 planes per CTA), all periodic.  Each leg runs
twice untimed, then REPS times (default 10) between CUDA events; one line per
leg gives the milliseconds per launch.  The default box is 256 x 256 x 512
cells (nz, ny, nx): 128 MiB per FP32 array.
"""
from __future__ import annotations

import sys

import torch

from . import PERIODIC, op_fused_leg, op_fx_step

SHAPES = {"down": (64, 32, 64), "down0": (64, 32, 64), "tma": (64, 32, 64), "tma0": (64, 32, 64), "upt": (64, 16, 64), "up": (64, 16, 64),
          "ud16": (64, 16, 128), "ud32": (64, 32, 64), "fx": (32, 16, 64)}


def main(argv):
    legs = argv[0].split(",")
    reps = int(argv[1]) if len(argv) > 1 else 10
    nz, ny, nx = (int(a) for a in argv[2:5]) if len(argv) > 4 else (256, 256, 512)
    g = torch.Generator(device="cuda").manual_seed(1)
    u = torch.rand((nz, ny, nx), device="cuda", generator=g)
    f = torch.rand((nz, ny, nx), device="cuda", generator=g)
    ec = torch.rand((nz // 2, ny // 2, nx // 2), device="cuda", generator=g)
    kinds = [PERIODIC] * 6
    h = 1.0 / nx
    if "fx" in legs:  # the fixed-point outer step's integer arrays
        phi = torch.randint(-2 ** 40, 2 ** 40, (nz, ny, nx), device="cuda", dtype=torch.int64,
                            generator=g)
        F = torch.randint(-2 ** 40, 2 ** 40, (nz, ny, nx), device="cuda", dtype=torch.int64,
                          generator=g)

    def run(leg):
        tile = SHAPES[leg]
        if leg == "fx":
            return op_fx_step(phi, u, 1024.0, F, kinds, 2.0 ** 40, 2.0 ** -40, cz=tile[2])
        if leg in ("down", "down0"):
            return op_fused_leg(0, u, f, h, kinds, zero_guess=(leg == "down0"), tile=tile)
        if leg in ("tma", "tma0"):
            return op_fused_leg(3, u, f, h, kinds, zero_guess=(leg == "tma0"), tile=tile)
        if leg == "up":
            return op_fused_leg(1, u, f, h, kinds, ec=ec, tile=tile)
        if leg == "upt":
            return op_fused_leg(4, u, f, h, kinds, ec=ec, tile=tile)
        return op_fused_leg(2, u, f, h, kinds, ec=ec, tile=tile)

    for leg in legs:
        for _ in range(2):
            run(leg)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            run(leg)
        b.record()
        torch.cuda.synchronize()
        print(f"{leg} {nz}x{ny}x{nx} tile {SHAPES[leg]}: {a.elapsed_time(b) / reps:.4f} ms per "
              f"launch (with the output tensors' allocation)", flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
