"""The no-allocation multipole-moment entry point, called through the C ABI.

It serves callers that cannot allocate device memory: a host application whose
device memory is all held by its own pool allocator and that forbids plugins to
allocate, or code that must not meet an out-of-memory failure or the
allocator's latency in the middle of a time step.  Its results must equal those
of mg_op_multipole_moments, the allocating entry point, on consecutive calls
that share its fixed scratch; at its size limit; and its first call on a fresh
context must leave the device's free memory unchanged.  This file is collected
last so that a failure here stops a -x run only after every other test has run.
"""
import ctypes
import json
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

import paper_2302_13903_gb300 as mg

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def call_noalloc(rho, h, lmax, use_com, origin, shape=None):
    nz, ny, nx = shape or rho.shape
    Q = np.zeros(25)
    org = np.array(origin, dtype=np.float64)
    st = mg.lib().mg_op_multipole_moments_noalloc(
        nx, ny, nz, h, rho.data_ptr(), lmax, int(use_com), org.ctypes.data_as(ctypes.c_void_p),
        Q.ctypes.data_as(ctypes.c_void_p), torch.cuda.current_stream().cuda_stream)
    return st, Q, org


def check_against_allocating(rho, h, origin):
    for use_com, lmax in ((True, 4), (False, 3)):
        Q_ref, o_ref = mg.op_multipole_moments(rho, h, lmax, use_com, origin)
        st, Q, o = call_noalloc(rho, h, lmax, use_com, origin)
        assert st == 0, mg.last_error()
        scale = np.abs(Q_ref).max()
        assert np.abs(Q - Q_ref).max() <= 1e-13 * scale
        assert np.abs(o - o_ref).max() <= 1e-13 * max(1.0, np.abs(o_ref).max())


def test_noalloc_moments_match_allocating_entry_point_on_two_calls():
    gen = torch.Generator(device="cuda").manual_seed(11)
    shapes = [(64, 48, 32), (16, 96, 128)]  # (nz, ny, nx); the second call reuses the scratch
    for call, shape in enumerate(shapes):
        rho = torch.rand(shape, dtype=torch.float64, device="cuda", generator=gen) + 0.1
        check_against_allocating(rho, 1.0 / max(shape), (0.01 * call, -0.02, 0.03))


def test_noalloc_at_its_row_limit():
    """ny * nz = 262144 rows fill every one of the 8192 partial blocks, the
    last of them ending where the result slots start."""
    gen = torch.Generator(device="cuda").manual_seed(12)
    rho = torch.rand((512, 512, 8), dtype=torch.float64, device="cuda", generator=gen)
    check_against_allocating(rho, 1.0 / 512, (0.0, 0.0, 0.0))
    # and a smaller grid after it, whose result must not mix with the big one's
    small = torch.rand((8, 8, 8), dtype=torch.float64, device="cuda", generator=gen) + 1.0
    check_against_allocating(small, 0.125, (0.1, 0.2, 0.3))


def test_noalloc_rejects_grids_beyond_its_scratch():
    rho = torch.zeros((2, 2, 2), dtype=torch.float64, device="cuda")
    for shape in [(5, 52429, 1), (1024, 1024, 8)]:  # 262145 and 1048576 rows
        st, _, _ = call_noalloc(rho, 0.1, 4, True, (0.0, 0.0, 0.0), shape=shape)
        assert st == 1  # MG_ERR_ARG, before any device work
        assert "rows" in mg.last_error()


CHILD = r"""
import ctypes, glob, json, os, sys
sys.path.insert(0, sys.argv[1])
import numpy as np
import paper_2302_13903_gb300 as mg
L = mg.lib()
# A CUDA runtime of its own for allocating the input and reading free memory,
# so that no other library's device code is loaded into this process.
cands = sorted(glob.glob(os.path.join(sys.argv[2], "lib64", "libcudart.so*")))
if not cands:
    print(json.dumps({"skip": "no libcudart.so under " + sys.argv[2]}))
    sys.exit(0)
rt = ctypes.CDLL(cands[0])
vp, sz = ctypes.c_void_p, ctypes.c_size_t
assert rt.cudaSetDevice(0) == 0
def dalloc(a):
    p = vp()
    assert rt.cudaMalloc(ctypes.byref(p), sz(a.nbytes)) == 0
    assert rt.cudaMemcpy(p, a.ctypes.data_as(vp), sz(a.nbytes), 1) == 0  # host to device
    return p
def free_bytes():
    f, t = sz(), sz()
    assert rt.cudaDeviceSynchronize() == 0
    assert rt.cudaMemGetInfo(ctypes.byref(f), ctypes.byref(t)) == 0
    return f.value
rho = dalloc(np.random.default_rng(1).random((32, 64, 64)) + 0.5)
tiny, tiny_c = dalloc(np.zeros(8)), dalloc(np.zeros(1))
# The library carries its own CUDA runtime, whose first call loads the
# library's device code (with CUDA_MODULE_LOADING=EAGER all of it, the fixed
# scratch included): make that first call through another entry point.
assert L.mg_op_restrict(0, 2, 2, 2, tiny, tiny_c, None) == 0
free = [free_bytes()]
for _ in range(3):
    Q = np.zeros(25); org = np.zeros(3)
    st = L.mg_op_multipole_moments_noalloc(64, 64, 32, 1.0 / 64, rho, 4, 1,
                                           org.ctypes.data_as(vp), Q.ctypes.data_as(vp), None)
    assert st == 0, st
    free.append(free_bytes())
print(json.dumps({"free": free, "Q00": Q[0]}))
"""


def test_noalloc_first_call_leaves_free_memory_unchanged():
    """In a fresh process that loads no other library's device code, once
    the library's own device code is loaded (CUDA_MODULE_LOADING=EAGER and one
    call of another entry point, so that loading the module, which holds the
    fixed scratch, is not counted), the first call of the no-allocation entry
    point -- which also does its per-device set-up -- and the calls after it
    change the device's free memory by nothing."""
    env = dict(os.environ, CUDA_MODULE_LOADING="EAGER")
    cuda_home = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    out = subprocess.run([sys.executable, "-c", CHILD, ROOT, cuda_home], capture_output=True,
                         text=True, env=env, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    rec = json.loads(out.stdout.strip().splitlines()[-1])
    if "skip" in rec:
        pytest.skip(rec["skip"])
    assert len(set(rec["free"])) == 1, rec["free"]
    assert rec["Q00"] > 0.0
