"""The no-allocation multipole-moment entry point, called through the C ABI.

It serves callers that cannot allocate device memory (their device memory is
held by another allocator, or an allocation failure mid-step is not
acceptable).  Its results must equal those of mg_op_multipole_moments, the
allocating entry point, on consecutive calls that share its fixed scratch.
This file is collected last so that a failure here stops a -x run only after
every other test has run.
"""
import ctypes

import numpy as np
import pytest
import torch

import paper_2302_13903_gb300 as mg

pytestmark = pytest.mark.gpu


def call_noalloc(rho, h, lmax, use_com, origin):
    nz, ny, nx = rho.shape
    Q = np.zeros(25)
    org = np.array(origin, dtype=np.float64)
    st = mg.lib().mg_op_multipole_moments_noalloc(
        nx, ny, nz, h, rho.data_ptr(), lmax, int(use_com), org.ctypes.data_as(ctypes.c_void_p),
        Q.ctypes.data_as(ctypes.c_void_p), torch.cuda.current_stream().cuda_stream)
    return st, Q, org


def test_noalloc_moments_match_allocating_entry_point_on_two_calls():
    gen = torch.Generator(device="cuda").manual_seed(11)
    shapes = [(64, 48, 32), (16, 96, 128)]  # (nz, ny, nx); the second call reuses the scratch
    for call, shape in enumerate(shapes):
        rho = torch.rand(shape, dtype=torch.float64, device="cuda", generator=gen) + 0.1
        h = 1.0 / max(shape)
        origin = (0.01 * call, -0.02, 0.03)
        for use_com, lmax in ((True, 4), (False, 3)):
            Q_ref, o_ref = mg.op_multipole_moments(rho, h, lmax, use_com, origin)
            st, Q, o = call_noalloc(rho, h, lmax, use_com, origin)
            assert st == 0
            scale = np.abs(Q_ref).max()
            assert np.abs(Q - Q_ref).max() <= 1e-13 * scale
            assert np.abs(o - o_ref).max() <= 1e-13 * max(1.0, np.abs(o_ref).max())


def test_noalloc_rejects_grids_beyond_its_scratch():
    rho = torch.zeros((2, 2, 2), dtype=torch.float64, device="cuda")
    Q = np.zeros(25)
    org = np.zeros(3)
    # 1024 * 1024 rows exceed the 262144-row limit; rejected before any device work
    st = mg.lib().mg_op_multipole_moments_noalloc(
        8, 1024, 1024, 0.1, rho.data_ptr(), 4, 1, org.ctypes.data_as(ctypes.c_void_p),
        Q.ctypes.data_as(ctypes.c_void_p), None)
    assert st == 1
