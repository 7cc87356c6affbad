"""Plain FP64 CPU multigrid oracle (test infrastructure only).

This package is the correctness oracle for the CUDA library: a slow,
obviously-correct C implementation of the multigrid method of Tomida & Stone
(Sec. 2.1-2.3 and App. A), bound here with ctypes.  Only the tests, the smoke
check and the CPU-baseline leg of ``bench.py`` may import it; the product path
never does.  It shares no code with the CUDA path.

Arrays are numpy float64, C-contiguous, shaped (nz, ny, nx) with x fastest.
Boundary kinds: 0 periodic, 1 fixed value, 2 zero gradient, 3 open
(multipole), 4 given face values (finest level only; tests of the dense solve),
5 (PER_FACE) a rule per face (periodic in pairs, fixed b_face or zero gradient), passed as
``faces=mixed_rule(kinds, values)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mg_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

PERIODIC, FIXED, ZEROGRAD, OPEN, FACES, PER_FACE = 0, 1, 2, 3, 4, 5
CORRECTION, FAS = 0, 1


def mixed_rule(kinds, values=(0.0,) * 6):
    """Descriptor of a rule per face (x-, x+, y-, y+, z-, z+): six kinds, then
    six values b_face (read on fixed faces)."""
    assert len(kinds) == 6 and len(values) == 6
    return np.array(list(kinds) + list(values), dtype=np.float64)
STATUS = {0: "ok", 1: "arg", 2: "oom", 4: "not_converged", 5: "diverged"}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no FP contraction, OpenMP)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = ctypes.CDLL(_LIB_PATH)
            d, i, p = ctypes.c_double, ctypes.c_int, ctypes.c_void_p
            L.orc_solve.restype = i
            L.orc_solve.argtypes = [i, i, i, d, i, d, p, i, i, p, d, i, i, i, i, i, i, d, d, d,
                                    p, p, p, i, p, p, p]
            L.orc_op_smooth.restype = i
            L.orc_op_smooth.argtypes = [i, i, i, d, i, d, p, d, i, i, p, p]
            L.orc_op_defect.restype = i
            L.orc_op_defect.argtypes = [i, i, i, d, i, d, p, p, p, p]
            L.orc_op_restrict.restype = i
            L.orc_op_restrict.argtypes = [i, i, i, p, p]
            L.orc_op_prolong.restype = i
            L.orc_op_prolong.argtypes = [i, i, i, i, d, p, i, i, p, p]
            L.orc_op_coarsest.restype = i
            L.orc_op_coarsest.argtypes = [i, i, i, d, i, d, p, p, p]
            L.orc_op_vcycle.restype = i
            L.orc_op_vcycle.argtypes = [i, i, i, d, i, d, p, d, i, i, i, i, p, p]
            L.orc_op_gravity.argtypes = [i, i, i, d, i, d, p, p, p]
            L.orc_op_gravity.restype = i
            L.orc_ylm.restype = d
            L.orc_ylm.argtypes = [i, i, d, d, d]
            L.orc_multipole_moments.restype = None
            L.orc_multipole_moments.argtypes = [i, i, i, d, p, i, i, p, p]
            L.orc_multipole_potential.restype = d
            L.orc_multipole_potential.argtypes = [p, i, d, p, d, d, d]
            L.orc_open_faces.restype = None
            L.orc_open_faces.argtypes = [i, i, i, d, p, i, d, p, p]
            L.orc_open_level_faces.restype = i
            L.orc_open_level_faces.argtypes = [i, i, i, d, p, i, i, p, d, i, p]
            L.orc_op_fx_step.restype = i
            L.orc_op_fx_step.argtypes = [i, i, i, p, p, d, p, p, ctypes.c_float, p, p,
                                         ctypes.c_float, p]
            L.orc_num_threads.restype = i
            L.orc_set_num_threads.argtypes = [i]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def faces_size(nx, ny, nz):
    return 2 * (ny + 2) * (nz + 2) + 2 * (nx + 2) * (nz + 2) + 2 * (nx + 2) * (ny + 2)


class SolveResult:
    def __init__(self, phi, hist, status, origin, Q):
        self.phi, self.hist, self.status, self.origin, self.Q = phi, hist, status, origin, Q

    @property
    def ok(self):
        return self.status == 0


def solve(rho, h, bc=PERIODIC, *, bc_value=0.0, faces=None, lmax=4, use_com=True,
          origin=(0.0, 0.0, 0.0), omega=1.15, pre=1, post=1, fmg=True, cycle=CORRECTION,
          max_cycles=50, stall_ratio=0.9, tol=1e-10, four_pi_G=1.0, phi0=None,
          hist_cap=256, coarse_literal=False) -> SolveResult:
    """FMG (or a given initial guess) then V-cycles to ||d||/||f|| < tol.

    coarse_literal: the coarse correction levels of a zero-gradient grid use
    zero fixed values (Sec. 2.3.6 read word for word) instead of the
    homogeneous zero-gradient rule."""
    rho = _f64(rho)
    nz, ny, nx = rho.shape
    phi = np.zeros_like(rho) if phi0 is None else _f64(phi0).copy()
    hist = np.zeros(hist_cap)
    nh = ctypes.c_int(0)
    org = np.array(origin, dtype=np.float64)
    org_out = np.zeros(3)
    Q = np.zeros(25)
    fa = None if faces is None else _f64(faces)
    st = lib().orc_solve(nx, ny, nz, h, bc, bc_value, _ptr(fa), lmax, int(use_com), _ptr(org),
                         omega, pre, post, int(fmg), cycle, int(coarse_literal), max_cycles,
                         stall_ratio, tol,
                         four_pi_G, _ptr(rho), _ptr(phi), _ptr(hist), hist_cap,
                         ctypes.byref(nh), _ptr(org_out), _ptr(Q))
    return SolveResult(phi, hist[: nh.value].copy(), st, org_out, Q)


def smooth(u, f, h, bc=PERIODIC, *, bc_value=0.0, faces=None, omega=1.15, steps=1, colours=0):
    """RB-SOR steps on one level; colours 0 = red then black, 1 = red, 2 = black."""
    u = _f64(u).copy()
    f = _f64(f)
    nz, ny, nx = u.shape
    fa = None if faces is None else _f64(faces)
    st = lib().orc_op_smooth(nx, ny, nz, h, bc, bc_value, _ptr(fa), omega, steps, colours,
                             _ptr(u), _ptr(f))
    assert st == 0
    return u


def defect(u, f, h, bc=PERIODIC, *, bc_value=0.0, faces=None):
    u, f = _f64(u), _f64(f)
    nz, ny, nx = u.shape
    d = np.zeros_like(u)
    fa = None if faces is None else _f64(faces)
    st = lib().orc_op_defect(nx, ny, nz, h, bc, bc_value, _ptr(fa), _ptr(u), _ptr(f), _ptr(d))
    assert st == 0
    return d


def restrict(uf):
    uf = _f64(uf)
    nz, ny, nx = uf.shape
    uc = np.zeros((nz // 2, ny // 2, nx // 2))
    assert lib().orc_op_restrict(nx, ny, nz, _ptr(uf), _ptr(uc)) == 0
    return uc


def prolong(uc, bc=PERIODIC, *, bc_value=0.0, coarse_faces=None, high_order=False, add=False,
            uf=None):
    """Trilinear (or FMG I') prolongation of a coarse array to the fine grid."""
    uc = _f64(uc)
    nz, ny, nx = (2 * s for s in uc.shape)
    out = np.zeros((nz, ny, nx)) if uf is None else _f64(uf).copy()
    fa = None if coarse_faces is None else _f64(coarse_faces)
    st = lib().orc_op_prolong(nx, ny, nz, bc, bc_value, _ptr(fa), int(high_order), int(add),
                              _ptr(uc), _ptr(out))
    assert st == 0
    return out


def gravity(phi, h, bc=PERIODIC, *, bc_value=0.0, faces=None):
    """Cell-centred acceleration (Sec. 3.2.3): array (3, nz, ny, nx) of g_x, g_y, g_z."""
    phi = _f64(phi)
    nz, ny, nx = phi.shape
    g = np.zeros((3, nz, ny, nx))
    fa = None if faces is None else _f64(faces)
    assert lib().orc_op_gravity(nx, ny, nz, h, bc, bc_value, _ptr(fa), _ptr(phi), _ptr(g)) == 0
    return g


def coarsest(f, h, bc=PERIODIC, *, bc_value=0.0, faces=None):
    f = _f64(f)
    nz, ny, nx = f.shape
    u = np.zeros_like(f)
    fa = None if faces is None else _f64(faces)
    assert lib().orc_op_coarsest(nx, ny, nz, h, bc, bc_value, _ptr(fa), _ptr(f), _ptr(u)) == 0
    return u


def vcycle(u, f, h, bc=PERIODIC, *, bc_value=0.0, faces=None, omega=1.15, pre=1, post=1,
           cycle=CORRECTION, coarse_literal=False):
    u = _f64(u).copy()
    f = _f64(f)
    nz, ny, nx = u.shape
    fa = None if faces is None else _f64(faces)
    st = lib().orc_op_vcycle(nx, ny, nz, h, bc, bc_value, _ptr(fa), omega, pre, post, cycle,
                             int(coarse_literal), _ptr(u), _ptr(f))
    assert st == 0
    return u


def ylm(l, m, x, y, z):
    return lib().orc_ylm(l, m, x, y, z)


def multipole_moments(rho, h, lmax=4, use_com=True, origin=(0.0, 0.0, 0.0)):
    rho = _f64(rho)
    nz, ny, nx = rho.shape
    org = np.array(origin, dtype=np.float64)
    Q = np.zeros(25)
    lib().orc_multipole_moments(nx, ny, nz, h, _ptr(rho), lmax, int(use_com), _ptr(org), _ptr(Q))
    return Q, org


def multipole_potential(Q, lmax, G, origin, x, y, z):
    Q = _f64(Q)
    org = np.array(origin, dtype=np.float64)
    return lib().orc_multipole_potential(_ptr(Q), lmax, G, _ptr(org), x, y, z)


def open_faces(nx, ny, nz, h, Q, lmax, G, origin):
    Q = _f64(Q)
    org = np.array(origin, dtype=np.float64)
    out = np.zeros(faces_size(nx, ny, nz))
    lib().orc_open_faces(nx, ny, nz, h, _ptr(Q), lmax, G, _ptr(org), _ptr(out))
    return out


def open_level_faces(rho, h, level, lmax=4, use_com=True, origin=(0.0, 0.0, 0.0),
                     four_pi_G=1.0):
    """Face values of level `level` (0 = coarsest) of an open-boundary solve of
    rho, as the solve sets them up (orc_open_level_faces)."""
    rho = _f64(rho)
    nz, ny, nx = rho.shape
    nlev = int(min(nx, ny, nz)).bit_length()  # levels down to a shortest side of 1
    shift = nlev - 1 - level
    out = np.zeros(faces_size(nx >> shift, ny >> shift, nz >> shift))
    org = _f64(origin)
    st = lib().orc_open_level_faces(nx, ny, nz, h, _ptr(rho), lmax, int(use_com), _ptr(org),
                                    four_pi_G, level, _ptr(out))
    assert st == 0, st
    return out


def fx_step(phi_in, e, c, F, kinds, values, two_pow_S, factor):
    """The exact integer defect of the fixed-point outer loop (orc_op_fx_step):
    returns (phi' int64, r float32).  phi_in may be None (zero); e float32 or
    None; F int64; kinds / values per face (x-, x+, y-, y+, z-, z+)."""
    F = np.ascontiguousarray(F, dtype=np.int64)
    nz, ny, nx = F.shape
    pin = None if phi_in is None else np.ascontiguousarray(phi_in, dtype=np.int64)
    e32 = None if e is None else np.ascontiguousarray(e, dtype=np.float32)
    k = np.ascontiguousarray(kinds, dtype=np.int32)
    b = _f64(values)
    out = np.empty_like(F)
    r = np.empty(F.shape, dtype=np.float32)
    st = lib().orc_op_fx_step(nx, ny, nz, _ptr(k), _ptr(b), float(two_pow_S), _ptr(pin), _ptr(e32),
                              float(c), _ptr(F), _ptr(out), float(factor), _ptr(r))
    assert st == 0
    return out, r


def num_threads():
    return lib().orc_num_threads()


def set_num_threads(n):
    lib().orc_set_num_threads(int(n))
