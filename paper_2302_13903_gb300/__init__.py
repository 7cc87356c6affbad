"""GB300 geometric-multigrid Poisson solver (Tomida & Stone 2023, Sec. 2-3).

Thin ctypes binding over the C ABI declared in ``include/mg.h``.  Every step
of a solve runs in the CUDA library ``_build/libmg_gb300.so``; this module only
marshals arguments (torch tensors give device pointers and streams).  There
is no CPU fallback: if the library is missing, loading it raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import _build

PERIODIC, FIXED, ZEROGRAD, OPEN, PER_FACE = 0, 1, 2, 3, 4  # PER_FACE: made by mg_create_faces
FP64, MIXED = 0, 1
STATUS = {0: "MG_OK", 1: "MG_ERR_ARG", 2: "MG_ERR_OOM", 3: "MG_ERR_CUDA",
          4: "MG_ERR_NOT_CONVERGED", 5: "MG_ERR_DIVERGED", 6: "MG_ERR_TIMEOUT", 7: "MG_ERR_BUSY"}

# Every symbol include/mg.h declares (checked by the ABI test).
EXPORTS = [
    "mg_opts_init", "mg_create", "mg_create_faces", "mg_solve", "mg_solve_host", "mg_destroy",
    "mg_ctx_device_bytes", "mg_ctx_last_launches", "mg_status_str", "mg_last_error",
    "mg_op_smooth", "mg_op_defect", "mg_op_defect_restrict", "mg_op_restrict", "mg_op_prolong",
    "mg_op_coarsest", "mg_op_multipole_moments", "mg_op_open_faces", "mg_faces_count",
    "mg_ctx_set_timing", "mg_ctx_kernel_time", "mg_op_multipole_moments_noalloc",
    "mg_op_vcycle_down", "mg_op_vcycle_up",
    "mg_batch_create", "mg_batch_solve", "mg_batch_destroy", "mg_batch_cells",
    "mg_batch_last_error", "mg_batch_graph", "mg_required_bytes", "mg_ctx_autotune",
    "mg_ctx_tile_config", "mg_batch_phase_ms", "mg_solve_gravity", "mg_op_gravity",
    "mg_server_create", "mg_server_submit", "mg_server_poll", "mg_server_wait",
    "mg_server_get_stats", "mg_server_destroy", "mg_server_last_error", "mg_op_convert",
    "mg_op_fused_leg", "mg_op_fx_step", "mg_batch_set_barrier_limit", "mg_batch_set_blocks",
    "mg_ctx_tensor_copies",
]
KERNELS = ["sor", "defect_restrict", "prolong", "fmg_prolong", "defect_norm", "outer_residual",
           "correct", "source", "fused_down", "fused_up", "gravity", "fused_down0",
           "fused_updown"]


class Opts(ctypes.Structure):
    _fields_ = [
        ("prec", ctypes.c_int), ("mode_fmg", ctypes.c_int), ("pre", ctypes.c_int),
        ("post", ctypes.c_int), ("omega", ctypes.c_double), ("max_cycles", ctypes.c_int),
        ("fixed_value", ctypes.c_double), ("lmax", ctypes.c_int), ("use_com", ctypes.c_int),
        ("origin", ctypes.c_double * 3), ("stall_ratio", ctypes.c_double),
        ("inner_fmg", ctypes.c_int), ("inner_cycles", ctypes.c_int),
        ("outer_fixed", ctypes.c_int), ("fas", ctypes.c_int), ("coarse_literal", ctypes.c_int),
        ("leg_pairs", ctypes.c_int), ("batch_small", ctypes.c_int),
        ("tensor_copies", ctypes.c_int), ("first_cycles", ctypes.c_int),
        ("reserved", ctypes.c_int * 1),
    ]


class Request(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int), ("nz", ctypes.c_int), ("dx", ctypes.c_double),
        ("bc", ctypes.c_int), ("fixed_value", ctypes.c_double), ("lmax", ctypes.c_int),
        ("rho", ctypes.c_void_p), ("four_pi_G", ctypes.c_double), ("tol", ctypes.c_double),
        ("phi", ctypes.c_void_p), ("per_face", ctypes.c_int), ("face_bc", ctypes.c_int * 6),
        ("face_value", ctypes.c_double * 6),
    ]


class Result(ctypes.Structure):
    _fields_ = [
        ("done", ctypes.c_int), ("status", ctypes.c_int), ("n_hist", ctypes.c_int),
        ("reserved", ctypes.c_int), ("queue_ms", ctypes.c_double), ("solve_ms", ctypes.c_double),
        ("total_ms", ctypes.c_double), ("h2d_ms", ctypes.c_double), ("d2h_ms", ctypes.c_double),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [
        ("submitted", ctypes.c_longlong), ("completed", ctypes.c_longlong),
        ("rejected", ctypes.c_longlong), ("evictions", ctypes.c_longlong),
        ("created", ctypes.c_longlong), ("cells_completed", ctypes.c_longlong),
        ("batched", ctypes.c_longlong), ("budget_bytes", ctypes.c_size_t),
        ("resident_bytes", ctypes.c_size_t), ("peak_bytes", ctypes.c_size_t), ("queued", ctypes.c_int), ("running", ctypes.c_int),
        ("slots", ctypes.c_int), ("resident", ctypes.c_int),
    ]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class MGError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Load the CUDA library (building it first if the sources are newer)."""
    global _lib
    with _lock:
        if _lib is None:
            if not _build.up_to_date():
                _build.build()
            if not os.path.exists(_build.LIB):
                raise RuntimeError(f"CUDA library not built: {_build.LIB}")
            L = ctypes.CDLL(_build.LIB)
            i, d, p, sz = ctypes.c_int, ctypes.c_double, ctypes.c_void_p, ctypes.c_size_t
            L.mg_opts_init.argtypes = [ctypes.POINTER(Opts)]
            L.mg_opts_init.restype = None
            L.mg_create.argtypes = [i, i, i, d, i, ctypes.POINTER(Opts), ctypes.POINTER(p)]
            L.mg_create.restype = i
            L.mg_create_faces.argtypes = [i, i, i, d, p, p, ctypes.POINTER(Opts),
                                          ctypes.POINTER(p)]
            L.mg_create_faces.restype = i
            L.mg_solve.argtypes = [p, p, d, d, p, p, i, ctypes.POINTER(i), p]
            L.mg_solve.restype = i
            L.mg_solve_host.argtypes = [p, p, d, d, p, p, i, ctypes.POINTER(i), p]
            L.mg_solve_gravity.argtypes = [p, p, d, d, p, p, p, i, ctypes.POINTER(i), p]
            L.mg_solve_gravity.restype = i
            L.mg_op_gravity.argtypes = [i, i, i, d, i, d, p, p, p, p]
            L.mg_op_gravity.restype = i
            L.mg_op_convert.argtypes = [i, ctypes.c_longlong, p, p, p]
            L.mg_op_convert.restype = i
            L.mg_solve_host.restype = i
            L.mg_destroy.argtypes = [p]
            L.mg_destroy.restype = i
            L.mg_ctx_device_bytes.argtypes = [p]
            L.mg_ctx_device_bytes.restype = sz
            L.mg_ctx_last_launches.argtypes = [p]
            L.mg_ctx_last_launches.restype = ctypes.c_longlong
            L.mg_status_str.argtypes = [i]
            L.mg_status_str.restype = ctypes.c_char_p
            L.mg_last_error.argtypes = [p]
            L.mg_last_error.restype = ctypes.c_char_p
            L.mg_op_smooth.argtypes = [i, i, i, i, d, i, d, p, d, i, i, p, p, p]
            L.mg_op_defect.argtypes = [i, i, i, i, d, i, d, p, p, p, p, p]
            L.mg_op_defect_restrict.argtypes = [i, i, i, i, d, i, d, p, p, p, p, p]
            L.mg_op_restrict.argtypes = [i, i, i, i, p, p, p]
            L.mg_op_prolong.argtypes = [i, i, i, i, i, d, p, i, i, p, p, p]
            L.mg_op_coarsest.argtypes = [i, d, i, d, p, p, p, p]
            L.mg_op_multipole_moments.argtypes = [i, i, i, d, p, i, i, p, p, p]
            L.mg_op_open_faces.argtypes = [i, i, i, d, p, i, d, p, p, p]
            L.mg_op_vcycle_down.argtypes = [i, i, i, d, i, d, i, p, p, p, p, p]
            L.mg_op_vcycle_down.restype = i
            L.mg_op_vcycle_up.argtypes = [i, i, i, d, i, d, p, p, p, p, p]
            L.mg_op_vcycle_up.restype = i
            L.mg_op_fused_leg.argtypes = [i, i, i, i, d, p, d, i, i, i, i, p, p, p, p, p, p]
            L.mg_op_fused_leg.restype = i
            L.mg_op_fx_step.argtypes = [i, i, i, p, p, d, i, p, p, ctypes.c_float, p, p,
                                        ctypes.c_float, p, p]
            L.mg_op_fx_step.restype = i
            L.mg_op_multipole_moments_noalloc.argtypes = [i, i, i, d, p, i, i, p, p, p]
            L.mg_op_multipole_moments_noalloc.restype = i
            for name in ("mg_op_smooth", "mg_op_defect", "mg_op_defect_restrict", "mg_op_restrict",
                         "mg_op_prolong", "mg_op_coarsest", "mg_op_multipole_moments",
                         "mg_op_open_faces"):
                getattr(L, name).restype = i
            L.mg_ctx_set_timing.argtypes = [p, i]
            L.mg_ctx_set_timing.restype = i
            L.mg_ctx_kernel_time.argtypes = [p, i, ctypes.POINTER(d), ctypes.POINTER(ctypes.c_longlong)]
            L.mg_ctx_kernel_time.restype = i
            L.mg_batch_create.argtypes = [i, p, p, p, p, ctypes.POINTER(Opts), ctypes.POINTER(p)]
            L.mg_batch_create.restype = i
            L.mg_batch_solve.argtypes = [p, p, p, p, p, p, i, p, p, p]
            L.mg_batch_solve.restype = i
            L.mg_batch_destroy.argtypes = [p]
            L.mg_batch_destroy.restype = i
            L.mg_batch_cells.argtypes = [p]
            L.mg_batch_cells.restype = ctypes.c_longlong
            L.mg_batch_phase_ms.argtypes = [p, p, i]
            L.mg_batch_phase_ms.restype = i
            L.mg_batch_graph.argtypes = [p]
            L.mg_batch_graph.restype = i
            L.mg_batch_set_barrier_limit.argtypes = [p, ctypes.c_longlong]
            L.mg_batch_set_barrier_limit.restype = i
            L.mg_batch_set_blocks.argtypes = [p, i]
            L.mg_batch_set_blocks.restype = i
            L.mg_batch_last_error.argtypes = [p]
            L.mg_batch_last_error.restype = ctypes.c_char_p
            L.mg_faces_count.argtypes = [i, i, i]
            L.mg_faces_count.restype = sz
            L.mg_ctx_tensor_copies.argtypes = [p, i, ctypes.POINTER(i), ctypes.POINTER(i),
                                               ctypes.POINTER(i)]
            L.mg_ctx_tensor_copies.restype = i
            L.mg_ctx_autotune.argtypes = [p, p]
            L.mg_ctx_autotune.restype = i
            L.mg_ctx_tile_config.argtypes = [p, i, i, ctypes.POINTER(i), ctypes.POINTER(i),
                                             ctypes.POINTER(i)]
            L.mg_ctx_tile_config.restype = i
            L.mg_required_bytes.argtypes = [i, i, i, i, ctypes.POINTER(Opts), ctypes.POINTER(sz)]
            L.mg_required_bytes.restype = i
            L.mg_server_create.argtypes = [sz, i, i, ctypes.POINTER(Opts), ctypes.POINTER(p)]
            L.mg_server_create.restype = i
            L.mg_server_submit.argtypes = [p, ctypes.POINTER(Request),
                                           ctypes.POINTER(ctypes.c_longlong)]
            L.mg_server_submit.restype = i
            L.mg_server_poll.argtypes = [p, ctypes.c_longlong, ctypes.POINTER(Result), p, i]
            L.mg_server_poll.restype = i
            L.mg_server_wait.argtypes = [p, ctypes.c_longlong, d, ctypes.POINTER(Result), p, i]
            L.mg_server_wait.restype = i
            L.mg_server_get_stats.argtypes = [p, ctypes.POINTER(ServerStats)]
            L.mg_server_get_stats.restype = i
            L.mg_server_destroy.argtypes = [p]
            L.mg_server_destroy.restype = i
            L.mg_server_last_error.argtypes = [p]
            L.mg_server_last_error.restype = ctypes.c_char_p
            _lib = L
    return _lib


def last_error(ctx=None) -> str:
    return lib().mg_last_error(ctx).decode()


def _check(st, ctx=None):
    if st != 0:
        raise MGError(st, last_error(ctx))


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().mg_opts_init(ctypes.byref(o))
    for k, v in kw.items():
        if k == "origin":
            o.origin[:] = list(v)
        elif k == "prec" and isinstance(v, str):
            o.prec = {"fp64": FP64, "mixed": MIXED}[v]
        else:
            setattr(o, k, v)
    return o


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


def _any_ptr(t):
    """Address of a contiguous float64 torch tensor on the device or the host."""
    import torch
    assert t.is_contiguous() and t.dtype == torch.float64, "expected contiguous float64"
    return t.data_ptr()


def _dptr(t, dtype=None):
    import torch
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    if dtype is not None:
        assert t.dtype == dtype, f"expected {dtype}, got {t.dtype}"
    return t.data_ptr()


class Solver:
    """One grid configuration: ``mg_create`` (or ``mg_create_faces``) on
    construction, ``mg_destroy`` on close."""

    def __init__(self, n, dx, bc=PERIODIC, face_values=None, **opts):
        """n: cells per side, or (nx, ny, nz) for a box (arrays are (nz, ny, nx)).
        bc: one rule, or six (x-, x+, y-, y+, z-, z+) with face_values the fixed
        faces' values (default 0)."""
        dims = (n, n, n) if isinstance(n, int) else tuple(int(v) for v in n)
        self.dims = dims
        self.n, self.dx, self.bc = min(dims), dx, bc
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        if isinstance(bc, (int, np.integer)):
            _check(lib().mg_create(*dims, dx, int(bc), ctypes.byref(self.opts), ctypes.byref(h)))
        else:
            kinds = np.ascontiguousarray(bc, dtype=np.int32)
            vals = np.zeros(6) if face_values is None else np.ascontiguousarray(face_values,
                                                                                  dtype=np.float64)
            if kinds.shape != (6,) or vals.shape != (6,):
                raise ValueError("a rule per face needs six kinds and six values")
            _check(lib().mg_create_faces(*dims, dx, kinds.ctypes.data, vals.ctypes.data,
                                         ctypes.byref(self.opts), ctypes.byref(h)))
        self.ctx = h

    def close(self):
        if self.ctx:
            lib().mg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def device_bytes(self):
        return lib().mg_ctx_device_bytes(self.ctx)

    @property
    def last_launches(self):
        return lib().mg_ctx_last_launches(self.ctx)

    def set_timing(self, on=True):
        _check(lib().mg_ctx_set_timing(self.ctx, int(on)), self.ctx)

    def autotune(self, stream=None):
        """Time the candidate launch shapes of the hot kernels and keep the fastest."""
        _check(lib().mg_ctx_autotune(self.ctx, _stream_ptr(stream)), self.ctx)

    def tensor_copies(self):
        """{level: (down, down0, up)} for the levels where the down leg (from
        a nonzero start, from zero) or the up leg takes its planes by tensor
        copies."""
        out = {}
        for l in range(self.n.bit_length()):
            a, b, c = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
            _check(lib().mg_ctx_tensor_copies(self.ctx, l, ctypes.byref(a), ctypes.byref(b),
                                              ctypes.byref(c)), self.ctx)
            if a.value or b.value or c.value:
                out[l] = (a.value, b.value, c.value)
        return out

    def tile_configs(self):
        """{"fused_down" | "fused_up" | "fused_updown" | "sor" | "outer_residual":
        {level: (tx, ty, cz)}} (0: built-in)."""
        out = {}
        levels = self.n.bit_length()
        for name in ("fused_down", "fused_up", "fused_updown", "sor", "outer_residual"):
            k = KERNELS.index(name)
            per = {}
            for l in range(levels):
                tx, ty, cz = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
                _check(lib().mg_ctx_tile_config(self.ctx, l, k, ctypes.byref(tx), ctypes.byref(ty),
                                                ctypes.byref(cz)), self.ctx)
                if tx.value or ty.value or cz.value:
                    per[l] = (tx.value, ty.value, cz.value)
            out[name] = per
        return out

    def kernel_times(self):
        """{kernel class: (total ms, launches)} of finest-level launches."""
        out = {}
        for k, name in enumerate(KERNELS):
            ms, n = ctypes.c_double(0), ctypes.c_longlong(0)
            _check(lib().mg_ctx_kernel_time(self.ctx, k, ctypes.byref(ms), ctypes.byref(n)))
            out[name] = (ms.value, n.value)
        return out

    def solve(self, rho, four_pi_G=1.0, tol=1e-10, phi=None, stream=None, hist_cap=256,
              raise_on_error=True):
        """rho: CUDA float64 (n, n, n).  Returns (phi, hist, status)."""
        import torch
        if phi is None:
            phi = torch.zeros_like(rho)
        hist = np.zeros(hist_cap)
        nh = ctypes.c_int(0)
        st = lib().mg_solve(self.ctx, _dptr(rho, torch.float64), four_pi_G, tol,
                            _dptr(phi, torch.float64), hist.ctypes.data_as(ctypes.c_void_p),
                            hist_cap, ctypes.byref(nh), _stream_ptr(stream))
        if raise_on_error and st not in (0, 4):
            _check(st, self.ctx)
        return phi, hist[: nh.value].copy(), st

    def solve_gravity(self, rho, four_pi_G=1.0, tol=1e-10, phi=None, g=None, stream=None,
                      hist_cap=256):
        """mg_solve_gravity: returns (phi, g, hist, status), g of shape (3, n, n, n)."""
        import torch
        if phi is None:
            phi = torch.zeros_like(rho)
        if g is None:
            g = torch.empty((3,) + tuple(rho.shape), dtype=torch.float64, device=rho.device)
        hist = np.zeros(hist_cap)
        nh = ctypes.c_int(0)
        st = lib().mg_solve_gravity(self.ctx, _dptr(rho, torch.float64), four_pi_G, tol,
                                    _dptr(phi, torch.float64), _dptr(g, torch.float64),
                                    hist.ctypes.data_as(ctypes.c_void_p), hist_cap,
                                    ctypes.byref(nh), _stream_ptr(stream))
        if st not in (0, 4):
            _check(st, self.ctx)
        return phi, g, hist[: nh.value].copy(), st

    def solve_host(self, rho, four_pi_G=1.0, tol=1e-10, phi=None, stream=None, hist_cap=256):
        """rho, phi: host float64 arrays (numpy or pinned torch CPU tensors)."""
        if phi is None:
            phi = np.zeros_like(rho)
        rp = rho.ctypes.data if isinstance(rho, np.ndarray) else rho.data_ptr()
        pp = phi.ctypes.data if isinstance(phi, np.ndarray) else phi.data_ptr()
        hist = np.zeros(hist_cap)
        nh = ctypes.c_int(0)
        st = lib().mg_solve_host(self.ctx, rp, four_pi_G, tol, pp,
                                 hist.ctypes.data_as(ctypes.c_void_p), hist_cap,
                                 ctypes.byref(nh), _stream_ptr(stream))
        if st not in (0, 4):
            _check(st, self.ctx)
        return phi, hist[: nh.value].copy(), st


def _prec_of(t):
    import torch
    return FP64 if t.dtype == torch.float64 else MIXED


def _faces_ptr(faces):
    import torch
    return _dptr(faces, torch.float64) if faces is not None else None


# mg_op_convert kinds: (input dtype, output dtype)
CONVERT_KINDS = {0: ("float64", "int64"), 1: ("int64", "float64"), 2: ("float64", "float32"),
                 3: ("float32", "int64"), 4: ("int64", "float32")}


def op_convert(kind, x, stream=None):
    """mg_op_convert: the fixed-point loop's exact conversion `kind` of a CUDA tensor."""
    import torch
    src, dst = CONVERT_KINDS[kind]
    if x.dtype != getattr(torch, src) or not x.is_contiguous():
        raise TypeError(f"kind {kind} converts contiguous {src} tensors")
    out = torch.empty(x.shape, dtype=getattr(torch, dst), device=x.device)
    _check(lib().mg_op_convert(kind, x.numel(), ctypes.c_void_p(x.data_ptr()),
                               ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))
    return out


def op_gravity(phi, h, bc=PERIODIC, bc_value=0.0, faces=None, stream=None):
    """mg_op_gravity: (3, nz, ny, nx) acceleration of a CUDA float64 potential."""
    import torch
    nz, ny, nx = phi.shape
    g = torch.empty((3, nz, ny, nx), dtype=torch.float64, device=phi.device)
    _check(lib().mg_op_gravity(nx, ny, nz, h, bc, bc_value, _faces_ptr(faces),
                               _dptr(phi, torch.float64), _dptr(g, torch.float64),
                               _stream_ptr(stream)))
    return g


def op_smooth(u, f, h, bc=PERIODIC, bc_value=0.0, faces=None, omega=1.15, steps=1, colours=0,
              stream=None):
    nz, ny, nx = u.shape
    _check(lib().mg_op_smooth(_prec_of(u), nx, ny, nz, h, bc, bc_value, _faces_ptr(faces), omega,
                              steps, colours, _dptr(u, u.dtype), _dptr(f, u.dtype),
                              _stream_ptr(stream)))
    return u


def op_defect(u, f, h, bc=PERIODIC, bc_value=0.0, faces=None, stream=None):
    import torch
    nz, ny, nx = u.shape
    d = torch.empty_like(u)
    _check(lib().mg_op_defect(_prec_of(u), nx, ny, nz, h, bc, bc_value, _faces_ptr(faces),
                              _dptr(u, u.dtype), _dptr(f, u.dtype), _dptr(d), _stream_ptr(stream)))
    return d


def op_defect_restrict(u, f, h, bc=PERIODIC, bc_value=0.0, faces=None, stream=None):
    import torch
    nz, ny, nx = u.shape
    fc = torch.empty((nz // 2, ny // 2, nx // 2), dtype=u.dtype, device=u.device)
    _check(lib().mg_op_defect_restrict(_prec_of(u), nx, ny, nz, h, bc, bc_value, _faces_ptr(faces),
                                       _dptr(u, u.dtype), _dptr(f, u.dtype), _dptr(fc),
                                       _stream_ptr(stream)))
    return fc


def op_restrict(uf, stream=None):
    import torch
    nz, ny, nx = uf.shape
    uc = torch.empty((nz // 2, ny // 2, nx // 2), dtype=uf.dtype, device=uf.device)
    _check(lib().mg_op_restrict(_prec_of(uf), nx, ny, nz, _dptr(uf), _dptr(uc), _stream_ptr(stream)))
    return uc


def op_prolong(uc, bc=PERIODIC, bc_value=0.0, coarse_faces=None, high_order=False, add=False,
               uf=None, stream=None):
    import torch
    nz, ny, nx = (2 * s for s in uc.shape)
    if uf is None:
        uf = torch.zeros((nz, ny, nx), dtype=uc.dtype, device=uc.device)
    _check(lib().mg_op_prolong(_prec_of(uc), nx, ny, nz, bc, bc_value, _faces_ptr(coarse_faces),
                               int(high_order), int(add), _dptr(uc, uc.dtype), _dptr(uf, uc.dtype),
                               _stream_ptr(stream)))
    return uf


def op_coarsest(f, h, bc=PERIODIC, bc_value=0.0, faces=None, stream=None):
    import torch
    u = torch.zeros_like(f)
    _check(lib().mg_op_coarsest(_prec_of(f), h, bc, bc_value, _faces_ptr(faces), _dptr(f), _dptr(u),
                                _stream_ptr(stream)))
    return u


def op_vcycle_down(u, f, h, bc=PERIODIC, omega=1.15, zero_guess=False, stream=None):
    """Fused down-leg on an FP32 level: returns (u_out, fc)."""
    import torch
    nz, ny, nx = f.shape
    uo = torch.empty_like(f)
    fc = torch.empty((nz // 2, ny // 2, nx // 2), dtype=f.dtype, device=f.device)
    _check(lib().mg_op_vcycle_down(nx, ny, nz, h, bc, omega, int(zero_guess),
                                   None if zero_guess else _dptr(u, torch.float32), _dptr(uo),
                                   _dptr(f, torch.float32), _dptr(fc), _stream_ptr(stream)))
    return uo, fc


def op_vcycle_up(u, f, ec, h, bc=PERIODIC, omega=1.15, stream=None):
    """Fused up-leg on an FP32 level: returns u_out."""
    import torch
    nz, ny, nx = f.shape
    uo = torch.empty_like(f)
    _check(lib().mg_op_vcycle_up(nx, ny, nz, h, bc, omega, _dptr(u, torch.float32), _dptr(uo),
                                 _dptr(f, torch.float32), _dptr(ec, torch.float32),
                                 _stream_ptr(stream)))
    return uo


def _face_kinds(kinds):
    k = (ctypes.c_int * 6)(*[int(x) for x in kinds])
    return k


def op_fused_leg(leg, u, f, h, kinds, omega=1.15, zero_guess=False, ec=None, tile=(0, 0, 0),
                 stream=None):
    """The fused FP32 kernels themselves (mg_op_fused_leg): leg 0 down returns
    (u_out, fc); leg 1 up returns u_out; leg 2 (up then down) returns (u_out,
    fc).  kinds: six face rules; tile = (tx, ty, cz), zeros for the built-in
    shape."""
    import torch
    nz, ny, nx = f.shape
    uo = torch.empty_like(f)
    fc = None
    if leg not in (1, 4):  # 3 / 4: the down / up leg with tensor copies
        fc = torch.empty((nz // 2, ny // 2, nx // 2), dtype=f.dtype, device=f.device)
    tx, ty, cz = tile
    _check(lib().mg_op_fused_leg(
        leg, nx, ny, nz, h, _face_kinds(kinds), omega, int(zero_guess), tx, ty, cz,
        None if (zero_guess or u is None) else _dptr(u, torch.float32), _dptr(uo),
        _dptr(f, torch.float32), None if ec is None else _dptr(ec, torch.float32),
        None if fc is None else _dptr(fc), _stream_ptr(stream)))
    return uo if leg in (1, 4) else (uo, fc)


def op_fx_step(phi_in, e, c, F, kinds, two_pow_S, factor, faces=None, cz=0, stream=None):
    """The fixed-point outer step (mg_op_fx_step): returns (phi' int64, r32)."""
    import torch
    nz, ny, nx = F.shape
    out = torch.empty_like(F)
    r = torch.empty(F.shape, dtype=torch.float32, device=F.device)
    _check(lib().mg_op_fx_step(
        nx, ny, nz, _face_kinds(kinds), _faces_ptr(faces), float(two_pow_S), cz,
        None if phi_in is None else _dptr(phi_in, torch.int64),
        None if e is None else _dptr(e, torch.float32), float(c), _dptr(F, torch.int64),
        _dptr(out), float(factor), _dptr(r), _stream_ptr(stream)))
    return out, r


def op_multipole_moments(rho, h, lmax=4, use_com=True, origin=(0.0, 0.0, 0.0), stream=None):
    import torch
    nz, ny, nx = rho.shape
    org = np.array(origin, dtype=np.float64)
    Q = np.zeros(25)
    _check(lib().mg_op_multipole_moments(nx, ny, nz, h, _dptr(rho, torch.float64), lmax,
                                         int(use_com), org.ctypes.data_as(ctypes.c_void_p),
                                         Q.ctypes.data_as(ctypes.c_void_p), _stream_ptr(stream)))
    return Q, org


def op_open_faces(n, h, Q, lmax, G, origin, device="cuda", stream=None):
    import torch
    cnt = lib().mg_faces_count(n, n, n)
    faces = torch.empty(cnt, dtype=torch.float64, device=device)
    Qa = np.ascontiguousarray(Q, dtype=np.float64)
    org = np.ascontiguousarray(origin, dtype=np.float64)
    _check(lib().mg_op_open_faces(n, n, n, h, Qa.ctypes.data_as(ctypes.c_void_p), lmax, G,
                                  org.ctypes.data_as(ctypes.c_void_p), _dptr(faces),
                                  _stream_ptr(stream)))
    return faces


def faces_count(nx, ny, nz):
    return lib().mg_faces_count(nx, ny, nz)


class Batch:
    """Many independent grids solved by one persistent launch (mg_batch_*)."""

    def __init__(self, sizes, dxs, bcs, fixed_values=None, **opts):
        self.n = len(sizes)
        opts.setdefault("prec", MIXED)
        opts.setdefault("max_cycles", 12)  # outer iterations unrolled into the phase list
        self.opts = default_opts(**opts)
        dims = np.repeat(np.asarray(sizes, dtype=np.int32), 3)
        dx = np.ascontiguousarray(dxs, dtype=np.float64)
        bc = np.ascontiguousarray(bcs, dtype=np.int32)
        fv = None if fixed_values is None else np.ascontiguousarray(fixed_values, dtype=np.float64)
        h = ctypes.c_void_p()
        st = lib().mg_batch_create(self.n, dims.ctypes.data, dx.ctypes.data, bc.ctypes.data,
                                   None if fv is None else fv.ctypes.data, ctypes.byref(self.opts),
                                   ctypes.byref(h))
        if st != 0:
            raise MGError(st, lib().mg_batch_last_error(None).decode())
        self.ptr = h
        self.sizes = list(sizes)

    @property
    def cells(self):
        return lib().mg_batch_cells(self.ptr)

    @property
    def graph(self):
        return bool(lib().mg_batch_graph(self.ptr))

    PHASES = ["source", "mean", "r0", "r0_norm", "down", "bottom", "up", "max_e",
              "set_fixed_point", "to_fixed_point", "outer_step", "stop_rule", "phi_sum",
              "phi_mean", "phi_sub"]

    def phase_ms(self):
        """{phase kind: device ms} of the last solve."""
        out = np.zeros(len(self.PHASES))
        st = lib().mg_batch_phase_ms(self.ptr, out.ctypes.data, len(out))
        if st != 0:
            raise MGError(st, lib().mg_batch_last_error(self.ptr).decode())
        return dict(zip(self.PHASES, out.tolist()))

    def solve(self, rhos, phis, four_pi_G=1.0, tol=1e-10, hist_cap=64, stream=None):
        """rhos, phis: lists of CUDA float64 tensors.  Returns (status, hists, statuses)."""
        import torch
        n = self.n
        # None in rhos leaves that slot out of this solve
        rp = np.array([0 if r is None else _dptr(r, torch.float64) for r in rhos], dtype=np.uint64)
        pp = np.array([0 if q is None else _dptr(q, torch.float64) for q in phis], dtype=np.uint64)
        fpg = np.broadcast_to(np.asarray(four_pi_G, dtype=np.float64), (n,)).copy()
        tl = np.broadcast_to(np.asarray(tol, dtype=np.float64), (n,)).copy()
        hist = np.zeros((n, hist_cap))
        nh = np.zeros(n, dtype=np.int32)
        sts = np.zeros(n, dtype=np.int32)
        st = lib().mg_batch_solve(self.ptr, rp.ctypes.data, fpg.ctypes.data, tl.ctypes.data,
                                  pp.ctypes.data, hist.ctypes.data, hist_cap, nh.ctypes.data,
                                  sts.ctypes.data, _stream_ptr(stream))
        if st in (3, 6):
            raise MGError(st, lib().mg_batch_last_error(self.ptr).decode())
        return st, [hist[g, : nh[g]].copy() for g in range(n)], sts

    def set_blocks(self, blocks):
        """CTAs of the persistent launch (0: all that fit)."""
        st = lib().mg_batch_set_blocks(self.ptr, int(blocks))
        if st != 0:
            raise MGError(st, lib().mg_batch_last_error(self.ptr).decode())

    def set_barrier_limit(self, cycles):
        """Clock cycles one grid-wide barrier wait may take before the solve
        gives up with MG_ERR_TIMEOUT (default 4e9)."""
        st = lib().mg_batch_set_barrier_limit(self.ptr, int(cycles))
        if st != 0:
            raise MGError(st, lib().mg_batch_last_error(self.ptr).decode())

    def close(self):
        if getattr(self, "ptr", None):
            lib().mg_batch_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def required_bytes(n, bc=PERIODIC, **opts) -> int:
    """Device bytes ``mg_create`` allocates for an n^3 grid (mg_required_bytes)."""
    o = default_opts(**opts)
    b = ctypes.c_size_t(0)
    _check(lib().mg_required_bytes(n, n, n, bc, ctypes.byref(o), ctypes.byref(b)))
    return b.value


class Server:
    """The serving loop (mg_server_*): submit solves, poll or wait for them."""

    def __init__(self, budget_bytes, slots=4, max_queue=1024, **opts):
        opts.setdefault("prec", MIXED)
        self.opts = default_opts(**opts)
        h = ctypes.c_void_p()
        st = lib().mg_server_create(int(budget_bytes), slots, max_queue, ctypes.byref(self.opts),
                                    ctypes.byref(h))
        if st != 0:
            raise MGError(st, lib().mg_server_last_error(None).decode())
        self.ptr = h

    def submit(self, rho, phi, dx=None, bc=PERIODIC, four_pi_G=1.0, tol=1e-10, lmax=4,
               fixed_value=0.0, face_values=None):
        """rho, phi: float64 (n, n, n) tensors kept alive until done, both on the
        device or both in host memory (pinned host tensors move fastest).  bc
        may be a list of six face rules (x-, x+, y-, y+, z-, z+), with
        face_values the fixed faces' values.  Returns the ticket, or raises
        MGError (MG_ERR_BUSY when the queue is full)."""
        import torch
        n = rho.shape[0]
        q = Request(n, n, n, 1.0 / n if dx is None else dx, 0, fixed_value, lmax,
                    _any_ptr(rho), four_pi_G, tol, _any_ptr(phi))
        if isinstance(bc, (list, tuple)):
            q.per_face = 1
            q.face_bc = (ctypes.c_int * 6)(*[int(k) for k in bc])
            q.face_value = (ctypes.c_double * 6)(*(face_values or [0.0] * 6))
        else:
            q.bc = bc
        t = ctypes.c_longlong(0)
        st = lib().mg_server_submit(self.ptr, ctypes.byref(q), ctypes.byref(t))
        if st != 0:
            raise MGError(st, lib().mg_server_last_error(self.ptr).decode())
        return t.value

    def _result(self, fn, ticket, *extra, hist_cap=64):
        r = Result()
        hist = np.zeros(hist_cap)
        st = fn(self.ptr, ticket, *extra, ctypes.byref(r), hist.ctypes.data, hist_cap)
        if st not in (0, 6):
            raise MGError(st, lib().mg_server_last_error(self.ptr).decode())
        return r, hist[: r.n_hist].copy()

    def poll(self, ticket):
        """(Result, hist); the ticket is retired once Result.done is 1."""
        return self._result(lib().mg_server_poll, ticket)

    def wait(self, ticket, timeout=60.0):
        """Block until done (or the timeout: Result.done stays 0)."""
        return self._result(lib().mg_server_wait, ticket, float(timeout))

    def stats(self):
        s = ServerStats()
        _check(lib().mg_server_get_stats(self.ptr, ctypes.byref(s)))
        return s.as_dict()

    def close(self):
        if getattr(self, "ptr", None):
            lib().mg_server_destroy(self.ptr)
            self.ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
