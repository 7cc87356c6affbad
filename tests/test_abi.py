"""The C-ABI library builds for sm_103a, loads without a GPU and exports every
entry point include/mg.h declares.  No compute call is made here."""
import ctypes
import os
import re
import subprocess

import pytest

import paper_2302_13903_gb300 as mg

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(mg_\w+)\s*\(", text))
    return names


def test_library_exports_every_declared_symbol():
    L = mg.lib()
    declared = declared_functions()
    assert declared, "no declarations found"
    assert declared == set(mg.EXPORTS), declared ^ set(mg.EXPORTS)
    for name in declared:
        assert hasattr(L, name), name
    raw = ctypes.CDLL(mg.library_path())
    for name in declared:
        getattr(raw, name)


def test_built_for_sm_103a_only():
    assert mg._build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
    assert os.path.exists(mg.library_path())


def test_default_options_layout():
    o = mg.default_opts()
    assert (o.prec, o.mode_fmg, o.pre, o.post) == (0, 1, 1, 1)
    assert o.omega == 1.15 and o.max_cycles == 50 and o.lmax == 4 and o.use_com == 1
    assert o.stall_ratio == 0.9 and o.inner_fmg == 0 and o.inner_cycles == 3
    assert o.outer_fixed == 1 and o.fas == 0
    assert o.coarse_literal == 0
    assert list(o.reserved) == [0] and o.batch_small == 0 and o.tensor_copies == 0
    assert o.first_cycles == 0
    assert o.leg_pairs == 0


@pytest.mark.parametrize("py,c", [(mg.Opts, "mg_opts"), (mg.Request, "mg_request"),
                                  (mg.Result, "mg_result"), (mg.ServerStats, "mg_server_stats")])
def test_struct_layout_matches_the_c_header(tmp_path, py, c):
    """Each ctypes mirror has the C compiler's size and offsets."""
    fields = [f for f, _ in py._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "mg.h"\nint main(void){\n'
                   + f'printf("%zu\\n", sizeof({c}));\n'
                   + "".join(f'printf("%zu\\n", offsetof({c}, {f}));\n' for f in fields)
                   + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = [int(x) for x in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert out[0] == ctypes.sizeof(py)
    assert out[1:] == [getattr(py, f).offset for f in fields]


def test_required_bytes_counts_the_hierarchy():
    """mg_required_bytes needs no device: FP64 keeps phi/f pyramids (the finest
    phi is the caller's), MIXED keeps FP32 pyramids plus FP64 f and the
    fixed-point buffer on the finest level."""
    n = 128
    fine = n ** 3
    pyramid = sum(8 ** l for l in range(8))  # 1^3 .. 128^3
    b64 = mg.required_bytes(n, mg.PERIODIC, prec=mg.FP64)
    assert 8 * (pyramid + pyramid - fine) <= b64 <= 8 * (2 * pyramid - fine) + 2 ** 20
    bmx = mg.required_bytes(n, mg.PERIODIC, prec=mg.MIXED)
    # u32 + f32 everywhere, a second u32 on the fused levels (32..128), f64 + int64 finest
    lo = 4 * 2 * pyramid + 4 * (fine + fine // 8 + fine // 64) + 16 * fine
    assert lo <= bmx <= lo + 2 ** 20
    assert mg.required_bytes(n, mg.OPEN, prec=mg.MIXED) > bmx  # boundary faces
    assert mg.required_bytes(2 * n, mg.PERIODIC, prec=mg.MIXED) > 7.9 * bmx
    L = mg.lib()
    b = ctypes.c_size_t(0)
    o = mg.default_opts()
    assert L.mg_required_bytes(12, 12, 12, 0, ctypes.byref(o), ctypes.byref(b)) == 1
    assert L.mg_required_bytes(8, 8, 8, 0, ctypes.byref(o), None) == 1


def test_server_argument_validation_needs_no_gpu():
    L = mg.lib()
    h = ctypes.c_void_p()
    o = mg.default_opts(prec=mg.MIXED)
    assert L.mg_server_create(0, 2, 8, ctypes.byref(o), ctypes.byref(h)) == 1
    assert L.mg_server_create(1 << 30, 0, 8, ctypes.byref(o), ctypes.byref(h)) == 1
    assert L.mg_server_create(1 << 30, 2, 0, ctypes.byref(o), ctypes.byref(h)) == 1
    bad = mg.default_opts(pre=5)
    assert L.mg_server_create(1 << 30, 2, 8, ctypes.byref(bad), ctypes.byref(h)) == 1
    assert not h.value
    assert L.mg_server_submit(None, None, None) == 1
    assert L.mg_server_destroy(None) == 0


def test_status_strings_and_faces_count():
    L = mg.lib()
    for code, name in mg.STATUS.items():
        assert L.mg_status_str(code).decode() == name
    n = 8
    assert L.mg_faces_count(n, n, n) == 6 * (n + 2) ** 2
    assert L.mg_faces_count(4, 8, 2) == 2 * 10 * 4 + 2 * 6 * 4 + 2 * 6 * 10


def test_argument_validation_needs_no_gpu():
    L = mg.lib()
    h = ctypes.c_void_p()
    o = mg.default_opts()
    for args in [(12, 12, 12, 0.1, 0), (4, 8, 8, 0.1, 0), (8, 8, 8, -1.0, 0), (8, 8, 8, 0.1, 7),
                 (1, 1, 1, 0.1, 0)]:
        assert L.mg_create(*args, ctypes.byref(o), ctypes.byref(h)) == 1
        assert not h.value
    bad = mg.default_opts(pre=3)
    assert L.mg_create(8, 8, 8, 0.1, 0, ctypes.byref(bad), ctypes.byref(h)) == 1
    bad = mg.default_opts(omega=2.5)
    assert L.mg_create(8, 8, 8, 0.1, 0, ctypes.byref(bad), ctypes.byref(h)) == 1
    bad = mg.default_opts(coarse_literal=2)
    assert L.mg_create(8, 8, 8, 0.1, 2, ctypes.byref(bad), ctypes.byref(h)) == 1
    # a rule per face: six kinds of periodic (in pairs), fixed or zero gradient,
    # finite values; MG_BC_MIXED is not a kind mg_create takes
    kinds = lambda *k: (ctypes.c_int * 6)(*k)
    vals = (ctypes.c_double * 6)(0, 0, 0, 0, 0.5, float("nan"))
    P, F, Z, OP = mg.PERIODIC, mg.FIXED, mg.ZEROGRAD, mg.OPEN
    for k, v in [(kinds(P, F, Z, Z, F, F), None), (kinds(OP, OP, Z, Z, F, F), None),
                 (kinds(P, P, Z, Z, F, F), vals), (kinds(P, P, Z, Z, 5, F), None)]:
        assert L.mg_create_faces(8, 8, 8, 0.1, k, v, ctypes.byref(o), ctypes.byref(h)) == 1
        assert not h.value
    assert L.mg_create_faces(8, 8, 8, 0.1, None, None, ctypes.byref(o), ctypes.byref(h)) == 1
    assert L.mg_create(8, 8, 8, 0.1, mg.PER_FACE, ctypes.byref(o), ctypes.byref(h)) == 1
    # the batched solve keeps the homogeneous coarse rules
    lit = mg.default_opts(prec=mg.MIXED, coarse_literal=1)
    dims = (ctypes.c_int * 3)(16, 16, 16)
    dx = (ctypes.c_double * 1)(1.0 / 16)
    bcs = (ctypes.c_int * 1)(mg.ZEROGRAD)
    assert L.mg_batch_create(1, dims, dx, bcs, None, ctypes.byref(lit), ctypes.byref(h)) == 1
    assert not h.value
    assert L.mg_solve(None, None, 1.0, 1e-10, None, None, 1, None, None) == 1
    assert L.mg_destroy(None) == 0
    assert L.mg_op_smooth(0, 8, 8, 8, 0.1, 3, 0.0, None, 1.15, 1, 0, None, None, None) == 1
    # mg_op_convert: a kind outside 0..4, a negative count, null arrays
    assert L.mg_op_convert(5, 1, ctypes.c_void_p(8), ctypes.c_void_p(8), None) == 1
    assert L.mg_op_convert(-1, 1, ctypes.c_void_p(8), ctypes.c_void_p(8), None) == 1
    assert L.mg_op_convert(0, -1, ctypes.c_void_p(8), ctypes.c_void_p(8), None) == 1
    assert L.mg_op_convert(2, 4, None, ctypes.c_void_p(8), None) == 1
    assert L.mg_op_convert(4, 0, None, None, None) == 0  # nothing to do, no launch
