"""The boundary from plain C: a C program built against include/mg.h and the
library solves the periodic sinusoid through mg_solve and mg_solve_host and
checks the exact discrete solution (Sec. 4.1)."""
import os
import subprocess

import pytest

import paper_2302_13903_gb300 as mg

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def test_c_caller_solves_the_sinusoid(tmp_path):
    lib = mg.library_path()
    mg.lib()  # built and loadable
    exe = tmp_path / "sinusoid_solve"
    libdir = os.path.dirname(lib)
    name = os.path.basename(lib)[3:-3]  # libNAME.so -> NAME
    subprocess.run(["gcc", "-std=c11", "-O1", "-Wall", "-Werror",
                    "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
                    os.path.join(HERE, "c", "sinusoid_solve.c"), "-o", str(exe),
                    "-L", libdir, "-l" + name, "-L", os.path.join(CUDA, "lib64"), "-lcudart",
                    "-lm", "-Wl,-rpath," + libdir, "-Wl,-rpath," + os.path.join(CUDA, "lib64")],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "C caller checks passed" in out.stdout
