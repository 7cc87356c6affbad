"""The serving loop's admission policy (HBM budget, resident hierarchies,
least-recently-used eviction, bounded bypass of a waiting request), checked
on the host by a small C++ program built from the library's own header."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2302_13903_gb300", "csrc")


def test_admission_policy(tmp_path):
    exe = tmp_path / "admission_check"
    subprocess.run(["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-I", CSRC,
                    os.path.join(HERE, "cpp", "admission_check.cpp"), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert out.returncode == 0, out.stderr
    assert "admission checks passed" in out.stdout


def test_ticket_book_threads(tmp_path):
    """Two or more threads waiting on one ticket while others poll it: every
    waiter receives the result, the record is freed exactly once, and a
    retired ticket answers "unknown" (mg_tickets.h, used by the serving loop).
    Built with the address and undefined-behaviour sanitizers where the
    compiler has them."""
    exe = tmp_path / "tickets_check"
    src = os.path.join(HERE, "cpp", "tickets_check.cpp")
    base = ["g++", "-std=c++17", "-O1", "-Wall", "-Werror", "-pthread", "-I", CSRC, src,
            "-o", str(exe)]
    r = subprocess.run(base[:1] + ["-fsanitize=address,undefined"] + base[1:],
                       capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(base, check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert out.returncode == 0, out.stderr
    assert "ticket checks passed" in out.stdout
