"""The C-ABI from plain C: tests/c_consumer.c compiles as C99 against include/isg.h alone, with
every warning an error, and links against libisg.so (CPU); on a GPU it runs and checks Table 1,
the sum and columns, ln Z and an error status (see the program's header)."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def build_consumer(tmp_path, isg):
    exe = os.path.join(str(tmp_path), "c_consumer")
    libdir = os.path.join(ROOT, "paper_1110_2561_gb300")
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_consumer.c"), "-o", exe, "-L", libdir, "-lisg", "-lm",
           "-Wl,-rpath," + libdir]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_consumer_compiles_and_links(tmp_path, isg):
    assert os.path.exists(build_consumer(tmp_path, isg))


@pytest.mark.gpu
def test_c_consumer_runs(tmp_path, isg, cuda):
    exe = build_consumer(tmp_path, isg)
    r = subprocess.run([exe, os.path.join(ROOT, "tests", "golden", "table1_4x4_periodic.txt")], capture_output=True,
                       text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "c consumer ok" in r.stdout
