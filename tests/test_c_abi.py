"""The C ABI from plain C: tests/c_abi/free_stream.c includes only af.h,
compiles as C99 with warnings as errors, links against libaf.so and, on a GPU,
keeps a uniform state uniform through five steps."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "free_stream.c")


def _build(tmp_path):
    from paper_2506_04857_gb300 import build
    lib = build.build()
    exe = str(tmp_path / "free_stream")
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-O1", "-I", os.path.join(ROOT, "include"), SRC,
           "-L", libdir, "-laf", "-Wl,-rpath," + libdir, "-lm", "-o", exe]
    subprocess.run(cmd, check=True)
    return exe


def test_header_is_plain_c_and_links(tmp_path):
    exe = _build(tmp_path)
    assert os.path.exists(exe)


@pytest.mark.gpu
def test_free_stream_from_c(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
