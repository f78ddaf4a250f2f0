"""The C ABI used from C alone: tests/c_abi_roundtrip.c includes only
include/pat.h and links the built library. On the CPU it must compile, link
and pass its host-only queries (folded layout, plan estimate); on the GPU it
runs H and H* on host arrays and checks the adjoint identity (Eq. 9)."""
import os
import shutil
import subprocess

import pytest

from paper_2603_28150_gb300 import build as pbuild
from paper_2603_28150_gb300 import pat

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _build(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pat.lib()  # builds libpat.so in-tree if needed
    libdir = os.path.dirname(pbuild.LIB)
    exe = str(tmp_path / "c_abi_roundtrip")
    cmd = [cc, "-std=c11", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
           os.path.join(ROOT, "tests", "c_abi_roundtrip.c"), "-o", exe, "-L", libdir, "-lpat",
           f"-Wl,-rpath,{libdir}", "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    return exe


def test_c_program_host_queries(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe, "--layout"], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "host queries ok" in r.stdout


@pytest.mark.gpu
def test_c_program_adjoint_identity(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "relative gap" in r.stdout
