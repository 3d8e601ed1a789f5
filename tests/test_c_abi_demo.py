"""The C ABI from plain C (tests/c_abi_demo.c): the header compiles as C99 and
the program links against libskipper.so and the CUDA runtime alone (CPU); on a
GPU it runs the worked example of Fig. 1 through the CSR, edge-list and server
calls and must print "ok"."""
import os
import subprocess

import pytest

from tests.conftest import cuda_ok

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CUDA = "/usr/local/cuda"


def _build(tmp_path):
    import paper_2507_04420_gb300  # noqa: F401  (the library must be built)
    lib_dir = os.path.join(ROOT, "paper_2507_04420_gb300", "_lib")
    exe = str(tmp_path / "c_abi_demo")
    cmd = ["gcc", "-std=c99", "-Wall", "-Werror", "-O1", os.path.join(ROOT, "tests", "c_abi_demo.c"),
           "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           "-L", lib_dir, "-lskipper", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           f"-Wl,-rpath,{lib_dir}", f"-Wl,-rpath,{os.path.join(CUDA, 'lib64')}", "-o", exe]
    subprocess.run(cmd, check=True, capture_output=True, text=True)
    return exe


def test_header_and_program_build_as_c(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
@pytest.mark.skipif(not cuda_ok(), reason="needs a CUDA GPU")
def test_c_program_runs(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip().endswith("ok"), r.stdout + r.stderr
