"""The C ABI used from plain C: compile tests/c_abi_droplet.c against include/lbm.h
and liblbm.so with gcc, no Python binding and no PyTorch on the path (the compile
check runs on the CPU; running the program needs a GPU)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi_droplet.c")
CUDA_LIB = "/usr/local/cuda/lib64"


def _compile(out):
    from paper_1507_07294_gb300 import _build
    lib = _build.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), SRC,
           "-o", out, "-L", os.path.dirname(lib), "-llbm", "-Wl,-rpath," + os.path.dirname(lib),
           "-Wl,-rpath," + CUDA_LIB, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr


def test_c_program_compiles_against_the_header(tmp_path):
    _compile(str(tmp_path / "c_abi_droplet"))


@pytest.mark.gpu
def test_c_program_runs_a_droplet(tmp_path):
    exe = str(tmp_path / "c_abi_droplet")
    _compile(exe)
    env = {k: v for k, v in os.environ.items() if k != "PYTHONPATH"}
    r = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
    print(r.stdout, r.stderr)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("steps=200 ")
