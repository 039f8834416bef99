"""A plain-C user of the library: ``tests/c_abi/rclupp_demo.c`` includes only
``rclupp.h`` and the CUDA runtime, links ``librclupp.so`` and ``libcudart``,
and factors a seeded 3000 x 24 matrix by RCLUPP (Algorithm 6), RCLUPPr
(Algorithm 7), CholeskyQR2 (Algorithm 2) and LC2 (Algorithm 4), checking
orthogonality, residual and the triangular R on the host.

The CPU test compiles and links it (the header is valid C and every entry it
calls is exported); the GPU test runs it.
"""
import glob
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_abi", "rclupp_demo.c")
PKG = os.path.join(ROOT, "paper_2412_06551_gb300")


def _cuda_home():
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))


def _build(tmp_path):
    from paper_2412_06551_gb300 import _build as b
    b.build()
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    cuda = _cuda_home()
    cands = [os.path.join(cuda, "lib64"), os.path.join(cuda, "lib")]
    cands += sorted(glob.glob(os.path.join(cuda, "targets", "*", "lib")))
    libdirs = [d for d in cands if os.path.exists(os.path.join(d, "libcudart.so"))]
    if not libdirs:
        pytest.skip("libcudart.so not found under " + cuda)
    exe = str(tmp_path / "rclupp_demo")
    cmd = [cc, "-std=c99", "-O2", "-Wall", "-Werror", "-I" + os.path.join(ROOT, "include"),
           "-I" + os.path.join(cuda, "include"), SRC, "-o", exe, "-L" + PKG, "-lrclupp"]
    cmd += ["-L" + d for d in libdirs] + ["-lcudart", "-lm", "-Wl,-rpath," + PKG]
    cmd += ["-Wl,-rpath," + d for d in libdirs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    return exe


def test_c_program_compiles_and_links(tmp_path):
    assert os.path.exists(_build(tmp_path))


@pytest.mark.gpu
def test_c_program_factors_on_the_device(tmp_path):
    exe = _build(tmp_path)
    r = subprocess.run([exe], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.strip().endswith("ok"), r.stdout
