"""The C ABI used from plain C (paper_1603_08357_gb300/examples/label_triangle.c):
it compiles and links against libccl.so on any host, and on a GPU its labels
match its own host union-find."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "paper_1603_08357_gb300", "examples", "label_triangle.c")
LIBDIR = os.path.join(ROOT, "paper_1603_08357_gb300", "_build")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")


def _compile(out):
    if shutil.which("gcc") is None or not os.path.exists(os.path.join(CUDA, "include", "cuda_runtime.h")):
        pytest.skip("gcc or the CUDA headers are not available")
    import paper_1603_08357_gb300  # noqa: F401  (the library is built)
    cmd = ["gcc", "-O2", "-std=c11", "-I", os.path.join(ROOT, "include"), "-I", os.path.join(CUDA, "include"),
           SRC, "-L", LIBDIR, "-lccl", "-L", os.path.join(CUDA, "lib64"), "-lcudart",
           "-Wl,-rpath," + LIBDIR, "-Wl,-rpath," + os.path.join(CUDA, "lib64"), "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]


def test_c_example_compiles_and_links(tmp_path):
    _compile(str(tmp_path / "label_triangle"))


@pytest.mark.gpu
def test_c_example_runs(tmp_path):
    exe = str(tmp_path / "label_triangle")
    _compile(exe)
    for L, p in (("300", "0.3473"), ("257", "0.6")):
        r = subprocess.run([exe, L, p], capture_output=True, text=True, timeout=300)
        assert r.returncode == 0, r.stdout + r.stderr
        assert r.stdout.strip().endswith("ok"), r.stdout
