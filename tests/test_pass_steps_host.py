"""Planner host check: the pass kernels' step table (row turns composed into
4x4 blocks) applies the same operator as the method's paired steps one by one.
Compiles tests/host/pass_steps_check.cpp against the planner sources with the
host compiler; no GPU and no device code involved."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_2608_13110_gb300", "csrc")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "vector_types.h")):
            return os.path.join(d, "include")
    return None


@pytest.fixture(scope="module")
def checker(tmp_path_factory):
    cxx = shutil.which("g++")
    inc = _cuda_include()
    if not cxx or not inc:
        pytest.skip("needs g++ and the CUDA headers")
    exe = str(tmp_path_factory.mktemp("pass_steps") / "pass_steps_check")
    srcs = [os.path.join(ROOT, "tests", "host", "pass_steps_check.cpp")] + [
        os.path.join(CSRC, f) for f in ("plan.cpp", "tc_plan.cpp", "open_plan.cpp")]
    r = subprocess.run([cxx, "-O2", "-std=c++17", "-I", inc, "-I", os.path.join(ROOT, "include"), "-I", CSRC,
                        *srcs, "-o", exe], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return exe


@pytest.mark.parametrize("args", [
    (8, 30), (6, 34), (9, 27), (6, 36, 8, 10, 9), (10, 28, 9, 10, 5), (6, 40, 9, 8, 6), (8, 44, 9, 10, 7), (9, 41, 6, 10, 7),
])
def test_pass_step_table_equals_method_steps(checker, args):
    r = subprocess.run([checker, *map(str, args)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "blocks=" in r.stdout and "blocks=0 " not in r.stdout, r.stdout
