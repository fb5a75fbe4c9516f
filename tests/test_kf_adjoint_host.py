"""The hand-written Kalman-filter adjoints of the CUDA path (csrc/kf.cuh: rotation, helix step, two-
coordinate and scalar measurement updates, and the step to the vertex) compiled in double precision
with the host compiler and compared with central differences of their forward functions
(tests/kf_adjoint_check.cpp).  No GPU; the oracle is not involved."""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def test_kf_adjoints_match_central_differences(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "kf_adjoint_check")
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_1712_09434_gb300", "csrc"),
                           os.path.join(HERE, "kf_adjoint_check.cpp"), "-o", exe])
    out = subprocess.check_output([exe], text=True).split()
    cases, worst = int(out[1]), float(out[3])
    assert cases >= 150
    assert worst < 1e-4, worst


def test_flop_counts_match_the_bench_roofline_constants(tmp_path):
    """The per-hit operation counts of the Kalman kernels that bench.py uses for the FP32 roofline
    are the counts of the implemented formulas (kf.cuh instantiated with a counting scalar)."""
    import bench
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    exe = str(tmp_path / "kf_flop_count")
    subprocess.check_call([cxx, "-O1", "-std=c++17", "-I", os.path.join(ROOT, "paper_1712_09434_gb300", "csrc"),
                           os.path.join(HERE, "kf_flop_count.cpp"), "-o", exe])
    got = {}
    for line in subprocess.check_output([exe], text=True).splitlines():
        name, n = line.split()[:2]
        got[name] = int(n)
    assert got == {"forward": bench.FLOP_FWD, "adjoint": bench.FLOP_ADJ, "sqrt_forward": bench.FLOP_SQRT_FWD}
