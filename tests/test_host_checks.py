"""Host-side logic of the GPU path checked on the CPU (no GPU needed).

ordered_key (the integer keys with which the corrector decides whether a
particle has left the domain box, in place of FP64 comparisons) must order
doubles exactly as the comparisons do, equate -0 and +0, and let no NaN pass a
two-sided bound test: a C++ driver built with the host compiler checks it over
edge cases and random bit patterns.
"""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1603_02421_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


def test_ordered_key_orders_doubles_like_comparisons(tmp_path):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("host C++ compiler or CUDA headers not available")
    exe = str(tmp_path / "ordered_key_check")
    src = os.path.join(ROOT, "tests", "host", "ordered_key_check.cpp")
    r = subprocess.run([cxx, "-std=c++17", "-O1", "-x", "c++", "-I", CSRC,
                        "-I", os.path.join(ROOT, "include"), "-I", CUDA_INC, src, "-o", exe],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([exe], capture_output=True, text=True)
    assert out.returncode == 0, out.stdout + out.stderr
    assert "mismatches 0" in out.stdout
