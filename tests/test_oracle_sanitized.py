"""The FP64 oracle under AddressSanitizer and UndefinedBehaviorSanitizer.

oracle/sanitize_check.c drives every oracle entry point over the method's
edge cases (no particles, one particle, coincident particles, pairs exactly
2h apart, a jittered patch with walls, surface tension and buffer
particles), in brute-force and cell-list modes; built with the sanitizers
set to abort on the first finding, it must exit 0.
"""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
ORACLE = os.path.join(ROOT, "oracle")


def test_oracle_is_clean_under_asan_and_ubsan():
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("gcc not available")
    with tempfile.TemporaryDirectory() as tmp:
        exe = os.path.join(tmp, "sanitize_check")
        cmd = [gcc, "-O1", "-g", "-std=c11", "-ffp-contract=off", "-fno-omit-frame-pointer",
               "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
               "-I", ORACLE, os.path.join(ORACLE, "sph_oracle.c"),
               os.path.join(ORACLE, "sanitize_check.c"), "-lm", "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0 and "sanitize" in r.stderr:
            pytest.skip("sanitizer runtime not available: " + r.stderr[-200:])
        assert r.returncode == 0, r.stderr
        env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0",
                   UBSAN_OPTIONS="print_stacktrace=1")
        run = subprocess.run([exe], capture_output=True, text=True, env=env, timeout=300)
        assert run.returncode == 0, run.stdout + run.stderr
        assert "oracle sanitized run ok" in run.stdout
