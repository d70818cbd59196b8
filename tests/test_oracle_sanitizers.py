"""The oracle under AddressSanitizer and UndefinedBehaviorSanitizer (CPU): a C
driver calls every oracle entry point on seeded inputs and edge cases; any
out-of-bounds access, leak or undefined operation fails the run."""
from __future__ import annotations

import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_runs_clean_under_asan_and_ubsan(tmp_path):
    cc = os.environ.get("CC", "gcc")
    if shutil.which(cc) is None:
        pytest.skip("no C compiler")
    exe = tmp_path / "oracle_sanitized"
    cmd = [cc, "-std=c99", "-O1", "-g", "-fno-omit-frame-pointer", "-ffp-contract=off",
           "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-pthread",
           os.path.join(ROOT, "oracle", "fpw_oracle.c"), os.path.join(ROOT, "oracle", "sanitize_driver.c"),
           "-o", str(exe), "-lm"]
    build = subprocess.run(cmd, capture_output=True, text=True)
    if build.returncode != 0 and "sanitize" in (build.stderr + build.stdout):
        pytest.skip(f"sanitizers unavailable: {build.stderr.strip()[:200]}")
    assert build.returncode == 0, build.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([str(exe)], capture_output=True, text=True, env=env, timeout=120)
    assert run.returncode == 0, run.stdout + run.stderr
    assert "oracle sanitizer run ok" in run.stdout
    assert "runtime error" not in run.stderr and "AddressSanitizer" not in run.stderr
