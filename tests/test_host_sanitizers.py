"""The library's host-side C++ (S_N tables, batch geometry, block-cyclic-reduction
schedule) built with AddressSanitizer and UndefinedBehaviorSanitizer and run on the CPU
against the invariants written out in tests/host_sanitize_check.cpp: any out-of-bounds
access, use after free, leak, signed overflow or broken invariant fails the test."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1907_13013_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"


def test_host_code_under_asan_and_ubsan(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.exists(os.path.join(CUDA_INC, "cuda_runtime.h")):
        pytest.skip("g++ or the CUDA headers are missing")
    exe = str(tmp_path / "host_check")
    cmd = [gxx, "-std=c++17", "-O1", "-g", "-fsanitize=address,undefined", "-fno-sanitize-recover=all",
           "-fno-omit-frame-pointer", "-I" + CUDA_INC, os.path.join(ROOT, "tests", "host_sanitize_check.cpp"),
           os.path.join(CSRC, "tables.cpp"), os.path.join(CSRC, "geometry.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0 and "sanitize" in r.stderr and ("cannot find" in r.stderr or "unrecognized" in r.stderr):
        pytest.skip("this compiler has no sanitizer runtime: " + r.stderr.strip().splitlines()[-1])
    assert r.returncode == 0, r.stderr
    env = dict(os.environ, ASAN_OPTIONS="detect_leaks=1:abort_on_error=0", UBSAN_OPTIONS="print_stacktrace=1")
    run = subprocess.run([exe], capture_output=True, text=True, timeout=300, env=env)
    assert run.returncode == 0 and "host check ok" in run.stdout, run.stdout[-3000:] + run.stderr[-3000:]
