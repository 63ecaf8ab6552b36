"""The kernels' row arithmetic under AddressSanitizer and UBSan (no GPU).

``host_row_check.cpp`` compiles elsr_row.cuh for the host with buffers of
exactly the kernels' shared-memory extents (A, C, L: T entries; P, Q and the
prefix tables: T + 1).  This test reruns tests/test_row_host.py in a child
process with that harness built under -fsanitize=address,undefined, so any
index outside those extents, any signed overflow or any invalid shift in the
decode, cache build or delta re-decode ends the child with an error.  Device
sanitizers are not available on the GPU pool; this covers the row code that
every kernel inlines.
"""
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def _runtime(name):
    out = subprocess.run(["gcc", f"-print-file-name={name}"], capture_output=True, text=True)
    path = out.stdout.strip()
    return path if out.returncode == 0 and os.path.isabs(path) and os.path.exists(path) else None


def test_row_arithmetic_under_sanitizers():
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("gcc sanitizer runtimes not installed")
    env = dict(os.environ, ELSR_HC_SANITIZE="1", LD_PRELOAD=f"{asan}:{ubsan}",
               ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, "test_row_host.py"),
                        "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=os.path.dirname(HERE), env=env, capture_output=True, text=True,
                       timeout=900)
    tail = (r.stdout + r.stderr)[-4000:]
    assert r.returncode == 0, tail
    assert "passed" in r.stdout and "ERROR: AddressSanitizer" not in tail, tail
