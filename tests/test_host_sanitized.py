"""The CPU oracle and the kernels' row arithmetic under AddressSanitizer and
UBSan (no GPU).

Each case reruns a test file in a child process with the C oracle
(``ELSR_ORACLE_SANITIZE=1``) and the host build of the kernels' row code
(``ELSR_HC_SANITIZE=1``) compiled with -fsanitize=address,undefined, so any
out-of-range index, signed overflow or invalid shift ends the child with an
error:

* tests/test_oracle_pins.py: the oracle's decode, neighbourhoods, VND, GVNS,
  fork-join and multi-start on every pinned case;
* tests/test_row_host.py: elsr_row.cuh (decode, row cache, delta re-decode)
  with buffers of exactly the kernels' shared-memory extents (A, C, L: T
  entries; P, Q and the prefix tables: T + 1), against the oracle.

No device-side sanitizer runs in this suite; this covers the oracle that
every parity test trusts and the row code every kernel inlines.
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


@pytest.mark.parametrize("target", ["test_oracle_pins.py", "test_row_host.py"])
def test_under_sanitizers(target):
    asan, ubsan = _runtime("libasan.so"), _runtime("libubsan.so")
    if not asan or not ubsan:
        pytest.skip("gcc sanitizer runtimes not installed")
    env = dict(os.environ, ELSR_HC_SANITIZE="1", ELSR_ORACLE_SANITIZE="1",
               LD_PRELOAD=f"{asan}:{ubsan}", ASAN_OPTIONS="detect_leaks=0:halt_on_error=1",
               UBSAN_OPTIONS="halt_on_error=1:print_stacktrace=1")
    r = subprocess.run([sys.executable, "-m", "pytest", os.path.join(HERE, target),
                        "-x", "-q", "-p", "no:cacheprovider"],
                       cwd=os.path.dirname(HERE), env=env, capture_output=True, text=True,
                       timeout=900)
    tail = (r.stdout + r.stderr)[-4000:]
    assert r.returncode == 0, tail
    assert "passed" in r.stdout and "Sanitizer" not in tail, tail
