"""The bounds-checked build (RTM_DEBUG=1 loads paper_2001_06444_gb300's
_build_debug/librtm.so).  Its kernels check the index of every global access
they compute from tables or launch scalars (items, samples, shots, receiver
entries, snapshot slots, trace samples, field and image planes); an index
outside its array skips the access and the call returns RTM_ERR_STATE with
the kernel source line, so nothing reads or writes past a buffer and nothing
traps.

The degenerate and ragged-grid parity cases, the source / receiver index
case, the flat reflector, the half-precision cases, the cases that make the
single-step, one-tile-per-block and persistent two-step kernels agree bit for
bit, and the Born cases run against the oracle in a child process that loads
the debug library: any failed check fails them."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_build_runs_the_parity_cases_cleanly():
    from paper_2001_06444_gb300 import build

    build.build(debug=True)
    env = dict(os.environ, RTM_DEBUG="1")
    which = subprocess.run(
        [sys.executable, "-c", "from paper_2001_06444_gb300 import rtm; print(rtm.lib()._name)"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert which.returncode == 0, which.stderr[-2000:]
    assert "_build_debug" in which.stdout, which.stdout
    cases = ("degenerate or ragged or indices or flat_reflector or half_precision_snapshots or "
             "bitwise or many_tiles or empty or born_matches_oracle or adjoint_matches")
    r = subprocess.run(
        [sys.executable, "-m", "pytest", "-x", "-q", "-m", "gpu", "-k", cases,
         "tests/test_gpu_parity.py", "tests/test_gpu_born.py"],
        cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-4000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "deselected" in r.stdout
