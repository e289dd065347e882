"""Parity with the oracle on the debug build of the library (-DFCIQMC_DEBUG: device table indices - occupied
lists, spawn queues, the per-warp determinant tables, the reference's table, the float integrals - checked
before use, a violation reported as FCIQMC_ERR_BOUNDS and the access skipped). A subset of the GPU parity tests
runs in a child process that loads the debug library: every list, counter and status must be as with the
normal build, i.e. no check ever fires on these workloads."""
from __future__ import annotations

import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_parity_subset_on_the_debug_build():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    tests = [os.path.join(ROOT, "tests", f) for f in
             ("test_gpu_parity.py", "test_gpu_hphf.py", "test_gpu_partition.py", "test_gpu_real.py", "test_gpu_edges.py",
              "test_gpu_space.py")]
    sel = ("plain_8e8o or initiator_12e24o or two_words or heavy_path or partitioned_12e24o or hybrid_8e8o "
           "or hybrid_24e60o or largest or one_electron or active_space")
    r = subprocess.run([sys.executable, "-m", "pytest", *tests, "-q", "-x", "-m", "gpu", "-k", sel,
                        "-p", "no:cacheprovider"], cwd=ROOT, env=dict(os.environ, FCIQMC_DEBUG_BUILD="1"),
                       capture_output=True, text=True, timeout=1800)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]
    assert " passed" in r.stdout and "deselected" in r.stdout
