"""The debug build of the library (-DFCIQMC_DEBUG: every device table index that the algorithm keeps in range by
construction is checked, and a violation is reported as FCIQMC_ERR_BOUNDS instead of being accessed) compiles
for sm_103a and exports every entry point the header declares. Runs on the CPU (no kernel is launched)."""
from __future__ import annotations

import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_debug_library_builds_and_exports_the_abi():
    code = ("import sys, ctypes; sys.path.insert(0, '.'); from paper_1305_6981_gb300 import _native; "
            "p = _native.build(); assert p.endswith('libfciqmc_debug.so'), p; L = ctypes.CDLL(p); "
            "missing = [s for s in _native.SYMBOLS if not hasattr(L, s)]; assert not missing, missing; "
            "assert L.fciqmc_strerror.__call__ is not None; print('ok', len(_native.SYMBOLS))")
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=dict(os.environ, FCIQMC_DEBUG_BUILD="1"),
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-2000:]
    assert r.stdout.strip().startswith("ok")
