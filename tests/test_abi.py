"""The C-ABI library builds, loads and exports every symbol include/fciqmc.h declares (CPU only;
only host-side entry points that need no GPU are called)."""
from __future__ import annotations

import ctypes
import os
import re
import subprocess

import pytest

from paper_1305_6981_gb300 import _native, synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "fciqmc.h")).read()
    return sorted(set(re.findall(r"\b(fciqmc_[a-z_]+)\s*\(", src)))


def test_header_and_binding_agree():
    assert declared_symbols() == sorted(_native.SYMBOLS)


def test_library_exports_every_declared_symbol():
    path = _native.build()
    L = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(L, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (fciqmc_[a-z_]+)$", out, flags=re.M))
    assert set(declared_symbols()) <= exported


def test_host_only_entry_points():
    L = _native.load()
    o = _native.Options()
    L.fciqmc_default_options(ctypes.byref(o))
    assert o.shift_period == 10 and o.initial_population == 10 and o.shift_damping == 0.05
    for s in (synth.tiny_8e8o(), synth.init_12e24o()):
        n = L.fciqmc_workspace_bytes(s.n_elec, s.n_orb, ctypes.byref(o))
        assert n > 0 and n % 256 == 0
    # limits: n_orb <= 64, n_elec < 2 n_orb
    assert L.fciqmc_workspace_bytes(8, 65, None) == 0
    assert L.fciqmc_workspace_bytes(16, 8, None) == 0
    assert L.fciqmc_strerror(-2).decode().startswith("capacity")


def test_workspace_grows_with_capacity():
    L = _native.load()
    o = _native.Options()
    L.fciqmc_default_options(ctypes.byref(o))
    o.main_capacity = 1 << 16
    a = L.fciqmc_workspace_bytes(24, 60, ctypes.byref(o))
    o.main_capacity = 1 << 18
    b = L.fciqmc_workspace_bytes(24, 60, ctypes.byref(o))
    assert b > a
    # two-word determinants: 16 bytes per slot per buffer at least
    assert b - a >= 2 * 16 * ((1 << 18) - (1 << 16))


def test_product_package_does_not_import_the_oracle():
    for name in os.listdir(os.path.join(ROOT, "paper_1305_6981_gb300")):
        if name.endswith(".py"):
            src = open(os.path.join(ROOT, "paper_1305_6981_gb300", name)).read()
            assert not re.search(r"^\s*(from|import)\s+oracle", src, flags=re.M), name
            assert "liboracle" not in src and "fciqmc_oracle" not in src, name


def test_struct_layouts_match_the_header(tmp_path):
    """Every public struct of include/fciqmc.h has the size and field offsets its ctypes mirror assumes
    (compiled with the host C compiler; the header is plain C)."""
    pairs = {"fciqmc_options": _native.Options, "fciqmc_row": _native.Row, "fciqmc_estimates": _native.Estimates,
             "fciqmc_state": _native.State, "fciqmc_info": _native.Info}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "fciqmc.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            lines.append(f'    printf("{cname} {f} %zu\\n", offsetof({cname}, {f}));')
    lines += ["    return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)])
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        cname, field, value = line.split()
        got[(cname, field)] = int(value)
    for cname, py in pairs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)
