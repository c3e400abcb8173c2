"""The CUDA library builds for sm_103a, loads, and exports every entry point
declared in include/basker.h (CPU only: no compute call is made)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_1601_05725_gb300 import basker, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = []
    for f in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(basker_[a-z_0-9]+)\s*\(", src)
    return sorted(set(names))


def test_library_builds_and_exports_all_symbols():
    path = build.build()
    assert os.path.exists(path)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT (basker_[a-z_0-9]+)", out))
    declared = _declared()
    assert declared, "no declarations found"
    missing = [n for n in declared if n not in exported]
    assert not missing, missing
    assert set(basker.EXPORTED) <= set(declared)


def test_library_loads_without_a_device():
    lib = basker.load()
    for name in _declared():
        assert hasattr(lib, name)
    assert lib.basker_strerror(4) == b"singular: no nonzero pivot candidate"
    opt = basker.default_options()
    assert opt.tau == 1e-3 and opt.slack == 1.0


def test_build_targets_sm_103a_only():
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]
