"""Host-side checks of the C ABI that need no GPU: the library builds for
sm_103a, loads, and exports every entry point include/wake.h declares; the
product package never imports the oracle."""
import ctypes
import os
import re

import pytest

from paper_2603_16623_gb300 import build as wbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wake_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    lib_path = wbuild.build()
    lib = ctypes.CDLL(lib_path)
    names = []
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            names += _declared(os.path.join(ROOT, "include", h))
    assert len(names) >= 13
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_limits_are_queryable_without_a_gpu():
    from paper_2603_16623_gb300 import wake
    assert wake.wake_max_rings("mixed") >= 8192
    assert wake.wake_max_slice_particles("fp64") >= 8192


def test_product_does_not_touch_the_oracle():
    pkg = os.path.join(ROOT, "paper_2603_16623_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle", src, re.M), f
                assert "wake_oracle" not in src and "liboracle" not in src, f
