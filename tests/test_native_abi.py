"""The C-ABI library loads and exports every entry point declared in include/mtp.h
(symbol lookup only: no compute call is made without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(mtp_[a-z0-9_]+)\s*\(", src))
    return names


def test_every_declared_symbol_is_exported(native_lib):
    lib = ctypes.CDLL(native_lib)
    names = declared_functions()
    assert len(names) >= 20
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing


def test_version_string(native_lib):
    from paper_2304_13144_gb300 import api
    assert b"sm_103a" in api.lib().mtp_version()
