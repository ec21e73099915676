"""The C ABI library builds for sm_103a, loads, and exports every entry
point that include/vd.h declares (no compute call: no GPU needed)."""
import ctypes
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(vd_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    from paper_2405_10050_gb300 import build, vd
    path = build.build()
    lib = ctypes.CDLL(path)
    names = _declared()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    assert set(vd.EXPORTS) <= set(names)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True).stdout
    for n in names:
        assert re.search(rf"\bT {n}\b", out), n


def test_status_strings_and_defaults_without_gpu():
    from paper_2405_10050_gb300 import vd
    L = vd.load()
    assert L.vd_status_str(0) == b"ok"
    assert L.vd_status_str(-5) == b"hash table full"
    cfg = vd.vd_config_default()
    assert cfg.box == 1 and cfg.precision == vd.VD_AUTO



def _prototypes():
    """name -> number of parameters of every function include/vd.h declares."""
    src = open(os.path.join(ROOT, "include", "vd.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    out = {}
    for m in re.finditer(r"\b(vd_[a-z0-9_]+)\s*\(([^;{]*?)\)\s*;", src, flags=re.S):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_signatures_match_the_header():
    """Every function the ctypes binding declares takes as many arguments as
    its prototype in include/vd.h (no GPU needed: the library only loads)."""
    from paper_2405_10050_gb300 import vd
    L = vd.load()
    protos = _prototypes()
    assert set(vd.EXPORTS) <= set(protos)
    for name in vd.EXPORTS:
        assert len(getattr(L, name).argtypes) == protos[name], name
