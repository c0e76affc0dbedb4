"""The C-ABI library builds, loads without a GPU, and exports every entry
point include/ebpoisson.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^[A-Za-z_][\w\s\*]*?\b(eb_\w+)\s*\(", src, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("eb_geom_build", "eb_poisson_setup", "eb_poisson_solve", "eb_field_eval"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_1809_03745_gb300 import build as B
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_and_validation_without_gpu():
    from paper_1809_03745_gb300 import ebpoisson as E
    from paper_1809_03745_gb300 import workloads as W
    lib = E.load(build_if_missing=True)
    assert lib.eb_status_str(0) == b"ok"
    assert lib.eb_status_str(6) == b"unsupported geometry"
    # host-side validation rejects bad sizes before any device work
    desc = W.rod_plane_2d(64)
    desc = dict(desc, n=(60, 60, 1))
    d, keep = E.make_desc(desc)
    h = ctypes.c_void_p()
    st = lib.eb_geom_build(ctypes.byref(d), None, ctypes.byref(h))
    assert st == E.EB_ERR_INVALID
    assert b"multiple of 8" in lib.eb_last_error()
    assert not h.value
    # a handle twice in one batch is refused before any handle is read
    fake = ctypes.c_void_p(0x1000)
    hs = (ctypes.c_void_p * 2)(fake, fake)
    ptrs = (ctypes.c_void_p * 2)(0x2000, 0x3000)
    st = lib.eb_poisson_solve_batched(hs, 2, ptrs, None, ptrs, None, None)
    assert st == E.EB_ERR_INVALID
    assert b"twice" in lib.eb_last_error()
    # a composite set-up with a negative primitive count is refused before any copy
    d2, keep2 = E.make_desc(W.rod_plane_2d(64))
    d2.n_prims = -1
    lo, hi = (ctypes.c_int * 3)(16, 16, 0), (ctypes.c_int * 3)(32, 32, 1)
    st = lib.eb_amr_setup(ctypes.byref(d2), lo, hi, None, None, ctypes.byref(h))
    assert st == E.EB_ERR_INVALID
    assert b"primitive" in lib.eb_last_error()


def test_binding_refuses_to_run_without_library(monkeypatch, tmp_path):
    from paper_1809_03745_gb300 import build as B
    from paper_1809_03745_gb300 import ebpoisson as E
    monkeypatch.setattr(B, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(E, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        E.load()
