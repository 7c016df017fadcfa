"""The C ABI library builds, loads without a GPU, and exports every function include/flix.h declares."""
import ctypes
import os
import re

import pytest

from tests.conftest import ROOT


def declared_functions():
    src = open(os.path.join(ROOT, "include", "flix.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(flix_\w+)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ("flix_create", "flix_bulk_load", "flix_insert", "flix_delete", "flix_lookup", "flix_successor",
              "flix_range", "flix_destroy", "flix_apply", "flix_restructure"):
        assert n in names


def test_library_exports_every_declared_symbol():
    from paper_2604_16725_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    import paper_2604_16725_gb300 as fx
    assert sorted(fx.SIGNATURES) == declared_functions()


def test_strerror_without_gpu():
    import paper_2604_16725_gb300 as fx
    L = fx.load()
    assert L.flix_strerror(0) == b"ok"
    assert b"KEY_MAX" in L.flix_strerror(-1)
