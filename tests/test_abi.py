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


def test_config_defaults_and_create_validation_without_gpu():
    """flix_config_default and every argument check of flix_create run on the host before any CUDA
    call: bad configurations are rejected with the documented codes and leave *out NULL."""
    import paper_2604_16725_gb300 as fx
    from paper_2604_16725_gb300.flix import Config
    L = fx.load()
    cfg = Config()
    L.flix_config_default(ctypes.byref(cfg), 1)            # FLIX_KEY_U64
    assert (cfg.key_type, cfg.node_size, cfg.fill_pct, cfg.grow) == (1, 64, 50, 1)
    assert cfg.restructure_in_one_pass == 1 and cfg.split_chains_over == 0 and cfg.merge_underfull == 0
    assert not cfg.dev_alloc and not cfg.dev_free
    L.flix_config_default(ctypes.byref(cfg), 0)            # FLIX_KEY_U32
    assert cfg.node_size == 32
    assert L.flix_create(None, None) == -1                  # FLIX_EINVAL

    def rejected(**fields):
        c = Config()
        L.flix_config_default(ctypes.byref(c), 1)
        for k, v in fields.items():
            setattr(c, k, v)
        h = ctypes.c_void_p(1234)
        code = L.flix_create(ctypes.byref(c), ctypes.byref(h))
        assert h.value is None
        return code

    assert rejected(key_type=7) == -4                       # FLIX_ETYPE
    assert rejected(node_size=3) == -4
    assert rejected(node_size=256) == -4
    assert rejected(fill_pct=0) == -1
    assert rejected(fill_pct=101) == -1
    assert rejected(sort_digit_bits=11) == -7               # FLIX_ENOTIMPL
    assert rejected(sort_variant=9) == -1
    assert rejected(dev_alloc=1) == -1                      # an allocator without its free
    assert rejected(dev_free=1) == -1
