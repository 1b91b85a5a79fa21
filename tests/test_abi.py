"""The C-ABI library loads and exports every symbol include/td.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    syms = set()
    for name in os.listdir(os.path.join(ROOT, "include")):
        if not name.endswith(".h"):
            continue
        text = open(os.path.join(ROOT, "include", name)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(td_[a-z0-9_]+)\s*\(", text):
            syms.add(m.group(1))
    return sorted(syms)


@pytest.fixture(scope="module")
def libtd():
    from paper_2603_06010_b300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_hot_path_calls():
    syms = declared_symbols()
    for name in ("td_segment_create", "td_factor", "td_loglike_batch", "td_logdet"):
        assert name in syms


def test_every_declared_symbol_is_exported(libtd):
    missing = [s for s in declared_symbols() if not hasattr(libtd, s)]
    assert not missing, missing


def test_binding_covers_every_symbol():
    from paper_2603_06010_b300 import td
    assert sorted(td.SIGNATURES) == declared_symbols()


def test_host_side_validation_without_gpu(libtd):
    """Argument checks run on the host before any device call."""
    from paper_2603_06010_b300 import td
    L = td.lib()
    out = ctypes.c_void_p()
    assert L.td_segment_create(None, 4, None, None, ctypes.byref(out)) == td.TD_ERR_INVALID
    import numpy as np
    bad = np.array([-1.0, 0.0])
    assert L.td_segment_create(bad.ctypes.data, 2, None, None, ctypes.byref(out)) == td.TD_ERR_INVALID
    assert b"acf[0]" in L.td_last_error()
    m = np.zeros(2, np.uint8)
    good = np.array([1.0, 0.0])
    assert L.td_segment_create(good.ctypes.data, 2, m.ctypes.data, None, ctypes.byref(out)) == td.TD_ERR_INVALID
    assert L.td_kept(None) == -1
    assert L.td_loglike_batch(None, None, 0, 0, None, None, None, None) == td.TD_ERR_INVALID
