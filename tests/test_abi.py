"""CPU checks of the boundary: the library builds, loads and exports every declared symbol."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header):
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(sph\w*)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2511_15908_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_every_declared_symbol_is_exported(lib):
    names = _declared("sph.h")
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_the_header(lib):
    from paper_2511_15908_gb300 import sph
    assert sorted(sph.SYMBOLS) == _declared("sph.h")


def test_workspace_size_and_argument_checks(lib):
    from paper_2511_15908_gb300 import scenes, sph
    L = sph.load()
    sc = scenes.dam_break()
    P = sph.make_params(sc.params, sc.fluid_spacing)
    cap = sph.Capacity(sc.n_total, 2, 0, 100)
    n = L.sph_workspace_bytes(ctypes.byref(P), ctypes.byref(cap))
    assert n > 160 * sc.n_total
    bad = sph.make_params(sc.params, sc.fluid_spacing)
    bad.cell = 0.5 * bad.h          # cell below h
    assert L.sph_workspace_bytes(ctypes.byref(bad), ctypes.byref(cap)) == 0
    cap_bad = sph.Capacity(sc.n_total, 65, 0, 100)
    assert L.sph_workspace_bytes(ctypes.byref(P), ctypes.byref(cap_bad)) == 0
    h = ctypes.c_void_p()
    # null workspace is rejected before any device call
    st = L.sph_create(ctypes.byref(P), ctypes.byref(cap), None, 0, None, 0, None, None,
                      ctypes.byref(h))
    assert st == sph.ERR_WORKSPACE
    st = L.sph_create(None, ctypes.byref(cap), None, 0, None, 0, None, None, ctypes.byref(h))
    assert st == sph.ERR_ARG


def test_grid_dims_match_oracle(lib):
    import numpy as np
    import oracle
    from paper_2511_15908_gb300 import scenes
    for sc in (scenes.dam_break(), scenes.tiny()):
        d = oracle.grid_dims(sc.params)
        assert np.all(d > 2)
