"""The C-ABI library builds for sm_103a, loads, and exports every entry point
that include/gs.h declares; host-only entry points give the layout the
oracle computes. No GPU needed (nothing is launched)."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2606_11390_gb300 import _native, build, scenes

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    with open(os.path.join(ROOT, "include", "gs.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gs_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    build.build()
    return _native.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert "gs_project" in names and "gs_bin_sort" in names
    assert "gs_rasterize_fwd" in names and "gs_rasterize_bwd" in names
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing
    # and the binding wraps each of them under the same name
    assert set(names) <= set(_native.exported_symbols())


def test_no_other_gs_symbols_exported(lib):
    # the library hides everything but the C ABI (-fvisibility=hidden)
    out = os.popen(f"nm -D --defined-only {build.LIB_PATH}").read()
    exported = sorted(set(re.findall(r" T (gs_[a-z0-9_]+)$", out, flags=re.M)))
    assert exported == _declared()


def test_layout_totals_match_oracle(lib, oracle):
    for s in (scenes.tiny(N=8), scenes.random_small(1, N=4, width=173, height=91, n_views=3, tile=8)):
        nt, npix = _native.gs_layout_totals(s["sizes"], s["cfg"])
        assert nt == oracle.num_tiles(s)
        assert npix == int((s["sizes"][:, 0].astype(np.int64) * s["sizes"][:, 1]).sum())


def test_host_side_argument_errors(lib):
    cfg = scenes.make_cfg(tile_w=12, tile_h=12)
    with pytest.raises(_native.GSError):
        _native.gs_layout_totals([[64, 64]], cfg)
    cfg = scenes.make_cfg()
    with pytest.raises(_native.GSError):
        _native.gs_layout_totals(np.zeros((0, 2), np.int32), cfg)
    with pytest.raises(_native.GSError):
        _native.gs_layout_totals([[0, 64]], cfg)
    assert _native.gs_version() >= 100
    assert lib.gs_status_string(1) == b"invalid argument"


def test_workspace_grows_with_capacity(lib):
    a = _native.gs_bin_sort_workspace_bytes(1000, 2, 10000, 100)
    b = _native.gs_bin_sort_workspace_bytes(1000, 2, 20000, 100)
    assert 0 < a < b
    assert a % 256 == 0


def _declared_arity():
    """Parameter count of every GS_API function in include/gs.h."""
    with open(os.path.join(ROOT, "include", "gs.h")) as f:
        text = f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    out = {}
    for m in re.finditer(r"GS_API\s+[\w\s\*]+?\b(gs_[a-z0-9_]+)\s*\(([^)]*)\)\s*;", text):
        params = m.group(2).strip()
        out[m.group(1)] = 0 if params in ("", "void") else len(params.split(","))
    return out


def test_binding_signatures_match_the_header():
    # the ctypes argument lists must follow every C-ABI change of the header
    declared = _declared_arity()
    assert len(declared) >= 20
    for name, (args, _res) in _native._SIGNATURES.items():
        assert name in declared, name
        assert len(args) == declared[name], (name, len(args), declared[name])
