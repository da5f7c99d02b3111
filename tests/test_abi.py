"""The C-ABI library loads and exports every entry point include/lbd.h
declares, with matching binding signatures; argument validation that happens
before any CUDA call is checked here without a GPU."""
import ctypes
import os
import re

import pytest

from paper_1711_10984_gb300 import lbd

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "lbd.h")


def declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbd_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_10984_gb300 import build
    build.build()
    return lbd.load()


def test_every_declared_symbol_is_exported(lib):
    names = declared()
    assert "lbd_create" in names and "lbd_step" in names
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    assert sorted(lbd.SIGNATURES) == declared()


def test_struct_layout_matches_header():
    # lbd_params: 11 doubles + int64 + 4 doubles + 4 int32 + 64 sources of 3 doubles
    assert ctypes.sizeof(lbd.lbd_params) == 11 * 8 + 8 + 4 * 8 + 4 * 4 + 64 * 24
    assert ctypes.sizeof(lbd.lbd_diag) == 8 * 8 + 8


def _create(**kw):
    p = lbd.make_params(**kw)
    g = lbd.lbd_grid(kw.pop("nx", 16), kw.pop("ny", 16))
    h = ctypes.c_void_p()
    return lbd.load().lbd_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h))


@pytest.mark.parametrize("bad", [dict(tau=0.5), dict(tau=0.2), dict(b=-1.0),
                                 dict(precision=7), dict(M=float("nan")), dict(flags=64)])
def test_create_rejects_bad_parameters(lib, bad):
    assert _create(**bad) == lbd.LBD_EINVAL


def test_create_rejects_bad_grid(lib):
    p = lbd.make_params()
    h = ctypes.c_void_p()
    for nx, ny in [(3, 16), (16, 2), (1 << 21, 8)]:
        g = lbd.lbd_grid(nx, ny)
        assert lib.lbd_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h)) == lbd.LBD_EINVAL


def test_strerror_names_codes(lib):
    for code in (0, -1, -2, -3, -4, -5, -6):
        assert lib.lbd_strerror(code).startswith(b"LBD_")
    assert (32, 8) in lbd.tiles() and (116, 64) in lbd.tiles() and (118, 64) in lbd.tiles()


HEADER3 = os.path.join(ROOT, "include", "lbd3.h")


def declared3():
    src = open(HEADER3).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lbd3_[a-z_0-9]+)\s*\(", src)))


def test_3d_symbols_exported_and_bound(lib):
    from paper_1711_10984_gb300 import lbd3
    names = declared3()
    assert "lbd3_create" in names and "lbd3_step" in names
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbd3.SIGNATURES) == names


def test_3d_struct_layout():
    from paper_1711_10984_gb300 import lbd3
    assert ctypes.sizeof(lbd3.lbd3_params) == ctypes.sizeof(lbd.lbd_params) + 2 * 8 + 2 * 4 + 64 * 32
    assert ctypes.sizeof(lbd3.lbd3_diag) == 7 * 8 + 8
    assert ctypes.sizeof(lbd3.lbd3_grid) == 12


@pytest.mark.parametrize("grid,bad", [((8, 8, 8), dict(tau=0.5)), ((8, 8, 8), dict(flags=16)),
                                      ((8, 8, 8), dict(b=-1.0)), ((0, 8, 8), {}),
                                      ((8, 8, 5000), {})])
def test_3d_create_rejects_bad_input(lib, grid, bad):
    from paper_1711_10984_gb300 import lbd3
    lbd3.load()
    p = lbd3.make_params(**bad)
    g = lbd3.lbd3_grid(*grid)
    h = ctypes.c_void_p()
    assert lib.lbd3_create(ctypes.byref(g), ctypes.byref(p), None, ctypes.byref(h)) == lbd.LBD_EINVAL


@pytest.mark.parametrize("nx,ny,pitch", [((1 << 20) + 1, 8, (1 << 20) + 1), (0, 8, 8),
                                         (16, 8, 15), (16, 8, (1 << 40) + 1),
                                         (1 << 20, 1 << 20, 1 << 40)])
def test_static_diagnostics_rejects_bad_shape(lib, nx, ny, pitch):
    """lbd_diagnostics_static refuses lattices beyond its scratch limits and
    pitches whose plane offsets would overflow, before any CUDA call."""
    out = lbd.lbd_diag()
    rc = lib.lbd_diagnostics_static(nx, ny, pitch, lbd.LBD_FP64, 1, 1, 1, 0.006, -0.05, 0.0, 0.0,
                                    None, ctypes.byref(out))
    assert rc == lbd.LBD_EINVAL
