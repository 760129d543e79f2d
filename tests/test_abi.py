"""The C ABI library builds, loads and exports every entry point of include/lbm.h, and
its host-side argument validation works without a GPU (no compute calls here)."""
import ctypes
import os
import re

import pytest

from paper_1507_07294_gb300 import lbm as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names.update(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    return L.load_library()


def test_header_declares_the_entry_points():
    names = declared_functions()
    for required in ("lbm_create", "lbm_init_phi", "lbm_step", "lbm_read_fields", "lbm_reduce",
                     "lbm_destroy", "lbm_last_error"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    assert set(declared_functions()) <= set(L._SIGNATURES)


def _create(lib, grid, params, alloc=None):
    out = ctypes.c_void_p()
    st = lib.lbm_create(ctypes.byref(grid), ctypes.byref(params), alloc, None, ctypes.byref(out))
    return st, out


def _good():
    grid = L.LbmGrid(8, 8, 8, 0)
    params = L.make_params(3.0, 1.0, 0.1, 0.1, 0.1, 4.0, 0.01)
    return grid, params


@pytest.mark.parametrize("mutate,expect", [
    (lambda g, p: setattr(g, "nx", 0), "grid sizes"),
    (lambda g, p: setattr(g, "walls_z", 2), "walls_z"),
    (lambda g, p: setattr(p, "rho_g", 0.0), "densities"),
    (lambda g, p: setattr(p, "nu_l", -1.0), "viscosities"),
    (lambda g, p: setattr(p, "A", 0.4), "A must"),
    (lambda g, p: p.sf.__setitem__(4, 2.0), "sf rates"),
    (lambda g, p: p.sf.__setitem__(2, 1.3), "s_1 = s_2 = s_3"),
    (lambda g, p: p.sg.__setitem__(0, 0.0), "sg rates"),
    (lambda g, p: setattr(p, "storage", 7), "storage"),
    (lambda g, p: setattr(p, "pattern", 2), "pattern"),
    (lambda g, p: setattr(p, "flags", 8), "flag"),
    (lambda g, p: (setattr(g, "nx", 2048), setattr(g, "ny", 1024), setattr(g, "nz", 1024)), "2^31"),
])
def test_create_rejects_bad_arguments(lib, mutate, expect):
    grid, params = _good()
    mutate(grid, params)
    st, out = _create(lib, grid, params)
    assert st == L.LBM_EINVAL
    assert out.value is None
    assert expect in lib.lbm_last_error(None).decode()


def test_viscous_rates_are_not_validated(lib):
    """lambda_9..13 come from nu(phi), so their input values are ignored."""
    grid, params = _good()
    params.sg[10] = 5.0
    grid.nx = 0  # still fails, but for the grid, not for sg[10]
    st, _ = _create(lib, grid, params)
    assert st == L.LBM_EINVAL
    assert "grid" in lib.lbm_last_error(None).decode()


def test_null_arguments(lib):
    grid, params = _good()
    assert lib.lbm_create(ctypes.byref(grid), ctypes.byref(params), None, None, None) == L.LBM_EINVAL
    assert lib.lbm_step(None, 1) == L.LBM_EINVAL
    assert lib.lbm_destroy(None) == L.LBM_EINVAL
    assert lib.lbm_init_phi(None, None, None, None) == L.LBM_EINVAL


def test_size_bound_of_the_grid():
    """Grids of up to 2^31 - 65 cells are admitted, 2^31 - 64 are not (lbm_memory_bytes
    applies lbm_create's checks without a GPU).  The largest grid with whole pairs of
    tiles per row, 2^31 - 128 = 128 x 1365 x 12291 cells, takes 92.6 B per cell with
    16-bit populations in place: 56 B of cell state (a 1792-byte tile per 32 cells),
    36 B of FP32 planes (phi, mu and seven staging planes) and 0.625 B of per-warp step
    sums (5 floats per 32 cells)."""
    params = L.make_params(3.0, 1.0, 0.1, 0.1, 0.1, 4.0, 0.01, storage="fp16", pattern="aa")
    n = 128 * 1365 * 12291
    assert n == 2 ** 31 - 128
    b = L.lbm_memory_bytes(L.LbmGrid(128, 1365, 12291, 0), params)
    assert 56 * n + 36 * n + 20 * n // 32 <= b <= 56 * n + 36 * n + 20 * n // 32 + (1 << 20)
    assert L.lbm_memory_bytes(L.LbmGrid(1, 1, 2 ** 31 - 65, 1), params) > 0
    with pytest.raises(L.LbmError) as e:
        L.lbm_memory_bytes(L.LbmGrid(64, 31, 1082401, 0), params)  # 2^31 - 64 cells
    assert e.value.status == L.LBM_EINVAL


def test_binding_constants_match_the_header():
    """Every numeric #define and status value of include/lbm.h has the same value in the
    Python binding."""
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    consts = dict(re.findall(r"^#define (LBM_[A-Z0-9_]+)\s+([0-9]+)u?\b", text, re.M))
    consts.update(re.findall(r"^\s*(LBM_[A-Z]+)\s*=\s*([0-9]+)", text, re.M))
    assert len(consts) >= 35
    wrong = {k: (v, getattr(L, k, None)) for k, v in consts.items() if getattr(L, k, None) != int(v)}
    assert not wrong, wrong
