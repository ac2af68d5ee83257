"""Host-side checks of the C ABI (no GPU): the library loads, exports every
entry point declared in include/lbps.h, and its pure-host helpers agree with
the oracle bit for bit."""
import ctypes
import re
from pathlib import Path

import numpy as np
import pytest

import oracle as O

ROOT = Path(__file__).resolve().parents[1]


@pytest.fixture(scope="module")
def lib():
    from paper_2301_00228_gb300 import build as B
    B.build()
    from paper_2301_00228_gb300 import lbps
    return lbps


def declared_symbols():
    text = (ROOT / "include" / "lbps.h").read_text()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbps_[a-z_0-9]+)\s*\(", text)))


def test_exports_every_declared_symbol(lib):
    so = ctypes.CDLL(str(lib._LIB_PATH))
    names = declared_symbols()
    assert len(names) >= 15
    missing = [n for n in names if not hasattr(so, n)]
    assert not missing, missing


def test_strerror(lib):
    assert lib.lbps_strerror(0) == "ok"
    assert "non-finite" in lib.lbps_strerror(lib.LBPS_ERR_NONFINITE)
    assert lib.lbps_strerror(-99) == "unknown error"


@pytest.mark.parametrize("nx,ny,px,py,et", [
    (5, 4, 0, 0, (1, 2, 1, 1)), (7, 9, 0, 0, (2, 2, 2, 2)), (3, 3, 0, 0, (1, 1, 1, 1)),
    (8, 6, 1, 0, (2, 1, 1, 2)), (6, 8, 0, 1, (1, 1, 2, 2)), (33, 17, 0, 0, (1, 2, 2, 1))])
def test_rect_bc_matches_oracle_bitwise(lib, nx, ny, px, py, et):
    ev = np.random.default_rng(nx * ny).uniform(-1e-3, 1e-3, 8)
    nt_l, bv_l = lib.lbps_rect_bc(nx, ny, px, py, 0.7, et, ev)
    nt_o, bv_o = O.rect_bc(nx, ny, et, ev, periodic_x=px, periodic_y=py, dh=0.7)
    assert np.array_equal(nt_l, nt_o)
    assert np.array_equal(bv_l.view(np.uint64), bv_o.view(np.uint64))


def test_rect_bc_rejects(lib):
    with pytest.raises(lib.LbpsError):
        lib.lbps_rect_bc(2, 5, 0, 0, 1.0, (1, 1, 1, 1), np.zeros(8))
    with pytest.raises(lib.LbpsError):
        lib.lbps_rect_bc(5, 5, 0, 0, 1.0, (1, 3, 1, 1), np.zeros(8))
    # a periodic direction ignores its edge types
    lib.lbps_rect_bc(5, 5, 1, 0, 1.0, (1, 0, 1, 0), np.zeros(8))


def test_state_bytes(lib):
    p = lib.lbps_params(100, 37, 1.0, 1.0, 1.0, 1.0, 0.9999, 0, 0, 0, 0, lib.LBPS_STORAGE_F32, 0, None)
    n32 = lib.lbps_state_bytes(p)
    p.storage = lib.LBPS_STORAGE_F64
    n64 = lib.lbps_state_bytes(p)
    px = 128
    assert n32 >= 2 * px * 37 * (10 * 4 + 4 * 8)
    assert n64 >= 2 * px * 37 * (10 * 8 + 4 * 8)
    assert n64 > n32
    for code in (lib.LBPS_STORAGE_BF16, lib.LBPS_STORAGE_F16, lib.LBPS_STORAGE_BFP13):
        p.storage = code
        n16 = lib.lbps_state_bytes(p)
        # FP32 f^0, Jx, Jy + two 16-bit sums per set: 32 B per point and copy
        assert 2 * px * 37 * (32 + 4 * 8) <= n16 < n32
        assert n32 - n16 >= 2 * px * 37 * 8
        # a lattice 3 wide along a non-periodic axis is rejected, a periodic one is not
        for nx, ny, pxp, pyp, ok in ((3, 37, 0, 0, False), (100, 3, 0, 0, False), (3, 37, 1, 0, True),
                                     (100, 3, 0, 1, True), (4, 4, 0, 0, True)):
            q = lib.lbps_params(nx, ny, 1.0, 1.0, 1.0, 1.0, 0.9999, pxp, pyp, 0, 0, code, 0, None)
            if ok:
                assert lib.lbps_state_bytes(q) > 0
            else:
                with pytest.raises(lib.LbpsError):
                    lib.lbps_state_bytes(q)
    for bad in (dict(nx=2), dict(mu=0.0), dict(rho=-1.0), dict(a0_phi=1.0), dict(bc_feq_mode=2),
                dict(storage=5), dict(storage=7), dict(storage=-1), dict(sync_every=-1), dict(dh=0.0), dict(pop_scale_exp=101),
                dict(pop_scale_exp=-101)):
        q = lib.lbps_params(100, 37, 1.0, 1.0, 1.0, 1.0, 0.9999, 0, 0, 0, 0, 0, 0, None)
        for k, v in bad.items():
            setattr(q, k, v)
        with pytest.raises(lib.LbpsError):
            lib.lbps_state_bytes(q)


def test_general_geometry_host_checks(lib):
    """Plate with a hole through the host-side checks of lbps_state_bytes_cells
    (no GPU needed): a valid hole costs the node-type plane and five stress
    slots per boundary point; invalid geometries are rejected."""
    nx, ny = 40, 36
    p = lib.lbps_params(nx, ny, 1.0, 1.0, 1.0, 1.0, 0.999, 0, 0, 0, 0, lib.LBPS_STORAGE_F32, 0, None)
    rect = lib.lbps_state_bytes(p)
    nt, bv, cell = lib.lbps_disk_cells(nx, ny, 1.0, 19.3, 17.6, 5.3, (1, 1, 1, 1), np.zeros(8))
    hole = lib.lbps_state_bytes_cells(p, nt, cell)
    assert hole >= rect + 64 * ny                       # + node types (pitched rows)
    assert lib.lbps_state_bytes_cells(p, None, None) == rect
    # a one-point ligament: column 1 then has no difference stencil along x
    bad = nt.copy()
    bad[:, 2] = lib.LBPS_VOID
    bad[:, 3] = lib.LBPS_NEUMANN
    with pytest.raises(lib.LbpsError):
        lib.lbps_state_bytes_cells(p, bad, None)
    wrong = nt.copy()
    wrong[nt == lib.LBPS_NEUMANN] = lib.LBPS_INTERIOR   # boundary points must be Neumann or Dirichlet
    with pytest.raises(lib.LbpsError):
        lib.lbps_state_bytes_cells(p, wrong, cell)
    badcell = cell.copy()
    badcell[nt == lib.LBPS_NEUMANN, 0] = 0.0              # zero cell area
    with pytest.raises(lib.LbpsError):
        lib.lbps_state_bytes_cells(p, nt, badcell)
    # 16-bit storage: a point between two boundary points along x is rejected
    two = np.zeros((ny, nx), np.uint8)
    two[:, [0, nx - 1]] = lib.LBPS_NEUMANN
    two[[0, ny - 1], :] = lib.LBPS_NEUMANN
    two[10:20, 12] = lib.LBPS_VOID                        # void column ...
    two[10:20, 14] = lib.LBPS_VOID                        # ... and another one two points away
    two[9:21, 11] = lib.LBPS_NEUMANN
    two[9:21, 15] = lib.LBPS_NEUMANN
    two[9, 12:15] = lib.LBPS_NEUMANN
    two[20, 12:15] = lib.LBPS_NEUMANN
    two[10:20, 13] = lib.LBPS_NEUMANN                     # the column between the voids
    q = lib.lbps_params(nx, ny, 1.0, 1.0, 1.0, 1.0, 0.999, 0, 0, 0, 0, lib.LBPS_STORAGE_F16, 0, None)
    with pytest.raises(lib.LbpsError):
        lib.lbps_state_bytes_cells(q, two, None)


def test_checked_build_compiles():
    """The range-checked build (LBPS_CHECKED, the sanitizer stand-in the GPU
    tests run) compiles from the same sources (host-side cross-compilation,
    no GPU)."""
    from paper_2301_00228_gb300 import build as B

    lib = B.build(checked=True)
    assert lib.exists() and lib.name == "liblbps_checked.so"
