"""General geometry on the GPU (reading R14: void points, clipped boundary
cells, one-sided differences next to them, streaming into every interior
neighbour): the plate with a hole of Sec. 4 against the FP64 oracle, a
uniform-strain patch test around a hole, batches, explicit rectangle cells,
and rejected geometries, through the C ABI."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2301_00228_gb300 import workloads as W
from tolerance import TARGET as TOL
from tolerance import judge

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("ux", "uy", "phi", "psi")


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def rel(got, ref, body):
    out = {}
    for grp in (("ux", "uy"), ("phi", "psi")):
        gn = math.sqrt(sum(np.linalg.norm(ref[k][body]) ** 2 for k in grp))
        for k in grp:
            den = max(np.linalg.norm(ref[k][body]), 1e-2 * gn, 1e-300)
            out[k] = float(np.linalg.norm((got[k] - ref[k])[body]) / den)
    return out


def gpu(L, n, d, nt, bv, cell, storage, sync=None):
    lat = L.Lattice(n, n, d.lam, d.mu, a0_phi=d.a0_phi, node_type=nt, bc_value=bv, cell=cell,
                    sync_every=d.sync_every if sync is None else sync, storage=storage)
    for kind, t_ramp, t_hold in d.loads:
        lat.set_load(kind, t_ramp, t_hold)
    return lat


def plate(L, d, n):
    """The plate's node types and cells, built by the library and, separately,
    by the oracle (the two must classify every point alike)."""
    ev = np.asarray(d.edge_value, float).ravel()
    lib = L.lbps_disk_cells(n, n, 1.0, *d.hole, d.edge_type, ev)
    ora = O.disk_cells(n, n, *d.hole, d.edge_type, ev)
    assert np.array_equal(lib[0], ora[0])
    return lib, ora


@pytest.fixture(scope="module")
def hole_case(L):
    n = 40
    d = W.hole_square(n, a0_phi=0.9999, horizon=0.4)
    (nt, bv, cell), (ont, obv, ocell) = plate(L, d, n)
    ref = O.OracleLattice(n, n, d.lam, d.mu, a0_phi=d.a0_phi, node_type=ont, bc_value=obv, cell=ocell,
                          sync_every=d.sync_every)
    for kind, t_ramp, t_hold in d.loads:
        ref.set_load(kind, t_ramp, t_hold)
    z = np.zeros((n, n))
    ref.init(z, z).step(d.steps)
    return n, d, nt, bv, cell, ref.fields()


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bfp13"])
def test_plate_with_hole_against_oracle(L, hole_case, storage):
    """The Sec. 4 plate with a hole (tension ramp, synchronised every 50
    steps) over 0.4 L/c_s, in uneven step chunks."""
    n, d, nt, bv, cell, ref = hole_case
    lat = gpu(L, n, d, nt, bv, cell, storage)
    z = np.zeros((n, n))
    lat.init(z, z)
    for chunk in (1, 49, 50, 777):
        lat.step(chunk)
    lat.step(d.steps - 877)
    got = {k: lat.read(k) for k in FIELDS}
    body = nt != 3
    errs = rel(got, ref, body)
    for k in FIELDS:
        assert np.abs(got[k][~body]).max() == 0.0, k          # void points hold nothing
    assert np.abs(ref["uy"]).max() > 1e-4
    judge(errs, storage, "plate with a hole")


def test_patch_uniform_strain_around_hole(L):
    """A uniform strain around a hole, every boundary cell loaded by the
    traction of the uniform stress (closure of the cell boundary), stays
    static on the GPU as in the oracle."""
    nx, ny, lam, mu = 33, 29, 1.3, 1.0
    nt, _, cell = L.lbps_disk_cells(nx, ny, 1.0, 15.6, 13.8, 4.6, (1, 1, 1, 1), np.zeros(8))
    exx, eyy, exy = 2e-4, -1e-4, 0.5e-4
    sxx, syy, sxy = lam * (exx + eyy) + 2 * mu * exx, lam * (exx + eyy) + 2 * mu * eyy, 2 * mu * exy
    fx = np.zeros((ny, nx))
    fy = np.zeros((ny, nx))
    for q, (ex, ey) in enumerate(((1, 0), (0, 1), (-1, 0), (0, -1))):
        fx -= (sxx * ex + sxy * ey) * cell[..., 1 + q]
        fy -= (sxy * ex + syy * ey) * cell[..., 1 + q]
    bv = np.stack([fx, fy], -1)
    bv[nt != 1] = 0.0
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    body = nt != 3
    ux, uy = (exx * X + exy * Y) * body, (exy * X + eyy * Y) * body
    lat = L.Lattice(nx, ny, lam, mu, a0_phi=0.99, node_type=nt, bc_value=bv, cell=cell, storage="f64")
    lat.init(ux, uy).step(300)
    assert np.abs(lat.read("ux") - ux)[body].max() <= 1e-13
    assert np.abs(lat.read("uy") - uy)[body].max() <= 1e-13


def test_explicit_rectangle_cells(L):
    """A rectangle given as general geometry (explicit cells of the clipped
    squares) runs the general boundary code and agrees with the rectangle
    path to round-off."""
    nx, ny = 47, 39
    ev = np.array([1e-4, -2e-4, 0, 3e-4, -1e-4, 0, 2e-4, 1e-4])
    et = (1, 2, 1, 1)
    nt, bv, cell = L.lbps_disk_cells(nx, ny, 1.0, -50.0, -50.0, 1.0, et, ev)
    ux, uy = W.pulse_displacement(nx, ny, 20.0, 17.0, 3.0, 1e-3, "rotation")
    a = L.Lattice.rectangle(nx, ny, 1.2, 1.0, et, ev, a0_phi=0.99, storage="f64").init(ux, uy).step(120)
    b = L.Lattice(nx, ny, 1.2, 1.0, a0_phi=0.99, node_type=nt, bc_value=bv, cell=cell, storage="f64")
    b.init(ux, uy).step(120)
    for k in FIELDS:
        x, y = a.read(k), b.read(k)
        assert np.abs(x - y).max() <= 1e-13 * np.abs(x).max(), k


def test_batch_with_holes_equals_single(L):
    shapes = [(40, 0.9999), (33, 0.9999), (51, 0.9999)]
    lats, solo = [], []
    for n, a0 in shapes:
        d = W.hole_square(n, a0_phi=a0, horizon=0.05, sync_every=0)
        nt, bv, cell = L.lbps_disk_cells(n, n, 1.0, *d.hole, d.edge_type, np.asarray(d.edge_value, float).ravel())
        z = np.zeros((n, n))
        one = gpu(L, n, d, nt, bv, cell, "f32").init(z, z).step(211)
        solo.append({k: one.read(k) for k in FIELDS})
        lats.append(gpu(L, n, d, nt, bv, cell, "f32").init(z, z))
    rect = L.Lattice.rectangle(30, 28, 1.0, 1.0, (1, 2, 1, 1), np.zeros(8), a0_phi=0.99)
    rect.init(*W.pulse_displacement(30, 28, 14.0, 12.0, 3.0, 1e-3, "dilatation"))
    b = L.Batch(lats + [rect])
    b.tune(repeats=2)
    b.step(100).step(111)
    assert b.check() == 0
    for q, (lat, want) in enumerate(zip(lats, solo)):
        for k in FIELDS:
            assert np.array_equal(lat.read(k), want[k]), (q, k)
    b.close()


def test_invalid_geometry_rejected(L):
    nx, ny = 30, 28
    nt, bv, cell = L.lbps_disk_cells(nx, ny, 1.0, 14.0, 13.0, 5.0, (1, 1, 1, 1), np.zeros(8))
    bad = nt.copy()
    bad[:, 2] = L.LBPS_VOID           # column 1 left without a stencil along x
    bad[:, 3] = L.LBPS_NEUMANN
    for nt_bad, cl in ((bad, None), (np.where(nt == 1, 0, nt).astype(np.uint8), cell)):
        with pytest.raises(L.LbpsError) as e:
            L.Lattice(nx, ny, 1.0, 1.0, node_type=nt_bad, bc_value=bv, cell=cl)
        assert e.value.code == L.LBPS_ERR_INVALID


def test_hole_rows_skipped_same_bits(L):
    """Warps whose rows lie inside the hole return without loading them. With
    8-row chunks many do; every launch shape must give the same bits, and the
    oracle's result within tolerance."""
    n = 96
    d = W.hole_square(n, a0_phi=0.99, horizon=0.2, sync_every=0)
    (nt, bv, cell), (ont, obv, ocell) = plate(L, d, n)
    ux, uy = W.pulse_displacement(n, n, 20.0, 30.0, 5.0, 1e-3, "dilatation")
    body = nt != 3
    ux, uy = ux * body, uy * body
    ref = O.OracleLattice(n, n, d.lam, d.mu, a0_phi=d.a0_phi, node_type=ont, bc_value=obv, cell=ocell)
    want = ref.init(ux, uy).step(150).fields()
    first = None
    for variant in range(8):
        for rows in (8, 16, 64):
            lat = L.Lattice(n, n, d.lam, d.mu, a0_phi=d.a0_phi, node_type=nt, bc_value=bv, cell=cell,
                            storage="f32")
            L.lbps_set_tuning(lat._h, variant, rows)
            got = lat.init(ux, uy).step(150).fields()
            if first is None:
                first = got
                errs = rel(got, want, body)
                assert all(v <= TOL["f32"] for v in errs.values()), errs
            else:
                for k in FIELDS:
                    assert np.array_equal(got[k], first[k]), (variant, rows, k)
            lat.close()
