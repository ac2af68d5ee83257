"""Energy densities and lbps_energy (FP64 reductions on the device) against
the oracle's energy densities (pinned by closed forms in test_oracle_pins):
point by point after many steps, on rectangles in every storage and on a
plate with a hole, and the summed energy against the oracle's sum."""
import numpy as np
import pytest

import oracle as O
from paper_2301_00228_gb300 import workloads as W
from tolerance import TARGET as TOL
from tolerance import judge

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def rect_case(seed=3, nx=61, ny=47):
    rng = np.random.default_rng(seed)
    et = (2, 1, 1, 2)
    ev = rng.uniform(-1e-4, 1e-4, 8)
    ux, uy = W.pulse_displacement(nx, ny, 25.0, 20.0, 4.0, 1e-3, "dilatation")
    rx, ry = W.pulse_displacement(nx, ny, 40.0, 30.0, 3.0, 1e-3, "rotation")
    return dict(nx=nx, ny=ny, lam=1.9, mu=1.0, rho=1.2, et=et, ev=ev, u=(ux + rx, uy + ry))


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16", "bfp13"])
def test_energy_matches_oracle(L, storage):
    c = rect_case()
    steps = 150
    lat = L.Lattice.rectangle(c["nx"], c["ny"], c["lam"], c["mu"], c["et"], c["ev"], rho=c["rho"], a0_phi=0.99,
                              storage=storage)
    lat.init(*c["u"]).step(steps)
    nt, bv = O.rect_bc(c["nx"], c["ny"], c["et"], c["ev"])
    ref = O.OracleLattice(c["nx"], c["ny"], c["lam"], c["mu"], c["rho"], a0_phi=0.99, node_type=nt, bc_value=bv)
    ref.init(*c["u"]).step(steps)
    want = {"kinetic_energy": ref.read(O.EKIN), "strain_energy": ref.read(O.ESTRAIN)}
    got = {k: lat.read(k) for k in want}
    e = lat.energy()
    lat.close()
    for q, k in enumerate(want):
        assert want[k].sum() > 0
        # the device's FP64 sum equals the host sum of the device's own densities
        assert abs(e[q] - got[k].sum()) <= 1e-12 * got[k].sum()
    assert e[2] == e[0] + e[1]
    # the densities are quadratic in the fields: their relative error is about
    # twice that of the fields, so half of it is held to the fields' tolerance
    errs = {k: rel(got[k], want[k]) / 2 for k in want}
    if storage in ("f16", "bf16", "bfp13"):
        judge(errs, storage, "energy densities")
    else:
        assert all(v <= TOL[storage] for v in errs.values()), errs
        for q, k in enumerate(want):
            assert abs(e[q] - want[k].sum()) <= 2 * TOL[storage] * want[k].sum(), k


def test_energy_hole_plate(L):
    n = 48
    d = W.hole_square(n, a0_phi=0.999, horizon=0.1, sync_every=50)
    ev = np.asarray(d.edge_value, float).ravel()
    nt, bv, cell = L.lbps_disk_cells(n, n, 1.0, *d.hole, d.edge_type, ev)
    ont, obv, ocell = O.disk_cells(n, n, *d.hole, d.edge_type, ev)
    u = W.pulse_displacement(n, n, 12.0, 30.0, 3.0, 1e-3, "rotation")
    u = tuple(np.where(nt == 3, 0.0, a) for a in u)
    steps = 200
    lat = L.Lattice(n, n, d.lam, d.mu, a0_phi=d.a0_phi, node_type=nt, bc_value=bv, cell=cell, storage="f64",
                    sync_every=d.sync_every)
    for kind, t_ramp, t_hold in d.loads:
        lat.set_load(kind, t_ramp, t_hold)
    lat.init(*u).step(steps)
    ref = O.OracleLattice(n, n, d.lam, d.mu, a0_phi=d.a0_phi, node_type=ont, bc_value=obv, cell=ocell,
                          sync_every=d.sync_every)
    for kind, t_ramp, t_hold in d.loads:
        ref.set_load(kind, t_ramp, t_hold)
    ref.init(*u).step(steps)
    for fid, k in ((O.EKIN, "kinetic_energy"), (O.ESTRAIN, "strain_energy")):
        want, got = ref.read(fid), lat.read(k)
        assert rel(got, want) <= 1e-10, k
        assert np.all(got[nt == 3] == 0.0)
    e = lat.energy()
    assert abs(e[1] - ref.read(O.ESTRAIN).sum()) <= 1e-10 * e[1]
    lat.close()


def test_energy_call_order(L):
    lat = L.Lattice.rectangle(20, 20, 1.0, 1.0, (1, 1, 1, 1), np.zeros(8))
    with pytest.raises(L.LbpsError) as e:
        lat.energy()
    assert e.value.code == L.LBPS_ERR_STATE
    lat.init(*W.pulse_displacement(20, 20, 10.0, 10.0, 3.0, 1e-3, "dilatation"))
    k0, s0, t0 = lat.energy()
    assert k0 == 0.0 and s0 > 0 and t0 == s0     # initial state at rest
    lat.close()
