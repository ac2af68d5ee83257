"""Seeded random parity cases, GPU against the FP64 oracle through the C ABI:
random sizes (ragged against the 30-column strips and 32-row chunks),
periodic axes, edge types and values, holes of random size and position,
material, a_0, both Eq. LBE_mod readings, synchronisation, ramped loads and
every storage.  Each case is small enough for the oracle to finish in a
fraction of a second."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2301_00228_gb300 import workloads as W
from tolerance import judge

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

N_CASES = 40


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def make_case(seed):
    rng = np.random.default_rng(1000 + seed)
    nx, ny = (int(v) for v in rng.integers(12, 90, 2))
    px, py = bool(rng.random() < 0.2), bool(rng.random() < 0.2)
    et = tuple(int(x) for x in rng.choice([1, 2], 4))
    ev = rng.uniform(-2e-4, 2e-4, 8)
    hole = (not px and not py and min(nx, ny) >= 24 and rng.random() < 0.5)
    storage = str(rng.choice(["f64", "f32", "f16", "bf16", "bfp13"]))
    case = dict(nx=nx, ny=ny, px=px, py=py, et=et, ev=ev, lam=float(rng.uniform(0.5, 3.0)),
                mu=float(rng.uniform(0.7, 1.5)), rho=float(rng.uniform(0.8, 1.6)),
                a0=float(rng.choice([0.99, 0.999])), mode=int(rng.integers(0, 2)),
                sync=int(rng.choice([0, 0, 13])), storage=storage, steps=int(rng.integers(20, 160)),
                ramp=bool(rng.random() < 0.3), cell=None, jmode=int(seed % 3 == 2))
    if hole:
        from paper_2301_00228_gb300 import lbps

        r = float(rng.uniform(2.5, min(nx, ny) / 5))
        cx = float(rng.uniform(r + 4, nx - 1 - r - 4))
        cy = float(rng.uniform(r + 4, ny - 1 - r - 4))
        # each side builds the plate's node types and cells itself
        nt, bv, cell = lbps.lbps_disk_cells(nx, ny, 1.0, cx, cy, r, et, ev)
        case.update(nt=nt, bv=bv, cell=cell, ora=O.disk_cells(nx, ny, cx, cy, r, et, ev))
    else:
        nt, bv = O.rect_bc(nx, ny, et, ev, periodic_x=px, periodic_y=py)
        case.update(nt=nt, bv=bv, ora=(nt, bv, None))
    body = case["nt"] != 3
    ux, uy = W.pulse_displacement(nx, ny, float(rng.uniform(0, nx - 1)), float(rng.uniform(0, ny - 1)),
                                  float(rng.uniform(2.0, max(2.5, min(nx, ny) / 5))), 1e-3,
                                  "dilatation" if rng.random() < 0.5 else "rotation")
    case.update(ux=ux * body, uy=uy * body)
    return case


def rel(got, ref, body):
    out = {}
    for grp in (("ux", "uy"), ("phi", "psi")):
        gn = math.sqrt(sum(np.linalg.norm(ref[k][body]) ** 2 for k in grp))
        for k in grp:
            den = max(np.linalg.norm(ref[k][body]), 1e-2 * gn, 1e-300)
            out[k] = float(np.linalg.norm((got[k] - ref[k])[body]) / den)
    return out


@pytest.mark.parametrize("seed", range(N_CASES))
def test_random_case(L, seed):
    c = make_case(seed)
    kw = dict(a0_phi=c["a0"], periodic_x=c["px"], periodic_y=c["py"], bc_feq_mode=c["mode"], bc_j_mode=c["jmode"],
              sync_every=c["sync"])
    ont, obv, ocell = c["ora"]
    assert np.array_equal(ont, c["nt"])
    ref = O.OracleLattice(c["nx"], c["ny"], c["lam"], c["mu"], c["rho"], node_type=ont, bc_value=obv, cell=ocell,
                          **kw)
    lat = L.Lattice(c["nx"], c["ny"], c["lam"], c["mu"], c["rho"], storage=c["storage"], node_type=c["nt"],
                    bc_value=c["bv"], cell=c["cell"], **kw)
    if c["ramp"]:
        ref.set_load(1, 30 * ref.dt, 60 * ref.dt)
        ref.set_load(2, 40 * ref.dt)
        lat.set_load(L.LBPS_NEUMANN, 30 * lat.dt, 60 * lat.dt)
        lat.set_load(L.LBPS_DIRICHLET, 40 * lat.dt)
    want = ref.init(c["ux"], c["uy"]).step(c["steps"]).fields()
    lat.init(c["ux"], c["uy"])
    half = c["steps"] // 2
    lat.step(half).step(c["steps"] - half)
    got = lat.fields()
    body = c["nt"] != 3
    errs = rel(got, want, body)
    lat.close()
    judge(errs, c["storage"], (seed, c["nx"], c["ny"]))
