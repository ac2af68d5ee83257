"""Time-dependent boundary data (Sec. 4 tension and shear examples) on the
GPU against the FP64 oracle, through the C ABI: the ramp-then-hold factor on
Neumann forces and Dirichlet targets, the device step counter across
lbps_step calls, batches and the autotuner."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2301_00228_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from tolerance import judge
FIELDS = ("ux", "uy", "phi", "psi")


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def rel(got, ref):
    out = {}
    for g in (("ux", "uy"), ("phi", "psi")):
        gn = math.sqrt(sum(np.linalg.norm(ref[k]) ** 2 for k in g))
        for k in g:
            out[k] = float(np.linalg.norm(got[k] - ref[k]) / max(np.linalg.norm(ref[k]), 1e-2 * gn, 1e-300))
    return out


def oracle_run(d, steps):
    nt, bv = O.rect_bc(d.nx, d.ny, d.edge_type, np.asarray(d.edge_value, float).ravel())
    ref = O.OracleLattice(d.nx, d.ny, d.lam, d.mu, a0_phi=d.a0_phi, node_type=nt, bc_value=bv,
                          sync_every=d.sync_every)
    for kind, t_ramp, t_hold in d.loads:
        ref.set_load(kind, t_ramp, t_hold)
    ux, uy = d.displacement()
    return ref.init(ux, uy).step(steps).fields()


def gpu_lattice(L, d, storage):
    lat = L.Lattice.rectangle(d.nx, d.ny, d.lam, d.mu, d.edge_type, np.asarray(d.edge_value, float).ravel(),
                              a0_phi=d.a0_phi, sync_every=d.sync_every, storage=storage)
    for kind, t_ramp, t_hold in d.loads:
        lat.set_load(kind, t_ramp, t_hold)
    return lat.init(*d.displacement())


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bfp13"])
@pytest.mark.parametrize("example", ["tension", "shear"])
def test_paper_examples_against_oracle(L, example, storage):
    """The tension (ramp to 0.005 mu at L/c_s, then held) and shear (ramp
    without end, clamped bottom) squares, synchronised every 50 steps, at
    a0 = 0.999 over 1.3 L/c_s, so the ramp, the hold and the synchronisation
    all happen; the steps are taken in uneven chunks."""
    mk = W.tension_square if example == "tension" else W.shear_square
    d = mk(24, a0_phi=0.999, horizon=1.3)
    ref = oracle_run(d, d.steps)
    lat = gpu_lattice(L, d, storage)
    done = 0
    for chunk in (1, 7, 50, 333):
        lat.step(chunk)
        done += chunk
    lat.step(d.steps - done)
    errs = rel({k: lat.read(k) for k in FIELDS}, ref)
    judge(errs, storage, example)
    assert np.abs(ref["uy" if example == "tension" else "ux"]).max() > 1e-4   # the load did act


def test_dirichlet_ramp_lands_on_target(L):
    """A Dirichlet edge with a ramped target: after step n the edge points sit
    at s(t_n) u*, exactly (Eq. acc_dirichlet lands u on the target)."""
    d = W.Domain(20, 16, 1.5, 1.0, a0_phi=0.99, edge_type=(2, 1, 1, 1),
                 edge_value=((2e-4, -1e-4), (0, 0), (0, 0), (0, 0)))
    lat = gpu_lattice(L, d, "f64")
    dt = lat.dt
    lat.set_load(L.LBPS_DIRICHLET, 40 * dt, 25 * dt)
    for n in (1, 10, 25, 40):
        lat.step(n - lat.steps)
        s = min(n, 25) / 40.0
        ux, uy = lat.read("ux"), lat.read("uy")
        assert np.allclose(ux[0, 1:-1], s * 2e-4, rtol=0, atol=1e-18), n
        assert np.allclose(uy[0, 1:-1], -s * 1e-4, rtol=0, atol=1e-18), n


def test_batch_with_ramps_equals_single(L):
    """Lattices with ramped data in a batch (graphs, the autotuner's repeated
    trial steps, single steps in between) end bit-identical to stepping them
    alone: the step counter that times the data is restored after tuning."""
    ds = [W.tension_square(30, a0_phi=0.99, horizon=0.2), W.shear_square(26, a0_phi=0.99, horizon=0.2),
          W.tension_square(41, a0_phi=0.999, horizon=0.1)]
    for d in ds:
        d.sync_every = 0
    steps = 157
    solo = []
    for d in ds:
        lat = gpu_lattice(L, d, "f32").step(steps)
        solo.append({k: lat.read(k) for k in FIELDS})
    lats = [gpu_lattice(L, d, "f32") for d in ds]
    b = L.Batch(lats)
    b.tune(repeats=2)
    b.step(40)
    lats[1].step(3)
    b.step(60)
    lats[1].step(steps - 103)
    lats[0].step(steps - 100)
    lats[2].step(steps - 100)
    for q, (lat, want) in enumerate(zip(lats, solo)):
        assert lat.steps == steps
        for k in FIELDS:
            assert np.array_equal(lat.read(k), want[k]), (q, k)
    b.close()


def test_set_load_rejects(L):
    d = W.tension_square(12)
    lat = gpu_lattice(L, d, "f32")
    for bad in ((0, 1.0, 1.0), (3, 1.0, 1.0), (1, -1.0, 1.0), (1, math.inf, 1.0), (1, 1.0, 0.0)):
        with pytest.raises(L.LbpsError) as e:
            lat.set_load(*bad)
        assert e.value.code == L.LBPS_ERR_INVALID
    lat.set_load(L.LBPS_NEUMANN, 0.0)   # constant data again
