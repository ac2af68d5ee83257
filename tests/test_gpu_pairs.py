"""Two time steps per sweep (lbps_set_step_pairs) against single steps, in
every storage, on ragged rectangles with mixed edges, both readings of the
boundary rules, ramped loads, synchronisation points that split pairs, odd
step counts, and steps replayed from CUDA graphs of every block length.  The
populations and step counts must be the same bits: no population reads u
between synchronisations.  u and du/dt of the points 3 or more from the
edges, which the two-step kernel integrates over both steps in one composed
Newmark update (newmark2), must agree with two single updates up to
rounding; a synchronisation rebuilds the populations from u, so after one
they agree up to that rounding too.  Both agree with the FP64 oracle within
the storage's tolerance.  Lattices the sweep does not apply to (periodic
axes, a hole, sides under 16) keep single steps, bit for bit."""
import numpy as np
import pytest

import oracle as O
from paper_2301_00228_gb300 import workloads as W
from tolerance import TARGET

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("ux", "uy", "vx", "vy", "f_phi", "f_psi")


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def case(seed, nx, ny):
    rng = np.random.default_rng(seed)
    et = tuple(int(x) for x in rng.choice([1, 2], 4))
    ev = rng.uniform(-2e-4, 2e-4, 8)
    ux, uy = W.pulse_displacement(nx, ny, nx / 3, ny / 2, max(2.0, nx / 10), 1e-3, "dilatation")
    rx, ry = W.pulse_displacement(nx, ny, 2 * nx / 3, ny / 3, max(2.0, ny / 12), 1e-3, "rotation")
    vx = 1e-4 * rng.standard_normal((ny, nx))
    return dict(nx=nx, ny=ny, et=et, ev=ev, lam=float(rng.uniform(0.5, 4.0)), u=(ux + rx, uy + ry, vx, -vx))


def run(L, c, storage, steps, pairs, graph_k=32, feq=0, jmode=0, sync=0, load=False, chunks=None):
    lat = L.Lattice.rectangle(c["nx"], c["ny"], c["lam"], 1.0, c["et"], c["ev"], a0_phi=0.99, storage=storage,
                              bc_feq_mode=feq, bc_j_mode=jmode, sync_every=sync)
    L.lbps_set_step_pairs(lat._h, int(pairs))
    L.lbps_set_graph_steps(lat._h, graph_k)
    if load:
        lat.set_load(L.LBPS_NEUMANN, 20 * lat.dt, 45 * lat.dt)
        lat.set_load(L.LBPS_DIRICHLET, 15 * lat.dt)
    lat.init(*c["u"])
    for n in (chunks or [steps]):
        lat.step(n)
    out = {k: lat.read(k) for k in FIELDS}
    out["steps"] = lat.steps
    assert lat.check() == 0
    lat.close()
    return out


def assert_same(a, b, what, storage="f32", sync=False):
    """Step counts and (without synchronisation) populations bit for bit; the
    rest within the rounding of the composed update: relative to the
    field's largest magnitude 1e-12 for FP64 storage, where the update's
    acceleration sums are FP64, and 1e-7 where they are FP32 (one FP32
    rounding of 3 a0 + a1 and a0 + a1 per pair); 1e-4 for 16-bit storage
    after a synchronisation."""
    tol = 1e-12 if storage == "f64" else 1e-7
    if sync and storage in ("f16", "bf16", "bfp13"):
        # populations rebuilt from u are rounded to 16 bits: a difference of
        # u can move a rounding by one 16-bit step
        tol = 1e-4
    for k in a:
        if k == "steps" or (k.startswith("f_") and not sync):
            assert np.array_equal(a[k], b[k]), (what, k)
        else:
            scale = max(float(np.abs(b[k]).max()), 1e-300)
            err = float(np.abs(a[k] - b[k]).max()) / scale
            assert err <= tol, (what, k, err)


@pytest.mark.parametrize("storage", ["f32", "f64", "f16", "bf16", "bfp13"])
@pytest.mark.parametrize("size", [(16, 16), (37, 53), (67, 45), (131, 97), (256, 200)])
def test_pairs_equal_single_steps(L, storage, size):
    c = case(sum(size), *size)
    want = run(L, c, storage, 41, pairs=False)
    got = run(L, c, storage, 41, pairs=True)
    assert_same(got, want, (storage, size), storage)


@pytest.mark.parametrize("storage", ["f64", "f32", "bfp13"])
def test_pairs_against_oracle(L, storage):
    """Two steps per sweep against the FP64 oracle (rel-L2 per field, as the
    parity tests take it) within the storage's tolerance."""
    c = case(7, 131, 97)
    got = run(L, c, storage, 121, pairs=True)
    nt, bv = O.rect_bc(c["nx"], c["ny"], c["et"], c["ev"])
    ref = O.OracleLattice(c["nx"], c["ny"], c["lam"], 1.0, a0_phi=0.99, node_type=nt, bc_value=bv)
    ref = ref.init(*c["u"]).step(121).fields()
    for grp in (("ux", "uy"), ("vx", "vy")):
        gn = np.sqrt(sum(np.linalg.norm(ref[k]) ** 2 for k in grp))
        for k in grp:
            err = np.linalg.norm(got[k] - ref[k]) / max(np.linalg.norm(ref[k]), 1e-2 * gn)
            assert err <= TARGET[storage], (storage, k, err)


@pytest.mark.parametrize("variant", ["feq1", "jmode1", "sync7", "loads", "chunks", "graphs2", "graphs4", "nographs"])
def test_pairs_equal_single_steps_variants(L, variant):
    c = case(5, 83, 71)
    kw = {"feq1": dict(feq=1), "jmode1": dict(jmode=1), "sync7": dict(sync=7), "loads": dict(load=True),
          "chunks": dict(chunks=[1, 2, 3, 5, 8, 13, 21, 34]), "graphs2": dict(graph_k=2),
          "graphs4": dict(graph_k=4), "nographs": dict(chunks=[1] * 9 + [3] * 3)}[variant]
    for storage in ("f32", "f16", "bfp13"):
        want = run(L, c, storage, 87, pairs=False, **kw)
        got = run(L, c, storage, 87, pairs=True, **kw)
        assert_same(got, want, (variant, storage), storage, sync=variant == "sync7")


def test_pairs_fall_back_where_they_do_not_apply(L):
    # periodic axes, a side under 16, a plate with a hole: single steps, same bits
    lats = []
    for periodic, nx, ny in ((True, 40, 40), (False, 15, 40)):
        c = case(9, nx, ny)
        for pairs in (False, True):
            lat = L.Lattice.rectangle(nx, ny, 1.5, 1.0, c["et"], c["ev"], periodic_x=periodic, a0_phi=0.99)
            L.lbps_set_step_pairs(lat._h, int(pairs))
            lats.append(lat.init(*c["u"][:2]).step(30))
    d = W.hole_square(48, a0_phi=0.999, horizon=0.1, sync_every=0)
    ev = np.asarray(d.edge_value, float).ravel()
    nt, bv, cell = L.lbps_disk_cells(48, 48, 1.0, *d.hole, d.edge_type, ev)
    for pairs in (False, True):
        lat = L.Lattice(48, 48, d.lam, d.mu, a0_phi=d.a0_phi, node_type=nt, bc_value=bv, cell=cell)
        L.lbps_set_step_pairs(lat._h, int(pairs))
        u = W.pulse_displacement(48, 48, 12.0, 30.0, 3.0, 1e-3, "rotation")
        lats.append(lat.init(*(np.where(nt == 3, 0.0, a) for a in u)).step(30))
    for q in range(0, len(lats), 2):
        for k in FIELDS:
            assert np.array_equal(lats[q].read(k), lats[q + 1].read(k)), (q, k)
    for lat in lats:
        lat.close()


def test_pairs_toggled_midway_and_checkpoint(L):
    c = case(11, 97, 64)
    want = run(L, c, "f32", 60, pairs=False)
    lat = L.Lattice.rectangle(c["nx"], c["ny"], c["lam"], 1.0, c["et"], c["ev"], a0_phi=0.99)
    lat.init(*c["u"])
    L.lbps_set_step_pairs(lat._h, 1)
    lat.step(17)
    saved = lat.save_state()
    L.lbps_set_step_pairs(lat._h, 0)
    lat.step(20)
    L.lbps_set_step_pairs(lat._h, 1)
    lat.step(23)
    got = {k: lat.read(k) for k in FIELDS}
    got["steps"] = lat.steps
    assert_same(got, want, "toggled")
    lat.load_state(saved).step(43)       # resume from step 17 with pairs on
    again = {k: lat.read(k) for k in FIELDS}
    again["steps"] = lat.steps
    assert_same(again, want, "resumed")
    for bad in (-1, 2):
        with pytest.raises(L.LbpsError):
            L.lbps_set_step_pairs(lat._h, bad)
    lat.close()


def test_pairs_report_nonfinite(L):
    c = case(2, 64, 64)
    lat = L.Lattice.rectangle(64, 64, 1.0, 1.0, c["et"], c["ev"], a0_phi=0.99)
    L.lbps_set_step_pairs(lat._h, 1)
    ux, uy = c["u"][:2]
    lat.init(ux * 1e300, uy * 1e300)
    with pytest.raises(L.LbpsError) as e:
        lat.step(10)
    assert e.value.code == L.LBPS_ERR_NONFINITE
    lat.close()


@pytest.mark.parametrize("storage", ["f32", "bfp13"])
def test_pair_implementations_same_bits(L, storage):
    """A lattice below 2^25 points takes its pairs as a batch of itself; with
    per-kernel timing on it takes them through the two-step kernel and the
    frame chain on the second stream.  Both give the same bits."""
    c = case(13, 131, 97)
    out = []
    for timed in (False, True):
        lat = L.Lattice.rectangle(c["nx"], c["ny"], c["lam"], 1.0, c["et"], c["ev"], a0_phi=0.99, storage=storage)
        L.lbps_set_step_pairs(lat._h, 1)
        L.lbps_profile(lat._h, int(timed))
        lat.init(*c["u"]).step(9).step(32)
        out.append({k: lat.read(k) for k in FIELDS})
        assert lat.check() == 0 and lat.steps == 41
        lat.close()
    for k in FIELDS:
        assert np.array_equal(out[0][k], out[1][k]), k
