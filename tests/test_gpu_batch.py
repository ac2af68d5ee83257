"""Batches: many lattices advanced by one launch per kernel per step.

Every lattice of a batch must end bit-for-bit where it ends when stepped on
its own (same per-point arithmetic), whatever the mix, the step counts, the
launch shape or interleaved single steps; and agree with the FP64 oracle."""
import numpy as np
import pytest

import oracle as O
from paper_2301_00228_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def domains(seed, count, lo=3, hi=150, periodic=True):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(count):
        nx, ny = (int(v) for v in rng.integers(lo, hi + 1, 2))
        px = bool(periodic and q % 5 == 3)
        py = bool(periodic and q % 7 == 5)
        et = tuple(int(x) for x in rng.choice([1, 2], 4))
        ev = rng.uniform(-2e-4, 2e-4, 8)
        lam = float(rng.uniform(0.5, 4.0))
        a0 = float(rng.choice([0.99, 0.9999]))
        kind = "dilatation" if q % 2 else "rotation"
        ux, uy = W.pulse_displacement(nx, ny, float(rng.uniform(0, nx - 1)), float(rng.uniform(0, ny - 1)),
                                      max(1.5, min(nx, ny) / 6), 1e-3, kind)
        out.append(dict(nx=nx, ny=ny, px=px, py=py, et=et, ev=ev, lam=lam, a0=a0, ux=ux, uy=uy))
    return out


def make(L, d, storage):
    lat = L.Lattice.rectangle(d["nx"], d["ny"], d["lam"], 1.0, d["et"], d["ev"], periodic_x=d["px"],
                              periodic_y=d["py"], a0_phi=d["a0"], storage=storage)
    return lat.init(d["ux"], d["uy"])


def assert_same(a, b, what):
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), (what, k)


@pytest.mark.parametrize("storage", ["f32", "f64", "bf16", "f16", "bfp13"])
def test_batch_equals_single(L, storage):
    ds = domains(7, 14, lo=3 if storage in ("f32", "f64") else 4)
    solo = [make(L, d, storage).step(37) for d in ds]
    lats = [make(L, d, storage) for d in ds]
    b = L.Batch(lats)
    b.step(10).step(27)
    assert b.check() == 0
    for q, (x, y) in enumerate(zip(lats, solo)):
        assert x.steps == 37
        assert_same(x, y, (storage, q))
    b.close()


def test_batch_tuning_and_interleaved_single_steps(L):
    ds = domains(8, 9, lo=20, hi=120)
    solo = [make(L, d, "f32").step(30) for d in ds]
    lats = [make(L, d, "f32") for d in ds]
    b = L.Batch(lats)
    v, r, ms = b.tune(repeats=2)
    assert v in (0, 1, 2, 4, 5, 6) and r in (8, 16, 32, 64, 128) and ms > 0
    assert b.graph_steps in (2, 4, 8, 16, 32)
    b.step(9)
    lats[2].step(1)        # one lattice stepped on its own in between
    lats[5].step(2)
    b.step(5)
    lats[2].step(15)       # catch up to 30 steps for every lattice
    lats[5].step(14)
    for q in (0, 1, 3, 4, 6, 7, 8):
        lats[q].step(16)
    for q, (x, y) in enumerate(zip(lats, solo)):
        assert x.steps == 30
        assert_same(x, y, q)
    for variant in range(3):
        b.set_tuning(variant, 8)
    b.close()


@pytest.mark.parametrize("storage", ["f32", "f64", "f16", "bfp13"])
def test_batch_every_launch_shape_same_bits(L, storage):
    """Every launch shape, with short and long row chunks: the same bits as
    the lattices stepped on their own."""
    ds = domains(11, 6, lo=5, hi=90)
    solo = [make(L, d, storage).step(21) for d in ds]
    for variant in range(8):
        for rows in (8, 40):
            lats = [make(L, d, storage) for d in ds]
            b = L.Batch(lats)
            b.set_tuning(variant, rows)
            b.step(21)
            assert b.check() == 0
            for q, (x, y) in enumerate(zip(lats, solo)):
                assert_same(x, y, (storage, variant, rows, q))
            b.close()
            for x in lats:
                x.close()


def test_batch_against_oracle(L):
    ds = domains(9, 5, lo=12, hi=60, periodic=False)
    lats = [make(L, d, "f64") for d in ds]
    b = L.Batch(lats)
    b.step(41)
    for d, lat in zip(ds, lats):
        nt, bv = O.rect_bc(d["nx"], d["ny"], d["et"], d["ev"])
        ref = O.OracleLattice(d["nx"], d["ny"], d["lam"], 1.0, a0_phi=d["a0"], node_type=nt, bc_value=bv)
        ref.init(d["ux"], d["uy"]).step(41)
        got, want = lat.fields(), ref.fields()
        for k in ("ux", "uy", "phi", "psi"):
            scale = max(np.abs(want["ux"]).max(), np.abs(want["uy"]).max()) if k[0] == "u" else \
                max(np.abs(want["phi"]).max(), np.abs(want["psi"]).max())
            assert np.abs(got[k] - want[k]).max() <= 1e-10 * scale, k
    b.close()


def test_batch_fp32_mixed_recipe_against_oracle(L):
    """The batching workload's recipe (random edges and values in
    U(-1e-3, 1e-3), lambda/mu in U(0.5, 4), a sigma = 4 pulse at a random
    point), scaled to sides 64..160 so the oracle finishes: FP32 storage,
    autotuned shape and graphs, 400 steps, every domain within the FP32
    tolerance (relative L2 per field, 1e-5) of the FP64 oracle."""
    def rel_errors(got, ref):
        # relative L2 per field against max(|ref|, 1e-2 |group|), groups (u), (v), (phi, psi)
        out = {}
        for g in (("ux", "uy"), ("vx", "vy"), ("phi", "psi")):
            gn = np.sqrt(sum(np.linalg.norm(ref[k]) ** 2 for k in g))
            for k in g:
                out[k] = float(np.linalg.norm(got[k] - ref[k]) / max(np.linalg.norm(ref[k]), 1e-2 * gn, 1e-300))
        return out

    ds = W.mixed_batch(count=6, seed=17, side_lo=64, side_hi=160)
    lats = [L.Lattice.rectangle(d.nx, d.ny, d.lam, d.mu, d.edge_type, np.asarray(d.edge_value, float).ravel(),
                                a0_phi=d.a0_phi, storage="f32").init(*d.displacement()) for d in ds]
    b = L.Batch(lats)
    b.tune(repeats=1)
    b.step(400)
    assert b.check() == 0
    for q, (d, lat) in enumerate(zip(ds, lats)):
        nt, bv = O.rect_bc(d.nx, d.ny, d.edge_type, np.asarray(d.edge_value, float).ravel())
        ref = O.OracleLattice(d.nx, d.ny, d.lam, d.mu, a0_phi=d.a0_phi, node_type=nt, bc_value=bv)
        ref.init(*d.displacement()).step(400)
        errs = rel_errors(lat.fields(), ref.fields())
        assert max(errs.values()) <= 1e-5, (q, errs)
    b.close()


def test_batch_rejects_and_reports(L):
    ds = domains(10, 3, lo=10, hi=30, periodic=False)
    a, c = make(L, ds[0], "f32"), make(L, ds[1], "f64")
    with pytest.raises(L.LbpsError):
        L.Batch([a, c])                       # mixed storage
    with pytest.raises(L.LbpsError):
        L.Batch([a, a])                       # the same lattice twice
    s = L.Lattice.rectangle(10, 10, 1.0, 1.0, (1, 1, 1, 1), np.zeros(8), sync_every=5).init(
        np.zeros((10, 10)), np.zeros((10, 10)))
    with pytest.raises(L.LbpsError):
        L.Batch([a, s])                       # synchronisation is per lattice only
    u = L.Lattice.rectangle(10, 10, 1.0, 1.0, (1, 1, 1, 1), np.zeros(8))
    with pytest.raises(L.LbpsError) as e:
        L.Batch([u])                          # not initialised
    assert e.value.code == L.LBPS_ERR_STATE
    big = np.full((ds[2]["ny"], ds[2]["nx"]), 1e300)
    bad = L.Lattice.rectangle(ds[2]["nx"], ds[2]["ny"], 1.0, 1.0, (1, 2, 1, 1), np.zeros(8)).init(big, 0 * big)
    b = L.Batch([a, bad])
    b.step(3)
    assert b.check() == L.LBPS_ERR_NONFINITE
    assert a.check() == 0
    b.close()


@pytest.mark.parametrize("k", [4, 8, 32])
def test_batch_graph_steps_same_bits(L, k):
    """Blocks of k steps per graph, then pairs, then an odd step: the same bits
    as stepping alone, for step counts around and below k."""
    ds = domains(12, 5, lo=6, hi=70)
    for n in (1, k - 1, k, 2 * k + 3):
        solo = [make(L, d, "f32").step(n) for d in ds]
        lats = [make(L, d, "f32") for d in ds]
        b = L.Batch(lats)
        b.set_graph_steps(k)
        assert b.graph_steps == k
        b.step(n)
        assert b.check() == 0
        for q, (x, y) in enumerate(zip(lats, solo)):
            assert x.steps == n
            assert_same(x, y, (k, n, q))
        b.close()
    b = L.Batch([make(L, ds[0], "f32")])
    for bad in (0, 3, 66, -2):
        with pytest.raises(L.LbpsError):
            b.set_graph_steps(bad)
    b.close()


@pytest.mark.parametrize("storage", ["f32", "f64", "f16", "bfp13"])
def test_batch_pairs_equal_lattices_alone(L, storage):
    """Two steps per sweep in the batch: every lattice ends with the same bits
    as the same lattice taking two steps per sweep on its own, over an odd
    step count in chunks (pairs, then a single step), and single steps taken
    again after turning the mode off continue alike."""
    ds = domains(17, 12, lo=16, hi=150, periodic=False)
    solo = []
    for d in ds:
        lat = make(L, d, storage)
        L.lbps_set_step_pairs(lat._h, 1)
        solo.append(lat.step(10).step(27))
    lats = [make(L, d, storage) for d in ds]
    b = L.Batch(lats)
    assert not b.step_pairs
    b.set_step_pairs(True)
    assert b.step_pairs
    b.step(10).step(27)
    assert b.check() == 0
    for q, (x, y) in enumerate(zip(lats, solo)):
        assert x.steps == 37
        assert_same(x, y, (storage, q))
    b.set_step_pairs(False)
    b.step(5)
    for y in solo:
        L.lbps_set_step_pairs(y._h, 0)
        y.step(5)
    for q, (x, y) in enumerate(zip(lats, solo)):
        assert_same(x, y, ("single after pairs", storage, q))
    b.close()


def test_batch_pairs_against_single_steps_and_oracle(L):
    """Against the batch's single steps: populations the same bits, u and
    du/dt within the rounding of the composed update; and against the FP64
    oracle within the FP32 tolerance."""
    ds = domains(23, 6, lo=16, hi=90, periodic=False)
    one = [make(L, d, "f32") for d in ds]
    two = [make(L, d, "f32") for d in ds]
    b1, b2 = L.Batch(one), L.Batch(two)
    b2.set_step_pairs(True)
    b1.step(40)
    b2.step(40)
    for q, (x, y) in enumerate(zip(two, one)):
        fx, fy = x.fields(), y.fields()
        for k in fx:
            if k in ("f_phi", "f_psi", "phi", "psi"):
                assert np.array_equal(fx[k], fy[k]), (q, k)
            else:
                scale = max(float(np.abs(fy[k]).max()), 1e-300)
                assert float(np.abs(fx[k] - fy[k]).max()) <= 1e-7 * scale, (q, k)
        d = ds[q]
        nt, bv = O.rect_bc(d["nx"], d["ny"], d["et"], d["ev"])
        ref = O.OracleLattice(d["nx"], d["ny"], d["lam"], 1.0, a0_phi=d["a0"], node_type=nt, bc_value=bv)
        ref = ref.init(d["ux"], d["uy"]).step(40).fields()
        for grp in (("ux", "uy"), ("phi", "psi")):
            gn = np.sqrt(sum(np.linalg.norm(ref[k]) ** 2 for k in grp))
            for k in grp:
                err = np.linalg.norm(fx[k] - ref[k]) / max(np.linalg.norm(ref[k]), 1e-2 * gn)
                assert err <= 1e-5, (q, k, err)
    b1.close()
    b2.close()


def test_batch_pairs_rejected_where_they_do_not_apply(L):
    """A periodic lattice or one under 16 points a side: LBPS_ERR_INVALID, the
    batch keeps single steps."""
    for d in (dict(domains(3, 1, lo=20, hi=40, periodic=False)[0], px=True),
              dict(domains(4, 1, lo=10, hi=12, periodic=False)[0])):
        good = make(L, domains(5, 1, lo=20, hi=40, periodic=False)[0], "f32")
        b = L.Batch([good, make(L, d, "f32")])
        with pytest.raises(L.LbpsError) as e:
            b.set_step_pairs(True)
        assert e.value.code == L.LBPS_ERR_INVALID
        assert not b.step_pairs
        b.step(3)
        assert b.check() == 0
        b.close()
