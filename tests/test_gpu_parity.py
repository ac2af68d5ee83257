"""Parity of the CUDA time loop with the FP64 oracle, through the C ABI.

Tolerances (tests/tolerance.py): FP64 population storage must match the
oracle to round-off (relative L2 <= 1e-10 per field); FP32 storage within
relative L2 <= 1e-5 per field; the 16-bit formats within 1e-3, a run that
misses it being reported as an expected failure with its measured error (the
format's precision limit) as long as it stays below a regression bound.
Relative L2 is taken per field against max(||ref||, 1e-2 ||ref group||)
where the groups are (ux, uy), (vx, vy), (phi, psi), so a field that is zero
by symmetry is compared on the scale of its partner.
"""
import numpy as np
import pytest

import oracle as O
import hand_cases as H
from paper_2301_00228_gb300 import workloads as W
from tolerance import TARGET as TOL
from tolerance import judge

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

GROUPS = (("ux", "uy"), ("vx", "vy"), ("phi", "psi"))


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def rel_errors(got, ref):
    out = {}
    for g in GROUPS:
        gn = np.sqrt(sum(np.linalg.norm(ref[k]) ** 2 for k in g))
        for k in g:
            den = max(np.linalg.norm(ref[k]), 1e-2 * gn, 1e-300)
            out[k] = float(np.linalg.norm(got[k] - ref[k]) / den)
    return out


def assert_parity(got, ref, tol, what="", storage=None):
    """Every field within tol; with a 16-bit storage named, a miss within the
    format's known limit is an expected failure (tests/tolerance.py)."""
    errs = rel_errors(got, ref)
    if storage in ("bf16", "f16", "bfp13"):
        return judge(errs, storage, what)
    bad = {k: v for k, v in errs.items() if not v <= tol}
    assert not bad, (what, bad, errs)
    return errs


# ------------------------------------------------------------ hand cases

def _gpu_factory(L, storage):
    def make(case, mode):
        c = H.load()["common"]
        return L.Lattice.rectangle(c["nx"], c["ny"], c["lambda"], c["mu"], case["edges"]["type"],
                                   H.edge_values(case), rho=c["rho"], a0_phi=c["a0_phi"], bc_feq_mode=mode,
                                   storage=storage)
    return make


def _gpu_read(lat, field, alpha):
    if field in ("f_phi", "f_psi"):
        return lat.read(field)[alpha]
    return lat.read(field)


@pytest.mark.parametrize("storage,tol", [("f64", 1e-12), ("f32", 1e-6)])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", [c["name"] for c in H.load()["cases"]])
def test_hand_cases(L, name, mode, storage, tol):
    g = H.load()
    case = next(c for c in g["cases"] if c["name"] == name)
    make = _gpu_factory(L, storage)
    dt = make(case, mode).dt
    fails = H.run_case(case, g["common"], mode, make, _gpu_read, dt, tol)
    assert not fails, fails


@pytest.mark.parametrize("storage,tol", [("f64", 1e-10), ("f32", 1e-5)])
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", [c["name"] for c in H.load()["cases"]])
def test_hand_inputs_partial_stream_j(L, name, mode, storage, tol):
    """The hand-computed lattices' inputs with J of Eq. correction-f taken
    from the partial LBE update (bc_j_mode 1), 12 steps, against the oracle."""
    g = H.load()
    c = g["common"]
    case = next(x for x in g["cases"] if x["name"] == name)
    ux, uy = H.initial_u(c)
    nt, bv = O.rect_bc(c["nx"], c["ny"], case["edges"]["type"], H.edge_values(case))
    ref = O.OracleLattice(c["nx"], c["ny"], c["lambda"], c["mu"], c["rho"], c["dh"], c["a0_phi"], node_type=nt,
                          bc_value=bv, bc_feq_mode=mode, bc_j_mode=1).init(ux, uy).step(12).fields()
    lat = L.Lattice.rectangle(c["nx"], c["ny"], c["lambda"], c["mu"], case["edges"]["type"], H.edge_values(case),
                              rho=c["rho"], a0_phi=c["a0_phi"], bc_feq_mode=mode, bc_j_mode=1, storage=storage)
    got = lat.init(ux, uy).step(12).fields()
    lat.close()
    for k in ref:
        scale = max(np.abs(ref[k]).max(), 1e-30)
        assert np.abs(got[k] - ref[k]).max() <= tol * scale, (k, storage)


# ------------------------------------------------------- mixed rectangles

def mixed_case(seed, nx, ny, periodic=(0, 0), a0=0.99, mode=0, sync=0, steps=200, jmode=0):
    rng = np.random.default_rng(seed)
    et = tuple(int(x) for x in rng.choice([1, 2], 4))
    ev = rng.uniform(-2e-4, 2e-4, 8)
    lam = float(rng.uniform(0.5, 4.0))
    cx, cy = float(rng.uniform(0, nx - 1)), float(rng.uniform(0, ny - 1))
    kind = "dilatation" if seed % 2 else "rotation"
    ux, uy = W.pulse_displacement(nx, ny, cx, cy, max(1.5, min(nx, ny) / 8), 1e-3, kind)
    return dict(nx=nx, ny=ny, et=et, ev=ev, lam=lam, px=periodic[0], py=periodic[1], a0=a0, mode=mode,
                sync=sync, steps=steps, ux=ux, uy=uy, jmode=jmode)


MIXED = [
    mixed_case(1, 67, 45),
    mixed_case(2, 130, 97, a0=0.9999, steps=300),
    mixed_case(3, 67, 45, mode=1),
    mixed_case(4, 96, 64, sync=7),
    mixed_case(5, 70, 41, periodic=(1, 0)),
    mixed_case(6, 41, 70, periodic=(0, 1), mode=1),
    mixed_case(7, 64, 48, periodic=(1, 1), a0=0.9),
    mixed_case(8, 3, 3, steps=50),
    mixed_case(9, 3, 11, steps=80),
    mixed_case(10, 13, 3, steps=80, mode=1),
    mixed_case(11, 33, 17, a0=0.5, steps=20),
]


def run_oracle(cs):
    nt, bv = O.rect_bc(cs["nx"], cs["ny"], cs["et"], cs["ev"], periodic_x=cs["px"], periodic_y=cs["py"])
    lat = O.OracleLattice(cs["nx"], cs["ny"], cs["lam"], 1.0, a0_phi=cs["a0"], periodic_x=cs["px"],
                          periodic_y=cs["py"], node_type=nt, bc_value=bv, bc_feq_mode=cs["mode"],
                          sync_every=cs["sync"], bc_j_mode=cs["jmode"])
    return lat.init(cs["ux"], cs["uy"]).step(cs["steps"]).fields()


def run_gpu(L, cs, storage):
    lat = L.Lattice.rectangle(cs["nx"], cs["ny"], cs["lam"], 1.0, cs["et"], cs["ev"], periodic_x=cs["px"],
                              periodic_y=cs["py"], a0_phi=cs["a0"], bc_feq_mode=cs["mode"], sync_every=cs["sync"],
                              storage=storage, bc_j_mode=cs["jmode"])
    f = lat.init(cs["ux"], cs["uy"]).step(cs["steps"]).fields()
    lat.close()
    return f


@pytest.mark.parametrize("jmode", [0, 1])
@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16", "bfp13"])
@pytest.mark.parametrize("k", range(len(MIXED)))
def test_mixed_rectangles(L, k, storage, jmode):
    """Both readings of J in Eq. correction-f (bc_j_mode 0 and 1)."""
    cs = dict(MIXED[k], jmode=jmode)
    if storage in ("bf16", "f16", "bfp13") and ((cs["nx"] == 3 and not cs["px"]) or (cs["ny"] == 3 and not cs["py"])):
        with pytest.raises(L.LbpsError) as e:       # 16-bit storage needs 4 points across
            run_gpu(L, cs, storage)
        assert e.value.code == L.LBPS_ERR_INVALID
        return
    assert_parity(run_gpu(L, cs, storage), run_oracle(cs), TOL[storage], (k, storage), storage)


# ------------------------------------------------- the 64 x 64 problem

@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16", "bfp13"])
def test_square_64_1000_steps(L, storage):
    """64 x 64, left edge clamped, others traction-free, centred dilatation pulse
    sigma = 4, lambda = mu = rho = 1, a_{0,phi} = 0.9999, 1000 steps."""
    d = W.square_64()
    ev = np.asarray(d.edge_value, float).ravel()
    ux, uy = d.displacement()
    nt, bv = O.rect_bc(64, 64, d.edge_type, ev)
    ref = O.OracleLattice(64, 64, 1.0, 1.0, node_type=nt, bc_value=bv).init(ux, uy).step(d.steps).fields()
    lat = L.Lattice.rectangle(64, 64, 1.0, 1.0, d.edge_type, ev, storage=storage)
    got = lat.init(ux, uy).step(d.steps).fields()
    assert_parity(got, ref, TOL[storage], "square_64", storage)


# ------------------------------------------- full size: periodic waves

def test_periodic_waves_full_size(L):
    """1024 x 1024 periodic, lambda/mu = 2, superposed dilatational and shear standing
    waves (wavelength 64), 10^4 FP32 steps, against the closed form of the scheme."""
    from test_oracle_pins import standing_wave_expected

    d = W.periodic_waves()
    m, n, amp_d, amp_s = d.wave
    lat = L.Lattice(d.nx, d.ny, d.lam, d.mu, periodic_x=True, periodic_y=True, storage="f32")
    ux, uy = d.displacement()
    lat.init(ux, uy).step(d.steps)
    ex = standing_wave_expected(d.nx, d.ny, m, n, amp_d, amp_s, d.lam, d.mu, d.rho, lat.a_phi, lat.a_psi, lat.dt,
                                d.steps)
    errs = assert_parity(lat.fields(), ex, TOL["f32"])
    print("periodic 1024^2 x 1e4 steps rel-L2:", errs)


# ---------------------------------------- full size: sampled windows

def test_many_pulses_full_size_sampled(L):
    """8192 x 8192, lambda/mu = 3, clamped bottom, 32 pulses (the largest single-GPU
    lattice), in the benchmark's launch configuration.  One step widens the domain of
    dependence by at most 5 points (a second-row point reads the reset state of its
    boundary neighbour, whose differences of the new u reach 2 points and whose
    boundary accelerations reach 2 more), so the oracle on a window of radius
    5 S + 16 around a sample reproduces the 13 x 13 points around it."""
    d = W.many_pulses(steps=24)
    S = d.steps
    R = 5 * S + 16
    ev = np.asarray(d.edge_value, float).ravel()
    lat = L.Lattice.rectangle(d.nx, d.ny, d.lam, d.mu, d.edge_type, ev, storage="f32")
    ux_d, uy_d = d.displacement_torch("cuda")
    lat.init(ux_d, uy_d).step(S)
    del ux_d, uy_d
    got = {k: lat.read_device(k) for k in ("ux", "uy", "phi", "psi")}
    samples = [(0, 0), (d.nx - 1, 0), (4000, 0), (0, 5000), (d.nx - 1, 3000), (2000, d.ny - 1),
               (d.nx - 1, d.ny - 1), (4100, 4100)]
    rng = np.random.default_rng(44)
    samples += [tuple(int(v) for v in rng.integers(0, d.nx, 2)) for _ in range(3)]
    for (si, sj) in samples:
        x0, x1 = max(0, si - R), min(d.nx, si + R + 1)
        y0, y1 = max(0, sj - R), min(d.ny, sj + R + 1)
        w, h = x1 - x0, y1 - y0
        ux, uy = d.displacement(window=(x0, y0, w, h))
        # crop edges that are real edges keep their type; cut edges get traction-free
        et = [d.edge_type[0] if y0 == 0 else 1, d.edge_type[1] if x1 == d.nx else 1,
              d.edge_type[2] if y1 == d.ny else 1, d.edge_type[3] if x0 == 0 else 1]
        nt, bv = O.rect_bc(w, h, et, ev)
        ref = O.OracleLattice(w, h, d.lam, d.mu, node_type=nt, bc_value=bv).init(ux, uy).step(S).fields()
        r = 6
        wx0, wx1 = max(0, si - r), min(d.nx, si + r + 1)
        wy0, wy1 = max(0, sj - r), min(d.ny, sj + r + 1)
        g = {k: got[k][wy0:wy1, wx0:wx1].cpu().numpy() for k in got}
        e = {k: ref[k][wy0 - y0:wy1 - y0, wx0 - x0:wx1 - x0] for k in got}
        for k in ("ux", "uy", "phi", "psi"):
            scale = max(np.abs(e["ux"]).max(), np.abs(e["uy"]).max()) if k in ("ux", "uy") else \
                max(np.abs(e["phi"]).max(), np.abs(e["psi"]).max())
            assert np.abs(g[k] - e[k]).max() <= 2e-6 * scale + 1e-18, ((si, sj), k)


def test_full_size_corner_bumps_long_run(L):
    """8192 x 8192 (clamped bottom, traction-free other edges, lambda/mu = 3) from
    three bumps of compact support: two at corners, one on the top edge.  After
    S = 120 steps the state can differ from zero only within 5 S points of a
    bump (the widening bound of the sampled test above), so (a) every point
    outside those regions is exactly zero on the GPU, over the whole lattice,
    and (b) inside them the GPU equals the oracle run on a crop around each
    region (cut edges traction-free, beyond the reach of the bumps), point for
    point: the boundary reset and the corners after many steps at full size."""
    d = W.many_pulses(steps=120)
    S, rad = d.steps, 6
    reach = 5 * S + rad + 8
    centres = [(rad, rad, "dilatation"), (d.nx - 1 - rad, d.ny - 1 - rad, "rotation"),
               (4000, d.ny - 1 - rad, "dilatation")]
    ux = np.zeros((d.ny, d.nx))
    uy = np.zeros((d.ny, d.nx))
    boxes = []
    for cx, cy, kind in centres:
        x0, x1 = max(0, cx - reach), min(d.nx, cx + reach + 1)
        y0, y1 = max(0, cy - reach), min(d.ny, cy + reach + 1)
        bx, by = W.bump_displacement(x1 - x0, y1 - y0, cx, cy, rad, 1e-3, kind, x0=x0, y0=y0)
        ux[y0:y1, x0:x1] += bx
        uy[y0:y1, x0:x1] += by
        boxes.append((x0, x1, y0, y1))
    ev = np.asarray(d.edge_value, float).ravel()
    lat = L.Lattice.rectangle(d.nx, d.ny, d.lam, d.mu, d.edge_type, ev, storage="f32")
    lat.init(ux, uy).step(S)
    inside = torch.zeros((d.ny, d.nx), dtype=torch.bool, device="cuda")
    for x0, x1, y0, y1 in boxes:
        inside[y0:y1, x0:x1] = True
    got = {}
    keys = ("ux", "uy", "vx", "vy", "phi", "psi")
    for k in keys:
        t = lat.read_device(k)
        assert int(torch.count_nonzero(t[~inside])) == 0, k
        got[k] = [t[y0:y1, x0:x1].cpu().numpy() for x0, x1, y0, y1 in boxes]
        del t
    lat.close()
    for b, (x0, x1, y0, y1) in enumerate(boxes):
        w, h = x1 - x0, y1 - y0
        et = [d.edge_type[0] if y0 == 0 else 1, d.edge_type[1] if x1 == d.nx else 1,
              d.edge_type[2] if y1 == d.ny else 1, d.edge_type[3] if x0 == 0 else 1]
        nt, bv = O.rect_bc(w, h, et, ev)
        ref = O.OracleLattice(w, h, d.lam, d.mu, node_type=nt, bc_value=bv).init(
            ux[y0:y1, x0:x1], uy[y0:y1, x0:x1]).step(S).fields()
        assert all(np.abs(ref[k]).max() > 0 for k in keys), b
        assert_parity({k: got[k][b] for k in keys}, {k: ref[k] for k in keys}, TOL["f32"], what=("bump", b))
        for k in keys:
            assert np.abs(got[k][b] - ref[k]).max() <= TOL["f32"] * np.abs(ref[k]).max(), (b, k)


# ----------------------------------------------------------- edge cases

def _small(L, **kw):
    args = dict(nx=20, ny=17, lam=1.0, mu=1.0, edge_type=(1, 2, 1, 1), edge_value=np.zeros(8))
    args.update(kw)
    return L.Lattice.rectangle(args.pop("nx"), args.pop("ny"), args.pop("lam"), args.pop("mu"),
                               args.pop("edge_type"), args.pop("edge_value"), **args)


def test_zero_steps_is_init(L):
    ux, uy = W.pulse_displacement(20, 17, 9.0, 8.0, 2.0, 1e-3, "rotation")
    lat = _small(L, storage="f64").init(ux, uy).step(0)
    nt, bv = O.rect_bc(20, 17, (1, 2, 1, 1), np.zeros(8))
    ref = O.OracleLattice(20, 17, 1.0, 1.0, node_type=nt, bc_value=bv).init(ux, uy)
    assert_parity(lat.fields(), ref.fields(), 1e-13)
    assert np.abs(lat.read("f_psi") - ref.read(O.F_PSI)).max() <= 1e-18
    assert lat.steps == 0


def test_invalid_inputs_rejected(L):
    nt, bv = L.lbps_rect_bc(10, 8, 0, 0, 1.0, (1, 1, 1, 1), np.zeros(8))
    bad = nt.copy()
    bad[3, 3] = 1  # interior point marked as boundary
    with pytest.raises(L.LbpsError) as e:
        L.Lattice(10, 8, 1.0, 1.0, node_type=bad, bc_value=bv)
    assert e.value.code == L.LBPS_ERR_INVALID
    bad = nt.copy()
    bad[0, 4] = 0  # boundary point left interior
    with pytest.raises(L.LbpsError):
        L.Lattice(10, 8, 1.0, 1.0, node_type=bad, bc_value=bv)
    bv2 = bv.copy()
    bv2[0, 0, 0] = np.nan
    with pytest.raises(L.LbpsError):
        L.Lattice(10, 8, 1.0, 1.0, node_type=nt, bc_value=bv2)
    with pytest.raises(L.LbpsError):
        L.Lattice(10, 8, 1.0, 1.0)  # bounded lattice without a mask
    with pytest.raises(L.LbpsError):
        L.Lattice(10, 8, 1.0, -1.0, periodic_x=True, periodic_y=True)


def test_call_order_and_capacity(L):
    lat = _small(L)
    assert L.lbps_step(lat._h, 1) == L.LBPS_ERR_STATE
    with pytest.raises(L.LbpsError) as e:
        lat.read("ux")
    assert e.value.code == L.LBPS_ERR_STATE
    ux = np.zeros((17, 20))
    lat.init(ux, ux)
    small = np.zeros(10)
    assert L._lib.lbps_read(lat._h, L.LBPS_UX, L._p(small), small.size) == L.LBPS_ERR_INVALID
    assert L._lib.lbps_read(lat._h, 42, L._p(small), small.size) == L.LBPS_ERR_INVALID
    assert L.lbps_step(lat._h, -1) == L.LBPS_ERR_INVALID
    bad = ux.copy()
    bad[2, 2] = np.inf
    with pytest.raises(L.LbpsError):
        lat.init(bad, ux)


def test_nonfinite_state_reported(L):
    """A displacement of 1e300 overflows FP32 populations; the step reports it."""
    ux = np.full((17, 20), 1e300)
    lat = _small(L, storage="f32").init(ux, np.zeros_like(ux))
    assert L.lbps_step(lat._h, 3) == L.LBPS_ERR_NONFINITE
    assert lat.check() == L.LBPS_ERR_NONFINITE
    lat.init(np.zeros_like(ux), np.zeros_like(ux))  # re-initialising clears the flag
    assert L.lbps_step(lat._h, 3) == L.LBPS_OK


def test_norms_match_host(L):
    ux, uy = W.pulse_displacement(50, 37, 20.0, 20.0, 4.0, 1e-3, "dilatation")
    lat = L.Lattice.rectangle(50, 37, 2.0, 1.0, (2, 1, 1, 1), np.zeros(8), a0_phi=0.99).init(ux, uy).step(30)
    for name in ("ux", "uy", "phi", "psi", "consistency"):
        x = lat.read(name)
        ref = torch.from_numpy(np.sin(np.arange(x.size)).reshape(x.shape) * 1e-3).cuda()
        n = lat.norms(name, ref)
        r = ref.cpu().numpy()
        assert n[0] == pytest.approx(((x - r) ** 2).sum(), rel=1e-12)
        assert n[1] == pytest.approx((r ** 2).sum(), rel=1e-12)
        assert abs(n[2] - x.sum()) <= 1e-12 * np.abs(x).sum() + 1e-300
        assert n[3] == np.abs(x).max()
        n0 = lat.norms(name)
        assert n0[0] == pytest.approx((x ** 2).sum(), rel=1e-12) and n0[1] == 0.0


def test_consistency_and_populations_match_oracle(L):
    nx, ny = 31, 26
    ux, uy = W.pulse_displacement(nx, ny, 12.0, 10.0, 3.0, 1e-3, "rotation")
    nt, bv = O.rect_bc(nx, ny, (1, 1, 2, 1), np.zeros(8))
    ref = O.OracleLattice(nx, ny, 1.0, 1.0, a0_phi=0.99, node_type=nt, bc_value=bv).init(ux, uy).step(40)
    lat = L.Lattice.rectangle(nx, ny, 1.0, 1.0, (1, 1, 2, 1), np.zeros(8), a0_phi=0.99, storage="f64")
    lat.init(ux, uy).step(40)
    e_ref = ref.read(O.ERR)
    assert np.abs(lat.read("consistency") - e_ref).max() <= 1e-10 * e_ref.max()
    for f, fid in (("f_phi", O.F_PHI), ("f_psi", O.F_PSI)):
        r = ref.read(fid)
        assert np.abs(lat.read(f) - r).max() <= 1e-10 * np.abs(r).max()


def test_sync_matches_oracle(L):
    nx, ny = 40, 30
    ux, uy = W.pulse_displacement(nx, ny, 15.0, 12.0, 3.0, 1e-3, "dilatation")
    nt, bv = O.rect_bc(nx, ny, (2, 1, 1, 1), np.zeros(8))
    ref = O.OracleLattice(nx, ny, 1.5, 1.0, a0_phi=0.99, node_type=nt, bc_value=bv).init(ux, uy).step(13).sync()
    for storage in ("f64", "f32"):
        lat = L.Lattice.rectangle(nx, ny, 1.5, 1.0, (2, 1, 1, 1), np.zeros(8), a0_phi=0.99, storage=storage)
        lat.init(ux, uy).step(13).sync()
        assert_parity(lat.fields(), ref.fields(), TOL[storage])
        assert lat.read("consistency").max() <= (1e-15 if storage == "f64" else 1e-10)


def test_device_init_equals_host_init(L):
    ux, uy = W.pulse_displacement(40, 33, 15.0, 12.0, 3.0, 1e-3, "dilatation")
    vx, vy = 1e-4 * uy, -1e-4 * ux
    a = _small(L, nx=40, ny=33, storage="f64").init(ux, uy, vx, vy).step(11)
    t = [torch.from_numpy(x).cuda() for x in (ux, uy, vx, vy)]
    b = _small(L, nx=40, ny=33, storage="f64").init(*t).step(11)
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k
    nt, bv = O.rect_bc(40, 33, (1, 2, 1, 1), np.zeros(8))
    ref = O.OracleLattice(40, 33, 1.0, 1.0, node_type=nt, bc_value=bv).init(ux, uy, vx, vy).step(11)
    assert_parity(fa, ref.fields(), TOL["f64"])


def test_library_owned_memory(L):
    """device_mem = NULL: the library allocates and frees the state itself."""
    p = L.lbps_params(24, 20, 1.0, 1.0, 1.0, 1.0, 0.99, 1, 1, 0, 0, L.LBPS_STORAGE_F32, 0, None)
    h = L.lbps_create(p, None, None, 0, 0)
    ux, uy = W.pulse_displacement(24, 20, 10.0, 9.0, 2.0, 1e-3, "dilatation")
    L.lbps_init(h, np.ascontiguousarray(ux), np.ascontiguousarray(uy))
    assert L.lbps_step(h, 10) == L.LBPS_OK
    out = np.zeros((20, 24))
    L.lbps_read(h, L.LBPS_UX, out)
    L.lbps_destroy(h)
    ref = O.OracleLattice(24, 20, 1.0, 1.0, a0_phi=0.99, periodic_x=True, periodic_y=True).init(ux, uy).step(10)
    r = ref.read(O.UX)
    assert np.linalg.norm(out - r) <= 1e-5 * np.linalg.norm(r)


def test_chunked_host_read(L):
    """Host reads larger than the staging buffer go through it in row blocks."""
    nx, ny = 640, 420
    d = W.Domain(nx, ny, 1.0, 1.0, pulses=[(300.0, 200.0, 20.0, 1e-3, "rotation")])
    lat = L.Lattice.rectangle(nx, ny, 1.0, 1.0, (1, 1, 1, 1), np.zeros(8), a0_phi=0.99)
    lat.init(*d.displacement()).step(5)
    for f in ("f_phi", "psi", "uy"):
        h = lat.read(f)
        dv = lat.read_device(f).cpu().numpy()
        assert np.array_equal(h, dv), f


def test_two_streams_independent(L):
    """Two lattices on two streams, stepped interleaved, give their solo results."""
    cs1, cs2 = MIXED[0], MIXED[3]
    solo1, solo2 = run_gpu(L, cs1, "f32"), run_gpu(L, cs2, "f32")
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()

    def mk(cs, st):
        return L.Lattice.rectangle(cs["nx"], cs["ny"], cs["lam"], 1.0, cs["et"], cs["ev"], a0_phi=cs["a0"],
                                   bc_feq_mode=cs["mode"], sync_every=cs["sync"], storage="f32", stream=st)

    a, b = mk(cs1, s1), mk(cs2, s2)
    a.init(cs1["ux"], cs1["uy"])
    b.init(cs2["ux"], cs2["uy"])
    for _ in range(max(cs1["steps"], cs2["steps"]) // 10):
        if a.steps < cs1["steps"]:
            a.step_async(10)
        if b.steps < cs2["steps"]:
            b.step_async(10)
    assert a.check() == 0 and b.check() == 0
    fa, fb = a.fields(), b.fields()
    for k in solo1:
        assert np.array_equal(fa[k], solo1[k]) and np.array_equal(fb[k], solo2[k]), k


def test_tunings_bit_identical(L):
    """Every launch shape of the interior kernel gives the same bits (ragged strip
    and row counts included)."""
    cs = mixed_case(21, 97, 83, steps=40)
    for storage in ("f32", "f16", "bfp13"):
        ref = None
        for variant in range(8):
            for rows in (1, 7, 64, 4096):
                lat = L.Lattice.rectangle(cs["nx"], cs["ny"], cs["lam"], 1.0, cs["et"], cs["ev"], a0_phi=cs["a0"],
                                          storage=storage)
                L.lbps_set_tuning(lat._h, variant, rows)
                f = lat.init(cs["ux"], cs["uy"]).step(cs["steps"]).fields()
                lat.close()
                if ref is None:
                    ref = f
                    assert_parity(f, run_oracle(cs), TOL[storage])
                for k in f:
                    assert np.array_equal(f[k], ref[k]), (storage, variant, rows, k)
    small = L.Lattice(8, 8, 1.0, 1.0, periodic_x=True, periodic_y=True)
    for bad in ((8, 64), (-1, 64), (0, 0), (0, 5000)):
        with pytest.raises(L.LbpsError):
            L.lbps_set_tuning(small._h, *bad)


def test_rejected_init_keeps_state(L):
    """lbps_init checks its input on the device after staging it in the copy
    that is not current: a rejected input leaves the lattice exactly where it
    was, and later steps (and void points of a general geometry) are
    unaffected."""
    ux, uy = W.pulse_displacement(47, 39, 20.0, 17.0, 3.0, 1e-3, "rotation")
    a = L.Lattice.rectangle(47, 39, 1.2, 1.0, (1, 2, 1, 1), np.zeros(8), a0_phi=0.99).init(ux, uy).step(7)
    b = L.Lattice.rectangle(47, 39, 1.2, 1.0, (1, 2, 1, 1), np.zeros(8), a0_phi=0.99).init(ux, uy).step(7)
    before = {k: a.read(k) for k in ("ux", "uy", "vx", "vy", "phi", "psi")}
    bad = np.full_like(ux, 3.0)
    bad[5, 9] = np.nan
    for args in ((bad, uy), (ux, uy, np.zeros_like(ux), np.where(ux > 1e-4, np.inf, 0.0))):
        with pytest.raises(L.LbpsError) as e:
            a.init(*args)
        assert e.value.code == L.LBPS_ERR_INVALID
    for k, v in before.items():
        assert np.array_equal(a.read(k), v), k
    a.step(13)
    b.step(13)
    for k in before:
        assert np.array_equal(a.read(k), b.read(k)), k
    # general geometry: garbage at void points of a rejected input never shows
    n = 40
    d = W.hole_square(n, a0_phi=0.999, horizon=0.05, sync_every=0)
    nt, bv, cell = L.lbps_disk_cells(n, n, 1.0, *d.hole, d.edge_type, np.asarray(d.edge_value, float).ravel())
    h = L.Lattice(n, n, d.lam, d.mu, a0_phi=d.a0_phi, node_type=nt, bc_value=bv, cell=cell)
    z = np.zeros((n, n))
    h.init(z, z)
    junk = np.where(nt == L.LBPS_VOID, 7.0, 0.0)
    junk[0, 0] = np.nan
    with pytest.raises(L.LbpsError):
        h.init(junk, junk)
    h.init(*W.pulse_displacement(n, n, 10.0, 10.0, 3.0, 1e-3, "dilatation"))
    h.step(5)
    void = nt == L.LBPS_VOID
    for k in ("ux", "uy", "vx", "vy"):
        assert np.abs(h.read(k)[void]).max() == 0.0, k


def test_caller_block_too_small_or_misaligned(L):
    """Host-side fault injection for allocation: a caller-provided device
    block smaller than lbps_state_bytes, or not 256-byte aligned, is refused
    with LBPS_ERR_OOM before anything is written to it."""
    p = L.lbps_params(40, 30, 1.0, 1.0, 1.0, 1.0, 0.99, 0, 0, 0, 0, L.LBPS_STORAGE_F32, 0, None)
    need = L.lbps_state_bytes(p)
    nt, bv = L.lbps_rect_bc(40, 30, 0, 0, 1.0, (2, 1, 1, 1), np.zeros(8))
    block = torch.zeros(need + 512, dtype=torch.uint8, device="cuda")
    for ptr, size in ((block.data_ptr(), need - 1), (block.data_ptr() + 64, need)):
        with pytest.raises(L.LbpsError) as e:
            L.lbps_create(p, nt, bv, ptr, size)
        assert e.value.code == L.LBPS_ERR_OOM
    assert int(block.sum()) == 0                      # nothing written
    h = L.lbps_create(p, nt, bv, block.data_ptr(), need)
    L._lib.lbps_destroy(h)


@pytest.mark.parametrize("jmode", [0, 1])
@pytest.mark.parametrize("size", [(3, 3), (4, 5), (7, 3)])
@pytest.mark.parametrize("edges", range(16))
def test_tiny_every_boundary_mix(L, size, edges, jmode):
    """Every Dirichlet/Neumann combination of the four edges (with the corner
    rule where a Dirichlet and a Neumann edge meet) on tiny lattices, from a
    random state, FP64 and FP32 against the oracle, in both readings of J in
    Eq. correction-f."""
    nx, ny = size
    et = tuple(1 + ((edges >> q) & 1) for q in range(4))
    rng = np.random.default_rng(1000 + 16 * nx + edges)
    ev = rng.uniform(-2e-4, 2e-4, 8)
    ux, uy = rng.uniform(-1e-4, 1e-4, (2, ny, nx))
    nt, bv = O.rect_bc(nx, ny, et, ev)
    ref = O.OracleLattice(nx, ny, 1.3, 1.0, a0_phi=0.9, node_type=nt, bc_value=bv, bc_j_mode=jmode)
    ref = ref.init(ux, uy).step(40).fields()
    for storage in ("f64", "f32"):
        lat = L.Lattice.rectangle(nx, ny, 1.3, 1.0, et, ev, a0_phi=0.9, storage=storage, bc_j_mode=jmode)
        got = lat.init(ux, uy).step(40).fields()
        lat.close()
        assert_parity(got, ref, TOL[storage], (size, et, storage))


@pytest.mark.parametrize("storage", ["f32", "f16", "bfp13"])
def test_step_graphs_same_bits(L, storage):
    """lbps_step replays blocks of k steps (and pairs) from captured CUDA
    graphs (one per starting copy); with per-kernel timing on it launches
    every kernel itself.  All give the same bits, for several k, across
    synchronisation points (every 7th step), a changed launch shape, a load
    schedule and a changed k set between calls (which make the graphs be
    captured again)."""
    cs = mixed_case(31, 71, 53, steps=0, a0=0.99)
    ev = cs["ev"]

    def run(timed, k=2):
        lat = L.Lattice.rectangle(cs["nx"], cs["ny"], cs["lam"], 1.0, cs["et"], ev, a0_phi=cs["a0"], storage=storage,
                                  sync_every=7)
        L.lbps_profile(lat._h, int(timed))
        L.lbps_set_graph_steps(lat._h, k)
        lat.init(cs["ux"], cs["uy"])
        lat.step(1).step(10).step(5)
        L.lbps_set_tuning(lat._h, 5, 16)
        lat.step(9)
        lat.set_load(L.LBPS_NEUMANN, 20 * lat.dt, 40 * lat.dt)
        lat.step(30).step(2)
        L.lbps_set_graph_steps(lat._h, 2 if k > 2 else 4)
        lat.step(13)
        out = {k: lat.read(k) for k in ("ux", "uy", "vx", "vy", "f_phi", "f_psi")}
        assert lat.steps == 70
        lat.close()
        return out

    a = run(True)
    for k in (2, 4, 6, 16):   # blocks of k steps, split by the synchronisation every 7th step or not
        b = run(False, k)
        for f in a:
            assert np.array_equal(a[f], b[f]), (storage, k, f)
    lat = L.Lattice(8, 8, 1.0, 1.0, periodic_x=True, periodic_y=True)
    for bad in (0, 1, 3, 66):
        with pytest.raises(L.LbpsError):
            L.lbps_set_graph_steps(lat._h, bad)
    lat.close()
