"""The slab decomposition on the GPU: one lattice split into 2 or 3 slabs on
one device (paper_2301_00228_gb300.slab plan and CUDA engine), their ghost
rows exchanged after every step through device buffers with lbps_halo_pack /
lbps_halo_unpack, and every slab's owned rows compared bit for bit with the
undivided lattice, in every storage format.  (Across GPUs the same exchange
runs through NCCL; that path is covered by the gloo rank tests on CPU.)"""
import numpy as np
import pytest

from paper_2301_00228_gb300 import slab as S
from paper_2301_00228_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("ux", "uy", "vx", "vy", "phi", "psi", "f_phi", "f_psi")


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def exchange(slabs):
    """The ghost-row exchange of slab.SlabRun, between slabs held in one
    process: each slab's owned rows next to a cut into the neighbour's ghost rows."""
    world = len(slabs)
    packed = []
    for eng, p in slabs:
        out = {}
        if p.up is not None:
            out["up"] = eng.pack(*p.send_up_rows())
        if p.down is not None:
            out["down"] = eng.pack(*p.send_down_rows())
        packed.append(out)
    for r, (eng, p) in enumerate(slabs):
        if p.down is not None:
            eng.unpack(*p.recv_down_rows(), packed[(r - 1) % world]["up"])
        if p.up is not None:
            eng.unpack(*p.recv_up_rows(), packed[(r + 1) % world]["down"])


def run_split(L, world, c, storage, scale_exp, steps):
    slabs = []
    void = None if c["nt"] is None else (c["nt"] == 3).any(axis=1)
    for r in range(world):
        p = S.plan(c["ny"], world, r, periodic_y=c["py"], void_rows=void)
        eng = S.CudaSlab(p, c["nx"], c["lam"], 1.0, node_type=c["nt"], bc_value=c["bv"], cell=c["cell"],
                         loads=c["loads"], periodic_x=c["px"], a0_phi=c["a0"], storage=storage,
                         pop_scale_exp=scale_exp, sync_every=c["sync"], bc_j_mode=c["jmode"])
        run = S.SlabRun(eng, p)
        eng.init(run.take(c["ux"]), run.take(c["uy"]))
        slabs.append((eng, p))
    exchange(slabs)
    for _ in range(steps):
        for eng, _ in slabs:
            eng.step(1)
        exchange(slabs)
    torch.cuda.synchronize()
    out = []
    for eng, p in slabs:
        assert eng.lat.check() == 0
        out.append((p, {k: S.SlabRun(eng, p).read_owned(k) for k in FIELDS}))
        eng.close()
    return out


def case_rect(L, py=False, jmode=0, sync=0, px=False):
    nx, ny = 70, 57
    rng = np.random.default_rng(8)
    et, ev = (2, 1, 1, 1), rng.uniform(-2e-4, 2e-4, 8)
    nt, bv = L.lbps_rect_bc(nx, ny, px, py, 1.0, et, ev)
    ux, uy = W.pulse_displacement(nx, ny, 30.0, 25.0, 4.0, 1e-3, "dilatation")
    rx, ry = W.pulse_displacement(nx, ny, 50.0, 45.0, 3.0, 1e-3, "rotation")
    return dict(nx=nx, ny=ny, lam=1.7, px=px, py=py, nt=nt, bv=bv, cell=None, ux=ux + rx, uy=uy + ry, a0=0.99,
                loads=(), sync=sync, jmode=jmode)


def case_hole(L):
    d = W.hole_square(48, a0_phi=0.999, horizon=0.1, sync_every=50)
    ev = np.asarray(d.edge_value, float).ravel()
    nt, bv, cell = L.lbps_disk_cells(48, 48, 1.0, *d.hole, d.edge_type, ev)
    z = np.zeros((48, 48))
    return dict(nx=48, ny=48, lam=d.lam, px=False, py=False, nt=nt, bv=bv, cell=cell, ux=z, uy=z, a0=d.a0_phi,
                loads=d.loads, sync=d.sync_every, jmode=0)


def whole(L, c, storage, steps):
    lat = L.Lattice(c["nx"], c["ny"], c["lam"], 1.0, periodic_x=c["px"], periodic_y=c["py"], node_type=c["nt"],
                    bc_value=c["bv"], cell=c["cell"], a0_phi=c["a0"], storage=storage, sync_every=c["sync"],
                    bc_j_mode=c["jmode"])
    for kind, t_ramp, t_hold in c["loads"]:
        lat.set_load(kind, t_ramp, t_hold)
    lat.init(c["ux"], c["uy"]).step(steps)
    out = {k: lat.read(k) for k in FIELDS}, lat.scale_exp
    lat.close()
    return out


@pytest.mark.parametrize("world", [2, 3])
@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16", "bfp13"])
def test_slabs_equal_whole_rectangle(L, storage, world):
    c = case_rect(L)
    steps = 150
    want, e = whole(L, c, storage, steps)
    covered = 0
    for p, got in run_split(L, world, c, storage, e, steps):
        covered += p.y1 - p.y0
        for k in FIELDS:
            assert np.array_equal(got[k], want[k][..., p.y0:p.y1, :]), (storage, world, p.rank, k)
    assert covered == c["ny"]


@pytest.mark.parametrize("variant", ["periodic_y", "periodic_both", "sync_j1", "hole"])
def test_slabs_equal_whole_variants(L, variant):
    if variant == "hole":
        c = case_hole(L)
    elif variant == "periodic_y":
        c = case_rect(L, py=True)
    elif variant == "periodic_both":
        c = case_rect(L, py=True, px=True)
        c["nt"] = c["bv"] = None
    else:
        c = case_rect(L, jmode=1, sync=11)
    steps = 130
    for world in (2, 3):
        want, e = whole(L, c, "f32", steps)
        for p, got in run_split(L, world, c, "f32", e, steps):
            for k in FIELDS:
                assert np.array_equal(got[k], want[k][..., p.y0:p.y1, :]), (variant, world, p.rank, k)


def test_halo_entry_points_check_arguments(L):
    lat = L.Lattice.rectangle(40, 30, 1.0, 1.0, (1, 1, 1, 1), np.zeros(8), a0_phi=0.99)
    n = L.lbps_halo_bytes(lat._h, 3)
    assert n == 3 * 64 * (40 + 32)                  # pitched rows of 10 FP32 + 4 FP64 planes
    buf = torch.zeros(n + 64, dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LbpsError) as e:
        L.lbps_halo_pack(lat._h, 0, 3, buf.data_ptr(), n)  # before init
    assert e.value.code == L.LBPS_ERR_STATE
    lat.init(*W.pulse_displacement(40, 30, 20.0, 15.0, 3.0, 1e-3, "dilatation"))
    for row0, rows, off, size in ((28, 3, 0, n), (0, 3, 8, n), (0, 3, 0, n - 1), (-1, 3, 0, n)):
        with pytest.raises(L.LbpsError) as e:
            L.lbps_halo_pack(lat._h, row0, rows, buf.data_ptr() + off, size)
        assert e.value.code == L.LBPS_ERR_INVALID
    # a pack/unpack round trip of the same rows changes nothing
    before = {k: lat.read(k) for k in ("ux", "f_phi")}
    L.lbps_halo_pack(lat._h, 10, 3, buf.data_ptr(), n)
    L.lbps_halo_unpack(lat._h, 10, 3, buf.data_ptr(), n)
    for k, v in before.items():
        assert np.array_equal(lat.read(k), v), k
    lat.close()
