"""The slab decomposition's plan and ghost-row exchange (paper_2301_00228_gb300.slab)
on CPU ranks: gloo process groups of 2 and 3 ranks (one spawned process per
rank, rendezvous on 127.0.0.1), each rank's slab advanced by the FP64 oracle
and its rows exchanged through torch.distributed after every step.  The
owned rows of every rank must equal the whole lattice's, bit for bit, for
rectangles with mixed edges, periodic axes, a plate with a hole, periodic
synchronisation, ramped loads and both readings of the boundary rules."""
import os
import socket
import sys
from pathlib import Path

import numpy as np
import pytest

torch = pytest.importorskip("torch")
ROOT = Path(__file__).resolve().parents[1]

FIELDS = ("ux", "uy", "vx", "vy", "phi", "psi", "f_phi", "f_psi")


class OracleSlab:
    """SlabRun engine on the FP64 oracle: rows move as host tensors of
    (14, rows, nx) doubles (ora_get_rows / ora_set_rows)."""

    device = "cpu"

    def __init__(self, p, nx, lam, mu, rho=1.0, dh=1.0, node_type=None, bc_value=None, cell=None, loads=(),
                 periodic_x=False, a0_phi=0.99, bc_feq_mode=0, bc_j_mode=0, sync_every=0):
        import oracle as O
        from paper_2301_00228_gb300 import slab

        self.O = O
        nt, bv, cl = slab.slab_description(p, nx, node_type, bc_value, cell, dh)
        self.nx = nx
        self.lat = O.OracleLattice(nx, p.rows, lam, mu, rho, dh, a0_phi=a0_phi, periodic_x=periodic_x,
                                   periodic_y=p.periodic_y and p.world == 1, node_type=nt, bc_value=bv, cell=cl,
                                   bc_feq_mode=bc_feq_mode, bc_j_mode=bc_j_mode, sync_every=sync_every)
        for kind, t_ramp, t_hold in loads:
            self.lat.set_load(kind, t_ramp, t_hold)

    def init(self, ux, uy, vx=None, vy=None):
        self.lat.init(ux, uy, vx, vy)

    def scale_exp(self):
        return None

    def empty(self, rows):
        return torch.empty((14, rows, self.nx), dtype=torch.float64)

    def pack(self, row0, rows):
        return torch.from_numpy(self.lat.get_rows(row0, rows))

    def unpack(self, row0, rows, buf):
        self.lat.set_rows(row0, buf.numpy())

    def step(self, n):
        self.lat.step(n)

    def read(self, field):
        O = self.O
        ids = {"ux": O.UX, "uy": O.UY, "vx": O.VX, "vy": O.VY, "phi": O.PHI, "psi": O.PSI, "f_phi": O.F_PHI,
               "f_psi": O.F_PSI}
        return self.lat.read(ids[field])


def cases():
    """(name, description) of the whole lattices; every field of a description
    is plain data so it can go to spawned processes."""
    from paper_2301_00228_gb300 import workloads as W

    out = []
    nx, ny = 23, 31
    rng = np.random.default_rng(4)
    ux, uy = W.pulse_displacement(nx, ny, 9.0, 14.0, 3.0, 1e-3, "dilatation")
    vx, vy = 1e-4 * rng.standard_normal((2, ny, nx))
    out.append(("mixed_edges", dict(nx=nx, ny=ny, lam=1.6, mu=1.0, et=(2, 1, 1, 2), ev=rng.uniform(-2e-4, 2e-4, 8),
                                    px=False, py=False, a0=0.9, steps=90, u=(ux, uy, vx, vy))))
    out.append(("mixed_edges_j1_feq1_sync", dict(nx=nx, ny=ny, lam=1.6, mu=1.0, et=(1, 2, 1, 1),
                                                 ev=rng.uniform(-2e-4, 2e-4, 8), px=False, py=False, a0=0.9,
                                                 steps=70, u=(ux, uy, None, None), jmode=1, feq=1, sync=9)))
    ux2, uy2 = W.pulse_displacement(20, 27, 4.0, 2.0, 3.0, 1e-3, "rotation")
    out.append(("periodic_y", dict(nx=20, ny=27, lam=2.0, mu=1.0, et=(1, 2, 1, 1), ev=np.zeros(8), px=False,
                                   py=True, a0=0.9, steps=80, u=(ux2, uy2, None, None))))
    ux3, uy3 = W.pulse_displacement(18, 24, 9.0, 1.0, 2.5, 1e-3, "dilatation")
    out.append(("periodic_both", dict(nx=18, ny=24, lam=2.0, mu=1.0, et=None, ev=None, px=True, py=True, a0=0.8,
                                      steps=60, u=(ux3, uy3, None, None))))
    d = W.tension_square(33, a0_phi=0.999, horizon=0.1, sync_every=50)
    d.hole = (16.0, 16.0, 4.3)
    out.append(("hole_tension", dict(nx=33, ny=33, lam=d.lam, mu=d.mu, et=d.edge_type,
                                     ev=np.asarray(d.edge_value, float).ravel(), px=False, py=False, a0=d.a0_phi,
                                     steps=min(d.steps, 120), u=(np.zeros((33, 33)), np.zeros((33, 33)), None, None),
                                     hole=d.hole, loads=d.loads, sync=d.sync_every)))
    return out


def whole_geometry(c):
    import oracle as O

    if c.get("hole"):
        return O.disk_cells(c["nx"], c["ny"], *c["hole"], c["et"], c["ev"])
    if c["et"] is None:
        return None, None, None
    nt, bv = O.rect_bc(c["nx"], c["ny"], c["et"], c["ev"], periodic_x=c["px"], periodic_y=c["py"])
    return nt, bv, None


def engine_kw(c):
    return dict(periodic_x=c["px"], a0_phi=c["a0"], bc_feq_mode=c.get("feq", 0), bc_j_mode=c.get("jmode", 0),
                sync_every=c.get("sync", 0), loads=c.get("loads", ()))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    sys.path.insert(0, str(ROOT))
    sys.path.insert(0, str(ROOT / "tests"))
    import torch.distributed as dist

    from paper_2301_00228_gb300 import slab
    from test_slab_host import OracleSlab, cases, engine_kw, whole_geometry

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = {}
    for name, c in cases():
        nt, bv, cell = whole_geometry(c)
        p = slab.plan(c["ny"], world, rank, periodic_y=c["py"],
                      void_rows=None if nt is None else (nt == 3).any(axis=1))
        eng = OracleSlab(p, c["nx"], c["lam"], c["mu"], node_type=nt, bc_value=bv, cell=cell, **engine_kw(c))
        run = slab.SlabRun(eng, p, dist)
        run.init(*c["u"])
        done = 0
        for chunk in (1, 2, c["steps"] - 3):    # the exchange runs after every step, whatever the chunks
            run.step(chunk)
            done += chunk
        res[name] = (p.y0, p.y1, {k: run.read_owned(k) for k in FIELDS})
    out.put((rank, res))
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_equal_whole_lattice(world):
    import oracle as O

    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for pr in procs:
        pr.start()
    got = {}
    import queue
    import time

    deadline = time.time() + 600
    while len(got) < world and time.time() < deadline:
        try:
            rank, res = q.get(timeout=2)      # drain before joining: a child holding queued data cannot exit
            got[rank] = res
        except queue.Empty:
            if any(pr.exitcode not in (None, 0) for pr in procs):
                break
    for pr in procs:
        pr.join(timeout=60)
        if pr.is_alive():
            pr.kill()
    assert all(pr.exitcode == 0 for pr in procs) and len(got) == world, "a rank failed (its traceback is above)"
    for name, c in cases():
        nt, bv, cell = whole_geometry(c)
        whole = O.OracleLattice(c["nx"], c["ny"], c["lam"], c["mu"], periodic_x=c["px"], periodic_y=c["py"],
                                node_type=nt, bc_value=bv, cell=cell, **{k: v for k, v in engine_kw(c).items()
                                                                          if k not in ("periodic_x", "loads")})
        for kind, t_ramp, t_hold in c.get("loads", ()):
            whole.set_load(kind, t_ramp, t_hold)
        whole.init(*c["u"]).step(c["steps"])
        ids = {"ux": O.UX, "uy": O.UY, "vx": O.VX, "vy": O.VY, "phi": O.PHI, "psi": O.PSI, "f_phi": O.F_PHI,
               "f_psi": O.F_PSI}
        covered = 0
        for rank in range(world):
            y0, y1, fields = got[rank][name]
            covered += y1 - y0
            for k in FIELDS:
                want = whole.read(ids[k])[..., y0:y1, :]
                assert np.array_equal(fields[k], want), (name, world, rank, k)
        assert covered == c["ny"]
        assert np.abs(whole.read(O.UX)).max() > 0


def test_plan_rows():
    from paper_2301_00228_gb300 import slab

    for ny, world, py in ((31, 3, False), (24, 2, True), (100, 7, False), (9, 3, True)):
        plans = [slab.plan(ny, world, r, periodic_y=py) for r in range(world)]
        assert plans[0].y0 == 0 and plans[-1].y1 == ny
        for a, b in zip(plans, plans[1:]):
            assert a.y1 == b.y0
        for pl in plans:
            assert pl.y1 - pl.y0 >= slab.HALO
            assert pl.lo == (slab.HALO if (pl.rank > 0 or py) else 0)
            assert pl.hi == (slab.HALO if (pl.rank < world - 1 or py) else 0)
            g = pl.global_rows()
            assert g[pl.lo] == pl.y0 and g[pl.rows - pl.hi - 1] == pl.y1 - 1
    with pytest.raises(ValueError):
        slab.plan(8, 3, 0)
    # a hole across the middle rows moves the cut clear of them
    void = np.zeros(40, bool)
    void[17:24] = True
    c = slab.cuts(40, 2, void)[0]
    assert not void[c - slab.HALO - 2:c + slab.HALO + 2].any()
    one = slab.plan(10, 1, 0, periodic_y=True)
    assert (one.lo, one.hi, one.rows) == (0, 0, 10)


def test_slab_description_fake_edges():
    import oracle as O
    from paper_2301_00228_gb300 import slab

    nt, bv = O.rect_bc(12, 20, (2, 1, 1, 2), np.arange(8) * 1e-4)
    p = slab.plan(20, 3, 1)
    snt, sbv, _ = slab.slab_description(p, 12, nt, bv)
    assert snt.shape == (p.rows, 12)
    assert np.all(snt[0] != 0) and np.all(snt[-1] != 0)        # fake edges
    assert np.array_equal(snt[1:-1], nt[p.first + 1:p.first + p.rows - 1])
    assert np.all(sbv[0, 1:-1] == 0) and np.all(sbv[-1, 1:-1] == 0)
    assert snt[0, 0] == 2 and snt[0, -1] == 1                   # left Dirichlet, right Neumann edges kept
