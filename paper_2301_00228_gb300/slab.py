"""One lattice split into slabs of rows, one slab per rank, with a ghost-row
exchange after every time step (a domain decomposition of the method's time
loop, Fig. 3; the paper only remarks that parallel computing is easy with
most LBMs, Sec. 1).

The plan.  Rank r of P owns rows [y0, y1) of the ny rows (as even as
possible).  Its lattice holds those rows and HALO = 3 ghost rows beyond each
cut to a neighbour (none beyond a non-periodic outer edge), so it has
y1 - y0 + 2 HALO rows in the middle of a non-periodic lattice.  The outermost
ghost row is made a traction-free edge of the slab's own lattice (a boundary
row the whole lattice does not have).  One step from a state that is right
everywhere but at that fake edge leaves wrong values only in the three ghost
rows:
  * the fake edge row itself (its accelerations, resets and stresses);
  * the next row: populations streamed from the fake edge, and u at its
    boundary points, whose Eq. acc_neumann reads stresses of the fake row;
  * the third row: at boundary points there, Eq. psi_phi_at_bound
    differentiates the wrong u of the second row, and the value they stream
    into their interior neighbour (Eq. LBE_mod) follows.
The owned rows read nothing else of the ghost rows, so they stay exact.
After the step each rank sends its three owned rows next to each cut to that
neighbour, which writes them over its ghost rows (lbps_halo_unpack also
recomputes the boundary stresses and mirror the library keeps with the
state); the whole slab is then right again except at the fake edge.  The
periodic synchronisation of Sec. 3.2 runs inside the step, before the
exchange, and keeps to the same rows.  The 16-bit formats also need the same
storage scale on every slab (the smallest exponent any slab chooses) and the
rounding key of the global rows (lbps_set_origin).

The exchange goes through torch.distributed (batch_isend_irecv): NCCL with
device buffers on GPUs, gloo with host buffers on CPU.  ``SlabRun`` is
written against a small engine interface (``make``, ``pack``, ``unpack``,
``empty``, ``step``, ``read``, ``scale_exp``) so the same plan and exchange
also drive other implementations of the step.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

HALO = 3
NEUMANN, DIRICHLET, VOID = 1, 2, 3


@dataclass
class SlabPlan:
    """Rows of one rank's slab of an nx x ny lattice split over `world` ranks."""
    rank: int
    world: int
    ny: int
    periodic_y: bool
    y0: int           # first owned row (global)
    y1: int           # one past the last owned row
    lo: int           # ghost rows below the owned ones
    hi: int           # ghost rows above

    @property
    def rows(self):
        return self.y1 - self.y0 + self.lo + self.hi

    @property
    def first(self):
        """Global row of the slab's row 0 (may be negative for a periodic lattice)."""
        return self.y0 - self.lo

    def global_rows(self):
        """Global row index of each slab row (wrapped on a periodic lattice)."""
        return [(self.first + j) % self.ny for j in range(self.rows)]

    @property
    def down(self):
        return (self.rank - 1) % self.world if self.lo else None

    @property
    def up(self):
        return (self.rank + 1) % self.world if self.hi else None

    # rows exchanged (slab coordinates)
    def send_down_rows(self):
        return self.lo, HALO            # owned rows next to the lower cut

    def send_up_rows(self):
        return self.rows - self.hi - HALO, HALO

    def recv_down_rows(self):
        return 0, HALO                  # ghost rows below

    def recv_up_rows(self):
        return self.rows - HALO, HALO


def cuts(ny, world, void_rows=None):
    """Row indices where slab k ends and slab k + 1 begins (world - 1 of them),
    as even as possible.  With ``void_rows`` (rows holding points outside the
    body, e.g. a hole), every cut moves to the nearest row whose ghost region
    with a margin, rows [c - HALO - 2, c + HALO + 2), holds none of them: a
    fake edge there has its one-sided differences inside the slab, and no
    point next to it changes from interior to boundary."""
    base, extra = divmod(ny, world)
    out = [(k + 1) * base + min(k + 1, extra) for k in range(world - 1)]
    if void_rows is None or not np.any(void_rows):
        return out
    bad = np.asarray(void_rows, bool)

    def clear(c):
        return not bad[max(c - HALO - 2, 0):min(c + HALO + 2, ny)].any()

    moved = []
    for c in out:
        for d in range(ny):
            cand = [x for x in (c - d, c + d) if HALO <= x <= ny - HALO and clear(x)]
            if cand:
                moved.append(cand[0])
                break
        else:
            raise ValueError("no cut position clear of void rows")
    return moved


def plan(ny, world, rank, periodic_y=False, void_rows=None):
    """Split ny rows over world ranks; every rank owns at least HALO rows.
    ``void_rows``: see ``cuts``."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("bad rank / world")
    if world > 1 and ny // world < HALO:
        raise ValueError(f"{ny} rows cannot be split over {world} slabs of at least {HALO} rows")
    c = [0] + cuts(ny, world, void_rows) + [ny]
    y0, y1 = c[rank], c[rank + 1]
    if any(b - a < HALO for a, b in zip(c, c[1:])):
        raise ValueError("a slab would own fewer than HALO rows")
    if world == 1:
        return SlabPlan(rank, world, ny, periodic_y, y0, y1, 0, 0)
    lo = HALO if (rank > 0 or periodic_y) else 0
    hi = HALO if (rank < world - 1 or periodic_y) else 0
    return SlabPlan(rank, world, ny, periodic_y, y0, y1, lo, hi)


def slab_description(p, nx, node_type=None, bc_value=None, cell=None, dh=1.0):
    """Node types, boundary values and cells of the slab's own lattice, cut
    from the whole lattice's (``node_type`` None: a lattice without boundary
    along y, i.e. only periodic in y, or fully periodic).  The fake edges
    (the outermost ghost rows beyond a cut) become traction-free Neumann
    points where they are not boundary points already; with explicit cells
    they get the cell of a straight edge."""
    rows = p.global_rows()
    ny = p.rows
    nt = np.zeros((ny, nx), np.uint8) if node_type is None else np.ascontiguousarray(node_type)[rows].copy()
    bv = np.zeros((ny, nx, 2)) if bc_value is None else np.ascontiguousarray(bc_value)[rows].copy()
    cl = None if cell is None else np.ascontiguousarray(cell)[rows].copy()
    fake = ([0] if p.lo else []) + ([ny - 1] if p.hi else [])
    for j in fake:
        body = nt[j] != VOID
        inner = body & (nt[j] == 0)
        nt[j, inner] = NEUMANN
        bv[j, inner] = 0.0
        if cl is not None:
            cl[j, inner] = (0.5 * dh * dh, dh / 2, 0.0 if j else dh, dh / 2, dh if j else 0.0)
    return nt, bv, cl


class SlabRun:
    """The time loop of one rank's slab: ``engine`` advances the slab's
    lattice and moves its rows; ``dist`` is torch.distributed (None for a
    single rank).  Call ``init`` with the whole lattice's initial fields (or
    just rows covering the slab, see ``take``), then ``step``."""

    def __init__(self, engine, p: SlabPlan, dist=None, group=None):
        self.e = engine
        self.p = p
        self.dist = dist
        self.group = group

    def take(self, a):
        """The slab's rows of a whole-lattice array [ny][nx] (or None)."""
        return None if a is None else np.ascontiguousarray(np.asarray(a)[self.p.global_rows()])

    def init(self, ux, uy, vx=None, vy=None):
        """Initial fields of the whole lattice ([ny][nx] arrays; v may be None)."""
        return self.init_rows(self.take(ux), self.take(uy), self.take(vx), self.take(vy))

    def init_rows(self, ux, uy, vx=None, vy=None):
        """As init with the slab's own rows (p.rows x nx, host or device arrays)."""
        self.e.init(ux, uy, vx, vy)
        if self.dist is not None and self.p.world > 1:
            # one storage scale for all slabs (16-bit formats): the smallest choice
            e = self.e.scale_exp()
            if e is not None:
                m = self.reduce_min(e)
                if m != e:
                    self.e.rescale(m)
                    self.e.init(ux, uy, vx, vy)
            self.exchange()
        return self

    def reduce_min(self, v):
        import torch

        t = torch.tensor([int(v)], dtype=torch.int64, device=self.e.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MIN, group=self.group)
        return int(t.item())

    def exchange(self):
        """Owned rows next to each cut to that neighbour, ghost rows from it.
        Phase 0: rows go up (send the upper owned rows, receive the lower
        ghost rows); phase 1: down.  The order is the same on every rank, so
        sends and receives between the same two ranks pair up even when the
        neighbour below is also the one above (two slabs, periodic)."""
        p, d = self.p, self.dist
        if d is None or p.world == 1:
            return
        ops, recvs = [], []
        for phase in (0, 1):
            if phase == 0:
                send, peer_s, recv, peer_r = p.send_up_rows(), p.up, p.recv_down_rows(), p.down
            else:
                send, peer_s, recv, peer_r = p.send_down_rows(), p.down, p.recv_up_rows(), p.up
            if peer_s is not None:
                ops.append(d.P2POp(d.isend, self.e.pack(*send), peer_s, self.group, tag=phase))
            if peer_r is not None:
                buf = self.e.empty(recv[1])
                ops.append(d.P2POp(d.irecv, buf, peer_r, self.group, tag=phase))
                recvs.append((recv, buf))
        if ops:
            for w in d.batch_isend_irecv(ops):
                w.wait()
        for (row0, rows), buf in recvs:
            self.e.unpack(row0, rows, buf)

    def step(self, n=1):
        for _ in range(int(n)):
            self.e.step(1)
            self.exchange()
        return self

    def read_owned(self, field):
        """The owned rows of a field: [y1 - y0][nx]."""
        a = self.e.read(field)
        return a[..., self.p.lo:self.p.rows - self.p.hi, :]


class CudaSlab:
    """Engine of SlabRun on the library: the slab is an ``lbps.Lattice`` on the
    current device; rows move through device buffers (lbps_halo_pack /
    lbps_halo_unpack)."""

    def __init__(self, p: SlabPlan, nx, lam, mu, rho=1.0, dh=1.0, node_type=None, bc_value=None, cell=None,
                 loads=(), **kw):
        import torch

        from . import lbps

        self.L, self.torch = lbps, torch
        self.p = p
        self.device = "cuda"
        nt, bv, cl = slab_description(p, nx, node_type, bc_value, cell, dh)
        self.args = dict(nx=nx, ny=p.rows, lam=lam, mu=mu, rho=rho, dh=dh,
                         periodic_y=p.periodic_y and p.world == 1, node_type=nt, bc_value=bv, cell=cl)
        self.kw = dict(kw)
        self.loads = tuple(loads)
        self._make()

    def _make(self):
        a = self.args
        # single steps: the ghost rows are exchanged after every step
        self.lat = self.L.Lattice(a["nx"], a["ny"], a["lam"], a["mu"], a["rho"], a["dh"],
                                  periodic_y=a["periodic_y"], node_type=a["node_type"], bc_value=a["bc_value"],
                                  cell=a["cell"], step_pairs=False, **self.kw)
        self.L.lbps_set_origin(self.lat._h, self.p.first)
        for kind, t_ramp, t_hold in self.loads:
            self.lat.set_load(kind, t_ramp, t_hold)

    def init(self, ux, uy, vx=None, vy=None):
        self.lat.init(ux, uy, vx, vy)

    def scale_exp(self):
        return self.lat.scale_exp if self.lat.storage in ("bf16", "f16", "bfp13") else None

    def rescale(self, e):
        self.lat.close()
        self.kw["pop_scale_exp"] = int(e)
        self._make()

    def empty(self, rows):
        n = self.L.lbps_halo_bytes(self.lat._h, rows)
        return self.torch.empty(n, dtype=self.torch.uint8, device="cuda")

    def pack(self, row0, rows):
        buf = self.empty(rows)
        self.L.lbps_halo_pack(self.lat._h, row0, rows, buf.data_ptr(), buf.numel())
        return buf

    def unpack(self, row0, rows, buf):
        self.L.lbps_halo_unpack(self.lat._h, row0, rows, buf.data_ptr(), buf.numel())

    def step(self, n):
        self.lat.step_async(n)

    def read(self, field):
        return self.lat.read(field)

    def close(self):
        self.lat.close()
