"""Seeded synthetic inputs for the plane-strain LBM.

This module only draws and samples initial displacement fields and boundary
descriptions.  It contains none of the method's arithmetic, so both the CUDA
path and the CPU oracle can take their inputs from it.

Recipes (lattice units, dh = 1):

* Gaussian pulses of dilatation or rotation are given through the exactly
  irrotational / solenoidal displacement fields
  ``u = A sigma^2 (1 - exp(-r^2 / (2 sigma^2))) / r`` along ``e_r`` (pure
  dilatation, div u = A exp(-r^2/(2 sigma^2)), curl u = 0) or along
  ``e_theta`` (pure rotation), sampled at the lattice points, u = 0 at r = 0.
* Plane waves on periodic lattices use integer wave numbers (m, n) so that
  they are periodic; the dilatational part points along k, the shear part
  along k rotated by 90 degrees.  Started at rest they are standing waves.
* Random rectangles draw each edge Dirichlet or Neumann with values in
  U(-1e-3, 1e-3)^2 and lambda/mu from U(0.5, 4) with mu = rho = 1.
* A plate with a hole is described by its rectangle, edges and the hole's
  centre and radius only; its node types and boundary cells are the
  method's preprocessing and are computed by the library or the oracle.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

NEUMANN, DIRICHLET = 1, 2
EDGES = ("bottom", "right", "top", "left")


def pulse_displacement(nx, ny, cx, cy, sigma, amp, kind="dilatation", dh=1.0, x0=0, y0=0):
    """Displacement of one Gaussian pulse centred at (cx, cy) (lattice coordinates),
    sampled on the nx x ny window whose first point is (x0, y0)."""
    x = (np.arange(x0, x0 + nx, dtype=np.float64) - cx) * dh
    y = (np.arange(y0, y0 + ny, dtype=np.float64) - cy) * dh
    X, Y = np.meshgrid(x, y)
    r = np.hypot(X, Y)
    s = sigma * dh
    with np.errstate(invalid="ignore", divide="ignore"):
        g = amp * s * s * (-np.expm1(-r * r / (2.0 * s * s))) / r
        g = np.where(r > 0.0, g / np.where(r > 0.0, r, 1.0), 0.0)  # g(r)/r
    if kind == "dilatation":
        return g * X, g * Y
    if kind == "rotation":
        return -g * Y, g * X
    raise ValueError(kind)


def bump_displacement(nx, ny, cx, cy, radius, amp, kind="dilatation", x0=0, y0=0):
    """A displacement bump of compact support centred at (cx, cy): magnitude
    amp (r/R)(1 - (r/R)^2)^3 for r < R = radius, zero beyond, along e_r
    (dilatation) or e_theta (rotation); sampled on the nx x ny window whose
    first point is (x0, y0)."""
    x = np.arange(x0, x0 + nx, dtype=np.float64) - cx
    y = np.arange(y0, y0 + ny, dtype=np.float64) - cy
    X, Y = np.meshgrid(x, y)
    q = np.hypot(X, Y) / radius
    g = np.where(q < 1.0, amp * (1.0 - q * q) ** 3, 0.0) / radius  # magnitude / r
    if kind == "dilatation":
        return g * X, g * Y
    if kind == "rotation":
        return -g * Y, g * X
    raise ValueError(kind)


def plane_wave_displacement(nx, ny, m, n, amp_d, amp_s):
    """u = amp_d khat sin(k.x) + amp_s khat_perp sin(k.x), k = 2 pi (m/nx, n/ny)."""
    kx, ky = 2.0 * math.pi * m / nx, 2.0 * math.pi * n / ny
    kn = math.hypot(kx, ky)
    ex, ey = kx / kn, ky / kn
    x = np.arange(nx, dtype=np.float64)
    y = np.arange(ny, dtype=np.float64)
    X, Y = np.meshgrid(x, y)
    ph = np.sin(kx * X + ky * Y)
    ux = (amp_d * ex - amp_s * ey) * ph
    uy = (amp_d * ey + amp_s * ex) * ph
    return ux, uy


def pick_wave_numbers(size, wavelength, rng):
    """Integer (m, n) whose |k| is nearest 2 pi / wavelength, at a random angle."""
    target = size / wavelength
    theta = rng.uniform(0.0, 2.0 * math.pi)
    m = int(round(target * math.cos(theta)))
    n = int(round(target * math.sin(theta)))
    best = None
    for dm in range(-2, 3):
        for dn in range(-2, 3):
            mm, nn = m + dm, n + dn
            if mm == 0 and nn == 0:
                continue
            err = abs(math.hypot(mm, nn) - target) + 1e-3 * abs(math.atan2(nn, mm) - theta)
            if best is None or err < best[0]:
                best = (err, mm, nn)
    return best[1], best[2]


@dataclass
class Domain:
    """A rectangular solve: sizes, material, boundary description, initial u."""
    nx: int
    ny: int
    lam: float
    mu: float
    rho: float = 1.0
    a0_phi: float = 0.9999
    periodic_x: bool = False
    periodic_y: bool = False
    edge_type: tuple = (NEUMANN, NEUMANN, NEUMANN, NEUMANN)
    edge_value: tuple = ((0.0, 0.0),) * 4
    pulses: list = field(default_factory=list)     # (cx, cy, sigma, amp, kind)
    wave: tuple | None = None                      # (m, n, amp_d, amp_s)
    steps: int = 0
    loads: tuple = ()                              # (kind, t_ramp, t_hold): ramped boundary data
    sync_every: int = 0
    hole: tuple | None = None                      # (cx, cy, r): traction-free circular hole

    def displacement(self, window=None):
        """u(x, 0) on the whole lattice, or on window = (x0, y0, w, h)."""
        x0, y0, w, h = window if window is not None else (0, 0, self.nx, self.ny)
        ux = np.zeros((h, w))
        uy = np.zeros((h, w))
        for (cx, cy, sg, amp, kind) in self.pulses:
            dx, dy = pulse_displacement(w, h, cx, cy, sg, amp, kind, x0=x0, y0=y0)
            ux += dx
            uy += dy
        if self.wave is not None:
            if window is not None:
                raise ValueError("plane waves are sampled on the whole lattice")
            dx, dy = plane_wave_displacement(self.nx, self.ny, *self.wave)
            ux += dx
            uy += dy
        return ux, uy

    def displacement_torch(self, device="cuda", rows=None):
        """u(x, 0) as FP64 torch tensors on ``device`` (same recipe as
        displacement()); ``rows`` = (first, count): only those rows (wrapped
        modulo ny, e.g. the rows of one slab of the lattice)."""
        import torch

        x = torch.arange(self.nx, dtype=torch.float64, device=device)
        if rows is None:
            y = torch.arange(self.ny, dtype=torch.float64, device=device)
        else:
            if self.wave is not None:
                raise ValueError("plane waves are sampled on the whole lattice")
            y = torch.remainder(torch.arange(rows[0], rows[0] + rows[1], device=device), self.ny).to(torch.float64)
        ux = torch.zeros((y.numel(), self.nx), dtype=torch.float64, device=device)
        uy = torch.zeros_like(ux)
        for (cx, cy, sg, amp, kind) in self.pulses:
            X = (x - cx)[None, :]
            Y = (y - cy)[:, None]
            r = torch.hypot(X, Y)
            g = amp * sg * sg * (-torch.expm1(-r * r / (2.0 * sg * sg)))
            g = torch.where(r > 0, g / torch.where(r > 0, r * r, torch.ones_like(r)), torch.zeros_like(r))
            if kind == "dilatation":
                ux += g * X
                uy += g * Y
            else:
                ux -= g * Y
                uy += g * X
        if self.wave is not None:
            dx, dy = plane_wave_displacement(self.nx, self.ny, *self.wave)
            ux += torch.from_numpy(dx).to(device)
            uy += torch.from_numpy(dy).to(device)
        return ux, uy

    def edge_arrays(self):
        return (np.asarray(self.edge_type, np.int32),
                np.asarray(self.edge_value, np.float64).reshape(4, 2))


def square_64():
    """64 x 64, lambda = mu = rho = 1, left edge clamped (u* = 0), others
    traction-free, centred dilatation pulse sigma = 4 cells, amplitude 1e-3,
    1000 steps."""
    return Domain(64, 64, 1.0, 1.0, edge_type=(NEUMANN, NEUMANN, NEUMANN, DIRICHLET),
                  pulses=[(31.5, 31.5, 4.0, 1e-3, "dilatation")], steps=1000)


def periodic_waves(size=1024, seed=2, wavelength=64.0, amp=1e-3, steps=10000):
    """Periodic size x size lattice, lambda/mu = 2, superposed dilatational and
    shear standing plane waves along a seeded direction."""
    rng = np.random.default_rng(seed)
    m, n = pick_wave_numbers(size, wavelength, rng)
    return Domain(size, size, 2.0, 1.0, periodic_x=True, periodic_y=True,
                  wave=(m, n, amp, amp), steps=steps)


def random_rectangle(rng, side_lo=64, side_hi=512, steps=2000, sigma=4.0, amp=1e-3):
    """One rectangle of the mixed-size batch: sides U{lo..hi}, random edges,
    lambda/mu in U(0.5, 4), one pulse at a random point."""
    nx = int(rng.integers(side_lo, side_hi + 1))
    ny = int(rng.integers(side_lo, side_hi + 1))
    et = tuple(int(x) for x in rng.choice([NEUMANN, DIRICHLET], size=4))
    ev = tuple((float(a), float(b)) for a, b in rng.uniform(-1e-3, 1e-3, size=(4, 2)))
    lam = float(rng.uniform(0.5, 4.0))
    cx = float(rng.integers(0, nx))
    cy = float(rng.integers(0, ny))
    kind = "dilatation" if rng.random() < 0.5 else "rotation"
    return Domain(nx, ny, lam, 1.0, edge_type=et, edge_value=ev,
                  pulses=[(cx, cy, sigma, amp, kind)], steps=steps)


def mixed_batch(count=256, seed=3, side_lo=64, side_hi=512, steps=2000):
    rng = np.random.default_rng(seed)
    return [random_rectangle(rng, side_lo, side_hi, steps) for _ in range(count)]


def many_pulses(size=8192, seed=4, count=32, steps=5000, amp=1e-3):
    """size x size, lambda/mu = 3, clamped bottom edge, traction-free others,
    32 random dilatation/rotation pulses with sigma in U(8, 64)."""
    rng = np.random.default_rng(seed)
    pulses = []
    for _ in range(count):
        kind = "dilatation" if rng.random() < 0.5 else "rotation"
        sg = float(rng.uniform(8.0, 64.0))
        cx, cy = (float(v) for v in rng.uniform(0, size - 1, size=2))
        pulses.append((cx, cy, sg, amp, kind))
    return Domain(size, size, 3.0, 1.0, edge_type=(DIRICHLET, NEUMANN, NEUMANN, NEUMANN),
                  pulses=pulses, steps=steps)


def crop(domain: Domain, x0, y0, w, h):
    """A w x h window of ``domain`` with the same boundary types on its edges and
    the pulses whose centres fall inside (re-centred)."""
    pulses = [(cx - x0, cy - y0, sg, amp, kind) for (cx, cy, sg, amp, kind) in domain.pulses
              if x0 <= cx < x0 + w and y0 <= cy < y0 + h]
    return Domain(w, h, domain.lam, domain.mu, domain.rho, domain.a0_phi,
                  edge_type=domain.edge_type, edge_value=domain.edge_value, pulses=pulses,
                  steps=domain.steps)


def tension_square(n=64, a0_phi=0.9999, horizon=1.0, sync_every=50):
    """Sec. 4, tension: an n x n square (lambda = mu, so c_s / c_d = 1/sqrt(3);
    rho = 1, dh = 1, side L = n - 1), traction t* = +-sigma_0(t) e_y on the
    top and bottom edges, the others traction-free.  sigma_0 rises linearly
    from 0 to 0.005 mu at t = L / c_s and is held; the body starts at rest.
    steps covers horizon x L / c_s.  The paper runs this example without
    synchronisation; with the boundary stencils read here its free corners
    then grow (about x20 per 10 dh / c_s), so the default synchronises every
    50 steps as the paper's other examples do (0 restores the paper's run)."""
    mu, lam = 1.0, 1.0
    L, cs, cd = n - 1.0, math.sqrt(mu), math.sqrt(lam + 2.0 * mu)
    T = L / cs
    dt = math.sqrt(2.0 * (1.0 - a0_phi) / 4.0) / cd
    s0 = 0.005 * mu
    return Domain(n, n, lam, mu, a0_phi=a0_phi, edge_type=(NEUMANN, NEUMANN, NEUMANN, NEUMANN),
                  edge_value=((0.0, -s0), (0.0, 0.0), (0.0, s0), (0.0, 0.0)),
                  loads=((NEUMANN, T, T),), steps=int(round(horizon * T / dt)), sync_every=sync_every)


def shear_square(n=64, a0_phi=0.9999, horizon=1.0, sync_every=50):
    """Sec. 4, simple shear: the same square, the top edge loaded by the
    shear traction sigma_0 = 0.005 mu t c_s / L (a ramp without hold), the
    bottom edge clamped (u* = 0), the sides traction-free; synchronisation
    every 50 steps."""
    mu, lam = 1.0, 1.0
    L, cs, cd = n - 1.0, math.sqrt(mu), math.sqrt(lam + 2.0 * mu)
    T = L / cs
    dt = math.sqrt(2.0 * (1.0 - a0_phi) / 4.0) / cd
    s0 = 0.005 * mu
    return Domain(n, n, lam, mu, a0_phi=a0_phi, edge_type=(DIRICHLET, NEUMANN, NEUMANN, NEUMANN),
                  edge_value=((0.0, 0.0), (0.0, 0.0), (s0, 0.0), (0.0, 0.0)),
                  loads=((NEUMANN, T, math.inf),), steps=int(round(horizon * T / dt)), sync_every=sync_every)


# ------------------------------------------------ plate with a circular hole

def hole_square(n=64, a0_phi=0.9999, horizon=1.0, sync_every=50):
    """Sec. 4, plate with a hole: the tension square of tension_square with
    a traction-free circular hole of diameter 0.266 L at its centre (taken
    centred; the text places the probe point Q at (-0.175 L, 0.025 L) from the
    hole's centre), synchronised every 50 steps as in the paper.  The hole is
    described by ``Domain.hole`` = (centre x, centre y, radius) in lattice
    units; the node types and boundary cells are the method's preprocessing
    and are built from it by the library (lbps_disk_cells) or the oracle."""
    d = tension_square(n, a0_phi=a0_phi, horizon=horizon, sync_every=sync_every)
    L = n - 1.0
    d.hole = (0.5 * L, 0.5 * L, 0.5 * 0.266 * L)
    return d


def busiest_crop(domain: Domain, side):
    """Origin (x0, y0) of the side x side window holding the most pulse
    centres (windows start on a grid of side / 4; the first in row-major
    order among equals).  With ``crop`` it makes a stand-alone problem of the
    same kind: the domain's edge types on the window's edges, the pulses
    centred inside."""
    step = max(1, side // 4)
    best = None
    for y0 in range(0, domain.ny - side + 1, step):
        for x0 in range(0, domain.nx - side + 1, step):
            n = sum(1 for (cx, cy, *_r) in domain.pulses if x0 <= cx < x0 + side and y0 <= cy < y0 + side)
            if best is None or n > best[0]:
                best = (n, x0, y0)
    return best[1], best[2]


def poisson_requests(count=10000, seed=5, rate_hz=1.0, side_lo=128, side_hi=2048, steps_lo=500,
                     steps_hi=20000):
    """Arrival times and domains of a serving stream: Poisson arrivals at
    rate_hz, sides log-uniform in [side_lo, side_hi] (independent nx, ny), step
    counts uniform in [steps_lo, steps_hi], edges, lambda/mu and one pulse
    drawn as in random_rectangle."""
    rng = np.random.default_rng(seed)
    t = np.cumsum(rng.exponential(1.0 / rate_hz, size=count))
    out = []
    for k in range(count):
        nx = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        ny = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
        et = tuple(int(x) for x in rng.choice([NEUMANN, DIRICHLET], size=4))
        ev = tuple((float(a), float(b)) for a, b in rng.uniform(-1e-3, 1e-3, size=(4, 2)))
        lam = float(rng.uniform(0.5, 4.0))
        kind = "dilatation" if rng.random() < 0.5 else "rotation"
        pulse = (float(rng.integers(0, nx)), float(rng.integers(0, ny)), 4.0, 1e-3, kind)
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        out.append((float(t[k]), Domain(nx, ny, lam, 1.0, edge_type=et, edge_value=ev, pulses=[pulse],
                                        steps=steps)))
    return out
