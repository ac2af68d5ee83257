"""Pins of the oracle's boundary cells for a plate with a circular hole
(reading R16; Sec. 3 preprocessing, Sec. 3.1.1 Eq. acc_neumann), and the
library's own cells against them (host code, no GPU).

The oracle computes a cell's area by Green's theorem along the clipped
boundary; the library integrates the disk column by column.  The pins here
are independent of both: hand-derived closed forms (tests/golden), the
tiling of the body by all points' cells, the closure of every cell boundary
(the outward normal integrates to zero), symmetry, and brute-force area by
sampling.
"""
import json
import math
from pathlib import Path

import numpy as np
import pytest

import oracle as O

GOLDEN = json.loads((Path(__file__).parent / "golden" / "disk_cells.json").read_text())
SIDES = ("l_E", "l_N", "l_W", "l_S")


def test_hand_cell_of_lattice():
    c = GOLDEN["lattice_case"]
    nt, bv, cell = O.disk_cells(c["nx"], c["ny"], *c["centre"], c["radius"], (1, 1, 1, 1), np.zeros(8),
                                dh=c["dh"])
    void = np.zeros((c["ny"], c["nx"]), bool)
    void[4:7, 4:7] = True
    assert np.array_equal(nt == 3, void)
    i, j = c["point"]
    assert nt[j, i] == 1
    want = c["expected"]
    got = cell[j, i]
    assert got[0] == pytest.approx(want["V_C"], abs=1e-15)
    for q, k in enumerate(SIDES):
        assert got[1 + q] == pytest.approx(want[k], abs=1e-15), k
    assert np.all(bv == 0.0)                                   # traction-free plate


@pytest.mark.parametrize("case", GOLDEN["clip_cases"], ids=lambda c: c["name"])
def test_hand_clip_cases(case):
    area, sides = O.clip_rect(*case["rect"], *case["centre"], case["radius"])
    want = case["expected"]
    assert area == pytest.approx(want["area"], abs=1e-14)
    for q, k in enumerate(SIDES):
        assert sides[q] == pytest.approx(want[k], abs=1e-14), k


def _square(x, y, h, Lx, Ly):
    return max(x - h / 2, 0.0), min(x + h / 2, Lx), max(y - h / 2, 0.0), min(y + h / 2, Ly)


@pytest.mark.parametrize("nx,ny,cx,cy,r,dh", [(40, 33, 19.3, 16.1, 7.3, 1.0), (25, 30, 12.0, 15.0, 6.0, 1.0),
                                              (60, 50, 7.4, 6.3, 3.9, 0.5), (31, 31, 15.0, 15.0, 10.5, 0.25)])
def test_cells_tile_the_body(nx, ny, cx, cy, r, dh):
    """The clipped squares of all lattice points (interior, boundary and void)
    tile the body rectangle, so their areas outside the disk add up to the
    rectangle's area minus the disk's (the disk lies inside the rectangle)."""
    Lx, Ly = (nx - 1) * dh, (ny - 1) * dh
    cx, cy, r = cx * dh, cy * dh, r * dh
    assert cx - r > 0 and cx + r < Lx and cy - r > 0 and cy + r < Ly
    total = 0.0
    for j in range(ny):
        for i in range(nx):
            total += O.clip_rect(*_square(i * dh, j * dh, dh, Lx, Ly), cx, cy, r)[0]
    assert total == pytest.approx(Lx * Ly - math.pi * r * r, abs=1e-11 * Lx * Ly)


def _circle_hits(x0, x1, y0, y1, cx, cy, r):
    """Points where the circle crosses the boundary of the rectangle (solved
    side by side here, independently of the oracle)."""
    pts = []
    for X in (x0, x1):
        d = r * r - (X - cx) ** 2
        if d > 0:
            for s in (-1, 1):
                y = cy + s * math.sqrt(d)
                if y0 <= y <= y1:
                    pts.append((X, y))
    for Y in (y0, y1):
        d = r * r - (Y - cy) ** 2
        if d > 0:
            for s in (-1, 1):
                x = cx + s * math.sqrt(d)
                if x0 <= x <= x1:
                    pts.append((x, Y))
    return pts


def test_cell_boundary_closes():
    """For every cell the circle cuts once (two crossings of the square's
    boundary), the outward normal integrated over the cell boundary vanishes:
    sum over the square's sides of length x normal, plus the integral over
    the arc, which is the chord rotated by 90 degrees and points from the
    centre towards the chord (n of the cell points into the disk there)."""
    nx, ny, cx, cy, r, h = 40, 36, 19.37, 17.81, 9.13, 1.0
    Lx, Ly = (nx - 1) * h, (ny - 1) * h
    checked = 0
    E = np.array([[1, 0], [0, 1], [-1, 0], [0, -1]], float)
    for j in range(ny):
        for i in range(nx):
            sq = _square(i * h, j * h, h, Lx, Ly)
            hits = _circle_hits(*sq, cx, cy, r)
            if len(hits) != 2:
                continue
            (ax, ay), (bx, by) = hits
            chord = math.hypot(bx - ax, by - ay)
            if chord < 1e-3:     # near tangency the crossings are ill-conditioned (sqrt of a tiny number)
                continue
            area, sides = O.clip_rect(*sq, cx, cy, r)
            flux_sides = sides @ E
            mx, my = 0.5 * (ax + bx) - cx, 0.5 * (ay + by) - cy
            m = math.hypot(mx, my)
            flux_arc = -chord * np.array([mx / m, my / m])   # the cell's outward normal on the arc
            assert np.abs(flux_sides + flux_arc).max() <= 1e-13, (i, j, flux_sides, flux_arc)
            checked += 1
    assert checked > 40


def test_cell_area_against_sampling():
    """Areas against a brute-force midpoint count on a fine grid (error of
    the count about perimeter x spacing)."""
    rng = np.random.default_rng(7)
    n = 2000
    g = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(g, g)
    for _ in range(20):
        cx, cy = rng.uniform(-0.6, 1.6, 2)
        r = rng.uniform(0.2, 1.5)
        area, sides = O.clip_rect(0.0, 1.0, 0.0, 1.0, cx, cy, r)
        count = np.mean((X - cx) ** 2 + (Y - cy) ** 2 >= r * r)
        assert area == pytest.approx(count, abs=5e-3)
        # side lengths by the same sampling along each side
        for q, (xs, ys) in enumerate(((np.ones(n), g), (g, np.ones(n)), (np.zeros(n), g), (g, np.zeros(n)))):
            frac = np.mean((xs - cx) ** 2 + (ys - cy) ** 2 >= r * r)
            assert sides[q] == pytest.approx(frac, abs=2e-3), q


def test_centred_hole_cells_symmetric():
    """A hole centred in a square plate: the cells are mirror-symmetric in x
    (E and W sides swapped) and in y, and symmetric about the diagonal."""
    n = 41
    c = 20.0
    nt, bv, cell = O.disk_cells(n, n, c, c, 7.7, (1, 1, 1, 1), np.zeros(8))
    mx = cell[:, ::-1][..., [0, 3, 2, 1, 4]]
    my = cell[::-1, :][..., [0, 1, 4, 3, 2]]
    dg = np.transpose(cell, (1, 0, 2))[..., [0, 2, 1, 4, 3]]
    for other in (mx, my, dg):
        assert np.abs(cell - other).max() <= 1e-13
    assert np.array_equal(nt, nt[:, ::-1]) and np.array_equal(nt, nt.T)


def test_outer_edge_tractions():
    """Neumann points on the outer edges carry the edge traction times the
    length of their external faces: dh on an edge, dh/2 per edge at a corner
    (the rectangle rule), when the hole is far from the edges."""
    nx, ny = 30, 24
    ev = np.array([1e-4, -2e-4, 3e-4, 0.5e-4, -1e-4, 2e-4, 0.7e-4, -0.3e-4])
    nt, bv, cell = O.disk_cells(nx, ny, 14.0, 11.5, 4.0, (1, 1, 1, 1), ev)
    nt0, bv0 = O.rect_bc(nx, ny, (1, 1, 1, 1), ev)
    ring = np.zeros((ny, nx), bool)
    ring[[0, -1], :] = True
    ring[:, [0, -1]] = True
    assert np.array_equal(nt[ring], nt0[ring])
    assert np.abs(bv[ring] - bv0[ring]).max() <= 1e-19
    assert np.all(bv[~ring] == 0.0)
    # Dirichlet edges: the mean u* of the Dirichlet edges through a point
    nt2, bv2, _ = O.disk_cells(nx, ny, 14.0, 11.5, 4.0, (2, 1, 2, 1), ev)
    nt3, bv3 = O.rect_bc(nx, ny, (2, 1, 2, 1), ev)
    assert np.array_equal(nt2[ring], nt3[ring]) and np.abs(bv2[ring] - bv3[ring]).max() <= 1e-19


@pytest.mark.parametrize("seed", range(12))
def test_library_cells_equal_oracle(seed):
    """The library's cells (column integration) against the oracle's (Green's
    theorem): node types bit-exact, areas and lengths to rounding (about
    eps x the radius, the size of the terms that cancel)."""
    from paper_2301_00228_gb300 import lbps

    rng = np.random.default_rng(300 + seed)
    nx, ny = (int(v) for v in rng.integers(8, 70, 2))
    dh = float(rng.choice([1.0, 0.5, 0.125]))
    r = float(rng.uniform(0.0, min(nx, ny) / 2.5)) * dh
    cx, cy = float(rng.uniform(-4, nx + 4)) * dh, float(rng.uniform(-4, ny + 4)) * dh
    et = rng.choice([1, 2], 4)
    ev = rng.uniform(-1e-3, 1e-3, 8)
    a = lbps.lbps_disk_cells(nx, ny, dh, cx, cy, r, et, ev)
    b = O.disk_cells(nx, ny, cx, cy, r, et, ev, dh=dh)
    assert np.array_equal(a[0], b[0])
    tol = 1e-15 * max(1.0, r / dh) * 8
    assert np.abs(a[1] - b[1]).max() <= tol * 1e-3 * dh + 1e-19
    assert np.abs(a[2][..., 0] - b[2][..., 0]).max() <= tol * dh * dh
    assert np.abs(a[2][..., 1:] - b[2][..., 1:]).max() <= tol * dh


def test_library_cells_large_plate():
    """The plate of the benchmark's hole workload at 1024^2: both builders agree."""
    from paper_2301_00228_gb300 import lbps

    n = 1024
    L = n - 1.0
    ev = np.array([0, -5e-3, 0, 0, 0, 5e-3, 0, 0], float)
    a = lbps.lbps_disk_cells(n, n, 1.0, 0.5 * L, 0.5 * L, 0.133 * L, (1, 1, 1, 1), ev)
    b = O.disk_cells(n, n, 0.5 * L, 0.5 * L, 0.133 * L, (1, 1, 1, 1), ev)
    assert np.array_equal(a[0], b[0])
    assert np.abs(a[2] - b[2]).max() <= 1e-15 * 0.133 * L * 8
    assert np.abs(a[1] - b[1]).max() <= 1e-18


def test_library_rejects_bad_input():
    from paper_2301_00228_gb300 import lbps

    for args in ((2, 10, 1.0, 5, 5, 1), (10, 10, 0.0, 5, 5, 1), (10, 10, 1.0, 5, 5, -1), (10, 10, 1.0, np.nan, 5, 1)):
        with pytest.raises(lbps.LbpsError):
            lbps.lbps_disk_cells(*args, (1, 1, 1, 1), np.zeros(8))
    with pytest.raises(lbps.LbpsError):
        lbps.lbps_disk_cells(10, 10, 1.0, 5, 5, 1, (1, 3, 1, 1), np.zeros(8))


def test_points_on_the_circle_belong_to_the_body():
    """The hole is the open disk: lattice points exactly on the circle (radius
    2 through (3, 5), (7, 5), (5, 3), (5, 7)) are body points, with a cell of
    area 1 - (area of the square in the disk)."""
    nt, bv, cell = O.disk_cells(11, 11, 5.0, 5.0, 2.0, (1, 1, 1, 1), np.zeros(8))
    for i, j in ((3, 5), (7, 5), (5, 3), (5, 7)):
        assert nt[j, i] == 1
        assert 0.0 < cell[j, i, 0] < 1.0
    assert nt[5, 4] == 3 and nt[4, 4] == 3
