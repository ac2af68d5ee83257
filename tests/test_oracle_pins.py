"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Every check here is independent of the oracle's own code: closed forms of the
discrete scheme derived on paper, continuum solutions, invariants, patch
tests and brute force.  None of them re-types an oracle formula.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2301_00228_gb300 import workloads as W

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def periodic_lattice(nx, ny, lam=2.0, mu=1.0, rho=1.0, a0=0.6, **kw):
    return O.OracleLattice(nx, ny, lam, mu, rho, a0_phi=a0, periodic_x=True, periodic_y=True, **kw)


# --------------------------------------------------------------- constants

def test_constants_wave_speed_ratio():
    """Sec. 4 fixes c_s/c_d = 1/sqrt(3) for its examples; with c_d = sqrt((lambda+2mu)/rho)
    and c_s = sqrt(mu/rho) that is lambda = mu."""
    lat = periodic_lattice(8, 8, lam=1.0, mu=1.0, rho=2.5, a0=0.9999)
    assert lat.cs / lat.cd == pytest.approx(1.0 / math.sqrt(3.0), rel=1e-14)
    assert lat.cd == pytest.approx(math.sqrt(3.0 / 2.5), rel=1e-14)


def test_constants_parameter_rules():
    """Eq. feq_req and Eq. conditions-parameters: a0 + 4a = 1 for both sets, one time step
    for both wave speeds, CFL c_d dt/dh <= 1."""
    for lam, mu, a0 in ((1.0, 1.0, 0.9999), (3.0, 0.7, 0.5), (0.5, 2.0, 0.0)):
        lat = O.OracleLattice(6, 5, lam, mu, 1.3, dh=0.25, a0_phi=a0, periodic_x=True, periodic_y=True)
        assert a0 + 4 * lat.a_phi == pytest.approx(1.0, abs=1e-15)
        assert lat.a0_psi + 4 * lat.a_psi == pytest.approx(1.0, abs=1e-15)
        assert lat.a0_psi >= 0.0
        dt_phi = 0.25 / lat.cd * math.sqrt(2 * lat.a_phi)
        dt_psi = 0.25 / lat.cs * math.sqrt(2 * lat.a_psi)
        assert lat.dt == pytest.approx(dt_phi, rel=1e-14)
        assert lat.dt == pytest.approx(dt_psi, rel=1e-14)
        assert lat.cd * lat.dt / 0.25 <= 1.0


# ---------------------------------------------------- interior = leapfrog

def test_leapfrog_equivalence():
    """With tau = dt/2 and J = 0 initially, the interior LBE is the five-point leapfrog
    s^{n+1} = 2 s^n - s^{n-1} + 2a (sum of 4 neighbours - 4 s^n), s^1 = s^0 + a(...)
    (a property of the D2Q5 wave model; derived by eliminating the populations)."""
    rng = np.random.default_rng(11)
    nx, ny = 24, 20
    ux0, uy0 = rng.standard_normal((2, ny, nx)) * 1e-3
    lat = periodic_lattice(nx, ny, lam=2.0, mu=1.0, a0=0.55)
    lat.init(ux0, uy0)
    s0 = {"phi": lat.read(O.PHI), "psi": lat.read(O.PSI)}
    a = {"phi": lat.a_phi, "psi": lat.a_psi}

    def lap(g):
        return np.roll(g, 1, 0) + np.roll(g, -1, 0) + np.roll(g, 1, 1) + np.roll(g, -1, 1) - 4 * g

    lf = {k: [s0[k], s0[k] + a[k] * lap(s0[k])] for k in s0}
    for n in range(2, 41):
        for k in lf:
            lf[k].append(2 * lf[k][-1] - lf[k][-2] + 2 * a[k] * lap(lf[k][-1]))
    for n in range(1, 41):
        lat.step(1)
        for k, fid in (("phi", O.PHI), ("psi", O.PSI)):
            scale = np.abs(s0[k]).max()
            assert np.abs(lat.read(fid) - lf[k][n]).max() <= 1e-12 * scale, (k, n)


# ----------------------------------------------- discrete standing wave

def standing_wave_expected(nx, ny, m, n, amp_d, amp_s, lam, mu, rho, a_phi, a_psi, dt, steps):
    """Closed form of the scheme for a periodic plane wave started at rest.

    u0 = A sin(k.x).  Central differences of sin/cos give
        phi0 = Phi cos(k.x),  Phi = A_x sin kx + A_y sin ky,
        psi0 = Psi cos(k.x),  Psi = A_y sin kx - A_x sin ky,
    the leapfrog gives phi_n = Phi cos(n w_phi) cos(k.x) with cos w = 1 - 2a(2 - cos kx - cos ky),
    the acceleration c_d^2 grad phi - c_s^2 curl(psi e_z) is sin(k.x) (P C_phi(n) + Q C_psi(n)),
    and the Newmark recurrences are summed as scalar sequences.
    """
    kx, ky = 2 * math.pi * m / nx, 2 * math.pi * n / ny
    kn = math.hypot(kx, ky)
    ex, ey = kx / kn, ky / kn
    Ax, Ay = amp_d * ex - amp_s * ey, amp_d * ey + amp_s * ex
    Phi = Ax * math.sin(kx) + Ay * math.sin(ky)
    Psi = Ay * math.sin(kx) - Ax * math.sin(ky)
    cd2, cs2 = (lam + 2 * mu) / rho, mu / rho
    K = 2 - math.cos(kx) - math.cos(ky)
    w_phi = math.acos(1 - 2 * a_phi * K)
    w_psi = math.acos(1 - 2 * a_psi * K)
    # d/dx cos(k.x) -> -sin(k.x) sin kx ; d/dy -> -sin(k.x) sin ky
    P = np.array([-cd2 * Phi * math.sin(kx), -cd2 * Phi * math.sin(ky)])
    Q = np.array([cs2 * Psi * math.sin(ky), -cs2 * Psi * math.sin(kx)])
    Ut = np.array([Ax, Ay], dtype=float)
    Vt = np.zeros(2)
    for q in range(steps):
        acc = P * math.cos(q * w_phi) + Q * math.cos(q * w_psi)
        Ut = Ut + dt * Vt + 0.5 * dt * dt * acc
        Vt = Vt + dt * acc
    X, Y = np.meshgrid(np.arange(nx), np.arange(ny))
    ph = kx * X + ky * Y
    return {
        "phi": Phi * math.cos(steps * w_phi) * np.cos(ph),
        "psi": Psi * math.cos(steps * w_psi) * np.cos(ph),
        "ux": Ut[0] * np.sin(ph), "uy": Ut[1] * np.sin(ph),
        "vx": Vt[0] * np.sin(ph), "vy": Vt[1] * np.sin(ph),
    }


@pytest.mark.parametrize("m,n,amp_d,amp_s", [(2, 1, 1e-3, 0.0), (1, 3, 0.0, 1e-3), (3, 2, 1e-3, -7e-4)])
def test_standing_wave_closed_form(m, n, amp_d, amp_s):
    nx, ny, lam, mu, rho, steps = 48, 40, 2.0, 1.0, 1.0, 300
    lat = periodic_lattice(nx, ny, lam, mu, rho, a0=0.6)
    ux0, uy0 = W.plane_wave_displacement(nx, ny, m, n, amp_d, amp_s)
    lat.init(ux0, uy0).step(steps)
    ex = standing_wave_expected(nx, ny, m, n, amp_d, amp_s, lam, mu, rho, lat.a_phi, lat.a_psi,
                                lat.dt, steps)
    got = lat.fields()
    groups = (("phi", "psi"), ("ux", "uy"), ("vx", "vy"))
    for g in groups:
        scale = max(np.abs(ex[k]).max() for k in g)
        for k in g:
            assert np.abs(got[k] - ex[k]).max() <= 1e-11 * scale, k


@pytest.mark.parametrize("field,speed", [("phi", "cd"), ("psi", "cs")])
def test_wave_speeds(field, speed):
    """The discrete frequency of a long plane wave gives the paper's wave speeds
    c_d = sqrt((lambda+2mu)/rho), c_s = sqrt(mu/rho) within the O((k dh)^2) dispersion."""
    nx, ny, lam, mu, rho = 256, 3, 3.0, 1.0, 1.7
    lat = O.OracleLattice(nx, ny, lam, mu, rho, a0_phi=0.99, periodic_x=True, periodic_y=True)
    k = 2 * math.pi * 4 / nx
    if field == "phi":
        ux0, uy0 = W.plane_wave_displacement(nx, ny, 4, 0, 1e-3, 0.0)
        fid = O.PHI
    else:
        ux0, uy0 = W.plane_wave_displacement(nx, ny, 4, 0, 0.0, 1e-3)
        fid = O.PSI
    lat.init(ux0, uy0)
    s0 = lat.read(fid)[1]
    i0 = int(np.argmax(np.abs(s0)))
    series = [s0[i0]]
    for _ in range(400):
        lat.step(1)
        series.append(lat.read(fid)[1, i0])
    series = np.array(series) / series[0]
    # least-squares fit of cos(w n) over a frequency scan, refined
    ns = np.arange(len(series))
    ws = np.linspace(1e-4, 0.2, 20001)
    err = [np.sum((series - np.cos(w * ns)) ** 2) for w in ws]
    w = ws[int(np.argmin(err))]
    c_meas = w / (k * lat.dt)
    c_ref = math.sqrt((lam + 2 * mu) / rho) if speed == "cd" else math.sqrt(mu / rho)
    assert abs(c_meas / c_ref - 1) < 3e-3


# ------------------------------------------------------------ conservation

def test_conservation_periodic():
    """Periodic lattice: sum phi, sum psi and sum J are invariants of the LBE
    (sum_alpha of 2 f_eq - f is s, its first moment is J); sum du/dt is invariant
    because central differences telescope; sum u grows by dt * sum du/dt."""
    rng = np.random.default_rng(5)
    nx, ny = 32, 24
    ux0, uy0, vx0, vy0 = rng.standard_normal((4, ny, nx)) * 1e-3
    lat = periodic_lattice(nx, ny, lam=1.5, mu=0.8, a0=0.7)
    lat.init(ux0, uy0, vx0, vy0)

    def totals():
        fphi, fpsi = lat.read(O.F_PHI), lat.read(O.F_PSI)
        c = 1.0 / lat.dt
        return (fphi.sum(), fpsi.sum(), c * (fphi[1] - fphi[3]).sum(), c * (fphi[2] - fphi[4]).sum(),
                c * (fpsi[1] - fpsi[3]).sum(), c * (fpsi[2] - fpsi[4]).sum(),
                lat.read(O.VX).sum(), lat.read(O.VY).sum())

    t0 = totals()
    sx0, sy0 = lat.read(O.UX).sum(), lat.read(O.UY).sum()
    lat.step(100)
    t1 = totals()
    for a, b in zip(t0, t1):
        assert abs(a - b) <= 1e-13 * nx * ny * 1e-3 * max(1.0, 1.0 / lat.dt)
    assert lat.read(O.UX).sum() == pytest.approx(sx0 + 100 * lat.dt * t0[6], abs=1e-12)
    assert lat.read(O.UY).sum() == pytest.approx(sy0 + 100 * lat.dt * t0[7], abs=1e-12)


# -------------------------------------------------------------- patch tests

def linear_field(nx, ny, G, d=(0.0, 0.0)):
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    return d[0] + G[0][0] * X + G[0][1] * Y, d[1] + G[1][0] * X + G[1][1] * Y


def hooke(G, lam, mu):
    """sigma for the uniform displacement gradient G (Eq. strain in Eq. hooke)."""
    eps = 0.5 * (np.array(G) + np.array(G).T)
    return lam * np.trace(eps) * np.eye(2) + 2 * mu * eps


def assert_static(lat, ux0, uy0, steps=60, tol=1e-13):
    lat.step(steps)
    scale = max(np.abs(ux0).max(), np.abs(uy0).max(), 1e-3)
    assert np.abs(lat.read(O.UX) - ux0).max() <= tol * scale
    assert np.abs(lat.read(O.UY) - uy0).max() <= tol * scale
    assert np.abs(lat.read(O.VX)).max() <= tol * scale / lat.dt
    assert np.abs(lat.read(O.VY)).max() <= tol * scale / lat.dt


@pytest.mark.parametrize("mode", [0, 1])
def test_patch_rigid_motions(mode):
    """Rigid translation and infinitesimal rigid rotation of a traction-free body stay at rest."""
    nx, ny = 12, 9
    nt, bv = O.rect_bc(nx, ny, (1, 1, 1, 1), np.zeros(8))
    for G, d in (([[0, 0], [0, 0]], (3e-4, -2e-4)), ([[0, -5e-4], [5e-4, 0]], (0.0, 0.0))):
        ux0, uy0 = linear_field(nx, ny, G, d)
        lat = O.OracleLattice(nx, ny, 1.3, 0.9, a0_phi=0.8, node_type=nt, bc_value=bv, bc_feq_mode=mode)
        lat.init(ux0, uy0)
        assert_static(lat, ux0, uy0)


@pytest.mark.parametrize("mode", [0, 1])
def test_patch_uniform_strain_neumann(mode):
    """A uniform displacement gradient with tractions t* = sigma n on every edge is an
    equilibrium: finite differences are exact on linear fields and the traction of a
    constant stress over a closed cell sums to zero, corners included."""
    nx, ny, lam, mu = 11, 8, 2.0, 0.7
    G = [[4e-4, 1.5e-4], [-0.5e-4, -2e-4]]
    sig = hooke(G, lam, mu)
    normals = ((0, -1), (1, 0), (0, 1), (-1, 0))  # bottom, right, top, left
    ev = np.concatenate([sig @ np.array(n, float) for n in normals])
    nt, bv = O.rect_bc(nx, ny, (1, 1, 1, 1), ev)
    ux0, uy0 = linear_field(nx, ny, G, (1e-4, 0.0))
    lat = O.OracleLattice(nx, ny, lam, mu, a0_phi=0.9, node_type=nt, bc_value=bv, bc_feq_mode=mode)
    lat.init(ux0, uy0)
    assert_static(lat, ux0, uy0)


def test_patch_uniform_strain_mixed():
    """The same equilibrium with the left edge and its corners held by Dirichlet values."""
    nx, ny, lam, mu = 9, 10, 1.0, 1.0
    G = [[-3e-4, 2e-4], [1e-4, 5e-4]]
    sig = hooke(G, lam, mu)
    normals = ((0, -1), (1, 0), (0, 1), (-1, 0))
    ev = np.concatenate([sig @ np.array(n, float) for n in normals])
    nt, bv = O.rect_bc(nx, ny, (1, 1, 1, 2), ev)
    ux0, uy0 = linear_field(nx, ny, G)
    dmask = nt == 2
    bv[dmask, 0] = ux0[dmask]
    bv[dmask, 1] = uy0[dmask]
    assert dmask[:, 0].all() and dmask.sum() == ny
    lat = O.OracleLattice(nx, ny, lam, mu, a0_phi=0.9999, node_type=nt, bc_value=bv)
    lat.init(ux0, uy0)
    assert_static(lat, ux0, uy0)


def test_dirichlet_reaches_target():
    """Eq. acc_dirichlet is chosen so that Eq. integration lands on u* after every step."""
    rng = np.random.default_rng(3)
    nx, ny = 10, 7
    ev = rng.uniform(-1e-3, 1e-3, 8)
    nt, bv = O.rect_bc(nx, ny, (2, 2, 2, 2), ev)
    ux0, uy0 = rng.standard_normal((2, ny, nx)) * 1e-3
    lat = O.OracleLattice(nx, ny, 1.0, 1.0, a0_phi=0.9, node_type=nt, bc_value=bv)
    lat.init(ux0, uy0)
    d = nt == 2
    for _ in range(5):
        lat.step(1)
        assert np.abs(lat.read(O.UX)[d] - bv[d, 0]).max() <= 1e-15
        assert np.abs(lat.read(O.UY)[d] - bv[d, 1]).max() <= 1e-15
    # corner of two Dirichlet edges: mean of the two prescribed values (corner reading)
    assert bv[0, 0, 0] == pytest.approx(0.5 * (ev[0] + ev[6]))


# ------------------------------------------------------ continuum convergence

def slab_error(N, kind, a0, sync_every, ny=3, rho=1.0):
    """Slab 0 <= x <= L, periodic in y, first standing mode of the continuum solution
    of Eq. navier1: traction-free edges (u = A cos(pi x/L) along x for the dilatational
    wave, along y for the shear wave) or clamped edges (u_x = A sin(pi x/L))."""
    L = N - 1
    et = (2, 2, 2, 2) if kind == "clamped" else (1, 1, 1, 1)
    nt, bv = O.rect_bc(N, ny, et, np.zeros(8), periodic_y=True)
    lat = O.OracleLattice(N, ny, 1.0, 1.0, rho, a0_phi=a0, periodic_y=True, node_type=nt,
                          bc_value=bv, sync_every=sync_every)
    X = np.arange(N)[None, :] * np.ones((ny, 1))
    k = math.pi / L
    A = 1e-3
    if kind == "free_d":
        base, c, fid = np.cos(k * X), lat.cd, O.UX
        lat.init(A * base, 0 * X)
    elif kind == "free_s":
        base, c, fid = np.cos(k * X), lat.cs, O.UY
        lat.init(0 * X, A * base)
    else:
        base, c, fid = np.sin(k * X), lat.cd, O.UX
        lat.init(A * base, 0 * X)
    steps = int(round(0.5 * (2 * math.pi / (c * k)) / lat.dt))
    lat.step(steps)
    exact = A * base * math.cos(c * k * steps * lat.dt)
    return np.abs(lat.read(fid) - exact).max() / A


@pytest.mark.parametrize("kind,a0,sync,rho", [("free_d", 0.99, 1, 1.0), ("free_s", 0.99, 1, 1.0),
                                              ("free_d", 0.99, 1, 2.5), ("clamped", 0.5, 0, 1.0)])
def test_slab_convergence(kind, a0, sync, rho):
    """Half a period of the first slab mode converges to the continuum solution at first
    order in dh (the printed Newmark update is first order in the velocity).  Traction-free
    edges need the synchronisation of Sec. 3.2 (here every step); clamped edges do not."""
    sizes = (33, 65, 129) if kind == "clamped" else (17, 33, 65)
    errs = [slab_error(N, kind, a0, sync, rho=rho) for N in sizes]
    assert errs[-1] < 3e-2
    for a, b in zip(errs, errs[1:]):
        assert a / b > 1.7


# ------------------------------------------------------ linearity, symmetry

def test_linearity():
    """The scheme is linear in (u0, v0) for homogeneous boundary data."""
    nx, ny = 20, 16
    nt, bv = O.rect_bc(nx, ny, (2, 1, 1, 2), np.zeros(8))
    u1 = W.pulse_displacement(nx, ny, 7.0, 8.0, 3.0, 1e-3, "dilatation")
    u2 = W.pulse_displacement(nx, ny, 12.0, 6.0, 2.5, 7e-4, "rotation")

    def run(ux, uy):
        lat = O.OracleLattice(nx, ny, 1.7, 1.0, a0_phi=0.9, node_type=nt, bc_value=bv)
        return lat.init(ux, uy).step(40).fields()

    a, b = run(*u1), run(*u2)
    c = run(u1[0] + u2[0], u1[1] + u2[1])
    for k in c:
        scale = np.abs(c[k]).max()
        assert np.abs(c[k] - a[k] - b[k]).max() <= 1e-12 * scale, k


def test_mirror_symmetry():
    """A pulse centred on a mirror line of a symmetric problem keeps the mirror symmetry."""
    nx, ny = 21, 15
    nt, bv = O.rect_bc(nx, ny, (1, 2, 1, 2), np.zeros(8))
    ux0, uy0 = W.pulse_displacement(nx, ny, 10.0, 7.0, 3.0, 1e-3, "dilatation")
    lat = O.OracleLattice(nx, ny, 1.0, 1.0, a0_phi=0.8, node_type=nt, bc_value=bv)
    f = lat.init(ux0, uy0).step(60).fields()
    s = np.abs(f["ux"]).max()
    assert np.abs(f["ux"] + f["ux"][:, ::-1]).max() <= 1e-13 * s
    assert np.abs(f["ux"] - f["ux"][::-1, :]).max() <= 1e-13 * s
    assert np.abs(f["uy"] - f["uy"][:, ::-1]).max() <= 1e-13 * s
    assert np.abs(f["uy"] + f["uy"][::-1, :]).max() <= 1e-13 * s
    assert np.abs(f["phi"] - f["phi"][:, ::-1]).max() <= 1e-13 * np.abs(f["phi"]).max()


# -------------------------------------------------------------- synchronise

def test_sync_restores_consistency():
    """After the synchronisation of Sec. 3.2 the consistency error e of Sec. 4 vanishes and
    the first moments are unchanged."""
    nx, ny = 18, 14
    nt, bv = O.rect_bc(nx, ny, (1, 1, 2, 1), np.zeros(8))
    ux0, uy0 = W.pulse_displacement(nx, ny, 9.0, 6.0, 2.0, 1e-3, "rotation")
    lat = O.OracleLattice(nx, ny, 1.0, 1.0, a0_phi=0.7, node_type=nt, bc_value=bv)
    lat.init(ux0, uy0).step(25)
    assert lat.read(O.ERR).max() > 1e-9
    f0 = lat.read(O.F_PHI)
    lat.sync()
    assert lat.read(O.ERR).max() <= 1e-17
    f1 = lat.read(O.F_PHI)
    assert np.abs((f1[1] - f1[3]) - (f0[1] - f0[3])).max() <= 1e-18


def test_sync_every_matches_manual():
    nx, ny = 12, 10
    nt, bv = O.rect_bc(nx, ny, (1, 1, 1, 1), np.zeros(8))
    u = W.pulse_displacement(nx, ny, 5.0, 5.0, 2.0, 1e-3, "dilatation")
    a = O.OracleLattice(nx, ny, 1.0, 1.0, a0_phi=0.8, node_type=nt, bc_value=bv, sync_every=4).init(*u)
    b = O.OracleLattice(nx, ny, 1.0, 1.0, a0_phi=0.8, node_type=nt, bc_value=bv).init(*u)
    a.step(12)
    for _ in range(3):
        b.step(4).sync()
    fa, fb = a.fields(), b.fields()
    for k in fa:
        assert np.array_equal(fa[k], fb[k]), k


def test_initial_state_consistent():
    """Fig. 3 initialises phi, psi by finite differences of u, so e(x, 0) = 0."""
    nx, ny = 15, 13
    nt, bv = O.rect_bc(nx, ny, (2, 1, 1, 1), np.zeros(8))
    u = W.pulse_displacement(nx, ny, 6.0, 7.0, 2.0, 1e-3, "dilatation")
    lat = O.OracleLattice(nx, ny, 1.0, 1.0, node_type=nt, bc_value=bv).init(*u)
    assert lat.read(O.ERR).max() <= 1e-15 * 1e-3


def test_init_polynomial_exact():
    """Second-order differences (central and one-sided) are exact on quadratics, so the
    initial phi, psi equal the analytic divergence and curl everywhere, edges included."""
    nx, ny = 7, 6
    nt, bv = O.rect_bc(nx, ny, (1, 1, 1, 1), np.zeros(8))
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    ux = 1e-4 * (X * X - 2 * X * Y + 3 * Y)
    uy = 1e-4 * (0.5 * Y * Y + X * Y - X)
    lat = O.OracleLattice(nx, ny, 1.0, 1.0, node_type=nt, bc_value=bv).init(ux, uy)
    div = 1e-4 * ((2 * X - 2 * Y) + (Y + X))
    curl = 1e-4 * ((Y - 1) - (-2 * X + 3))
    assert np.abs(lat.read(O.PHI) - div).max() <= 1e-17
    assert np.abs(lat.read(O.PSI) - curl).max() <= 1e-17


def test_consistency_error_peaks_at_second_row():
    """Sec. 4 (tension example, Fig. 9): under a traction on the top and bottom edges the
    consistency error appears at the 'second row' points of the loaded edges.  The
    magnitude 4.3e-12 printed there cannot be reproduced (resolution not given)."""
    nx = ny = 33
    s0 = 5e-3
    ev = np.array([0, -s0, 0, 0, 0, s0, 0, 0], float)  # bottom -sigma0 e_y, top +sigma0 e_y
    nt, bv = O.rect_bc(nx, ny, (1, 1, 1, 1), ev)
    lat = O.OracleLattice(nx, ny, 1.0, 1.0, a0_phi=0.9999, node_type=nt, bc_value=bv)
    lat.init(np.zeros((ny, nx)), np.zeros((ny, nx))).step(3)
    e = lat.read(O.ERR)
    j, i = np.unravel_index(int(np.argmax(e)), e.shape)
    assert j in (1, ny - 2)


# ------------------------------------------------------------ rect helper

def test_rect_bc_types_and_values():
    nx, ny = 5, 4
    ev = np.array([1, 2, 3, 4, 5, 6, 7, 8], float)  # bottom, right, top, left
    nt, bv = O.rect_bc(nx, ny, (1, 2, 1, 1), ev, dh=0.5)
    expected_types = np.array([
        [1, 1, 1, 1, 2],
        [1, 0, 0, 0, 2],
        [1, 0, 0, 0, 2],
        [1, 1, 1, 1, 2]], np.uint8)
    assert np.array_equal(nt, expected_types)
    # Neumann edge point: t* times dh
    assert np.allclose(bv[0, 2], [0.5, 1.0])
    # Neumann-Neumann corner (bottom-left): half faces of both edges
    assert np.allclose(bv[0, 0], [0.25 * 1 + 0.25 * 7, 0.25 * 2 + 0.25 * 8])
    # Dirichlet right edge dominates its corners: u* of the right edge
    assert np.allclose(bv[0, 4], [3, 4]) and np.allclose(bv[3, 4], [3, 4])
    assert np.allclose(bv[1, 1], [0, 0])


def test_rect_bc_periodic():
    nt, bv = O.rect_bc(6, 5, (2, 0, 1, 0), np.array([1, 1, 0, 0, 2, 2, 0, 0.]), periodic_x=True)
    assert (nt[0] == 2).all() and (nt[-1] == 1).all() and (nt[1:-1] == 0).all()
    assert np.allclose(bv[-1], [2, 2])


def test_rejects_bad_masks():
    nt, bv = O.rect_bc(6, 5, (1, 1, 1, 1), np.zeros(8))
    nt[2, 2] = 1
    with pytest.raises(ValueError):
        O.OracleLattice(6, 5, 1.0, 1.0, node_type=nt, bc_value=bv)
    with pytest.raises(ValueError):
        O.OracleLattice(2, 5, 1.0, 1.0, periodic_x=True, periodic_y=True)


# ------------------------------------------- time-dependent boundary data

STATE_FIELDS = (O.UX, O.UY, O.VX, O.VY, O.F_PHI, O.F_PSI)


def _loaded_lattice(et, ev, a0=0.99):
    nt, bv = O.rect_bc(12, 10, et, ev)
    return O.OracleLattice(12, 10, 1.7, 1.0, a0_phi=a0, node_type=nt, bc_value=bv)


def _state(lat):
    return [lat.read(f).copy() for f in STATE_FIELDS]


@pytest.mark.parametrize("kind,et", [(1, (1, 1, 1, 1)), (2, (2, 1, 2, 1))])
@pytest.mark.parametrize("ramp,hold", [(7, 7), (5, 13), (9, 1e9)])
def test_load_ramp_superposition(kind, et, ramp, hold):
    """The scheme is linear and time-invariant in the boundary data, so from a
    body at rest the state after N steps under data s_n g is
    sum_n s_n (y_{N-n} - y_{N-n-1}), with y_m the state after m steps under
    constant data g.  The factor of step n is s(n dt) for Neumann forces and
    s((n+1) dt) for Dirichlet targets (reading R13); a wrong time index, a
    missing hold or a factor on the wrong kind of point breaks the identity."""
    ev = np.array([3e-4, -2e-4, 1e-4, 5e-4, -4e-4, 2e-4, 1.5e-4, -1e-4])
    # only the ramped kind carries data (the other kind's edges are traction-free)
    ev = np.where(np.repeat(np.asarray(et) == kind, 2), ev, 0.0)
    N = 24
    zero = np.zeros((10, 12))
    const = _loaded_lattice(et, ev).init(zero, zero)
    y = [_state(const)]
    for _ in range(N):
        const.step(1)
        y.append(_state(const))
    ramped = _loaded_lattice(et, ev).init(zero, zero)
    dt = ramped.dt
    ramped.set_load(kind, ramp * dt, hold * dt)
    ramped.step(N)
    got = _state(ramped)
    shift = 0 if kind == 1 else 1
    s = [min((n + shift) * dt, hold * dt) / (ramp * dt) for n in range(N)]
    for q, g in enumerate(got):
        want = sum(s[n] * (y[N - n][q] - y[N - n - 1][q]) for n in range(N))
        scale = max(np.abs(want).max(), 1e-300)
        assert np.abs(g - want).max() <= 1e-11 * scale, (STATE_FIELDS[q], np.abs(g - want).max() / scale)
    assert np.abs(got[0]).max() > 0


def test_load_ramp_only_scales_its_kind():
    """A schedule on one kind leaves the other kind's data constant: with
    Dirichlet edges only, a Neumann schedule changes nothing; t_ramp = 0
    restores constant data."""
    ev = np.array([3e-4, -2e-4, 1e-4, 5e-4, -4e-4, 2e-4, 1.5e-4, -1e-4])
    zero = np.zeros((10, 12))
    a = _loaded_lattice((2, 2, 2, 2), ev).init(zero, zero).step(15)
    b = _loaded_lattice((2, 2, 2, 2), ev).init(zero, zero)
    b.set_load(1, 4 * b.dt, 4 * b.dt).step(15)
    c = _loaded_lattice((2, 2, 2, 2), ev).init(zero, zero)
    c.set_load(2, 4 * c.dt).set_load(2, 0.0).step(15)
    for f in STATE_FIELDS:
        assert np.array_equal(a.read(f), b.read(f)) and np.array_equal(a.read(f), c.read(f))
    with pytest.raises(ValueError):
        a.set_load(3, 1.0)
    with pytest.raises(ValueError):
        a.set_load(1, -1.0)


# ------------------------------------------ general geometry (plate with hole)

def _hole_closure_force(nt, cell, sxx, syy, sxy):
    """Per boundary point, the traction of a uniform stress integrated over
    the cell's external boundary: by closure of the cell boundary, minus the
    stress times the sum of e_d l_d over its sides (reading R14)."""
    E = ((1, 0), (0, 1), (-1, 0), (0, -1))
    fx = np.zeros(nt.shape)
    fy = np.zeros(nt.shape)
    for q, (ex, ey) in enumerate(E):
        l = cell[..., 1 + q]
        fx -= (sxx * ex + sxy * ey) * l
        fy -= (sxy * ex + syy * ey) * l
    bv = np.stack([fx, fy], axis=-1)
    bv[nt != 1] = 0.0
    return bv


def test_hole_patch_uniform_strain():
    """A uniform strain in a plate with a hole, loaded on every boundary cell
    by the traction sigma n of the uniform stress, stays static: the
    one-sided differences at the hole are exact for a linear field, and the
    cell faces (with sigma_k on sides facing the hole) balance the external
    force exactly (readings R4, R14)."""
    nx, ny, lam, mu = 31, 27, 1.3, 1.0
    nt, _, cell = O.disk_cells(nx, ny, 14.6, 12.8, 4.4, (1, 1, 1, 1), np.zeros(8))
    exx, eyy, exy = 2e-4, -1e-4, 0.5e-4
    sxx = lam * (exx + eyy) + 2 * mu * exx
    syy = lam * (exx + eyy) + 2 * mu * eyy
    sxy = 2 * mu * exy
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    ux = exx * X + exy * Y
    uy = exy * X + eyy * Y
    ux[nt == 3] = 0.0
    uy[nt == 3] = 0.0
    bv = _hole_closure_force(nt, cell, sxx, syy, sxy)
    lat = O.OracleLattice(nx, ny, lam, mu, a0_phi=0.99, node_type=nt, bc_value=bv, cell=cell)
    lat.init(ux, uy).step(300)
    body = nt != 3
    assert np.abs(lat.read(O.UX) - ux)[body].max() <= 1e-13
    assert np.abs(lat.read(O.UY) - uy)[body].max() <= 1e-13
    assert np.abs(lat.read(O.UX)[~body]).max() == 0.0


def test_explicit_rectangle_cells_equal_default():
    """Cells from the general geometry generator on a rectangle without hole
    are the clipped squares of R6; given explicitly they give the same bits
    as the built-in rule."""
    nx, ny = 17, 13
    ev = np.array([1e-4, -2e-4, 0, 3e-4, -1e-4, 0, 2e-4, 1e-4])
    et = (1, 2, 1, 1)
    nt, bv, cell = O.disk_cells(nx, ny, -50.0, -50.0, 1.0, et, ev)
    nt0, bv0 = O.rect_bc(nx, ny, et, ev)
    assert np.array_equal(nt, nt0) and np.array_equal(bv, bv0)
    ux, uy = W.pulse_displacement(nx, ny, 7.0, 6.0, 2.5, 1e-3, "rotation")
    a = O.OracleLattice(nx, ny, 1.2, 1.0, a0_phi=0.99, node_type=nt, bc_value=bv).init(ux, uy).step(40)
    b = O.OracleLattice(nx, ny, 1.2, 1.0, a0_phi=0.99, node_type=nt, bc_value=bv, cell=cell).init(ux, uy).step(40)
    for f in (O.UX, O.UY, O.VX, O.VY, O.F_PHI, O.F_PSI):
        assert np.array_equal(a.read(f), b.read(f)), f


def test_hole_mirror_symmetry():
    """A centred hole and a centred dilatation pulse in a traction-free
    plate: the solution is mirror-symmetric in x and in y."""
    n = 33
    nt, bv, cell = O.disk_cells(n, n, 16.0, 16.0, 5.5, (1, 1, 1, 1), np.zeros(8))
    ux, uy = W.pulse_displacement(n, n, 16.0, 16.0, 6.0, 1e-3, "dilatation")
    ux[nt == 3] = 0.0
    uy[nt == 3] = 0.0
    lat = O.OracleLattice(n, n, 2.0, 1.0, a0_phi=0.999, node_type=nt, bc_value=bv, cell=cell).init(ux, uy)
    lat.step(400)
    gx, gy = lat.read(O.UX), lat.read(O.UY)
    scale = np.abs(gx).max()
    assert scale > 1e-5
    assert np.abs(gx + gx[:, ::-1]).max() <= 1e-12 * scale
    assert np.abs(gy - gy[:, ::-1]).max() <= 1e-12 * scale
    assert np.abs(gx - gx[::-1, :]).max() <= 1e-12 * scale
    assert np.abs(gx - gy.T).max() <= 1e-12 * scale                   # diagonal symmetry


def test_geometry_rejected_without_stencil():
    """A body point whose differences have no stencil (a one-point-thin
    ligament next to the hole) or a wrong node type makes the lattice
    invalid."""
    nx, ny = 12, 9
    nt, bv = O.rect_bc(nx, ny, (1, 1, 1, 1), np.zeros(8))
    bad = nt.copy()
    bad[:, 2] = 3            # void column: column 1 is left with one neighbour column (0)
    bad[:, 3] = 1
    bad[0, 2] = bad[-1, 2] = 3
    with pytest.raises(ValueError):
        O.OracleLattice(nx, ny, 1.0, 1.0, node_type=bad, bc_value=bv)
    wrong = nt.copy()
    wrong[4, 5] = 1          # an interior point marked Neumann
    with pytest.raises(ValueError):
        O.OracleLattice(nx, ny, 1.0, 1.0, node_type=wrong, bc_value=bv)


def test_hole_init_quadratic_exact():
    """Initialisation of a plate with a hole from a quadratic u: phi, psi by
    the differences of R4/R14 (one-sided three-point next to the hole) equal
    the exact divergence and curl at every body point."""
    nx, ny = 30, 26
    nt, bv, cell = O.disk_cells(nx, ny, 13.7, 12.2, 4.8, (1, 1, 1, 1), np.zeros(8))
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    ux = 1e-4 * (0.3 * X * X - 0.2 * X * Y + 0.1 * Y * Y + X)
    uy = 1e-4 * (-0.1 * X * X + 0.4 * X * Y - 0.25 * Y * Y + 2 * Y)
    div = 1e-4 * (0.6 * X - 0.2 * Y + 1) + 1e-4 * (0.4 * X - 0.5 * Y + 2)
    curl = 1e-4 * (-0.2 * X + 0.4 * Y) - 1e-4 * (-0.2 * X + 0.2 * Y)
    body = nt != 3
    lat = O.OracleLattice(nx, ny, 1.0, 1.0, node_type=nt, bc_value=bv, cell=cell).init(ux * body, uy * body)
    scale = np.abs(div).max()
    assert np.abs(lat.read(O.PHI) - div)[body].max() <= 1e-12 * scale
    assert np.abs(lat.read(O.PSI) - curl)[body].max() <= 1e-12 * scale
    assert np.abs(lat.read(O.PHI)[~body]).max() == 0.0


# ------------------------------------------ travelling wave from du/dt (R9)

@pytest.mark.parametrize("m,n,P", [(3, 2, (1e-3, 0.4e-3)), (1, -2, (-0.3e-3, 0.8e-3)), (2, 0, (0.0, 1e-3))])
def test_travelling_wave_from_initial_velocity(m, n, P):
    """Reading R9 (J_phi = -v, J_psi = (-v_y, v_x), in lattice units scaled by
    dt/dh) against a closed form of the discrete scheme.  On a periodic
    lattice with u0 = P sin(k.x) and du/dt(0) = Q cos(k.x):
      phi0 = (P.s) cos(k.x), psi0 = (s x P) cos(k.x), s = (sin kx, sin ky)
    (central differences).  The LBE's first step from f = f_eq(phi0, J) is
      phi1 = phi0 + a lap5(phi0) - div_c(Jbar) = phi0 cos(w) - div_c(Jbar),
    cos w = 1 - 2a(2 - cos kx - cos ky), and every later step is the
    five-point leapfrog.  With Jbar_phi = -dt Q cos(k.x), -div_c Jbar_phi =
    -dt (Q.s) sin(k.x), so phi_n = (P.s) cos(k.x - w_phi n) exactly when
    -dt (Q.s) = (P.s) sin(w_phi); likewise Jbar_psi = dt (-Q_y, Q_x) cos(k.x)
    gives psi_n = (s x P) cos(k.x - w_psi n) when -dt (s x Q) = (s x P) sin(w_psi).
    Q is chosen so: a pure travelling wave in both fields, which runs at
    w/(|k| dt) -> c_d, c_s.  A wrong sign of J_psi makes psi travel backwards,
    a wrong dt scaling mixes in the opposite wave; both fail here."""
    nx, ny, lam, mu, steps = 48, 40, 2.0, 1.0, 120
    lat = periodic_lattice(nx, ny, lam, mu, 1.0, a0=0.6)
    kx, ky = 2 * math.pi * m / nx, 2 * math.pi * n / ny
    s = np.array([math.sin(kx), math.sin(ky)])
    Pv = np.array(P, float)
    A_phi = float(Pv @ s)
    A_psi = float(s[0] * Pv[1] - s[1] * Pv[0])
    K = 2 - math.cos(kx) - math.cos(ky)
    w_phi = math.acos(1 - 2 * lat.a_phi * K)
    w_psi = math.acos(1 - 2 * lat.a_psi * K)
    sn = float(np.linalg.norm(s))
    shat, sperp = s / sn, np.array([-s[1], s[0]]) / sn
    q1 = -A_phi * math.sin(w_phi) / (lat.dt * sn)      # Q.s = q1 |s|
    q2 = -A_psi * math.sin(w_psi) / (lat.dt * sn)      # s x Q = q2 |s|
    Q = q1 * shat + q2 * sperp
    X, Y = np.meshgrid(np.arange(nx, dtype=float), np.arange(ny, dtype=float))
    ph = kx * X + ky * Y
    ux0, uy0 = Pv[0] * np.sin(ph), Pv[1] * np.sin(ph)
    vx0, vy0 = Q[0] * np.cos(ph), Q[1] * np.cos(ph)
    lat.init(ux0, uy0, vx0, vy0)
    scale = max(abs(A_phi), abs(A_psi))
    for done in (1, 2, 7, 40, steps):
        lat.step(done - lat.steps)
        assert np.abs(lat.read(O.PHI) - A_phi * np.cos(ph - w_phi * done)).max() <= 1e-12 * scale, ("phi", done)
        assert np.abs(lat.read(O.PSI) - A_psi * np.cos(ph - w_psi * done)).max() <= 1e-12 * scale, ("psi", done)


# ------------------------------------------- J of Eq. correction-f (R15)

def test_bc_j_mode_partial_stream():
    """Reading R15, bc_j_mode 1: after a step the boundary populations are
    f^0 = a0 s, f^alpha = a s + e_alpha.Jbar/2 (Eq. correction-f), so their
    first moment is the Jbar used; it must be the first moment of what the
    LBE streams into the point from its body neighbours (2 a s - f^opp there)
    with the point's own populations kept for directions from outside.  This
    evaluates that definition from the populations before the step.  (The
    reading is not pinned against the paper: it is one of two readings.)"""
    nx, ny = 9, 7
    rng = np.random.default_rng(5)
    et, ev = (1, 2, 1, 1), rng.uniform(-2e-4, 2e-4, 8)
    nt, bv = O.rect_bc(nx, ny, et, ev)
    ux, uy = rng.uniform(-1e-4, 1e-4, (2, ny, nx))
    lat = O.OracleLattice(nx, ny, 1.4, 1.0, a0_phi=0.9, node_type=nt, bc_value=bv, bc_j_mode=1)
    lat.init(ux, uy).step(6)
    a = {0: lat.a_phi, 1: lat.a_psi}
    before = {0: lat.read(O.F_PHI), 1: lat.read(O.F_PSI)}
    lat.step(1)
    after = {0: lat.read(O.F_PHI), 1: lat.read(O.F_PSI)}
    EX, EY, OPP = (0, 1, 0, -1, 0), (0, 0, 1, 0, -1), (0, 3, 4, 1, 2)
    checked = 0
    for set_ in (0, 1):
        f = before[set_]
        for j in range(ny):
            for i in range(nx):
                if nt[j, i] == 0:
                    continue
                g = [f[q, j, i] for q in range(5)]
                for q in range(1, 5):
                    si, sj = i - EX[q], j - EY[q]
                    if 0 <= si < nx and 0 <= sj < ny:
                        g[q] = 2 * a[set_] * f[:, sj, si].sum() - f[OPP[q], sj, si]
                jx, jy = g[1] - g[3], g[2] - g[4]
                h = after[set_][:, j, i]
                assert h[1] - h[3] == pytest.approx(jx, abs=1e-18), (set_, i, j)
                assert h[2] - h[4] == pytest.approx(jy, abs=1e-18), (set_, i, j)
                checked += 1
    assert checked == 2 * (2 * nx + 2 * (ny - 2))


@pytest.mark.parametrize("jmode", [0, 1])
def test_bc_j_mode_patch_static(jmode):
    """Both readings of J keep the uniform-strain patch test static (a body
    in equilibrium has J = 0 everywhere, and so has every partial stream)."""
    nx, ny, lam, mu = 11, 8, 2.0, 0.7
    G = [[4e-4, 1.5e-4], [-0.5e-4, -2e-4]]
    sig = hooke(G, lam, mu)
    normals = ((0, -1), (1, 0), (0, 1), (-1, 0))
    ev = np.concatenate([sig @ np.array(nn, float) for nn in normals])
    nt, bv = O.rect_bc(nx, ny, (1, 1, 1, 1), ev)
    ux0, uy0 = linear_field(nx, ny, G, (1e-4, 0.0))
    lat = O.OracleLattice(nx, ny, lam, mu, a0_phi=0.9, node_type=nt, bc_value=bv, bc_j_mode=jmode)
    lat.init(ux0, uy0)
    assert_static(lat, ux0, uy0)


def test_bc_j_mode_changes_boundary_moments():
    """The two readings give different boundary populations once a wave has
    reached the boundary (so the parity cases of both modes test something)."""
    nx, ny = 21, 17
    nt, bv = O.rect_bc(nx, ny, (2, 1, 1, 1), np.zeros(8))
    ux, uy = W.pulse_displacement(nx, ny, 10.0, 8.0, 2.0, 1e-3, "dilatation")
    res = [O.OracleLattice(nx, ny, 1.0, 1.0, a0_phi=0.9, node_type=nt, bc_value=bv, bc_j_mode=jm)
           .init(ux, uy).step(40).read(O.F_PHI) for jm in (0, 1)]
    assert np.abs(res[0] - res[1]).max() > 1e-3 * np.abs(res[0]).max()


# ------------------------------------------------- energy densities (diagnostic)

def _closed_form_strain_energy(G, lam, mu):
    """Strain energy density of the uniform displacement gradient G (plane strain):
    eps = sym(G), W = lambda tr(eps)^2 / 2 + mu eps : eps, written out by hand."""
    exx, eyy = G[0][0], G[1][1]
    exy = 0.5 * (G[0][1] + G[1][0])
    return 0.5 * lam * (exx + eyy) ** 2 + mu * (exx * exx + eyy * eyy + 2.0 * exy * exy)


@pytest.mark.parametrize("geometry", ["rectangle", "hole"])
def test_energy_density_linear_fields(geometry):
    """For a linear displacement field the finite differences are exact at every
    body point (central and one-sided alike), so the strain energy density
    equals the closed form of the uniform strain everywhere, 0 at void points;
    an infinitesimal rigid rotation stores none (only the symmetric part of the
    gradient counts); a uniform velocity gives rho |v|^2 / 2 at every body point."""
    nx, ny, lam, mu, rho = 23, 19, 1.7, 0.8, 1.3
    if geometry == "rectangle":
        nt, bv = O.rect_bc(nx, ny, (2, 1, 1, 1), np.zeros(8))
        cell = None
    else:
        nt, bv, cell = O.disk_cells(nx, ny, 11.3, 9.6, 3.7, (1, 1, 1, 1), np.zeros(8))
    body = nt != 3
    G = [[3e-4, -1.2e-4], [2.1e-4, -0.7e-4]]
    ux, uy = linear_field(nx, ny, G, (1e-4, -2e-4))
    ux[~body] = 0.0
    uy[~body] = 0.0
    vx, vy = np.full((ny, nx), 2e-3), np.full((ny, nx), -1e-3)
    lat = O.OracleLattice(nx, ny, lam, mu, rho, node_type=nt, bc_value=bv, cell=cell)
    lat.init(ux, uy, vx, vy)
    w = lat.read(O.ESTRAIN)
    want = _closed_form_strain_energy(G, lam, mu)
    assert want > 0
    assert np.abs(w[body] - want).max() <= 1e-12 * want
    assert np.all(w[~body] == 0.0)
    k = lat.read(O.EKIN)
    assert np.abs(k[body] - 0.5 * rho * (4e-6 + 1e-6)).max() <= 1e-18
    assert np.all(k[~body] == 0.0)
    rot = [[0.0, -4e-4], [4e-4, 0.0]]
    rx, ry = linear_field(nx, ny, rot)
    rx[~body] = 0.0
    ry[~body] = 0.0
    lat.init(rx, ry)
    assert np.abs(lat.read(O.ESTRAIN)).max() <= 1e-22


def test_energy_density_plane_wave():
    """u = A e_x sin(k x) on a periodic lattice: the central difference gives
    eps_xx = A sin(k dh) / dh cos(k x) exactly, so the strain energy density is
    (lambda / 2 + mu) eps_xx^2 point by point, and its lattice sum is
    (lambda / 2 + mu) (A sin(k dh) / dh)^2 N / 2 (a full number of periods)."""
    nx, ny, lam, mu, A = 64, 8, 2.0, 1.0, 1e-3
    m = 3
    k = 2 * math.pi * m / nx
    X = np.tile(np.arange(nx, dtype=float), (ny, 1))
    lat = O.OracleLattice(nx, ny, lam, mu, periodic_x=True, periodic_y=True)
    lat.init(A * np.sin(k * X), np.zeros((ny, nx)))
    w = lat.read(O.ESTRAIN)
    exx = A * math.sin(k) * np.cos(k * X)
    assert np.abs(w - (0.5 * lam + mu) * exx ** 2).max() <= 1e-12 * (0.5 * lam + mu) * A * A
    total = (0.5 * lam + mu) * (A * math.sin(k)) ** 2 * nx * ny / 2
    assert abs(w.sum() - total) <= 1e-12 * total
