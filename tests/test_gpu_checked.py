"""The range-checked build (the stand-in for a memory sanitizer): every device
access of the time-loop kernels is checked for alignment and against the
device blocks of the live lattices, and the first violation is recorded
instead of performed.  A child process builds it, runs random single-lattice
cases, hole plates under every launch shape, lattices taking two steps per
sweep (their scratch copy registered as a live block) and a batch of uneven
lattices through it, and reads the record: no access may fall outside."""
import os
import subprocess
import sys
from pathlib import Path

import pytest

pytestmark = pytest.mark.gpu
ROOT = Path(__file__).resolve().parents[1]

CHILD = r"""
import os, sys
sys.path.insert(0, ROOT); sys.path.insert(0, os.path.join(ROOT, "tests"))
from paper_2301_00228_gb300 import build
build.build(checked=True)
os.environ["LBPS_CHECKED"] = "1"
import numpy as np
from paper_2301_00228_gb300 import lbps as L
from paper_2301_00228_gb300 import workloads as W
import test_gpu_fuzz as F

runs = 0
for seed in range(12):                       # random sizes, holes, periodic axes, storages, sync, ramps
    c = F.make_case(seed)
    lat = L.Lattice(c["nx"], c["ny"], c["lam"], c["mu"], c["rho"], a0_phi=c["a0"], periodic_x=c["px"],
                    periodic_y=c["py"], node_type=c["nt"], bc_value=c["bv"], bc_feq_mode=c["mode"],
                    sync_every=c["sync"], cell=c["cell"], storage=c["storage"])
    if c["ramp"]:
        lat.set_load(L.LBPS_NEUMANN, 30 * lat.dt, 60 * lat.dt)
    lat.init(c["ux"], c["uy"]).step(40)
    lat.fields()
    lat.close()
    runs += 1
n = 40                                        # hole plate: every launch shape, row chunks inside the hole
d = W.hole_square(n, a0_phi=0.999, horizon=0.05, sync_every=0)
nt, bv, cell = L.lbps_disk_cells(n, n, 1.0, *d.hole, d.edge_type, np.asarray(d.edge_value, float).ravel())
for variant in range(8):
    lat = L.Lattice(n, n, d.lam, d.mu, a0_phi=d.a0_phi, node_type=nt, bc_value=bv, cell=cell, storage="f32")
    L.lbps_set_tuning(lat._h, variant, 8)
    lat.init(*W.pulse_displacement(n, n, 12.0, 12.0, 3.0, 1e-3, "dilatation")).step(30)
    bad = np.zeros((n, n)); bad[3, 3] = np.nan
    try:
        lat.init(bad, bad)                    # rejected input (device check in the idle copy)
    except L.LbpsError:
        pass
    lat.step(5).close()
    runs += 1
for storage, (nx, ny) in (("f32", (16, 16)), ("f16", (67, 45)), ("f64", (131, 37))):  # two steps per sweep
    lat = L.Lattice.rectangle(nx, ny, 1.7, 1.0, (2, 1, 1, 2), np.full(8, 1e-4), a0_phi=0.99, storage=storage,
                              sync_every=7)
    L.lbps_set_step_pairs(lat._h, 1)
    lat.init(*W.pulse_displacement(nx, ny, nx / 3, ny / 2, 3.0, 1e-3, "dilatation")).step(41)
    lat.close()
    runs += 1
lats = []                                     # a batch of uneven rectangles and hole plates
for dom in W.mixed_batch(count=10)[::2]:
    lats.append(L.Lattice.rectangle(dom.nx, dom.ny, dom.lam, dom.mu, dom.edge_type,
                                    np.asarray(dom.edge_value, float).ravel(), a0_phi=dom.a0_phi)
                .init(*dom.displacement()))
for m in (40, 52):
    dd = W.hole_square(m, a0_phi=0.999, horizon=0.05, sync_every=0)
    nt2, bv2, cell2 = L.lbps_disk_cells(m, m, 1.0, *dd.hole, dd.edge_type, np.asarray(dd.edge_value, float).ravel())
    lats.append(L.Lattice(m, m, dd.lam, dd.mu, a0_phi=dd.a0_phi, node_type=nt2, bc_value=bv2, cell=cell2)
                .init(*W.pulse_displacement(m, m, 10.0, 10.0, 3.0, 1e-3, "rotation")))
b = L.Batch(lats)
b.tune(repeats=1)
b.step(25)
assert b.check() == 0
b.close()
runs += 1
rc, line, addr = L.lbps_check_report()
print("REPORT", rc, line, addr, runs)
"""


def test_checked_build_records_no_violation():
    env = dict(os.environ)
    env.pop("LBPS_CHECKED", None)
    out = subprocess.run([sys.executable, "-c", f"ROOT = {str(ROOT)!r}\n" + CHILD], capture_output=True, text=True,
                         timeout=1200, env=env, cwd=str(ROOT))
    report = [ln for ln in out.stdout.splitlines() if ln.startswith("REPORT")]
    assert out.returncode == 0 and report, out.stdout[-2000:] + out.stderr[-3000:]
    rc, line, addr, runs = (int(x) for x in report[-1].split()[1:])
    assert rc == 1, "the checked build was not loaded"
    assert (line, addr) == (0, 0), f"first violation at source line {line}, address {addr:#x}"
    assert runs == 24
