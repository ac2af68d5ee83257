"""Loader for the hand-computed 3x3 lattices of tests/golden/hand_3x3.json.

The same fixtures check the FP64 oracle (tests/test_oracle_golden.py) and the
CUDA library (tests/test_gpu_parity.py).  ``run_case`` takes a factory that
returns an object with ``init(ux, uy)``, ``step(n)`` and ``read(name)``.
"""
import json
from pathlib import Path

import numpy as np

GOLDEN = Path(__file__).resolve().parent / "golden" / "hand_3x3.json"
DELTA, TAU = 1e-3, 2e-4


def load():
    return json.loads(GOLDEN.read_text())


def edge_values(case):
    return np.array([TAU if v == "t" else float(v) for v in case["edges"]["value"]], np.float64)


def initial_u(common):
    nx, ny = common["nx"], common["ny"]
    ux = np.zeros((ny, nx))
    uy = np.zeros((ny, nx))
    ux[1, 1] = DELTA
    return ux, uy


def expected(check, dt):
    return float(eval(check["expr"], {"__builtins__": {}}, {"d": DELTA, "t": TAU, "dt": dt}))


def checks_by_step(case, mode):
    out = {}
    for c in case["checks"]:
        if "mode" in c and c["mode"] != mode:
            continue
        out.setdefault(c["steps"], []).append(c)
    return out


def run_case(case, common, mode, make, read, dt, tol):
    """Advance a lattice built by ``make(case, mode)`` and compare every check.

    ``read(lattice, field, alpha)`` returns a [ny][nx] array.  Returns the list of
    (check, got, want) that failed ``|got - want| <= tol * DELTA``.
    """
    lat = make(case, mode)
    ux, uy = initial_u(common)
    lat.init(ux, uy)
    fails = []
    done = 0
    by_step = checks_by_step(case, mode)
    for steps in sorted(by_step):
        if steps > done:
            lat.step(steps - done)
            done = steps
        for c in by_step[steps]:
            i, j = c["node"]
            got = float(read(lat, c["field"], c.get("alpha"))[j, i])
            want = expected(c, dt)
            if not abs(got - want) <= tol * DELTA:
                fails.append((c, got, want))
    return fails
