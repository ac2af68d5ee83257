"""The FP64 oracle reproduces the hand-computed 3x3 lattices (both readings of the
equilibrium in Eq. LBE_mod)."""
import numpy as np
import pytest

import oracle as O
import hand_cases as H

FIELDS = {"ux": O.UX, "uy": O.UY, "vx": O.VX, "vy": O.VY, "phi": O.PHI, "psi": O.PSI}


def make(case, mode):
    c = H.load()["common"]
    nt, bv = O.rect_bc(c["nx"], c["ny"], case["edges"]["type"], H.edge_values(case))
    return O.OracleLattice(c["nx"], c["ny"], c["lambda"], c["mu"], c["rho"], c["dh"], c["a0_phi"],
                           node_type=nt, bc_value=bv, bc_feq_mode=mode)


def read(lat, field, alpha):
    if field in ("f_phi", "f_psi"):
        return lat.read(O.F_PHI if field == "f_phi" else O.F_PSI)[alpha]
    return lat.read(FIELDS[field])


@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("name", [c["name"] for c in H.load()["cases"]])
def test_hand_case(name, mode):
    g = H.load()
    case = next(c for c in g["cases"] if c["name"] == name)
    dt = make(case, mode).dt
    assert dt * dt == pytest.approx(1.0 / 12.0, rel=1e-14)
    fails = H.run_case(case, g["common"], mode, make, read, dt, tol=1e-12)
    assert not fails, fails
