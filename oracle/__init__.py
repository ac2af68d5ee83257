"""FP64 CPU oracle for the plane-strain lattice Boltzmann method (arXiv:2301.00228).

TEST INFRASTRUCTURE ONLY.  The oracle is the plain, slow reference the CUDA
library is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import it.  It shares no code with the
CUDA path: the arithmetic lives in ``lbm_oracle.c`` (compiled with gcc,
``-ffp-contract=off`` so results do not depend on FMA contraction), and this
module only marshals arrays through ctypes.

Parity status of each function is recorded in ``PINS`` below: every part of
the time loop is pinned by a test against a closed form, an invariant, a
hand-computed lattice or brute force, except what is listed in
``PARITY_UNPINNED`` (pinned oracle-to-CUDA only).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
from pathlib import Path

import numpy as np

_HERE = Path(__file__).resolve().parent
_SRC = _HERE / "lbm_oracle.c"
_LIB = _HERE / "liblbm_oracle.so"

# Which test pins which part of the oracle (file::test).
PINS = {
    "constants (Eq. conditions-parameters)": "tests/test_oracle_pins.py::test_constants_*",
    "interior LBE = five-point leapfrog": "tests/test_oracle_pins.py::test_leapfrog_equivalence",
    "discrete standing wave, phi/psi/u/v": "tests/test_oracle_pins.py::test_standing_wave_closed_form",
    "wave speeds c_d, c_s": "tests/test_oracle_pins.py::test_wave_speeds",
    "conservation (periodic)": "tests/test_oracle_pins.py::test_conservation_periodic",
    "patch tests (Neumann cells, corners, Dirichlet)": "tests/test_oracle_pins.py::test_patch_*",
    "Dirichlet target u*": "tests/test_oracle_pins.py::test_dirichlet_reaches_target",
    "hand-computed 3x3 lattices": "tests/test_oracle_golden.py",
    "convergence to continuum slab modes": "tests/test_oracle_pins.py::test_slab_convergence",
    "linearity / mirror symmetry": "tests/test_oracle_pins.py::test_linearity, ::test_mirror_symmetry",
    "synchronisation (Sec. 3.2)": "tests/test_oracle_pins.py::test_sync_*",
    "rectangle boundary helper": "tests/test_oracle_pins.py::test_rect_bc_*",
    "time-dependent boundary data (readings R12, R13)": "tests/test_oracle_pins.py::test_load_ramp_*",
    "general geometry: void points, clipped cells, one-sided stencils (reading R14)":
        "tests/test_oracle_pins.py::test_hole_*, ::test_explicit_rectangle_cells_equal_default, "
        "::test_geometry_rejected_without_stencil",
    "cells of the plate with a hole, areas by Green's theorem (reading R16)":
        "tests/test_oracle_cells.py (hand-derived cells in tests/golden/disk_cells.json, tiling of the body, "
        "closure of every cell boundary, sampling, symmetry)",
    "initial first moments from du/dt (reading R9)":
        "tests/test_oracle_pins.py::test_travelling_wave_from_initial_velocity (discrete travelling wave)",
    "J of Eq. correction-f, both readings (R7, R15)":
        "tests/test_oracle_pins.py::test_bc_j_mode_* (mode 1 against its definition; patch tests)",
    "energy densities (diagnostic; Eq. hooke, Eq. strain)":
        "tests/test_oracle_pins.py::test_energy_density_* (uniform strain and rigid rotation on a rectangle "
        "and a plate with a hole, uniform velocity, discrete plane wave)",
}
# Readings with no pin against the paper itself.
PARITY_UNPINNED = (
    "J of Eq. correction-f with bc_j_mode 1 (reading R15): an alternative reading of the paper's J(x_k, t); "
    "pinned to its own definition and oracle-to-CUDA only",
    "consistency-error magnitude of Fig. 9 (4.3e-12): lattice resolution not given",
)

UX, UY, VX, VY, PHI, PSI, F_PHI, F_PSI, ERR, AX, AY, EKIN, ESTRAIN = range(13)


def build(force: bool = False) -> Path:
    """Compile lbm_oracle.c into a shared library beside it (gcc, FP64, OpenMP)."""
    if _LIB.exists() and not force and _LIB.stat().st_mtime >= _SRC.stat().st_mtime:
        return _LIB
    tmp = _LIB.with_suffix(f".so.{os.getpid()}")
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-o", str(tmp), str(_SRC), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("lam", ctypes.c_double), ("mu", ctypes.c_double), ("rho", ctypes.c_double),
                ("dh", ctypes.c_double), ("a0_phi", ctypes.c_double),
                ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("bc_feq_mode", ctypes.c_int32), ("sync_every", ctypes.c_int32),
                ("bc_j_mode", ctypes.c_int32)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(str(_LIB))
        vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
        L.ora_create.restype = vp
        L.ora_create.argtypes = [ctypes.POINTER(_Params), vp, vp]
        L.ora_create_cells.restype = vp
        L.ora_create_cells.argtypes = [ctypes.POINTER(_Params), vp, vp, vp]
        L.ora_destroy.argtypes = [vp]
        L.ora_constants.argtypes = [vp, dp]
        L.ora_init.argtypes = [vp, vp, vp, vp, vp]
        L.ora_step.argtypes = [vp, ctypes.c_int64]
        L.ora_set_load.argtypes = [vp, ctypes.c_int32, ctypes.c_double, ctypes.c_double]
        L.ora_sync.argtypes = [vp]
        L.ora_read.argtypes = [vp, ctypes.c_int32, vp]
        L.ora_steps_done.restype = ctypes.c_int64
        L.ora_steps_done.argtypes = [vp]
        L.ora_rect_bc.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_double, vp, vp, vp, vp]
        L.ora_disk_cells.argtypes = [ctypes.c_int32, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_double, vp, vp, vp, vp, vp]
        L.ora_clip_rect.argtypes = [ctypes.c_double] * 7 + [vp]
        L.ora_get_rows.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp]
        L.ora_set_rows.argtypes = [vp, ctypes.c_int32, ctypes.c_int32, vp]
        L.ora_set_threads.argtypes = [ctypes.c_int32]
        L.ora_get_threads.restype = ctypes.c_int32
        _lib = L
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def set_threads(n: int) -> None:
    lib().ora_set_threads(int(n))


def rect_bc(nx, ny, edge_type, edge_value, periodic_x=False, periodic_y=False, dh=1.0):
    """Node types and boundary values of a rectangle (edges: bottom, right, top, left)."""
    et = np.ascontiguousarray(edge_type, dtype=np.int32).reshape(4)
    ev = np.ascontiguousarray(edge_value, dtype=np.float64).reshape(8)
    nt = np.zeros((ny, nx), np.uint8)
    bv = np.zeros((ny, nx, 2), np.float64)
    rc = lib().ora_rect_bc(nx, ny, int(periodic_x), int(periodic_y), float(dh), _ptr(et), _ptr(ev),
                           _ptr(nt), _ptr(bv))
    if rc != 0:
        raise ValueError("invalid rectangle boundary description")
    return nt, bv


def disk_cells(nx, ny, cx, cy, r, edge_type, edge_value, dh=1.0):
    """Node types, boundary values and cells of an nx x ny rectangle of lattice
    points with a traction-free circular hole of centre (cx, cy) and radius r
    (lengths in the units of dh; reading R16, areas by Green's theorem)."""
    et = np.ascontiguousarray(edge_type, dtype=np.int32).reshape(4)
    ev = np.ascontiguousarray(edge_value, dtype=np.float64).reshape(8)
    nt = np.zeros((ny, nx), np.uint8)
    bv = np.zeros((ny, nx, 2), np.float64)
    cell = np.zeros((ny, nx, 5), np.float64)
    rc = lib().ora_disk_cells(int(nx), int(ny), float(dh), float(cx), float(cy), float(r), _ptr(et), _ptr(ev),
                              _ptr(nt), _ptr(bv), _ptr(cell))
    if rc != 0:
        raise ValueError("invalid plate-with-hole description")
    return nt, bv, cell


def clip_rect(x0, x1, y0, y1, cx, cy, r):
    """(area, lengths of the sides x = x1, y = y1, x = x0, y = y0) of the part of
    the rectangle [x0, x1] x [y0, y1] outside the open disk."""
    out = np.zeros(5, np.float64)
    lib().ora_clip_rect(float(x0), float(x1), float(y0), float(y1), float(cx), float(cy), float(r), _ptr(out))
    return float(out[0]), out[1:].copy()


class OracleLattice:
    """One lattice of the FP64 oracle."""

    def __init__(self, nx, ny, lam, mu, rho=1.0, dh=1.0, a0_phi=0.9999, periodic_x=False,
                 periodic_y=False, node_type=None, bc_value=None, bc_feq_mode=0, sync_every=0, cell=None,
                 bc_j_mode=0):
        self.nx, self.ny = int(nx), int(ny)
        p = _Params(self.nx, self.ny, lam, mu, rho, dh, a0_phi, int(periodic_x), int(periodic_y),
                    int(bc_feq_mode), int(sync_every), int(bc_j_mode))
        if node_type is None:
            node_type = np.zeros((ny, nx), np.uint8)
        self._nt = np.ascontiguousarray(node_type, dtype=np.uint8)
        self._bv = None if bc_value is None else np.ascontiguousarray(bc_value, dtype=np.float64)
        self._cell = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64)
        self._h = lib().ora_create_cells(ctypes.byref(p), _ptr(self._nt), _ptr(self._bv), _ptr(self._cell))
        if not self._h:
            raise ValueError("oracle rejected the lattice description")
        c = np.zeros(6)
        lib().ora_constants(self._h, c.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        self.cd, self.cs, self.a_phi, self.a_psi, self.a0_psi, self.dt = (float(x) for x in c)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().ora_destroy(h)
            self._h = None

    def init(self, ux0, uy0, vx0=None, vy0=None):
        a = [np.ascontiguousarray(x, dtype=np.float64) if x is not None else None
             for x in (ux0, uy0, vx0, vy0)]
        if lib().ora_init(self._h, *[_ptr(x) for x in a]) != 0:
            raise ValueError("non-finite initial data")
        return self

    def set_load(self, kind, t_ramp, t_hold=float("inf")):
        """Ramp-then-hold factor on the boundary data of one kind (1 Neumann,
        2 Dirichlet): s(t) = min(t, t_hold) / t_ramp; t_ramp = 0: constant."""
        if lib().ora_set_load(self._h, int(kind), float(t_ramp), float(t_hold)) != 0:
            raise ValueError("ora_set_load: bad arguments")
        return self

    def step(self, n=1):
        if lib().ora_step(self._h, int(n)) != 0:
            raise RuntimeError("oracle step failed")
        return self

    def sync(self):
        lib().ora_sync(self._h)
        return self

    @property
    def steps(self):
        return int(lib().ora_steps_done(self._h))

    def read(self, field):
        planes = 5 if field in (F_PHI, F_PSI) else 1
        out = np.zeros((planes, self.ny, self.nx), np.float64)
        if lib().ora_read(self._h, int(field), _ptr(out)) != 0:
            raise ValueError("bad field id")
        return out if planes == 5 else out[0]

    def get_rows(self, row0, rows):
        """Rows [row0, row0 + rows) of the state: (14, rows, nx) doubles (the five
        populations of each set, u_x, u_y, v_x, v_y)."""
        out = np.zeros((14, rows, self.nx), np.float64)
        if lib().ora_get_rows(self._h, int(row0), int(rows), _ptr(out)) != 0:
            raise ValueError("bad row range or lattice not initialised")
        return out

    def set_rows(self, row0, block):
        block = np.ascontiguousarray(block, np.float64)
        if lib().ora_set_rows(self._h, int(row0), int(block.shape[1]), _ptr(block)) != 0:
            raise ValueError("bad row range or lattice not initialised")
        return self

    def fields(self):
        return {name: self.read(fid) for name, fid in
                (("ux", UX), ("uy", UY), ("vx", VX), ("vy", VY), ("phi", PHI), ("psi", PSI))}


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print(_LIB)
