"""Thin ctypes binding of the C ABI in include/lbps.h.

The functions ``lbps_*`` here have the names and arguments of the C entry
points and only marshal arguments; every step of the time loop runs in the
CUDA kernels of liblbps.so.  There is no host fallback: if the library is
missing, importing this module raises.  PyTorch supplies device memory (the
lattice state lives in a torch uint8 tensor) and the CUDA stream.

``Lattice`` is the convenience wrapper used by the tests and the benchmark.
"""
from __future__ import annotations

import ctypes
import os
from pathlib import Path

import numpy as np

# LBPS_CHECKED=1 selects the range-checked build (liblbps_checked.so).
_LIB_PATH = Path(__file__).resolve().parent / (
    "liblbps_checked.so" if os.environ.get("LBPS_CHECKED") == "1" else "liblbps.so")

LBPS_OK = 0
LBPS_ERR_INVALID = -1
LBPS_ERR_OOM = -2
LBPS_ERR_CUDA = -3
LBPS_ERR_NONFINITE = -4
LBPS_ERR_TIMEOUT = -5
LBPS_ERR_STATE = -6

LBPS_INTERIOR, LBPS_NEUMANN, LBPS_DIRICHLET, LBPS_VOID = 0, 1, 2, 3
LBPS_STORAGE_F32, LBPS_STORAGE_F64, LBPS_STORAGE_BF16, LBPS_STORAGE_F16, LBPS_STORAGE_BFP13 = 0, 1, 2, 3, 4
(LBPS_UX, LBPS_UY, LBPS_VX, LBPS_VY, LBPS_PHI, LBPS_PSI, LBPS_F_PHI, LBPS_F_PSI, LBPS_CONSISTENCY,
 LBPS_KINETIC_ENERGY, LBPS_STRAIN_ENERGY) = range(11)
FIELDS = {"ux": LBPS_UX, "uy": LBPS_UY, "vx": LBPS_VX, "vy": LBPS_VY, "phi": LBPS_PHI, "psi": LBPS_PSI,
          "f_phi": LBPS_F_PHI, "f_psi": LBPS_F_PSI, "consistency": LBPS_CONSISTENCY,
          "kinetic_energy": LBPS_KINETIC_ENERGY, "strain_energy": LBPS_STRAIN_ENERGY}
STORAGES = {"f32": LBPS_STORAGE_F32, "f64": LBPS_STORAGE_F64, "bf16": LBPS_STORAGE_BF16,
            "f16": LBPS_STORAGE_F16, "bfp13": LBPS_STORAGE_BFP13}


class lbps_params(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32),
                ("lambda_", ctypes.c_double), ("mu", ctypes.c_double), ("rho", ctypes.c_double),
                ("dh", ctypes.c_double), ("a0_phi", ctypes.c_double),
                ("periodic_x", ctypes.c_int32), ("periodic_y", ctypes.c_int32),
                ("bc_feq_mode", ctypes.c_int32), ("sync_every", ctypes.c_int32),
                ("storage", ctypes.c_int32), ("pop_scale_exp", ctypes.c_int32),
                ("cuda_stream", ctypes.c_void_p), ("bc_j_mode", ctypes.c_int32)]


class LbpsError(RuntimeError):
    def __init__(self, code, what="", cuda_code=0):
        self.code = code
        self.cuda_code = cuda_code
        msg = f"{lbps_strerror(code)} ({code})"
        if cuda_code:
            msg += f", cudaError {cuda_code}"
        super().__init__(f"{what}: {msg}" if what else msg)


def _load():
    if not _LIB_PATH.exists():
        raise ImportError(f"CUDA library {_LIB_PATH.name} is not built; run __graft_entry__.build()")
    L = ctypes.CDLL(str(_LIB_PATH))
    vp, i32, i64, sz = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
    P = ctypes.POINTER
    sig = {
        "lbps_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        "lbps_rect_bc": (ctypes.c_int, [i32, i32, i32, i32, ctypes.c_double, vp, vp, vp, vp]),
        "lbps_state_bytes": (ctypes.c_int, [P(lbps_params), P(sz)]),
        "lbps_create": (ctypes.c_int, [P(lbps_params), vp, vp, vp, sz, P(vp)]),
        "lbps_state_bytes_cells": (ctypes.c_int, [P(lbps_params), vp, vp, P(sz)]),
        "lbps_create_cells": (ctypes.c_int, [P(lbps_params), vp, vp, vp, vp, sz, P(vp)]),
        "lbps_disk_cells": (ctypes.c_int, [i32, i32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, vp, vp, vp, vp, vp]),
        "lbps_init": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "lbps_init_device": (ctypes.c_int, [vp, vp, vp, vp, vp]),
        "lbps_step": (ctypes.c_int, [vp, i64]),
        "lbps_step_async": (ctypes.c_int, [vp, i64]),
        "lbps_check": (ctypes.c_int, [vp]),
        "lbps_sync": (ctypes.c_int, [vp]),
        "lbps_read": (ctypes.c_int, [vp, i32, vp, sz]),
        "lbps_read_device": (ctypes.c_int, [vp, i32, vp, sz]),
        "lbps_norms": (ctypes.c_int, [vp, i32, vp, vp]),
        "lbps_energy": (ctypes.c_int, [vp, vp]),
        "lbps_norms_noalloc": (ctypes.c_int, [vp, vp, sz, vp, vp]),
        "lbps_info": (ctypes.c_int, [vp, vp, P(i64)]),
        "lbps_scale_exp": (ctypes.c_int, [vp, P(i32)]),
        "lbps_codec16": (ctypes.c_int, [i32, i32, vp, vp, i64, ctypes.c_uint32, i32, vp]),
        "lbps_set_load": (ctypes.c_int, [vp, i32, ctypes.c_double, ctypes.c_double]),
        "lbps_state_size": (ctypes.c_int, [vp, P(sz)]),
        "lbps_state_save": (ctypes.c_int, [vp, vp, sz]),
        "lbps_state_load": (ctypes.c_int, [vp, vp, sz]),
        "lbps_check_report": (ctypes.c_int, [vp]),
        "lbps_last_cuda_error": (ctypes.c_int, [vp]),
        "lbps_set_tuning": (ctypes.c_int, [vp, i32, i32]),
        "lbps_set_graph_steps": (ctypes.c_int, [vp, i32]),
        "lbps_set_step_pairs": (ctypes.c_int, [vp, i32]),
        "lbps_step_pairs": (ctypes.c_int, [vp]),
        "lbps_profile": (ctypes.c_int, [vp, i32]),
        "lbps_profile_read": (ctypes.c_int, [vp, vp]),
        "lbps_set_stream": (ctypes.c_int, [vp, vp]),
        "lbps_halo_bytes": (ctypes.c_int, [vp, i32, P(sz)]),
        "lbps_halo_pack": (ctypes.c_int, [vp, i32, i32, vp, sz]),
        "lbps_halo_unpack": (ctypes.c_int, [vp, i32, i32, vp, sz]),
        "lbps_set_origin": (ctypes.c_int, [vp, i64]),
        "lbps_destroy": (None, [vp]),
        "lbps_batch_create": (ctypes.c_int, [vp, i32, vp, P(vp)]),
        "lbps_batch_step": (ctypes.c_int, [vp, i64]),
        "lbps_batch_check": (ctypes.c_int, [vp]),
        "lbps_batch_set_tuning": (ctypes.c_int, [vp, i32, i32]),
        "lbps_batch_set_graph_steps": (ctypes.c_int, [vp, i32]),
        "lbps_batch_graph_steps": (ctypes.c_int, [vp]),
        "lbps_batch_set_step_pairs": (ctypes.c_int, [vp, i32]),
        "lbps_batch_step_pairs": (ctypes.c_int, [vp]),
        "lbps_batch_tune": (ctypes.c_int, [vp, i32, P(i32), P(i32), P(ctypes.c_double)]),
        "lbps_batch_last_cuda_error": (ctypes.c_int, [vp]),
        "lbps_batch_destroy": (None, [vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    return L


_lib = _load()


def _p(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _check(rc, what):
    if rc != LBPS_OK:
        raise LbpsError(rc, what)


# ---- C entry points under their own names ---------------------------------

def lbps_strerror(code):
    return _lib.lbps_strerror(int(code)).decode()


def lbps_rect_bc(nx, ny, periodic_x, periodic_y, dh, edge_type, edge_value):
    et = np.ascontiguousarray(edge_type, np.int32).reshape(4)
    ev = np.ascontiguousarray(edge_value, np.float64).reshape(8)
    nt = np.zeros((ny, nx), np.uint8)
    bv = np.zeros((ny, nx, 2), np.float64)
    _check(_lib.lbps_rect_bc(nx, ny, int(periodic_x), int(periodic_y), float(dh), _p(et), _p(ev), _p(nt), _p(bv)),
           "lbps_rect_bc")
    return nt, bv


def lbps_state_bytes(params):
    n = ctypes.c_size_t(0)
    _check(_lib.lbps_state_bytes(ctypes.byref(params), ctypes.byref(n)), "lbps_state_bytes")
    return int(n.value)


def lbps_create(params, node_type, bc_value, device_ptr, device_bytes):
    h = ctypes.c_void_p()
    _check(_lib.lbps_create(ctypes.byref(params), _p(node_type), _p(bc_value),
                            ctypes.c_void_p(device_ptr) if device_ptr else None, device_bytes, ctypes.byref(h)),
           "lbps_create")
    return h


def lbps_state_bytes_cells(params, node_type, cell):
    n = ctypes.c_size_t(0)
    _check(_lib.lbps_state_bytes_cells(ctypes.byref(params), _p(node_type), _p(cell), ctypes.byref(n)),
           "lbps_state_bytes_cells")
    return int(n.value)


def lbps_create_cells(params, node_type, bc_value, cell, device_ptr, device_bytes):
    h = ctypes.c_void_p()
    _check(_lib.lbps_create_cells(ctypes.byref(params), _p(node_type), _p(bc_value), _p(cell),
                                  ctypes.c_void_p(device_ptr) if device_ptr else None, device_bytes,
                                  ctypes.byref(h)), "lbps_create_cells")
    return h


def lbps_disk_cells(nx, ny, dh, cx, cy, r, edge_type, edge_value):
    """(node_type, bc_value, cell) of a rectangle with a circular hole."""
    et = np.ascontiguousarray(edge_type, np.int32).reshape(4)
    ev = np.ascontiguousarray(edge_value, np.float64).reshape(8)
    nt = np.zeros((ny, nx), np.uint8)
    bv = np.zeros((ny, nx, 2), np.float64)
    cell = np.zeros((ny, nx, 5), np.float64)
    _check(_lib.lbps_disk_cells(int(nx), int(ny), float(dh), float(cx), float(cy), float(r), _p(et), _p(ev),
                                _p(nt), _p(bv), _p(cell)), "lbps_disk_cells")
    return nt, bv, cell


def lbps_init(h, ux0, uy0, vx0=None, vy0=None):
    _check(_lib.lbps_init(h, _p(ux0), _p(uy0), _p(vx0), _p(vy0)), "lbps_init")


def lbps_init_device(h, d_ux0, d_uy0, d_vx0=0, d_vy0=0):
    _check(_lib.lbps_init_device(h, ctypes.c_void_p(d_ux0), ctypes.c_void_p(d_uy0),
                                 ctypes.c_void_p(d_vx0) if d_vx0 else None,
                                 ctypes.c_void_p(d_vy0) if d_vy0 else None), "lbps_init_device")


def lbps_step(h, n):
    return _lib.lbps_step(h, int(n))


def lbps_step_async(h, n):
    return _lib.lbps_step_async(h, int(n))


def lbps_check(h):
    return _lib.lbps_check(h)


def lbps_sync(h):
    _check(_lib.lbps_sync(h), "lbps_sync")


def lbps_read(h, field, dst):
    _check(_lib.lbps_read(h, int(field), _p(dst), dst.size), "lbps_read")
    return dst


def lbps_read_device(h, field, d_dst, count):
    _check(_lib.lbps_read_device(h, int(field), ctypes.c_void_p(d_dst), int(count)), "lbps_read_device")


def lbps_energy(h):
    out = np.zeros(3, np.float64)
    _check(_lib.lbps_energy(h, _p(out)), "lbps_energy")
    return out


def lbps_norms(h, field, d_ref=0):
    out = np.zeros(4, np.float64)
    _check(_lib.lbps_norms(h, int(field), ctypes.c_void_p(d_ref) if d_ref else None, _p(out)), "lbps_norms")
    return out


LBPS_NOALLOC_MAX_POINTS = 65536 * 4096


def lbps_norms_noalloc(d_x, d_ref, n, stream_ptr=0):
    """FP64 norms of caller-owned device arrays without any allocation (the
    scratch is a fixed array inside the library; see include/lbps.h)."""
    out = np.zeros(4, np.float64)
    _check(_lib.lbps_norms_noalloc(ctypes.c_void_p(d_x), ctypes.c_void_p(d_ref) if d_ref else None, int(n),
                                   ctypes.c_void_p(stream_ptr) if stream_ptr else None, _p(out)),
           "lbps_norms_noalloc")
    return out


def lbps_codec16(storage, encode, d_x, d_code, n, key0=0, stochastic=False, stream_ptr=0):
    """The value codec of a 16-bit storage format on device arrays (FP32
    values d_x, 16-bit codes d_code; see include/lbps.h)."""
    _check(_lib.lbps_codec16(STORAGES[storage] if isinstance(storage, str) else int(storage), int(encode),
                             ctypes.c_void_p(d_x), ctypes.c_void_p(d_code), int(n), int(key0) & 0xffffffff,
                             int(bool(stochastic)), ctypes.c_void_p(stream_ptr) if stream_ptr else None),
           "lbps_codec16")


def lbps_info(h):
    out = np.zeros(6, np.float64)
    steps = ctypes.c_int64(0)
    _check(_lib.lbps_info(h, _p(out), ctypes.byref(steps)), "lbps_info")
    return out, int(steps.value)


def lbps_set_load(h, kind, t_ramp, t_hold=float("inf")):
    _check(_lib.lbps_set_load(h, int(kind), float(t_ramp), float(t_hold)), "lbps_set_load")


def lbps_state_size(h):
    n = ctypes.c_size_t(0)
    _check(_lib.lbps_state_size(h, ctypes.byref(n)), "lbps_state_size")
    return int(n.value)


def lbps_state_save(h, dst):
    _check(_lib.lbps_state_save(h, _p(dst), dst.nbytes), "lbps_state_save")
    return dst


def lbps_state_load(h, src):
    src = np.ascontiguousarray(src, np.uint8)
    _check(_lib.lbps_state_load(h, _p(src), src.nbytes), "lbps_state_load")


def lbps_scale_exp(h):
    e = ctypes.c_int32(0)
    _check(_lib.lbps_scale_exp(h, ctypes.byref(e)), "lbps_scale_exp")
    return int(e.value)


def lbps_check_report():
    out = np.zeros(2, np.uint64)
    rc = _lib.lbps_check_report(_p(out))
    if rc < 0:
        raise LbpsError(rc, "lbps_check_report")
    return rc, int(out[0]), int(out[1])


def lbps_set_step_pairs(h, on):
    _check(_lib.lbps_set_step_pairs(h, int(on)), "lbps_set_step_pairs")


def lbps_step_pairs(h):
    return int(_lib.lbps_step_pairs(h))


def lbps_set_graph_steps(h, k):
    _check(_lib.lbps_set_graph_steps(h, int(k)), "lbps_set_graph_steps")


def lbps_set_tuning(h, variant, rows_per_warp):
    _check(_lib.lbps_set_tuning(h, int(variant), int(rows_per_warp)), "lbps_set_tuning")


def lbps_profile(h, enable):
    _check(_lib.lbps_profile(h, int(bool(enable))), "lbps_profile")


def lbps_profile_read(h):
    out = np.zeros(4, np.float64)
    _check(_lib.lbps_profile_read(h, _p(out)), "lbps_profile_read")
    return out


def lbps_set_stream(h, stream_ptr):
    _check(_lib.lbps_set_stream(h, ctypes.c_void_p(stream_ptr) if stream_ptr else None), "lbps_set_stream")


def lbps_destroy(h):
    _lib.lbps_destroy(h)


def lbps_halo_bytes(h, rows):
    n = ctypes.c_size_t(0)
    _check(_lib.lbps_halo_bytes(h, int(rows), ctypes.byref(n)), "lbps_halo_bytes")
    return int(n.value)


def lbps_halo_pack(h, row0, rows, d_buf, nbytes):
    _check(_lib.lbps_halo_pack(h, int(row0), int(rows), ctypes.c_void_p(d_buf), int(nbytes)), "lbps_halo_pack")


def lbps_halo_unpack(h, row0, rows, d_buf, nbytes):
    _check(_lib.lbps_halo_unpack(h, int(row0), int(rows), ctypes.c_void_p(d_buf), int(nbytes)), "lbps_halo_unpack")


def lbps_set_origin(h, row0):
    _check(_lib.lbps_set_origin(h, int(row0)), "lbps_set_origin")


# ---- convenience wrapper --------------------------------------------------

# From about this many points two time steps per sweep are faster than one
# (FP32, lbps_step with CUDA graphs: 8192^2 72.1 against 43.2 GLUPS, 4096^2
# 63.1 against 41.9, 2048^2 46.6 against 37.1, 1536^2 32.5 against 33.6;
# FP64 storage is bound by its FP64 population arithmetic, so not there).
PAIRS_AUTO_POINTS = 3_000_000


class Lattice:
    """One lattice on the current CUDA device, its state in a torch tensor."""

    def __init__(self, nx, ny, lam, mu, rho=1.0, dh=1.0, a0_phi=0.9999, periodic_x=False, periodic_y=False,
                 node_type=None, bc_value=None, bc_feq_mode=0, sync_every=0, storage="f32", pop_scale_exp=0,
                 stream=None, cell=None, bc_j_mode=0, step_pairs="auto"):
        """step_pairs: two time steps per sweep (lbps_set_step_pairs); "auto"
        turns them on for lattices of at least PAIRS_AUTO_POINTS points where
        they apply (rectangles without periodic axes) and the storage is not
        FP64, where they are faster (the scratch state copy they need is
        allocated then)."""
        import torch

        self.nx, self.ny = int(nx), int(ny)
        self._torch = torch
        self.stream = stream if stream is not None else torch.cuda.current_stream()
        self.params = lbps_params(self.nx, self.ny, lam, mu, rho, dh, a0_phi, int(periodic_x), int(periodic_y),
                                  int(bc_feq_mode), int(sync_every), STORAGES[storage], int(pop_scale_exp),
                                  ctypes.c_void_p(self.stream.cuda_stream), int(bc_j_mode))
        self.storage = storage
        nt = None if node_type is None else np.ascontiguousarray(node_type, np.uint8)
        bv = None if bc_value is None else np.ascontiguousarray(bc_value, np.float64)
        cl = None if cell is None else np.ascontiguousarray(cell, np.float64)
        self.nbytes = lbps_state_bytes_cells(self.params, nt, cl)
        with torch.cuda.stream(self.stream):
            self._mem = torch.empty(self.nbytes, dtype=torch.uint8, device="cuda")
        self._h = lbps_create_cells(self.params, nt, bv, cl, self._mem.data_ptr(), self.nbytes)
        c, _ = lbps_info(self._h)
        self.cd, self.cs, self.a_phi, self.a_psi, self.a0_psi, self.dt = (float(x) for x in c)
        if step_pairs == "auto":  # FP64 storage is FP64-bound with single steps already
            step_pairs = self.nx * self.ny >= PAIRS_AUTO_POINTS and storage != "f64"
        if step_pairs:
            lbps_set_step_pairs(self._h, 1)
            if not lbps_step_pairs(self._h):  # does not apply here: free the scratch copy
                lbps_set_step_pairs(self._h, 0)

    @classmethod
    def rectangle(cls, nx, ny, lam, mu, edge_type, edge_value, periodic_x=False, periodic_y=False, dh=1.0, **kw):
        nt, bv = lbps_rect_bc(nx, ny, periodic_x, periodic_y, dh, edge_type, edge_value)
        return cls(nx, ny, lam, mu, dh=dh, periodic_x=periodic_x, periodic_y=periodic_y, node_type=nt,
                   bc_value=bv, **kw)

    def close(self):
        if getattr(self, "_h", None):
            self.stream.synchronize()
            lbps_destroy(self._h)
            self._h = None
            self._mem = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def init(self, ux0, uy0, vx0=None, vy0=None):
        torch = self._torch
        if isinstance(ux0, torch.Tensor):
            t = [None if x is None else x.contiguous().to(torch.float64) for x in (ux0, uy0, vx0, vy0)]
            self._init_keep = t
            lbps_init_device(self._h, t[0].data_ptr(), t[1].data_ptr(), t[2].data_ptr() if t[2] is not None else 0,
                             t[3].data_ptr() if t[3] is not None else 0)
        else:
            a = [None if x is None else np.ascontiguousarray(x, np.float64) for x in (ux0, uy0, vx0, vy0)]
            lbps_init(self._h, *a)
        return self

    def step(self, n=1):
        rc = lbps_step(self._h, n)
        if rc != LBPS_OK:
            raise LbpsError(rc, "lbps_step", _lib.lbps_last_cuda_error(self._h))
        return self

    def step_async(self, n=1):
        rc = lbps_step_async(self._h, n)
        if rc != LBPS_OK:
            raise LbpsError(rc, "lbps_step_async", _lib.lbps_last_cuda_error(self._h))
        return self

    def check(self):
        return lbps_check(self._h)

    def sync(self):
        lbps_sync(self._h)
        return self

    @property
    def steps(self):
        return lbps_info(self._h)[1]

    @property
    def scale_exp(self):
        return lbps_scale_exp(self._h)

    def save_state(self):
        """Checkpoint of the current state (host bytes, numpy uint8)."""
        return lbps_state_save(self._h, np.empty(lbps_state_size(self._h), np.uint8))

    def load_state(self, buf):
        lbps_state_load(self._h, buf)
        return self

    def set_load(self, kind, t_ramp, t_hold=float("inf")):
        """Ramp-then-hold factor on the boundary data of one kind
        (LBPS_NEUMANN or LBPS_DIRICHLET): s(t) = min(t, t_hold) / t_ramp."""
        lbps_set_load(self._h, kind, t_ramp, t_hold)
        return self

    def read(self, field):
        fid = FIELDS[field] if isinstance(field, str) else int(field)
        planes = 5 if fid in (LBPS_F_PHI, LBPS_F_PSI) else 1
        out = np.zeros((planes, self.ny, self.nx), np.float64)
        lbps_read(self._h, fid, out)
        return out if planes == 5 else out[0]

    def read_device(self, field, out=None):
        torch = self._torch
        fid = FIELDS[field] if isinstance(field, str) else int(field)
        planes = 5 if fid in (LBPS_F_PHI, LBPS_F_PSI) else 1
        if out is None:
            out = torch.empty((planes, self.ny, self.nx), dtype=torch.float64, device="cuda")
        lbps_read_device(self._h, fid, out.data_ptr(), out.numel())
        return out if planes == 5 else out[0]

    def norms(self, field, ref=None):
        fid = FIELDS[field] if isinstance(field, str) else int(field)
        if ref is not None:
            ref = ref.contiguous()
            return lbps_norms(self._h, fid, ref.data_ptr())
        return lbps_norms(self._h, fid)

    def energy(self):
        """(kinetic, strain, total) energy of the current state (FP64, on the device)."""
        return lbps_energy(self._h)

    def fields(self):
        return {k: self.read(k) for k in ("ux", "uy", "vx", "vy", "phi", "psi")}


# ---- batches -----------------------------------------------------------------

def lbps_batch_create(handles, stream_ptr=0):
    arr = (ctypes.c_void_p * len(handles))(*[h.value if isinstance(h, ctypes.c_void_p) else h for h in handles])
    b = ctypes.c_void_p()
    _check(_lib.lbps_batch_create(arr, len(handles), ctypes.c_void_p(stream_ptr) if stream_ptr else None,
                                  ctypes.byref(b)), "lbps_batch_create")
    return b


def lbps_batch_step(b, n):
    return _lib.lbps_batch_step(b, int(n))


def lbps_batch_check(b):
    return _lib.lbps_batch_check(b)


def lbps_batch_set_tuning(b, variant, rows_per_warp):
    _check(_lib.lbps_batch_set_tuning(b, int(variant), int(rows_per_warp)), "lbps_batch_set_tuning")


def lbps_batch_set_graph_steps(b, k):
    _check(_lib.lbps_batch_set_graph_steps(b, int(k)), "lbps_batch_set_graph_steps")


def lbps_batch_graph_steps(b):
    return int(_lib.lbps_batch_graph_steps(b))


def lbps_batch_set_step_pairs(b, on):
    _check(_lib.lbps_batch_set_step_pairs(b, int(on)), "lbps_batch_set_step_pairs")


def lbps_batch_step_pairs(b):
    return int(_lib.lbps_batch_step_pairs(b))


def lbps_batch_tune(b, repeats=3):
    v, r, ms = ctypes.c_int32(0), ctypes.c_int32(0), ctypes.c_double(0)
    _check(_lib.lbps_batch_tune(b, int(repeats), ctypes.byref(v), ctypes.byref(r), ctypes.byref(ms)),
           "lbps_batch_tune")
    return int(v.value), int(r.value), float(ms.value)


def lbps_batch_destroy(b):
    _lib.lbps_batch_destroy(b)


class Batch:
    """Lattices advanced together (one launch per kernel per step, graphs)."""

    def __init__(self, lattices, stream=None):
        self.lattices = list(lattices)
        self.stream = stream
        self._h = lbps_batch_create([l._h for l in self.lattices], stream.cuda_stream if stream is not None else 0)

    def step(self, n=1):
        rc = lbps_batch_step(self._h, n)
        if rc != LBPS_OK:
            raise LbpsError(rc, "lbps_batch_step", _lib.lbps_batch_last_cuda_error(self._h))
        return self

    def check(self):
        return lbps_batch_check(self._h)

    def tune(self, repeats=3):
        return lbps_batch_tune(self._h, repeats)

    def set_tuning(self, variant, rows_per_warp):
        lbps_batch_set_tuning(self._h, variant, rows_per_warp)

    @property
    def graph_steps(self):
        return lbps_batch_graph_steps(self._h)

    def set_graph_steps(self, k):
        lbps_batch_set_graph_steps(self._h, k)

    @property
    def step_pairs(self):
        return bool(lbps_batch_step_pairs(self._h))

    def set_step_pairs(self, on):
        """Two time steps per sweep for every lattice (lbps_batch_set_step_pairs)."""
        lbps_batch_set_step_pairs(self._h, on)

    def close(self):
        if getattr(self, "_h", None):
            lbps_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
