"""Checkpoint / resume through the C ABI: n steps equal k steps, save, load
into a fresh lattice created the same way, n - k steps, bit for bit, in every
storage format, with ramped boundary data (the step counter travels with
the state), into host or device memory, and inside a batch afterwards."""
import numpy as np
import pytest

from paper_2301_00228_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

FIELDS = ("ux", "uy", "vx", "vy", "phi", "psi", "f_phi", "f_psi")


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def make(L, storage, nx=45, ny=38, init=True):
    d = W.tension_square(24, a0_phi=0.999)
    lat = L.Lattice.rectangle(nx, ny, 1.3, 1.0, (1, 2, 1, 1), np.asarray(d.edge_value, float).ravel(),
                              a0_phi=0.99, storage=storage)
    lat.set_load(L.LBPS_NEUMANN, 60 * lat.dt, 90 * lat.dt)
    if init:
        ux, uy = W.pulse_displacement(nx, ny, 20.0, 15.0, 4.0, 1e-3, "rotation")
        lat.init(ux, uy)
    return lat


def same(a, b, what):
    for k in FIELDS:
        assert np.array_equal(a.read(k), b.read(k)), (what, k)


@pytest.mark.parametrize("storage", ["f64", "f32", "bf16", "f16", "bfp13"])
def test_resume_is_bit_exact(L, storage):
    n, k = 130, 47
    a = make(L, storage).step(n)
    b = make(L, storage).step(k)
    buf = b.save_state()
    assert buf.nbytes == L.lbps_state_size(b._h)
    c = make(L, storage, init=False).load_state(buf)
    assert c.steps == k and c.scale_exp == b.scale_exp
    c.step(n - k)
    same(a, c, storage)


def test_device_buffer_and_batch_after_resume(L):
    n, k = 90, 33
    a = make(L, "f32").step(n)
    b = make(L, "f32").step(k)
    dev = torch.empty(L.lbps_state_size(b._h), dtype=torch.uint8, device="cuda")
    assert L._lib.lbps_state_save(b._h, L.ctypes.c_void_p(dev.data_ptr()), dev.numel()) == 0
    c = make(L, "f32", init=False)
    assert L._lib.lbps_state_load(c._h, L.ctypes.c_void_p(dev.data_ptr()), dev.numel()) == 0
    other = make(L, "f32", nx=30, ny=30)
    batch = L.Batch([c, other])
    batch.step(n - k)
    assert batch.check() == 0
    batch.close()
    same(a, c, "batch")


def test_load_rejects_mismatch(L):
    b = make(L, "f32").step(3)
    buf = b.save_state()
    for bad in (make(L, "f32", nx=46, init=False), make(L, "f64", init=False), make(L, "f16", init=False)):
        with pytest.raises(L.LbpsError) as e:
            bad.load_state(buf)
        assert e.value.code == L.LBPS_ERR_INVALID
    with pytest.raises(L.LbpsError):
        make(L, "f32", init=False).load_state(buf[:-1])
    corrupt = buf.copy()
    corrupt[0] ^= 0xFF
    with pytest.raises(L.LbpsError):
        make(L, "f32", init=False).load_state(corrupt)
    with pytest.raises(L.LbpsError) as e:
        make(L, "f32", init=False).save_state()
    assert e.value.code == L.LBPS_ERR_STATE


def test_load_rejects_other_setup(L):
    """A state saved by one lattice does not load into a lattice of the same
    size and storage created otherwise: another material, another edge value,
    another reading of the boundary rules, or a plate with a hole."""
    nx, ny = 45, 38
    buf = make(L, "f32").step(3).save_state()
    d = W.tension_square(24, a0_phi=0.999)
    ev = np.asarray(d.edge_value, float).ravel()
    others = [L.Lattice.rectangle(nx, ny, 1.4, 1.0, (1, 2, 1, 1), ev, a0_phi=0.99),
              L.Lattice.rectangle(nx, ny, 1.3, 1.0, (1, 2, 1, 1), ev * 1.5, a0_phi=0.99),
              L.Lattice.rectangle(nx, ny, 1.3, 1.0, (1, 2, 1, 1), ev, a0_phi=0.99, bc_j_mode=1),
              L.Lattice.rectangle(nx, ny, 1.3, 1.0, (1, 2, 1, 1), ev, a0_phi=0.99, bc_feq_mode=1)]
    nt, bv, cell = L.lbps_disk_cells(nx, ny, 1.0, 22.0, 19.0, 6.0, (1, 2, 1, 1), ev)
    others.append(L.Lattice(nx, ny, 1.3, 1.0, a0_phi=0.99, node_type=nt, bc_value=bv, cell=cell))
    for q, o in enumerate(others):
        with pytest.raises(L.LbpsError) as e:
            o.load_state(buf)
        assert e.value.code == L.LBPS_ERR_INVALID, q
    same_again = make(L, "f32", init=False).load_state(buf)
    assert same_again.steps == 3
