"""The allocation-free norms entry point (lbps_norms_noalloc) against lbps_norms.

lbps_norms_noalloc serves callers that cannot allocate device memory (a
serving loop whose memory all sits in its own pool under a fixed budget, or a
loop that must not stall on cudaFree); its scratch is a fixed array inside the
library.  This file is collected last so a failure here leaves every other
test already run.  It passes alone in a fresh process and after the others.
"""
import numpy as np
import pytest

from paper_2301_00228_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-12  # relative: both sides sum in FP64, in different orders


@pytest.fixture(scope="module")
def L():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import lbps
    return lbps


def close(a, b, what):
    assert abs(a[0] - b[0]) <= TOL * max(abs(b[0]), 1e-300), (what, a, b)
    assert abs(a[1] - b[1]) <= TOL * max(abs(b[1]), 1e-300), (what, a, b)
    assert a[3] == b[3], (what, a, b)


def test_noalloc_norms_match_lattice_norms_twice(L):
    nx, ny = 301, 223
    ux, uy = W.pulse_displacement(nx, ny, 140.0, 100.0, 8.0, 1e-3, "dilatation")
    lat = L.Lattice.rectangle(nx, ny, 2.0, 1.0, (2, 1, 1, 1), np.zeros(8), a0_phi=0.99)
    lat.init(ux, uy).step(25)
    stream = torch.cuda.current_stream().cuda_stream
    for name in ("ux", "phi", "psi", "consistency"):
        x = lat.read_device(name).contiguous()
        ref = torch.sin(torch.arange(x.numel(), dtype=torch.float64, device="cuda")).reshape(x.shape) * 1e-3
        want = lat.norms(name, ref)
        want0 = lat.norms(name)
        torch.cuda.synchronize()
        for _ in range(2):  # two calls in a row share the scratch
            got = L.lbps_norms_noalloc(x.data_ptr(), ref.data_ptr(), x.numel(), stream)
            close(got, want, name)
            assert abs(got[2] - want[2]) <= 1e-12 * float(x.abs().sum()) + 1e-300
            got0 = L.lbps_norms_noalloc(x.data_ptr(), 0, x.numel(), stream)
            close(got0, want0, name + " (no ref)")


def test_noalloc_smaller_second_call_ignores_stale_scratch(L):
    """A call after a larger one reads only its own partial slots."""
    big = torch.rand(5_000_000, dtype=torch.float64, device="cuda")
    small = torch.rand(3000, dtype=torch.float64, device="cuda") - 0.5
    L.lbps_norms_noalloc(big.data_ptr(), 0, big.numel())
    got = L.lbps_norms_noalloc(small.data_ptr(), 0, small.numel())
    s = small.double().cpu().numpy()
    assert got[0] == pytest.approx((s * s).sum(), rel=1e-12)
    assert got[2] == pytest.approx(s.sum(), rel=1e-9, abs=1e-12)
    assert got[3] == np.abs(s).max()


def test_noalloc_rejects_oversize_and_bad_args(L):
    x = torch.zeros(16, dtype=torch.float64, device="cuda")
    for n in (L.LBPS_NOALLOC_MAX_POINTS + 1, 0):
        with pytest.raises(L.LbpsError) as e:
            L.lbps_norms_noalloc(x.data_ptr(), 0, n)
        assert e.value.code == L.LBPS_ERR_INVALID
    got = L.lbps_norms_noalloc(x.data_ptr(), 0, 16)
    assert list(got) == [0.0, 0.0, 0.0, 0.0]


def test_noalloc_keeps_nan_and_refuses_a_capturing_stream(L):
    """A NaN in x shows in the max slot; a call on a stream that is being
    captured into a graph is refused before any device work (it would end
    with a host copy and a wait), and the capture stays valid."""
    x = torch.arange(1000, dtype=torch.float64, device="cuda")
    x[17] = float("nan")
    got = L.lbps_norms_noalloc(x.data_ptr(), 0, x.numel())
    assert np.isnan(got[3]) and np.isnan(got[0])
    g = torch.cuda.CUDAGraph()
    y = torch.zeros_like(x)
    with torch.cuda.graph(g):
        with pytest.raises(L.LbpsError) as e:
            L.lbps_norms_noalloc(x.data_ptr(), 0, x.numel(), torch.cuda.current_stream().cuda_stream)
        y.copy_(x * 2.0)
    assert e.value.code == L.LBPS_ERR_INVALID
    g.replay()
    torch.cuda.synchronize()
    assert float(y[3]) == 6.0
