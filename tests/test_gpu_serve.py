"""Continuous-batching serving: every request's result is the same alone and in
the mix, admission respects the device-memory budget, and the batched server
overlaps requests that arrive while others run."""
import numpy as np
import pytest

from paper_2301_00228_gb300 import workloads as W

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_2301_00228_gb300 import serve
    return serve


def stream(seed, count, rate_hz, side_lo=16, side_hi=96, steps_lo=20, steps_hi=200):
    from paper_2301_00228_gb300.serve import Request
    reqs = []
    for rid, (t, d) in enumerate(W.poisson_requests(count=count, seed=seed, rate_hz=rate_hz, side_lo=side_lo,
                                                    side_hi=side_hi, steps_lo=steps_lo, steps_hi=steps_hi)):
        d.a0_phi = 0.99
        reqs.append(Request(rid, t, d, d.steps))
    return reqs


def alone(S, req):
    lat = S._lattice(req.domain, "f32")
    lat.step(req.steps)
    out = lat.read("ux"), lat.read("uy")
    lat.close()
    return out


def test_results_same_alone_and_in_the_mix(S):
    reqs = stream(5, 24, rate_hz=400.0)
    rep = S.serve_batched(reqs, budget_bytes=8 << 30, max_chunk=64)
    assert len(rep.results) == len(reqs)
    assert rep.max_active > 1                    # requests overlapped on the device
    base = S.serve_one_at_a_time(reqs)
    for req, r, b in zip(reqs, rep.results, base.results):
        ux, uy = alone(S, req)
        assert r.rid == req.rid == b.rid
        assert np.array_equal(r.ux, ux) and np.array_equal(r.uy, uy), req.rid
        assert np.array_equal(b.ux, ux) and np.array_equal(b.uy, uy), req.rid
        assert r.completed >= r.admitted >= r.arrival
    s = rep.summary()
    assert s["solves"] == 24 and s["p99_latency_s"] >= s["p50_latency_s"] > 0


def test_admission_budget_binds(S):
    reqs = stream(6, 12, rate_hz=1000.0, side_lo=40, side_hi=60)
    per = max(S.footprint(r.domain) for r in reqs)
    budget = 3 * per
    rep = S.serve_batched(reqs, budget_bytes=budget, max_chunk=50)
    assert len(rep.results) == 12
    assert rep.max_active <= 3
    assert rep.peak_bytes <= budget
    for req, r in zip(reqs, rep.results):
        ux, uy = alone(S, req)
        assert np.array_equal(r.ux, ux) and np.array_equal(r.uy, uy), req.rid


def test_request_larger_than_budget_is_refused(S):
    reqs = stream(7, 2, rate_hz=10.0)
    with pytest.raises(ValueError):
        S.serve_batched(reqs, budget_bytes=1024)


class StepClock:
    """A clock that advances one second at every reading: the server's
    timeline (arrivals, chunk boundaries, withdrawals) becomes deterministic."""

    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


def test_withdrawn_requests_leave_queue_and_batch(S):
    """A request withdrawn before admission never runs; one withdrawn while
    in the batch leaves it at the next chunk boundary and gives its memory
    back; the others end with the same bits as alone."""
    reqs = stream(8, 6, rate_hz=10.0, steps_lo=150, steps_hi=200)
    for r in reqs:
        r.arrival = 0.0
    reqs[1].cancel_at = 0.0      # withdrawn while waiting
    reqs[3].cancel_at = 3.5      # admitted at t = 1, withdrawn after its first chunk
    rep = S.serve_batched(reqs, budget_bytes=8 << 30, max_chunk=20, clock=StepClock())
    assert sorted(rep.cancelled) == [1, 3]
    assert [r.rid for r in rep.results] == [0, 2, 4, 5]
    assert rep.max_active == 5
    for r in rep.results:
        ux, uy = alone(S, reqs[r.rid])
        assert np.array_equal(r.ux, ux) and np.array_equal(r.uy, uy), r.rid
    base = S.serve_one_at_a_time(reqs, clock=StepClock())
    assert 1 in base.cancelled and len(base.results) + len(base.cancelled) == 6


def test_results_with_two_steps_per_sweep(S):
    """With pairs the batch takes two steps per sweep: every result matches
    the solve alone up to the rounding of the composed two-step update of u,
    and the admission charge includes the scratch copy."""
    reqs = stream(8, 16, rate_hz=400.0, side_lo=16, side_hi=80)
    rep = S.serve_batched(reqs, budget_bytes=8 << 30, max_chunk=64, pairs=True)
    assert len(rep.results) == len(reqs) and rep.max_active > 1
    for req, r in zip(reqs, rep.results):
        ux, uy = alone(S, req)
        for got, want in ((r.ux, ux), (r.uy, uy)):
            scale = max(float(np.abs(want).max()), 1e-300)
            assert float(np.abs(got - want).max()) <= 1e-7 * scale, req.rid
    d = reqs[0].domain
    assert S.footprint(d, pairs=True) == S.footprint(d) + S.footprint(d) // 2
