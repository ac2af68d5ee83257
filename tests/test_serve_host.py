"""Host logic of the continuous-batching server, on the CPU: lattices, batches
and lbps_step are replaced by fakes that count the steps each solve takes,
so admission, chunking, completion, withdrawal and the lone-request path are
checked without a GPU."""
from types import SimpleNamespace

import numpy as np
import pytest

from paper_2301_00228_gb300 import serve as S

# a scheduling bug tends to loop forever rather than fail: bound each test
pytestmark = pytest.mark.timeout(60)


class FakeLattice:
    def __init__(self, d):
        self.d, self.done, self.closed = d, 0, False
        self._h = self

    def read(self, name):
        return np.full((2, 2), float(self.done))

    def norms(self, name):
        return None

    def close(self):
        self.closed = True


class FakeBatch:
    built = []

    def __init__(self, lats, stream=None):
        assert len(lats) > 1, "a lone solve is stepped directly"
        self.lats = list(lats)
        FakeBatch.built.append(tuple(l.d.rid for l in lats))

    def set_tuning(self, variant, rows):
        pass

    def step(self, k):
        for lat in self.lats:
            assert not lat.closed
            lat.done += k

    def check(self):
        return 0

    def close(self):
        pass


class StepClock:
    def __init__(self):
        self.t = 0.0

    def __call__(self):
        self.t += 1.0
        return self.t


@pytest.fixture
def fakes(monkeypatch):
    lats = []

    def make(d, storage, u0=None, stream=None):
        lats.append(FakeLattice(d))
        return lats[-1]

    def lone_step(h, k):
        h.done += k
        return 0

    FakeBatch.built = []
    monkeypatch.setattr(S, "_lattice", make)
    monkeypatch.setattr(S, "footprint", lambda d, storage="f32": d.bytes)
    monkeypatch.setattr(S.lbps, "Batch", FakeBatch)
    monkeypatch.setattr(S.lbps, "lbps_step_async", lone_step)
    monkeypatch.setattr(S.lbps, "lbps_check", lambda h: 0)
    return lats


def req(rid, steps, arrival=0.0, nbytes=100, cancel_at=None):
    return S.Request(rid, arrival, SimpleNamespace(rid=rid, bytes=nbytes), steps, cancel_at)


def test_every_solve_takes_exactly_its_steps(fakes):
    reqs = [req(0, 130), req(1, 500), req(2, 75), req(3, 1000), req(4, 1)]
    rep = S.serve_batched(reqs, budget_bytes=10_000, max_chunk=64, clock=StepClock())
    assert [r.rid for r in rep.results] == [0, 1, 2, 3, 4]
    for r, q in zip(rep.results, reqs):
        assert r.ux[0, 0] == q.steps          # stepped exactly its step count
    assert all(lat.closed for lat in fakes)
    assert rep.max_active == 5
    assert rep.memory_waits == 0 and rep.memory_wait_s == 0.0


def test_budget_bounds_the_resident_solves(fakes):
    reqs = [req(k, 50 * (k + 1), nbytes=300) for k in range(6)]
    rep = S.serve_batched(reqs, budget_bytes=900, max_chunk=40, clock=StepClock())
    assert rep.max_active == 3 and rep.peak_bytes <= 900
    assert rep.memory_waits > 0 and rep.memory_wait_s > 0
    assert [r.ux[0, 0] for r in rep.results] == [q.steps for q in reqs]
    assert all(r.completed >= r.admitted >= r.arrival for r in rep.results)


def test_lone_request_is_stepped_directly(fakes):
    rep = S.serve_batched([req(0, 700)], budget_bytes=1000, max_chunk=500, clock=StepClock())
    assert FakeBatch.built == [] and rep.rebuilds == 0
    assert rep.results[0].ux[0, 0] == 700 and rep.chunks == 2      # chunks of 500 and 200


def test_withdrawn_requests_free_their_memory(fakes):
    reqs = [req(0, 400, nbytes=500), req(1, 400, nbytes=500, cancel_at=0.0), req(2, 400, nbytes=500, cancel_at=3.5),
            req(3, 400, nbytes=500)]
    # budget for two: 0 and 2 are admitted (1 is withdrawn while waiting); 2 is
    # withdrawn after its first chunk, which lets 3 in
    rep = S.serve_batched(reqs, budget_bytes=1000, max_chunk=100, clock=StepClock())
    assert sorted(rep.cancelled) == [1, 2]
    assert [r.rid for r in rep.results] == [0, 3]
    assert all(r.ux[0, 0] == 400 for r in rep.results)
    assert rep.peak_bytes <= 1000
    assert all(lat.closed for lat in fakes)


def test_request_larger_than_budget_is_refused(fakes):
    with pytest.raises(ValueError):
        S.serve_batched([req(0, 10, nbytes=2000)], budget_bytes=1000)
