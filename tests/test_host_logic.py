"""Host-side logic without a GPU: the serving scheduler's admission by HBM footprint, the
autotune cache, and the wedge-covariance helpers.

The server's device calls (workspace size, free memory, contexts, streams, events) are replaced
by fakes, so that what is tested is its scheduling: continuous batching of requests into
contexts keyed by (nmesh, l_max), admission against the HBM budget and the device's free
memory, least-recently-used eviction of idle contexts, and waiting when everything is busy.
"""
import math
import types

import numpy as np
import pytest

from paper_1704_02357_gb300 import covariance, serve, tune
from oracle import systematics as OS


# ----------------------------------------------------------------------------- serving
class FakeEvent:
    def __init__(self):
        self.done = False

    def record(self, stream):
        stream.events.append(self)

    def query(self):
        return self.done


class FakeStream:
    def __init__(self, device=None):
        self.events = []


class FakeTensor:
    def __init__(self, a):
        self.a = np.asarray(a)

    def __getitem__(self, i):
        return FakeTensor(self.a[i])

    def cpu(self):
        return self

    def numpy(self):
        return self.a


class FakeEstimator:
    created = []

    def __init__(self, nmesh, ell_max, stream, **kw):
        self.nmesh, self.ell_max, self.stream = nmesh, ell_max, stream
        self.kw = kw
        self.closed = False
        self.randoms = None
        FakeEstimator.created.append(self)

    def set_randoms(self, r):
        self.randoms = r

    def run_batch(self, pos, ells, edges, use_graph=True):
        nk = len(edges) - 1
        return {"P": FakeTensor(np.full((1, len(ells), nk), float(self.nmesh))), "sums": FakeTensor(np.zeros((1, 4)))}

    def close(self):
        self.closed = True


@pytest.fixture
def fake_server(monkeypatch):
    import torch
    FakeEstimator.created = []
    monkeypatch.setattr(serve, "Estimator", FakeEstimator)
    monkeypatch.setattr(torch.cuda, "Stream", FakeStream)
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "empty_cache", lambda: None)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda *a: None)
    clock = types.SimpleNamespace(t=0.0)

    def make(budget, free=1 << 50, footprints=None, **kw):
        s = serve.Server(box_size=1000.0, box_corner=(0.0, 0.0, 0.0), randoms_for=lambda n: f"randoms{n}",
                         hbm_budget=budget, clock=lambda: clock.t, **kw)
        fp = footprints or {}
        s._footprint = lambda nmesh, ell_max, tables=None: fp.get((nmesh, ell_max), nmesh ** 3)
        s._free_device_bytes = lambda: free - s.used()
        s.headroom = 0
        return s

    make.clock = clock
    return make


def _req(rid, nmesh, ell_max=4):
    return serve.Request(rid=rid, nmesh=nmesh, ell_max=ell_max, pos=None, k_edges=np.linspace(0, 0.1, 5))


def _finish(server, nmesh=None):
    for s in server.slots:
        if s.busy is not None and (nmesh is None or s.key[0] == nmesh):
            s.event.done = True


def test_requests_of_one_shape_share_and_reuse_a_context(fake_server):
    s = fake_server(budget=10 * 64 ** 3)
    for i in range(3):
        s.submit(_req(i, 64))
    s.step()
    # at most max_slots_per_shape (2) contexts per shape; the third request waits
    assert len(s.slots) == 2 and len(s.queue) == 1
    assert all(e.randoms == "randoms64" for e in FakeEstimator.created)
    _finish(s)
    s.step()
    assert len(s.done) == 2 and len(s.queue) == 0 and len(s.slots) == 2
    assert len(FakeEstimator.created) == 2  # the waiting request reused a warm context
    _finish(s)
    s.step()
    assert sorted(r.rid for r in s.done) == [0, 1, 2]
    for r in s.done:
        assert r.P.shape == (3, 4) and np.all(r.P == 64.0)
        assert r.t_admit >= r.t_arrival and r.t_done >= r.t_admit


def test_shapes_whose_tables_would_crowd_the_budget_are_served_without_them(fake_server):
    """A context holds the Y_lm tables only when its footprint with them is at most
    table_fraction of the budget; the policy is decided once per shape."""
    s = fake_server(budget=100, table_fraction=0.5)
    big = {True: 80, False: 30}
    small = {True: 40, False: 20}
    s._footprint = lambda nmesh, ell_max, tables=None: (
        (big if nmesh == 512 else small)[s.tables_for(nmesh, ell_max) if tables is None else tables])
    assert s.tables_for(512, 16) is False and s.tables_for(128, 4) is True
    s.submit(_req(0, 512, 16))
    s.submit(_req(1, 128, 4))
    s.step()
    assert sorted(sl.footprint for sl in s.slots) == [30, 40]
    assert {e.nmesh: e.kw["ylm_table"] for e in FakeEstimator.created} == {512: False, 128: True}


def test_prewarm_builds_contexts_before_the_stream(fake_server):
    s = fake_server(budget=10 * 64 ** 3)
    s.prewarm([(64, 4), (32, 2)], edges_for=lambda n: np.linspace(0, 0.1, 5), pos_for=lambda n: None)
    assert sorted(sl.key for sl in s.slots) == [(32, 2), (32, 2), (64, 4), (64, 4)]
    n0 = len(FakeEstimator.created)
    s.submit(_req(0, 64))
    s.step()
    assert len(FakeEstimator.created) == n0  # served by a prewarmed context, none built on admission
    assert any(sl.busy is not None for sl in s.slots if sl.key == (64, 4))


def test_admission_evicts_the_least_recently_used_idle_context(fake_server):
    fp = {(64, 4): 4, (96, 4): 4, (128, 4): 4}
    s = fake_server(budget=8, footprints=fp)
    s.submit(_req(0, 64))
    s.submit(_req(1, 96))
    s.step()
    assert s.used() == 8
    fake_server.clock.t = 1.0
    _finish(s, 64)
    s.step()
    fake_server.clock.t = 2.0
    _finish(s, 96)
    s.step()
    # both idle; 64 was used least recently, so it goes for the 128^3 context
    s.submit(_req(2, 128))
    s.step()
    keys = sorted(sl.key for sl in s.slots)
    assert keys == [(96, 4), (128, 4)] and s.used() == 8
    assert [e.closed for e in FakeEstimator.created[:2]] == [True, False]


def test_a_request_waits_while_every_context_is_busy(fake_server):
    s = fake_server(budget=8, footprints={(64, 4): 8, (96, 4): 8})
    s.submit(_req(0, 64))
    s.submit(_req(1, 96))
    s.step()
    assert len(s.slots) == 1 and [r.rid for r in s.queue] == [1]
    assert math.isnan(s.queue[0].t_admit)
    _finish(s)
    s.step()  # the 64^3 request finishes; its idle context is evicted for the 96^3 one
    assert [sl.key for sl in s.slots] == [(96, 4)] and not s.queue
    assert s.busy()
    _finish(s)
    s.step()
    assert not s.busy() and sorted(r.rid for r in s.done) == [0, 1]


def test_the_device_free_memory_also_bounds_admission(fake_server):
    # the budget would allow two contexts, the device only has room for one
    s = fake_server(budget=100, free=10, footprints={(64, 4): 6, (96, 4): 6})
    s.submit(_req(0, 64))
    s.submit(_req(1, 96))
    s.step()
    assert len(s.slots) == 1 and len(s.queue) == 1


def test_over_budget_and_nothing_to_evict_are_errors(fake_server):
    s = fake_server(budget=5, footprints={(64, 4): 6})
    s.submit(_req(0, 64))
    with pytest.raises(ValueError):
        s.step()
    s = fake_server(budget=100, free=3, footprints={(64, 4): 6})
    s.submit(_req(0, 64))
    with pytest.raises(MemoryError):
        s.step()


def test_latency_summary():
    done = []
    for i, (ta, tq, td) in enumerate([(0.0, 0.1, 0.5), (1.0, 1.0, 1.2), (2.0, 2.5, 3.0)]):
        r = _req(i, 64)
        r.t_arrival, r.t_admit, r.t_done = ta, tq, td
        done.append(r)
    s = serve.latency_summary(done, wall=4.0)
    lat = np.array([0.5, 0.2, 1.0])
    assert s["requests"] == 3 and s["throughput_per_s"] == 0.75
    assert s["p50_ms"] == pytest.approx(np.percentile(lat, 50) * 1e3)
    assert s["p99_ms"] == pytest.approx(np.percentile(lat, 99) * 1e3)
    assert s["mean_queue_wait_ms"] == pytest.approx(np.mean([0.1, 0.0, 0.5]) * 1e3)


# ----------------------------------------------------------------------------- autotune cache
class FakeTunable:
    def __init__(self):
        self.applied = None
        self.tuned_calls = 0

    def set_tuning(self, **kw):
        self.applied = kw

    def autotune(self, data_pos, randoms_pos, ells, k_edges, reps=2, **cat):
        self.tuned_calls += 1
        return {"tile_y": 1, "ylm_harmonics": 9, "bin_blocks_per_sm": 2, "paint_binned": 1}


def test_tuning_cache_round_trip_and_reuse(tmp_path, monkeypatch):
    path = str(tmp_path / "sub" / "tuning.json")
    assert tune.load_cache(path) == {}
    monkeypatch.setattr(tune, "key_for", lambda est: "GPU|N512|fp32|l4|w0|i1")
    est = FakeTunable()
    first = tune.tuned(est, None, None, [0, 2, 4], [0.0, 0.1], path=path)
    assert first["cached"] is False and est.tuned_calls == 1
    assert tune.load_cache(path) == {"GPU|N512|fp32|l4|w0|i1": {k: v for k, v in first.items() if k != "cached"}}
    est2 = FakeTunable()
    second = tune.tuned(est2, None, None, [0, 2, 4], [0.0, 0.1], path=path)
    assert second["cached"] is True and est2.tuned_calls == 0
    assert est2.applied == {k: v for k, v in first.items() if k != "cached"}


def test_a_corrupt_tuning_cache_reads_as_empty(tmp_path):
    p = tmp_path / "tuning.json"
    p.write_text("{not json")
    assert tune.load_cache(str(p)) == {}


# ----------------------------------------------------------------------------- wedge covariance
def test_correlation_and_condition_number_match_the_oracle():
    rng = np.random.default_rng(3)
    A = rng.standard_normal((6, 6))
    C = A @ A.T + 6 * np.eye(6)
    np.testing.assert_allclose(covariance.correlation(C), OS.correlation(C), rtol=1e-14)
    assert covariance.condition_number(C) == pytest.approx(OS.condition_number(C), rel=1e-12)
    assert covariance.condition_number(np.eye(4)) == 1.0


def test_pooled_correlation_recovers_a_known_correlation():
    rng = np.random.default_rng(5)
    R = np.array([[1.0, 0.6, -0.2], [0.6, 1.0, 0.1], [-0.2, 0.1, 1.0]])
    L = np.linalg.cholesky(R)
    n, nk = 4000, 6
    W = np.einsum("ij,mjk->mik", L, rng.standard_normal((n, 3, nk)))
    W = W * np.arange(1, nk + 1)[None, None, :] + 7.0  # scale and offset per k bin do not matter
    W[:, :, 2] = np.nan          # a bin with non-finite wedges is left out
    W[:, :, 4] = 1.0             # and so is one whose wedges do not vary
    P = covariance.pooled_correlation(W)
    np.testing.assert_allclose(np.diag(P), 1.0, rtol=1e-12)
    np.testing.assert_allclose(P, P.T, rtol=1e-12)
    assert np.max(np.abs(P - R)) < 0.05
    with pytest.raises(ValueError):
        covariance.pooled_correlation(np.ones((10, 3, 2)))


def test_autotune_keeps_the_exact_paint_where_the_context_holds_its_buffers(tmp_path, monkeypatch):
    import types
    monkeypatch.setattr(tune, "key_for", lambda est: "key")

    class DirectFaster(FakeTunable):
        def __init__(self, max_particles):
            super().__init__()
            self.params = types.SimpleNamespace(max_particles=max_particles)

        def autotune(self, *a, **kw):
            self.tuned_calls += 1
            return {"tile_y": 0, "ylm_harmonics": 8, "bin_blocks_per_sm": 0, "paint_binned": 0}

    est = DirectFaster(10 ** 6)
    got = tune.tuned(est, None, None, [0, 2, 4], [0.0, 0.1], path=str(tmp_path / "a.json"))
    assert got["paint_binned"] == 1 and est.applied["paint_binned"] == 1
    assert tune.load_cache(str(tmp_path / "a.json"))["key"]["paint_binned"] == 1
    # without tile buffers the direct paint is the only one, and the search's choice stands
    est0 = DirectFaster(0)
    assert tune.tuned(est0, None, None, [0, 2, 4], [0.0, 0.1], path=str(tmp_path / "b.json"))["paint_binned"] == 0
    # the caller may let the search choose the direct paint
    est1 = DirectFaster(10 ** 6)
    got1 = tune.tuned(est1, None, None, [0, 2, 4], [0.0, 0.1], path=str(tmp_path / "c.json"), keep_exact_paint=False)
    assert got1["paint_binned"] == 0
