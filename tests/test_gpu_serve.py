"""Continuous-batching server: each result is the same alone and in the mix, and admission
respects the HBM budget."""
import math

import numpy as np
import pytest

import synth
from oracle import estimator as E
from tests._parity import check_fp32

pytestmark = pytest.mark.gpu

L = 400.0
CORNER = (0.0, 0.0, 0.0)
OBS = (-300.0, -200.0, -250.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02357_gb300 import build
    build.build()


def _edges(n):
    return np.linspace(0.0, math.pi * n / L, 7)


def _requests(device):
    import torch
    from paper_1704_02357_gb300.serve import Request
    rng = np.random.default_rng(5)
    shapes = [(32, 4), (48, 2), (64, 4), (32, 2), (48, 4), (64, 2), (32, 4), (48, 4)]
    reqs, cats = [], []
    for i, (n, l) in enumerate(shapes):
        cat = synth.uniform_box(int(rng.integers(800, 4000)), L, CORNER, 300 + i)
        cats.append(cat)
        reqs.append(Request(rid=i, nmesh=n, ell_max=l, pos=torch.as_tensor(cat.pos, device=device),
                            k_edges=_edges(n)))
    return reqs, cats


def _server(randoms_dev, budget, slots=2):
    from paper_1704_02357_gb300.serve import Server
    return Server(L, CORNER, randoms_for=lambda n: randoms_dev, hbm_budget=budget, observer=OBS, window="tsc",
                  interlaced=True, P0=1e4, nbar=1e-5, max_kbins=16, max_particles=5000, max_slots_per_shape=slots)


def test_results_alone_equal_results_in_the_mix():
    import torch
    dev = torch.device("cuda", 0)
    randoms = synth.uniform_box(12000, L, CORNER, 9)
    rdev = torch.as_tensor(randoms.pos, device=dev)
    reqs, cats = _requests(dev)
    # alone: one request at a time on an otherwise idle server
    srv = _server(rdev, budget=8 << 30)
    alone = {}
    for r in reqs:
        srv.submit(r)
        while srv.busy():
            srv.step()
        alone[r.rid] = srv.done[-1].P.copy()
    srv.close()
    # mixed: everything arrives at once and overlaps on the device
    reqs2, _ = _requests(dev)
    srv = _server(rdev, budget=8 << 30)
    done = srv.run(reqs2, [0.0] * len(reqs2))
    srv.close()
    assert len(done) == len(reqs2)
    for r in done:
        i = r.rid
        p = E.Params(nmesh=r.nmesh, box_size=L, box_corner=CORNER, observer=OBS, window="tsc", interlaced=True,
                     compensate=True, P0=1e4, nbar=1e-5)
        ells = list(range(0, r.ell_max + 1, 2))
        o = E.multipoles(cats[i], randoms, p, ells, r.k_edges)
        scale = np.abs(o["P"][0]) + o["S"] / o["I"]
        assert np.all(np.abs(r.P - alone[i]) <= 1e-5 * scale[None, :]), i
        check_fp32({"P": r.P}, o, ells, scale=scale)


def test_admission_respects_the_hbm_budget():
    import torch
    dev = torch.device("cuda", 0)
    randoms = synth.uniform_box(12000, L, CORNER, 9)
    rdev = torch.as_tensor(randoms.pos, device=dev)
    reqs, _ = _requests(dev)
    probe = _server(rdev, budget=1 << 40)
    fp = {n: probe._footprint(n, 4) for n in (32, 48, 64)}
    probe.close()
    budget = fp[64] + fp[48]  # never room for all three shapes at once
    srv = _server(rdev, budget=budget, slots=1)
    peak = 0
    order = list(range(len(reqs)))
    pending = [reqs[i] for i in order]
    for r in pending:
        srv.submit(r)
    while srv.busy():
        srv.step()
        peak = max(peak, srv.used())
    assert peak <= budget
    assert len(srv.done) == len(reqs)
    assert any(r.queue_wait > 0 for r in srv.done)
    srv.close()
