"""Batched mocks against one cached randoms catalog (pspec_set_randoms / pspec_run_batch).

Each mock of a batch must give what the single-catalog path (pspec_paint + pspec_multipoles)
and the oracle give for that mock with the shared randoms; the graph-replayed batch must
agree with the eager one.
"""
import math

import numpy as np
import pytest

import synth
from oracle import estimator as E
from tests._parity import check_fp32, gpu_estimator, run_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02357_gb300 import build
    build.build()


L = 400.0
CORNER = (0.0, 0.0, 0.0)


def _mocks(n, seed0=40, base=1500):
    out = []
    for i in range(n):
        out.append(synth.uniform_box(base + 400 * i, L, CORNER, seed0 + i))
    return out


def _params(nmesh, window="tsc", interlaced=True, precision_nbar=1e-5):
    return E.Params(nmesh=nmesh, box_size=L, box_corner=CORNER, observer=(-300.0, -200.0, -250.0), window=window,
                    interlaced=interlaced, compensate=True, P0=1e4, nbar=precision_nbar)


@pytest.mark.parametrize("use_graph", [True, False])
@pytest.mark.parametrize("nmesh,window,interlaced", [(32, "tsc", True), (48, "cic", False)])
def test_batch_matches_single_path_and_oracle(use_graph, nmesh, window, interlaced):
    p = _params(nmesh, window, interlaced)
    randoms = synth.uniform_box(9000, L, CORNER, 7)
    mocks = _mocks(4)
    edges = np.linspace(0.0, math.pi * nmesh / L, 9)
    ells = [0, 2, 4]
    est = gpu_estimator(p, precision="fp32", ell_max=4, cache_randoms=True,
                        max_particles=max(m.size for m in mocks))
    est.set_randoms(randoms.pos)
    res = est.run_batch([m.pos for m in mocks], ells, edges, use_graph=use_graph)
    import torch
    torch.cuda.synchronize()
    Pb = res["P"].cpu().numpy()
    sums = res["sums"].cpu().numpy()
    for i, m in enumerate(mocks):
        o = E.multipoles(m, randoms, p, ells, edges)
        g = run_gpu(p, m, randoms, ells, edges, precision="fp32")
        np.testing.assert_array_equal(res["n_modes"].cpu().numpy(), o["n_modes"])
        scale = np.abs(o["P"][0]) + o["S"] / o["I"]
        check_fp32({"P": Pb[i]}, o, ells, scale=scale)
        assert np.all(np.abs(Pb[i] - g["P"]) <= 2e-5 * scale[None, :])
        assert abs(sums[i, 0] - o["alpha"]) <= 1e-14 * o["alpha"]
        assert abs(sums[i, 1] - o["I"]) <= 1e-12 * o["I"]
        assert abs(sums[i, 2] - o["S"]) <= 1e-12 * o["S"]
    info = est.plan_info()
    assert info["kernel_launches"] > 0
    est.close()


def test_batch_fp64_matches_oracle():
    p = _params(32)
    randoms = synth.uniform_box(6000, L, CORNER, 8)
    mocks = _mocks(3, seed0=60)
    edges = np.linspace(0.0, math.pi * 32 / L, 7)
    ells = [0, 2, 4, 6]
    est = gpu_estimator(p, precision="fp64", ell_max=6, cache_randoms=True)
    est.set_randoms(randoms.pos)
    res = est.run_batch([m.pos for m in mocks], ells, edges)
    Pb = res["P"].cpu().numpy()
    for i, m in enumerate(mocks):
        o = E.multipoles(m, randoms, p, ells, edges)
        scale = (np.abs(o["P"][0]) + o["S"] / o["I"]).max()
        np.testing.assert_allclose(Pb[i], o["P"], rtol=1e-8, atol=1e-10 * scale)
    est.close()


def test_batch_runner_groups_mesh_sizes():
    from paper_1704_02357_gb300.batch import BatchRunner
    randoms = synth.uniform_box(8000, L, CORNER, 9)
    mocks = _mocks(5, seed0=80)
    meshes = [32, 48, 32, 48, 32]
    ells = [0, 2]
    edges_for = lambda n: np.linspace(0.0, math.pi * n / L, 7)
    br = BatchRunner(L, CORNER, randoms.pos, observer=(-300.0, -200.0, -250.0), window="tsc", interlaced=True,
                     P0=1e4, nbar=1e-5, ell_max=2)
    out = br.run([m.pos for m in mocks], meshes, ells, edges_for)
    for i, m in enumerate(mocks):
        p = _params(meshes[i])
        o = E.multipoles(m, randoms, p, ells, edges_for(meshes[i]))
        check_fp32({"P": out[i]["P"].cpu().numpy()}, o, ells, scale=np.abs(o["P"][0]) + o["S"] / o["I"])
    br.close()


def test_batch_requires_cached_randoms():
    from paper_1704_02357_gb300 import PspecError, pspec
    p = _params(32)
    m = _mocks(1)[0]
    edges = np.linspace(0.0, 0.2, 5)
    est = gpu_estimator(p, precision="fp32", ell_max=2)
    with pytest.raises(PspecError) as e:
        est.set_randoms(m.pos)
    assert e.value.status == pspec.ESTATE
    est.close()
    est = gpu_estimator(p, precision="fp32", ell_max=2, cache_randoms=True)
    with pytest.raises(PspecError) as e:
        est.run_batch([m.pos], [0, 2], edges)
    assert e.value.status == pspec.ESTATE
    est.close()


def test_graph_replay_writes_the_current_calls_buffers():
    """A batch graph captured in one call and replayed in the next writes that next call's output
    tensors: the first call's buffers (filled with NaN in between) stay untouched, and the second
    call's results equal the first's for the same mocks. (Graph nodes keep the pointers they were
    captured with, so the destinations are read from device memory.)"""
    import torch
    p = _params(32, "cic", True)
    randoms = synth.uniform_box(9000, L, CORNER, 7)
    mocks = _mocks(2)
    edges = np.linspace(0.0, math.pi * 32 / L, 9)
    est = gpu_estimator(p, precision="fp32", ell_max=4, cache_randoms=True,
                        max_particles=max(m.size for m in mocks))
    est.set_randoms(randoms.pos)
    first = est.run_batch([m.pos for m in mocks], [0, 2], edges, use_graph=True)
    torch.cuda.synchronize()
    P1, s1 = first["P"].clone(), first["sums"].clone()
    first["P"].fill_(float("nan"))
    first["sums"].fill_(float("nan"))
    torch.cuda.synchronize()
    second = est.run_batch([m.pos for m in mocks], [0, 2], edges, use_graph=True)
    torch.cuda.synchronize()
    assert torch.isnan(first["P"]).all() and torch.isnan(first["sums"]).all()
    # equal up to the order of the FP64 bin atomics
    np.testing.assert_allclose(second["P"].cpu().numpy(), P1.cpu().numpy(), rtol=1e-12, atol=0)
    np.testing.assert_allclose(second["sums"].cpu().numpy(), s1.cpu().numpy(), rtol=1e-12, atol=0)
