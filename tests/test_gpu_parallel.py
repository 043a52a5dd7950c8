"""Harmonic ranges on one GPU: the ranks of a sharded run played one after another.

Raw bins of ranges that cover the harmonic list once, summed and finalized, must give what
one pspec_multipoles call gives and what the oracle gives.
"""
import math

import numpy as np
import pytest

import synth
from oracle import estimator as E
from tests._parity import check_fp32, gpu_estimator

pytestmark = pytest.mark.gpu

L = 400.0
CORNER = (0.0, 0.0, 0.0)
OBS = (-300.0, -200.0, -250.0)


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02357_gb300 import build
    build.build()


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
@pytest.mark.parametrize("world", [2, 3, 7])
def test_ranges_summed_equal_the_whole(precision, world):
    import torch
    from paper_1704_02357_gb300.parallel import harmonic_items, split
    p = E.Params(nmesh=48, box_size=L, box_corner=CORNER, observer=OBS, window="tsc", interlaced=True,
                 compensate=True, P0=1e4, nbar=1e-5)
    data = synth.uniform_box(4000, L, CORNER, 71)
    randoms = synth.uniform_box(16000, L, CORNER, 72)
    ells = [0, 2, 4, 6]
    edges = np.linspace(0.0, math.pi * 48 / L, 9)
    est = gpu_estimator(p, precision=precision, ell_max=6)
    est.paint(data.pos, randoms.pos)
    whole = est.multipoles(ells, edges)
    n = len(harmonic_items(ells))
    total = None
    for r in range(world):
        q0, q1 = split(n, world, r)
        b = est.multipoles_range(ells, edges, q0, q1, include_p0=(r == 0))
        total = b.clone() if total is None else total + b
    res = est.finalize_bins(total, ells, edges)
    torch.cuda.synchronize()
    P = res["P"].cpu().numpy()
    np.testing.assert_array_equal(res["n_modes"].cpu().numpy(), whole["n_modes"])
    o = E.multipoles(data, randoms, p, ells, edges)
    scale = np.abs(o["P"][0]) + o["S"] / o["I"]
    tol = 1e-6 if precision == "fp32" else 1e-11
    assert np.all(np.abs(P - whole["P"]) <= tol * scale[None, :])
    if precision == "fp32":
        check_fp32({"P": P}, o, ells, scale=scale)
    else:
        np.testing.assert_allclose(P, o["P"], rtol=1e-8, atol=1e-10 * scale.max())
    est.close()


def test_range_arguments_are_checked():
    from paper_1704_02357_gb300 import PspecError, pspec
    p = E.Params(nmesh=32, box_size=L, box_corner=CORNER, observer=OBS, window="cic", interlaced=False,
                 compensate=True, P0=1e4, nbar=1e-5)
    data = synth.uniform_box(1000, L, CORNER, 73)
    randoms = synth.uniform_box(4000, L, CORNER, 74)
    edges = np.linspace(0.0, 0.2, 5)
    est = gpu_estimator(p, precision="fp32", ell_max=4)
    with pytest.raises(PspecError) as e:
        est.multipoles_range([0, 2], edges, 0, 5)
    assert e.value.status == pspec.ESTATE
    est.paint(data.pos, randoms.pos)
    with pytest.raises(PspecError) as e:
        est.multipoles_range([0, 2], edges, 3, 1)
    assert e.value.status == pspec.EINVAL
    # an empty range gives the l = 0 bins only
    b = est.multipoles_range([0, 2], edges, 0, 0).cpu().numpy()
    assert np.all(b[1] == 0) and np.any(b[0] != 0)
    est.close()
