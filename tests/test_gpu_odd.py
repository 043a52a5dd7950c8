"""Odd multipoles (end-point line of sight, wide-angle terms) on the CUDA path against the oracle.

For odd l the shell average of eq. Pell-yama is purely imaginary and P_l reports its
imaginary part; the oracle's odd l are pinned to the direct particle sum in
test_oracle_pins.py. On the FP32 path the even l read Y_lm(khat) from the table and the odd
l evaluate it in the binning kernel, so both routes are covered here.
"""
import math

import numpy as np
import pytest

import synth
from oracle import estimator as E
from tests._parity import run_gpu, check_fp32, gpu_estimator, kf, uniform_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02357_gb300 import build
    build.build()


def _offnode(nmesh, window="tsc", interlaced=True, compensate=True, seed=5, nd=3000, nr=9000,
             observer=(-300.0, -200.0, -250.0)):
    L = 400.0
    corner = (0.0, 0.0, 0.0)
    d = synth.uniform_box(nd, L, corner, seed)
    r = synth.uniform_box(nr, L, corner, seed + 1)
    p = E.Params(nmesh=nmesh, box_size=L, box_corner=corner, observer=observer, window=window,
                 interlaced=interlaced, compensate=compensate, P0=1e4, nbar=nd / L ** 3)
    edges = np.linspace(0.0, math.pi * nmesh / L, 9)
    return d, r, p, edges


def test_on_node_odd_fp64_matches_oracle():
    nmesh = 16
    L = 10.0 * nmesh
    corner = (11.0, 7.0, 5.0)
    d = synth.on_node_catalog(40, nmesh, L, corner, 11)
    r = synth.on_node_catalog(90, nmesh, L, corner, 1011)
    p = E.Params(nmesh=nmesh, box_size=L, box_corner=corner, observer=(-37.0, -51.0, -23.0), window="cic",
                 interlaced=False, compensate=False, P0=2000.0, nbar=3e-4)
    edges = np.arange(0.5, nmesh / 2, 1.0) * kf(p)
    ells = [0, 1, 2, 3, 4, 5]
    g = run_gpu(p, d, r, ells, edges, precision="fp64")
    o = E.multipoles(d, r, p, ells, edges)
    scale = np.max(np.abs(o["P"][0]))
    assert np.max(np.abs(o["P"][1])) > 1e-3 * scale  # the odd terms are not trivially zero
    np.testing.assert_allclose(g["P"], o["P"], rtol=1e-8, atol=1e-10 * scale)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nmesh,window,interlaced,compensate", [
    (32, "tsc", True, True), (48, "cic", True, True), (64, "cic", False, True), (96, "tsc", False, False)])
def test_offnode_odd_matches_oracle(precision, nmesh, window, interlaced, compensate):
    d, r, p, edges = _offnode(nmesh, window, interlaced, compensate)
    ells = [0, 1, 2, 3, 4, 5, 7]
    g = run_gpu(p, d, r, ells, edges, precision=precision, ell_max=7)
    o = E.multipoles(d, r, p, ells, edges)
    np.testing.assert_array_equal(g["n_modes"], o["n_modes"])
    scale = np.abs(o["P"][0]) + o["S"] / o["I"]
    if precision == "fp64":
        np.testing.assert_allclose(g["P"], o["P"], rtol=1e-8, atol=1e-10 * scale.max())
    else:
        check_fp32(g, o, ells, scale=scale)


def test_odd_with_and_without_the_ylm_table():
    """FP32: a context with the Y table (even l from it, odd l evaluated) and one without
    (every l evaluated) give the oracle's odd and even multipoles alike."""
    d, r, p, edges = _offnode(48, "tsc", True, True, seed=9)
    ells = [0, 1, 2, 3, 4]
    o = E.multipoles(d, r, p, ells, edges)
    scale = np.abs(o["P"][0]) + o["S"] / o["I"]
    for table in (True, False):
        g = run_gpu(p, d, r, ells, edges, precision="fp32", ylm_table=table)
        assert (g["plan"]["ylm_table_bytes"] > 0) == table
        check_fp32(g, o, ells, scale=scale)


def test_survey_shaped_dipole_fp32():
    """A survey cap seen from the observer at the origin: the wide-angle dipole and octupole
    of the end-point line of sight, FP32, under the tolerance rule on the bins where
    |P_l| > 1% |P_0|."""
    geo = synth.survey_geometry()
    fld = synth.lognormal_field(64, geo.box_size, geo.box_corner, seed=3)
    d = synth.survey_catalog(fld, geo, nbar=1e-4, seed=33)
    r = synth.survey_randoms(5 * d.size, geo, seed=4)
    r.nbar = np.full(r.size, 1e-4)
    p = E.Params(nmesh=96, box_size=geo.box_size, box_corner=tuple(geo.box_corner), window="tsc",
                 interlaced=True, compensate=True, P0=1e4, nbar=1e-4)
    edges = uniform_edges(0.005, 0.145, 0.01)
    ells = [0, 1, 2, 3, 4]
    o = E.multipoles(d, r, p, ells, edges)
    g = run_gpu(p, d, r, ells, edges, precision="fp32")
    rep = {}
    check_fp32(g, o, ells, report=rep)
    assert rep[0]["bins_checked"] == len(edges) - 1
    assert rep[1]["max_abs_over_P0"] < 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_odd_harmonic_ranges_sum_to_the_whole(precision):
    import torch
    from paper_1704_02357_gb300.parallel import harmonic_items, split
    d, r, p, edges = _offnode(32, "cic", True, True, seed=21)
    ells = [0, 1, 2, 3]
    est = gpu_estimator(p, precision=precision, ell_max=3)
    est.paint(d.pos, r.pos)
    whole = est.multipoles(ells, edges)
    n = len(harmonic_items(ells))
    assert n == 3 + 5 + 7
    total = None
    for rank in range(3):
        q0, q1 = split(n, 3, rank)
        b = est.multipoles_range(ells, edges, q0, q1, include_p0=(rank == 0))
        total = b.clone() if total is None else total + b
    res = est.finalize_bins(total, ells, edges)
    torch.cuda.synchronize()
    P = res["P"].cpu().numpy()
    o = E.multipoles(d, r, p, ells, edges)
    scale = np.abs(o["P"][0]) + o["S"] / o["I"]
    tol = 1e-6 if precision == "fp32" else 1e-11
    assert np.all(np.abs(P - whole["P"]) <= tol * scale[None, :])
    est.close()


def test_odd_l_is_refused_where_it_is_undefined():
    import torch
    from paper_1704_02357_gb300 import PspecError, pspec, wedges
    d, r, p, edges = _offnode(32, "cic", False, True, seed=23, nd=500, nr=2000)
    est = gpu_estimator(p, precision="fp32", ell_max=4, cartesian=True)
    est.paint(d.pos, r.pos)
    with pytest.raises(PspecError) as e:
        est.multipoles([0, 5], edges)  # above the context's ell_max
    assert e.value.status == pspec.EUNSUPPORTED
    with pytest.raises(PspecError) as e:
        est.multipoles_cartesian([0, 1], edges)
    assert e.value.status == pspec.EUNSUPPORTED
    est.close()
    P = torch.zeros((2, 4), dtype=torch.float64, device="cuda")
    with pytest.raises(PspecError) as e:
        wedges(P, [0, 1], np.array([0.0, 0.5, 1.0]))
    assert e.value.status == pspec.EUNSUPPORTED
