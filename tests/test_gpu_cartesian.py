"""The Cartesian-decomposition route (pspec_multipoles_cartesian) against the oracle.

For l <= 4 the Cartesian route and the spherical-harmonic route compute the same estimator
(the oracle pins the two against each other to rounding); here the GPU's Cartesian route must
meet the same FP32 tolerance against the oracle and agree with the GPU's own SH route, and it
spends 1 + 6 + 15 transforms where the SH route spends 1 + 5 + 9 (Sec. 2.1).
"""
import math

import numpy as np
import pytest

import synth
from oracle import estimator as E
from oracle import brute as B
from tests._parity import check_fp32, gpu_estimator, uniform_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02357_gb300 import build
    build.build()


def _run(p, d, r, ells, edges):
    est = gpu_estimator(p, precision="fp32", ell_max=4, cartesian=True)
    est.paint(d.pos, r.pos, d.weight, d.nbar, r.weight, r.nbar)
    cart = est.multipoles_cartesian(ells, edges)
    n_cart = est.plan_info()["transforms_executed"]
    sh = est.multipoles(ells, edges)
    n_sh = est.plan_info()["transforms_executed"]
    info = est.plan_info()
    est.close()
    return cart, sh, n_cart, n_sh, info


def test_cartesian_route_on_a_survey_cap():
    geo = synth.survey_geometry()
    fld = synth.lognormal_field(64, geo.box_size, geo.box_corner, seed=7)
    d = synth.survey_catalog(fld, geo, nbar=1e-4, seed=37)
    r = synth.survey_randoms(5 * d.size, geo, seed=8)
    p = E.Params(nmesh=64, box_size=geo.box_size, box_corner=tuple(geo.box_corner), window="cic",
                 interlaced=True, compensate=True, P0=1e4, nbar=1e-4)
    edges = uniform_edges(0.005, 0.095, 0.01)
    ells = [0, 2, 4]
    o = E.multipoles(d, r, p, ells, edges)
    cart, sh, n_cart, n_sh, info = _run(p, d, r, ells, edges)
    rep = {}
    check_fp32(cart, o, ells, report=rep)
    assert rep[2]["bins_checked"] > 0 and rep[4]["bins_checked"] > 0
    np.testing.assert_array_equal(cart["n_modes"], o["n_modes"])
    scale = np.abs(o["P"][0])
    assert np.all(np.abs(cart["P"] - sh["P"]) <= 2e-5 * scale[None, :])
    # interlaced: F1, F2 and the round trip, then 6 + 15 (Cartesian) or 5 + 9 (SH) transforms
    assert n_cart == 3 + 6 + 15 and n_sh == 3 + 5 + 9
    assert info["cartesian_table_bytes"] == 64 * 64 * 32 * 4 * 21


@pytest.mark.parametrize("nmesh,window,interlaced", [(48, "tsc", True), (32, "cic", False)])
def test_cartesian_route_matches_the_oracle_cartesian_route(nmesh, window, interlaced):
    L = 400.0
    p = E.Params(nmesh=nmesh, box_size=L, box_corner=(0.0, 0.0, 0.0), observer=(-300.0, -200.0, -250.0),
                 window=window, interlaced=interlaced, compensate=True, P0=1e4, nbar=1e-5)
    d = synth.uniform_box(3000, L, (0.0, 0.0, 0.0), 51)
    r = synth.uniform_box(12000, L, (0.0, 0.0, 0.0), 52)
    edges = np.linspace(0.0, math.pi * nmesh / L, 8)
    ells = [0, 2, 4]
    fl = E.density_fields(d, r, p)
    bidx, mult, _ = E.mode_binning(nmesh, L, edges)
    oc = B.cartesian_multipoles(fl.f, fl.F0, p, fl.sums["I"], fl.sums["S"], ells, edges, (bidx, mult))
    cart, sh, _, _, _ = _run(p, d, r, ells, edges)
    scale = np.abs(oc["P"][0]) + fl.sums["S"] / fl.sums["I"]
    check_fp32(cart, oc, ells, scale=scale)


def test_cartesian_route_errors():
    from paper_1704_02357_gb300 import PspecError, pspec
    p = E.Params(nmesh=32, box_size=400.0, box_corner=(0.0, 0.0, 0.0), window="cic", interlaced=False,
                 compensate=True, P0=1e4, nbar=1e-5)
    d = synth.uniform_box(500, 400.0, (0.0, 0.0, 0.0), 53)
    r = synth.uniform_box(2000, 400.0, (0.0, 0.0, 0.0), 54)
    edges = np.linspace(0.0, 0.2, 5)
    est = gpu_estimator(p, precision="fp32", ell_max=6)
    est.paint(d.pos, r.pos)
    with pytest.raises(PspecError) as e:
        est.multipoles_cartesian([0, 2], edges)  # context made without the Cartesian table
    assert e.value.status == pspec.EUNSUPPORTED
    est.close()
    est = gpu_estimator(p, precision="fp32", ell_max=6, cartesian=True)
    est.paint(d.pos, r.pos)
    with pytest.raises(PspecError) as e:
        est.multipoles_cartesian([0, 6], edges)
    assert e.value.status == pspec.EUNSUPPORTED
    est.close()
    with pytest.raises(PspecError) as e:
        gpu_estimator(p, precision="fp64", ell_max=4, cartesian=True)
    assert e.value.status == pspec.EUNSUPPORTED
