"""The survey workloads against the FP64 oracle, bin by bin, under the stated tolerances: a 96^3
survey cap at l <= 16, and at full size the benchmark's 512^3 workload (CIC + interlacing,
l = 0, 2, 4, FP32) and its l <= 16 TSC configuration.

At 512^3 the l <= 16 check uses the oracle's stored values (recomputing them would need ~150
full transforms and Y_lm evaluations, over an hour). The worst bins here sit close to the FP32
rounding floor of the transforms, so this file is collected after every other GPU test: a run
stopping at the first failure has run the rest.
"""
import math

import numpy as np
import pytest

import synth
from oracle import estimator as E
from tests._parity import check_fp32, run_gpu, uniform_edges

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02357_gb300 import build
    build.build()


def test_survey_shaped_high_ell_fp32():
    """A survey cap (lognormal, redshift-space, TSC + interlacing) at l <= 16, FP32, with
    the stated tolerances on bins where |P_l| > 1% |P_0|."""
    geo = synth.survey_geometry()
    fld = synth.lognormal_field(64, geo.box_size, geo.box_corner, seed=3)
    d = synth.survey_catalog(fld, geo, nbar=1e-4, seed=33)
    r = synth.survey_randoms(5 * d.size, geo, seed=4)
    r.nbar = np.full(r.size, 1e-4)
    p = E.Params(nmesh=96, box_size=geo.box_size, box_corner=tuple(geo.box_corner), window="tsc",
                 interlaced=True, compensate=True, P0=1e4, nbar=1e-4)
    edges = uniform_edges(0.005, 0.145, 0.01)
    ells = list(range(0, 17, 2))
    o = E.multipoles(d, r, p, ells, edges)
    g = run_gpu(p, d, r, ells, edges, precision="fp32")
    rep = {}
    check_fp32(g, o, ells, report=rep)
    assert rep[0]["bins_checked"] == len(edges) - 1
    assert rep[2]["bins_checked"] > 0 and rep[4]["bins_checked"] > 0


@pytest.fixture(scope="module")
def survey512_l4():
    """The benchmark's 512^3 catalog and the oracle's multipoles of it (computed once here)."""
    geo = synth.survey_geometry(box_size=2000.0)
    fld = synth.lognormal_field(256, geo.box_size, geo.box_corner, seed=3)
    d = synth.survey_catalog(fld, geo, nbar=3e-4, seed=33)
    r = synth.survey_randoms(20 * d.size, geo, seed=4)
    d.nbar = None
    p = E.Params(nmesh=512, box_size=2000.0, box_corner=tuple(geo.box_corner), window="cic", interlaced=True,
                 compensate=True, P0=1e4, nbar=3e-4)
    kn = math.pi * 512 / 2000.0
    edges = 0.005 * np.arange(int(kn / 0.005) + 1)
    ells = [0, 2, 4]
    return d, r, p, edges, ells, E.multipoles(d, r, p, ells, edges)


# fp32: the library default (exact-add harmonic and inverse transforms); fp32_plain: plain FP32
# radix trees, the transforms the benchmark's headline runs
@pytest.mark.parametrize("precision", ["fp32", "fp32_plain"])
def test_survey_512_l4_matches_oracle(survey512_l4, precision):
    d, r, p, edges, ells, o = survey512_l4
    g = run_gpu(p, d, r, ells, edges, precision=precision, max_particles=d.size + r.size)
    np.testing.assert_array_equal(g["n_modes"], o["n_modes"])
    np.testing.assert_allclose(g["k_mean"], o["k_mean"], rtol=1e-6)
    assert abs(g["stats"]["alpha"] - o["alpha"]) <= 1e-14 * o["alpha"]
    rep = {}
    check_fp32(g, o, ells, report=rep)
    assert rep[0]["bins_checked"] == len(edges) - 1 and rep[2]["bins_checked"] > 20 and rep[4]["bins_checked"] > 0
    print("full-size parity", precision, rep)


def test_survey_512_tsc_l16_matches_golden():
    """The l <= 16 benchmark configuration (512^3, TSC + interlacing + compensation, even l
    up to 16, FP32) against the FP64 oracle's values stored by
    tests/golden/make_survey512_tsc_l16.py (too slow to run here: ~150 full transforms),
    under 1e-5 (l <= 4) and 1e-4 (l <= 16) on bins where |P_l| > 1% |P_0|."""
    import importlib.util
    import os
    gold_dir = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_l16", os.path.join(gold_dir, "make_survey512_tsc_l16.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    d, r, p, edges = mk.case()
    gold = np.load(os.path.join(gold_dir, "survey512_tsc_l16.npz"))
    assert d.size == int(gold["n_data"]) and r.size == int(gold["n_randoms"])
    np.testing.assert_array_equal(edges, gold["edges"])
    ells = [int(x) for x in gold["ells"]]
    g = run_gpu(p, d, r, ells, edges, precision="fp32", max_particles=d.size + r.size)
    np.testing.assert_array_equal(g["n_modes"], gold["n_modes"])
    np.testing.assert_allclose(g["k_mean"], gold["k_mean"], rtol=1e-6)
    assert abs(g["stats"]["alpha"] - float(gold["alpha"])) <= 1e-14 * float(gold["alpha"])
    rep = {}
    check_fp32(g, {"P": gold["P"]}, ells, report=rep)
    assert all(rep[ell]["bins_checked"] > 100 for ell in ells)
    print("full-size l <= 16 parity:", {ell: (v["bins_checked"], f'{v["max_rel"]:.2e}') for ell, v in rep.items()})


@pytest.mark.parametrize("precision", ["fp32", "fp32_plain"])
def test_survey_512_l4_second_draw_matches_golden(precision):
    """A second Poisson draw of the 512^3 survey catalog (data seed 34), against the FP64
    oracle's values stored by tests/golden/make_survey512_cic_l4_s34.py. One of its high-k bins
    has P_4 = 1.4% of P_0, so any error that does not average down over the k shell (an FP32
    real-space Y_lm evaluation left 1.9e-5 there) shows under the 1e-5 rule."""
    import importlib.util
    import os
    gold_dir = os.path.join(os.path.dirname(__file__), "golden")
    spec = importlib.util.spec_from_file_location("make_s34", os.path.join(gold_dir, "make_survey512_cic_l4_s34.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    d, r, p, edges = mk.case()
    gold = np.load(os.path.join(gold_dir, "survey512_cic_l4_s34.npz"))
    assert d.size == int(gold["n_data"]) and r.size == int(gold["n_randoms"])
    np.testing.assert_array_equal(edges, gold["edges"])
    ells = [int(x) for x in gold["ells"]]
    g = run_gpu(p, d, r, ells, edges, precision=precision, max_particles=d.size + r.size)
    np.testing.assert_array_equal(g["n_modes"], gold["n_modes"])
    assert abs(g["stats"]["alpha"] - float(gold["alpha"])) <= 1e-14 * float(gold["alpha"])
    rep = {}
    check_fp32(g, {"P": gold["P"]}, ells, report=rep)
    assert all(rep[ell]["bins_checked"] > 100 for ell in ells)
    print("second draw, 512^3 l <= 4 parity:", {ell: (v["bins_checked"], f'{v["max_rel"]:.2e}') for ell, v in rep.items()})
