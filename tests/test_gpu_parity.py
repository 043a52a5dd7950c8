"""CUDA path (libpspec through its C ABI) against the FP64 oracle, element by element.

Sizes here are ones the oracle finishes in seconds; they span several FFT tiles and
include radix-3 meshes (48, 96). The survey workloads under the stated tolerances (96^3 at
l <= 16, 512^3 at l <= 4 and l <= 16) live in test_zzz_survey.py.
"""
import math

import numpy as np
import pytest

import synth
from oracle import estimator as E
from tests._parity import run_gpu, check_fp32, uniform_edges, kf, gpu_estimator

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02357_gb300 import build
    build.build()


def _tiny(nmesh, seed=11, observer=(-37.0, -51.0, -23.0)):
    L = 10.0 * nmesh
    corner = (11.0, 7.0, 5.0)
    d = synth.on_node_catalog(40, nmesh, L, corner, seed)
    r = synth.on_node_catalog(90, nmesh, L, corner, seed + 1000)
    p = E.Params(nmesh=nmesh, box_size=L, box_corner=corner, observer=observer, window="cic",
                 interlaced=False, compensate=False, P0=2000.0, nbar=3e-4)
    edges = np.arange(0.5, nmesh / 2, 1.0) * kf(p)
    return d, r, p, edges


@pytest.mark.parametrize("nmesh", [16, 48, 64])
def test_on_node_fp64_matches_oracle(nmesh):
    d, r, p, edges = _tiny(nmesh)
    ells = [0, 2, 4, 6, 8]
    g = run_gpu(p, d, r, ells, edges, precision="fp64")
    o = E.multipoles(d, r, p, ells, edges)
    np.testing.assert_array_equal(g["n_modes"], o["n_modes"])
    np.testing.assert_allclose(g["k_mean"], o["k_mean"], rtol=1e-12)
    scale = np.abs(o["P"][0]).max()
    np.testing.assert_allclose(g["P"], o["P"], rtol=1e-9, atol=1e-11 * scale)
    assert abs(g["stats"]["alpha"] - o["alpha"]) <= 1e-15 * o["alpha"]
    assert abs(g["stats"]["I"] - o["I"]) <= 1e-13 * o["I"]
    assert abs(g["stats"]["S"] - o["S"]) <= 1e-13 * o["S"]


@pytest.mark.parametrize("nmesh", [16, 48])
def test_on_node_fp32_matches_oracle(nmesh):
    d, r, p, edges = _tiny(nmesh)
    ells = [0, 2, 4, 6, 8]
    g = run_gpu(p, d, r, ells, edges, precision="fp32")
    o = E.multipoles(d, r, p, ells, edges)
    np.testing.assert_array_equal(g["n_modes"], o["n_modes"])
    scale = np.abs(o["P"][0]) + o["S"] / o["I"]
    check_fp32(g, o, ells, scale=scale)


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


@pytest.mark.parametrize("nmesh,window,interlaced,compensate", [
    (32, "tsc", True, True), (48, "cic", True, True), (32, "cic", False, True), (96, "tsc", False, False),
    (64, "tsc", True, False)])
def test_offnode_fp64_matches_oracle(nmesh, window, interlaced, compensate):
    d, r, p, edges = _offnode(nmesh, window, interlaced, compensate)
    ells = [0, 2, 4, 6, 8]
    g = run_gpu(p, d, r, ells, edges, precision="fp64")
    o = E.multipoles(d, r, p, ells, edges)
    np.testing.assert_array_equal(g["n_modes"], o["n_modes"])
    scale = (np.abs(o["P"][0]) + o["S"] / o["I"]).max()
    np.testing.assert_allclose(g["P"], o["P"], rtol=1e-8, atol=1e-10 * scale)


@pytest.mark.parametrize("nmesh,window,interlaced", [(32, "tsc", True), (48, "cic", True), (64, "cic", False)])
def test_offnode_fp32_matches_oracle(nmesh, window, interlaced):
    d, r, p, edges = _offnode(nmesh, window, interlaced)
    ells = [0, 2, 4, 6, 8, 10, 12, 14, 16]
    g = run_gpu(p, d, r, ells, edges, precision="fp32")
    o = E.multipoles(d, r, p, ells, edges)
    np.testing.assert_array_equal(g["n_modes"], o["n_modes"])
    scale = np.abs(o["P"][0]) + o["S"] / o["I"]
    check_fp32(g, o, ells, scale=scale)


def test_config_plain_box_64():
    """64^3, 1000 Mpc/h box with its corner 500 Mpc/h from the observer, 2e4 data and 1e5
    randoms uniform (seeds 1, 2), unit weights, CIC, k bins 0-0.3 in steps of 0.01."""
    L, corner = 1000.0, (500.0, 500.0, 500.0)
    d = synth.uniform_box(20000, L, corner, 1)
    r = synth.uniform_box(100000, L, corner, 2)
    p = E.Params(nmesh=64, box_size=L, box_corner=corner, window="cic", interlaced=False, compensate=True,
                 nbar=20000 / L ** 3)
    edges = uniform_edges(0.0, 0.3, 0.01)
    ells = [0, 2, 4]
    o = E.multipoles(d, r, p, ells, edges)
    g64 = run_gpu(p, d, r, ells, edges, precision="fp64")
    g32 = run_gpu(p, d, r, ells, edges, precision="fp32")
    fin = np.isfinite(o["P"])
    np.testing.assert_array_equal(np.isfinite(g64["P"]), fin)
    np.testing.assert_array_equal(g64["n_modes"], o["n_modes"])
    np.testing.assert_array_equal(g32["n_modes"], o["n_modes"])
    scale = np.nanmax(np.abs(o["P"][0])) + o["S"] / o["I"]
    assert np.nanmax(np.abs(g64["P"] - o["P"])) <= 1e-10 * scale
    check_fp32(g32, o, ells, scale=np.abs(o["P"][0]) + o["S"] / o["I"])


def test_transform_counts_follow_the_paper():
    d, r, p, edges = _offnode(16, seed=2, nd=200, nr=600)
    est = gpu_estimator(p, precision="fp32", ell_max=16)
    est.paint(d.pos, r.pos)
    est.multipoles([0, 2, 4], edges)
    info = est.plan_info()
    assert info["sh_transforms"] == 15
    # executed: F1, F2 (interlaced), the inverse of the combined field, and 2l+1 per l >= 2
    assert info["transforms_executed"] == 3 + 5 + 9
    est.multipoles(list(range(0, 17, 2)), edges)
    assert est.plan_info()["sh_transforms"] == 153
    est.close()


def test_repeat_and_empty_data():
    d, r, p, edges = _offnode(16, seed=3, nd=300, nr=900)
    est = gpu_estimator(p, precision="fp64", ell_max=4)
    est.paint(d.pos, r.pos)
    a = est.multipoles([0, 2, 4], edges)
    b = est.multipoles([4, 0], edges)
    np.testing.assert_allclose(b["P"][1], a["P"][0], rtol=1e-12)
    np.testing.assert_allclose(b["P"][0], a["P"][2], rtol=1e-12)
    empty = synth.Catalog(pos=np.zeros((0, 3)))
    st = est.paint(empty.pos, r.pos)
    assert st["W_d"] == 0.0 and st["alpha"] == 0.0
    o = E.multipoles(empty, r, p, [0, 2], edges)
    g = est.multipoles([0, 2], edges)
    np.testing.assert_allclose(g["P"], o["P"], rtol=1e-9, equal_nan=True)
    est.close()


def test_bins_beyond_nyquist_are_empty_nan():
    d, r, p, _ = _offnode(16, seed=4, nd=300, nr=900)
    kn = math.pi * p.nmesh / p.box_size
    edges = np.array([0.0, 0.5 * kn, kn, 3.0 * kn, 4.0 * kn])
    g = run_gpu(p, d, r, [0, 2], edges, precision="fp64")
    o = E.multipoles(d, r, p, [0, 2], edges)
    np.testing.assert_array_equal(g["n_modes"], o["n_modes"])
    assert g["n_modes"][3] == 0 and np.all(np.isnan(g["P"][:, 3])) and np.isnan(g["k_mean"][3])
    np.testing.assert_allclose(g["P"][:, :3], o["P"][:, :3], rtol=1e-9)


def test_wedges_match_oracle():
    import torch
    from paper_1704_02357_gb300 import wedges
    rng = np.random.default_rng(1)
    ells = list(range(0, 17, 2))
    P = rng.standard_normal((len(ells), 37))
    mu = np.array([0.0, 0.05, 0.2, 0.4, 0.6, 0.8, 1.0])
    out = wedges(torch.tensor(P, device="cuda"), ells, mu)
    torch.cuda.synchronize()
    np.testing.assert_allclose(out.cpu().numpy(), E.wedges(P, ells, mu), rtol=1e-13, atol=1e-14)


def test_wedges_of_host_multipoles_through_a_device_copy():
    """The boundary as a caller uses it: pspec_multipoles returns host P_l; the caller copies
    them to the device and pspec_wedges combines them there (Sec. 2.2 eqs. wedge-est, Lbar).
    Against the oracle's wedges of the oracle's multipoles, and exactly the oracle's wedges of
    the host P (the wedge step is FP64 on both sides)."""
    import torch
    from paper_1704_02357_gb300 import wedges
    d, r, p, edges = _offnode(48, "tsc", True, seed=31)
    ells = [0, 2, 4, 6]
    mu = np.array([0.0, 0.05, 0.2, 0.4, 0.6, 0.8, 1.0])
    g = run_gpu(p, d, r, ells, edges, precision="fp32")          # host arrays out
    Pd = torch.as_tensor(g["P"]).to("cuda")                      # the caller's device copy
    out = wedges(Pd, ells, mu)
    torch.cuda.synchronize()
    w = out.cpu().numpy()
    np.testing.assert_allclose(w, E.wedges(g["P"], ells, mu), rtol=1e-13, atol=1e-12 * np.abs(g["P"]).max())
    o = E.multipoles(d, r, p, ells, edges)
    wo = E.wedges(o["P"], ells, mu)
    scale = np.abs(o["P"][0]) + o["S"] / o["I"]
    # |Lbar_l| <= 1, so a wedge moves by at most the sum of the multipoles' tolerances
    bound = sum(1e-5 if ell <= 4 else 1e-4 for ell in ells) * scale
    assert np.all(np.abs(w - wo) <= bound[None, :])


def test_errors_are_reported_not_faulted():
    from paper_1704_02357_gb300 import PspecError
    from paper_1704_02357_gb300 import pspec
    d, r, p, edges = _offnode(16, seed=6, nd=100, nr=300)
    est = gpu_estimator(p, precision="fp32", ell_max=4)
    with pytest.raises(PspecError) as e:
        est.multipoles([0], edges)
    assert e.value.status == pspec.ESTATE
    est.paint(d.pos, r.pos)
    for ells, ed, st in [([5], edges, pspec.EUNSUPPORTED), ([6], edges, pspec.EUNSUPPORTED),
                         ([0, 0], edges, pspec.EINVAL), ([0], edges[::-1], pspec.EINVAL),
                         ([0], np.array([0.1]), pspec.EINVAL), ([0], np.array([0.0, np.nan]), pspec.EINVAL)]:
        with pytest.raises(PspecError) as e:
            est.multipoles(ells, ed)
        assert e.value.status == st, (ells, ed)
    bad = d.pos.copy()
    bad[5, 1] = np.nan
    with pytest.raises(PspecError) as e:
        est.paint(bad, r.pos)
    assert e.value.status == pspec.EINVAL
    with pytest.raises(PspecError) as e:
        est.paint(d.pos, np.zeros((0, 3)))
    assert e.value.status == pspec.EINVAL
    # the context is still usable
    est.paint(d.pos, r.pos)
    g = est.multipoles([0, 2], edges)
    assert np.all(np.isfinite(g["P"][:, 1:]))
    est.close()
    with pytest.raises(PspecError):
        gpu_estimator(E.Params(nmesh=20, box_size=1.0, box_corner=(0, 0, 0)))


def test_float32_positions_and_weights():
    d, r, p, edges = _offnode(32, seed=8, nd=2000, nr=6000)
    d.weight = 0.5 + np.random.default_rng(0).random(d.size)
    r.nbar = np.full(r.size, p.nbar * 1.3)
    o = E.multipoles(d, r, p, [0, 2], edges)
    g = run_gpu(p, d, r, [0, 2], edges, precision="fp64")
    np.testing.assert_allclose(g["P"], o["P"], rtol=1e-8, atol=1e-10 * np.abs(o["P"][0]).max())
    d32 = synth.Catalog(pos=d.pos.astype(np.float32), weight=d.weight)
    r32 = synth.Catalog(pos=r.pos.astype(np.float32), nbar=r.nbar)
    o32 = E.multipoles(synth.Catalog(pos=d32.pos.astype(np.float64), weight=d.weight),
                       synth.Catalog(pos=r32.pos.astype(np.float64), nbar=r.nbar), p, [0, 2], edges)
    g32 = run_gpu(p, d32, r32, [0, 2], edges, precision="fp64")
    np.testing.assert_allclose(g32["P"], o32["P"], rtol=1e-8, atol=1e-10 * np.abs(o["P"][0]).max())


@pytest.mark.parametrize("nmesh,window,interlaced", [(32, "tsc", True), (48, "cic", True), (64, "cic", False),
                                                      (32, "tsc", False)])
def test_tile_binned_paint_matches_oracle_and_direct(nmesh, window, interlaced):
    """The tile-binned paint (FP32 meshes) gives the oracle's multipoles within the FP32
    tolerance, including particles outside the box (painted periodically), and agrees with
    the direct atomic paint."""
    d, r, p, edges = _offnode(nmesh, window, interlaced, seed=12)
    rng = np.random.default_rng(3)
    shift = rng.integers(-1, 2, size=(d.size, 3)) * p.box_size
    d = synth.Catalog(pos=d.pos + shift * (rng.random((d.size, 1)) < 0.1))
    ells = [0, 2, 4, 6]
    o = E.multipoles(d, r, p, ells, edges)
    gb = run_gpu(p, d, r, ells, edges, precision="fp32", max_particles=d.size + r.size)
    gd = run_gpu(p, d, r, ells, edges, precision="fp32", max_particles=0)
    assert gb["stats"]["n_wrapped"] > 0
    assert gb["stats"]["n_wrapped"] == gd["stats"]["n_wrapped"]
    scale = np.abs(o["P"][0]) + o["S"] / o["I"]
    check_fp32(gb, o, ells, scale=scale)
    assert np.all(np.abs(gb["P"] - gd["P"]) <= 2e-5 * scale[None, :])


def test_tile_binned_paint_falls_back_when_catalog_exceeds_capacity():
    d, r, p, edges = _offnode(32, seed=13, nd=2000, nr=6000)
    o = E.multipoles(d, r, p, [0, 2], edges)
    g = run_gpu(p, d, r, [0, 2], edges, precision="fp32", max_particles=1000)
    check_fp32(g, o, [0, 2], scale=np.abs(o["P"][0]) + o["S"] / o["I"])


@pytest.mark.parametrize("knobs", [dict(tile_y=1), dict(ylm_harmonics=2), dict(bin_blocks_per_sm=1),
                                   dict(paint_binned=0), dict(tile_y=1, ylm_harmonics=3, bin_blocks_per_sm=2)])
def test_tuning_knobs_keep_parity(knobs):
    """Every runtime knob setting is a different launch shape of the same computation."""
    d, r, p, edges = _offnode(64, "tsc", True, seed=21)
    ells = [0, 2, 4, 6]
    o = E.multipoles(d, r, p, ells, edges)
    est = gpu_estimator(p, precision="fp32", ell_max=6, max_particles=d.size + r.size)
    est.set_tuning(**knobs)
    est.paint(d.pos, r.pos)
    g = est.multipoles(ells, edges)
    est.close()
    check_fp32(g, o, ells, scale=np.abs(o["P"][0]) + o["S"] / o["I"])


def test_autotune_picks_valid_knobs_and_caches(tmp_path):
    from paper_1704_02357_gb300 import tune
    d, r, p, edges = _offnode(64, "cic", True, seed=22)
    ells = [0, 2, 4]
    est = gpu_estimator(p, precision="fp32", ell_max=4, max_particles=d.size + r.size)
    path = str(tmp_path / "tuning.json")
    first = tune.tuned(est, d.pos, r.pos, ells, edges, path=path)
    assert not first["cached"] and first["paint_binned"] in (0, 1) and first["tile_y"] in (0, 1)
    second = tune.tuned(est, d.pos, r.pos, ells, edges, path=path)
    assert second["cached"] and all(second[k] == first[k] for k in ("paint_binned", "ylm_harmonics",
                                                                      "bin_blocks_per_sm", "tile_y"))
    est.paint(d.pos, r.pos)
    g = est.multipoles(ells, edges)
    est.close()
    o = E.multipoles(d, r, p, ells, edges)
    check_fp32(g, o, ells, scale=np.abs(o["P"][0]) + o["S"] / o["I"])


def test_ylm_table_and_per_mode_paths_match_oracle():
    """FP32 binning with the Y_lm(khat) table (default) and with per-mode FP32 evaluation
    (ylm_table = -1) both meet the tolerance; the plan reports the table it holds."""
    geo = synth.survey_geometry()
    fld = synth.lognormal_field(64, geo.box_size, geo.box_corner, seed=5)
    d = synth.survey_catalog(fld, geo, nbar=1e-4, seed=35)
    r = synth.survey_randoms(5 * d.size, geo, seed=6)
    p = E.Params(nmesh=64, box_size=geo.box_size, box_corner=tuple(geo.box_corner), window="cic",
                 interlaced=True, compensate=True, P0=1e4, nbar=1e-4)
    edges = uniform_edges(0.005, 0.095, 0.01)
    ells = [0, 2, 4, 6]
    o = E.multipoles(d, r, p, ells, edges)
    out = {}
    for table in (True, False):
        g = run_gpu(p, d, r, ells, edges, precision="fp32", ylm_table=table)
        check_fp32(g, o, ells)
        nbytes = 64 * 64 * 32 * 4 * (5 + 9 + 13)
        assert g["plan"]["ylm_table_bytes"] == (nbytes if table else 0)
        assert g["plan"]["ylm_rtable_bytes"] == (2 * nbytes if table else 0)  # Y_lm(rhat) of every node
        out[table] = g["P"]
    scale = np.abs(o["P"][0])
    assert np.all(np.abs(out[True] - out[False]) <= 2e-5 * scale[None, :])
    # FP64 contexts never hold the table
    g = run_gpu(p, d, r, [0, 2], edges, precision="fp64", ell_max=6)
    assert g["plan"]["ylm_table_bytes"] == 0


@pytest.mark.parametrize("form", ["jing", "sinc_per_mode"])
@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("nmesh,window,interlaced", [(32, "cic", False), (48, "tsc", True)])
def test_compensation_forms_match_oracle(form, precision, nmesh, window, interlaced):
    """compensate = 2: the alias-summed divisor of Jing (2005) in place of prod sinc^p;
    compensate = 3: the field left as painted and 1/W^2 applied to each binned mode."""
    from dataclasses import replace
    d, r, p, edges = _offnode(nmesh, window, interlaced, seed=31)
    p = replace(p, compensation=form)
    ells = [0, 2, 4]
    o = E.multipoles(d, r, p, ells, edges)
    g = run_gpu(p, d, r, ells, edges, precision=precision)
    scale = np.abs(o["P"][0]) + o["S"] / o["I"]
    if precision == "fp64":
        np.testing.assert_allclose(g["P"], o["P"], rtol=1e-8, atol=1e-10 * scale.max())
    else:
        check_fp32(g, o, ells, scale=scale)
    # and it differs from the field-level sinc form (the test has teeth)
    o_sinc = E.multipoles(d, r, replace(p, compensation="sinc"), ells, edges)
    k = 0 if form == "jing" else 1  # per mode, l = 0 is identical by construction
    assert np.max(np.abs(o_sinc["P"][k] - o["P"][k]) / scale) > 1e-4


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_columns_beyond_the_last_bin_are_skipped_exactly(precision):
    """Bins ending well below k_N: the harmonics' y pass stores, and the binning pass reads,
    only x columns (ky, kz) that hold a binned mode (whole y-pass slabs drop out here). The
    result equals the oracle's, also when the same context alternates low and full edges."""
    d, r, p, _ = _offnode(64, "tsc", True, True, seed=31)
    ells = [0, 1, 2, 4]
    low = np.linspace(0.0, 0.3 * math.pi * 64 / p.box_size, 6)
    full = np.linspace(0.0, math.pi * 64 / p.box_size * math.sqrt(3.0), 7)
    est = gpu_estimator(p, precision=precision, ell_max=4)
    est.paint(d.pos, r.pos)
    for edges in (low, full, low):
        g = est.multipoles(ells, edges)
        o = E.multipoles(d, r, p, ells, edges)
        np.testing.assert_array_equal(g["n_modes"], o["n_modes"])
        fin = o["n_modes"] > 0
        scale = (np.abs(o["P"][0]) + o["S"] / o["I"])[fin]
        if precision == "fp64":
            np.testing.assert_allclose(g["P"][:, fin], o["P"][:, fin], rtol=1e-8, atol=1e-10 * scale.max())
        else:
            check_fp32({"P": g["P"][:, fin]}, {"P": o["P"][:, fin]}, ells, scale=scale)
    est.close()
