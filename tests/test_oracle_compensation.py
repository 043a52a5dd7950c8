"""Pins of the compensation forms (Sec. 2.3, which cites Jing 2005 for the aliasing correction)."""
import math

import numpy as np
import pytest

import synth
from oracle import estimator as E


@pytest.mark.parametrize("window,p", [("cic", 2), ("tsc", 3)])
def test_jing_form_is_the_alias_sum_of_the_window(window, p):
    """prod_d C_p: the closed form of sum_m sinc^{2p}(pi (n/N + m)), checked against the sum itself."""
    n = 16
    W2 = E.window_transfer(n, window, "jing") ** 2
    full = np.fft.fftfreq(n, d=1.0 / n)
    m = np.arange(-4000, 4001)[:, None]
    a = np.pi * (full[None, :] / n + m)
    c1 = np.sum(np.where(a == 0, 1.0, np.sin(a) / np.where(a == 0, 1.0, a)) ** (2 * p), axis=0)
    ref = c1[:, None, None] * c1[None, :, None] * c1[None, None, : n // 2 + 1][..., : W2.shape[2]]
    np.testing.assert_allclose(W2, ref[:, :, : W2.shape[2]], rtol=0, atol=1e-9)


def test_jing_compensation_flattens_the_aliased_shot_noise():
    """Uniform Poisson points, non-interlaced CIC: with the Jing form P_0 (noise subtracted)
    stays near zero up to k_N; the plain sinc form leaves the alias excess, which matches
    the mean of C(k)/W^2(k) - 1 over the bin's modes."""
    L, n = 500.0, 32
    d = synth.uniform_box(40000, L, (0, 0, 0), 1)
    r = synth.uniform_box(400000, L, (0, 0, 0), 2)
    edges = np.linspace(0.0, math.pi * n / L, 9)
    res = {}
    for form in ("sinc", "jing"):
        p = E.Params(nmesh=n, box_size=L, box_corner=(0, 0, 0), observer=(L / 2, L / 2, -1e7), window="cic",
                     interlaced=False, compensate=True, compensation=form, P0=0.0, nbar=40000 / L ** 3)
        o = E.multipoles(d, r, p, [0], edges)
        res[form] = o["P"][0] / (o["S"] / o["I"])
    assert np.all(np.abs(res["jing"][-2:]) < 0.05)
    # expected sinc excess in the top bin: mean over its modes of C/W^2 - 1
    b, mult, _ = E.mode_binning(n, L, edges)
    ratio = (E.window_transfer(n, "cic", "jing") / E.window_transfer(n, "cic", "sinc")) ** 2 - 1.0
    top = b == len(edges) - 2
    expect = np.sum((mult * ratio)[top]) / np.sum(mult[top])
    assert expect > 0.15
    assert abs(res["sinc"][-1] - expect) < 0.05


def _offnode_case(observer):
    L, n = 400.0, 16
    d = synth.uniform_box(800, L, (0.0, 0.0, 0.0), 5)
    r = synth.uniform_box(3000, L, (0.0, 0.0, 0.0), 6)
    edges = np.linspace(0.0, math.pi * n / L, 6)
    return d, r, L, n, edges


@pytest.mark.parametrize("interlaced", [False, True])
def test_per_mode_compensation_equals_field_compensation_where_it_must(interlaced):
    """|X/W|^2 = |X|^2/W^2, so P_0 agrees for any observer; in the distant-observer limit
    Y_lm(rhat) is constant and every P_l agrees; with a near observer P_2 differs."""
    from dataclasses import replace
    ells = [0, 2, 4]
    for obs, all_equal in (((-300.0, -200.0, -250.0), False), ((200.0, 200.0, -1e13), True)):
        d, r, L, n, edges = _offnode_case(obs)
        p = E.Params(nmesh=n, box_size=L, box_corner=(0, 0, 0), observer=obs, window="tsc", interlaced=interlaced,
                     compensate=True, P0=1e4, nbar=800 / L ** 3)
        a = E.multipoles(d, r, p, ells, edges)
        b = E.multipoles(d, r, replace(p, compensation="sinc_per_mode"), ells, edges)
        scale = np.max(np.abs(a["P"][0]) + a["S"] / a["I"])
        np.testing.assert_allclose(b["P"][0], a["P"][0], rtol=1e-10, atol=1e-12 * scale)
        if all_equal:
            np.testing.assert_allclose(b["P"], a["P"], rtol=1e-6, atol=1e-8 * scale)
        else:
            assert np.max(np.abs(b["P"][1] - a["P"][1])) > 1e-4 * scale
