"""Pins of the oracle's transverse-systematics functions (Sec. 3.1)."""
import numpy as np
import pytest
from scipy import integrate, special

from oracle import systematics as S


@pytest.mark.parametrize("ell_max", [2, 4, 8, 16])
def test_response_closed_form_equals_the_multipole_sum(ell_max):
    """Eq. response (Christoffel summation) equals the truncated Legendre expansion of the spike."""
    mu = np.linspace(-1.0, 1.0, 401)
    np.testing.assert_allclose(S.response_closed(ell_max, mu), S.response_sum(ell_max, mu), atol=1e-12)


def test_response_values():
    # l_max = 2: -(3/2) L_2(0) L_3(mu)/mu; at mu = 1: -(3/2)(-1/2)(1) = 0.75
    assert S.response_closed(2, [1.0])[0] == pytest.approx(0.75, abs=1e-15)
    # the reconstructed spike integrates to 1 over [-1, 1] (the delta's weight) for every l_max
    for lm in (2, 4, 16):
        val, _ = integrate.quad(lambda m: -S.response_sum(lm, m), -1.0, 1.0)
        assert val == pytest.approx(1.0, abs=1e-12)


@pytest.mark.parametrize("ell_max", [2, 4, 6, 8, 16])
def test_nonuniform_edges_cancel_the_spike_beyond_the_first_wedge(ell_max):
    e = S.mu_edges_nonuniform(ell_max)
    assert len(e) == ell_max // 2 + 2 and e[0] == 0.0 and e[-1] == 1.0
    assert np.all(np.diff(e) > 0)
    for a, b in zip(e[1:-1], e[2:]):
        val, _ = integrate.quad(lambda t: special.eval_legendre(ell_max + 1, t) / t, a, b, epsabs=1e-14)
        assert abs(val) < 1e-10
    # the first wedge's width follows the uniform 1/(l_max/2 + 1) closely (Sec. 3.1)
    assert abs(e[1] - 1.0 / (ell_max / 2 + 1)) < 0.1 / (ell_max / 2 + 1)
    r = S.spike_wedge_ratios(ell_max, e)
    assert np.all(np.abs(r[1:]) < 1e-9)


def test_uniform_wedges_stay_contaminated():
    r = S.spike_wedge_ratios(16, np.linspace(0.0, 1.0, 10))
    assert np.max(np.abs(r[1:])) > 0.05
