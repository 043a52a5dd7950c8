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


@pytest.mark.parametrize("ell_max", [4, 16])
def test_lbar_quadrature_matches_the_antiderivative(ell_max):
    """Mean Legendre polynomial over a wedge: quadrature against [L_{l+1} - L_{l-1}]/((2l+1) dmu)."""
    e = np.linspace(0.0, 1.0, 10)
    ells = list(range(0, ell_max + 1, 2))
    Lb = S.lbar_matrix(ells, e)
    for w, (a, b) in enumerate(zip(e[:-1], e[1:])):
        for i, l in enumerate(ells):
            ref = 1.0 if l == 0 else ((special.eval_legendre(l + 1, b) - special.eval_legendre(l - 1, b))
                                      - (special.eval_legendre(l + 1, a) - special.eval_legendre(l - 1, a))) / ((2 * l + 1) * (b - a))
            assert Lb[w, i] == pytest.approx(ref, abs=1e-12)


def test_gamma_without_rsd_is_the_orthogonality_form():
    """beta = 0: int dmu/2 L_l L_l' = delta_ll'/(2l+1), so gamma = Lbar diag(2l+1) Lbar^T."""
    e = S.mu_edges_nonuniform(8)
    ells = list(range(0, 9, 2))
    Lb = S.lbar_matrix(ells, e)
    ref = Lb @ np.diag([2.0 * l + 1 for l in ells]) @ Lb.T
    np.testing.assert_allclose(S.gamma_kaiser(8, e, 0.0), ref, rtol=1e-10, atol=1e-12)


def test_gamma_is_symmetric_positive_definite_with_as_many_wedges_as_multipoles():
    e = np.linspace(0.0, 1.0, 6)
    g = S.gamma_kaiser(8, e, 0.35)
    np.testing.assert_allclose(g, g.T, atol=1e-12)
    assert np.all(np.linalg.eigvalsh(g) > 0)


def test_uniform_wedges_become_ill_conditioned_at_high_lmax():
    """Sec. 4.1: with N_mu = l_max/2 + 1 wedges both binnings are well conditioned at l_max = 4;
    the uniform one becomes nearly singular by l_max = 16 while the non-uniform one does not."""
    def conds(lm):
        u = np.linspace(0.0, 1.0, lm // 2 + 2)
        nu = S.mu_edges_nonuniform(lm)
        return S.condition_number(S.gamma_kaiser(lm, u, 0.35)), S.condition_number(S.gamma_kaiser(lm, nu, 0.35))
    cu4, cn4 = conds(4)
    cu16, cn16 = conds(16)
    assert cu4 > 0.1 and cn4 > 0.1
    assert cu16 < 1e-4 and cn16 > 1e-2
    ells = list(range(0, 17, 2))
    assert S.condition_number(S.lbar_matrix(ells, np.linspace(0, 1, 10))) < 1e-3
    assert S.condition_number(S.lbar_matrix(ells, S.mu_edges_nonuniform(16))) > 5e-2
