"""Transverse (mu = 0) systematics, Sec. 3.1 and the box test of Sec. 3.2, on the GPU path.

A lattice catalog whose weights carry a sinusoidal modulation in the plane of the sky (the
x direction; the observer is far along z) puts all the power of one k bin in two modes at
mu = 0: the toy model's spike. Its multipoles up to l = 16 turned into wedges leave the spike
in every uniform wedge, in the proportions the response predicts, and only in the first of
the non-uniform wedges.
"""
import math

import numpy as np
import pytest

from oracle import estimator as E
from oracle import systematics as S
from tests._parity import gpu_estimator

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02357_gb300 import build
    build.build()


@pytest.mark.parametrize("ell_max", [2, 4, 8, 16])
def test_host_functions_match_the_oracle(ell_max):
    from paper_1704_02357_gb300 import pspec as P
    np.testing.assert_allclose(P.mu_edges_nonuniform(ell_max), S.mu_edges_nonuniform(ell_max), atol=1e-10)
    mu = np.linspace(-1.0, 1.0, 257)
    np.testing.assert_allclose(P.transverse_response(ell_max, mu), S.response_closed(ell_max, mu), atol=1e-11)


def test_host_functions_reject_bad_arguments():
    from paper_1704_02357_gb300 import PspecError, pspec as P
    for bad in (0, 3, 18):
        with pytest.raises(PspecError):
            P.mu_edges_nonuniform(bad)
    with pytest.raises(PspecError):
        P.transverse_response(4, np.array([1.5]))


class _Cat:
    def __init__(self, pos, weight):
        self.pos, self.weight, self.nbar = pos, weight, None


def _lattice_case(n=64, L=1000.0, m=8, amp=0.5):
    H = L / n
    g = np.arange(n) * H
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pos = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    data = _Cat(pos, 1.0 + amp * np.cos(2.0 * math.pi * m * pos[:, 0] / L))
    randoms = _Cat(pos.copy(), np.ones(len(pos)))
    p = E.Params(nmesh=n, box_size=L, box_corner=(0.0, 0.0, 0.0), observer=(L / 2, L / 2, -1e7), window="cic",
                 interlaced=False, compensate=False, P0=0.0, nbar=n ** 3 / L ** 3)
    kf = 2.0 * math.pi / L
    edges = np.array([m - 1.5, m - 0.5, m + 0.5, m + 1.5]) * kf  # the spike sits in bin 1
    return p, data, randoms, edges


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_nonuniform_wedges_confine_a_transverse_spike(precision):
    import torch
    from paper_1704_02357_gb300 import pspec as P
    p, d, r, edges = _lattice_case()
    ells = list(range(0, 17, 2))
    est = gpu_estimator(p, precision=precision, ell_max=16)
    est.paint(d.pos, r.pos, d.weight, None, r.weight, None)
    nk = len(edges) - 1
    Pd = torch.empty(len(ells) * nk, dtype=torch.float64, device="cuda")
    km = torch.empty(nk, dtype=torch.float64, device="cuda")
    nm = torch.empty(nk, dtype=torch.float64, device="cuda")
    est.multipoles_device(ells, edges, Pd, km, nm)
    Pl = Pd.view(len(ells), nk)
    tol = 1e-4 if precision == "fp64" else 2e-4
    for mu_edges, theory in ((np.linspace(0.0, 1.0, 10), True), (P.mu_edges_nonuniform(16), False)):
        W = P.wedges(Pl, ells, mu_edges).cpu().numpy()
        spike = W[:, 1] - W[:, 0]  # bin 0 holds only the constant noise offset of P_0
        ratio = spike / spike[0]
        if theory:
            np.testing.assert_allclose(ratio, S.spike_wedge_ratios(16, mu_edges), atol=tol)
            assert np.max(np.abs(ratio[1:])) > 0.05
        else:
            assert np.max(np.abs(ratio[1:])) < tol, ratio
    est.close()


@pytest.mark.parametrize("ell_max", [4, 16])
def test_wedge_statistics_host_functions_match_the_oracle(ell_max):
    from paper_1704_02357_gb300 import pspec as P
    ells = list(range(0, ell_max + 1, 2))
    for e in (np.linspace(0.0, 1.0, 10), P.mu_edges_nonuniform(ell_max)):
        np.testing.assert_allclose(P.wedge_lbar(ells, e), S.lbar_matrix(ells, e), atol=1e-12)
        for beta in (0.0, 0.35):
            g = P.wedge_gamma_kaiser(ell_max, e, beta)
            np.testing.assert_allclose(g, S.gamma_kaiser(ell_max, e, beta), rtol=1e-9, atol=1e-10 * np.abs(g).max())


def test_mock_wedge_covariance_follows_the_gaussian_prediction():
    """Poisson boxes (white noise only, so beta = 0 in the Gaussian prediction) through the
    batched path at l <= 16; wedge correlations pooled over k bins against gamma_mn, for 9
    uniform and 9 non-uniform wedges, and the non-uniform ones are the more diagonal."""
    import torch
    import synth
    from paper_1704_02357_gb300 import covariance as CV, pspec as P
    L, n, nm = 600.0, 64, 128
    p = E.Params(nmesh=n, box_size=L, box_corner=(0.0, 0.0, 0.0), observer=(L / 2, L / 2, -1e7), window="cic",
                 interlaced=True, compensate=True, P0=0.0, nbar=30000 / L ** 3)
    kf = 2.0 * math.pi / L
    edges = kf * np.arange(6.0, 31.0, 2.0)
    ells = list(range(0, 17, 2))
    est = gpu_estimator(p, precision="fp32", ell_max=16, cache_randoms=True)
    est.set_randoms(synth.uniform_box(600000, L, (0.0, 0.0, 0.0), 199).pos)
    mocks = [synth.uniform_box(30000, L, (0.0, 0.0, 0.0), 200 + i).pos for i in range(nm)]
    res = est.run_batch(mocks, ells, edges)
    torch.cuda.synchronize()
    rms = {}
    for name, e in (("uniform", np.linspace(0.0, 1.0, 10)), ("nonuniform", P.mu_edges_nonuniform(16))):
        W = CV.mock_wedges(res["P"], ells, e).cpu().numpy()
        rho = CV.pooled_correlation(W)
        rho_th = S.correlation(S.gamma_kaiser(16, e, 0.0))
        assert np.max(np.abs(rho - rho_th)) < 0.12, (name, np.round(rho - rho_th, 3))
        off = rho[~np.eye(9, dtype=bool)]
        rms[name] = float(np.sqrt(np.mean(off ** 2)))
    assert rms["nonuniform"] < rms["uniform"]
    est.close()
