"""Oracle (test infrastructure only): transverse mu = 0 systematics of Sec. 3.1, in FP64.

* ``response_closed``: R(mu) of eq. response, -(l_max+1)/(2 mu) L_lmax(0) L_{lmax+1}(mu).
* ``response_sum``: the same leakage from its definition, eq. Pobs-model: the reconstruction of
  a delta(mu) spike from the even multipoles up to l_max, with the sign of eq. response
  (observed minus true, per unit P_c): -sum_l (2l+1)/2 L_l(0) L_l(mu).
* ``mu_edges_nonuniform``: the wedge edges of eq. nonuniform-bins, found with numerical
  quadrature of L_{lmax+1}(t)/t and bracketing root finding.
* ``spike_wedge_ratios``: the wedges of the reconstructed spike relative to the first wedge.

Only tests and bench.py's baseline leg use this module.
"""
from __future__ import annotations

import numpy as np
from scipy import integrate, optimize, special


def response_closed(ell_max: int, mu):
    mu = np.asarray(mu, dtype=np.float64)
    lm0 = special.eval_legendre(ell_max, 0.0)
    with np.errstate(invalid="ignore", divide="ignore"):
        q = special.eval_legendre(ell_max + 1, mu) / mu
    # mu -> 0: L_{lmax+1}(mu)/mu -> L'_{lmax+1}(0)
    d0 = special.legendre(ell_max + 1).deriv()(0.0)
    q = np.where(mu == 0.0, d0, q)
    return -0.5 * (ell_max + 1) * lm0 * q


def response_sum(ell_max: int, mu):
    mu = np.asarray(mu, dtype=np.float64)
    s = np.zeros_like(mu)
    for ell in range(0, ell_max + 1, 2):
        s += 0.5 * (2 * ell + 1) * special.eval_legendre(ell, 0.0) * special.eval_legendre(ell, mu)
    return -s


def _g(ell_max: int, mu: float) -> float:
    f = lambda t: special.eval_legendre(ell_max + 1, t) / t if t != 0.0 else 0.0
    val, _ = integrate.quad(f, 0.0, mu, epsabs=1e-14, epsrel=1e-13, limit=200)
    return val


def mu_edges_nonuniform(ell_max: int) -> np.ndarray:
    g1 = _g(ell_max, 1.0)
    h = lambda m: _g(ell_max, m) - g1
    grid = np.linspace(1e-9, 1.0 - 1e-9, 4001)
    hv = np.array([h(m) for m in grid])
    roots = []
    for i in range(len(grid) - 1):
        if hv[i] == 0.0:
            roots.append(grid[i])
        elif np.sign(hv[i]) != np.sign(hv[i + 1]):
            roots.append(optimize.brentq(h, grid[i], grid[i + 1], xtol=1e-15, rtol=1e-15))
    return np.concatenate([[0.0], roots, [1.0]])


def spike_wedge_ratios(ell_max: int, mu_edges) -> np.ndarray:
    """Mean over each wedge of the reconstructed spike sum_l (2l+1)/2 L_l(0) L_l(mu), divided by
    its value in the first wedge."""
    e = np.asarray(mu_edges, dtype=np.float64)
    w = []
    for a, b in zip(e[:-1], e[1:]):
        val, _ = integrate.quad(lambda m: -response_sum(ell_max, m), a, b, epsabs=1e-14, limit=200)
        w.append(val / (b - a))
    w = np.array(w)
    return w / w[0]


# --------------------------------------------------------------------------- wedge statistics (Sec. 4.1)
def lbar_matrix(ells, mu_edges) -> np.ndarray:
    """(n_mu, n_ells) mean of L_l over each wedge, by numerical quadrature."""
    e = np.asarray(mu_edges, dtype=np.float64)
    out = np.empty((len(e) - 1, len(ells)))
    for w, (a, b) in enumerate(zip(e[:-1], e[1:])):
        for i, ell in enumerate(ells):
            val, _ = integrate.quad(lambda m: special.eval_legendre(ell, m), a, b, epsabs=1e-14)
            out[w, i] = val / (b - a)
    return out


def gamma_kaiser(ell_max: int, mu_edges, beta: float) -> np.ndarray:
    """gamma_mn of eq. gamma over the even multipoles 0..l_max, the mu integrals by quadrature."""
    ells = list(range(0, ell_max + 1, 2))
    Lb = lbar_matrix(ells, mu_edges)
    I = np.empty((len(ells), len(ells)))
    for a, la in enumerate(ells):
        for b, lb in enumerate(ells):
            f = lambda m: 0.5 * special.eval_legendre(la, m) * special.eval_legendre(lb, m) * (1 + beta * m * m) ** 4
            I[a, b], _ = integrate.quad(f, -1.0, 1.0, epsabs=1e-14, limit=200)
    D = np.array([2 * l + 1 for l in ells], dtype=np.float64)
    M = Lb * D[None, :]
    return M @ I @ M.T


def condition_number(M) -> float:
    """Smallest over largest singular value (the paper's definition, Sec. 4.1)."""
    s = np.linalg.svd(np.asarray(M, dtype=np.float64), compute_uv=False)
    return float(s.min() / s.max())


def correlation(C) -> np.ndarray:
    d = np.sqrt(np.diag(C))
    return C / np.outer(d, d)
