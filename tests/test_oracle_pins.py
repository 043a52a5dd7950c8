"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test ties one part of ``oracle.estimator`` to the paper's mathematics: a closed form,
a brute-force sum, an independent decomposition, an invariance or a printed number.
"""
import json
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.special import eval_legendre

from oracle import estimator as E
from oracle import brute as B
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _unit_vectors(n, seed):
    v = np.random.default_rng(seed).standard_normal((n, 3))
    return v / np.linalg.norm(v, axis=1)[:, None]


# ----------------------------------------------------------------------------- harmonics
@pytest.mark.parametrize("ell", list(range(0, 17)))
def test_addition_theorem(ell):
    """sum_m Y_lm(a) Y_lm(b) = (2l+1)/(4 pi) L_l(a.b) for the real harmonics (eq. add-theorem)."""
    a = _unit_vectors(2000, 1)
    b = _unit_vectors(2000, 2)
    lhs = sum(E.real_ylm(ell, m, *a.T) * E.real_ylm(ell, m, *b.T) for m in range(-ell, ell + 1))
    rhs = (2 * ell + 1) / (4 * math.pi) * eval_legendre(ell, np.sum(a * b, axis=1))
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * (2 * ell + 1)


def test_ylm_orthonormal():
    """Gauss-Legendre x trapezoid quadrature of Y_lm Y_l'm' over the sphere gives delta."""
    nth, nph = 40, 80
    x, wx = np.polynomial.legendre.leggauss(nth)
    phi = np.arange(nph) * 2 * math.pi / nph
    X, PH = np.meshgrid(x, phi, indexing="ij")
    W = np.repeat(wx[:, None], nph, axis=1) * (2 * math.pi / nph)
    s = np.sqrt(1 - X ** 2)
    ux, uy, uz = s * np.cos(PH), s * np.sin(PH), X
    lm = [(l, m) for l in range(0, 9) for m in range(-l, l + 1)]
    Y = np.array([E.real_ylm(l, m, ux, uy, uz).ravel() for l, m in lm])
    gram = (Y * W.ravel()) @ Y.T
    assert np.max(np.abs(gram - np.eye(len(lm)))) < 1e-12


def test_ylm_l2_closed_forms():
    forms = json.load(open(os.path.join(GOLDEN, "ylm_l2.json")))["forms"]
    u = _unit_vectors(500, 3)
    x, y, z = u.T
    ref = {
        0: math.sqrt(5 / math.pi) / 4 * (3 * z ** 2 - 1),
        1: -math.sqrt(15 / math.pi) / 2 * x * z,
        -1: -math.sqrt(15 / math.pi) / 2 * y * z,
        2: math.sqrt(15 / math.pi) / 4 * (x ** 2 - y ** 2),
        -2: math.sqrt(15 / math.pi) / 2 * x * y,
    }
    assert set(int(k) for k in forms) == set(ref)
    for m, r in ref.items():
        np.testing.assert_allclose(E.real_ylm(2, m, x, y, z), r, atol=1e-14)
    assert abs(E.real_ylm(0, 0, 1.0, 0.0, 0.0) - 1 / math.sqrt(4 * math.pi)) < 1e-15
    assert E.real_ylm(2, 0, 0.0, 0.0, 0.0) == 0.0


# ----------------------------------------------------------------------------- transform counts
def test_fft_counts_printed():
    g = json.load(open(os.path.join(GOLDEN, "fft_counts.json")))
    assert E.fft_count_sh(4) == g["ell_max_4"]["sh"] == 15
    assert E.fft_count_cartesian(4) == g["ell_max_4"]["cartesian"] == 22
    assert E.fft_count_sh(16) == g["ell_max_16"]["sh"] == 153
    assert E.fft_count_cartesian(16) == g["ell_max_16"]["cartesian"] == 525
    assert round(525 / 153, 1) == g["ell_max_16"]["ratio"]
    assert 2 * 4 + 1 == g["hexadecapole_alone"]["sh"]
    assert (4 + 1) * (4 + 2) // 2 == g["hexadecapole_alone"]["cartesian"]
    assert round(1 - 9 / 15, 2) == g["hexadecapole_alone"]["fewer_fraction"]
    for lmax in range(0, 33, 2):
        assert E.fft_count_sh(lmax) == (lmax + 2) * (lmax + 1) // 2
        assert E.fft_count_cartesian(lmax) == (lmax + 2) * (lmax + 4) * (2 * lmax + 3) // 24


# ----------------------------------------------------------------------------- DFT convention
@pytest.mark.parametrize("n", [4, 6, 8])
def test_rfft_is_half_of_brute_dft(n):
    x = np.random.default_rng(n).standard_normal((n, n, n))
    full = B.dft_brute(x)
    import scipy.fft as sfft
    half = sfft.rfftn(x)
    np.testing.assert_allclose(half, full[:, :, : n // 2 + 1], atol=1e-10)


# ----------------------------------------------------------------------------- painting
@pytest.mark.parametrize("window", ["cic", "tsc"])
@pytest.mark.parametrize("shift", [0.0, 0.5])
def test_paint_matches_loop(window, shift):
    p = E.Params(nmesh=8, box_size=80.0, box_corner=(-3.0, 5.0, 1.0), window=window)
    rng = np.random.default_rng(7)
    pos = np.asarray(p.box_corner) + rng.random((60, 3)) * 80.0
    pos[:5] = np.asarray(p.box_corner) + np.floor(rng.random((5, 3)) * 8) * 10.0  # on nodes
    vals = rng.standard_normal(60)
    np.testing.assert_allclose(E.paint(pos, vals, p, shift), B.paint_loop(pos, vals, p, shift), atol=1e-13)


@pytest.mark.parametrize("window", ["cic", "tsc"])
def test_paint_conserves_mass_and_on_node(window):
    p = E.Params(nmesh=8, box_size=8.0, box_corner=(0.0, 0.0, 0.0), window=window)
    rng = np.random.default_rng(3)
    pos = rng.random((100, 3)) * 8.0
    vals = rng.random(100)
    assert abs(E.paint(pos, vals, p).sum() - vals.sum()) < 1e-12
    mesh = E.paint(np.array([[3.0, 4.0, 5.0]]), np.array([1.0]), p)
    if window == "cic":
        assert mesh[3, 4, 5] == 1.0 and mesh.sum() == 1.0
    else:  # TSC on a node: 3/4 in the middle, 1/8 either side, per axis
        assert abs(mesh[3, 4, 5] - 0.75 ** 3) < 1e-15
        assert abs(mesh[2, 4, 5] - 0.125 * 0.75 ** 2) < 1e-15


@pytest.mark.parametrize("window", ["cic", "tsc"])
def test_window_transfer_is_kernel_fourier_transform(window):
    """Averaging the painted mesh's DFT x exp(i q u) over the particle's sub-cell offset u
    integrates the kernel over the whole line: the result is the kernel's Fourier
    transform, which the compensation must equal (Sec. 2.3 compensation)."""
    n = 16
    p = E.Params(nmesh=n, box_size=float(n), box_corner=(0.0, 0.0, 0.0), window=window)
    nu = 1024
    us = (np.arange(nu) + 0.5) / nu
    acc = np.zeros(n // 2, dtype=complex)
    import scipy.fft as sfft
    for u in us:
        mesh = E.paint(np.array([[5.0 + u, 2.0, 9.0]]), np.array([1.0]), p)
        F = sfft.rfftn(mesh)[:n // 2, 0, 0]
        q = 2 * math.pi * np.arange(n // 2) / n
        acc += F * np.exp(1j * q * (5.0 + u))
    acc /= nu
    W = E.window_transfer(n, window)[: n // 2, 0, 0]
    np.testing.assert_allclose(acc.real, W, atol=2e-6)
    assert np.max(np.abs(acc.imag)) < 2e-6


@pytest.mark.parametrize("window,p_ord", [("cic", 2), ("tsc", 3)])
@pytest.mark.parametrize("interlaced", [False, True])
def test_single_particle_alias_sum(window, p_ord, interlaced):
    """The combined field of one particle equals its Poisson alias sum; interlacing keeps
    only the even aliases, which pins the sign of the interlacing phase."""
    n = 16
    prm = E.Params(nmesh=n, box_size=float(n), box_corner=(0.0, 0.0, 0.0), window=window)
    u = 6.3137
    pos = np.array([[u, 0.0, 0.0]])
    import scipy.fft as sfft
    F1 = sfft.rfftn(E.paint(pos, np.array([1.0]), prm))
    if interlaced:
        F2 = sfft.rfftn(E.paint(pos, np.array([1.0]), prm, shift=0.5))
        X = 0.5 * (F1 + E.interlace_phase(n) * F2)
    else:
        X = F1
    for nx in range(0, n // 2):
        q = 2 * math.pi * nx / n
        ref = B.alias_sum_1d(q, u, p_ord, interlaced, nalias=4000 if p_ord == 2 else 1000)
        tol = 3e-5 if p_ord == 2 else 1e-7
        assert abs(X[nx, 0, 0] - ref) < tol, (nx, X[nx, 0, 0], ref)


# ----------------------------------------------------------------------------- the estimator
def _tiny_case(nmesh, seed, observer=(-37.0, -51.0, -23.0)):
    L = 10.0 * nmesh
    corner = (11.0, 7.0, 5.0)
    d = synth.on_node_catalog(40, nmesh, L, corner, seed)
    r = synth.on_node_catalog(90, nmesh, L, corner, seed + 1000)
    p = E.Params(nmesh=nmesh, box_size=L, box_corner=corner, observer=observer,
                 window="cic", interlaced=False, compensate=False, P0=2000.0, nbar=3e-4)
    kf = 2 * math.pi / L
    edges = np.arange(0.5, nmesh / 2, 1.0) * kf
    return d, r, p, edges


@pytest.mark.parametrize("nmesh", [8, 12, 16])
def test_mesh_estimator_equals_direct_sum(nmesh):
    """On-node particles, CIC, no compensation/interlacing: the SH-FFT estimator equals
    the local plane-parallel estimator summed over particles (eq. Pell-yama) exactly, odd l
    included (their imaginary part; the real part of an odd l and the imaginary part of an
    even l vanish)."""
    d, r, p, edges = _tiny_case(nmesh, 11)
    ells = [0, 1, 2, 3, 4, 5, 6, 8]
    a = E.multipoles(d, r, p, ells, edges)
    b = B.direct_multipoles(d, r, p, ells, edges)
    np.testing.assert_array_equal(a["n_modes"], b["n_modes"])
    np.testing.assert_allclose(a["k_mean"], b["k_mean"], rtol=1e-13)
    scale = np.max(np.abs(b["P"][0]))
    np.testing.assert_allclose(a["P"], b["P"], rtol=1e-9, atol=1e-10 * scale)
    assert np.max(np.abs(b["P_other"])) < 1e-10 * scale
    # the observer sits near the box: the end-point line of sight gives odd multipoles
    assert np.max(np.abs(b["P"][ells.index(1)])) > 1e-3 * scale
    assert abs(a["S"] - b["S"]) < 1e-12 * b["S"] and abs(a["I"] - b["I"]) < 1e-12 * b["I"]


def test_mirror_image_keeps_every_multipole():
    """Reflecting the catalogs and the observer through a plane maps each k shell onto itself
    and each end-point line of sight onto its mirror, so every P_l is unchanged, odd l
    included (pins the per-axis geometry of the moving line of sight; the sign of odd l is
    pinned by the direct sum above)."""
    d, r, p, edges = _tiny_case(12, 17)
    ells = [0, 1, 2, 3]
    a = E.multipoles(d, r, p, ells, edges)
    # the plane through c + (N - 1) H / 2 maps node i onto node N - 1 - i
    c = np.asarray(p.box_corner)
    x0 = 2 * c[0] + (p.nmesh - 1) * p.cell
    mirror = lambda x: np.column_stack([x0 - x[:, 0], x[:, 1], x[:, 2]])
    import copy
    d2, r2 = copy.deepcopy(d), copy.deepcopy(r)
    d2.pos, r2.pos = mirror(d.pos), mirror(r.pos)
    o = np.asarray(p.observer)
    p2 = E.Params(**{**p.__dict__, "observer": (x0 - o[0], o[1], o[2])})
    b = E.multipoles(d2, r2, p2, ells, edges)
    scale = np.max(np.abs(a["P"][0]))
    np.testing.assert_allclose(b["P"], a["P"], atol=1e-9 * scale)


def _offnode_case(nmesh=16, window="tsc", interlaced=True, compensate=True, seed=5,
                  observer=(-300.0, -200.0, -250.0)):
    L = 400.0
    corner = (0.0, 0.0, 0.0)
    d = synth.uniform_box(300, L, corner, seed)
    r = synth.uniform_box(900, L, corner, seed + 1)
    p = E.Params(nmesh=nmesh, box_size=L, box_corner=corner, observer=observer, window=window,
                 interlaced=interlaced, compensate=compensate, P0=1e4, nbar=1e-5)
    edges = np.linspace(0.0, math.pi * nmesh / L, 6)
    return d, r, p, edges


@pytest.mark.parametrize("window,interlaced", [("tsc", True), ("cic", False), ("cic", True)])
def test_sh_equals_cartesian_decomposition(window, interlaced):
    """For l <= 4 the spherical-harmonic route and the Cartesian route agree to rounding,
    and the Cartesian route spends 22 transforms (Sec. 2.1)."""
    d, r, p, edges = _offnode_case(window=window, interlaced=interlaced)
    fl = E.density_fields(d, r, p)
    ells = [0, 2, 4]
    a = E.multipoles_from_fields(fl, p, ells, edges)
    bidx, mult, _ = E.mode_binning(p.nmesh, p.box_size, edges)
    c = B.cartesian_multipoles(fl.f, fl.F0, p, fl.sums["I"], fl.sums["S"], ells, edges, (bidx, mult))
    assert c["n_fft"] == 22
    scale = np.max(np.abs(a["P"][0]))
    np.testing.assert_allclose(a["P"], c["P"], atol=1e-11 * scale, rtol=1e-10)


def test_distant_observer_limit():
    """With the observer very far along z the moving line of sight is fixed, and P_l is
    the ordinary mu-multipole (2l+1)/(I N_b) sum |F0|^2 L_l(khat_z) - delta_l0 S/I."""
    d, r, p, edges = _offnode_case(observer=(0.0, 0.0, -1e13), nmesh=16)
    fl = E.density_fields(d, r, p)
    ells = [0, 1, 2, 3, 4, 6, 8]
    a = E.multipoles_from_fields(fl, p, ells, edges)
    bidx, mult, n2 = E.mode_binning(p.nmesh, p.box_size, edges)
    _, _, khz = E.mode_khat(p.nmesh)
    sel = bidx >= 0
    nk = len(edges) - 1
    nm = np.bincount(bidx[sel], weights=mult[sel], minlength=nk)
    pw = np.abs(fl.F0) ** 2
    scale = np.max(np.abs(a["P"][0]))
    for li, ell in enumerate(ells):
        s = np.bincount(bidx[sel], weights=(mult * pw * eval_legendre(ell, khz))[sel], minlength=nk)
        # odd l: L_l(khat_z) |F0|^2 is odd in k, so the full shell average is 0
        ref = (2 * ell + 1) * s / (fl.sums["I"] * nm) if ell % 2 == 0 else np.zeros(nk)
        if ell == 0:
            ref = ref - fl.sums["S"] / fl.sums["I"]
        np.testing.assert_allclose(a["P"][li], ref, atol=1e-9 * scale)


def test_randoms_weight_rescaling_invariance():
    """Scaling every random's completeness weight by c divides alpha by c: alpha n_s, I and
    S are unchanged, so P_l is too (eq. FKP-density: alpha only normalises the randoms)."""
    d, r, p, edges = _offnode_case(nmesh=12)
    a = E.multipoles(d, r, p, [0, 2, 4], edges)
    r2 = synth.Catalog(pos=r.pos, weight=np.full(r.size, 3.7))
    b = E.multipoles(d, r2, p, [0, 2, 4], edges)
    assert abs(b["alpha"] * 3.7 - a["alpha"]) < 1e-15 * a["alpha"] * 10
    np.testing.assert_allclose(a["P"], b["P"], rtol=1e-10, atol=1e-12 * np.abs(a["P"]).max())


def test_translation_by_cells_invariance():
    d, r, p, edges = _offnode_case(nmesh=12)
    a = E.multipoles(d, r, p, [0, 2, 4], edges)
    sh = np.array([3, -2, 5]) * p.cell
    d2 = synth.Catalog(pos=d.pos + sh)
    r2 = synth.Catalog(pos=r.pos + sh)
    p2 = E.Params(**{**p.__dict__, "box_corner": tuple(np.asarray(p.box_corner) + sh),
                     "observer": tuple(np.asarray(p.observer) + sh)})
    b = E.multipoles(d2, r2, p2, [0, 2, 4], edges)
    np.testing.assert_allclose(a["P"], b["P"], rtol=1e-9, atol=1e-11 * np.abs(a["P"]).max())


def test_axis_permutation_invariance():
    d, r, p, edges = _offnode_case(nmesh=12)
    a = E.multipoles(d, r, p, [0, 2, 4, 6], edges)
    perm = [2, 0, 1]
    d2 = synth.Catalog(pos=d.pos[:, perm])
    r2 = synth.Catalog(pos=r.pos[:, perm])
    p2 = E.Params(**{**p.__dict__, "box_corner": tuple(np.asarray(p.box_corner)[perm]),
                     "observer": tuple(np.asarray(p.observer)[perm])})
    b = E.multipoles(d2, r2, p2, [0, 2, 4, 6], edges)
    np.testing.assert_allclose(a["P"], b["P"], rtol=1e-9, atol=1e-11 * np.abs(a["P"]).max())


def test_uniform_poisson_noise_and_normalisation():
    """Uniform Poisson points, CIC, no compensation: <|F0|^2> = S prod_d (1 - 2/3 sin^2(pi n_d/N))
    (the alias sum of the squared CIC window), and I = n̄^2 V for unit weights."""
    L, n = 1000.0, 32
    d = synth.uniform_box(20000, L, (500.0,) * 3, 1)
    r = synth.uniform_box(100000, L, (500.0,) * 3, 2)
    nbar = 20000 / L ** 3
    p = E.Params(nmesh=n, box_size=L, box_corner=(500.0,) * 3, window="cic",
                 interlaced=False, compensate=False, nbar=nbar)
    fl = E.density_fields(d, r, p)
    assert abs(fl.sums["I"] - nbar ** 2 * L ** 3) < 1e-12 * nbar ** 2 * L ** 3
    assert abs(fl.sums["alpha"] - 0.2) < 1e-15
    assert abs(fl.sums["S"] - (20000 + 0.04 * 100000)) < 1e-8
    full, half = E.int_freqs(n)
    c = lambda f: 1 - 2.0 / 3.0 * np.sin(math.pi * f / n) ** 2
    C = c(full)[:, None, None] * c(full)[None, :, None] * c(half)[None, None, :]
    ratio = np.abs(fl.F0) ** 2 / (fl.sums["S"] * C)
    sel = ~E.nyquist_mask(n)
    sel[0, 0, 0] = False
    m = ratio[sel].mean()
    assert abs(m - 1.0) < 5.0 / math.sqrt(sel.sum()), m


def test_offnode_mesh_close_to_direct_sum():
    """TSC + interlacing + compensation on off-node particles approximates the exact
    particle sum (eq. Pell-yama) at k < k_N/2 at the 1e-3 level or better (Sec. 2.3), and
    interlacing beats the same mesh without it. l = 2 is held loosely: there the mesh
    evaluates Y_lm at nodes instead of at particles, which moves the shot-noise quadrupole
    at the 1e-2 level."""
    obs = (-3000.0, -2000.0, -2500.0)
    err = {}
    for inter in (True, False):
        d, r, p, _ = _offnode_case(nmesh=32, seed=9, observer=obs, interlaced=inter)
        kn = math.pi * p.nmesh / p.box_size
        edges = np.linspace(0.05 * kn, 0.5 * kn, 5)
        a = E.multipoles(d, r, p, [0, 2], edges)
        b = B.direct_multipoles(d, r, p, [0, 2], edges)
        scale = np.max(np.abs(b["P"][0] + b["S"] / b["I"]))
        err[inter] = np.max(np.abs(a["P"] - b["P"]), axis=1) / scale
    assert err[True][0] < 2e-4, err
    assert err[True][0] < 0.5 * err[False][0], err
    assert err[True][1] < 2e-2, err


# ----------------------------------------------------------------------------- wedges
def test_lbar_closed_form_vs_quadrature():
    edges = [0.0, 0.05, 0.2, 0.4, 0.6, 0.8, 1.0]
    for ell in range(0, 17, 2):
        for lo, hi in zip(edges[:-1], edges[1:]):
            q = integrate.quad(lambda x: eval_legendre(ell, x), lo, hi, epsabs=1e-14)[0] / (hi - lo)
            assert abs(E.lbar(ell, lo, hi) - q) < 1e-12


def test_wedges_refuse_odd_multipoles():
    with pytest.raises(ValueError):
        E.wedges(np.ones((2, 3)), [0, 1], [0.0, 0.5, 1.0])


def test_wedge_sum_rule_and_pure_multipole():
    rng = np.random.default_rng(0)
    ells = list(range(0, 17, 2))
    P = rng.standard_normal((len(ells), 7))
    edges = np.array([0.0, 0.05, 0.2, 0.4, 0.6, 0.8, 1.0])
    w = E.wedges(P, ells, edges)
    np.testing.assert_allclose((np.diff(edges)[:, None] * w).sum(axis=0), P[0], atol=1e-13)
    pure = np.zeros_like(P)
    pure[3] = 1.0
    w = E.wedges(pure, ells, edges)
    ref = [E.lbar(6, a, b) for a, b in zip(edges[:-1], edges[1:])]
    np.testing.assert_allclose(w[:, 0], ref, atol=1e-15)
