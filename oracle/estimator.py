"""Plain FP64 restatement of the SH-FFT multipole estimator (Hand, Li, Slepian & Seljak 2017).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__``). Written for a reader checking it
against the paper by eye: no blocking, fusion or reordering beyond what the paper states.
Library primitives used as steps: ``numpy.fft``/``scipy.fft`` (r2c and c2r DFTs),
``scipy.special.lpmv`` (associated Legendre functions), ``scipy.special.eval_legendre``.

Conventions, and the readings of the paper they encode:

* Mesh: N^3 nodes at x_i = corner + i*H, H = L/N, index order (x, y, z), z fastest.
* Forward DFT with exp(-i k.x), unnormalised; integer frequencies n in [-N/2, N/2).
* F(r) = w (n - alpha n_s) is kept unnormalised; the 1/I is applied once (Sec. 2.1,
  eq. FKP-density; the text divides by I twice, we divide once).
* alpha = sum of data completeness weights / sum of randoms completeness weights.
* I = alpha * sum_randoms nbar * w_c * w_fkp^2  (discrete form of int w^2 nbar^2).
* S = sum_data v^2 + alpha^2 sum_randoms v^2 with v = w_c * w_fkp: the i = j terms of the
  pair sum, subtracted from l = 0 only (Sec. 2.1, shot-noise equation and the sentence
  after it).
* Painting: CIC nodes floor(u), floor(u)+1; TSC nodes around c = floor(u + 1/2); periodic
  wrap; the interlaced second mesh is painted at u - 1/2 (Sec. 2.3).
* Interlacing: X = (F1 + exp(-i k.s) F2)/2 with s = (H/2)(1,1,1) (Sec. 2.3).
* Compensation: X /= prod_d sinc^p(pi n_d / N), p = 2 (CIC) or 3 (TSC), applied to the
  combined field before the inverse transform (Sec. 2.3 is silent on where).
* When interlacing or compensation is on, every mode with some n_d = -N/2 is zeroed in X
  before the inverse transform, and f = c2r(X)/N^3 is the field that gets Y_lm weights
  (Sec. 2.3: sum in Fourier space, inverse transform, then weight). With neither, f is the
  painted mesh itself.
* Binning: modes with some n_d = -N/2 and the k = 0 mode are left out. Mode n is in bin b
  iff t_b <= |n|^2 < t_{b+1}, t_b = (k_b L / 2 pi)^2 evaluated in FP64. In the half
  spectrum a mode with n_z = 0 counts once, 0 < n_z < N/2 twice (itself and -n).
* P_0(k_b) = (sum_b mult |F0|^2 / N_b - S) / I;
  P_l(k_b) = 4 pi / (I N_b) * sum_b mult * sum_m Y_lm(khat) Re[G_lm conj(F0)], l >= 2,
  with G_lm = DFT[f * Y_lm(rhat)] (Sec. 2.1 eqs. Pell-ours and Fell: the (2l+1) in front
  cancels the 4 pi/(2l+1) of the addition theorem).
* Odd l: eq. Pell-yama's shell average of A_l(k) conj(A_0(k)) (A = sum v L_l exp(-i k.r)) is
  purely imaginary for odd l (the terms at k and -k are complex conjugates up to the sign of
  L_l), so P_l reports its imaginary part, 4 pi/(I N_b) sum mult sum_m Y_lm(khat)
  Im[G_lm conj(F0)]; no shot noise. Eq. Pell-ours as printed, with F_l(-k), would flip the
  sign of odd l; the definition followed is eq. Pell-yama, the estimator being accelerated.
* Real spherical harmonics per eq. real-Ylm; Y_lm at the zero vector is 0 for l > 0.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from typing import Dict, Optional, Sequence

import numpy as np
import scipy.fft as sfft
from scipy.special import eval_legendre, lpmv, gammaln

CIC, TSC = "cic", "tsc"
WINDOW_ORDER = {CIC: 2, TSC: 3}


def _workers() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


@dataclass
class Params:
    nmesh: int
    box_size: float
    box_corner: Sequence[float]
    observer: Sequence[float] = (0.0, 0.0, 0.0)
    window: str = CIC
    interlaced: bool = False
    compensate: bool = True
    P0: float = 0.0          # FKP P0; 0 means w_fkp = 1
    nbar: float = 0.0        # n̄ used when a catalog carries none
    compensation: str = "sinc"  # "sinc": prod_d sinc^p; "jing": the alias-summed form of Jing (2005)

    @property
    def cell(self) -> float:
        return self.box_size / self.nmesh


# --------------------------------------------------------------------------- catalog sums
def fkp_weight(nbar: np.ndarray, P0: float) -> np.ndarray:
    """FKP weight w = 1 / (1 + n̄ P0) (Sec. 2.1, the weighting w(r) of eq. FKP-density)."""
    nbar = np.asarray(nbar, dtype=np.float64)
    if P0 <= 0.0:
        return np.ones_like(nbar)
    return 1.0 / (1.0 + nbar * P0)


def _cat_arrays(cat, params: Params):
    n = cat.pos.shape[0]
    wc = np.ones(n) if cat.weight is None else np.asarray(cat.weight, dtype=np.float64)
    nb = np.full(n, params.nbar) if cat.nbar is None else np.asarray(cat.nbar, dtype=np.float64)
    return wc, nb


def catalog_sums(data, randoms, params: Params) -> Dict[str, float]:
    """alpha, I and S of the FKP field (Sec. 2.1, eq. FKP-density and the noise term)."""
    wc_d, nb_d = _cat_arrays(data, params)
    wc_r, nb_r = _cat_arrays(randoms, params)
    wf_d = fkp_weight(nb_d, params.P0)
    wf_r = fkp_weight(nb_r, params.P0)
    W_d = float(np.sum(wc_d))
    W_r = float(np.sum(wc_r))
    alpha = W_d / W_r
    I = alpha * float(np.sum(nb_r * wc_r * wf_r ** 2))
    v_d = wc_d * wf_d
    v_r = wc_r * wf_r
    S = float(np.sum(v_d ** 2)) + alpha ** 2 * float(np.sum(v_r ** 2))
    return {"alpha": alpha, "I": I, "S": S, "W_d": W_d, "W_r": W_r}


def painted_values(data, randoms, params: Params, alpha: float):
    """Per-particle painted values: +w_c w_fkp for data, -alpha w_c w_fkp for randoms."""
    wc_d, nb_d = _cat_arrays(data, params)
    wc_r, nb_r = _cat_arrays(randoms, params)
    return wc_d * fkp_weight(nb_d, params.P0), -alpha * wc_r * fkp_weight(nb_r, params.P0)


# --------------------------------------------------------------------------- painting
def window_weights_1d(u: np.ndarray, window: str):
    """Node offsets and weights of the 1-D assignment kernel at grid coordinate u.

    Returns (base, [w_0, w_1, ...]): node base + a gets weight w_a.
    CIC: base = floor(u), weights (1 - d, d), d = u - base.
    TSC: c = floor(u + 1/2), d = u - c in [-1/2, 1/2), base = c - 1,
         weights ((1/2 - d)^2 / 2, 3/4 - d^2, (1/2 + d)^2 / 2).
    """
    if window == CIC:
        base = np.floor(u)
        d = u - base
        return base.astype(np.int64), [1.0 - d, d]
    if window == TSC:
        c = np.floor(u + 0.5)
        d = u - c
        return (c - 1).astype(np.int64), [0.5 * (0.5 - d) ** 2, 0.75 - d * d, 0.5 * (0.5 + d) ** 2]
    raise ValueError(window)


def paint(pos: np.ndarray, values: np.ndarray, params: Params, shift: float = 0.0) -> np.ndarray:
    """Mass assignment onto the N^3 mesh (Sec. 2.3): mesh_j += v_p W(u_p - shift - j).

    u = (pos - corner)/H; ``shift`` = 1/2 paints the interlaced second mesh, whose node j
    sits at corner + (j + 1/2) H. Nodes wrap periodically.
    """
    n = params.nmesh
    u = (np.asarray(pos, dtype=np.float64) - np.asarray(params.box_corner, dtype=np.float64)) \
        / params.cell - shift
    mesh = np.zeros(n * n * n)
    bx, wx = window_weights_1d(u[:, 0], params.window)
    by, wy = window_weights_1d(u[:, 1], params.window)
    bz, wz = window_weights_1d(u[:, 2], params.window)
    for a, wa in enumerate(wx):
        ia = (bx + a) % n
        for b, wb in enumerate(wy):
            ib = (by + b) % n
            for c, wcz in enumerate(wz):
                ic = (bz + c) % n
                mesh += np.bincount((ia * n + ib) * n + ic, weights=values * wa * wb * wcz, minlength=n ** 3)
    return mesh.reshape(n, n, n)


# --------------------------------------------------------------------------- k-space helpers
def int_freqs(n: int):
    """Signed integer frequencies along a full axis (length n) and a half axis (n/2 + 1)."""
    full = np.fft.fftfreq(n, d=1.0 / n).astype(np.int64)   # [0..n/2-1, -n/2..-1]
    half = np.arange(n // 2 + 1, dtype=np.int64)           # rfft axis: 0..n/2
    return full, half


def nyquist_mask(n: int) -> np.ndarray:
    """True where some n_d = -N/2 (the rfft axis index N/2 is that frequency too)."""
    full, half = int_freqs(n)
    fx = full[:, None, None] == -n // 2
    fy = full[None, :, None] == -n // 2
    fz = half[None, None, :] == n // 2
    return fx | fy | fz


def window_transfer(n: int, window: str, form: str = "sinc") -> np.ndarray:
    """The compensation divisor over the half spectrum (Sec. 2.3, which cites Jing 2005).

    "sinc": W(k) = prod_d sinc^p(pi n_d / N). "jing": prod_d sqrt(C_p(n_d)), C_p the sum of
    sinc^{2p} over the aliases n_d + m N, in its closed form for CIC (1 - 2/3 s^2) and TSC
    (1 - s^2 + 2/15 s^4), s = sin(pi n_d / N): dividing the field by it removes the aliased
    shot noise of a non-interlaced mesh on average."""
    p = WINDOW_ORDER[window]
    full, half = int_freqs(n)

    def axis(v):
        if form in ("sinc", "sinc_per_mode"):
            return np.sinc(v / n) ** p    # numpy sinc(x) = sin(pi x)/(pi x)
        s2 = np.sin(np.pi * v / n) ** 2
        c = 1.0 - 2.0 / 3.0 * s2 if p == 2 else 1.0 - s2 + 2.0 / 15.0 * s2 * s2
        return np.sqrt(c)
    sx, sz = axis(full), axis(half)
    return sx[:, None, None] * sx[None, :, None] * sz[None, None, :]


def interlace_phase(n: int) -> np.ndarray:
    """exp(-i k.s), s = (H/2)(1,1,1): exp(-i pi (n_x + n_y + n_z) / N)."""
    full, half = int_freqs(n)
    tot = full[:, None, None] + full[None, :, None] + half[None, None, :]
    return np.exp(-1j * math.pi * tot / n)


def mode_binning(n: int, box_size: float, k_edges: np.ndarray):
    """Bin index (or -1) and half-spectrum multiplicity of every stored mode.

    Mode n lies in bin b iff t_b <= |n|^2 < t_{b+1}, t_b = (k_b L/(2 pi))^2 (FP64). The
    k = 0 mode and modes with some n_d = -N/2 get -1. Multiplicity: 1 on n_z = 0, else 2.
    """
    full, half = int_freqs(n)
    n2 = (full[:, None, None] ** 2 + full[None, :, None] ** 2 + half[None, None, :] ** 2)
    t = (np.asarray(k_edges, dtype=np.float64) * box_size / (2.0 * math.pi)) ** 2
    n2f = n2.astype(np.float64)
    b = np.searchsorted(t, n2f, side="right") - 1
    b[(n2f < t[0]) | (n2f >= t[-1])] = -1
    b[n2 == 0] = -1
    b[nyquist_mask(n)] = -1
    mult = np.where(half[None, None, :] == 0, 1.0, 2.0) * np.ones_like(n2f)
    return b, mult, n2


# --------------------------------------------------------------------------- harmonics
def real_ylm(ell: int, m: int, x: np.ndarray, y: np.ndarray, z: np.ndarray) -> np.ndarray:
    """Real spherical harmonic of eq. real-Ylm at unit vectors (x, y, z).

    m > 0: sqrt((2l+1)/(2pi) (l-m)!/(l+m)!) P_l^m(cos t) cos(m phi)
    m = 0: sqrt((2l+1)/(4pi)) P_l(cos t)
    m < 0: sqrt((2l+1)/(2pi) (l-|m|)!/(l+|m|)!) P_l^|m|(cos t) sin(|m| phi)
    P_l^m from scipy.special.lpmv. Zero-length vectors (all of x, y, z = 0) give 0 for l > 0.
    """
    x = np.asarray(x, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    z = np.asarray(z, dtype=np.float64)
    zero = (x == 0) & (y == 0) & (z == 0)
    ct = np.clip(z, -1.0, 1.0)
    phi = np.arctan2(y, x)
    am = abs(m)
    plm = lpmv(am, ell, ct)
    if m == 0:
        out = math.sqrt((2 * ell + 1) / (4 * math.pi)) * plm
    else:
        norm = math.sqrt((2 * ell + 1) / (2 * math.pi) * math.exp(gammaln(ell - am + 1) - gammaln(ell + am + 1)))
        trig = np.cos(am * phi) if m > 0 else np.sin(am * phi)
        out = norm * plm * trig
    if ell > 0:
        out = np.where(zero, 0.0, out)
    return out


def _unit(vx, vy, vz):
    r = np.sqrt(vx * vx + vy * vy + vz * vz)
    safe = np.where(r > 0, r, 1.0)
    return vx / safe, vy / safe, vz / safe


def node_rhat(params: Params, ix: np.ndarray):
    """Unit vectors from the observer to the nodes corner + (i, j, k) H for x-planes ``ix``."""
    n = params.nmesh
    h = params.cell
    c = np.asarray(params.box_corner, dtype=np.float64)
    o = np.asarray(params.observer, dtype=np.float64)
    ax = c[0] + ix * h - o[0]
    ay = c[1] + np.arange(n) * h - o[1]
    az = c[2] + np.arange(n) * h - o[2]
    vx = np.broadcast_to(ax[:, None, None], (len(ix), n, n))
    vy = np.broadcast_to(ay[None, :, None], (len(ix), n, n))
    vz = np.broadcast_to(az[None, None, :], (len(ix), n, n))
    return _unit(vx, vy, vz)


def mode_khat(n: int):
    full, half = int_freqs(n)
    kx = np.broadcast_to(full[:, None, None].astype(np.float64), (n, n, n // 2 + 1))
    ky = np.broadcast_to(full[None, :, None].astype(np.float64), (n, n, n // 2 + 1))
    kz = np.broadcast_to(half[None, None, :].astype(np.float64), (n, n, n // 2 + 1))
    return _unit(kx, ky, kz)


# --------------------------------------------------------------------------- the estimator
@dataclass
class Fields:
    """Intermediate products of the density step (for tests)."""

    sums: Dict[str, float]
    mesh1: np.ndarray
    mesh2: Optional[np.ndarray]
    F0: np.ndarray          # combined, compensated field X (half spectrum)
    f: np.ndarray           # real field that gets the Y_lm weights
    extra: dict = field(default_factory=dict)


def density_fields(data, randoms, params: Params) -> Fields:
    """Sums, painting, interlacing, compensation and the round trip (Sec. 2.1, Sec. 2.3)."""
    n = params.nmesh
    sums = catalog_sums(data, randoms, params)
    v_d, v_r = painted_values(data, randoms, params, sums["alpha"])
    mesh1 = paint(data.pos, v_d, params) + paint(randoms.pos, v_r, params)
    F1 = sfft.rfftn(mesh1, workers=_workers())
    mesh2 = None
    if params.interlaced:
        mesh2 = paint(data.pos, v_d, params, shift=0.5) + paint(randoms.pos, v_r, params, shift=0.5)
        F2 = sfft.rfftn(mesh2, workers=_workers())
        X = 0.5 * (F1 + interlace_phase(n) * F2)
        del F2
    else:
        X = F1
    # "sinc_per_mode": the field is left uncompensated and each mode's binned product is
    # divided by W(k)^2 instead (multipoles_from_fields)
    field_comp = params.compensate and params.compensation != "sinc_per_mode"
    if field_comp:
        X = X / window_transfer(n, params.window, params.compensation)
    if params.interlaced or field_comp:
        X = np.where(nyquist_mask(n), 0.0, X)
        f = sfft.irfftn(X, s=(n, n, n), workers=_workers())
    else:
        f = mesh1
    return Fields(sums=sums, mesh1=mesh1, mesh2=mesh2, F0=X, f=f)


def harmonic_spectrum(f: np.ndarray, params: Params, ell: int, m: int, chunk: int = 32) -> np.ndarray:
    """G_lm(k) = DFT[f(x) Y_lm(rhat_x)] (Sec. 2.1 eq. Fell, one term of the m sum)."""
    n = params.nmesh
    weighted = np.empty_like(f)
    for i0 in range(0, n, chunk):
        ix = np.arange(i0, min(n, i0 + chunk))
        ux, uy, uz = node_rhat(params, ix)
        weighted[ix] = f[ix] * real_ylm(ell, m, ux, uy, uz)
    return sfft.rfftn(weighted, workers=_workers())


def multipoles_from_fields(fl: Fields, params: Params, ells: Sequence[int], k_edges) -> Dict[str, np.ndarray]:
    """Angular averages in k shells (Sec. 2.1 eqs. Pell-ours and Fell)."""
    n = params.nmesh
    k_edges = np.asarray(k_edges, dtype=np.float64)
    nk = len(k_edges) - 1
    b, mult, n2 = mode_binning(n, params.box_size, k_edges)
    sel = b >= 0
    bs = b[sel]
    ms = mult[sel]
    n_modes = np.bincount(bs, weights=ms, minlength=nk)
    kmag = (2.0 * math.pi / params.box_size) * np.sqrt(n2[sel].astype(np.float64))
    ksum = np.bincount(bs, weights=ms * kmag, minlength=nk)
    with np.errstate(invalid="ignore", divide="ignore"):
        k_mean = ksum / n_modes
    I, S = fl.sums["I"], fl.sums["S"]
    F0 = fl.F0
    # compensation per mode: 1/W^2 on every binned product
    wm = (1.0 / window_transfer(n, params.window, "sinc")[sel] ** 2
          if params.compensate and params.compensation == "sinc_per_mode" else 1.0)
    ms = ms * wm
    P = np.zeros((len(ells), nk))
    khat = None
    for li, ell in enumerate(ells):
        if ell == 0:
            p2 = np.bincount(bs, weights=ms * np.abs(F0[sel]) ** 2, minlength=nk)
            with np.errstate(invalid="ignore", divide="ignore"):
                P[li] = (p2 / n_modes - S) / I
            continue
        if khat is None:
            khat = mode_khat(n)
        acc = np.zeros(F0.shape)
        for m in range(-ell, ell + 1):
            G = harmonic_spectrum(fl.f, params, ell, m)
            prod = G * np.conj(F0)
            acc += real_ylm(ell, m, *khat) * (np.imag(prod) if ell % 2 else np.real(prod))
            del G
        s = np.bincount(bs, weights=ms * acc[sel], minlength=nk)
        with np.errstate(invalid="ignore", divide="ignore"):
            P[li] = 4.0 * math.pi * s / (I * n_modes)
    return {"P": P, "k_mean": k_mean, "n_modes": n_modes}


def multipoles(data, randoms, params: Params, ells: Sequence[int], k_edges) -> Dict[str, np.ndarray]:
    """P_l(k) of the estimator for the catalogs (the whole hot path, FP64)."""
    fl = density_fields(data, randoms, params)
    out = multipoles_from_fields(fl, params, ells, k_edges)
    out.update(fl.sums)
    return out


# --------------------------------------------------------------------------- wedges
def legendre(ell: int, mu):
    return eval_legendre(ell, np.asarray(mu, dtype=np.float64))


def lbar(ell: int, mu_lo: float, mu_hi: float) -> float:
    """Mean of L_l over [mu_lo, mu_hi] (Sec. 2.2 eq. Lbar), from the antiderivative
    int L_l = (L_{l+1} - L_{l-1}) / (2l + 1) for l >= 1, and mu for l = 0."""
    if ell == 0:
        return 1.0
    def anti(mu):
        return (legendre(ell + 1, mu) - legendre(ell - 1, mu)) / (2 * ell + 1)
    return float((anti(mu_hi) - anti(mu_lo)) / (mu_hi - mu_lo))


def wedges(P: np.ndarray, ells: Sequence[int], mu_edges) -> np.ndarray:
    """P(k_i, mu_m) = sum_l P_l(k_i) Lbar_l(mu_m, mu_{m+1}) (Sec. 2.2 eq. wedge-est), even l only."""
    if any(int(ell) % 2 for ell in ells):
        raise ValueError("wedges are built from even multipoles")
    mu_edges = np.asarray(mu_edges, dtype=np.float64)
    nmu = len(mu_edges) - 1
    out = np.zeros((nmu, P.shape[1]))
    for w in range(nmu):
        for li, ell in enumerate(ells):
            out[w] += P[li] * lbar(ell, mu_edges[w], mu_edges[w + 1])
    return out


# --------------------------------------------------------------------------- FFT counts
def fft_count_sh(ell_max: int) -> int:
    """Transforms for all even l <= l_max with 2l+1 per multipole (Sec. 2.1)."""
    return sum(2 * l + 1 for l in range(0, ell_max + 1, 2))


def fft_count_cartesian(ell_max: int) -> int:
    """Transforms with (l+1)(l+2)/2 per multipole, the Cartesian route (Sec. 2.1)."""
    return sum((l + 1) * (l + 2) // 2 for l in range(0, ell_max + 1, 2))
