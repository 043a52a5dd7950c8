"""Independent routes that pin the oracle's estimator (test infrastructure only).

None of these share code with ``oracle.estimator`` beyond the Params container and the
catalog arrays: each restates its quantity from its own definition.

* ``direct_multipoles``: eq. Pell-yama of Sec. 2.1 evaluated as an explicit sum over
  particles and over every mode of the full N^3 grid (no FFT, no spherical harmonics:
  the Legendre polynomial of khat.rhat is evaluated directly).
* ``cartesian_multipoles``: the Cartesian decomposition of Sec. 2.1 (the route of Bianchi
  et al. and Scoccimarro) for l <= 4: L_l(khat.rhat) expanded in powers of
  mu = sum_a khat_a rhat_a, 1 + 6 + 15 = 22 transforms.
* ``dft_brute``: the O(N^6) sum defining the 3-D DFT.
* ``paint_loop``: per-particle mass assignment written from the kernel shapes as
  functions of distance.
* ``alias_sum_1d``: the Fourier transform of a mesh painted from one particle, written as
  the Poisson sum over aliases of the continuous kernel sinc^p, with or without
  interlacing.
"""
from __future__ import annotations

import itertools
import math
from typing import Dict, Sequence

import numpy as np
from scipy.special import eval_legendre


# --------------------------------------------------------------------------- direct sum
def _values(cat, P0, nbar_default):
    n = cat.pos.shape[0]
    wc = np.ones(n) if cat.weight is None else np.asarray(cat.weight, dtype=np.float64)
    nb = np.full(n, nbar_default) if cat.nbar is None else np.asarray(cat.nbar, dtype=np.float64)
    wf = np.ones(n) if P0 <= 0 else 1.0 / (1.0 + nb * P0)
    return wc, nb, wf


def direct_multipoles(data, randoms, params, ells: Sequence[int], k_edges) -> Dict[str, np.ndarray]:
    """Local plane-parallel estimator by explicit sums (Sec. 2.1 eq. Pell-yama).

    P_l(k_b) = (2l+1)/(I N_b) sum_{k in b} A_l(k) conj(A_0(k)) - delta_l0 S/I with
    A_l(k) = sum_p v_p L_l(khat . rhat_p) exp(-i k . r_p) over data (v = w) and randoms
    (v = -alpha w); S/I removes the p = q pairs for l = 0. The modes are every n in
    [-N/2, N/2)^3 with no component equal to -N/2, n != 0, each counted once.
    Equals the mesh estimator when particles sit on nodes and no compensation or
    interlacing is applied. The shell sum is complex: "P" holds its real part for even l and
    its imaginary part for odd l, "P_other" the other part (zero up to rounding, since the
    terms at k and -k are conjugate for even l and minus conjugate for odd l).
    """
    n = params.nmesh
    L = params.box_size
    wc_d, nb_d, wf_d = _values(data, params.P0, params.nbar)
    wc_r, nb_r, wf_r = _values(randoms, params.P0, params.nbar)
    alpha = wc_d.sum() / wc_r.sum()
    I = alpha * np.sum(nb_r * wc_r * wf_r ** 2)
    pos = np.concatenate([data.pos, randoms.pos], axis=0)
    v = np.concatenate([wc_d * wf_d, -alpha * wc_r * wf_r])
    rel = pos - np.asarray(params.observer, dtype=np.float64)
    rr = np.sqrt(np.sum(rel ** 2, axis=1))
    rhat = rel / np.where(rr > 0, rr, 1.0)[:, None]

    freqs = np.arange(-n // 2, n // 2)
    nvec = np.array(list(itertools.product(freqs, freqs, freqs)), dtype=np.int64)
    keep = np.all(nvec != -n // 2, axis=1) & np.any(nvec != 0, axis=1)
    nvec = nvec[keep]
    n2 = np.sum(nvec ** 2, axis=1)
    t = (np.asarray(k_edges, dtype=np.float64) * L / (2 * math.pi)) ** 2
    nk = len(k_edges) - 1
    b = np.full(n2.shape, -1)
    for i in range(nk):
        b[(n2 >= t[i]) & (n2 < t[i + 1])] = i
    kvec = nvec * (2 * math.pi / L)
    khat = nvec / np.sqrt(n2)[:, None]
    phase = np.exp(-1j * (kvec @ pos.T))          # (modes, particles)
    A0 = phase @ v
    mu = khat @ rhat.T                            # (modes, particles)
    n_modes = np.array([np.sum(b == i) for i in range(nk)], dtype=np.float64)
    kmag = np.sqrt(n2) * (2 * math.pi / L)
    k_mean = np.array([kmag[b == i].mean() if n_modes[i] else np.nan for i in range(nk)])
    S = np.sum(v ** 2)
    P = np.zeros((len(ells), nk))
    other = np.zeros((len(ells), nk))
    for li, ell in enumerate(ells):
        Al = (phase * eval_legendre(ell, mu)) @ v
        val = Al * np.conj(A0)
        for i in range(nk):
            s = (2 * ell + 1) * val[b == i].sum() / (I * n_modes[i])
            P[li, i], other[li, i] = (s.imag, s.real) if ell % 2 else (s.real, s.imag)
            if ell == 0:
                P[li, i] -= S / I
    return {"P": P, "P_other": other, "k_mean": k_mean, "n_modes": n_modes, "I": I, "S": S, "alpha": alpha}


# --------------------------------------------------------------------------- Cartesian route
def cartesian_multipoles(f: np.ndarray, F0: np.ndarray, params, I: float, S: float,
                         ells: Sequence[int], k_edges, binning) -> Dict[str, np.ndarray]:
    """l in {0, 2, 4} from products of Cartesian components (Sec. 2.1).

    M_j(k) = DFT[f mu^j] with mu^j = sum over multisets of axes (multinomial weights) of
    khat and rhat component products; L_2 = (3 mu^2 - 1)/2, L_4 = (35 mu^4 - 30 mu^2 + 3)/8.
    ``binning`` = (bin index, multiplicity) over the half spectrum, supplied by the caller.
    Returns P and the number of transforms used (1 + 6 + 15 = 22 for l_max = 4).
    """
    import scipy.fft as sfft

    n = params.nmesh
    h = params.box_size / n
    c = np.asarray(params.box_corner, dtype=np.float64)
    o = np.asarray(params.observer, dtype=np.float64)
    ax = [c[d] + np.arange(n) * h - o[d] for d in range(3)]
    X = np.broadcast_to(ax[0][:, None, None], (n, n, n))
    Y = np.broadcast_to(ax[1][None, :, None], (n, n, n))
    Z = np.broadcast_to(ax[2][None, None, :], (n, n, n))
    R = np.sqrt(X * X + Y * Y + Z * Z)
    Rs = np.where(R > 0, R, 1.0)
    rh = [X / Rs, Y / Rs, Z / Rs]
    fr = np.fft.fftfreq(n, d=1.0 / n)
    hf = np.arange(n // 2 + 1, dtype=np.float64)
    KX = np.broadcast_to(fr[:, None, None], (n, n, n // 2 + 1))
    KY = np.broadcast_to(fr[None, :, None], (n, n, n // 2 + 1))
    KZ = np.broadcast_to(hf[None, None, :], (n, n, n // 2 + 1))
    K = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    Ks = np.where(K > 0, K, 1.0)
    kh = [KX / Ks, KY / Ks, KZ / Ks]
    nfft = 0

    def mu_power(j):
        nonlocal nfft
        out = np.zeros(F0.shape, dtype=np.complex128)
        for combo in itertools.combinations_with_replacement(range(3), j):
            cnt = [combo.count(a) for a in range(3)]
            coef = math.factorial(j) / (math.factorial(cnt[0]) * math.factorial(cnt[1]) * math.factorial(cnt[2]))
            wr = np.ones((n, n, n))
            wk = np.ones(F0.shape)
            for a in combo:
                wr = wr * rh[a]
                wk = wk * kh[a]
            out += coef * wk * sfft.rfftn(f * wr)
            nfft += 1
        return out

    b, mult = binning
    sel = b >= 0
    nk = len(k_edges) - 1
    n_modes = np.bincount(b[sel], weights=mult[sel], minlength=nk)
    need = max(ells)
    F = sfft.rfftn(f)
    nfft += 1
    M2 = mu_power(2) if need >= 2 else None
    M4 = mu_power(4) if need >= 4 else None
    P = np.zeros((len(ells), nk))
    for li, ell in enumerate(ells):
        if ell == 0:
            Fl = F
        elif ell == 2:
            Fl = (3.0 * M2 - F) / 2.0
        elif ell == 4:
            Fl = (35.0 * M4 - 30.0 * M2 + 3.0 * F) / 8.0
        else:
            raise ValueError("Cartesian route implemented for l <= 4")
        val = np.real(Fl * np.conj(F0))
        s = np.bincount(b[sel], weights=mult[sel] * val[sel], minlength=nk)
        P[li] = (2 * ell + 1) * s / (I * n_modes)
        if ell == 0:
            P[li] -= S / I
    return {"P": P, "n_fft": nfft}


# --------------------------------------------------------------------------- DFT
def dft_brute(x: np.ndarray) -> np.ndarray:
    """X(k) = sum_x x(r) exp(-2 pi i k.r / N) over the full N^3 grid, by explicit sums."""
    n = x.shape[0]
    idx = np.arange(n)
    r = np.array(list(itertools.product(idx, idx, idx)))
    vals = np.array([x[tuple(p)] for p in r])
    out = np.zeros((n, n, n), dtype=np.complex128)
    for k in itertools.product(idx, idx, idx):
        ph = np.exp(-2j * math.pi * (r @ np.array(k)) / n)
        out[k] = np.sum(vals * ph)
    return out


# --------------------------------------------------------------------------- paint by loop
def _kernel(window: str, s: float) -> float:
    a = abs(s)
    if window == "cic":
        return max(0.0, 1.0 - a)
    if window == "tsc":
        if a < 0.5:
            return 0.75 - a * a
        if a < 1.5:
            return 0.5 * (1.5 - a) ** 2
        return 0.0
    raise ValueError(window)


def paint_loop(pos, values, params, shift: float = 0.0) -> np.ndarray:
    """mesh_j = sum_p v_p prod_d K(u_pd - shift - j_d), K the CIC or TSC kernel shape."""
    n = params.nmesh
    mesh = np.zeros((n, n, n))
    u_all = (np.asarray(pos) - np.asarray(params.box_corner)) / (params.box_size / n) - shift
    for u, v in zip(u_all, values):
        base = np.floor(u).astype(int)
        cand = [range(b - 2, b + 3) for b in base]
        for j in itertools.product(*cand):
            w = _kernel(params.window, u[0] - j[0]) * _kernel(params.window, u[1] - j[1]) \
                * _kernel(params.window, u[2] - j[2])
            if w != 0.0:
                mesh[j[0] % n, j[1] % n, j[2] % n] += v * w
    return mesh


# --------------------------------------------------------------------------- alias sums
def alias_sum_1d(q: float, u: float, p: int, interlaced: bool, nalias: int = 2000) -> complex:
    """DFT at q = 2 pi n/N (cell units) of a 1-D mesh painted from one particle at u.

    By Poisson summation, sum_j K(u - j) exp(-i q j) = sum_a exp(-i (q + 2 pi a) u) Kt(q + 2 pi a)
    with Kt(w) = sinc^p(w/2) the Fourier transform of the kernel. Interlacing keeps only
    the even a (the odd aliases cancel in (F1 + exp(-i q/2) F2)/2).
    """
    a = np.arange(-nalias, nalias + 1)
    if interlaced:
        a = a[a % 2 == 0]
    w = q + 2 * math.pi * a
    kt = np.sinc(w / (2 * math.pi)) ** p    # sinc(w/2) with numpy's normalised sinc
    return complex(np.sum(np.exp(-1j * w * u) * kt))
