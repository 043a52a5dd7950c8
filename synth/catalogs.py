"""Seeded synthetic catalogs with the shapes of the paper's workloads.

The paper measures on BOSS DR12 CMASS mocks, QPM boxes and periodic simulations
(Sec. 3.2, Sec. 4.1). None of those are available, so these generators stand in for them:

* ``uniform_box``: uniform Poisson points in a cube (the periodic-box case).
* ``survey_catalog``: a lognormal galaxy field, Poisson sampled, moved into redshift
  space along the radial line of sight with the Zel'dovich displacement, then cut to a
  spherical cap and radial shell (the survey-shaped case), and ``survey_randoms``: the
  matching uniform randoms.
* ``on_node_catalog``: a handful of particles placed exactly on mesh nodes, for which the
  mesh estimator equals the direct sum over particles.

Everything is seeded with ``numpy.random.default_rng`` so every caller sees identical bytes.
The Fourier transforms below only build the input density field; they are not part of the
estimator.
"""
from __future__ import annotations

import math
import os
from dataclasses import dataclass, field
from typing import Optional

import numpy as np

__all__ = [
    "Catalog", "SurveyGeometry", "LognormalField", "uniform_box", "on_node_catalog",
    "survey_geometry", "lognormal_field", "survey_catalog", "survey_randoms",
    "box_randoms", "mock_batch_spec",
]


@dataclass
class Catalog:
    """Particles: FP64 positions (n, 3), optional completeness weight and n̄ per particle."""

    pos: np.ndarray
    weight: Optional[np.ndarray] = None
    nbar: Optional[np.ndarray] = None

    @property
    def size(self) -> int:
        return int(self.pos.shape[0])


@dataclass
class SurveyGeometry:
    """A spherical cap (axis, half-angle) times a radial shell, inside a cubic box."""

    axis: np.ndarray
    half_angle_deg: float
    r_min: float
    r_max: float
    box_size: float
    box_corner: np.ndarray
    observer: np.ndarray = field(default_factory=lambda: np.zeros(3))

    @property
    def volume(self) -> float:
        solid = 2.0 * math.pi * (1.0 - math.cos(math.radians(self.half_angle_deg)))
        return solid * (self.r_max ** 3 - self.r_min ** 3) / 3.0


def _workers() -> int:
    try:
        return max(1, len(os.sched_getaffinity(0)))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def uniform_box(n: int, box_size: float, corner, seed: int) -> Catalog:
    """Exactly ``n`` uniform points in [corner, corner + box_size)^3."""
    rng = np.random.default_rng(seed)
    corner = np.asarray(corner, dtype=np.float64)
    pos = corner + rng.random((n, 3)) * box_size
    return Catalog(pos=pos)


def box_randoms(n: int, box_size: float, corner, seed: int) -> Catalog:
    return uniform_box(n, box_size, corner, seed)


def on_node_catalog(n: int, nmesh: int, box_size: float, corner, seed: int,
                    distinct: bool = True, weights: bool = True) -> Catalog:
    """``n`` particles sitting exactly on mesh nodes corner + i*H (i integer).

    With ``distinct`` the nodes are all different. Weights are drawn in [0.5, 1.5) when
    ``weights`` is set, else left as None (unit).
    """
    rng = np.random.default_rng(seed)
    corner = np.asarray(corner, dtype=np.float64)
    h = box_size / nmesh
    if distinct:
        flat = rng.choice(nmesh ** 3, size=n, replace=False)
    else:
        flat = rng.integers(0, nmesh ** 3, size=n)
    idx = np.stack(np.unravel_index(flat, (nmesh,) * 3), axis=1).astype(np.float64)
    pos = corner + idx * h
    w = 0.5 + rng.random(n) if weights else None
    return Catalog(pos=pos, weight=w)


def survey_geometry(box_size: float = 2000.0, half_angle_deg: float = 60.0,
                    r_min: float = 600.0, r_max: float = 1400.0) -> SurveyGeometry:
    """The survey-shaped geometry: cap about (1,1,1)/sqrt(3) so that it fits the box.

    A cap of 60 degrees about the z axis out to 1400 Mpc/h is 2425 Mpc/h wide and does
    not fit a 2000 Mpc/h box; about the diagonal it spans [-585.9, 1400] on every axis.
    The box is centred on that span.
    """
    axis = np.ones(3) / math.sqrt(3.0)
    cos_a = 1.0 / math.sqrt(3.0)  # cos of the angle between the diagonal and each axis
    ang_to_axis = math.acos(cos_a)
    lo = r_max * math.cos(ang_to_axis + math.radians(half_angle_deg))
    hi = r_max if ang_to_axis <= math.radians(half_angle_deg) else \
        r_max * math.cos(ang_to_axis - math.radians(half_angle_deg))
    centre = 0.5 * (lo + hi)
    corner = np.full(3, centre - 0.5 * box_size)
    return SurveyGeometry(axis=axis, half_angle_deg=half_angle_deg, r_min=r_min,
                          r_max=r_max, box_size=box_size, box_corner=corner)


def _in_geometry(pos: np.ndarray, geo: SurveyGeometry) -> np.ndarray:
    rel = pos - geo.observer
    r = np.sqrt(np.einsum("ij,ij->i", rel, rel))
    cosang = (rel @ geo.axis) / np.maximum(r, 1e-300)
    return (r >= geo.r_min) & (r < geo.r_max) & \
        (cosang >= math.cos(math.radians(geo.half_angle_deg)))


def survey_randoms(n: int, geo: SurveyGeometry, seed: int) -> Catalog:
    """Exactly ``n`` points uniform in the cap x shell (r^3 and cos(theta) uniform)."""
    rng = np.random.default_rng(seed)
    u = rng.random((n, 3))
    r = np.cbrt(geo.r_min ** 3 + u[:, 0] * (geo.r_max ** 3 - geo.r_min ** 3))
    cmin = math.cos(math.radians(geo.half_angle_deg))
    cth = cmin + u[:, 1] * (1.0 - cmin)
    sth = np.sqrt(np.maximum(0.0, 1.0 - cth * cth))
    phi = 2.0 * math.pi * u[:, 2]
    a = geo.axis
    # orthonormal frame (e1, e2, a)
    t = np.array([1.0, 0.0, 0.0]) if abs(a[0]) < 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(a, t)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(a, e1)
    d = (sth * np.cos(phi))[:, None] * e1 + (sth * np.sin(phi))[:, None] * e2 + cth[:, None] * a
    pos = geo.observer + r[:, None] * d
    return Catalog(pos=pos)


@dataclass
class LognormalField:
    """A lognormal overdensity and a Zel'dovich displacement on a generation grid."""

    delta: np.ndarray     # (ng, ng, ng) float64, mean ~0
    psi: np.ndarray       # (3, ng, ng, ng) float64 displacement
    box_size: float
    corner: np.ndarray


def _plaw_pk(k: np.ndarray) -> np.ndarray:
    """P(k) = 2e4 (k/0.02) / (1 + (k/0.02)^2.4)  [(Mpc/h)^3]."""
    x = k / 0.02
    return 2.0e4 * x / (1.0 + x ** 2.4)


def lognormal_field(ngen: int, box_size: float, corner, seed: int, pk=_plaw_pk) -> LognormalField:
    """Gaussian field G with spectrum ``pk``; delta = exp(G - sigma^2/2) - 1; psi = i k/k^2 G."""
    import scipy.fft as sfft

    rng = np.random.default_rng(seed)
    white = rng.standard_normal((ngen,) * 3)
    dv = (box_size / ngen) ** 3
    kf = 2.0 * math.pi / box_size
    kx = np.fft.fftfreq(ngen, d=1.0 / ngen) * kf
    kz = np.fft.rfftfreq(ngen, d=1.0 / ngen) * kf
    k2 = kx[:, None, None] ** 2 + kx[None, :, None] ** 2 + kz[None, None, :] ** 2
    amp = np.sqrt(pk(np.sqrt(k2)) / dv)
    amp[0, 0, 0] = 0.0
    wk = sfft.rfftn(white, workers=_workers())
    gk = wk * amp
    del wk, white
    g = sfft.irfftn(gk, s=(ngen,) * 3, workers=_workers())
    sigma2 = float(np.var(g))
    delta = np.exp(g - 0.5 * sigma2) - 1.0
    del g
    k2s = k2.copy()
    k2s[0, 0, 0] = 1.0
    psi = np.empty((3, ngen, ngen, ngen))
    for ax, kk in enumerate((kx[:, None, None], kx[None, :, None], kz[None, None, :])):
        psi[ax] = sfft.irfftn(1j * kk / k2s * gk, s=(ngen,) * 3, workers=_workers())
    return LognormalField(delta=delta, psi=psi, box_size=box_size,
                          corner=np.asarray(corner, dtype=np.float64))


def _interp_cic(grid: np.ndarray, u: np.ndarray) -> np.ndarray:
    """Periodic trilinear interpolation of ``grid`` at grid coordinates u (n, 3)."""
    ng = grid.shape[0]
    i0 = np.floor(u).astype(np.int64)
    d = u - i0
    out = np.zeros(u.shape[0])
    for a in (0, 1):
        wa = d[:, 0] if a else 1.0 - d[:, 0]
        ia = (i0[:, 0] + a) % ng
        for b in (0, 1):
            wb = d[:, 1] if b else 1.0 - d[:, 1]
            ib = (i0[:, 1] + b) % ng
            for c in (0, 1):
                wc = d[:, 2] if c else 1.0 - d[:, 2]
                ic = (i0[:, 2] + c) % ng
                out += wa * wb * wc * grid[ia, ib, ic]
    return out


def survey_catalog(field_: LognormalField, geo: SurveyGeometry, nbar: float, seed: int,
                   growth_rate: float = 0.75) -> Catalog:
    """Poisson-sample nbar(1+delta) over the box, move radially by f (psi.rhat) rhat, cut.

    The cut (cap and shell) is applied in redshift space. The returned catalog carries a
    constant n̄ per particle.
    """
    rng = np.random.default_rng(seed)
    ng = field_.delta.shape[0]
    h = field_.box_size / ng
    lam = nbar * h ** 3 * np.clip(1.0 + field_.delta, 0.0, None)
    counts = rng.poisson(lam.ravel())
    cells = np.repeat(np.arange(counts.size, dtype=np.int64), counts)
    idx = np.stack(np.unravel_index(cells, (ng,) * 3), axis=1).astype(np.float64)
    u = idx + rng.random(idx.shape)
    pos = field_.corner + u * h
    rel = pos - geo.observer
    rhat = rel / np.sqrt(np.einsum("ij,ij->i", rel, rel))[:, None]
    psi_r = sum(_interp_cic(field_.psi[a], u - 0.5) * rhat[:, a] for a in range(3))
    pos = pos + growth_rate * psi_r[:, None] * rhat
    keep = _in_geometry(pos, geo)
    pos = pos[keep]
    return Catalog(pos=pos, nbar=np.full(pos.shape[0], nbar))


def mock_batch_spec(n_mocks: int = 64, seed0: int = 100, n_min: float = 3e5, n_max: float = 3e6,
                    meshes=(256, 384)):
    """(seed, n_data, nmesh) for a campaign of mocks: N_d log-uniform, meshes alternating."""
    out = []
    for i in range(n_mocks):
        s = seed0 + i
        rng = np.random.default_rng(s)
        nd = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        out.append((s, nd, meshes[s % len(meshes)]))
    return out
