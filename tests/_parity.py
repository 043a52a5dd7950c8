"""Shared helpers of the GPU parity tests: run the oracle and the CUDA path on the same
seeded catalogs and compare under the stated tolerances."""
import math

import numpy as np

from oracle import estimator as E


def gpu_estimator(p: E.Params, precision="fp32", ell_max=4, max_kbins=512, **kw):
    from paper_1704_02357_gb300 import Estimator
    comp = p.compensation if p.compensate else False
    return Estimator(nmesh=p.nmesh, box_size=p.box_size, box_corner=p.box_corner, observer=p.observer,
                     window=p.window, interlaced=p.interlaced, compensate=comp, precision=precision,
                     ell_max=ell_max, P0=p.P0, nbar=p.nbar, max_kbins=max_kbins, **kw)


def run_gpu(p, data, randoms, ells, edges, precision="fp32", ell_max=None, **kw):
    """Paint + multipoles on a fresh context. FP32 contexts get the exact tile-binned paint
    (max_particles covers both catalogs) unless the caller passes max_particles (0: direct
    atomic paint)."""
    if precision != "fp64":
        kw.setdefault("max_particles", data.size + randoms.size)
    est = gpu_estimator(p, precision=precision, ell_max=ell_max if ell_max is not None else max(ells), **kw)
    stats = est.paint(data.pos, randoms.pos, data.weight, data.nbar, randoms.weight, randoms.nbar)
    out = est.multipoles(ells, edges)
    out["stats"] = stats
    out["plan"] = est.plan_info()
    est.close()
    return out


def tol_for(ell):
    """Max relative error allowed for the FP32 path: 1e-5 for l <= 4, 1e-4 for l <= 16."""
    return 1e-5 if ell <= 4 else 1e-4


def check_fp32(gpu, ora, ells, scale=None, report=None):
    """Tolerance rule: |dP_l| / |P_l| <= tol(l) in bins where |P_l| > 1% |P_0|.

    ``scale`` replaces |P_0| as the reference amplitude when the monopole carries no
    signal (uniform Poisson points: P_0 ~ 0); the rule is then |dP_l| <= tol(l) * scale.
    Returns a dict with, per l, the bins checked, the max relative error there and
    max |dP_l| / ref over all bins (so the check is never vacuous).
    """
    Pg, Po = gpu["P"], ora["P"]
    i0 = ells.index(0)
    ref = np.abs(Po[i0]) if scale is None else np.broadcast_to(scale, Po[i0].shape)
    res = {}
    for li, ell in enumerate(ells):
        fin = np.isfinite(Po[li]) & (ref > 0)
        d = np.abs(Pg[li] - Po[li])
        assert np.all(np.isfinite(Pg[li][fin])), (ell, Pg[li])
        if scale is None:
            mask = fin & (np.abs(Po[li]) > 0.01 * ref)
            rel = d[mask] / np.abs(Po[li][mask])
            worst = float(rel.max()) if mask.any() else 0.0
            res[ell] = {"bins_checked": int(mask.sum()), "max_rel": worst,
                        "max_abs_over_P0": float((d[fin] / ref[fin]).max())}
            assert worst <= tol_for(ell), (ell, worst, res[ell])
        else:
            worst = float((d[fin] / ref[fin]).max())
            res[ell] = {"bins_checked": int(fin.sum()), "max_rel": worst, "max_abs_over_P0": worst}
            assert worst <= tol_for(ell), (ell, worst)
    if report is not None:
        report.update(res)
    return res


def uniform_edges(kmin, kmax, dk):
    n = int(round((kmax - kmin) / dk))
    return kmin + dk * np.arange(n + 1)


def kf(p):
    return 2 * math.pi / p.box_size
