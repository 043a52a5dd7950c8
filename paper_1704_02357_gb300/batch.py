"""Batched mock campaigns: many data catalogs against one shared randoms catalog.

Mocks are grouped by mesh side; each group gets one estimator context whose randoms meshes
are painted once, and the group runs as one persistent launch sequence (a CUDA graph
replayed per mock, see pspec_run_batch). All arithmetic happens in libpspec.
"""
from __future__ import annotations

from typing import Dict, List, Sequence

import numpy as np

from .pspec import Estimator


class BatchRunner:
    """Runs mocks of possibly different mesh sides; results come back in input order."""

    def __init__(self, box_size, box_corner, randoms_pos, observer=(0.0, 0.0, 0.0), window="cic",
                 interlaced=True, compensate=True, precision="fp32", ell_max=4, P0=0.0, nbar=0.0,
                 randoms_weight=None, randoms_nbar=None, max_kbins=512, device=None, stream=None):
        self.kw = dict(box_size=box_size, box_corner=box_corner, observer=observer, window=window,
                       interlaced=interlaced, compensate=compensate, precision=precision, ell_max=ell_max, P0=P0,
                       nbar=nbar, max_kbins=max_kbins, device=device, stream=stream)
        self.randoms = (randoms_pos, randoms_weight, randoms_nbar)
        self.contexts: Dict[int, Estimator] = {}

    def context(self, nmesh: int, max_particles: int) -> Estimator:
        est = self.contexts.get(nmesh)
        if est is not None and est.params.max_particles >= max_particles:
            return est
        if est is not None:
            est.close()
        est = Estimator(nmesh=nmesh, cache_randoms=True, max_particles=int(max_particles), **self.kw)
        est.set_randoms(*self.randoms)
        self.contexts[nmesh] = est
        return est

    def run(self, mocks: Sequence, nmeshes: Sequence[int], ells: Sequence[int], k_edges_for,
            use_graph: bool = True) -> List[dict]:
        """mocks[i] = pos or (pos, weight, nbar); nmeshes[i] its mesh side; k_edges_for(nmesh)
        gives the k edges of that side. Returns, per mock, P (n_ells, nk) and its sums as
        device tensors."""
        out: List[dict] = [None] * len(mocks)
        for n in sorted(set(nmeshes)):
            idx = [i for i, m in enumerate(nmeshes) if m == n]
            group = [mocks[i] for i in idx]
            count = max(int((g[0] if isinstance(g, (tuple, list)) else g).shape[0]) for g in group)
            est = self.context(n, count)
            res = est.run_batch(group, ells, k_edges_for(n), use_graph=use_graph)
            for j, i in enumerate(idx):
                out[i] = {"P": res["P"][j], "sums": res["sums"][j], "k_mean": res["k_mean"],
                          "n_modes": res["n_modes"], "nmesh": n}
        return out

    def close(self):
        for est in self.contexts.values():
            est.close()
        self.contexts.clear()
