"""Sharding one catalog's harmonics over ranks (host logic, CPU, gloo).

Each rank's share of the work is played by a stand-in estimator built from the oracle's own
steps (the raw bin sums of a harmonic range, Sec. 2.1 eqs. Pell-ours and Fell). The gloo runs
check that the ranges cover the harmonic list once, that the l = 0 bins are counted once, and
that the all-reduced, finalized result is the oracle's single-process answer.
"""
import math
import os
import socket
import tempfile

import numpy as np
import pytest

import synth
from oracle import estimator as E
from paper_1704_02357_gb300.parallel import harmonic_items, sharded_multipoles, split

L = 300.0
CORNER = (0.0, 0.0, 0.0)
OBS = (-250.0, -150.0, -200.0)
ELLS = [0, 2, 4]


@pytest.mark.parametrize("n_items", [0, 1, 5, 14, 17, 153])
@pytest.mark.parametrize("world", [1, 2, 3, 4, 8])
def test_split_covers_each_item_once(n_items, world):
    seen = []
    sizes = []
    prev = 0
    for r in range(world):
        q0, q1 = split(n_items, world, r)
        assert q0 == prev and q1 >= q0
        prev = q1
        seen.extend(range(q0, q1))
        sizes.append(q1 - q0)
    assert seen == list(range(n_items))
    assert max(sizes) - min(sizes) <= 1


def test_split_rejects_bad_ranks():
    with pytest.raises(ValueError):
        split(5, 0, 0)
    with pytest.raises(ValueError):
        split(5, 2, 2)


def test_harmonic_items_order_and_count():
    items = harmonic_items([0, 2, 4, 16])
    assert len(items) == 5 + 9 + 33
    assert items[:5] == [(2, 0), (2, 1), (2, -1), (2, 2), (2, -2)]
    assert items[5] == (4, 0) and items[-1] == (16, -16)
    # every (l, m) once; with the one l = 0 transform this is the SH transform count
    assert len(set(items)) == len(items)
    assert len(harmonic_items(range(0, 9, 2))) + 1 == E.fft_count_sh(8)
    # odd l: 2l+1 harmonics each, in the order asked
    odd = harmonic_items([3, 0, 1])
    assert len(odd) == 7 + 3 and odd[:3] == [(3, 0), (3, 1), (3, -1)] and odd[-3:] == [(1, 0), (1, 1), (1, -1)]


class OracleShard:
    """Stand-in for an Estimator holding painted meshes: raw bins of a harmonic range."""

    def __init__(self, params, data, randoms):
        import torch
        self.p = params
        self.fl = E.density_fields(data, randoms, params)
        self.torch = torch

    def _binning(self, k_edges):
        b, mult, n2 = E.mode_binning(self.p.nmesh, self.p.box_size, np.asarray(k_edges, dtype=np.float64))
        sel = b >= 0
        return b[sel], mult[sel], n2[sel], sel

    def multipoles_range(self, ells, k_edges, q0, q1, include_p0=True):
        nk = len(k_edges) - 1
        bs, ms, _, sel = self._binning(k_edges)
        bins = np.zeros((1 + len(ells), nk))
        F0 = self.fl.F0
        if include_p0:
            bins[0] = np.bincount(bs, weights=ms * np.abs(F0[sel]) ** 2, minlength=nk)
        khat = E.mode_khat(self.p.nmesh)
        for q, (ell, m) in enumerate(harmonic_items(ells)):
            if not q0 <= q < q1:
                continue
            G = E.harmonic_spectrum(self.fl.f, self.p, ell, m)
            prod = G * np.conj(F0)
            acc = E.real_ylm(ell, m, *khat) * (np.imag(prod) if ell % 2 else np.real(prod))
            bins[1 + list(ells).index(ell)] += np.bincount(bs, weights=ms * acc[sel], minlength=nk)
        return self.torch.from_numpy(bins)

    def finalize_bins(self, bins, ells, k_edges):
        bins = bins.numpy()
        bs, ms, _, _ = self._binning(k_edges)
        nmodes = np.bincount(bs, weights=ms, minlength=len(k_edges) - 1)
        I, S = self.fl.sums["I"], self.fl.sums["S"]
        P = np.zeros((len(ells), len(k_edges) - 1))
        for i, ell in enumerate(ells):
            P[i] = (bins[0] / nmodes - S) / I if ell == 0 else 4.0 * math.pi * bins[1 + i] / (I * nmodes)
        return {"P": P, "n_modes": nmodes}


def _case():
    p = E.Params(nmesh=16, box_size=L, box_corner=CORNER, observer=OBS, window="tsc", interlaced=True,
                 compensate=True, P0=1e4, nbar=1e-5)
    data = synth.uniform_box(1500, L, CORNER, 21)
    randoms = synth.uniform_box(6000, L, CORNER, 22)
    edges = np.linspace(0.0, math.pi * 16 / L, 6)
    return p, data, randoms, edges


def _rank_main(rank, world, port, out_dir, ells=ELLS):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, data, randoms, edges = _case()
        res = sharded_multipoles(OracleShard(p, data, randoms), ells, edges)
        np.save(os.path.join(out_dir, f"P{rank}.npy"), res["P"])
    finally:
        dist.destroy_process_group()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("world,ells", [(2, ELLS), (3, ELLS), (2, [0, 1, 2, 3])])
def test_sharded_multipoles_over_gloo_ranks(world, ells):
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with tempfile.TemporaryDirectory() as d:
        port = _free_port()
        procs = [ctx.Process(target=_rank_main, args=(r, world, port, d, ells)) for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=240)
        assert all(pr.exitcode == 0 for pr in procs), [pr.exitcode for pr in procs]
        Ps = [np.load(os.path.join(d, f"P{r}.npy")) for r in range(world)]
    p, data, randoms, edges = _case()
    o = E.multipoles(data, randoms, p, ells, edges)
    scale = (np.abs(o["P"][0]) + o["S"] / o["I"]).max()
    for P in Ps:
        np.testing.assert_allclose(P, o["P"], rtol=1e-10, atol=1e-12 * scale)
        np.testing.assert_array_equal(P, Ps[0])


def test_single_rank_runs_everything_without_a_process_group():
    p, data, randoms, edges = _case()
    res = sharded_multipoles(OracleShard(p, data, randoms), ELLS, edges, rank=0, world=1)
    o = E.multipoles(data, randoms, p, ELLS, edges)
    scale = (np.abs(o["P"][0]) + o["S"] / o["I"]).max()
    np.testing.assert_allclose(res["P"], o["P"], rtol=1e-10, atol=1e-12 * scale)


def test_dropping_a_rank_share_is_detected():
    """A range that skips one harmonic changes the answer: the check above has teeth."""
    p, data, randoms, edges = _case()
    sh = OracleShard(p, data, randoms)
    n = len(harmonic_items(ELLS))
    full = sh.multipoles_range(ELLS, edges, 0, n)
    part = sh.multipoles_range(ELLS, edges, 0, n - 1)
    P_full = sh.finalize_bins(full, ELLS, edges)["P"]
    P_part = sh.finalize_bins(part, ELLS, edges)["P"]
    assert np.max(np.abs(P_full[2] - P_part[2])) > 1e-6 * np.max(np.abs(P_full[0]))


class ContractShard(OracleShard):
    """OracleShard that checks every call against the contract of Estimator.multipoles_range /
    finalize_bins (pspec_multipoles_range, pspec_finalize_bins): the range [q0, q1) is this
    rank's contiguous share of the flat harmonic list, only rank 0 asks for the l = 0 bins, the
    raw bins are a float64 torch tensor of shape (1 + n_ells, nk) whose row 0 is zero without
    include_p0, and finalize_bins receives that same tensor, summed over the ranks in place."""

    def __init__(self, params, data, randoms, rank, world):
        super().__init__(params, data, randoms)
        self.rank, self.world = rank, world
        self.calls = []

    def multipoles_range(self, ells, k_edges, q0, q1, include_p0=True):
        assert (q0, q1) == split(len(harmonic_items(ells)), self.world, self.rank)
        assert bool(include_p0) == (self.rank == 0)
        bins = super().multipoles_range(ells, k_edges, q0, q1, include_p0=include_p0)
        assert bins.dtype == self.torch.float64 and tuple(bins.shape) == (1 + len(ells), len(k_edges) - 1)
        if not include_p0:
            assert not bins[0].any()
        self.local = bins.clone()
        self.bins = bins
        self.calls.append(("range", q0, q1, bool(include_p0)))
        return bins

    def finalize_bins(self, bins, ells, k_edges):
        assert bins is self.bins  # the all-reduce works in place on the returned tensor
        self.calls.append(("finalize",))
        return super().finalize_bins(bins, ells, k_edges)


def _contract_rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        p, data, randoms, edges = _case()
        sh = ContractShard(p, data, randoms, rank, world)
        res = sharded_multipoles(sh, ELLS, edges)
        assert [c[0] for c in sh.calls] == ["range", "finalize"]
        np.save(os.path.join(out_dir, f"P{rank}.npy"), res["P"])
        np.save(os.path.join(out_dir, f"local{rank}.npy"), sh.local.numpy())
        np.save(os.path.join(out_dir, f"summed{rank}.npy"), sh.bins.numpy())
    finally:
        dist.destroy_process_group()


def test_sharded_multipoles_follow_the_range_contract_over_gloo():
    """Two gloo ranks drive sharded_multipoles through a stand-in that checks the product's
    range contract; the summed bins are the sum of the ranks' local bins, the same on both
    ranks, and finalize to the oracle's single-process multipoles."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    world = 2
    with tempfile.TemporaryDirectory() as d:
        port = _free_port()
        procs = [ctx.Process(target=_contract_rank, args=(r, world, port, d)) for r in range(world)]
        for pr in procs:
            pr.start()
        for pr in procs:
            pr.join(timeout=240)
        assert all(pr.exitcode == 0 for pr in procs), [pr.exitcode for pr in procs]
        local = [np.load(os.path.join(d, f"local{r}.npy")) for r in range(world)]
        summed = [np.load(os.path.join(d, f"summed{r}.npy")) for r in range(world)]
        Ps = [np.load(os.path.join(d, f"P{r}.npy")) for r in range(world)]
    np.testing.assert_array_equal(summed[0], summed[1])
    np.testing.assert_allclose(summed[0], local[0] + local[1], rtol=1e-15, atol=0)
    assert local[0][0].any() and not local[1][0].any()
    p, data, randoms, edges = _case()
    o = E.multipoles(data, randoms, p, ELLS, edges)
    scale = (np.abs(o["P"][0]) + o["S"] / o["I"]).max()
    np.testing.assert_allclose(Ps[0], o["P"], rtol=1e-10, atol=1e-12 * scale)
