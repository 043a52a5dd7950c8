"""pspec_catalog_sums_noalloc against pspec_paint, through the C ABI, on two calls in a row.

The no-allocation entry point serves callers that cannot call cudaMalloc (for example code
running while a CUDA graph is captured, or a framework whose memory pool owns the device).
Its scratch is a fixed array inside the library, shared by every call, so the second call
below, on a different catalog, also checks that nothing from the first call leaks into it.
This file is collected last so that a run stopping at the first failure has run the rest.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1704_02357_gb300 import build
    build.build()


def _catalogs(seed, device):
    import torch
    L, corner = 400.0, (0.0, 0.0, 0.0)
    rng = np.random.default_rng(seed)
    d = synth.uniform_box(5000 + 1000 * seed, L, corner, seed)
    r = synth.uniform_box(20000 + 3000 * seed, L, corner, seed + 100)
    dw = 0.5 + rng.random(d.size)
    rw = 0.5 + rng.random(r.size)
    dn = np.full(d.size, 1e-4 * (1 + seed))
    rn = 1e-4 * (1 + seed) * (0.9 + 0.2 * rng.random(r.size))
    t = lambda a: torch.as_tensor(a, dtype=torch.float64, device=device).contiguous()
    return t(d.pos), t(r.pos), t(dw), t(dn), t(rw), t(rn)


def test_noalloc_matches_paint_on_two_calls():
    import torch
    from paper_1704_02357_gb300 import Estimator, pspec
    dev = torch.device("cuda", 0)
    est = Estimator(nmesh=32, box_size=400.0, box_corner=(0.0, 0.0, 0.0), P0=1e4, nbar=1e-4, device=dev)
    out = torch.full((10,), float("nan"), dtype=torch.float64, device=dev)
    for seed in (1, 2):
        dp, rp, dw, dn, rw, rn = _catalogs(seed, dev)
        ref = est.paint(dp, rp, dw, dn, rw, rn)          # the existing entry point
        torch.cuda.synchronize()
        before = torch.cuda.memory_allocated(dev)
        pspec.catalog_sums_noalloc(est.params, dp, rp, out, dw, dn, rw, rn)
        torch.cuda.synchronize()
        assert torch.cuda.memory_allocated(dev) == before
        got = out.cpu().numpy()
        for key, idx in (("W_d", 0), ("W_r", 1), ("alpha", 2), ("I", 3), ("S", 4)):
            assert abs(got[idx] - ref[key]) <= 1e-12 * abs(ref[key]), (seed, key, got[idx], ref[key])
    est.close()


def test_noalloc_rejects_more_partials_than_its_scratch_holds():
    import torch
    from paper_1704_02357_gb300 import Estimator, PspecError, pspec
    dev = torch.device("cuda", 0)
    est = Estimator(nmesh=32, box_size=400.0, box_corner=(0.0, 0.0, 0.0), P0=1e4, nbar=1e-4, device=dev)
    out = torch.zeros(10, dtype=torch.float64, device=dev)
    dp, rp, dw, dn, rw, rn = _catalogs(3, dev)
    with pytest.raises(PspecError) as e:
        pspec.catalog_sums_noalloc(est.params, dp, rp, out, dw, dn, rw, rn, nblocks=1025)
    assert e.value.status == pspec.EINVAL
    pspec.catalog_sums_noalloc(est.params, dp, rp, out, dw, dn, rw, rn, nblocks=1024)
    torch.cuda.synchronize()
    ref = est.paint(dp, rp, dw, dn, rw, rn)
    assert abs(out[2].item() - ref["alpha"]) <= 1e-12 * ref["alpha"]
    est.close()


def test_noalloc_binding_checks_its_buffers_instead_of_copying():
    """The Python binding refuses what would make it allocate or write out of bounds: a short
    or non-float64 `out`, and catalog arrays that are not already contiguous tensors on `out`'s
    device (it would otherwise have to copy them there)."""
    import torch
    from paper_1704_02357_gb300 import Estimator, pspec
    dev = torch.device("cuda", 0)
    est = Estimator(nmesh=32, box_size=400.0, box_corner=(0.0, 0.0, 0.0), P0=1e4, nbar=1e-4, device=dev)
    dp, rp, dw, dn, rw, rn = _catalogs(4, dev)
    for bad in (torch.zeros(9, dtype=torch.float64, device=dev), torch.zeros(10, dtype=torch.float32, device=dev),
                torch.zeros(10, dtype=torch.float64)):
        with pytest.raises(ValueError):
            pspec.catalog_sums_noalloc(est.params, dp, rp, bad, dw, dn, rw, rn)
    out = torch.zeros(10, dtype=torch.float64, device=dev)
    with pytest.raises(ValueError):
        pspec.catalog_sums_noalloc(est.params, dp.cpu().numpy(), rp, out)
    with pytest.raises(ValueError):
        pspec.catalog_sums_noalloc(est.params, dp, rp, out, dw[:-1])
    est.close()
