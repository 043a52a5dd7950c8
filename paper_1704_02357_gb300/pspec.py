"""ctypes binding of libpspec (include/pspec.h): argument marshalling only.

Every step of the estimator runs in the library's CUDA kernels. PyTorch supplies device
memory (the workspace and the catalogs) and the CUDA stream. If libpspec.so is missing the
binding raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libpspec.so")

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ECANCELED, EUNSUPPORTED, ESTATE = range(8)
WINDOWS = {"cic": 2, "tsc": 3}
PRECISIONS = {"fp32": 0, "fp64": 1, "fp32_plain": 2}
K_NAMES = ["catalog_sums", "paint", "r2c_z", "fft_y", "fft_x", "combine_x", "ylm_r2c_z", "bin_x",
           "c2r_z", "finalize", "other"]


class PspecError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"pspec status {status}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("nmesh", C.c_int32), ("window", C.c_int32), ("interlaced", C.c_int32),
                ("compensate", C.c_int32), ("precision", C.c_int32), ("ell_max", C.c_int32),
                ("box_size", C.c_double), ("box_corner", C.c_double * 3), ("observer", C.c_double * 3),
                ("P0", C.c_double), ("nbar", C.c_double), ("max_group_bytes", C.c_int64),
                ("max_particles", C.c_int64), ("cache_randoms", C.c_int32), ("ylm_table", C.c_int32),
                ("cartesian", C.c_int32)]


class Catalog(C.Structure):
    _fields_ = [("pos", C.c_void_p), ("pos_dtype", C.c_int32), ("weight", C.c_void_p),
                ("nbar", C.c_void_p), ("count", C.c_int64)]


class Stats(C.Structure):
    _fields_ = [("alpha", C.c_double), ("I", C.c_double), ("S", C.c_double), ("W_d", C.c_double),
                ("W_r", C.c_double), ("n_nonfinite", C.c_int64), ("n_wrapped", C.c_int64)]


class Tuning(C.Structure):
    _fields_ = [("paint_binned", C.c_int32), ("ylm_harmonics", C.c_int32), ("bin_blocks_per_sm", C.c_int32),
                ("tile_y", C.c_int32)]


class PlanInfo(C.Structure):
    _fields_ = [("nmesh", C.c_int32), ("precision", C.c_int32), ("ell_max", C.c_int32),
                ("tile_y", C.c_int32), ("tile_x", C.c_int32), ("tile_bin", C.c_int32), ("rows_z", C.c_int32),
                ("group_max", C.c_int32), ("bin_ctas", C.c_int32), ("sh_transforms", C.c_int64),
                ("transforms_executed", C.c_int64), ("kernel_launches", C.c_int64),
                ("model_bytes_last", C.c_double), ("ylm_table_bytes", C.c_int64),
                ("cartesian_table_bytes", C.c_int64), ("ylm_rtable_bytes", C.c_int64)]


_lib = None

# (name, restype, argtypes) for every entry point of include/pspec.h
SIGNATURES = [
    ("pspec_workspace_size", C.c_int32, [C.POINTER(Params), C.c_int32, C.POINTER(C.c_int64)]),
    ("pspec_create", C.c_int32, [C.POINTER(Params), C.c_int32, C.c_void_p, C.c_void_p, C.c_int64, C.c_int32,
                                 C.POINTER(C.c_void_p)]),
    ("pspec_destroy", C.c_int32, [C.c_void_p]),
    ("pspec_paint", C.c_int32, [C.c_void_p, C.POINTER(Catalog), C.POINTER(Catalog), C.POINTER(Stats)]),
    ("pspec_multipoles", C.c_int32, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_double),
                                     C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double),
                                     C.POINTER(C.c_double)]),
    ("pspec_multipoles_device", C.c_int32, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32,
                                            C.POINTER(C.c_double), C.c_int32, C.c_void_p, C.c_void_p,
                                            C.c_void_p]),
    ("pspec_wedges", C.c_int32, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.c_int32,
                                 C.POINTER(C.c_double), C.c_int32, C.c_void_p, C.c_void_p]),
    ("pspec_get_plan_info", C.c_int32, [C.c_void_p, C.POINTER(PlanInfo)]),
    ("pspec_set_profiling", C.c_int32, [C.c_void_p, C.c_int32]),
    ("pspec_kernel_times", C.c_int32, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_double),
                                       C.POINTER(C.c_double)]),
    ("pspec_kernel_name", C.c_char_p, [C.c_int32]),
    ("pspec_strerror", C.c_char_p, [C.c_int32]),
    ("pspec_last_error", C.c_char_p, [C.c_void_p]),
    ("pspec_version", C.c_char_p, []),
    ("pspec_set_randoms", C.c_int32, [C.c_void_p, C.POINTER(Catalog)]),
    ("pspec_run_batch", C.c_int32, [C.c_void_p, C.POINTER(Catalog), C.c_int32, C.POINTER(C.c_int32), C.c_int32,
                                    C.POINTER(C.c_double), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                    C.c_int32]),
    ("pspec_get_tuning", C.c_int32, [C.c_void_p, C.POINTER(Tuning)]),
    ("pspec_set_tuning", C.c_int32, [C.c_void_p, C.POINTER(Tuning)]),
    ("pspec_autotune", C.c_int32, [C.c_void_p, C.POINTER(Catalog), C.POINTER(Catalog), C.POINTER(C.c_int32),
                                   C.c_int32, C.POINTER(C.c_double), C.c_int32, C.c_int32, C.POINTER(Tuning)]),
    ("pspec_multipoles_cartesian", C.c_int32, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32,
                                               C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double),
                                               C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    ("pspec_transverse_response", C.c_int32, [C.c_int32, C.POINTER(C.c_double), C.c_int32, C.POINTER(C.c_double)]),
    ("pspec_mu_edges_nonuniform", C.c_int32, [C.c_int32, C.POINTER(C.c_double)]),
    ("pspec_wedge_lbar", C.c_int32, [C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_double), C.c_int32,
                                     C.POINTER(C.c_double)]),
    ("pspec_wedge_gamma_kaiser", C.c_int32, [C.c_int32, C.POINTER(C.c_double), C.c_int32, C.c_double,
                                             C.POINTER(C.c_double)]),
    ("pspec_multipoles_range", C.c_int32, [C.c_void_p, C.POINTER(C.c_int32), C.c_int32, C.POINTER(C.c_double),
                                           C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_void_p]),
    ("pspec_finalize_bins", C.c_int32, [C.c_void_p, C.c_void_p, C.POINTER(C.c_int32), C.c_int32,
                                        C.POINTER(C.c_double), C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    ("pspec_catalog_sums_noalloc", C.c_int32, [C.POINTER(Params), C.POINTER(Catalog), C.POINTER(Catalog), C.c_int32,
                                               C.c_void_p, C.c_void_p]),
]


def compensation_code(compensate) -> int:
    """False/True, or a form: "sinc" (1), "jing" (2), "sinc_per_mode" (3, 1/W^2 on each binned mode)."""
    codes = {False: 0, True: 1, 0: 0, 1: 1, 2: 2, 3: 3, "sinc": 1, "jing": 2, "sinc_per_mode": 3}
    if compensate not in codes:
        raise ValueError(f"unknown compensation {compensate!r}")
    return codes[compensate]


def load(path: str = LIB_PATH):
    """Load libpspec.so and declare its signatures. Raises if it is not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"{path} is missing: build it with `python -m paper_1704_02357_gb300.build`")
    lib = C.CDLL(path)
    for name, res, args in SIGNATURES:
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(st: int, ctx=None):
    if st != OK:
        lib = load()
        detail = lib.pspec_last_error(ctx).decode() if ctx else ""
        raise PspecError(st, f"{lib.pspec_strerror(st).decode()} {detail}".strip())


def _ptr(t) -> Optional[int]:
    return None if t is None else int(t.data_ptr())


def _dev_tensor(x, dtype, device, name):
    import torch
    if x is None:
        return None
    if not isinstance(x, torch.Tensor):
        x = torch.as_tensor(np.ascontiguousarray(x))
    if x.dtype != dtype:
        x = x.to(dtype)
    return x.to(device).contiguous()


def _catalog(pos, weight, nbar, device, keep):
    import torch
    p = pos if isinstance(pos, torch.Tensor) else torch.as_tensor(np.ascontiguousarray(pos))
    if p.dim() != 2 or p.shape[1] != 3:
        raise ValueError("positions must be (n, 3)")
    if p.dtype not in (torch.float64, torch.float32):
        p = p.to(torch.float64)
    p = p.to(device).contiguous()
    w = _dev_tensor(weight, torch.float64, device, "weight")
    nb = _dev_tensor(nbar, torch.float64, device, "nbar")
    keep.extend([p, w, nb])
    return Catalog(_ptr(p) if p.numel() else None, 1 if p.dtype == torch.float32 else 0, _ptr(w), _ptr(nb),
                   int(p.shape[0]))


class Estimator:
    """One estimator context: a mesh geometry, window and precision, on one device/stream."""

    def __init__(self, nmesh: int, box_size: float, box_corner, observer=(0.0, 0.0, 0.0), window="cic",
                 interlaced=False, compensate=True, precision="fp32", ell_max=4, P0=0.0, nbar=0.0,
                 max_group_bytes=0, max_kbins=512, max_particles=0, cache_randoms=False, device=None,
                 stream=None, ylm_table=True, cartesian=False):
        import torch
        lib = load()
        self.device = torch.device(device if device is not None else "cuda", )
        if self.device.index is None:
            self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        comp = compensation_code(compensate)
        self.params = Params(int(nmesh), WINDOWS[window], int(bool(interlaced)), comp,
                             PRECISIONS[precision], int(ell_max), float(box_size),
                             (C.c_double * 3)(*box_corner), (C.c_double * 3)(*observer), float(P0), float(nbar),
                             int(max_group_bytes), int(max_particles), int(bool(cache_randoms)),
                             0 if ylm_table else -1, int(bool(cartesian)))
        self.max_kbins = int(max_kbins)
        nbytes = C.c_int64(0)
        with torch.cuda.device(self.device):
            _check(lib.pspec_workspace_size(C.byref(self.params), self.max_kbins, C.byref(nbytes)))
            self.workspace_bytes = int(nbytes.value)
            self._ws = torch.empty(self.workspace_bytes + 256, dtype=torch.uint8, device=self.device)
        base = self._ws.data_ptr()
        self._ws_ptr = (base + 255) // 256 * 256
        ctx = C.c_void_p()
        _check(lib.pspec_create(C.byref(self.params), self.device.index, C.c_void_p(self.stream.cuda_stream),
                                C.c_void_p(self._ws_ptr), self.workspace_bytes, self.max_kbins, C.byref(ctx)))
        self._ctx = ctx
        self._keep = []

    # ------------------------------------------------------------------ a1 + a2
    def paint(self, data_pos, randoms_pos, data_weight=None, data_nbar=None, randoms_weight=None,
              randoms_nbar=None, stats=True):
        lib = load()
        keep = []
        d = _catalog(data_pos, data_weight, data_nbar, self.device, keep)
        r = _catalog(randoms_pos, randoms_weight, randoms_nbar, self.device, keep)
        self._keep = keep  # inputs must outlive the enqueued kernels
        st = Stats()
        _check(lib.pspec_paint(self._ctx, C.byref(d), C.byref(r), C.byref(st) if stats else None), self._ctx)
        if not stats:
            return None
        return {f: getattr(st, f) for f, _ in Stats._fields_}

    # ------------------------------------------------------------------ a3..a6
    def multipoles(self, ells: Sequence[int], k_edges) -> dict:
        lib = load()
        ells = [int(e) for e in ells]
        edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        nk = len(edges) - 1
        el = (C.c_int32 * len(ells))(*ells)
        P = np.empty((len(ells), nk))
        km = np.empty(nk)
        nm = np.empty(nk)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        _check(lib.pspec_multipoles(self._ctx, el, len(ells), dp(edges), nk, dp(P), dp(km), dp(nm)), self._ctx)
        return {"P": P, "k_mean": km, "n_modes": nm, "ells": ells}

    def multipoles_cartesian(self, ells: Sequence[int], k_edges) -> dict:
        """l in {0, 2, 4} through the Cartesian decomposition (22 transforms for l <= 4); needs
        an FP32 context created with cartesian=True."""
        lib = load()
        ells = [int(e) for e in ells]
        edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        nk = len(edges) - 1
        el = (C.c_int32 * len(ells))(*ells)
        P = np.empty((len(ells), nk))
        km = np.empty(nk)
        nm = np.empty(nk)
        dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
        _check(lib.pspec_multipoles_cartesian(self._ctx, el, len(ells), dp(edges), nk, dp(P), dp(km), dp(nm)),
               self._ctx)
        return {"P": P, "k_mean": km, "n_modes": nm, "ells": ells}

    def multipoles_device(self, ells: Sequence[int], k_edges, P_out, kmean_out, nmodes_out):
        """Enqueue without synchronising; outputs are float64 CUDA tensors (n_ells*nk, nk, nk)."""
        lib = load()
        ells = [int(e) for e in ells]
        edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        el = (C.c_int32 * len(ells))(*ells)
        _check(lib.pspec_multipoles_device(self._ctx, el, len(ells), edges.ctypes.data_as(C.POINTER(C.c_double)),
                                           len(edges) - 1, C.c_void_p(_ptr(P_out)), C.c_void_p(_ptr(kmean_out)),
                                           C.c_void_p(_ptr(nmodes_out))), self._ctx)

    def multipoles_range(self, ells: Sequence[int], k_edges, q0: int, q1: int, include_p0=True, bins=None):
        """Raw FP64 bin sums, shape (1 + n_ells, nk), of items [q0, q1) of the flat harmonic list
        (l >= 2 in the order of ells, m = 0, +1, -1, +2, ... within l). Enqueued, not synchronised."""
        import torch
        lib = load()
        ells = [int(e) for e in ells]
        edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        nk = len(edges) - 1
        if bins is None:
            # allocated on the context's stream, which writes it (the caching allocator keeps it
            # there until that stream's work on it is done)
            with torch.cuda.stream(self.stream):
                bins = torch.empty((1 + len(ells), nk), dtype=torch.float64, device=self.device)
        el = (C.c_int32 * len(ells))(*ells)
        _check(lib.pspec_multipoles_range(self._ctx, el, len(ells), edges.ctypes.data_as(C.POINTER(C.c_double)), nk,
                                          int(q0), int(q1), int(bool(include_p0)), C.c_void_p(_ptr(bins))), self._ctx)
        return bins

    def finalize_bins(self, bins, ells: Sequence[int], k_edges) -> dict:
        """Multipoles from summed raw bins (device tensors out, enqueued on the context stream)."""
        import torch
        lib = load()
        ells = [int(e) for e in ells]
        edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        nk = len(edges) - 1
        with torch.cuda.stream(self.stream):  # written by the context's stream
            P = torch.empty((len(ells), nk), dtype=torch.float64, device=self.device)
            km = torch.empty(nk, dtype=torch.float64, device=self.device)
            nm = torch.empty(nk, dtype=torch.float64, device=self.device)
        el = (C.c_int32 * len(ells))(*ells)
        _check(lib.pspec_finalize_bins(self._ctx, C.c_void_p(_ptr(bins)), el, len(ells),
                                       edges.ctypes.data_as(C.POINTER(C.c_double)), nk, C.c_void_p(_ptr(P)),
                                       C.c_void_p(_ptr(km)), C.c_void_p(_ptr(nm))), self._ctx)
        return {"P": P, "k_mean": km, "n_modes": nm, "ells": ells}

    # ------------------------------------------------------------------ batched mocks
    def set_randoms(self, pos, weight=None, nbar=None):
        """Paint the shared randoms once into the cached meshes (needs cache_randoms=True)."""
        keep = []
        r = _catalog(pos, weight, nbar, self.device, keep)
        self._rkeep = keep
        _check(load().pspec_set_randoms(self._ctx, C.byref(r)), self._ctx)

    def run_batch(self, mocks, ells: Sequence[int], k_edges, use_graph=True):
        """Multipoles of every mock (list of (pos[, weight[, nbar]])) against the cached randoms.

        Returns device tensors P (n_mocks, n_ells, nk), sums (n_mocks, 4: alpha, I, S, W_d),
        k_mean (nk), n_modes (nk); enqueued on the context's stream.
        """
        import torch
        ells = [int(e) for e in ells]
        edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        nk = len(edges) - 1
        keep = []
        cats = []
        for m in mocks:
            m = m if isinstance(m, (tuple, list)) else (m,)
            cats.append(_catalog(m[0], m[1] if len(m) > 1 else None, m[2] if len(m) > 2 else None, self.device, keep))
        arr = (Catalog * len(cats))(*cats)
        with torch.cuda.stream(self.stream):  # written by the context's stream
            P = torch.empty((len(cats), len(ells), nk), dtype=torch.float64, device=self.device)
            sums = torch.empty((len(cats), 4), dtype=torch.float64, device=self.device)
            km = torch.empty(nk, dtype=torch.float64, device=self.device)
            nm = torch.empty(nk, dtype=torch.float64, device=self.device)
        el = (C.c_int32 * len(ells))(*ells)
        _check(load().pspec_run_batch(self._ctx, arr, len(cats), el, len(ells),
                                      edges.ctypes.data_as(C.POINTER(C.c_double)), nk, C.c_void_p(P.data_ptr()),
                                      C.c_void_p(sums.data_ptr()), C.c_void_p(km.data_ptr()),
                                      C.c_void_p(nm.data_ptr()), int(bool(use_graph))), self._ctx)
        self._bkeep = keep
        return {"P": P, "sums": sums, "k_mean": km, "n_modes": nm, "ells": ells}

    # ------------------------------------------------------------------ tuning
    def tuning(self) -> dict:
        t = Tuning()
        _check(load().pspec_get_tuning(self._ctx, C.byref(t)), self._ctx)
        return {f: getattr(t, f) for f, _ in Tuning._fields_}

    def set_tuning(self, **kw):
        cur = self.tuning()
        cur.update({k: int(v) for k, v in kw.items()})
        t = Tuning(*[cur[f] for f, _ in Tuning._fields_])
        _check(load().pspec_set_tuning(self._ctx, C.byref(t)), self._ctx)

    def autotune(self, data_pos, randoms_pos, ells, k_edges, reps=2, data_weight=None, data_nbar=None,
                 randoms_weight=None, randoms_nbar=None) -> dict:
        """Time candidate knob settings on these catalogs (native search) and keep the best."""
        keep = []
        d = _catalog(data_pos, data_weight, data_nbar, self.device, keep)
        r = _catalog(randoms_pos, randoms_weight, randoms_nbar, self.device, keep)
        ells = [int(e) for e in ells]
        edges = np.ascontiguousarray(k_edges, dtype=np.float64)
        el = (C.c_int32 * len(ells))(*ells)
        best = Tuning()
        _check(load().pspec_autotune(self._ctx, C.byref(d), C.byref(r), el, len(ells),
                                     edges.ctypes.data_as(C.POINTER(C.c_double)), len(edges) - 1, int(reps),
                                     C.byref(best)), self._ctx)
        self._keep = keep
        return {f: getattr(best, f) for f, _ in Tuning._fields_}

    def plan_info(self) -> dict:
        info = PlanInfo()
        _check(load().pspec_get_plan_info(self._ctx, C.byref(info)), self._ctx)
        return {f: getattr(info, f) for f, _ in PlanInfo._fields_}

    def set_profiling(self, on: bool):
        _check(load().pspec_set_profiling(self._ctx, int(bool(on))), self._ctx)

    def kernel_times(self) -> dict:
        n = len(K_NAMES)
        la = (C.c_int64 * n)()
        ms = (C.c_double * n)()
        by = (C.c_double * n)()
        _check(load().pspec_kernel_times(self._ctx, la, ms, by), self._ctx)
        return {K_NAMES[k]: {"launches": la[k], "ms": ms[k], "bytes": by[k]} for k in range(n)}

    def close(self):
        """Destroy the context and release its workspace (and the inputs it kept alive)."""
        if getattr(self, "_ctx", None):
            load().pspec_destroy(self._ctx)
            self._ctx = None
        self._ws = None
        self._keep = []

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def wedges(P, ells: Sequence[int], mu_edges, stream=None):
    """P(k, mu) wedges from multipoles (a float64 CUDA tensor (n_ells, nk)); returns (n_mu, nk)."""
    import torch
    lib = load()
    P = P.contiguous()
    if P.dtype != torch.float64 or not P.is_cuda:
        raise ValueError("P must be a float64 CUDA tensor")
    mu = np.ascontiguousarray(mu_edges, dtype=np.float64)
    ells = [int(e) for e in ells]
    n_mu = len(mu) - 1
    s = stream if stream is not None else torch.cuda.current_stream(P.device)
    with torch.cuda.stream(s):  # written by the kernel on `s`
        out = torch.empty((n_mu, P.shape[1]), dtype=torch.float64, device=P.device)
    el = (C.c_int32 * len(ells))(*ells)
    _check(lib.pspec_wedges(C.c_void_p(P.data_ptr()), el, len(ells), int(P.shape[1]),
                            mu.ctypes.data_as(C.POINTER(C.c_double)), n_mu, C.c_void_p(out.data_ptr()),
                            C.c_void_p(s.cuda_stream)))
    return out


def catalog_sums_noalloc(params: Params, data_pos, randoms_pos, out, data_weight=None, data_nbar=None,
                         randoms_weight=None, randoms_nbar=None, nblocks=0, stream=None):
    """Enqueue pspec_catalog_sums_noalloc (the catalog sums of paint, without device allocation).

    Every array must already be a contiguous CUDA tensor on `out`'s device: positions float64
    or float32 (n, 3), weights and nbar float64. Nothing is copied or converted here, so the
    call allocates no device memory (a host array or a tensor on another device raises
    ValueError instead of being copied over). `out` is a contiguous float64 CUDA tensor of at
    least 10 elements; it receives the values in the order of the library's derived layout
    (W_d, W_r, alpha, I, S, ...). The call is enqueued on `stream` (default: the current stream
    of `out`'s device) with that device current.
    """
    import torch
    if not (isinstance(out, torch.Tensor) and out.is_cuda and out.dtype == torch.float64
            and out.is_contiguous() and out.numel() >= 10):
        raise ValueError("out must be a contiguous float64 CUDA tensor of at least 10 elements")

    def dev_array(a, name, dtypes, ndim):
        if a is None:
            return None
        if not (isinstance(a, torch.Tensor) and a.is_cuda and a.device == out.device and a.is_contiguous()):
            raise ValueError(f"{name} must be a contiguous CUDA tensor on {out.device} (no copies are made)")
        if a.dtype not in dtypes or a.dim() != ndim or (ndim == 2 and a.shape[1] != 3):
            raise ValueError(f"{name} has dtype {a.dtype} and shape {tuple(a.shape)}")
        return a

    pos_t = (torch.float64, torch.float32)
    f64 = (torch.float64,)
    dp = dev_array(data_pos, "data_pos", pos_t, 2)
    rp = dev_array(randoms_pos, "randoms_pos", pos_t, 2)
    if dp is None or rp is None:
        raise ValueError("data_pos and randoms_pos are required")
    dw, dn = dev_array(data_weight, "data_weight", f64, 1), dev_array(data_nbar, "data_nbar", f64, 1)
    rw, rn = dev_array(randoms_weight, "randoms_weight", f64, 1), dev_array(randoms_nbar, "randoms_nbar", f64, 1)
    for a, n in ((dw, dp), (dn, dp), (rw, rp), (rn, rp)):
        if a is not None and a.shape[0] != n.shape[0]:
            raise ValueError("a weight or nbar array does not match its positions")
    lib = load()
    with torch.cuda.device(out.device):
        keep = []
        d = _catalog(dp, dw, dn, out.device, keep)
        r = _catalog(rp, rw, rn, out.device, keep)
        s = stream if stream is not None else torch.cuda.current_stream(out.device)
        st = lib.pspec_catalog_sums_noalloc(C.byref(params), C.byref(d), C.byref(r), int(nblocks),
                                            C.c_void_p(out.data_ptr()), C.c_void_p(s.cuda_stream))
    _check(st)
    return keep


def transverse_response(ell_max: int, mu) -> np.ndarray:
    """R(mu) of a mu = 0 spike reconstructed from even multipoles up to ell_max (Sec. 3.1)."""
    mu = np.ascontiguousarray(mu, dtype=np.float64)
    out = np.empty_like(mu)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    _check(load().pspec_transverse_response(int(ell_max), dp(mu), mu.size, dp(out)))
    return out


def mu_edges_nonuniform(ell_max: int) -> np.ndarray:
    """Wedge edges confining a mu = 0 spike to the first wedge (Sec. 3.1, ell_max/2 + 1 wedges)."""
    out = np.empty(int(ell_max) // 2 + 2)
    _check(load().pspec_mu_edges_nonuniform(int(ell_max), out.ctypes.data_as(C.POINTER(C.c_double))))
    return out


def wedge_lbar(ells: Sequence[int], mu_edges) -> np.ndarray:
    """(n_mu, n_ells) mean Legendre polynomials over each wedge (Sec. 2.2 eq. Lbar)."""
    mu = np.ascontiguousarray(mu_edges, dtype=np.float64)
    ells = [int(e) for e in ells]
    out = np.empty((len(mu) - 1, len(ells)))
    el = (C.c_int32 * len(ells))(*ells)
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    _check(load().pspec_wedge_lbar(el, len(ells), dp(mu), len(mu) - 1, dp(out)))
    return out


def wedge_gamma_kaiser(ell_max: int, mu_edges, beta: float) -> np.ndarray:
    """gamma_mn of Sec. 4.1 (Kaiser-model wedge covariance, angular part)."""
    mu = np.ascontiguousarray(mu_edges, dtype=np.float64)
    out = np.empty((len(mu) - 1, len(mu) - 1))
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    _check(load().pspec_wedge_gamma_kaiser(int(ell_max), dp(mu), len(mu) - 1, float(beta), dp(out)))
    return out
