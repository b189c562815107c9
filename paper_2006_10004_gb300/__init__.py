"""Python binding of the GB300 spectral TV decomposition library (``include/tvspec.h``).

Argument marshalling only: every step of the decomposition runs in the CUDA kernels of
``libtvspec.so``. There is no CPU fallback; if the library or a CUDA device is missing, the
calls raise.

Host arrays (numpy) use the host-memory mode of the C ABI; CUDA tensors (torch) use the
device-memory mode on the current torch stream.
"""
from __future__ import annotations

import ctypes
import math
import os
import threading

import numpy as np

from . import _build

__all__ = ["Plan", "Config", "TvSpecError", "load", "build", "STATUS"]

STATUS = {0: "TVSPEC_OK", 1: "TVSPEC_EINVAL", 2: "TVSPEC_ENOMEM", 3: "TVSPEC_ECUDA",
          4: "TVSPEC_ETIMEOUT", 5: "TVSPEC_ENOTREADY", 6: "TVSPEC_ECANCELLED", 7: "TVSPEC_ENOTSUP"}
OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENOTREADY, ECANCELLED, ENOTSUP = range(8)
SOLVER_CHAMBOLLE, SOLVER_FGP, SOLVER_PDHG, SOLVER_FGP_REFERENCE = range(4)
SOLVERS = {"chambolle": SOLVER_CHAMBOLLE, "fgp": SOLVER_FGP, "pdhg": SOLVER_PDHG,
           "fgp_reference": SOLVER_FGP_REFERENCE}
P_FP32, P_FP16, P_BF16, P_SNORM16 = 0, 1, 2, 3
MEM_HOST, MEM_DEVICE = 0, 1
KERNEL_AUTO, KERNEL_NAIVE, KERNEL_TILED = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_fp = ctypes.POINTER(ctypes.c_float)


class TvSpecError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        super().__init__(f"{where}: {STATUS.get(status, status)} ({detail})")


class Config(ctypes.Structure):
    _fields_ = [("p_storage", ctypes.c_int), ("warm_start", ctypes.c_int), ("tau", ctypes.c_float),
                ("kernel", ctypes.c_int), ("tile", ctypes.c_int), ("temporal_block", ctypes.c_int),
                ("use_graphs", ctypes.c_int), ("fast_math", ctypes.c_int),
                ("mem_budget_bytes", ctypes.c_size_t), ("max_batch", ctypes.c_int), ("pdl", ctypes.c_int),
                ("persistent", ctypes.c_int), ("barrier_timeout_ms", ctypes.c_int),
                ("test_barrier_noshow", ctypes.c_int), ("resident", ctypes.c_int),
                ("resident_variant", ctypes.c_int), ("acc_mode", ctypes.c_int),
                ("tune_cache", ctypes.c_char_p), ("test_fail_alloc", ctypes.c_int),
                ("test_guard_bytes", ctypes.c_int), ("tma", ctypes.c_int)]


class Request(ctypes.Structure):
    _fields_ = [("f", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int),
                ("dt", ctypes.c_double), ("K", ctypes.c_int), ("n_inner", ctypes.c_int),
                ("band_edges", ctypes.c_void_p), ("n_edges", ctypes.c_int),
                ("bands", ctypes.c_void_p), ("residual", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("u_trace", ctypes.c_void_p), ("mem_kind", ctypes.c_int),
                ("n_filters", ctypes.c_int), ("filter_H", ctypes.c_void_p),
                ("filter_residual", ctypes.c_void_p), ("filtered", ctypes.c_void_p),
                ("S_parseval", ctypes.c_void_p)]


class Crop(ctypes.Structure):
    _fields_ = [("src", ctypes.c_int), ("y", ctypes.c_int), ("x", ctypes.c_int), ("scale", ctypes.c_int)]


class TrainingRequest(ctypes.Structure):
    _fields_ = [("n_sources", ctypes.c_int), ("sources", ctypes.c_void_p), ("source_H", ctypes.c_void_p),
                ("source_W", ctypes.c_void_p), ("n_crops", ctypes.c_int), ("crops", ctypes.c_void_p),
                ("size", ctypes.c_int), ("standardize", ctypes.c_int), ("mean_std", ctypes.c_double * 2),
                ("dt", ctypes.c_double), ("K", ctypes.c_int), ("n_inner", ctypes.c_int),
                ("band_edges", ctypes.c_void_p), ("n_edges", ctypes.c_int), ("crops_out", ctypes.c_void_p),
                ("bands", ctypes.c_void_p), ("residual", ctypes.c_void_p), ("S", ctypes.c_void_p),
                ("stats", ctypes.c_void_p), ("mem_kind", ctypes.c_int)]


class RofRequest(ctypes.Structure):
    _fields_ = [("g", ctypes.c_void_p), ("H", ctypes.c_int), ("W", ctypes.c_int), ("lam", ctypes.c_double),
                ("solver", ctypes.c_int), ("max_iter", ctypes.c_int), ("gap_tol", ctypes.c_double),
                ("check_every", ctypes.c_int), ("pdhg_tau", ctypes.c_float), ("pdhg_sigma", ctypes.c_float),
                ("pdhg_gamma", ctypes.c_float), ("p1_in", ctypes.c_void_p), ("p2_in", ctypes.c_void_p),
                ("u", ctypes.c_void_p), ("p1", ctypes.c_void_p), ("p2", ctypes.c_void_p),
                ("mem_kind", ctypes.c_int), ("iterations", ctypes.c_int), ("gap", ctypes.c_double)]


class Stats(ctypes.Structure):
    _fields_ = [("kernel_launches", ctypes.c_uint64), ("graph_launches", ctypes.c_uint64),
                ("graphs_built", ctypes.c_uint64), ("decompositions", ctypes.c_uint64),
                ("workspace_bytes", ctypes.c_size_t), ("last_tile", ctypes.c_int),
                ("last_temporal_block", ctypes.c_int)]


_lock = threading.Lock()
_lib = None

# name -> (restype, argtypes) for every entry point of include/tvspec.h
_SIGS = {
    "tvspec_config_init": (None, [ctypes.POINTER(Config)]),
    "tvspec_plan_create": (ctypes.c_int, [ctypes.POINTER(Config), ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
    "tvspec_plan_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "tvspec_validate": (ctypes.c_int, [ctypes.POINTER(Request)]),
    "tvspec_decompose": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                        ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                        ctypes.c_int, ctypes.c_void_p]),
    "tvspec_decompose_ex": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.c_void_p]),
    "tvspec_resident_variant_count": (ctypes.c_int, []),
    "tvspec_resident_variant_info": (ctypes.c_int, [ctypes.c_int] + [ctypes.POINTER(ctypes.c_int)] * 4),
    "tvspec_rof_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(RofRequest), ctypes.c_void_p]),
    "tvspec_training_set": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(TrainingRequest), ctypes.c_void_p]),
    "tvspec_decompose_batch": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(Request),
                                              ctypes.c_void_p]),
    "tvspec_submit": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]),
    "tvspec_poll": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "tvspec_wait": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int]),
    "tvspec_cancel": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint64]),
    "tvspec_serving_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64),
                                            _dp, _dp]),
    "tvspec_checkpoint_bytes": (ctypes.c_size_t, [ctypes.c_void_p, ctypes.POINTER(Request)]),
    "tvspec_decompose_steps": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Request), ctypes.c_int,
                                              ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]),
    "tvspec_rof_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int, ctypes.c_int,
                                       ctypes.c_double, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                       ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p]),
    "tvspec_chambolle_iterate": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_void_p]),
    "tvspec_decompose_noalloc": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                                ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                                ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                                ctypes.c_void_p]),
    "tvspec_tile_count": (ctypes.c_int, []),
    "tvspec_tile_info": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]),
    "tvspec_plan_stats": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(Stats)]),
    "tvspec_status_str": (ctypes.c_char_p, [ctypes.c_int]),
    "tvspec_last_error": (ctypes.c_char_p, []),
    "tvspec_version": (ctypes.c_char_p, []),
}


def build(force: bool = False) -> str:
    return _build.build(force=force)


def load(build_if_missing: bool = True):
    """Load ``libtvspec.so`` (building it first if needed). Raises if it cannot be built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(_build.LIB) or (build_if_missing and not _build.up_to_date()):
                if not build_if_missing:
                    raise RuntimeError(f"{_build.LIB} is missing; run __graft_entry__.build()")
                _build.build()
            lib = ctypes.CDLL(_build.LIB)
            for name, (res, args) in _SIGS.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


def library_path() -> str:
    return _build.LIB


def _check(status: int, where: str):
    if status != OK:
        detail = load().tvspec_last_error()
        raise TvSpecError(status, where, detail.decode() if detail else "")


def tile_shapes() -> list:
    L = load()
    out = []
    for i in range(L.tvspec_tile_count()):
        v, r, w, tb = (ctypes.c_int() for _ in range(4))
        _check(L.tvspec_tile_info(i, ctypes.byref(v), ctypes.byref(r), ctypes.byref(w), ctypes.byref(tb)),
               "tvspec_tile_info")
        out.append({"V": v.value, "R": r.value, "RW": w.value, "TB": tb.value})
    return out


def resident_variants() -> list:
    """Thread layouts of the resident small-image kernel: largest image, threads, CTAs per SM."""
    L = load()
    out = []
    for i in range(L.tvspec_resident_variant_count()):
        h, w, t, m = (ctypes.c_int() for _ in range(4))
        _check(L.tvspec_resident_variant_info(i, ctypes.byref(h), ctypes.byref(w), ctypes.byref(t),
                                              ctypes.byref(m)), "tvspec_resident_variant_info")
        out.append({"max_H": h.value, "max_W": w.value, "threads": t.value, "min_ctas_per_sm": m.value})
    return out


_pinned_ok = None


def _host_empty(shape, dtype) -> np.ndarray:
    """An uninitialised host array (every element is written by the library), page-locked
    through torch's caching host allocator when a CUDA device is present, else plain numpy."""
    global _pinned_ok
    if _pinned_ok is None:
        try:
            import torch

            _pinned_ok = bool(torch.cuda.is_available())
        except Exception:
            _pinned_ok = False
    if _pinned_ok:
        import torch

        tdt = {np.dtype(np.float32): torch.float32, np.dtype(np.float64): torch.float64}[np.dtype(dtype)]
        return torch.empty(tuple(shape), dtype=tdt, pin_memory=True).numpy()
    return np.empty(shape, dtype)


def _is_torch_cuda(x) -> bool:
    return hasattr(x, "is_cuda") and bool(getattr(x, "is_cuda"))


def _stream_ptr(stream) -> int:
    """cudaStream_t of a torch stream (None: torch's current stream).

    torch's default stream is the legacy NULL stream, whose handle is 0; the C ABI reads a NULL
    stream as "the plan's own stream", so it is passed as cudaStreamLegacy (handle 1) instead.
    """
    if stream is None:
        import torch

        stream = torch.cuda.current_stream()
    ptr = int(getattr(stream, "cuda_stream", stream))
    return ptr if ptr != 0 else 1


class Result(dict):
    """bands (n_bands, H, W), residual (H, W), S (K-1,), optional u (K+1, H, W)."""


class Plan:
    """A tvspec plan bound to one CUDA device."""

    def __init__(self, device: int = 0, **cfg):
        L = load()
        c = Config()
        L.tvspec_config_init(ctypes.byref(c))
        for k, v in cfg.items():
            if not hasattr(c, k):
                raise TypeError(f"unknown config field {k}")
            if k == "tune_cache" and isinstance(v, str):
                v = v.encode()
            setattr(c, k, v)
        self.config = c
        h = ctypes.c_void_p()
        _check(L.tvspec_plan_create(ctypes.byref(c), int(device), ctypes.byref(h)), "tvspec_plan_create")
        self._h = h
        self._lib = L
        self._keep = {}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.tvspec_plan_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- request marshalling -----------------------------------------------------------------
    @staticmethod
    def _edges(edges) -> np.ndarray:
        return np.ascontiguousarray(np.asarray(edges, dtype=np.float64))

    @staticmethod
    def _filters(filters, K):
        """filters: list of (H_values, h_r), H_values[k-1] = H(t_k) for k = 1..K-1."""
        nf = len(filters) if filters else 0
        if nf == 0:
            return 0, None, None
        fH = np.ascontiguousarray(np.stack([np.asarray(h, np.float64).reshape(max(K - 1, 0))
                                            for h, _ in filters]))
        fr = np.ascontiguousarray(np.asarray([float(r) for _, r in filters], np.float64))
        return nf, fH, fr

    @staticmethod
    def _out_specs(nb, H, W, K, trace, nf, parseval):
        """(name, shape, is_float64) of every output array of one request."""
        specs = [("bands", (nb, H, W), False), ("residual", (H, W), False), ("S", (max(K - 1, 0),), True)]
        if trace:
            specs.append(("u", (K + 1, H, W), True))
        if nf:
            specs.append(("filtered", (nf, H, W), False))
        if parseval:
            specs.append(("S_parseval", (max(K - 1, 1),), True))
        return specs

    @staticmethod
    def _alloc_outputs(spec_lists, device):
        """Results for several requests carved out of one float32 and one float64 buffer (on
        `device`, or page-locked host memory when device is None); views start 256-byte
        aligned."""
        import math as _m

        tot = [0, 0]
        offs = []
        for specs in spec_lists:
            o = []
            for name, shape, f64 in specs:
                al = 32 if f64 else 64
                tot[f64] = (tot[f64] + al - 1) // al * al
                o.append(tot[f64])
                tot[f64] += int(_m.prod(shape))
            offs.append(o)
        if device is not None:
            import torch

            bufs = [torch.empty((max(tot[0], 1),), dtype=torch.float32, device=device),
                    torch.empty((max(tot[1], 1),), dtype=torch.float64, device=device)]
        else:
            bufs = [_host_empty((max(tot[0], 1),), np.float32), _host_empty((max(tot[1], 1),), np.float64)]
        results = []
        for specs, o in zip(spec_lists, offs):
            res = Result()
            for (name, shape, f64), start in zip(specs, o):
                n = int(_m.prod(shape))
                res[name] = bufs[f64][start:start + n].reshape(shape)
            results.append(res)
        return results

    def _make_request(self, f, dt, K, n_inner, edges, trace, keep, filters=None, parseval=False, out=None):
        e = self._edges(edges)
        keep.append(e)
        nb = len(e) - 1
        nf, fH, fr = self._filters(filters, K)
        keep.extend([fH, fr])
        if _is_torch_cuda(f):
            import torch

            f = f.contiguous()
            if f.dtype != torch.float32 or f.dim() != 2:
                raise TypeError("f must be a 2-D float32 CUDA tensor")
            H, W = f.shape
            if out is None:
                out = self._alloc_outputs([self._out_specs(nb, H, W, K, trace, nf, parseval)], f.device)[0]
            ptr = lambda t: t.data_ptr()
            kind = MEM_DEVICE
        else:
            f = np.ascontiguousarray(np.asarray(f, dtype=np.float32))
            if f.ndim != 2:
                raise TypeError("f must be 2-D")
            H, W = f.shape
            # outputs in page-locked memory: the device-to-host copies run at full speed
            if out is None:
                out = self._alloc_outputs([self._out_specs(nb, H, W, K, trace, nf, parseval)], None)[0]
            ptr = lambda a: a.ctypes.data
            kind = MEM_HOST
        keep.append(f)
        r = Request(f=ptr(f), H=H, W=W, dt=float(dt), K=int(K), n_inner=int(n_inner),
                    band_edges=e.ctypes.data, n_edges=len(e), bands=ptr(out["bands"]),
                    residual=ptr(out["residual"]), S=ptr(out["S"]) if K > 1 else ptr(out["residual"]),
                    u_trace=ptr(out["u"]) if trace else None, mem_kind=kind, n_filters=nf,
                    filter_H=fH.ctypes.data if nf else None,
                    filter_residual=fr.ctypes.data if nf else None,
                    filtered=ptr(out["filtered"]) if nf else None,
                    S_parseval=ptr(out["S_parseval"]) if parseval else None)
        return r, out, kind

    def decompose(self, f, dt: float, K: int, n_inner: int, edges, trace: bool = False, stream=None,
                  filters=None, parseval: bool = False):
        """Decompose one image; returns a Result (numpy for host input, torch for CUDA input).

        ``filters``: optional list of (H_values, h_r) spectral filters (Eq. filteredTVtrafo);
        the Result then holds ``filtered`` ((n_filters, H, W)). ``parseval`` adds ``S_parseval``
        ((K-1,), the Parseval-type spectrum <phi_k, f>).
        """
        keep = []
        r, out, kind = self._make_request(f, dt, K, n_inner, edges, trace, keep, filters, parseval)
        st = _stream_ptr(stream) if kind == MEM_DEVICE else None
        _check(self._lib.tvspec_decompose_ex(self._h, ctypes.byref(r), st), "tvspec_decompose_ex")
        return out

    def decompose_raw(self, f_ptr, H, W, dt, K, n_inner, edges, bands_ptr, residual_ptr, S_ptr,
                      mem_kind, stream=0):
        """The plain C entry with caller-owned buffers (pointers as integers)."""
        e = self._edges(edges)
        _check(self._lib.tvspec_decompose(self._h, f_ptr, H, W, float(dt), K, n_inner, e.ctypes.data,
                                          len(e), bands_ptr, residual_ptr, S_ptr, mem_kind, stream),
               "tvspec_decompose")

    def decompose_batch(self, jobs, trace: bool = False, stream=None, parseval: bool = False):
        """jobs: iterable of (f, dt, K, n_inner, edges[, filters]). Returns a list of Results."""
        keep = []
        reqs, outs, kinds = [], [], set()
        jobs = list(jobs)
        # all outputs of the batch carved out of one buffer per element type
        specs = []
        dev = None
        for job in jobs:
            f, K, edges = job[0], int(job[2]), job[4]
            flt = job[5] if len(job) > 5 else None
            specs.append(self._out_specs(len(edges) - 1, f.shape[0], f.shape[1], K, trace,
                                         len(flt) if flt else 0, parseval))
            if _is_torch_cuda(f):
                dev = f.device
        pre = self._alloc_outputs(specs, dev) if jobs else []
        for job, o_pre in zip(jobs, pre):
            f, dt, K, n_inner, edges = job[:5]
            r, o, k = self._make_request(f, dt, K, n_inner, edges, trace, keep,
                                         job[5] if len(job) > 5 else None, parseval, out=o_pre)
            reqs.append(r)
            outs.append(o)
            kinds.add(k)
        if len(kinds) != 1:
            raise TypeError("all images of a batch must be host arrays or all CUDA tensors")
        arr = (Request * len(reqs))(*reqs)
        st = _stream_ptr(stream) if MEM_DEVICE in kinds else None
        _check(self._lib.tvspec_decompose_batch(self._h, len(reqs), arr, st), "tvspec_decompose_batch")
        return outs

    # ---- checkpoint / resume -------------------------------------------------------------------
    def checkpoint_bytes(self, f, dt: float, K: int, n_inner: int, edges, trace: bool = False,
                         filters=None, parseval: bool = False) -> int:
        """Bytes of a decomposition's saved state under this plan's configuration."""
        keep = []
        r, _, _ = self._make_request(f, dt, K, n_inner, edges, trace, keep, filters, parseval)
        n = int(self._lib.tvspec_checkpoint_bytes(self._h, ctypes.byref(r)))
        if n == 0:
            raise TvSpecError(EINVAL, "tvspec_checkpoint_bytes", "invalid request")
        return n

    def decompose_steps(self, f, dt: float, K: int, n_inner: int, edges, k_begin: int, k_end: int,
                        state=None, trace: bool = False, filters=None, parseval: bool = False):
        """ROF steps [k_begin, k_end) of one decomposition. From k_begin > 0 it resumes from
        ``state`` (a uint8 array returned by an earlier call that stopped at k_begin). Returns
        (Result, None) when k_end == K, else (None, state after step k_end - 1)."""
        keep = []
        r, out, kind = self._make_request(f, dt, K, n_inner, edges, trace, keep, filters, parseval)
        state_out = None
        if k_end < K:
            n = int(self._lib.tvspec_checkpoint_bytes(self._h, ctypes.byref(r)))
            if n == 0:
                raise TvSpecError(EINVAL, "tvspec_checkpoint_bytes", "invalid request")
            state_out = np.empty(n, np.uint8)
        sin = None
        if state is not None:
            state = np.ascontiguousarray(state, dtype=np.uint8)
            sin = state.ctypes.data
        if kind == MEM_DEVICE:
            import torch

            torch.cuda.synchronize()  # the call runs on the plan's own stream
        _check(self._lib.tvspec_decompose_steps(self._h, ctypes.byref(r), int(k_begin), int(k_end), sin,
                                                None if state_out is None else state_out.ctypes.data),
               "tvspec_decompose_steps")
        return (out, None) if k_end == K else (None, state_out)

    # ---- training-data generation (Sec. 4.1) ---------------------------------------------------
    def training_set(self, sources, crops, size: int, standardize: int, dt: float, K: int, n_inner: int,
                     edges, mean_std=(0.0, 1.0), want_crops: bool = True, want_stats: bool = True,
                     stream=None) -> Result:
        """Crops (src, y, x, scale) of the sources, standardised (0 none, 1 over the crops,
        2 per crop, 3 by mean_std) and decomposed. Host (numpy) or CUDA (torch) sources; the
        Result holds ``crops`` (n, size, size), ``bands`` (n, n_bands, size, size),
        ``residual`` (n, size, size), ``S`` (n, K-1) and ``stats`` (host float64)."""
        e = self._edges(edges)
        nb = len(e) - 1
        n = len(crops)
        device = all(_is_torch_cuda(x) for x in sources) and len(sources) > 0
        if device:
            import torch

            srcs = [x.contiguous() for x in sources]
            for x in srcs:
                if x.dtype != torch.float32 or x.dim() != 2:
                    raise TypeError("sources must be 2-D float32 tensors")
            dev = srcs[0].device
            mk = lambda *shape, dt=torch.float32: torch.empty(shape, dtype=dt, device=dev)
            out = Result(bands=mk(n, nb, size, size), residual=mk(n, size, size),
                         S=mk(n, max(K - 1, 0), dt=torch.float64))
            if want_crops:
                out["crops"] = mk(n, size, size)
            ptr = lambda t: t.data_ptr()
            kind = MEM_DEVICE
        else:
            srcs = [np.ascontiguousarray(np.asarray(x, np.float32)) for x in sources]
            if any(x.ndim != 2 for x in srcs):
                raise TypeError("sources must be 2-D")
            out = Result(bands=np.zeros((n, nb, size, size), np.float32), residual=np.zeros((n, size, size), np.float32),
                         S=np.zeros((n, max(K - 1, 0)), np.float64))
            if want_crops:
                out["crops"] = np.zeros((n, size, size), np.float32)
            ptr = lambda a: a.ctypes.data
            kind = MEM_HOST
        ptrs = (ctypes.c_void_p * len(srcs))(*[ptr(x) for x in srcs])
        hs = np.ascontiguousarray([x.shape[0] for x in srcs], np.int32)
        ws = np.ascontiguousarray([x.shape[1] for x in srcs], np.int32)
        ca = (Crop * max(n, 1))(*[Crop(int(c[0]), int(c[1]), int(c[2]), int(c[3])) for c in crops])
        stats = np.zeros(max(2, 2 * n) if standardize == 2 else 2, np.float64)
        r = TrainingRequest(n_sources=len(srcs), sources=ctypes.cast(ptrs, ctypes.c_void_p),
                            source_H=hs.ctypes.data, source_W=ws.ctypes.data, n_crops=n,
                            crops=ctypes.cast(ca, ctypes.c_void_p), size=int(size), standardize=int(standardize),
                            dt=float(dt), K=int(K), n_inner=int(n_inner), band_edges=e.ctypes.data,
                            n_edges=len(e), crops_out=ptr(out["crops"]) if want_crops else None,
                            bands=ptr(out["bands"]), residual=ptr(out["residual"]),
                            S=ptr(out["S"]) if K > 1 else ptr(out["residual"]),
                            stats=stats.ctypes.data if want_stats else None, mem_kind=kind)
        r.mean_std[0], r.mean_std[1] = float(mean_std[0]), float(mean_std[1])
        st = _stream_ptr(stream) if kind == MEM_DEVICE else None
        _check(self._lib.tvspec_training_set(self._h, ctypes.byref(r), st), "tvspec_training_set")
        if want_stats:
            out["stats"] = stats[:2 * n] if standardize == 2 else stats[:2]
        return out

    # ---- serving -------------------------------------------------------------------------------
    def submit(self, f, dt, K, n_inner, edges, trace: bool = False, filters=None, parseval: bool = False):
        """Queue one host-memory request; returns (ticket, Result). Keep the Result alive."""
        keep = []
        r, out, kind = self._make_request(f, dt, K, n_inner, edges, trace, keep, filters, parseval)
        if kind != MEM_HOST:
            raise TypeError("serving takes host (numpy) images")
        t = ctypes.c_uint64()
        _check(self._lib.tvspec_submit(self._h, ctypes.byref(r), ctypes.byref(t)), "tvspec_submit")
        self._keep[t.value] = (keep, out)
        return t.value, out

    def poll(self, ticket: int) -> int:
        s = int(self._lib.tvspec_poll(self._h, ctypes.c_uint64(ticket)))
        if s != ENOTREADY:
            self._keep.pop(ticket, None)  # finished: the library no longer writes its buffers
        return s

    def wait(self, ticket: int, timeout_ms: int = -1) -> int:
        s = int(self._lib.tvspec_wait(self._h, ctypes.c_uint64(ticket), int(timeout_ms)))
        if s not in (ENOTREADY, ETIMEOUT):
            self._keep.pop(ticket, None)
        return s

    def cancel(self, ticket: int) -> int:
        return int(self._lib.tvspec_cancel(self._h, ctypes.c_uint64(ticket)))

    def serving_stats(self, reset: bool = False):
        n = ctypes.c_uint64()
        p50 = ctypes.c_double()
        p99 = ctypes.c_double()
        _check(self._lib.tvspec_serving_stats(self._h, 1 if reset else 0, ctypes.byref(n), ctypes.byref(p50),
                                              ctypes.byref(p99)), "tvspec_serving_stats")
        return {"count": n.value, "p50_ms": p50.value, "p99_ms": p99.value}

    # ---- lower-level entry points ------------------------------------------------------------
    def rof_step(self, g, lam: float, n_iter: int, p1=None, p2=None, stream=None):
        """One ROF step by n_iter dual iterations; returns (u, p1, p2) (float32)."""
        if _is_torch_cuda(g):
            import torch

            g = g.contiguous().float()
            p1 = torch.zeros_like(g) if p1 is None else p1.contiguous().float().clone()
            p2 = torch.zeros_like(g) if p2 is None else p2.contiguous().float().clone()
            u = torch.empty_like(g)
            ptr = lambda t: t.data_ptr()
            kind, st = MEM_DEVICE, _stream_ptr(stream)
        else:
            g = np.ascontiguousarray(np.asarray(g, np.float32))
            p1 = np.zeros_like(g) if p1 is None else np.array(p1, np.float32, copy=True, order="C")
            p2 = np.zeros_like(g) if p2 is None else np.array(p2, np.float32, copy=True, order="C")
            u = np.empty_like(g)
            ptr = lambda a: a.ctypes.data
            kind, st = MEM_HOST, None
        H, W = g.shape
        _check(self._lib.tvspec_rof_step(self._h, ptr(g), H, W, float(lam), int(n_iter), ptr(p1), ptr(p2),
                                         ptr(u), kind, st), "tvspec_rof_step")
        return u, p1, p2

    def rof_solve(self, g, lam: float, solver="chambolle", max_iter: int = 1000, gap_tol: float = 0.0,
                  check_every: int = 50, p_in=None, tau: float = 0.25, sigma: float = 0.5, gamma: float = 0.7,
                  stream=None) -> dict:
        """One ROF step by the chosen solver ("chambolle", "fgp", "pdhg"); stops at the first
        check with duality gap <= gap_tol (if > 0). Returns u, p1, p2, iterations, gap."""
        sv = SOLVERS[solver] if isinstance(solver, str) else int(solver)
        if _is_torch_cuda(g):
            import torch

            g = g.contiguous().float()
            u = torch.empty_like(g)
            p1 = torch.empty_like(g)
            p2 = torch.empty_like(g)
            pin = None if p_in is None else (p_in[0].contiguous().float(), p_in[1].contiguous().float())
            ptr = lambda t: t.data_ptr()
            kind, st = MEM_DEVICE, _stream_ptr(stream)
        else:
            g = np.ascontiguousarray(np.asarray(g, np.float32))
            u, p1, p2 = np.empty_like(g), np.empty_like(g), np.empty_like(g)
            pin = None if p_in is None else tuple(np.ascontiguousarray(np.asarray(x, np.float32)) for x in p_in)
            ptr = lambda a: a.ctypes.data
            kind, st = MEM_HOST, None
        H, W = g.shape
        r = RofRequest(g=ptr(g), H=H, W=W, lam=float(lam), solver=sv, max_iter=int(max_iter),
                       gap_tol=float(gap_tol), check_every=int(check_every), pdhg_tau=float(tau),
                       pdhg_sigma=float(sigma), pdhg_gamma=float(gamma),
                       p1_in=ptr(pin[0]) if pin else None, p2_in=ptr(pin[1]) if pin else None,
                       u=ptr(u), p1=ptr(p1), p2=ptr(p2), mem_kind=kind)
        _check(self._lib.tvspec_rof_solve(self._h, ctypes.byref(r), st), "tvspec_rof_solve")
        return {"u": u, "p1": p1, "p2": p2, "iterations": r.iterations, "gap": r.gap}

    def chambolle_iterate(self, gl, p1, p2, H: int, W: int, pitch: int, n_iter: int, stream=None):
        """Dual iterations on pitched CUDA tensors (gl, p1, p2 of H*pitch float32), in place."""
        _check(self._lib.tvspec_chambolle_iterate(self._h, gl.data_ptr(), p1.data_ptr(), p2.data_ptr(), H, W,
                                                  pitch, int(n_iter), _stream_ptr(stream)),
               "tvspec_chambolle_iterate")

    def stats(self) -> dict:
        s = Stats()
        _check(self._lib.tvspec_plan_stats(self._h, ctypes.byref(s)), "tvspec_plan_stats")
        return {k: getattr(s, k) for k, _ in Stats._fields_}


def decompose_noalloc(f, dt: float, K: int, n_inner: int, edges, stream=None, out=None) -> Result:
    """The decomposition through tvspec_decompose_noalloc, which allocates no device memory.

    For callers that may not call cudaMalloc where they run (see include/tvspec.h). ``f`` is a
    2-D float32 CUDA tensor; the call runs with ``f``'s device current. The outputs are
    allocated here by torch, outside the entry point, as such a caller would pre-allocate them,
    unless ``out`` gives them (a Result / dict with float32 ``bands`` (n_edges-1, H, W) and
    ``residual`` (H, W) and float64 ``S`` (at least max(K-1, 1)) on ``f``'s device), in which
    case nothing is allocated here either. Images up to about 1.1 megapixels.
    """
    import torch

    L = load()
    if not isinstance(f, torch.Tensor) or f.dtype != torch.float32 or f.dim() != 2 or not f.is_cuda:
        raise TypeError("f must be a 2-D float32 CUDA tensor")
    if not f.is_contiguous():
        raise TypeError("f must be contiguous")
    e = np.ascontiguousarray(np.asarray(edges, dtype=np.float64))
    H, W = f.shape
    with torch.cuda.device(f.device):
        if out is None:
            out = Result(bands=torch.empty((len(e) - 1, H, W), dtype=torch.float32, device=f.device),
                         residual=torch.empty((H, W), dtype=torch.float32, device=f.device),
                         S=torch.empty((max(K - 1, 1),), dtype=torch.float64, device=f.device))
        else:
            b, r, S = out["bands"], out["residual"], out["S"]
            ok = (b.dtype == torch.float32 and tuple(b.shape) == (len(e) - 1, H, W) and b.is_contiguous()
                  and r.dtype == torch.float32 and tuple(r.shape) == (H, W) and r.is_contiguous()
                  and S.dtype == torch.float64 and S.dim() == 1 and S.numel() >= max(K - 1, 1)
                  and S.is_contiguous() and all(t.device == f.device for t in (b, r, S)))
            if not ok:
                raise TypeError("out: bands (n_edges-1, H, W) float32, residual (H, W) float32 and "
                                "S (>= K-1,) float64, contiguous, on f's device")
            out = Result(bands=b, residual=r, S=S)
        _check(L.tvspec_decompose_noalloc(f.data_ptr(), H, W, float(dt), int(K), int(n_inner), e.ctypes.data,
                                          len(e), out["bands"].data_ptr(), out["residual"].data_ptr(),
                                          out["S"].data_ptr(), _stream_ptr(stream)), "tvspec_decompose_noalloc")
    out["S"] = out["S"][: max(K - 1, 0)]
    return out


def validate(f_shape, dt, K, n_inner, edges, f=None, mem_kind=MEM_HOST, filters=None) -> int:
    """Host-only argument check through tvspec_validate (no GPU needed); returns the status."""
    L = load()
    H, W = f_shape
    e = np.ascontiguousarray(np.asarray(edges, np.float64))
    fa = np.zeros((H, W), np.float32) if f is None else np.ascontiguousarray(np.asarray(f, np.float32))
    dummy = np.zeros(max(1, (len(e) - 1) * H * W), np.float32)
    S = np.zeros(max(1, K), np.float64)
    nf = len(filters) if filters else 0
    fH = np.ascontiguousarray(np.concatenate([np.asarray(h, np.float64).ravel() for h, _ in filters])) if nf else None
    fr = np.ascontiguousarray(np.asarray([float(r) for _, r in filters], np.float64)) if nf else None
    fout = np.zeros(max(1, nf * H * W), np.float32)
    r = Request(f=fa.ctypes.data, H=H, W=W, dt=float(dt), K=int(K), n_inner=int(n_inner),
                band_edges=e.ctypes.data, n_edges=len(e), bands=dummy.ctypes.data, residual=dummy.ctypes.data,
                S=S.ctypes.data, u_trace=None, mem_kind=mem_kind, n_filters=nf,
                filter_H=fH.ctypes.data if nf else None, filter_residual=fr.ctypes.data if nf else None,
                filtered=fout.ctypes.data if nf else None)
    return int(L.tvspec_validate(ctypes.byref(r)))


def pitch_for(W: int) -> int:
    return int(math.ceil(W / 4) * 4)
