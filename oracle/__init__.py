"""FP64 CPU oracle of the classical spectral TV decomposition (arXiv 2006.10004, Sec. 2).

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs
of ``bench.py`` may import this package. The CUDA product path
(``paper_2006_10004_gb300``) never imports it, and the two share no code.

The arithmetic lives in ``tvspec_oracle.c`` (plain loops, double precision, compiled with
``-ffp-contract=off``); this module only compiles it with gcc and marshals numpy arrays.

Functions and the passages they follow:

* ``grad`` / ``div``  -- forward differences with Neumann boundary and the negative adjoint
  (the discrete form of J_TV, Eq. TV; Chambolle 2004 as cited in Sec. 4.3).
* ``chambolle``      -- fixed-iteration Chambolle projection for one ROF step (Eq. ROF).
* ``rof_gap``        -- duality gap of a ROF step (diagnostic).
* ``fgp`` / ``pdhg`` / ``rof_gap_pair`` -- other inner solvers of the ROF step (Beck-Teboulle's
  fast gradient projection on the same dual; Chambolle-Pock's primal-dual method, the family
  of the GPU toolbox Sec. 4.3 times) and the gap of a primal-dual pair.
* ``decompose``      -- TV flow by implicit Euler (Eq. TVflow, Eq. ROF), phi (Eq. TVtrafo),
  S(t) (Sec. 2.1), bands (Eq. spectral_bands), residual (Eq. finite_inverse_trafo) and
  filtered images (Eq. filteredTVtrafo substituted into Eq. finite_inverse_trafo).
* ``crop`` / ``standardize`` / ``training_set`` -- the ground-truth generation of Sec. 4.1:
  fixed-size crops (some from twice-as-large windows downsampled by 2), standardisation to
  zero mean and unit standard deviation, then ``decompose`` of every crop.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tvspec_oracle.c")
_LIBDIR = os.path.join(_HERE, "_lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_handle = None

_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, OpenMP, no FP contraction). Returns the .so path."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if (not force and os.path.exists(_LIB)
            and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-fno-fast-math", "-std=c11", _SRC, "-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _lib():
    global _handle
    with _lock:
        if _handle is None:
            build()
            h = ctypes.CDLL(_LIB)
            h.orc_grad.argtypes = [_dp, ctypes.c_int, ctypes.c_int, _dp, _dp]
            h.orc_grad.restype = None
            h.orc_div.argtypes = [_dp, _dp, ctypes.c_int, ctypes.c_int, _dp]
            h.orc_div.restype = None
            h.orc_chambolle.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
            h.orc_chambolle.restype = ctypes.c_int
            h.orc_rof_gap.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                      _dp, _dp]
            h.orc_rof_gap.restype = ctypes.c_double
            h.orc_band_of.argtypes = [ctypes.c_double, _dp, ctypes.c_int]
            h.orc_band_of.restype = ctypes.c_int
            h.orc_decompose.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, ctypes.c_int, ctypes.c_double,
                                        ctypes.c_int, _dp, ctypes.c_int, _dp, _dp, _dp, _dp]
            h.orc_decompose.restype = ctypes.c_int
            h.orc_decompose_filtered.argtypes = h.orc_decompose.argtypes + [ctypes.c_int, _dp, _dp, _dp]
            h.orc_decompose_filtered.restype = ctypes.c_int
            h.orc_decompose_full.argtypes = h.orc_decompose_filtered.argtypes + [_dp]
            h.orc_decompose_full.restype = ctypes.c_int
            h.orc_crop.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_int, ctypes.c_int, _dp]
            h.orc_crop.restype = ctypes.c_int
            h.orc_standardize.argtypes = [_dp, ctypes.c_int, ctypes.c_size_t, ctypes.c_int, _dp, _dp]
            h.orc_standardize.restype = ctypes.c_int
            h.orc_fgp.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int, _dp, _dp, _dp]
            h.orc_fgp.restype = ctypes.c_int
            h.orc_pdhg.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                   ctypes.c_double, ctypes.c_double, ctypes.c_double, _dp, _dp, _dp]
            h.orc_pdhg.restype = ctypes.c_int
            h.orc_rof_gap_pair.argtypes = [_dp, ctypes.c_int, ctypes.c_int, ctypes.c_double, _dp, _dp, _dp]
            h.orc_rof_gap_pair.restype = ctypes.c_double
            h.orc_set_threads.argtypes = [ctypes.c_int]
            h.orc_set_threads.restype = ctypes.c_int
            h.orc_max_threads.argtypes = []
            h.orc_max_threads.restype = ctypes.c_int
            _handle = h
        return _handle


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_dp)


def set_threads(n: int) -> int:
    """OpenMP threads of later calls (n >= 1); returns the new count."""
    return int(_lib().orc_set_threads(int(n)))


def max_threads() -> int:
    """OpenMP threads the oracle uses (set OMP_NUM_THREADS before the first call)."""
    return int(_lib().orc_max_threads())


def grad(u):
    """Forward-difference gradient (grad^1 along rows, grad^2 along columns), Neumann."""
    u = _f64(u)
    H, W = u.shape
    g1 = np.empty_like(u)
    g2 = np.empty_like(u)
    _lib().orc_grad(_ptr(u), H, W, _ptr(g1), _ptr(g2))
    return g1, g2


def div(p1, p2):
    """Discrete divergence = -grad^T."""
    p1 = _f64(p1)
    p2 = _f64(p2)
    H, W = p1.shape
    d = np.empty_like(p1)
    _lib().orc_div(_ptr(p1), _ptr(p2), H, W, _ptr(d))
    return d


def chambolle(g, lam: float, n_iter: int, tau: float = 0.125, p1=None, p2=None):
    """``n_iter`` Chambolle iterations of the ROF step with weight ``lam`` (Eq. ROF).

    Returns ``(u, p1, p2)`` with ``u = g - lam div p``. ``p1``/``p2`` default to zero.
    """
    g = _f64(g)
    H, W = g.shape
    p1 = np.zeros_like(g) if p1 is None else _f64(p1).copy()
    p2 = np.zeros_like(g) if p2 is None else _f64(p2).copy()
    u = np.empty_like(g)
    rc = _lib().orc_chambolle(_ptr(g), H, W, float(lam), float(tau), int(n_iter),
                              _ptr(p1), _ptr(p2), _ptr(u))
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    return u, p1, p2


def fgp(g, lam: float, n_iter: int, p1=None, p2=None):
    """``n_iter`` fast-gradient-projection iterations on the ROF dual; returns (u, p1, p2)."""
    g = _f64(g)
    H, W = g.shape
    p1 = np.zeros_like(g) if p1 is None else _f64(p1).copy()
    p2 = np.zeros_like(g) if p2 is None else _f64(p2).copy()
    u = np.empty_like(g)
    if _lib().orc_fgp(_ptr(g), H, W, float(lam), int(n_iter), _ptr(p1), _ptr(p2), _ptr(u)) != 0:
        raise MemoryError("oracle: allocation failed")
    return u, p1, p2


def pdhg(g, lam: float, n_iter: int, tau: float = 0.25, sigma: float = 0.5, gamma: float = 0.7,
         u=None, p1=None, p2=None):
    """``n_iter`` primal-dual iterations of the ROF step (gamma > 0: accelerated); returns
    (u, p1, p2) with p the dual in Chambolle's scaling (|p| <= 1)."""
    g = _f64(g)
    H, W = g.shape
    u = g.copy() if u is None else _f64(u).copy()
    p1 = np.zeros_like(g) if p1 is None else _f64(p1).copy()
    p2 = np.zeros_like(g) if p2 is None else _f64(p2).copy()
    if _lib().orc_pdhg(_ptr(g), H, W, float(lam), int(n_iter), float(tau), float(sigma), float(gamma),
                       _ptr(u), _ptr(p1), _ptr(p2)) != 0:
        raise MemoryError("oracle: allocation failed")
    return u, p1, p2


def rof_gap_pair(g, lam: float, u, p1, p2) -> float:
    """P(u) - D(p) of the ROF step for a primal-dual pair (|p| <= 1)."""
    g, u, p1, p2 = _f64(g), _f64(u), _f64(p1), _f64(p2)
    H, W = g.shape
    return float(_lib().orc_rof_gap_pair(_ptr(g), H, W, float(lam), _ptr(u), _ptr(p1), _ptr(p2)))


def rof_gap(g, lam: float, p1, p2) -> float:
    """Duality gap P(u) - D(p) of the ROF step at the dual point p (|p| <= 1)."""
    g = _f64(g)
    p1 = _f64(p1)
    p2 = _f64(p2)
    H, W = g.shape
    return float(_lib().orc_rof_gap(_ptr(g), H, W, float(lam), _ptr(p1), _ptr(p2)))


def band_of(t: float, edges) -> int:
    e = _f64(edges)
    return int(_lib().orc_band_of(float(t), _ptr(e), len(e)))


def decompose(f, dt: float, K: int, n_inner: int, edges, tau: float = 0.125,
              warm_start: bool = True, trace: bool = False, filters=None) -> dict:
    """Spectral TV decomposition of ``f`` (H x W).

    Returns a dict with ``bands`` ((n_edges-1, H, W)), ``residual`` ((H, W)), ``S`` ((K-1,)),
    ``S_parseval`` ((K-1,), <phi_k, f>) and, when ``trace`` is set, ``u`` ((K+1, H, W)) holding
    u_0..u_K. All float64.
    ``filters``: optional list of (H_values, h_r) with H_values[k-1] = H(t_k) for k=1..K-1;
    adds ``filtered`` ((n_filters, H, W)) = sum_k H(t_k) phi_k dt + h_r f_r (Eq. filteredTVtrafo).
    """
    f = _f64(f)
    if f.ndim != 2:
        raise ValueError("f must be 2-D")
    H, W = f.shape
    e = _f64(edges)
    nb = len(e) - 1
    bands = np.zeros((nb, H, W))
    residual = np.zeros((H, W))
    S = np.zeros(max(K - 1, 0))
    ut = np.zeros((K + 1, H, W)) if trace else None
    nf = len(filters) if filters else 0
    fH = _f64([np.asarray(h, np.float64).reshape(K - 1) for h, _ in filters]) if nf else np.zeros(1)
    fr = _f64([r for _, r in filters]) if nf else np.zeros(1)
    filtered = np.zeros((max(nf, 1), H, W))
    S_par = np.zeros(max(K - 1, 0))
    rc = _lib().orc_decompose_full(_ptr(f), H, W, float(dt), int(K), int(n_inner), float(tau),
                                   1 if warm_start else 0, _ptr(e), len(e), _ptr(bands),
                                   _ptr(residual), _ptr(S), _ptr(ut) if trace else None,
                                   nf, _ptr(fH), _ptr(fr), _ptr(filtered), _ptr(S_par))
    if rc == -2:
        raise ValueError("oracle: invalid arguments")
    if rc != 0:
        raise MemoryError("oracle: allocation failed")
    out = {"bands": bands, "residual": residual, "S": S, "S_parseval": S_par}
    if nf:
        out["filtered"] = filtered
    if trace:
        out["u"] = ut
    return out


def crop(src, y: int, x: int, size: int, scale: int = 1) -> np.ndarray:
    """The ``scale``-fold block average of the (scale*size)^2 window of ``src`` at (y, x),
    rounded to float32 values (returned as float64)."""
    src = _f64(src)
    sH, sW = src.shape
    out = np.zeros((size, size))
    rc = _lib().orc_crop(_ptr(src), sH, sW, int(y), int(x), int(size), int(scale), _ptr(out))
    if rc != 0:
        raise ValueError("oracle: crop window outside the source image")
    return out


def standardize(x, mode: int, mean_std=None):
    """Standardise images x ((n, H, W)): mode 0 none, 1 over all of x, 2 per image, 3 by the
    given (mean, std). Returns (out, mean_std) with mean_std of length 2 (modes 1, 3) or 2n."""
    x = _f64(x)
    n = x.shape[0]
    npx = int(np.prod(x.shape[1:]))
    ms = np.zeros(max(2, 2 * n))
    if mode == 3:
        ms[0], ms[1] = float(mean_std[0]), float(mean_std[1])
    out = np.zeros_like(x)
    rc = _lib().orc_standardize(_ptr(x), n, npx, int(mode), _ptr(ms), _ptr(out))
    if rc != 0:
        raise ValueError("oracle: bad standardisation mode")
    return out, (ms[:2 * n] if mode == 2 else ms[:2])


def training_set(sources, crops, size: int, standardize_mode: int, dt: float, K: int, n_inner: int,
                 edges, mean_std=None, tau: float = 0.125, warm_start: bool = True) -> dict:
    """Ground-truth generation (Sec. 4.1). ``crops``: list of (src_index, y, x, scale).

    Returns ``crops`` ((n, size, size), standardised), ``mean_std``, ``bands``
    ((n, n_bands, size, size)), ``residual`` ((n, size, size)) and ``S`` ((n, K-1)).
    """
    raw = np.stack([crop(sources[c[0]], c[1], c[2], size, c[3]) for c in crops]) if crops else \
        np.zeros((0, size, size))
    x, ms = standardize(raw, standardize_mode, mean_std)
    nb = len(edges) - 1
    bands = np.zeros((len(crops), nb, size, size))
    residual = np.zeros((len(crops), size, size))
    S = np.zeros((len(crops), max(K - 1, 0)))
    for i in range(len(crops)):
        r = decompose(x[i], dt, K, n_inner, edges, tau=tau, warm_start=warm_start)
        bands[i], residual[i], S[i] = r["bands"], r["residual"], r["S"]
    return {"crops": x, "mean_std": ms, "bands": bands, "residual": residual, "S": S}
