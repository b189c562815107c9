"""Parity bars between the CUDA path and the FP64 oracle.

The bars are those the decomposition's accuracy target states:
  u(t_k)          L_inf <= 1e-4 max|f|
  bands           L_inf <= 1e-3 max|f|   and   relative L2 <= 1e-4 (over the stacked bands)
  reconstruction  L_inf(sum bands + residual - f) <= 1e-5 max|f|
S(t) and the residual have no separate bar; they are reported and bounded loosely here by
the same derivation (S is an L1 norm of phi; the residual is u_{K-1} - T D_{K-1}).
"""
import numpy as np

U_INF = 1e-4
BAND_INF = 1e-3
BAND_REL_L2 = 1e-4
RECON_INF = 1e-5


def parity_metrics(gpu: dict, ref: dict, f) -> dict:
    f = np.asarray(f, np.float64)
    mf = max(float(np.abs(f).max()), 1e-30)
    gb = np.asarray(gpu["bands"], np.float64)
    rb = np.asarray(ref["bands"], np.float64)
    m = {
        "band_inf": float(np.abs(gb - rb).max()) / mf,
        "band_rel_l2": float(np.linalg.norm(gb - rb) / max(np.linalg.norm(rb), 1e-300)),
        "recon_inf": float(np.abs(gb.sum(0) + np.asarray(gpu["residual"], np.float64) - f).max()) / mf,
        "residual_inf": float(np.abs(np.asarray(gpu["residual"], np.float64) - ref["residual"]).max()) / mf,
        "S_rel": float(np.abs(np.asarray(gpu["S"]) - ref["S"]).max() / max(np.abs(ref["S"]).max(), 1e-300))
        if len(ref["S"]) else 0.0,
    }
    if "u" in gpu and "u" in ref:
        m["u_inf"] = float(np.abs(np.asarray(gpu["u"]) - ref["u"]).max()) / mf
    return m


def assert_parity(gpu: dict, ref: dict, f, label: str = "") -> dict:
    m = parity_metrics(gpu, ref, f)
    msg = f"{label} {m}"
    if "u_inf" in m:
        assert m["u_inf"] <= U_INF, msg
    assert m["band_inf"] <= BAND_INF, msg
    if np.linalg.norm(ref["bands"]) > 0:
        assert m["band_rel_l2"] <= BAND_REL_L2, msg
    assert m["recon_inf"] <= RECON_INF, msg
    assert m["residual_inf"] <= BAND_INF, msg
    assert m["S_rel"] <= 1e-3, msg
    return m
