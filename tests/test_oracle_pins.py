"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: a closed form, an invariant
of the method, a textbook special case, an independent solver (``refsolvers``), or a
hand-derived fixture under ``tests/golden``. Together they are chosen so that a plausible
mistake anywhere in the oracle (a dropped term, a wrong sign or index, a transposed operand,
a wrong time index, band boundary or residual formula) fails at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import refsolvers as rs
import synthetic as syn

INF = float("inf")


def _rand(H, W, seed, scale=1.0):
    return np.random.default_rng(seed).normal(size=(H, W)) * scale


# --------------------------------------------------------------------------------------------
# Operators: grad is the forward difference with Neumann boundary, div is exactly -grad^T.
# (J_TV of Eq. TV: sup over |phi| <= 1 of <u, div phi> needs div = -grad^*.)
# --------------------------------------------------------------------------------------------
@pytest.mark.parametrize("H,W", [(5, 7), (1, 6), (6, 1), (1, 1), (2, 2)])
def test_grad_matches_explicit_matrix_and_div_is_negative_transpose(H, W):
    D = rs.grad_matrix(H, W)
    N = H * W
    u = _rand(H, W, 1)
    g1, g2 = oracle.grad(u)
    ref = D @ u.ravel()
    np.testing.assert_allclose(g1.ravel(), ref[:N], rtol=0, atol=1e-14)
    np.testing.assert_allclose(g2.ravel(), ref[N:], rtol=0, atol=1e-14)
    p1 = _rand(H, W, 2)
    p2 = _rand(H, W, 3)
    d = oracle.div(p1, p2)
    np.testing.assert_allclose(d.ravel(), -(D.T @ np.concatenate([p1.ravel(), p2.ravel()])),
                               rtol=0, atol=1e-14)


def test_div_sums_to_zero():
    # Neumann divergence has zero sum, which is why the flow preserves the mean (Eq. inverse_trafo's f-bar)
    d = oracle.div(_rand(9, 13, 4), _rand(9, 13, 5))
    assert abs(d.sum()) < 1e-12


# --------------------------------------------------------------------------------------------
# One ROF step (Eq. ROF) run to convergence equals the exact minimiser.
# --------------------------------------------------------------------------------------------
def test_two_pixel_rof_closed_form(golden_dir):
    data = json.load(open(os.path.join(golden_dir, "two_pixel_rof.json")))
    for case in data["cases"]:
        g = np.array(case["g"], dtype=np.float64).reshape(1, 2)
        u, p1, p2 = oracle.chambolle(g, case["lam"], 20000)
        np.testing.assert_allclose(u.ravel(), case["u"], rtol=0, atol=1e-10)


def _frac_array(rows):
    from fractions import Fraction

    return np.array([[float(Fraction(v)) for v in row] for row in rows], dtype=np.float64)


def test_chambolle_one_and_two_iterations_hand_derived(golden_dir):
    # A fixed iteration count, not the converged step, is what the decomposition computes, so
    # the iterates themselves are pinned: a slip in tau or lambda that keeps the fixed point
    # (tau/2, a denominator 1 + tau |G|^2, w = div p - lam g, ...) changes these values.
    from fractions import Fraction

    data = json.load(open(os.path.join(golden_dir, "chambolle_iterations.json")))
    tau = float(Fraction(data["tau"]))
    assert tau == 0.125
    for case in data["cases"]:
        g = _frac_array(case["g"])
        lam = float(Fraction(case["lam"]))
        prev = None
        for it in case["iterations"]:
            exp_p1, exp_p2, exp_u = (_frac_array(it[k]) for k in ("p1", "p2", "u"))
            u, p1, p2 = oracle.chambolle(g, lam, it["n"], tau=tau)
            for got, exp in ((p1, exp_p1), (p2, exp_p2), (u, exp_u)):
                np.testing.assert_allclose(got, exp, rtol=0, atol=4e-15, err_msg=case["name"])
            # the same iterate reached from the previous one (warm start of the dual)
            if prev is not None:
                u2, q1, q2 = oracle.chambolle(g, lam, it["n"] - prev[0], tau=tau, p1=prev[1], p2=prev[2])
                np.testing.assert_allclose(q1, exp_p1, rtol=0, atol=4e-15)
                np.testing.assert_allclose(q2, exp_p2, rtol=0, atol=4e-15)
                np.testing.assert_allclose(u2, exp_u, rtol=0, atol=4e-15)
            prev = (it["n"], p1, p2)
            # the transposed image gives the transposed iterate with the components swapped
            uT, p1T, p2T = oracle.chambolle(g.T.copy(), lam, it["n"], tau=tau)
            np.testing.assert_allclose(p1T, exp_p2.T, rtol=0, atol=4e-15)
            np.testing.assert_allclose(p2T, exp_p1.T, rtol=0, atol=4e-15)
            np.testing.assert_allclose(uT, exp_u.T, rtol=0, atol=4e-15)


def test_1d_segments_closed_form(golden_dir):
    data = json.load(open(os.path.join(golden_dir, "segments_1d_rof.json")))
    for case in data["cases"]:
        prof = np.concatenate([np.full(m, v, dtype=np.float64)
                               for m, v in zip(case["lengths"], case["values"])])
        expect = np.concatenate([np.full(m, v) for m, v in zip(case["lengths"], case["u_segments"])])
        # as a column profile (varies along i) and as a row profile (varies along j)
        for g in (np.tile(prof[:, None], (1, 3)), np.tile(prof[None, :], (4, 1))):
            u, _, _ = oracle.chambolle(g, case["lam"], 200000)
            ref = np.broadcast_to(expect[:, None] if g.shape[1] == 3 else expect[None, :], g.shape)
            np.testing.assert_allclose(u, ref, rtol=0, atol=1e-10)


@pytest.mark.parametrize("seed,lam", [(0, 0.2), (1, 0.7), (2, 1.5)])
def test_1d_stripe_matches_exact_bvls(seed, lam):
    prof = np.random.default_rng(seed).normal(size=12)
    exact = rs.rof_1d_bvls(prof, lam)
    g = np.tile(prof[:, None], (1, 4))
    u, _, _ = oracle.chambolle(g, lam, 300000)
    np.testing.assert_allclose(u, np.tile(exact[:, None], (1, 4)), rtol=0, atol=1e-9)


@pytest.mark.parametrize("seed,lam", [(3, 0.3), (4, 0.08), (6, 0.15), (5, 1.0)])
def test_8x8_rof_matches_bruteforce_dual_fista(seed, lam):
    g = _rand(8, 8, seed)
    u_bf, gap, _ = rs.rof_fista(g, lam, gap_tol=1e-13)
    assert gap <= 1e-12
    u, p1, p2 = oracle.chambolle(g, lam, 200000)
    gap_o = oracle.rof_gap(g, lam, p1, p2)
    # |u - u*|^2 <= 2 gap for both points, so they are within the sum of the two radii
    bound = math.sqrt(2 * max(gap_o, 0.0)) + math.sqrt(2 * max(gap, 0.0)) + 1e-12
    assert np.linalg.norm(u - u_bf) <= bound
    assert gap_o <= 1e-4  # sublinear convergence for large lam; the bound above is the pin
    if gap_o <= 1e-20:
        np.testing.assert_allclose(u, u_bf, rtol=0, atol=1e-9)


def test_fixed_iterations_gap_decreases():
    # the duality gap of a fixed-iteration step shrinks as the iteration count grows
    g = _rand(16, 16, 7)
    gaps = []
    for n in (10, 100, 1000):
        _, p1, p2 = oracle.chambolle(g, 0.5, n)
        gaps.append(oracle.rof_gap(g, 0.5, p1, p2))
    assert gaps[0] > gaps[1] > gaps[2] >= -1e-12


def test_dual_stays_feasible():
    # the Chambolle update keeps |p_ij| <= 1 (it is a projection-like step)
    g = _rand(20, 24, 8, 5.0)
    _, p1, p2 = oracle.chambolle(g, 0.5, 300)
    assert np.max(np.sqrt(p1 ** 2 + p2 ** 2)) <= 1.0 + 1e-15
    assert np.all(p1[-1, :] == 0.0) and np.all(p2[:, -1] == 0.0)


# --------------------------------------------------------------------------------------------
# The decomposition: constant image, reconstruction, bands, mean, S.
# --------------------------------------------------------------------------------------------
def test_constant_image_gives_zero_spectrum():
    f = np.full((12, 17), 0.7)
    out = oracle.decompose(f, 0.5, 6, 50, syn.DYADIC_EDGES, trace=True)
    assert np.all(out["S"] == 0.0)
    assert np.all(out["bands"] == 0.0)
    assert np.array_equal(out["residual"], f)
    assert np.all(out["u"] == 0.7)


@pytest.mark.parametrize("warm", [True, False])
@pytest.mark.parametrize("dt,K,edges", [(0.5, 12, syn.DYADIC_EDGES),
                                         (0.25, 9, (0.0, 0.6, 1.1, INF)),
                                         (1.0, 2, (0.0, INF))])
def test_reconstruction_identity(warm, dt, K, edges):
    # Eq. finite_inverse_trafo / spectral_bands: f = sum_m b^m + f_r, by telescoping
    f = syn.make_image(23, 31, 5, (2, 8), (0.1, 1.0), 0.05, seed=11).astype(np.float64)
    out = oracle.decompose(f, dt, K, 40, edges, warm_start=warm)
    rec = out["bands"].sum(axis=0) + out["residual"]
    assert np.max(np.abs(rec - f)) <= 1e-12 * np.max(np.abs(f))


def test_band_index_ranges_match_golden(golden_dir):
    data = json.load(open(os.path.join(golden_dir, "band_ranges.json")))
    for case in data["cases"]:
        edges = [INF if e == "inf" else float(e) for e in case["edges"]]
        assert syn.band_index_ranges(case["dt"], case["K"], edges) == case["k_per_band"]
        for m, ks in enumerate(case["k_per_band"]):
            for k in ks:
                assert oracle.band_of(k * case["dt"], edges) == m


def test_bands_equal_closed_form_telescoping():
    # sum_{k=a}^{b} phi_k dt = t_b D_b - t_a D_{a-1} - (u_b - u_a),  D_k = (u_{k+1}-u_k)/dt.
    # Pins phi's formula, its time index, its quadrature weight and band membership at once.
    dt, K = 0.5, 14
    edges = (0.0, 1.0, 2.0, 4.0, INF)
    f = syn.make_image(19, 21, 6, (2, 7), (0.1, 1.0), 0.02, seed=12).astype(np.float64)
    out = oracle.decompose(f, dt, K, 30, edges, trace=True)
    u = out["u"]
    D = lambda k: (u[k + 1] - u[k]) / dt
    for m, ks in enumerate(syn.band_index_ranges(dt, K, edges)):
        if not ks:
            assert np.all(out["bands"][m] == 0.0)
            continue
        a, b = ks[0], ks[-1]
        closed = b * dt * D(b) - a * dt * D(a - 1) - (u[b] - u[a])
        np.testing.assert_allclose(out["bands"][m], closed, rtol=0, atol=1e-11)
    # residual: f_r = u(T) - T u_t(T), T = t_{K-1}, forward difference
    T = (K - 1) * dt
    np.testing.assert_allclose(out["residual"], u[K - 1] - T * D(K - 1), rtol=0, atol=1e-12)
    assert np.array_equal(u[0], f)


def test_mean_preserved_and_phi_zero_sum():
    f = syn.make_image(30, 26, 8, (2, 9), (0.1, 1.0), 0.05, seed=13).astype(np.float64)
    out = oracle.decompose(f, 0.5, 10, 60, syn.DYADIC_EDGES, trace=True)
    for k in range(out["u"].shape[0]):
        assert abs(out["u"][k].sum() - f.sum()) <= 1e-11 * np.abs(f).sum()
    # bands carry no mean; the residual carries f-bar (Eq. inverse_trafo)
    for m in range(out["bands"].shape[0]):
        assert abs(out["bands"][m].sum()) <= 1e-10 * np.abs(f).sum()
    assert abs(out["residual"].mean() - f.mean()) <= 1e-12


def test_S_is_l1_norm_of_phi_and_nonnegative():
    dt, K = 0.5, 8
    f = syn.make_image(16, 16, 4, (2, 6), (0.1, 1.0), 0.02, seed=14).astype(np.float64)
    out = oracle.decompose(f, dt, K, 40, syn.DYADIC_EDGES, trace=True)
    u = out["u"]
    assert out["S"].shape == (K - 1,)
    for k in range(1, K):
        phi = k * dt * (u[k + 1] - 2 * u[k] + u[k - 1]) / dt ** 2
        assert out["S"][k - 1] == pytest.approx(np.abs(phi).sum(), rel=1e-12, abs=1e-15)
    assert np.all(out["S"] >= 0.0)


# --------------------------------------------------------------------------------------------
# Invariances the paper states (Sec. 2.1, Sec. 4.2): one-homogeneity, rotation, translation.
# --------------------------------------------------------------------------------------------
def test_one_homogeneity_exact():
    # (c f, c dt) leaves g/lambda unchanged, so u scales exactly by c = 2 and phi(2t) = phi(t)
    f = syn.make_image(21, 18, 5, (2, 7), (0.1, 1.0), 0.02, seed=15).astype(np.float64)
    edges = (0.0, 1.0, 2.0, 4.0, INF)
    a = oracle.decompose(f, 0.5, 9, 40, edges, trace=True)
    b = oracle.decompose(2.0 * f, 1.0, 9, 40, tuple(2 * e for e in edges), trace=True)
    assert np.array_equal(b["u"], 2.0 * a["u"])
    assert np.array_equal(b["bands"], 2.0 * a["bands"])
    assert np.array_equal(b["residual"], 2.0 * a["residual"])
    assert np.array_equal(b["S"], a["S"])


def test_transpose_equivariance_exact():
    f = syn.make_image(17, 29, 6, (2, 7), (0.1, 1.0), 0.05, seed=16).astype(np.float64)
    a = oracle.decompose(f, 0.5, 8, 50, syn.DYADIC_EDGES)
    b = oracle.decompose(f.T.copy(), 0.5, 8, 50, syn.DYADIC_EDGES)
    assert np.array_equal(b["bands"], np.transpose(a["bands"], (0, 2, 1)))
    assert np.array_equal(b["residual"], a["residual"].T)
    np.testing.assert_allclose(b["S"], a["S"], rtol=1e-13)


@pytest.mark.parametrize("op", ["flipud", "fliplr", "rot90", "rot180", "rot270"])
def test_flips_and_rotations_exact_on_stripes(op):
    # a stripe image makes the problem 1-D, where the forward-difference scheme is mirror
    # symmetric, so flips and 90-degree rotations commute with the decomposition exactly
    prof = syn.make_image(1, 40, 4, (2, 6), (0.1, 1.0), 0.03, seed=17)[0].astype(np.float64)
    f = np.tile(prof[:, None], (1, 11))
    fn = {"flipud": np.flipud, "fliplr": np.fliplr, "rot90": lambda x: np.rot90(x, 1),
          "rot180": lambda x: np.rot90(x, 2), "rot270": lambda x: np.rot90(x, 3)}[op]
    a = oracle.decompose(f, 0.5, 7, 60, syn.DYADIC_EDGES)
    b = oracle.decompose(fn(f).copy(), 0.5, 7, 60, syn.DYADIC_EDGES)
    for m in range(a["bands"].shape[0]):
        np.testing.assert_allclose(b["bands"][m], fn(a["bands"][m]), rtol=0, atol=1e-13)
    np.testing.assert_allclose(b["residual"], fn(a["residual"]), rtol=0, atol=1e-13)
    np.testing.assert_allclose(b["S"], a["S"], rtol=1e-12)


@pytest.mark.parametrize("op", ["flipud", "rot90"])
def test_flips_and_rotations_approximate_in_general(op):
    # forward differences are not mirror symmetric in 2-D: equivariance is approximate
    f = syn.make_image(48, 48, 6, (3, 12), (0.1, 1.0), 0.0, seed=18).astype(np.float64)
    fn = {"flipud": np.flipud, "rot90": lambda x: np.rot90(x, 1)}[op]
    a = oracle.decompose(f, 0.5, 12, 150, syn.DYADIC_EDGES)
    b = oracle.decompose(fn(f).copy(), 0.5, 12, 150, syn.DYADIC_EDGES)
    ba = np.stack([fn(x) for x in a["bands"]])
    rel = np.linalg.norm(b["bands"] - ba) / np.linalg.norm(ba)
    relS = np.abs(b["S"] - a["S"]).sum() / np.abs(a["S"]).sum()
    assert rel < 0.2 and relS < 0.05, (rel, relS)


def test_translation_keeps_disk_spectrum_peak():
    # On a bounded Neumann domain translation equivariance is approximate only (the zero
    # background is not calibrable and feels the borders); the impulse time does not move.
    base = syn.disk_image(40, 40, 6.0, 1.0, cy=16, cx=15).astype(np.float64)
    moved = np.roll(np.roll(base, 5, axis=0), 7, axis=1)
    a = oracle.decompose(base, 0.5, 10, 1000, syn.DYADIC_EDGES)
    b = oracle.decompose(moved, 0.5, 10, 1000, syn.DYADIC_EDGES)
    assert np.argmax(a["S"]) == np.argmax(b["S"])


# --------------------------------------------------------------------------------------------
# Eigenfunctions: a disk gives an impulse of S near t* (Sec. 2.1, Sec. 4.3 disk experiment).
# --------------------------------------------------------------------------------------------
def _disk_tstar(f, h):
    # finite Neumann domain: disk level falls at Per/|D|, background rises at Per/|Omega\D|;
    # they meet at t* = h |D| |Omega\D| / (Per |Omega|)  (continuum limit: r h / 2)
    H, W = f.shape
    Dm = rs.grad_matrix(H, W)
    per = rs.tv_iso(f / h, Dm)
    area = float((f > 0).sum())
    return h * area * (H * W - area) / (per * H * W)


@pytest.mark.parametrize("r,h", [(8.0, 1.0), (6.0, 1.0)])
def test_disk_spectrum_peaks_near_eigenvalue_time(r, h):
    dt, K = 0.1, 70
    f = syn.disk_image(48, 48, r, h).astype(np.float64)
    tstar = _disk_tstar(f, h)
    out = oracle.decompose(f, dt, K, 300, (0.0, INF))
    S = out["S"]
    tk = dt * np.arange(1, K)
    t_peak = tk[np.argmax(S)]
    assert abs(t_peak - tstar) <= 0.15 * tstar + dt, (t_peak, tstar)
    near = S[np.abs(tk - tstar) <= 0.25 * tstar].sum() / S.sum()
    assert near >= 0.7, near


def test_disk_contrast_doubles_peak_time():
    # one-homogeneity with the same dt: doubling the contrast doubles the impulse time
    dt, K = 0.1, 70
    f = syn.disk_image(40, 40, 5.0, 1.0).astype(np.float64)
    a = oracle.decompose(f, dt, K, 300, (0.0, INF))
    b = oracle.decompose(2 * f, dt, 2 * K, 300, (0.0, INF))
    ta = dt * (1 + np.argmax(a["S"]))
    tb = dt * (1 + np.argmax(b["S"]))
    assert abs(tb - 2 * ta) <= 2 * dt, (ta, tb)


# --------------------------------------------------------------------------------------------
# Degenerate and invalid inputs.
# --------------------------------------------------------------------------------------------
def test_zero_inner_iterations_is_identity_flow():
    f = _rand(6, 5, 19)
    out = oracle.decompose(f, 0.5, 4, 0, syn.DYADIC_EDGES)
    assert np.all(out["bands"] == 0.0) and np.all(out["S"] == 0.0)
    assert np.array_equal(out["residual"], f)


def test_single_pixel_and_single_row():
    for shape in [(1, 1), (1, 9), (9, 1)]:
        f = _rand(*shape, 20)
        out = oracle.decompose(f, 0.5, 5, 30, syn.DYADIC_EDGES)
        rec = out["bands"].sum(axis=0) + out["residual"]
        assert np.max(np.abs(rec - f)) <= 1e-12 * max(1.0, np.abs(f).max())
    out = oracle.decompose(np.ones((1, 1)), 0.5, 5, 30, syn.DYADIC_EDGES)
    assert np.all(out["S"] == 0.0)


def test_invalid_arguments_rejected():
    f = np.zeros((4, 4))
    with pytest.raises(ValueError):
        oracle.decompose(f, 0.5, 1, 10, syn.DYADIC_EDGES)
    with pytest.raises(ValueError):
        oracle.decompose(f, 0.0, 4, 10, syn.DYADIC_EDGES)
    with pytest.raises(ValueError):
        oracle.decompose(f, 0.5, 4, -1, syn.DYADIC_EDGES)


def test_warm_and_cold_start_agree_when_converged():
    # both start points of the dual iteration converge to the same ROF minimiser per step
    f = syn.make_image(12, 12, 3, (2, 5), (0.2, 1.0), 0.0, seed=21).astype(np.float64)
    diffs = []
    for n in (2000, 20000):
        a = oracle.decompose(f, 0.5, 4, n, syn.DYADIC_EDGES, warm_start=True, trace=True)
        b = oracle.decompose(f, 0.5, 4, n, syn.DYADIC_EDGES, warm_start=False, trace=True)
        diffs.append(np.abs(a["u"] - b["u"]).max())
    assert diffs[1] <= 1e-4 and diffs[1] < 0.5 * diffs[0], diffs


# --------------------------------------------------------------------------------------------
# Spectral filtering (Eq. filteredTVtrafo): f_H = sum_k H(t_k) phi_k dt + h_r f_r
# --------------------------------------------------------------------------------------------
def _filt_setup():
    dt, K = 0.5, 12
    f = syn.make_image(22, 27, 6, (2, 8), (0.1, 1.0), 0.03, seed=31).astype(np.float64)
    tk = dt * np.arange(1, K)
    return f, dt, K, tk


def test_all_pass_filter_reconstructs_the_image():
    f, dt, K, tk = _filt_setup()
    out = oracle.decompose(f, dt, K, 40, syn.DYADIC_EDGES, filters=[(np.ones(K - 1), 1.0)])
    assert np.max(np.abs(out["filtered"][0] - f)) <= 1e-12 * np.abs(f).max()


def test_band_indicator_filter_equals_the_band_exactly():
    f, dt, K, tk = _filt_setup()
    e = syn.DYADIC_EDGES
    filters = [(((e[m] <= tk) & (tk < e[m + 1])).astype(float), 0.0) for m in range(len(e) - 1)]
    out = oracle.decompose(f, dt, K, 40, e, filters=filters)
    assert np.array_equal(out["filtered"], out["bands"])


def test_complementary_filters_sum_to_the_image_and_filters_are_linear():
    f, dt, K, tk = _filt_setup()
    low = np.exp(-tk / 2.0)            # passes small scales
    high = 1.0 - low
    a, b = 0.7, -1.3
    out = oracle.decompose(f, dt, K, 40, syn.DYADIC_EDGES,
                           filters=[(low, 0.25), (high, 0.75), (a * low + b * high, a * 0.25 + b * 0.75)])
    fl, fh, fc = out["filtered"]
    assert np.max(np.abs(fl + fh - f)) <= 1e-12 * np.abs(f).max()
    assert np.max(np.abs(fc - (a * fl + b * fh))) <= 1e-12 * np.abs(f).max()


def test_filtering_is_one_homogeneous_exactly():
    f, dt, K, tk = _filt_setup()
    h = np.cos(tk)
    a = oracle.decompose(f, dt, K, 40, syn.DYADIC_EDGES, filters=[(h, 0.5)])
    b = oracle.decompose(2 * f, 2 * dt, K, 40, tuple(2 * x for x in syn.DYADIC_EDGES), filters=[(h, 0.5)])
    assert np.array_equal(b["filtered"], 2 * a["filtered"])


# --------------------------------------------------------------------------------------------
# Parseval-type spectrum <phi_k, f> (the alternative spectrum Sec. 2.1 names): its Riemann sum
# with the residual's pairing is |f|^2, each band's pairing with f is its share of that sum,
# it is exactly one-homogeneous, and for a disk it peaks where S(t) does.
# --------------------------------------------------------------------------------------------
def test_parseval_spectrum_sums_to_the_energy():
    f, dt, K, tk = _filt_setup()
    out = oracle.decompose(f, dt, K, 40, syn.DYADIC_EDGES)
    total = out["S_parseval"].sum() * dt + float((out["residual"] * f).sum())
    assert abs(total - float((f * f).sum())) <= 1e-11 * float((f * f).sum())


def test_parseval_spectrum_splits_over_the_bands():
    f, dt, K, tk = _filt_setup()
    e = syn.DYADIC_EDGES
    out = oracle.decompose(f, dt, K, 40, e)
    for m, ks in enumerate(syn.band_index_ranges(dt, K, e)):
        want = float((out["bands"][m] * f).sum())
        got = sum(out["S_parseval"][k - 1] for k in ks) * dt
        assert abs(got - want) <= 1e-11 * max(1.0, abs(want)), (m, got, want)


def test_parseval_spectrum_one_homogeneous_and_constant_image():
    f, dt, K, tk = _filt_setup()
    a = oracle.decompose(f, dt, K, 40, syn.DYADIC_EDGES)
    b = oracle.decompose(2 * f, 2 * dt, K, 40, tuple(2 * x for x in syn.DYADIC_EDGES))
    assert np.array_equal(b["S_parseval"], 2 * a["S_parseval"])
    c = oracle.decompose(np.full((9, 7), 0.4), dt, K, 40, syn.DYADIC_EDGES)
    assert np.all(c["S_parseval"] == 0)


def test_parseval_spectrum_of_a_disk_peaks_with_S():
    dt, K = 0.1, 70
    f = syn.disk_image(48, 48, 8.0, 1.0).astype(np.float64)
    out = oracle.decompose(f, dt, K, 300, (0.0, INF))
    assert abs(int(np.argmax(out["S_parseval"])) - int(np.argmax(out["S"]))) <= 1
