"""Randomised checks of the oracle against what the method fixes for any input (hypothesis
draws the image size, the schedule and the image): the telescoping reconstruction of
Eq. spectral_bands / Eq. finite_inverse_trafo, mean preservation and zero-sum phi (div has zero
sum), S as the L1 norm of phi, exact one-homogeneity under (c f, c dt) with c = 2 (the dual
iterations see g / dt unchanged), and exact transpose equivariance of u and the bands (the
isotropic norm is symmetric; S, a sum in row-major order, up to rounding). The fixed-seed
versions of these pins live in test_oracle_pins.py; here the sizes include 1-pixel rows and
columns and the schedules include n_inner = 0. Derandomised: the same draws on every run."""
import math

import numpy as np
import pytest

hypothesis = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402

import oracle  # noqa: E402

EDGE_SETS = ([0.0, math.inf], [0.0, 1.0, 2.0, 4.0, math.inf], [0.5, 3.0, math.inf], [0.0, 0.25, 0.75, 10.0])


@st.composite
def problems(draw):
    H = draw(st.integers(1, 12))
    W = draw(st.integers(1, 12))
    K = draw(st.integers(2, 7))
    n_inner = draw(st.integers(0, 25))
    dt = draw(st.sampled_from([0.125, 0.25, 0.5, 1.0]))
    edges = draw(st.sampled_from(EDGE_SETS))
    seed = draw(st.integers(0, 2 ** 31 - 1))
    rng = np.random.default_rng(seed)
    f = (rng.standard_normal((H, W)) * draw(st.sampled_from([0.1, 1.0, 10.0]))).astype(np.float32)
    return f, dt, K, n_inner, edges


@settings(max_examples=60, deadline=None, derandomize=True)
@given(problems(), st.booleans())
def test_reconstruction_mean_and_l1(p, warm):
    f, dt, K, n, edges = p
    r = oracle.decompose(f, dt, K, n, edges, warm_start=warm, trace=True)
    f64 = f.astype(np.float64)
    scale = max(1.0, float(np.abs(f64).max()))
    # Eq. spectral_bands + Eq. finite_inverse_trafo: bands cover [e_0, e_last); with e_0 > 0 or
    # a finite last edge some t_k fall outside every band, so reconstruct from phi directly
    u = r["u"]
    phi = [(k * dt) * (u[k + 1] - 2 * u[k] + u[k - 1]) / dt ** 2 for k in range(1, K)]
    rec = sum(p_ * dt for p_ in phi) + r["residual"] if phi else r["residual"]
    assert np.abs(rec - f64).max() <= 1e-12 * scale
    if edges[0] == 0.0 and math.isinf(edges[-1]):
        assert np.abs(r["bands"].sum(0) + r["residual"] - f64).max() <= 1e-12 * scale
    for k in range(K + 1):  # div has zero sum: the mean stays in u
        assert abs(u[k].sum() - f64.sum()) <= 1e-12 * scale * f.size
    for k, p_ in enumerate(phi, start=1):
        assert abs(p_.sum()) <= 1e-9 * scale * f.size
        assert r["S"][k - 1] == pytest.approx(np.abs(p_).sum(), rel=1e-12, abs=1e-300)


@settings(max_examples=40, deadline=None, derandomize=True)
@given(problems())
def test_one_homogeneity_and_transpose_exact(p):
    f, dt, K, n, edges = p
    a = oracle.decompose(f, dt, K, n, edges, trace=True)
    b = oracle.decompose(2 * f, 2 * dt, K, n, [2 * e for e in edges], trace=True)
    assert np.array_equal(b["u"], 2 * a["u"])
    assert np.array_equal(b["bands"], 2 * a["bands"])
    assert np.array_equal(b["S"], a["S"])
    t = oracle.decompose(np.ascontiguousarray(f.T), dt, K, n, edges, trace=True)
    assert np.array_equal(t["u"], np.transpose(a["u"], (0, 2, 1)))
    assert np.array_equal(t["bands"], np.transpose(a["bands"], (0, 2, 1)))
    # S sums |phi| in row-major order, which the transpose permutes: equal up to rounding
    np.testing.assert_allclose(t["S"], a["S"], rtol=1e-12, atol=0)


@settings(max_examples=25, deadline=None, derandomize=True)
@given(st.integers(2, 4), st.integers(0, 6), st.integers(0, 2 ** 31 - 1))
def test_finite_propagation_speed(K, n, seed):
    # an iteration moves information one pixel (w reads p one pixel up / left, the update reads
    # w one pixel down / right, u_{k+1} reads p one pixel up / left): after K steps of n
    # iterations an output depends only on inputs within K (n + 1) pixels, so a window with that
    # margin reproduces the full image's outputs on its centre bit for bit (the premise of the
    # largest-image GPU test, which compares windows)
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((80, 84)).astype(np.float32)
    edges = [0.0, 1.0, math.inf]
    full = oracle.decompose(f, 0.5, K, n, edges)
    m, y0, x0, side = K * (n + 1), 35, 37, 6  # the window stays inside the image (m <= 28)
    win = oracle.decompose(f[y0 - m:y0 + side + m, x0 - m:x0 + side + m], 0.5, K, n, edges)
    c = (slice(None), slice(m, m + side), slice(m, m + side))
    assert np.array_equal(win["bands"][c], full["bands"][:, y0:y0 + side, x0:x0 + side])
    assert np.array_equal(win["residual"][c[1:]], full["residual"][y0:y0 + side, x0:x0 + side])


@settings(max_examples=40, deadline=None, derandomize=True)
@given(problems(), st.integers(0, 2 ** 31 - 1))
def test_filters_and_parseval_identities(p, seed):
    # Eq. filteredTVtrafo in Eq. finite_inverse_trafo: the all-pass filter (H = 1, h_r = 1)
    # reconstructs f; filtering is linear in H; and the Parseval-type spectrum splits the energy,
    # sum_k <phi_k, f> dt + <f_r, f> = |f|^2
    f, dt, K, n, edges = p
    rng = np.random.default_rng(seed)
    h1, h2 = rng.standard_normal(K - 1), rng.standard_normal(K - 1)
    r1, r2 = float(rng.standard_normal()), float(rng.standard_normal())
    out = oracle.decompose(f, dt, K, n, edges,
                           filters=[(np.ones(K - 1), 1.0), (h1, r1), (h2, r2), (h1 + 2 * h2, r1 + 2 * r2)])
    f64 = f.astype(np.float64)
    scale = max(1.0, float(np.abs(f64).max()))
    F = out["filtered"]
    assert np.abs(F[0] - f64).max() <= 1e-12 * scale
    lin_scale = scale * max(1.0, float(np.abs(np.concatenate([h1, h2, [r1, r2]])).max()))
    assert np.abs(F[3] - (F[1] + 2 * F[2])).max() <= 1e-11 * lin_scale
    energy = float((f64 * f64).sum())
    total = out["S_parseval"].sum() * dt + float((out["residual"] * f64).sum())
    assert abs(total - energy) <= 1e-10 * max(energy, scale * scale)


@settings(max_examples=60, deadline=None, derandomize=True)
@given(st.integers(1, 10), st.integers(1, 10), st.floats(0.01, 5.0), st.integers(0, 2 ** 31 - 1))
def test_weak_duality_of_the_rof_gap(H, W, lam, seed):
    # Eq. ROF: for any u and any dual field with |p| <= 1 the primal value
    # 1/2 |u - g|^2 + lam J_TV(u) is at least the dual value 1/2 |g|^2 - 1/2 |g - lam div p|^2,
    # so both gap functions are non-negative; with u = g - lam div p they coincide; at the
    # optimum the gap is zero
    rng = np.random.default_rng(seed)
    g = rng.standard_normal((H, W))
    u = rng.standard_normal((H, W)) * rng.choice([0.01, 1.0, 10.0])
    ang = rng.uniform(0, 2 * np.pi, (H, W))
    mag = rng.uniform(0, 1, (H, W))
    p1, p2 = mag * np.cos(ang), mag * np.sin(ang)
    scale = 1.0 + float((g * g).sum() + (u * u).sum())
    assert oracle.rof_gap_pair(g, lam, u, p1, p2) >= -1e-12 * scale
    assert oracle.rof_gap(g, lam, p1, p2) >= -1e-12 * scale
    uc, q1, q2 = oracle.chambolle(g, lam, 0, p1=p1, p2=p2)  # u = g - lam div p
    assert oracle.rof_gap_pair(g, lam, uc, p1, p2) == pytest.approx(oracle.rof_gap(g, lam, p1, p2),
                                                                    rel=1e-9, abs=1e-12 * scale)
    # and the gap closes at the optimum (fast gradient projection, O(1/k^2)): strong duality
    us, s1, s2 = oracle.fgp(g, lam, 3000)
    gap = oracle.rof_gap_pair(g, lam, us, s1, s2)
    gs = 1.0 + float((g * g).sum())
    assert -1e-9 * gs <= gap <= 1e-6 * gs


@settings(max_examples=60, deadline=None, derandomize=True)
@given(st.integers(1, 8), st.integers(1, 3), st.integers(0, 2 ** 31 - 1))
def test_crop_and_standardisation(size, scale, seed):
    # the training-data preparation (Sec. 4.1): a crop is the scale x scale block average of
    # its (scale size)^2 window, rounded to float32 (numpy's block mean, to one float32 ulp);
    # standardising over the set gives mean 0 and population std 1, per image likewise
    rng = np.random.default_rng(seed)
    sH, sW = int(rng.integers(scale * size, scale * size + 20)), int(rng.integers(scale * size, scale * size + 20))
    src = (rng.standard_normal((sH, sW)) * 3 + 1).astype(np.float32)
    y = int(rng.integers(0, sH - scale * size + 1))
    x = int(rng.integers(0, sW - scale * size + 1))
    c = oracle.crop(src, y, x, size, scale)
    win = src[y:y + scale * size, x:x + scale * size].astype(np.float64)
    want = win.reshape(size, scale, size, scale).mean(axis=(1, 3)).astype(np.float32)
    assert np.all(np.abs(c - want) <= np.spacing(np.abs(want).astype(np.float32)))
    imgs = np.stack([oracle.crop(src, int(rng.integers(0, sH - scale * size + 1)),
                                 int(rng.integers(0, sW - scale * size + 1)), size, scale)
                     for _ in range(3)])
    if np.ptp(imgs) > 0:
        z, ms = oracle.standardize(imgs, 1)
        assert abs(z.mean()) <= 1e-6 and abs(z.std() - 1.0) <= 1e-6
    z2, ms2 = oracle.standardize(imgs, 2)
    for i in range(3):
        if np.ptp(imgs[i]) > 0:
            assert abs(z2[i].mean()) <= 1e-6 and abs(z2[i].std() - 1.0) <= 1e-6
