"""Pins of the oracle's other ROF solvers (fast gradient projection, primal-dual hybrid
gradient) and of the pair duality gap: closed forms, an exact 1-D solve, a certified
reference, the gap's lower bound, and the ordering of convergence the methods promise."""
import json
import math
import os

import numpy as np
import pytest

import oracle
import refsolvers as rs
import synthetic as syn

SOLVERS = {
    "fgp": lambda g, lam, n: oracle.fgp(g, lam, n),
    "pdhg": lambda g, lam, n: oracle.pdhg(g, lam, n),
    "pdhg_basic": lambda g, lam, n: oracle.pdhg(g, lam, n, tau=1 / math.sqrt(8), sigma=1 / math.sqrt(8), gamma=0.0),
}


def _gap(g, lam, u, p1, p2):
    return oracle.rof_gap_pair(g, lam, u, p1, p2)


def _near(u, exact, g, lam, p1, p2, name):
    """u within the gap's certificate of the exact minimiser, and the gap small. The
    accelerated primal-dual method converges in u only like 1/N in its tail, so its bar is
    the certificate |u - u*| <= sqrt(2 gap); the others must also be close pointwise."""
    gap = _gap(g, lam, u, p1, p2)
    assert -1e-12 <= gap <= 1e-9, (name, gap)
    # the gap is a difference of O(1) energies: allow for its rounding (1e-13 absolute)
    assert np.linalg.norm(u - exact) <= math.sqrt(2 * max(gap, 0.0) + 1e-13), name
    if name == "fgp":
        np.testing.assert_allclose(u, exact, rtol=0, atol=1e-8)


@pytest.mark.parametrize("name", list(SOLVERS))
def test_two_pixel_closed_form(golden_dir, name):
    data = json.load(open(os.path.join(golden_dir, "two_pixel_rof.json")))
    for case in data["cases"]:
        g = np.asarray(case["g"], np.float64).reshape(1, 2)
        u, p1, p2 = SOLVERS[name](g, case["lam"], 20000)
        _near(u, np.asarray(case["u"], np.float64).reshape(1, 2), g, case["lam"], p1, p2, name)


@pytest.mark.parametrize("name", list(SOLVERS))
def test_1d_segments_closed_form(golden_dir, name):
    data = json.load(open(os.path.join(golden_dir, "segments_1d_rof.json")))
    for case in data["cases"]:
        prof = np.concatenate([np.full(m, v, dtype=np.float64) for m, v in zip(case["lengths"], case["values"])])
        expect = np.concatenate([np.full(m, v) for m, v in zip(case["lengths"], case["u_segments"])])
        g = np.tile(prof[:, None], (1, 3))
        u, p1, p2 = SOLVERS[name](g, case["lam"], 20000)
        _near(u, np.broadcast_to(expect[:, None], g.shape), g, case["lam"], p1, p2, name)


@pytest.mark.parametrize("name", list(SOLVERS))
@pytest.mark.parametrize("seed,lam", [(0, 0.2), (2, 1.5)])
def test_1d_stripe_matches_exact_bvls(name, seed, lam):
    prof = np.random.default_rng(seed).normal(size=12)
    exact = rs.rof_1d_bvls(prof, lam)
    g = np.tile(prof[:, None], (1, 4))
    u, p1, p2 = SOLVERS[name](g, lam, 30000)
    _near(u, np.tile(exact[:, None], (1, 4)), g, lam, p1, p2, name)


@pytest.mark.parametrize("name", list(SOLVERS))
def test_8x8_certified_by_the_gap(name):
    g = np.random.default_rng(3).normal(size=(8, 8))
    lam = 0.3
    u_ref, gap_ref, _ = rs.rof_fista(g, lam, gap_tol=1e-13)
    u, p1, p2 = SOLVERS[name](g, lam, 5000)
    gap = _gap(g, lam, u, p1, p2)
    assert gap >= -1e-12
    # 1/2 |u - u*|^2 <= gap for both points
    assert np.linalg.norm(u - u_ref) <= math.sqrt(2 * max(gap, 0)) + math.sqrt(2 * max(gap_ref, 0)) + 1e-12
    assert gap <= 1e-6


def test_pair_gap_bounds_the_distance_to_the_minimiser():
    g = syn.make_image(20, 24, 4, (2, 6), (0.1, 1.0), 0.05, seed=4).astype(np.float64)
    lam = 0.5
    u_star, gs, _ = rs.rof_fista(g, lam, gap_tol=1e-12)
    for n in (5, 30, 200):
        for name in SOLVERS:
            u, p1, p2 = SOLVERS[name](g, lam, n)
            gap = _gap(g, lam, u, p1, p2)
            assert 0.5 * np.sum((u - u_star) ** 2) <= gap + gs + 1e-12, (name, n)
            assert np.max(np.sqrt(p1 ** 2 + p2 ** 2)) <= 1.0 + 1e-12


def test_pair_gap_agrees_with_the_dual_gap_on_the_dual_primal():
    g = np.random.default_rng(9).normal(size=(11, 13))
    _, p1, p2 = oracle.chambolle(g, 0.4, 37)
    u = g - 0.4 * oracle.div(p1, p2)
    assert abs(_gap(g, 0.4, u, p1, p2) - oracle.rof_gap(g, 0.4, p1, p2)) <= 1e-12


def test_accelerated_methods_beat_chambolle_at_equal_iterations():
    # O(1/k^2) methods against Chambolle's O(1/k) on the same problem and start
    g = syn.make_image(48, 48, 6, (3, 14), (0.1, 1.0), 0.02, seed=1).astype(np.float64)
    lam = 0.5
    for n in (100, 400):
        _, a, b = oracle.chambolle(g, lam, n)
        gc = oracle.rof_gap(g, lam, a, b)
        u, a, b = oracle.fgp(g, lam, n)
        gf = _gap(g, lam, u, a, b)
        u, a, b = oracle.pdhg(g, lam, n)
        gp = _gap(g, lam, u, a, b)
        assert gf < 0.2 * gc and gp < 0.2 * gc, (n, gc, gf, gp)


def test_fgp_zero_iterations_and_warm_start_at_the_optimum():
    g = np.random.default_rng(5).normal(size=(9, 10))
    u, p1, p2 = oracle.fgp(g, 0.3, 0)
    assert np.array_equal(u, g)
    _, q1, q2 = oracle.fgp(g, 0.3, 20000)
    u1, r1, r2 = oracle.fgp(g, 0.3, 50, q1, q2)  # starting at the optimum stays there
    assert _gap(g, 0.3, u1, r1, r2) <= 1e-9
