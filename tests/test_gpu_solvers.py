"""Inner ROF solvers on the GPU (tvspec_rof_solve): Chambolle's projection, fast gradient
projection and the primal-dual method against the oracle's solvers, the gap kernel against
the oracle's pair gap, gap-based stopping and its certificate."""
import math

import numpy as np
import pytest

import oracle
import synthetic as syn
from tolerances import U_INF

pytestmark = pytest.mark.gpu
NAMES = ("chambolle", "fgp", "pdhg")


@pytest.fixture(scope="module")
def tv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_10004_gb300 as tvm

    tvm.load()
    return tvm


@pytest.fixture(scope="module")
def plan(tv):
    p = tv.Plan(0)
    yield p
    p.close()


def _img(H, W, seed):
    return syn.make_image(H, W, 6, (2.0, 14.0), (0.1, 1.0), 0.02, seed)


def _oracle(name, g, lam, n):
    if name == "chambolle":
        return oracle.chambolle(g, lam, n)
    if name == "fgp":
        return oracle.fgp(g, lam, n)
    return oracle.pdhg(g, lam, n)


@pytest.mark.parametrize("name", NAMES)
@pytest.mark.parametrize("H,W,n", [(64, 64, 200), (37, 101, 50), (130, 70, 120), (1, 9, 30)])
def test_fixed_iterations_parity(plan, name, H, W, n):
    g = _img(H, W, H * 7 + W)
    lam = 0.5
    r = plan.rof_solve(g, lam, name, max_iter=n)
    u, p1, p2 = _oracle(name, g.astype(np.float64), lam, n)
    assert r["iterations"] == n
    err = np.max(np.abs(r["u"] - u)) / np.max(np.abs(g))
    assert err <= U_INF, (name, err)
    # the GPU's gap is the pair gap of its own (float) outputs, reduced in float64
    want = oracle.rof_gap_pair(g, lam, r["u"], r["p1"], r["p2"])
    assert abs(r["gap"] - want) <= 1e-9 * max(1.0, abs(want)), (r["gap"], want)


@pytest.mark.parametrize("name", NAMES)
def test_gap_stopping_and_its_certificate(plan, name):
    g = _img(96, 80, 5)
    lam, tol = 0.5, 0.15  # Chambolle's O(1/k) needs ~10^4 iterations for this on 96x80
    r = plan.rof_solve(g, lam, name, max_iter=50000, gap_tol=tol, check_every=25)
    assert r["gap"] <= tol and r["iterations"] % 25 == 0 and r["iterations"] < 50000
    u_star, q1, q2 = oracle.fgp(g.astype(np.float64), lam, 4000)
    gap_star = oracle.rof_gap_pair(g, lam, u_star, q1, q2)
    dist = np.linalg.norm(r["u"].astype(np.float64) - u_star)
    assert dist <= math.sqrt(2 * max(r["gap"], 0)) + math.sqrt(2 * max(gap_star, 0)) + 1e-6


def test_accelerated_solvers_reach_a_smaller_gap_at_equal_iterations(plan):
    g = _img(128, 128, 9)
    gaps = {name: plan.rof_solve(g, 0.5, name, max_iter=200)["gap"] for name in NAMES}
    assert gaps["fgp"] < 0.2 * gaps["chambolle"] and gaps["pdhg"] < 0.2 * gaps["chambolle"], gaps


def test_warm_start_at_the_optimum_stays_there(plan):
    g = _img(50, 60, 3)
    best = plan.rof_solve(g, 0.5, "fgp", max_iter=3000)
    for name in ("chambolle", "fgp"):
        r = plan.rof_solve(g, 0.5, name, max_iter=40, p_in=(best["p1"], best["p2"]))
        assert r["gap"] <= max(2 * best["gap"], 1e-6), (name, r["gap"], best["gap"])


def test_device_memory_matches_host(plan):
    import torch

    g = _img(70, 45, 11)
    for name in NAMES:
        h = plan.rof_solve(g, 0.5, name, max_iter=60)
        d = plan.rof_solve(torch.from_numpy(g).cuda(), 0.5, name, max_iter=60)
        torch.cuda.synchronize()
        assert np.array_equal(h["u"], d["u"].cpu().numpy()) and h["gap"] == d["gap"], name


def test_invalid_solver_arguments(plan, tv):
    g = _img(16, 16, 1)
    for kw in (dict(solver=7), dict(check_every=0), dict(solver="pdhg", tau=0.5, sigma=0.5),
               dict(max_iter=-1), dict(solver="pdhg", gamma=-1.0)):
        args = dict(solver="chambolle", max_iter=10)
        args.update(kw)
        with pytest.raises(tv.TvSpecError) as ei:
            plan.rof_solve(g, 0.5, **args)
        assert ei.value.status == tv.EINVAL
    assert np.isfinite(plan.rof_solve(g, 0.5, "pdhg", max_iter=10)["u"]).all()


@pytest.mark.parametrize("H,W,n", [(64, 64, 37), (200, 333, 21), (1, 9, 9), (130, 70, 8), (517, 260, 50)])
def test_blocked_fgp_matches_the_one_iteration_kernel_bit_for_bit(plan, H, W, n):
    # register tiles with overlapped halos change where an iteration is computed, not its bits
    g = _img(H, W, 3 * H + W)
    a = plan.rof_solve(g, 0.5, "fgp", max_iter=n)
    b = plan.rof_solve(g, 0.5, "fgp_reference", max_iter=n)
    for k in ("u", "p1", "p2"):
        assert np.array_equal(a[k], b[k]), k
    assert a["gap"] == b["gap"]
