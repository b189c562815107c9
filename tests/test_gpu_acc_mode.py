"""The compensated-float32 epilogue (acc_mode = 1, float-float arithmetic) against the FP64
oracle at the same bars as the float64 epilogue, and bit-identity across the paths."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from tolerances import RECON_INF, assert_parity

pytestmark = pytest.mark.gpu


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
    p = tv.Plan(0, acc_mode=1)
    yield p
    p.close()


def _img(H, W, seed):
    return syn.make_image(H, W, 6, (2.0, 14.0), (0.1, 1.0), 0.02, seed)


def _same(a, b, keys=("bands", "residual", "S")):
    for k in keys:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def test_config0_parity_with_trace(plan):
    job = syn.config0().jobs[0]
    g = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, trace=True)
    ref = oracle.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, trace=True)
    m = assert_parity(g, ref, job.f, "config0 acc_mode 1")
    print(m)


@pytest.mark.parametrize("H,W,K,dt", [(37, 53, 9, 0.5), (130, 70, 6, 0.25), (1, 17, 5, 1.0), (200, 333, 5, 0.5)])
def test_ragged_parity(plan, H, W, K, dt):
    f = _img(H, W, H + W)
    g = plan.decompose(f, dt, K, 30, syn.DYADIC_EDGES, trace=True)
    ref = oracle.decompose(f, dt, K, 30, syn.DYADIC_EDGES, trace=True)
    assert_parity(g, ref, f, f"{H}x{W}")


def test_config1_full_size_parity(plan):
    job = syn.config1().jobs[0]
    g = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges)
    ref = oracle.decompose(job.f, job.dt, job.K, job.n_inner, job.edges)
    print(assert_parity(g, ref, job.f, "config1 acc_mode 1"))


def test_close_to_the_float64_epilogue(tv, plan):
    f = _img(90, 110, 4)
    with tv.Plan(0) as p64:
        a = p64.decompose(f, 0.5, 12, 40, syn.DYADIC_EDGES, trace=True)
    b = plan.decompose(f, 0.5, 12, 40, syn.DYADIC_EDGES, trace=True)
    # g/dt is rounded to float32 for the dual iterations; where the two modes round it apart,
    # the iterations move by a float32 ulp: float32-level agreement, not float64-level
    assert np.max(np.abs(a["u"] - b["u"])) <= 1e-5 * np.max(np.abs(f))
    assert np.max(np.abs(a["S"] - b["S"])) <= 1e-4 * np.max(np.abs(a["S"]))
    recon = np.asarray(b["bands"], np.float64).sum(0) + b["residual"]
    assert np.max(np.abs(recon - f)) <= RECON_INF * np.max(np.abs(f))


def test_resident_batch_alone_and_device_bit_identical(tv, plan):
    import torch

    crops = [_img(50 + (i % 3) * 7, 64, 80 + i) for i in range(34)]
    jobs = [(c, 0.5, 7, 25, syn.DYADIC_EDGES) for c in crops]
    with tv.Plan(0, acc_mode=1, resident=2) as r, tv.Plan(0, acc_mode=1, resident=0) as s:
        a = r.decompose_batch(jobs, parseval=True)
        b = s.decompose_batch(jobs, parseval=True)
    for x, y in zip(a, b):
        _same(x, y, ("bands", "residual", "S", "S_parseval"))
    alone = plan.decompose(*jobs[5])
    _same(alone, b[5])
    d = plan.decompose(torch.from_numpy(crops[5]).cuda(), 0.5, 7, 25, syn.DYADIC_EDGES)
    torch.cuda.synchronize()
    assert np.array_equal(d["bands"].cpu().numpy(), alone["bands"])


def test_filters_and_served_requests(tv, plan):
    job = syn.config0().jobs[0]
    bank = [(np.ones(job.K - 1), 1.0), (np.exp(-0.5 * np.arange(1, job.K)), 0.25)]
    g = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=bank, parseval=True)
    ref = oracle.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=bank)
    scale = np.max(np.abs(job.f))
    assert np.max(np.abs(g["filtered"] - ref["filtered"])) <= 1e-3 * scale
    assert np.max(np.abs(g["filtered"][0] - job.f)) <= RECON_INF * scale
    assert np.max(np.abs(g["S_parseval"] - ref["S_parseval"])) <= 1e-3 * np.max(np.abs(ref["S_parseval"]))
    with tv.Plan(0, acc_mode=1) as p:
        t, out = p.submit(job.f, job.dt, job.K, job.n_inner, job.edges)
        assert p.wait(t, 60000) == tv.OK
    _same(out, g)


def test_training_set_in_compensated_mode(tv):
    srcs = [syn.make_image(200, 240, 12, (2.0, 24.0), (0.05, 1.0), 0.02, seed=s) for s in (1, 2)]
    crops = [(i % 2, 10 + i, 20 + 2 * i, 1 + i % 2) for i in range(40)]
    with tv.Plan(0, acc_mode=1) as p:
        g = p.training_set(srcs, crops, 32, 1, 0.5, 6, 30, syn.DYADIC_EDGES)
    ref = oracle.training_set(srcs, crops, 32, 1, 0.5, 6, 30, syn.DYADIC_EDGES)
    for i in (0, 17, 39):
        gi = {k: np.asarray(g[k][i]) for k in ("bands", "residual", "S")}
        ri = {k: ref[k][i] for k in ("bands", "residual", "S")}
        assert_parity(gi, ri, np.asarray(g["crops"][i], np.float64), f"crop {i}")


def test_invalid_acc_mode(tv):
    with pytest.raises(tv.TvSpecError):
        tv.Plan(0, acc_mode=2)
