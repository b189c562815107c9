"""The Parseval-type spectrum <phi_k, f> and fine band sets on the GPU, against the oracle and
against the identities the definitions fix."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from tolerances import RECON_INF, assert_parity

pytestmark = pytest.mark.gpu
INF = float("inf")


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


@pytest.mark.parametrize("H,W,K,n_inner", [(64, 64, 20, 200), (45, 99, 10, 50), (200, 130, 8, 40)])
def test_parseval_spectrum_parity_and_energy_identity(plan, H, W, K, n_inner):
    f = _img(H, W, H + 3 * W)
    g = plan.decompose(f, 0.5, K, n_inner, syn.DYADIC_EDGES, parseval=True)
    ref = oracle.decompose(f, 0.5, K, n_inner, syn.DYADIC_EDGES)
    sp, rp = np.asarray(g["S_parseval"]), ref["S_parseval"]
    assert np.max(np.abs(sp - rp)) <= 1e-3 * np.max(np.abs(rp)), np.max(np.abs(sp - rp)) / np.max(np.abs(rp))
    fd = f.astype(np.float64)
    energy = sp.sum() * 0.5 + float((np.asarray(g["residual"], np.float64) * fd).sum())
    assert abs(energy - float((fd * fd).sum())) <= RECON_INF * float((fd * fd).sum())


def test_parseval_request_leaves_other_outputs_unchanged(plan):
    f = _img(70, 90, 5)
    a = plan.decompose(f, 0.5, 8, 30, syn.DYADIC_EDGES)
    b = plan.decompose(f, 0.5, 8, 30, syn.DYADIC_EDGES, parseval=True)
    for k in ("bands", "residual", "S"):
        assert np.array_equal(a[k], b[k]), k


def test_parseval_resident_per_step_host_device_served_bit_identical(tv):
    import torch

    crops = [_img(60, 64, 400 + j) for j in range(36)]
    jobs = [(c, 0.5, 7, 25, syn.DYADIC_EDGES) for c in crops]
    outs = {}
    for mode in (0, 2):
        with tv.Plan(0, resident=mode) as p:
            outs[mode] = p.decompose_batch(jobs, parseval=True)
    for a, b in zip(outs[0], outs[2]):
        assert np.array_equal(a["S_parseval"], b["S_parseval"])
        assert np.array_equal(a["S"], b["S"])
    with tv.Plan(0) as p:
        d = p.decompose(torch.from_numpy(crops[0]).cuda(), 0.5, 7, 25, syn.DYADIC_EDGES, parseval=True)
        torch.cuda.synchronize()
        assert np.array_equal(d["S_parseval"].cpu().numpy(), outs[0][0]["S_parseval"])
        t, o = p.submit(crops[1], 0.5, 7, 25, syn.DYADIC_EDGES, parseval=True)
        assert p.wait(t, 60000) == tv.OK
        assert np.array_equal(o["S_parseval"], outs[0][1]["S_parseval"])


def test_twenty_five_log_spaced_bands(plan):
    # a fine band set (25 bands, log-spaced in t) at the parity bars
    edges = (0.0,) + tuple(float(x) for x in np.logspace(-0.5, 1.4, 24)) + (INF,)
    f = _img(96, 80, 77)
    g = plan.decompose(f, 0.25, 60, 60, edges)
    ref = oracle.decompose(f, 0.25, 60, 60, edges)
    assert g["bands"].shape == (25, 96, 80)
    assert_parity(g, ref, f, "25 bands")
