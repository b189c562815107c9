"""Spectral filtering on the GPU (Eq. filteredTVtrafo substituted into Eq. finite_inverse_trafo).

The filter bank runs inside the per-step float64 epilogue; these tests compare it with the
FP64 oracle's ``filtered`` output and check the properties the definition fixes exactly on
the GPU's own outputs: an indicator filter of a band reproduces that band bit for bit, and the
all-pass filter reconstructs f within the reconstruction bar.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn
from tolerances import BAND_INF, BAND_REL_L2, RECON_INF

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
    p = tv.Plan(0)
    yield p
    p.close()


def _bank(dt, K, edges):
    """All-pass, ideal low/high/band-pass in t, a smooth one and a random one."""
    t = dt * np.arange(1, K)
    rng = np.random.default_rng(K)
    return [
        (np.ones(K - 1), 1.0),                               # all-pass: reconstructs f
        ((t < 2.0).astype(np.float64), 0.0),                 # small scales only
        ((t >= 2.0).astype(np.float64), 1.0),                # large scales + residual
        (((t >= 1.0) & (t < 4.0)).astype(np.float64), 0.0),  # band-pass
        (np.exp(-t / 4.0), 0.5),                             # smooth attenuation
        (rng.uniform(-1.0, 2.0, K - 1), -0.25),              # arbitrary weights
    ]


def _filtered_parity(g, ref, f, what):
    scale = float(np.max(np.abs(f))) or 1.0
    a = np.asarray(g, np.float64)
    b = np.asarray(ref, np.float64)
    inf = float(np.max(np.abs(a - b))) / scale
    rel = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
    assert inf <= BAND_INF, (what, inf)
    assert rel <= BAND_REL_L2 or np.linalg.norm(b) < 1e-12, (what, rel)
    return inf, rel


@pytest.mark.parametrize("H,W,K,n_inner", [(64, 64, 20, 200), (37, 101, 12, 60), (130, 70, 9, 40)])
def test_filter_bank_parity(plan, H, W, K, n_inner):
    f = syn.make_image(H, W, 6, (2.0, 16.0), (0.1, 1.0), 0.01, seed=H + W + K)
    bank = _bank(0.5, K, syn.DYADIC_EDGES)
    g = plan.decompose(f, 0.5, K, n_inner, syn.DYADIC_EDGES, filters=bank)
    ref = oracle.decompose(f, 0.5, K, n_inner, syn.DYADIC_EDGES, filters=bank)
    assert g["filtered"].shape == (len(bank), H, W)
    for q in range(len(bank)):
        _filtered_parity(g["filtered"][q], ref["filtered"][q], f, f"filter {q}")


def test_all_pass_reconstructs_f(plan):
    job = syn.config0().jobs[0]
    bank = [(np.ones(job.K - 1), 1.0)]
    g = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=bank)
    err = float(np.max(np.abs(g["filtered"][0].astype(np.float64) - job.f))) / float(np.max(np.abs(job.f)))
    assert err <= RECON_INF, err


def test_band_indicator_filters_equal_bands_bit_for_bit(plan):
    job = syn.config0().jobs[0]
    ranges = syn.band_index_ranges(job.dt, job.K, job.edges)
    bank = []
    for ks in ranges:
        Hv = np.zeros(job.K - 1)
        for k in ks:
            Hv[k - 1] = 1.0
        bank.append((Hv, 0.0))
    g = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=bank)
    assert np.array_equal(g["filtered"], g["bands"])


def test_filters_leave_other_outputs_unchanged(plan):
    job = syn.config0().jobs[0]
    a = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges)
    b = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=_bank(job.dt, job.K, job.edges))
    for k in ("bands", "residual", "S"):
        assert np.array_equal(a[k], b[k]), k


def test_resident_and_per_step_filters_bit_identical(tv):
    crops = [syn.make_image(48 + (i % 3) * 8, 56, 4, (2.0, 10.0), (0.1, 1.0), 0.02, seed=70 + i)
             for i in range(40)]
    bank = _bank(0.5, 8, syn.DYADIC_EDGES)
    jobs = [(c, 0.5, 8, 30, syn.DYADIC_EDGES, bank) for c in crops]
    outs = {}
    for mode in (0, 2):
        with tv.Plan(0, resident=mode) as p:
            outs[mode] = p.decompose_batch(jobs)
    for a, b in zip(outs[0], outs[2]):
        assert np.array_equal(a["filtered"], b["filtered"])
        assert np.array_equal(a["bands"], b["bands"])


def test_device_memory_filters_match_host(plan):
    import torch

    job = syn.config0().jobs[0]
    bank = _bank(job.dt, job.K, job.edges)
    h = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=bank)
    d = plan.decompose(torch.from_numpy(job.f).cuda(), job.dt, job.K, job.n_inner, job.edges, filters=bank)
    torch.cuda.synchronize()
    assert np.array_equal(h["filtered"], d["filtered"].cpu().numpy())


def test_serving_filters_match_alone(tv):
    job = syn.config0().jobs[0]
    bank = _bank(job.dt, job.K, job.edges)
    with tv.Plan(0) as p:
        alone = p.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=bank)
        t, out = p.submit(job.f, job.dt, job.K, job.n_inner, job.edges, filters=bank)
        assert p.wait(t, 60000) == tv.OK
    assert np.array_equal(alone["filtered"], out["filtered"])


def test_invalid_filters_rejected_and_plan_usable(plan, tv):
    job = syn.config0().jobs[0]
    bad = [(np.full(job.K - 1, np.nan), 0.0)]
    with pytest.raises(tv.TvSpecError):
        plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=bad)
    too_many = [(np.ones(job.K - 1), 1.0)] * 65
    with pytest.raises(tv.TvSpecError):
        plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=too_many)
    g = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, filters=[(np.ones(job.K - 1), 1.0)])
    assert np.isfinite(g["filtered"]).all()
