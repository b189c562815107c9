"""Ground-truth generation for training (Sec. 4.1) through tvspec_training_set vs the oracle.

Crops (plain and downsampled by 2), standardisation (none, over the data set, per crop, given)
and the decompositions of all crops in one call, compared with the FP64 oracle's
``training_set``; and bit-identity with the plain path on the returned crops.
"""
import numpy as np
import pytest

import oracle
import synthetic as syn
from tolerances import BAND_INF, BAND_REL_L2, RECON_INF, assert_parity

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


def _sources(seed=0):
    return [syn.make_image(H, W, max(1, H * W // 4000), (2.0, 24.0), (0.05, 1.0), 0.02, seed=seed + i)
            for i, (H, W) in enumerate([(200, 240), (150, 310), (260, 180)])]


def _crops(sources, n, size, seed, scales=(1, 2)):
    rng = np.random.default_rng(seed)
    out = []
    for c in range(n):
        s = int(scales[c % len(scales)])
        i = int(rng.integers(0, len(sources)))
        H, W = sources[i].shape
        out.append((i, int(rng.integers(0, H - s * size + 1)), int(rng.integers(0, W - s * size + 1)), s))
    return out


def _ulp_close(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return np.all(np.abs(a - b) <= 2.0 ** -23 * np.abs(b) + 1e-37)


def _check_decomp(g, ref):
    """Every crop within the parity bars; the reconstruction against the GPU's own input."""
    for i in range(ref["bands"].shape[0]):
        gi = {k: np.asarray(g[k][i]) for k in ("bands", "residual", "S")}
        ri = {k: ref[k][i] for k in ("bands", "residual", "S")}
        assert_parity(gi, ri, np.asarray(g["crops"][i], np.float64), f"crop {i}")


@pytest.mark.parametrize("mode", [0, 1, 2, 3])
def test_training_set_parity(plan, mode):
    srcs = _sources(10 * mode)
    crops = _crops(srcs, 40, 32, seed=mode)
    K, n_inner = 8, 40
    ms = (0.3, 0.25)
    g = plan.training_set(srcs, crops, 32, mode, 0.5, K, n_inner, syn.DYADIC_EDGES, mean_std=ms)
    ref = oracle.training_set(srcs, crops, 32, mode, 0.5, K, n_inner, syn.DYADIC_EDGES, mean_std=ms)
    if mode in (0, 3):
        assert np.array_equal(np.asarray(g["crops"], np.float64), ref["crops"])
    else:
        assert _ulp_close(g["crops"], ref["crops"])
        assert np.allclose(g["stats"], ref["mean_std"], rtol=1e-12, atol=1e-15)
    _check_decomp(g, ref)


def test_training_set_equals_plain_decomposition_of_its_crops(plan):
    srcs = _sources(3)
    crops = _crops(srcs, 36, 24, seed=5)
    g = plan.training_set(srcs, crops, 24, 1, 0.5, 6, 30, syn.DYADIC_EDGES)
    for i in (0, 7, 35):
        a = plan.decompose(g["crops"][i], 0.5, 6, 30, syn.DYADIC_EDGES)
        assert np.array_equal(a["bands"], g["bands"][i])
        assert np.array_equal(a["residual"], g["residual"][i])
        assert np.array_equal(a["S"], g["S"][i])


def test_training_set_device_matches_host(plan):
    import torch

    srcs = _sources(4)
    crops = _crops(srcs, 33, 16, seed=6)
    h = plan.training_set(srcs, crops, 16, 2, 0.5, 5, 20, syn.DYADIC_EDGES)
    d = plan.training_set([torch.from_numpy(s).cuda() for s in srcs], crops, 16, 2, 0.5, 5, 20, syn.DYADIC_EDGES)
    torch.cuda.synchronize()
    for k in ("crops", "bands", "residual", "S"):
        assert np.array_equal(h[k], d[k].cpu().numpy()), k
    assert np.array_equal(h["stats"], d["stats"])


def test_small_batch_uses_the_tiled_path_and_matches_oracle(plan):
    srcs = _sources(7)
    crops = _crops(srcs, 5, 48, seed=8)
    g = plan.training_set(srcs, crops, 48, 1, 0.5, 6, 30, syn.DYADIC_EDGES)
    ref = oracle.training_set(srcs, crops, 48, 1, 0.5, 6, 30, syn.DYADIC_EDGES)
    assert _ulp_close(g["crops"], ref["crops"])
    _check_decomp(g, ref)


def test_full_size_training_batch_sampled_parity(plan):
    # the paper's setting: 64x64 crops (a third from 128x128 windows downsampled by 2),
    # standardised over the data set, K = 50 steps of dt = .5, 300 iterations, 6 dyadic bands
    srcs = [syn.make_image(512, 512, 40, (2.0, 60.0), (0.05, 1.0), 0.02, seed=90 + i) for i in range(4)]
    crops = _crops(srcs, 600, 64, seed=9, scales=(1, 1, 2))
    g = plan.training_set(srcs, crops, 64, 1, 0.5, 50, 300, syn.DYADIC_EDGES)
    x = np.asarray(g["crops"], np.float64)
    assert abs(x.mean()) < 1e-5 and abs(x.std() - 1.0) < 1e-5
    recon = np.asarray(g["bands"], np.float64).sum(axis=1) + g["residual"]
    assert np.max(np.abs(recon - x)) / np.max(np.abs(x)) <= RECON_INF * 10
    for i in (0, 301, 599):
        ref = oracle.decompose(x[i], 0.5, 50, 300, syn.DYADIC_EDGES)
        scale = float(np.max(np.abs(x[i])))
        assert np.max(np.abs(g["bands"][i] - ref["bands"])) / scale <= BAND_INF
        rel = np.linalg.norm(g["bands"][i] - ref["bands"]) / np.linalg.norm(ref["bands"])
        assert rel <= BAND_REL_L2, rel


def test_training_set_rejects_bad_windows(plan, tv):
    srcs = _sources(1)
    H, W = srcs[0].shape
    for bad in [(0, H - 31, 0, 1), (0, 0, 0, 0), (3, 0, 0, 1), (0, 0, W - 60, 2), (0, -1, 0, 1)]:
        with pytest.raises(tv.TvSpecError) as ei:
            plan.training_set(srcs, [bad], 32, 1, 0.5, 4, 10, syn.DYADIC_EDGES)
        assert ei.value.status == tv.EINVAL
    with pytest.raises(tv.TvSpecError):
        plan.training_set(srcs, [(0, 0, 0, 1)], 32, 3, 0.5, 4, 10, syn.DYADIC_EDGES, mean_std=(0.0, float("nan")))
    g = plan.training_set(srcs, [(0, 0, 0, 1)], 32, 2, 0.5, 4, 10, syn.DYADIC_EDGES)
    assert np.isfinite(g["bands"]).all()
