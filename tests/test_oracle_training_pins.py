"""Pins of the oracle's training-sample preparation (Sec. 4.1: crops, downsampling by 2,
standardisation of the data set), against closed forms, numpy and invariants."""
import numpy as np
import pytest

import oracle
import synthetic as syn

INF = float("inf")


def test_plain_crop_is_the_window():
    rng = np.random.default_rng(1)
    src = rng.normal(size=(37, 53)).astype(np.float32)
    for (y, x, n) in [(0, 0, 8), (5, 11, 16), (37 - 9, 53 - 9, 9), (3, 40, 13)]:
        c = oracle.crop(src, y, x, n, 1)
        assert np.array_equal(c, src[y:y + n, x:x + n].astype(np.float64))


def test_downsampled_crop_of_a_bilinear_field_is_its_centre_value():
    # the average of a + b i + c j + d i j over an s x s block is its value at the block centre
    H, W = 40, 44
    i = np.arange(H, dtype=np.float64)[:, None]
    j = np.arange(W, dtype=np.float64)[None, :]
    fn = lambda ii, jj: 3.0 + 2.0 * ii - jj + 0.5 * ii * jj
    src = fn(i, j)
    y, x, n = 3, 6, 8
    c2 = oracle.crop(src, y, x, n, 2)
    ii = np.arange(n, dtype=np.float64)[:, None]
    jj = np.arange(n, dtype=np.float64)[None, :]
    assert np.array_equal(c2, fn(y + 2 * ii + 0.5, x + 2 * jj + 0.5))  # all values exact
    c3 = oracle.crop(src, y, x, n, 3)
    want = fn(y + 3 * ii + 1.0, x + 3 * jj + 1.0)
    assert np.allclose(c3, want, rtol=2e-7, atol=0)


def test_downsampled_crop_matches_block_mean_and_kills_a_checkerboard():
    rng = np.random.default_rng(2)
    src = rng.uniform(-1, 1, (70, 90)).astype(np.float32)
    y, x, n = 4, 9, 16
    win = src[y:y + 2 * n, x:x + 2 * n].astype(np.float64)
    want = win.reshape(n, 2, n, 2).mean(axis=(1, 3)).astype(np.float32).astype(np.float64)
    assert np.max(np.abs(oracle.crop(src, y, x, n, 2) - want)) <= 1e-7 * np.max(np.abs(want))
    cb = np.where((np.arange(32)[:, None] + np.arange(32)[None, :]) % 2 == 0, 1.0, -1.0)
    assert np.array_equal(oracle.crop(cb, 0, 0, 16, 2), np.zeros((16, 16)))


def test_crop_window_outside_is_rejected():
    src = np.zeros((20, 20))
    for args in [(0, 0, 11, 2), (-1, 0, 4, 1), (0, 17, 4, 1), (10, 10, 6, 2)]:
        with pytest.raises(ValueError):
            oracle.crop(src, *args)


def test_dataset_standardisation_matches_numpy_mean_and_population_std():
    rng = np.random.default_rng(3)
    x = rng.normal(0.7, 2.5, (6, 12, 12)).astype(np.float32)
    out, ms = oracle.standardize(x, 1)
    xd = x.astype(np.float64)
    assert abs(ms[0] - xd.mean()) <= 1e-12 * abs(xd.mean())
    assert abs(ms[1] - xd.std()) <= 1e-12 * xd.std()          # ddof = 0
    assert abs(out.mean()) < 1e-6 and abs(out.std() - 1.0) < 1e-6
    # per-pixel: (x - mean) / std rounded to float32
    want = ((xd - ms[0]) / ms[1]).astype(np.float32).astype(np.float64)
    assert np.array_equal(out, want)


def test_per_image_standardisation():
    rng = np.random.default_rng(4)
    x = np.stack([rng.normal(m, s, (10, 10)) for m, s in [(0, 1), (5, 0.1), (-3, 7)]]).astype(np.float32)
    out, ms = oracle.standardize(x, 2)
    for c in range(3):
        xd = x[c].astype(np.float64)
        assert abs(ms[2 * c] - xd.mean()) <= 1e-12 * max(1.0, abs(xd.mean()))
        assert abs(ms[2 * c + 1] - xd.std()) <= 1e-12 * xd.std()
        assert abs(out[c].mean()) < 1e-6 and abs(out[c].std() - 1.0) < 1e-6


def test_given_statistics_and_degenerate_cases():
    x = np.arange(32, dtype=np.float32).reshape(2, 4, 4)
    out, ms = oracle.standardize(x, 3, (10.0, 4.0))
    assert np.array_equal(out, (x.astype(np.float64) - 10.0) / 4.0)
    const = np.full((2, 5, 5), 0.25, np.float32)
    out, ms = oracle.standardize(const, 2)
    assert np.array_equal(out, np.zeros_like(out)) and ms[1] == 0.0
    out, _ = oracle.standardize(x, 0)
    assert np.array_equal(out, x.astype(np.float64))


def test_standardisation_is_affine_invariant():
    rng = np.random.default_rng(5)
    x = rng.uniform(0, 1, (4, 9, 9)).astype(np.float32)
    a, _ = oracle.standardize(x, 1)
    b, _ = oracle.standardize((3.0 * x.astype(np.float64) + 0.5), 1)
    assert np.max(np.abs(a - b)) < 1e-6


def test_training_set_is_the_decomposition_of_the_standardised_crops():
    srcs = [syn.make_image(96, 80, 8, (3.0, 14.0), (0.1, 1.0), 0.02, seed=s) for s in (11, 12)]
    crops = [(0, 3, 5, 1), (1, 10, 2, 2), (0, 40, 30, 1), (1, 0, 0, 2)]
    size, K, n_inner = 24, 6, 40
    ts = oracle.training_set(srcs, crops, size, 1, 0.5, K, n_inner, syn.DYADIC_EDGES)
    assert ts["crops"].shape == (4, size, size) and ts["bands"].shape == (4, 6, size, size)
    raw = np.stack([oracle.crop(srcs[c[0]], c[1], c[2], size, c[3]) for c in crops])
    x, ms = oracle.standardize(raw, 1)
    assert np.array_equal(ts["crops"], x) and np.array_equal(ts["mean_std"], ms)
    for i in range(4):
        r = oracle.decompose(x[i], 0.5, K, n_inner, syn.DYADIC_EDGES)
        assert np.array_equal(ts["bands"][i], r["bands"])
        assert np.array_equal(ts["S"][i], r["S"])
        recon = ts["bands"][i].sum(axis=0) + ts["residual"][i]
        assert np.max(np.abs(recon - x[i])) < 1e-10
