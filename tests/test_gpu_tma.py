"""Tile loads by the tensor memory accelerator (config `tma`): the dual iterations give the same
bits as the per-thread loads and the one-iteration reference kernel, for every shape that takes
them, at ragged sizes and at the bench size, alone, stepped and with the workspace guards on."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
TMA_SHAPES = (8, 24, 25)


@pytest.fixture(scope="module")
def tv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_10004_gb300 as tvm

    tvm.load()
    return tvm


def _img(H, W, seed):
    return syn.make_image(H, W, 8, (2.0, 20.0), (0.1, 1.0), 0.02, seed)


def _same(a, b, keys=("bands", "residual", "S", "u")):
    for k in keys:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


# (130, 70): edge-aligned tiles whose last column of tiles starts off the 4-float grid (per-thread
# loads instead); (97, 512), (136, 132): edge-aligned TMA boxes, the last at W - 64
@pytest.mark.parametrize("H,W", [(1, 1), (19, 1), (1, 130), (37, 53), (130, 70), (200, 333), (97, 512),
                                 (136, 132)])
def test_every_tma_shape_matches_the_reference_kernel(tv, H, W):
    f = _img(H, W, 5 * H + W)
    args = (f, 0.5, 5, 23, syn.DYADIC_EDGES)
    with tv.Plan(0, kernel=tv.KERNEL_NAIVE) as p:
        base = p.decompose(*args, trace=True)
    for s in TMA_SHAPES:
        for depth in sorted({4, tv.tile_shapes()[s]["TB"] // 4 * 4}):
            with tv.Plan(0, kernel=tv.KERNEL_TILED, tile=s, temporal_block=depth, tma=1,
                         test_guard_bytes=256) as p:
                _same(p.decompose(*args, trace=True), base)


def test_bench_image_autotuned_and_stepped(tv):
    job = syn.config1().jobs[0]
    args = (job.f, job.dt, 6, job.n_inner, job.edges)
    with tv.Plan(0) as p:
        want = p.decompose(*args, trace=True)
    with tv.Plan(0, tma=1) as p:
        for _ in range(3):  # plain, captured, replayed
            _same(p.decompose(*args, trace=True), want)
        _, st = p.decompose_steps(*args, 0, 2)
        out, _ = p.decompose_steps(*args, 2, 6, state=st)
        _same(out, want, ("bands", "residual", "S"))


def test_batches_and_other_storage_ignore_the_option(tv):
    jobs = [(_img(60 + 7 * i, 90, 40 + i), 0.5, 4, 20, syn.DYADIC_EDGES) for i in range(4)]
    with tv.Plan(0) as p0, tv.Plan(0, tma=1) as p1:
        for a, b in zip(p0.decompose_batch(jobs), p1.decompose_batch(jobs)):
            _same(a, b, ("bands", "residual", "S"))
    f = _img(100, 120, 3)
    with tv.Plan(0, p_storage=tv.P_BF16) as p0, tv.Plan(0, p_storage=tv.P_BF16, tma=1) as p1:
        _same(p0.decompose(f, 0.5, 4, 20, syn.DYADIC_EDGES), p1.decompose(f, 0.5, 4, 20, syn.DYADIC_EDGES),
              ("bands", "residual", "S"))
