"""Write checks of every kernel that touches an image's workspace (compute-sanitizer is not
available): with test_guard_bytes each array of the workspace is fenced by guard regions of a
known content, checked after every call, across the launch forms, tile shapes, storage types,
epilogue modes, optional outputs, batches (tiled and resident), stepped and served runs. A
guard byte found changed fails the call; results must also equal the unguarded plan's."""
import numpy as np
import pytest

import synthetic as syn

pytestmark = pytest.mark.gpu
G = 512


@pytest.fixture(scope="module")
def tv():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_10004_gb300 as tvm

    tvm.load()
    return tvm


def _img(H, W, seed):
    return syn.make_image(H, W, 6, (2.0, 14.0), (0.1, 1.0), 0.02, seed)


def _same(a, b, keys=("bands", "residual", "S")):
    for k in keys:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


SIZES = [(1, 1), (19, 1), (37, 53), (200, 333)]


def test_every_tile_shape_and_the_reference_kernel(tv):
    for H, W in SIZES:
        f = _img(H, W, H * 3 + W)
        args = (f, 0.5, 4, 13, syn.DYADIC_EDGES)
        with tv.Plan(0) as p0:
            want = p0.decompose(*args, trace=True)
        with tv.Plan(0, kernel=tv.KERNEL_NAIVE, test_guard_bytes=G) as p:
            _same(p.decompose(*args, trace=True), want)
        for i, s in enumerate(tv.tile_shapes()):
            with tv.Plan(0, kernel=tv.KERNEL_TILED, tile=i, test_guard_bytes=G) as p:
                _same(p.decompose(*args, trace=True), want, ("bands", "residual", "S", "u"))


@pytest.mark.parametrize("cfg", [dict(p_storage=1), dict(p_storage=2), dict(p_storage=3),
                                 dict(acc_mode=1), dict(warm_start=0), dict(fast_math=0),
                                 dict(persistent=1), dict(use_graphs=0), dict(pdl=0)])
def test_configurations(tv, cfg):
    f = _img(150, 170, 4)
    K = 6
    bank = [(np.ones(K - 1), 1.0), (np.linspace(0, 1, K - 1), 0.0)]
    args = (f, 0.25, K, 20, syn.DYADIC_EDGES)
    with tv.Plan(0, **cfg) as p0:
        want = p0.decompose(*args, trace=True, filters=bank, parseval=True)
    with tv.Plan(0, test_guard_bytes=G, **cfg) as p:
        for _ in range(3):  # the third call replays a captured graph
            got = p.decompose(*args, trace=True, filters=bank, parseval=True)
    _same(got, want, ("bands", "residual", "S", "u", "filtered", "S_parseval"))


def test_batches_tiled_and_resident_and_device_memory(tv):
    import torch

    small = [(_img(40 + (i % 5) * 5, 64, 100 + i), 0.5, 5, 15, syn.DYADIC_EDGES) for i in range(36)]
    mixed = [(_img(60 + 17 * i, 90 + 11 * i, 200 + i), 0.5, 3 + i % 4, 18, syn.DYADIC_EDGES)
             for i in range(6)]
    for jobs in (small, mixed, small[:3] + mixed):
        with tv.Plan(0) as p0:
            want = p0.decompose_batch(jobs, parseval=True)
        with tv.Plan(0, test_guard_bytes=G) as p:
            got = p.decompose_batch(jobs, parseval=True)
            dev = p.decompose_batch([(torch.from_numpy(j[0]).cuda(),) + j[1:] for j in jobs])
            torch.cuda.synchronize()
        for a, b, d in zip(got, want, dev):
            _same(a, b, ("bands", "residual", "S", "S_parseval"))
            assert np.array_equal(d["bands"].cpu().numpy(), b["bands"])


def test_stepped_and_served_runs(tv):
    f = _img(120, 100, 7)
    args = (f, 0.5, 8, 20, syn.DYADIC_EDGES)
    with tv.Plan(0) as p0:
        want = p0.decompose(*args)
        plain_bytes = p0.stats()["workspace_bytes"]
    with tv.Plan(0, test_guard_bytes=G) as p:
        _, st = p.decompose_steps(*args, 0, 3)
        assert p.stats()["workspace_bytes"] >= plain_bytes + 20 * G  # the guards are there
        out, _ = p.decompose_steps(*args, 3, 8, state=st)
        _same(out, want)
        # the check itself: a state whose last byte (the workspace's trailing guard) was
        # changed on the host is restored, run, and caught
        bad = st.copy()
        bad[-1] ^= 0xFF
        with pytest.raises(tv.TvSpecError) as ei:
            p.decompose_steps(*args, 3, 8, state=bad)
        assert ei.value.status == tv.ECUDA and "guard" in str(ei.value)
        tickets = [p.submit(_img(50 + 30 * i, 70, 300 + i), 0.5, 4 + i, 15, syn.DYADIC_EDGES)
                   for i in range(5)] + [p.submit(*args)]
        for t, _ in tickets:
            assert p.wait(t, 120000) == tv.OK
        _same(tickets[-1][1], want)
