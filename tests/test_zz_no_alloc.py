"""tvspec_decompose_noalloc: the entry point for callers that cannot allocate device memory.

Some callers may not call cudaMalloc (or anything that allocates device memory) where they
run: a thread that works while another thread captures a CUDA graph in global mode (an
allocation anywhere in the process is then an error that also spoils that capture), real-time
loops that cannot take the device synchronisation an allocation may cause, and frameworks that
own all device memory. They pass device buffers for the image and the outputs only; the
library takes its workspace from one fixed device array. These tests check that the results
equal the plan path's bit for bit on two calls in a row (the second finds the first one's
leftovers in the array), agree with the oracle, that a call allocates nothing, and that it
runs beside another thread's global-mode graph capture. This file is collected last so that a
failure here does not stop a run before the other tests.
"""
import threading

import numpy as np
import pytest

import oracle
import synthetic as syn
from tolerances import BAND_INF, BAND_REL_L2, RECON_INF, U_INF

pytestmark = pytest.mark.gpu


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


def _cases():
    a = syn.config1(K=12).jobs[0]                     # 512 x 512, 300 iterations per step
    b_img = syn.make_image(100, 37, 5, (2.0, 9.0), (0.1, 1.0), 0.02, seed=5)
    return [(a.f, a.dt, a.K, a.n_inner, a.edges), (b_img, 0.25, 6, 25, syn.DYADIC_EDGES)]


def _np(out):
    return {k: out[k].cpu().numpy() for k in ("bands", "residual", "S")}


def _assert_equal(got, ref):
    for k in ("bands", "residual", "S"):
        assert got[k].shape == ref[k].shape, k
        assert np.array_equal(got[k], ref[k]), (k, float(np.abs(got[k].astype(np.float64) - ref[k]).max()))


def test_noalloc_matches_plan_path_on_two_calls_in_a_row():
    torch = _torch()
    import paper_2006_10004_gb300 as tv

    cases = _cases()
    dev = [torch.from_numpy(c[0]).cuda() for c in cases]
    with tv.Plan(0) as plan:
        refs = [_np(plan.decompose(x, *c[1:])) for x, c in zip(dev, cases)]
        torch.cuda.synchronize()
    # the two no-allocation calls back to back: the second finds the first one's leftovers
    outs = [tv.decompose_noalloc(x, *c[1:]) for x, c in zip(dev, cases)]
    torch.cuda.synchronize()
    for out, ref in zip(outs, refs):
        _assert_equal(_np(out), ref)   # same per-pixel operations as the plan path: same bits
    # and again in the other order
    outs = [tv.decompose_noalloc(x, *c[1:]) for x, c in reversed(list(zip(dev, cases)))]
    torch.cuda.synchronize()
    for out, ref in zip(outs, reversed(refs)):
        _assert_equal(_np(out), ref)


def test_noalloc_small_case_matches_the_oracle():
    torch = _torch()
    import paper_2006_10004_gb300 as tv

    f, dt, K, n_inner, edges = _cases()[1]
    got = _np(tv.decompose_noalloc(torch.from_numpy(f).cuda(), dt, K, n_inner, edges))
    ref = oracle.decompose(f, dt, K, n_inner, edges)
    mf = float(np.abs(f).max())
    b = got["bands"].astype(np.float64)
    assert np.abs(b - ref["bands"]).max() <= BAND_INF * mf
    assert np.linalg.norm(b - ref["bands"]) <= BAND_REL_L2 * np.linalg.norm(ref["bands"])
    assert np.abs(got["residual"] - ref["residual"]).max() <= U_INF * mf
    assert np.abs(b.sum(0) + got["residual"] - f).max() <= RECON_INF * mf
    assert np.abs(got["S"] - ref["S"]).max() <= 1e-3 * np.abs(ref["S"]).max()


def test_noalloc_allocates_nothing():
    torch = _torch()
    import paper_2006_10004_gb300 as tv

    f, dt, K, n_inner, edges = _cases()[1]
    x = torch.from_numpy(f).cuda()
    out = {"bands": torch.empty((len(edges) - 1,) + f.shape, dtype=torch.float32, device="cuda"),
           "residual": torch.empty(f.shape, dtype=torch.float32, device="cuda"),
           "S": torch.empty((K - 1,), dtype=torch.float64, device="cuda")}
    tv.decompose_noalloc(x, dt, K, n_inner, edges, out=out)       # loads the module and kernels
    torch.cuda.synchronize()
    first = _np(out)
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    reserved0 = torch.cuda.memory_reserved()
    for _ in range(3):
        tv.decompose_noalloc(x, dt, K, n_inner, edges, out=out)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)
    assert torch.cuda.memory_allocated() == alloc0
    assert torch.cuda.memory_reserved() == reserved0
    _assert_equal(_np(out), first)


def test_noalloc_runs_beside_another_threads_global_graph_capture():
    torch = _torch()
    import paper_2006_10004_gb300 as tv

    f, dt, K, n_inner, edges = _cases()[1]
    x = torch.from_numpy(f).cuda()
    with tv.Plan(0) as plan:
        ref = _np(plan.decompose(x, dt, K, n_inner, edges))
    out = {"bands": torch.empty((len(edges) - 1,) + f.shape, dtype=torch.float32, device="cuda"),
           "residual": torch.empty(f.shape, dtype=torch.float32, device="cuda"),
           "S": torch.empty((K - 1,), dtype=torch.float64, device="cuda")}
    tv.decompose_noalloc(x, dt, K, n_inner, edges, out=out)       # first call: before any capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    a = torch.ones(1 << 16, device="cuda")
    b = torch.empty_like(a)
    capturing, called = threading.Event(), threading.Event()
    errors = []

    def worker():
        try:
            assert capturing.wait(60)
            tv.decompose_noalloc(x, dt, K, n_inner, edges, stream=side, out=out)
        except BaseException as e:  # reported by the main thread
            errors.append(e)
        finally:
            called.set()

    t = threading.Thread(target=worker)
    t.start()
    g = torch.cuda.CUDAGraph()
    try:
        with torch.cuda.graph(g, capture_error_mode="global"):
            b.copy_(a * 3.0)
            capturing.set()
            assert called.wait(120)
    finally:
        capturing.set()
        t.join(120)
    assert not errors, errors
    g.replay()
    side.synchronize()
    torch.cuda.synchronize()
    assert torch.equal(b, a * 3.0)
    _assert_equal(_np(out), ref)


def test_noalloc_rejects_images_beyond_its_array():
    torch = _torch()
    import paper_2006_10004_gb300 as tv

    f = torch.zeros((2048, 2048), dtype=torch.float32, device="cuda")
    with pytest.raises(tv.TvSpecError) as ei:
        tv.decompose_noalloc(f, 0.5, 4, 10, syn.DYADIC_EDGES)
    assert ei.value.status == tv.EINVAL and "48 MiB" in str(ei.value)


def test_noalloc_rejects_host_buffers_before_enqueueing_anything():
    torch = _torch()
    import paper_2006_10004_gb300 as tv

    L = tv.load()
    H, W, K = 8, 8, 4
    e = np.ascontiguousarray(syn.DYADIC_EDGES, dtype=np.float64)
    f_host = np.zeros((H, W), np.float32)
    bands = torch.empty((len(e) - 1, H, W), dtype=torch.float32, device="cuda")
    residual = torch.empty((H, W), dtype=torch.float32, device="cuda")
    S = torch.empty((K - 1,), dtype=torch.float64, device="cuda")
    st = L.tvspec_decompose_noalloc(f_host.ctypes.data, H, W, 0.5, K, 5, e.ctypes.data, len(e),
                                    bands.data_ptr(), residual.data_ptr(), S.data_ptr(), None)
    assert st == tv.EINVAL
    assert b"device memory" in L.tvspec_last_error()
