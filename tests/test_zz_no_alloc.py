"""tvspec_decompose_noalloc: the entry point for callers that cannot allocate device memory.

Such callers (a thread working while another one captures a CUDA graph in global mode,
real-time loops that cannot take the synchronisation an allocation may cause, frameworks that
own all device memory) pass device buffers for the image and the outputs only; the library
takes its workspace from one fixed device array. This file is collected last so that a
failure here does not stop a run before the other tests.
"""
import numpy as np
import pytest

import synthetic as syn
from tolerances import BAND_INF, BAND_REL_L2, RECON_INF

pytestmark = pytest.mark.gpu


def _close(out, ref, f):
    mf = float(np.abs(f).max())
    b = out["bands"].cpu().numpy().astype(np.float64)
    rb = ref["bands"].cpu().numpy().astype(np.float64)
    assert np.abs(b - rb).max() <= BAND_INF * mf
    if np.linalg.norm(rb) > 0:
        assert np.linalg.norm(b - rb) / np.linalg.norm(rb) <= BAND_REL_L2
    r = out["residual"].cpu().numpy().astype(np.float64)
    rr = ref["residual"].cpu().numpy().astype(np.float64)
    assert np.abs(r - rr).max() <= BAND_INF * mf
    assert np.abs(b.sum(0) + r - f).max() <= RECON_INF * mf
    S = out["S"].cpu().numpy()
    rS = ref["S"].cpu().numpy()
    assert np.abs(S - rS).max() <= 1e-3 * max(np.abs(rS).max(), 1e-300)


def test_noalloc_matches_plan_path_on_two_calls_in_a_row():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_10004_gb300 as tv

    a = syn.config1(K=12).jobs[0]                     # 512 x 512, 300 iterations per step
    b_img = syn.make_image(100, 37, 5, (2.0, 9.0), (0.1, 1.0), 0.02, seed=5)
    cases = [(a.f, a.dt, a.K, a.n_inner, a.edges), (b_img, 0.25, 6, 25, syn.DYADIC_EDGES)]
    dev = [torch.from_numpy(c[0]).cuda() for c in cases]
    with tv.Plan(0) as plan:
        refs = [plan.decompose(x, *c[1:]) for x, c in zip(dev, cases)]
        torch.cuda.synchronize()
    # the two no-allocation calls back to back: the second finds the first one's leftovers
    outs = [tv.decompose_noalloc(x, *c[1:]) for x, c in zip(dev, cases)]
    torch.cuda.synchronize()
    for out, ref, c in zip(outs, refs, cases):
        _close(out, ref, c[0].astype(np.float64))


def test_noalloc_rejects_images_beyond_its_array():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2006_10004_gb300 as tv

    f = torch.zeros((2048, 2048), dtype=torch.float32, device="cuda")
    with pytest.raises(tv.TvSpecError) as ei:
        tv.decompose_noalloc(f, 0.5, 4, 10, syn.DYADIC_EDGES)
    assert ei.value.status == tv.EINVAL and "48 MiB" in str(ei.value)
