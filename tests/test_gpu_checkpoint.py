"""Checkpoint / resume (tvspec_decompose_steps): a decomposition stopped after any ROF step,
its state held in host memory and resumed, in the same plan or another one of the same
configuration, gives the bits of the uninterrupted run; the state is tied to its request,
configuration and step."""
import numpy as np
import pytest

import oracle
import synthetic as syn
from tolerances import assert_parity

pytestmark = pytest.mark.gpu


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


def _same(a, b, keys=("bands", "residual", "S")):
    for k in keys:
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k


def _resumed(plan, args, cuts, **kw):
    K = args[2]
    state = None
    edges = [0] + list(cuts) + [K]
    out = None
    for k0, k1 in zip(edges[:-1], edges[1:]):
        out, state = plan.decompose_steps(*args, k0, k1, state=state, **kw)
    return out


@pytest.mark.parametrize("H,W", [(130, 170), (64, 64), (1, 33), (301, 97)])
def test_resumed_run_is_bit_identical(tv, H, W):
    f = _img(H, W, H + W)
    args = (f, 0.5, 12, 40, syn.DYADIC_EDGES)
    with tv.Plan(0) as p:
        whole = p.decompose(*args, trace=True)
        for cuts in ([1], [5], [1, 2, 3], [11], [4, 9]):
            _same(_resumed(p, args, cuts, trace=True), whole, ("bands", "residual", "S", "u"))
        # one call over all steps is the plain run too
        out, st = p.decompose_steps(*args, 0, 12)
        assert st is None
        _same(out, whole)


def test_resume_in_another_plan_with_another_launch_parity(tv):
    # 40 iterations: 5 launches per step at depth 8 (tile 24), 10 at depth 4 (tiles 4 and 26,
    # whose 6-iteration halo runs 4 per launch, a multiple of the fold interval): the copy of p
    # a step reads differs, the resumed run must move it
    f = _img(150, 140, 3)
    args = (f, 0.5, 9, 40, syn.DYADIC_EDGES)
    with tv.Plan(0) as p:
        whole = p.decompose(*args)
    for a, b in ((24, 4), (4, 26), (26, 24)):
        with tv.Plan(0, kernel=tv.KERNEL_TILED, tile=a) as pa, tv.Plan(0, kernel=tv.KERNEL_TILED, tile=b) as pb:
            _, st = pa.decompose_steps(*args, 0, 3)
            _, st = pb.decompose_steps(*args, 3, 6, state=st)
            out, _ = pa.decompose_steps(*args, 6, 9, state=st)
        _same(out, whole)


def test_filters_parseval_acc_mode_and_cold_start(tv):
    f = _img(96, 120, 9)
    K = 10
    bank = [(np.ones(K - 1), 1.0), (np.exp(-0.3 * np.arange(1, K)), 0.5)]
    args = (f, 0.25, K, 30, syn.DYADIC_EDGES)
    for cfg in (dict(), dict(acc_mode=1), dict(warm_start=0), dict(p_storage=tv.P_BF16)):
        with tv.Plan(0, **cfg) as p:
            whole = p.decompose(*args, filters=bank, parseval=True)
            out = _resumed(p, args, [2, 7], filters=bank, parseval=True)
        _same(out, whole, ("bands", "residual", "S", "filtered", "S_parseval"))


def test_resumed_run_matches_the_oracle(tv):
    job = syn.config0().jobs[0]
    args = (job.f, job.dt, job.K, job.n_inner, job.edges)
    with tv.Plan(0) as p:
        out = _resumed(p, args, [6, 13])
    ref = oracle.decompose(*args)
    assert_parity(out, ref, job.f, "config0 resumed")


def test_state_is_checked(tv):
    f = _img(80, 90, 5)
    args = (f, 0.5, 8, 20, syn.DYADIC_EDGES)
    with tv.Plan(0) as p:
        n = p.checkpoint_bytes(*args)
        _, st = p.decompose_steps(*args, 0, 4)
        assert st.nbytes == n
        for bad in ((args, 5, 8, st),                                    # saved at 4
                    ((f, 0.25, 8, 20, syn.DYADIC_EDGES), 4, 8, st),    # another dt
                    ((f, 0.5, 9, 20, syn.DYADIC_EDGES), 4, 9, st),     # another K
                    (args, 4, 8, None),                                  # no state
                    (args, 3, 3, st), (args, 0, 9, None)):              # bad ranges
            a, k0, k1, s = bad
            with pytest.raises(tv.TvSpecError) as ei:
                p.decompose_steps(*a, k0, k1, state=s)
            assert ei.value.status == tv.EINVAL
        corrupt = st.copy()
        corrupt[:8] = 0
        with pytest.raises(tv.TvSpecError):
            p.decompose_steps(*args, 4, 8, state=corrupt)
        out, _ = p.decompose_steps(*args, 4, 8, state=st)  # the plan is still usable
        _same(out, p.decompose(*args))
    with tv.Plan(0, acc_mode=1) as q:  # another configuration
        with pytest.raises(tv.TvSpecError) as ei:
            q.decompose_steps(*args, 4, 8, state=st)
        assert ei.value.status == tv.EINVAL


def test_device_memory_request(tv):
    import torch

    f = _img(70, 75, 6)
    args_h = (f, 0.5, 7, 25, syn.DYADIC_EDGES)
    args_d = (torch.from_numpy(f).cuda(), 0.5, 7, 25, syn.DYADIC_EDGES)
    with tv.Plan(0) as p:
        whole = p.decompose(*args_h)
        _, st = p.decompose_steps(*args_d, 0, 3)
        out, _ = p.decompose_steps(*args_d, 3, 7, state=st)
        torch.cuda.synchronize()
        assert np.array_equal(out["bands"].cpu().numpy(), whole["bands"])
        assert np.array_equal(out["S"].cpu().numpy() if hasattr(out["S"], "cpu") else out["S"], whole["S"])
