"""CUDA path vs the FP64 oracle, through the C ABI (Python binding = marshalling only).

Parity bars are in ``tolerances.py``. Bit-identity tests check what the design promises:
the result of the float32 dual iterations does not depend on the tile shape, the iterations
per launch, graph replay, the memory mode, or the batch an image runs in.
"""
import math

import numpy as np
import pytest

import oracle
import synthetic as syn
from tolerances import assert_parity, parity_metrics

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


def _img(H, W, seed, n=6, r=(2.0, 12.0)):
    return syn.make_image(H, W, n, r, (0.1, 1.0), 0.02, seed)


def _same(a, b):
    for k in ("bands", "residual", "S"):
        assert np.array_equal(np.asarray(a[k]), np.asarray(b[k])), k
    if "u" in a and "u" in b:
        assert np.array_equal(np.asarray(a["u"]), np.asarray(b["u"])), "u"


# ---------------------------------------------------------------------------------------------
def test_config0_full_parity(plan):
    job = syn.config0().jobs[0]
    g = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, trace=True)
    ref = oracle.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, trace=True)
    m = assert_parity(g, ref, job.f, "config0")
    print("config0", m)


@pytest.mark.parametrize("H,W", [(37, 53), (130, 70), (1, 1), (1, 17), (19, 1), (2, 3), (65, 129),
                                 (200, 333)])
def test_ragged_sizes_parity(plan, H, W):
    f = _img(H, W, seed=H * 1000 + W)
    g = plan.decompose(f, 0.5, 6, 25, syn.DYADIC_EDGES, trace=True)
    ref = oracle.decompose(f, 0.5, 6, 25, syn.DYADIC_EDGES, trace=True)
    assert_parity(g, ref, f, f"{H}x{W}")


def test_constant_image_exact(plan):
    f = np.full((40, 70), 0.3, np.float32)
    g = plan.decompose(f, 0.5, 5, 40, syn.DYADIC_EDGES, trace=True)
    assert np.all(g["bands"] == 0) and np.all(g["S"] == 0)
    assert np.array_equal(g["residual"], f)
    assert np.all(g["u"] == np.float64(np.float32(0.3)))


def test_zero_inner_iterations(plan):
    f = _img(20, 30, 3)
    g = plan.decompose(f, 0.5, 4, 0, syn.DYADIC_EDGES)
    assert np.all(g["bands"] == 0) and np.all(g["S"] == 0)
    assert np.array_equal(g["residual"], f)


def test_band_edges_not_covering_time_range(plan):
    # a band set that starts after t_1 and ends before t_{K-1}: only the covered phi_k count
    f = _img(33, 41, 4)
    edges = (0.75, 1.5, 2.25)
    g = plan.decompose(f, 0.25, 14, 30, edges, trace=True)
    ref = oracle.decompose(f, 0.25, 14, 30, edges, trace=True)
    m = parity_metrics(g, ref, f)
    assert m["band_inf"] <= 1e-3 and m["u_inf"] <= 1e-4, m


# ---------------------------------------------------------------------------------------------
# bit-identity of the implementation choices
# ---------------------------------------------------------------------------------------------
# 100 x 150: edge-aligned tiles for the V = 2 shapes up to 100 rows, masked ones for V = 4 (150
# is not a multiple of 4) and the taller shapes; 120 x 200: edge-aligned for V = 2 and V = 4;
# 56 x 64: exactly one tile of the 64 x 56 shapes (all four borders in one tile)
@pytest.mark.parametrize("H,W", [(100, 150), (120, 200), (56, 64)])
def test_every_tile_shape_and_depth_bit_identical(tv, H, W):
    f = _img(H, W, 7 + H)
    args = (f, 0.5, 4, 23, syn.DYADIC_EDGES)
    with tv.Plan(0, kernel=tv.KERNEL_NAIVE) as p:
        base = p.decompose(*args, trace=True)
    for i, s in enumerate(tv.tile_shapes()):
        # iterations per launch: multiples of the compensated update's fold interval (4)
        for depth in sorted({4, s["TB"] // 4 * 4}):
            with tv.Plan(0, kernel=tv.KERNEL_TILED, tile=i, temporal_block=depth) as p:
                out = p.decompose(*args, trace=True)
                assert p.stats()["last_tile"] == i
            _same(out, base)


# 1000 x 1100: edge-aligned tiles for every shape; 1001 x 999 (odd width): masked border tiles
@pytest.mark.parametrize("H,W", [(1000, 1100), (1001, 999)])
def test_many_waves_of_tiles_bit_identical_and_parity(tv, H, W):
    # an image with many more tiles than the GPU holds at once: later tiles read halos that
    # earlier tiles of the same launch have already finished (the ping-pong copies of p must
    # make that irrelevant), and the run must be reproducible
    f = syn.make_image(H, W, 120, (2.0, 60.0), (0.05, 1.0), 0.02, seed=77 + H - 1000)
    args = (f, 0.5, 3, 40, syn.DYADIC_EDGES)
    with tv.Plan(0, kernel=tv.KERNEL_NAIVE) as p:
        base = p.decompose(*args, trace=True)
    for tile in (0, 5, 8, 10, 11, 24):  # 8 and 24: the shapes the autotuner picks for large and 512^2 images
        with tv.Plan(0, kernel=tv.KERNEL_TILED, tile=tile) as p:
            a = p.decompose(*args, trace=True)
            b = p.decompose(*args, trace=True)
        _same(a, base)
        _same(b, base)
    ref = oracle.decompose(*args, trace=True)
    assert_parity(base, ref, f, f"{H}x{W}")


def test_graph_and_plain_launches_bit_identical(tv):
    f = _img(90, 77, 8)
    args = (f, 0.5, 5, 31, syn.DYADIC_EDGES)
    with tv.Plan(0, use_graphs=1) as a, tv.Plan(0, use_graphs=0) as b:
        ra = a.decompose(*args, trace=True)   # first use: launched directly
        ra2 = a.decompose(*args, trace=True)  # second use: captured into a graph and replayed
        ra3 = a.decompose(*args, trace=True)  # replay
        rb = b.decompose(*args, trace=True)
        assert a.stats()["graph_launches"] == 2 and a.stats()["graphs_built"] == 1
        assert b.stats()["graph_launches"] == 0
    _same(ra, rb)
    _same(ra, ra2)
    _same(ra, ra3)


def test_programmatic_dependent_launch_bit_identical(tv):
    f = _img(160, 140, 10)
    args = (f, 0.5, 5, 37, syn.DYADIC_EDGES)
    with tv.Plan(0, pdl=1) as a, tv.Plan(0, pdl=0) as b:
        _same(a.decompose(*args, trace=True), b.decompose(*args, trace=True))


@pytest.mark.parametrize("H,W", [(64, 64), (1, 1), (1, 17), (19, 1), (37, 53), (100, 37), (40, 70),
                                 (64, 128), (128, 64), (63, 127)])
@pytest.mark.parametrize("warm", [1, 0])
def test_resident_small_image_kernel_bit_identical(tv, H, W, warm):
    # the whole decomposition in one CTA vs one launch per block and step
    f = _img(H, W, 7 * H + W)
    args = (f, 0.5, 6, 27, syn.DYADIC_EDGES)
    with tv.Plan(0, resident=2, warm_start=warm) as a, tv.Plan(0, resident=0, warm_start=warm) as b:
        ra = a.decompose(*args, trace=True)
        assert a.stats()["kernel_launches"] == 1  # one launch for the whole decomposition
        _same(ra, b.decompose(*args, trace=True))
    ref = oracle.decompose(*args, trace=True, warm_start=bool(warm))
    assert_parity(ra, ref, f, f"resident {H}x{W}")


def test_every_resident_variant_bit_identical(tv):
    # every thread layout of the resident kernel that holds the image gives the per-step bits
    shapes = [(64, 64), (33, 50), (7, 64), (64, 5), (120, 60), (60, 120)]
    imgs = {s: _img(*s, seed=13 * s[0] + s[1]) for s in shapes}
    with tv.Plan(0, resident=0) as b:
        want = {s: b.decompose(f, 0.5, 5, 23, syn.DYADIC_EDGES, trace=True) for s, f in imgs.items()}
    for v, info in enumerate(tv.resident_variants()):
        with tv.Plan(0, resident=2, resident_variant=v) as a:
            for s, f in imgs.items():
                if s[0] <= info["max_H"] and s[1] <= info["max_W"]:
                    _same(a.decompose(f, 0.5, 5, 23, syn.DYADIC_EDGES, trace=True), want[s])


def test_resident_batch_of_crops(tv):
    # the training-data use: many 64^2 crops, K = 50, dyadic bands, in one launch (the default
    # chooses the resident kernel from 32 eligible images on)
    jobs = [(_img(64, 64, 300 + j), 0.5, 50, 60, syn.DYADIC_EDGES) for j in range(40)]
    with tv.Plan(0) as p:
        outs = p.decompose_batch(jobs)
        assert p.stats()["kernel_launches"] == 1
    with tv.Plan(0) as p:
        p.decompose_batch(jobs[:8])
        assert p.stats()["kernel_launches"] > 1  # too few images: per-step path
    for job, out in zip(jobs[:3], outs[:3]):
        assert_parity(out, oracle.decompose(*job), job[0], "crop")


@pytest.mark.parametrize("persistent", [1, 2])
def test_persistent_step_kernel_bit_identical(tv, persistent):
    # one cooperative launch per step (tiles resident; grid barriers, or waits on the
    # neighbouring tiles' progress only) vs one launch per block
    for H, W in [(256, 300), (512, 512), (37, 53), (1, 700), (700, 1)]:
        f = _img(H, W, 11 + H)
        args = (f, 0.5, 4, 41, syn.DYADIC_EDGES)
        with tv.Plan(0, persistent=persistent) as a, tv.Plan(0, persistent=0) as b:
            got = a.decompose(*args, trace=True)
            n0 = a.stats()["kernel_launches"]
            again = a.decompose(*args, trace=True)
            # one dual-iteration launch per step (+ the two epilogue parts, + the init)
            assert a.stats()["kernel_launches"] - n0 <= 3 * 4 + 1
            _same(got, b.decompose(*args, trace=True))
            _same(again, got)


@pytest.mark.parametrize("tile", [5, 11, 14, 20, 24, 26])
def test_neighbour_synchronised_kernel_every_depth_bit_identical(tv, tile):
    # the neighbour-flag persistent kernel against the reference kernel for several tile
    # shapes and depths, on an image with many tiles and ragged edges; the flags must also
    # carry over from step to step within a decomposition (epochs keep increasing)
    f = _img(300, 413, 5 + tile)
    args = (f, 0.5, 5, 29, syn.DYADIC_EDGES)
    with tv.Plan(0, kernel=tv.KERNEL_NAIVE) as p:
        base = p.decompose(*args, trace=True)
    s = tv.tile_shapes()[tile]
    for depth in sorted({4, s["TB"] // 4 * 4}):
        with tv.Plan(0, kernel=tv.KERNEL_TILED, tile=tile, temporal_block=depth, persistent=2) as p:
            _same(p.decompose(*args, trace=True), base)
            _same(p.decompose(*args, trace=True), base)  # graph replay: flags cleared per run


@pytest.mark.parametrize("persistent", [1, 2])
def test_persistent_barrier_timeout_is_reported_and_plan_recovers(tv, persistent):
    # fault injection on the host side of the contract: one CTA never arrives at its barrier
    # (or never publishes its progress), the others give up after the bounded wait and the
    # call reports TVSPEC_ETIMEOUT; the device stays usable
    f = _img(200, 200, 12)
    with tv.Plan(0, persistent=persistent, barrier_timeout_ms=20, test_barrier_noshow=0) as p:
        with pytest.raises(tv.TvSpecError) as ei:
            p.decompose(f, 0.5, 3, 30, syn.DYADIC_EDGES)
        assert ei.value.status == tv.ETIMEOUT
    with tv.Plan(0) as p:
        out = p.decompose(f, 0.5, 3, 30, syn.DYADIC_EDGES)
    ref = oracle.decompose(f, 0.5, 3, 30, syn.DYADIC_EDGES)
    assert_parity(out, ref, f, "after timeout")


def test_device_and_host_memory_bit_identical(plan):
    import torch

    f = _img(64, 96, 9)
    h = plan.decompose(f, 0.5, 6, 30, syn.DYADIC_EDGES, trace=True)
    ft = torch.from_numpy(f).cuda()
    d = plan.decompose(ft, 0.5, 6, 30, syn.DYADIC_EDGES, trace=True)
    torch.cuda.synchronize()
    _same(h, {k: v.cpu().numpy() for k, v in d.items()})


def test_batch_matches_alone_bit_identical_and_oracle(plan):
    rng = np.random.default_rng(11)
    jobs = []
    for j in range(7):
        H, W = int(rng.integers(20, 140)), int(rng.integers(20, 140))
        K = int(rng.integers(3, 9))
        dt = float(rng.choice([0.25, 0.5, 1.0]))
        jobs.append((_img(H, W, 100 + j), dt, K, 30, syn.DYADIC_EDGES))
    outs = plan.decompose_batch(jobs, trace=True)
    for job, out in zip(jobs, outs):
        alone = plan.decompose(*job, trace=True)
        _same(out, alone)
        ref = oracle.decompose(*job, trace=True)
        assert_parity(out, ref, job[0])


def test_device_batch_copy_list_matches_host_batch(plan):
    # device batches move inputs and outputs with one copy-list launch each; the inputs here are
    # views into one flat buffer at offsets that are not 16-byte aligned
    import torch

    rng = np.random.default_rng(12)
    imgs = [_img(int(rng.integers(5, 90)), int(rng.integers(5, 90)), 200 + j) for j in range(9)]
    flat = torch.zeros(sum(x.size for x in imgs) + 3 * len(imgs) + 1, dtype=torch.float32, device="cuda")
    views, off = [], 1
    for x in imgs:
        v = flat[off:off + x.size].view(x.shape)
        v.copy_(torch.from_numpy(x))
        views.append(v)
        off += x.size + 3
    bank = [(np.linspace(0.0, 1.0, 4), 0.5)]
    host = plan.decompose_batch([(x, 0.5, 5, 20, syn.DYADIC_EDGES, bank) for x in imgs], trace=True)
    dev = plan.decompose_batch([(v, 0.5, 5, 20, syn.DYADIC_EDGES, bank) for v in views], trace=True)
    torch.cuda.synchronize()
    for h, d in zip(host, dev):
        for k in ("bands", "residual", "S", "u", "filtered"):
            assert np.array_equal(h[k], d[k].cpu().numpy()), k


# ---------------------------------------------------------------------------------------------
# invariances (Sec. 2.1), exact on the GPU path too
# ---------------------------------------------------------------------------------------------
def test_one_homogeneity_exact(plan):
    f = _img(70, 50, 12)
    e = (0.0, 1.0, 2.0, 4.0, INF)
    a = plan.decompose(f, 0.5, 7, 40, e, trace=True)
    b = plan.decompose(2 * f, 1.0, 7, 40, tuple(2 * x for x in e), trace=True)
    assert np.array_equal(b["u"], 2 * a["u"])
    assert np.array_equal(b["bands"], 2 * a["bands"])
    assert np.array_equal(b["residual"], 2 * a["residual"])
    assert np.array_equal(b["S"], a["S"])


def test_transpose_exact(plan):
    f = _img(45, 77, 13)
    a = plan.decompose(f, 0.5, 6, 35, syn.DYADIC_EDGES)
    b = plan.decompose(np.ascontiguousarray(f.T), 0.5, 6, 35, syn.DYADIC_EDGES)
    assert np.array_equal(b["bands"], np.transpose(a["bands"], (0, 2, 1)))
    assert np.array_equal(b["residual"], a["residual"].T)
    np.testing.assert_allclose(b["S"], a["S"], rtol=1e-13)


# ---------------------------------------------------------------------------------------------
# the ROF step alone (Eq. ROF by Chambolle's iterations)
# ---------------------------------------------------------------------------------------------
@pytest.mark.parametrize("n_iter", [1, 7, 100, 1000])
def test_rof_step_matches_oracle(plan, n_iter):
    g = _img(48, 40, 14)
    u, p1, p2 = plan.rof_step(g, 0.5, n_iter)
    ru, rp1, rp2 = oracle.chambolle(g, 0.5, n_iter)
    assert np.abs(u - ru).max() <= 1e-5 * max(1.0, np.abs(g).max())
    assert np.abs(p1 - rp1).max() <= 1e-5 and np.abs(p2 - rp2).max() <= 1e-5


def test_rof_step_warm_start_input(plan):
    g = _img(30, 33, 15)
    _, p1, p2 = oracle.chambolle(g, 0.7, 40)
    u, q1, q2 = plan.rof_step(g, 0.7, 60, p1, p2)
    ru, _, _ = oracle.chambolle(g, 0.7, 60, p1=p1, p2=p2)
    assert np.abs(u - ru).max() <= 1e-5


# ---------------------------------------------------------------------------------------------
# full sizes
# ---------------------------------------------------------------------------------------------
def test_config1_full_size_parity(plan):
    # the bench workload as the bench runs it: device-resident input on a side stream, the
    # plan's tile choice, graph replay from the second call on
    import torch

    job = syn.config1().jobs[0]
    st = torch.cuda.Stream()
    f_dev = torch.from_numpy(job.f).cuda()
    torch.cuda.synchronize()
    outs = []
    with torch.cuda.stream(st):
        for _ in range(3):
            outs.append(plan.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, trace=True,
                                       stream=st))
    st.synchronize()
    g = {k: v.cpu().numpy() for k, v in outs[-1].items()}
    for o in outs[:-1]:
        for k in ("bands", "residual", "S", "u"):
            assert np.array_equal(o[k].cpu().numpy(), g[k]), k
    ref = oracle.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, trace=True)
    m = assert_parity(g, ref, job.f, "config1")
    print("config1", m)


def test_config1_full_size_cold_start_parity(tv):
    # p restarted from zero at every ROF step (the warm_start = 0 option), the whole config-1 run
    job = syn.config1().jobs[0]
    with tv.Plan(0, warm_start=0) as p:
        g = p.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, trace=True)
    ref = oracle.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, trace=True, warm_start=False)
    print("config1 cold start", assert_parity(g, ref, job.f, "config1 cold start"))


def test_m1024_full_size_parity_as_benchmarked(plan):
    # the 1024^2 workload of the decompositions/s figure, whole (K=50, 300 iterations), from
    # device memory on a side stream as the bench runs it
    import torch

    job = syn.m1024().jobs[0]
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        g = plan.decompose(torch.from_numpy(job.f).cuda(), job.dt, job.K, job.n_inner, job.edges,
                           stream=st)
    st.synchronize()
    g = {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in g.items()}
    ref = oracle.decompose(job.f, job.dt, job.K, job.n_inner, job.edges)
    print("m1024", assert_parity(g, ref, job.f, "m1024"))


def test_maximum_size_sampled_parity(plan):
    # the largest image the ABI accepts (H*W = 2^28), checked where the oracle can follow it. An
    # iteration moves information at most one pixel (w reads p one pixel up / left, the update
    # reads w one pixel down / right, u_{k+1} reads p one pixel up / left), so after K steps of
    # n_inner iterations an output depends only on inputs within K (n_inner + 1) pixels: the
    # oracle run on a window with a wider margin reproduces the window's centre. Plus exact
    # reconstruction everywhere and S against the band it feeds.
    H = W = 1 << 14
    K, n_inner, dt = 2, 2, 0.5
    edges = [0.0, 1.0, math.inf]
    rng = np.random.default_rng(2024)
    f = rng.standard_normal((H, W), dtype=np.float32)
    f[1000:3000, 5000:9000] += 4.0
    f[H - 700:, :300] -= 3.0
    g = plan.decompose(f, dt, K, n_inner, edges)
    scale = float(np.abs(f).max())
    for y0 in range(0, H, 2048):  # reconstruction, in slabs
        sl = slice(y0, y0 + 2048)
        rec = g["bands"][:, sl].astype(np.float64).sum(0) + g["residual"][sl]
        assert np.abs(rec - f[sl]).max() <= 1e-5 * scale
    # K = 2: S(t_1) = sum |phi_1|, and band 0 holds phi_1 dt (t_1 = 0.5 in [0, 1))
    s_band = np.abs(g["bands"][0].astype(np.float64)).sum() / dt
    assert abs(g["S"][0] - s_band) <= 1e-5 * g["S"][0]
    m = K * (n_inner + 1) + 4
    side = 48
    for y0, x0 in ((0, 0), (H - side, W - side), (0, W // 2), (1000 - side // 2, 5000 - side // 2),
                   (H // 2 + 7, 123)):
        ya, yb = max(0, y0 - m), min(H, y0 + side + m)
        xa, xb = max(0, x0 - m), min(W, x0 + side + m)
        ref = oracle.decompose(f[ya:yb, xa:xb], dt, K, n_inner, edges)
        cy, cx = slice(y0 - ya, y0 - ya + side), slice(x0 - xa, x0 - xa + side)
        gy, gx = slice(y0, y0 + side), slice(x0, x0 + side)
        assert np.abs(g["bands"][:, gy, gx] - ref["bands"][:, cy, cx]).max() <= 1e-3 * scale
        assert np.abs(g["residual"][gy, gx] - ref["residual"][cy, cx]).max() <= 1e-3 * scale


def test_config3_full_size_first_steps_parity(plan):
    # full 2048^2 spatial size and iteration count, the first 3 ROF steps (the oracle's share)
    job = syn.config3().jobs[0]
    g = plan.decompose(job.f, job.dt, 3, job.n_inner, job.edges, trace=True)
    ref = oracle.decompose(job.f, job.dt, 3, job.n_inner, job.edges, trace=True)
    assert_parity(g, ref, job.f, "config3 K=3")


def test_config3_full_run_properties(plan):
    # the whole 2048^2, K=50, 500-iteration run: reconstruction and exact one-homogeneity
    job = syn.config3().jobs[0]
    a = plan.decompose(job.f, job.dt, job.K, job.n_inner, job.edges)
    rec = a["bands"].astype(np.float64).sum(0) + a["residual"]
    assert np.abs(rec - job.f).max() <= 1e-5 * np.abs(job.f).max()
    assert np.all(np.isfinite(a["S"])) and np.all(a["S"] >= 0)
    b = plan.decompose(2 * job.f, 2 * job.dt, job.K, job.n_inner, tuple(2 * e for e in job.edges))
    assert np.array_equal(b["bands"], 2 * a["bands"]) and np.array_equal(b["S"], a["S"])


def test_config2_full_batch_as_benchmarked(plan):
    # the whole config-2 batch (64 images 128..1024 square-ish, K 20..60, three dt) in the
    # launch configuration the bench times (device memory, one batch): every image
    # reconstructs, the smallest ones match the oracle in full, and each sampled image is
    # bit-identical to its decomposition alone
    import torch

    wl = syn.config2()
    jobs = [(torch.from_numpy(j.f).cuda(), j.dt, j.K, j.n_inner, j.edges) for j in wl.jobs]
    outs = plan.decompose_batch(jobs)
    torch.cuda.synchronize()
    for j, o in zip(wl.jobs, outs):
        rec = o["bands"].double().sum(0).cpu().numpy() + o["residual"].cpu().numpy()
        assert np.abs(rec - j.f).max() <= 1e-5 * np.abs(j.f).max()
        assert bool(torch.isfinite(o["S"]).all()) and bool((o["S"] >= 0).all())
    order = sorted(range(len(wl.jobs)), key=lambda i: wl.jobs[i].f.size)
    for i in order[:2]:
        j = wl.jobs[i]
        ref = oracle.decompose(j.f, j.dt, j.K, j.n_inner, j.edges)
        got = {k: outs[i][k].cpu().numpy() for k in ("bands", "residual", "S")}
        assert_parity(got, ref, j.f, f"config2 image {i} {j.f.shape}")
    for i in (order[0], order[len(order) // 2], order[-1]):
        alone = plan.decompose(*jobs[i])
        torch.cuda.synchronize()
        for k in ("bands", "residual", "S"):
            assert torch.equal(alone[k], outs[i][k]), (i, k)


@pytest.mark.parametrize("storage", [1, 2, 3])
def test_16bit_dual_storage_reports_error(tv, storage):
    # fp16 / bf16 / snorm16 storage of p between launches: errors are reported, no bar is promised;
    # the reconstruction identity holds regardless (it telescopes in float64)
    job = syn.config1(H=256, W=256, K=20).jobs[0]
    with tv.Plan(0, p_storage=storage) as p:
        g = p.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, trace=True)
    ref = oracle.decompose(job.f, job.dt, job.K, job.n_inner, job.edges, trace=True)
    m = parity_metrics(g, ref, job.f)
    print("p_storage", storage, m)
    assert m["recon_inf"] <= 1e-5
    assert m["u_inf"] < 1.0


# ---------------------------------------------------------------------------------------------
# serving
# ---------------------------------------------------------------------------------------------
def test_serving_results_match_alone(tv):
    rng = np.random.default_rng(21)
    jobs = []
    for j in range(8):
        s = int(rng.choice([48, 64, 96, 130]))
        jobs.append((_img(s, s + 7, 200 + j), 0.5, int(rng.integers(3, 8)), 30, syn.DYADIC_EDGES))
    with tv.Plan(0) as p:
        tickets = [p.submit(*j, trace=True) for j in jobs]
        for (t, out), job in zip(tickets, jobs):
            assert p.wait(t, 120000) == tv.OK
        st = p.serving_stats()
        assert st["count"] == len(jobs) and st["p99_ms"] >= st["p50_ms"] > 0
        for (t, out), job in zip(tickets, jobs):
            alone = p.decompose(*job, trace=True)
            _same(out, alone)


def test_serving_admits_a_request_mid_flight_same_as_alone(tv):
    # Continuous batching, forced by construction rather than by timing: with two slots, A
    # (short) and B (long) take both; C waits in the queue until A retires, so C joins while B
    # is on the GPU between two of its steps, and C's steps then run in the same launches as
    # B's. C must give the bits it gives alone, and match the oracle; B, whose launches changed
    # when A left and C joined, must too.
    A = (_img(96, 80, 301), 0.5, 6, 40, syn.DYADIC_EDGES)
    B = (_img(128, 150, 302), 0.5, 2000, 40, syn.DYADIC_EDGES)
    C = (_img(70, 111, 303), 0.5, 8, 40, syn.DYADIC_EDGES)
    with tv.Plan(0, max_batch=2) as p:
        ta, oa = p.submit(*A, trace=True)
        tb, ob = p.submit(*B)
        tc, oc = p.submit(*C, trace=True)
        assert p.wait(tc, 120000) == tv.OK
        # C is done while B (2000 steps, admitted no later than A's retirement after 6) still runs
        b_running = p.poll(tb) == tv.ENOTREADY
        assert p.wait(ta, 120000) == tv.OK and p.wait(tb, 120000) == tv.OK
        assert b_running
        for out, job in ((oa, A), (ob, B), (oc, C)):
            alone = p.decompose(*job, trace="u" in out)
            _same(out, alone)
    ref = oracle.decompose(*C, trace=True)
    assert_parity(oc, ref, C[0], "served mid-flight")


def test_serving_budget_and_cancel(tv):
    f = _img(64, 64, 30)
    with tv.Plan(0, mem_budget_bytes=1 << 16) as p:
        t, _ = p.submit(f, 0.5, 4, 10, syn.DYADIC_EDGES)
        assert p.wait(t, 60000) == tv.ENOMEM
    with tv.Plan(0, max_batch=1) as p:
        t1, _ = p.submit(_img(256, 256, 31), 0.5, 40, 300, syn.DYADIC_EDGES)
        t2, _ = p.submit(f, 0.5, 4, 10, syn.DYADIC_EDGES)
        assert p.cancel(t2) == tv.OK
        assert p.wait(t2, 60000) == tv.ECANCELLED
        assert p.wait(t1, 120000) == tv.OK
        assert p.poll(12345) == tv.EINVAL


def test_slow_and_absent_clients(tv):
    # a client that polls late gets its finished results (they were retired into its buffers
    # meanwhile); one that never waits does not hold up the others, and closing the plan with
    # requests queued and running cancels them without hanging; the device stays usable
    import time

    jobs = [(_img(64 + 20 * i, 80, 400 + i), 0.5, 4 + i % 3, 20, syn.DYADIC_EDGES) for i in range(6)]
    with tv.Plan(0) as p0:
        want = [p0.decompose(*j) for j in jobs]
    with tv.Plan(0) as p:
        tickets = [p.submit(*j) for j in jobs]
        time.sleep(1.0)  # nobody waits meanwhile
        for (t, out), w in zip(tickets[:3], want[:3]):
            assert p.poll(t) in (tv.OK, tv.ENOTREADY)
            assert p.wait(t, 60000) == tv.OK
            _same(out, w)
        # tickets[3:] are never claimed
    with tv.Plan(0, max_batch=2) as p:
        for _ in range(3):
            p.submit(_img(512, 512, 41), 0.5, 50, 300, syn.DYADIC_EDGES)
        p.submit(*jobs[0])
        t0 = time.perf_counter()
    assert time.perf_counter() - t0 < 60.0  # closing cancelled the queue instead of draining it
    with tv.Plan(0) as p:
        _same(p.decompose(*jobs[1]), want[1])


def test_cached_batch_workspaces_stay_within_the_budget(tv):
    imgs = [_img(120 + 10 * i, 130, 60 + i) for i in range(6)]
    a = [(imgs[i], 0.5, 5, 20, syn.DYADIC_EDGES) for i in range(3)]
    b = [(imgs[i], 0.5, 6, 20, syn.DYADIC_EDGES) for i in range(3, 6)]
    with tv.Plan(0) as p0:
        want_a = p0.decompose_batch(a)
        bytes_a = p0.stats()["workspace_bytes"]
        want_b = p0.decompose_batch(b)
        assert p0.stats()["workspace_bytes"] > bytes_a  # both kept under the default budget
    budget = int(1.6 * bytes_a)
    with tv.Plan(0, mem_budget_bytes=budget) as p:
        for x, y in zip(p.decompose_batch(a), want_a):
            _same(x, y)
        for x, y in zip(p.decompose_batch(b), want_b):
            _same(x, y)
        assert p.stats()["workspace_bytes"] <= budget  # a's workspace made room for b's
        both = p.decompose_batch(a + b)  # larger than the budget on its own: runs alone
        assert p.stats()["workspace_bytes"] > budget
        for x, y in zip(both, want_a + want_b):
            _same(x, y)
        for x, y in zip(p.decompose_batch(a), want_a):
            _same(x, y)


def test_injected_workspace_allocation_failure(tv):
    # host-side fault injection (no device fault): the plan's n-th workspace allocation fails
    # once with ENOMEM. With other workspaces cached the plan drops them and retries; with none
    # the call reports ENOMEM and the plan stays usable.
    a = [(_img(90 + 5 * i, 100, 70 + i), 0.5, 4, 20, syn.DYADIC_EDGES) for i in range(3)]
    b = [(_img(60, 80 + 3 * i, 80 + i), 0.5, 5, 20, syn.DYADIC_EDGES) for i in range(2)]
    with tv.Plan(0) as p0:
        want_a = p0.decompose_batch(a)
        want_b = p0.decompose_batch(b)
    with tv.Plan(0, test_fail_alloc=4) as p:  # a takes allocations 1-3, b's first one fails
        for x, y in zip(p.decompose_batch(a), want_a):
            _same(x, y)
        for x, y in zip(p.decompose_batch(b), want_b):
            _same(x, y)
        assert p.stats()["workspace_bytes"] > 0
        for x, y in zip(p.decompose_batch(a), want_a):  # rebuilt after the eviction
            _same(x, y)
    with tv.Plan(0, test_fail_alloc=2) as p:  # nothing cached to give back: the call fails
        with pytest.raises(tv.TvSpecError) as ei:
            p.decompose_batch(a)
        assert ei.value.status == tv.ENOMEM
        assert p.stats()["workspace_bytes"] == 0
        for x, y in zip(p.decompose_batch(a), want_a):
            _same(x, y)


def test_invalid_arguments_leave_plan_usable(plan, tv):
    f = _img(16, 16, 40)
    with pytest.raises(tv.TvSpecError) as ei:
        plan.decompose(f, 0.5, 1, 10, syn.DYADIC_EDGES)
    assert ei.value.status == tv.EINVAL
    bad = f.copy()
    bad[3, 3] = np.nan
    with pytest.raises(tv.TvSpecError):
        plan.decompose(bad, 0.5, 4, 10, syn.DYADIC_EDGES)
    out = plan.decompose(f, 0.5, 4, 10, syn.DYADIC_EDGES)
    assert np.all(np.isfinite(out["bands"]))


def test_tune_cache_file_round_trip(tv, tmp_path):
    # the first plan tunes and appends its choice; a later plan reads choices from the file
    path = str(tmp_path / "tune.txt")
    f = _img(40, 60, 3)
    args = (f, 0.5, 4, 16, syn.DYADIC_EDGES)
    with tv.Plan(0, tune_cache=path) as a:
        ra = a.decompose(*args)
    lines = open(path).read().split("\n")
    prefix, key, shape, depth, pdl = lines[0].split()  # pdl: dependent launch chosen or not
    forced = 3 if int(shape) != 3 else 2
    with open(path, "w") as fh:
        fh.write(f"{prefix} {key} {forced} 4 0\n")
        fh.write(f"another-gpu/sm1/shapes1-0 {key} 0 1\n")  # ignored: other GPU / build
    with tv.Plan(0, tune_cache=path) as b:
        rb = b.decompose(*args)
        assert b.stats()["last_tile"] == forced
    _same(ra, rb)  # every tile shape gives the same bits
