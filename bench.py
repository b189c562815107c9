"""Benchmark of the spectral TV decomposition on GB300.

Default workload: one 512x512 float32 image (40 disks/rectangles + noise), K = 50 implicit
TV-flow steps at dt = 0.5, 300 Chambolle iterations per step, 6 dyadic bands + residual.
One bench step = one whole decomposition. Metric: Chambolle Mpx*iter/s
(= H*W*K*n_inner / time / 1e6), whole job over all ranks.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
                  [--workload config1|m1024|config2|config3|config4] [--quick]

Printed: one JSON line on rank 0. `value` is device-timed (inputs resident in HBM, L2
flushed before every timed step); `e2e` is the same metric through the C ABI with host
buffers, host<->device copies inside the timed region; `roofline` is for the dominant kernel
(the tiled dual-iteration kernel) timed alone on the same image; `cpu_baseline` is the FP64
oracle on this host's cores on a bounded sample of the workload.

The reference arm (--impl reference) times the FP64 oracle (the only implementation of the
method besides this one), on a bounded sample per step.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

ALG_BYTES_FP32 = 20  # read p (8) + read g/lambda (4) + write p (8) per pixel per iteration


def kernel_source_hash() -> str:
    """Hash of the dual-iteration kernel's sources: DRAM traffic recorded from an ncu capture
    (profiles/traffic.json) is only reported while the kernel is unchanged since the capture."""
    import hashlib

    h = hashlib.sha1()
    for f in ("k_tiled.cuh", "chambolle_math.cuh", "k_step_coop.cuh"):
        with open(os.path.join(ROOT, "paper_2006_10004_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:12]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _workload(name: str):
    if name == "config1":
        return syn.config1()
    if name == "m1024":
        return syn.m1024()
    if name == "config2":
        return syn.config2()
    if name == "config3":
        return syn.config3()
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 50 ms while running. Entering waits
    (up to 3 s) for nvidia-smi's first sample, and only samples that arrive after that count,
    so the summary describes the region inside the ``with`` block."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t_end = time.perf_counter() + 3.0
            while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.lines = []  # samples from before the region do not count
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate_over_ranks(t_sec: float, units: float, dist=None):
    """Whole-job throughput of weak-scaled replicas: every rank processed `units` (pixel-
    iterations) in `t_sec` seconds of device time; the job's time is the slowest rank's, and
    the value is all ranks' units over it. With dist (torch.distributed, any backend) the
    ranks synchronise on a barrier and agree on the maximum; returns (value, t_max)."""
    import torch

    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return units / t_sec, t_sec
    ws = dist.get_world_size()
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    dist.barrier()
    t = torch.tensor([t_sec], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([units], dtype=torch.float64, device=dev)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    t_max = float(t.item())
    return float(u.item()) / t_max, t_max


def _oracle_sample(job, max_k: int):
    """FP64 oracle on a bounded sample of the job: the first max_k ROF steps of the same image."""
    import oracle

    K = min(job.K, max_k)
    t = time.perf_counter()
    oracle.decompose(job.f, job.dt, K, job.n_inner, job.edges)
    el = time.perf_counter() - t
    px_it = job.f.size * K * job.n_inner
    return px_it / el / 1e6, el, K, oracle.max_threads()


def _oracle_batch_sample(jobs):
    """FP64 oracle on whole decompositions of a fixed subset of a batch's images."""
    import oracle

    t = time.perf_counter()
    for j in jobs:
        oracle.decompose(j.f, j.dt, j.K, j.n_inner, j.edges)
    el = time.perf_counter() - t
    return sum(j.px_iters for j in jobs) / el / 1e6, el, oracle.max_threads()


def _reference_line(args, ws, metric, unit, value, times, workload, sample, cores):
    return {"impl": "reference", "metric": metric, "value": value, "unit": unit,
            "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * np.mean(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": workload, "sample": sample},
            "cpu_baseline": {"value": value, "unit": unit, "cores": cores, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": unit, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def run_reference(args):
    """The reference arm: the FP64 oracle (the only other implementation of the method) on the
    host's cores, each step a bounded sample of the workload."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle

    kk_req = max(2, args.ref_steps_k)
    if args.workload == "training":
        # whole decompositions (K = 50, 300 iterations) of the first 8 crops of the set
        srcs, crops = training_workload(8)
        run = lambda: oracle.training_set(srcs, crops, 64, 1, 0.5, 50, 300, syn.DYADIC_EDGES)
        px_it = 8 * 64 * 64 * 50 * 300
        for _ in range(args.warmup):
            oracle.training_set(srcs, crops[:1], 64, 1, 0.5, 2, 300, syn.DYADIC_EDGES)
        times = []
        for _ in range(args.steps):
            t = time.perf_counter()
            run()
            times.append(time.perf_counter() - t)
        value = px_it * len(times) / sum(times) / 1e6
        sample = "8 crops of 64x64 (whole decompositions, K=50, 300 iterations) of the training set"
        line = _reference_line(args, ws, "Chambolle Mpx*iter/s", "Mpx*iter/s", value, times,
                               training_workload_name(args.crops), sample, oracle.max_threads())
    elif args.workload == "config4":
        # served images/s of the oracle one request at a time: the first kk ROF steps of each of
        # the first 4 requests at 100 req/s, each request's time scaled to its K steps
        _, jobs = config4_requests(config4_pool(), 100.0, 4)
        for _ in range(args.warmup):
            oracle.decompose(jobs[0][0][:64, :64], 0.5, 2, 300, syn.DYADIC_EDGES)
        times = []
        for _ in range(args.steps):
            est = 0.0
            for f, dt, K, n, e in jobs:
                kk = min(K, kk_req)
                t = time.perf_counter()
                oracle.decompose(f, dt, kk, n, e)
                est += (time.perf_counter() - t) * K / kk
            times.append(est / len(jobs))
        value = len(times) / sum(times)
        sample = (f"first {kk_req} ROF steps of each of the first 4 requests of the 100 req/s "
                  "stream, each request's time scaled by K / steps run; one request at a time")
        line = _reference_line(args, ws, "served images/s", "images/s", value, times, "config4_serving",
                               sample, oracle.max_threads())
    else:
        wl = _workload(args.workload)
        # one image (config 2: the first two images of the batch), its first kk ROF steps
        jobs = wl.jobs[:2] if args.workload == "config2" else wl.jobs[:1]
        for _ in range(args.warmup):
            _oracle_sample(jobs[0], 2)
        times = []
        px_it = 0
        for _ in range(args.steps):
            el = 0.0
            px_it = 0
            for job in jobs:
                kk = max(2, min(job.K, kk_req))
                _, e, _, _ = _oracle_sample(job, kk)
                el += e
                px_it += job.f.size * kk * job.n_inner
            times.append(el)
        value = px_it * len(times) / sum(times) / 1e6
        sample = "; ".join(f"first {max(2, min(j.K, kk_req))} of {j.K} ROF steps of the "
                           f"{j.f.shape[0]}x{j.f.shape[1]} image, {j.n_inner} iterations each" for j in jobs)
        line = _reference_line(args, ws, "Chambolle Mpx*iter/s", "Mpx*iter/s", value, times, wl.name,
                               sample, oracle.max_threads())
    print(json.dumps(line))
    return 0


def run_gb300(args):
    import torch

    ws, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
        pg = dist
    import paper_2006_10004_gb300 as tv

    if args.kernel_only:
        return run_kernel_only(args, tv, torch, local)
    if args.workload == "config2":
        return run_batched(args, tv, torch, local, ws)
    if args.workload == "config4":
        return run_serving(args, tv, torch, local, ws)
    if args.workload == "training":
        return run_training(args, tv, torch, local, ws)
    wl = _workload(args.workload)
    plan = tv.Plan(local, acc_mode=args.acc_mode, tma=1 if args.tma else 0,
                   **({"kernel": tv.KERNEL_TILED, "tile": args.tile} if args.tile >= 0 else {}))
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2

    # ---- device-resident timed region ------------------------------------------------------
    if args.workload == "config2":
        jobs = [(torch.from_numpy(j.f).to(dev), j.dt, j.K, j.n_inner, j.edges) for j in wl.jobs]
        run = lambda: plan.decompose_batch(jobs, stream=stream)
        px_it = wl.px_iters
        shape_desc = {"images": len(jobs)}
    else:
        job = wl.jobs[0]
        f_dev = torch.from_numpy(job.f).to(dev)
        run = lambda: plan.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, stream=stream)
        px_it = job.px_iters
        shape_desc = {"H": job.f.shape[0], "W": job.f.shape[1], "K": job.K, "n_inner": job.n_inner,
                      "dt": job.dt, "n_bands": len(job.edges) - 1}
    for _ in range(max(args.warmup, 3) if args.warmup >= 3 else args.warmup):
        run()
    torch.cuda.synchronize()
    st0 = plan.stats()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if pg:
        pg.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xff)  # evict the previous step's state from L2 (not timed)
            evs[i][0].record(stream)
            run()
            evs[i][1].record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    if pg:
        pg.barrier()
    st1 = plan.stats()
    dev_ms = sum(a.elapsed_time(b) for a, b in evs)
    value, t_sec = aggregate_over_ranks(dev_ms / 1000.0, float(px_it * args.steps), pg)
    value /= 1e6
    launches = int(st1["kernel_launches"] - st0["kernel_launches"])

    result = {"metric": "Chambolle Mpx*iter/s", "value": value, "unit": "Mpx*iter/s", "n_gpus": ws,
              "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * t_sec / args.steps,
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
              "data": "synthetic",
              "config": {"workload": wl.name, **shape_desc,
                         "arith": "dual iterations f32, epilogue (u, phi, S, bands, residual) "
                                  + ("f64" if args.acc_mode == 0 else "float-float (compensated f32), S f64"),
                         "l2": "flushed before every timed step (256 MiB write, untimed)",
                         "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                         "tile": st1["last_tile"], "temporal_block": st1["last_temporal_block"]},
              "gpu_launches": launches, "clocks": clk.summary(),
              "wall_s_timed_region": wall}

    # ---- end to end through the C ABI with host buffers ------------------------------------
    if not args.no_e2e and args.workload != "config2":
        f_host = torch.from_numpy(job.f).pin_memory().numpy()
        for _ in range(2):  # untimed, as the device-timed steps above
            plan.decompose(f_host, job.dt, job.K, job.n_inner, job.edges)
        n_e2e = max(1, min(args.steps, 5))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(n_e2e):
            out = plan.decompose(f_host, job.dt, job.K, job.n_inner, job.edges)
        el = time.perf_counter() - t0
        d2h = out["bands"].nbytes + out["residual"].nbytes + out["S"].nbytes
        result["e2e"] = {"value": px_it * n_e2e / el / 1e6, "unit": "Mpx*iter/s",
                         "h2d_bytes_per_step": int(job.f.nbytes), "d2h_bytes_per_step": int(d2h),
                         "steps": n_e2e, "ms_per_step": 1000 * el / n_e2e}

    # ---- roofline of the dominant kernel: dual iterations timed alone -----------------------
    if args.workload != "config2":
        result["roofline"], result["roofline_issue"] = measure_roofline(tv, torch, plan, wl.name, job,
                                                                        dev, stream)

    # ---- CPU baseline: the FP64 oracle on this host -------------------------------------------
    if rank == 0 and not args.no_cpu_baseline and args.workload != "config2":
        v, el, K, cores = _oracle_sample(job, args.cpu_k)
        result["cpu_baseline"] = {"value": v, "unit": "Mpx*iter/s", "cores": cores, "kind": "oracle",
                                  "sample": f"first {K} of {job.K} ROF steps of the same image ({el:.1f} s)"}
        # the same oracle on one core, on a shorter sample
        import oracle

        oracle.set_threads(1)
        v1, el1, K1, _ = _oracle_sample(job, max(1, args.cpu_k // 10))
        oracle.set_threads(cores)
        result["cpu_baseline"]["single_thread"] = {
            "value": v1, "cores": 1, "sample": f"first {K1} of {job.K} ROF steps ({el1:.1f} s)"}

    if rank == 0 and not args.quick and args.workload == "config3":
        result["precision_study"] = measure_precision(tv, torch, local, job, f_dev, stream)

    if rank == 0 and not args.quick and args.workload == "config1":
        # the other two parts of the metric: 1024^2 decompositions/s and served p50/p99,
        # plus the batched-vs-plain comparison
        m = syn.m1024().jobs[0]
        fm = torch.from_numpy(m.f).to(dev)
        for _ in range(2):  # the second use captures the graph the timed runs replay
            plan.decompose(fm, m.dt, m.K, m.n_inner, m.edges, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(3):
            plan.decompose(fm, m.dt, m.K, m.n_inner, m.edges, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 3
        result["m1024"] = {"workload": syn.m1024.__doc__.strip().splitlines()[0], "decomps_per_s": 1000.0 / ms,
                           "ms_per_decomp": ms, "Mpx_iter_per_s": m.px_iters / ms / 1e3}
        # the largest single-image workload (2048^2, K = 50, 500 iterations: its 80 MB dual state
        # is 0.6 of the L2) with its own rooflines
        result["config3"] = measure_decomposition(tv, torch, local, syn.config3(), dev, stream, flush)
        result["filter_bank_config1"] = measure_filters(tv, torch, plan, job, f_dev, stream, flush)
        result["inner_solvers"] = measure_solvers(tv, torch, plan, job, stream)
        result["acc_mode_compare"] = measure_acc_modes(tv, torch, local, job, f_dev, stream, flush)
        result["batched_config2"] = measure_batched(tv, torch, local, 2, 1)
        result["training_crops"] = measure_crops(tv, torch, local)
        # config 4's load points (20-200 req/s), each with a shortened request count
        rates = [float(x) for x in str(args.serve_rates).split(",")]
        pts = measure_serving(tv, local, rates, args.serve_requests)
        result["serving_config4"] = [{k: v for k, v in sv.items() if k != "clocks"} for sv in pts]
        result["config"]["serving_requests_per_rate"] = args.serve_requests

    if rank == 0:
        print(json.dumps(result))
    plan.close()
    if pg:
        pg.destroy_process_group()
    return 0


SM_COUNT = 152          # GB300
ISSUE_PER_SM_CLK = 4    # warp instructions issued per SM per clock (four schedulers)


def _profile_record(key: str):
    """The ncu record of a kernel launch (DRAM bytes, warp instructions, iterations of the
    captured launch) from profiles/traffic.json, if one was taken of the current sources."""
    tf = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        rec = json.load(open(tf)).get(key)
    except Exception:
        return None
    return rec if isinstance(rec, dict) else None


def measure_roofline(tv, torch, plan, wl_name, job, dev, stream, reps: int = 5):
    """The dual-iteration kernel timed alone on the workload's image (per-launch duration by
    CUDA events on the launch stream), against two ceilings:
      hbm   -- algorithmic bytes (20 B per pixel-iteration: read p and g/lambda, write p) per
               launch / duration, over the measured copy bandwidth; with temporal blocking
               this can exceed 1 (the state is re-read from registers, not HBM);
      issue -- warp instructions per launch (ncu count of the current sources, scaled by
               iterations) / duration, over the SM count x 4 issue slots x the maximum clock.
    `traffic` (DRAM bytes per launch) and the instruction count come from profiles/traffic.json
    only while the kernel sources are those the capture was taken of."""
    H, W = job.f.shape
    pitch = tv.pitch_for(W)
    gl = torch.zeros((H, pitch), dtype=torch.float32, device=dev)
    gl[:, :W] = torch.from_numpy(job.f / job.dt).to(dev)
    p1 = torch.zeros_like(gl)
    p2 = torch.zeros_like(gl)
    iters = job.n_inner
    plan.chambolle_iterate(gl, p1, p2, H, W, pitch, iters, stream=stream)  # tunes + warms
    torch.cuda.synchronize()
    s0 = plan.stats()
    depth = max(1, s0["last_temporal_block"])
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        plan.chambolle_iterate(gl, p1, p2, H, W, pitch, iters, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    s1 = plan.stats()
    n_launch = max(int(s1["kernel_launches"] - s0["kernel_launches"]), 1)
    per_launch_s = e0.elapsed_time(e1) / 1000.0 / n_launch
    # n_inner need not be a multiple of the temporal block (300 = 37 x 8 + 4): an average
    # launch does the iterations of all launches over their number
    it_per_launch = iters * reps / n_launch
    alg_bytes = ALG_BYTES_FP32 * H * W * it_per_launch
    achieved = alg_bytes / per_launch_s / 1e9
    peak, src = _peaks()
    key = f"{wl_name}/tile{s1['last_tile']}/tb{depth}/{kernel_source_hash()}"
    rec = _profile_record(key)
    # DRAM bytes per launch (tile loads and stores: the same for a launch of fewer iterations)
    traffic = rec.get("dram_bytes") if rec else None
    hbm = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
           "traffic": traffic,
           "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else src,
           "kernel": "k_tiled", "per_launch_us": per_launch_s * 1e6, "temporal_block": depth,
           "iters_per_launch": it_per_launch, "algorithmic_bytes_per_launch": alg_bytes,
           "profile_key": key}
    issue = None
    if rec and rec.get("warp_inst"):
        mhz = _max_sm_mhz()
        inst = rec["warp_inst"] * it_per_launch / rec.get("iters", it_per_launch)
        ipeak = SM_COUNT * ISSUE_PER_SM_CLK * mhz * 1e6 / 1e9
        ia = inst / per_launch_s / 1e9
        issue = {"bound": "issue", "achieved": ia, "peak": ipeak, "unit": "Gwarp_inst/s", "frac": ia / ipeak,
                 "peak_source": f"{SM_COUNT} SMs x {ISSUE_PER_SM_CLK} issue slots x {mhz:.0f} MHz (nominal)",
                 "warp_inst_per_launch": inst,
                 "thread_inst_per_px_iter": 32 * inst / (H * W * it_per_launch),
                 "source": "ncu smsp__inst_executed.sum of the current sources (profiles/traffic.json)"}
    return hbm, issue


def _max_sm_mhz() -> float:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["sm_max_mhz"])
    except Exception:
        return 2070.0


def measure_decomposition(tv, torch, local, wl, dev, stream, flush, steps: int = 5, warmup: int = 3):
    """A second single-image workload of the default run: whole decompositions, device-timed
    (L2 flushed before each), with the dual-iteration kernel's rooflines on the same image."""
    job = wl.jobs[0]
    with tv.Plan(local) as plan:
        f_dev = torch.from_numpy(job.f).to(dev)
        for _ in range(warmup):
            plan.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, stream=stream)
        torch.cuda.synchronize()
        ts = []
        for i in range(steps):
            flush.fill_(i & 0xff)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, stream=stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        st = plan.stats()
        ms = float(np.median(ts))
        out = {"workload": wl.name, "H": job.f.shape[0], "W": job.f.shape[1], "K": job.K,
               "n_inner": job.n_inner, "ms_per_decomp": ms, "Mpx_iter_per_s": job.px_iters / ms / 1e3,
               "decomps_per_s": 1000.0 / ms, "tile": st["last_tile"], "temporal_block": st["last_temporal_block"],
               "steps": steps, "l2": "flushed before every timed decomposition"}
        out["roofline"], out["roofline_issue"] = measure_roofline(tv, torch, plan, wl.name, job, dev, stream)
    return out


def filter_bank(dt: float, K: int, n: int = 6):
    """n spectral filters H(t_k): all-pass, ideal low / high / band-pass in t, and smooth ones."""
    t = dt * np.arange(1, K)
    bank = [(np.ones(K - 1), 1.0), ((t < 2.0) * 1.0, 0.0), ((t >= 2.0) * 1.0, 1.0),
            (((t >= 1.0) & (t < 4.0)) * 1.0, 0.0)]
    s = 2.0
    while len(bank) < n:
        bank.append((np.exp(-t / s), 0.5))
        s *= 2.0
    return bank[:n]


def measure_filters(tv, torch, plan, job, f_dev, stream, flush, n_filters: int = 6, reps: int = 3):
    """Spectral filtering fused into the epilogue (Eq. filteredTVtrafo): device time of the
    decomposition with a bank of filters against the same decomposition without, L2 flushed."""
    bank = filter_bank(job.dt, job.K, n_filters)

    def timed(fn):
        fn()
        fn()  # the second use captures the graph the timed runs replay
        torch.cuda.synchronize()
        evs = []
        for i in range(reps):
            flush.fill_(i & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(x.elapsed_time(y) for x, y in evs) / reps

    plain = timed(lambda: plan.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, stream=stream))
    filt = timed(lambda: plan.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, stream=stream,
                                        filters=bank))
    return {"filters": n_filters, "ms_with_filters": filt, "ms_without": plain,
            "overhead_frac": filt / plain - 1.0,
            "Mpx_iter_per_s_with_filters": job.px_iters / filt / 1e3}


def measure_precision(tv, torch, local, job, f_dev, stream):
    """Config 3's precision study: the dual field stored as fp32 / fp16 / bf16 / snorm16 between
    launches. Per storage: device time of one decomposition and the bands' and residual's
    deviation from the fp32 run (L-inf relative to max|f|, relative L2)."""
    out = {}
    ref = None
    fmax = float(f_dev.abs().max())
    for name, st_kind in (("fp32", 0), ("fp16", 1), ("bf16", 2), ("snorm16", 3)):
        with tv.Plan(local, p_storage=st_kind) as p:
            for _ in range(2):
                r = p.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, stream=stream)
            torch.cuda.synchronize()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            r = p.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, stream=stream)
            b.record(stream)
            torch.cuda.synchronize()
            row = {"ms": a.elapsed_time(b), "tile": p.stats()["last_tile"]}
        if ref is None:
            ref = r
        else:
            db = (r["bands"].double() - ref["bands"].double())
            row["bands_inf_rel_maxf"] = float(db.abs().max()) / fmax
            row["bands_rel_l2"] = float(db.norm() / ref["bands"].double().norm())
            row["residual_inf_rel_maxf"] = float((r["residual"] - ref["residual"]).abs().max()) / fmax
        out[name] = row
    return out


def measure_acc_modes(tv, torch, local, job, f_dev, stream, flush, reps: int = 3):
    """Device time of the decomposition with the float64 epilogue and with the compensated
    float32 (float-float) epilogue, L2 flushed before every timed run."""
    out = {}
    for mode in (0, 1):
        with tv.Plan(local, acc_mode=mode) as p:
            for _ in range(2):
                p.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, stream=stream)
            torch.cuda.synchronize()
            tot = 0.0
            for i in range(reps):
                flush.fill_(i & 0xff)
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                p.decompose(f_dev, job.dt, job.K, job.n_inner, job.edges, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                tot += a.elapsed_time(b)
            out[f"acc_mode_{mode}_ms"] = tot / reps
    out["speedup_compensated"] = out["acc_mode_0_ms"] / out["acc_mode_1_ms"]
    return out


def measure_solvers(tv, torch, plan, job, stream, targets=(1e-4, 1e-5), check_every: int = 25):
    """Inner solvers of one ROF step (the first step of the bench image, lambda = dt): for each
    per-pixel duality-gap target, the iterations and wall time (gap checks included) each
    solver needs, and each solver's device time per iteration."""
    g = torch.from_numpy(job.f).to(stream.device)
    N = job.f.size
    out = {"image": f"{job.f.shape[0]}x{job.f.shape[1]}", "lambda": job.dt, "check_every": check_every}
    for name in ("chambolle", "fgp", "pdhg"):
        plan.rof_solve(g, job.dt, name, max_iter=100, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = plan.rof_solve(g, job.dt, name, max_iter=1000, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        row = {"us_per_iteration": e0.elapsed_time(e1) * 1e3 / 1000, "gap_at_1000": r["gap"] / N}
        for tgt in targets:
            t0 = time.perf_counter()
            r = plan.rof_solve(g, job.dt, name, max_iter=50000, gap_tol=tgt * N, check_every=check_every,
                               stream=stream)
            row[f"to_{tgt:g}"] = {"iterations": r["iterations"], "ms": 1e3 * (time.perf_counter() - t0),
                                 "gap_per_px": r["gap"] / N}
        out[name] = row
    return out


def measure_batched(tv, torch, local, steps: int, warmup: int, with_clocks=None):
    """Config 2: 64 images of uneven sizes and schedules. Device time of the batched path (one
    set of launches per step over all images, graph-replayed) against the plain path (the same
    images decomposed one at a time, each graph-replayed); L2 flushed before every timed step."""
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    wl = syn.config2()
    jobs = [(torch.from_numpy(j.f).to(dev), j.dt, j.K, j.n_inner, j.edges) for j in wl.jobs]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    plan = tv.Plan(local)
    plain_plan = tv.Plan(local)

    def timed(fn, n):
        evs = []
        for i in range(n):
            flush.fill_(i & 0xff)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            evs.append((a, b))
        torch.cuda.synchronize()
        return sum(x.elapsed_time(y) for x, y in evs) / 1000.0

    batch = lambda: plan.decompose_batch(jobs, stream=stream)

    def plain():
        for j in jobs:
            plain_plan.decompose(*j, stream=stream)

    for _ in range(max(2, warmup)):
        batch()
    plain()
    torch.cuda.synchronize()
    s0 = plan.stats()
    t_batch = timed(batch, steps)
    s1 = plan.stats()
    n_plain = max(1, steps // 2)
    t_plain = timed(plain, n_plain)
    # the plain form without graph replay: one image at a time, every launch from the host
    nograph = tv.Plan(local, use_graphs=0)

    def plain_nograph():
        for j in jobs:
            nograph.decompose(*j, stream=stream)

    plain_nograph()
    t_nograph = timed(plain_nograph, 1)
    nograph.close()
    n_img = len(jobs)
    out = {"workload": wl.name, "images": n_img, "px_iters_per_batch": wl.px_iters,
           "batched_images_per_s": n_img * steps / t_batch, "batched_ms": 1000 * t_batch / steps,
           "batched_Mpx_iter_per_s": wl.px_iters * steps / t_batch / 1e6,
           "plain_images_per_s": n_img * n_plain / t_plain, "plain_ms": 1000 * t_plain / n_plain,
           "plain_no_graph_images_per_s": n_img / t_nograph,
           "tile": s1["last_tile"], "temporal_block": s1["last_temporal_block"],
           "gpu_launches": int(s1["kernel_launches"] - s0["kernel_launches"])}
    out["batched_over_plain"] = out["batched_images_per_s"] / out["plain_images_per_s"]
    plan.close()
    plain_plan.close()
    return out


def training_workload_name(n: int) -> str:
    return (f"{n} crops 64x64 (1/3 from 128x128 downsampled by 2) of 16 sources 512x512, "
            "standardised over the set, K=50, dt=.5, 300 iterations, 6 dyadic bands")


def training_workload(n: int = 3000, size: int = 64, n_sources: int = 16, seed: int = 9000):
    """The paper's ground-truth generation (Sec. 4.1): n crops of size^2 from synthetic
    512^2 greyscale sources, one third of them from (2 size)^2 windows downsampled by 2;
    crop positions drawn here (seeded) and passed in."""
    srcs = [syn.make_image(512, 512, 40, (2.0, 60.0), (0.05, 1.0), 0.02, seed + i) for i in range(n_sources)]
    rng = np.random.default_rng(seed)
    crops = []
    for c in range(n):
        s = 2 if c % 3 == 2 else 1
        i = int(rng.integers(0, n_sources))
        crops.append((i, int(rng.integers(0, 512 - s * size + 1)), int(rng.integers(0, 512 - s * size + 1)), s))
    return srcs, crops


# Algorithmic float32 operations of one Chambolle iteration at one pixel (FMA = 2): w = div p - g/l
# (4), G = grad w (2), |G|^2 (3), 1 + tau |G| (2), p + tau G (4), times 1/(1 + tau |G|) (2); plus
# one square root and one reciprocal on the special-function unit, not counted.
ALG_FLOPS_PER_PX_ITER = 17
# float32 peak of the SMs: 152 SMs x 128 FP32 lanes x 2 flop per FMA x 2.07 GHz (maximum SM clock)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
# special-function (XU) pipe: 16 results per SM per clock (nominal) x 152 SMs x 2.07 GHz
XU_PEAK_GOPS = 152 * 16 * 2.07e9 / 1e9


def measure_crops(tv, torch, local, n: int = 3000, compare: bool = True, acc_mode: int = 0,
                  steps: int = 2, warmup: int = 3):
    """Training-data generation: crops + standardisation over the set + decompositions
    (K = 50 steps of dt = .5, 300 iterations, 6 dyadic bands) of n 64x64 crops through
    tvspec_training_set (device memory); with ``compare``, against the same standardised crops
    decomposed as a batch on the per-step path and on the resident path."""
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    srcs, crops = training_workload(n)
    srcs_d = [torch.from_numpy(x).to(dev) for x in srcs]
    out = {"workload": training_workload_name(n)}

    def timed(fn, reps=2, warm=3):
        # the untimed calls (the second one captures the graph) are still running on the
        # device while the timed calls are prepared on the host: no host-side gaps
        for _ in range(max(2, warm)):
            fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    px_it = n * 64 * 64 * 50 * 300
    with tv.Plan(local, acc_mode=acc_mode) as p:
        run = lambda: p.training_set(srcs_d, crops, 64, 1, 0.5, 50, 300, syn.DYADIC_EDGES, want_stats=False,
                                     stream=stream)
        s0 = p.stats()
        ms = timed(run, reps=steps, warm=warmup)
        s1 = p.stats()
        x = run()["crops"]
        torch.cuda.synchronize()
        calls = max(2, warmup) + steps
        out["training_set"] = {"images_per_s": n / ms * 1e3, "ms": ms, "Mpx_iter_per_s": px_it / ms / 1e3,
                               "steps": steps, "warmup": max(2, warmup),
                               "gpu_launches_per_call": int(s1["kernel_launches"] - s0["kernel_launches"]) // calls}
    if compare:
        jobs = [(x[i], 0.5, 50, 300, syn.DYADIC_EDGES) for i in range(n)]
        for name, res in (("resident_batch", 1), ("per_step_batch", 0)):
            with tv.Plan(local, resident=res) as p:
                ms = timed(lambda: p.decompose_batch(jobs, stream=stream), reps=1, warm=2)
                out[name] = {"images_per_s": n / ms * 1e3, "ms": ms, "Mpx_iter_per_s": px_it / ms / 1e3}
        out["training_set_over_per_step"] = (out["training_set"]["images_per_s"]
                                             / out["per_step_batch"]["images_per_s"])
    return out


def run_training(args, tv, torch, local, ws):
    dev = torch.device("cuda", local)
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    with ClockSampler(local) as clk:
        m = measure_crops(tv, torch, local, args.crops, compare=not args.quick, acc_mode=args.acc_mode,
                          steps=args.steps, warmup=args.warmup)
    t = m["training_set"]
    # the resident kernel is one launch per call and > 99 % of its device time (launch list in
    # profiles/); the call's event-timed duration bounds the kernel's from above
    flops = ALG_FLOPS_PER_PX_ITER * args.crops * 64 * 64 * 50 * 300
    achieved = flops / (t["ms"] / 1e3) / 1e12
    result = {"metric": "Chambolle Mpx*iter/s", "value": t["Mpx_iter_per_s"], "unit": "Mpx*iter/s",
              "n_gpus": ws, "steps": t["steps"], "warmup": t["warmup"], "ms_per_step": t["ms"], "higher_is_better": True,
              "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
              "config": {"workload": m["workload"], "images": args.crops,
                         "l2": "inputs and workspace (~0.5 GB) larger than L2"},
              "gpu_launches": t["gpu_launches_per_call"] * t["steps"],
              "roofline": {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                           "frac": achieved / FP32_PEAK_TFLOPS, "traffic": None, "kernel": "k_resident",
                           "peak_source": "nominal, not measured: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz",
                           "algorithmic_flops_per_launch": flops},
              # the square root and the reciprocal of every pixel-iteration run on the XU pipe
              # (16 results per SM per clock, nominal): the second ceiling of this kernel
              "roofline_xu": {"bound": "alu", "unit": "Gop/s", "kernel": "k_resident",
                              "achieved": 2 * flops / ALG_FLOPS_PER_PX_ITER / (t["ms"] / 1e3) / 1e9,
                              "peak": XU_PEAK_GOPS,
                              "frac": 2 * flops / ALG_FLOPS_PER_PX_ITER / (t["ms"] / 1e3) / 1e9 / XU_PEAK_GOPS,
                              "peak_source": "nominal, not measured: 152 SMs x 16 XU results per clock x 2.07 GHz",
                              "ops_per_px_iter": 2},
              "clocks": clk.summary(), "training": m}
    print(json.dumps(result))
    return 0


def run_batched(args, tv, torch, local, ws):
    dev = torch.device("cuda", local)
    torch.cuda.set_stream(torch.cuda.Stream(dev))
    with ClockSampler(local) as clk:
        m = measure_batched(tv, torch, local, args.steps, args.warmup)
    result = {"metric": "Chambolle Mpx*iter/s", "value": m["batched_Mpx_iter_per_s"], "unit": "Mpx*iter/s",
              "n_gpus": ws, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["batched_ms"],
              "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
              "data": "synthetic",
              "config": {"workload": m["workload"], "images": m["images"], "l2": "flushed before every timed step",
                         "tile": m["tile"], "temporal_block": m["temporal_block"]},
              "gpu_launches": m["gpu_launches"], "clocks": clk.summary(), "batched": m}
    if _dist()[1] == 0 and not args.no_cpu_baseline:
        sample = syn.config2().jobs[:8]
        v, el, cores = _oracle_batch_sample(sample)
        result["cpu_baseline"] = {"value": v, "unit": "Mpx*iter/s", "cores": cores, "kind": "oracle",
                                  "sample": f"the first 8 of the 64 images, all their ROF steps ({el:.1f} s); "
                                            "Mpx*iter/s applies to the whole batch by its px*iter"}
    print(json.dumps(result))
    return 0


def config4_pool():
    """8 synthetic images per served size (config-1 generator, shapes scaled with the area)."""
    return {s: [syn.make_image(s, s, max(1, int(40 * s * s / 512 ** 2)), (2.0, 60.0), (0.05, 1.0), 0.02,
                               4000 + 10 * s + k) for k in range(8)] for s in (256, 512, 1024, 2048)}


def config4_requests(pool, rate: float, n_req: int):
    """Poisson arrivals at `rate` req/s of requests: size 256^2..2048^2 with weights
    .4/.3/.2/.1, K ~ U{20..50}, dt .5, 300 iterations, 6 dyadic bands (seeded by the rate)."""
    rng = np.random.default_rng(4000 + int(rate))
    arrivals, jobs = [], []
    t = 0.0
    for j in range(n_req):
        t += float(rng.exponential(1.0 / rate))
        s = int(rng.choice([256, 512, 1024, 2048], p=[0.4, 0.3, 0.2, 0.1]))
        K = int(rng.integers(20, 51))
        arrivals.append(t)
        jobs.append((pool[s][j % 8], 0.5, K, 300, syn.DYADIC_EDGES))
    return arrivals, jobs


def measure_serving(tv, local, rates, n_req):
    """Config 4: Poisson arrivals of single-image requests (sizes 256^2..2048^2 with weights
    .4/.3/.2/.1, K ~ U{20..50}, dt .5, 300 iterations, 6 bands) into the serving loop
    (continuous batching, 60 GiB budget). Per rate: images/s and p50/p99 latency (submit to
    finish, host clock); the same requests through the plain path one at a time, and as
    offline batches of up to 500 (each timed on its second run: workspace, tile choice and graph
    built by the first), for images/s. A pool of 8 images per size is reused (timing does not
    depend on the picture)."""
    pool = config4_pool()
    points = []
    for rate in rates:
        arrivals, jobs = config4_requests(pool, rate, n_req)
        px_it = sum(j[0].size * j[2] * j[3] for j in jobs)
        with tv.Plan(local) as plan:
            tw, _ = plan.submit(*jobs[0])  # warm the scheduler thread and its tile choice
            plan.wait(tw)
            plan.serving_stats(reset=True)
            tickets = []
            t0 = time.perf_counter()
            with ClockSampler(local) as clk:
                for a, job in zip(arrivals, jobs):
                    dt_wait = t0 + a - time.perf_counter()
                    if dt_wait > 0:
                        time.sleep(dt_wait)
                    tickets.append(plan.submit(*job)[0])
                for tk in tickets:
                    st = plan.wait(tk)
                    if st != 0:
                        raise SystemExit(f"served request failed: {st}")
            wall = time.perf_counter() - t0
            lat = plan.serving_stats()
        with tv.Plan(local) as plain:
            for job in jobs[:8]:
                plain.decompose(*job)
            t1 = time.perf_counter()
            for job in jobs:
                plain.decompose(*job)
            t_plain = time.perf_counter() - t1
            # offline batches of at most 500 requests (their host outputs stay a few GB)
            t_batch = 0.0
            for c0 in range(0, len(jobs), 500):
                part = jobs[c0:c0 + 500]
                plain.decompose_batch(part)  # workspace, tile choice and graph of this set
                t2 = time.perf_counter()
                plain.decompose_batch(part)
                t_batch += time.perf_counter() - t2
        points.append({"rate_req_per_s": rate, "requests": n_req, "served_images_per_s": n_req / wall,
                       "served_Mpx_iter_per_s": px_it / wall / 1e6,
                       "p50_ms": lat["p50_ms"], "p99_ms": lat["p99_ms"], "count": lat["count"],
                       "plain_images_per_s": n_req / t_plain,
                       "offline_batch_images_per_s": n_req / t_batch,
                       "plain_Mpx_iter_per_s": px_it / t_plain / 1e6,
                       "offered_duration_s": arrivals[-1], "wall_s": wall, "clocks": clk.summary()})
    return points


def run_serving(args, tv, torch, local, ws):
    rates = [float(x) for x in args.rates.split(",")]
    out = {"metric": "served images/s and p50/p99 latency", "workload": "config4_serving", "n_gpus": ws,
           "requests_per_rate": args.requests, "data": "synthetic"}
    out["load_points"] = measure_serving(tv, local, rates, args.requests)
    for p in out["load_points"]:
        print(json.dumps(p), flush=True)
    print(json.dumps(out))
    return 0


def run_kernel_only(args, tv, torch, local):
    """The dual-iteration kernel alone on an N x N image (config-1 generator, shapes scaled
    with the area): a small, self-contained case for profiler captures."""
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    torch.cuda.set_stream(stream)
    n = args.size
    f = syn.make_image(n, n, max(1, int(40 * n * n / 512 ** 2)), (2.0, 60.0), (0.05, 1.0), 0.02, 1000)
    plan = tv.Plan(local, tma=1 if args.tma else 0,
                   **({"kernel": tv.KERNEL_TILED, "tile": args.tile} if args.tile >= 0 else {}))
    pitch = tv.pitch_for(n)
    gl = torch.zeros((n, pitch), dtype=torch.float32, device=dev)
    gl[:, :n] = torch.from_numpy(f / 0.5).to(dev)
    p1 = torch.zeros_like(gl)
    p2 = torch.zeros_like(gl)
    plan.chambolle_iterate(gl, p1, p2, n, n, pitch, 8, stream=stream)
    torch.cuda.synchronize()
    depth = max(1, plan.stats()["last_temporal_block"])
    iters = depth * args.launches
    plan.chambolle_iterate(gl, p1, p2, n, n, pitch, iters, stream=stream)  # same call, untimed
    torch.cuda.synchronize()
    s0 = plan.stats()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.chambolle_iterate(gl, p1, p2, n, n, pitch, iters, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    s1 = plan.stats()
    nl = int(s1["kernel_launches"] - s0["kernel_launches"])
    us = e0.elapsed_time(e1) * 1000 / max(nl, 1)
    alg = ALG_BYTES_FP32 * n * n * depth
    print(json.dumps({"kernel_only": True, "size": n, "tile": s1["last_tile"], "depth": depth,
                      "launches": nl, "per_launch_us": us, "effective_GBps": alg / (us * 1e-6) / 1e9,
                      "Mpx_iter_per_s": n * n * depth / (us * 1e-6) / 1e6}))
    plan.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--crops", type=int, default=3000, help="crops of the training workload")
    ap.add_argument("--acc-mode", type=int, default=0, choices=[0, 1],
                    help="epilogue arithmetic: 0 float64, 1 compensated float32")
    ap.add_argument("--workload", default="config1",
                    choices=["config1", "m1024", "config2", "config3", "config4", "training"])
    ap.add_argument("--rates", default="20,50,100,200", help="config4: Poisson arrival rates (req/s)")
    ap.add_argument("--requests", type=int, default=200, help="config4: requests per rate")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-k", type=int, default=50, help="ROF steps of the oracle's CPU sample")
    ap.add_argument("--ref-steps-k", type=int, default=6, help="ROF steps per reference-arm step")
    ap.add_argument("--quick", action="store_true",
                    help="skip the 1024^2, batched and serving summaries of the default run")
    ap.add_argument("--serve-rates", default="20,50,100,200", help="config4 load points of the default run (req/s)")
    ap.add_argument("--serve-requests", type=int, default=300,
                    help="requests per load point of the default run (config 4 specifies 2000)")
    ap.add_argument("--kernel-only", action="store_true",
                    help="time only the dual-iteration kernel on a --size x --size image")
    ap.add_argument("--size", type=int, default=4096)
    ap.add_argument("--launches", type=int, default=6)
    ap.add_argument("--tma", action="store_true",
                    help="tile loads by the tensor memory accelerator (config tma = 1)")
    ap.add_argument("--tile", type=int, default=-1,
                    help="fixed tile shape of the dual-iteration kernel (-1 = autotune), e.g. to pin the "
                         "autotuner's choice under a profiler")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
