#!/usr/bin/env python3
"""Benchmark: shaded point-sphere pairs per second, forward + backward.

Workload: the human-scale G-buffer -- 512 x 512 shading points from a
synthetic capsule-body depth map, 100 occluder spheres, 16 SH coefficients
(n = 4 bands) x 3 colour channels.  One step is one analysis-by-synthesis
pass of the whole shading path: the forward shading (per-pair log-visibility,
SH exponential, cosine lobe, triple product, lighting) followed by the L2 loss
against a perturbed target render and the adjoint pass (gradients for
lighting, albedo, sphere centres and radii).  Units: P x N pairs per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 oracle on the host cores instead (a
deliberately slow baseline, bounded sample of the same workload).
Under torchrun each rank shades its own copy of the workload (weak scaling,
no collective on the data path); rank 0 prints one JSON line.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

# The oracle baseline is timed single-threaded; pin BLAS pools before numpy loads.
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")

import numpy as np  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "shaded point-sphere pairs/sec fwd+bwd (512², 100 spheres, 16 SH coeffs); p50/p99 latency"
WORKLOAD = "capsule-body G-buffer 512x512 points, 100 spheres, n_bands=4 (16 SH coeffs x 3 ch), fwd + L2 loss + bwd"
N_BANDS = 4
SMS = 152
FP32_LANES_PER_SM = 128
SM_MAX_MHZ = 2070.0


def gaunt_nnz(n):
    """(nnz of C_ijk, nnz over j <= k) for n bands -- for the flop model."""
    sys.path.insert(0, os.path.join(ROOT, "paper_2104_00359_gb300", "csrc"))
    try:
        import gen_tables
        g = gen_tables.gaunt_monomial(n)
    finally:
        sys.path.pop(0)
    nnz_sym = len(g)
    nnz = sum(1 if j == k else 2 for (_, j, k) in g)
    return nnz, nnz_sym


def flop_model(n, n_spheres, k_mean):
    """Algorithmic FP32 flops per shading point:
    pair terms 4n^2+5n+14 (fwd) and 9n^2+10n+50 (bwd) per sphere; tails
    2 nnz_sym k + 2 nnz + 10K (fwd) and 2 nnz_sym k + 2 nnz k + 6 nnz + 18K (bwd)."""
    K = n * n
    nnz, nnz_sym = gaunt_nnz(n)
    pf = 4 * n * n + 5 * n + 14
    pb = 9 * n * n + 10 * n + 50
    tf = 2 * nnz_sym * k_mean + 2 * nnz + 10 * K
    tb = 2 * nnz_sym * k_mean + 2 * nnz * k_mean + 6 * nnz + 18 * K
    return dict(fwd=n_spheres * pf + tf, bwd=n_spheres * pb + tb)


KERNEL_SOURCES = ("paper_2104_00359_gb300/csrc/shs_kern.cu", "paper_2104_00359_gb300/csrc/shs_internal.h",
                  "paper_2104_00359_gb300/csrc/shs_exp.cuh", "paper_2104_00359_gb300/csrc/shs_warp.cuh",
                  "paper_2104_00359_gb300/csrc/generated/shs_sh_gen.cuh")


def kernel_source_hash():
    """Short hash of the sources the shading kernels are compiled from."""
    import hashlib
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_value(tag, kernel, workload_tag):
    """A per-launch figure of ``kernel`` recorded in a committed ncu summary,
    or None when the kernel sources changed since it was taken.  The summary
    carries lines '<tag> <kernel> <workload> <value> <source hash>'; tags:
    'traffic' (DRAM read + write bytes), 'flops' (executed FP32 flop: 2 per
    FFMA, 4 per FFMA2, 1 per FADD / FMUL, 2 per FADD2 / FMUL2)."""
    import glob
    want = kernel_source_hash()
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        with open(path) as fh:
            for line in fh:
                parts = line.strip().strip("`").split()
                if len(parts) == 5 and parts[0] == tag and parts[1] == kernel and parts[2] == workload_tag:
                    if parts[4] == want:
                        return float(parts[3])
    return None


def profiled_traffic(kernel, workload_tag):
    return profiled_value("traffic", kernel, workload_tag)


def read_ol_table(path):
    """(a, b, s_max) of a fitted optimal linear table file (columns s a b;
    s_max on the '# n_bands' header line)."""
    rows, s_max = [], None
    with open(path) as fh:
        for line in fh:
            if line.startswith("# n_bands"):
                s_max = float(line.split()[4])
            elif line.strip() and not line.startswith("#"):
                rows.append([float(x) for x in line.split()])
    rows = np.array(rows)
    return rows[:, 1].copy(), rows[:, 2].copy(), s_max


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.15)
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        rows = []
        for line in (self.out or "").splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        backend = "gloo" if args.impl == "reference" else "nccl"
        dist.init_process_group(backend)
        pg = dist
    return world, rank, local, pg


def bench_ours(args, world, rank, local, dist):
    import torch
    from paper_2104_00359_gb300 import Config, Scene, synthetic, _lib

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()
    sc = synthetic.capsule_body_scene(seed=1 + 1000 * rank, n_bands=N_BANDS)
    tgt_sc = synthetic.perturb_scene(sc, seed=2 + 1000 * rank)
    P = sc["points"].shape[0]
    Nsph = sc["centers"].shape[0]
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in ("points", "normals", "albedo", "centers", "radii", "light")}
    cfg = Config(n_bands=N_BANDS, deterministic=not args.atomic)
    # target render with the perturbed scene through the same library
    tscene = Scene(torch.from_numpy(tgt_sc["centers"]).to(dev), torch.from_numpy(tgt_sc["radii"]).to(dev),
                   torch.from_numpy(tgt_sc["light"]).to(dev), cfg)
    target = tscene.shade(T["points"], T["normals"], torch.from_numpy(tgt_sc["albedo"]).to(dev))
    torch.cuda.synchronize()
    tscene.close()

    scene = Scene(T["centers"], T["radii"], T["light"], cfg)
    saved = scene.new_saved(P, dev)
    radiance = torch.empty((P, 3), device=dev)
    want = ("light", "albedo", "centers", "radii")
    g = scene._grad_buffers(P, dev, want)
    loss = torch.empty((), device=dev)
    stream = torch.cuda.current_stream()
    sp = _lib.ptr
    sptr = _lib.ctypes.c_void_p(stream.cuda_stream)

    def step():
        _lib.check(lib.shs_shade(scene.handle, P, sp(T["points"]), sp(T["normals"]), sp(T["albedo"]),
                                 sp(radiance), sp(saved), sptr), "shs_shade")
        ev_mid.record(stream)
        _lib.check(lib.shs_shade_backward_l2(scene.handle, P, sp(T["points"]), sp(T["normals"]),
                                             sp(T["albedo"]), sp(saved), sp(radiance), sp(target), sp(loss),
                                             sp(g["d_light"]), sp(g["d_albedo"]), sp(g["d_centers"]),
                                             sp(g["d_radii"]), None, None, sptr), "shs_shade_backward_l2")

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MiB > L2
    W, K = args.warmup, args.steps
    ev_mid = torch.cuda.Event(enable_timing=True)
    for _ in range(W):
        step()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    mids = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = lib.shs_launch_count()
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for i in range(K):
            flush.zero_()
            starts[i].record(stream)
            ev_mid = mids[i]
            step()
            ends[i].record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        launches = lib.shs_launch_count() - launches0
        # latency distribution: a separate loop of >= 200 steps (and >= ~3 s,
        # so clock samples see the GPU under load), L2 flushed before each
        # step as above, CUDA events around each step
        est_ms = (t1 - t0) * 1e3 / K
        NL = args.latency_reps or int(min(20000, max(200, 3000.0 / max(est_ms, 1e-3))))
        ls = [torch.cuda.Event(enable_timing=True) for _ in range(NL)]
        le = [torch.cuda.Event(enable_timing=True) for _ in range(NL)]
        lm = [torch.cuda.Event(enable_timing=True) for _ in range(NL)]
        for i in range(NL):
            flush.zero_()
            ls[i].record(stream)
            ev_mid = lm[i]
            step()
            le[i].record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    lat_ms = sorted(s.elapsed_time(e) for s, e in zip(ls, le))
    step_ms = [s.elapsed_time(e) for s, e in zip(starts, ends)]
    fwd_ms = [s.elapsed_time(m) for s, m in zip(starts, mids)]
    bwd_ms = [m.elapsed_time(e) for m, e in zip(mids, ends)]
    mean_ms = statistics.fmean(step_ms)
    if dist:
        t = torch.tensor([mean_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        mean_ms = float(t.item())
    pairs = P * Nsph
    value = world * pairs / (mean_ms * 1e-3)
    kvals = scene.saved_views(saved, P)[1].float()
    k_mean = float(kvals.mean())
    fm = flop_model(N_BANDS, Nsph, k_mean)
    bwd_mean = statistics.fmean(bwd_ms)
    fwd_mean = statistics.fmean(fwd_ms)
    peak = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    # work per launch: the smaller of the algorithmic model and the FP32 flop
    # ncu counted in the kernel (recorded in profiles/ for these sources)
    exec_b = profiled_value("flops", "backward_kernel_t", "capsule512_n4")
    exec_f = profiled_value("flops", "forward_kernel_t", "capsule512_n4")
    work_b = min(P * fm["bwd"], exec_b) if exec_b else P * fm["bwd"]
    work_f = min(P * fm["fwd"], exec_f) if exec_f else P * fm["fwd"]
    achieved = work_b / (bwd_mean * 1e-3) / 1e12
    achieved_fwd = work_f / (fwd_mean * 1e-3) / 1e12
    p50 = lat_ms[len(lat_ms) // 2]
    p99 = lat_ms[min(len(lat_ms) - 1, int(round(0.99 * (len(lat_ms) - 1))))]

    # end to end through the public API: each step uploads its points, normals,
    # albedo and target from pinned host memory and downloads the gradients and
    # the loss; HostStepPipeline overlaps step i's kernels with the copies of
    # steps i-1 and i+1 on separate streams
    from paper_2104_00359_gb300.pipeline import HostStepPipeline
    host = {k: torch.from_numpy(sc[k]).pin_memory() for k in ("points", "normals", "albedo")}
    host["target"] = target.cpu().pin_memory()
    pipe = HostStepPipeline(scene, P, want=want, depth=2, device=dev)

    def e2e_run(n):
        for i in range(n):
            pipe.submit(host["points"], host["normals"], host["albedo"], host["target"])
            if i:
                pipe.result(i - 1 + base[0])
        pipe.result(n - 1 + base[0])
        base[0] += n

    base = [0]
    e2e_run(3)
    KE = max(3, min(K, 500))
    if dist:
        dist.barrier()
    te0 = time.perf_counter()
    e2e_run(KE)
    te1 = time.perf_counter()
    e2e_s = (te1 - te0) / KE
    if dist:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    h2d, d2h = pipe.bytes_per_step()
    pipe.synchronize()
    status = scene.device_status()
    scene.close()
    peaks = load_peaks()
    fma_peak = measure_fma_peak(lib, dev, stream)
    return dict(
        metric=METRIC, value=value, unit="pairs/s", n_gpus=world, steps=K, warmup=W,
        ms_per_step=mean_ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic", impl="ours",
        config={"workload": WORKLOAD, "points": P, "spheres": Nsph, "sh_coeffs": N_BANDS ** 2,
                "pairs_per_step": pairs, "l2_flush_between_steps": True,
                "deterministic_reduction": not args.atomic, "parallelism": f"replicas{world}"},
        latency_ms={"p50": p50, "p99": p99, "reps": len(lat_ms), "max": lat_ms[-1],
                    "source": "separate loop after the timed steps: CUDA events per step, L2 flushed before each",
                    "fwd_mean": fwd_mean, "bwd_mean": bwd_mean},
        roofline={"bound": "alu", "kernel": "backward (pair adjoints + tail adjoint)",
                  "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                  "traffic": profiled_traffic("backward_kernel_t", "capsule512_n4"),
                  "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per launch (profiles/), "
                                    "null when the kernel sources changed since",
                  "kernel_source_hash": kernel_source_hash(),
                  "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz",
                  "flops_per_point": work_b / P, "flops_per_point_model": fm["bwd"],
                  "flops_per_point_executed": exec_b / P if exec_b else None,
                  "work_basis": "min(model, ncu-executed FP32 flop)" if exec_b else "model (no current ncu count)",
                  "k_mean": k_mean,
                  "peak_measured": fma_peak, "frac_of_measured": achieved / fma_peak if fma_peak else None,
                  "peak_measured_source": "shs_fp32_fma_probe: 1216 x 256 threads x 8 FMA chains, CUDA events",
                  "forward": {"achieved": achieved_fwd, "frac": achieved_fwd / peak,
                              "frac_of_measured": achieved_fwd / fma_peak if fma_peak else None,
                              "flops_per_point": work_f / P, "flops_per_point_model": fm["fwd"],
                              "flops_per_point_executed": exec_f / P if exec_f else None}},
        e2e={"value": world * pairs / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": h2d,
             "d2h_bytes_per_step": d2h, "ms_per_step": e2e_s * 1e3, "steps": KE,
             "api": "HostStepPipeline (pinned host in/out, 3 streams, depth 2)"},
        gpu_launches=int(launches), clocks=clk.summary(), device_status=status,
        wall_s_timed=t1 - t0, hbm_peak_gbs=peaks.get("hbm_gbs"),
        cpu_baseline=cpu_baseline(args) if (rank == 0 and world == 1 and not args.no_cpu) else None,
    )


def measure_fma_peak(lib, dev, stream, iters=1 << 16, blocks=152 * 8):
    """FP32 FMA throughput (TFLOP/s) of the library's probe kernel: best of 3."""
    import ctypes
    import torch
    from paper_2104_00359_gb300 import _lib
    out = torch.empty(blocks * 256, device=dev)
    sptr = ctypes.c_void_p(stream.cuda_stream)
    best = None
    for _ in range(4):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        _lib.check(lib.shs_fp32_fma_probe(blocks, iters, _lib.ptr(out), sptr), "shs_fp32_fma_probe")
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return 16.0 * iters * blocks * 256 / (best * 1e-3) / 1e12


def _oracle_step(O, cfg, sc, idx, dB_seed=0):
    args = [sc[k][idx] for k in ("points", "normals", "albedo")] + [sc["centers"], sc["radii"], sc["light"]]
    fw = O.shade_forward(cfg, *args)
    dB = np.random.default_rng(dB_seed).normal(size=(len(idx), 3))
    O.shade_backward(cfg, *args, dB)
    return fw


def _oracle_cost(O, cfg, sc, rng):
    """(fixed seconds per call, seconds per point) of one oracle fwd + bwd
    call: its time is a per-call cost (the loop over spheres) plus a
    per-point cost, fitted from two timed calls after a warm-up call."""
    P = sc["points"].shape[0]
    _oracle_step(O, cfg, sc, rng.choice(P, 64, replace=False))
    t = time.perf_counter()
    _oracle_step(O, cfg, sc, rng.choice(P, 128, replace=False))
    t1 = time.perf_counter() - t
    t = time.perf_counter()
    _oracle_step(O, cfg, sc, rng.choice(P, 640, replace=False))
    t2 = time.perf_counter() - t
    per_pt = max((t2 - t1) / 512, 1e-7)
    return max(t1 - 128 * per_pt, 0.0), per_pt


_WORKER = {}


def _oracle_worker_init():
    from oracle import shs_oracle as O
    from paper_2104_00359_gb300 import synthetic
    _WORKER["O"] = O
    _WORKER["sc"] = synthetic.capsule_body_scene(seed=1, n_bands=N_BANDS)
    _WORKER["cfg"] = O.Config(n_bands=N_BANDS)


def _oracle_worker(task):
    seed, n = task
    sc = _WORKER["sc"]
    idx = np.random.default_rng(seed).choice(sc["points"].shape[0], n, replace=True)
    _oracle_step(_WORKER["O"], _WORKER["cfg"], sc, idx)
    return n


def cpu_baseline_all_cores(fixed, per_pt, budget_s=15.0):
    """The same oracle step on every host core: one single-threaded process
    per core (spawned: this process already holds a CUDA context), two point
    chunks per process, timed around the parallel map after a warm-up."""
    import multiprocessing as mp
    cores = max(1, os.cpu_count() or 1)
    chunk = int(max(256, (budget_s / 2 - fixed) / per_pt))
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=cores, initializer=_oracle_worker_init) as pool:
        pool.map(_oracle_worker, [(1000 + i, 64) for i in range(cores)], chunksize=1)
        t = time.perf_counter()
        done = pool.map(_oracle_worker, [(i, chunk) for i in range(2 * cores)], chunksize=1)
        dt = time.perf_counter() - t
    return {"value": sum(done) * 100 / dt, "unit": "pairs/s", "cores": cores, "kind": "oracle",
            "sample": f"{2 * cores} chunks of {chunk} random points (with replacement) of the 512x512 "
                      f"capsule-body G-buffer x 100 spheres, fwd + bwd, float64 numpy, {cores} single-threaded "
                      f"processes, {dt:.1f} s"}


def cpu_baseline(args, budget_s=15.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload:
    single-threaded, and on every host core (``all_cores``)."""
    from oracle import shs_oracle as O
    from paper_2104_00359_gb300 import synthetic
    sc = synthetic.capsule_body_scene(seed=1, n_bands=N_BANDS)
    cfg = O.Config(n_bands=N_BANDS)
    rng = np.random.default_rng(0)
    fixed, per_pt = _oracle_cost(O, cfg, sc, rng)
    n = int(max(512, min(65536, (budget_s - fixed) / per_pt)))
    idx = rng.choice(sc["points"].shape[0], n, replace=False)
    t = time.perf_counter()
    _oracle_step(O, cfg, sc, idx)
    dt = time.perf_counter() - t
    pairs = n * sc["centers"].shape[0]
    out = {"value": pairs / dt, "unit": "pairs/s", "cores": 1, "kind": "oracle",
           "sample": f"{n} random points of the 512x512 capsule-body G-buffer x 100 spheres, "
                     f"fwd + bwd, float64 numpy, 1 thread, {dt:.1f} s"}
    try:
        out["all_cores"] = cpu_baseline_all_cores(fixed, per_pt)
    except Exception as e:                      # report, never fail the GPU bench over the baseline
        out["all_cores"] = {"error": f"{type(e).__name__}: {e}"}
    return out


def bench_reference(args, world, rank, budget_s=120.0):
    """The oracle as the reference arm: same metric and workload, K timed
    steps of a bounded point sample each.  The oracle has a per-call cost of
    about a second (its loop over spheres); when K + W such calls would not
    end within the budget, G consecutive steps' samples go through one call
    and each step is charged 1/G of that call's time."""
    if rank != 0:
        return None
    from oracle import shs_oracle as O
    from paper_2104_00359_gb300 import synthetic
    sc = synthetic.capsule_body_scene(seed=1, n_bands=N_BANDS)
    cfg = O.Config(n_bands=N_BANDS)
    rng = np.random.default_rng(0)
    fixed, per_pt = _oracle_cost(O, cfg, sc, rng)
    K, W = args.steps, args.warmup
    lo = 16
    if (K + W) * (fixed + lo * per_pt) <= budget_s:
        G = 1
        n = int(max(lo, min(16384, (budget_s / (K + W) - fixed) / per_pt)))
    else:
        n = lo
        left = max(budget_s - (K + W) * n * per_pt, fixed)
        G = int(np.ceil((K + W) * fixed / left))
    P = sc["points"].shape[0]

    def calls(steps):
        out = []
        while steps > 0:
            g = min(G, steps)
            out.append(g)
            steps -= g
        return out

    for g in calls(W):
        _oracle_step(O, cfg, sc, rng.choice(P, n * g, replace=False))
    times = []
    for g in calls(K):
        idx = rng.choice(P, n * g, replace=False)
        t = time.perf_counter()
        _oracle_step(O, cfg, sc, idx)
        times += [(time.perf_counter() - t) / g] * g
    Nsph = sc["centers"].shape[0]
    mean_s = statistics.fmean(times)
    value = n * Nsph / mean_s
    srt = sorted(times)
    sample = (f"{n} random points per step of the 512x512 capsule-body G-buffer x 100 spheres, "
              f"{G} step(s) per oracle call, fwd + bwd, float64 numpy, 1 thread")
    return dict(metric=METRIC, value=value, unit="pairs/s", n_gpus=world, steps=K, warmup=W,
                ms_per_step=mean_s * 1e3, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f64",
                data="synthetic", impl="reference",
                config={"workload": WORKLOAD, "points": int(P), "spheres": Nsph,
                        "sh_coeffs": N_BANDS ** 2, "points_per_step_sampled": n, "steps_per_oracle_call": G},
                latency_ms={"p50": srt[len(srt) // 2] * 1e3, "p99": srt[min(len(srt) - 1, int(0.99 * (len(srt) - 1)))] * 1e3},
                cpu_baseline={"value": value, "unit": "pairs/s", "cores": 1, "kind": "oracle", "sample": sample},
                e2e={"value": value, "unit": "pairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0})


def bench_serving(args, world, rank, local):
    """The serving mix: 64 resident jobs (16,384 to 1,048,576 points, log-
    uniform; 20 to 500 spheres; 4 or 6 SH bands), 2,000 Poisson requests (70 %
    forward, 30 % forward + L2 backward) at 80 % of the per-call capacity,
    served by the continuous-batching server and, for comparison, by per-call
    launches in arrival order.  Throughput in pairs/s; latency from arrival to
    completion."""
    import torch
    from paper_2104_00359_gb300 import Config, Scene, serve, synthetic
    torch.cuda.set_device(local)
    rng = np.random.default_rng(4 + 1000 * rank)
    n_jobs, n_req = args.serve_jobs, args.serve_requests
    srv = serve.Server(hbm_budget_bytes=80e9, n_slots=args.serve_slots, max_batch=32, chunk_points=args.serve_chunk,
                       batch_work=args.serve_batch_work, small_work=args.serve_small_work)
    for j in range(n_jobs):
        P = int(np.exp(rng.uniform(np.log(16384), np.log(1048576))))
        N = int(rng.integers(20, 501))
        n = 4 if rng.random() < 0.5 else 6
        sc = synthetic.serving_job(10_000 + j, P, N, n)
        cfg = Config(n_bands=n, deterministic=False)
        dev = torch.device("cuda", local)
        light_t = torch.from_numpy(sc["light"]).to(dev)
        tsc = Scene(torch.from_numpy(sc["centers"]).to(dev), torch.from_numpy(sc["radii"]).to(dev),
                    light_t + 0.05 * torch.randn_like(light_t), cfg)
        target = tsc.shade(*(torch.from_numpy(sc[k]).to(dev) for k in ("points", "normals", "albedo")))
        torch.cuda.synchronize()
        tsc.close()
        srv.add_job(j, sc["points"], sc["normals"], sc["albedo"], sc["centers"], sc["radii"], sc["light"],
                    cfg, target=target)
    runner = serve.PerCallRunner(srv.jobs)
    # per-call capacity: one fwd and one fwdbwd per job, timed on the device
    t_fwd, t_fb = [], []
    for j in range(n_jobs):
        for op, acc in (("fwd", t_fwd), ("fwdbwd", t_fb)):
            runner.run(serve.Request(-1, j, op, 0.0)).synchronize()
            t0 = time.perf_counter()
            runner.run(serve.Request(-1, j, op, 0.0)).synchronize()
            acc.append(time.perf_counter() - t0)
    mean_service = 0.7 * statistics.fmean(t_fwd) + 0.3 * statistics.fmean(t_fb)
    rate = 0.8 / mean_service
    gaps = rng.exponential(1.0 / rate, n_req)
    arrivals = np.cumsum(gaps)
    req_jobs = rng.integers(0, n_jobs, n_req)
    req_ops = np.where(rng.random(n_req) < 0.3, "fwdbwd", "fwd")

    def run_server():
        t0 = time.perf_counter()
        reqs, i = [], 0
        while i < n_req or not srv.idle():
            now = time.perf_counter() - t0
            while i < n_req and arrivals[i] <= now:
                reqs.append(srv.submit(int(req_jobs[i]), str(req_ops[i]), arrival=t0 + arrivals[i]))
                i += 1
            srv.poll()
        return reqs, t0

    def run_percall():
        t0 = time.perf_counter()
        done, inflight, i = [], deque(), 0
        while i < n_req or inflight:
            now = time.perf_counter() - t0
            while i < n_req and arrivals[i] <= now:
                r = serve.Request(i, int(req_jobs[i]), str(req_ops[i]), t0 + arrivals[i])
                inflight.append((r, runner.run(r)))
                i += 1
            while inflight and inflight[0][1].query():
                r, _ = inflight.popleft()
                r.done = time.perf_counter()
                job = srv.jobs[r.job_id]
                r.pairs = job.P * job.N
                done.append(r)
        return done, t0

    def summarise(reqs, t0):
        lat = [r.latency * 1e3 for r in reqs]
        span = max(r.done for r in reqs) - t0
        pairs = sum(r.pairs for r in reqs)
        out = {"value": pairs / span, "p50_ms": serve.percentile(lat, 0.5), "p99_ms": serve.percentile(lat, 0.99),
               "span_s": span, "requests": len(reqs)}
        # latency by request size: jobs under 100k points, and the rest
        for name, test in (("under_100k_points", lambda P: P < 100_000), ("100k_points_and_up", lambda P: P >= 100_000)):
            sel = [r.latency * 1e3 for r in reqs if test(srv.jobs[r.job_id].P)]
            out[name] = {"requests": len(sel), "p50_ms": serve.percentile(sel, 0.5),
                         "p99_ms": serve.percentile(sel, 0.99)}
        return out

    from collections import deque
    pc_reqs, pc_t0 = run_percall()
    torch.cuda.synchronize()
    sv_reqs, sv_t0 = run_server()
    torch.cuda.synchronize()
    sv = summarise(sv_reqs, sv_t0)
    pc = summarise(pc_reqs, pc_t0)
    # saturated: every request available at t = 0 (capacity of each path)
    saved_arrivals = arrivals.copy()
    arrivals[:] = 0.0
    pcs_reqs, pcs_t0 = run_percall()
    torch.cuda.synchronize()
    svs_reqs, svs_t0 = run_server()
    torch.cuda.synchronize()
    arrivals[:] = saved_arrivals
    svs = summarise(svs_reqs, svs_t0)
    pcs = summarise(pcs_reqs, pcs_t0)
    srv.close()
    return dict(metric="serving mix: shaded point-sphere pairs/sec (64 jobs, 2000 Poisson requests); p50/p99 latency",
                value=sv["value"], unit="pairs/s", n_gpus=world, higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f32", data="synthetic", impl="ours",
                config={"workload": "serving mix: 64 resident jobs, 16,384-1,048,576 points (log-uniform), "
                                    "20-500 spheres, n_bands 4 or 6, 70% fwd / 30% fwd+L2 bwd, Poisson arrivals "
                                    "at 80% of per-call capacity, 80 GB HBM budget",
                        "jobs": n_jobs, "requests": n_req, "rate_per_s": rate,
                        "mean_per_call_service_ms": mean_service * 1e3, "slots": args.serve_slots, "max_batch": 32,
                        "small_work": srv.small_work},
                latency_ms={"p50": sv["p50_ms"], "p99": sv["p99_ms"],
                            "under_100k_points": sv["under_100k_points"],
                            "100k_points_and_up": sv["100k_points_and_up"]},
                batches=srv.batches, max_batches_in_flight=srv.max_inflight, chunk_points=srv.chunk_points,
                batch_work=srv.batch_work,
                per_call_baseline={"value": pc["value"], "unit": "pairs/s",
                                   "latency_ms": {"p50": pc["p50_ms"], "p99": pc["p99_ms"],
                                                  "under_100k_points": pc["under_100k_points"],
                                                  "100k_points_and_up": pc["100k_points_and_up"]}},
                span_s={"server": sv["span_s"], "per_call": pc["span_s"]},
                saturated={"server": {"value": svs["value"], "span_s": svs["span_s"]},
                           "per_call": {"value": pcs["value"], "span_s": pcs["span_s"]},
                           "unit": "pairs/s"})


def bench_heightfield(args, world, rank, local):
    """The precision workload: 1,048,576 points of a 1024x1024 height field,
    300 spheres (radii log-uniform [0.01, 0.2]), n_bands = 8 (64 SH coeffs):
    forward and backward times per precision, and the error of every output
    against the FP64 oracle: the shading and adjoint of a random sample of
    256 points (radiance and each gradient, the scene sums over the sample)."""
    import torch
    from oracle import shs_oracle as O
    from paper_2104_00359_gb300 import Config, Scene, synthetic
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    sc = synthetic.height_field_scene(seed=3, res=args.hf_res)
    fields = ("points", "normals", "albedo", "centers", "radii", "light")
    T = {k: torch.from_numpy(sc[k]).to(dev) for k in fields}
    P, N = sc["points"].shape[0], sc["centers"].shape[0]
    sel = np.sort(np.random.default_rng(1).choice(P, 256, replace=False))
    Ts = {k: (T[k][torch.from_numpy(sel).to(dev)].contiguous() if k in ("points", "normals", "albedo") else T[k])
          for k in fields}
    args_o = [sc[f][sel] if f in ("points", "normals", "albedo") else sc[f] for f in fields]
    dBs = np.random.default_rng(2).normal(size=(len(sel), 3)).astype(np.float32)
    out = {}
    # (name, precision, exp_mode): precision 2 / 1 / 3 are the tensor-core
    # tails in BF16 / TF32 / FP16; exp_mode 1 is the projected-exponential
    # variant, 2 the optimal linear step with the fitted 8-band table
    all_precs = (("fp32", 0, 0), ("bf16_tc", 2, 0), ("tf32_tc", 1, 0), ("fp16_tc", 3, 0), ("fp32_projexp", 0, 1),
                 ("bf16_tc_projexp", 2, 1), ("tf32_tc_projexp", 1, 1), ("fp32_oltable", 0, 2))
    # the library stores the table as float32: give the oracle the same values
    table = tuple(np.float32(x).astype(np.float64) if i < 2 else x for i, x in
                  enumerate(read_ol_table(os.path.join(ROOT, "tests", "golden", "ol_table_n8.txt"))))
    fine = None
    fma_peak = None
    oracle_cache = {}
    grads = ("d_light", "d_albedo", "d_centers", "d_radii", "d_points", "d_normals")
    for prec_name, prec, mode in [x for x in all_precs if x[0] in args.precisions.split(",")]:
        scene = Scene(T["centers"], T["radii"], T["light"], Config(n_bands=8, precision=prec, exp_mode=mode))
        if mode == 2:
            scene.set_ol_table(*table)
        saved = scene.new_saved(P, dev)
        dB = torch.randn((P, 3), device=dev)
        times_f, times_b = [], []
        for it in range(args.warmup + args.steps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            B = scene.shade(T["points"], T["normals"], T["albedo"], saved=saved)
            e1.record()
            scene.backward(T["points"], T["normals"], T["albedo"], dB, saved=saved,
                           want=("light", "albedo", "centers", "radii"))
            e2.record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                times_f.append(e0.elapsed_time(e1))
                times_b.append(e1.elapsed_time(e2))
        k = scene.saved_views(saved, P)[1].cpu().numpy().astype(np.int64)
        # the exponential and shading alone (shs_shade_tail), and the adjoint
        # without the pair terms (only lighting, albedo and normal gradients)
        tail_f, tail_b = [], []
        Bt = torch.empty_like(B)
        for it in range(args.warmup + args.steps):
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            scene.shade_tail(T["normals"], T["albedo"], saved, out=Bt)
            e1.record()
            scene.backward(T["points"], T["normals"], T["albedo"], dB, saved=saved,
                           want=("light", "albedo", "normals"))
            e2.record()
            torch.cuda.synchronize()
            if it >= args.warmup:
                tail_f.append(e0.elapsed_time(e1))
                tail_b.append(e1.elapsed_time(e2))
        # every output on the sample: shading and adjoint of the 256 sampled points
        svs = scene.new_saved(len(sel), dev)
        Bs = scene.shade(Ts["points"], Ts["normals"], Ts["albedo"], saved=svs)
        gs = scene.backward(Ts["points"], Ts["normals"], Ts["albedo"], torch.from_numpy(dBs).to(dev), saved=svs)
        torch.cuda.synchronize()
        ks = scene.saved_views(svs, len(sel))[1].cpu().numpy().astype(np.int64)
        ocfg = O.Config(n_bands=8, exp_mode=mode, ol_table=table if mode == 2 else None)
        key = (mode, ks.tobytes())
        if key not in oracle_cache:
            oracle_cache[key] = O.shade_backward(ocfg, *args_o, dBs.astype(np.float64), k=ks)
        ref = oracle_cache[key]
        errs = {"radiance": _norm_err(Bs.cpu().numpy(), ref["forward"]["radiance"])}
        for name in grads:
            errs[name] = _norm_err(gs[name].cpu().numpy(), ref[name], ref.get("abs_" + name))
        got_full = B.cpu().numpy()[sel]
        out[prec_name] = {"fwd_ms": statistics.fmean(times_f), "bwd_ms": statistics.fmean(times_b),
                          "pairs_per_s_fwd": P * N / (statistics.fmean(times_f) * 1e-3),
                          "pairs_per_s_fwd_bwd": P * N / ((statistics.fmean(times_f) + statistics.fmean(times_b)) * 1e-3),
                          "max_rel_err_vs_fp64": errs,
                          "full_size_radiance_matches_sample": bool(np.allclose(got_full, Bs.cpu().numpy(), rtol=0,
                                                                                atol=1e-6 * np.abs(got_full).max())),
                          "k_mean": float(k.mean()),
                          "tail_fwd_ms": statistics.fmean(tail_f), "tail_bwd_ms": statistics.fmean(tail_b)}
        if prec != 0:
            out[prec_name]["roofline_tail"] = _tc_tail_roofline(prec, k, statistics.fmean(tail_f),
                                                                statistics.fmean(tail_b), mode)
        elif mode == 0:
            if fma_peak is None:
                from paper_2104_00359_gb300 import _lib
                fma_peak = measure_fma_peak(_lib.load(), dev, torch.cuda.current_stream())
            out[prec_name]["roofline"] = _fp32_roofline_n8(P, N, float(k.mean()), statistics.fmean(times_f),
                                                           statistics.fmean(times_b), fma_peak)
        if mode in (1, 2):
            # accuracy of the exponential methods (FP64) against the projection of
            # exp(f) by a fine rule (64 x 128 nodes) on the same sample
            if fine is None:
                fine = O.shade_forward(O.Config(n_bands=8, exp_mode=1, exp_rule=(64, 128)), *args_o)["radiance"]

            def rel(x):
                d = np.abs(x - fine) / np.maximum(np.abs(fine), 1e-3 * np.abs(fine).max())
                return {"max": float(d.max()), "median": float(np.median(d))}
            sq = O.shade_forward(O.Config(n_bands=8), *args_o)["radiance"]
            out[prec_name]["vs_fine_projection_fp64"] = {
                "projected_2n_x_4n" if mode == 1 else "fitted_ol_table": rel(ref["forward"]["radiance"]),
                "scaling_squaring": rel(sq)}
        scene.close()
    first = next(iter(out.values()))
    return dict(metric="height field 1024^2 x 300 spheres, n_bands=8: pairs/sec and error vs FP64 per precision",
                value=first["pairs_per_s_fwd_bwd"], unit="pairs/s", n_gpus=world, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f32", data="synthetic", impl="ours",
                config={"workload": f"height field {args.hf_res}x{args.hf_res} points, 300 spheres, n_bands=8 (64 SH coeffs)",
                        "points": P, "spheres": N, "error_sample_points": int(len(sel))},
                precisions=out)


def _fp32_roofline_n8(P, N, k_mean, fwd_ms, bwd_ms, fma_peak):
    """The FP32 CUDA-core 8-band step against the FP32 FMA peak.  Work per
    point = the smaller of the flop model (flop_model) and the FP32 flop the
    kernels execute per point, counted by ncu on the 512 x 512 height field
    (same 300 spheres; 'flops <kernel> heightfield512_n8' lines in profiles/,
    used only while the kernel sources are unchanged).  Forward: the shading
    kernel; backward: the tail adjoint pass and the pair pass (the lighting
    reduction is not counted)."""
    fm = flop_model(8, N, k_mean)
    peak = SMS * FP32_LANES_PER_SM * 2 * SM_MAX_MHZ * 1e6 / 1e12
    pts512 = 512 * 512
    ex_f = profiled_value("flops", "forward_kernel_t", "heightfield512_n8")
    ex_t = profiled_value("flops", "backward_kernel_t", "heightfield512_n8")
    ex_p = profiled_value("flops", "bwd_pairs_t_kernel", "heightfield512_n8")
    ex_f = ex_f / pts512 if ex_f else None
    ex_b = (ex_t + ex_p) / pts512 if (ex_t and ex_p) else None
    wf = min(fm["fwd"], ex_f) if ex_f else fm["fwd"]
    wb = min(fm["bwd"], ex_b) if ex_b else fm["bwd"]
    af = wf * P / (fwd_ms * 1e-3) / 1e12
    ab = wb * P / (bwd_ms * 1e-3) / 1e12
    return {"bound": "alu", "unit": "TFLOP/s", "peak": peak,
            "peak_source": f"{SMS} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 flop x {SM_MAX_MHZ:.0f} MHz",
            "peak_measured": fma_peak,
            "forward": {"achieved": af, "frac": af / peak, "frac_of_measured": af / fma_peak if fma_peak else None,
                        "flops_per_point": wf, "flops_per_point_model": fm["fwd"],
                        "flops_per_point_executed": ex_f},
            "backward": {"achieved": ab, "frac": ab / peak, "frac_of_measured": ab / fma_peak if fma_peak else None,
                         "flops_per_point": wb, "flops_per_point_model": fm["bwd"],
                         "flops_per_point_executed": ex_b},
            "work_basis": "min(model, ncu-executed FP32 flop per point)" if (ex_f and ex_b)
                          else "model (no current ncu count)",
            "k_mean": k_mean, "kernel_source_hash": kernel_source_hash()}


def _tc_tail_roofline(prec, k, fwd_ms, bwd_ms, mode=0):
    """Tensor-core tails against the measured dense peak of their operand type.
    Work = the MMAs the method issues: per 128-point tile (kt = the tile's
    largest k) and pass over the Q quadrature directions, the evaluation
    GEMM X = S Y^T and the projection GEMM (X o X)(w Y) are 2 x 128 x Q x 64
    flop each, times the product terms of the split operands (BF16: 6, TF32 /
    FP16: 3).  Forward: kt squaring passes (2 GEMMs) and a shading pass (1).
    Adjoint: kt recomputed squarings (2), the shading adjoint (1 + 2) and kt
    squaring adjoints (2 evaluations + 1 projection): 5 kt + 3.  Squarings:
    Q = 256 (the 11 x 22 product rule); the projected exponential (mode 1):
    Q = 512 (its 16 x 32 rule) and kt = 1 (one exp pass)."""
    peaks = load_peaks()
    bf16 = peaks.get("bf16_tflops") or 1900.0
    terms = 6 if prec == 2 else 3
    # TF32 at the recipe's nominal ratio to BF16 (1.1 / 2.25 PFLOP/s dense)
    peak = bf16 * (1.1 / 2.25) if prec == 1 else bf16
    P = k.shape[0]
    kt = np.array([k[i:i + 128].max() for i in range(0, P, 128)], np.int64)
    Q = 256
    if mode == 1:
        kt = np.ones_like(kt)
        Q = 512
    gemm = 2.0 * 128 * Q * 64 * terms
    f_fwd = gemm * float(np.sum(2 * kt + 1))
    f_bwd = gemm * float(np.sum(5 * kt + 3))
    a_f = f_fwd / (fwd_ms * 1e-3) / 1e12
    a_b = f_bwd / (bwd_ms * 1e-3) / 1e12
    return {"bound": "tensor", "unit": "TFLOP/s", "peak": peak,
            "peak_source": "MEASURED_PEAKS bf16_tflops (burst)" + (" x 1.1/2.25 (TF32 nominal ratio)" if prec == 1 else ""),
            "forward": {"achieved": a_f, "frac": a_f / peak, "flop": f_fwd, "ms": fwd_ms},
            "adjoint": {"achieved": a_b, "frac": a_b / peak, "flop": f_bwd, "ms": bwd_ms,
                        "note": "includes the fixed-order lighting reduction launch"},
            "terms": terms, "tiles": int(kt.shape[0]), "kt_mean": float(kt.mean())}


def _norm_err(got, ref, abs_terms=None):
    """Largest normalised error |x - x_ref| / max(|x_ref|, 1e-3 max |x_ref|),
    with 1e-2 x the sum of absolute terms added to the scale of sums."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    scale = np.maximum(np.abs(ref), 1e-3 * max(np.abs(ref).max(), 1e-30))
    if abs_terms is not None:
        scale = np.maximum(scale, 1e-2 * np.asarray(abs_terms, np.float64))
    return float((np.abs(got - ref) / scale).max())


def bench_chain(args, world, rank, local):
    """Mesh-deformation batch: 16 views x 50,000 vertices, 200 spheres, 60
    deformation parameters, n = 4.  A step renders every view (chain kernels
    -> shading) and back-propagates to the parameters and poses.  The chain
    kernels are HBM-bound (the [M, 3, D] basis read once per pass): their
    bytes/s, with L2 flushed before each timed launch, against the measured
    copy bandwidth."""
    import ctypes
    import torch
    from paper_2104_00359_gb300 import Config, _lib, chain, synthetic
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()
    m = synthetic.mesh_deformation_scene(seed=2 + rank)
    T = {k: torch.from_numpy(np.ascontiguousarray(v)).to(dev) for k, v in m.items() if k != "n_bands"}
    M, D = int(T["v0"].shape[0]), int(T["A_v"].shape[2])
    V, N = int(T["poses"].shape[0]), int(T["c0"].shape[0])
    stream = torch.cuda.current_stream()
    sptr = ctypes.c_void_p(stream.cuda_stream)
    flush = torch.empty(256 * 2 ** 20 // 4, device=dev)
    # chain kernels alone, on the vertex array
    p = torch.from_numpy(np.random.default_rng(1).normal(0, 1, D).astype(np.float32)).to(dev)
    q = T["poses"][0].contiguous()
    x = torch.empty((M, 3), device=dev)
    g = torch.randn((M, 3), device=dev)
    d_p, d_q = torch.empty(D, device=dev), torch.empty(6, device=dev)
    need = int(lib.shs_chain_workspace_bytes(M, D))
    ws = torch.empty(need // 4 + 4, device=dev)
    tf, tb = [], []
    for it in range(args.warmup + max(3, min(args.steps, 50))):
        flush.zero_()
        e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
        e0.record(stream)
        _lib.check(lib.shs_chain_forward(_lib.ptr(T["v0"]), _lib.ptr(T["A_v"]), M, D, _lib.ptr(p), _lib.ptr(q), 0,
                                         None, _lib.ptr(x), sptr), "shs_chain_forward")
        e1.record(stream)
        flush.zero_()
        e2.record(stream)
        _lib.check(lib.shs_chain_backward(_lib.ptr(T["v0"]), _lib.ptr(T["A_v"]), M, D, _lib.ptr(p), _lib.ptr(q), 0,
                                          _lib.ptr(g), _lib.ptr(d_p), _lib.ptr(d_q), _lib.ptr(ws), need, sptr),
                   "shs_chain_backward")
        e3.record(stream)
        torch.cuda.synchronize()
        if it >= args.warmup:
            tf.append(e0.elapsed_time(e1))
            tb.append(e2.elapsed_time(e3))
    fwd_ms, bwd_ms = statistics.fmean(tf), statistics.fmean(tb)
    chain_bytes = 4 * (M * 3 * D + 2 * M * 3)          # basis + base in, x out (backward: g in)
    # the whole step: every view through the chain kernels and the shading path
    pp = torch.zeros(D, device=dev, requires_grad=True)
    poses = T["poses"].clone().requires_grad_(True)
    cfg = Config(n_bands=m["n_bands"])
    scenes = chain.make_view_scenes(V, T["c0"], T["radii"], T["light"], cfg)
    views = chain.ViewBatch(V, M, T["c0"], T["radii"], T["light"], cfg)
    W = torch.randn((V, M, 3), device=dev)
    steps = max(3, min(args.steps, 20))

    def run_steps(batched):
        times, launches = [], 0
        for it in range(args.warmup + steps):
            l0 = lib.shs_launch_count()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            pp.grad = None
            poses.grad = None
            e0.record(stream)
            if batched:
                B = chain.render_views_batched(pp, poses, T, T["radii"], T["light"], T["albedo"], views)
            else:
                B = chain.render_views(pp, poses, T, T["radii"], T["light"], T["albedo"], scenes)
            (B * W).sum().backward()
            e1.record(stream)
            torch.cuda.synchronize()
            if it >= args.warmup:
                times.append(e0.elapsed_time(e1))
                launches += lib.shs_launch_count() - l0
        return statistics.fmean(times), launches

    # the step as one batched launch per pass (all views), and view by view
    with ClockSampler(local) as clk:
        step_ms, launches = run_steps(True)
    per_view_ms, per_view_launches = run_steps(False)
    for sc in scenes:
        sc.close()
    views.close()
    hbm = load_peaks().get("hbm_gbs")
    ach = chain_bytes / (fwd_ms * 1e-3) / 1e9
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        from oracle import chain_oracle as CO
        gn = g.cpu().numpy()
        t = time.perf_counter()
        CO.deform_pose(m["v0"], m["A_v"], p.cpu().numpy(), q.cpu().numpy())
        CO.deform_pose_backward(m["v0"], m["A_v"], p.cpu().numpy(), q.cpu().numpy(), gn)
        dt = time.perf_counter() - t
        cpu = {"value": 2 * chain_bytes / dt, "unit": "bytes/s", "cores": 1, "kind": "oracle",
               "sample": f"chain forward + backward on the {M} x 3 x {D} vertex basis, float64 numpy, {dt:.1f} s"}
    return dict(
        metric="mesh-deformation batch: point-sphere pairs/sec fwd+bwd through chain + shading (16 views)",
        value=V * M * N / (step_ms * 1e-3), unit="pairs/s", n_gpus=world, steps=steps, warmup=args.warmup,
        ms_per_step=step_ms, higher_is_better=True, scaling="weak", vs_baseline=None, dtype="f32",
        data="synthetic", impl="ours",
        config={"workload": f"mesh deformation {V} views x {M} vertices, {N} spheres, {D} parameters, n_bands=4",
                "views": V, "vertices": M, "spheres": N, "params": D, "l2_flush_between_chain_launches": True},
        chain_kernels={"fwd_ms": fwd_ms, "bwd_ms": bwd_ms, "bytes_per_launch": chain_bytes},
        step={"batched_views_ms": step_ms, "launches_per_step": launches / steps,
              "per_view_calls_ms": per_view_ms, "per_view_launches_per_step": per_view_launches / steps},
        roofline={"bound": "hbm", "kernel": "chain_forward_kernel (vertices)", "achieved": ach, "peak": hbm,
                  "unit": "GB/s", "frac": ach / hbm if hbm else None, "traffic": None,
                  "backward": {"achieved": chain_bytes / (bwd_ms * 1e-3) / 1e9,
                               "frac": chain_bytes / (bwd_ms * 1e-3) / 1e9 / hbm if hbm else None}},
        gpu_launches=int(launches), clocks=clk.summary(), cpu_baseline=cpu)


def bench_envmap(args, world, rank, local):
    """Eq. 9 projection of an equirectangular HDR map (default 4096 x 8192,
    402 MB, larger than L2) onto SH lighting, n = 8 and n = 4.  The kernel
    streams the map once: bytes/s against the measured HBM copy bandwidth."""
    import ctypes
    import torch
    from paper_2104_00359_gb300 import _lib, synthetic
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = _lib.load()
    H, W = args.env_res, 2 * args.env_res
    env_np = synthetic.environment_map(seed=5 + rank, height=H, width=W)
    env = torch.from_numpy(env_np).to(dev)
    nbytes = env.numel() * 4
    sptr = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    stream = torch.cuda.current_stream()
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs")
    out = {}
    for n in (8, 4):
        light = torch.empty((3, n * n), device=dev)
        need = int(lib.shs_envmap_workspace_bytes(H, W, n))
        ws = torch.empty(need // 4, device=dev)

        def step():
            _lib.check(lib.shs_project_envmap(_lib.ptr(env), H, W, n, _lib.ptr(light), _lib.ptr(ws), need, sptr),
                       "shs_project_envmap")

        for _ in range(args.warmup):
            step()
        torch.cuda.synchronize()
        K = max(3, min(args.steps, 200))
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(K)]
        launches0 = lib.shs_launch_count()
        with ClockSampler(local) as clk:
            for e0, e1 in evs:
                e0.record(stream)
                step()
                e1.record(stream)
            torch.cuda.synchronize()
        ms = statistics.fmean(a.elapsed_time(b) for a, b in evs)
        out[f"n{n}"] = {"ms": ms, "bytes_per_s": nbytes / (ms * 1e-3), "gpu_launches": lib.shs_launch_count() - launches0,
                        "clocks": clk.summary()}
    # end to end: pinned host map -> device -> light back to the host
    host = torch.from_numpy(env_np).pin_memory()
    light_h = torch.empty((3, 64)).pin_memory()
    light = torch.empty((3, 64), device=dev)
    need = int(lib.shs_envmap_workspace_bytes(H, W, 8))
    ws = torch.empty(need // 4, device=dev)
    KE = 10
    for i in range(KE + 2):
        if i == 2:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        env.copy_(host, non_blocking=True)
        _lib.check(lib.shs_project_envmap(_lib.ptr(env), H, W, 8, _lib.ptr(light), _lib.ptr(ws), need, sptr),
                   "shs_project_envmap")
        light_h.copy_(light, non_blocking=True)
        stream.synchronize()
    e2e_s = (time.perf_counter() - t0) / KE
    main = out["n8"]
    achieved = main["bytes_per_s"] / 1e9
    cpu = None
    if not args.no_cpu and rank == 0 and world == 1:
        from oracle import shs_oracle as O
        rows = max(1, min(H, int(4e6 // W)))
        t = time.perf_counter()
        O.project_envmap(8, env_np[:rows])
        dt = time.perf_counter() - t
        cpu = {"value": rows * W * 12 / dt, "unit": "bytes/s", "cores": 1, "kind": "oracle",
               "sample": f"first {rows} rows of the {H}x{W} map, n_bands=8, float64 numpy, 1 thread, {dt:.1f} s"}
    return dict(
        metric="equirectangular HDR map -> SH lighting (Eq. 9), map bytes/s", value=main["bytes_per_s"],
        unit="bytes/s", n_gpus=world, steps=K, warmup=args.warmup, ms_per_step=main["ms"], higher_is_better=True,
        scaling="weak", vs_baseline=None, dtype="f32", data="synthetic", impl="ours",
        config={"workload": f"environment map {H}x{W}x3 float32 ({nbytes / 1e6:.0f} MB, larger than L2), n_bands=8",
                "height": H, "width": W},
        per_band_count=out,
        roofline={"bound": "hbm", "kernel": "envmap_rows_kernel<8> + envmap_reduce_kernel",
                  "achieved": achieved, "peak": hbm, "unit": "GB/s",
                  "frac": (achieved / hbm) if hbm else None, "traffic": None,
                  "peak_source": "MEASURED_PEAKS.json hbm_gbs (copy bandwidth, read + write bytes)",
                  "bytes_per_launch": nbytes},
        e2e={"value": nbytes / e2e_s, "unit": "bytes/s", "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": 3 * 64 * 4,
             "ms_per_step": e2e_s * 1e3},
        gpu_launches=main["gpu_launches"], clocks=main["clocks"], cpu_baseline=cpu)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--atomic", action="store_true", help="unordered (atomic) scene-gradient reduction")
    ap.add_argument("--no-cpu", action="store_true", help="skip the oracle CPU baseline")
    ap.add_argument("--latency-reps", type=int, default=0,
                    help="steps of the latency loop (default: >= 200 and about 3 s)")
    ap.add_argument("--workload", choices=("capsule", "serving", "heightfield", "envmap", "chain"), default="capsule",
                    help="capsule: the 512x512 G-buffer step (default); serving: the mixed request stream")
    ap.add_argument("--hf-res", type=int, default=1024, help="height-field grid side (heightfield workload)")
    ap.add_argument("--precisions", default="fp32,bf16_tc,tf32_tc,fp16_tc,fp32_projexp,bf16_tc_projexp,"
                    "tf32_tc_projexp,fp32_oltable",
                    help="heightfield workload: comma list of fp32, bf16_tc, tf32_tc, fp16_tc, fp32_projexp, "
                         "bf16_tc_projexp, tf32_tc_projexp, "
                         "fp32_oltable")
    ap.add_argument("--env-res", type=int, default=4096, help="environment map rows (width = 2 x rows)")
    ap.add_argument("--serve-jobs", type=int, default=64)
    ap.add_argument("--serve-batch-work", type=float, default=3.0e8,
                    help="serving: estimated work one batch may carry (serve.task_work units)")
    ap.add_argument("--serve-chunk", type=int, default=1 << 40,
                    help="serving: largest chunk of a request in one launch (points)")
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-slots", type=int, default=3, help="serving: batch slots (streams) in flight")
    ap.add_argument("--serve-small-work", type=float, default=None,
                    help="serving: tasks up to this estimated work fill a batch first (0: arrival order)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    if args.serve_small_work is None:
        from paper_2104_00359_gb300 import serve as _serve
        args.serve_small_work = _serve.SMALL_WORK
    world, rank, local, dist = dist_init(args)
    if args.impl == "reference":
        res = bench_reference(args, world, rank)
    elif args.workload == "serving":
        res = bench_serving(args, world, rank, local)
    elif args.workload == "heightfield":
        res = bench_heightfield(args, world, rank, local)
    elif args.workload == "envmap":
        res = bench_envmap(args, world, rank, local)
    elif args.workload == "chain":
        res = bench_chain(args, world, rank, local)
    else:
        res = bench_ours(args, world, rank, local, dist)
    if rank == 0 and res is not None:
        print(json.dumps(res))
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
