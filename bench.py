#!/usr/bin/env python3
"""Benchmark: preconditioned-SPS iterations/s on one GB300 for the 2-D fan-beam
MBIR workload (512x512 at 0.5 mm, 720 views over 360 deg, 888 curved bins,
SID 500 / SDD 1000 mm, water phantom with inserts, I0 = 1e5, beta = 1e4,
Haar-wavelet preconditioner with the line search), plus wall time to a 1e-4
relative objective gap for PSPS and for plain SPS on the same GPU.

A step is one full preconditioned SPS iteration (model, backprojection,
preconditioner applies, projection, line search, update) replayed as a CUDA
graph.  L2 (129 MB) is flushed with a 256 MB write between timed steps; each
step is timed with CUDA events on the launching stream.

--impl reference times the FP64 CPU oracle's iteration on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "precond-SPS iters/s & time to 1e-4 rel objective gap vs plain SPS, one GB300"
WORKLOAD = "c2_fan2d_512_haar"

# other workloads (python bench.py --workload NAME): problem builder,
# preconditioner, description
# Bytes per step copied back by psps_step with a host history: the history
# (2 doubles for one iteration) plus the device line-search record.
DEVLS_BYTES = 80

# Counters of the dominant kernel from one ncu capture of the same kernel and
# workload (summaries under profiles/): DRAM bytes read + written per launch,
# and the unit that binds it.  Remove an entry when its kernel changes.
NCU_CAPTURES = {
    ("c2_fan2d_512_haar", "backproject"): {
        "traffic": 16.12e6,
        "binding": {"unit": "SM instruction issue (issue active, % of cycles)", "frac_of_peak": 0.858,
                    "source": "profiles/back_tile_2d_c2_fan512.md"},
    },
}

WORKLOADS = {
    "c2_fan2d_512_haar": ("config2", "haar", "512x512@0.5mm, 720x888 fan curved, Haar(M0, lattice 3)"),
    "c1_par2d_64_modfourier": ("config1", "mod_fourier", "64x64@1mm, 90x96 parallel, modified Fourier"),
    "c3_projdomain_block": ("config3", "block", "720x888 rays, 2 materials x 2 kVp channels, per-ray 2x2 blocks"),
    "c4_mbmd_512_blockfourier": ("config4_slice", "block_fourier",
                                 "512x512@0.5mm, 3 materials x 4 PC channels (101 energies), 3x3 blocks + "
                                 "cross-material Fourier"),
    "c4_mbmd_512_blockhaar": ("config4_slice", "block_haar",
                              "512x512@0.5mm, 3 materials x 4 PC channels (101 energies), 3x3 blocks + "
                              "cross-material wavelet (Haar)"),
    "c4_mbmd_16slices_blockfourier": ("config4", "block_fourier",
                                      "16 slices 256^2..512^2 @0.5mm (seeded sizes), 720 views, 3 materials x 4 PC "
                                      "channels, 3x3 blocks + cross-material Fourier, one graph per batch iteration"),
    "c5_cone3d_256_block": ("config5", "block", "256^3@0.5mm, 360x384x512 cone flat, 2 materials x 2 kVp, 2x2 "
                                                "per-voxel blocks"),
    "c5_cone3d_256_blockfourier": ("config5", "block_fourier", "256^3@0.5mm, 360x384x512 cone flat, 2 materials x "
                                                              "2 kVp, 2x2 per-voxel blocks + 3-D cross-material Fourier"),
    "c5_cone3d_128_block": ("config5", "block", "128^3@1mm, 180x192x256 cone flat (the 256^3 scan scaled down), "
                                                "2 materials x 2 kVp, 2x2 per-voxel blocks",
                            {"n": 128, "n_views": 180, "n_u": 256, "n_v": 192}),
    "c5_cone3d_128_blockhaar": ("config5", "block_haar", "128^3@1mm, 180x192x256 cone flat (the 256^3 scan scaled "
                                                         "down), 2 materials x 2 kVp, 2x2 per-voxel blocks + 3-D "
                                                         "cross-material wavelet (Haar)",
                                {"n": 128, "n_views": 180, "n_u": 256, "n_v": 192}),
    "c2_fan2d_512_haar_blur1": ("config2", "haar", "config 2 read out through a 3-tap detector blur along the "
                                                   "888-bin rows (outer operator B S)", {"blur": "r1"}),
    "c4_mbmd_512_blockfourier_blur3": ("config4_slice", "block_fourier",
                                       "config 4 slice read out through a 7-tap asymmetric detector blur along the "
                                       "888-bin rows (outer operator B S), 3x3 blocks + cross-material Fourier",
                                       {"blur": "r3"}),
    "c4_mbmd_512_blockfourier_corr": ("config4_slice", "block_fourier",
                                      "config 4 slice with correlated detector noise (correlation 0.4^|j-k| along "
                                      "the 888-bin rows) and a 3-tap detector blur, 3x3 blocks + cross-material "
                                      "Fourier", {"blur": "r1", "noise": 0.4}),
}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def shard(n_units: int, rank: int, world: int) -> list:
    """Independent units (the slices of a batch) of one rank: every world-th
    unit from the rank's own index; the ranks' shards cover every unit once.
    No data moves between ranks: each rank reconstructs its own slices."""
    return list(range(rank, n_units, world))


def job_max(value: float, world: int, device) -> float:
    """The job's figure over all ranks: the slowest rank's time (all-reduce
    MAX; the only collective, outside the timed region)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_sum(value: float, world: int, device) -> float:
    """Sum over all ranks (kernel launch counts)."""
    if world == 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d.get("hbm_gbs", 6800.0)), "measured"
    return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index: int):
        self.proc = None
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")
        self.index = index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}",
                 "--query-gpu=clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower() in ("active", "1"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(prob, n_iter: int):
    """The FP64 oracle's PSPS iteration on the same workload, timed; the Haar
    eigenvalues are built with the paper's single test function (one
    Hessian application) to keep the sample bounded -- the per-iteration
    work does not depend on the eigenvalue values."""
    import oracle
    from oracle import build as obuild, model, precond, psps as opsps
    st = opsps.Setup(oracle.Projector(prob.geom), prob.Q, prob.S, prob.y, prob.beta)
    F = obuild.fisher(st)
    aH = obuild.make_apply_H(st, F)
    m0 = obuild.m0_blocks(st, F)[:, 0, 0].reshape(st.shape)
    lam = precond.haar_eigenvalues(lambda v: m0[None] * aH(m0[None] * v), st.shape, lattice=0)
    P = precond.Haar(lam, m0)
    t0 = time.perf_counter()
    opsps.run(st, P, n_iter, opsps.LineSearch())
    dt = time.perf_counter() - t0
    # run() adds one final exact projection + objective; count it as overhead
    return n_iter / dt, dt


def reference_arm(args, prob):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build_c()
    t_start = time.perf_counter()
    rate_w, _ = oracle_sample(prob, 1)
    per = 1.0 / rate_w
    budget = 150.0
    k = max(1, min(args.steps, int(budget / max(per, 1e-3))))
    rate, dt = oracle_sample(prob, k)
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "iter/s", "n_gpus": args.gpus,
            "steps": k, "warmup": 1, "ms_per_step": 1000.0 / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (host)"},
            "cpu_baseline": {"kind": "oracle", "value": rate, "unit": "iter/s", "cores": 1,
                             "sample": f"{k} FP64 oracle PSPS-Haar iterations of the full 512^2 / 720x888 "
                                       f"fan-beam workload (single-threaded C projector + NumPy)"},
            "e2e": {"value": rate, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)


def gap_runs(p, plan, spec, yd, beta, pc, n_star: int, n_cmp: int):
    """Objective histories for PSPS and plain SPS (with and without the line
    search); Phi* from a long PSPS run."""
    st = p.State(plan, spec, pc, yd, beta, graph=True)
    h_star = p.psps_step(st, n_star)
    out = {}
    for name, pcx, ls in [("psps", pc, True), ("sps", None, False), ("sps_ls", None, True)]:
        s = p.State(plan, spec, pcx, yd, beta, line_search=ls, graph=True)
        out[name] = p.psps_step(s, n_cmp)
    phi_star = min(float(np.min(h_star)), *[float(np.min(v)) for v in out.values()])
    return phi_star, out


def ours(args, prob, workload=WORKLOAD, kind="haar", desc="", blur=None, noise=None):
    import torch

    import paper_2010_01371_gb300 as p

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    y_host = torch.as_tensor(prob.y.astype(np.float32)).pin_memory()
    yd = y_host.to(dev)
    t0 = time.perf_counter()
    plan = p.Plan(prob.geom) if prob.geom is not None else None
    spec = p.Spectrum(prob.Q, prob.S)
    if blur is not None:
        spec.set_blur(blur, prob.geom.n_u)
    if noise is not None:
        spec.set_noise(noise, prob.geom.n_u)
    beta = prob.beta if plan is not None else None
    pc = p.Precond(plan, spec, kind, yd, beta)
    tuned = plan.autotune(2 * prob.Q.shape[1]) if plan is not None else None
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    st = p.State(plan, spec, pc, yd, beta, line_search=True, graph=True)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    for _ in range(args.warmup):
        p.psps_step(st, 1, history=False)
    torch.cuda.synchronize()
    p.psps_profile(st, True)
    p.psps_step(st, 1, history=False)          # re-capture the graph with timers
    p.psps_profile(st, True)                   # reset totals
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = p.psps_launch_count(st)
    times = []
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p.psps_step(st, 1, history=False)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = job_max(float(np.sum(times)), world, dev)
    clk = clocks.stop()
    launches = int(job_sum(p.psps_launch_count(st) - launches0, world, dev))
    prof = p.psps_profile_read(st)
    p.psps_profile(st, False)
    ms_step = ms / args.steps
    value = world * args.steps / (ms / 1000.0)

    # end to end through the public API with host buffers: every step uploads
    # the measured counts from pinned host memory into the state
    # (psps_state_set_data) and reads back the objective history and the
    # line-search record (psps_step with a host history synchronises).
    st2 = p.State(plan, spec, pc, yd, beta, line_search=True, graph=True)
    p.psps_step(st2, 1, history=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        p.psps_state_set_data(st2, y_host)
        p.psps_step(st2, 1, history=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0

    # roofline of the dominant stage
    n_rays = int(prob.n_rays)
    n_pix = plan.n_pix if plan is not None else n_rays
    stage_ms = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in prof.items()}
    dom = max(stage_ms, key=stage_ms.get)
    nm, nc = prob.Q.shape[1], prob.S.shape[0]
    alg_bytes = {
        "backproject": 2 * nm * 4 * (n_rays + n_pix),     # 2 n_mat channels: sinograms in, images out
        "project": nm * 4 * (n_rays + n_pix),
        "model": 4 * n_rays * (nm + nc + nm + 2 * nm),     # l, y, gamma in; g, kappa out
        "linesearch": 4 * n_rays * (2 * nm + nc) * 4,      # l, q, y per evaluation, 3 Newton + 1 halving pass
        "precond": 4 * n_pix * nm * 16,
        "update": 4 * 2 * nm * (n_pix + n_rays),
        "reproject": nm * 4 * (n_rays + n_pix),
    }[dom]
    hbm, src = peaks()
    achieved = alg_bytes / (stage_ms[dom] * 1e-3) / 1e9 if stage_ms[dom] > 0 else 0.0
    cap = NCU_CAPTURES.get((workload, dom))
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": cap["traffic"] if cap else None, "peak_source": src,
                "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()}}
    if cap:
        roofline["binding"] = cap["binding"]

    line = {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "problem": desc or WORKLOADS[workload][2], "precond": kind,
                       "line_search": True, "graph": True,
                       "l2": "flushed (256 MB write) between timed steps", "build_s": round(build_s, 3),
                       "views_per_cta": tuned},
            "gpu_launches": launches, "clocks": clk, "roofline": roofline,
            "e2e": {"value": args.steps / e2e_s, "unit": "iter/s", "h2d_bytes_per_step": int(y_host.numel() * 4),
                    "d2h_bytes_per_step": 2 * 8 + DEVLS_BYTES}}
    if rank == 0 and not args.no_gap:
        t0 = time.perf_counter()
        phi_star, runs = gap_runs(p, plan, spec, yd, beta, pc, args.gap_star, args.gap_iters)
        # per-iteration times of each method from short timed runs
        per_iter = {}
        for name, pcx, ls in [("psps", pc, True), ("sps", None, False), ("sps_ls", None, True)]:
            s = p.State(plan, spec, pcx, yd, beta, line_search=ls, graph=True)
            p.psps_step(s, 3, history=False)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.psps_step(s, 20, history=False)
            e1.record(stream)
            torch.cuda.synchronize()
            per_iter[name] = e0.elapsed_time(e1) / 20
        gap = {"target": 1e-4, "phi_star": phi_star, "phi_star_iters": args.gap_star}
        for name, h in runs.items():
            g = (h - phi_star) / (h[0] - phi_star)
            hit = np.nonzero(g <= 1e-4)[0]
            it = int(hit[0]) if hit.size else None
            gap[name] = {"iters": it, "ms_per_iter": per_iter[name],
                         "ms_to_gap": (it * per_iter[name]) if it is not None else None,
                         "gap_at_end": float(g[-1]), "iters_run": len(h) - 1}
        gap["wall_s"] = time.perf_counter() - t0
        line["time_to_gap"] = gap
    if rank == 0 and not args.no_cpu and workload == WORKLOAD:
        import oracle
        oracle.build_c()
        rate, dt = oracle_sample(prob, args.cpu_iters)
        line["cpu_baseline"] = {"value": rate, "unit": "iter/s", "cores": 1, "kind": "oracle",
                                "sample": f"{args.cpu_iters} FP64 oracle PSPS-Haar iterations of the same "
                                          f"workload ({dt:.1f} s, single-threaded)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def ours_batch(args, probs, workload, kind, desc):
    """The batched workload: every slice has its own plan (autotuned view
    split), spectrum handle, preconditioner and state; one psps_batch_step
    iteration advances all slices through one CUDA graph.  value = batch
    iterations per second (each advances every slice once)."""
    import torch

    import paper_2010_01371_gb300 as p

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n_total = len(probs)
    probs = [probs[i] for i in shard(n_total, rank, world)]
    t0 = time.perf_counter()
    slices, tuned = [], []
    for prob in probs:
        plan = p.Plan(prob.geom)
        tuned.append(plan.autotune(2))
        spec = p.Spectrum(prob.Q, prob.S)
        y_host = torch.as_tensor(prob.y.astype(np.float32)).reshape(-1).pin_memory()
        yd = y_host.to(dev)
        pc = p.Precond(plan, spec, kind, yd, prob.beta)
        slices.append({"prob": prob, "plan": plan, "spec": spec, "y_host": y_host, "yd": yd, "pc": pc})
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    states = [p.State(s["plan"], s["spec"], s["pc"], s["yd"], s["prob"].beta, graph=True) for s in slices]
    batch = p.Batch(states)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)   # 256 MB > L2
    for _ in range(args.warmup):
        p.psps_batch_step(batch, 1, history=False)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    launches0 = p.psps_batch_launch_count(batch)
    times = []
    torch.cuda.nvtx.range_push("timed")
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p.psps_batch_step(batch, 1, history=False)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    torch.cuda.nvtx.range_pop()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    launches = int(job_sum(p.psps_batch_launch_count(batch) - launches0, world, dev))
    ms = job_max(float(np.sum(times)), world, dev)
    value = args.steps / (ms / 1000.0)   # iterations of the whole batch per second

    # dominant kernel: the 2 n_mat-channel transpose of every slice, timed
    # alone per slice (CUDA events, L2 flushed) and summed over the batch
    back_ms, alg_bytes = 0.0, 0
    for s in slices:
        prob, plan = s["prob"], s["plan"]
        nm = prob.Q.shape[1]
        sino = torch.rand((2 * nm, plan.n_rays), device=dev)
        img = torch.empty((2 * nm,) + plan.image_shape, device=dev)
        p.mbir_backproject(plan, sino, img)
        reps = []
        for _ in range(5):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            p.mbir_backproject(plan, sino, img)
            e1.record(stream)
            torch.cuda.synchronize()
            reps.append(e0.elapsed_time(e1))
        back_ms += float(np.median(reps))
        alg_bytes += 2 * nm * 4 * (plan.n_rays + plan.n_pix)
    hbm, src = peaks()
    achieved = alg_bytes / (back_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "backproject (rank 0's slices, timed alone)", "achieved": achieved,
                "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None, "peak_source": src,
                "backproject_ms_per_iter": round(back_ms, 4)}

    # end to end: every step uploads each slice's counts from pinned host
    # memory and reads back every slice's objective history
    states2 = [p.State(s["plan"], s["spec"], s["pc"], s["yd"], s["prob"].beta, graph=True) for s in slices]
    batch2 = p.Batch(states2)
    p.psps_batch_step(batch2, 1, history=True)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        for st, s in zip(states2, slices):
            p.psps_state_set_data(st, s["y_host"])
        p.psps_batch_step(batch2, 1, history=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t1
    sizes = [int(s["prob"].geom.nx) for s in slices]
    e2e_s = job_max(e2e_s, world, dev)
    line = {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "problem": desc, "precond": kind, "line_search": True,
                       "graph": "one per batch iteration (one branch per slice)", "slices": n_total,
                       "slices_per_rank": len(slices), "sharding": "slices round-robin over ranks, no collective "
                                                                   "in the data path",
                       "slice_sizes_rank0": sizes, "views_per_cta_rank0": tuned,
                       "slice_iters_per_s": value * n_total,
                       "l2": "flushed (256 MB write) between timed steps", "build_s": round(build_s, 3)},
            "gpu_launches": launches, "clocks": clk, "roofline": roofline,
            "e2e": {"value": args.steps / e2e_s, "unit": "iter/s",
                    "h2d_bytes_per_step": int(job_sum(sum(s["y_host"].numel() for s in slices) * 4, world, dev)),
                    "d2h_bytes_per_step": int(job_sum(len(slices) * (2 * 8 + DEVLS_BYTES), world, dev))}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def kernel_bench(args, prob):
    """Times the projector and transpose variants alone on the workload's
    geometry (CUDA events, L2 flushed between launches)."""
    import torch

    import paper_2010_01371_gb300 as p
    dev = torch.device("cuda", 0)
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device=dev)
    plan = p.Plan(prob.geom)
    rng = np.random.default_rng(0)
    x1 = torch.as_tensor(prob.truth.astype(np.float32), device=dev)
    s2 = torch.as_tensor(rng.random((2, plan.n_rays)).astype(np.float32), device=dev)
    out = {}

    def timeit(fn, reps=20):
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return float(np.median(ts))
    l1 = torch.empty((1, plan.n_rays), device=dev)
    g2 = torch.empty((2,) + plan.image_shape, device=dev)
    for mode in ["tile", "ray"]:
        plan.set_projector(mode)
        out[f"project_{mode}_1ch_ms"] = timeit(lambda: p.mbir_project(plan, x1, l1))
    for mode in ["tile", "gather", "atomic"]:
        plan.set_backprojector(mode)
        out[f"backproject_{mode}_2ch_ms"] = timeit(lambda: p.mbir_backproject(plan, s2, g2))
    plan.set_backprojector("tile")
    for vs in [30, 45, 60, 90, 120, 180]:
        plan.set_tiling(vs)
        out[f"backproject_tile{vs}_2ch_ms"] = timeit(lambda: p.mbir_backproject(plan, s2, g2))
        out[f"backproject_tile{vs}_1ch_ms"] = timeit(lambda: p.mbir_backproject(plan, s2[:1], g2[:1]))
    plan.set_tiling(60)
    print(json.dumps({"kernels": out, "workload": WORKLOAD}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-gap", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--gap-iters", type=int, default=300)
    ap.add_argument("--gap-star", type=int, default=1500)
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--kernels", action="store_true", help="time the projector variants alone")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    args = ap.parse_args()
    import synth
    if args.kernels:
        kernel_bench(args, synth.config2())
        return
    if args.impl == "reference":
        reference_arm(args, synth.config2())
        return
    builder, kind, desc, *kw = WORKLOADS[args.workload]
    kw = dict(kw[0]) if kw else {}
    blur = kw.pop("blur", None)
    noise = kw.pop("noise", None)
    prob = getattr(synth, builder)(**kw)
    if blur is not None:
        blur = synth.BLUR_TAPS[blur]
        prob = synth.with_detector_blur(prob, blur)
    if args.workload != WORKLOAD:
        args.no_cpu = True
    if isinstance(prob, list):
        ours_batch(args, prob, args.workload, kind, desc)
        return
    ours(args, prob, args.workload, kind, desc, blur, noise)


if __name__ == "__main__":
    main()
