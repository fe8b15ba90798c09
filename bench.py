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

The default run (one GPU) adds, under "largest", the same measurements for the
two largest workloads: the 16-slice one-step MBMD batch (256^2..512^2, 3
materials x 4 photon-counting channels, one CUDA graph per batch iteration)
and the 256^3 cone-beam one-step MBMD (2 materials x 2 kVp, 360 x 384 x 512
rays), with the time to the 1e-4 gap of the cone scan at 128^3.

--impl reference times the FP64 CPU oracle's iteration on the same workload
on every host core (independent replicas, one per core).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "precond-SPS iters/s & time to 1e-4 rel objective gap vs plain SPS, one GB300"
WORKLOAD = "c2_fan2d_512_haar"

# Bytes per step copied back by psps_step with a host history: the history
# (2 doubles for one iteration) plus the device line-search record.
DEVLS_BYTES = 80

# Counters of the dominant kernel from one ncu capture of the same kernel and
# workload (summaries under profiles/): DRAM bytes read + written per launch,
# and the unit that binds it.  Remove an entry when its kernel changes.
NCU_CAPTURES = {
    # 128^3 capture of the same kernel (back_cone_tile_kernel<4, 0>), 340.4 MB
    # per launch, scaled by the rays and voxels processed (8x each) to 256^3
    ("c5_cone3d_256_block", "backproject"): {
        "traffic": 8 * 340.4e6,
        "binding": {"unit": "SM instruction issue (issue active, % of cycles)", "frac_of_peak": 0.792,
                    "source": "profiles/back_cone_tile_c5_128.md"},
    },
    ("c2_fan2d_512_haar", "backproject"): {
        "traffic": 16.12e6,
        "binding": {"unit": "SM instruction issue (issue active, % of cycles)", "frac_of_peak": 0.858,
                    "source": "profiles/back_tile_2d_c2_fan512.md"},
    },
}

# other workloads (python bench.py --workload NAME): problem builder,
# preconditioner, description[, builder keywords]
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

# the two largest single-GPU workloads, measured by the default run
LARGEST = ["c4_mbmd_16slices_blockfourier", "c5_cone3d_256_block"]


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


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class Clocks:
    """nvidia-smi sampling during the timed region (into a temporary file)."""

    def __init__(self, index: int):
        self.proc = None
        self.index = index
        self.f = None

    def start(self):
        try:
            self.f = tempfile.TemporaryFile(mode="w+")
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
        self.f.seek(0)
        lines = self.f.read().splitlines()
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
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


# ---------------------------------------------------------------------------
# the FP64 oracle on the host cores
# ---------------------------------------------------------------------------

def build_problem(workload: str, views: int | None = None):
    """The workload's seeded problem.  views: only the first `views` views
    of the cone scan (a bounded sample whose per-iteration work is
    proportional to the views kept).  A batch gives its smallest slice."""
    import synth
    builder, kind, desc, *kw = WORKLOADS[workload]
    kw = dict(kw[0]) if kw else {}
    kw.pop("blur", None)
    kw.pop("noise", None)
    if views is not None:
        kw["first_views"] = views
    prob = getattr(synth, builder)(**kw)
    if isinstance(prob, list):
        prob = min(prob, key=lambda q: q.geom.nx)
    return prob


def oracle_sample(prob, kind: str, n_iter: int):
    """The FP64 oracle's PSPS iteration (line search on) on a problem, timed.
    The preconditioner is built with its cheapest estimate (Haar: the
    paper's single test function, one Hessian application) to keep the
    sample bounded -- the per-iteration work does not depend on the
    eigenvalue values.  Returns (iterations/s, seconds)."""
    import oracle
    from oracle import build as obuild, precond, psps as opsps
    oracle.build_c()
    A = oracle.Projector(prob.geom) if prob.geom is not None else oracle.IdentityProjector(prob.n_rays)
    st = opsps.Setup(A, prob.Q, prob.S, prob.y, prob.beta if prob.geom is not None else None)
    F = obuild.fisher(st)
    if kind == "haar":
        aH = obuild.make_apply_H(st, F)
        m0 = obuild.m0_blocks(st, F)[:, 0, 0].reshape(st.shape)
        lam = precond.haar_eigenvalues(lambda v: m0[None] * aH(m0[None] * v), st.shape, lattice=0)
        P = precond.Haar(lam, m0)
    else:
        P = obuild.build(st, kind)
    t0 = time.perf_counter()
    opsps.run(st, P, n_iter, opsps.LineSearch())
    dt = time.perf_counter() - t0
    return n_iter / dt, dt


def _oracle_worker(job):
    workload, kind, n_iter, views = job
    return oracle_sample(build_problem(workload, views), kind, n_iter)


def oracle_all_cores(workload: str, kind: str, n_iter: int, views=None, replicas=None):
    """Independent oracle replicas of the same sample, one per host core
    (spawned processes with single-threaded BLAS): aggregate iterations/s of
    the machine's CPU.  Returns (aggregate rate, replicas, slowest seconds)."""
    cores = host_cores()
    n = replicas or cores
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            res = pool.map(_oracle_worker, [(workload, kind, n_iter, views)] * n)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return float(sum(r for r, _ in res)), n, float(max(dt for _, dt in res))


def mem_replicas(per_replica_gb: float) -> int:
    """Replicas that fit the host's available memory (half of it), at most
    one per core."""
    avail = None
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                avail = float(line.split()[1]) / 1e6
    except OSError:
        pass
    n = host_cores()
    if avail:
        n = max(1, min(n, int(0.5 * avail / per_replica_gb)))
    return n


def cpu_baseline(workload: str, kind: str, prob, n_iter: int, views=None, scale: float = 1.0,
                 per_replica_gb: float = 1.0, what: str = ""):
    """Single-threaded and all-core oracle timings of a bounded sample;
    `scale` converts the sample's iterations/s into the workload's
    (views kept / views of the scan)."""
    single, dt1 = oracle_sample(prob, kind, n_iter)
    agg, n, dtn = oracle_all_cores(workload, kind, n_iter, views, mem_replicas(per_replica_gb))
    return {"value": agg * scale, "unit": "iter/s", "cores": n, "kind": "oracle",
            "single_thread": {"value": single * scale, "cores": 1, "seconds": round(dt1, 1)},
            "sample": f"{n_iter} FP64 oracle PSPS iterations ({kind}) {what}; single-threaded {dt1:.1f} s, then "
                      f"{n} independent replicas on {n} host cores (slowest {dtn:.1f} s), value = their summed "
                      f"rate" + (f", scaled by {scale:.4g} to the full scan" if scale != 1.0 else "")}


def reference_arm(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import oracle
    oracle.build_c()
    t_start = time.perf_counter()
    prob = build_problem(WORKLOAD)
    per = 1.0 / oracle_sample(prob, "haar", 1)[0]
    k = max(1, min(args.steps, int(60.0 / max(per, 1e-3))))
    rate, n, dt = oracle_all_cores(WORKLOAD, "haar", k, replicas=mem_replicas(1.0))
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": "iter/s", "n_gpus": args.gpus,
            "steps": k, "warmup": 1, "ms_per_step": 1000.0 / rate, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "l2": "n/a (host)"},
            "cpu_baseline": {"kind": "oracle", "value": rate, "unit": "iter/s", "cores": n,
                             "single_thread": {"value": 1.0 / per, "cores": 1},
                             "sample": f"{k} FP64 oracle PSPS-Haar iterations of the full 512^2 / 720x888 fan-beam "
                                       f"workload in each of {n} independent replicas on {n} host cores "
                                       f"(C projector + NumPy, single-threaded BLAS each; slowest {dt:.1f} s); "
                                       f"value = their summed rate"},
            "e2e": {"value": rate, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "wall_s": time.perf_counter() - t_start}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU path
# ---------------------------------------------------------------------------

def time_to_gap(p, stream, plan, spec, yd, beta, pc, n_star: int, n_cmp: int, build_s: float):
    """Objective histories for PSPS and plain SPS (with and without the line
    search), Phi* the lowest objective of a long PSPS run and of the compared
    runs (relative gap (Phi_n - Phi*) / (Phi_0 - Phi*)); time to the 1e-4
    gap = iterations x measured ms per iteration, plus the preconditioner
    build for PSPS."""
    import torch
    t0 = time.perf_counter()
    st = p.State(plan, spec, pc, yd, beta, graph=True)
    h_star = p.psps_step(st, n_star)
    runs, per_iter = {}, {}
    for name, pcx, ls in [("psps", pc, True), ("sps", None, False), ("sps_ls", None, True)]:
        s = p.State(plan, spec, pcx, yd, beta, line_search=ls, graph=True)
        runs[name] = p.psps_step(s, n_cmp)
        s = p.State(plan, spec, pcx, yd, beta, line_search=ls, graph=True)
        p.psps_step(s, 3, history=False)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        p.psps_step(s, 20, history=False)
        e1.record(stream)
        torch.cuda.synchronize()
        per_iter[name] = e0.elapsed_time(e1) / 20
    phi_star = min(float(np.min(h_star)), *[float(np.min(v)) for v in runs.values()])
    gap = {"target": 1e-4, "phi_star": phi_star, "phi_star_iters": n_star, "build_ms": round(1000 * build_s, 2)}
    for name, h in runs.items():
        g = (h - phi_star) / (h[0] - phi_star)
        hit = np.nonzero(g <= 1e-4)[0]
        it = int(hit[0]) if hit.size else None
        ms = it * per_iter[name] if it is not None else None
        gap[name] = {"iters": it, "ms_per_iter": per_iter[name], "ms_to_gap_iterations": ms,
                     "ms_to_gap": (ms + (1000 * build_s if name == "psps" else 0.0)) if ms is not None else None,
                     "gap_at_end": float(g[-1]), "iters_run": len(h) - 1}
    gap["wall_s"] = round(time.perf_counter() - t0, 2)
    return gap


ALG_NOTE = ("algorithmic bytes: backproject 2 n_mat (n_rays + n_pix) 4 B, project n_mat (n_rays + n_pix) 4 B, "
            "model 4 n_rays (4 n_mat + n_chan) B, line search 4 (2 n_mat + n_chan) n_rays B per evaluation x 4")


def alg_bytes(stage: str, nm: int, nc: int, n_rays: int, n_pix: int) -> int:
    return {
        "backproject": 2 * nm * 4 * (n_rays + n_pix),     # 2 n_mat channels: sinograms in, images out
        "project": nm * 4 * (n_rays + n_pix),
        "model": 4 * n_rays * (nm + nc + nm + 2 * nm),     # l, y, gamma in; g, kappa out
        "linesearch": 4 * n_rays * (2 * nm + nc) * 4,      # l, q, y per evaluation, 3 Newton + 1 halving pass
        "precond": 4 * n_pix * nm * 16,
        "update": 4 * 2 * nm * (n_pix + n_rays),
        "reproject": nm * 4 * (n_rays + n_pix),
    }[stage]


def ours(args, prob, workload=WORKLOAD, kind="haar", desc="", blur=None, noise=None, gap=None, cpu=None):
    """One reconstruction: `steps` timed iterations (CUDA events, L2 flushed),
    an end-to-end leg through the C ABI with host buffers, the roofline of the
    dominant stage, and optionally the time to the 1e-4 gap (gap = (n_star,
    n_cmp)) and a CPU baseline (cpu = callable returning the dict).  Returns
    the JSON line (dict)."""
    import torch

    import paper_2010_01371_gb300 as p

    rank, world, local = dist_env()
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
    t1 = time.perf_counter()
    for _ in range(args.steps):
        p.psps_state_set_data(st2, y_host)
        p.psps_step(st2, 1, history=True)
    torch.cuda.synchronize()
    e2e_s = job_max(time.perf_counter() - t1, world, dev)
    del st2

    # roofline of the dominant stage
    n_rays = int(prob.n_rays)
    n_pix = plan.n_pix if plan is not None else n_rays
    stage_ms = {k: (v[0] / v[1] if v[1] else 0.0) for k, v in prof.items()}
    dom = max(stage_ms, key=stage_ms.get)
    nm, nc = prob.Q.shape[1], prob.S.shape[0]
    hbm, src = peaks()
    ab = alg_bytes(dom, nm, nc, n_rays, n_pix)
    achieved = ab / (stage_ms[dom] * 1e-3) / 1e9 if stage_ms[dom] > 0 else 0.0
    cap = NCU_CAPTURES.get((workload, dom))
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": cap["traffic"] if cap else None, "peak_source": src,
                "alg_bytes_per_launch": ab, "stage_ms": {k: round(v, 4) for k, v in stage_ms.items()},
                "note": ALG_NOTE}
    if cap:
        roofline["binding"] = cap["binding"]

    line = {"metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "problem": desc or WORKLOADS[workload][2], "precond": kind,
                       "line_search": True, "graph": True,
                       "l2": "flushed (256 MB write) between timed steps", "build_s": round(build_s, 3),
                       "views_per_cta": tuned, "tuning": plan.tuning() if plan is not None else None},
            "gpu_launches": launches, "clocks": clk, "roofline": roofline,
            "e2e": {"value": world * args.steps / e2e_s, "unit": "iter/s",
                    "h2d_bytes_per_step": int(y_host.numel() * 4), "d2h_bytes_per_step": 2 * 8 + DEVLS_BYTES}}
    del st
    if rank == 0 and gap is not None and not args.no_gap:
        line["time_to_gap"] = time_to_gap(p, stream, plan, spec, yd, beta, pc, gap[0], gap[1], build_s)
    if rank == 0 and cpu is not None and not args.no_cpu:
        line["cpu_baseline"] = cpu()
    return line


def ours_batch(args, probs, workload, kind, desc, cpu=None):
    """The batched workload: every slice has its own plan (autotuned view
    split), spectrum handle, preconditioner and state; one psps_batch_step
    iteration advances all slices through one CUDA graph.  value = batch
    iterations per second (each advances every slice once)."""
    import torch

    import paper_2010_01371_gb300 as p

    rank, world, local = dist_env()
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    n_total = len(probs)
    probs = [probs[i] for i in shard(n_total, rank, world)]
    t0 = time.perf_counter()
    slices, tuned = [], []
    for prob in probs:
        plan = p.Plan(prob.geom)
        tuned.append(plan.autotune(2 * prob.Q.shape[1]))
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
    del batch, states

    # dominant kernel: the 2 n_mat-channel transpose of every slice, timed
    # alone per slice (CUDA events, L2 flushed) and summed over the batch
    back_ms, ab = 0.0, 0
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
        ab += 2 * nm * 4 * (plan.n_rays + plan.n_pix)
    hbm, src = peaks()
    achieved = ab / (back_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "kernel": "backproject (rank 0's slices, timed alone)", "achieved": achieved,
                "peak": hbm, "unit": "GB/s", "frac": achieved / hbm, "traffic": None, "peak_source": src,
                "alg_bytes_per_launch": ab, "backproject_ms_per_iter": round(back_ms, 4), "note": ALG_NOTE}

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
    e2e_s = job_max(time.perf_counter() - t1, world, dev)
    del batch2, states2
    sizes = [int(s["prob"].geom.nx) for s in slices]
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
    if rank == 0 and cpu is not None and not args.no_cpu:
        line["cpu_baseline"] = cpu()
    return line


def cone_gap(args):
    """Time to the 1e-4 gap of the cone-beam one-step MBMD at 128^3 (the
    256^3 scan scaled down; 1500 + 3 x 300 iterations fit a few seconds
    there, not at 256^3)."""
    import torch

    import paper_2010_01371_gb300 as p
    prob = build_problem("c5_cone3d_128_block")
    y = torch.as_tensor(prob.y.astype(np.float32), device="cuda")
    t0 = time.perf_counter()
    plan, spec = p.Plan(prob.geom), p.Spectrum(prob.Q, prob.S)
    pc = p.Precond(plan, spec, "block", y, prob.beta)
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    gap = time_to_gap(p, torch.cuda.current_stream(), plan, spec, y, prob.beta, pc, args.gap_star, args.gap_iters,
                      build_s)
    gap["workload"] = "c5_cone3d_128_block"
    return gap


def largest(args):
    """The largest workloads, each with its own roofline, clocks, end-to-end
    leg and CPU baseline (bounded oracle samples scaled to the workload)."""
    import synth
    out = {}
    name = LARGEST[0]
    probs = synth.config4()
    small = min(probs, key=lambda q: q.geom.nx)
    pix = sum(q.geom.nx * q.geom.ny for q in probs)

    def cpu4():
        # one oracle iteration of the smallest (256^2) slice, scaled by the
        # batch's total pixels: per-slice work grows with pixels x rays / views
        # ~ N^2 at fixed views (the bins scale with N)
        return cpu_baseline(name, "block_fourier", small, 1, scale=small.geom.nx * small.geom.ny / pix,
                            per_replica_gb=2.0, what=f"on the {small.geom.nx}^2 slice of the batch")
    out[name] = ours_batch(args, probs, name, "block_fourier", WORKLOADS[name][2], cpu=cpu4)
    del probs
    name = LARGEST[1]
    prob = build_problem(name)
    views = 4

    def cpu5():
        sample = build_problem(name, views)
        return cpu_baseline(name, "block", sample, 1, views=views, scale=views / prob.geom.n_views,
                            per_replica_gb=4.0, what=f"on {views} of the {prob.geom.n_views} views of the scan "
                                                     f"(full 256^3 volume)")
    out[name] = ours(args, prob, name, "block", WORKLOADS[name][2], gap=None, cpu=cpu5)
    if not args.no_gap:
        out[name]["time_to_gap"] = cone_gap(args)
    return out


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
    out = {}
    if prob.geom.kind == 2:
        # cone beam: forward of the basis images, and the 2 n_mat-channel
        # transposes (fixed-point tile scatter, direct and split-table gathers)
        nm = x1.shape[0]
        s4 = torch.as_tensor(rng.random((2 * nm, plan.n_rays)).astype(np.float32), device=dev)
        l = torch.empty((nm, plan.n_rays), device=dev)
        img = torch.empty((2 * nm,) + plan.image_shape, device=dev)

        def timec(fn, reps=5):
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
        for mode in ["ray", "aligned"]:
            plan.set_projector(mode)
            out[f"project_{mode}_{nm}ch_ms"] = timec(lambda: p.mbir_project(plan, x1, l))
        for mode in ["tile", "tile8", "gather", "split"]:
            plan.set_backprojector("tile" if mode == "tile8" else mode)
            plan.set_cone_tile(8 if mode == "tile8" else 16)
            out[f"backproject_{mode}_{2 * nm}ch_ms"] = timec(lambda: p.mbir_backproject(plan, s4, img))
        print(json.dumps({"kernels": out, "workload": args.workload}), flush=True)
        return
    s2 = torch.as_tensor(rng.random((2, plan.n_rays)).astype(np.float32), device=dev)

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
    x3 = torch.as_tensor(np.concatenate([prob.truth] * 3).astype(np.float32), device=dev)
    l3 = torch.empty((3, plan.n_rays), device=dev)
    for mode in ["tile", "ray", "strip"]:
        plan.set_projector(mode)
        out[f"project_{mode}_1ch_ms"] = timeit(lambda: p.mbir_project(plan, x1, l1))
        out[f"project_{mode}_3ch_ms"] = timeit(lambda: p.mbir_project(plan, x3, l3))
    plan.set_projector("ray")
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
    ap.add_argument("--no-largest", action="store_true", help="skip the largest workloads of the default run")
    ap.add_argument("--gap-iters", type=int, default=300)
    ap.add_argument("--gap-star", type=int, default=1500)
    ap.add_argument("--cpu-iters", type=int, default=2)
    ap.add_argument("--kernels", action="store_true", help="time the projector variants alone")
    ap.add_argument("--workload", default=WORKLOAD, choices=sorted(WORKLOADS))
    args = ap.parse_args()
    import synth
    if args.kernels:
        if args.workload.startswith("c5"):       # geometry and phantom only
            kw = dict(WORKLOADS[args.workload][3]) if len(WORKLOADS[args.workload]) > 3 else {}
            kernel_bench(args, synth.config5(**kw, rays=False))
        else:
            kernel_bench(args, synth.config2())
        return
    if args.impl == "reference":
        reference_arm(args)
        return
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    builder, kind, desc, *kw = WORKLOADS[args.workload]
    kw = dict(kw[0]) if kw else {}
    blur = kw.pop("blur", None)
    noise = kw.pop("noise", None)
    prob = getattr(synth, builder)(**kw)
    if blur is not None:
        blur = synth.BLUR_TAPS[blur]
        prob = synth.with_detector_blur(prob, blur)
    if isinstance(prob, list):
        line = ours_batch(args, prob, args.workload, kind, desc)
    else:
        headline = args.workload == WORKLOAD
        cpu = (lambda: cpu_baseline(WORKLOAD, "haar", prob, args.cpu_iters, what="of the same workload")) \
            if headline else None
        line = ours(args, prob, args.workload, kind, desc, blur, noise,
                    gap=(args.gap_star, args.gap_iters), cpu=cpu)
        if headline and world == 1 and not args.no_largest:
            del prob
            line["largest"] = largest(args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
