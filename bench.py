#!/usr/bin/env python
"""Benchmark of the PRIEST hot path on GB300: projected sample-iterations per
second of full solves (Alg. 1: sample, K projection iterations, residual and
cost, elites, refit, Cholesky).

Default line: the batched workload of 256 uneven 2-D problems (obstacles
log-uniform in [10, 400], N in {256, 512, 1024, 2048}, n_p in {60, 100,
150}, K = 60, L = 3) solved by priest_plan_batch: per CEM iteration one
persistent projection launch over every problem's samples, one selection and
one refit launch, replayed as a CUDA graph.  One step = one batched solve of
all 256 problems; units per step = sum over problems of N K L.  The line also
carries the single-problem 2-D clutter solve (N = 1000, n_p = 100, K = 100,
L = 5) and the point-to-point solves (the paper's N_b = 110, 13 CEM
iterations) as extra keys.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload batched|clutter2d|...]

Under torchrun each rank solves its own 256 problems (a disjoint share of a
256 N problem set; no collective on the data path); rank 0 prints one JSON
line.  ``--impl reference`` times the FP64 CPU oracle on a bounded sample of
the same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2309_08235_gb300 import replicas as R  # noqa: E402

METRIC = "projected sample-iters/s; solves/s & p99 latency vs plain GPU path, at oracle tol"
UNIT = "sample-iters/s"
FP32_LANES = 128
BATCH_K, BATCH_L, BATCH_N = 60, 3, 256

WORKLOADS = {"clutter2d": "clutter2d_fp32", "ellipsoid3d": "ellipsoid3d_mixed", "p2p2d": "p2p2d", "p2p3d": "p2p3d",
             "clutter2d_bounds": "clutter2d_bounds", "dynamic2d": "dynamic2d"}


def workload_desc(p, cem, precision="fp32", name="clutter2d"):
    prec = ("FP32 projection" if precision == "fp32" else
            "FP32 projection, pair tests selected by a split-BF16 tensor-core product")
    if name in ("p2p2d", "p2p3d", "dynamic2d"):
        return (f"{name}: {p['n_obs']} obstacles, dims {p['dims']}, N={cem['n_samples']} samples, n_p={p['n_p']}, "
                f"K={cem['proj_iters']}, L={cem['cem_iters']} CEM iters (the paper's N_b = 110, N = 13), "
                f"{cem['n_elite']} elites, cost {'BARN-style' if p.get('cost_kind', 0) == 1 else 'sum |acc|^2'}, "
                f"{prec}")
    if name == "clutter2d_bounds":
        return (f"2-D clutter with workspace rows (box [0, 30]^2) and the paper's four boundary rows per axis "
                f"(end position only): {p['n_obs']} circles (10 moving), N={cem['n_samples']} samples, "
                f"n_p={p['n_p']}, K={cem['proj_iters']}, L={cem['cem_iters']}, {cem['n_elite']} elites, {prec}")
    if p["dims"] == 3:
        return (f"3-D point-to-point: {p['n_obs']} static ellipsoids in 20x20x8 m, N={cem['n_samples']} samples, "
                f"n_p={p['n_p']}, degree {p['degree']}, K={cem['proj_iters']} projection iters, "
                f"L={cem['cem_iters']} CEM iters, {cem['n_elite']} elites, {prec}")
    return (f"2-D clutter: {p['n_obs'] - int(np.count_nonzero(np.abs(p['vel']).sum(1)))} static + "
            f"{int(np.count_nonzero(np.abs(p['vel']).sum(1)))} moving circles in 30x30 m, "
            f"N={cem['n_samples']} samples, n_p={p['n_p']}, degree {p['degree']}, "
            f"K={cem['proj_iters']} projection iters, L={cem['cem_iters']} CEM iters, "
            f"{cem['n_elite']} elites, {prec}")


BATCH_DESC = ("batched: 256 uneven 2-D problems (obstacles log-uniform 10-400, 10 % moving; N in {256, 512, 1024, "
              "2048}; n_p in {60, 100, 150}; degree 10), K=60 projection iters, L=3 CEM iters, N/10 elites, FP32 "
              "projection; one persistent projection launch per CEM iteration over all problems, CUDA graph replay")


def flops_per_sample_iter(p, nf=5):
    """Algorithmic FP32 flops of one projected sample-iteration, the per-unit
    figure of the hot-path scope: per (point, obstacle) pair the direct polar
    test (offset, scaled squared distance, activity test: 14 flops in 2-D, 22
    in 3-D; the rare active pairs' rsqrt is not counted), the velocity /
    acceleration blocks (12 flops per point and block), the two basis products
    of the affine map over all n_v columns (2 x dims x 2 x 3 n_p n_v) and the
    shared-inverse step (2 x dims x n_v^2)."""
    dims, n_p, n_o = p["dims"], p["n_p"], p["n_obs"]
    nv = p.get("degree", 10) + 1
    pair = 14 if dims == 2 else 22
    return n_p * n_o * pair + 2 * n_p * 12 + 2 * dims * (2 * 3 * n_p * nv) + 2 * dims * nv * nv


def free_coefficients(p):
    """Free Bernstein coefficients per axis: n_v minus the three start
    conditions minus the end conditions of the final mask."""
    fixed_end = {7: 3, 3: 2, 1: 1, 0: 0}[int(p.get("bc_final_mask", 7))]
    return p.get("degree", 10) + 1 - 3 - fixed_end


def sm_count(dev=None):
    import torch

    return int(torch.cuda.get_device_properties(dev if dev is not None else 0).multi_processor_count)


def sm_max_mhz(clocks):
    """The SM clock ceiling: nvidia-smi's maximum seen during the run, else
    the measured peaks file, else the part's nominal 2070 MHz."""
    if clocks.get("sm_max_mhz"):
        return float(clocks["sm_max_mhz"])
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            return float(json.load(open(path))["sm_max_mhz"])
        except Exception:
            pass
    return 2070.0


def fp32_peak_tflops(n_sm, mhz):
    return n_sm * FP32_LANES * 2 * mhz * 1e6 / 1e12


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "100",
                 "-i", str(self.device)], stdout=self.file, stderr=subprocess.DEVNULL)
            time.sleep(0.5)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.3)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 10:
                    rows.append(parts)
        os.unlink(self.file.name)
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        busy = [s for s in sm if s > 0.5 * (max(mx) if mx else 1)]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[6 + k].lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(busy or sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(rows)}


def dist_env():
    return R.env()


def stored_profile(key):
    """A figure of the committed ncu summary (profiles/traffic.txt: DRAM bytes
    per launch, issue / pipe utilisation of the dominant kernels), or None."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path):
        return None
    for ln in open(path):
        if ln.startswith(key + ":"):
            return float(ln.split(":", 1)[1].split()[0])
    return None


SCREEN_NOTE = ("achieved counts the scope table's per-unit work: the direct polar test of every (point, obstacle) pair "
               "in every iteration.  The point-owner kernel tests only each point's listed pairs exactly; it screens "
               "for its lists only when it rebuilds them (the first iteration, and after a point of the CTA moved 7/8 "
               "of the list margin), then the static obstacles of the point's grid cell and every moving one; the "
               "pairs left out are provably inactive (zero residual rows), so its results equal full screening "
               "(bitwise) and achieved can exceed the FP32 peak.  'executed' holds the kernel's own issue and "
               "FMA-pipe utilisation from the committed ncu capture.")


def executed(prefix):
    out = {k: stored_profile(f"{prefix}_{k}") for k in ("issue_active_pct", "fma_pipe_pct", "alu_pipe_pct")}
    if all(v is None for v in out.values()):
        return None
    out["note"] = "ncu capture committed under profiles/ (not measured in this run)"
    return out


# ---------------------------------------------------------------------------
# The FP64 oracle on the host cores (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_projection_rate(jobs, threads):
    """Projected sample-iterations/s of the FP64 oracle on `jobs`, a list of
    (problem, samples, K): each job's K projection iterations + residual /
    cost.  threads > 1 runs the jobs' rows in parallel (the oracle is plain
    reentrant C called through ctypes, which releases the interpreter lock),
    one chunk of rows per task."""
    import oracle as O

    O.build()
    tasks = []
    for p, xi, K in jobs:
        step = max(1, int(np.ceil(len(xi) / max(1, threads))) if threads > 1 else len(xi))
        for a in range(0, len(xi), step):
            tasks.append((p, xi[a:a + step], K))

    def run(t):
        p, xi, K = t
        xb, _ = O.project(p, xi, K)
        O.residual_cost(p, xb)

    units = sum(len(xi) * K for _, xi, K in jobs)
    t0 = time.perf_counter()
    if threads > 1:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(run, tasks))
    else:
        for t in tasks:
            run(t)
    dt = time.perf_counter() - t0
    return units / dt, dt


def batched_oracle_jobs(scale=8, n_sub=16, seed=0):
    """The bounded sample of the batched workload: the first n_sub of its
    seeded problems, scale * N_i / 256 rows of problem i (so the rows keep
    the workload's weighting of problems by sample count), K = 60."""
    import oracle as O
    from paper_2309_08235_gb300 import workloads as W

    O.build()
    jobs = []
    for i, (p, N) in enumerate(W.batched_problems(n_sub)):
        m = max(1, scale * N // 256)
        xi = O.default_mean(p) + 2.0 * W.normals(seed * 1000 + i, (m, 22))
        jobs.append((p, xi, BATCH_K))
    return jobs


def single_oracle_jobs(p, cem, n_samples, seed=0):
    import oracle as O
    from paper_2309_08235_gb300 import workloads as W

    O.build()
    D = p["dims"] * (p["degree"] + 1)
    xi = O.default_mean(p) + cem["init_std"] * W.normals(seed, (n_samples, D))
    return [(p, xi, cem["proj_iters"])]


def cpu_baselines(jobs, sample_desc):
    """The oracle on all host cores and on one thread (same sample)."""
    cores = os.cpu_count() or 1
    rate_all, dt_all = oracle_projection_rate(jobs, cores)
    rate_1, dt_1 = oracle_projection_rate(jobs, 1)
    return {"value": rate_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{sample_desc}; FP64 oracle, rows split over {cores} threads, {dt_all:.1f} s",
            "single_thread": {"value": rate_1, "unit": UNIT, "cores": 1, "seconds": dt_1}}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2309_08235_gb300 import workloads as W

    cores = os.cpu_count() or 1
    if args.workload == "batched":
        desc = BATCH_DESC
        make = lambda k: batched_oracle_jobs(scale=args.ref_scale, seed=k)  # noqa: E731
        sample = (f"rows {args.ref_scale} N_i / 256 of each of the first 16 seeded problems of the batched "
                  f"workload (K=60 projection iterations + residual / cost) per step")
    else:
        p, cem = W.workload(WORKLOADS[args.workload])
        desc = workload_desc(p, cem, name=args.workload)
        # calibrate, then size each step so the whole run stays within ~2 minutes
        rate, _ = oracle_projection_rate(single_oracle_jobs(p, dict(cem, proj_iters=10), cores), cores)
        per_step_s = 120.0 / max(1, args.steps + args.warmup)
        m = max(cores, int(per_step_s * rate / cem["proj_iters"]))
        make = lambda k: single_oracle_jobs(p, cem, m, seed=k)  # noqa: E731
        sample = f"{m} samples x {cem['proj_iters']} projection iterations (+ residual / cost) per step"
    for k in range(args.warmup):
        oracle_projection_rate(make(100 + k), cores)
    units, secs = 0.0, 0.0
    times = []
    for k in range(args.steps):
        jobs = make(k + 1)
        rate, dt = oracle_projection_rate(jobs, cores)
        units += rate * dt
        secs += dt
        times.append(dt)
    value = units / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": desc, "impl": "FP64 CPU oracle"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample + f", FP64 oracle, rows split over {cores} threads"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------
# One problem per step (the 2-D clutter, 3-D, point-to-point workloads)
# ---------------------------------------------------------------------------

def measure_single(args, name, steps, warmup, precision="fp32", plain_steps=0, e2e=True, cpu=False, dist=None):
    """Full solves of one problem per step on this rank's GPU: the device
    timed rate, the projection kernel's roofline, optionally the end-to-end
    rate through priest_plan_z with host buffers, the plain per-problem path
    and the oracle's baseline.  Returns the line's dict."""
    import torch

    from paper_2309_08235_gb300 import priest as P
    from paper_2309_08235_gb300 import workloads as W

    rank, world, local = dist_env()
    p, cem = W.workload(WORKLOADS[name])
    N, K, L = cem["n_samples"], cem["proj_iters"], cem["cem_iters"]
    D = p["dims"] * (p["degree"] + 1)
    units = N * K * L
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)
    prec = P.PRIEST_MIXED_BF16 if precision == "mixed" else P.PRIEST_FP32
    ctx = P.Context(p, cem, precision=prec, stream=stream.cuda_stream)
    prob, keep = P.make_problem(p, cem, per_problem_shape=True)
    h = P.priest_load(ctx.h, prob)
    z_host = torch.from_numpy(W.normals(1000 + rank, (L, N, D))).pin_memory()
    z_dev = z_host.to(dev)
    out = torch.zeros(D + 4, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        P.priest_plan_device(ctx.h, h, z_dev.data_ptr(), out.data_ptr())

    with torch.cuda.stream(stream):
        for _ in range(max(3, warmup)):
            step()
    stream.synchronize()
    P.priest_sync(ctx.h)

    # ---- timed region: device-resident inputs, L2 flushed between steps
    sampler = ClockSampler(local)
    sampler.start()
    P.priest_profile_read(ctx.h)
    P.priest_profile_enable(ctx.h, 1)
    l0 = ctx.launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    R.barrier(dist)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            step()
            e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    R.barrier(dist)
    clocks = sampler.stop()
    P.priest_profile_enable(ctx.h, 0)
    launches = ctx.launches() - l0
    kind = P.priest_last_kernel(ctx.h)
    n_proj_launch, proj_ms = P.priest_profile_read(ctx.h)
    P.priest_sync(ctx.h)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    value, t_max, _ = R.job_rate(units * steps, sum(step_ms) / 1e3, dist, dev)
    total_ms = 1e3 * t_max

    # ---- roofline of the dominant kernel (the fused projection)
    avg_proj_ms = proj_ms / max(1, n_proj_launch)
    flops_launch = flops_per_sample_iter(p) * N * K
    n_sm = sm_count(dev)
    mhz = sm_max_mhz(clocks)
    peak = fp32_peak_tflops(n_sm, mhz)
    achieved = flops_launch / (avg_proj_ms / 1e3) / 1e12
    kname = {0: "project_kernel (FP32 chunked projection)", 1: "pts_kernel (FP32 point-owner projection)",
             2: "project_tc_kernel (tcgen05 pair tests)"}.get(kind, "projection kernel")
    # the committed ncu figures of this workload's point-owner launch, where one was captured
    prof = {"clutter2d": "pts_kernel", "ellipsoid3d": "pts_kernel_3d"}.get(name) if kind == 1 else None
    traffic = stored_profile(f"{prof}_bytes_per_launch") if prof else None
    traffic = None if traffic is None else int(traffic)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": f"{kname}, {p['dims']}-D", "avg_launch_ms": avg_proj_ms,
                "launches": n_proj_launch, "flops_per_launch": flops_launch,
                "flops_note": "algorithmic: direct polar pair test 14 (2-D) / 22 (3-D) flops per pair, "
                              "vel/acc blocks, both basis products over all n_v columns, shared-inverse step",
                "peak_note": f"FP32 FMA peak derived: {n_sm} SMs x 128 lanes x 2 flop x {mhz:g} MHz",
                "traffic_note": ("dram bytes per launch from one ncu capture (profiles/traffic.txt), not measured "
                                 "in this run") if traffic else None}
    if kind == 1:
        roofline["note"] = SCREEN_NOTE
        if prof:
            roofline["executed"] = executed(prof)
    if clocks.get("sm_mhz"):
        roofline["frac_at_median_clock"] = achieved / fp32_peak_tflops(n_sm, clocks["sm_mhz"])
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload_desc(p, cem, precision, name),
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": "replicas" if world > 1 else "single GPU", "units_per_step": units},
            "solves_per_s": steps * world / (total_ms / 1e3),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "roofline": roofline, "gpu_launches": int(launches), "clocks": clocks}

    if e2e:
        # ---- end to end through the host-pointer C ABI (pinned z in, result out)
        res = P.priest_result()
        z_np = z_host.numpy()
        for _ in range(2):
            P.priest_plan_z(ctx.h, prob, None, None, z_np, res)
        e2e_steps = max(3, min(steps, 50))
        R.barrier(dist)
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            P.priest_plan_z(ctx.h, prob, None, None, z_np, res)
        e2e_rate, _, _ = R.job_rate(units * e2e_steps, time.perf_counter() - t0, dist, dev)
        obs_bytes = 8 * (p["n_obs"] * (2 * p["dims"] + 2))
        line["e2e"] = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(z_np.nbytes + obs_bytes),
                       "d2h_bytes_per_step": int(8 * (D + 4 + D)), "api": "priest_plan_z (host buffers, blocking)"}

    if plain_steps > 0:
        # ---- the plain per-problem FP32 GPU path on the same workload and draws
        out_p = torch.zeros(D + 4, dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            P.priest_plan_plain_device(ctx.h, h, z_dev.data_ptr(), out_p.data_ptr())
        P.priest_sync(ctx.h)
        pev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(plain_steps)]
        with torch.cuda.stream(stream):
            for e0, e1 in pev:
                flush.zero_()
                e0.record(stream)
                P.priest_plan_plain_device(ctx.h, h, z_dev.data_ptr(), out_p.data_ptr())
                e1.record(stream)
        P.priest_sync(ctx.h)
        pms = sum(a.elapsed_time(b) for a, b in pev) / len(pev)
        line["plain_gpu"] = {"value": units / (pms / 1e3), "unit": UNIT, "ms_per_step": pms, "steps": len(pev),
                             "speedup_of_fused": pms / (total_ms / steps),
                             "c_aug": float(out_p.cpu().numpy()[D + 2]), "c_aug_fused": float(out.cpu().numpy()[D + 2]),
                             "path": "priest_plan_plain_device: one kernel per step, HBM trajectory / residual tiles"}
    if cpu and rank == 0 and world == 1:
        line["cpu_baseline"] = cpu_baselines(single_oracle_jobs(p, cem, args.cpu_samples),
                                             f"{args.cpu_samples} samples x {K} projection iterations "
                                             "(+ residual / cost) of the same workload")
    P.priest_unload(ctx.h, h)
    ctx.close()
    return line


def run_single(args):
    import torch

    from paper_2309_08235_gb300 import build as B

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    B.build()
    line = measure_single(args, args.workload, args.steps, args.warmup, args.precision, args.plain_steps,
                          e2e=True, cpu=not args.no_cpu_baseline, dist=dist)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------------------
# The batched workload (the default line)
# ---------------------------------------------------------------------------

def run_batched(args):
    """256 uneven 2-D problems per rank in shared launches (priest_plan_batch,
    graph replay): device-timed rate, roofline of the persistent projection
    kernel, end-to-end rate through priest_plan_batch_host, the plain
    per-problem path on the same problems and draws, the oracle's baseline,
    and the single-problem workloads as extra keys."""
    import torch

    from paper_2309_08235_gb300 import build as B
    from paper_2309_08235_gb300 import priest as P
    from paper_2309_08235_gb300 import workloads as W

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    B.build()
    dev = torch.device("cuda", local)
    K, L, n = BATCH_K, BATCH_L, args.batch_problems
    # this rank's share of an n x world problem set (weak scaling: n per rank)
    share = R.shard(n * world, rank, world)
    probs = W.batched_problems(len(share), seed0=100 + share.start)
    stream = torch.cuda.Stream(device=dev)
    p0, n0 = probs[0]
    ctx = P.Context(p0, W.cem_settings(n0, K, L), precision=P.PRIEST_FP32, stream=stream.cuda_stream)
    handles, structs, keep, z_host, z_dev, outs = [], [], [], [], [], []
    units = flops_launch = pairs = 0
    h2d_obs = 0
    for i, (p, N) in enumerate(probs):
        cem = W.cem_settings(N, K, L)
        prob, kp = P.make_problem(p, cem, per_problem_shape=True)
        keep.append(kp)
        structs.append(prob)
        handles.append(P.priest_load(ctx.h, prob))
        zh = torch.from_numpy(W.normals(2000 + share.start + i, (L, N, 22))).pin_memory()
        z_host.append(zh)
        z_dev.append(zh.to(dev))
        outs.append(torch.zeros(26, dtype=torch.float64, device=dev))
        units += N * K * L
        pairs += N * K * L * p["n_p"] * p["n_obs"]
        flops_launch += flops_per_sample_iter(p) * N * K
        h2d_obs += 8 * (p["n_obs"] * (2 * p["dims"] + 2) + 18)
    zp = [z.data_ptr() for z in z_dev]
    op = [o.data_ptr() for o in outs]
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    t_setup = time.perf_counter()
    with torch.cuda.stream(stream):
        for _ in range(max(3, args.warmup)):  # the first call tunes tilings and records the graph
            P.priest_plan_batch(ctx.h, handles, zp, op)
    P.priest_sync(ctx.h)
    t_setup = time.perf_counter() - t_setup
    kind = P.priest_last_kernel(ctx.h)

    # ---- timed region: device-resident inputs, L2 flushed between steps
    sampler = ClockSampler(local)
    sampler.start()
    P.priest_profile_read(ctx.h)
    P.priest_profile_enable(ctx.h, 1)
    l0 = ctx.launches()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    R.barrier(dist)
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for e0, e1 in evs:
            flush.zero_()
            e0.record(stream)
            P.priest_plan_batch(ctx.h, handles, zp, op)
            e1.record(stream)
    stream.synchronize()
    torch.cuda.synchronize()
    R.barrier(dist)
    clocks = sampler.stop()
    P.priest_profile_enable(ctx.h, 0)
    launches = ctx.launches() - l0
    n_proj_launch, proj_ms = P.priest_profile_read(ctx.h)
    P.priest_sync(ctx.h)
    step_ms = [e0.elapsed_time(e1) for e0, e1 in evs]
    value, t_max, _ = R.job_rate(units * args.steps, sum(step_ms) / 1e3, dist, dev)
    total_ms = 1e3 * t_max

    # ---- roofline of the persistent projection kernel
    avg_proj_ms = proj_ms / max(1, n_proj_launch)
    n_sm = sm_count(dev)
    mhz = sm_max_mhz(clocks)
    peak = fp32_peak_tflops(n_sm, mhz)
    achieved = flops_launch / (avg_proj_ms / 1e3) / 1e12
    kname = {0: "project_batch_kernel (FP32 chunked, persistent)",
             1: "pts_batch_kernel (FP32 point-owner, persistent)"}.get(kind, "batched projection kernel")
    traffic = stored_profile("pts_batch_kernel_bytes_per_launch") if kind == 1 else None
    traffic = None if traffic is None else int(traffic)
    roofline = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                "traffic": traffic, "kernel": kname, "avg_launch_ms": avg_proj_ms, "launches": n_proj_launch,
                "flops_per_launch": flops_launch,
                "flops_note": "algorithmic, summed over the launch's problems: N_i K x (n_p n_o x 14 flops per "
                              "direct polar pair test + vel/acc blocks + both basis products over all n_v columns "
                              "+ shared-inverse step)",
                "peak_note": f"FP32 FMA peak derived: {n_sm} SMs x 128 lanes x 2 flop x {mhz:g} MHz",
                "traffic_note": ("dram bytes per launch from one ncu capture of this workload "
                                 "(profiles/traffic.txt), not measured in this run") if traffic else None}
    if kind == 1:
        roofline["note"] = SCREEN_NOTE
        roofline["executed"] = executed("pts_batch_kernel")
    if clocks.get("sm_mhz"):
        roofline["frac_at_median_clock"] = achieved / fp32_peak_tflops(n_sm, clocks["sm_mhz"])

    # ---- end to end through the host-buffer C ABI: problems, pinned draws in, results out
    res = (P.priest_result * len(probs))()
    z_np = [z.numpy() for z in z_host]
    # the argument arrays of the repeated call, built once as a serving loop would keep them
    parr, zarr = P.priest_problem_array(structs), P.pointer_array(z_np)
    for _ in range(2):  # the first call makes the resident set, tunes nothing new and records its graph
        P.priest_plan_batch_host(ctx.h, parr, zarr, res)
    e2e_steps = max(3, min(args.steps, 20))
    R.barrier(dist)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        P.priest_plan_batch_host(ctx.h, parr, zarr, res)
    e2e_rate, _, _ = R.job_rate(units * e2e_steps, time.perf_counter() - t0, dist, dev)
    h2d_z = sum(z.nbytes for z in z_np)
    e2e = {"value": e2e_rate, "unit": UNIT, "h2d_bytes_per_step": int(h2d_z + h2d_obs),
           "d2h_bytes_per_step": int(8 * len(probs) * (30 + 22)),
           "api": "priest_plan_batch_host (host problem structs and pinned draws in, results out, blocking)"}
    ok = sum(1 for i in range(len(probs)) if res[i].status == 0)

    # ---- the plain per-problem FP32 path: the same problems and draws, one at a time
    plain = None
    if args.plain_steps > 0:
        outp = torch.zeros(26, dtype=torch.float64, device=dev)
        with torch.cuda.stream(stream):
            P.priest_plan_plain_device(ctx.h, handles[0], zp[0], outp.data_ptr())
        P.priest_sync(ctx.h)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            flush.zero_()
            e0.record(stream)
            for h, z in zip(handles, zp):
                P.priest_plan_plain_device(ctx.h, h, z, outp.data_ptr())
            e1.record(stream)
        P.priest_sync(ctx.h)
        pms = e0.elapsed_time(e1)
        plain = {"value": units / (pms / 1e3), "unit": UNIT, "ms_per_step": pms, "steps": 1,
                 "speedup_of_fused": pms / (total_ms / args.steps),
                 "path": "priest_plan_plain_device on each of the same problems in turn (one kernel per step, "
                         "HBM trajectory / residual tiles), same draws"}
    for h in handles:
        P.priest_unload(ctx.h, h)
    ctx.close()

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": BATCH_DESC, "problems_per_gpu": len(probs), "units_per_step": units,
                       "pair_tests_per_step": pairs,
                       "l2": "flushed between timed steps (256 MB write); the draws alone are 130 MB",
                       "parallelism": f"dp{world}: a disjoint share of {n * world} problems per GPU"
                       if world > 1 else "single GPU"},
            "solves_per_s": len(probs) * args.steps * world / (total_ms / 1e3),
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99)),
                           "note": "per batched solve of all problems"},
            "roofline": roofline, "e2e": e2e, "gpu_launches": int(launches), "clocks": clocks,
            "results_ok": ok, "first_call_s": t_setup, "plain_gpu": plain}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baselines(
            batched_oracle_jobs(scale=args.ref_scale),
            f"rows {args.ref_scale} N_i / 256 of each of the first 16 seeded problems of the batched workload "
            "(K=60 projection iterations + residual / cost; the rows keep the workload's weighting by N_i)")
    if not args.no_extra:
        # the single-problem workloads on the same GPU, as extra keys
        extra = {}
        c2 = measure_single(args, "clutter2d", max(3, min(args.steps, 50)), 3, plain_steps=3, e2e=True, dist=dist)
        extra["clutter2d"] = {k: c2[k] for k in ("value", "ms_per_step", "solves_per_s", "config", "e2e",
                                                 "plain_gpu")}
        extra["clutter2d"]["roofline"] = {k: c2["roofline"].get(k) for k in
                                          ("kernel", "achieved", "peak", "frac", "avg_launch_ms", "traffic")}
        extra["clutter2d"]["roofline"]["executed"] = c2["roofline"].get("executed")
        for name in ("p2p2d", "p2p3d", "dynamic2d"):
            r = measure_single(args, name, 20, 3, e2e=False, dist=dist)
            extra[name] = {"ms_per_solve": r["ms_per_step"], "value": r["value"],
                           "projection_launch_ms": r["roofline"]["avg_launch_ms"],
                           "workload": r["config"]["workload"]}
        line["extra_workloads"] = extra
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()
    return 0


def fifo_latencies(arrivals, service):
    """Completion-minus-arrival times of a single FIFO server (Lindley's
    recursion) that serves request i for service[i] seconds."""
    free_at = 0.0
    out = []
    for a, s in zip(arrivals, service):
        start = max(a, free_at)
        free_at = start + s
        out.append(free_at - a)
    return out


def run_serving(args):
    """Serving workload: a Poisson stream of 2-D / 3-D planning requests
    (sizes as the batched workload, 20 % 3-D, 30 % warm replans of an earlier
    robot) submitted in real time to priest_submit; the library's serving loop
    batches them continuously under an HBM budget.  Reports solves/s, p50 /
    p99 latency and projected sample-iters/s, next to the same stream served
    one request at a time by priest_plan (service times measured on the GPU,
    queueing replayed for a single FIFO server).  Not the default bench line."""
    import threading

    import torch

    from paper_2309_08235_gb300 import build as B
    from paper_2309_08235_gb300 import priest as P
    from paper_2309_08235_gb300 import workloads as W

    B.build()
    torch.cuda.init()
    K, L = 60, 3
    reqs = W.serving_requests(rate=args.rate, duration=args.duration, seed=7)
    p0 = reqs[0][1]
    budget = int(args.budget_gb * (1 << 30))
    ctx = P.Context(p0, W.cem_settings(256, K, L), precision=P.PRIEST_FP32, hbm_budget=budget)
    cems = [W.cem_settings(N, K, L, dims=p["dims"]) for (_, p, N, _) in reqs]
    # warm-up, untimed: a burst from another stream of the same mix (every
    # kernel variant loaded, staging buffers sized), then a short paced run
    warm = W.serving_requests(rate=args.rate, duration=0.5, seed=8)
    wt = [ctx.submit(p, W.cem_settings(N, K, L, dims=p["dims"]), robot_id=10**9 + rid) for (_, p, N, rid) in warm]
    for t in wt:
        ctx.wait(t)
    st0 = ctx.serve_stats()
    tickets = [None] * len(reqs)
    sampler = ClockSampler(0)
    sampler.start()
    t0 = time.perf_counter()

    def submitter():
        for i, ((ta, p, N, rid), cem) in enumerate(zip(reqs, cems)):
            dt = t0 + ta - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = ctx.submit(p, cem, robot_id=rid)

    th = threading.Thread(target=submitter)
    th.start()
    res = []
    for i in range(len(reqs)):
        while tickets[i] is None:
            time.sleep(0.0005)
        res.append(ctx.wait(tickets[i]))
    t_end = time.perf_counter()
    th.join()
    clocks = sampler.stop()
    st = ctx.serve_stats()
    wall = t_end - t0
    lat = np.array([r["latency_ms"] for r in res])
    ok = sum(1 for r in res if r["status"] == 0)
    units = sum(cem["n_samples"] * K * L for cem in cems)
    steps = st["steps"] - st0["steps"]
    served = {
        "requests": len(reqs), "ok": ok, "wall_s": wall, "solves_per_s": len(reqs) / wall,
        "sample_iters_per_s": units / wall, "offered_sample_iters_per_s": units / args.duration,
        "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
        "max_ms": float(lat.max()), "steps": steps,
        "mean_batch": (st["slot_steps"] - st0["slot_steps"]) / max(1, steps), "max_active": st["max_active"],
        "warm_starts": st["warm_starts"] - st0["warm_starts"], "peak_bytes": st["peak_bytes"],
        "budget_bytes": st["budget_bytes"], "deferred": st["deferred"] - st0["deferred"],
    }
    if args.dump:
        np.savez(args.dump, arrival=np.array([r[0] for r in reqs]), latency_ms=lat,
                 dims=np.array([r[1]["dims"] for r in reqs]), n=np.array([r[2] for r in reqs]),
                 n_obs=np.array([r[1]["n_obs"] for r in reqs]), n_p=np.array([r[1]["n_p"] for r in reqs]),
                 robot=np.array([r[3] for r in reqs]))
    ctx.close()
    # one request at a time through the plain per-problem FP32 path (load,
    # device draws, solve, result read, unload): measured service times of a
    # sample, FIFO queueing replayed on the full arrival stream
    n_seq = min(len(reqs), args.seq_sample)
    stride = max(1, len(reqs) // n_seq)
    idx = list(range(0, len(reqs), stride))[:n_seq]
    pctx = P.Context(p0, W.cem_settings(256, K, L), precision=P.PRIEST_FP32)
    svc = []
    for rep, i in enumerate([idx[0]] + idx):  # the first one again as a warm-up
        _, p, N, _ = reqs[i]
        cem = cems[i]
        D = p["dims"] * 11
        torch.cuda.synchronize()
        a = time.perf_counter()
        prob, kp = P.make_problem(p, cem, per_problem_shape=True)
        hh = P.priest_load(pctx.h, prob)
        z = torch.empty(L * N * D, dtype=torch.float64, device="cuda")
        P.priest_rng_normal_device(p["seed"], z.numel(), z.data_ptr(), torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        o = torch.zeros(D + 4, dtype=torch.float64, device="cuda")
        P.priest_plan_plain_device(pctx.h, hh, z.data_ptr(), o.data_ptr())
        P.priest_sync(pctx.h)
        _ = o.cpu()
        P.priest_unload(pctx.h, hh)
        if rep > 0:
            svc.append(time.perf_counter() - a)
    pctx.close()
    mean_svc = float(np.mean(svc))
    rng = np.random.default_rng(0)
    service = rng.choice(np.array(svc), size=len(reqs))
    seq_lat = np.array(fifo_latencies([r[0] for r in reqs], service)) * 1e3
    seq = {"service_ms_mean": 1e3 * mean_svc, "solves_per_s_capacity": 1.0 / mean_svc,
           "p50_ms": float(np.percentile(seq_lat, 50)), "p99_ms": float(np.percentile(seq_lat, 99)),
           "sample": f"{len(idx)} requests timed one at a time, FIFO replay of all {len(reqs)} arrivals",
           "method": "replayed: the plain path's measured per-request service times (load, device draws, solve, "
                     "result read, unload) fed to a single FIFO server over the same arrival times (Lindley's "
                     "recursion), not a live run of the stream"}
    line = {"metric": METRIC, "value": served["sample_iters_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": steps, "warmup": len(warm), "ms_per_step": 1e3 * wall / max(1, steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"serving: Poisson {args.rate:g} req/s for {args.duration:g} s, sizes as the "
                                   "batched workload, 20% 3-D, 30% warm replans, K=60, L=3, "
                                   f"{args.budget_gb:g} GB budget"},
            "serving": served, "plain_gpu_one_at_a_time": seq, "clocks": clocks}
    print(json.dumps(line), flush=True)
    return 0


def run_dpriest(args):
    """D-PRIEST scaling (the paper's per-iteration time against the number
    of distributions): the 2-D clutter scene with M distributions of a fixed
    N_b / M = 1000 samples each, K = 100, L = 5, one stacked projection launch
    per CEM iteration.  Reports per-iteration time and projected
    sample-iters/s for each M.  Not the default bench line."""
    import torch

    from paper_2309_08235_gb300 import build as B
    from paper_2309_08235_gb300 import priest as P
    from paper_2309_08235_gb300 import workloads as W

    B.build()
    p, cem0 = W.workload("clutter2d_fp32")
    K, L, nj = cem0["proj_iters"], cem0["cem_iters"], 1000
    prec = P.PRIEST_MIXED_BF16 if args.precision == "mixed" else P.PRIEST_FP32
    rows = []
    for M in (1, 2, 4, 8):
        cem = W.cem_settings(M * nj, K, L, n_elite=100 * M)
        z = W.normals(3000 + M, (L, M * nj, 22))
        with P.Context(p, cem, precision=prec) as ctx:
            for _ in range(max(1, args.warmup)):
                ctx.plan_multi(p, M, z=z)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                r = ctx.plan_multi(p, M, z=z)
            dt = (time.perf_counter() - t0) / args.steps
        rows.append({"M": M, "samples": M * nj, "ms_per_solve": 1e3 * dt, "ms_per_cem_iteration": 1e3 * dt / L,
                     "sample_iters_per_s": M * nj * K * L / dt, "best_dist": r["dist"],
                     "best_c_aug": r["best"]["c_aug"]})
    line = {"metric": METRIC, "value": rows[-1]["sample_iters_per_s"], "unit": UNIT, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rows[-1]["ms_per_solve"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "D-PRIEST sweep on the 2-D clutter scene: M distributions x 1000 samples, "
                                   "K=100, L=5 (host draws, blocking priest_plan_multi)"},
            "sweep": rows}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-samples", type=int, default=160)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true", help="batched: skip the single-problem extra keys")
    ap.add_argument("--ref-scale", type=int, default=8,
                    help="batched oracle sample: rows ref_scale * N_i / 256 of each of 16 problems")
    ap.add_argument("--workload", choices=["clutter2d", "clutter2d_bounds", "ellipsoid3d", "p2p2d", "p2p3d", "dynamic2d",
                                           "batched", "serving", "dpriest"],
                    default="batched",
                    help="batched: the default line (256 uneven problems); the single-problem workloads print "
                         "their own line; serving: Poisson request stream; dpriest: distribution sweep")
    ap.add_argument("--batch-problems", type=int, default=BATCH_N)
    ap.add_argument("--rate", type=float, default=500.0)
    ap.add_argument("--duration", type=float, default=60.0)
    ap.add_argument("--budget-gb", type=float, default=8.0)
    ap.add_argument("--seq-sample", type=int, default=300)
    ap.add_argument("--plain-steps", type=int, default=10, help="timed solves of the plain per-problem path")
    ap.add_argument("--precision", choices=["fp32", "mixed"], default="fp32",
                    help="fp32: FMA pair tests; mixed: pair tests selected by the BF16 tensor-core product")
    ap.add_argument("--dump", default=None, help="serving: save per-request arrival / latency / sizes (.npz)")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload in ("serving", "dpriest"):
            args.workload = "batched"
        return run_reference(args)
    if args.workload == "batched":
        return run_batched(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "dpriest":
        return run_dpriest(args)
    return run_single(args)


if __name__ == "__main__":
    sys.exit(main())
