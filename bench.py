"""Benchmark: adaptive image ray-tracing (AIR) of a block-AMR cone-shock grid
on one GB300, against the fixed-resolution image and the FP64 CPU oracle.

A step is one adaptive image: base image traced, then scan / balance / refine /
trace sweeps until nothing is flagged, then leaf output and band flux, all in
the library's CUDA kernels through the C ABI. The grid is resident in HBM
(uploaded once, outside the timed region); L2 is flushed before every timed
step by writing a 256 MiB buffer.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line (rank 0). With N > 1 (torchrun) every rank renders the
same image independently (replicas, weak scaling) and value = total steps of
all ranks / max time over ranks. `--impl reference` times the oracle on the
host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import scenes  # noqa: E402

METRIC = "AIR image time & ray-cell steps/s on 1 GB300 vs fixed-res, at ≤1e-4 rel error"
UNIT = "ray-cell steps/s"
WORKLOAD = dict(
    workload="cone-shock block-AMR grid: 128^3 base cells in 16^3 bricks, 3 refinement levels "
             "(1024^3 effective), FP32 rho/T with sigma=0.3 lognormal clumping, 64-bin "
             "Lambda(T), 1 band (1-10 keV) with absorption; view +z; AIR base 256^2, "
             "max level 4 (4096^2 equivalent), xi_crit 0.5, Eq. 2 axis-sum norm, refine on I",
    seed=0, n_base=128, brick=16, levels=3, base_res=256, max_level=4, xi_crit=0.5,
    fixed_res=4096)
BYTES_PER_STEP = 8  # rho (f32) + table coordinate of T (u32) fetched per ray-cell segment


def sample_clocks_start(path):
    dev = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    cmd = ["nvidia-smi", "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,"
           "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "200"]
    if dev.strip().isdigit():
        cmd[1:1] = ["-i", dev.strip()]
    try:
        f = open(path, "w")
        return subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def sample_clocks_stop(proc, f, path):
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.close()
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        p = [x.strip() for x in line.split(",")]
        if len(p) < 9:
            continue
        try:
            sm.append(float(p[1]))
            mx.append(float(p[2]))
        except ValueError:
            continue
        for k, nm in enumerate(names):
            if p[5 + k].lower().startswith("active"):
                reasons.add(nm)
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
            "samples": len(sm)}


def oracle_sample_rate(sc, view, lv, ii, jj, n0, budget_s=12.0):
    """Oracle (as it stands) on a bounded sample of rays: ray-cell steps/s."""
    import oracle
    o = oracle.Oracle(sc)
    steps, t_used, done = 0, 0.0, 0
    chunk = 256
    while t_used < budget_s and done < len(lv):
        sl = slice(done, done + chunk)
        t = time.perf_counter()
        _, _, st = o.trace(view, n0, lv[sl], ii[sl], jj[sl])
        t_used += time.perf_counter() - t
        steps += int(st.sum())
        done += len(st)
    return steps / t_used, done, t_used


def omp_threads():
    v = os.environ.get("OMP_NUM_THREADS")
    return int(v) if v and v.isdigit() else (os.cpu_count() or 1)


def finest_sample(n, seed=1):
    W = WORKLOAD
    nf = W["base_res"] << W["max_level"]
    rng = np.random.default_rng(seed)
    return (np.full(n, W["max_level"], np.int32), rng.integers(0, nf, n).astype(np.int32),
            rng.integers(0, nf, n).astype(np.int32))


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    W = WORKLOAD
    sc = scenes.cone_shock_amr(W["seed"], n_base=W["n_base"], brick=W["brick"], levels=W["levels"])
    view = scenes.axis_view("+z")
    import oracle
    o = oracle.Oracle(sc)
    per_step = 600
    lv, ii, jj = finest_sample(per_step * (args.steps + args.warmup), seed=7)
    times, steps = [], 0
    for s in range(args.warmup + args.steps):
        sl = slice(s * per_step, (s + 1) * per_step)
        t = time.perf_counter()
        _, _, st = o.trace(view, W["base_res"], lv[sl], ii[sl], jj[sl])
        dt = time.perf_counter() - t
        if s >= args.warmup:
            times.append(dt)
            steps += int(st.sum())
    tot = sum(times)
    val = steps / tot
    sample = (f"{per_step} rays per step drawn uniformly from the 4096^2 finest pixels of the "
              f"same view and grid; FP64 oracle, OpenMP over rays")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {k: v for k, v in W.items()},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="one adaptive image of the workload after --warmup images, then exit "
                         "(the case profiled with ncu)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    assert args.warmup >= 3 or args.profile_case, "at least 3 warm-up steps"

    import torch
    import torch.distributed as dist
    import paper_1010_5534_gb300 as air

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    air.build()

    W = WORKLOAD
    t0 = time.perf_counter()
    sc = scenes.cone_shock_amr(W["seed"], n_base=W["n_base"], brick=W["brick"], levels=W["levels"])
    gen_s = time.perf_counter() - t0
    view = scenes.axis_view("+z")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = air.Grid(sc)
    torch.cuda.synchronize()
    load_s = time.perf_counter() - t0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def render(mem="device", cap=None):
        return g.render_adaptive(view, W["base_res"], W["max_level"], W["xi_crit"], mem=mem,
                                 capacity=cap)

    if args.profile_case:
        for _ in range(args.warmup + 1):
            r = render()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "air", "rays": r["n_rays"], "steps": r["n_steps"],
                          "sweeps": r["n_sweeps"]}), flush=True)
        return
    r = render()
    cap = r["n_out"]
    for _ in range(args.warmup):
        render(cap=cap)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed: device-resident outputs
    st = torch.cuda.current_stream()
    clk_path = os.path.join(ROOT, "gpurun_out", f"clocks_rank{rank}.csv") \
        if os.path.isdir(os.path.join(ROOT, "gpurun_out")) else f"/tmp/air_clocks_{os.getpid()}.csv"
    proc, fh = sample_clocks_start(clk_path)
    g.profile(True)
    barrier()
    step_ms, n_steps, n_rays = [], 0, 0
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        r = render(cap=cap)
        e1.record(st)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        n_steps += r["n_steps"]
        n_rays += r["n_rays"]
    barrier()
    prof = g.profile_read()
    g.profile(False)
    clocks = sample_clocks_stop(proc, fh, clk_path)
    tot_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([tot_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        tot_ms = float(t.item())
        s = torch.tensor([n_steps], device="cuda", dtype=torch.float64)
        dist.all_reduce(s)
        total_steps = float(s.item())
    else:
        total_steps = float(n_steps)
    value = total_steps / (tot_ms * 1e-3)

    # ---- end to end: host (pinned) outputs through the C ABI
    e2e_ms, e2e_steps, d2h = [], 0, 0
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rh = render(mem="host", cap=cap)
        e1.record(st)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        e2e_steps += rh["n_steps"]
        n = rh["n_out"]
        d2h = n * (4 + 4 + 4 + 1 + 4 + 4 * g.n_bands + 4) + 8 * g.n_bands
    e2e_val = e2e_steps / (sum(e2e_ms) * 1e-3)
    if world > 1:
        t = torch.tensor([e2e_val], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        e2e_val = float(t.item()) * world

    # ---- the fixed-resolution comparison arm (same grid, 4096^2)
    f = g.render_fixed(view, W["fixed_res"], fields=("band_flux",))
    fixed_ms = []
    for _ in range(2):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        f = g.render_fixed(view, W["fixed_res"], fields=("band_flux",))
        e1.record(st)
        e1.synchronize()
        fixed_ms.append(e0.elapsed_time(e1))
    air_flux = float(r["band_flux"][0])
    fix_flux = float(f["band_flux"][0])
    flux_err = abs(air_flux - fix_flux) / abs(fix_flux)

    # ---- roofline of the dominant kernel (the march)
    march_ms, march_launches = prof["march"]
    per_step_steps = n_steps / args.steps
    algo_bytes_per_launch = BYTES_PER_STEP * n_steps / max(march_launches, 1)
    achieved = BYTES_PER_STEP * n_steps / (march_ms * 1e-3) / 1e9
    peaks = {}
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(pk_path):
        peaks = json.load(open(pk_path))
    hbm = peaks.get("hbm_gbs", 6800.0)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s",
                "kernel": "k_march (AMR)", "algorithmic_bytes_per_launch": algo_bytes_per_launch,
                "march_share_of_step": march_ms / tot_ms if world == 1 else None}

    gpu_launches = sum(v[1] for v in prof.values())

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        lv, ii, jj = finest_sample(20000, seed=7)
        rate, nr, secs = oracle_sample_rate(sc, view, lv, ii, jj, W["base_res"], budget_s=12.0)
        cpu = {"value": rate, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
               "sample": f"{nr} rays drawn uniformly from the 4096^2 finest pixels of the same "
                         f"view and grid ({secs:.1f} s of CPU time)"}

    if rank == 0:
        cfg = {k: v for k, v in W.items()}
        cfg.update(
            images_per_s=1e3 / (tot_ms / args.steps),
            air_rays_per_image=n_rays // args.steps, air_leaves=int(r["n_leaves"]),
            air_sweeps=int(r["n_sweeps"]), steps_per_image=int(per_step_steps),
            fixed_ms=min(fixed_ms), fixed_rays=W["fixed_res"] ** 2,
            air_speedup_vs_fixed=min(fixed_ms) / (tot_ms / args.steps),
            pixel_saving_vs_fixed=W["fixed_res"] ** 2 / (n_rays / args.steps),
            flux_rel_err_vs_fixed=flux_err,
            phase_ms_per_image={k: v[0] / args.steps for k, v in prof.items()},
            grid_cells=int(sc.n_cells), grid_bricks=int(len(sc.brick_level)),
            grid_upload_s=load_s, scene_gen_s=gen_s,
            l2="flushed before every timed step (256 MiB write)",
            parallelism=f"replicas x{world}" if world > 1 else "single GPU")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic", "config": cfg, "roofline": roofline, "cpu_baseline": cpu,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 112,
                        "d2h_bytes_per_step": int(d2h),
                        "ms_per_step": sum(e2e_ms) / args.steps},
                "gpu_launches": int(gpu_launches), "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
