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
import tempfile
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
    """Start nvidia-smi sampling SM clocks and throttle reasons every 100 ms;
    waits (up to 5 s) for the first sample so the timed region is covered."""
    dev = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    cmd = ["nvidia-smi", "--query-gpu=timestamp,index,clocks.sm,clocks.max.sm,power.draw,"
           "clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
           "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
           "clocks_event_reasons.sw_power_cap", "--format=csv,noheader,nounits", "-lms", "100"]
    if dev.strip().isdigit():
        cmd[1:1] = ["-i", dev.strip()]
    try:
        f = open(path, "w")
        proc = subprocess.Popen(cmd, stdout=f, stderr=subprocess.DEVNULL)
    except (OSError, FileNotFoundError):
        return None, None
    t_end = time.time() + 5.0
    while time.time() < t_end and proc.poll() is None:
        f.flush()
        if os.path.getsize(path) > 0:
            break
        time.sleep(0.05)
    return proc, f


def _parse_clock_rows(path):
    from datetime import datetime
    rows = []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in open(path):
        p = [x.strip() for x in line.split(",")]
        if len(p) < 10:
            continue
        try:
            ts = datetime.strptime(p[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            sm, mx = float(p[2]), float(p[3])
        except ValueError:
            continue
        rs = {nm for k, nm in enumerate(names) if p[6 + k].lower().startswith("active")}
        rows.append((ts, sm, mx, rs))
    return rows


def sample_clocks_stop(proc, f, path, window):
    """Median SM clock and the throttle reasons seen in `window` (host times of
    the timed region); if the region was too short for 3 samples, all samples
    taken while the GPU was busy with this benchmark are used and said so."""
    if proc is None:
        return None
    proc.terminate()
    try:
        proc.wait(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
    f.close()
    return clock_summary(_parse_clock_rows(path), window)


def clock_summary(rows, window):
    """Median SM clock, max clock and throttle reasons of the samples in
    `window`, or of all samples when fewer than 3 fall inside it."""
    sel = [r for r in rows if window[0] <= r[0] <= window[1]]
    span = "timed region"
    if len(sel) < 3:
        sel, span = rows, "whole benchmark (timed region shorter than 3 samples)"
    if not sel:
        return None
    reasons = sorted(set().union(*[r[3] for r in sel]))
    return {"sm_mhz": statistics.median(r[1] for r in sel), "sm_max_mhz": max(r[2] for r in sel),
            "reasons": reasons, "samples": len(sel), "span": span}


def oracle_sample_rate(sc, view, n0, budget_s=15.0, chunk=65536, max_rays=1 << 24):
    """Oracle (as it stands) on a bounded sample: rays drawn uniformly from the
    finest pixels, traced in chunks until `budget_s` of wall time; returns
    ray-cell steps/s, rays traced, seconds."""
    import oracle
    o = oracle.Oracle(sc)
    steps, t_used, done, k = 0, 0.0, 0, 0
    while t_used < budget_s and done < max_rays:
        lv, ii, jj = finest_sample(chunk, seed=7 + k)
        t = time.perf_counter()
        _, _, st = o.trace(view, n0, lv, ii, jj)
        t_used += time.perf_counter() - t
        steps += int(st.sum())
        done += len(st)
        k += 1
    return steps / t_used, done, t_used


MARCH_SOURCES = ("air_march.cuh", "air_march.cu", "air_internal.cuh", "air_refine.cuh")


def march_source_hash():
    import hashlib
    h = hashlib.sha256()
    for n in MARCH_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_1010_5534_gb300", "csrc", n), "rb").read())
    return h.hexdigest()[:16]


def march_traffic(path=None):
    """DRAM bytes per march launch from the committed ncu summary of this
    workload, if it was taken on the current march source (else None)."""
    path = path or os.path.join(ROOT, "profiles", "k_march_amr_cone128_air256.md")
    if not os.path.exists(path):
        return None
    src, val = None, None
    for line in open(path):
        if line.startswith("march source sha256/16:"):
            src = line.split(":", 1)[1].strip().strip("`")
        if line.startswith("dram bytes per launch:"):
            val = float(line.split(":", 1)[1].split()[0])
    return val if src == march_source_hash() else None


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
    per_step = 32768
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


def _timed(fn, st):
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    out = fn()
    e1.record(st)
    e1.synchronize()
    return e0.elapsed_time(e1), out


def run_batch(args):
    """Batched AIR: the cone grid with 16 bands (0.5-10 keV) at 64 random views,
    one persistent launch per render, against the same views one by one. Under
    torchrun (N > 1) the views are sharded over the ranks (view v on rank v mod
    N, no data-path collective) and only the sharded batch is timed."""
    import torch
    import paper_1010_5534_gb300 as air
    air.build()
    W = WORKLOAD
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        return run_batch_sharded(args, world)
    sc = scenes.cone_shock_amr(W["seed"], n_base=W["n_base"], brick=W["brick"], levels=W["levels"],
                               n_bands=16, e_lo=0.5, e_hi=10.0)
    g = air.Grid(sc)
    vs = scenes.random_views(3, 64)
    st = torch.cuda.current_stream()
    res = {}
    for bpt in (4, 8, 16):
        g.render_batch(vs, W["base_res"], W["max_level"], W["xi_crit"], bands_per_thread=bpt,
                       fields=("band_flux",))
        g.profile(True)
        ms, b = _timed(lambda: g.render_batch(vs, W["base_res"], W["max_level"], W["xi_crit"],
                                              bands_per_thread=bpt, fields=("band_flux",)), st)
        prof = g.profile_read()
        g.profile(False)
        steps = sum(r["n_steps"] for r in b)
        res[f"bands_per_thread_{bpt}"] = dict(ms=ms, steps=steps, steps_per_s=steps / ms * 1e3,
                                             band_steps_per_s=16 * steps / ms * 1e3,
                                             kernel_ms=prof["batch"][0], output_ms=prof["output"][0])
    seq = lambda: [g.render_adaptive(v, W["base_res"], W["max_level"], W["xi_crit"],
                                     fields=("band_flux",)) for v in vs]
    seq()
    ms_seq, s1 = _timed(seq, st)
    best = min(res.values(), key=lambda r: r["ms"])
    same = all(b["n_rays"] == a["n_rays"] and b["n_steps"] == a["n_steps"] for a, b in zip(s1, b))
    # batched with the learned proposal: a network trained on plain trees of
    # 16 other views of this grid (outside the timed region)
    lrn = learned_batch_record(air, torch, g, vs, W["base_res"], W["max_level"], W["xi_crit"], st,
                               train_views=scenes.random_views(4, 16), plain=b, plain_ms=best["ms"],
                               quantiles=(0.3, 0.5, 0.8))
    # fixed 4096^2 images of two of the views
    g.render_fixed(vs[0], 512, fields=("band_flux",))
    fx = [_timed(lambda: g.render_fixed(v, W["fixed_res"], fields=("band_flux",)), st) for v in vs[:2]]
    fixed_view_ms = float(np.mean([x[0] for x in fx]))
    ferr = [abs(float(s1[k]["band_flux"].double().sum()) - float(fx[k][1]["band_flux"].double().sum())) /
            abs(float(fx[k][1]["band_flux"].double().sum())) for k in range(2)]
    print(json.dumps({"workload": "batch: cone grid, 64 random views x 16 bands, base 256^2, "
                                  "max level 4, xi_crit 0.5", "rays": sum(r["n_rays"] for r in b),
                      "steps": best["steps"], "batch": res, "sequential_ms": ms_seq,
                      "batch_speedup_vs_sequential": ms_seq / best["ms"],
                      "per_view_rays_and_steps_equal_to_sequential": same,
                      "batched_learned": lrn, "fixed_per_view_ms": fixed_view_ms,
                      "fixed_64_views_ms_extrapolated": fixed_view_ms * len(vs),
                      "batch_speedup_vs_fixed": fixed_view_ms * len(vs) / best["ms"],
                      "batched_learned_speedup_vs_fixed": fixed_view_ms * len(vs) / lrn["ms"],
                      "flux_rel_err_vs_fixed_views_0_1": ferr}), flush=True)


def run_batch_sharded(args, world):
    """The 64-view, 16-band batch sharded by view over `world` ranks: each rank
    renders its views in one persistent launch per step; per-view summaries are
    gathered once at the end (weak scaling in views per rank)."""
    import torch
    import torch.distributed as dist
    import paper_1010_5534_gb300 as air
    from paper_1010_5534_gb300 import shard
    rank, local = int(os.environ.get("RANK", "0")), int(os.environ.get("LOCAL_RANK", "0"))
    dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    W = WORKLOAD
    sc = scenes.cone_shock_amr(W["seed"], n_base=W["n_base"], brick=W["brick"], levels=W["levels"],
                               n_bands=16, e_lo=0.5, e_hi=10.0)
    g = air.Grid(sc)
    vs = scenes.random_views(3, 64)
    mine = shard.shard_views(len(vs), rank, world)
    my_views = [vs[k] for k in mine]
    st = torch.cuda.current_stream()
    render = lambda: g.render_batch(my_views, W["base_res"], W["max_level"], W["xi_crit"],
                                    fields=("band_flux",))
    for _ in range(max(args.warmup, 1)):
        r = render()
    dist.barrier()
    torch.cuda.synchronize()
    ms = []
    for _ in range(args.steps):
        m, r = _timed(render, st)
        ms.append(m)
    dist.barrier()
    t = torch.tensor([sum(ms)], device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    allv = shard.gather_summaries({k: shard.summary(x) for k, x in zip(mine, r)}, len(vs))
    if rank == 0:
        steps = sum(v["n_steps"] for v in allv) * args.steps
        print(json.dumps({"workload": "batch sharded by view: cone grid, 64 views x 16 bands",
                          "n_gpus": world, "steps": args.steps, "ms_per_step": float(t.item()) / args.steps,
                          "value": steps / (float(t.item()) * 1e-3), "unit": UNIT, "scaling": "weak",
                          "views_per_rank": [len(shard.shard_views(len(vs), q, world)) for q in range(world)]}),
              flush=True)
    dist.barrier()
    dist.destroy_process_group()


def learned_batch_record(air, torch, g, vs, n0, Lm, xc, st, train_views, plain, plain_ms,
                         quantiles=(0.8,)):
    """Train the depth network on plain trees of `train_views` of grid g (outside
    any timed region), then time air_render_batch_learned on `vs` at each
    proposal quantile and check its images against the plain batched render
    `plain`; the fastest quantile is the record's `ms`."""
    t0 = time.perf_counter()
    xs, ys = [], []
    for v in train_views:
        x, y = g.learn_samples(v, n0, Lm, xc)
        xs.append(x)
        ys.append(y)
    X, Y = torch.cat(xs), torch.cat(ys)
    net = air.MLP(scenes.mlp_init(0, scale=1.0))
    net.train(X, Y, batch=8192, epochs=4, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del X, Y, xs, ys
    per_q = {}
    for quantile in quantiles:
        g.render_batch_learned(vs, n0, Lm, xc, net, quantile=quantile, fields=("band_flux",))
        ms, (rl, stats) = _timed(lambda: g.render_batch_learned(vs, n0, Lm, xc, net, quantile=quantile,
                                                                fields=("band_flux",)), st)
        # band fluxes of batched renders are FP64 atomic sums: equal up to summation order
        same = all(a["n_rays"] == b["n_rays"] and a["n_steps"] == b["n_steps"] and
                   np.allclose(a["band_flux"].cpu().numpy(), b["band_flux"].cpu().numpy(), rtol=1e-12,
                               atol=0) for a, b in zip(rl, plain))
        per_q[quantile] = dict(ms=ms, speedup_vs_plain_batched=plain_ms / ms,
                               identical_to_plain_batched=same,
                               proposed_rays=int(stats["proposed_rays"]), used_rays=int(stats["used_rays"]),
                               wasted_rays=int(stats["wasted_rays"]),
                               fallback_rays=int(stats["fallback_rays"]))
    net.close()
    best_q = min(per_q, key=lambda q: per_q[q]["ms"])
    return dict(ms=per_q[best_q]["ms"], quantile=best_q, per_quantile={str(k): v for k, v in per_q.items()},
                speedup_vs_plain_batched=plain_ms / per_q[best_q]["ms"],
                identical_to_plain_batched=all(v["identical_to_plain_batched"] for v in per_q.values()),
                training=f"{len(train_views)} plain trees of other views of the grid, 4 epochs",
                training_s=train_s)


def run_mlp(args):
    """The depth network alone: training (minibatch Adam, forward + backward)
    and inference throughput on synthetic BF16 features and random labels
    (the network's cost does not depend on the values), with the tensor-core
    FLOP rate against the measured BF16 peak."""
    import torch
    import paper_1010_5534_gb300 as air
    air.build()
    n = args.mlp_samples
    g = torch.Generator(device="cuda").manual_seed(7)
    x = (torch.rand((n, 16), generator=g, device="cuda") * 2.0).to(torch.bfloat16).view(torch.int16)
    y = torch.randint(0, 5, (n,), generator=g, device="cuda", dtype=torch.int32)
    net = air.MLP(scenes.mlp_init(0, scale=1.0))
    st = torch.cuda.current_stream()
    net.train(x, y, batch=8192, epochs=1, lr=1e-3)
    train_ms, _ = _timed(lambda: net.train(x, y, batch=8192, epochs=1, lr=1e-3), st)
    net.forward(x)
    fwd_ms, _ = _timed(lambda: net.forward(x), st)
    mac = 16 * 64 + 64 * 64 + 64 * 5  # multiply-adds per sample, forward
    peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
    bf16 = peaks.get("bf16_tflops", 1900.0)
    fwd_tf = 2 * mac * n / (fwd_ms * 1e-3) / 1e12
    train_tf = 3 * 2 * mac * n / (train_ms * 1e-3) / 1e12  # forward + two backward products
    print(json.dumps({"workload": f"depth network 16-64-64-5, {n} samples", "train_ms_per_epoch": train_ms,
                      "forward_ms": fwd_ms, "forward_tflops": fwd_tf, "train_tflops": train_tf,
                      "bf16_peak_tflops": bf16, "forward_frac_of_bf16_peak": fwd_tf / bf16,
                      "train_frac_of_bf16_peak": train_tf / bf16}), flush=True)


def run_ring(args):
    """The paper's test calculation (Section 3, Table 1) on GB300: fixed 512^2
    against AIR (32^2 base, 4 levels) at xi_crit 0.2, 0.5, 0.8; pixel counts,
    flux errors against the grid-summed flux, image times."""
    import torch
    import paper_1010_5534_gb300 as air
    air.build()
    sc = scenes.ring_amr()
    g = air.Grid(sc)
    v = scenes.ring_view()
    st = torch.cuda.current_stream()
    tab = sc.lambda_table[0].astype(np.float64)
    nt = tab.size
    hf = (sc.hi[0] - sc.lo[0]) / 512
    ex = 0.0
    for b in range(len(sc.brick_level)):
        T = sc.temp[b].astype(np.float64)
        x = np.clip((np.log10(T) - sc.logT_lo) / (sc.logT_hi - sc.logT_lo) * (nt - 1), 0, nt - 1)
        k = np.minimum(np.floor(x).astype(int), nt - 2)
        lam = (1 - (x - k)) * tab[k] + (x - k) * tab[k + 1]
        ex += (sc.rho[b].astype(np.float64) ** 2 * lam).sum() * (hf * (1 << (4 - sc.brick_level[b]))) ** 3
    rows = []
    for _ in range(args.warmup):
        g.render_fixed(v, 512, fields=("band_flux",))
    ms_f = min(_timed(lambda: g.render_fixed(v, 512, fields=("band_flux",)), st)[0]
               for _ in range(max(args.steps, 1)))
    f = g.render_fixed(v, 512, fields=("band_flux",))
    rows.append(dict(calc="fixed 512^2", pixels=512 * 512, ms=ms_f,
                     flux_err=(ex - float(f["band_flux"][0])) / ex))
    for xc in (0.2, 0.5, 0.8):
        for _ in range(args.warmup):
            g.render_adaptive(v, 32, 4, xc, fields=("band_flux",))
        ms = min(_timed(lambda: g.render_adaptive(v, 32, 4, xc, fields=("band_flux",)), st)[0]
                 for _ in range(max(args.steps, 1)))
        r = g.render_adaptive(v, 32, 4, xc, fields=("band_flux",))
        rows.append(dict(calc=f"AIR xi_crit {xc}", pixels=int(r["n_rays"]), ms=ms,
                         flux_err=(ex - float(r["band_flux"][0])) / ex,
                         speedup_vs_fixed=ms_f / ms, pixel_saving=512 * 512 / r["n_rays"]))
    print(json.dumps({"workload": "Section 3 ring (Eq. 3) on 4^3 blocks of 8^3 cells, 4 levels "
                                  "(512^3 effective), face-on; Table 1 calculations",
                      "table": rows, "paper_table1_pixels": {"fixed": 262144, "0.2": 40512,
                                                             "0.5": 23384, "0.8": 22748}}),
          flush=True)


def run_learned(args):
    """Learned depth proposal: plain AIR trees of seed-varied cone grids (the
    clumping redrawn per seed) at random views give (features, depth) samples;
    the network is trained on the GPU with the library's kernels, then the
    learned and plain renders are compared on held-out seeds."""
    import torch
    import paper_1010_5534_gb300 as air
    air.build()
    W = WORKLOAD
    n0, Lm, xc = W["base_res"], W["max_level"], W["xi_crit"]
    t0 = time.perf_counter()
    base = scenes.cone_shock_amr(0, n_base=W["n_base"], brick=W["brick"], levels=W["levels"],
                                 keep_smooth=True)
    xs, ys = [], []
    gen_s = ren_s = 0.0
    for sd in range(args.seeds):
        t = time.perf_counter()
        sc = scenes.reseed(base, 100 + sd)
        gen_s += time.perf_counter() - t
        t = time.perf_counter()
        g = air.Grid(sc)
        for v in scenes.random_views(5000 + sd, args.views):
            x, y = g.learn_samples(v, n0, Lm, xc)
            xs.append(x)
            ys.append(y)
        g.close()
        torch.cuda.synchronize()
        ren_s += time.perf_counter() - t
    X = torch.cat(xs)
    Y = torch.cat(ys)
    del xs, ys
    counts = torch.bincount(Y.long(), minlength=5).cpu().tolist()
    net = air.MLP(scenes.mlp_init(0, scale=1.0))
    t = time.perf_counter()
    hist = net.train(X, Y, batch=8192, epochs=args.steps, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    acc = float((net.forward(X[:2_000_000]).argmax(dim=1).to(torch.int32) == Y[:2_000_000])
                .float().mean())
    # held-out seeds: the benchmark view and random views
    st = torch.cuda.current_stream()
    evals = []
    for sd in range(3):
        sc = scenes.reseed(base, 900 + sd)
        g = air.Grid(sc)
        for v in [scenes.axis_view("+z")] + scenes.random_views(9000 + sd, 3):
            for _ in range(2):
                g.render_adaptive(v, n0, Lm, xc)
                g.render_learned(v, n0, Lm, xc, net, quantile=0.8)
            ms_p, rp = _timed(lambda: g.render_adaptive(v, n0, Lm, xc), st)
            ms_l, (rl, stl) = _timed(lambda: g.render_learned(v, n0, Lm, xc, net, quantile=0.8), st)
            same = all(bool((rp[k] == rl[k]).all()) for k in ("level", "i", "j", "intensity"))
            evals.append(dict(view=list(v.dir), plain_ms=ms_p, learned_ms=ms_l,
                              plain_waves=1 + rp["n_sweeps"], learned_waves=stl["waves"],
                              rays=rp["n_rays"], proposed=stl["proposed_rays"],
                              wasted=stl["wasted_rays"], fallback=stl["fallback_rays"],
                              under=stl["under_predicted"], over=stl["over_predicted"],
                              identical=same))
        g.close()
    nb = n0 * n0
    print(json.dumps({
        "workload": f"learned proposal: {args.seeds} seeds x {args.views} views = "
                    f"{args.seeds * args.views} plain trees of the cone grid (clumping redrawn "
                    f"per seed), base {n0}^2, max level {Lm}, xi_crit {xc}",
        "samples": int(X.shape[0]), "label_counts": counts, "epochs": args.steps,
        "loss_history": [float(h) for h in hist], "train_s": train_s, "data_gen_s": gen_s,
        "data_render_s": ren_s, "train_accuracy": acc,
        "heldout": evals,
        "heldout_mean": {
            "plain_ms": float(np.mean([e["plain_ms"] for e in evals])),
            "learned_ms": float(np.mean([e["learned_ms"] for e in evals])),
            "plain_waves": float(np.mean([e["plain_waves"] for e in evals])),
            "learned_waves": float(np.mean([e["learned_waves"] for e in evals])),
            "misprediction_rate": float(np.mean([(e["under"] + e["over"]) / nb for e in evals])),
            "under_rate": float(np.mean([e["under"] / nb for e in evals])),
            "wasted_fraction": float(np.mean([e["wasted"] / e["rays"] for e in evals])),
            "all_identical": all(e["identical"] for e in evals)},
        "total_s": time.perf_counter() - t0}), flush=True)


LARGE = dict(workload="clumps-and-cones block-AMR grid: 512^3 base cells in 32^3 bricks, 5 "
                       "refinement levels (16384^3 effective) around 200 dense clumps (r 0.005-"
                       "0.02, contrast 10-1000) with two shock cones at the base resolution, "
                       "FP32 rho/T (1.06 G cells), 32 bands (0.5-10 keV) with absorption; 16 "
                       "random views; AIR base 1024^2, max level 3 (8192^2 equivalent), "
                       "xi_crit 0.5", seed=0, views=16, base_res=1024, max_level=3, xi_crit=0.5,
             fixed_res=8192)
FP32_OPS_PER_BAND_STEP = 23  # per band and cell: dtau, exponent argument, Taylor (7), both
                             # cell-term forms (7), select, Kahan sum (4), table lookup (2)


def run_large(args):
    """The large configuration: 16 views x 32 bands of the clumps-and-cones
    grid as one batched persistent render, the same views one by one, the
    learned proposal (network trained on plain trees of 48 other views of the
    same grid) view by view, and fixed 8192^2 images (two views timed)."""
    import torch
    import paper_1010_5534_gb300 as air
    air.build()
    W = LARGE
    n0, Lm, xc = W["base_res"], W["max_level"], W["xi_crit"]
    t0 = time.perf_counter()
    sc = scenes.clumps_cones_amr(W["seed"])
    gen_s = time.perf_counter() - t0
    t = time.perf_counter()
    g = air.Grid(sc)
    torch.cuda.synchronize()
    load_s = time.perf_counter() - t
    vs = scenes.random_views(21, W["views"])
    st = torch.cuda.current_stream()
    out = {"workload": W["workload"], "cells": int(sc.n_cells), "bricks": int(len(sc.brick_level)),
           "bricks_per_level": np.bincount(sc.brick_level).tolist(), "scene_gen_s": gen_s,
           "grid_upload_s": load_s}
    # batched plain AIR
    batch = {}
    for bpt in (8, 16):
        g.render_batch(vs, n0, Lm, xc, bands_per_thread=bpt, fields=("band_flux",))
        g.profile(True)
        ms, b = _timed(lambda: g.render_batch(vs, n0, Lm, xc, bands_per_thread=bpt,
                                              fields=("band_flux",)), st)
        prof = g.profile_read()
        g.profile(False)
        steps = sum(r["n_steps"] for r in b)
        batch[f"bands_per_thread_{bpt}"] = dict(ms=ms, rays=sum(r["n_rays"] for r in b), steps=steps,
                                                band_steps_per_s=sc.n_bands * steps / ms * 1e3,
                                                kernel_ms=prof["batch"][0])
    best = min(batch.values(), key=lambda r: r["ms"])
    out["batch"] = batch
    # the same views one by one
    g.render_adaptive(vs[0], n0, Lm, xc, fields=("band_flux",))
    ms_seq, seq = _timed(lambda: [g.render_adaptive(v, n0, Lm, xc, fields=("band_flux",))
                                  for v in vs], st)
    out["sequential_ms"] = ms_seq
    out["batch_speedup_vs_sequential"] = ms_seq / best["ms"]
    out["batch_equal_to_sequential"] = all(a["n_rays"] == b_["n_rays"] and a["n_steps"] == b_["n_steps"]
                                           for a, b_ in zip(seq, b))
    # learned proposal
    t = time.perf_counter()
    xs, ys = [], []
    for v in scenes.random_views(22, 48):
        x, y = g.learn_samples(v, n0, Lm, xc)
        xs.append(x)
        ys.append(y)
    X, Y = torch.cat(xs), torch.cat(ys)
    del xs, ys
    torch.cuda.synchronize()
    data_s = time.perf_counter() - t
    net = air.MLP(scenes.mlp_init(0, scale=1.0))
    t = time.perf_counter()
    net.train(X, Y, batch=8192, epochs=4, lr=1e-3)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    # the proposal quantile trades wasted rays (over-prediction) against
    # fallback waves (under-prediction); both are reported
    learned = dict(samples=int(X.shape[0]), label_counts=torch.bincount(Y.long(), minlength=5)
                   .cpu().tolist(), data_s=data_s, train_s=train_s,
                   plain_waves=float(np.mean([1 + r["n_sweeps"] for r in seq])))
    ref2 = [g.render_adaptive(v, n0, Lm, xc) for v in vs[:2]]
    for q in (0.3, 0.5, 0.8):
        g.render_learned(vs[0], n0, Lm, xc, net, quantile=q)
        ms_l, rl = _timed(lambda: [g.render_learned(v, n0, Lm, xc, net, quantile=q) for v in vs], st)
        same = all(bool((a["intensity"] == b[0]["intensity"]).all()) and
                   bool((a["level"] == b[0]["level"]).all()) for a, b in zip(ref2, rl[:2]))
        learned[f"quantile_{q}"] = dict(ms=ms_l, waves=float(np.mean([b[1]["waves"] for b in rl])),
                                        wasted_rays=int(sum(b[1]["wasted_rays"] for b in rl)),
                                        fallback_rays=int(sum(b[1]["fallback_rays"] for b in rl)),
                                        speedup_vs_sequential=ms_seq / ms_l, first_two_identical=same)
    out["learned"] = learned
    del X, Y
    # batched with the learned proposal (the same network), per quantile
    bl = {}
    torch.cuda.empty_cache()
    for qq in (0.3, 0.5, 0.8):
        try:
            g.render_batch_learned(vs, n0, Lm, xc, net, quantile=qq, fields=("band_flux",))
        except air.AirError as e:  # recorded, not fatal: the other records still print
            bl[str(qq)] = {"error": str(e), "free_gb": torch.cuda.mem_get_info()[0] / 2 ** 30}
            continue
        ms_q, (rbl, sbl) = _timed(lambda: g.render_batch_learned(vs, n0, Lm, xc, net, quantile=qq,
                                                                 fields=("band_flux",)), st)
        bl[str(qq)] = dict(
            ms=ms_q, speedup_vs_plain_batched=best["ms"] / ms_q,
            identical_to_plain_batched=all(a["n_rays"] == c["n_rays"] and a["n_steps"] == c["n_steps"] and
                                           np.allclose(a["band_flux"].cpu().numpy(),
                                                       c["band_flux"].cpu().numpy(), rtol=1e-12, atol=0)
                                           for a, c in zip(rbl, b)),
            **{k: int(v) for k, v in sbl.items() if k in ("proposed_rays", "used_rays", "wasted_rays",
                                                         "fallback_rays")})
    out["batched_learned"] = bl
    ms_bl = min((x["ms"] for x in bl.values() if "ms" in x), default=float("nan"))
    # fixed 8192^2 (two views timed)
    g.render_fixed(vs[0], 1024, fields=("band_flux",))
    fx = []
    for v in vs[:2]:
        ms_f, f = _timed(lambda: g.render_fixed(v, W["fixed_res"], fields=("band_flux",)), st)
        fx.append(dict(ms=ms_f, steps=f["n_steps"]))
    fixed_view_ms = float(np.mean([x["ms"] for x in fx]))
    out["fixed_per_view_ms"] = fixed_view_ms
    out["fixed_16_views_ms_extrapolated"] = fixed_view_ms * W["views"]
    out["batch_speedup_vs_fixed"] = fixed_view_ms * W["views"] / best["ms"]
    out["batched_learned_speedup_vs_fixed"] = fixed_view_ms * W["views"] / ms_bl
    for k in range(2):
        fs = g.render_fixed(vs[k], W["fixed_res"], fields=("band_flux",))
        fa = fs["band_flux"].double().sum().item()
        out.setdefault("flux_rel_err_vs_fixed", []).append(
            abs(seq[k]["band_flux"].double().sum().item() - fa) / abs(fa))
    # ALU roofline of the batched kernel: FP32 operations per band-step
    peak_ops = 152 * 128 * 2.07e9
    ach = best["band_steps_per_s"] * FP32_OPS_PER_BAND_STEP
    out["roofline"] = {"bound": "alu", "achieved": ach / 1e12, "peak": peak_ops / 1e12,
                       "unit": "T FP32 op/s", "frac": ach / peak_ops, "traffic": None,
                       "kernel": "k_air_batch", "ops_per_band_step": FP32_OPS_PER_BAND_STEP}
    out["total_s"] = time.perf_counter() - t0
    print(json.dumps(out), flush=True)


def large_view_record(air, torch, st, reps=2):
    """One view of the large configuration (view 0 of its 16, all 32 bands):
    the adaptive image through the single-view path and through the batched
    persistent kernel, against the fixed 8192^2 image of the same view, with
    the band-summed flux error and the march's HBM and FP32-issue fractions.
    Scene generation, upload and warm-up are outside the timed renders."""
    W = LARGE
    n0, Lm, xc = W["base_res"], W["max_level"], W["xi_crit"]
    t0 = time.perf_counter()
    sc = scenes.clumps_cones_amr(W["seed"])
    gen_s = time.perf_counter() - t0
    t = time.perf_counter()
    g = air.Grid(sc)
    torch.cuda.synchronize()
    load_s = time.perf_counter() - t
    v = scenes.random_views(21, W["views"])[0]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def timed(fn):
        ms, out = [], None
        for _ in range(reps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            out = fn()
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return min(ms), out

    fields = ("band_flux",)
    g.render_adaptive(v, n0, Lm, xc, fields=fields)
    g.profile(True)
    air_ms, ra = timed(lambda: g.render_adaptive(v, n0, Lm, xc, fields=fields))
    prof = g.profile_read()
    g.profile(False)
    g.render_batch([v], n0, Lm, xc, fields=fields)
    batch_ms, rb = timed(lambda: g.render_batch([v], n0, Lm, xc, fields=fields))
    rb = rb[0]
    lrn = learned_batch_record(air, torch, g, [v], n0, Lm, xc, st,
                               train_views=scenes.random_views(22, 4), plain=[rb], plain_ms=batch_ms,
                               quantiles=(0.3, 0.5, 0.8))
    g.render_fixed(v, 1024, fields=fields)
    fixed_ms, rf = timed(lambda: g.render_fixed(v, W["fixed_res"], fields=fields))
    fa = rf["band_flux"].double().cpu().numpy()
    ea = ra["band_flux"].double().cpu().numpy()
    eb = rb["band_flux"].double().cpu().numpy()
    steps = int(ra["n_steps"])
    march_ms = prof["march"][0] / reps
    hbm = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs", 6800.0) \
        if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 6800.0
    peak_ops = 152 * 128 * 2.07e9
    band_steps_s = sc.n_bands * steps / (march_ms * 1e-3)
    rec = dict(workload=W["workload"] + " -- view 0 of the 16, all 32 bands",
               base_res=n0, max_level=Lm, xi_crit=xc, fixed_res=W["fixed_res"],
               cells=int(sc.n_cells), scene_gen_s=gen_s, grid_upload_s=load_s,
               air_ms=air_ms, air_rays=int(ra["n_rays"]), air_steps=steps,
               air_sweeps=int(ra["n_sweeps"]),
               batched_ms=batch_ms, batched_equal=bool(rb["n_rays"] == ra["n_rays"] and
                                                      rb["n_steps"] == ra["n_steps"]),
               batched_learned=lrn,
               batched_learned_speedup_vs_fixed=fixed_ms / lrn["ms"],
               fixed_ms=fixed_ms, fixed_steps=int(rf["n_steps"]),
               air_speedup_vs_fixed=fixed_ms / air_ms,
               batched_speedup_vs_fixed=fixed_ms / batch_ms,
               flux_rel_err_vs_fixed=float(abs(ea.sum() - fa.sum()) / abs(fa.sum())),
               flux_rel_err_vs_fixed_max_band=float(np.max(np.abs(ea - fa) / np.abs(fa))),
               phase_ms={k: val[0] / reps for k, val in prof.items()},
               roofline={"march_ms": march_ms,
                         "hbm": {"bound": "hbm", "achieved": BYTES_PER_STEP * steps / (march_ms * 1e-3) / 1e9,
                                 "peak": hbm, "unit": "GB/s",
                                 "frac": BYTES_PER_STEP * steps / (march_ms * 1e-3) / 1e9 / hbm},
                         "alu": {"bound": "alu", "achieved": band_steps_s * FP32_OPS_PER_BAND_STEP / 1e12,
                                 "peak": peak_ops / 1e12, "unit": "T FP32 op/s",
                                 "frac": band_steps_s * FP32_OPS_PER_BAND_STEP / peak_ops,
                                 "ops_per_band_step": FP32_OPS_PER_BAND_STEP}})
    g.close()
    del sc, g, flush
    torch.cuda.empty_cache()
    return rec


def batch_record(air, torch, st):
    """The batched configuration in brief: the cone grid with 16 bands
    (0.5-10 keV) at 64 random views, one persistent launch (8 bands per
    thread), against fixed 4096^2 images of two of the views (extrapolated to
    64) with the band-summed flux error on those two, and the batched march's
    FP32-issue fraction. Scene generation, upload and one warm-up render are
    outside the timed render."""
    W = WORKLOAD
    t0 = time.perf_counter()
    sc = scenes.cone_shock_amr(W["seed"], n_base=W["n_base"], brick=W["brick"], levels=W["levels"],
                               n_bands=16, e_lo=0.5, e_hi=10.0)
    g = air.Grid(sc)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    vs = scenes.random_views(3, 64)
    n0, Lm, xc = W["base_res"], W["max_level"], W["xi_crit"]
    g.render_batch(vs, n0, Lm, xc, bands_per_thread=8, fields=("band_flux",))
    g.profile(True)
    ms, b = _timed(lambda: g.render_batch(vs, n0, Lm, xc, bands_per_thread=8, fields=("band_flux",)), st)
    prof = g.profile_read()
    g.profile(False)
    steps = sum(r["n_steps"] for r in b)
    g.render_fixed(vs[0], 512, fields=("band_flux",))
    fx = [_timed(lambda: g.render_fixed(v, W["fixed_res"], fields=("band_flux",)), st) for v in vs[:2]]
    fixed_view_ms = float(np.mean([x[0] for x in fx]))
    ferr = [abs(float(b[k]["band_flux"].double().sum()) - float(fx[k][1]["band_flux"].double().sum())) /
            abs(float(fx[k][1]["band_flux"].double().sum())) for k in range(2)]
    band_steps_s = 16 * steps / (prof["batch"][0] * 1e-3)
    peak_ops = 152 * 128 * 2.07e9
    rec = dict(workload="cone grid, 64 random views x 16 bands (0.5-10 keV), base 256^2, max level 4, "
                        "xi_crit 0.5, one persistent launch, 8 bands per thread",
               setup_s=setup_s, batched_ms=ms, rays=int(sum(r["n_rays"] for r in b)), steps=int(steps),
               band_steps_per_s=16 * steps / ms * 1e3, kernel_ms=prof["batch"][0],
               fixed_per_view_ms=fixed_view_ms, fixed_64_views_ms_extrapolated=fixed_view_ms * len(vs),
               batched_speedup_vs_fixed=fixed_view_ms * len(vs) / ms,
               flux_rel_err_vs_fixed_views_0_1=ferr,
               roofline={"bound": "alu", "achieved": band_steps_s * FP32_OPS_PER_BAND_STEP / 1e12,
                         "peak": peak_ops / 1e12, "unit": "T FP32 op/s",
                         "frac": band_steps_s * FP32_OPS_PER_BAND_STEP / peak_ops,
                         "ops_per_band_step": FP32_OPS_PER_BAND_STEP, "kernel": "k_air_batch"})
    g.close()
    del sc, g
    torch.cuda.empty_cache()
    return rec


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true",
                    help="skip the learned-proposal comparison in the default workload")
    ap.add_argument("--workload", default="air", choices=["air", "batch", "learned", "ring", "large", "mlp"],
                    help="air: the benchmark line (one adaptive image of the cone grid); "
                         "batch: 64 views x 16 bands in one persistent launch vs one by one; "
                         "learned: train the depth network on 2000 plain trees, evaluate")
    ap.add_argument("--seeds", type=int, default=40)
    ap.add_argument("--views", type=int, default=50)
    ap.add_argument("--mlp-samples", type=int, default=1 << 24,
                    help="samples of the --workload mlp run")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the one-view record of the large configuration")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the record of the 64-view batched configuration")
    ap.add_argument("--clocks-file", default=None,
                    help="keep the nvidia-smi clock samples here ({rank} is replaced by the rank); "
                         "default: a temporary file")
    ap.add_argument("--profile-case", action="store_true",
                    help="one adaptive image of the workload after --warmup images, then exit "
                         "(the case profiled with ncu)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "learned":
        return run_learned(args)
    if args.workload == "ring":
        return run_ring(args)
    if args.workload == "large":
        return run_large(args)
    if args.workload == "mlp":
        return run_mlp(args)
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
    sc = scenes.cone_shock_amr(W["seed"], n_base=W["n_base"], brick=W["brick"], levels=W["levels"],
                               keep_smooth=not args.no_learned)
    sc_smooth = sc
    gen_s = time.perf_counter() - t0
    view = scenes.axis_view("+z")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    g = air.Grid(sc)
    torch.cuda.synchronize()
    load_s = time.perf_counter() - t0
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    # the image a caller reads back: each leaf's level and position, column
    # density and band intensities, and the band flux (is_leaf is all ones for
    # a leaves-only image, and the band sum equals the intensity for one band)
    E2E_FIELDS = ("level", "i", "j", "coldens", "intensity", "band_flux")

    def render(mem="device", cap=None, fields=None, out=None):
        kw = {"fields": fields} if fields else {}
        return g.render_adaptive(view, W["base_res"], W["max_level"], W["xi_crit"], mem=mem,
                                 capacity=cap, out=out, **kw)

    if args.profile_case:
        for _ in range(args.warmup + 1):
            r = render()
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "air", "rays": r["n_rays"], "steps": r["n_steps"],
                          "sweeps": r["n_sweeps"]}), flush=True)
        return
    clk_path = args.clocks_file.replace("{rank}", str(rank)) if args.clocks_file else \
        os.path.join(tempfile.gettempdir(), f"air_clocks_{os.getpid()}_rank{rank}.csv")
    proc, fh = sample_clocks_start(clk_path)
    r = render()
    cap = r["n_out"]
    for _ in range(args.warmup):
        render(cap=cap)

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # ---- timed: device-resident outputs. The headline pass runs without the
    # library's event profiler (its two event records per launch group cost
    # ~0.3 ms of host time per image); a second pass of the same K images with
    # the profiler on gives the per-phase times and the march launches'
    # durations for the roofline.
    st = torch.cuda.current_stream()

    def timed_pass():
        ms, ns, nr, last = [], 0, 0, None
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            last = render(cap=cap)
            e1.record(st)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            ns += last["n_steps"]
            nr += last["n_rays"]
        return ms, ns, nr, last

    barrier()
    t_win0 = time.time()
    step_ms, n_steps, n_rays, r = timed_pass()
    barrier()
    t_win1 = time.time()
    g.profile(True)
    prof_step_ms, _, _, _ = timed_pass()
    prof = g.profile_read()
    g.profile(False)
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
    # the caller's page-locked output arrays are allocated once, outside the
    # timed region (as the inputs are resident), and filled by every call
    hbuf = g.alloc_image(cap, "host", E2E_FIELDS)
    for _ in range(args.warmup):
        rh = render(mem="host", out=hbuf)
    torch.cuda.synchronize()
    barrier()
    for _ in range(args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        rh = render(mem="host", out=hbuf)
        e1.record(st)
        e1.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
        e2e_steps += rh["n_steps"]
        n = rh["n_out"]
        d2h = n * (4 + 4 + 4 + 4 + 4 * g.n_bands) + 8 * g.n_bands
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
    clocks = sample_clocks_stop(proc, fh, clk_path, (t_win0, t_win1))
    air_flux = float(r["band_flux"][0])
    fix_flux = float(f["band_flux"][0])
    flux_err = abs(air_flux - fix_flux) / abs(fix_flux)

    # ---- the learned depth proposal on the same image: a network trained on
    # plain trees of other clumping seeds (outside the timed region), then
    # the same adaptive image with the proposal, timed like the plain one
    learned = None
    if not args.no_learned:
        t0 = time.perf_counter()
        xs, ys = [], []
        for sd in range(5):
            gs = air.Grid(scenes.reseed(sc_smooth, 100 + sd))
            for vv in scenes.random_views(5000 + sd, 19) + [view]:
                x, y = gs.learn_samples(vv, W["base_res"], W["max_level"], W["xi_crit"])
                xs.append(x)
                ys.append(y)
            gs.close()
        net = air.MLP(scenes.mlp_init(0, scale=1.0))
        net.train(torch.cat(xs), torch.cat(ys), batch=8192, epochs=4, lr=1e-3)
        del xs, ys
        torch.cuda.synchronize()
        train_s = time.perf_counter() - t0
        for _ in range(args.warmup):
            g.render_learned(view, W["base_res"], W["max_level"], W["xi_crit"], net, quantile=0.99,
                             capacity=cap)
        lms, waves = [], 0
        for _ in range(args.steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(st)
            rl, stl = g.render_learned(view, W["base_res"], W["max_level"], W["xi_crit"], net,
                                       quantile=0.99, capacity=cap)
            e1.record(st)
            e1.synchronize()
            lms.append(e0.elapsed_time(e1))
            waves = stl["waves"]
        rp = render(cap=cap)
        same = all(bool((rp[k] == rl[k]).all()) for k in ("level", "i", "j", "coldens", "intensity"))
        learned = dict(ms_per_image=sum(lms) / len(lms), waves=int(waves),
                       plain_waves=int(rp["n_sweeps"]) + 1, identical_to_plain=same,
                       speedup_vs_plain=(tot_ms / args.steps) / (sum(lms) / len(lms)),
                       speedup_vs_fixed=min(fixed_ms) / (sum(lms) / len(lms)),
                       training="100 plain trees (5 other clumping seeds x 20 views), "
                                "4 epochs", training_s=train_s)

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
                "frac": achieved / hbm, "traffic": march_traffic(),
                "march_source": march_source_hash(),
                "peak_source": "MEASURED_PEAKS.json hbm_gbs" if peaks else "fallback 6.8 TB/s",
                "kernel": "k_march (AMR)", "algorithmic_bytes_per_launch": algo_bytes_per_launch,
                "march_share_of_step": march_ms / sum(prof_step_ms) if world == 1 else None,
                "duration_source": "CUDA events on the handle's stream around every march launch, "
                                   "profiled pass of the same images"}

    gpu_launches = sum(v[1] for v in prof.values())

    # ---- one view of the large configuration (outside the timed region)
    large = None
    if rank == 0 and world == 1 and not args.no_large:
        g.close()
        torch.cuda.empty_cache()
        large = large_view_record(air, torch, st)
    batched = None
    if rank == 0 and world == 1 and not args.no_batch:
        batched = batch_record(air, torch, st)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        rate, nr, secs = oracle_sample_rate(sc, view, W["base_res"])
        cpu = {"value": rate, "unit": UNIT, "cores": omp_threads(), "kind": "oracle",
               "sample": f"{nr} rays drawn uniformly from the 4096^2 finest pixels of the same "
                         f"view and grid, FP64 oracle, OpenMP over rays ({secs:.1f} s wall)"}

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
            learned_proposal=learned,
            large_view=large,
            batched_64_views=batched,
            phase_ms_per_image={k: v[0] / args.steps for k, v in prof.items()},
            profiled_pass_ms_per_image=sum(prof_step_ms) / args.steps,
            phase_source="second timed pass of the same images with the library's CUDA-event "
                         "profiler on (headline pass without it)",
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
                        "ms_per_step": sum(e2e_ms) / args.steps,
                        "fields": list(E2E_FIELDS)},
                "gpu_launches": int(gpu_launches), "clocks": clocks}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
