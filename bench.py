#!/usr/bin/env python
"""Benchmark of the InIm cartogram iteration on one GB300 (or N replicas).

Workload (the time-varying configuration): 200 jittered Voronoi regions,
~50k vertices, 1024^2 texture, 24 time steps of log-normal random-walk values,
50 iterations per step, shape parameter swept over {0.25, 0.5, 0.75}, in
direct mode (72 independent solves, one batch) and cumulative mode (3 shape
series, 24 rounds of a 3-solve batch).  One step = that whole sweep =
2 * 3 * 24 * 50 = 7200 InIm iterations.

Printed (one JSON line, rank 0): iterations/s with inputs resident in HBM,
the same through host (pinned) buffers (e2e), the dominant kernel's roofline
from CUDA events on the library's stream, SM clocks sampled during the timed
region, the CPU oracle on a bounded sample (cpu_baseline), the plain
unfused GPU form on a bounded sample, and time-to-epsilon plain vs fused.

--impl reference times the CPU oracle on the same workload and metric (the
reference arm: the paper's own implementation is not available).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

SHAPES = (0.25, 0.5, 0.75)
ITERS = 50
T_STEPS = 24
ITERS_PER_STEP = 2 * len(SHAPES) * T_STEPS * ITERS
METRIC = "InIm iterations/s"
WORKLOAD = "voronoi200_v50k_res1024_T24_it50_shapes3_direct+cumulative"


def whole_job_rate(local_ms, iters_per_rank, world, dist=None, device="cpu"):
    """Replicas: the slowest rank's time (max over ranks) and the whole-job
    rate, every rank's iterations divided by that time."""
    import torch
    t = torch.tensor([float(local_ms)], device=device, dtype=torch.float64)
    if dist is not None and world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    ms_max = float(t.item())
    return ms_max, iters_per_rank * world / (ms_max / 1e3)


def stage_bytes(n_jobs, N, V, R, E, K, nb):
    """Algorithmic bytes per launch of every stage over a batch of n_jobs
    (FP32; per job: P = N^2 pixels, V vertices, R regions, E ring edges, K
    crossing keys, nb bands)."""
    Ppx = N * N
    return {
        "crossings": n_jobs * (8 * E + 8 * V + 4 * K),
        "raster_rows": n_jobs * (4 * K + 2 * Ppx),
        "density_table": n_jobs * (12 * R),
        "scan_phase1": n_jobs * (2 * Ppx + 3 * nb * N * 4),
        "scan_carry": n_jobs * (2 * 3 * nb * N * 4),
        "scan_phase3": n_jobs * (2 * Ppx + 8 * Ppx + 3 * nb * N * 4),
        "gather_move": n_jobs * 48 * V,
        "areas_errors": n_jobs * (8 * E + 8 * V + 8 * R),
        # single pass: labels read once, S and T written, band aggregates and
        # carries written (the look-back's reads of earlier bands stay in L2)
        "scan_fused": n_jobs * (2 * Ppx + 8 * Ppx + 2 * 3 * nb * N * 4),
    }


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from
# ncu captures of `bench.py --ncu-case <batch>` with the kernels and tiles of
# this source; keyed by (batch, stage, band rows, columns per thread, threads).
# The 3-solve batch's textures stay in L2, so its kernels move far fewer DRAM
# bytes than their algorithmic bytes.  Kernels changed since their capture
# have no entry (the crossing keys, the gather, the parallel-rows phase 3).
TRAFFIC = {
    ("chain3", "raster_rows", 8, 0, 256): 0.876e6,
    ("chain3", "scan_phase1", 8, 0, 256): 6.363e6,
    ("chain3", "scan_carry", 8, 0, 256): 4.750e6,
    ("chain3", "areas_errors", 8, 0, 256): 1.988e6,
    ("direct72", "scan_phase1", 64, 4, 256): 161.4e6,
    ("direct72", "scan_phase3", 16, 4, 256): 755.632e6,
    ("direct72", "scan_phase3", 32, 4, 256): 731.673e6,
    ("direct72", "scan_phase3", 64, 4, 256): 718.129e6,
}


def roofline(batches, bn, sn, pk):
    b = batches[bn]
    t = b["tile"]
    achieved = b["algo"][sn] / (b["stages"][sn] / 1e3) / 1e9
    return {"bound": "hbm", "kernel": sn, "batch": bn, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / pk["hbm_gbs"],
            "traffic": TRAFFIC.get((bn, sn, t["band_rows"], t["cols_per_thread"], t["threads"])),
            "algorithmic_bytes_per_launch": b["algo"][sn], "launch_ms": b["stages"][sn],
            "launches_per_step": b["per_step"],
            "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "fallback" not in pk else "fallback"}


def crossings_count(mesh, N):
    """Crossing keys of one raster of the map at its start positions: for
    every ring edge, the texture rows whose pixel centres it spans."""
    y = mesh.verts[:, 1]
    K = 0
    for r in range(len(mesh.ring_off) - 1):
        ids = mesh.ring_idx[mesh.ring_off[r]:mesh.ring_off[r + 1]]
        y0, y1 = y[ids], y[np.roll(ids, -1)]
        lo, hi = np.minimum(y0, y1), np.maximum(y0, y1)
        K += int(np.maximum(np.ceil(hi * N - 0.5) - np.ceil(lo * N - 0.5), 0).sum())
    return K


def _oracle_worker(task):
    """One CPU worker of the all-core baseline: `iters` oracle iterations of
    one solve (its own shape and time step), single-threaded numpy."""
    arrays, verts, values, k, shape, iters = task
    from oracle import inim_oracle as O
    t0 = O.transform_uniform(1 << k)
    xy = verts.astype(np.float64)
    t = time.perf_counter()
    for _ in range(iters):
        xy, _ = O.iterate(xy, arrays, values, k, shape, t0=t0)
    return iters, time.perf_counter() - t


def cpu_all_cores(mesh, values, k, iters_per_worker=3):
    """The oracle on every host core the process may use: one independent solve
    per core (shapes and time steps of the sweep), iterations / wall time."""
    import multiprocessing as mp
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    arrays = (mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)
    tasks = [(arrays, mesh.verts_f32(), values[c % len(values)], k, SHAPES[c % len(SHAPES)], iters_per_worker)
             for c in range(cores)]
    env = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in env:
        os.environ[v] = "1"                        # one thread per worker process
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            pool.map(_oracle_worker, [tasks[0][:5] + (1,)] * cores)      # start-up and imports, untimed
            t = time.perf_counter()
            res = pool.map(_oracle_worker, tasks)
            wall = time.perf_counter() - t
    finally:
        for v, x in env.items():
            if x is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = x
    n = sum(r[0] for r in res)
    return {"value": n / wall, "unit": "iterations/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} independent solves of the 1024^2 map (one per core, the sweep's shapes and "
                      f"time steps), {iters_per_worker} oracle iterations each, {wall:.1f} s wall"}


def quick_warm_start_network(n_maps=1536, epochs=10):
    """A warm-start network trained on the spot (fields the method generates on
    the training maps of the learned part, as in warmstart.py, fewer maps);
    returns (parameter blob, seconds)."""
    from paper_2604_13880_gb300 import warmstart as W
    import paper_2604_13880_gb300 as P
    t = time.perf_counter()
    maps = W.generate_maps(range(50000, 50000 + n_maps), workers=min(16, os.cpu_count() or 1))
    X, Y, _ = W.build_dataset(maps, eps_target=0.05, max_iters=512)
    net, _ = W.train(X, Y, epochs=epochs)
    blob = P.inim_cnn_get_params(net)
    net.close()
    return blob, time.perf_counter() - t


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "fallback": True}


# ---------------------------------------------------------------------------
# clocks sampled during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if "Active" in r[5 + k] and "Not" not in r[5 + k]})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


# ---------------------------------------------------------------------------
# the reference arm: the CPU oracle
# ---------------------------------------------------------------------------
def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from oracle import inim_oracle as O
    from paper_2604_13880_gb300 import synth
    w = synth.time_varying_workload()
    mesh = w["mesh"]
    arrays = (mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)
    t0 = O.transform_uniform(1 << w["log2_res"])
    xy = mesh.verts_f32().astype(np.float64)
    per_step = 2

    def step():
        nonlocal xy
        for _ in range(per_step):
            xy, _ = O.iterate(xy, arrays, w["values"][0], w["log2_res"], 0.5, t0=t0)

    for _ in range(args.warmup):
        step()
    t = time.perf_counter()
    for _ in range(args.steps):
        step()
    dt = time.perf_counter() - t
    value = args.steps * per_step / dt
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": f"{per_step} oracle iterations per step (shape 0.5, t=0)"},
            "cpu_baseline": {"value": value, "unit": "iterations/s", "cores": 1, "kind": "oracle",
                             "sample": f"{per_step} iterations of the 1024^2 map per step"},
            "e2e": {"value": value, "unit": "iterations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# precision study: the 4096^2 workload in the three precisions
# ---------------------------------------------------------------------------
def precision_study(args):
    import torch
    import paper_2604_13880_gb300 as P
    from paper_2604_13880_gb300 import synth
    w = synth.precision_workload()
    mesh = w["mesh"]
    vals = w["values"][0].astype(np.float32)
    m = P.inim_map_create(mesh)
    xy0 = mesh.verts_f32()
    K = args.precision_study
    res = {"workload": w["name"], "iterations": K, "precisions": {}}
    outs = {}
    for name, prec in (("fp32", P.INIM_FP32), ("fix64", P.INIM_FIX64), ("kahan", P.INIM_KAHAN)):
        p = P.params(log2_res=12, shape=0.5, precision=prec)
        x = torch.as_tensor(xy0, device="cuda")
        v = torch.as_tensor(vals, device="cuda")
        # scan tiles of this precision chosen by the autotuner on the job itself
        ja = (P.inim_job * 1)()
        ja[0].map = m.handle
        ja[0].values = v.data_ptr()
        ja[0].init_xy = None
        ja[0].out_xy = x.data_ptr()
        ja[0].params = p
        ja[0].stats = None
        P.inim_autotune_scan(ja, reps=3)
        P.inim_iterate(m, x.clone(), v, p, 2)             # warm
        torch.cuda.synchronize()
        t = time.perf_counter()
        st, _ = P.inim_iterate(m, x, v, p, K)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        outs[name] = x.cpu().numpy()
        res["precisions"][name] = {"ms_per_iteration": 1e3 * dt / K, "eps": st["eps"], "xi": st["xi"]}
        # stage times of this 4096^2 job and its dominant kernel against the copy bandwidth
        stages = P.inim_profile_stages(reps=5)
        N = 1 << 12
        tile = P.inim_get_scan_tile(12, prec, 1)
        E = int(P.inim_map_info(m)["n_edges"])
        algo = stage_bytes(1, N, mesh.n_verts, mesh.n_regions, E, crossings_count(mesh, N), -(-N // tile["band_rows"]))
        if prec != P.INIM_FP32:                     # 64-bit sums: 8 more bytes per pixel in S and T
            for sn in ("scan_phase3", "scan_fused"):
                algo[sn] += 8 * N * N
        dom = max((sn for sn in stages if stages[sn] > 0), key=lambda sn: stages[sn])
        pk = peaks()
        gbs = algo[dom] / (stages[dom] / 1e3) / 1e9
        res["precisions"][name].update(stages_ms=stages, dominant=dom, dominant_gbs=gbs,
                                       dominant_frac=gbs / pk["hbm_gbs"], scan_tile=tile)
    np.savez_compressed(args.study_out, verts=xy0, ring_off=mesh.ring_off, ring_idx=mesh.ring_idx,
                        ring_region=mesh.ring_region, n_regions=mesh.n_regions, values=vals, iterations=K,
                        **{f"gpu_{k}": v for k, v in outs.items()})
    print(json.dumps(res))
    return 0


# ---------------------------------------------------------------------------
# quality measures (Sec. 3.3) of the sweep's map against a cartogram of it
# ---------------------------------------------------------------------------
def quality_timing(args):
    """inim_quality on the sweep's map (1024^2, 200 regions; or, with
    --quality-map 4096, the 4096^2 map of 2000 regions of the precision study)
    against its cartogram after 20 iterations on the last time step's values:
    host wall time per call (both rasters, the kernels, the call's own
    allocations)."""
    import torch
    import paper_2604_13880_gb300 as P
    from paper_2604_13880_gb300 import synth
    w = synth.precision_workload() if args.quality_map == 4096 else synth.time_varying_workload()
    mesh = w["mesh"]
    k = w.get("log2_res", 12)
    m = P.inim_map_create(mesh)
    x = torch.as_tensor(mesh.verts_f32(), device="cuda")
    v = torch.as_tensor(w["values"][-1].astype(np.float32), device="cuda")
    P.inim_iterate(m, x, v, P.params(log2_res=k, shape=0.5), 20)
    res, _ = P.inim_quality(m, x, k)                       # warm
    times = []
    for _ in range(args.quality):
        torch.cuda.synchronize()
        t = time.perf_counter()
        res, _ = P.inim_quality(m, x, k)
        times.append(time.perf_counter() - t)
    print(json.dumps({"quality": w["name"], "log2_res": k, "n_regions": mesh.n_regions, "calls": args.quality,
                      "ms_per_call_median": 1e3 * float(np.median(times)), "ms_per_call_min": 1e3 * min(times),
                      **res}))
    return 0


# ---------------------------------------------------------------------------
# dynamic area (Sec. 4.3, Eq. (Mb)) on the sweep's map and values
# ---------------------------------------------------------------------------
def dynamic_timing(args):
    """inim_run_dynamic on the sweep's map (1024^2, 200 regions) and its 24
    time steps, area fractions 0.45 .. 0.65, K fixed iterations per step, in
    direct and in cumulative mode: iterations/s through the public call (host
    values in, host vertices out, CUDA events around the call), and the same
    steps with a fixed background (inim_run) for comparison."""
    import torch
    import paper_2604_13880_gb300 as P
    from paper_2604_13880_gb300 import synth
    w = synth.time_varying_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    vals = np.ascontiguousarray(w["values"].astype(np.float32))
    T = vals.shape[0]
    m = P.inim_map_create(mesh)
    a_min, a_max, K = 0.45, 0.65, args.dynamic
    res = {"dynamic": w["name"], "steps": T, "iterations_per_step": K, "area_fractions": [a_min, a_max]}
    bdv, frac = P.inim_background_values(vals, k, a_min, a_max)
    res["background_value_range"] = [float(np.min(bdv)), float(np.max(bdv))]
    for name, mode in (("direct", P.INIM_DIRECT), ("cumulative", P.INIM_CUMULATIVE)):
        p = P.params(log2_res=k, shape=0.5, max_iters=K, xi_stop=0.0, stall_window=0, mode=mode)
        for call, fn in (("dynamic", lambda: P.inim_run_dynamic(m, vals, p, a_min, a_max)),
                         ("fixed_background", lambda: P.inim_run(m, vals, p))):
            fn()                                                   # warm: batches, graphs
            torch.cuda.synchronize()
            ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            ev0.record()
            out, stats, _ = fn()
            ev1.record()
            torch.cuda.synchronize()
            ms = ev0.elapsed_time(ev1)
            res[f"{name}_{call}"] = {"ms": ms, "iterations_per_s": T * K / (ms / 1e3),
                                     "eps_last": float(stats[-1]["eps"])}
    print(json.dumps(res))
    return 0


# ---------------------------------------------------------------------------
# direct vs cumulative (Sec. 5.5) on a random walk with large jumps
# ---------------------------------------------------------------------------
def coherence_study(args):
    """The sweep's map under T steps of a log-normal random walk with step
    sigma --coherence-sigma, solved in both modes with the stop rule of
    Sec. 4.1 (xi < 0.01, 32-iteration stall, 512 iterations; shape 0.5): per
    step the iterations, eps, xi and the quality of the cartogram against the
    original map (inim_quality: tau, shape distortion, R), and each mode's
    wall time for the whole series."""
    import torch
    import paper_2604_13880_gb300 as P
    from paper_2604_13880_gb300 import synth
    w = synth.time_varying_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    T = args.coherence_study
    vals = synth.random_walk_values(mesh.n_regions, T, seed=202, sigma=args.coherence_sigma).astype(np.float32)
    m = P.inim_map_create(mesh)
    res = {"coherence_study": w["name"], "steps": T, "sigma": args.coherence_sigma, "modes": {}}
    for name, mode in (("direct", P.INIM_DIRECT), ("cumulative", P.INIM_CUMULATIVE)):
        p = P.params(log2_res=k, shape=0.5, mode=mode)
        P.inim_run(m, vals[:2], p)                         # warm: graphs, scan tiles
        torch.cuda.synchronize()
        t = time.perf_counter()
        out, stats, _ = P.inim_run(m, vals, p)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        steps = []
        for s in range(T):
            q, _ = P.inim_quality(m, out[s], k)
            steps.append({"iters": stats[s]["iters"], "eps": stats[s]["eps"], "xi": stats[s]["xi"],
                          "tau": q["tau"], "shape": q["shape"], "rel_pos": q["rel_pos"]})
        res["modes"][name] = {"wall_s": dt, "iterations": int(sum(x["iters"] for x in steps)), "per_step": steps}
    print(json.dumps(res))
    return 0


# ---------------------------------------------------------------------------
# the batched workload: 64 independent maps of uneven texture sizes
# ---------------------------------------------------------------------------
def batched_config(args):
    """64 maps (N from {256, 512, 1024, 2048}, 20-500 regions, log-normal
    values, FP32, shape 0.5) solved together in one batch: iterations/s of 50
    fixed iterations per map (inputs resident in HBM; and through pinned host
    buffers), the dominant kernel's roofline from stage timings, and the same
    batch with the stop rule of Sec. 4.1 (time until every map stops)."""
    import torch
    import paper_2604_13880_gb300 as P
    from paper_2604_13880_gb300 import _lib, synth
    lib = _lib.load()
    t_gen = time.perf_counter()
    w = synth.batched_workload()
    t_gen = time.perf_counter() - t_gen
    maps = [P.inim_map_create(x["mesh"]) for x in w]
    B = len(w)
    vals_h = [torch.as_tensor(np.ascontiguousarray(x["values"][0], dtype=np.float32)).pin_memory() for x in w]
    vals_d = [v.cuda() for v in vals_h]
    out_h = [torch.empty((x["mesh"].n_verts, 2)).pin_memory() for x in w]
    out_d = [torch.empty((x["mesh"].n_verts, 2), device="cuda") for x in w]
    iters = ITERS

    def jobs(vals, outs, max_iters=iters, rule=False):
        arr = (P.inim_job * B)()
        for q, x in enumerate(w):
            arr[q].map = maps[q].handle
            arr[q].values = vals[q].data_ptr()
            arr[q].init_xy = None
            arr[q].out_xy = outs[q].data_ptr()
            arr[q].params = P.params(log2_res=x["log2_res"], shape=0.5, max_iters=max_iters,
                                     xi_stop=0.01 if rule else 0.0, stall_window=32 if rule else 0)
            arr[q].stats = None
        return arr

    jd = jobs(vals_d, out_d)
    P.inim_autotune_scan(jd, reps=5)                         # tiles of every size group of the batch
    tiles = {f"{1 << kk}": {"small": P.inim_get_scan_tile(kk, P.INIM_FP32, 0),
                            "large": P.inim_get_scan_tile(kk, P.INIM_FP32, 1)} for kk in (8, 9, 10, 11)}

    def run(a):
        _lib.check(lib.inim_run_batch(a, B, None), "batched")

    for _ in range(args.warmup):
        run(jd)
    torch.cuda.synchronize()
    clocks = ClockSampler()
    launches0 = P.inim_launch_count()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record()
    for _ in range(args.steps):
        run(jd)
    ev1.record()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = P.inim_launch_count() - launches0
    clk = clocks.stop()
    value = B * iters * args.steps / (ms / 1e3)
    # through the public API with pinned host buffers (values in, vertices out)
    jh = jobs(vals_h, out_h)
    run(jh)
    torch.cuda.synchronize()
    t = time.perf_counter()
    for _ in range(args.steps):
        run(jh)
    torch.cuda.synchronize()
    e2e = B * iters * args.steps / (time.perf_counter() - t)
    # stop rule: until every map stops (xi < 0.01, 32 iterations without a new best xi, or 512)
    stats = (P.inim_step_stats * B)()
    jr = jobs(vals_d, out_d, 512, True)
    for q in range(B):
        jr[q].stats = ctypes.pointer(stats[q])
    run(jr)
    torch.cuda.synchronize()
    t = time.perf_counter()
    run(jr)
    torch.cuda.synchronize()
    rule_s = time.perf_counter() - t
    its = [stats[q].iters for q in range(B)]
    # stage timings of the batch and the dominant kernel against the copy bandwidth
    run(jd)
    stages = P.inim_profile_stages(reps=5)
    pk = peaks()
    algo = {}
    for q, x in enumerate(w):
        mesh = x["mesh"]
        N = 1 << x["log2_res"]
        E = int(P.inim_map_info(maps[q])["n_edges"])
        K = crossings_count(mesh, N)
        large = sum(1 << (2 * y["log2_res"]) for y in w if y["log2_res"] == x["log2_res"]) >= (1 << 23)
        H = tiles[str(N)]["large" if large else "small"]["band_rows"]
        for st_name, b in stage_bytes(1, N, mesh.n_verts, mesh.n_regions, E, K, -(-N // H)).items():
            algo[st_name] = algo.get(st_name, 0) + b
    dom = max((sn for sn in stages if stages[sn] > 0), key=lambda sn: stages[sn])
    achieved = algo[dom] / (stages[dom] / 1e3) / 1e9
    px = sum(1 << (2 * x["log2_res"]) for x in w)
    V = sum(x["mesh"].n_verts for x in w)
    line = {"metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batched64_res256-2048_regions20-500_it50", "maps": B,
                       "textures": {str(1 << kk): sum(1 for x in w if x["log2_res"] == kk) for kk in (8, 9, 10, 11)},
                       "pixels": px, "vertices": V, "iterations_per_map": iters,
                       "l2": f"inputs larger than L2 ({px * 12 / 1e9:.2f} GB of texture traffic per iteration)",
                       "scan_tiles_autotuned": tiles, "map_generation_s": t_gen},
            "e2e": {"value": e2e, "unit": "iterations/s", "h2d_bytes_per_step": sum(4 * x["mesh"].n_regions for x in w),
                    "d2h_bytes_per_step": 8 * V, "host_buffers": "pinned"},
            "gpu_launches": int(launches),
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": pk["hbm_gbs"], "unit": "GB/s",
                         "frac": achieved / pk["hbm_gbs"], "traffic": None,
                         "algorithmic_bytes_per_launch": algo[dom], "launch_ms": stages[dom],
                         "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)" if "fallback" not in pk else "fallback"},
            "stages_ms": stages,
            "stages_gbs": {sn: algo[sn] / (stages[sn] / 1e3) / 1e9 for sn in stages if stages[sn] > 0 and sn in algo},
            "iteration_bytes": px * 12 + V * 48,
            "iteration_gbs": (px * 12 + V * 48) / (ms / 1e3 / (iters * args.steps)) / 1e9,
            "stop_rule": {"wall_ms": 1e3 * rule_s, "iters_mean": float(np.mean(its)), "iters_max": int(max(its)),
                          "iterations_per_s": float(sum(its)) / rule_s,
                          "converged_xi_below_0.01": int(sum(stats[q].xi < 0.01 for q in range(B)))}}
    if clk:
        line["clocks"] = clk
    if not args.no_extras:
        # CPU oracle: one iteration of each of a few maps on one core
        from oracle import inim_oracle as O
        t = time.perf_counter()
        n = 0
        for x in sorted(w, key=lambda y: y["log2_res"])[::8]:
            mesh = x["mesh"]
            O.iterate(mesh.verts_f32().astype(np.float64), (mesh.ring_off, mesh.ring_idx, mesh.ring_region,
                      mesh.n_regions), x["values"][0], x["log2_res"], 0.5)
            n += 1
        cpu_s = time.perf_counter() - t
        line["cpu_baseline"] = {"value": n / cpu_s, "unit": "iterations/s", "cores": 1, "kind": "oracle",
                                "sample": f"one iteration of each of {n} maps of the batch (every 8th by size), "
                                          f"{cpu_s:.1f} s"}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
# in-graph kernel timeline of both batch shapes of the sweep
# ---------------------------------------------------------------------------
def timeline_study(args):
    """The sweep's two batch shapes run alone (the 72-solve direct batch and
    the 3-solve batch of the cumulative chain), 50 iterations each under the
    library's CUDA graphs with programmatic launches, with the kernel
    timeline on: per kernel the median time from its first block's start to
    its last block's end, the median gap to the next kernel's first block,
    and the time per iteration (medians over iterations 5-49).  Scan tiles
    from --tiles (default: the tiles the sweep uses).  Also the chain's
    kernel timeline at later rounds of its cumulative series
    (chain_rounds_timeline) and the step split by series kind
    (series_split)."""
    import torch
    import paper_2604_13880_gb300 as P
    from paper_2604_13880_gb300 import _lib, synth
    lib = _lib.load()
    w = synth.time_varying_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    vals = np.ascontiguousarray(w["values"].astype(np.float32))
    m = P.inim_map_create(mesh)
    tl = [tuple(int(x) for x in t.split(",")) for t in args.tiles.split(":")] if args.tiles else \
        [(64, 4, 256), (8, 0, 256)]
    P.inim_set_scan_tile(k, P.INIM_FP32, 1, *tl[0])
    P.inim_set_scan_tile(k, P.INIM_FP32, 0, *tl[1])
    P.inim_timeline(True)
    names = P.TIMELINE_KERNELS
    res = {"timeline": w["name"], "tiles": {"large": tl[0], "small": tl[1]}, "iterations": ITERS, "batches": {}}
    for name, jobs in (("chain3", [(sh, 0) for sh in SHAPES]),
                       ("direct72", [(sh, t) for sh in SHAPES for t in range(T_STEPS)])):
        arr = (P.inim_job * len(jobs))()
        outs = [np.empty((mesh.n_verts, 2), np.float32) for _ in jobs]
        for q, (sh, t) in enumerate(jobs):
            arr[q].map = m.handle
            arr[q].values = vals[t].ctypes.data
            arr[q].init_xy = None
            arr[q].out_xy = outs[q].ctypes.data
            arr[q].params = P.params(log2_res=k, shape=sh, max_iters=ITERS, xi_stop=0.0, stall_window=0)
            arr[q].stats = None
        # the same run without the timeline (its block counters are atomics on
        # one address per kernel, which add to every launch): CUDA events
        P.inim_timeline(False)
        for _ in range(2):
            _lib.check(lib.inim_run_batch(arr, len(arr), None), "timeline")
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record()
        for _ in range(4):
            _lib.check(lib.inim_run_batch(arr, len(arr), None), "timeline")
        ev1.record()
        torch.cuda.synchronize()
        plain_us = 1e3 * ev0.elapsed_time(ev1) / (4 * ITERS)
        P.inim_timeline(True)
        for _ in range(2):                                # graphs, buffers, warm caches
            _lib.check(lib.inim_run_batch(arr, len(arr), None), "timeline")
        P.inim_timeline_read()
        _lib.check(lib.inim_run_batch(arr, len(arr), None), "timeline")
        st, en = P.inim_timeline_read()
        ran = [q for q in range(len(names)) if st[q, 5] > 0]
        lo, hi = 5, ITERS
        kern = {names[q]: float(np.median(en[q, lo:hi] - st[q, lo:hi])) / 1e3 for q in ran}
        path = [q for q in ran if names[q] != "areas_errors"]
        gaps = {f"{names[a]}->{names[b]}": float(np.median(st[b, lo:hi] - en[a, lo:hi])) / 1e3
                for a, b in zip(path[:-1], path[1:])}
        gaps[f"{names[path[-1]]}->next {names[path[0]]}"] = float(
            np.median(st[path[0], lo + 1:hi] - en[path[-1], lo:hi - 1])) / 1e3
        res["batches"][name] = {"jobs": len(jobs), "us_per_iteration": float(np.median(np.diff(st[0, lo:hi]))) / 1e3,
                                "us_per_iteration_timeline_off": plain_us, "kernel_us": kern, "gap_us": gaps}
    P.inim_timeline(False)
    res["chain3_rounds"] = chain_rounds_timeline(P, _lib, lib, m, mesh, k, vals, names)
    res["series_split_ms"] = series_split(P, _lib, lib, m, mesh, k, vals)
    print(json.dumps(res))
    return 0


def chain_rounds_timeline(P, _lib, lib, m, mesh, k, vals, names, sample=(0, 12, 23)):
    """The cumulative chain advanced round by round from the initial map (each
    round starts from the previous round's 50-iteration result), with the
    kernel timeline of the sampled rounds: their maps stretch, rows hold more
    crossings and regions fold over.  Per sampled round: median kernel times
    and time per iteration (iterations 5-49), the mean crossings per row and
    the flags of the three solves."""
    import torch
    xy = [torch.as_tensor(mesh.verts_f32(), device="cuda").contiguous() for _ in SHAPES]
    out = [torch.empty_like(x) for x in xy]
    N = 1 << k

    def run_round(t):
        arr = (P.inim_job * len(SHAPES))()
        stats = (P.inim_step_stats * len(SHAPES))()
        for q, sh in enumerate(SHAPES):
            arr[q].map = m.handle
            arr[q].values = vals[t].ctypes.data
            arr[q].init_xy = xy[q].data_ptr()
            arr[q].out_xy = out[q].data_ptr()
            arr[q].params = P.params(log2_res=k, shape=sh, max_iters=ITERS, xi_stop=0.0, stall_window=0)
            arr[q].stats = ctypes.cast(ctypes.byref(stats[q]), ctypes.POINTER(P.inim_step_stats))
        _lib.check(lib.inim_run_batch(arr, len(arr), None), "chain round")
        return stats

    rounds = {}
    for t in range(T_STEPS):
        if t in sample:
            P.inim_timeline(True)
            for _ in range(2):
                run_round(t)
            P.inim_timeline_read()
            stats = run_round(t)
            st, en = P.inim_timeline_read()
            P.inim_timeline(False)
            ran = [q for q in range(len(names)) if st[q, 5] > 0]
            rows = float(np.mean([crossings_count(mesh_at(mesh, x.cpu().numpy()), N) for x in xy])) / N
            rounds[str(t)] = {
                "us_per_iteration": float(np.median(np.diff(st[0, 5:ITERS]))) / 1e3,
                "kernel_us": {names[q]: float(np.median(en[q, 5:ITERS] - st[q, 5:ITERS])) / 1e3 for q in ran},
                "crossings_per_row": rows,
                "foldover": [int(x.foldover) for x in stats], "overlap": [int(x.overlap) for x in stats]}
        run_round(t)
        torch.cuda.synchronize()
        for q in range(len(SHAPES)):
            xy[q].copy_(out[q])
    return rounds


def mesh_at(mesh, xy):
    """The mesh with its vertices moved to xy."""
    from paper_2604_13880_gb300 import synth
    return synth.Mesh(np.asarray(xy, np.float64), mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)


def series_split(P, _lib, lib, m, mesh, k, vals, reps=5):
    """One sweep step as inim_run_series calls: both series kinds (the
    benchmark's step), the 3 direct series alone and the 3 cumulative series
    alone; median wall ms of `reps` calls after 3 warm-up calls."""
    import torch
    V = mesh.n_verts
    vals_d = torch.as_tensor(vals, device="cuda").contiguous()
    out_d = torch.empty((len(SHAPES) * T_STEPS, V, 2), device="cuda")
    out_c = torch.empty((len(SHAPES) * T_STEPS, V, 2), device="cuda")

    def series(kinds):
        ser = (P.inim_series * (len(kinds) * len(SHAPES)))()
        for a, (mode, buf) in enumerate(kinds):
            for b, sh in enumerate(SHAPES):
                x = ser[a * len(SHAPES) + b]
                x.map = m.handle
                x.values = vals_d.data_ptr()
                x.T = T_STEPS
                x.init_xy = None
                x.out_xy = buf.data_ptr() + b * T_STEPS * V * 8
                x.params = P.params(log2_res=k, shape=sh, max_iters=ITERS, xi_stop=0.0, stall_window=0, mode=mode)
                x.stats = None
        return ser

    res = {}
    for name, kinds in (("both", [(P.INIM_DIRECT, out_d), (P.INIM_CUMULATIVE, out_c)]),
                        ("direct_only", [(P.INIM_DIRECT, out_d)]),
                        ("cumulative_only", [(P.INIM_CUMULATIVE, out_c)])):
        ser = series(kinds)
        for _ in range(3):
            _lib.check(lib.inim_run_series(ser, len(ser), None), name)
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            _lib.check(lib.inim_run_series(ser, len(ser), None), name)
            torch.cuda.synchronize()
            ts.append((time.perf_counter() - t0) * 1e3)
        res[name] = float(np.median(ts))
    return res


# ---------------------------------------------------------------------------
# small fixed cases for profiler captures (ncu): one batch, two iterations
# ---------------------------------------------------------------------------
def ncu_case(args):
    """direct72: the sweep's 72-solve direct batch; chain3: the 3-solve batch
    of its cumulative series.  Scan tiles from --tiles, else 16/4/256 for the
    72-solve batch and 8 rows in the parallel-rows form for the 3-solve
    batch.  Per iteration the batch launches, in order: k_crossings,
    k_raster_rows, k_scan_band*<...,1> (which builds the density table),
    k_scan_carry*, k_scan_band*<...,3>, k_gather_move, k_areas_errors (after
    k_raster_reset)."""
    import torch
    import paper_2604_13880_gb300 as P
    from paper_2604_13880_gb300 import _lib, synth
    w = synth.time_varying_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    vals = np.ascontiguousarray(w["values"].astype(np.float32))
    m = P.inim_map_create(mesh)
    tl = [tuple(int(x) for x in t.split(",")) for t in args.tiles.split(":")] if args.tiles else \
        [(16, 4, 256), (8, 0, 256)]
    P.inim_set_scan_tile(k, P.INIM_FP32, 1, *tl[0])
    P.inim_set_scan_tile(k, P.INIM_FP32, 0, *tl[1])
    steps = range(T_STEPS) if args.ncu_case == "direct72" else range(1)
    jobs = [(sh, t) for sh in SHAPES for t in steps]
    arr = (P.inim_job * len(jobs))()
    outs = [np.empty((mesh.n_verts, 2), np.float32) for _ in jobs]
    for q, (sh, t) in enumerate(jobs):
        arr[q].map = m.handle
        arr[q].values = vals[t].ctypes.data
        arr[q].init_xy = None
        arr[q].out_xy = outs[q].ctypes.data
        arr[q].params = P.params(log2_res=k, shape=sh, max_iters=2, xi_stop=0.0, stall_window=0)
        arr[q].stats = None
    _lib.check(_lib.load().inim_run_batch(arr, len(arr), None), "ncu case")
    torch.cuda.synchronize()
    print(json.dumps({"ncu_case": args.ncu_case, "jobs": len(jobs), "iterations": 2}))
    return 0


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip plain form, time-to-eps and CPU baseline")
    ap.add_argument("--tiles", default=None, metavar="H,C,T:H,C,T",
                    help="scan tiles (band rows, columns per thread (0 = parallel rows), threads) of the "
                         "72-solve and the 3-solve batch, instead of the autotuner and the step-level choice")
    ap.add_argument("--precision-study", type=int, default=0, metavar="K",
                    help="instead of the sweep: K iterations of the 4096^2 precision workload in FP32, "
                         "FIX64 and compensated sums; results to --study-out for the FP64 oracle comparison")
    ap.add_argument("--study-out", default="precision_study.npz")
    ap.add_argument("--coherence-study", type=int, default=0, metavar="T",
                    help="instead of the sweep: T steps of a random walk with large jumps in direct and "
                         "cumulative mode with the stop rule, with per-step errors and quality measures")
    ap.add_argument("--coherence-sigma", type=float, default=0.6)
    ap.add_argument("--quality", type=int, default=0, metavar="K",
                    help="instead of the sweep: time K calls of inim_quality on the sweep's map")
    ap.add_argument("--quality-map", type=int, default=1024, choices=[1024, 4096],
                    help="the map of --quality: the sweep's (1024^2) or the precision study's (4096^2)")
    ap.add_argument("--dynamic", type=int, default=0, metavar="K",
                    help="instead of the sweep: the dynamic-area series (Eq. (Mb)) with K iterations per step")
    ap.add_argument("--timeline", action="store_true",
                    help="instead of the sweep: in-graph kernel timeline of the sweep's two batch shapes")
    ap.add_argument("--config", choices=["sweep", "batched"], default="sweep",
                    help="batched: the 64-map batched workload instead of the time-varying sweep")
    ap.add_argument("--ncu-case", choices=["direct72", "chain3"], default=None,
                    help="instead of the sweep: one batch for two iterations (small profiler captures)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        return run_reference(args)
    if args.precision_study:
        return precision_study(args)
    if args.ncu_case:
        return ncu_case(args)
    if args.quality:
        return quality_timing(args)
    if args.coherence_study:
        return coherence_study(args)
    if args.dynamic:
        return dynamic_timing(args)
    if args.config == "batched":
        return batched_config(args)
    if args.timeline:
        return timeline_study(args)

    import torch
    import paper_2604_13880_gb300 as P
    from paper_2604_13880_gb300 import _lib, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    lib = _lib.load()

    w = synth.time_varying_workload()
    mesh = w["mesh"]
    k = w["log2_res"]
    V, R = mesh.n_verts, mesh.n_regions
    vals = w["values"].astype(np.float32)                     # [24, 200]
    m = P.inim_map_create(mesh)

    def prm(shape, **kw):
        return P.params(log2_res=k, shape=shape, max_iters=ITERS, xi_stop=0.0, stall_window=0, **kw)

    def job_array(entries):
        arr = (P.inim_job * len(entries))()
        for q, (vp, ip, op, p) in enumerate(entries):
            arr[q].map = m.handle
            arr[q].values = vp
            arr[q].init_xy = ip
            arr[q].out_xy = op
            arr[q].params = p
            arr[q].stats = None
        return arr

    def make_plan(vals_buf, out_direct, out_cum, stride):
        """The sweep as one inim_run_series call (3 direct + 3 cumulative series)
        over the given buffers (device or pinned host), plus job arrays of the
        two batch shapes for the autotuner and the stage profile."""
        vp = lambda t: vals_buf.data_ptr() + t * R * 4                    # noqa: E731
        op = lambda buf, q: buf.data_ptr() + q * V * 2 * 4                 # noqa: E731
        ser = (P.inim_series * (2 * len(SHAPES)))()
        for q, (mode, buf) in enumerate(((P.INIM_DIRECT, out_direct), (P.INIM_CUMULATIVE, out_cum))):
            for s_, sh in enumerate(SHAPES):
                x = ser[q * len(SHAPES) + s_]
                x.map = m.handle
                x.values = vp(0)
                x.T = T_STEPS
                x.init_xy = None
                x.out_xy = op(buf, s_ * T_STEPS)
                x.params = prm(sh, mode=mode)
                x.stats = None
        direct = job_array([(vp(t), None, op(out_direct, s * T_STEPS + t), prm(sh))
                            for s, sh in enumerate(SHAPES) for t in range(T_STEPS)])
        small = job_array([(vp(0), None, op(out_cum, s * T_STEPS), prm(sh)) for s, sh in enumerate(SHAPES)])
        return ser, direct, small

    def run_step(plan):
        ser = plan[0]
        _lib.check(lib.inim_run_series(ser, len(ser), None), "sweep")

    # device-resident inputs and outputs
    vals_d = torch.as_tensor(vals, device=dev).contiguous()
    out_dir_d = torch.empty((len(SHAPES) * T_STEPS, V, 2), device=dev)
    out_cum_d = torch.empty((len(SHAPES) * T_STEPS, V, 2), device=dev)
    plan_d = make_plan(vals_d, out_dir_d, out_cum_d, None)

    # scan tiles chosen by the autotuner on the two batch shapes of the step
    fixed = [tuple(int(x) for x in t.split(",")) for t in args.tiles.split(":")] if args.tiles else None
    if fixed:
        P.inim_set_scan_tile(k, P.INIM_FP32, 1, *fixed[0])
        P.inim_set_scan_tile(k, P.INIM_FP32, 0, *fixed[1])
    else:
        P.inim_autotune_scan(plan_d[1], reps=5)
        P.inim_autotune_scan(plan_d[2], reps=20)
    # The autotuner times each batch's scan alone; in the step the 72-solve
    # batch shares the GPU with the latency-bound cumulative chain, where
    # other tiles can win.  Time the step with the tuned large tile, two other
    # band heights of its form and the parallel-rows tile, keep the fastest.
    tuned = P.inim_get_scan_tile(k, P.INIM_FP32, 1)
    tuned_t = (tuned["band_rows"], tuned["cols_per_thread"], tuned["threads"])
    cands = []
    if not fixed:
        cands = [tuned_t]
        if tuned_t[1] > 0:
            cands += [(h, tuned_t[1], tuned_t[2]) for h in (16, 32, 64) if h != tuned_t[0]]
        else:
            cands += [(h, 4, 256) for h in (16, 32, 64)]
        if (1 << k) in (512, 1024):
            cands += [(h, 0, 256) for h in (8, 16) if (h, 0, 256) != tuned_t]
    step_times = {}
    for t in cands:
        P.inim_set_scan_tile(k, P.INIM_FP32, 1, *t)
        run_step(plan_d)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        run_step(plan_d)
        torch.cuda.synchronize()
        step_times[t] = time.perf_counter() - t0
    if step_times:
        best_t = min(step_times, key=step_times.get)
        P.inim_set_scan_tile(k, P.INIM_FP32, 1, *best_t)
    tiles = {cls: P.inim_get_scan_tile(k, P.INIM_FP32, large) for cls, large in (("large", 1), ("small", 0))}

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(args.warmup):
        run_step(plan_d)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    barrier()
    clocks = ClockSampler(uuid) if rank == 0 else None
    launches0 = P.inim_launch_count()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record()
    t_wall = time.perf_counter()
    torch.cuda.nvtx.range_push("timed_step")       # profilers can capture exactly the timed steps
    for _ in range(args.steps):
        run_step(plan_d)
    torch.cuda.nvtx.range_pop()
    ev1.record()
    barrier()
    wall = time.perf_counter() - t_wall
    ms = ev0.elapsed_time(ev1)
    launches = P.inim_launch_count() - launches0
    clk = clocks.stop() if clocks else None
    ms_max, value = whole_job_rate(ms, ITERS_PER_STEP * args.steps, world, dist, dev)

    # e2e: the same sweep through the public API with pinned host buffers
    vals_h = torch.as_tensor(vals).pin_memory()
    out_dir_h = torch.empty((len(SHAPES) * T_STEPS, V, 2)).pin_memory()
    out_cum_h = torch.empty((len(SHAPES) * T_STEPS, V, 2)).pin_memory()
    plan_h = make_plan(vals_h, out_dir_h, out_cum_h, None)
    run_step(plan_h)
    barrier()
    e_steps = args.steps                           # the same step count as the device-resident value
    t = time.perf_counter()
    for _ in range(e_steps):
        run_step(plan_h)
    barrier()
    e2e_s = time.perf_counter() - t
    _, e2e_value = whole_job_rate(1e3 * e2e_s, ITERS_PER_STEP * e_steps, world, dist, dev)
    n_sol = 2 * len(SHAPES) * T_STEPS
    h2d = n_sol * R * 4            # the values of every solve
    d2h = n_sol * V * 8            # the vertices after every solve

    line = {"metric": METRIC, "value": value, "unit": "iterations/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "texture": "1024x1024", "regions": R, "vertices": V,
                       "iterations_per_step": ITERS_PER_STEP,
                       "l2": "inputs larger than L2 (72 solves x ~13 MB of textures per batched iteration)",
                       "parallelism": f"replicas{world}",
                       ("scan_tiles_fixed" if fixed else "scan_tiles_autotuned"): tiles,
                       "large_tile_by_step_ms": {",".join(map(str, h)): round(1e3 * t, 2)
                                                 for h, t in step_times.items()}},
            "e2e": {"value": e2e_value, "unit": "iterations/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "host_buffers": "pinned"},
            "gpu_launches": int(launches), "wall_s_timed": wall,
            # completed cartograms (time steps of a series, ITERS iterations each) per second
            "cartograms_per_s": {"value": value / ITERS, "e2e": e2e_value / ITERS, "unit": "cartograms/s"}}
    if clk:
        line["clocks"] = clk

    if rank == 0:
        # stage times of both batch shapes of the step (CUDA events around each
        # stage on the library's stream); the step's dominant kernel is the one
        # with the largest time per step (launch time x launches per step)
        N = 1 << k
        E = int(P.inim_map_info(m)["n_edges"])
        K = crossings_count(mesh, N)
        run_step(plan_d)
        _lib.check(lib.inim_run_batch(plan_d[1], len(plan_d[1]), None), "direct batch")
        stages_d = P.inim_profile_stages(reps=10)
        _lib.check(lib.inim_run_batch(plan_d[2], len(plan_d[2]), None), "3-solve batch")
        stages_c = P.inim_profile_stages(reps=20)
        batches = {
            "direct72": dict(stages=stages_d, jobs=len(SHAPES) * T_STEPS, tile=tiles["large"], per_step=ITERS),
            "chain3": dict(stages=stages_c, jobs=len(SHAPES), tile=tiles["small"], per_step=T_STEPS * ITERS),
        }
        pk = peaks()
        for name, b in batches.items():
            b["algo"] = stage_bytes(b["jobs"], N, V, R, E, K, -(-N // b["tile"]["band_rows"]))
        dom_b, dom_s = max(((bn, sn) for bn, b in batches.items() for sn in b["stages"]),
                           key=lambda x: batches[x[0]]["stages"][x[1]] * batches[x[0]]["per_step"])
        line["roofline"] = roofline(batches, dom_b, dom_s, pk)
        dd = max(stages_d, key=stages_d.get)
        line["roofline_direct72"] = roofline(batches, "direct72", dd, pk)
        line["stages_ms"] = stages_d
        # (a stage timed 0 is not in the iteration: the density table built by scan phase 1)
        line["stages_gbs"] = {st: batches["direct72"]["algo"][st] / (stages_d[st] / 1e3) / 1e9
                              for st in stages_d if stages_d[st] > 0}
        line["stages_3solve_ms"] = stages_c
        line["stage_ms_per_step"] = {f"{bn}:{sn}": round(b["stages"][sn] * b["per_step"], 3)
                                     for bn, b in batches.items() for sn in b["stages"]}
        # the sweep with the cumulative series in one persistent launch instead
        # (runs after the direct batch), with its phase times per iteration
        P.inim_set_persistent(True)
        run_step(plan_d)
        torch.cuda.synchronize()
        P.inim_persistent_phase_times(True)
        t = time.perf_counter()
        run_step(plan_d)
        torch.cuda.synchronize()
        pers_s = time.perf_counter() - t
        ph = P.inim_persistent_phase_times(False)
        P.inim_set_persistent(False)
        line["persistent_variant"] = {
            "value": ITERS_PER_STEP / pers_s, "unit": "iterations/s",
            "phase_us_per_iteration": {k: 1e3 * v / (T_STEPS * ITERS) for k, v in ph.items()}}

    if rank == 0 and not args.no_extras:
        # plain unfused form on a bounded sample: 2 time steps x 3 shapes, direct
        tp = time.perf_counter()
        for sh in SHAPES:
            P.inim_run(m, vals[:2], prm(sh, form=P.INIM_FORM_PLAIN))
        torch.cuda.synchronize()
        plain_s = time.perf_counter() - tp
        plain_value = 2 * len(SHAPES) * ITERS / plain_s
        line["plain_form"] = {"value": plain_value, "unit": "iterations/s",
                              "sample": "3 shapes x 2 time steps x 50 iterations, one solve at a time",
                              "fused_over_plain": value / world / plain_value}
        # time to cartographic error eps, the same target for every form:
        # one solve (time step 0, shape 0.5) in the plain and the fused form,
        # with and without the learned warm start, and all 24 time steps as
        # one batch (direct), cold and warm
        eps_target = 0.1
        tte = {"eps_target": eps_target, "max_iters": 512, "shape": 0.5}

        def to_eps(vv, form=P.INIM_FORM_FUSED, warm=0):
            p = P.params(log2_res=k, shape=0.5, max_iters=512, xi_stop=0.0, stall_window=0, eps_stop=eps_target,
                         form=form, warm_start=warm)
            P.inim_run(m, vv, p)                                          # warm-up: graphs, buffers
            torch.cuda.synchronize()
            t = time.perf_counter()
            _, st, _ = P.inim_run(m, vv, p)
            torch.cuda.synchronize()
            its = [x["iters"] for x in st]
            return {"ms": 1e3 * (time.perf_counter() - t), "iters": int(sum(its)),
                    "reached": int(sum(x["eps"] < eps_target for x in st)), "solves": len(st),
                    "eps_max": float(max(x["eps"] for x in st))}

        tte["plain"] = to_eps(vals[:1], P.INIM_FORM_PLAIN)
        tte["fused"] = to_eps(vals[:1])
        tte["fused_batched_24_steps"] = to_eps(vals)
        blob, train_s = quick_warm_start_network()
        P.inim_warmstart_load(blob)
        tte["warm_start_network"] = {"training_maps": 1536, "epochs": 10, "seconds": train_s,
                                     "note": "trained in this run on fields the method generates (512^2 maps)"}
        tte["fused_warm"] = to_eps(vals[:1], warm=1)
        tte["fused_batched_24_steps_warm"] = to_eps(vals, warm=1)
        line["time_to_eps"] = tte
        # animation frames (Sec. 5.5): 10 frames per time step, the values
        # interpolated linearly between steps (231 frames of the 24 steps), a
        # cartogram of 50 iterations (shape 0.5) for every frame; direct (every
        # frame from the map, one batch) and cumulative (frame after frame)
        fv = torch.as_tensor(P.inim_interpolate_values(vals, 10), device=dev).contiguous()
        nf = int(fv.shape[0])
        fout = torch.empty((nf, V, 2), device=dev)
        fr = {"frames_per_step": 10, "frames": nf, "iterations_per_frame": ITERS, "shape": 0.5}
        for name, mode in (("direct", P.INIM_DIRECT), ("cumulative", P.INIM_CUMULATIVE)):
            ser = [dict(map=m, values=fv, params=prm(0.5, mode=mode), out_xy=fout)]
            P.inim_run_series(ser)                                         # warm-up: buffers, graphs
            torch.cuda.synchronize()
            t = time.perf_counter()
            P.inim_run_series(ser)
            torch.cuda.synchronize()
            dt = time.perf_counter() - t
            fr[name] = {"frames_per_s": nf / dt, "seconds": dt, "iterations_per_s": nf * ITERS / dt}
        line["frames"] = fr
        # CPU oracle on a bounded sample (this host's cores): one core, then all
        from oracle import inim_oracle as O
        arrays = (mesh.ring_off, mesh.ring_idx, mesh.ring_region, mesh.n_regions)
        t0 = O.transform_uniform(1 << k)
        xy = mesh.verts_f32().astype(np.float64)
        n_cpu = 0
        t = time.perf_counter()
        while n_cpu < 40 and (n_cpu < 3 or time.perf_counter() - t < 15.0):
            xy, _ = O.iterate(xy, arrays, w["values"][0], k, 0.5, t0=t0)
            n_cpu += 1
        cpu_s = time.perf_counter() - t
        line["cpu_baseline"] = {"value": n_cpu / cpu_s, "unit": "iterations/s", "cores": 1, "kind": "oracle",
                                "sample": f"{n_cpu} oracle iterations of the 1024^2 map (shape 0.5, t=0), "
                                          f"{cpu_s:.1f} s"}
        line["cpu_baseline_all_cores"] = cpu_all_cores(mesh, w["values"], k)
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
