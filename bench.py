#!/usr/bin/env python3
"""Throughput of the micro-continuum (VoS) time step on GB300.

Workload (default ``rock256``): synthetic 3D carbonate-like rock, 256^3
voxels, overlapping spheres with lognormal radii (median 12 voxels, log-sd
0.3) shifted to porosity 0.20, fluid bands at inlet/outlet, no-slip lateral
walls; Pe = 10, Da = 1, iVoS; mixed precision (FP32 multigrid / Krylov
inner solves, FP64 refinement, FP64 fields and reductions), pressure and
momentum solved to a relative residual of 1e-8, concentration to 1e-10.
A step is one full vos_step (S1-S7).  The plain-FP64 path is timed on the
same workload beside it (``fp64``).

Every leg runs W warm-up steps from rest and then K timed steps, all at one
fixed time step (``config.dt``; 1e-3 on the rock, below the CFL-0.5 limit
of its developed flow, which the line reports as ``dt_cfl05_after``),
so the mixed, FP64 and learned legs advance the same state and their ratios
are like for like; ``config.momentum_precond`` says which momentum
preconditioner that dt selects.

Metric: cell-steps/s (cells x steps / device time of the timed steps,
CUDA events on the caller's stream; each step is one CUDA-graph replay with
device-side solver loops).  Inputs stay resident in HBM and exceed L2 (each
FP64 field is 134 MB), so no L2 flush is used.  The roofline figure comes
from a short window after the timed steps in which the dominant kernel's
launches are bracketed by CUDA events (eager launch sequence, same kernels).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W]
                       [--impl ours|reference] [--workload rock256|micromodel|calcite]
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

# Hardware work queues of this process's CUDA context (read when the context
# is created): the 64-instance batch replays one graph branch per instance,
# and 32 queues instead of the default 8 let more branches run at once
# (measured 250.5 -> 222.2 ms per batch step; the single-grid steps do not
# change).  A per-process setting, not a device setting.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2204_07019_gb300 import inputs as I  # noqa: E402

METRIC = "cell-steps/s at 1e-8 residual"
UNIT = "cell-steps/s"


def workload(name, size=256):
    """(eps_s, params, description) of a named workload (``size`` scales the
    rock; radii scale with it so that the pore structure is the same)."""
    if name == "rock256":
        r = 12.0 * size / 256.0
        es = I.sphere_rock_3d(size, seed=0, median_r=r)
        prm = I.make_params(es.shape, Pe=10.0, Da=1.0, L=2.0 * r, method="ivos", precision=1)
        desc = f"3D sphere rock {size}^3, porosity 0.20, Pe=10, Da=1, iVoS"
    elif name == "micromodel":
        es = I.disc_micromodel_2d(1024, 512, seed=0)
        prm = I.make_params(es.shape, Pe=100.0, Da=1.0, L=40.0, method="ivos", precision=1)
        desc = "2D polydisperse discs 1024x512, porosity 0.60, Pe=100, Da=1, iVoS"
    elif name == "calcite":
        es = I.calcite_post_2d()
        prm = I.make_params(es.shape, Pe=1.0, Da=0.1, L=32.0, method="ivos", precision=0)
        desc = "2D calcite post 256x64, Pe=1, Da=0.1, iVoS"
    else:
        raise SystemExit(f"unknown workload {name}")
    prm.update(p_rtol=1e-8, u_rtol=1e-8, c_rtol=1e-10, max_iter=2000)
    # the pressure correction starts from the previous step's correction
    # (VOS_PRECOND_P_WARM: 64 -> 57.4 iterations per step on the rock, 109.1
    # -> 104.0 ms) and the momentum solves from 2 u^n - u^{n-1}
    # (VOS_PRECOND_U_EXTRAP: 44.1 -> 42.9 iterations, 104.0 -> 103.2 ms)
    prm["precond"] = int(prm.get("precond", 0)) | 8 | 16
    return es, prm, desc


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None
        self.th = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        if self.th is not None:
            self.th.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "", 1).isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "", 1).isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def init_dist(world, device):
    if world <= 1:
        return None
    import torch.distributed as dist
    dist.init_process_group("nccl" if device.type == "cuda" else "gloo")
    return dist


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


TRAFFIC_PER_ALG_BYTE = {
    # DRAM bytes (read + write) per algorithmic byte from one ncu capture of
    # the bench workload at 192^3 (7,077,888 cells, above L2, about 4.8 GB on
    # the device), scaled to a launch by the units processed: the reads scale
    # exactly (every input word once); the part of the writes that reaches
    # DRAM inside the launch depends on the L2, so the write part is an
    # estimate.
    # FP32 x/r update: 113.28 MB read (16 B per unknown) + 9.04 MB written
    # against 24 B per unknown
    "pcg_xr_f32_L0": ((113283840.0 + 9038848.0) / (24.0 * 7077888.0), "ncu dram bytes of a 192^3 launch scaled by units"),
    # matrix-free pressure Jacobi sweep (four cells per thread): 84.95 MB read
    # (12.0 B per cell) + 6.61 MB written against 16 B per cell
    "mg_jac_mf_f32_L0": ((84949248.0 + 6610688.0) / (16.0 * 7077888.0), "ncu dram bytes of a 192^3 launch scaled by cells"),
    # two-kernel diagonal PCG (momentum), mean of eight launches each:
    # x/r update + preconditioner: 141.61 MB read (20.0 B per unknown) +
    # 31.93 MB written against 32 B per unknown; direction update + matvec:
    # 84.98 MB read (12.0 B) + 20.85 MB written against 20 B per unknown
    "pcg_xrz_f32_L0": ((141609984.0 + 31928000.0) / (32.0 * 7077888.0),
                       "ncu dram bytes of 192^3 launches scaled by units"),
    "pcg_pmv_mfc_f32_L0": ((84976992.0 + 20846368.0) / (20.0 * 7077888.0),
                           "ncu dram bytes of 192^3 launches scaled by units"),
}


# Fixed time steps: on the rock 1e-3 lies below the CFL-0.5 limit of the
# interstitial speed that vos_suggest_dt reports once the flow has developed
# (1.2e-3 measured after 7 steps at 2.5e-3).
DEFAULT_DT = {"rock256": 1.0e-3, "micromodel": 0.02, "calcite": 0.25}


def _stats_row(s):
    return (s["iters_u"], s["iters_p"], s["iters_c"], s["res_p"], s["outer_u"], s["outer_p"], s["outer_c"])


def time_gpu(V, es, prm, steps, warmup, dt, torch, profile=True, keep_fields=False):
    """Create, run ``warmup`` untimed steps from rest, time ``steps`` steps
    with CUDA events (all at the same fixed dt), then -- untimed -- take a
    per-kernel breakdown of one step and event-time the dominant kernel's
    launches over a few more steps."""
    h = V.vos_create(es, prm)
    try:
        for _ in range(warmup):
            V.vos_step(h, dt)
        # timed steps: CUDA-graph replay (default launch mode), no per-kernel timing
        stream = torch.cuda.current_stream()
        iters = []
        l0 = V.vos_kernel_launches()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            V.vos_step(h, dt)
            iters.append(_stats_row(V.vos_get_stats(h)))
        e1.record(stream)
        torch.cuda.synchronize()
        launches = V.vos_kernel_launches() - l0
        ms = e0.elapsed_time(e1) / steps
        final = V.vos_get_stats(h)
        fields = V.vos_fields(h, ("eps", "c", "u", "p")) if keep_fields else None
        dt_cfl = V.vos_suggest_dt(h, 0.5, 0.005)
        breakdown, top, roof = None, None, None
        if profile:
            V.vos_prof_reset()
            V.vos_prof_enable("*")
            torch.cuda.synchronize()
            e0.record()
            V.vos_step(h, dt)
            e1.record()
            torch.cuda.synchronize()
            step_ms = e0.elapsed_time(e1)
            rep = V.vos_prof_report()
            V.vos_prof_enable(None)
            V.vos_prof_reset()
            tot = sum(v[1] for v in rep.values())
            breakdown = sorted(({"kernel": k, "launches": v[0], "ms": v[1], "share": v[1] / tot if tot else 0.0,
                                 "gbs": v[2] / (v[1] * 1e6) if v[1] > 0 else None} for k, v in rep.items()),
                               key=lambda r: -r["ms"])
            top = breakdown[0]["kernel"] if breakdown else None
            breakdown = {"step_ms_profiled": step_ms, "kernel_ms_sum": tot, "kernels": breakdown[:48]}
        if top:
            # roofline window: further steps with the dominant kernel's
            # launches bracketed by CUDA events on the launching stream
            # (per-kernel timing uses the eager launch sequence)
            V.vos_prof_reset()
            V.vos_prof_enable(top)
            for _ in range(max(2, min(steps, 4))):
                V.vos_step(h, dt)
            rep = V.vos_prof_report()
            V.vos_prof_enable(None)
            V.vos_prof_reset()
            n, kms, kbytes = rep.get(top, (0, 0.0, 0.0))
            peak, src = measured_peaks()
            if n > 0 and kms > 0:
                ach = kbytes / (kms * 1e-3) / 1e9
                tr = TRAFFIC_PER_ALG_BYTE.get(top)
                traffic = kbytes / n * tr[0] if tr else None
                roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                        "traffic": traffic, "kernel": top, "launches": n, "avg_launch_us": kms * 1e3 / n,
                        "alg_bytes_per_launch": kbytes / n, "peak_source": src,
                        "window": "steps after the timed ones, same handle and dt, kernel launches event-timed",
                        "traffic_source": tr[1] if tr else None}
        tiles = {}
        for lev in (0, 1):
            try:
                tx, ty, zc, tuned = V.vos_tile_config(h, 3, lev)
                tiles["p_L%d" % lev] = {"tile": [tx, ty], "zc": zc, "tuned": bool(tuned)}
            except V.VosError:
                pass
        return dict(ms=ms, dt=dt, iters=iters, dev_bytes=V.vos_device_bytes(h), breakdown=breakdown,
                    roofline=roof, launches=launches, tiles=tiles, final=final, fields=fields, dt_cfl=dt_cfl)
    finally:
        V.vos_destroy(h)


def _gen_rock(args):
    size, seed, r = args
    return I.sphere_rock_3d(size, seed=seed, median_r=r)


def _gen_batch_item(args):
    seed, b, nx, ny = args
    return I.disc_micromodel_2d(nx, ny, seed=seed * 1000 + b + 1)


def _spawn_map(fn, items):
    """Seeded geometry generators are numpy-only; run them in a pool of
    spawned processes (a process forked after CUDA initialisation may hang)."""
    import multiprocessing as mp
    n = min(len(items), max(1, (os.cpu_count() or 1)), 16)
    if n <= 1:
        return [fn(a) for a in items]
    with mp.get_context("spawn").Pool(n) as pool:
        return pool.map(fn, items)


def mom_precond_name(prm, dt):
    """Which momentum preconditioner vos_step picks (include/vos.h rule)."""
    fl = int(prm.get("precond", 0))
    if fl & 2:
        return "diag"
    if fl & 4:
        return "mg"
    return "mg" if 2.0 * prm["dim"] * prm["nu"] * dt / prm["dx"] ** 2 > 30.0 else "diag"


def measured_bf16_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, "fallback"


def _unet_eval(V, es, prm, dt, steps, warmup, params, torch):
    """Steps of the workload with a network of the given parameters attached
    to the pressure solve (flexible CG, MG-PCG fallback; eager launches):
    ms per step and iteration counts."""
    net = V.UNet(es.shape, train=False)
    net.set_params(params)
    h = V.vos_create(es, prm)
    try:
        for _ in range(max(warmup - 1, 0)):
            V.vos_step(h, dt)
        V.vos_set_unet_preconditioner(h, net)
        V.vos_step(h, dt)  # last warm-up step, with the network
        stream = torch.cuda.current_stream()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        its, nets, fbs = [], [], []
        e0.record(stream)
        for _ in range(steps):
            V.vos_step(h, dt)
            s = V.vos_get_stats(h)
            ni, fb = V.vos_unet_solve_stats(h)
            its.append(s["iters_p"])
            nets.append(ni)
            fbs.append(fb)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        V.vos_prof_reset()
        V.vos_prof_enable("unet_conv")
        V.vos_step(h, dt)
        rep = V.vos_prof_report()
        V.vos_prof_enable(None)
        V.vos_prof_reset()
    finally:
        V.vos_destroy(h)
        net.close()
    return ms, its, nets, fbs, rep


def learned_leg(V, es, prm, dt, steps, warmup, torch, train_size=128, seeds=tuple(range(1, 21)), adam_per_seed=12,
                lr=2e-3, init_seed=0):
    """The learned pressure preconditioner under the held-out protocol:
    train the U-Net with the library's own kernels on MG-PCG residual
    snapshots of short runs on independently seeded rocks (seeds 1-20,
    train_size^3, the same generator and parameters), then evaluate it on
    the workload's own rock (seed 0, not seen in training) against the
    untrained network and against MG-PCG alone, at the same dt and step
    sequence.  Also the tensor-core convolution throughput."""
    t0 = time.time()
    net_t = V.UNet((train_size,) * 3, train=True)
    p0 = V.UNet.he_init(init_seed)
    net_t.set_params(p0)
    snap_iters = [0, 2, 5, 10, 20, 40]
    losses = []
    r = 12.0 * train_size / 256.0
    rocks = _spawn_map(_gen_rock, [(train_size, sd, r) for sd in seeds])
    for seed, est in zip(seeds, rocks):
        prt = dict(prm)
        prt.update(nx=train_size, ny=train_size, nz=train_size)
        h = V.vos_create(est, prt)
        try:
            for _ in range(max(warmup, 1)):
                V.vos_step(h, dt)
            snaps = torch.empty((len(snap_iters), train_size ** 3), dtype=torch.float32, device="cuda")
            V.vos_pressure_snapshots(h, snap_iters, snaps)
            for k in range(adam_per_seed):
                losses.append(net_t.train_step(h, snaps[k % len(snap_iters)], lr))
        finally:
            V.vos_destroy(h)
    params = net_t.get_params()
    net_t.close()
    torch.cuda.synchronize()
    train_s = time.time() - t0
    ms, its, nets, fbs, rep = _unet_eval(V, es, prm, dt, steps, warmup, params, torch)
    ms_u, its_u, nets_u, fbs_u, _ = _unet_eval(V, es, prm, dt, steps, warmup, p0, torch)
    nconv, cms, cflops = rep.get("unet_conv", (0, 0.0, 0.0))
    peak, src = measured_bf16_peak()
    tf = cflops / (cms * 1e-3) / 1e12 if cms > 0 else None
    return {"ms_per_step": ms, "value": es.size / (ms * 1e-3), "iters_p_mean": float(np.mean(its)),
            "net_iters_mean": float(np.mean(nets)), "fallbacks": int(sum(fbs)), "steps": steps,
            "untrained": {"ms_per_step": ms_u, "iters_p_mean": float(np.mean(its_u)),
                          "net_iters_mean": float(np.mean(nets_u)), "fallbacks": int(sum(fbs_u))},
            "train": {"protocol": f"snapshots of {len(seeds)} seeded {train_size}^3 rocks (seeds "
                                  f"{seeds[0]}-{seeds[-1]}); evaluated on the held-out seed-0 rock",
                      "seconds": train_s, "adam_steps": len(losses), "snapshot_iters": snap_iters,
                      "loss_first": float(np.mean(losses[:6])), "loss_last": float(np.mean(losses[-6:]))},
            "conv": {"launches": nconv, "ms": cms, "tflops": tf, "peak_tflops": peak, "peak_source": src,
                     "frac": (tf / peak) if tf else None, "bound": "tensor"}}


def batch_workload(count=64):
    """64 disc micromodels, side lengths U[128, 768], log-uniform Pe in [1, 100]
    and Da in [0.01, 100], iVoS, mixed precision (the draws of
    inputs.batched_micromodels, geometries generated in parallel)."""
    rng = np.random.default_rng(0)
    draws = []
    for b in range(count):
        nx, ny = (int(v) for v in rng.integers(128, 768 + 1, size=2))
        Pe = float(10 ** rng.uniform(0.0, 2.0))
        Da = float(10 ** rng.uniform(-2.0, 2.0))
        draws.append((nx, ny, Pe, Da))
    geoms = _spawn_map(_gen_batch_item, [(0, b, nx, ny) for b, (nx, ny, _, _) in enumerate(draws)])
    items = [(es, Pe, Da) for es, (_, _, Pe, Da) in zip(geoms, draws)]
    eps, prms = [], []
    for es, Pe, Da in items:
        p = I.make_params(es.shape, Pe=Pe, Da=Da, L=40.0, method="ivos", precision=1)
        p.update(p_rtol=1e-8, u_rtol=1e-8, c_rtol=1e-10, max_iter=2000)
        eps.append(es)
        prms.append(p)
    return eps, prms


def time_batch(V, eps, prms, steps, warmup, torch, nthreads=16, dt=0.02):
    b = V.vos_batch_create(eps, prms, nthreads=nthreads)
    try:
        dts = [dt] * len(eps)
        for _ in range(max(warmup, 1)):
            V.vos_batch_step(b, dts)
        l0 = V.vos_kernel_launches()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        status = [V.vos_batch_step(b, dts) for _ in range(steps)]
        e1.record()
        torch.cuda.synchronize()
        launches = V.vos_kernel_launches() - l0
        ms = e0.elapsed_time(e1) / steps
        its = [V.vos_get_stats(h) for h in b.handles]
        return dict(ms=ms, launches=launches, status=status,
                    iters_p_mean=float(np.mean([s["iters_p"] for s in its])),
                    dt_range=[min(dts), max(dts)])
    finally:
        V.vos_batch_destroy(b)


def _event_loop(V, h, steps, dt_fn, torch):
    stream = torch.cuda.current_stream()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    its = []
    e0.record(stream)
    for _ in range(steps):
        V.vos_step(h, dt_fn())
        s = V.vos_get_stats(h)
        its.append(s["iters_p"])
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / steps, float(np.mean(its))


def extra_workloads(V, torch, c1_steps=10, c3_steps=3):
    """The other configurations of the build, each measured briefly on the same
    GPU (the step count of each is part of its record):
    calcite post 256 x 64, FP64 iVoS, 50 steps with dt from vos_suggest_dt at
    CFL 0.5 (and App. D's 0.005); the 1024 x 512 disc micromodel in three
    (Pe, Da) regimes x three methods x {FP64, mixed}, fixed dt 0.05; the batch
    of 64 micromodels (one CUDA graph per batch step)."""
    out = {}
    es = I.calcite_post_2d()
    prm = I.make_params(es.shape, Pe=1.0, Da=0.1, L=32.0, method="ivos", precision=0)
    prm.update(p_rtol=1e-8, u_rtol=1e-8, c_rtol=1e-10, max_iter=2000)
    h = V.vos_create(es, prm)
    try:
        V.vos_step(h, 0.1)
        ms, ip = _event_loop(V, h, 50, lambda: min(V.vos_suggest_dt(h, 0.5, 0.005), 1.0), torch)
        s = V.vos_get_stats(h)
        out["calcite_256x64_fp64_ivos"] = {"steps": 50, "ms_per_step": ms, "cell_steps_per_s": es.size / (ms * 1e-3),
                                           "iters_p_mean": ip, "t_end": s["t"], "porosity": s["porosity"],
                                           "dt": "vos_suggest_dt(0.5, 0.005) per step"}
    finally:
        V.vos_destroy(h)
    es = I.disc_micromodel_2d(1024, 512, seed=0)
    rows = []
    for Pe, Da in ((1.0, 0.1), (100.0, 1.0), (100.0, 100.0)):
        for method in ("psi", "psi_prime", "ivos"):
            for prec in (0, 1):
                prm = I.make_params(es.shape, Pe=Pe, Da=Da, L=40.0, method=method, precision=prec)
                prm.update(p_rtol=1e-8, u_rtol=1e-8, c_rtol=1e-10, max_iter=2000)
                h = V.vos_create(es, prm)
                try:
                    for _ in range(2):
                        V.vos_step(h, 0.05)
                    ms, ip = _event_loop(V, h, c1_steps, lambda: 0.05, torch)
                finally:
                    V.vos_destroy(h)
                rows.append({"Pe": Pe, "Da": Da, "method": method, "precision": "mixed" if prec else "fp64",
                             "ms_per_step": round(ms, 3), "cell_steps_per_s": es.size / (ms * 1e-3),
                             "iters_p_mean": ip})
    out["micromodel_1024x512"] = {"steps": c1_steps, "warmup": 2, "dt": 0.05, "runs": rows}
    eps, prms = batch_workload(64)
    r = time_batch(V, eps, prms, c3_steps, 2, torch, dt=0.02)
    N = int(sum(e.size for e in eps))
    out["batch64_micromodels"] = {"steps": c3_steps, "warmup": 2, "dt": 0.02, "cells": N, "ms_per_batch_step": r["ms"],
                                  "cell_steps_per_s": N / (r["ms"] * 1e-3), "iters_p_mean": r["iters_p_mean"]}
    return out


def time_e2e(V, es, prm, steps, dt):
    """End to end through the C ABI with host buffers: create from host eps_s,
    ``steps`` steps, copy eps and c back; wall clock."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = V.vos_create(es, prm)
    for _ in range(steps):
        V.vos_step(h, dt)
    f = V.vos_fields(h, ("eps", "c"))
    V.vos_destroy(h)
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    n = es.size
    return {"value": n * steps / (t1 - t0), "unit": UNIT, "h2d_bytes_per_step": int(n * 8 / steps),
            "d2h_bytes_per_step": int(2 * n * 8 / steps), "steps": steps, "checksum": float(f["c"].sum())}


def oracle_sample(es, prm, dt, budget_s=20.0, crop=40):
    """The CPU oracle on a bounded crop (crop^3 for 3D, crop x crop... for 2D)
    of the same geometry and parameters; returns (cell-steps/s, steps, shape,
    wall seconds, threads used = process CPU time / wall time over the timed
    steps, at least 1)."""
    from oracle import vos_oracle as O
    nz, ny, nx = es.shape
    if nz > 1:
        sub = np.ascontiguousarray(es[:crop, :crop, :crop])
    else:
        sub = np.ascontiguousarray(es[:, : min(ny, 4 * crop), : min(nx, 4 * crop)])
    p = dict(prm)
    p.update(nz=sub.shape[0], ny=sub.shape[1], nx=sub.shape[2])
    st = O.init_state(sub, p)
    t0 = time.perf_counter()
    c0 = time.process_time()
    n = 0
    while True:
        st, _ = O.step(st, dt, p, solver="iterative", rtol=p["p_rtol"])
        n += 1
        if time.perf_counter() - t0 > budget_s or n >= 20:
            break
    dt = time.perf_counter() - t0
    cores = max(1, int(round((time.process_time() - c0) / dt)))
    return sub.size * n / dt, n, sub.shape, dt, cores


def reference_arm(args, rank, world):
    """The CPU oracle as it stands, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    es, prm, desc = workload(args.workload, args.size)
    dt_step = args.dt if args.dt else DEFAULT_DT[args.workload]
    cells = []
    for _ in range(max(args.warmup, 0)):
        oracle_sample(es, prm, dt_step, budget_s=2.0)
    rates, used = [], []
    for _ in range(args.steps):
        r, n, shp, dt, cores = oracle_sample(es, prm, dt_step, budget_s=5.0)
        rates.append(r)
        cells.append(shp)
        used.append(cores)
    v = float(np.mean(rates))
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "higher_is_better": True, "scaling": "weak",
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "desc": desc, "dt": dt_step},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": max(used), "kind": "oracle",
                            "sample": f"oracle step(s) on a {cells[0]} crop of the workload geometry, "
                                      "scipy CG/BiCGStab to the same tolerances, ~5 s per timed step"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rock256", choices=["rock256", "micromodel", "calcite", "batch64"])
    ap.add_argument("--size", type=int, default=256, help="edge of the rock workload (profiling runs only)")
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="0 skips the FP64 leg; otherwise it runs the same W + K steps as the mixed leg")
    ap.add_argument("--dt", type=float, default=None, help="fixed time step of every leg (default per workload)")
    ap.add_argument("--mom-precond", default="auto", choices=["auto", "diag", "mg"],
                    help="momentum preconditioner: the library's rule, or forced")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the brief measurements of the other configurations (calcite post, micromodel grid, "
                         "batch of 64)")
    ap.add_argument("--p-cold", action="store_true",
                    help="start each pressure-correction solve from zero instead of the previous step's correction")
    ap.add_argument("--u-plain", action="store_true",
                    help="start each momentum solve from u^n instead of the extrapolation 2 u^n - u^{n-1}")
    ap.add_argument("--scalar-sweeps", action="store_true",
                    help="one cell per thread in the matrix-free pressure sweeps (same results; for comparison)")
    ap.add_argument("--fused-mask", type=int, default=None,
                    help="vos_set_fused_pcg mask (default: the library's, all fused forms)")
    ap.add_argument("--four-kernel-pcg", action="store_true",
                    help="the FP32 inner Krylov solves with separate kernels (vos_set_fused_pcg(0)) instead of "
                         "the fused forms (for comparison)")
    ap.add_argument("--coarse-cycle", action="store_true",
                    help="run the coarse multigrid levels as one cluster launch per V-cycle instead of one "
                         "launch per operation (same results; for comparison)")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-preconditioner leg")
    ap.add_argument("--eager", action="store_true",
                    help="launch the step's kernels one by one instead of replaying CUDA graphs "
                         "(the same kernels; for profilers)")
    args = ap.parse_args()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    import torch
    from paper_2204_07019_gb300 import build_lib
    from paper_2204_07019_gb300 import vos as V
    if rank == 0 or world == 1:
        build_lib.build()
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    dist = init_dist(world, device)
    if dist is not None:
        dist.barrier()
    V.load_library()
    if args.eager:
        V.vos_set_launch_mode(0)
    if args.coarse_cycle:
        V.vos_set_coarse_cycle(1)
    if args.scalar_sweeps:
        V.vos_set_vector_sweeps(0)
    if args.four_kernel_pcg:
        V.vos_set_fused_pcg(0)
    elif args.fused_mask is not None:
        V.vos_set_fused_pcg(args.fused_mask)
    if args.workload == "batch64":
        eps, prms = batch_workload(64)
        N = int(sum(e.size for e in eps))
        clocks = ClockSampler(local)
        clocks.start()
        r = time_batch(V, eps, prms, args.steps, args.warmup, torch, dt=args.dt or 0.02)
        ck = clocks.stop()
        out = {"metric": METRIC, "value": N / (r["ms"] * 1e-3), "unit": UNIT, "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": r["ms"], "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
               "config": {"workload": "batch64", "desc": "64 disc micromodels, sides U[128,768], Pe U_log[1,100], "
                          "Da U_log[0.01,100], iVoS, mixed; each batch step one CUDA graph with "
                          "every instance as a parallel branch",
                          "cells": N, "dt_range": r["dt_range"]},
               "gpu_launches": r["launches"], "iters_p_mean": r["iters_p_mean"], "clocks": ck,
               "roofline": None}
        if rank == 0:
            print(json.dumps(out), flush=True)
        return
    es, prm, desc = workload(args.workload, args.size)
    if args.mom_precond != "auto":
        prm["precond"] = int(prm.get("precond", 0)) | (2 if args.mom_precond == "diag" else 4)
    if args.p_cold:
        prm["precond"] = int(prm.get("precond", 0)) & ~8
    if args.u_plain:
        prm["precond"] = int(prm.get("precond", 0)) & ~16
    dt = args.dt if args.dt else DEFAULT_DT[args.workload]
    N = es.size
    clocks = ClockSampler(local)
    if dist is not None:
        dist.barrier()
    clocks.start()
    r = time_gpu(V, es, prm, args.steps, args.warmup, dt, torch, keep_fields=args.fp64_steps > 0)
    ck = clocks.stop()
    ms, iters = r["ms"], r["iters"]
    t = torch.tensor([ms], device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
    ms = float(t.item())
    value = N * world / (ms * 1e-3)
    # FP64-only solver leg: same workload, dt and step sequence (warm-up W,
    # then K timed steps), so its fields after W + K steps are the FP64
    # counterpart of the mixed leg's (--fp64-steps 0 skips it)
    r64, prec = None, None
    if args.fp64_steps > 0:
        p64 = dict(prm)
        p64["precision"] = 0
        r64 = time_gpu(V, es, p64, args.steps, args.warmup, dt, torch, profile=False, keep_fields=True)
        f32, f64 = r["fields"], r64["fields"]
        prec = {"steps": args.warmup + args.steps,
                "porosity_err": abs(r["final"]["porosity"] - r64["final"]["porosity"]),
                "rel_l2": {n: float(np.linalg.norm(f32[n] - f64[n]) / max(np.linalg.norm(f64[n]), 1e-300))
                           for n in f64},
                "reference": "the FP64 GPU path (parity-tested against the FP64 oracle to 1e-9) after the same steps"}
    e2e = time_e2e(V, es, prm, max(2, args.steps // 2), dt)
    learned = None
    if not args.no_learned and es.ndim == 3 and min(es.shape) >= 64:
        learned = learned_leg(V, es, prm, dt, 3, args.warmup, torch,
                              train_size=min(128, es.shape[0]))
        learned["vs_fp64"] = learned["value"] / (N / (r64["ms"] * 1e-3)) if r64 else None
        learned["vs_mixed"] = learned["value"] / (N / (r["ms"] * 1e-3))
        learned["mgpcg_iters_p_mean"] = float(np.mean([i[1] for i in iters]))
    fp64_value = N * world / (r64["ms"] * 1e-3) if r64 else None
    mom = mom_precond_name(prm, dt)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
           "config": {"workload": args.workload, "desc": desc, "cells": N, "dt": dt,
                      "dt_rule": "fixed for every leg and step (warm-up from rest included)",
                      "dt_cfl05_after": r["dt_cfl"],
                      "p_rtol": prm["p_rtol"], "u_rtol": prm["u_rtol"], "c_rtol": prm["c_rtol"],
                      "momentum_precond": mom, "precond_flags": int(prm.get("precond", 0)),
                      "residual": "diagonally scaled, FP64",
                      "l2": "inputs larger than L2 (no flush)", "parallelism": f"replicas{world}",
                      "launch": "eager" if args.eager else "graph", "tiles": r["tiles"],
                      "coarse_cycle": "cluster-resident" if args.coarse_cycle else "separate launches",
                      "fused_mask": 0 if args.four_kernel_pcg else (7 if args.fused_mask is None else args.fused_mask)},
           "roofline": r["roofline"], "gpu_launches": r["launches"],
           "fp64_value": fp64_value, "fp64_ms_per_step": r64["ms"] if r64 else None,
           "mixed_vs_fp64": (value / fp64_value) if fp64_value else None,
           "learned_value": learned["value"] if learned else None,
           "learned_vs_fp64": learned["vs_fp64"] if learned else None,
           "iters_p": float(np.mean([i[1] for i in iters])),
           "iters_u": [float(np.mean([i[0][a] for i in iters])) for a in range(3)],
           "porosity_err": prec["porosity_err"] if prec else None,
           "fp64": ({"value": fp64_value, "ms_per_step": r64["ms"],
                     "iters_p_mean": float(np.mean([i[1] for i in r64["iters"]]))} if r64 else None),
           "mixed_precision_error": prec,
           "solver": {"iters_u_mean": [float(np.mean([i[0][a] for i in iters])) for a in range(3)],
                      "iters_p_mean": float(np.mean([i[1] for i in iters])),
                      "iters_c_mean": float(np.mean([i[2] for i in iters])),
                      "res_p_max": float(max(i[3] for i in iters)),
                      "outer_passes_mean": {"u": [float(np.mean([i[4][a] for i in iters])) for a in range(3)],
                                            "p": float(np.mean([i[5] for i in iters])),
                                            "c": float(np.mean([i[6] for i in iters]))}},
           "device_bytes": r["dev_bytes"], "e2e": e2e, "clocks": ck, "learned": learned,
           "breakdown": r["breakdown"]}
    if rank == 0 and not args.no_extra and args.workload == "rock256":
        out["workloads"] = extra_workloads(V, torch)
    if rank == 0 and not args.no_cpu:
        r, n, shp, dtc, cores = oracle_sample(es, prm, dt, budget_s=15.0)
        out["cpu_baseline"] = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                               "sample": f"{n} oracle step(s) on a {tuple(shp)} crop of the same geometry "
                                         f"({dtc:.1f} s), scipy CG/BiCGStab at the same tolerances"}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
