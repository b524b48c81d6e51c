#!/usr/bin/env python
"""Benchmark: gradient Gcell-updates/s of the superposition adjoint method.

One step = one full wave_adjoint_sensitivity call over the workload (all
shots: forward, superposed backward pass, sensitivity, misfit).  One gradient
cell-update = one cell advanced one time step in both passes, so a step is
worth sum_s ncells * N_s units.

Default workload: 3D 512^3, 8th order, layered velocity, 16 shots with record
lengths 1500-2500 (the batched multi-shot configuration).  Inputs are resident
in HBM before the timed region; the state of one shot (2 x 537 MB) and the
coefficient and accumulator grids are each larger than the 129 MB L2.

`--impl reference` times the FP64 CPU oracle on a bounded sample of the same
workload (the reference arm); it never touches the GPU.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "gradient Gcell-updates/s (fwd+adjoint+sens), % HBM roofline, batched vs plain"
UNIT = "Gcell-updates/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="w2", choices=["w0", "w1", "w2", "w3", "w4"])
    ap.add_argument("--mode", default="auto", choices=["auto", "plain", "batched"])
    ap.add_argument("--forward-curve", action="store_true",
                    help="forward time per step versus grid size (2D and 3D, order 2) instead of the benchmark")
    ap.add_argument("--grad-mode", default="superposition", choices=["superposition", "symmetric", "reverse"],
                    help="gradient: Algorithm 1, the +-k mean, or the two-field reverse-time adjoint "
                         "(the last two are exact and run shot by shot)")
    ap.add_argument("--kahan", dest="kahan", action="store_true", default=None,
                    help="Kahan-compensated sensitivity (default: on for w4, whose configuration names it)")
    ap.add_argument("--no-kahan", dest="kahan", action="store_false")
    ap.add_argument("--k-ratio", type=float, default=None,
                    help="ratio r of the automatic k = r |psi| / |f_adj| (default: the library's, 1e-2 for the "
                         "velocity form); it sets the accuracy against the exact gradient, not the speed")
    ap.add_argument("--tiling", default=None,
                    help="zblock:rows:depth:pipeline for the 3D step kernel instead of the autotuner's pick")
    ap.add_argument("--cta-order", type=int, default=None, choices=[0, 1],
                    help="launch order of the 3D step CTAs (0 z-block fastest, 1 plane-major) instead of the "
                         "autotuner's pick (with --tiling: default 1)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain-path comparison")
    ap.add_argument("--no-graph", action="store_true", help="time eager calls instead of CUDA-graph replays")
    ap.add_argument("--storage", default="f32", choices=["f32", "bf16", "f16"],
                    help="storage type of the resident time levels (stencil arithmetic stays FP32)")
    ap.add_argument("--compare-exact", action="store_true",
                    help="after the timed region, the exact discrete gradient (the history-free +-k mean and, "
                         "where it fits, the stored-history adjoint) as the reference of the timed result")
    ap.add_argument("--fd-check", action="store_true",
                    help="after the timed region, a central finite difference of C along a smooth random "
                         "direction against <grad, direction>")
    ap.add_argument("--refined-data", action="store_true",
                    help="observed data from the true model on a grid twice as fine with twice the steps "
                         "(no inverse crime), generated with the GPU forward")
    # reduced sizes, for profiling captures only (the line is marked "reduced")
    ap.add_argument("--shape", default=None, help="override the grid shape, e.g. 256,256,256")
    ap.add_argument("--shots", type=int, default=None, help="use the first K shots")
    ap.add_argument("--nt", type=int, default=None, help="override every record length")
    return ap.parse_args()


def make_workload(name, shape=None, shots=None, nt=None):
    from paper_2509_15744_gb300 import workloads as WL
    if shape is not None:
        shape = tuple(int(v) for v in shape.split(","))
        if name == "w2":
            wl = WL.workload2(shape=shape)
        elif name == "w0":
            wl = WL.workload0(n=shape[0])
        elif name == "w1":
            wl = WL.workload1(n=shape[0])
        elif name == "w3":
            wl = WL.workload3(n=shape[0])
        else:
            wl = WL.workload4(n=shape[0])
    else:
        wl = {"w0": WL.workload0, "w1": WL.workload1, "w2": WL.workload2, "w3": WL.workload3,
              "w4": WL.workload4}[name]()
    if shots is not None:
        wl.sources, wl.receivers, wl.nt = wl.sources[:shots], wl.receivers[:shots], wl.nt[:shots]
    if nt is not None:
        wl.nt = [int(nt)] * len(wl.nt)
    if shape is not None or shots is not None or nt is not None:
        wl.name += "_reduced"
    return wl


def units_of(wl):
    return float(sum(wl.ncells * n for n in wl.nt))


def aggregate(ms_local, units_local, dist=None, device=None):
    """Whole-job timing over ranks: the slowest rank's time and the sum of the
    units every rank processed (replicas: each rank runs its own copy of the
    workload, so there is no exchange on the data path)."""
    if dist is None:
        return ms_local, units_local
    import torch
    t = torch.tensor([ms_local], dtype=torch.float64, device=device)
    u = torch.tensor([units_local], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


# ---------------------------------------------------------------------------
# CPU oracle sample (cpu_baseline leg and the reference arm): the FP64 oracle
# on every host core, one process per core, each running Algorithm 1 for one
# shot on a crop of the workload
# ---------------------------------------------------------------------------
def _oracle_shot(job):
    """One process's share: Algorithm 1 (one shot, nt steps each way) on a
    crop; returns the seconds it took."""
    import numpy as np
    import oracle as O
    physics, param, h, order, bc, vmax, cfl, nt, seed = job
    shape = param.shape
    dt = O.cfl_dt(h, vmax, len(shape), order, cfl)
    med = O.Medium(physics, param, h, dt, order, bc)
    rng = np.random.default_rng(seed)
    mid = [int(rng.integers(n // 4, 3 * n // 4)) for n in shape]
    mid[0] = min(2, shape[0] - 1)
    src = int(np.ravel_multi_index(tuple(mid), shape))
    rec = np.arange(0, shape[-1], 2, dtype=np.int64)
    wav = np.ones(nt + 1)
    shot = O.Shot(src, wav, rec, np.zeros((len(rec), nt + 1)), 1.0)
    t0 = time.perf_counter()
    O.superposition_gradient(med, [shot], nt, 1.0)
    return time.perf_counter() - t0


def cpu_model():
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith(("model name", "cpu part")):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    import platform
    return platform.processor() or platform.machine()


class OracleSampler:
    """The oracle's Algorithm 1 on all host cores: `procs` processes (spawned,
    so safe after CUDA initialisation), each one shot of `nt` steps each way
    on a crop of the workload (3D: 128^3; 2D: 1024^2)."""

    def __init__(self, wl, nt=6, procs=None):
        import multiprocessing as mp
        import numpy as np
        self.procs = procs or (os.cpu_count() or 1)
        crop = 128 if wl.ndim == 3 else 1024
        shape = tuple(min(crop, n) for n in wl.shape)
        sl = tuple(slice(0, n) for n in shape)
        param = np.ascontiguousarray(np.asarray(wl.init_param)[sl]).astype(np.float64)
        self.jobs = [(wl.physics, param, wl.h, wl.order, wl.bc, wl.vmax, wl.cfl_fraction, nt, i)
                     for i in range(self.procs)]
        self.units = float(np.prod(shape)) * nt * self.procs
        self.desc = (f"FP64 numpy oracle, Algorithm 1, {self.procs} processes on {self.procs} host cores "
                     f"({cpu_model()}), each one shot of {nt} steps each way on a {'x'.join(map(str, shape))} "
                     f"crop of the workload")
        self.pool = mp.get_context("spawn").Pool(self.procs)

    def sample(self):
        """Wall seconds and gradient cell-updates/s of one round."""
        t0 = time.perf_counter()
        self.pool.map(_oracle_shot, self.jobs, chunksize=1)
        el = time.perf_counter() - t0
        return el, self.units / el / 1e9

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args, rank, world):
    if rank != 0:
        return
    wl = make_workload(args.workload, args.shape, args.shots, args.nt)
    sampler = OracleSampler(wl)
    rates, secs = [], []
    for i in range(args.warmup + args.steps):
        el, r = sampler.sample()
        if i >= args.warmup:
            rates.append(r)
            secs.append(el)
    sampler.close()
    value = statistics.median(rates)
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.median(secs),
        "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "shape": list(wl.shape), "order": wl.order, "physics": wl.physics,
                   "shots": wl.nshots, "nt_total": int(sum(wl.nt)), "mode": "oracle sample",
                   "sample": sampler.desc},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": sampler.procs, "kind": "oracle",
                         "sample": sampler.desc},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples (one CSV line per 200 ms) go to WAVE_BENCH_CLOCKS_DIR, else the temp directory
        out = os.environ.get("WAVE_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out, f"clocks_bench_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), float(parts[3]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return None
        sm = [r[0] for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for n, v in zip(names, r[3]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "power_w_max": max(r[2] for r in rows), "samples": len(rows), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def kernel_traffic(kernel_file, workload_name, tiling=None):
    """dram bytes per launch of the step kernel from a committed ncu summary
    (profiles/*_traffic.txt) taken on the current kernel source, this workload
    and (when the summary names one) this tiling, else None."""
    src = open(os.path.join(ROOT, "paper_2509_15744_gb300", "csrc", kernel_file), "rb").read()
    digest = hashlib.sha256(src).hexdigest()[:16]
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*_traffic.txt"))):
        vals = {}
        for line in open(path):
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":", 1)
                vals[k.strip()] = v.strip()
        if "tiling" in vals and tiling is not None and \
                [int(v) for v in vals["tiling"].split(",")] != [int(v) for v in tiling]:
            continue
        if vals.get("kernel_source_sha256_16") == digest and vals.get("workload") == workload_name:
            try:
                return float(vals["dram_bytes_per_launch_full_size"])
            except (KeyError, ValueError):
                return None
    return None


def forward_curve(W, torch, nt=40, warm=5):
    """Forward solver time per step versus cells (Sec. 3.2's computation-time
    study): 2D and 3D, order 2, velocity form, one point source and receiver,
    device-resident inputs, CUDA events around the forward call."""
    import numpy as np
    dev = torch.device("cuda")
    sides = {2: [128, 256, 512, 1024, 2048, 2896, 4096, 8192, 16384, 32768],
             3: [32, 64, 100, 128, 160, 200, 256, 320, 400, 512, 640, 800, 1024]}
    points = []
    for ndim, ns in sides.items():
        for n in ns:
            shape = (n,) * ndim
            cells = n ** ndim
            dt = W.cfl_dt(ndim, 2, 10.0, 3000.0, 0.5)
            v = torch.full(shape, 2500.0, device=dev)
            m = W.Model(v, 10.0, dt, 2, "velocity", "dirichlet")
            src = int(np.ravel_multi_index(tuple(s // 2 for s in shape), shape))
            wav = W.wavelet("ricker", 15.0, dt, nt, device=dev)
            rec = torch.tensor([src], dtype=torch.int64, device=dev)
            warm_shot = W.Shot(src, wav[: warm + 1].contiguous(), rec)
            m.forward([warm_shot])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            m.forward([W.Shot(src, wav, rec)])
            e1.record()
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / nt
            points.append({"ndim": ndim, "cells": cells, "ms_per_step": ms, "Gcell_steps_per_s": cells / ms / 1e6,
                           "working_set_MB": 16.0 * cells / 1e6})
            del m, v
            torch.cuda.empty_cache()
    print(json.dumps({"metric": "forward time per step vs cells (order 2, velocity)", "unit": "ms",
                      "points": points}), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import numpy as np
    import torch

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    import __graft_entry__ as ge
    ge.build()
    from paper_2509_15744_gb300 import wave as W
    if args.forward_curve:
        forward_curve(W, torch)
        return

    wl = make_workload(args.workload, args.shape, args.shots, args.nt)
    if args.kahan is None:
        args.kahan = args.workload == "w4"
    dt = W.cfl_dt(wl.ndim, wl.order, wl.h, wl.vmax, wl.cfl_fraction)
    batched_ok = wl.ndim == 3 and wl.physics == "velocity" and wl.nshots > 1
    mode = args.mode if args.mode != "auto" else ("batched" if batched_ok else "plain")
    if args.grad_mode != "superposition":
        mode = "plain"

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    # ---- inputs resident in HBM --------------------------------------------
    param0 = torch.from_numpy(np.ascontiguousarray(wl.init_param, dtype=np.float32)).to(dev)
    wk = {"ricker": "ricker", "sine_burst": "sine_burst"}[wl.wavelet.kind]
    wavs = [W.wavelet(wk, wl.wavelet.freq, dt, n, nc=wl.wavelet.nc, psi0=wl.wavelet.psi0, device=dev)
            for n in wl.nt]
    recs = [torch.from_numpy(r).to(dev) for r in wl.receivers]
    observed = [None] * wl.nshots
    if wl.objective == "l2" and args.refined_data:
        from paper_2509_15744_gb300 import workloads as WL
        fine = WL.refined(wl, 2)
        dtf = W.cfl_dt(fine.ndim, fine.order, fine.h, fine.vmax, fine.cfl_fraction)
        ptrue = torch.from_numpy(np.ascontiguousarray(fine.true_param, dtype=np.float32)).to(dev)
        mtrue = W.Model(ptrue, fine.h, dtf, fine.order, fine.physics, fine.bc)
        for i in range(wl.nshots):
            wf = W.wavelet(wk, fine.wavelet.freq, dtf, fine.nt[i], nc=fine.wavelet.nc, psi0=fine.wavelet.psi0,
                           device=dev)
            tr = mtrue.forward([W.Shot(fine.sources[i], wf, torch.from_numpy(fine.receivers[i]).to(dev))])[0]
            observed[i] = tr[:, ::2].contiguous()   # coarse level n = fine level 2n
        del mtrue, ptrue
    elif wl.objective == "l2":
        ptrue = torch.from_numpy(np.ascontiguousarray(wl.true_param, dtype=np.float32)).to(dev)
        mtrue = W.Model(ptrue, wl.h, dt, wl.order, wl.physics, wl.bc)
        for i in range(wl.nshots):
            observed[i] = mtrue.forward([W.Shot(wl.sources[i], wavs[i], recs[i])])[0]
        del mtrue, ptrue
    shots = [W.Shot(wl.sources[i], wavs[i], recs[i], observed[i]) for i in range(wl.nshots)]
    model = W.Model(param0, wl.h, dt, wl.order, wl.physics, wl.bc, kahan=args.kahan, storage=args.storage)
    gkw = dict(objective=wl.objective, patch_sign=wl.patch_sign, batched=(mode == "batched"), mode=args.grad_mode,
               k_ratio=args.k_ratio)
    from paper_2509_15744_gb300 import tune
    if args.tiling:
        tiling = tuple(int(v) for v in args.tiling.split(":"))
        model.set_tiling(*tiling)
    else:
        tiling = tune.tune(model, shots, batched=(mode == "batched"))
    if args.cta_order is not None:
        model.set_schedule(args.cta_order)
    cta_order = model.cta_order

    # ---- warm-up -----------------------------------------------------------
    for _ in range(args.warmup):
        model.gradient(shots, **gkw)
    barrier()
    W.timing_enable(True)   # creates the timing events (none may be created while capturing)
    launches_eager = W.launch_count()
    model.gradient(shots, **gkw)
    barrier()
    launches_per_call = W.launch_count() - launches_eager

    # ---- the timed step: replays of the gradient call captured in a CUDA
    # graph (the whole call: both passes, sparse kernels, misfit, k, finish);
    # the step-kernel events are captured too, so the replays time every
    # step launch (--no-graph: eager calls instead) --------------------------
    stream = torch.cuda.current_stream()
    use_graph = not args.no_graph
    graph = None
    W.timing_enable(True)
    if use_graph:
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            grad, mis, kd = model.gradient(shots, **gkw)
        graph.replay()   # one more warm-up, as a replay
        barrier()
    clocks = ClockSampler(local)
    clocks.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if not use_graph:
        W.timing_enable(True)
    barrier()
    torch.cuda.nvtx.range_push("timed")   # lets a profiler select the timed launches
    e0.record(stream)
    for _ in range(args.steps):
        if use_graph:
            graph.replay()
        else:
            grad, mis, kd = model.gradient(shots, **gkw)
    e1.record(stream)
    barrier()
    torch.cuda.nvtx.range_pop()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    step_ms, step_launches, step_bytes = W.timing_read()
    W.timing_enable(False)
    if use_graph:   # the events hold the last replay: one gradient call
        kernel_ms_per_call, calls_timed = step_ms, 1
    else:
        kernel_ms_per_call, calls_timed = step_ms / args.steps, args.steps
    launches = launches_per_call * args.steps
    grad_norm = float(model.grad_norm.item())   # FP64 device reduction of the finish pass
    misfit_val = float(mis.item())
    k_val = float(kd.item())
    grad = grad.clone()
    del graph
    ms, units = aggregate(ms, units_of(wl), dist, dev)
    value = units * args.steps / (ms / 1e3) / 1e9

    # ---- plain path (one shot per launch) over the same shots on the same GPU ------
    plain = None
    if mode == "batched" and not args.no_plain:
        plain_tiling = tune.tune(model, shots, batched=False) if not args.tiling else tiling
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        gp, mp_, kp = model.gradient(shots, objective=wl.objective, patch_sign=wl.patch_sign, k=k_val)
        b.record(stream)
        barrier()
        plain = {"value": units_of(wl) / (a.elapsed_time(b) / 1e3) / 1e9, "unit": UNIT, "shots": wl.nshots,
                 "tiling": list(plain_tiling),
                 "grad_rel_diff_vs_batched": float(torch.linalg.vector_norm((gp - grad).double()).item()) /
                 max(grad_norm, 1e-300)}
        plain["cta_order"] = model.cta_order
        model.set_tiling(*tiling)
        model.set_schedule(cta_order)

    # ---- end to end through the public API with host buffers ------------------
    e2e = None
    if not args.no_e2e:
        e2e_steps = min(args.steps, 3)
        h_param = torch.from_numpy(np.ascontiguousarray(wl.init_param, dtype=np.float32)).pin_memory()
        h_obs = [o.cpu().pin_memory() if o is not None else None for o in observed]
        h_wav = [w.cpu().pin_memory() for w in wavs]
        h_rec = [r.cpu().pin_memory() for r in recs]
        h_grad = torch.empty(wl.init_param.shape, dtype=torch.float32).pin_memory()
        h_mis = torch.empty(1, dtype=torch.float64).pin_memory()
        h2d = h_param.numel() * 4 + sum(o.numel() * 4 for o in h_obs if o is not None) + \
            sum(w.numel() * 4 for w in h_wav) + sum(r.numel() * 8 for r in h_rec)
        d2h = h_grad.numel() * 4 + 8
        barrier()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            p = h_param.to(dev, non_blocking=True)
            sh = [W.Shot(wl.sources[i], h_wav[i].to(dev, non_blocking=True), h_rec[i].to(dev, non_blocking=True),
                         h_obs[i].to(dev, non_blocking=True) if h_obs[i] is not None else None)
                  for i in range(wl.nshots)]
            m2 = W.Model(p, wl.h, dt, wl.order, wl.physics, wl.bc, kahan=args.kahan, storage=args.storage)
            m2.set_tiling(*tiling)
            m2.set_schedule(cta_order)
            g2, mi2, _ = m2.gradient(sh, **gkw)
            h_grad.copy_(g2, non_blocking=True)
            h_mis.copy_(mi2, non_blocking=True)
            torch.cuda.synchronize()
        barrier()
        el, _ = aggregate(time.perf_counter() - t0, 0.0, dist, dev)
        e2e = {"value": units * e2e_steps / el / 1e9, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
               "d2h_bytes_per_step": int(d2h), "steps": e2e_steps,
               "mode": "eager calls: model built from host buffers every step"}

    # ---- roofline of the dominant kernel (the fused step) ---------------------
    peak, peak_kind = measured_peak()
    achieved = step_bytes / (step_ms / 1e3) / 1e9 if step_ms > 0 else 0.0
    if wl.physics == "density":
        kfile = "step_density.cu"
    elif wl.ndim == 3:   # the 3D FP32 step kernel of the chosen pipeline
        kfile = {0: "step3d_ring.cu", 3: "step3d_queue.cu",
                 4: "step3d_pair.cu" if mode == "batched" else "step3d_queue.cu",
                 5: "step3d_stream.cu" if mode == "batched" else "step3d_queue.cu"}[tiling[3]]
    else:
        kfile = "step_velocity.cu"
    traffic = kernel_traffic(kfile, wl.name, tiling)
    nl = max(step_launches, 1)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_kind,
                "traffic": traffic,
                "algorithmic_bytes_per_launch": step_bytes / nl,
                "kernel": kfile.replace(".cu", ""), "launches_per_call": step_launches,
                "avg_launch_ms": step_ms / nl,
                "kernel_share_of_step": kernel_ms_per_call / (ms / args.steps) if ms > 0 else None,
                "timing": "CUDA events around every step launch of the last timed call"
                          if use_graph else "CUDA events around every step launch of the timed calls"}
    if traffic:
        # DRAM bytes actually moved, over the same launch time (re-reads count here)
        roofline["dram_achieved"] = traffic / (step_ms / nl / 1e3) / 1e9
        roofline["dram_frac"] = roofline["dram_achieved"] / peak
        roofline["traffic_source"] = "ncu capture on a smaller case of the same kernel, scaled by shot-cells"

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        sampler = OracleSampler(wl)
        sampler.sample()                 # worker start-up and imports
        _, r = sampler.sample()
        sampler.close()
        cpu = {"value": r, "unit": UNIT, "cores": sampler.procs, "kind": "oracle", "sample": sampler.desc}

    # ---- accuracy of the timed result at full size ----------------------------
    accuracy = None
    if args.compare_exact or args.fd_check:
        accuracy = {}
        gsum = torch.linalg.vector_norm(grad.double()).item()
        ref_model = model
        if args.storage != "f32":   # the references are computed with FP32 storage
            ref_model = W.Model(param0, wl.h, dt, wl.order, wl.physics, wl.bc, kahan=args.kahan)
            ref_model.set_tiling(*tiling)
            ref_model.set_schedule(cta_order)
        if args.compare_exact:
            gs, _, _ = ref_model.gradient(shots, objective=wl.objective, patch_sign=wl.patch_sign, mode="symmetric")
            barrier()
            ns = torch.linalg.vector_norm(gs.double()).item()
            dn = torch.linalg.vector_norm((grad - gs).double()).item()
            accuracy["exact_symmetric"] = {
                "rel_l2_of_timed_result": dn / ns if ns > 0 else None,
                "exact_norm": ns,
                "what": "exact discrete gradient from the +-k mean (history-free, pinned to the FP64 oracle)"}
            hist_bytes = (max(wl.nt) + 2) * wl.ncells * 4
            free, _ = torch.cuda.mem_get_info(dev)
            if wl.physics == "velocity" and hist_bytes < 0.8 * free:
                del model._gws
                model._gws = None
                a0, b0 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a0.record(stream)
                ge, _, _ = ref_model.gradient(shots, objective=wl.objective, patch_sign=wl.patch_sign, mode="exact")
                b0.record(stream)
                barrier()
                ne = torch.linalg.vector_norm(ge.double()).item()
                accuracy["exact_stored"] = {
                    "rel_l2_of_timed_result": torch.linalg.vector_norm((grad - ge).double()).item() / ne
                    if ne > 0 else None,
                    "rel_l2_symmetric_vs_stored": torch.linalg.vector_norm((gs - ge).double()).item() / ne
                    if ne > 0 else None,
                    "history_GB": hist_bytes / 1e9,
                    "Gcell_updates_per_s": units_of(wl) / (a0.elapsed_time(b0) / 1e3) / 1e9,
                    "what": "standard adjoint over the stored forward history (memory grows with N)"}
                del ge
                ref_model._gws = None
            del gs
        if args.fd_check:
            # C(p + e d) - C(p - e d) over 2e against <grad, d>, d smooth and random
            gen = torch.Generator(device=dev)
            gen.manual_seed(12)
            d = torch.randn(param0.shape, generator=gen, device=dev)
            for _ in range(3):   # smooth by repeated neighbour averaging along every axis
                for ax in range(d.dim()):
                    d = (d + torch.roll(d, 1, ax) + torch.roll(d, -1, ax)) / 3
            if wl.physics == "density":
                # keep the design below 1: the material interpolation stiffens
                # steeply towards gamma = 1 and the time step must stay stable
                d = d * (param0 < 0.9).to(d.dtype)
            d = d / d.abs().max()
            eps = (1e-3 if wl.physics == "velocity" else 1e-2) * float(param0.abs().max())
            cs = []
            for sgn in (1.0, -1.0):
                mp = W.Model((param0 + sgn * eps * d).contiguous(), wl.h, dt, wl.order, wl.physics, wl.bc,
                             kahan=args.kahan)
                mp.set_tiling(*tiling)
                mp.set_schedule(cta_order)
                _, c_, _ = mp.gradient(shots, objective=wl.objective, patch_sign=wl.patch_sign, mode="symmetric",
                                       grad_wrt="param")
                cs.append(float(c_.item()))
                del mp
            fd = (cs[0] - cs[1]) / (2 * eps)
            gp, _, _ = ref_model.gradient(shots, objective=wl.objective, patch_sign=wl.patch_sign, grad_wrt="param")
            dirv = float((gp.double() * d.double()).sum().item())
            accuracy["finite_difference"] = {"fd": fd, "directional_derivative": dirv,
                                             "rel_err": abs(dirv - fd) / max(abs(fd), 1e-300), "eps": eps,
                                             "what": "central difference of C along a smooth random direction "
                                                     "vs <dC/dparam of the timed method, direction>"}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32" if args.storage == "f32" else f"f32 arithmetic, {args.storage} storage",
            "data": "synthetic",
            "config": {"workload": wl.name, "shape": list(wl.shape), "order": wl.order, "physics": wl.physics,
                       "shots": wl.nshots, "nt_total": int(sum(wl.nt)),
                       "mode": mode + (", graph replay" if use_graph else ", eager calls"),
                       "gradient": args.grad_mode, "k_ratio": args.k_ratio, "kahan": args.kahan,
                       "storage": args.storage, "parallelism": f"replicas x{world}", "tiling": list(tiling),
                       "cta_order": cta_order,
                       "l2": "inputs larger than L2 (each resident grid > 129 MB)",
                       "observed_data": "true model on a 2x grid with 2x steps" if args.refined_data
                       else "true model on the same grid"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": int(launches),
            "plain": plain, "check": {"misfit": misfit_val, "grad_l2": grad_norm, "k": k_val},
            "accuracy": accuracy,
        }
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
