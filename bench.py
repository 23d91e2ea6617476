#!/usr/bin/env python
"""Throughput of the shaped-stencil acoustic forward on one or more GB300s.

Workload (default, one bench step): the 3D smooth-random model of 400^3
physical nodes (h = 10 m, 1500-5000 m/s, 30-node sponge -> 460^3 padded),
1500 time steps, 15 Hz Ricker source, 100 x 100 surface receivers, run once
with each of Cross(4) Taylor, Cross(8) Taylor and Rhombus(4) DispLS weights
(dt = 0.5 x the Taylor CFL limit of radius M at 5000 m/s).  Metric: grid-point
updates per second (padded points x steps / time), in Gpts/s.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs the same workload on its own GPU (independent
problems, weak scaling); the time is the max over ranks.  --impl reference
times the FP64 CPU oracle on a bounded sample of the same workload.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

STENCILS = [("cross", 4, "spatte"), ("cross", 8, "spatte"), ("rhombus", 4, "displs")]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--n", type=int, default=400, help="physical nodes per axis")
    ap.add_argument("--nt", type=int, default=1500)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def workload(n, nt):
    from workloads import gradient_random_3d
    return gradient_random_3d(n=n, nt=nt)


def taylor_dt(F, M, h, vmax):
    return 0.5 * F.fd_cfl_limit(F.stencil_desc(3, "cross", M)) * h / vmax


class ClockSampler:
    """nvidia-smi sampled every 200 ms while the timed region runs."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm = [float(r[1]) for r in rows if len(r) > 8 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) > 8 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) > 8 for i in range(4)
                          if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def run_gpu(args):
    import torch
    import torch.distributed as dist
    import paper_2606_04882_gb300 as F
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pr = workload(args.n, args.nt)
    h, nt, nb, vmax = pr.h, pr.nt, pr.nb, pr.vmax
    vel = torch.from_numpy(pr.vel).to(dev)
    src_idx, rec_idx = None, None
    runs = []
    for shape, M, scheme in STENCILS:
        dt = taylor_dt(F, M, h, vmax)
        desc = F.stencil_desc(3, shape, M, 0, scheme, courant=vmax * dt / h)
        plan = F.Plan(pr.shape, h, dt, nt, nb, vmax, desc)
        plan0 = F.Plan(pr.shape, h, dt, 0, nb, vmax, desc)      # set-up only (nt = 0)
        if src_idx is None:
            src_idx = plan.linear_index(pr.src)
            rec_idx = plan.linear_index(pr.rec)
        wav = torch.from_numpy(F.fd_ricker(pr.f0, dt, nt)[:, None].copy()).to(dev)
        tr = torch.empty((nt, len(rec_idx)), device=dev)
        ws = F.workspace(plan.forward_workspace_size(1, len(rec_idx)), dev)
        runs.append(dict(name="%s%d_%s" % (shape, M, scheme), plan=plan, plan0=plan0, wav=wav,
                         tr=tr, ws=ws, dt=dt))
    inf = runs[0]["plan"].info()
    pts = int(inf.padded[0] * inf.padded[1] * inf.padded[2])
    stream = torch.cuda.current_stream()

    def one_step(ev=None):
        for i, r in enumerate(runs):
            if ev is not None:
                ev[i][0].record(stream)
            F.fd_forward(r["plan"], vel, src_idx, r["wav"], rec_idx, r["tr"], r["ws"])
            if ev is not None:
                ev[i][1].record(stream)

    def barrier():
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # set-up cost per stencil (nt = 0), subtracted to get the step kernel's time
    setup_ms = []
    for r in runs:
        for _ in range(2):
            F.fd_forward(r["plan0"], vel, src_idx, r["wav"], rec_idx, r["tr"], r["ws"])
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(5):
            F.fd_forward(r["plan0"], vel, src_idx, r["wav"], rec_idx, r["tr"], r["ws"])
        b.record(stream)
        torch.cuda.synchronize()
        setup_ms.append(a.elapsed_time(b) / 5)

    for _ in range(args.warmup):
        one_step()
    for r in runs:
        assert F.fd_status_read(r["plan"], r["ws"]) == 0, F.last_error()
    sampler = ClockSampler(local)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in runs] for _ in range(args.steps)]
    barrier()
    sampler.start()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        one_step(ev[k])
    t1.record(stream)
    barrier()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    per_run_ms = [statistics.mean(ev[k][i][0].elapsed_time(ev[k][i][1]) for k in range(args.steps))
                  for i in range(len(runs))]
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    work = pts * nt * len(runs) * args.steps * world
    value = work / (ms * 1e-3) / 1e9

    # e2e: host model in, host traces out, through the same calls
    e2e = None
    if not args.no_e2e:
        hvel = torch.from_numpy(pr.vel).pin_memory()
        hwav = [r["wav"].cpu().pin_memory() for r in runs]
        htr = [torch.empty(r["tr"].shape, dtype=torch.float32).pin_memory() for r in runs]
        dvel = torch.empty_like(vel)
        dwav = [torch.empty_like(r["wav"]) for r in runs]

        def e2e_step():
            dvel.copy_(hvel, non_blocking=True)
            for i, r in enumerate(runs):
                dwav[i].copy_(hwav[i], non_blocking=True)
                F.fd_forward(r["plan"], dvel, src_idx, dwav[i], rec_idx, r["tr"], r["ws"])
                htr[i].copy_(r["tr"], non_blocking=True)
            stream.synchronize()

        e2e_step()
        barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            e2e_step()
        b.record(stream)
        barrier()
        ems = a.elapsed_time(b)
        if world > 1:
            t = torch.tensor([ems], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ems = float(t.item())
        h2d = hvel.numel() * 4 + sum(w.numel() * 4 for w in hwav)
        d2h = sum(t.numel() * 4 for t in htr)
        e2e = {"value": work / (ems * 1e-3) / 1e9, "unit": "Gpts/s", "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h}

    peak, peak_kind = load_peaks()
    kernels = []
    for i, r in enumerate(runs):
        launch_ms = max(per_run_ms[i] - setup_ms[i], 1e-9) / nt
        gbs = 16.0 * pts / (launch_ms * 1e-3) / 1e9
        kernels.append({"stencil": r["name"], "ms_per_launch": launch_ms,
                        "achieved_gbs": gbs, "frac": gbs / peak,
                        "gpts": pts / (launch_ms * 1e-3) / 1e9})
    dom = max(range(len(runs)), key=lambda i: per_run_ms[i])
    roof = {"bound": "hbm", "achieved": kernels[dom]["achieved_gbs"], "peak": peak,
            "unit": "GB/s", "frac": kernels[dom]["frac"], "traffic": None,
            "kernel": "step3d " + kernels[dom]["stencil"],
            "bytes_per_point": 16, "peak_source": peak_kind}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(pr, runs[0]["dt"])
    out = {"metric": "grid-point updates/s (forward, 3D 400^3 + 30-node sponge, 1500 steps)",
           "value": value, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "3d_gradient_random_%d (%d^3 padded), %d steps, stencils %s"
                                  % (args.n, inf.padded[0], nt, ",".join(r["name"] for r in runs)),
                      "padded_points": pts, "receivers": len(rec_idx), "l2": "inputs larger than L2",
                      "parallelism": "independent replicas per GPU"},
           "e2e": e2e, "roofline": roof, "kernels": kernels, "cpu_baseline": cpu,
           "clocks": clocks, "gpu_launches": args.steps * len(runs) * (nt + 1)}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(pr, dt, steps=2):
    """The FP64 oracle on a bounded sample: `steps` time steps of the full
    460^3 grid with the Cross(4) stencil on all host cores."""
    from oracle import physics as P
    from oracle import wave as W
    st = W.Setup(pr.vel, pr.h, dt, pr.nb, pr.vmax, 3, "cross", 4)
    wav = P.ricker(pr.f0, steps, dt)[:, None]
    threads = W.default_threads()
    t = time.perf_counter()
    W.forward(st, steps, pr.src, wav, pr.rec, threads=threads)
    el = time.perf_counter() - t
    pts = int(np.prod(st.pshape))
    return {"value": pts * steps / el / 1e9, "unit": "Gpts/s", "cores": threads, "kind": "oracle",
            "sample": "%d time steps of the %d^3 padded grid, Cross(4), FP64 C oracle" % (steps, st.pshape[0])}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from oracle import physics as P
    from oracle import stencil as S
    from oracle import wave as W
    pr = workload(args.n, args.nt)
    setups = []
    for shape, M, scheme in STENCILS:
        pw = S.expand(3, "cross", M, 0, S.weights(3, "cross", M))
        dt = 0.5 * S.cfl_limit(pw, 3) * pr.h / pr.vmax
        setups.append(W.Setup(pr.vel, pr.h, dt, pr.nb, pr.vmax, 3, shape, M, 0, scheme))
    threads = W.default_threads()
    pts = int(np.prod(setups[0].pshape))

    def step(i):
        st = setups[i % len(setups)]
        W.forward(st, 1, pr.src, P.ricker(pr.f0, 1, st.dt)[:, None], pr.rec, threads=threads)

    for i in range(args.warmup):
        step(i)
    t = time.perf_counter()
    for i in range(args.steps):
        step(i)
    el = time.perf_counter() - t
    v = pts * args.steps / el / 1e9
    out = {"impl": "reference", "metric": "grid-point updates/s (forward, 3D 400^3 + 30-node sponge, 1500 steps)",
           "value": v, "unit": "Gpts/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": el * 1e3 / max(args.steps, 1),
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": "3d_gradient_random_%d (%d^3 padded), stencils cross4,cross8,rhombus4"
                                  % (args.n, setups[0].pshape[0])},
           "cpu_baseline": {"value": v, "unit": "Gpts/s", "cores": threads, "kind": "oracle",
                            "sample": "one time step of the full padded grid per bench step, "
                                      "cycling through the three stencils"},
           "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_gpu(a)
