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
    ap.add_argument("--workload", default="3d", choices=["3d", "2d", "batched", "fwi", "metrics"],
                    help="3d: 400^3 forward (default); 2d: 1001^2 x 18 stencils; batched: "
                         "48 2D shots on three grids; fwi: 256^3 gradient, 16 shots; metrics: "
                         "DFT dispersion metric of a 2000-sample x 1001-receiver gather pair")
    ap.add_argument("--shots", type=int, default=0, help="fwi/batched: use the first N shots")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-gradient", action="store_true",
                    help="3d: skip the FWI-gradient sub-record")
    ap.add_argument("--variants", default="",
                    help="3d: comma-separated y tiles (fd_plan_variants values) for the three "
                         "stencils instead of autotuning, e.g. 16,8,8")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# DRAM bytes per padded point of one step launch (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of the 300^3 case, 360^3 padded;
# scaled to the bench grid by its point count), valid only for the kernel
# sources whose digest is recorded with them.
TRAFFIC_SOURCES = ("paper_2606_04882_gb300/csrc/step3d.cu",
                   "paper_2606_04882_gb300/csrc/step3d_cross.cu",
                   "paper_2606_04882_gb300/csrc/step3d_planar.cu",
                   "paper_2606_04882_gb300/csrc/step3d_common.cuh",
                   "paper_2606_04882_gb300/csrc/device_common.cuh",
                   "paper_2606_04882_gb300/csrc/internal.h")
TRAFFIC_DIGEST = "50d1f10be7ca390c5f97e54fd4550e088068405780c0a2f9f8045b10ecbfd251"
TRAFFIC_B_PER_POINT = {"cross4_spatte": 16.487, "cross8_spatte": 16.776, "rhombus4_displs": 16.485}


def traffic_per_launch(stencil, pts):
    import hashlib
    h = hashlib.sha256()
    for rel in TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    if h.hexdigest() != TRAFFIC_DIGEST or stencil not in TRAFFIC_B_PER_POINT:
        return None
    return TRAFFIC_B_PER_POINT[stencil] * pts


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
    fixed = [int(v) for v in args.variants.split(",")] if args.variants else None
    for i, (shape, M, scheme) in enumerate(STENCILS):
        dt = taylor_dt(F, M, h, vmax)
        desc = F.stencil_desc(3, shape, M, 0, scheme, courant=vmax * dt / h)
        plan = F.Plan(pr.shape, h, dt, nt, nb, vmax, desc)
        plan0 = F.Plan(pr.shape, h, dt, 0, nb, vmax, desc)      # set-up only (nt = 0)
        if fixed:                                                # a given tile, cost-model z-chunk
            tile = list(plan.set_variant(fixed[i], 0).tile)
        else:
            tile = list(plan.autotune(vel).tile)                 # untimed tile-shape choice
        if src_idx is None:
            src_idx = plan.linear_index(pr.src)
            rec_idx = plan.linear_index(pr.rec)
        wav = torch.from_numpy(F.fd_ricker(pr.f0, dt, nt)[:, None].copy()).to(dev)
        tr = torch.empty((nt, len(rec_idx)), device=dev)
        # the nt = 0 plan keeps the default tile shape: size for both plans
        ws = F.workspace(max(plan.forward_workspace_size(1, len(rec_idx)),
                             plan0.forward_workspace_size(1, len(rec_idx))), dev)
        runs.append(dict(name="%s%d_%s" % (shape, M, scheme), plan=plan, plan0=plan0, wav=wav,
                         tr=tr, ws=ws, dt=dt, tile=tile))
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
        kernels.append({"stencil": r["name"], "tile": r["tile"], "ms_per_launch": launch_ms,
                        "achieved_gbs": gbs, "frac": gbs / peak,
                        "gpts": pts / (launch_ms * 1e-3) / 1e9})
    dom = max(range(len(runs)), key=lambda i: per_run_ms[i])
    roof = {"bound": "hbm", "achieved": kernels[dom]["achieved_gbs"], "peak": peak,
            "unit": "GB/s", "frac": kernels[dom]["frac"],
            "traffic": traffic_per_launch(kernels[dom]["stencil"], pts),
            "traffic_note": "DRAM bytes per launch, ncu on 360^3 scaled by points",
            "kernel": "step3d " + kernels[dom]["stencil"],
            "bytes_per_point": 16, "peak_source": peak_kind}

    grad_rec = None if args.no_gradient else bench_gradient(args, dev, stream, peak, peak_kind, world)

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
           "clocks": clocks, "gpu_launches": args.steps * len(runs) * (nt + 1),
           "gradient": grad_rec}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


# Algorithmic bytes per padded point and time step of the checkpointed
# gradient: three sweeps of the 16 B/pt step (forward, recompute, adjoint);
# the checkpoint copies, two fields read and written when stored every k
# steps and again when restored for the segment's recompute (32/k); the D
# store of the recompute and its load in the adjoint (4 + 4); and the
# gradient accumulator read and written in the adjoint (4 + 4).
GRAD_K = 20
GRAD_BYTES_PER_POINT = 3 * 16.0 + 32.0 / GRAD_K + 8.0 + 8.0


def bench_gradient(args, dev, stream, peak, peak_kind, world):
    """FWI gradient of the 256^3 workload (296^3 padded, 1200 steps, Cross(4),
    checkpoints every 20 steps): `args.steps` full shots timed with CUDA events
    after one untimed shot, and the same through host buffers (m in, dJ/dm
    out).  Metric: padded points x time steps of gradient per second."""
    import torch
    import torch.distributed as dist
    import paper_2606_04882_gb300 as F
    import workloads as WL
    probs, _ = WL.fwi_3d()
    pr = probs[0]
    dt = 0.5 * F.fd_cfl_limit(F.stencil_desc(3, "cross", 4)) * pr.h / pr.vmax
    plan = F.Plan(pr.shape, pr.h, dt, pr.nt, pr.nb, pr.vmax, F.stencil_desc(3, "cross", 4))
    m_host = (1.0 / pr.vel.astype(np.float64) ** 2).astype(np.float32)
    m = torch.from_numpy(m_host).to(dev)
    ri = plan.linear_index(pr.rec)
    wav = torch.from_numpy(F.fd_ricker(pr.f0, dt, pr.nt)[:, None].copy()).to(dev)
    resid = torch.randn((pr.nt, len(ri)), device=dev, generator=torch.Generator(dev).manual_seed(5))
    grad = torch.empty_like(m)
    ws = F.workspace(plan.gradient_workspace_size(1, len(ri), GRAD_K), dev)
    inf = plan.info()
    pts = int(inf.padded[0] * inf.padded[1] * inf.padded[2])
    shots = [plan.linear_index(probs[i % len(probs)].src) for i in range(max(args.steps, 1))]

    def shot(si, mm, gg):
        F.fd_adjoint_gradient(plan, mm, si, wav, ri, resid, GRAD_K, gg, ws,
                              model_kind=F.FD_MODEL_SLOWNESS2)

    shot(shots[0], m, grad)
    assert F.fd_status_read(plan, ws) == 0, F.last_error()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for si in shots:
        shot(si, m, grad)
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / len(shots)
    hm = torch.from_numpy(m_host).pin_memory()
    hg = torch.empty(m_host.shape, dtype=torch.float32).pin_memory()
    dm, dg = torch.empty_like(m), torch.empty_like(grad)
    a.record(stream)
    for si in shots:
        dm.copy_(hm, non_blocking=True)
        shot(si, dm, dg)
        hg.copy_(dg, non_blocking=True)
    b.record(stream)
    torch.cuda.synchronize()
    ems = a.elapsed_time(b) / len(shots)
    assert F.fd_status_read(plan, ws) == 0, F.last_error()
    keep = keep_all_d(plan, pr, m, shots, wav, ri, resid, grad, stream, peak, peak_kind, pts)
    if world > 1:
        t = torch.tensor([ms, ems], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms, ems = float(t[0]), float(t[1])
    work = pts * pr.nt * world
    gbs = GRAD_BYTES_PER_POINT * pts * pr.nt / (ms * 1e-3) / 1e9
    return {"metric": "FWI gradient grid-point updates/s (3D 256^3 + 20-node sponge, 1200 steps, "
                      "Cross(4), checkpoints every %d steps)" % GRAD_K,
            "value": work / (ms * 1e-3) / 1e9, "unit": "Gpts/s", "ms_per_shot": ms,
            "shots_timed": len(shots), "padded_points": pts,
            "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                         "frac": gbs / peak, "traffic": None, "peak_source": peak_kind,
                         "bytes_per_point": GRAD_BYTES_PER_POINT,
                         "note": "per padded point and time step of the gradient: forward, "
                                 "recompute and adjoint sweeps 3 x 16 B, checkpoint store and "
                                 "restore 32/k, D store and load 8, gradient accumulator 8"},
            "e2e": {"value": work / (ems * 1e-3) / 1e9, "unit": "Gpts/s",
                    "h2d_bytes_per_step": m.numel() * 4, "d2h_bytes_per_step": grad.numel() * 4},
            "gpu_launches": len(shots) * (3 * pr.nt + 2), "keep_all_d": keep}


KEEP_BYTES_PER_POINT = 2 * 16 + 8 + 8


def keep_all_d(plan, pr, m, shots, wav, ri, resid, grad_k, stream, peak, peak_kind, pts):
    """The same gradient with ckpt_every = nt: D of all 1200 steps stays in HBM
    (about 124 GB), so the forward sweep stores D and nothing is recomputed.
    Timed like the checkpointed run when the GPU has the room (else null); the
    last shot's gradient is compared bit for bit with the checkpointed one."""
    import torch
    import paper_2606_04882_gb300 as F
    need = plan.gradient_workspace_size(1, len(ri), pr.nt)
    free, _ = torch.cuda.mem_get_info()
    if need + (4 << 30) > free:
        return None
    ws = F.workspace(need, m.device)
    g = torch.empty_like(grad_k)

    def shot(si):
        F.fd_adjoint_gradient(plan, m, si, wav, ri, resid, pr.nt, g, ws,
                              model_kind=F.FD_MODEL_SLOWNESS2)

    shot(shots[0])
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for si in shots:
        shot(si)
    b.record(stream)
    torch.cuda.synchronize()
    assert F.fd_status_read(plan, ws) == 0, F.last_error()
    ms = a.elapsed_time(b) / len(shots)
    gbs = KEEP_BYTES_PER_POINT * pts * pr.nt / (ms * 1e-3) / 1e9
    out = {"value": pts * pr.nt / (ms * 1e-3) / 1e9, "unit": "Gpts/s", "ms_per_shot": ms,
           "workspace_gb": need / 1e9, "bitwise_equal_to_checkpointed": bool(torch.equal(g, grad_k)),
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                        "frac": gbs / peak, "peak_source": peak_kind,
                        "bytes_per_point": KEEP_BYTES_PER_POINT,
                        "note": "forward sweep storing D (16 + 4 B) and adjoint sweep (16 B, D load "
                                "4 B, gradient accumulator 8 B) per padded point and time step"},
           "gpu_launches": len(shots) * (2 * pr.nt + 2)}
    del ws
    torch.cuda.empty_cache()
    return out


def run_other(args):
    """2D, batched and FWI-gradient workloads (same JSON contract)."""
    import torch
    import torch.distributed as dist
    import paper_2606_04882_gb300 as F
    import workloads as WL
    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()
    jobs = []          # (name, enqueue(nt0: bool), points, nt, launches per run)
    h2d = d2h = 0
    if args.workload == "2d":
        pr = WL.layered_random_2d()
        vel = torch.from_numpy(pr.vel).to(dev)
        for st in pr.stencils:
            pw_dt = 0.5 * F.fd_cfl_limit(F.stencil_desc(2, "cross", st.M)) * pr.h / pr.vmax
            desc = F.stencil_desc(2, st.shape, st.M, 0, st.scheme, courant=pr.vmax * pw_dt / pr.h)
            plan = F.Plan(pr.shape, pr.h, pw_dt, pr.nt, pr.nb, pr.vmax, desc)
            plan0 = F.Plan(pr.shape, pr.h, pw_dt, 0, pr.nb, pr.vmax, desc)
            plan.autotune(vel)                                       # untimed tile choice
            si, ri = plan.linear_index(pr.src), plan.linear_index(pr.rec)
            wav = torch.from_numpy(F.fd_ricker(pr.f0, pw_dt, pr.nt)[:, None].copy()).to(dev)
            tr = torch.empty((pr.nt, len(ri)), device=dev)
            ws = F.workspace(max(plan.forward_workspace_size(1, len(ri)),
                                 plan0.forward_workspace_size(1, len(ri))), dev)
            inf = plan.info()
            pts = int(inf.padded[0] * inf.padded[2])

            def enq(zero, plan=plan, plan0=plan0, si=si, ri=ri, wav=wav, tr=tr, ws=ws):
                F.fd_forward(plan0 if zero else plan, vel, si, wav, ri, tr, ws)
            jobs.append(("%s%d_%s" % (st.shape, st.M, st.scheme), enq, pts, pr.nt, pr.nt + 1))
            d2h += tr.numel() * 4
        h2d = vel.numel() * 4
        wl = "2d_layered_random_1001 (1081^2 padded), 2000 steps, 18 stencils"
    elif args.workload == "batched":
        probs = WL.batched_shots_2d()
        if args.shots:
            probs = probs[:args.shots]
        dt = min(0.5 * F.fd_cfl_limit(F.stencil_desc(2, "cross", 4)) * p.h / p.vmax for p in probs)
        nt = probs[0].nt

        def make(nt_):
            shots, keep = [], []
            for pr in probs:
                plan = F.Plan(pr.shape, pr.h, dt, nt_, pr.nb, pr.vmax, F.stencil_desc(2, "cross", 4))
                shots.append(dict(plan=plan, model=torch.from_numpy(pr.vel).to(dev),
                                  src_idx=plan.linear_index(pr.src),
                                  wavelet=torch.from_numpy(F.fd_ricker(pr.f0, dt, nt)[:, None].copy()).to(dev),
                                  rec_idx=plan.linear_index(pr.rec),
                                  traces=torch.empty((nt, len(pr.rec)), device=dev)))
            return shots
        shots, shots0 = make(nt), make(0)
        ws = F.workspace(max(F.batched_workspace_size(shots), F.batched_workspace_size(shots0)), dev)
        F.fd_forward_batched_autotune(shots, ws)                 # untimed tile choice
        pts = 0
        for d in shots:
            inf = d["plan"].info()
            pts += int(inf.padded[0] * inf.padded[2])

        def enq(zero):
            F.fd_forward_batched(shots0 if zero else shots, ws)
        jobs.append(("batched_cross4_%dshots" % len(probs), enq, pts, nt, nt + len(probs)))
        h2d = sum(d["model"].numel() * 4 for d in shots)
        d2h = sum(d["traces"].numel() * 4 for d in shots)
        wl = "2d_batched %d shots on 1201x601/801x401/2001x801 (+20 sponge), 3000 steps, cross4" % len(probs)
    else:   # fwi
        probs, true = WL.fwi_3d()
        if args.shots:
            probs = probs[:args.shots]
        pr0 = probs[0]
        dt = 0.5 * F.fd_cfl_limit(F.stencil_desc(3, "cross", 4)) * pr0.h / pr0.vmax
        plan = F.Plan(pr0.shape, pr0.h, dt, pr0.nt, pr0.nb, pr0.vmax, F.stencil_desc(3, "cross", 4))
        m = torch.from_numpy((1.0 / pr0.vel.astype(np.float64) ** 2).astype(np.float32)).to(dev)
        ri = plan.linear_index(pr0.rec)
        wav = torch.from_numpy(F.fd_ricker(pr0.f0, dt, pr0.nt)[:, None].copy()).to(dev)
        resid = torch.randn((pr0.nt, len(ri)), device=dev, generator=torch.Generator(dev).manual_seed(5))
        grad = torch.empty_like(m)
        k = GRAD_K
        ws = F.workspace(plan.gradient_workspace_size(1, len(ri), k), dev)
        inf = plan.info()
        pts = int(inf.padded[0] * inf.padded[1] * inf.padded[2])
        for i, pr in enumerate(probs):
            si = plan.linear_index(pr.src)

            def enq(zero, si=si):
                if zero:
                    return
                F.fd_adjoint_gradient(plan, m, si, wav, ri, resid, k, grad, ws,
                                      model_kind=F.FD_MODEL_SLOWNESS2)
            jobs.append(("gradient_shot%d" % i, enq, pts, pr0.nt, 3 * pr0.nt + 1))
        h2d = m.numel() * 4
        d2h = m.numel() * 4
        wl = "3d_fwi_256 (296^3 padded), %d shots, 1200 steps, cross4, checkpoints every 20" % len(probs)

    def step(ev=None):
        for i, (_, enq, _, _, _) in enumerate(jobs):
            if ev is not None:
                ev[i][0].record(stream)
            enq(False)
            if ev is not None:
                ev[i][1].record(stream)

    setup_ms = []
    for (_, enq, _, _, _) in jobs:
        enq(True)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        enq(True)
        b.record(stream)
        torch.cuda.synchronize()
        setup_ms.append(a.elapsed_time(b))
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    ev = [[(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in jobs] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for kk in range(args.steps):
        step(ev[kk])
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    ms = t0.elapsed_time(t1)
    if world > 1:
        t = torch.tensor([ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    work = sum(j[2] * j[3] for j in jobs) * args.steps * world
    value = work / (ms * 1e-3) / 1e9
    peak, peak_kind = load_peaks()
    kernels = []
    bpp = 16.0 if args.workload != "fwi" else GRAD_BYTES_PER_POINT
    for i, (name, _, pts, nt, _) in enumerate(jobs):
        run_ms = statistics.mean(ev[kk][i][0].elapsed_time(ev[kk][i][1]) for kk in range(args.steps))
        per = max(run_ms - setup_ms[i], 1e-9) / nt
        gbs = bpp * pts / (per * 1e-3) / 1e9
        kernels.append({"run": name, "ms_per_time_step": per, "achieved_gbs": gbs, "frac": gbs / peak,
                        "gpts": pts / (per * 1e-3) / 1e9, "run_ms": run_ms})
    dom = max(range(len(jobs)), key=lambda i: kernels[i]["run_ms"])
    roof = {"bound": "hbm", "achieved": kernels[dom]["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": kernels[dom]["frac"], "traffic": None, "kernel": kernels[dom]["run"],
            "bytes_per_point": bpp, "peak_source": peak_kind}
    compare = batched_vs_single(args, dev, stream, shots) if args.workload == "batched" else None
    if args.workload == "2d":
        roof["note"] = "fields (4.7 MB) are L2-resident: the HBM fraction is nominal"
    if args.workload == "fwi":
        roof["note"] = ("bytes per point per time step of the whole gradient: forward, recompute "
                        "and adjoint sweeps (3 x 16) + checkpoint store and restore (32/k) + "
                        "D store/load (8) + gradient accumulator (8)")
    out = {"metric": "grid-point updates/s (%s)" % args.workload, "value": value, "unit": "Gpts/s",
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": wl, "l2": "see roofline note" if args.workload == "2d" else "inputs larger than L2"},
           "e2e": None, "roofline": roof, "kernels": kernels, "cpu_baseline": None,
           "clocks": clocks,
           "gpu_launches": args.steps * sum(j[4] for j in jobs)}
    if compare is not None:
        out["batched_vs_single_shot"] = compare
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        dist.destroy_process_group()


def batched_vs_single(args, dev, stream, shots, grad_shots=8, k=GRAD_K):
    """The batched forward of all shots against one fd_forward call per shot on
    the same inputs, and the batched gradient of the first `grad_shots` shots
    against one fd_adjoint_gradient call per shot (checkpoints every k steps,
    seeded residuals).  Same arithmetic, so the traces and gradients are
    checked to be bitwise equal; times are CUDA events, best of `args.steps`."""
    import torch
    import paper_2606_04882_gb300 as F

    def best(fn):
        fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(max(args.steps, 1)):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return min(ts)

    nt = shots[0]["plan"].nt
    pts = [int(np.prod(d["plan"].padded_shape)) for d in shots]
    ws = F.workspace(F.batched_workspace_size(shots), dev)
    ms_b = best(lambda: F.fd_forward_batched(shots, ws))
    tr_b = [d["traces"].clone() for d in shots]
    wss = [F.workspace(d["plan"].forward_workspace_size(len(d["src_idx"]), len(d["rec_idx"])), dev)
           for d in shots]

    def single():
        for d, w in zip(shots, wss):
            F.fd_forward(d["plan"], d["model"], d["src_idx"], d["wavelet"], d["rec_idx"], d["traces"], w)
    ms_s = best(single)
    same_fwd = all(torch.equal(a, d["traces"]) for a, d in zip(tr_b, shots))
    del ws, wss
    gs = []
    for i, d in enumerate(shots[:grad_shots]):
        g = torch.Generator(dev).manual_seed(100 + i)
        gs.append(dict(d, resid=torch.randn(d["traces"].shape, device=dev, generator=g),
                       grad=torch.empty_like(d["model"])))
    wsg = F.workspace(F.batched_gradient_workspace_size(gs, k), dev)
    gms_b = best(lambda: F.fd_adjoint_gradient_batched(gs, k, wsg))
    g_b = [d["grad"].clone() for d in gs]
    del wsg
    wsgs = [F.workspace(d["plan"].gradient_workspace_size(len(d["src_idx"]), len(d["rec_idx"]), k), dev)
            for d in gs]

    def single_grad():
        for d, w in zip(gs, wsgs):
            F.fd_adjoint_gradient(d["plan"], d["model"], d["src_idx"], d["wavelet"], d["rec_idx"],
                                  d["resid"], k, d["grad"], w)
    gms_s = best(single_grad)
    same_grad = all(torch.equal(a, d["grad"]) for a, d in zip(g_b, gs))
    del wsgs
    # the batched gradient with every shot's D kept in HBM (ckpt_every = nt)
    keep = None
    need = F.batched_gradient_workspace_size(gs, nt)
    torch.cuda.empty_cache()
    if need + (4 << 30) < torch.cuda.mem_get_info()[0]:
        wsk = F.workspace(need, dev)
        kms = best(lambda: F.fd_adjoint_gradient_batched(gs, nt, wsk))
        del wsk
        keep = {"batched_gpts": sum(pts[:len(gs)]) * nt / (kms * 1e-3) / 1e9, "batched_ms": kms,
                "workspace_gb": need / 1e9,
                "bitwise_equal": all(torch.equal(a, d["grad"]) for a, d in zip(g_b, gs))}
    work = sum(pts) * nt
    gwork = sum(pts[:len(gs)]) * nt
    return {"forward": {"shots": len(shots), "batched_gpts": work / (ms_b * 1e-3) / 1e9,
                        "single_shot_gpts": work / (ms_s * 1e-3) / 1e9, "batched_ms": ms_b,
                        "single_shot_ms": ms_s, "speedup": ms_s / ms_b, "bitwise_equal": same_fwd},
            "gradient": {"shots": len(gs), "ckpt_every": k,
                         "batched_gpts": gwork / (gms_b * 1e-3) / 1e9,
                         "single_shot_gpts": gwork / (gms_s * 1e-3) / 1e9, "batched_ms": gms_b,
                         "single_shot_ms": gms_s, "speedup": gms_s / gms_b,
                         "bitwise_equal": same_grad, "keep_all_d": keep},
            "note": "gradient points per second count padded points x time steps of the "
                    "gradient (its three sweeps)"}


def run_metrics(args):
    """Appendix A's DFT dispersion metric (fd_dft_gamma) on a pair of gathers of
    the 1001^2 workload's receiver size (2000 samples x 1001 receivers, all
    nt/2 + 1 frequencies): numerical = reference delayed by two samples plus
    noise.  Metric: complex multiply-adds of the two direct DFTs per second.
    The wavelet metric (fd_cwt_gamma) on the first trace pair at all 1001
    scales is timed separately and listed under kernels."""
    import torch
    import paper_2606_04882_gb300 as F
    dev = torch.device("cuda")
    nt, nrec = 2000, 1001
    nfreq = nt // 2 + 1
    g = torch.Generator(dev).manual_seed(11)
    ref = (torch.randn((nt, nrec), device=dev, generator=g).cumsum(0) * 1e-2).contiguous()
    num = (torch.roll(ref, 2, 0) + 1e-3 * torch.randn((nt, nrec), device=dev, generator=g)).contiguous()
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        F.fd_dft_gamma(num, ref)
    torch.cuda.synchronize()
    sampler = ClockSampler(0)
    sampler.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(args.steps):
        _, _, agg, _ = F.fd_dft_gamma(num, ref)
    b.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    ms = a.elapsed_time(b) / args.steps
    macs = 2.0 * nt * nrec * nfreq
    value = macs / (ms * 1e-3) / 1e9
    # the wavelet metric on one trace pair at all nt/2 + 1 scales (the paper's
    # analysis at one point), timed on its own
    nscale = nt // 2 + 1
    num1, ref1 = num[:, :1].contiguous(), ref[:, :1].contiguous()
    for _ in range(args.warmup):
        F.fd_cwt_gamma(num1, ref1, nscale)
    torch.cuda.synchronize()
    a.record(stream)
    for _ in range(args.steps):
        _, cw_norm, _, _, _ = F.fd_cwt_gamma(num1, ref1, nscale)
    b.record(stream)
    torch.cuda.synchronize()
    ms_w = a.elapsed_time(b) / args.steps
    macs_w = 2.0 * nscale * nt * (nt // 2)
    # per sample: 2 FMAs (accumulate) + 4 multiplies and 2 adds (twiddle rotation)
    gflops = 8.0 * macs / (ms * 1e-3) / 1e9
    out = {"metric": "DFT dispersion metric: complex multiply-adds per second (2 x 2000 x 1001 x 1001)",
           "value": value, "unit": "G/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "f64", "data": "synthetic",
           "config": {"workload": "metrics_dft_gamma 2000 samples x 1001 receivers, 1001 frequencies"},
           "roofline": {"bound": "alu", "achieved": gflops, "peak": 1250.0, "unit": "GFLOP/s",
                        "frac": gflops / 1250.0, "traffic": None,
                        "peak_source": "nominal FP64 rate of a GB300 (not measured)"},
           "result": {"gamma_norm_avg": float(agg[0]), "gamma_norm_max": float(agg[1]),
                      "gamma_w_norm_trace0": float(cw_norm[0])},
           "kernels": [{"run": "dft_gamma 2000 samples x 1001 receivers", "ms": ms, "gmacs": value},
                       {"run": "cwt_gamma 2000 samples x 1 receiver, 1001 scales", "ms": ms_w,
                        "gmacs": macs_w / (ms_w * 1e-3) / 1e9,
                        "frac": 8.0 * macs_w / (ms_w * 1e-3) / 1e9 / 1250.0}],
           "clocks": clocks, "gpu_launches": args.steps * 4}
    print(json.dumps(out))


def cpu_model():
    """The host CPU as /proc/cpuinfo names it (model name on x86; implementer
    and part numbers on Arm, e.g. 0x41/0xd4f for a Neoverse V2)."""
    try:
        info = open("/proc/cpuinfo").read().splitlines()
    except OSError:
        return "unknown"
    kv = {}
    for ln in info:
        if ":" in ln:
            k, v = ln.split(":", 1)
            kv.setdefault(k.strip().lower(), v.strip())
    if "model name" in kv:
        return kv["model name"]
    if "cpu implementer" in kv:
        return "Arm implementer %s part %s" % (kv["cpu implementer"], kv.get("cpu part", "?"))
    return "unknown"


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
            "cpu": cpu_model(), "sample": "%d time steps of the %d^3 padded grid, Cross(4), FP64 C oracle" % (steps, st.pshape[0])}


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
           "config": {"workload": "3d_gradient_random_%d (%d^3 padded), %d steps, stencils %s"
                                  % (args.n, setups[0].pshape[0], args.nt,
                                     ",".join("%s%d_%s" % st for st in STENCILS))},
           "cpu_baseline": {"value": v, "unit": "Gpts/s", "cores": threads, "kind": "oracle",
                            "cpu": cpu_model(), "sample": "one time step of the full padded grid per bench step, "
                                      "cycling through the three stencils"},
           "e2e": {"value": v, "unit": "Gpts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.workload == "3d":
        run_gpu(a)
    elif a.workload == "metrics":
        run_metrics(a)
    else:
        run_other(a)
