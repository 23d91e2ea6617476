"""Accuracy experiments of Section 6 on the GPU: the homogeneous velocity
model (Section 6, "Homogeneous Velocity Model", Table table1:homogeneo) and
the two-layer model (Section 6, "Two Layers Velocity Model", Table
table1:hetero).

Every finite-difference scheme of Section 4 runs on the paper's grid for
M = 1..6, with 1 <= N <= M for the cross-rhombus and 0 <= N <= M for the
cross-square shapes (Section 6, "General Considerations").  The reference
runs on a grid refined 16 times in space and time (same section) with the
Taylor cross of radius 8, and is sampled at the coarse nodes and times.
For each scheme the snapshot at the paper's time and the seismic trace at
the paper's point are compared with the reference: the error norms of
Section 5.3 (Eqs. snapnorm1, snapnorm2, snapnormmax) and the trace's DFT and
CWT dispersion norms (Appendix A, Eqs. norm2gammastdft, norm2gammastcwt),
all computed by the library's GPU metrics.

Readings where the tables are silent or inconsistent:
- a run lasts nt steps of dt (the tables' printed end times, 1500 ms and
  "1500s", disagree with nt * dt);
- the damping layer is the library's sponge, nb = 40 nodes on each side of
  the coarse grid and 16 nb on the reference grid, so its physical width and
  profile are the same;
- the weights of the velocity-dependent schemes use the model's maximum
  velocity (Section 6, "General Considerations");
- the trace norms substitute tau for h in the snapshot norms' scale
  factors (Section 5.3): 1/tau^2 and 1/tau;
- the CWT norm uses nt/2 + 1 scales with omega0 = 6.

Usage: ``python -m paper_2606_04882_gb300.experiments e1 e2 --out results.json``
(GPU required).
"""
from __future__ import annotations

import argparse
import json
import time
from dataclasses import dataclass
from typing import Callable, Dict, List, Optional, Tuple

import numpy as np

from . import (FdError, Plan, fd_cwt_gamma, fd_dft_gamma, fd_error_norms, fd_forward,
               fd_ricker, fd_status_read, stencil_desc, workspace)


@dataclass
class Experiment:
    name: str
    n: int                       # physical nodes per axis (square grid)
    h: float                     # node spacing (m)
    dt: float                    # time step (s)
    nt: int                      # time steps
    f0: float                    # Ricker peak frequency (Hz)
    velocity: Callable[[np.ndarray], np.ndarray]   # depth z (m) -> velocity (m/s)
    src: Tuple[float, float]     # (z, x) in m
    trace: Tuple[float, float]   # (z, x) in m
    t_snap: float                # snapshot time (s)
    nb: int = 40

    @property
    def vmax(self) -> float:
        z = np.arange(self.n) * self.h
        return float(self.velocity(z).max())

    def model(self, refine: int) -> np.ndarray:
        """Velocity on the physical grid refined `refine` times, [nz][nx] float32."""
        n = (self.n - 1) * refine + 1
        z = np.arange(n) * (self.h / refine)
        col = self.velocity(z).astype(np.float32)
        return np.ascontiguousarray(np.repeat(col[:, None], n, axis=1))

    def node(self, pos: Tuple[float, float], refine: int) -> Tuple[int, int]:
        hr = self.h / refine
        return int(round(pos[0] / hr)), int(round(pos[1] / hr))

    @property
    def n_snap(self) -> int:
        return int(round(self.t_snap / self.dt))


def homogeneous() -> Experiment:
    """Table table1:homogeneo: 6 km x 6 km, 401^2 nodes, h = 15 m, dt = 2 ms,
    nt = 1500, f0 = 30 Hz, c = 3 km/s, source at the centre; snapshot at
    1.05 s, trace at x = 1200 m, z = 3000 m."""
    return Experiment("homogeneous", 401, 15.0, 2.0e-3, 1500, 30.0,
                      lambda z: np.full(z.shape, 3000.0), src=(3000.0, 3000.0),
                      trace=(3000.0, 1200.0), t_snap=1.05)


def two_layer() -> Experiment:
    """Table table1:hetero: 4 km x 4 km, 401^2 nodes, h = 10 m, dt = 1 ms,
    nt = 1500, f0 = 25 Hz; 1.5 km/s down to z = 1200 m and 3 km/s below;
    source at x = 2000 m, z = 1600 m; snapshot at 1.08 s, trace at x = 1000 m,
    z = 2000 m."""
    return Experiment("two_layer", 401, 10.0, 1.0e-3, 1500, 25.0,
                      lambda z: np.where(z <= 1200.0, 1500.0, 3000.0), src=(1600.0, 2000.0),
                      trace=(2000.0, 1000.0), t_snap=1.08)


EXPERIMENTS = {"e1": homogeneous, "e2": two_layer}


def schemes(m_max: int = 6) -> List[Tuple[str, str, int, int, str]]:
    """(label, shape, M, N, scheme) for every scheme of the sweep."""
    out = []
    for M in range(1, m_max + 1):
        out.append(("SpatTE-Cross(%d)" % M, "cross", M, 0, "spatte"))
        out.append(("SpecTE-theta-Cross(%d)" % M, "cross", M, 0, "specte_theta"))
        for sch, tag in (("dispte", "DispTE"), ("displs", "DispLS"), ("specls", "SpecLS")):
            for N in range(1, M + 1):
                out.append(("%s-CrossRb(%d,%d)" % (tag, M, N), "cross_rhombus", M, N, sch))
            for N in range(0, M + 1):
                out.append(("%s-CrossSq(%d,%d)" % (tag, M, N), "cross_square", M, N, sch))
    return out


def _run(ex: Experiment, refine: int, desc, vel_d, rec: Tuple[int, int], dev):
    """Forward run on the grid refined `refine` times: returns (snapshot on the
    physical grid at step refine * n_snap, trace [refine * nt], status)."""
    import torch
    dt = ex.dt / refine
    nt = ex.nt * refine
    n1 = ex.n_snap * refine
    nb = ex.nb * refine
    h = ex.h / refine
    shape = tuple(vel_d.shape)
    wav = torch.from_numpy(fd_ricker(ex.f0, dt, nt)[:, None].copy()).to(dev)
    src = ex.node(ex.src, refine)
    traces = torch.zeros((nt, 1), dtype=torch.float32, device=dev)
    status = 0
    state = None
    snap = None
    for t0, steps in ((0, n1), (n1, nt - n1)):
        plan = Plan(shape, h, dt, steps, nb, ex.vmax, desc)
        ws = workspace(plan.forward_workspace_size(1, 1), dev)
        out = torch.empty((2,) + tuple(plan.padded_shape), dtype=torch.float32, device=dev)
        fd_forward(plan, vel_d, plan.linear_index([src]), wav[t0:t0 + steps],
                   plan.linear_index([rec]), traces[t0:t0 + steps], ws, state_in=state,
                   state_out=out)
        status = status or fd_status_read(plan, ws)
        if t0 == 0:
            snap = out[0, nb:nb + shape[0], nb:nb + shape[1]].clone(
                memory_format=torch.contiguous_format)
        state = out
    return snap, traces[:, 0], status


def run(ex: Experiment, refine: int = 16, m_max: int = 6, ref_M: int = 8,
        only: Optional[List[str]] = None) -> Dict:
    """Run the sweep of `ex` against its refined reference; returns a dict of
    norms per scheme (GPU required)."""
    import torch
    dev = torch.device("cuda")
    t_start = time.perf_counter()
    # reference: Taylor cross of radius ref_M on the refined grid
    vel_r = torch.from_numpy(ex.model(refine)).to(dev)
    c_ref = ex.vmax * (ex.dt / refine) / (ex.h / refine)
    d_ref = stencil_desc(2, "cross", ref_M, 0, "spatte", courant=c_ref)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    snap_r, tr_r, st_r = _run(ex, refine, d_ref, vel_r, ex.node(ex.trace, refine), dev)
    torch.cuda.synchronize()
    t_ref = time.perf_counter() - t0
    pad = (ex.n - 1) * refine + 1 + 2 * ex.nb * refine
    ref_pts = float(pad) ** 2 * ex.nt * refine
    snap_ref = snap_r[::refine, ::refine].contiguous()
    # trace sample n of the coarse run is u at t^{n+1}: reference sample refine (n+1) - 1
    tr_ref = tr_r[refine - 1::refine].contiguous()
    del vel_r, snap_r, tr_r
    snap_ref_n = fd_error_norms(snap_ref, torch.zeros_like(snap_ref), 1.0 / ex.h ** 2,
                                1.0 / ex.h).cpu().numpy()
    tr_ref_n = fd_error_norms(tr_ref, torch.zeros_like(tr_ref), 1.0 / ex.dt ** 2,
                              1.0 / ex.dt).cpu().numpy()
    vel_c = torch.from_numpy(ex.model(1)).to(dev)
    C = ex.vmax * ex.dt / ex.h
    rows = []
    for label, shape, M, N, sch in schemes(m_max):
        if only and label not in only:
            continue
        row = {"scheme": label, "shape": shape, "M": M, "N": N, "weights": sch}
        try:
            snap, tr, st = _run(ex, 1, stencil_desc(2, shape, M, N, sch, courant=C), vel_c,
                                ex.node(ex.trace, 1), dev)
        except FdError as e:
            row["status"] = "rejected: %s" % e
            rows.append(row)
            continue
        if st != 0:
            row["status"] = "device status %d" % st
        elif not (torch.isfinite(snap).all() and torch.isfinite(tr).all()):
            row["status"] = "unstable (non-finite field)"
        else:
            row["status"] = "ok"
        if row["status"] == "ok":
            s = fd_error_norms(snap, snap_ref, 1.0 / ex.h ** 2, 1.0 / ex.h).cpu().numpy()
            t = fd_error_norms(tr, tr_ref, 1.0 / ex.dt ** 2, 1.0 / ex.dt).cpu().numpy()
            _, gn, _, _ = fd_dft_gamma(tr[:, None].contiguous(), tr_ref[:, None].contiguous(),
                                       with_gamma=False)
            _, wn, _, _, _ = fd_cwt_gamma(tr[:, None].contiguous(), tr_ref[:, None].contiguous(),
                                          with_gamma=False)
            row.update(snap_l1=float(s[0]), snap_l2=float(s[1]), snap_linf=float(s[2]),
                       trace_l1=float(t[0]), trace_l2=float(t[1]), trace_linf=float(t[2]),
                       snap_rel_l2=float(s[1] / snap_ref_n[1]),
                       trace_rel_l2=float(t[1] / tr_ref_n[1]),
                       gamma_dft=float(gn[0]), gamma_cwt=float(wn[0]))
        rows.append(row)
    torch.cuda.synchronize()
    return {"experiment": ex.name, "n": ex.n, "h": ex.h, "dt": ex.dt, "nt": ex.nt, "f0": ex.f0,
            "vmax": ex.vmax, "courant": C, "nb": ex.nb, "t_snap": ex.t_snap,
            "src": ex.src, "trace": ex.trace, "refine": refine,
            "reference": {"stencil": "SpatTE-Cross(%d)" % ref_M, "status": st_r,
                          "seconds": t_ref, "gpts_per_s": ref_pts / t_ref / 1e9,
                          "snap_l2": float(snap_ref_n[1]), "snap_linf": float(snap_ref_n[2]),
                          "trace_l2": float(tr_ref_n[1]), "trace_linf": float(tr_ref_n[2])},
            "seconds": time.perf_counter() - t_start, "schemes": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("which", nargs="+", choices=sorted(EXPERIMENTS))
    ap.add_argument("--refine", type=int, default=16)
    ap.add_argument("--m-max", type=int, default=6)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    res = [run(EXPERIMENTS[w](), a.refine, a.m_max) for w in a.which]
    txt = json.dumps(res, indent=1)
    if a.out:
        with open(a.out, "w") as f:
            f.write(txt)
    else:
        print(txt)


if __name__ == "__main__":
    main()
