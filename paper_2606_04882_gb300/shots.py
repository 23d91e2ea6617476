"""Shot-parallel execution across ranks.

Shots are independent forward problems and independent terms of the FWI
misfit J = sum_s 1/2 ||d_s - d_obs,s||^2, so ranks split the shot list and the
only exchange is one sum of (J, dJ/dm) at the end (torch.distributed
all-reduce: NCCL between GPUs, gloo on CPU).  The per-shot work is a callable,
so the same host logic drives the CUDA path (``gpu_shot_fn``) and, in tests,
CPU stand-ins on gloo ranks.
"""
from __future__ import annotations

from typing import Callable, List, Optional, Sequence, Tuple

import numpy as np


def shard(nshots: int, rank: int, world: int) -> List[int]:
    """Contiguous, balanced block of shot indices for `rank` (sizes differ by
    at most one; ranks beyond nshots get none)."""
    if world < 1 or not (0 <= rank < world):
        raise ValueError("bad rank/world %d/%d" % (rank, world))
    base, extra = divmod(nshots, world)
    lo = rank * base + min(rank, extra)
    hi = lo + base + (1 if rank < extra else 0)
    return list(range(lo, hi))


class RankFailure(RuntimeError):
    """Another rank failed its shots: raised on the ranks that did not, in
    place of the reduction (which would mix in a partial gradient)."""


def _dist():
    try:
        import torch.distributed as dist
        if dist.is_available() and dist.is_initialized():
            return dist
    except Exception:
        pass
    return None


def misfit_and_gradient(template, nshots: int,
                        per_shot: Callable[[int], Tuple[float, "object"]],
                        rank: Optional[int] = None, world: Optional[int] = None):
    """Sum (J_s, g_s) over this rank's shots, then all-reduce the sums over
    ranks.  ``per_shot(s)`` returns (J_s, g_s) with g_s a tensor shaped like
    `template` (which fixes shape, dtype and device, so that ranks without
    shots contribute zeros).  Returns (J, g), identical on every rank.

    Failures: the ranks first all-reduce a count of failed ranks.  A rank
    whose shots raised re-raises its exception after that exchange, and the
    others raise RankFailure, so no rank waits in the reduction for a rank
    that has given up.  A rank that never reaches the exchange (it died or
    hangs) is caught by the process group's timeout, which ends the
    collective with an error on the others."""
    import torch
    dist = _dist()
    if rank is None or world is None:
        rank, world = (dist.get_rank(), dist.get_world_size()) if dist else (0, 1)
    g = torch.zeros_like(template)
    J = 0.0
    err = None
    try:
        for s in shard(nshots, rank, world):
            Js, gs = per_shot(s)
            J += float(Js)
            g.add_(gs)
    except Exception as e:        # reported to the other ranks below
        err = e
    if dist is not None and world > 1:
        failed = torch.tensor([0.0 if err is None else 1.0], dtype=torch.float64, device=g.device)
        dist.all_reduce(failed)
        if err is not None:
            raise err
        if failed.item() > 0:
            raise RankFailure("%d of %d ranks failed their shots" % (int(failed.item()), world))
        Jt = torch.tensor([J], dtype=g.dtype, device=g.device)
        dist.all_reduce(Jt)
        dist.all_reduce(g)
        J = float(Jt.item())
    elif err is not None:
        raise err
    return J, g


def gpu_shot_fn(plan, model_m, src_idx: Sequence[np.ndarray], wavelets, rec_idx: np.ndarray,
                d_obs, k=None):
    """Per-shot (J_s, dJ/dm) on the GPU for m = 1/v^2: forward traces, residual
    d - d_obs, adjoint gradient.  k = None: when every step's D fits the
    device, one forward sweep keeps them (fd_gradient_forward) and the adjoint
    runs from them (fd_gradient_adjoint); else, or with an integer k, a plain
    forward for the traces and fd_adjoint_gradient with checkpoints every k
    (20 by default) steps.  The results are bitwise the same."""
    import torch
    from . import (FD_MODEL_SLOWNESS2, check_status, fd_adjoint_gradient, fd_forward,
                   fd_gradient_adjoint, fd_gradient_forward, workspace)
    dev = model_m.device
    nrec = len(rec_idx)
    if k is None:
        need = plan.gradient_workspace_size(1, nrec, plan.nt)
        if need + (4 << 30) < torch.cuda.mem_get_info(dev)[0]:
            wss = workspace(need, dev)

            def run_split(s):
                tr = torch.empty((plan.nt, nrec), device=dev)
                fd_gradient_forward(plan, model_m, src_idx[s], wavelets[s], rec_idx, tr, wss,
                                    model_kind=FD_MODEL_SLOWNESS2)
                check_status(plan, wss, "forward of shot %d" % s)
                r = tr - d_obs[s]
                J = 0.5 * float((r.double() ** 2).sum())
                g = torch.empty_like(model_m)
                fd_gradient_adjoint(plan, src_idx[s], rec_idx, r, g, wss)
                check_status(plan, wss, "gradient of shot %d" % s)
                return J, g

            return run_split
        k = 20
    wsf = workspace(plan.forward_workspace_size(1, nrec), dev)
    wsg = workspace(plan.gradient_workspace_size(1, nrec, k), dev)

    def run(s):
        tr = torch.empty((plan.nt, nrec), device=dev)
        fd_forward(plan, model_m, src_idx[s], wavelets[s], rec_idx, tr, wsf,
                   model_kind=FD_MODEL_SLOWNESS2)
        check_status(plan, wsf, "forward of shot %d" % s)
        r = tr - d_obs[s]
        J = 0.5 * float((r.double() ** 2).sum())
        g = torch.empty_like(model_m)
        fd_adjoint_gradient(plan, model_m, src_idx[s], wavelets[s], rec_idx, r, k, g, wsg,
                            model_kind=FD_MODEL_SLOWNESS2)
        check_status(plan, wsg, "gradient of shot %d" % s)
        return J, g

    return run
