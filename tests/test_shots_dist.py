"""Multi-rank host logic on CPU: shot sharding and the single misfit/gradient
reduction, run as gloo ranks (world_size 2 and 3) with the FP64 oracle as the
per-shot computation, against the single-process sum."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_04882_gb300.shots import misfit_and_gradient, shard


def test_shard_covers_every_shot_once():
    for n in range(0, 13):
        for w in range(1, 6):
            parts = [shard(n, r, w) for r in range(w)]
            flat = [s for p in parts for s in p]
            assert flat == list(range(n))
            sizes = [len(p) for p in parts]
            assert max(sizes) - min(sizes) <= 1


def _problem():
    from oracle import physics as P
    from oracle import stencil as S
    from oracle import wave as W
    from workloads import smooth_velocity
    n, nb, nt, h, vmax = 24, 4, 60, 10.0, 3000.0
    v = smooth_velocity((n, n), 4, 1500.0, 2900.0, sigma=3.0).astype(np.float64)
    vt = smooth_velocity((n, n), 9, 1500.0, 2900.0, sigma=2.0).astype(np.float64)
    pw = S.expand(2, "cross", 2, 0, S.weights(2, "cross", 2))
    dt = 0.5 * S.cfl_limit(pw, 2) * h / vmax
    srcs = [np.array([[2, x]]) for x in (3, 9, 15, 21, 12)]
    rec = np.array([[2, x] for x in range(n)])
    wav = P.ricker(25.0, nt, dt)[:, None]
    st = W.Setup(v, h, dt, nb, vmax, 2, "cross", 2)
    stt = W.Setup(vt, h, dt, nb, vmax, 2, "cross", 2)

    def per_shot(s):
        dobs = W.forward(stt, nt, srcs[s], wav, rec, threads=1)[0]
        d = W.forward(st, nt, srcs[s], wav, rec, threads=1)[0]
        g, _ = W.gradient(st, nt, srcs[s], wav, rec, d - dobs, threads=1)
        return 0.5 * float(np.sum((d - dobs) ** 2)), torch.from_numpy(g)

    return per_shot, len(srcs), (n, n)


def _rank_main(rank, world, port, nshots, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    per_shot, _, shape = _problem()
    J, g = misfit_and_gradient(torch.zeros(shape, dtype=torch.float64), nshots, per_shot)
    out[rank] = (J, g.numpy().copy())
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


@pytest.mark.parametrize("world,nshots", [(2, 5), (3, 2)])
def test_gloo_ranks_reduce_to_the_single_process_sum(world, nshots):
    per_shot, _, shape = _problem()
    J0 = 0.0
    g0 = np.zeros(shape)
    for s in range(nshots):
        Js, gs = per_shot(s)
        J0 += Js
        g0 += gs.numpy()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_rank_main, args=(world, _free_port(), nshots, out), nprocs=world,
                       join=True, start_method="spawn")
    for r in range(world):
        J, g = out[r]
        assert abs(J - J0) <= 1e-12 * abs(J0)
        assert np.allclose(g, g0, rtol=1e-12, atol=1e-12 * np.abs(g0).max())
