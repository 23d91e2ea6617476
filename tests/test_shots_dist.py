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


def _failing_rank_main(rank, world, port, mode, out):
    """mode 'raise': rank 1's shot raises; mode 'absent': rank 1 never joins
    the reduction (it leaves between steps)."""
    import datetime
    import time
    from paper_2606_04882_gb300.shots import RankFailure
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world,
                            timeout=datetime.timedelta(seconds=5))

    def per_shot(s):
        if rank == 1 and mode == "raise":
            raise ValueError("shot %d failed" % s)
        return 1.0, torch.ones(4, dtype=torch.float64)

    t0 = time.time()
    if rank == 1 and mode == "absent":
        time.sleep(8)             # past the others' collective timeout
        out[rank] = ("left", 0.0)
        return
    try:
        misfit_and_gradient(torch.zeros(4, dtype=torch.float64), 4, per_shot)
        out[rank] = ("ok", time.time() - t0)
    except RankFailure:
        out[rank] = ("rank_failure", time.time() - t0)
    except ValueError:
        out[rank] = ("own_error", time.time() - t0)
    except RuntimeError:
        out[rank] = ("collective_error", time.time() - t0)
    dist.destroy_process_group()


def test_a_failing_rank_is_reported_to_the_others():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_failing_rank_main, args=(2, _free_port(), "raise", out), nprocs=2,
                       join=True, start_method="spawn")
    assert out[1][0] == "own_error"
    assert out[0][0] == "rank_failure" and out[0][1] < 5.0


def test_an_absent_rank_ends_the_collective_by_timeout():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_failing_rank_main, args=(2, _free_port(), "absent", out), nprocs=2,
                       join=True, start_method="spawn")
    assert out[1][0] == "left"
    assert out[0][0] == "collective_error" and out[0][1] < 8.0
