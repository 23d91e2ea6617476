"""Batched shots (one launch per time step over the tiles of every shot,
captured once into a CUDA graph and replayed) against single-shot runs and
the FP64 oracle, on grids of uneven size."""
import numpy as np
import pytest

from gpu_cases import Case, rel_l2
from workloads import faulted_layers_2d, smooth_velocity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_04882_gb300 import build
    build.build()


def _shots(M=4, scheme="spatte", dim=2, nt=120):
    cases = []
    if dim == 2:
        grids = [(61, 121), (41, 81), (81, 201)]
        for gi, (nz, nx) in enumerate(grids):
            vel = faulted_layers_2d(nz, nx, 40 + gi)
            for sx in (nx // 4, 3 * nx // 4):
                rec = np.array([[2, x] for x in range(0, nx, 3)])
                cases.append(Case(vel, 10.0, nt, 10, 5500.0, "cross", M, 0, scheme,
                                  src=[[2, sx]], rec=rec, f0=20.0))
    else:
        for gi, n in enumerate(((20, 24, 28), (26, 22, 30))):
            vel = smooth_velocity(n, 50 + gi, 1500.0, 3000.0)
            rec = np.array([[2, 3, x] for x in range(0, n[2], 2)])
            cases.append(Case(vel, 10.0, nt, 6, 3000.0, "cross", M, 0, scheme,
                              src=[[3, n[1] // 2, n[2] // 2]], rec=rec, f0=20.0))
    # one dt for the batch (the smallest)
    dt = min(c.dt for c in cases)
    for c in cases:
        c.dt = dt
        c.C = c.vmax * dt / c.h
    return cases


def _batched(cases, repeat=1, rows=0, autotune=False, status=None):
    import torch
    import paper_2606_04882_gb300 as F
    dev = torch.device("cuda")
    shots, keep = [], []
    for c in cases:
        plan = c.plan()
        tr = torch.zeros((c.nt, len(c.rec)), device=dev)
        d = dict(plan=plan, model=torch.from_numpy(c.vel).to(dev), src_idx=plan.linear_index(c.src),
                 wavelet=torch.from_numpy(c.wavelet32()).to(dev), rec_idx=plan.linear_index(c.rec),
                 traces=tr)
        shots.append(d)
    ws = F.workspace(F.batched_workspace_size(shots))
    if rows:
        F.fd_forward_batched_set_variant(shots, rows)
    if autotune:
        F.fd_forward_batched_autotune(shots, ws)
    outs = []
    for _ in range(repeat):
        for d in shots:
            d["traces"].zero_()
        F.fd_forward_batched(shots, ws)
        torch.cuda.synchronize()
        outs.append([d["traces"].cpu().numpy() for d in shots])
        if status is not None:   # shot 0's status word holds the batch's conditions
            status.append(F.fd_status_read(shots[0]["plan"], ws))
    return outs


@pytest.mark.parametrize("M,scheme", [(4, "spatte"), (2, "spatte"), (3, "spatte"), (8, "spatte"),
                                      (4, "displs")])
def test_batched_2d_matches_single_shot_and_oracle(M, scheme):
    """The batched kernel runs the single-shot kernel's per-point arithmetic,
    so its traces are bitwise those of single-shot runs."""
    cases = _shots(M, scheme)
    outs = _batched(cases, repeat=2)
    for i, c in enumerate(cases):
        tr, _, rc = c.gpu_forward()
        assert rc == 0
        assert np.array_equal(outs[0][i], tr), (i, rel_l2(outs[0][i], tr))
        assert np.array_equal(outs[0][i], outs[1][i]), i      # graph replay
    otr, _ = cases[-1].oracle_forward(threads=8)
    assert rel_l2(outs[0][-1], otr) < 1e-4


@pytest.mark.parametrize("nt", [121, 2, 3])
def test_batched_two_step_odd_and_short_runs(nt, monkeypatch):
    """With FDWAVE_BATCH_2STEP=1, Cross(2) and Cross(4) batches advance two
    steps per pass (an odd first step runs alone); traces equal single-shot
    runs and the one-step pass bitwise, for odd, minimal and short step
    counts."""
    for M in (4, 2):
        cases = _shots(M, "spatte", nt=nt)
        monkeypatch.setenv("FDWAVE_BATCH_2STEP", "1")
        two = _batched(cases)[0]
        monkeypatch.delenv("FDWAVE_BATCH_2STEP")
        one = _batched(cases)[0]
        for i, c in enumerate(cases):
            tr, _, rc = c.gpu_forward()
            assert rc == 0
            assert np.array_equal(two[i], tr), (M, nt, i, rel_l2(two[i], tr))
            assert np.array_equal(one[i], tr), (M, nt, i)


def test_batched_3d_per_shot_launches():
    cases = _shots(4, "spatte", dim=3, nt=50)
    outs = _batched(cases)
    for i, c in enumerate(cases):
        tr, _, _ = c.gpu_forward()
        assert rel_l2(outs[0][i], tr) < 1e-6, i


@pytest.mark.parametrize("M", [2, 4, 8])
def test_batched_tile_shapes_and_autotune_keep_the_bits(M):
    """Every tile shape of the batched kernel (R = 2 and 4 rows per thread, set
    by hand) and the autotuner's choice give the single-shot traces bit for
    bit, on a first call and on a graph replay."""
    cases = _shots(M, "spatte", nt=70)
    ref = [c.gpu_forward()[0] for c in cases]
    for kw in (dict(rows=4), dict(rows=2), dict(autotune=True)):
        outs = _batched(cases, repeat=2, **kw)
        for i in range(len(cases)):
            assert np.array_equal(outs[0][i], ref[i]), (kw, i)
            assert np.array_equal(outs[1][i], ref[i]), (kw, i)


@pytest.mark.parametrize("M", [2, 4, 8])
def test_batched_persistent_launch_keeps_the_bits(M, monkeypatch):
    """With FDWAVE_BATCH_PERSISTENT=1 the batch runs every step in one
    cooperative launch (a grid barrier between steps); traces equal the
    single-shot runs bit for bit for both tile shapes, on a long, a ragged and a
    one-step run, and the status word stays clear."""
    for nt in (70, 33, 1):
        cases = _shots(M, "spatte", nt=nt)
        ref = [c.gpu_forward()[0] for c in cases]
        monkeypatch.setenv("FDWAVE_BATCH_PERSISTENT", "1")
        try:
            for rows in (2, 4):
                st = []
                outs = _batched(cases, repeat=2, rows=rows, status=st)
                assert st == [0, 0], (nt, rows, st)
                for i in range(len(cases)):
                    assert np.array_equal(outs[0][i], ref[i]), (nt, rows, i)
                    assert np.array_equal(outs[1][i], ref[i]), (nt, rows, i)
        finally:
            monkeypatch.delenv("FDWAVE_BATCH_PERSISTENT")
