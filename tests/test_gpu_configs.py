"""Parity at the workloads' full sizes, in the launch configuration bench.py
times (default plan variant).  Where a full FP64 trajectory is too long for
the oracle, the check is one that holds at any size:

* restart: from a GPU state after n steps of the full run, a few GPU steps
  equal the oracle's steps from that same state (relative L2 <= 1e-5: the
  inputs are identical, only the steps' FP32 arithmetic differs);
* batched = single-shot runs (bitwise up to 1e-6) on the full 48-shot batch;
* FWI at 296^3 x 1200 steps: the adjoint's dot-product test, checkpoint
  interval invariance, and the oracle gradient on the full grid with fewer
  steps.
The 1001^2 workload is also run for its full 2000 steps against the oracle
for two of its stencils."""
import numpy as np
import pytest

import workloads as WL
from gpu_cases import Case, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_04882_gb300 import build
    build.build()


def _restart_check(c: Case, n_mid: int, k: int, tol=1e-5):
    """GPU state after n_mid steps, then k more steps on GPU and oracle."""
    _, st_mid, rc = c.gpu_forward(nt=n_mid)
    assert rc == 0
    assert np.all(np.isfinite(st_mid))
    assert np.abs(st_mid).max() > 0
    tr_g, st_g, rc = c.gpu_forward(nt=k, state_in=st_mid, t0=n_mid)
    assert rc == 0
    tr_o, st_o = c.oracle_forward(nt=k, state_in=st_mid, t0=n_mid)
    assert rel_l2(st_g[0], st_o[0]) < tol
    if len(c.rec) and np.abs(tr_o).max() > 0:
        assert rel_l2(tr_g, tr_o) < tol


@pytest.fixture(scope="module")
def cfg2():
    return WL.layered_random_2d()


def _case_from(pr, st, dt_taylor=True):
    import paper_2606_04882_gb300 as F
    dim = pr.dim
    dt = 0.5 * F.fd_cfl_limit(F.stencil_desc(dim, "cross", st.M)) * pr.h / pr.vmax
    return Case(pr.vel, pr.h, pr.nt, pr.nb, pr.vmax, st.shape, st.M, st.N, st.scheme,
                src=pr.src, rec=pr.rec, f0=pr.f0, dt=dt)


def test_layered_1001_all_18_stencils_restart(cfg2):
    for st in cfg2.stencils:
        c = _case_from(cfg2, st)
        _restart_check(c, n_mid=1000, k=3)


@pytest.mark.parametrize("shape,M,scheme", [("cross", 4, "spatte"), ("rhombus", 4, "displs")])
def test_layered_1001_full_run(cfg2, shape, M, scheme):
    st = WL.Stencil(shape, M, 0, scheme)
    c = _case_from(cfg2, st)
    tr, sf, rc = c.gpu_forward()
    assert rc == 0
    otr, ost = c.oracle_forward()
    assert rel_l2(tr, otr) < 1e-4
    assert rel_l2(sf[0], ost[0]) < 1e-4


def test_gradient_random_400_restart():
    pr = WL.gradient_random_3d()
    for st in pr.stencils:
        c = _case_from(pr, st)
        _restart_check(c, n_mid=750, k=2)


def test_batched_48_shots_full():
    import torch
    import paper_2606_04882_gb300 as F
    probs = WL.batched_shots_2d()
    dt = min(0.5 * F.fd_cfl_limit(F.stencil_desc(2, "cross", 4)) * p.h / p.vmax for p in probs)
    dev = torch.device("cuda")
    cases = [Case(p.vel, p.h, p.nt, p.nb, p.vmax, "cross", 4, 0, "spatte", src=p.src, rec=p.rec,
                  f0=p.f0, dt=dt) for p in probs]
    shots = []
    for c in cases:
        plan = c.plan()
        shots.append(dict(plan=plan, model=torch.from_numpy(c.vel).to(dev),
                          src_idx=plan.linear_index(c.src),
                          wavelet=torch.from_numpy(c.wavelet32()).to(dev),
                          rec_idx=plan.linear_index(c.rec),
                          traces=torch.zeros((c.nt, len(c.rec)), device=dev)))
    ws = F.workspace(F.batched_workspace_size(shots))
    F.fd_forward_batched(shots, ws)
    torch.cuda.synchronize()
    for i in (0, 17, 47):
        tr, _, rc = cases[i].gpu_forward()
        assert rc == 0
        assert rel_l2(shots[i]["traces"].cpu().numpy(), tr) < 1e-6, i
    _restart_check(cases[33], n_mid=1500, k=3)


def _fwi_case(nt=None):
    import paper_2606_04882_gb300 as F
    probs, _ = WL.fwi_3d()
    pr = probs[0]
    dt = 0.5 * F.fd_cfl_limit(F.stencil_desc(3, "cross", 4)) * pr.h / pr.vmax
    return Case(pr.vel, pr.h, nt or pr.nt, pr.nb, pr.vmax, "cross", 4, 0, "spatte", src=pr.src,
                rec=pr.rec, f0=pr.f0, dt=dt)


def _gpu_grad(c, resid, k, wavelet=None):
    import torch
    import paper_2606_04882_gb300 as F
    plan = c.plan()
    dev = torch.device("cuda")
    m = torch.from_numpy(c.vel).to(dev)
    wav = torch.from_numpy(c.wavelet32() if wavelet is None else wavelet).to(dev)
    g = torch.empty_like(m)
    wg = torch.zeros((c.nt, 1), device=dev)
    ws = F.workspace(plan.gradient_workspace_size(1, len(c.rec), k))
    F.fd_adjoint_gradient(plan, m, plan.linear_index(c.src), wav, plan.linear_index(c.rec),
                          torch.from_numpy(np.ascontiguousarray(resid, np.float32)).to(dev), k, g, ws,
                          wavelet_grad=wg)
    assert F.fd_status_read(plan, ws) == 0
    torch.cuda.synchronize()
    out = g.cpu().numpy(), wg.cpu().numpy()
    del ws
    return out


def test_fwi_256_dot_product_and_checkpoint_invariance():
    import torch
    import paper_2606_04882_gb300 as F
    c = _fwi_case()
    rng = np.random.default_rng(1)
    s = rng.standard_normal((c.nt, 1)).astype(np.float32)
    d = rng.standard_normal((c.nt, len(c.rec))).astype(np.float32)
    plan = c.plan()
    dev = torch.device("cuda")
    tr = torch.zeros((c.nt, len(c.rec)), device=dev)
    ws = F.workspace(plan.forward_workspace_size(1, len(c.rec)))
    F.fd_forward(plan, torch.from_numpy(c.vel).to(dev), plan.linear_index(c.src),
                 torch.from_numpy(s).to(dev), plan.linear_index(c.rec), tr, ws)
    g20, wg = _gpu_grad(c, d, 20, wavelet=s)
    lhs = float(np.sum(tr.cpu().numpy().astype(np.float64) * d))
    rhs = float(np.sum(s.astype(np.float64) * wg))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)
    g40, _ = _gpu_grad(c, d, 40, wavelet=s)
    assert np.array_equal(g20, g40)
    # k = nt: D of every step resident (~124 GB), no checkpoint and no recompute
    plan = c.plan()
    torch.cuda.empty_cache()
    if plan.gradient_workspace_size(1, len(c.rec), c.nt) + (8 << 30) < torch.cuda.mem_get_info()[0]:
        g_all, _ = _gpu_grad(c, d, c.nt, wavelet=s)
        assert np.array_equal(g20, g_all)


def test_fwi_256_gradient_matches_oracle_on_full_grid():
    from oracle import physics as P
    from oracle import wave as W
    c = _fwi_case(nt=40)
    resid = np.random.default_rng(2).standard_normal((c.nt, len(c.rec)))
    g, _ = _gpu_grad(c, resid, 20)
    st = c.setup()
    og, _ = W.gradient(st, c.nt, c.src, P.ricker(c.f0, c.nt, c.dt)[:, None], c.rec, resid, seg=20)
    assert rel_l2(g, og) < 1e-4
