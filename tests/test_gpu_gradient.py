"""Adjoint / FWI-gradient parity of the CUDA path against the FP64 oracle,
the dot-product test of the GPU adjoint, checkpoint invariance and the
autograd.Function."""
import numpy as np
import pytest

from gpu_cases import Case, rel_l2
from oracle import physics as P
from oracle import wave as W
from workloads import smooth_velocity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_04882_gb300 import build
    build.build()


def _gpu_gradient(c: Case, resid, k, model_kind=0, model=None):
    import torch
    import paper_2606_04882_gb300 as F
    plan = c.plan()
    dev = torch.device("cuda")
    m = torch.from_numpy(np.ascontiguousarray(model if model is not None else c.vel, np.float32)).to(dev)
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    r = torch.from_numpy(np.ascontiguousarray(resid, np.float32)).to(dev)
    grad = torch.empty_like(m)
    tr = torch.zeros((c.nt, len(c.rec)), device=dev)
    wg = torch.zeros((c.nt, len(c.src)), device=dev)
    ws = F.workspace(plan.gradient_workspace_size(len(c.src), len(c.rec), k))
    F.fd_adjoint_gradient(plan, m, plan.linear_index(c.src), wav, plan.linear_index(c.rec), r, k,
                          grad, ws, traces=tr, wavelet_grad=wg, model_kind=model_kind)
    rc = F.fd_status_read(plan, ws)
    torch.cuda.synchronize()
    return grad.cpu().numpy(), tr.cpu().numpy(), wg.cpu().numpy(), rc


def _case(dim, nt, seed=5, shape="cross", M=4, scheme="spatte"):
    n = (60, 71) if dim == 2 else (26, 29, 33)
    vel = smooth_velocity(n, seed, 1500.0, 3000.0, sigma=3.0)
    rng = np.random.default_rng(seed)
    rec = np.stack([np.full(25, 2)] + [rng.integers(0, s, 25) for s in n[1:]], axis=1)
    src = np.array([[3] + [s // 2 for s in n[1:]]])
    return Case(vel, 10.0, nt, 6, 3000.0, shape, M, 0, scheme, src=src, rec=rec, f0=25.0)


@pytest.mark.parametrize("dim,shape,M,scheme", [(2, "cross", 4, "spatte"), (2, "rhombus", 4, "displs"),
                                               (3, "cross", 4, "spatte"), (3, "cross", 2, "spatte")])
def test_gradient_matches_oracle(dim, shape, M, scheme):
    c = _case(dim, 120 if dim == 2 else 80, shape=shape, M=M, scheme=scheme)
    resid = np.random.default_rng(1).standard_normal((c.nt, len(c.rec)))
    g, tr, wg, rc = _gpu_gradient(c, resid, k=13)
    assert rc == 0
    st = c.setup()
    wav = P.ricker(c.f0, c.nt, c.dt)[:, None]
    og, adj = W.gradient(st, c.nt, c.src, wav, c.rec, resid, adj_pos=c.src, threads=8)
    assert rel_l2(g, og) < 1e-4, rel_l2(g, og)
    otr = W.forward(st, c.nt, c.src, wav, c.rec, threads=8)[0]
    assert rel_l2(tr, otr) < 1e-4
    # dJ/ds(t^n) = nu^{n+1}(x_s) tau^2 / h^dim
    assert rel_l2(wg, adj * c.dt ** 2 / c.h ** dim) < 1e-4


@pytest.mark.parametrize("dim", [2, 3])
def test_dot_product_of_gpu_adjoint(dim):
    """<F s, d> = <s, F* d> for the map wavelet -> traces, both sides computed
    by the GPU (F by fd_forward, F* by the adjoint's wavelet gradient)."""
    import torch
    import paper_2606_04882_gb300 as F
    c = _case(dim, 100 if dim == 2 else 60, seed=8)
    rng = np.random.default_rng(2)
    s = rng.standard_normal((c.nt, 1)).astype(np.float32)
    d = rng.standard_normal((c.nt, len(c.rec))).astype(np.float32)
    plan = c.plan()
    dev = torch.device("cuda")
    vel = torch.from_numpy(c.vel).to(dev)
    tr = torch.zeros((c.nt, len(c.rec)), device=dev)
    ws = F.workspace(plan.forward_workspace_size(1, len(c.rec)))
    F.fd_forward(plan, vel, plan.linear_index(c.src), torch.from_numpy(s).to(dev),
                 plan.linear_index(c.rec), tr, ws)
    _, _, wg, rc = _gpu_gradient(c, d, k=10)
    lhs = float(np.sum(tr.cpu().numpy().astype(np.float64) * d))
    rhs = float(np.sum(s.astype(np.float64) * wg))
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs), (lhs, rhs)


@pytest.mark.parametrize("dim,shape", [(2, "cross"), (3, "cross"), (3, "rhombus")])
def test_checkpoint_interval_is_bitwise_invariant(dim, shape):
    """The store-D recompute reproduces the forward sweep bit for bit, so the
    gradient does not depend on the checkpoint interval (in 3D the forward,
    store-D and adjoint sweeps run different kernel instantiations)."""
    c = _case(dim, 90 if dim == 2 else 70, shape=shape)
    resid = np.random.default_rng(4).standard_normal((c.nt, len(c.rec)))
    g1, tr1, wg1, _ = _gpu_gradient(c, resid, k=1)
    for k in (7, 30, 90, 500):   # k >= nt keeps every D and recomputes nothing
        g, tr, wg, rc = _gpu_gradient(c, resid, k=k)
        assert rc == 0
        assert np.array_equal(g1, g), k
        assert np.array_equal(tr1, tr) and np.array_equal(wg1, wg), k


@pytest.mark.parametrize("dim,shape", [(2, "cross"), (3, "cross"), (3, "rhombus")])
def test_split_gradient_equals_one_call(dim, shape):
    """fd_gradient_forward (forward sweep keeping every D, traces out) then
    fd_gradient_adjoint (adjoint sweep for a residual) give the traces,
    gradient and wavelet gradient of fd_adjoint_gradient bit for bit; one
    stored forward serves two adjoints; two stored forwards on one plan are
    both usable; a workspace rewritten by fd_forward is refused."""
    import torch
    import paper_2606_04882_gb300 as F
    c = _case(dim, 60, shape=shape)
    resid = np.random.default_rng(12).standard_normal((c.nt, len(c.rec)))
    g1, tr1, wg1, rc = _gpu_gradient(c, resid, k=7)
    assert rc == 0
    plan = c.plan()
    dev = torch.device("cuda")
    m = torch.from_numpy(c.vel).to(dev)
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    r = torch.from_numpy(resid.astype(np.float32)).to(dev)
    si, ri = plan.linear_index(c.src), plan.linear_index(c.rec)
    need = plan.gradient_workspace_size(len(c.src), len(c.rec), c.nt)
    wss = [F.workspace(need), F.workspace(need)]
    for ws in wss:
        tr = torch.zeros((c.nt, len(c.rec)), device=dev)
        F.fd_gradient_forward(plan, m, si, wav, ri, tr, ws)
        assert F.fd_status_read(plan, ws) == 0
        assert np.array_equal(tr.cpu().numpy(), tr1)
    for ws in (wss[0], wss[0], wss[1]):
        g = torch.empty_like(m)
        wg = torch.zeros((c.nt, len(c.src)), device=dev)
        F.fd_gradient_adjoint(plan, si, ri, r, g, ws, wavelet_grad=wg)
        assert F.fd_status_read(plan, ws) == 0
        assert np.array_equal(g.cpu().numpy(), g1)
        assert np.array_equal(wg.cpu().numpy(), wg1)
    F.fd_forward(plan, m, si, wav, ri, torch.zeros((c.nt, len(c.rec)), device=dev), wss[1])
    with pytest.raises(F.FdError) as e:
        F.fd_gradient_adjoint(plan, si, ri, r, torch.empty_like(m), wss[1])
    assert e.value.code == F.FD_ERR_ARG


def test_slowness_parameterisation_and_autograd():
    import torch
    import paper_2606_04882_gb300 as F
    c = _case(2, 80, seed=3)
    m = (1.0 / c.vel.astype(np.float64) ** 2).astype(np.float32)
    resid = np.random.default_rng(6).standard_normal((c.nt, len(c.rec)))
    g_v = _gpu_gradient(c, resid, k=8)[0]
    g_m = _gpu_gradient(c, resid, k=8, model_kind=F.FD_MODEL_SLOWNESS2, model=m)[0]
    assert rel_l2(g_m, g_v) < 1e-5
    plan = c.plan()
    mt = torch.from_numpy(m).cuda().requires_grad_(True)
    wav = torch.from_numpy(c.wavelet32()).cuda()
    tr = F.acoustic_traces(mt, plan, plan.linear_index(c.src), wav, plan.linear_index(c.rec), k=8)
    loss = (tr * torch.from_numpy(resid.astype(np.float32)).cuda()).sum()
    loss.backward()
    assert rel_l2(mt.grad.cpu().numpy(), g_m) < 1e-6
    # the default interval (every D kept when it fits) gives the same bits
    g8 = mt.grad.clone()
    mt.grad = None
    tr = F.acoustic_traces(mt, plan, plan.linear_index(c.src), wav, plan.linear_index(c.rec))
    (tr * torch.from_numpy(resid.astype(np.float32)).cuda()).sum().backward()
    assert torch.equal(mt.grad, g8)


def test_shot_driver_on_the_gpu_matches_the_oracle_sum():
    """shots.gpu_shot_fn (forward, residual d - d_obs, adjoint gradient of each
    shot, with the device status checked after each call), summed over three
    shots by shots.misfit_and_gradient in one process, against the FP64
    oracle's misfit J = sum_s 1/2 ||d_s - d_obs,s||^2 and its dJ/dm."""
    import torch
    import paper_2606_04882_gb300 as F
    from paper_2606_04882_gb300.shots import gpu_shot_fn, misfit_and_gradient
    n, nb, nt, h, vmax, f0 = (48, 64), 6, 150, 10.0, 3000.0, 25.0
    m32 = (1.0 / smooth_velocity(n, 4, 1500.0, 2900.0, sigma=3.0).astype(np.float64) ** 2).astype(np.float32)
    v = (1.0 / np.sqrt(m32.astype(np.float64))).astype(np.float32)
    vt = smooth_velocity(n, 9, 1500.0, 2900.0, sigma=2.0)
    srcs = [np.array([[2, x]]) for x in (5, 30, 58)]
    rec = np.array([[2, x] for x in range(n[1])])
    c = Case(v, h, nt, nb, vmax, "cross", 4, src=srcs[0], rec=rec, f0=f0)
    st, stt = c.setup(), Case(vt, h, nt, nb, vmax, "cross", 4, rec=rec, dt=c.dt).setup()
    wav64 = P.ricker(f0, nt, c.dt)[:, None]
    dobs = [W.forward(stt, nt, s, wav64, rec, threads=8)[0] for s in srcs]
    J_o, g_o = 0.0, np.zeros(n)
    for s, d in zip(srcs, dobs):
        r = W.forward(st, nt, s, wav64, rec, threads=8)[0] - d
        J_o += 0.5 * float(np.sum(r ** 2))
        g_o += W.gradient(st, nt, s, wav64, rec, r, threads=8)[0]
    dev = torch.device("cuda")
    plan = c.plan()
    m = torch.from_numpy(m32).to(dev)
    wav = torch.from_numpy(F.fd_ricker(f0, c.dt, nt)[:, None].copy()).to(dev)
    run = gpu_shot_fn(plan, m, [plan.linear_index(s) for s in srcs], [wav] * 3,
                      plan.linear_index(rec), [torch.from_numpy(d.astype(np.float32)).to(dev) for d in dobs],
                      k=16)
    J, g = misfit_and_gradient(m, 3, run)
    assert abs(J - J_o) < 1e-4 * J_o
    assert rel_l2(g.cpu().numpy(), g_o) < 1e-4
    # the default (every D kept, one forward sweep per shot) gives the same bits
    run = gpu_shot_fn(plan, m, [plan.linear_index(s) for s in srcs], [wav] * 3,
                      plan.linear_index(rec), [torch.from_numpy(d.astype(np.float32)).to(dev) for d in dobs])
    J2, g2 = misfit_and_gradient(m, 3, run)
    assert J2 == J and torch.equal(g2, g)


@pytest.mark.parametrize("shape,M,scheme", [("rhombus", 4, "displs"), ("cross", 4, "spatte")])
def test_gradient_is_bitwise_equal_across_3d_variants(shape, M, scheme):
    """The forward, recompute and adjoint sweeps of every 3D kernel variant
    give the same gradient bit for bit."""
    import torch
    import paper_2606_04882_gb300 as F
    c = _case(3, 40, shape=shape, M=M, scheme=scheme)
    resid = np.random.default_rng(2).standard_normal((c.nt, len(c.rec))).astype(np.float32)
    plan = c.plan()
    dev = torch.device("cuda")
    m = torch.from_numpy(c.vel).to(dev)
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    r = torch.from_numpy(resid).to(dev)
    ref = None
    for v in plan.variants():
        plan.set_variant(v, 0)
        g = torch.empty_like(m)
        ws = F.workspace(plan.gradient_workspace_size(1, len(c.rec), 9))
        F.fd_adjoint_gradient(plan, m, plan.linear_index(c.src), wav, plan.linear_index(c.rec), r, 9,
                              g, ws)
        assert F.fd_status_read(plan, ws) == 0
        g = g.cpu().numpy()
        if ref is None:
            ref = g
        assert np.array_equal(g, ref), v


@pytest.mark.parametrize("shape,M,scheme,rows", [("cross", 4, "spatte", 2), ("cross", 4, "spatte", 4),
                                                 ("cross", 2, "spatte", 2), ("cross", 8, "spatte", 4),
                                                 ("rhombus", 4, "displs", 0)])
def test_batched_gradient_equals_per_shot_gradients(shape, M, scheme, rows):
    """fd_adjoint_gradient_batched over five shots on two grids of different
    size (one launch per step over every shot's tiles for the cross, with the
    batched kernel's 64 x 32 or 64 x 64 tiles; shot by shot for the rhombus)
    gives each shot's gradient and traces bit for bit as fd_adjoint_gradient
    does, and one shot matches the FP64 oracle."""
    import torch
    import paper_2606_04882_gb300 as F
    dev = torch.device("cuda")
    nt, nb, h, vmax, k = 90, 6, 10.0, 3000.0, 11
    grids = [(61, 83), (45, 130)]
    dt = min(Case(np.zeros(g, np.float32), h, nt, nb, vmax, "cross", M).dt for g in grids)
    shots, ref = [], []
    for i in range(5):
        g = grids[i % 2]
        vel = smooth_velocity(g, 30 + i, 1500.0, 2900.0, sigma=3.0)
        rng = np.random.default_rng(40 + i)
        rec = np.stack([np.full(20, 2), rng.integers(0, g[1], 20)], axis=1)
        src = np.array([[3, (7 + 13 * i) % g[1]]])
        c = Case(vel, h, nt, nb, vmax, shape, M, 0, scheme, src=src, rec=rec, f0=25.0, dt=dt)
        plan = c.plan()
        resid = torch.from_numpy(rng.standard_normal((nt, len(rec))).astype(np.float32)).to(dev)
        d = dict(plan=plan, model=torch.from_numpy(c.vel).to(dev), src_idx=plan.linear_index(src),
                 wavelet=torch.from_numpy(c.wavelet32()).to(dev), rec_idx=plan.linear_index(rec),
                 resid=resid, grad=torch.full(g, float("nan"), device=dev),
                 traces=torch.full((nt, len(rec)), float("nan"), device=dev))
        shots.append(d)
        g1 = torch.empty(g, device=dev)
        tr1 = torch.zeros((nt, len(rec)), device=dev)
        ws1 = F.workspace(plan.gradient_workspace_size(1, len(rec), k))
        F.fd_adjoint_gradient(plan, d["model"], d["src_idx"], d["wavelet"], d["rec_idx"], resid, k, g1,
                              ws1, traces=tr1)
        assert F.fd_status_read(plan, ws1) == 0
        ref.append((g1.cpu().numpy(), tr1.cpu().numpy(), c, resid.cpu().numpy()))
    if rows:
        F.fd_forward_batched_set_variant(shots, rows)
    ws = F.workspace(F.batched_gradient_workspace_size(shots, k))
    F.fd_adjoint_gradient_batched(shots, k, ws)
    assert F.fd_status_read(shots[0]["plan"], ws) == 0
    for d, (g1, tr1, _, _) in zip(shots, ref):
        assert np.array_equal(d["grad"].cpu().numpy(), g1)
        assert np.array_equal(d["traces"].cpu().numpy(), tr1)
    # ckpt_every >= nt: every shot's D kept, no checkpoint and no recompute, the same bits
    del ws
    ws = F.workspace(F.batched_gradient_workspace_size(shots, nt))
    for d in shots:
        d["grad"].fill_(float("nan"))
        d["traces"].fill_(float("nan"))
    F.fd_adjoint_gradient_batched(shots, nt, ws)
    assert F.fd_status_read(shots[0]["plan"], ws) == 0
    for d, (g1, tr1, _, _) in zip(shots, ref):
        assert np.array_equal(d["grad"].cpu().numpy(), g1)
        assert np.array_equal(d["traces"].cpu().numpy(), tr1)
    g1, _, c, resid = ref[3]
    og, _ = W.gradient(c.setup(), nt, c.src, P.ricker(c.f0, nt, c.dt)[:, None], c.rec,
                       resid.astype(np.float64), threads=8)
    assert rel_l2(g1, og) < 1e-4


@pytest.mark.parametrize("shape,M,N,scheme", [("cross_rhombus", 4, 2, "displs"), ("cross", 5, 0, "spatte")])
def test_gradient_3d_generic_kernel_matches_oracle(shape, M, N, scheme):
    """The generic 3D kernel's recompute and adjoint modes: gradient parity with
    the oracle's exact discrete adjoint."""
    n = (22, 20, 26)
    vel = smooth_velocity(n, 31, 1500.0, 3000.0, sigma=3.0)
    rng = np.random.default_rng(31)
    rec = np.stack([np.full(18, 2), rng.integers(0, n[1], 18), rng.integers(0, n[2], 18)], axis=1)
    c = Case(vel, 10.0, 40, 5, 3000.0, shape, M, N, scheme, src=[[3, 10, 13]], rec=rec, f0=25.0)
    resid = rng.standard_normal((c.nt, len(rec)))
    g, tr, wg, rc = _gpu_gradient(c, resid, k=7)
    assert rc == 0
    og, _ = W.gradient(c.setup(), c.nt, c.src, P.ricker(c.f0, c.nt, c.dt)[:, None], c.rec, resid,
                       threads=8)
    assert rel_l2(g, og) < 1e-4
