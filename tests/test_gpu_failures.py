"""Failure detection on the GPU, without a GPU fault.

* A bounded device wait that runs out.  A test hook (environment variables
  read by the library on each call) shortens the waits of the 3D kernels to a
  millisecond and makes the producer warp of CTA 0 skip one ring slot.  That
  CTA's consumers then wait for copies that never come, give up, and the call
  reports FD_ERR_TIMEOUT through the status word; the producer gives up on
  their release the same way.  Every wait is bounded and no access is skipped
  or redirected, so nothing faults.  The next call on the same plan and
  workspace must be clean and match the oracle.
* Unbounded growth.  A non-finite initial state, and a model faster than the
  plan's vmax (Courant number above the von Neumann limit of Eq. full_disp),
  must come back as FD_ERR_UNSTABLE from the growth check that every step
  kernel runs on every 32nd step and the last one.
* The differentiable traces and the shot driver raise on those conditions.
"""
import numpy as np
import pytest

from gpu_cases import Case, rel_l2
from workloads import smooth_velocity

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_04882_gb300 import build
    build.build()


def _run(c, plan, ws, state_in=None):
    """fd_forward of case c on an existing plan and workspace; (traces, state, status)."""
    import torch
    import paper_2606_04882_gb300 as F
    dev = torch.device("cuda")
    vel = torch.from_numpy(c.vel).to(dev)
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    nrec = len(c.rec)
    tr = torch.zeros((c.nt, max(nrec, 1)), device=dev)
    st = torch.zeros((2,) + tuple(plan.padded_shape), device=dev)
    sin = None if state_in is None else torch.from_numpy(np.ascontiguousarray(state_in, np.float32)).to(dev)
    F.fd_forward(plan, vel, plan.linear_index(c.src), wav,
                 plan.linear_index(c.rec) if nrec else np.zeros(0, np.int64),
                 tr if nrec else None, ws, state_in=sin, state_out=st)
    rc = F.fd_status_read(plan, ws)
    return tr.cpu().numpy()[:, :nrec], st.cpu().numpy(), rc


def _case3d(shape, M, scheme, nt=40):
    nz, ny, nx = 30, 34, 40
    vel = smooth_velocity((nz, ny, nx), 5, 1500.0, 3000.0, sigma=3.0)
    rec = [[2, y, x] for y in (3, 17, 30) for x in range(0, nx, 7)]
    return Case(vel, 10.0, nt, 4, 3000.0, shape, M, 0, scheme, src=[[15, 17, 20]], rec=rec, f0=25.0)


@pytest.mark.parametrize("shape,M,scheme", [("cross", 4, "spatte"), ("cross", 8, "spatte"),
                                            ("rhombus", 4, "displs")])
def test_forced_wait_timeout_is_reported_and_the_next_call_is_clean(monkeypatch, shape, M, scheme):
    import paper_2606_04882_gb300 as F
    c = _case3d(shape, M, scheme)
    plan = c.plan()
    ws = F.workspace(plan.forward_workspace_size(len(c.src), len(c.rec)))
    monkeypatch.setenv("FDWAVE_DEBUG_WAIT_CYCLES", "2000000")
    monkeypatch.setenv("FDWAVE_DEBUG_DROP_SLOT", "0")
    _, _, rc = _run(c, plan, ws)
    assert rc == F.FD_ERR_TIMEOUT
    assert "timed out" in F.last_error()
    monkeypatch.delenv("FDWAVE_DEBUG_WAIT_CYCLES")
    monkeypatch.delenv("FDWAVE_DEBUG_DROP_SLOT")
    tr, st, rc = _run(c, plan, ws)
    assert rc == F.FD_OK
    otr, ost = c.oracle_forward(threads=8)
    assert rel_l2(tr, otr) < TOL and rel_l2(st[0], ost[0]) < TOL


def test_forced_wait_timeout_in_the_gradient(monkeypatch):
    import torch
    import paper_2606_04882_gb300 as F
    c = _case3d("cross", 4, "spatte", nt=24)
    plan = c.plan()
    dev = torch.device("cuda")
    vel = torch.from_numpy(c.vel).to(dev)
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    resid = torch.ones((c.nt, len(c.rec)), device=dev)
    g = torch.empty_like(vel)
    ws = F.workspace(plan.gradient_workspace_size(1, len(c.rec), 8))
    monkeypatch.setenv("FDWAVE_DEBUG_WAIT_CYCLES", "2000000")
    monkeypatch.setenv("FDWAVE_DEBUG_DROP_SLOT", "1")
    F.fd_adjoint_gradient(plan, vel, plan.linear_index(c.src), wav, plan.linear_index(c.rec),
                          resid, 8, g, ws)
    assert F.fd_status_read(plan, ws) == F.FD_ERR_TIMEOUT
    monkeypatch.delenv("FDWAVE_DEBUG_WAIT_CYCLES")
    monkeypatch.delenv("FDWAVE_DEBUG_DROP_SLOT")
    F.fd_adjoint_gradient(plan, vel, plan.linear_index(c.src), wav, plan.linear_index(c.rec),
                          resid, 8, g, ws)
    assert F.fd_status_read(plan, ws) == F.FD_OK
    assert torch.isfinite(g).all()


@pytest.mark.parametrize("dim", [2, 3])
def test_non_finite_state_is_reported_unstable(dim):
    import paper_2606_04882_gb300 as F
    n = (50, 60) if dim == 2 else (20, 22, 26)
    vel = smooth_velocity(n, 3, 1500.0, 3000.0, sigma=3.0)
    c = Case(vel, 10.0, 10, 3, 3000.0, "cross", 4, src=np.zeros((0, dim)), rec=None)
    plan = c.plan()
    ws = F.workspace(plan.forward_workspace_size(0, 0))
    st0 = np.zeros((2,) + tuple(plan.padded_shape), np.float32)
    st0[(0,) + tuple(s // 2 for s in plan.padded_shape)] = np.nan
    _, _, rc = _run(c, plan, ws, state_in=st0)
    assert rc == F.FD_ERR_UNSTABLE
    assert "non-finite" in F.last_error()
    _, _, rc = _run(c, plan, ws)          # a clean run on the same workspace
    assert rc == F.FD_OK


@pytest.mark.parametrize("dim", [2, 3])
def test_growth_beyond_the_stability_limit_is_reported(dim):
    """The plan is built for vmax and dt = 0.5 C_max h / vmax; a model 2.5 times
    faster runs at 1.25 C_max, where the leapfrog amplifies the shortest waves
    by up to 4 per step.  The status must say so (velocity and growth)."""
    import paper_2606_04882_gb300 as F
    n = (60, 70) if dim == 2 else (24, 26, 28)
    vmax = 2000.0
    c = Case(np.full(n, 2.5 * vmax, np.float32), 10.0, 200, 4, vmax, "cross", 4,
             rec=[[2] * (dim - 1) + [5]])
    plan = c.plan()
    ws = F.workspace(plan.forward_workspace_size(1, 1))
    _, _, rc = _run(c, plan, ws)
    assert rc == F.FD_ERR_UNSTABLE
    assert "grew without bound" in F.last_error()


def test_gradient_growth_is_reported():
    import torch
    import paper_2606_04882_gb300 as F
    vmax = 2000.0
    c = Case(np.full((50, 60), 2.5 * vmax, np.float32), 10.0, 150, 4, vmax, "cross", 4,
             rec=[[2, x] for x in range(0, 60, 6)])
    plan = c.plan()
    dev = torch.device("cuda")
    vel = torch.from_numpy(c.vel).to(dev)
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    g = torch.empty_like(vel)
    ws = F.workspace(plan.gradient_workspace_size(1, len(c.rec), 10))
    F.fd_adjoint_gradient(plan, vel, plan.linear_index(c.src), wav, plan.linear_index(c.rec),
                          torch.ones((c.nt, len(c.rec)), device=dev), 10, g, ws)
    assert F.fd_status_read(plan, ws) == F.FD_ERR_UNSTABLE


def test_differentiable_traces_raise_on_device_conditions():
    import torch
    import paper_2606_04882_gb300 as F
    vmax = 2000.0
    n = (40, 48)
    c = Case(np.full(n, 1800.0, np.float32), 10.0, 60, 4, vmax, "cross", 4,
             rec=[[2, x] for x in range(0, 48, 4)])
    plan = c.plan()
    dev = torch.device("cuda")
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    fast = torch.full(n, 1.0 / (2.5 * vmax) ** 2, device=dev, requires_grad=True)
    with pytest.raises(F.FdError) as e:
        F.acoustic_traces(fast, plan, plan.linear_index(c.src), wav, plan.linear_index(c.rec))
    assert e.value.code == F.FD_ERR_UNSTABLE
    ok = torch.full(n, 1.0 / 1800.0 ** 2, device=dev, requires_grad=True)
    tr = F.acoustic_traces(ok, plan, plan.linear_index(c.src), wav, plan.linear_index(c.rec))
    tr.square().sum().backward()
    assert torch.isfinite(ok.grad).all()
