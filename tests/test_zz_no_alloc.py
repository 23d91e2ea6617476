"""fd_forward_noalloc: the forward entry point for callers that cannot
allocate device memory (it uses the library's own 32 MiB static device
scratch instead of a caller-provided workspace).  Checked through the C ABI
against fd_forward with a workspace, on two calls in a row: the second call
reuses the array the first one left behind.  This file is collected last."""
import numpy as np
import pytest

from gpu_cases import Case, rel_l2
from workloads import smooth_velocity

pytestmark = pytest.mark.gpu
TOL = 1e-4   # the relative-L2 tolerance of the forward parity tests


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_04882_gb300 import build
    build.build()


def test_noalloc_forward_matches_workspace_forward_twice():
    import torch
    import paper_2606_04882_gb300 as F
    nz, nx = 140, 171
    vel = smooth_velocity((nz, nx), 21, 1500.0, 3000.0, sigma=4.0)
    rec = np.array([[3, x] for x in range(0, nx, 2)])
    c = Case(vel, 10.0, 160, 12, 3000.0, "rhombus", 4, 0, "displs",
             src=[[nz // 2, nx // 2], [4, 9]], rec=rec, f0=20.0)
    ref_tr, ref_st, rc = c.gpu_forward()
    assert rc == 0
    plan = c.plan()
    dev = torch.device("cuda")
    v = torch.from_numpy(c.vel).to(dev)
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    for call in range(2):
        tr = torch.full((c.nt, len(rec)), float("nan"), device=dev)
        st = torch.full((2,) + tuple(plan.padded_shape), float("nan"), device=dev)
        F.fd_forward_noalloc(plan, v, plan.linear_index(c.src), wav, plan.linear_index(c.rec), tr,
                             state_out=st)
        torch.cuda.synchronize()
        assert rel_l2(tr.cpu().numpy(), ref_tr) < TOL, call
        assert rel_l2(st.cpu().numpy(), ref_st) < TOL, call


def test_noalloc_rejects_problems_larger_than_the_static_scratch():
    import paper_2606_04882_gb300 as F
    d = F.stencil_desc(2, "cross", 4)
    plan = F.Plan((2000, 2000), 10.0, 1e-3, 5, 20, 3000.0, d)    # ~51 MB of scratch
    assert plan.forward_workspace_size(1, 1) > (32 << 20)
    with pytest.raises(F.FdError) as e:
        F.fd_forward_noalloc(plan, 0, np.array([0]), 0, np.array([0]), 0)
    assert e.value.code == F.FD_ERR_NOMEM
    assert "static scratch" in F.last_error()


def test_noalloc_device_status_is_readable():
    """A model faster than the plan's vmax is recorded in the status word in the
    static array, which fd_status_read_noalloc reads and clears; a clean call
    then reads FD_OK."""
    import torch
    import paper_2606_04882_gb300 as F
    vel = np.full((40, 50), 2000.0, np.float32)
    c = Case(vel, 10.0, 40, 4, 2500.0, "cross", 4, rec=[[2, 7]])
    plan = c.plan()
    dev = torch.device("cuda")
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    tr = torch.zeros((c.nt, 1), device=dev)
    fast = torch.full((40, 50), 2600.0, device=dev)
    F.fd_forward_noalloc(plan, fast, plan.linear_index(c.src), wav, plan.linear_index(c.rec), tr)
    assert F.fd_status_read_noalloc(plan) == F.FD_ERR_UNSTABLE
    assert "vmax" in F.last_error()
    F.fd_forward_noalloc(plan, torch.from_numpy(vel).to(dev), plan.linear_index(c.src), wav,
                         plan.linear_index(c.rec), tr)
    assert F.fd_status_read_noalloc(plan) == F.FD_OK
