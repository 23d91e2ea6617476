"""GPU evaluation metrics (fd_error_norms, fd_dft_gamma) against the FP64
oracle's, on traces of two stencils' runs and on synthetic gathers of the
1001^2 workload's size (2000 samples x 1001 receivers)."""
import numpy as np
import pytest

from gpu_cases import Case
from oracle import metrics as X
from workloads import smooth_velocity

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_04882_gb300 import build
    build.build()


def _check_gamma(num, ref, nfreq=0):
    import torch
    import paper_2606_04882_gb300 as F
    dev = torch.device("cuda")
    tn = torch.from_numpy(np.ascontiguousarray(num, np.float32)).to(dev)
    tr = torch.from_numpy(np.ascontiguousarray(ref, np.float32)).to(dev)
    g, norms, agg, (sn, sr) = F.fd_dft_gamma(tn, tr, nfreq)
    torch.cuda.synchronize()
    n32, r32 = num.astype(np.float32), ref.astype(np.float32)
    og, onorm, oavg, omax = X.dft_gamma(n32, r32, nfreq or None)
    nf = og.shape[1]
    An = X.dft(n32, nf).T
    spec = sn.cpu().numpy()
    assert np.allclose(spec[..., 0] + 1j * spec[..., 1], An, rtol=1e-10,
                       atol=1e-10 * np.abs(An).max())
    assert np.allclose(norms.cpu().numpy(), onorm, rtol=1e-9, atol=1e-12)
    assert np.allclose(agg.cpu().numpy(), [oavg, omax], rtol=1e-9, atol=1e-12)
    # gamma entry by entry, except where the phase difference sits at +-pi
    # (either sign is the same wrapped value)
    d = np.angle(X.dft(n32, nf)) - np.angle(X.dft(r32, nf))
    d = np.where(d > np.pi, d - 2 * np.pi, np.where(d < -np.pi, d + 2 * np.pi, d)).T
    edge = np.abs(np.abs(d) - np.pi) < 1e-6
    gg = g.cpu().numpy()
    assert np.allclose(gg[~edge], og[~edge], atol=2e-6)
    assert np.allclose(np.abs(gg[edge]), np.abs(og[edge]), atol=2e-6)
    return gg, norms.cpu().numpy()


def test_dft_gamma_of_two_stencils_runs():
    """Traces of Cross(4) Taylor (numerical) against Cross(8) Taylor (reference)."""
    nz, nx = 90, 140
    vel = smooth_velocity((nz, nx), 21, 1500.0, 3000.0, sigma=4.0)
    rec = [[3, x] for x in range(0, nx, 4)]
    outs = []
    for M in (4, 8):
        c = Case(vel, 10.0, 400, 12, 3000.0, "cross", M, 0, "spatte", src=[[3, nx // 2]],
                 rec=rec, f0=25.0, dt=1.0e-3)
        tr, _, rc = c.gpu_forward()
        assert rc == 0
        outs.append(tr)
    g, norms = _check_gamma(outs[0], outs[1])
    assert norms.max() > 0
    _check_gamma(outs[0], outs[1], nfreq=57)


def test_dft_gamma_edge_cases():
    rng = np.random.default_rng(4)
    u = rng.standard_normal((64, 5))
    g, norms = _check_gamma(u, u)
    assert np.all(g == 0) and np.all(norms == 0)
    z = u.copy()
    z[:, 2] = 0.0                                   # a zero numerical trace: gamma 0
    g, norms = _check_gamma(z, u)
    assert np.all(g[2] == 0) and norms[2] == 0
    _check_gamma(u[:1], u[:1], nfreq=1)             # a single sample


def test_dft_gamma_at_workload_size():
    rng = np.random.default_rng(6)
    ref = rng.standard_normal((2000, 1001)).cumsum(axis=0) * 1e-2
    num = np.roll(ref, 2, axis=0) + 1e-3 * rng.standard_normal(ref.shape)
    _check_gamma(num, ref)


@pytest.mark.parametrize("n", [1, 1000, 3_000_001])
def test_error_norms_match_oracle(n):
    import torch
    import paper_2606_04882_gb300 as F
    rng = np.random.default_rng(n)
    a = rng.standard_normal(n).astype(np.float32)
    b = (a + 1e-3 * rng.standard_normal(n)).astype(np.float32)
    s1, s2 = X.snapshot_scales(10.0)
    out = F.fd_error_norms(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), s1, s2)
    got = out.cpu().numpy()
    exp = X.error_norms(a, b, s1, s2)
    assert np.allclose(got, exp, rtol=1e-12, atol=0)


# --- wavelet (CWT) dispersion metric -------------------------------------------------


def _check_cwt(num, ref, nscale=0, omega0=6.0):
    import torch
    import paper_2606_04882_gb300 as F
    dev = torch.device("cuda")
    tn = torch.from_numpy(np.ascontiguousarray(num, np.float32)).to(dev)
    tr = torch.from_numpy(np.ascontiguousarray(ref, np.float32)).to(dev)
    g, norms, agg, amax, (sn, sr) = F.fd_cwt_gamma(tn, tr, nscale, omega0)
    torch.cuda.synchronize()
    n32, r32 = num.astype(np.float32), ref.astype(np.float32)
    ns = nscale or num.shape[0] // 2 + 1
    og, onorm, oavg, omax, oamax = X.cwt_gamma(n32, r32, ns, omega0)
    for got, sig in ((sn, n32), (sr, r32)):
        S = X.cwt(sig, ns, omega0)
        gs = got.cpu().numpy()
        tol = 1e-10 * max(np.abs(S).max(), 1e-300)
        assert np.abs(gs[..., 0] + 1j * gs[..., 1] - S).max() <= tol
    assert np.allclose(amax.cpu().numpy(), oamax, rtol=1e-10, atol=0)
    assert np.allclose(norms.cpu().numpy(), onorm, rtol=1e-9, atol=1e-12)
    assert np.allclose(agg.cpu().numpy(), [oavg, omax], rtol=1e-9, atol=1e-12)
    # gamma entry by entry, except where the phase difference sits at +-pi
    Sn, Sr = X.cwt(n32, ns, omega0), X.cwt(r32, ns, omega0)
    d = np.angle(Sn) - np.angle(Sr)
    d = np.where(d > np.pi, d - 2 * np.pi, np.where(d < -np.pi, d + 2 * np.pi, d))
    edge = np.abs(np.abs(d) - np.pi) < 1e-6
    gg = g.cpu().numpy()
    assert np.allclose(gg[~edge], og[~edge], atol=2e-6)
    assert np.allclose(np.abs(gg[edge]), np.abs(og[edge]), atol=2e-6)
    return gg, norms.cpu().numpy()


def test_cwt_gamma_of_two_stencils_runs():
    """Traces of Cross(4) Taylor (numerical) against Cross(8) Taylor (reference)."""
    nz, nx = 90, 140
    vel = smooth_velocity((nz, nx), 21, 1500.0, 3000.0, sigma=4.0)
    rec = [[3, x] for x in range(0, nx, 4)]
    outs = []
    for M in (4, 8):
        c = Case(vel, 10.0, 400, 12, 3000.0, "cross", M, 0, "spatte", src=[[3, nx // 2]],
                 rec=rec, f0=25.0, dt=1.0e-3)
        tr, _, rc = c.gpu_forward()
        assert rc == 0
        outs.append(tr)
    g, norms = _check_cwt(outs[0], outs[1])
    assert norms.max() > 0
    _check_cwt(outs[0], outs[1], nscale=57, omega0=8.0)


def test_cwt_gamma_edge_cases():
    rng = np.random.default_rng(12)
    u = rng.standard_normal((64, 5))
    g, norms = _check_cwt(u, u)
    assert np.all(g == 0) and np.all(norms == 0)
    z = u.copy()
    z[:, 2] = 0.0                                   # a zero numerical trace: gamma 0
    g, norms = _check_cwt(z, u)
    assert np.all(g[2] == 0) and norms[2] == 0
    _check_cwt(u[:1], u[:1], nscale=1)              # a single sample: no positive line
    _check_cwt(u[:2], u[:2][::-1].copy(), nscale=2)
    _check_cwt(u[:3], u[:3][::-1].copy(), nscale=3)  # odd nt


def test_cwt_gamma_single_trace_at_workload_length():
    """One trace of 2000 samples at all 1001 scales (the paper's analysis at
    one point), and a trace long enough that its DFT lines take more than
    48 KB of shared memory."""
    rng = np.random.default_rng(13)
    ref = rng.standard_normal((2000, 1)).cumsum(axis=0) * 1e-2
    num = np.roll(ref, 2, axis=0) + 1e-3 * rng.standard_normal(ref.shape)
    _check_cwt(num, ref)
    ref = rng.standard_normal((8000, 1)).cumsum(axis=0) * 1e-2
    num = np.roll(ref, 3, axis=0)
    _check_cwt(num, ref, nscale=16)


def test_cwt_gamma_rejects_bad_arguments():
    import torch
    import paper_2606_04882_gb300 as F
    t = torch.zeros((64, 2), dtype=torch.float32, device="cuda")
    with pytest.raises(F.FdError):
        F.fd_cwt_gamma(t, t, nscale=65)                 # more scales than samples
    with pytest.raises(F.FdError):
        F.fd_cwt_gamma(t, t, omega0=0.0)
    big = torch.zeros((29056, 1), dtype=torch.float32, device="cuda")
    with pytest.raises(F.FdError):
        F.fd_cwt_gamma(big, big, nscale=1)              # DFT lines exceed shared memory
