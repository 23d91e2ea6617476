"""Pins of the oracle's time loop, source, damping and adjoint (CPU only).

* exact discrete plane waves (undamped and with a uniform damping term) pin
  the stencil application, the leapfrog update, the damping discretisation
  and the dispersion relation of Eq. full_disp together;
* the analytic 2D/3D Green's functions pin source scaling, sign and timing;
* the von Neumann bound is checked on both sides of the stability limit;
* the adjoint is pinned by the dot-product test and by finite differences of
  the misfit, and checkpointing by agreement with the store-all schedule.
"""
import math

import numpy as np
import pytest

from oracle import physics as P
from oracle import stencil as S
from oracle import wave as W


def _setup(n, dim, C, shape="cross", M=4, N=0, scheme="spatte", nb=0, h=10.0):
    """Uniform model with Courant number C (kappa = C^2 everywhere)."""
    v = 1500.0
    dt = C * h / v
    vel = np.full((n,) * dim, v, dtype=np.float32)
    return W.Setup(vel, h, dt, nb, v, dim, shape, M, N, scheme)


def _grid(n, dim):
    return np.meshgrid(*([np.arange(n, dtype=np.float64)] * dim), indexing="ij")


@pytest.mark.parametrize("dim,shape,M,scheme,k", [
    (2, "cross", 4, "spatte", (0.31, 0.57)),
    (2, "rhombus", 4, "displs", (0.9, -0.4)),
    (2, "square", 2, "dispte", (0.2, 1.1)),
    (3, "cross", 2, "spatte", (0.3, 0.5, -0.7)),
    (3, "rhombus", 3, "displs", (0.6, 0.2, 0.4)),
])
def test_discrete_plane_wave_is_exact(dim, shape, M, scheme, k):
    n, nsteps, C = (48 if dim == 2 else 26), 4, 0.3
    st = _setup(n, dim, C, shape, M, 0, scheme)
    X = _grid(n, dim)
    phase = sum(ki * xi for ki, xi in zip(k, X))
    Sk = S.symbol(st.points, np.array([k]))[0]
    wt = math.acos(1.0 + 0.5 * C * C * Sk)          # omega tau, Eq. full_disp
    _, un, _ = W.forward(st, nsteps, None, None, None, u0=np.cos(phase),
                         um1=np.cos(phase + wt), threads=4)
    exact = np.cos(phase - nsteps * wt)
    r = M * nsteps
    inner = tuple(slice(r, n - r) for _ in range(dim))
    assert np.max(np.abs(un[inner] - exact[inner])) < 1e-11


def test_damped_plane_wave_is_exact():
    """With uniform gamma the mode mu^n e^{ik.x} solves the damped scheme iff
    (1 + g) mu^2 - (2 + C^2 S) mu + (1 - g) = 0 (centred u_t)."""
    n, nsteps, C, g = 48, 5, 0.35, 0.07
    st = _setup(n, 2, C)
    st.gamma = np.full(st.pshape, g)
    k = np.array([0.45, 0.8])
    Z, X = _grid(n, 2)
    phase = k[0] * Z + k[1] * X
    Sk = S.symbol(st.points, k[None])[0]
    mu = np.roots([1 + g, -(2 + C * C * Sk), 1 - g])[0]
    assert abs(mu) < 1
    u0 = np.real(np.exp(1j * phase))
    um1 = np.real(np.exp(1j * phase) / mu)
    _, un, _ = W.forward(st, nsteps, None, None, None, u0=u0, um1=um1, threads=4)
    exact = np.real(mu ** nsteps * np.exp(1j * phase))
    r = 4 * nsteps
    assert np.max(np.abs(un[r:-r, r:-r] - exact[r:-r, r:-r])) < 1e-12


def test_green_function_2d():
    """u_tt - c^2 Lap u = s(t) delta(x): u(r,t) = 1/(2 pi c^2) *
    int_0^{acosh(ct/r)} s(t - (r/c) cosh xi) dxi (2D Green's function
    convolved with the wavelet)."""
    from scipy.integrate import quad
    n, h, c, f0, M = 241, 5.0, 1500.0, 15.0, 8
    pw = S.expand(2, "cross", M, 0, S.weights(2, "cross", M))
    dt = 0.5 * S.cfl_limit(pw, 2) * h / c
    nt = int(0.30 / dt)
    vel = np.full((n, n), c, dtype=np.float32)
    st = W.Setup(vel, h, dt, 0, c, 2, "cross", M)
    src = np.array([[n // 2, n // 2]])
    rec = np.array([[n // 2, n // 2 + 40]])
    wav = P.ricker(f0, nt, dt)
    tr, _, _ = W.forward(st, nt, src, wav, rec, threads=8)
    r = 40 * h
    s = lambda t: (1 - 2 * (math.pi * f0 * (t - 1 / f0)) ** 2) * math.exp(-(math.pi * f0 * (t - 1 / f0)) ** 2)
    ref = np.zeros(nt)
    for i in range(nt):
        t = (i + 1) * dt
        if c * t > r:
            ref[i] = quad(lambda xi: s(t - r / c * math.cosh(xi)), 0, math.acosh(c * t / r),
                          limit=200)[0] / (2 * math.pi * c * c)
    err = np.linalg.norm(tr[:, 0] - ref) / np.linalg.norm(ref)
    assert err < 2e-2, err


def test_green_function_3d():
    """3D: u(r,t) = s(t - r/c) / (4 pi c^2 r)."""
    n, h, c, f0, M = 81, 10.0, 1500.0, 8.0, 4
    pw = S.expand(3, "cross", M, 0, S.weights(3, "cross", M))
    dt = 0.5 * S.cfl_limit(pw, 3) * h / c
    nt = int(0.42 / dt)
    vel = np.full((n, n, n), c, dtype=np.float32)
    st = W.Setup(vel, h, dt, 0, c, 3, "cross", M)
    ctr = n // 2
    src = np.array([[ctr, ctr, ctr]])
    rec = np.array([[ctr, ctr, ctr + 16]])
    wav = P.ricker(f0, nt, dt)
    tr, _, _ = W.forward(st, nt, src, wav, rec, threads=8)
    r = 16 * h
    t = (np.arange(nt) + 1) * dt
    ref = (
        (1 - 2 * (math.pi * f0 * (t - r / c - 1 / f0)) ** 2)
        * np.exp(-(math.pi * f0 * (t - r / c - 1 / f0)) ** 2)) / (4 * math.pi * c * c * r)
    err = np.linalg.norm(tr[:, 0] - ref) / np.linalg.norm(ref)
    assert err < 3e-2, err


@pytest.mark.parametrize("dim", [2, 3])
def test_cfl_limit_separates_stable_and_unstable(dim):
    n = 40 if dim == 2 else 16
    pw = S.expand(dim, "cross", 4, 0, S.weights(dim, "cross", 4))
    cmax = S.cfl_limit(pw, dim)
    rng = np.random.default_rng(0)
    u0 = rng.standard_normal((n,) * dim)
    out = {}
    for f in (0.99, 1.01):
        st = _setup(n, dim, f * cmax)
        _, un, _ = W.forward(st, 600, None, None, None, u0=u0, um1=u0, threads=4)
        out[f] = np.max(np.abs(un))
    assert out[0.99] < 20 * np.max(np.abs(u0))
    assert out[1.01] > 1e6 * np.max(np.abs(u0))


def _hetero_setup(n=36, nb=6, dim=2, seed=1, M=4, shape="cross", scheme="spatte"):
    from workloads import smooth_velocity
    vel = smooth_velocity((n,) * dim, seed, 1500.0, 3000.0, sigma=3.0)
    h = 10.0
    pw = S.expand(dim, "cross", M, 0, S.weights(dim, "cross", M))
    dt = 0.5 * S.cfl_limit(pw, dim) * h / 3000.0
    return W.Setup(vel, h, dt, nb, 3000.0, dim, shape, M, 0, scheme), vel, dt


@pytest.mark.parametrize("dim", [2, 3])
def test_adjoint_dot_product(dim):
    """<F a, d> = <a, F* d> for the linear map from injected source values to
    receiver traces (damping and heterogeneous kappa included)."""
    n = 30 if dim == 2 else 14
    st, vel, dt = _hetero_setup(n, 5, dim, shape="rhombus", scheme="displs", M=3)
    rng = np.random.default_rng(3)
    nt = 60
    src = rng.integers(0, n, size=(2, dim))
    rec = rng.integers(0, n, size=(7, dim))
    amp = rng.standard_normal((nt, 2))
    wav = amp / (st.dt ** 2 / st.h ** dim)              # forward injects wav*dt^2/h^dim = amp
    tr, _, _ = W.forward(st, nt, src, wav, rec, threads=4)
    d = rng.standard_normal(tr.shape)
    _, adj = W.gradient(st, nt, src, np.zeros((nt, 2)), rec, d, adj_pos=src, threads=4)
    lhs = np.sum(tr * d)
    rhs = np.sum(amp * adj)
    assert abs(lhs - rhs) <= 1e-12 * max(abs(lhs), 1e-300) * 10, (lhs, rhs)


@pytest.mark.parametrize("dim", [2, 3])
def test_gradient_matches_finite_differences(dim):
    """dJ/dm for J = 1/2 ||traces(m) - d_obs||^2, m = 1/v^2 on the physical
    grid, against central differences of J along a smooth direction."""
    from workloads import smooth_velocity
    n = 28 if dim == 2 else 12
    nb, nt, h, vmax = 5, 120 if dim == 2 else 70, 10.0, 3200.0
    v = smooth_velocity((n,) * dim, 4, 1500.0, 3000.0, sigma=3.0).astype(np.float64)
    vtrue = smooth_velocity((n,) * dim, 5, 1500.0, 3000.0, sigma=2.0).astype(np.float64)
    m0 = 1.0 / v ** 2
    pw = S.expand(dim, "cross", 4, 0, S.weights(dim, "cross", 4))
    dt = 0.5 * S.cfl_limit(pw, dim) * h / vmax
    c = n // 2
    src = np.array([[2] + [c] * (dim - 1)])
    rec = np.array([[2] + list(p) for p in np.ndindex(*([n] * (dim - 1)))][:: 2])
    wav = P.ricker(25.0, nt, dt)

    def run(m):
        st = W.Setup(1.0 / np.sqrt(m), h, dt, nb, vmax, dim, "cross", 4)
        return st, W.forward(st, nt, src, wav, rec, threads=4)[0]

    _, dobs = run(1.0 / vtrue ** 2)
    st, d0 = run(m0)
    g, _ = W.gradient(st, nt, src, wav, rec, d0 - dobs, threads=4)
    dm = smooth_velocity((n,) * dim, 6, -1.0, 1.0, sigma=2.0).astype(np.float64) * 0.02 * m0
    eps = 1e-3
    J = lambda m: 0.5 * np.sum((run(m)[1] - dobs) ** 2)
    fd = (J(m0 + eps * dm) - J(m0 - eps * dm)) / (2 * eps)
    an = np.sum(g * dm)
    assert abs(fd - an) <= 1e-6 * abs(fd), (fd, an)


def test_checkpointing_does_not_change_gradient():
    st, vel, dt = _hetero_setup(24, 4)
    nt = 50
    src = np.array([[3, 12]])
    rec = np.array([[3, x] for x in range(24)])
    wav = P.ricker(20.0, nt, dt)
    r = np.random.default_rng(9).standard_normal((nt, 24))
    g1, a1 = W.gradient(st, nt, src, wav, rec, r, adj_pos=src, seg=nt, threads=2)
    for seg in (1, 7, 20):
        g2, a2 = W.gradient(st, nt, src, wav, rec, r, adj_pos=src, seg=seg, threads=2)
        assert np.array_equal(g1, g2) and np.array_equal(a1, a2)


def test_restart_from_state_is_identical():
    st, vel, dt = _hetero_setup(30, 5)
    nt1, nt2 = 17, 23
    src = np.array([[4, 15]])
    rec = np.array([[2, x] for x in range(30)])
    wav = P.ricker(20.0, nt1 + nt2, dt)
    tr, un, unm1 = W.forward(st, nt1 + nt2, src, wav, rec, threads=2)
    tra, ua, uam1 = W.forward(st, nt1, src, wav[:nt1], rec, threads=2)
    trb, ub, ubm1 = W.forward(st, nt2, src, wav[nt1:], rec, u0=ua, um1=uam1, threads=2)
    assert np.array_equal(tr, np.concatenate([tra, trb]))
    assert np.array_equal(un, ub) and np.array_equal(unm1, ubm1)


def test_ricker_closed_form_properties():
    f0 = 15.0
    at = lambda t: P.ricker(f0, 2, t)[1]                   # s(t) = sample n = 1 with dt = t
    assert abs(at(1 / f0) - 1.0) < 1e-15                   # peak 1 at t0 = 1/f0
    tz = 1 / f0 + 1 / (math.pi * f0 * math.sqrt(2))        # zeros at t0 +- 1/(pi f0 sqrt 2)
    assert abs(at(tz)) < 1e-15
    assert abs(at(1 / f0 - (tz - 1 / f0))) < 1e-15
    tm = 1 / f0 + math.sqrt(1.5) / (math.pi * f0)          # minima -2 exp(-3/2)
    assert abs(at(tm) + 2 * math.exp(-1.5)) < 1e-14
    assert abs(P.ricker(f0, 1, 1.0)[0] - (1 - 2 * math.pi ** 2) * math.exp(-math.pi ** 2)) < 1e-15
    dt = 1e-4
    s = P.ricker(f0, 4000, dt)
    assert abs(np.sum(s) * dt) < 1e-5                       # zero mean (tail before t = 0 is tiny)


def test_damping_profile():
    g = P.gamma_field((10, 12), 5, 1e-3, 10.0, 3000.0)
    assert g.shape == (20, 22)
    assert np.all(g[5:15, 5:17] == 0)
    em = P.eta_max(3000.0, 5, 10.0)
    assert abs(em - 3 * 3000.0 * math.log(1e3) / (2 * 5 * 10.0)) < 1e-12
    assert abs(g[0, 10] - 0.5e-3 * em) < 1e-15           # outermost row, one axis
    assert abs(g[0, 0] - 2 * 0.5e-3 * em) < 1e-15         # corner: both axes
    assert abs(g[3, 10] / g[1, 10] - (2 / 4) ** 2) < 1e-12  # quadratic in distance


def test_pad_fold_adjoint():
    rng = np.random.default_rng(2)
    for shape in ((7, 9), (5, 6, 4)):
        x = rng.standard_normal(shape)
        y = rng.standard_normal(tuple(s + 6 for s in shape))
        assert abs(np.sum(P.pad(x, 3) * y) - np.sum(x * P.fold(y, 3))) < 1e-10


def test_symbol_positive_stencil_grows_at_the_predicted_rate():
    """DispTE-CrossSq(2, 1) (weights at C = 0.3) run at a tenth of the Taylor
    Cross(2) limit: its symbol peaks at S* > 0, so the largest root of
    lambda^2 - (2 + C^2 S*) lambda + 1 = 0 exceeds 1 and a random field grows
    by that factor per step (slightly less on a finite grid, whose modes only
    approach the worst wave number)."""
    w = S.weights(2, "cross_square", 2, 1, "dispte", C=0.3)
    _, smax = S.symbol_range(S.expand(2, "cross_square", 2, 1, w), 2)
    C = 0.1 * S.cfl_limit(S.expand(2, "cross", 2, 0, S.weights(2, "cross", 2)), 2)
    n, v, h = 64, 1500.0, 10.0
    st = W.Setup(np.full((n, n), v, dtype=np.float32), h, C * h / v, 0, v, 2,
                 "cross_square", 2, 1, "dispte", weights=w)
    u0 = np.random.default_rng(0).standard_normal((n, n))
    amp = {}
    for ns in (100, 150):
        _, un, _ = W.forward(st, ns, None, None, None, u0=u0, um1=u0, threads=4)
        amp[ns] = np.max(np.abs(un))
    assert amp[100] > 1e6 * np.max(np.abs(u0))
    x = 2.0 + C * C * smax
    rate = math.log((x + math.sqrt(x * x - 4.0)) / 2.0)
    measured = math.log(amp[150] / amp[100]) / 50
    assert 0.9 * rate < measured <= 1.001 * rate, (measured, rate)
