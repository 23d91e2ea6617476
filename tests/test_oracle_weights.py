"""Pins of the oracle's stencil geometry and weight schemes (CPU only).

Each test checks the oracle against something other than itself: textbook
weights (tests/golden), the closed form of the centred second derivative,
the paper's counting formulas, exact polynomial reproduction, the order of
the dispersion error the scheme is defined by, the paper's special-case
reductions, and an independent evaluation of the least-squares functional.
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

from oracle import stencil as S

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _read(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                rows.append(line.split())
    return rows


def test_taylor_matches_textbook_weights():
    for row in _read("taylor_second_derivative_weights.txt"):
        M = int(row[0])
        c = [Fraction(x) for x in row[1:]]
        a = S.taylor_cross_exact(M, dim=1)
        assert a[0] == c[0]
        assert a[1:] == c[1:]
        a2 = S.taylor_cross_exact(M, dim=2)
        assert a2[0] == 2 * c[0] and a2[1:] == c[1:]
        a3 = S.taylor_cross_exact(M, dim=3)
        assert a3[0] == 3 * c[0] and a3[1:] == c[1:]


@pytest.mark.parametrize("M", range(1, 11))
def test_taylor_closed_form(M):
    # a_m = 2 (-1)^(m+1) (M!)^2 / (m^2 (M-m)! (M+m)!)
    a = S.taylor_cross_exact(M, dim=2)
    for m in range(1, M + 1):
        ref = Fraction(2 * (-1) ** (m + 1) * math.factorial(M) ** 2,
                       m * m * math.factorial(M - m) * math.factorial(M + m))
        assert a[m] == ref
    assert a[0] == -4 * sum(a[1:])


def test_shape_weight_counts_match_paper_formulas():
    for sh, M, N, cnt in _read("shape_weight_counts.txt"):
        pts = S.point_set(2, sh, int(M), int(N))
        assert len(S.orbits(pts)) == int(cnt), (sh, M, N)


def test_shape_point_sets():
    # rhombus = {|p|+|q| <= M}, square = {max <= M}, cross-square = thick cross
    for M in range(1, 7):
        rh = set(S.point_set(2, "rhombus", M))
        assert rh == {(a, b) for a in range(-M, M + 1) for b in range(-M, M + 1) if abs(a) + abs(b) <= M}
        sq = set(S.point_set(2, "square", M))
        assert len(sq) == (2 * M + 1) ** 2
        for N in range(0, M + 1):
            cs = set(S.point_set(2, "cross_square", M, N))
            assert cs == {(a, b) for a in range(-M, M + 1) for b in range(-M, M + 1)
                          if min(abs(a), abs(b)) <= N}
    # paper: CrossRb(M,1) = CrossSq(M,0) = Cross(M); CrossRb(M,M) = Rhombus(M); CrossSq(M,M) = Square(M)
    for M in range(1, 7):
        cr = set(S.point_set(2, "cross", M))
        assert set(S.point_set(2, "cross_rhombus", M, 1)) == cr
        assert set(S.point_set(2, "cross_square", M, 0)) == cr
        assert set(S.point_set(2, "cross_rhombus", M, M)) == set(S.point_set(2, "rhombus", M))
        assert set(S.point_set(2, "cross_square", M, M)) == set(S.point_set(2, "square", M))
    # 3D planar-union rhombus of radius 4 has 97 points; cross has 6M+1
    assert len(S.point_set(3, "rhombus", 4)) == 97
    assert len(S.point_set(3, "cross", 8)) == 49


def _monomial_check(dim, pw, degree):
    """Apply the stencil to every monomial of total degree <= degree at the
    origin with exact rationals; compare with the exact Laplacian at 0."""
    import itertools
    for e in itertools.product(range(degree + 1), repeat=dim):
        if sum(e) > degree:
            continue
        val = Fraction(0)
        for o, w in pw:
            t = Fraction(w)
            for oi, ei in zip(o, e):
                t *= Fraction(oi) ** ei
            val += t
        # Laplacian of prod x_i^e_i at 0 is 2 if exactly one e_i == 2 and the rest 0
        exact = 2 if (sorted(e) == [0] * (dim - 1) + [2]) else 0
        assert val == exact, (e, val)


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("M", [1, 2, 4, 6])
def test_taylor_polynomial_exactness(dim, M):
    a = S.taylor_cross_exact(M, dim)
    pw = [(tuple([0] * dim), a[0])]
    for m in range(1, M + 1):
        for ax in range(dim):
            for sgn in (1, -1):
                o = [0] * dim
                o[ax] = sgn * m
                pw.append((tuple(o), a[m]))
    _monomial_check(dim, pw, 2 * M + 1)


def _dispersion_error(pw, C, k):
    """cos(omega tau) of the scheme minus the exact cos(C |k|) (Eq. full_disp)."""
    return 1.0 + 0.5 * C * C * S.symbol(pw, k) - np.cos(C * np.linalg.norm(k, axis=1))


@pytest.mark.parametrize("shape,M,N,thetas,order", [
    ("cross", 2, 0, (0.0,), 6), ("cross", 4, 0, (0.0,), 10),
    ("rhombus", 3, 0, (0.1, 0.5, 1.0), 8), ("rhombus", 4, 0, (0.1, 0.5, 1.0), 10),
    ("cross_rhombus", 4, 2, (0.0,), 10), ("cross_rhombus", 4, 2, (0.3, 0.8), 6)])
def test_dispte_dispersion_order(shape, M, N, thetas, order):
    """DispTE is defined by matching the time-space dispersion relation term
    by term (Section 3.4.2): with all mixed equations (rhombus) the error
    falls like beta^(2M+2) in every direction; along the axes it does so for
    every shape; with mixed equations up to order N off-axis directions keep
    order 2N+2."""
    C = 0.35
    w = S.weights(2, shape, M, N, "dispte", C=C)
    pw = S.expand(2, shape, M, N, w)
    for th in thetas:
        kh = np.array([[np.sin(th), np.cos(th)]])
        e1 = abs(_dispersion_error(pw, C, 0.4 * kh)[0])
        e2 = abs(_dispersion_error(pw, C, 0.2 * kh)[0])
        rate = math.log2(e1 / e2)
        assert rate > order - 1.0, (th, rate)


def test_spatte_spectral_order():
    """SpatTE: S(k) + |k|^2 = O(|k|^(2M+2)) in every direction."""
    for M, s0 in ((2, 0.4), (4, 0.4), (8, 1.0)):   # s0 keeps errors above fp64 round-off
        pw = S.expand(2, "cross", M, 0, S.weights(2, "cross", M))
        for th in (0.2, 0.7):
            kh = np.array([[np.sin(th), np.cos(th)]])
            e = [abs(S.symbol(pw, s * kh)[0] + s * s) for s in (s0, s0 / 2)]
            assert math.log2(e[0] / e[1]) > 2 * M + 2 - 1.0


def test_specte_theta_reductions():
    # theta = 0 recovers SpatTE (Section 4.2, second bullet)
    for M in (2, 4, 6):
        a = S.weights(2, "cross", M, 0, "specte_theta", theta=0.0)
        b = S.weights(2, "cross", M, 0, "spatte")
        for k in b:
            assert abs(a[k] - b[k]) < 1e-9 * max(1, abs(b[k]))
    # at theta = pi/8 the symbol is accurate to order 2M along that direction only
    M, th = 4, np.pi / 8
    pw = S.expand(2, "cross", M, 0, S.weights(2, "cross", M, 0, "specte_theta", theta=th))
    kh = np.array([[np.sin(th), np.cos(th)]])
    e = [abs(S.symbol(pw, s * kh)[0] + s * s) for s in (0.4, 0.2)]
    assert math.log2(e[0] / e[1]) > 2 * M + 2 - 1.0


def test_dispte_reduces_to_spatte_at_zero_courant():
    for M in (2, 4, 6):
        a = S.weights(2, "cross", M, 0, "dispte", C=0.0)
        b = S.weights(2, "cross", M, 0, "spatte")
        for k in b:
            assert abs(a[k] - b[k]) < 1e-8 * max(1, abs(b[k]))


@pytest.mark.parametrize("scheme", ["dispte", "displs", "specls"])
def test_cross_rhombus_n1_equals_cross(scheme):
    for M in (2, 4):
        a = S.weights(2, "cross_rhombus", M, 1, scheme, C=0.3)
        b = S.weights(2, "cross", M, 0, scheme, C=0.3)
        c = S.weights(2, "cross_square", M, 0, scheme, C=0.3)
        assert set(a) == set(b) == set(c)
        for k in b:
            assert abs(a[k] - b[k]) < 1e-9 * max(1, abs(b[k]))
            assert abs(c[k] - b[k]) < 1e-9 * max(1, abs(b[k]))


@pytest.mark.parametrize("dim,shape,M,scheme", [(2, "cross", 4, "displs"), (2, "rhombus", 4, "displs"),
                                                (2, "square", 2, "specls"), (3, "rhombus", 4, "displs"),
                                                (2, "cross", 8, "dispte")])
def test_weights_sum_to_zero(dim, shape, M, scheme):
    w = S.weights(dim, shape, M, 0, scheme, C=0.3)
    pw = S.expand(dim, shape, M, 0, w)
    assert abs(sum(x for _, x in pw)) < 1e-9


def _paper_displs_functional(a_axis, a_off, M, C, b, n_beta=40, n_theta=180):
    """E_disp(b) of Eq. LS_disp_error with the cosine basis of Eqs.
    phim_continuous2 / phipq_continuous2 written in the paper's notation:
    axis weights a_{m,0}, off-axis a_{p,q} for the listed (p, q) (each paired
    with its symmetric counterpart a_{q,p} = a_{p,q}).  Different quadrature
    (Gauss-Legendre with 40 nodes in beta, midpoint rule in theta)."""
    xb, wb = np.polynomial.legendre.leggauss(n_beta)
    beta = 0.5 * b * (xb + 1)
    wbeta = 0.5 * b * wb
    th = (np.arange(n_theta) + 0.5) * 2 * np.pi / n_theta
    B, T = np.meshgrid(beta, th, indexing="ij")
    psi2 = (2 - 2 * np.cos(C * B)) / C ** 2
    acc = np.zeros_like(B)
    for m, am in a_axis.items():
        acc += am * (4 - 2 * np.cos(m * B * np.cos(T)) - 2 * np.cos(m * B * np.sin(T))) / psi2
    for (p, q), apq in a_off.items():
        f = lambda pp, qq: (4 - 2 * np.cos(qq * B * np.cos(T) + pp * B * np.sin(T))
                            - 2 * np.cos(qq * B * np.cos(T) - pp * B * np.sin(T))) / psi2
        acc += apq * (f(p, q) + (f(q, p) if p != q else 0.0))
    return float(np.sum((acc - 1.0) ** 2 * wbeta[:, None]) * 2 * np.pi / n_theta)


@pytest.mark.parametrize("shape,M", [("cross", 4), ("cross", 8), ("rhombus", 4), ("square", 3)])
def test_displs_minimises_paper_functional(shape, M):
    """The DispLS weights minimise the paper's E_disp(b) (Eq. LS_disp_error):
    every coordinate perturbation increases the independently evaluated
    functional and its finite-difference gradient vanishes."""
    C, b = 0.3, np.pi / 2
    w = S.weights(2, shape, M, 0, "displs", C=C, b=b)
    axis = {k[0]: v for k, v in w.items() if k[0] > 0 and k[1] == 0}
    off = {k: v for k, v in w.items() if k[1] > 0}
    E0 = _paper_displs_functional(axis, off, M, C, b)
    scale = max(E0, 1e-12)
    eps = 1e-4
    for key in list(axis) + list(off):
        def E(d):
            ax = dict(axis)
            of = dict(off)
            if key in ax:
                ax[key] += d
            else:
                of[key] += d
            return _paper_displs_functional(ax, of, M, C, b)
        Ep, Em = E(eps), E(-eps)
        assert Ep > E0 and Em > E0
        grad = (Ep - Em) / (2 * eps)
        curv = (Ep + Em - 2 * E0) / eps ** 2
        # stationarity: the minimiser of the quadratic sits within |grad/curv| of a
        assert abs(grad / curv) < 1e-6 * max(1.0, abs(axis.get(key, off.get(key, 1.0)))), key


def test_ls_small_band_tends_to_taylor():
    """As the band b shrinks, the cosine-basis least squares on low wave
    numbers approaches the Taylor conditions (SpecLS -> SpatTE)."""
    t = S.weights(2, "cross", 3, 0, "spatte")
    errs = []
    for b in (0.4, 0.2, 0.1):
        w = S.weights(2, "cross", 3, 0, "specls", b=b, basis="cosine")
        errs.append(max(abs(w[k] - t[k]) for k in t))
    # the gap closes like b^2
    assert 3.0 < errs[0] / errs[1] < 5.5 and 3.0 < errs[1] / errs[2] < 5.5, errs
    assert errs[2] < 1e-3, errs


@pytest.mark.parametrize("dim,shape,M", [(2, "rhombus", 4), (2, "square", 3), (3, "rhombus", 2)])
def test_specls_taylor_basis_reproduces_spatte(dim, shape, M):
    """With the Taylor basis adopted for SpecLS (Eq. taylor_laplacian_spec_disp
    _linsys) the target beta^2 lies in the span of the basis (the r = 1
    term), so the least-squares residual is zero: the stencil has the full
    Taylor spectral order 2M in every direction, and where that solution is
    unique (rhombus) it is the SpatTE stencil with vanishing off-axis
    weights.  (For the square, with more orbits than equations, the
    minimum-norm exact solution is returned instead.)"""
    w = S.weights(dim, shape, M, 0, "specls")
    t = S.weights(dim, shape, M, 0, "spatte")
    pw = S.expand(dim, shape, M, 0, w)
    for th in (0.3, 0.9):
        kh = np.array([[np.sin(th), np.cos(th)] if dim == 2 else [np.sin(th), 0.6 * np.cos(th), 0.8 * np.cos(th)]])
        e = [abs(S.symbol(pw, s * kh)[0] + s * s) for s in (0.6, 0.3)]
        assert math.log2(e[0] / e[1]) > 2 * M + 2 - 1.0
    if shape == "rhombus":
        for k in t:
            assert abs(w[k] - t[k]) < 1e-10 * max(1.0, abs(t[k])), k


def test_cfl_closed_form_and_brute_force():
    # -S_max = 4 d sum_{m odd} a_m for the Taylor cross (attained at k = (pi,...,pi))
    for dim in (2, 3):
        for M in (1, 2, 4, 8):
            a = S.taylor_cross_exact(M, dim)
            smax = 4 * dim * float(sum(a[m] for m in range(1, M + 1, 2)))
            pw = S.expand(dim, "cross", M, 0, S.weights(dim, "cross", M))
            assert abs(S.cfl_limit(pw, dim) - 2 / math.sqrt(smax)) < 1e-9
    pw = S.expand(2, "cross", 1, 0, S.weights(2, "cross", 1))
    assert abs(S.cfl_limit(pw, 2) - 1 / math.sqrt(2)) < 1e-12
    pw = S.expand(3, "cross", 1, 0, S.weights(3, "cross", 1))
    assert abs(S.cfl_limit(pw, 3) - 1 / math.sqrt(3)) < 1e-12
    # Cross(4), 2D: 2 / sqrt(8 * 512/315)
    pw = S.expand(2, "cross", 4, 0, S.weights(2, "cross", 4))
    assert abs(S.cfl_limit(pw, 2) - 2 / math.sqrt(8 * 512 / 315)) < 1e-9
    # brute force over a fine grid of a LS stencil never exceeds the bound's symbol max
    w = S.weights(2, "square", 4, 0, "displs", C=0.3)
    pw = S.expand(2, "square", 4, 0, w)
    cm = S.cfl_limit(pw, 2)
    g = np.linspace(0, np.pi, 301)
    K = np.array(np.meshgrid(g, g, indexing="ij")).reshape(2, -1).T
    assert np.max(-S.symbol(pw, K)) <= 4 / cm ** 2 * (1 + 1e-9)


@pytest.mark.parametrize("scheme,C", [("displs", 0.3), ("displs", 0.6), ("specls", 0.0)])
def test_ls_single_unknown_has_the_closed_form_minimiser(scheme, C):
    """Cross(1) in 2D has one least-squares unknown a (the axis weight), so
    the minimiser of the functional over beta in [0, b], theta in [0, 2 pi]
    (Eqs. cont_dotprod, LS_disp_error, cosine basis) is a = <Phi, 1> / <Phi, Phi>
    with Phi = (4 - 2 cos(beta cos theta) - 2 cos(beta sin theta)) / Psi(beta),
    Psi = (2 - 2 cos C beta)/C^2 (DispLS) or beta^2 (SpecLS).  Evaluated here
    by adaptive quadrature in half-angle form, independent of the oracle's
    Gauss-Legendre and trapezoid rules."""
    integrate = pytest.importorskip("scipy.integrate")
    b = np.pi / 2

    def phi(th, beta):
        num = 4 * np.sin(0.5 * beta * np.cos(th)) ** 2 + 4 * np.sin(0.5 * beta * np.sin(th)) ** 2
        psi = (2 * np.sin(0.5 * C * beta) / C) ** 2 if C > 0 else beta ** 2
        return num / psi

    opts = dict(epsabs=1e-14, epsrel=1e-13)
    p1 = integrate.dblquad(lambda th, beta: phi(th, beta), 0, b, 0, 2 * np.pi, **opts)[0]
    p2 = integrate.dblquad(lambda th, beta: phi(th, beta) ** 2, 0, b, 0, 2 * np.pi, **opts)[0]
    a = p1 / p2
    w = S.weights(2, "cross", 1, 0, scheme, C=C, b=b, basis="cosine")
    assert abs(w[(1, 0)] - a) < 1e-10 * abs(a)
    assert abs(w[(0, 0)] + 4 * a) < 1e-10 * abs(a)


def test_ls_single_unknown_closed_form_in_3d():
    """The same for the 3D Cross(1) DispLS weight, with directions over the
    unit sphere (mu = cos of the polar angle, azimuth phi):
    Phi = (6 - 2 cos(beta kx) - 2 cos(beta ky) - 2 cos(beta kz)) / Psi(beta)."""
    integrate = pytest.importorskip("scipy.integrate")
    b, C = np.pi / 2, 0.4

    def phi(ph, mu, beta):
        st = np.sqrt(max(0.0, 1.0 - mu * mu))
        k = (st * np.cos(ph), st * np.sin(ph), mu)
        num = sum(4 * np.sin(0.5 * beta * kc) ** 2 for kc in k)
        return num / (2 * np.sin(0.5 * C * beta) / C) ** 2

    opts = dict(epsabs=1e-12, epsrel=1e-11)
    p1 = integrate.tplquad(lambda ph, mu, beta: phi(ph, mu, beta), 0, b, -1, 1, 0, 2 * np.pi, **opts)[0]
    p2 = integrate.tplquad(lambda ph, mu, beta: phi(ph, mu, beta) ** 2, 0, b, -1, 1, 0, 2 * np.pi,
                           **opts)[0]
    a = p1 / p2
    w = S.weights(3, "cross", 1, 0, "displs", C=C, b=b, basis="cosine")
    assert abs(w[(1, 0, 0)] - a) < 1e-8 * abs(a)
    assert abs(w[(0, 0, 0)] + 6 * a) < 1e-8 * abs(a)


@pytest.mark.parametrize("shape,orbits", [
    ("cross", {(1, 0): [(1, 0), (-1, 0), (0, 1), (0, -1)],
               (2, 0): [(2, 0), (-2, 0), (0, 2), (0, -2)]}),
    ("rhombus", {(1, 0): [(1, 0), (-1, 0), (0, 1), (0, -1)],
                 (2, 0): [(2, 0), (-2, 0), (0, 2), (0, -2)],
                 (1, 1): [(1, 1), (1, -1), (-1, 1), (-1, -1)]}),
])
def test_ls_normal_equations_by_adaptive_quadrature(shape, orbits):
    """DispLS for radius 2 (two and three unknowns): the weights solve the
    normal equations <Phi_i, Phi_j> a_j = <Phi_i, 1> of the paper's functional
    (cosine basis, Eq. displs_cont_linsys), with every inner product taken by
    adaptive quadrature from orbit point lists written out here."""
    integrate = pytest.importorskip("scipy.integrate")
    b, C = np.pi / 2, 0.3
    keys = list(orbits)

    def phi(key, th, beta):
        kz, kx = np.sin(th), np.cos(th)
        num = sum(4 * np.sin(0.5 * beta * (kz * o[0] + kx * o[1])) ** 2 / 2 for o in orbits[key])
        return num / (2 * np.sin(0.5 * C * beta) / C) ** 2

    def ip(f):
        return integrate.dblquad(lambda th, beta: f(th, beta), 0, b, 0, 2 * np.pi,
                                 epsabs=1e-13, epsrel=1e-12)[0]

    G = np.array([[ip(lambda th, be, i=i, j=j: phi(i, th, be) * phi(j, th, be)) for j in keys]
                  for i in keys])
    r = np.array([ip(lambda th, be, i=i: phi(i, th, be)) for i in keys])
    a = np.linalg.solve(G, r)
    w = S.weights(2, shape, 2, 0, "displs", C=C, b=b, basis="cosine")
    for k, v in zip(keys, a):
        assert abs(w[k] - v) < 1e-8 * np.abs(a).max(), (k, w[k], v)


def _brute_force_symbol_max(pts, wo, n=241):
    """max over a regular (kz, kx) grid of [0, pi]^2 of S(k) = sum_o w_o cos(k . o),
    summed here offset by offset."""
    g = np.linspace(0.0, np.pi, n)
    best = -np.inf
    for kz in g:
        s = np.zeros_like(g)
        for (dz, dx), wi in zip(pts, wo):
            s += wi * np.cos(kz * dz + g * dx)
        best = max(best, float(s.max()))
    return best


@pytest.mark.parametrize("M,N", [(2, 1), (4, 2), (6, 3)])
def test_symbol_positive_stencil_has_no_stable_time_step(M, N):
    """The leapfrog's amplification equation lambda^2 - (2 + C^2 S) lambda + 1 = 0
    (Eq. full_disp) has a root above 1 wherever S(k) > 0, at every C > 0.
    DispTE-CrossSq(M, N) at C = 0.3 has such wave numbers: the brute-force
    maximum of its symbol is far above 0, and the bound must say that no time
    step is stable instead of returning 2 / sqrt(max -S)."""
    w = S.weights(2, "cross_square", M, N, "dispte", C=0.3)
    pts = S.point_set(2, "cross_square", M, N)
    wo = [w[tuple(sorted((abs(v) for v in o), reverse=True))] for o in pts]
    smax = _brute_force_symbol_max(pts, wo)
    assert smax > 1.0
    pw = S.expand(2, "cross_square", M, N, w)
    lo, hi = S.symbol_range(pw, 2)
    assert smax - 1e-9 <= hi <= smax + 0.05 * smax
    assert lo < 0
    with pytest.raises(ValueError, match="unstable at every time step"):
        S.cfl_limit(pw, 2)


@pytest.mark.parametrize("dim,shape,M,N,scheme", [
    (2, "cross", 4, 0, "spatte"), (2, "rhombus", 4, 0, "displs"), (2, "square", 4, 0, "displs"),
    (2, "cross_square", 4, 2, "displs"), (3, "cross", 4, 0, "spatte"),
])
def test_stable_stencils_have_non_positive_symbol(dim, shape, M, N, scheme):
    """Stencils the workloads run keep S(k) <= 0 up to round-off (S(0) = 0),
    so the bound stays 2 / sqrt(max -S)."""
    pw = S.expand(dim, shape, M, N, S.weights(dim, shape, M, N, scheme, C=0.3))
    lo, hi = S.symbol_range(pw, dim, n_grid=65 if dim == 3 else 129)
    assert hi <= 1e-12 * abs(lo)
    assert abs(S.cfl_limit(pw, dim) - 2 / math.sqrt(-lo)) < 1e-12


def _orbit_offsets(key, dim):
    """Every offset of a symmetry orbit: all permutations and sign changes of
    its sorted absolute offsets (zero-padded to dim components)."""
    full = tuple(key) + (0,) * (dim - len(key))
    out = set()
    for perm in itertools.permutations(full):
        for sg in itertools.product((1, -1), repeat=dim):
            out.add(tuple(s * v for s, v in zip(sg, perm)))
    return sorted(out)


def _displs_design(dim, keys, C, b, n_beta=24, n_dir=16):
    """Design matrix of E_disp(b) (Eq. LS_disp_error, cosine basis of Eq.
    displs_cont_linsys: Phi_orb = sum_{o in orb} (1 - cos(beta khat.o)) / Psi2,
    Psi2 = (2 - 2 cos C beta) / C^2, target 1) on this test's own quadrature:
    Gauss-Legendre in beta; in 2D the midpoint rule on one eighth of the
    circle (the integrand has the square's eight-fold symmetry), in 3D
    Gauss-Legendre in the polar angle (weight sin) and the midpoint rule in
    azimuth.  Returns (A, quadrature weights)."""
    xb, wb = np.polynomial.legendre.leggauss(n_beta)
    beta, wbeta = 0.5 * b * (xb + 1), 0.5 * b * wb
    if dim == 2:
        th = (np.arange(n_dir) + 0.5) * (np.pi / 4) / n_dir
        dirs = np.stack([np.sin(th), np.cos(th)], 1)
        wd = np.full(n_dir, 8 * (np.pi / 4) / n_dir)
    else:
        xt, wt = np.polynomial.legendre.leggauss(n_dir)
        pol = 0.5 * np.pi * (xt + 1)
        wpol = 0.5 * np.pi * wt * np.sin(pol)
        az = (np.arange(2 * n_dir) + 0.5) * np.pi / n_dir
        dirs = np.stack([np.repeat(np.cos(pol), len(az)), np.outer(np.sin(pol), np.sin(az)).ravel(),
                         np.outer(np.sin(pol), np.cos(az)).ravel()], 1)
        wd = np.outer(wpol, np.full(len(az), np.pi / n_dir)).ravel()
    Bt = np.repeat(beta, len(wd))
    K = Bt[:, None] * np.tile(dirs, (n_beta, 1))
    psi2 = (2 - 2 * np.cos(C * Bt)) / C ** 2
    cols = [np.sum(1 - np.cos(K @ np.array(_orbit_offsets(k, dim), float).T), 1) / psi2 for k in keys]
    return np.stack(cols, 1), np.outer(wbeta, wd).ravel()


def _exact_minimum(A, W, dps=50):
    """min_x sum W (A x - 1)^2 by the normal equations in `dps`-digit arithmetic
    (exact for the float64 entries of A and W, whatever their conditioning).
    Returns (minimum, minimiser)."""
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = dps
    n = A.shape[1]
    G = mpmath.matrix(n, n)
    g = mpmath.matrix(n, 1)
    tot = mpmath.mpf(0)
    for r in range(A.shape[0]):
        row = [mpmath.mpf(float(x)) for x in A[r]]
        w = mpmath.mpf(float(W[r]))
        tot += w
        for i in range(n):
            wi = w * row[i]
            g[i] += wi
            for j in range(i, n):
                G[i, j] += wi * row[j]
    for i in range(n):
        for j in range(i):
            G[i, j] = G[j, i]
    x = mpmath.lu_solve(G, g)
    return float(tot - sum(g[i] * x[i] for i in range(n))), np.array([float(v) for v in x])


@pytest.mark.parametrize("dim,shape,M", [(2, "rhombus", 8), (2, "square", 4), (2, "square", 8),
                                         (3, "rhombus", 4), (2, "rhombus", 4), (2, "cross", 8)])
def test_displs_weights_of_the_workloads_reach_the_exact_minimum(dim, shape, M):
    """Every DispLS stencil the 1001^2 and 400^3 workloads run, at C = 0.3 and
    b = pi/2, against the exact minimum of the paper's functional E_disp(b)
    built and minimised here (see _displs_design, _exact_minimum).
    - Where the design matrix keeps every singular value above the cutoff
      (1e-10 sigma_max), the oracle's weights are the minimiser: E(w) is
      within 1e-6 of the minimum.
    - Square(8) has condition number ~7e14; the minimum-norm solution drops
      the directions below the cutoff.  E(w) then exceeds the minimum by less
      than 1e-12 of the functional's scale E(0) (an RMS relative dispersion
      error of about 1e-8 either way), with weights far smaller than the
      exact minimiser's, whose cancelling entries FP32 rounding would spoil.
    A dropped term, a wrong sign, a transposed offset or the missing factor 2
    of Psi2 changes E(w) by orders of magnitude more than these margins."""
    C, b = 0.3, np.pi / 2
    w = S.weights(dim, shape, M, 0, "displs", C=C, b=b)
    keys = [k for k in w if any(k)]
    A, W = _displs_design(dim, keys, C, b, n_dir=16 if dim == 2 else 20)
    x = np.array([w[k] for k in keys])
    E = float(np.sum(W * (A @ x - 1) ** 2))
    Emin, xmin = _exact_minimum(A, W)
    E0 = float(np.sum(W))
    assert Emin <= E * (1 + 1e-9)
    if (shape, M) == ("square", 8):
        assert E - Emin < 1e-12 * E0
        assert np.linalg.norm(x) < 0.1 * np.linalg.norm(xmin)
    else:
        assert E <= Emin * (1 + 1e-6), (E, Emin)
    # and a plausible mistake is far outside that margin: the factor 2 of Psi2
    # dropped (the garbled Eq. psibeta2) or the weights' sign flipped
    assert float(np.sum(W * (0.5 * (A @ x) - 1) ** 2)) > 1e3 * Emin
    assert float(np.sum(W * (-(A @ x) - 1) ** 2)) > 1e3 * Emin
