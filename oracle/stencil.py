"""Stencil geometry, weight schemes and stability bound (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

Notation follows the paper: the 2D Laplacian is approximated as
(1/h^2) * sum over offsets o of a_o * u(x + o h) (Eq. spacexz_derivative2_sym),
with a_o equal on every offset of one symmetry orbit {(+-p,+-q), (+-q,+-p)}.
Unknowns are one weight per orbit ("orbit form"), which is the unambiguous
reading of the symmetric c_{p,q} = a_{p,q} + a_{q,p} passage of Section 4.1.
3D stencils are the union of the 2D shape in the three coordinate planes.
"""
from __future__ import annotations

import itertools
import math
from fractions import Fraction
from typing import Dict, List, Sequence, Tuple

import numpy as np

LS_RCOND = 1e-10

SHAPES = ("cross", "cross_rhombus", "rhombus", "cross_square", "square")
SCHEMES = ("spatte", "specte_theta", "specls", "dispte", "dispte_theta", "displs")


# ---------------------------------------------------------------------------
# Geometry (Section 4.1 "Basic shapes", Eq. spacexz_derivative2_sym)
# ---------------------------------------------------------------------------

def _offaxis_ranges(shape: str, M: int, N: int):
    """(Q, P0(q), P(q)) of the paper's shape definitions (Section 4.1):
    cross: Q = 0; rhombus: Q = floor(M/2), P0 = q, P = M - q;
    cross-rhombus: Q = floor(N/2), P0 = q, P = N - q;
    square: Q = M, P0 = q, P = M; cross-square: Q = N, P0 = q, P = M."""
    if shape == "cross":
        return 0, None, None
    if shape == "rhombus":
        return M // 2, (lambda q: q), (lambda q: M - q)
    if shape == "cross_rhombus":
        return N // 2, (lambda q: q), (lambda q: N - q)
    if shape == "square":
        return M, (lambda q: q), (lambda q: M)
    if shape == "cross_square":
        return N, (lambda q: q), (lambda q: M)
    raise ValueError("unknown shape %r" % shape)


def point_set_2d(shape: str, M: int, N: int = 0) -> List[Tuple[int, int]]:
    """All offsets (p, q) (p along x, q along z) of a 2D stencil."""
    pts = {(0, 0)}
    for m in range(1, M + 1):
        pts |= {(m, 0), (-m, 0), (0, m), (0, -m)}
    Q, P0, P = _offaxis_ranges(shape, M, N)
    for q in range(1, Q + 1):
        for p in range(P0(q), P(q) + 1):
            for sp, sq in itertools.product((1, -1), (1, -1)):
                pts.add((sp * p, sq * q))
                pts.add((sq * q, sp * p))   # symmetric counterpart a_{q,p}
    return sorted(pts)


def point_set(dim: int, shape: str, M: int, N: int = 0) -> List[Tuple[int, ...]]:
    """Offsets of a ``dim``-D stencil; 3D is the union of the 2D shape in the
    xy, xz and yz planes (offsets ordered (dz, dy, dx) for 3D and (dz, dx)
    for 2D, matching the [z][y][x] array layout)."""
    p2 = point_set_2d(shape, M, N)
    if dim == 2:
        return sorted((q, p) for (p, q) in p2)
    if dim != 3:
        raise ValueError("dim must be 2 or 3")
    pts = set()
    for (a, b) in p2:
        pts.add((0, a, b))   # xy plane (dz = 0)
        pts.add((a, 0, b))   # xz plane
        pts.add((a, b, 0))   # yz plane
    return sorted(pts)


def orbit_key(o: Sequence[int]) -> Tuple[int, ...]:
    return tuple(sorted((abs(v) for v in o), reverse=True))


def orbits(points: Sequence[Tuple[int, ...]]) -> Dict[Tuple[int, ...], List[Tuple[int, ...]]]:
    """Group offsets into symmetry orbits keyed by sorted absolute values."""
    out: Dict[Tuple[int, ...], List[Tuple[int, ...]]] = {}
    for o in points:
        out.setdefault(orbit_key(o), []).append(tuple(o))
    return dict(sorted(out.items()))


# ---------------------------------------------------------------------------
# Classical Taylor weights (Section 3.3.1, Eq. taylor_system), exact
# ---------------------------------------------------------------------------

def _solve_exact(A: List[List[Fraction]], b: List[Fraction]) -> List[Fraction]:
    n = len(A)
    M = [row[:] + [bb] for row, bb in zip(A, b)]
    for c in range(n):
        piv = next(r for r in range(c, n) if M[r][c] != 0)
        M[c], M[piv] = M[piv], M[c]
        for r in range(n):
            if r != c and M[r][c] != 0:
                f = M[r][c] / M[c][c]
                M[r] = [x - f * y for x, y in zip(M[r], M[c])]
    return [M[i][n] / M[i][i] for i in range(n)]


def _rank_rows(A: List[List[Fraction]]) -> List[int]:
    """Indices of a maximal set of linearly independent rows (exact)."""
    keep, basis = [], []
    for i, row in enumerate(A):
        v = row[:]
        for piv, brow in basis:
            if v[piv] != 0:
                f = v[piv] / brow[piv]
                v = [x - f * y for x, y in zip(v, brow)]
        piv = next((j for j, x in enumerate(v) if x != 0), None)
        if piv is not None:
            basis.append((piv, v))
            keep.append(i)
    return keep


def lstsq_rational(A, b) -> List[float]:
    """Minimum-norm least-squares solution computed exactly in rationals
    (float inputs are converted exactly).  Full column rank: normal equations
    (A^T A) x = A^T b; otherwise x = A_r^T (A_r A_r^T)^{-1} b_r on a maximal
    independent row subset (the consistent under-determined case)."""
    A = [[Fraction(x) for x in row] for row in A]
    b = [Fraction(x) for x in b]
    n = len(A[0])
    rows = _rank_rows(A)
    if len(rows) == n:
        At = list(zip(*A))
        AtA = [[sum(x * y for x, y in zip(ci, cj)) for cj in At] for ci in At]
        Atb = [sum(x * y for x, y in zip(ci, b)) for ci in At]
        return [float(v) for v in _solve_exact(AtA, Atb)]
    Ar = [A[i] for i in rows]
    br = [b[i] for i in rows]
    G = [[sum(x * y for x, y in zip(ri, rj)) for rj in Ar] for ri in Ar]
    y = _solve_exact(G, br)
    return [float(sum(Ar[k][j] * y[k] for k in range(len(Ar)))) for j in range(n)]


def taylor_cross_exact(M: int, dim: int = 2) -> List[Fraction]:
    """Exact solution of the Taylor system (Eq. taylor_system): unknowns
    a_{0,0}, a_{1,0}..a_{M,0}; a_{0,0} + 2*dim*sum a_m = 0 (r = 0; 4 in 2D),
    sum m^2 a_m = 1 (r = 1), sum m^(2r) a_m = 0 (1 < r <= M)."""
    n = M + 1
    A = [[Fraction(0)] * n for _ in range(n)]
    b = [Fraction(0)] * n
    A[0][0] = Fraction(1)
    for m in range(1, M + 1):
        A[0][m] = Fraction(2 * dim)
    for r in range(1, M + 1):
        for m in range(1, M + 1):
            A[r][m] = Fraction(m) ** (2 * r)
    b[1] = Fraction(1)
    return _solve_exact(A, b)


# ---------------------------------------------------------------------------
# Moment systems: SpatTE / DispTE (Eqs. taylor_system_r0 .. r_s and
# taylor_system_r0_disp .. r_s_disp) and their theta variants
# (Eqs. taylor_system_r*_spec, taylor_system_r*_disp_theta)
# ---------------------------------------------------------------------------

def _exponent_tuples(r: int, dim: int):
    """Sorted exponent tuples e_1 >= ... >= e_dim >= 0 with sum r."""
    out = []
    for e in itertools.product(range(r + 1), repeat=dim):
        if sum(e) == r and list(e) == sorted(e, reverse=True):
            out.append(e)
    return out


def moment_target(e: Sequence[int], C: float) -> float:
    """Right-hand side of the moment equation for exponents e (sum r):
    matching the coefficient of prod (k_i h)^(2 e_i) of the stencil symbol
    against (2/C^2)(cos(C beta) - 1) expanded with the multinomial theorem
    (Eq. full_disp_spec_taylor_cos_omega).  r = 0 gives 0; C = 0 gives the
    spatial Taylor system (only r = 1 non-zero)."""
    r = sum(e)
    if r == 0:
        return Fraction(0)
    multinom = Fraction(math.factorial(r), math.prod(math.factorial(x) for x in e))
    multinom2 = Fraction(math.factorial(2 * r), math.prod(math.factorial(2 * x) for x in e))
    cpow = Fraction(1) if r == 1 else Fraction(C) ** (2 * r - 2)
    return 2 * cpow * multinom / multinom2


def mixed_order(shape: str, M: int, N: int) -> int:
    """Highest order r of the mixed-derivative equations kept in the DispTE
    system.  The paper states that DispTE-CrossRb(M,N) has as many equations
    as weights (Section 4.2); that holds when the mixed equations stop at
    r = N (they number floor(N/2)ceil(N/2), the off-axis orbit count).  The
    cross keeps none (CrossRb(M,1) = Cross(M)); rhombus, square and cross-square
    keep all r <= M (the square and wide cross-square systems are then
    under-determined, the case the paper calls ill-posed)."""
    if shape == "cross":
        return 1
    if shape == "cross_rhombus":
        return max(1, N)
    return M


def moment_system(dim: int, orbs, M: int, C: float, rmix: int = None):
    """Orbit-form moment equations for r = 0..M: sum_orb a_orb * sum_{o in
    orb} prod_i o_i^(2 e_i) = target(e); mixed equations (two or more
    non-zero exponents) only up to order ``rmix``.  Returns (A, b, keys)."""
    keys = list(orbs.keys())
    rows, rhs = [], []
    if rmix is None:
        rmix = M
    for r in range(0, M + 1):
        for e in _exponent_tuples(r, dim):
            if sum(1 for x in e if x) >= 2 and r > rmix:
                continue
            row = []
            for k in keys:
                s = 0
                for o in orbs[k]:
                    t = 1
                    for oi, ei in zip(o, e):
                        t *= oi ** (2 * ei)
                    s += t
                row.append(s)
            rows.append(row)
            rhs.append(moment_target(e, C))
    return rows, rhs, keys


def theta_system(orbs, M: int, C: float, theta: float):
    """SpecTE-theta (C = 0) / DispTE-theta moment equations at one wave-number
    angle theta (2D): r = 0: sum mult * a = 0; r >= 1:
    sum_orb a_orb sum_{o in orb} (o . khat)^(2r) = 2 C^(2r-2),
    khat = (cos theta, sin theta) (Eqs. taylor_system_r1_spec/_r_s0_spec and
    taylor_system_r1_disp_theta/_r_s0_disp_theta, multiplied by 2)."""
    keys = list(orbs.keys())
    kh = np.array([np.sin(theta), np.cos(theta)])   # offsets are (dz, dx)
    rows, rhs = [], []
    rows.append([float(len(orbs[k])) for k in keys])
    rhs.append(0.0)
    for r in range(1, M + 1):
        rows.append([sum(float(np.dot(o, kh)) ** (2 * r) for o in orbs[k]) for k in keys])
        rhs.append(2.0 * (1.0 if r == 1 else C ** (2 * r - 2)))
    return np.array(rows), np.array(rhs), keys


# ---------------------------------------------------------------------------
# Least-squares schemes (Section 3.3.3 SpecLS, Section 3.4.3 DispLS)
# ---------------------------------------------------------------------------

def _directions(dim: int, n_ang: int):
    """Quadrature over wave-number directions: theta in [0, 2 pi) with the
    trapezoid rule (2D); the unit sphere with Gauss-Legendre in cos(polar)
    (at most 48 nodes) and the trapezoid rule in azimuth (twice as many
    nodes) (3D).  Returns (khat [n, dim], weights)."""
    if dim == 2:
        th = 2 * np.pi * np.arange(n_ang) / n_ang
        w = np.full(n_ang, 2 * np.pi / n_ang)
        return np.stack([np.sin(th), np.cos(th)], axis=1), w   # (dz, dx)
    n_ang = min(n_ang, 48)
    mu, wmu = np.polynomial.legendre.leggauss(n_ang)
    ph = 2 * np.pi * np.arange(2 * n_ang) / (2 * n_ang)
    st = np.sqrt(1 - mu ** 2)
    kz = np.repeat(mu, len(ph))
    ky = np.outer(st, np.sin(ph)).ravel()
    kx = np.outer(st, np.cos(ph)).ravel()
    w = np.outer(wmu, np.full(len(ph), 2 * np.pi / len(ph))).ravel()
    return np.stack([kz, ky, kx], axis=1), w


def _taylor_cos(x: np.ndarray, M: int) -> np.ndarray:
    """Truncated series sum_{r=0}^{M} (-1)^r x^(2r)/(2r)! of cos(x)."""
    return sum(((-1) ** r) * x ** (2 * r) / math.factorial(2 * r) for r in range(M + 1))


def ls_weights(dim: int, orbs, M: int, scheme: str, C: float, b: float,
               basis: str = "paper", n_beta: int = 64, n_ang: int = 256):
    """Least-squares weights.  Unknowns: one weight per non-centre orbit; the
    centre weight follows from the r = 0 condition (Eq. taylor_system_r0_spec).

    basis "taylor" (Eqs. taylor_laplacian_spec_disp_phim/_phipq1):
        phi_orb(beta, khat) = sum_{o in orb} [1 - T_M(beta khat.o)],
        T_M the cosine series truncated at r = M; target phi_1 = beta^2
        (SpecLS, Eq. taylor_laplacian_spec_disp_linsys) or
        phi_2 = (2 - 2 cos C beta)/C^2 (DispLS, Eq. ..._linsys1).
    basis "cosine" (Eqs. phim_continuous, phipq_continuous):
        Phi_orb = sum_{o in orb} [1 - cos(beta khat.o)] / Psi(beta),
        Psi_1 = beta^2 (SpecLS, Eq. specls_cont_linsys) or
        Psi_2 = (2 - 2 cos C beta)/C^2 (DispLS, Eq. displs_cont_linsys, with the
        factor 2 of phi_2 restored in the garbled Eq. psibeta2); target 1.
    basis "paper" picks the variant the paper adopts: Taylor basis for SpecLS
    (end of Section 3.3.3) and cosine basis for DispLS (end of 3.4.3).

    Inner product (Eq. cont_dotprod): integral over beta in [0, b] (Gauss-
    Legendre) and over all directions (2D: theta in [0, 2 pi]; 3D: the unit
    sphere).  Solved as the minimum-norm least-squares problem (Section 4.2,
    third bullet) with singular values below LS_RCOND * sigma_max dropped: the
    design matrices are ill-conditioned (up to ~1e13 for Square(8)) with no
    spectral gap, and a fixed relative cutoff makes the solution well defined
    to ~1e-6 independent of the solver."""
    if basis == "paper":
        basis = "taylor" if scheme == "specls" else "cosine"
    keys = [k for k in orbs.keys() if any(k)]
    xb, wb = np.polynomial.legendre.leggauss(n_beta)
    beta = 0.5 * b * (xb + 1.0)
    wbeta = 0.5 * b * wb
    khat, wang = _directions(dim, n_ang)
    nb_, na_ = len(beta), len(wang)
    Bm = np.repeat(beta, na_)
    W = np.outer(wbeta, wang).ravel()
    cols = []
    for k in keys:
        acc = np.zeros(nb_ * na_)
        for o in orbs[k]:
            proj = np.repeat(beta, na_) * np.tile(khat @ np.array(o, dtype=np.float64), nb_)
            acc += 1.0 - (_taylor_cos(proj, M) if basis == "taylor" else np.cos(proj))
        cols.append(acc)
    Phi = np.stack(cols, axis=1)
    if scheme == "specls":
        target = Bm ** 2
    elif scheme == "displs":
        target = (2.0 - 2.0 * np.cos(C * Bm)) / C ** 2 if C > 0 else Bm ** 2
    else:
        raise ValueError(scheme)
    if basis == "cosine":
        Phi = Phi / target[:, None]
        target = np.ones_like(target)
    sw = np.sqrt(W)
    a, *_ = np.linalg.lstsq(Phi * sw[:, None], target * sw, rcond=LS_RCOND)
    w = {k: float(v) for k, v in zip(keys, a)}
    center = tuple([0] * dim)
    w[center] = -sum(len(orbs[k]) * w[k] for k in keys)
    return w


def weights(dim: int, shape: str, M: int, N: int = 0, scheme: str = "spatte",
            C: float = 0.0, theta: float = np.pi / 8, b: float = np.pi / 2,
            basis: str = "paper") -> Dict[Tuple[int, ...], float]:
    """Orbit weights {orbit key: a} for any shape and scheme (Section 4.2).

    SpatTE and SpecTE-theta solve only the main (axis) equations with every
    off-axis weight set to zero, as Section 3.3.1 and the first two bullets of
    Section 4.2 prescribe; the shape then only adds zero weights."""
    orbs = orbits(point_set(dim, shape, M, N))
    if scheme in ("spatte", "specte_theta"):
        axis = {k: v for k, v in orbs.items() if sum(1 for x in k if x) <= 1}
        if scheme == "spatte":
            ex = taylor_cross_exact(M, dim)
            w = {k: 0.0 for k in orbs}
            for k in axis:
                w[k] = float(ex[k[0]])
            return w
        if dim != 2:
            raise ValueError("theta schemes are defined for 2D only")
        A, rhs, keys = theta_system(axis, M, 0.0, theta)
        a = lstsq_rational(A, rhs)
        w = {k: 0.0 for k in orbs}
        w.update({k: float(v) for k, v in zip(keys, a)})
        return w
    if scheme == "dispte":
        A, rhs, keys = moment_system(dim, orbs, M, C, mixed_order(shape, M, N))
    elif scheme == "dispte_theta":
        if dim != 2:
            raise ValueError("theta schemes are defined for 2D only")
        A, rhs, keys = theta_system(orbs, M, C, theta)
    elif scheme in ("specls", "displs"):
        return ls_weights(dim, orbs, M, scheme, C, b, basis)
    else:
        raise ValueError(scheme)
    a = lstsq_rational(A, rhs)
    return {k: float(v) for k, v in zip(keys, a)}


def expand(dim: int, shape: str, M: int, N: int, w: Dict[Tuple[int, ...], float]):
    """Per-offset list [(offset tuple, weight)] from orbit weights."""
    orbs = orbits(point_set(dim, shape, M, N))
    return [(o, w[k]) for k, os_ in orbs.items() for o in os_]


# ---------------------------------------------------------------------------
# Dispersion symbol and stability (Eqs. full_disp, full_disp_omegaFD, courant)
# ---------------------------------------------------------------------------

def symbol(pts_w, k: np.ndarray) -> np.ndarray:
    """S(k) = sum_o a_o cos(k . o) for wave-number vectors k (rows, ordered
    like the offsets, units of 1/h).  The scheme's dispersion relation is
    cos(omega tau) = 1 + (C^2 / 2) S(k h)."""
    offs = np.array([o for o, _ in pts_w], dtype=np.float64)
    ws = np.array([w for _, w in pts_w], dtype=np.float64)
    return np.cos(np.atleast_2d(k) @ offs.T) @ ws


def omega_fd(pts_w, k: np.ndarray, C: float, tau: float) -> np.ndarray:
    """Numerical angular frequency (Eq. full_disp_omegaFD)."""
    return np.arccos(1.0 + 0.5 * C * C * symbol(pts_w, k)) / tau


SYMBOL_POSITIVE_TOL = 1e-9


def _extreme_symbol(pts_w, dim: int, sign: float, n_grid: int):
    """max_k sign * S(k) over k in [0, pi]^dim: brute force on a regular grid
    (which contains every corner), refined by a bounded local search."""
    g = np.linspace(0.0, np.pi, n_grid)
    best, kbest = -np.inf, None
    slabs = [None] if dim == 2 else list(g)
    for a in slabs:
        if dim == 2:
            K = np.array(np.meshgrid(g, g, indexing="ij")).reshape(2, -1).T
        else:
            K = np.array(np.meshgrid([a], g, g, indexing="ij")).reshape(3, -1).T
        s = sign * symbol(pts_w, K)
        i = int(np.argmax(s))
        if s[i] > best:
            best, kbest = float(s[i]), K[i]
    try:
        from scipy.optimize import minimize
        res = minimize(lambda k: -sign * symbol(pts_w, np.clip(k, 0, np.pi))[0], kbest,
                       method="L-BFGS-B", bounds=[(0, np.pi)] * dim)
        if -float(res.fun) > best:
            best, kbest = -float(res.fun), np.clip(res.x, 0, np.pi)
    except Exception:  # pragma: no cover
        pass
    return best, kbest


def symbol_range(pts_w, dim: int, n_grid: int = 129):
    """(min_k S(k), max_k S(k)) over k in [0, pi]^dim (the symbol is even and
    2 pi-periodic in every component, so this is its range on all of R^dim)."""
    neg, _ = _extreme_symbol(pts_w, dim, -1.0, n_grid)
    pos, _ = _extreme_symbol(pts_w, dim, +1.0, n_grid)
    return -neg, pos


def cfl_limit(pts_w, dim: int, n_grid: int = 129) -> float:
    """Von Neumann bound of the leapfrog scheme (Eq. full_disp written as the
    amplification equation lambda^2 - (2 + C^2 S) lambda + 1 = 0): the product
    of the two roots is 1, so both stay on the unit circle iff their sum
    2 + C^2 S(k) lies in [-2, 2], i.e. iff -4 <= C^2 S(k) <= 0 for every k.

    - If S(k) > 0 anywhere, one root is real and larger than 1 for every
      C > 0: no time step is stable and a ValueError is raised.  S(0) = 0 for a
      consistent stencil, so "positive" means above SYMBOL_POSITIVE_TOL times
      max(-S), far above the round-off of S(0) and far below a real violation.
    - Otherwise C_max = 2 / sqrt(max_k -S(k))."""
    smin, smax = symbol_range(pts_w, dim, n_grid)
    if -smin <= 0:
        raise ValueError("stencil symbol is non-negative: no stable time step")
    if smax > SYMBOL_POSITIVE_TOL * (-smin):
        raise ValueError("stencil symbol reaches %.6g > 0: the leapfrog is unstable "
                         "at every time step" % smax)
    return 2.0 / math.sqrt(-smin)
