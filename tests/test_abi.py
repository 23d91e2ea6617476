"""C-ABI checks that need no GPU: the library loads, exports every symbol
declared in include/fdwave.h, and its host-side entry points (weights, CFL
bound, Ricker wavelet, plan validation, workspace sizing) agree with the FP64
oracle and reject bad arguments."""
import math
import os
import re

import numpy as np
import pytest

import paper_2606_04882_gb300 as F
from oracle import physics as P
from oracle import stencil as S

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_2606_04882_gb300 import build
    build.build()


def _declared_symbols():
    txt = open(os.path.join(ROOT, "include", "fdwave.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?(?:int|void|char|double|size_t)\s*\*?\s*(fd_\w+)\s*\(",
                       txt, flags=re.M)
    return sorted(set(names))


def test_every_declared_symbol_is_exported():
    names = _declared_symbols()
    assert len(names) >= 15, names
    L = F.lib()
    for n in names:
        assert hasattr(L, n), n
    # and the binding exposes the same names
    for n in names:
        assert n in F._SIGS, n


@pytest.mark.parametrize("dim,shape,M,N,scheme", [
    (2, "cross", 1, 0, "spatte"), (2, "cross", 4, 0, "spatte"), (2, "cross", 8, 0, "spatte"),
    (3, "cross", 4, 0, "spatte"), (3, "cross", 8, 0, "spatte"), (2, "cross", 16, 0, "spatte"),
    (2, "rhombus", 4, 0, "dispte"), (2, "cross_rhombus", 5, 3, "dispte"),
    (2, "square", 3, 0, "dispte"), (2, "cross_square", 4, 2, "dispte"),
    (2, "cross", 4, 0, "specte_theta"), (2, "rhombus", 4, 0, "dispte_theta"),
    (2, "cross", 4, 0, "displs"), (2, "rhombus", 4, 0, "displs"), (2, "square", 2, 0, "specls"),
    (3, "rhombus", 4, 0, "displs"), (2, "cross", 8, 0, "displs"),
])
def test_weights_and_cfl_match_oracle(dim, shape, M, N, scheme):
    C = 0.3
    d = F.stencil_desc(dim, shape, M, N, scheme, courant=C)
    keys, mult, w = F.fd_weights(d)
    ow = S.weights(dim, shape, M, N, scheme, C=C)
    orbs = S.orbits(S.point_set(dim, shape, M, N))
    assert len(keys) == len(ow)
    scale = max(abs(x) for x in w)
    # least-squares design matrices have condition numbers up to ~1e7 (cross 8)
    tol = (1e-9 if M <= 4 else 1e-6) if scheme in ("displs", "specls") else 1e-12
    for i, k in enumerate(keys):
        kk = tuple(int(x) for x in k[:dim])
        assert mult[i] == len(orbs[kk])
        assert abs(w[i] - ow[kk]) <= tol * scale, (kk, w[i], ow[kk])
    try:
        oc = S.cfl_limit(S.expand(dim, shape, M, N, ow), dim)
    except ValueError:
        # the symbol is positive somewhere: both sides must refuse every dt
        with pytest.raises(F.FdError) as e:
            F.fd_cfl_limit(d)
        assert e.value.code == F.FD_ERR_UNSTABLE
        return
    c = F.fd_cfl_limit(d)
    assert abs(c - oc) < 1e-7 * oc


def test_square8_displs_within_ls_cutoff_agreement():
    # the most ill-conditioned LS problem: both solvers truncate at the same
    # relative cutoff and agree to ~1e-6
    d = F.stencil_desc(2, "square", 8, 0, "displs", courant=0.3)
    _, _, w = F.fd_weights(d)
    ow = S.weights(2, "square", 8, 0, "displs", C=0.3)
    keys, _, _ = F.fd_weights(d)
    err = max(abs(w[i] - ow[tuple(int(x) for x in k[:2])]) for i, k in enumerate(keys))
    assert err < 1e-6 * max(abs(x) for x in w)


def test_ricker_matches_oracle():
    f0, dt, nt = 15.0, 1e-3, 300
    a = F.fd_ricker(f0, dt, nt)
    b = P.ricker(f0, nt, dt)
    assert a.dtype == np.float32
    assert np.max(np.abs(a - b)) < 1e-7


def test_plan_validation_and_stability_check():
    d = F.stencil_desc(2, "cross", 4)
    cm = F.fd_cfl_limit(d)
    h, v = 10.0, 3000.0
    ok = F.Plan((50, 60), h, 0.99 * cm * h / v, 10, 5, v, d)
    inf = ok.info()
    assert tuple(inf.padded) == (60, 1, 70)
    assert inf.pitch % 32 == 0 and inf.pitch >= 70
    assert abs(inf.courant_max - cm) < 1e-12
    with pytest.raises(F.FdError) as e:
        F.Plan((50, 60), h, 1.01 * cm * h / v, 10, 5, v, d)
    assert e.value.code == F.FD_ERR_UNSTABLE
    with pytest.raises(F.FdError) as e:
        F.Plan((50, 60), -1.0, 1e-3, 10, 5, v, d)
    assert e.value.code == F.FD_ERR_ARG
    bad = F.stencil_desc(2, "cross_rhombus", 4, 7, "dispte")
    with pytest.raises(F.FdError) as e:
        F.fd_weights(bad)
    assert e.value.code == F.FD_ERR_ARG
    with pytest.raises(F.FdError) as e:
        F.fd_weights(F.stencil_desc(3, "cross", 4, 0, "specte_theta"))
    assert e.value.code == F.FD_ERR_UNSUPPORTED
    # 3D shapes without a specialised kernel run the generic kernel (kernel id ends in 1)
    gp = F.Plan((20, 20, 20), h, 1e-4, 5, 2, v, F.stencil_desc(3, "cross_square", 4, 2, "displs", courant=0.1))
    assert gp.info().kernel % 10 == 1 and gp.variants() == []
    with pytest.raises(F.FdError) as e:   # its DispTE weights have S(k) > 0: no stable dt
        F.Plan((20, 20, 20), h, 1e-4, 5, 2, v, F.stencil_desc(3, "cross_square", 4, 2, "dispte", courant=0.1))
    assert e.value.code == F.FD_ERR_UNSTABLE


def test_taylor_rhombus_reduces_to_cross_kernel():
    d = F.stencil_desc(2, "rhombus", 4, 0, "spatte")
    p = F.Plan((40, 40), 10.0, 5e-4, 4, 4, 3000.0, d)
    assert p.info().effective_shape == F.SHAPES["cross"]
    d = F.stencil_desc(2, "rhombus", 4, 0, "displs", courant=0.15)
    p = F.Plan((40, 40), 10.0, 5e-4, 4, 4, 3000.0, d)
    assert p.info().effective_shape == F.SHAPES["rhombus"]


def test_workspace_sizes():
    d = F.stencil_desc(3, "cross", 4)
    p = F.Plan((30, 31, 32), 10.0, 1e-3, 100, 6, 3000.0, d)
    f = p.forward_workspace_size(1, 100)
    g = p.gradient_workspace_size(1, 100, 10)
    inf = p.info()
    field = inf.padded[0] * inf.padded[1] * inf.pitch * 4
    assert f >= 3 * field
    # gradient: 4 buffers + kappa + gacc + 2*10 checkpoints + 10 segment fields
    assert g >= (6 + 20 + 10) * field
    assert p.gradient_workspace_size(1, 100, 5) > g


def test_gradient_adjoint_needs_a_stored_forward():
    """fd_gradient_adjoint checks, before touching the device, that the plan has
    a stored forward for this workspace and these counts."""
    d = F.stencil_desc(2, "cross", 4)
    p = F.Plan((30, 40), 10.0, 1e-3, 20, 6, 3000.0, d)
    ws = np.zeros(256, np.uint8)
    with pytest.raises(F.FdError) as e:
        F._check(F.lib().fd_gradient_adjoint(p.ptr, 0, None, 0, None, None, ws.ctypes.data, None,
                                             ws.ctypes.data, ws.nbytes, None))
    assert e.value.code == F.FD_ERR_ARG
    assert "fd_gradient_forward" in F.last_error()


@pytest.mark.parametrize("M,N", [(2, 1), (4, 2), (6, 3)])
def test_symbol_positive_stencil_is_rejected(M, N):
    """A stencil whose symbol is positive somewhere (DispTE-CrossSq at C = 0.3)
    has no stable time step: fd_cfl_limit and fd_plan_create refuse it, at any
    dt, while the Taylor cross of the same radius is still accepted."""
    d = F.stencil_desc(2, "cross_square", M, N, "dispte", courant=0.3)
    with pytest.raises(F.FdError) as e:
        F.fd_cfl_limit(d)
    assert e.value.code == F.FD_ERR_UNSTABLE
    assert "unstable at every time step" in str(e.value)
    h, v = 10.0, 3000.0
    for dt in (1e-6, 0.3 * h / v):
        with pytest.raises(F.FdError) as e:
            F.Plan((40, 40), h, dt, 10, 5, v, d)
        assert e.value.code == F.FD_ERR_UNSTABLE
    dc = F.stencil_desc(2, "cross", M)
    F.Plan((40, 40), h, 0.5 * F.fd_cfl_limit(dc) * h / v, 10, 5, v, dc)


def test_weights_conditioning():
    """fd_weights_conditioning against matrices built here.
    - SpatTE Cross(M), 2D: the Taylor system in orbit form (Eq. taylor_system),
      rows r = 0..M, columns (centre, axis orbits m = 1..M): row 0 holds the
      orbit sizes (1, 4, ..., 4), row r >= 1 holds sum over the orbit of
      x^(2r) = 2 m^(2r).
    - DispLS: the design matrix of E_disp(b) on this suite's own quadrature;
      singular values of a smooth Gram operator barely depend on the rule.
    - Square(8) DispLS keeps fewer singular values than unknowns (the
      minimum-norm cutoff fixes part of the weights), and the under-determined
      DispTE square reports its equation count as rank."""
    from test_oracle_weights import _displs_design
    for M in (1, 2, 4, 8):
        A = np.zeros((M + 1, M + 1))
        A[0] = [1] + [4] * M
        for r in range(1, M + 1):
            A[r, 1:] = [2.0 * m ** (2 * r) for m in range(1, M + 1)]
        c, r, n = F.fd_weights_conditioning(F.stencil_desc(2, "cross", M))
        assert (r, n) == (M + 1, M + 1)
        # at M = 8 (condition ~2e15) two double-precision SVDs agree to ~1 %
        assert abs(c / np.linalg.cond(A) - 1) < (1e-6 if M <= 4 else 2e-2)
    for shape, M in (("cross", 4), ("rhombus", 4), ("square", 4)):
        d = F.stencil_desc(2, shape, M, 0, "displs", courant=0.3)
        c, r, n = F.fd_weights_conditioning(d)
        keys = [k for k in S.weights(2, shape, M, 0, "displs", C=0.3) if any(k)]
        A, W = _displs_design(2, keys, 0.3, np.pi / 2, n_beta=48, n_dir=24)
        assert (r, n) == (len(keys), len(keys))
        assert abs(c / np.linalg.cond(A * np.sqrt(W)[:, None]) - 1) < 0.05, (shape, c)
    c, r, n = F.fd_weights_conditioning(F.stencil_desc(2, "square", 8, 0, "displs", courant=0.3))
    assert n == 44 and r < n and c > 1e12
    c, r, n = F.fd_weights_conditioning(F.stencil_desc(2, "square", 3, 0, "dispte", courant=0.3))
    assert n == 10 and r < n and np.isfinite(c)
