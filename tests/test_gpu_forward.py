"""Forward parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerance: relative L2 <= 1e-4 on traces and final wavefields (the contract
for FP32 wavefields after the full run).  Small cases span several tiles with
ragged tails in every axis; the homogeneous 201^2 workload runs at full size
and length."""
import numpy as np
import pytest

from gpu_cases import Case, per_receiver_errors, rel_l2
from workloads import homogeneous_2d, smooth_velocity

pytestmark = pytest.mark.gpu
TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def built():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_04882_gb300 import build
    build.build()


def _case2d(shape, M, N, scheme, nz=131, nx=157, nb=10, nt=150, seed=11):
    vel = smooth_velocity((nz, nx), seed, 1500.0, 3000.0, sigma=4.0)
    rng = np.random.default_rng(seed)
    src = np.array([[nz // 2, nx // 3], [5, nx - 3]])
    rec = np.stack([rng.integers(0, nz, 40), rng.integers(0, nx, 40)], axis=1)
    rec[0] = (0, 0)
    rec[1] = (nz - 1, nx - 1)
    return Case(vel, 10.0, nt, nb, 3000.0, shape, M, N, scheme, src=src, rec=rec, f0=20.0)


@pytest.mark.parametrize("shape,M,N,scheme", [
    ("cross", 1, 0, "spatte"), ("cross", 2, 0, "spatte"), ("cross", 4, 0, "spatte"),
    ("cross", 8, 0, "spatte"), ("cross", 3, 0, "dispte"), ("cross", 12, 0, "spatte"),
    ("rhombus", 2, 0, "displs"), ("rhombus", 4, 0, "displs"), ("rhombus", 8, 0, "displs"),
    ("square", 2, 0, "displs"), ("square", 4, 0, "displs"), ("square", 8, 0, "displs"),
    ("rhombus", 5, 0, "dispte"), ("cross_rhombus", 4, 2, "dispte"),
    ("cross_square", 4, 2, "displs"), ("cross", 4, 0, "specte_theta"),
])
def test_forward_2d_matches_oracle(shape, M, N, scheme):
    c = _case2d(shape, M, N, scheme)
    tr, st, rc = c.gpu_forward()
    assert rc == 0
    otr, ost = c.oracle_forward(threads=8)
    assert rel_l2(tr, otr) < TOL
    assert per_receiver_errors(tr, otr).max() < 10 * TOL
    assert rel_l2(st[0], ost[0]) < TOL and rel_l2(st[1], ost[1]) < TOL


@pytest.mark.parametrize("shape,M,scheme", [
    ("cross", 1, "spatte"), ("cross", 2, "spatte"), ("cross", 4, "spatte"), ("cross", 8, "spatte"),
    ("rhombus", 2, "displs"), ("rhombus", 4, "displs"), ("cross", 3, "spatte"),
    ("square", 2, "specls"), ("square", 4, "displs"), ("cross", 6, "spatte"),
])
def test_forward_3d_matches_oracle(shape, M, scheme):
    nz, ny, nx, nb = 38, 45, 52, 8
    vel = smooth_velocity((nz, ny, nx), 7, 1500.0, 3000.0, sigma=3.0)
    rng = np.random.default_rng(3)
    rec = np.stack([rng.integers(0, n, 60) for n in (nz, ny, nx)], axis=1)
    src = np.array([[nz // 2, ny // 2, nx // 2], [2, 3, nx - 2]])
    c = Case(vel, 10.0, 70, nb, 3000.0, shape, M, 0, scheme, src=src, rec=rec, f0=25.0)
    tr, st, rc = c.gpu_forward()
    assert rc == 0
    otr, ost = c.oracle_forward(threads=8)
    assert rel_l2(tr, otr) < TOL
    assert per_receiver_errors(tr, otr).max() < 10 * TOL
    assert rel_l2(st[0], ost[0]) < TOL


def test_homogeneous_201_full_run():
    """The 201^2 homogeneous workload (h = 10 m, v = 1500 m/s, Cross(4)
    Taylor, dt = 0.5 CFL, 500 steps, 15 Hz Ricker at the centre, 201
    receivers at 20 m depth, 20-node sponge) at full size and length."""
    pr = homogeneous_2d()
    c = Case(pr.vel, pr.h, pr.nt, pr.nb, pr.vmax, "cross", 4, 0, "spatte", src=pr.src,
             rec=pr.rec, f0=pr.f0)
    tr, st, rc = c.gpu_forward()
    assert rc == 0
    otr, ost = c.oracle_forward(threads=8)
    assert rel_l2(tr, otr) < TOL
    assert rel_l2(st[0], ost[0]) < TOL


def test_restart_from_state_is_bitwise_and_matches_oracle():
    c = _case2d("cross", 4, 0, "spatte", nt=120)
    tr, st, rc = c.gpu_forward()
    tra, sta, _ = c.gpu_forward(nt=50)
    trb, stb, _ = c.gpu_forward(nt=70, state_in=sta, t0=50)
    assert np.array_equal(tr, np.concatenate([tra, trb]))
    assert np.array_equal(st, stb)
    # one GPU step from a mid-run state equals one oracle step from that state
    otr, ost = c.oracle_forward(nt=70, state_in=sta, t0=50)
    assert rel_l2(trb, otr) < TOL and rel_l2(stb[0], ost[0]) < TOL


def test_edge_cases():
    # grid smaller than one tile, no sponge, source and receiver on corners
    vel = np.full((5, 7), 2000.0, np.float32)
    c = Case(vel, 10.0, 20, 0, 2000.0, "cross", 2, 0, "spatte", src=[[0, 0]], rec=[[4, 6], [0, 0], [0, 0]])
    tr, st, rc = c.gpu_forward()
    otr, ost = c.oracle_forward()
    assert rc == 0 and rel_l2(tr, otr) < TOL and rel_l2(st[0], ost[0]) < TOL
    assert np.array_equal(tr[:, 1], tr[:, 2])        # duplicated receiver
    # stencil radius larger than the grid
    vel = np.full((6, 9), 2000.0, np.float32)
    c = Case(vel, 10.0, 15, 0, 2000.0, "cross", 8, 0, "spatte", src=[[3, 4]], rec=[[1, 1]])
    tr, st, rc = c.gpu_forward()
    otr, ost = c.oracle_forward()
    assert rel_l2(tr, otr) < TOL and rel_l2(st[0], ost[0]) < TOL
    # no sources, no receivers, non-zero initial state
    vel = smooth_velocity((40, 50), 1, 1500.0, 2500.0)
    c = Case(vel, 10.0, 30, 4, 2500.0, "rhombus", 4, 0, "displs", src=np.zeros((0, 2)), rec=None)
    st0 = np.random.default_rng(0).standard_normal((2, 48, 58)).astype(np.float32)
    _, st, rc = c.gpu_forward(state_in=st0)
    _, ost = c.oracle_forward(state_in=st0)
    assert rc == 0 and rel_l2(st[0], ost[0]) < TOL
    # zero steps returns the initial state
    c0 = Case(vel, 10.0, 0, 4, 2500.0, "cross", 4, src=np.zeros((0, 2)))
    _, st, _ = c0.gpu_forward(state_in=st0)
    assert np.array_equal(st, st0)


def test_velocity_above_vmax_is_reported():
    import paper_2606_04882_gb300 as F
    vel = np.full((20, 20), 2000.0, np.float32)
    vel[5, 5] = 2600.0
    c = Case(vel, 10.0, 5, 2, 2500.0, "cross", 2, src=[[10, 10]], rec=[[1, 1]])
    _, _, rc = c.gpu_forward()
    assert rc == F.FD_ERR_UNSTABLE


@pytest.mark.parametrize("dim,shape,M,scheme", [(3, "cross", 4, "spatte"), (3, "rhombus", 4, "displs"),
                                                (2, "cross", 4, "spatte")])
def test_autotune_keeps_results_bitwise(dim, shape, M, scheme):
    """The tile shape the autotuner picks changes the schedule, not the
    arithmetic of any point: traces and fields are bitwise identical."""
    import torch
    import paper_2606_04882_gb300 as F
    n = (120, 150) if dim == 2 else (40, 44, 70)
    vel = smooth_velocity(n, 12, 1500.0, 3000.0, sigma=3.0)
    rec = np.array([[2] * (dim - 1) + [x] for x in range(0, n[-1], 3)])
    c = Case(vel, 10.0, 40, 8, 3000.0, shape, M, 0, scheme, src=[[s // 2 for s in n]], rec=rec)
    tr0, st0, _ = c.gpu_forward()
    plan = c.plan()
    plan.autotune(torch.from_numpy(c.vel).cuda())
    after = plan.info()
    dev = torch.device("cuda")
    tr = torch.zeros((c.nt, len(rec)), device=dev)
    ws = F.workspace(plan.forward_workspace_size(1, len(rec)))
    F.fd_forward(plan, torch.from_numpy(c.vel).to(dev), plan.linear_index(c.src),
                 torch.from_numpy(c.wavelet32()).to(dev), plan.linear_index(c.rec), tr, ws)
    assert np.array_equal(tr.cpu().numpy(), tr0)
    # a second plan of the same problem takes the cached choice
    p2 = c.plan()
    p2.autotune(torch.from_numpy(c.vel).cuda())
    assert tuple(p2.info().tile) == tuple(after.tile)


def test_time_loop_schedules_are_bitwise_equal(monkeypatch):
    """The time loop runs as a captured CUDA graph (default, replayed on repeat
    calls), as plain launches, or as one persistent cooperative launch (opt-in
    for small 2D grids); all three give bitwise identical results."""
    c = _case2d("rhombus", 4, 0, "displs", nz=300, nx=280, nt=200)
    tr_g, st_g, rc = c.gpu_forward()
    assert rc == 0
    tr_g2, st_g2, _ = c.gpu_forward()
    monkeypatch.setenv("FDWAVE_GRAPHS", "0")
    tr_s, st_s, rc = c.gpu_forward()
    assert rc == 0
    monkeypatch.setenv("FDWAVE_PERSISTENT", "1")
    tr_p, st_p, rc = c.gpu_forward()
    assert rc == 0
    for tr, st in ((tr_g2, st_g2), (tr_s, st_s), (tr_p, st_p)):
        assert np.array_equal(tr, tr_g) and np.array_equal(st, st_g)


def test_graph_cache_survives_plan_and_buffer_reuse(monkeypatch):
    """Plans and tensors freed and re-created at recycled addresses with a
    different stencil must not replay another plan's captured time loop: the
    graph cache is keyed by plan ids, never by addresses."""
    runs = [("cross", 2, "spatte"), ("cross", 4, "spatte"), ("rhombus", 4, "displs"),
            ("cross", 2, "spatte"), ("square", 2, "displs")]
    got = []
    for shape, M, scheme in runs:
        c = _case2d(shape, M, 0, scheme, nz=90, nx=100, nt=40)
        got.append(c.gpu_forward())
    monkeypatch.setenv("FDWAVE_GRAPHS", "0")
    for (shape, M, scheme), (tr, st, rc) in zip(runs, got):
        c = _case2d(shape, M, 0, scheme, nz=90, nx=100, nt=40)
        tr0, st0, rc0 = c.gpu_forward()
        assert rc == 0 and rc0 == 0
        assert np.array_equal(tr, tr0) and np.array_equal(st, st0), (shape, M, scheme)


@pytest.mark.parametrize("dim,shape,M,N,scheme", [
    (2, "cross", 4, 0, "spatte"), (2, "rhombus", 4, 0, "displs"), (2, "square", 8, 0, "displs"),
    (2, "cross_rhombus", 4, 2, "dispte"), (2, "cross", 3, 0, "dispte"),
    (3, "cross", 4, 0, "spatte"), (3, "cross", 8, 0, "spatte"), (3, "rhombus", 4, 0, "displs"),
    (3, "square", 2, 0, "specls"),
])
def test_constant_field_is_a_fixed_point(dim, shape, M, N, scheme):
    """A constant field (u^n = u^{n-1} = c) is an exact fixed point of one step
    wherever the whole stencil lies in the grid and there is no sponge: the
    kernels sum a_o (u(x+o) - u(x)), which is exactly zero there whatever the
    FP32 rounding of the weights (a literal sum of a_o u(x+o) leaves
    c * sum_o fl(a_o) != 0)."""
    n = (40, 52) if dim == 2 else (24, 28, 36)
    nb = 8
    vel = smooth_velocity(n, 4, 1500.0, 3000.0, sigma=3.0)
    c = Case(vel, 10.0, 1, nb, 3000.0, shape, M, N, scheme, src=np.zeros((0, dim)), rec=None)
    pshape = tuple(s + 2 * nb for s in n)
    st0 = np.full((2,) + pshape, 0.3712, np.float32)
    _, st, rc = c.gpu_forward(state_in=st0)
    assert rc == 0
    inner = (slice(None),) + tuple(slice(nb, nb + s) for s in n)
    assert np.array_equal(st[inner][0], st0[inner][0])


@pytest.mark.parametrize("shape,M,scheme", [("cross", 4, "spatte"), ("cross", 8, "spatte"),
                                            ("rhombus", 4, "displs"), ("square", 2, "specls")])
def test_edge_cases_3d(shape, M, scheme):
    """3D grids smaller than one tile and than the stencil radius, sources and
    receivers on corners, no sponge, and a thin grid whose z extent is shorter
    than the stencil, each against the oracle."""
    # grid smaller than a tile and than the radius in every axis
    vel = np.full((5, 6, 7), 2000.0, np.float32)
    c = Case(vel, 10.0, 12, 0, 2000.0, shape, M, 0, scheme, src=[[0, 0, 0]],
             rec=[[4, 5, 6], [0, 0, 0], [2, 3, 4]])
    tr, st, rc = c.gpu_forward()
    otr, ost = c.oracle_forward()
    assert rc == 0 and rel_l2(tr, otr) < TOL and rel_l2(st[0], ost[0]) < TOL
    # thin in z, wide in x and y (several tiles with ragged tails), with a sponge
    vel = smooth_velocity((3, 37, 131), 9, 1500.0, 3000.0, sigma=3.0)
    c = Case(vel, 10.0, 25, 2, 3000.0, shape, M, 0, scheme, src=[[1, 18, 65], [2, 36, 130]],
             rec=[[0, y, x] for y in (0, 36) for x in range(0, 131, 13)])
    tr, st, rc = c.gpu_forward()
    otr, ost = c.oracle_forward()
    assert rc == 0 and rel_l2(tr, otr) < TOL and rel_l2(st[0], ost[0]) < TOL


@pytest.mark.parametrize("shape,M,scheme", [("rhombus", 4, "displs"), ("cross", 4, "spatte"),
                                            ("cross", 8, "spatte"), ("rhombus", 2, "displs"),
                                            ("square", 2, "specls")])
def test_every_3d_variant_gives_the_same_bits(shape, M, scheme):
    """Every kernel variant built for a 3D stencil (y tile, kernel form, z-chunk;
    fd_plan_variants / fd_plan_set_variant) schedules the same per-point
    arithmetic: traces and final fields are bitwise equal to the default
    variant's, which matches the oracle.  The grid has ragged tiles in every
    axis for every tile shape."""
    import torch
    import paper_2606_04882_gb300 as F
    n = (37, 45, 70)
    vel = smooth_velocity(n, 17, 1500.0, 3000.0, sigma=3.0)
    rng = np.random.default_rng(17)
    rec = np.stack([rng.integers(0, k, 50) for k in n], axis=1)
    c = Case(vel, 10.0, 30, 8, 3000.0, shape, M, 0, scheme, src=[[18, 22, 35], [2, 44, 69]], rec=rec,
             f0=25.0)
    tr0, st0, rc = c.gpu_forward()
    assert rc == 0
    otr, ost = c.oracle_forward(threads=8)
    assert rel_l2(tr0, otr) < TOL and rel_l2(st0[0], ost[0]) < TOL
    plan = c.plan()
    dev = torch.device("cuda")
    vel_t = torch.from_numpy(c.vel).to(dev)
    wav = torch.from_numpy(c.wavelet32()).to(dev)
    variants = plan.variants()
    assert variants
    for v in variants:
        for zc in (0, 5):
            info = plan.set_variant(v, zc)
            tr = torch.zeros((c.nt, len(rec)), device=dev)
            st = torch.zeros((2,) + tuple(plan.padded_shape), device=dev)
            ws = F.workspace(plan.forward_workspace_size(len(c.src), len(rec)))
            F.fd_forward(plan, vel_t, plan.linear_index(c.src), wav, plan.linear_index(c.rec), tr, ws,
                         state_out=st)
            assert F.fd_status_read(plan, ws) == 0
            assert np.array_equal(tr.cpu().numpy(), tr0), (v, zc, tuple(info.tile))
            assert np.array_equal(st.cpu().numpy(), st0), (v, zc, tuple(info.tile))


@pytest.mark.parametrize("shape,M,N,scheme", [
    ("cross_rhombus", 4, 2, "displs"), ("cross_square", 4, 2, "displs"), ("cross", 5, 0, "spatte"),
    ("rhombus", 5, 0, "displs"), ("square", 3, 0, "specls"), ("cross", 12, 0, "spatte"),
])
def test_forward_3d_generic_kernel_matches_oracle(shape, M, N, scheme):
    """3D stencils without a specialised kernel (cross-rhombus, cross-square,
    radii outside the compiled lists, M up to 16) run the generic kernel:
    parity with the oracle on a grid with ragged tiles in every axis, sources
    and receivers inside and on faces."""
    import paper_2606_04882_gb300 as F
    n = (21, 19, 70)
    vel = smooth_velocity(n, 23, 1500.0, 3000.0, sigma=3.0)
    rng = np.random.default_rng(23)
    rec = np.stack([rng.integers(0, k, 40) for k in n], axis=1)
    rec[0] = (0, 0, 0)
    c = Case(vel, 10.0, 30, 5, 3000.0, shape, M, N, scheme, src=[[10, 9, 35], [0, 18, 69]], rec=rec,
             f0=25.0)
    assert c.plan().info().kernel % 10 == 1
    tr, st, rc = c.gpu_forward()
    assert rc == 0
    otr, ost = c.oracle_forward(threads=8)
    assert rel_l2(tr, otr) < TOL
    assert rel_l2(st[0], ost[0]) < TOL and rel_l2(st[1], ost[1]) < TOL
