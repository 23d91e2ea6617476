"""Host-side set-up of the accuracy experiments (no GPU): the scheme sweep,
the refined models and the node and time mapping between the coarse grid
and the refined reference."""
import numpy as np

from paper_2606_04882_gb300 import experiments as E


def test_scheme_sweep_covers_every_shape_and_order():
    s = E.schemes(6)
    # per M: SpatTE + SpecTE-theta crosses, 3 weight schemes x (M rhombus + M+1 square)
    assert len(s) == sum(2 + 3 * (2 * M + 1) for M in range(1, 7)) == 156
    assert len({r[0] for r in s}) == len(s)
    for label, shape, M, N, sch in s:
        if shape == "cross_rhombus":
            assert 1 <= N <= M
        elif shape == "cross_square":
            assert 0 <= N <= M
        else:
            assert shape == "cross" and N == 0 and sch in ("spatte", "specte_theta")


def test_tables_of_the_paper():
    e1, e2 = E.homogeneous(), E.two_layer()
    assert (e1.n - 1) * e1.h == 6000.0 and (e2.n - 1) * e2.h == 4000.0
    assert (e1.dt, e1.nt, e1.f0, e1.vmax) == (2.0e-3, 1500, 30.0, 3000.0)
    assert (e2.dt, e2.nt, e2.f0, e2.vmax) == (1.0e-3, 1500, 25.0, 3000.0)
    assert e1.n_snap == 525 and e2.n_snap == 1080          # 1.05 s and 1.08 s
    assert e1.node(e1.src, 1) == (200, 200)                 # centre of the domain
    assert e1.node(e1.trace, 1) == (200, 80)                # x = 1200 m, z = 3000 m
    assert e2.node(e2.src, 1) == (160, 200)                 # x = 2000 m, z = 1600 m
    assert e2.node(e2.trace, 1) == (200, 100)               # x = 1000 m, z = 2000 m


def test_refined_grid_contains_the_coarse_nodes():
    for ex in (E.homogeneous(), E.two_layer()):
        for r in (2, 4, 16):
            assert ex.node(ex.src, r) == tuple(r * i for i in ex.node(ex.src, 1))
            assert ex.node(ex.trace, r) == tuple(r * i for i in ex.node(ex.trace, 1))
        coarse = ex.model(1)
        fine = ex.model(4)
        assert fine.shape == (4 * (ex.n - 1) + 1,) * 2
        assert np.array_equal(fine[::4, ::4], coarse)


def test_two_layer_interface():
    v = E.two_layer().model(1)
    assert np.all(v[:121] == 1500.0) and np.all(v[121:] == 3000.0)   # z <= 1200 m is slow
    assert np.all(E.homogeneous().model(1) == 3000.0)
