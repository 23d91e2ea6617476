"""Pins of the oracle's evaluation metrics (Section 2.4 norms, Appendix A DFT
dispersion metric) against closed forms."""
import numpy as np

from oracle import metrics as X


def test_error_norms_closed_form():
    num = np.array([[1.0, -2.0], [3.0, 0.5]])
    ref = np.array([[0.0, 0.0], [1.0, 0.5]])
    s1, s2 = X.snapshot_scales(10.0)
    a, b, c = X.error_norms(num, ref, s1, s2)
    assert np.isclose(a, 5.0 / 100.0)           # |1| + |-2| + |2| + 0, times 1/h^2
    assert np.isclose(b, 3.0 / 10.0)            # sqrt(1 + 4 + 4), times 1/h
    assert c == 2.0
    assert X.error_norms(num, num, 1.0, 1.0) == (0.0, 0.0, 0.0)


def test_dft_of_a_delta_and_a_cosine():
    nt = 64
    u = np.zeros((nt, 2))
    u[0, 0] = 1.0
    u[:, 1] = np.cos(2 * np.pi * 5 * np.arange(nt) / nt)
    A = X.dft(u, nt // 2 + 1)
    assert np.allclose(A[:, 0], 1.0)                          # delta: flat spectrum
    expect = np.zeros(nt // 2 + 1)
    expect[5] = nt / 2                                         # cosine: one line of height nt/2
    assert np.allclose(A[:, 1], expect, atol=1e-9)


def test_gamma_of_identical_traces_is_zero():
    rng = np.random.default_rng(3)
    u = rng.standard_normal((200, 4))
    g, n, avg, mx = X.dft_gamma(u, u)
    assert np.all(g == 0) and np.all(n == 0) and avg == 0 and mx == 0


def test_gamma_of_a_phase_shifted_cosine():
    """num = cos(w n + delta), ref = cos(w n) on an exact DFT line: gamma is
    delta/pi at that line (where the amplitude is the maximum) and 0 elsewhere."""
    nt, k0 = 128, 9
    n = np.arange(nt)
    for delta in (0.3, -1.2, 2.9):
        num = np.cos(2 * np.pi * k0 * n / nt + delta)[:, None]
        ref = np.cos(2 * np.pi * k0 * n / nt)[:, None]
        g, norms, _, _ = X.dft_gamma(num, ref)
        assert np.isclose(g[0, k0], delta / np.pi)
        others = np.delete(g[0], k0)
        assert np.max(np.abs(others)) < 1e-10
        assert np.isclose(norms[0], abs(delta) / np.pi / np.sqrt(nt // 2 + 1))


def test_phase_difference_wraps_into_minus_pi_pi():
    """Phases 3.0 (num) and -3.0 (ref) differ by 6.0 - 2 pi, not by 6.0."""
    nt, k0 = 64, 4
    n = np.arange(nt)
    num = np.cos(2 * np.pi * k0 * n / nt + 3.0)[:, None]
    ref = np.cos(2 * np.pi * k0 * n / nt - 3.0)[:, None]
    g, _, _, _ = X.dft_gamma(num, ref)
    assert np.isclose(g[0, k0], (6.0 - 2 * np.pi) / np.pi)


def test_gamma_of_a_time_delay():
    """A pure delay by m samples of a periodic trace rotates line k by
    -2 pi k m / nt (wrapped): gamma_k follows that, weighted by |A_k| / max."""
    rng = np.random.default_rng(5)
    nt, m = 96, 3
    ref = rng.standard_normal((nt, 1))
    num = np.roll(ref, m, axis=0)
    g, _, avg, mx = X.dft_gamma(num, ref)
    A = np.abs(np.fft.fft(ref[:, 0]))[: nt // 2 + 1]
    k = np.arange(nt // 2 + 1)
    ph = -2 * np.pi * k * m / nt
    ph = (ph + np.pi) % (2 * np.pi) - np.pi
    expect = ph / np.pi * A / A.max()
    edge = np.isclose(np.abs(ph), np.pi)       # a shift of exactly pi is +pi or -pi
    assert np.allclose(g[0][~edge], expect[~edge], atol=1e-9)
    assert np.allclose(np.abs(g[0][edge]), np.abs(expect[edge]), atol=1e-9)
    assert avg == mx


# --- wavelet (CWT) dispersion metric -------------------------------------------------


def test_cwt_tone_peaks_at_its_matched_scale():
    """A pure tone on DFT line k1: its wavelet power over the scales peaks at
    the scale matched to line k1 (the stationary point of the power in s),
    its envelope is constant in time and its phase advances 2 pi k1 / nt per
    sample."""
    nt = 256
    n = np.arange(nt)
    for k1, w0 in ((9, 6.0), (23, 6.0), (40, 8.0)):
        u = np.cos(2 * np.pi * k1 * n / nt + 0.4)[:, None]
        S = X.cwt(u, 60, w0)[0]
        power = (np.abs(S) ** 2).mean(axis=1)
        assert np.argmax(power) == k1
        env = np.abs(S[k1])
        assert env.std() < 1e-12 * env.mean()
        step = np.angle(S[k1, 1:] / S[k1, :-1])
        assert np.allclose(step, 2 * np.pi * k1 / nt, atol=1e-12)
        assert np.all(S[0] == 0)


def test_cwt_of_an_impulse_has_unit_energy_per_scale():
    """The normalisation (2 pi s / tau)^(1/2) pi^(-1/4) gives every wavelet unit
    energy: for a unit impulse, sum_n |S_{n,k}|^2 = 1 at every scale whose
    Gaussian lies well inside (0, nt/2]."""
    nt = 1024
    u = np.zeros((nt, 1))
    u[0, 0] = 1.0
    S = X.cwt(u, 120)[0]
    e = (np.abs(S) ** 2).sum(axis=1)
    assert np.allclose(e[15:120], 1.0, rtol=1e-6)


def test_cwt_of_a_delayed_trace_is_the_delayed_cwt():
    """Circularly delaying the trace by m samples delays each scale's row by m
    (this fixes the sign of the inverse transform's exponent)."""
    rng = np.random.default_rng(7)
    nt, m = 200, 13
    u = rng.standard_normal((nt, 3))
    S = X.cwt(u, 50)
    Sd = X.cwt(np.roll(u, m, axis=0), 50)
    assert np.allclose(Sd, np.roll(S, m, axis=2), atol=1e-12 * np.abs(S).max())


def test_cwt_rows_hold_only_positive_frequencies():
    """The Heaviside factor: every scale's row is an analytic signal, with no
    zero-frequency and no negative-frequency content."""
    rng = np.random.default_rng(8)
    nt = 150
    S = X.cwt(rng.standard_normal((nt, 2)), 40)
    F = np.fft.fft(S, axis=2)
    tol = 1e-12 * np.abs(F).max()
    assert np.abs(F[..., 0]).max() < tol
    assert np.abs(F[..., nt // 2 + 1:]).max() < tol


def test_gamma_w_of_a_phase_shifted_tone():
    """num = cos(w n + delta), ref = cos(w n), w on DFT line k1: every S^num is
    e^{i delta} S^ref, so gamma^W = (delta/pi) |S^num| / max |S^num|; it is
    delta/pi along the matched scale, where the amplitude is largest."""
    nt, k1 = 128, 11
    n = np.arange(nt)
    for delta in (0.5, -2.0, 3.0):
        num = np.cos(2 * np.pi * k1 * n / nt + delta)[:, None]
        ref = np.cos(2 * np.pi * k1 * n / nt)[:, None]
        g, norms, avg, mx, amax = X.cwt_gamma(num, ref, 30)
        assert np.allclose(g[0, k1], delta / np.pi, atol=1e-12)
        assert np.abs(g).max() <= abs(delta) / np.pi + 1e-12
        assert avg == mx == norms[0] > 0


def test_gamma_w_wraps_and_vanishes_where_it_should():
    nt, k1 = 64, 5
    n = np.arange(nt)
    num = np.cos(2 * np.pi * k1 * n / nt + 3.0)[:, None]
    ref = np.cos(2 * np.pi * k1 * n / nt - 3.0)[:, None]
    g, _, _, _, _ = X.cwt_gamma(num, ref, 12)
    assert np.allclose(g[0, k1], (6.0 - 2 * np.pi) / np.pi, atol=1e-12)
    rng = np.random.default_rng(9)
    u = rng.standard_normal((80, 3))
    g, norms, avg, mx, amax = X.cwt_gamma(u, u)
    assert np.all(g == 0) and np.all(norms == 0) and avg == mx == 0 and np.all(amax > 0)
    z = u.copy()
    z[:, 1] = 0.0
    g, norms, _, _, amax = X.cwt_gamma(z, u)
    assert np.all(g[1] == 0) and norms[1] == 0 and amax[1] == 0
