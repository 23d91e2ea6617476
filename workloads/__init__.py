"""Seeded synthetic inputs for the acoustic shaped-stencil workloads.

This module is shared by the CUDA path's tests/bench and by the FP64 oracle's
tests.  It holds only problem *inputs*: grid sizes, spacing, step counts,
source/receiver node positions and seeded velocity models.  It contains none
of the method's arithmetic (no stencil weights, no CFL bound, no wavelet, no
damping profile): each side computes those on its own.

Index conventions (shared by both sides):
  * 2D arrays are [z][x], 3D arrays are [z][y][x]; x is contiguous.
  * Sizes are physical node counts (the paper's grid has n_x+1 nodes for
    i = 0..n_x, Section 3.1); the sponge of ``nb`` nodes is added on every
    side by the solver, not here.
  * Positions are physical node indices (z, x) or (z, y, x).

The workloads restate the acquisition geometry of the paper's experiments
(surface sources, dense surface receivers, Ricker wavelets; Section 6) on
synthetic models.  The SEG/EAGE salt and Marmousi models used in Section 6.4
and 6.5 are not available, so the layered/faulted and smooth-random models
below stand in for them.
"""
from __future__ import annotations

import dataclasses
from typing import List, Optional, Sequence, Tuple

import numpy as np

try:  # scipy is present on both the build host and the GPU host
    from scipy.ndimage import gaussian_filter as _gaussian_filter
except Exception:  # pragma: no cover - fallback keeps the module importable
    _gaussian_filter = None


@dataclasses.dataclass
class Stencil:
    """Stencil choice: shape name, radius M, inner size N, weight scheme."""
    shape: str = "cross"        # cross | cross_rhombus | rhombus | cross_square | square
    M: int = 4
    N: int = 0
    scheme: str = "spatte"      # spatte | specte_theta | specls | dispte | displs
    theta: float = np.pi / 8
    b: float = np.pi / 2


@dataclasses.dataclass
class Problem:
    """One acoustic run (inputs only; dt is derived by each solver)."""
    name: str
    dim: int
    shape: Tuple[int, ...]          # physical nodes, (nz, nx) or (nz, ny, nx)
    h: float
    nt: int
    f0: float
    nb: int
    cfl_fraction: float             # dt = cfl_fraction * C_max * h / vmax
    vmax: float
    vel: np.ndarray                 # float32 physical model, m/s
    src: np.ndarray                 # int64 [nsrc, dim] physical node positions
    rec: np.ndarray                 # int64 [nrec, dim] physical node positions
    stencils: List[Stencil] = dataclasses.field(default_factory=list)

    @property
    def padded_shape(self) -> Tuple[int, ...]:
        return tuple(n + 2 * self.nb for n in self.shape)

    @property
    def padded_points(self) -> int:
        return int(np.prod(self.padded_shape))


def _smooth_noise(rng: np.random.Generator, shape, sigma: float) -> np.ndarray:
    """Zero-mean white noise, Gaussian-filtered, scaled to unit max-abs."""
    w = rng.standard_normal(shape)
    if _gaussian_filter is not None:
        w = _gaussian_filter(w, sigma=sigma, mode="nearest")
    m = np.max(np.abs(w))
    return w / m if m > 0 else w


def linear_index(pos: np.ndarray, shape: Sequence[int]) -> np.ndarray:
    """Row-major linear indices of integer node positions into ``shape``."""
    pos = np.asarray(pos, dtype=np.int64)
    return np.ravel_multi_index(tuple(pos.T), tuple(shape)).astype(np.int64)


# ---------------------------------------------------------------------------
# The five workloads (sizes, models, geometry)
# ---------------------------------------------------------------------------

def homogeneous_2d(n: int = 201, h: float = 10.0, v: float = 1500.0, nt: int = 500,
                   f0: float = 15.0, nb: int = 20, rec_depth_m: float = 20.0,
                   stencil: Optional[Stencil] = None) -> Problem:
    """2D homogeneous medium, Cross(4) Taylor, source at the centre and one
    receiver on every x of the row at depth ``rec_depth_m``."""
    vel = np.full((n, n), v, dtype=np.float32)
    c = n // 2
    src = np.array([[c, c]], dtype=np.int64)
    zr = int(round(rec_depth_m / h))
    rec = np.array([[zr, x] for x in range(n)], dtype=np.int64)
    return Problem("2d_homogeneous_%d" % n, 2, (n, n), h, nt, f0, nb, 0.5, v, vel, src, rec,
                   [stencil or Stencil("cross", 4, 0, "spatte")])


def layered_random_2d(n: int = 1001, h: float = 5.0, nt: int = 2000, f0: float = 20.0,
                      nb: int = 40, seed: int = 2) -> Problem:
    """2D smooth random model: three flat interfaces plus Gaussian-filtered
    noise (sigma 15 nodes, +-300 m/s), clipped to [1500, 4500] m/s.  The
    stencil list spans Cross/Rhombus/Square x M in {2,4,8} x {Taylor,
    least-squares dispersion-optimised}."""
    rng = np.random.default_rng(seed)
    z = np.arange(n)[:, None]
    base = np.select([z < 250, z < 500, z < 750], [1800.0, 2600.0, 3400.0], 4200.0)
    base = np.broadcast_to(base, (n, n)).astype(np.float64)
    vel = base + 300.0 * _smooth_noise(rng, (n, n), 15.0)
    vel = np.clip(vel, 1500.0, 4500.0).astype(np.float32)
    src = np.array([[10, n // 2]], dtype=np.int64)
    rec = np.array([[10, x] for x in range(n)], dtype=np.int64)
    stencils = [Stencil(s, M, 0, sch) for s in ("cross", "rhombus", "square")
                for M in (2, 4, 8) for sch in ("spatte", "displs")]
    return Problem("2d_layered_random_%d" % n, 2, (n, n), h, nt, f0, nb, 0.5, 4500.0, vel,
                   src, rec, stencils)


def gradient_random_3d(n: int = 400, h: float = 10.0, nt: int = 1500, f0: float = 15.0,
                       nb: int = 30, seed: int = 3, nrec_side: int = 100) -> Problem:
    """3D smooth random model: linear 1500->4700 m/s gradient in depth plus
    Gaussian-filtered noise (sigma 10 nodes, +-300 m/s), clipped to
    [1500, 5000] m/s.  Source near the surface at the centre; a square grid of
    ``nrec_side``^2 receivers at depth index 2 (every 4th node from 2)."""
    rng = np.random.default_rng(seed)
    zz = np.linspace(1500.0, 4700.0, n)[:, None, None]
    noise = _smooth_noise(rng, (n, n, n), 10.0).astype(np.float32)
    vel = (zz + 300.0 * noise).astype(np.float64)
    vel = np.clip(vel, 1500.0, 5000.0).astype(np.float32)
    c = n // 2
    src = np.array([[5, c, c]], dtype=np.int64)
    step = max(1, (n - 4) // max(1, nrec_side))
    xs = [2 + step * i for i in range(nrec_side) if 2 + step * i < n]
    rec = np.array([[2, y, x] for y in xs for x in xs], dtype=np.int64)
    stencils = [Stencil("cross", 4, 0, "spatte"), Stencil("cross", 8, 0, "spatte"),
                Stencil("rhombus", 4, 0, "displs")]
    return Problem("3d_gradient_random_%d" % n, 3, (n, n, n), h, nt, f0, nb, 0.5, 5000.0, vel,
                   src, rec, stencils)


def faulted_layers_2d(nz: int, nx: int, seed: int, h: float = 10.0,
                      n_layers: int = 6, vmin: float = 1500.0, vmax: float = 5500.0) -> np.ndarray:
    """Layered model with interfaces dipping at seeded angles in [-10, 10]
    degrees and two normal faults with seeded throws of 5-20 nodes."""
    rng = np.random.default_rng(seed)
    vlayers = np.linspace(vmin, vmax, n_layers)
    depths = np.sort(rng.uniform(0.1, 0.95, n_layers - 1)) * nz
    dips = np.tan(np.deg2rad(rng.uniform(-10.0, 10.0, n_layers - 1)))
    fault_x = np.sort(rng.uniform(0.2, 0.8, 2)) * nx
    throws = rng.uniform(5.0, 20.0, 2)
    x = np.arange(nx)[None, :].astype(np.float64)
    z = np.arange(nz)[:, None].astype(np.float64)
    shift = np.zeros((1, nx))
    for fx, th in zip(fault_x, throws):
        shift = shift + np.where(x > fx, th, 0.0)
    vel = np.full((nz, nx), vlayers[0])
    for k in range(n_layers - 1):
        zi = depths[k] + dips[k] * (x - nx / 2.0) + shift
        vel = np.where(z >= zi, vlayers[k + 1], vel)
    return vel.astype(np.float32)


def batched_shots_2d(nt: int = 3000, f0: float = 15.0, nb: int = 20, seed: int = 4,
                     shots_per_grid: int = 16,
                     grids: Sequence[Tuple[int, int]] = ((601, 1201), (401, 801), (801, 2001))
                     ) -> List[Problem]:
    """Batched 2D shots: ``shots_per_grid`` shots on each of three grids of a
    layered model with dipping faults (1500-5500 m/s, h = 10 m), sources spaced
    evenly along physical row 2, receivers on every x of row 2."""
    probs = []
    for gi, (nz, nx) in enumerate(grids):
        vel = faulted_layers_2d(nz, nx, seed + 100 * gi)
        xs = np.linspace(nx / (shots_per_grid + 1), nx * shots_per_grid / (shots_per_grid + 1),
                         shots_per_grid).round().astype(np.int64)
        rec = np.array([[2, x] for x in range(nx)], dtype=np.int64)
        for si, sx in enumerate(xs):
            src = np.array([[2, int(sx)]], dtype=np.int64)
            probs.append(Problem("2d_batched_g%d_s%d" % (gi, si), 2, (nz, nx), 10.0, nt, f0, nb,
                                 0.5, 5500.0, vel, src, rec, [Stencil("cross", 4, 0, "spatte")]))
    return probs


def fwi_models_3d(n: int = 256, seed: int = 5, n_anom: int = 8) -> Tuple[np.ndarray, np.ndarray]:
    """True and initial 3D models for the FWI-gradient workload: smooth
    background 1500->4000 m/s in depth plus ``n_anom`` seeded Gaussian
    anomalies (sigma 6-12 nodes, +-300 m/s); the initial model is the
    background smoothed with sigma = 10 nodes, without anomalies."""
    rng = np.random.default_rng(seed)
    zz = np.linspace(1500.0, 4000.0, n)[:, None, None]
    bg = np.broadcast_to(zz, (n, n, n)).astype(np.float64)
    true = bg.copy()
    g = np.arange(n, dtype=np.float64)
    for _ in range(n_anom):
        cz, cy, cx = rng.uniform(0.2 * n, 0.8 * n, 3)
        sig = rng.uniform(6.0, 12.0)
        amp = rng.choice([-300.0, 300.0])
        ez = np.exp(-((g - cz) ** 2) / (2 * sig * sig))[:, None, None]
        ey = np.exp(-((g - cy) ** 2) / (2 * sig * sig))[None, :, None]
        ex = np.exp(-((g - cx) ** 2) / (2 * sig * sig))[None, None, :]
        true = true + amp * ez * ey * ex
    init = bg.copy()
    if _gaussian_filter is not None:
        init = _gaussian_filter(init, sigma=10.0, mode="nearest")
    return true.astype(np.float32), init.astype(np.float32)


def fwi_geometry_3d(n: int = 256, n_shot_side: int = 4, rec_every: int = 4,
                    depth: int = 2) -> Tuple[np.ndarray, np.ndarray]:
    """Shots on a square surface grid at depth index ``depth`` and receivers on
    every ``rec_every``-th node of that plane."""
    sx = np.linspace(n / (n_shot_side + 1), n * n_shot_side / (n_shot_side + 1),
                     n_shot_side).round().astype(np.int64)
    shots = np.array([[depth, y, x] for y in sx for x in sx], dtype=np.int64)
    r = np.arange(0, n, rec_every, dtype=np.int64)
    rec = np.array([[depth, y, x] for y in r for x in r], dtype=np.int64)
    return shots, rec


def fwi_3d(n: int = 256, h: float = 12.5, nt: int = 1200, f0: float = 15.0, nb: int = 20,
           seed: int = 5, n_shot_side: int = 4) -> Tuple[List[Problem], np.ndarray]:
    """FWI-gradient workload: one Problem per shot on the initial model, and the
    true model (for synthesising observed data)."""
    true, init = fwi_models_3d(n, seed)
    shots, rec = fwi_geometry_3d(n, n_shot_side)
    probs = [Problem("3d_fwi_%d_s%d" % (n, i), 3, (n, n, n), h, nt, f0, nb, 0.5, 4300.0,
                     init, shots[i:i + 1], rec, [Stencil("cross", 4, 0, "spatte")])
             for i in range(len(shots))]
    return probs, true


def random_field(shape: Sequence[int], seed: int, lo: float = -1.0, hi: float = 1.0) -> np.ndarray:
    """Seeded uniform random float64 field (initial states, residuals)."""
    return np.random.default_rng(seed).uniform(lo, hi, size=tuple(shape))


def smooth_velocity(shape: Sequence[int], seed: int, vmin: float, vmax: float,
                    sigma: float = 3.0) -> np.ndarray:
    """Seeded smooth random velocity in [vmin, vmax] (float32) for small cases."""
    rng = np.random.default_rng(seed)
    w = _smooth_noise(rng, tuple(shape), sigma)
    v = 0.5 * (vmin + vmax) + 0.5 * (vmax - vmin) * w
    return np.clip(v, vmin, vmax).astype(np.float32)
