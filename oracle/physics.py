"""Source wavelet, sponge damping and model padding (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).  The paper names a Ricker
source (Section 3.1, below Eq. wave_eq) and a damping layer of extra
eta(x) u_t (same passage) without formulas; the readings taken here are:

* Ricker: s(t) = (1 - 2 pi^2 f0^2 (t - t0)^2) exp(-pi^2 f0^2 (t - t0)^2),
  t0 = 1/f0, sampled at t^n = n tau.
* Damping: eta(d) = eta_max (d / nb)^2 summed over axes, d the node distance
  into the layer (0 in the physical domain), eta_max = 3 c_max ln(1/R) /
  (2 nb h) with R = 1e-3, and gamma = eta tau / 2 (centred u_t).
* Padding: the physical model is extended into the sponge by edge
  replication; the field is zero outside the padded grid.
"""
from __future__ import annotations

import math
from typing import Sequence

import numpy as np


def ricker(f0: float, nt: int, dt: float) -> np.ndarray:
    t = np.arange(nt, dtype=np.float64) * dt - 1.0 / f0
    a = (math.pi * f0 * t) ** 2
    return (1.0 - 2.0 * a) * np.exp(-a)


def eta_max(vmax: float, nb: int, h: float, R: float = 1e-3) -> float:
    return 3.0 * vmax * math.log(1.0 / R) / (2.0 * nb * h) if nb > 0 else 0.0


def layer_distance(n_phys: int, nb: int) -> np.ndarray:
    """Node distance into the sponge along one padded axis of n_phys + 2 nb."""
    i = np.arange(n_phys + 2 * nb)
    return np.maximum(np.maximum(nb - i, i - (nb + n_phys - 1)), 0).astype(np.float64)


def gamma_field(phys_shape: Sequence[int], nb: int, dt: float, h: float, vmax: float,
                R: float = 1e-3) -> np.ndarray:
    """gamma = eta dt / 2 on the padded grid (float64)."""
    if nb == 0:
        return np.zeros(tuple(phys_shape))
    em = eta_max(vmax, nb, h, R)
    ds = [(layer_distance(n, nb) / nb) ** 2 for n in phys_shape]
    grids = np.meshgrid(*ds, indexing="ij")
    return 0.5 * dt * em * sum(grids)


def pad(model: np.ndarray, nb: int) -> np.ndarray:
    return np.pad(np.asarray(model, dtype=np.float64), nb, mode="edge")


def fold(gpad: np.ndarray, nb: int) -> np.ndarray:
    """Adjoint of ``pad``: each padded value is added to the physical node it
    replicates."""
    g = np.asarray(gpad, dtype=np.float64)
    for ax in range(g.ndim):
        n = g.shape[ax] - 2 * nb
        lo = np.take(g, range(0, nb + 1), axis=ax).sum(axis=ax, keepdims=True)
        hi = np.take(g, range(nb + n - 1, n + 2 * nb), axis=ax).sum(axis=ax, keepdims=True)
        mid = np.take(g, range(nb + 1, nb + n - 1), axis=ax)
        g = np.concatenate([lo, mid, hi], axis=ax) if n > 1 else lo + hi - np.take(g, [nb], axis=ax)
    return g
