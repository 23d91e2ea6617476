"""Python driver of the FP64 C oracle (test infrastructure only).

Builds ``wave_oracle.c`` with gcc (OpenMP) into ``oracle/_objs`` and calls it
through ctypes.  Everything here is FP64; inputs that the CUDA path receives
as FP32 (velocity model, wavelet) are passed in already rounded to FP32 by the
tests so that both sides see identical data.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from typing import Optional, Sequence

import numpy as np

from . import physics, stencil

_HERE = os.path.dirname(os.path.abspath(__file__))
_OBJ = os.path.join(_HERE, "_objs")
_SO = os.path.join(_OBJ, "liboracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle (plain gcc -O2 -fopenmp, no target-specific flags)."""
    src = os.path.join(_HERE, "wave_oracle.c")
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        os.makedirs(_OBJ, exist_ok=True)
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c99",
                               "-o", tmp, src, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        i64, i32, dp = ctypes.c_int64, ctypes.c_int, ctypes.c_void_p
        _lib.oracle_forward.argtypes = [i64, i64, i64, dp, dp, i32, dp, dp, i32, i32, dp, dp,
                                        i32, dp, dp, dp, dp, i32]
        _lib.oracle_gradient.argtypes = [i64, i64, i64, dp, dp, i32, dp, dp, i32, i32, dp, dp,
                                         i32, dp, dp, i32, dp, dp, dp, i32, i32]
        _lib.oracle_forward.restype = i32
        _lib.oracle_gradient.restype = i32
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def default_threads() -> int:
    return int(os.environ.get("ORACLE_THREADS", os.cpu_count() or 1))


class Setup:
    """Padded FP64 inputs of one run (Section 3.1): kappa = (v tau / h)^2,
    gamma of the sponge, the stencil's offset list, source amplitudes
    tau^2 s(t^n) / h^dim and padded receiver indices."""

    def __init__(self, vel: np.ndarray, h: float, dt: float, nb: int, vmax: float,
                 dim: int, shape: str = "cross", M: int = 4, N: int = 0,
                 scheme: str = "spatte", weights=None, theta: float = np.pi / 8,
                 b: float = np.pi / 2, damp_R: float = 1e-3):
        vel = np.asarray(vel, dtype=np.float64)
        assert vel.ndim == dim
        self.dim, self.h, self.dt, self.nb = dim, h, dt, nb
        self.phys_shape = vel.shape
        vp = physics.pad(vel, nb)
        self.pshape = vp.shape
        self.kappa = np.ascontiguousarray((vp * dt / h) ** 2)
        self.m = 1.0 / vp ** 2
        self.gamma = np.ascontiguousarray(physics.gamma_field(vel.shape, nb, dt, h, vmax, damp_R))
        if weights is None:
            C = vmax * dt / h
            weights = stencil.weights(dim, shape, M, N, scheme, C, theta, b)
        self.orbit_weights = weights
        pw = stencil.expand(dim, shape, M, N, weights)
        self.points = pw
        off = np.zeros((len(pw), 3), dtype=np.int32)
        for i, (o, _) in enumerate(pw):
            if dim == 2:
                off[i] = (o[0], 0, o[1])
            else:
                off[i] = o
        self.off = off
        self.w = np.array([w for _, w in pw], dtype=np.float64)

    @property
    def dims3(self):
        if self.dim == 2:
            return self.pshape[0], 1, self.pshape[1]
        return self.pshape

    def padded_index(self, pos: np.ndarray) -> np.ndarray:
        pos = np.asarray(pos, dtype=np.int64) + self.nb
        return np.ravel_multi_index(tuple(pos.T), self.pshape).astype(np.int64)

    def source_amp(self, wavelet: np.ndarray) -> np.ndarray:
        """[nt][nsrc] injected values tau^2 s(t^n) / h^dim (Eq. wave_eq with
        f = s(t) delta(x - x_s), the delta discretised as 1/h^dim)."""
        w = np.asarray(wavelet, dtype=np.float64)
        if w.ndim == 1:
            w = w[:, None]
        return np.ascontiguousarray(w * self.dt ** 2 / self.h ** self.dim)


def forward(st: Setup, nt: int, src_pos: np.ndarray, wavelet: np.ndarray,
            rec_pos: np.ndarray, u0: Optional[np.ndarray] = None,
            um1: Optional[np.ndarray] = None, threads: Optional[int] = None):
    """Run nt steps; returns (traces [nt, nrec], u^{nt}, u^{nt-1}) on the
    padded grid.  ``u0``/``um1`` are optional initial states u^0, u^{-1}."""
    lib = _load()
    nz, ny, nx = st.dims3
    cur = np.zeros(st.pshape) if u0 is None else np.array(u0, dtype=np.float64, copy=True)
    prev = np.zeros(st.pshape) if um1 is None else np.array(um1, dtype=np.float64, copy=True)
    src_idx = st.padded_index(np.atleast_2d(src_pos)) if src_pos is not None and len(src_pos) else np.zeros(0, np.int64)
    amp = st.source_amp(wavelet) if len(src_idx) else None
    rec_idx = st.padded_index(np.atleast_2d(rec_pos)) if rec_pos is not None and len(rec_pos) else np.zeros(0, np.int64)
    traces = np.zeros((nt, len(rec_idx)))
    rc = lib.oracle_forward(nz, ny, nx, _p(st.kappa), _p(st.gamma), len(st.w), _p(st.off),
                            _p(st.w), nt, len(src_idx), _p(src_idx), _p(amp), len(rec_idx),
                            _p(rec_idx), _p(traces), _p(prev), _p(cur),
                            threads or default_threads())
    assert rc == 0
    return traces, cur, prev


def gradient(st: Setup, nt: int, src_pos: np.ndarray, wavelet: np.ndarray,
             rec_pos: np.ndarray, resid: np.ndarray, adj_pos: Optional[np.ndarray] = None,
             seg: Optional[int] = None, threads: Optional[int] = None, padded: bool = False):
    """dJ/dm for m = 1/v^2 with residual r = dJ/dtrace [nt, nrec].  Returns
    (grad on the physical grid (or padded if ``padded``), adj_trace [nt, nadj])
    where adj_trace[n] = nu^{n+1} at ``adj_pos``."""
    lib = _load()
    nz, ny, nx = st.dims3
    src_idx = st.padded_index(np.atleast_2d(src_pos)) if src_pos is not None and len(src_pos) else np.zeros(0, np.int64)
    amp = st.source_amp(wavelet) if len(src_idx) else None
    rec_idx = st.padded_index(np.atleast_2d(rec_pos))
    resid = np.ascontiguousarray(resid, dtype=np.float64)
    assert resid.shape == (nt, len(rec_idx))
    adj_idx = st.padded_index(np.atleast_2d(adj_pos)) if adj_pos is not None else np.zeros(0, np.int64)
    adj_trace = np.zeros((nt, len(adj_idx)))
    G = np.zeros(st.pshape)
    if seg is None:
        seg = max(1, int(np.sqrt(2 * nt)))
    rc = lib.oracle_gradient(nz, ny, nx, _p(st.kappa), _p(st.gamma), len(st.w), _p(st.off),
                             _p(st.w), nt, len(src_idx), _p(src_idx), _p(amp), len(rec_idx),
                             _p(rec_idx), _p(resid), len(adj_idx), _p(adj_idx), _p(adj_trace),
                             _p(G), seg, threads or default_threads())
    assert rc == 0
    gpad = -(st.kappa / st.m) * G
    if padded:
        return gpad, adj_trace
    return physics.fold(gpad, st.nb), adj_trace
