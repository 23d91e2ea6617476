"""GB300 shaped-stencil acoustic wave engine: Python binding of libfdwave.

Thin ctypes layer over the C ABI declared in ``include/fdwave.h``; the names
match the C entry points (``fd_weights``, ``fd_forward``, ...).  PyTorch
supplies device memory and streams only; every step of the time loop runs in
the library's CUDA kernels.  There is no CPU fallback: if the shared library
is missing or no GPU is present, the device calls raise.

The ``Plan`` helper and ``AcousticTraces`` (a ``torch.autograd.Function``
mapping m = 1/v^2 to receiver traces, with the exact discrete adjoint as its
backward) are conveniences built only from those entry points.
"""
from __future__ import annotations

import ctypes
import enum
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libfdwave.so")

# ----------------------------------------------------------------------------
# enums and structs (mirror include/fdwave.h)
# ----------------------------------------------------------------------------
FD_OK, FD_ERR_ARG, FD_ERR_CUDA, FD_ERR_UNSTABLE = 0, -1, -2, -3
FD_ERR_SINGULAR, FD_ERR_TIMEOUT, FD_ERR_NOMEM, FD_ERR_UNSUPPORTED = -4, -5, -6, -7

SHAPES = {"cross": 0, "cross_rhombus": 1, "rhombus": 2, "cross_square": 3, "square": 4}
SCHEMES = {"spatte": 0, "specte_theta": 1, "specls": 2, "dispte": 3, "dispte_theta": 4,
           "displs": 5}
LS_BASIS = {"paper": 0, "taylor": 1, "cosine": 2}
FD_MODEL_VELOCITY, FD_MODEL_SLOWNESS2 = 0, 1
FD_MAX_ORBITS = 160


class fd_stencil_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("shape", ctypes.c_int32), ("M", ctypes.c_int32),
                ("N", ctypes.c_int32), ("scheme", ctypes.c_int32), ("ls_basis", ctypes.c_int32),
                ("courant", ctypes.c_double), ("theta", ctypes.c_double),
                ("band", ctypes.c_double)]


class fd_problem(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("nb", ctypes.c_int32), ("n", ctypes.c_int64 * 3),
                ("nt", ctypes.c_int32), ("reserved", ctypes.c_int32), ("h", ctypes.c_double),
                ("dt", ctypes.c_double), ("vmax", ctypes.c_double), ("damp_R", ctypes.c_double)]


class fd_plan_info(ctypes.Structure):
    _fields_ = [("padded", ctypes.c_int64 * 3), ("pitch", ctypes.c_int64),
                ("n_orbits", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("courant_max", ctypes.c_double), ("tile", ctypes.c_int32 * 3),
                ("effective_shape", ctypes.c_int32)]


class fd_shot(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("model_kind", ctypes.c_int32),
                ("nsrc", ctypes.c_int32), ("nrec", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("model_d", ctypes.c_void_p), ("src_idx", ctypes.c_void_p),
                ("wavelet_d", ctypes.c_void_p), ("rec_idx", ctypes.c_void_p),
                ("traces_d", ctypes.c_void_p)]


class fd_grad_shot(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("model_kind", ctypes.c_int32),
                ("nsrc", ctypes.c_int32), ("nrec", ctypes.c_int32), ("reserved", ctypes.c_int32),
                ("model_d", ctypes.c_void_p), ("src_idx", ctypes.c_void_p),
                ("wavelet_d", ctypes.c_void_p), ("rec_idx", ctypes.c_void_p),
                ("resid_d", ctypes.c_void_p), ("grad_d", ctypes.c_void_p),
                ("traces_d", ctypes.c_void_p)]


class FdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("fdwave error %d: %s" % (code, msg))
        self.code = code


_lib = None
_P, _I, _I64, _D, _SZ = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double, ctypes.c_size_t
_SIGS = {
    "fd_error_norms": (_I, [_P, _P, _I64, _D, _D, _P, _P]),
    "fd_dft_gamma": (_I, [_P, _P, _I, _I, _I, _P, _P, _P, _P, _P, _P]),
    "fd_cwt_gamma": (_I, [_P, _P, _I, _I, _I, _D, _P, _P, _P, _P, _P, _P, _P, _P, _P]),
    "fd_weights": (_I, [_P, _I, _P, _P, _P, _P]),
    "fd_cfl_limit": (_I, [_P, _P]),
    "fd_weights_conditioning": (_I, [_P, _P, _P, _P]),
    "fd_ricker": (_I, [_D, _D, _I, _P]),
    "fd_plan_create": (_I, [_P, _P, _P]),
    "fd_plan_destroy": (None, [_P]),
    "fd_plan_get_info": (_I, [_P, _P]),
    "fd_plan_autotune": (_I, [_P, _I, _P, _P, _SZ, _P]),
    "fd_plan_variants": (_I, [_P, _I, _P, _P]),
    "fd_plan_set_variant": (_I, [_P, _I, _I]),
    "fd_forward_workspace_size": (_I, [_P, _I, _I, _P]),
    "fd_forward": (_I, [_P, _I, _P, _I, _P, _P, _I, _P, _P, _P, _P, _P, _SZ, _P]),
    "fd_status_read": (_I, [_P, _P, _P]),
    "fd_gradient_workspace_size": (_I, [_P, _I, _I, _I, _P]),
    "fd_adjoint_gradient": (_I, [_P, _I, _P, _I, _P, _P, _I, _P, _P, _I, _P, _P, _P, _P, _SZ, _P]),
    "fd_gradient_forward": (_I, [_P, _I, _P, _I, _P, _P, _I, _P, _P, _P, _SZ, _P]),
    "fd_gradient_adjoint": (_I, [_P, _I, _P, _I, _P, _P, _P, _P, _P, _SZ, _P]),
    "fd_forward_batched_workspace_size": (_I, [_I, _P, _P]),
    "fd_forward_batched": (_I, [_I, _P, _P, _SZ, _P]),
    "fd_forward_batched_autotune": (_I, [_I, _P, _P, _SZ, _P]),
    "fd_forward_batched_set_variant": (_I, [_I, _P, _I]),
    "fd_forward_noalloc": (_I, [_P, _I, _P, _I, _P, _P, _I, _P, _P, _P, _P, _P]),
    "fd_adjoint_gradient_batched_workspace_size": (_I, [_I, _P, _I, _P]),
    "fd_adjoint_gradient_batched": (_I, [_I, _P, _I, _P, _SZ, _P]),
    "fd_status_read_noalloc": (_I, [_P, _P]),
    "fd_last_error": (ctypes.c_char_p, []),
    "fd_version": (ctypes.c_char_p, []),
}


def lib() -> ctypes.CDLL:
    """The loaded libfdwave.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libfdwave.so is not built (run __graft_entry__.build() or "
                               "python -m paper_2606_04882_gb300.build); there is no CPU fallback")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def last_error() -> str:
    return lib().fd_last_error().decode()


def _check(rc: int):
    if rc != FD_OK:
        raise FdError(rc, last_error())


def _addr(x) -> Optional[int]:
    """Device/host address of a tensor/array (None for None)."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    return int(x)


# ----------------------------------------------------------------------------
# host entry points
# ----------------------------------------------------------------------------

def stencil_desc(dim: int, shape: str = "cross", M: int = 4, N: int = 0, scheme: str = "spatte",
                 courant: float = 0.0, theta: float = np.pi / 8, band: float = np.pi / 2,
                 ls_basis: str = "paper") -> fd_stencil_desc:
    return fd_stencil_desc(dim, SHAPES[shape], M, N, SCHEMES[scheme], LS_BASIS[ls_basis],
                           courant, theta, band)


def fd_weights(desc: fd_stencil_desc):
    """Orbit keys [n, 3], multiplicities [n] and FP64 weights [n]."""
    n = ctypes.c_int(0)
    keys = np.zeros((FD_MAX_ORBITS, 3), np.int32)
    mult = np.zeros(FD_MAX_ORBITS, np.int32)
    w = np.zeros(FD_MAX_ORBITS, np.float64)
    _check(lib().fd_weights(ctypes.byref(desc), FD_MAX_ORBITS, ctypes.byref(n), keys.ctypes.data,
                            mult.ctypes.data, w.ctypes.data))
    k = n.value
    return keys[:k].copy(), mult[:k].copy(), w[:k].copy()


def fd_cfl_limit(desc: fd_stencil_desc) -> float:
    c = ctypes.c_double(0.0)
    _check(lib().fd_cfl_limit(ctypes.byref(desc), ctypes.byref(c)))
    return c.value


def fd_weights_conditioning(desc: fd_stencil_desc):
    """(condition number, numerical rank, unknowns) of the weight system."""
    c, r, n = ctypes.c_double(0.0), ctypes.c_int(0), ctypes.c_int(0)
    _check(lib().fd_weights_conditioning(ctypes.byref(desc), ctypes.byref(c), ctypes.byref(r),
                                         ctypes.byref(n)))
    return c.value, r.value, n.value


def fd_ricker(f0: float, dt: float, nt: int) -> np.ndarray:
    out = np.zeros(nt, np.float32)
    _check(lib().fd_ricker(f0, dt, nt, out.ctypes.data))
    return out


def fd_version() -> str:
    return lib().fd_version().decode()


# ----------------------------------------------------------------------------
# plans and device calls (torch supplies memory and streams)
# ----------------------------------------------------------------------------

def _torch():
    import torch
    return torch


def _stream_ptr(stream=None) -> int:
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


class Plan:
    """Owns an fd_plan (host only).  ``shape`` is the physical grid (nz, nx) or
    (nz, ny, nx)."""

    def __init__(self, shape: Sequence[int], h: float, dt: float, nt: int, nb: int, vmax: float,
                 stencil: fd_stencil_desc, damp_R: float = 0.0):
        dim = len(shape)
        n = (shape[0], 1, shape[1]) if dim == 2 else tuple(shape)
        self.prob = fd_problem(dim, nb, (ctypes.c_int64 * 3)(*n), nt, 0, h, dt, vmax, damp_R)
        self.stencil = stencil
        self.shape = tuple(shape)
        self.dim, self.nb, self.nt, self.h, self.dt = dim, nb, nt, h, dt
        p = ctypes.c_void_p(0)
        _check(lib().fd_plan_create(ctypes.byref(self.prob), ctypes.byref(stencil), ctypes.byref(p)))
        self.ptr = p

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            _lib.fd_plan_destroy(self.ptr)
            self.ptr = None

    def info(self) -> fd_plan_info:
        inf = fd_plan_info()
        _check(lib().fd_plan_get_info(self.ptr, ctypes.byref(inf)))
        return inf

    @property
    def padded_shape(self):
        inf = self.info()
        p = tuple(inf.padded)
        return (p[0], p[2]) if self.dim == 2 else p

    def autotune(self, model, model_kind: int = FD_MODEL_VELOCITY, stream=None):
        """fd_plan_autotune on a scratch workspace (torch allocation)."""
        ws = workspace(self.forward_workspace_size(0, 0) + 4096, model.device)
        _check(lib().fd_plan_autotune(self.ptr, model_kind, _addr(model), _addr(ws), ws.numel(),
                                      _stream_ptr(stream)))
        return self.info()

    def variants(self):
        """Kernel variants built for this plan's stencil (fd_plan_variants)."""
        n = ctypes.c_int(0)
        buf = (ctypes.c_int * 16)()
        _check(lib().fd_plan_variants(self.ptr, 16, ctypes.byref(n), buf))
        return list(buf[:n.value])

    def set_variant(self, variant: int, z_chunk: int = 0):
        """fd_plan_set_variant; returns the plan info."""
        _check(lib().fd_plan_set_variant(self.ptr, variant, z_chunk))
        return self.info()

    def forward_workspace_size(self, nsrc: int, nrec: int) -> int:
        b = ctypes.c_size_t(0)
        _check(lib().fd_forward_workspace_size(self.ptr, nsrc, nrec, ctypes.byref(b)))
        return b.value

    def gradient_workspace_size(self, nsrc: int, nrec: int, k: int) -> int:
        b = ctypes.c_size_t(0)
        _check(lib().fd_gradient_workspace_size(self.ptr, nsrc, nrec, k, ctypes.byref(b)))
        return b.value

    def linear_index(self, pos) -> np.ndarray:
        pos = np.atleast_2d(np.asarray(pos, np.int64))
        if self.dim == 2:
            return (pos[:, 0] * self.shape[1] + pos[:, 1]).astype(np.int64)
        return ((pos[:, 0] * self.shape[1] + pos[:, 1]) * self.shape[2] + pos[:, 2]).astype(np.int64)


def workspace(nbytes: int, device="cuda"):
    """A 256-byte aligned device workspace (torch allocation)."""
    torch = _torch()
    return torch.empty(max(int(nbytes), 1), dtype=torch.uint8, device=device)


def fd_forward(plan: Plan, model, src_idx: np.ndarray, wavelet, rec_idx: np.ndarray, traces,
               ws, state_in=None, state_out=None, model_kind: int = FD_MODEL_VELOCITY,
               stream=None):
    """Enqueue the forward run (all tensors on the device, indices on the host)."""
    src_idx = np.ascontiguousarray(src_idx, np.int64)
    rec_idx = np.ascontiguousarray(rec_idx, np.int64)
    _check(lib().fd_forward(plan.ptr, model_kind, _addr(model), len(src_idx),
                            src_idx.ctypes.data if len(src_idx) else None, _addr(wavelet),
                            len(rec_idx), rec_idx.ctypes.data if len(rec_idx) else None,
                            _addr(traces), _addr(state_in), _addr(state_out), _addr(ws),
                            ws.numel(), _stream_ptr(stream)))


def fd_forward_noalloc(plan: Plan, model, src_idx: np.ndarray, wavelet, rec_idx: np.ndarray, traces,
                       state_in=None, state_out=None, model_kind: int = FD_MODEL_VELOCITY,
                       stream=None):
    """fd_forward for callers that cannot allocate device memory: the library
    uses its own 32 MiB static device scratch (see include/fdwave.h); larger
    problems raise FdError(FD_ERR_NOMEM).  Calls must not overlap on the GPU."""
    src_idx = np.ascontiguousarray(src_idx, np.int64)
    rec_idx = np.ascontiguousarray(rec_idx, np.int64)
    _check(lib().fd_forward_noalloc(plan.ptr, model_kind, _addr(model), len(src_idx),
                                    src_idx.ctypes.data if len(src_idx) else None, _addr(wavelet),
                                    len(rec_idx), rec_idx.ctypes.data if len(rec_idx) else None,
                                    _addr(traces), _addr(state_in), _addr(state_out),
                                    _stream_ptr(stream)))


def fd_status_read(plan: Plan, ws, stream=None) -> int:
    return lib().fd_status_read(plan.ptr, _addr(ws), _stream_ptr(stream))


def fd_status_read_noalloc(plan: Plan, stream=None) -> int:
    """Device status of the last fd_forward_noalloc call on the current device."""
    return lib().fd_status_read_noalloc(plan.ptr, _stream_ptr(stream))


def check_status(plan: Plan, ws, what: str = "device run", stream=None) -> None:
    """Raise FdError when the device status word of the last call that used
    `ws` reports a condition (time-out, vmax exceeded, unbounded growth)."""
    rc = fd_status_read(plan, ws, stream)
    if rc != FD_OK:
        raise FdError(rc, "%s: %s" % (what, last_error()))


def fd_error_norms(num, ref, scale1: float = 1.0, scale2: float = 1.0, out=None, stream=None):
    """(scale1 sum|num - ref|, scale2 sqrt(sum (num - ref)^2), max|num - ref|) as a
    float64 device tensor [3] (Section 2.4); num and ref are float32 device
    tensors of the same size."""
    import torch
    assert num.dtype == torch.float32 and ref.dtype == torch.float32 and num.numel() == ref.numel()
    out = torch.empty(3, dtype=torch.float64, device=num.device) if out is None else out
    _check(lib().fd_error_norms(_addr(num), _addr(ref), num.numel(), scale1, scale2, _addr(out),
                                _stream_ptr(stream)))
    return out


def fd_dft_gamma(num, ref, nfreq: int = 0, with_gamma: bool = True, stream=None):
    """DFT dispersion metric of Appendix A for traces num, ref [nt, nrec]
    (float32 device tensors).  Returns (gamma [nrec, nfreq] float32 or None,
    trace norms [nrec] float64, (average, maximum) float64 [2], and the two
    spectra [nrec, nfreq, 2] float64); nfreq defaults to nt // 2 + 1."""
    import torch
    nt, nrec = num.shape
    assert ref.shape == num.shape and num.dtype == torch.float32 and ref.dtype == torch.float32
    nfreq = nfreq or nt // 2 + 1
    dev = num.device
    sn = torch.empty((nrec, nfreq, 2), dtype=torch.float64, device=dev)
    sr = torch.empty_like(sn)
    g = torch.empty((nrec, nfreq), dtype=torch.float32, device=dev) if with_gamma else None
    norms = torch.empty(nrec, dtype=torch.float64, device=dev)
    agg = torch.empty(2, dtype=torch.float64, device=dev)
    _check(lib().fd_dft_gamma(_addr(num), _addr(ref), nt, nrec, nfreq, _addr(sn), _addr(sr),
                              _addr(g) if g is not None else None, _addr(norms), _addr(agg),
                              _stream_ptr(stream)))
    return g, norms, agg, (sn, sr)


def fd_cwt_gamma(num, ref, nscale: int = 0, omega0: float = 6.0, with_gamma: bool = True,
                 stream=None):
    """Wavelet (CWT) dispersion metric of Appendix A for traces num, ref
    [nt, nrec] (float32 device tensors).  Returns (gamma [nrec, nscale, nt]
    float32 or None, trace norms [nrec] float64, (average, maximum) float64
    [2], largest |S^num| per trace [nrec] float64, and the two transforms
    [nrec, nscale, nt, 2] float64); nscale defaults to nt // 2 + 1."""
    import torch
    nt, nrec = num.shape
    assert ref.shape == num.shape and num.dtype == torch.float32 and ref.dtype == torch.float32
    nscale = nscale or nt // 2 + 1
    dev = num.device
    spn = torch.empty((nrec, nt // 2 + 1, 2), dtype=torch.float64, device=dev)
    spr = torch.empty_like(spn)
    sn = torch.empty((nrec, nscale, nt, 2), dtype=torch.float64, device=dev)
    sr = torch.empty_like(sn)
    g = torch.empty((nrec, nscale, nt), dtype=torch.float32, device=dev) if with_gamma else None
    amax = torch.empty(nrec, dtype=torch.float64, device=dev)
    norms = torch.empty(nrec, dtype=torch.float64, device=dev)
    agg = torch.empty(2, dtype=torch.float64, device=dev)
    _check(lib().fd_cwt_gamma(_addr(num), _addr(ref), nt, nrec, nscale, omega0, _addr(spn),
                              _addr(spr), _addr(sn), _addr(sr),
                              _addr(g) if g is not None else None, _addr(amax), _addr(norms),
                              _addr(agg), _stream_ptr(stream)))
    return g, norms, agg, amax, (sn, sr)


def fd_adjoint_gradient(plan: Plan, model, src_idx, wavelet, rec_idx, resid, k: int, grad, ws,
                        traces=None, wavelet_grad=None, model_kind: int = FD_MODEL_VELOCITY,
                        stream=None):
    src_idx = np.ascontiguousarray(src_idx, np.int64)
    rec_idx = np.ascontiguousarray(rec_idx, np.int64)
    _check(lib().fd_adjoint_gradient(plan.ptr, model_kind, _addr(model), len(src_idx),
                                     src_idx.ctypes.data if len(src_idx) else None,
                                     _addr(wavelet), len(rec_idx),
                                     rec_idx.ctypes.data if len(rec_idx) else None, _addr(resid),
                                     k, _addr(grad), _addr(traces), _addr(wavelet_grad),
                                     _addr(ws), ws.numel(), _stream_ptr(stream)))


def fd_gradient_forward(plan: Plan, model, src_idx, wavelet, rec_idx, traces, ws,
                        model_kind: int = FD_MODEL_VELOCITY, stream=None):
    """Forward sweep of the gradient keeping every step's D in ws (sized by
    plan.gradient_workspace_size(nsrc, nrec, plan.nt))."""
    src_idx = np.ascontiguousarray(src_idx, np.int64)
    rec_idx = np.ascontiguousarray(rec_idx, np.int64)
    _check(lib().fd_gradient_forward(plan.ptr, model_kind, _addr(model), len(src_idx),
                                     src_idx.ctypes.data if len(src_idx) else None,
                                     _addr(wavelet), len(rec_idx),
                                     rec_idx.ctypes.data if len(rec_idx) else None, _addr(traces),
                                     _addr(ws), ws.numel(), _stream_ptr(stream)))


def fd_gradient_adjoint(plan: Plan, src_idx, rec_idx, resid, grad, ws, wavelet_grad=None,
                        stream=None):
    """Adjoint sweep after fd_gradient_forward on the same plan and ws."""
    src_idx = np.ascontiguousarray(src_idx, np.int64)
    rec_idx = np.ascontiguousarray(rec_idx, np.int64)
    _check(lib().fd_gradient_adjoint(plan.ptr, len(src_idx),
                                     src_idx.ctypes.data if len(src_idx) else None, len(rec_idx),
                                     rec_idx.ctypes.data if len(rec_idx) else None, _addr(resid),
                                     _addr(grad), _addr(wavelet_grad), _addr(ws), ws.numel(),
                                     _stream_ptr(stream)))


def fd_forward_batched(shots: Sequence[dict], ws, stream=None):
    """shots: dicts with plan, model, src_idx, wavelet, rec_idx, traces
    (and optional model_kind)."""
    arr = (fd_shot * len(shots))()
    keep = []
    for i, s in enumerate(shots):
        si = np.ascontiguousarray(s["src_idx"], np.int64)
        ri = np.ascontiguousarray(s["rec_idx"], np.int64)
        keep += [si, ri]
        arr[i] = fd_shot(s["plan"].ptr.value, s.get("model_kind", FD_MODEL_VELOCITY), len(si),
                         len(ri), 0, _addr(s["model"]), si.ctypes.data, _addr(s["wavelet"]),
                         ri.ctypes.data, _addr(s["traces"]))
    _check(lib().fd_forward_batched(len(shots), arr, _addr(ws), ws.numel(), _stream_ptr(stream)))


def _fwd_shots(shots: Sequence[dict]):
    arr = (fd_shot * len(shots))()
    keep = []
    for i, s in enumerate(shots):
        si = np.ascontiguousarray(s["src_idx"], np.int64)
        ri = np.ascontiguousarray(s["rec_idx"], np.int64)
        keep += [si, ri]
        arr[i] = fd_shot(s["plan"].ptr.value, s.get("model_kind", FD_MODEL_VELOCITY), len(si),
                         len(ri), 0, _addr(s["model"]), si.ctypes.data, _addr(s["wavelet"]),
                         ri.ctypes.data, _addr(s["traces"]))
    return arr, keep


def fd_forward_batched_autotune(shots: Sequence[dict], ws, stream=None):
    """Time the batched kernel's tile shapes on this batch and keep the fastest."""
    arr, keep = _fwd_shots(shots)
    _check(lib().fd_forward_batched_autotune(len(shots), arr, _addr(ws), ws.numel(),
                                             _stream_ptr(stream)))


def fd_forward_batched_set_variant(shots: Sequence[dict], rows: int):
    """Choose the batched kernel's rows per thread (2 or 4) for this batch."""
    arr, keep = _fwd_shots(shots)
    _check(lib().fd_forward_batched_set_variant(len(shots), arr, rows))


def batched_workspace_size(shots: Sequence[dict]) -> int:
    arr = (fd_shot * len(shots))()
    for i, s in enumerate(shots):
        arr[i] = fd_shot(s["plan"].ptr.value, 0, len(s["src_idx"]), len(s["rec_idx"]), 0,
                         None, None, None, None, None)
    b = ctypes.c_size_t(0)
    _check(lib().fd_forward_batched_workspace_size(len(shots), arr, ctypes.byref(b)))
    return b.value


def _grad_shots(shots: Sequence[dict]):
    arr = (fd_grad_shot * len(shots))()
    keep = []
    for i, s in enumerate(shots):
        si = np.ascontiguousarray(s.get("src_idx", np.zeros(0)), np.int64)
        ri = np.ascontiguousarray(s.get("rec_idx", np.zeros(0)), np.int64)
        keep += [si, ri]
        arr[i] = fd_grad_shot(s["plan"].ptr.value, s.get("model_kind", FD_MODEL_VELOCITY), len(si),
                              len(ri), 0, _addr(s.get("model")), si.ctypes.data if len(si) else None,
                              _addr(s.get("wavelet")), ri.ctypes.data if len(ri) else None,
                              _addr(s.get("resid")), _addr(s.get("grad")), _addr(s.get("traces")))
    return arr, keep


def batched_gradient_workspace_size(shots: Sequence[dict], k: int) -> int:
    arr, _ = _grad_shots(shots)
    b = ctypes.c_size_t(0)
    _check(lib().fd_adjoint_gradient_batched_workspace_size(len(shots), arr, k, ctypes.byref(b)))
    return b.value


def fd_adjoint_gradient_batched(shots: Sequence[dict], k: int, ws, stream=None):
    """shots: dicts with plan, model, src_idx, wavelet, rec_idx, resid, grad
    (and optional traces, model_kind); each shot's gradient is written to its
    grad tensor."""
    arr, keep = _grad_shots(shots)
    _check(lib().fd_adjoint_gradient_batched(len(shots), arr, k, _addr(ws), ws.numel(),
                                             _stream_ptr(stream)))


# ----------------------------------------------------------------------------
# autograd: m = 1/v^2 -> traces, backward by the discrete adjoint
# ----------------------------------------------------------------------------

def _make_traces_fn():
    torch = _torch()

    class AcousticTraces(torch.autograd.Function):
        """traces = F(m); grad_m = F'(m)^T grad_traces by the discrete adjoint.
        ``k = None``: when the device has room for every step's D, the forward
        keeps them (fd_gradient_forward) and the backward runs only the
        adjoint sweep (fd_gradient_adjoint); else the backward calls
        fd_adjoint_gradient with checkpoints every 20 steps.  An integer ``k``
        always takes the second path with that interval.  The gradient is
        bitwise the same either way."""

        @staticmethod
        def forward(ctx, m, plan, src_idx, wavelet, rec_idx, k):
            nt = plan.nt
            traces = torch.empty((nt, len(rec_idx)), dtype=torch.float32, device=m.device)
            ctx.store = None
            if k is None and ctx.needs_input_grad[0]:
                need = plan.gradient_workspace_size(len(src_idx), len(rec_idx), nt)
                if need + (4 << 30) < torch.cuda.mem_get_info(m.device)[0]:
                    ws = workspace(need, m.device)
                    fd_gradient_forward(plan, m, src_idx, wavelet, rec_idx, traces, ws,
                                        model_kind=FD_MODEL_SLOWNESS2)
                    check_status(plan, ws, "acoustic_traces forward")
                    ctx.store = ws
            if ctx.store is None:
                ws = workspace(plan.forward_workspace_size(len(src_idx), len(rec_idx)), m.device)
                fd_forward(plan, m, src_idx, wavelet, rec_idx, traces, ws,
                           model_kind=FD_MODEL_SLOWNESS2)
                check_status(plan, ws, "acoustic_traces forward")
            ctx.save_for_backward(m, wavelet)
            ctx.plan, ctx.src_idx, ctx.rec_idx, ctx.k = plan, src_idx, rec_idx, k
            return traces

        @staticmethod
        def backward(ctx, grad_traces):
            m, wavelet = ctx.saved_tensors
            plan = ctx.plan
            grad = torch.empty_like(m)
            if ctx.store is not None:
                ws, ctx.store = ctx.store, None
                fd_gradient_adjoint(plan, ctx.src_idx, ctx.rec_idx, grad_traces.contiguous().float(),
                                    grad, ws)
            else:
                k = 20 if ctx.k is None else ctx.k
                ws = workspace(plan.gradient_workspace_size(len(ctx.src_idx), len(ctx.rec_idx), k),
                               m.device)
                fd_adjoint_gradient(plan, m, ctx.src_idx, wavelet, ctx.rec_idx,
                                    grad_traces.contiguous().float(), k, grad, ws,
                                    model_kind=FD_MODEL_SLOWNESS2)
            check_status(plan, ws, "acoustic_traces backward")
            return grad, None, None, None, None, None

    return AcousticTraces


_traces_fn = None


def acoustic_traces(m, plan: Plan, src_idx, wavelet, rec_idx, k=None):
    """Differentiable traces(m) for m = 1/v^2 on the physical grid.  ``k`` is
    the backward pass's checkpoint interval; None keeps every step's D in
    device memory from the forward when it fits (the backward then runs only
    the adjoint sweep), else checkpoints every 20."""
    global _traces_fn
    if _traces_fn is None:
        _traces_fn = _make_traces_fn()
    return _traces_fn.apply(m, plan, np.asarray(src_idx, np.int64), wavelet,
                            np.asarray(rec_idx, np.int64), k)
