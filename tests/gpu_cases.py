"""Shared drivers for the GPU parity tests: run the CUDA path through the C ABI
and the FP64 oracle on the same seeded inputs, and compare."""
import numpy as np

import paper_2606_04882_gb300 as F
from oracle import physics as P
from oracle import stencil as S
from oracle import wave as W


def rel_l2(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def per_receiver_errors(tr, otr, floor=1e-3):
    """Relative L2 error of each receiver's trace [nt, nrec], with the
    denominator floored at `floor` times the largest trace norm (receivers the
    wave barely reaches carry the FP32 noise of the field around them, not of
    their own small signal).  One wrong receiver among many shows here even
    when the global norm hides it."""
    tr = np.asarray(tr, np.float64)
    otr = np.asarray(otr, np.float64)
    e = np.linalg.norm(tr - otr, axis=0)
    o = np.linalg.norm(otr, axis=0)
    return e / np.maximum(o, floor * (o.max() if o.size else 1.0))


def taylor_dt(dim, M, h, vmax, frac=0.5):
    """dt = frac * C_max(Taylor cross of radius M) * h / vmax (oracle bound)."""
    pw = S.expand(dim, "cross", M, 0, S.weights(dim, "cross", M))
    return frac * S.cfl_limit(pw, dim) * h / vmax


class Case:
    def __init__(self, vel, h, nt, nb, vmax, shape="cross", M=4, N=0, scheme="spatte",
                 src=None, rec=None, f0=15.0, dt=None, frac=0.5):
        self.vel = np.ascontiguousarray(vel, np.float32)
        self.dim = self.vel.ndim
        self.h, self.nt, self.nb, self.vmax = h, nt, nb, vmax
        self.shape, self.M, self.N, self.scheme = shape, M, N, scheme
        self.dt = dt if dt is not None else taylor_dt(self.dim, M, h, vmax, frac)
        self.C = vmax * self.dt / h
        self.src = np.atleast_2d(np.asarray(src if src is not None else [[s // 2 for s in self.vel.shape]], np.int64))
        self.rec = np.atleast_2d(np.asarray(rec, np.int64)) if rec is not None else np.zeros((0, self.dim), np.int64)
        self.f0 = f0

    def desc(self):
        return F.stencil_desc(self.dim, self.shape, self.M, self.N, self.scheme, courant=self.C)

    def plan(self, nt=None):
        return F.Plan(self.vel.shape, self.h, self.dt, self.nt if nt is None else nt, self.nb,
                      self.vmax, self.desc())

    def wavelet32(self, nt=None):
        nt = self.nt if nt is None else nt
        w = F.fd_ricker(self.f0, self.dt, nt)
        return np.ascontiguousarray(np.repeat(w[:, None], len(self.src), axis=1))

    def gpu_forward(self, nt=None, state_in=None, t0=0):
        import torch
        nt = self.nt if nt is None else nt
        plan = self.plan(nt)
        dev = torch.device("cuda")
        vel = torch.from_numpy(self.vel).to(dev)
        wav = torch.from_numpy(self.wavelet32(self.nt)[t0:t0 + nt].copy()).to(dev)
        nrec = len(self.rec)
        traces = torch.zeros((nt, max(nrec, 1)), device=dev)
        ws = F.workspace(plan.forward_workspace_size(len(self.src), nrec))
        pshape = plan.padded_shape
        sin = None if state_in is None else torch.from_numpy(np.ascontiguousarray(state_in, np.float32)).to(dev)
        sout = torch.zeros((2,) + tuple(pshape), device=dev)
        F.fd_forward(plan, vel, plan.linear_index(self.src), wav,
                     plan.linear_index(self.rec) if nrec else np.zeros(0, np.int64),
                     traces if nrec else None, ws, state_in=sin, state_out=sout)
        rc = F.fd_status_read(plan, ws)
        torch.cuda.synchronize()
        return traces.cpu().numpy()[:, :nrec], sout.cpu().numpy(), rc

    def setup(self):
        return W.Setup(self.vel, self.h, self.dt, self.nb, self.vmax, self.dim, self.shape,
                       self.M, self.N, self.scheme)

    def oracle_forward(self, nt=None, state_in=None, t0=0, threads=None):
        nt = self.nt if nt is None else nt
        st = self.setup()
        wav = np.repeat(P.ricker(self.f0, self.nt, self.dt)[:, None], len(self.src), axis=1)[t0:t0 + nt]
        u0 = um1 = None
        if state_in is not None:
            u0, um1 = state_in[0].astype(np.float64), state_in[1].astype(np.float64)
        tr, u, up = W.forward(st, nt, self.src, wav, self.rec if len(self.rec) else None,
                              u0=u0, um1=um1, threads=threads)
        return tr, np.stack([u, up])
