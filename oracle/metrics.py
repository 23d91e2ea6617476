"""FP64 evaluation metrics of the paper (test infrastructure only; the CUDA
path never imports this module).

* Classical error norms of a numerical against a reference data object
  (Section 2.4, Eqs. snapnorm1, snapnorm2, snapnormmax): sum |d| and
  sqrt(sum d^2) with the paper's scale factors, and max |d|.
* The DFT-based dispersion metric of Appendix A: per trace the DFT
  coefficients A_k (Eq. dft), their amplitude and phase (Eqs. ampldft,
  phasedft; the amplitude read as sqrt(Re^2 + Im^2)), the phase difference
  numerical minus reference brought back into [-pi, pi] by one 2 pi shift
  (Eqs. phasesdifdft, phasesdifdftajusted), gamma_k = (phase difference / pi)
  (|A_k^num| / max_k |A_k^num|) (Eq. gammadft), the trace's 2-norm
  sqrt(mean_k gamma_k^2) over the n_freq frequencies computed (Eq.
  norm2gammastdft, whose printed bounds are garbled), and the average and
  maximum of those norms over the receivers (Eqs. norm2gammarecdftavg,
  norm2gammarecdftmax).  A trace whose numerical spectrum is zero has
  gamma = 0 (the ratio is undefined).
"""
from __future__ import annotations

import numpy as np


def error_norms(num, ref, scale1: float, scale2: float):
    """(scale1 * sum|num - ref|, scale2 * sqrt(sum (num - ref)^2), max|num - ref|)."""
    d = np.asarray(num, np.float64) - np.asarray(ref, np.float64)
    return scale1 * np.abs(d).sum(), scale2 * np.sqrt((d * d).sum()), (np.abs(d).max() if d.size else 0.0)


def snapshot_scales(h: float):
    """Scale factors of Eqs. snapnorm1 and snapnorm2 for a 2D snapshot: 1/h^2, 1/h."""
    return 1.0 / (h * h), 1.0 / h


def dft(traces, nfreq: int):
    """A[k, p] = sum_n u[n, p] exp(-2 pi i k n / nt), k < nfreq (Eq. dft)."""
    u = np.asarray(traces, np.float64)
    return np.fft.fft(u, axis=0)[:nfreq]


def dft_gamma(num, ref, nfreq: int | None = None):
    """gamma [nrec, nfreq], per-trace norms [nrec], and their average and maximum
    for traces num, ref of shape [nt, nrec]."""
    num = np.asarray(num, np.float64)
    ref = np.asarray(ref, np.float64)
    nt = num.shape[0]
    if nfreq is None:
        nfreq = nt // 2 + 1
    An, Ar = dft(num, nfreq), dft(ref, nfreq)
    d = np.angle(An) - np.angle(Ar)
    d = np.where(d > np.pi, d - 2 * np.pi, d)
    d = np.where(d < -np.pi, d + 2 * np.pi, d)
    amp = np.abs(An)
    amax = amp.max(axis=0)
    safe = np.where(amax > 0, amax, 1.0)
    gamma = np.where(amax > 0, (d / np.pi) * (amp / safe), 0.0)
    norms = np.sqrt((gamma * gamma).mean(axis=0))
    return gamma.T, norms, norms.mean(), norms.max()
