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
* The wavelet (CWT) dispersion metric of Appendix A, read as the
  DFT-based Morlet transform of Torrence and Compo that the appendix cites
  (its printed form is garbled: Eq. cwt applies an inverse DFT to a sum that
  already is one, and the IDFT of Eq. idft carries the wrong sign and a
  1/n_freq factor).  The reading used:
  - omega_k = 2 pi k / (nt tau) for 1 <= k <= nt/2 (Eq. omegak); the
    Heaviside factor of Eq. cwt3 removes k = 0 and every k > nt/2, so the
    printed sign of the negative branch never matters;
  - S_{n,k} = (1/nt) sum_k' A_k' Psi^*(s_k omega_k') exp(+2 pi i k' n / nt)
    (Eqs. cwt1 and cwt taken as one inverse DFT), with
    Psi^*(s omega) = (2 pi s / tau)^(1/2) pi^(-1/4) H(omega)
    exp(-(s omega - omega0)^2 / 2) (Eqs. cwt2, cwt3), omega0 = 6 by default;
  - the k-th scale is the one whose Fourier period is line k's period:
    s_k = (omega0 + sqrt(2 + omega0^2)) / (2 omega_k) for k >= 1 (the scale
    at which the wavelet power of a pure tone of line k peaks); the k = 0
    line has no finite scale and S_{n,0} = 0.  tau cancels: s_k omega_k' =
    c k'/k and 2 pi s_k / tau = c nt / k, c = (omega0 + sqrt(2 + omega0^2))/2;
  - amplitude |S| (Eq. amplcwt read as sqrt(Re^2 + Im^2)), phase atan2 (Eq.
    phasecwt), the wrapped phase difference (Eqs. phasesdifcwt,
    phasesdifcwtajusted), gamma_{n,k} of Eq. gammacwt with the largest |S^num|
    over all (n, k) of the trace (Eq. amplmaxcwt), the trace norm
    sqrt(mean over n and k of gamma^2) (Eq. norm2gammastcwt), and its average
    and maximum over the receivers (Eqs. norm2gammareccwtavg,
    norm2gammareccwtmax).
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


def morlet_scale_factor(omega0: float = 6.0) -> float:
    """c = (omega0 + sqrt(2 + omega0^2)) / 2, so that s_k omega_k = c."""
    return 0.5 * (omega0 + np.sqrt(2.0 + omega0 * omega0))


def cwt(traces, nscale: int, omega0: float = 6.0):
    """S [nrec, nscale, nt] complex: the Morlet CWT of each trace of
    traces [nt, nrec] at the scales matched to DFT lines k = 0 .. nscale-1
    (S[:, 0, :] = 0), following Eqs. dft, omegak, cwt2, cwt3, cwt1, cwt."""
    u = np.asarray(traces, np.float64)
    nt, nrec = u.shape
    A = np.fft.fft(u, axis=0)                                 # Eq. dft, all lines
    kp = np.arange(nt)
    positive = (kp >= 1) & (2 * kp <= nt)                     # H(omega_k') = 1
    c = morlet_scale_factor(omega0)
    S = np.zeros((nrec, nscale, nt), np.complex128)
    for k in range(1, nscale):
        s_omega = c * kp / k                                  # s_k omega_k'
        psi = np.sqrt(c * nt / k) * np.pi ** -0.25 * np.exp(-0.5 * (s_omega - omega0) ** 2)
        psi = np.where(positive, psi, 0.0)
        # (1/nt) sum_k' (A_k' psi_k') exp(+2 pi i k' n / nt)
        S[:, k, :] = np.fft.ifft(A * psi[:, None], axis=0).T
    return S


def cwt_gamma(num, ref, nscale: int | None = None, omega0: float = 6.0):
    """gamma^W [nrec, nscale, nt], the per-trace norms [nrec], their average and
    maximum, and the largest |S^num| of each trace, for traces num, ref [nt, nrec]."""
    num = np.asarray(num, np.float64)
    ref = np.asarray(ref, np.float64)
    nt = num.shape[0]
    if nscale is None:
        nscale = nt // 2 + 1
    Sn, Sr = cwt(num, nscale, omega0), cwt(ref, nscale, omega0)
    d = np.angle(Sn) - np.angle(Sr)
    d = np.where(d > np.pi, d - 2 * np.pi, d)
    d = np.where(d < -np.pi, d + 2 * np.pi, d)
    amp = np.abs(Sn)
    amax = amp.max(axis=(1, 2))
    safe = np.where(amax > 0, amax, 1.0)[:, None, None]
    gamma = np.where(amax[:, None, None] > 0, (d / np.pi) * (amp / safe), 0.0)
    norms = np.sqrt((gamma * gamma).mean(axis=(1, 2)))
    return gamma, norms, norms.mean(), norms.max(), amax
