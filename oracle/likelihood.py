"""Fourier transform, Sangria analytic PSD, matched-filter inner product and
log-likelihood (Sec. II.B: the inner product of the A, E, T channels and the
PSD equations).

Readings of the paper taken here:
* logL = -1/2 sum_c (h_c - d_c | h_c - d_c) (the complete definition given in
  the footnote; the displayed form has the opposite sign of the cross term).
* (a|b) = 4 df Re sum_{k: f_lo <= f_k <= f_hi} a_k conj(b_k) / S(f_k),
  a_k = dt sum_n a_n exp(-2 pi i k n / N), k = 0 .. N/2, df = 1/(N dt);
  rectangular window.
* PSD arm factor x = 2 pi f L / c; A_acc = 2.4e-15; TDI-2 PSDs = TDI-1.5
  PSDs times 4 sin^2(2x).
"""
import math

import numpy as np

from . import consts as K


def dft(a, dt):
    """One-sided DFT a_k = dt sum_n a_n e^{-2 pi i k n/N} (library FFT)."""
    return dt * np.fft.rfft(np.asarray(a, dtype=np.float64))


def dft_brute(a, dt):
    """The same sum evaluated term by term (O(N^2); test use on small N)."""
    a = np.asarray(a, dtype=np.float64)
    n = a.shape[0]
    k = np.arange(n // 2 + 1)[:, None]
    j = np.arange(n)[None, :]
    ang = -2.0 * math.pi * ((k * j) % n) / n
    return dt * np.sum(a[None, :] * (np.cos(ang) + 1j * np.sin(ang)), axis=1)


def freqs(n, dt):
    return np.arange(n // 2 + 1) / (n * dt)


def psd_components(f):
    """S_acc and S_op in fractional-frequency units."""
    f = np.asarray(f, dtype=np.float64)
    w = 2.0 * math.pi * f
    s_acc = (K.A_ACC ** 2 * (1.0 + (4e-4 / f) ** 2) * (1.0 + (f / 8e-3) ** 4)
             * w ** -4 * (w / K.C_SI) ** 2)
    s_op = K.A_OMS ** 2 * (1.0 + (2e-3 / f) ** 4) * (w / K.C_SI) ** 2
    return s_acc, s_op


def psd_aet(f, gen):
    """(S_AE, S_T) at frequencies f for TDI generation 15 or 20."""
    s_acc, s_op = psd_components(f)
    x = 2.0 * math.pi * np.asarray(f) * K.ARM_S
    sx2 = np.sin(x) ** 2
    s_ae = 8.0 * sx2 * (2.0 * s_acc * (3.0 + 2.0 * np.cos(x) + np.cos(2.0 * x))
                        + s_op * (2.0 + np.cos(x)))
    s_t = (16.0 * s_op * (1.0 - np.cos(x)) * sx2
           + 128.0 * s_acc * sx2 * np.sin(0.5 * x) ** 4)
    if gen == 20:
        g = 4.0 * np.sin(2.0 * x) ** 2
        s_ae, s_t = s_ae * g, s_t * g
    return s_ae, s_t


def band(n, dt, f_lo, f_hi):
    f = freqs(n, dt)
    return (f >= f_lo) & (f <= f_hi)


def inner(a_f, b_f, s, df, mask):
    """(a|b) = 4 df Re sum_band a conj(b) / S."""
    return 4.0 * df * float(np.sum((a_f[mask] * np.conj(b_f[mask])).real / s[mask]))


def loglike(h_aet, d_aet, dt, f_lo, f_hi, gen, channel_mask=7):
    """logL = -1/2 sum_{c in mask} (h_c - d_c | h_c - d_c)."""
    n = np.asarray(h_aet[0]).shape[0]
    f = freqs(n, dt)
    mask = band(n, dt, f_lo, f_hi)
    with np.errstate(divide="ignore", invalid="ignore"):
        s_ae, s_t = psd_aet(np.where(f > 0, f, 1.0), gen)
    df = 1.0 / (n * dt)
    total = 0.0
    for c in range(3):
        if not (channel_mask >> c) & 1:
            continue
        r = dft(np.asarray(h_aet[c]) - 0.0, dt) - dft(np.asarray(d_aet[c]), dt)
        total += inner(r, r, s_t if c == 2 else s_ae, df, mask)
    return -0.5 * total
