"""Coloured Gaussian noise for the A, E, T channels: data = signal + noise
rather than the zero-noise injections of Sec. II.C (the paper's stated next
step, Sec. IV).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Definition: for each band bin k (f_lo <= f_k <= f_hi) the DFT of the noise is
    N_k = sqrt(n S_c(f_k) / (2 dt)) (x_k + i y_k) / sqrt(2),
x_k, y_k standard normal (passed in), zero outside the band, so that
E|N_k|^2 = n S_c(f_k) / (2 dt) -- the one-sided PSD S_c -- and the noise is the
real inverse DFT n_j = (1/n) sum_k N_k e^{2 pi i j k / n} (Hermitian
extension).  With the inner product of the likelihood, (n|n) = sum over band
bins of x_k^2 + y_k^2 exactly (expectation 2 per bin).
"""
import numpy as np

from . import likelihood


def noise_aet(z, n, dt, f_lo, f_hi, gen):
    """z: standard normals [3][2][n//2 + 1] -> noise [3][n] (channels A, E, T)."""
    z = np.asarray(z, dtype=np.float64)
    f = likelihood.freqs(n, dt)
    mask = likelihood.band(n, dt, f_lo, f_hi)
    with np.errstate(divide="ignore", invalid="ignore"):
        s_ae, s_t = likelihood.psd_aet(np.where(f > 0, f, 1.0), gen)
    out = np.zeros((3, n))
    for c in range(3):
        s = s_t if c == 2 else s_ae
        sig = np.sqrt(n * s / (2.0 * dt))
        spec = np.where(mask, sig * (z[c, 0] + 1j * z[c, 1]) / np.sqrt(2.0), 0.0)
        out[c] = np.fft.irfft(spec, n)
    return out
