"""Host checks (no GPU) of the arithmetic identities the CUDA kernels rely on,
each restated here in Python and compared with an independent reference:

* the FFT stages divide j by L with a multiply-high by floor((2^32 - 1) / L) + 1
  (exact for j, L < 2^16; plan_fft keeps every transform below 2^16 points);
* the projection's paired Lagrange weights: nodes o and 1 - o paired as
  s + o (1 - o) with s = eps (eps - 1), the 1 / prod (j - m) absorbed into
  per-pair scalings, give the centred Lagrange weights (oracle);
* the radix-5 and radix-7 butterflies in symmetric form give the DFT.
"""
import math

import numpy as np
import pytest

from oracle import response


def _div_magic(j, L):
    if L == 1:
        return j
    mag = (0xFFFFFFFF // L) + 1
    return (j * mag) >> 32


def test_multiply_high_division_is_exact_below_2_16():
    rng = np.random.default_rng(0)
    Ls = list(range(1, 1100)) + [1080, 960, 4096, 2401, 3375, 65535] + \
        rng.integers(1, 1 << 16, 400).tolist()
    for L in Ls:
        js = list(range(0, 300)) + rng.integers(0, 1 << 16, 300).tolist() + [(1 << 16) - 1]
        for j in js:
            assert _div_magic(j, L) == j // L, (j, L)


def _paired_weights(eps, K):
    """The paired form in float64 (the kernel evaluates it in float32)."""
    NP, H = K // 2, (K - 2) // 2
    cinv = [1.0 / math.prod(float(j - m) for m in range(K) if m != j) for j in range(K)]
    la = [math.log(abs(cinv[k])) for k in range(NP)]
    sg = [math.copysign(1.0, cinv[k]) for k in range(NP)]
    lL = sum(la) / (NP - 1)
    lam = [sg[k] * math.exp(lL - la[k]) for k in range(NP)]
    s = eps * (eps - 1.0)
    P = [lam[k] * (s + (k - H) * (1.0 - (k - H))) for k in range(NP)]
    w = np.zeros(K)
    for k in range(NP):
        R = math.prod(P[q] for q in range(NP) if q != k)
        w[k] = (eps + (k - H - 1)) * R
        w[K - 1 - k] = ((k - H) - eps) * R
    return w


@pytest.mark.parametrize("K", [8, 16, 32])
def test_paired_lagrange_weights_equal_the_lagrange_weights(K):
    for eps in np.linspace(0.0, 0.999, 37):
        want = response.lagrange_weights(eps, K - 1)
        got = _paired_weights(float(eps), K)
        assert np.max(np.abs(got - want)) <= 1e-10 * max(1.0, np.max(np.abs(want))), (K, eps)


def _dft_sym(a, R):
    """The symmetric butterfly: t_q = a_q + a_{R-q}, u_q = a_q - a_{R-q};
    X_s = a_0 + sum t_q cos(2 pi q s / R) - i sum u_q sin(2 pi q s / R), X_{R-s}
    with +i."""
    M = (R - 1) // 2
    t = [a[q] + a[R - q] for q in range(1, M + 1)]
    u = [a[q] - a[R - q] for q in range(1, M + 1)]
    X = np.zeros(R, complex)
    X[0] = a[0] + sum(t)
    for s in range(1, M + 1):
        b = a[0] + sum(t[q - 1] * math.cos(2 * math.pi * q * s / R) for q in range(1, M + 1))
        d = sum(u[q - 1] * math.sin(2 * math.pi * q * s / R) for q in range(1, M + 1))
        X[s] = b - 1j * d
        X[R - s] = b + 1j * d
    return X


@pytest.mark.parametrize("R", [3, 5, 7])
def test_symmetric_odd_radix_butterflies_are_the_dft(R):
    rng = np.random.default_rng(R)
    for _ in range(20):
        a = rng.normal(size=R) + 1j * rng.normal(size=R)
        assert np.max(np.abs(_dft_sym(a, R) - np.fft.fft(a))) <= 1e-13
