"""Wigner rotation matrices and spin-weighted spherical harmonics, written from
their textbook definitions (used by the two-step twist-up of Sec. II.A).

Conventions (declared):
* Euler angles are z-y-z: R(alpha, beta, gamma) = R_z(alpha) R_y(beta) R_z(gamma).
* D^l_{m m'}(alpha, beta, gamma) = exp(-i m alpha) d^l_{m m'}(beta) exp(-i m' gamma),
  with Wigner's explicit sum for the small-d matrix; D is a representation,
  D(R1 R2) = D(R1) D(R2).
* sY_lm(theta, phi) from Goldberg's explicit sum with the (-1)^m prefactor,
  which gives -2Y_22 = sqrt(5/64pi)(1+cos theta)^2 exp(2 i phi).
"""
import math

import numpy as np


def _f(n):
    return math.factorial(n)


def small_d(l, mp, m, beta):
    """Wigner small-d d^l_{mp, m}(beta) (explicit finite sum)."""
    beta = np.asarray(beta, dtype=np.float64)
    c = np.cos(0.5 * beta)
    s = np.sin(0.5 * beta)
    pref = math.sqrt(_f(l + mp) * _f(l - mp) * _f(l + m) * _f(l - m))
    out = np.zeros_like(beta)
    for k in range(0, 2 * l + 1):
        a, b, cc, dd = l + m - k, k, mp - m + k, l - mp - k
        if min(a, b, cc, dd) < 0:
            continue
        coef = (-1.0) ** (mp - m + k) * pref / (_f(a) * _f(b) * _f(cc) * _f(dd))
        out = out + coef * c ** (2 * l + m - mp - 2 * k) * s ** (mp - m + 2 * k)
    return out


def wigner_D(l, mp, m, alpha, beta, gamma):
    """D^l_{mp, m}(alpha, beta, gamma) = e^{-i mp alpha} d^l_{mp m}(beta) e^{-i m gamma}."""
    return (np.exp(-1j * mp * np.asarray(alpha)) * small_d(l, mp, m, beta)
            * np.exp(-1j * m * np.asarray(gamma)))


def sYlm(s, l, m, theta, phi):
    """Spin-weighted spherical harmonic sY_lm(theta, phi) (Goldberg et al.)."""
    theta = np.asarray(theta, dtype=np.float64)
    phi = np.asarray(phi, dtype=np.float64)
    pref = (-1.0) ** m * math.sqrt(
        _f(l + m) * _f(l - m) * (2 * l + 1) / (4.0 * math.pi * _f(l + s) * _f(l - s)))
    sh = np.sin(0.5 * theta)
    ch = np.cos(0.5 * theta)
    acc = np.zeros(np.broadcast(theta, phi).shape, dtype=np.complex128)
    for r in range(0, l - s + 1):
        j = r + s - m
        if j < 0 or j > l + s:
            continue
        k = 2 * r + s - m                 # power of cot(theta/2)
        coef = math.comb(l - s, r) * math.comb(l + s, j) * (-1.0) ** (l - r - s)
        acc = acc + coef * sh ** (2 * l - k) * ch ** k
    return pref * acc * np.exp(1j * m * phi)
