"""Host checks (no GPU) of the arithmetic identities the CUDA kernels rely on,
each restated here in Python and compared with an independent reference:

* the FFT stages divide j by L with a multiply-high by floor((2^32 - 1) / L) + 1
  (exact for j, L < 2^16; plan_fft keeps every transform below 2^16 points);
* the projection's paired Lagrange weights: nodes o and 1 - o paired as
  s + o (1 - o) with s = eps (eps - 1), the 1 / prod (j - m) absorbed into
  per-pair scalings, give the centred Lagrange weights (oracle);
* the radix-5 and radix-7 butterflies in symmetric form give the DFT;
* the waveform kernels' single-sum twist-up (Eq. newtwistup): the unit
  quaternion of each Euler rotation, their Hamilton product
  conj(q(alpha, beta, gamma)) conj(q(rot0)) q(phi_ref, iota, 0), and
  sqrt((2l+1)/4pi) D^l_{m,2} as a sum of non-negative powers of
  Q_a = q0 + i q3, Q_b = q2 + i q1, equal the oracle's two-step twist-up.
"""
import math

import numpy as np
import pytest

from oracle import consts as K
from oracle import response, waveform


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


def _quat_euler(a, b, g):
    cb, sb = math.cos(0.5 * b), math.sin(0.5 * b)
    return np.array([cb * math.cos(0.5 * (a + g)), -sb * math.sin(0.5 * (a - g)),
                     sb * math.cos(0.5 * (a - g)), cb * math.sin(0.5 * (a + g))])


def _qmul(a, b):
    return np.array([a[0] * b[0] - a[1] * b[1] - a[2] * b[2] - a[3] * b[3],
                     a[0] * b[1] + a[1] * b[0] + a[2] * b[3] - a[3] * b[2],
                     a[0] * b[2] - a[1] * b[3] + a[2] * b[0] + a[3] * b[1],
                     a[0] * b[3] + a[1] * b[2] - a[2] * b[1] + a[3] * b[0]])


def _conj(q):
    return np.array([q[0], -q[1], -q[2], -q[3]])


def _ylm_from_quat(l, m, q):
    Qa, Qb = complex(q[0], q[3]), complex(q[2], q[1])
    acc = 0j
    for r in range(max(0, m - 2), min(l + m, l - 2) + 1):
        c = math.comb(l + m, r) * math.comb(l - m, l - 2 - r) * (-1.0) ** r
        acc += c * Qa ** (l + m - r) * Qa.conjugate() ** (l - 2 - r) * \
            Qb ** (2 - m + r) * Qb.conjugate() ** r
    f = math.factorial
    return acc * math.sqrt(f(l + 2) * f(l - 2) / (f(l + m) * f(l - m))) * \
        math.sqrt((2 * l + 1) / (4 * math.pi))


@pytest.mark.parametrize("tilt", [0.3, 1.6, 2.9])
def test_quaternion_single_sum_equals_the_oracle_twist_up(tilt):
    th = np.array([6.2e5, 1.9e5, 0.8, tilt, 1.1, 0.4, 0.9, 2.0, 5.0, 0.7, 2.3,
                   0.2, 4.0, 0.0, 0.9 * 10 * 86400.0])
    src = waveform.source(th, True)
    t = np.linspace(src["tm"] - 3e5, src["tm"] + 300.0, 24)
    al, be, ga, rot0 = waveform.euler_angles(src, t)
    hp, hx = waveform.plus_cross(th, t, 0.0, 31, True)
    want = hp - 1j * hx
    q03 = _qmul(_conj(_quat_euler(*rot0)), _quat_euler(src["phi_ref"], src["iota"], 0.0))
    got = np.zeros(t.size, complex)
    for (l, m) in K.MODES:
        h = waveform.mode(src, l, m, t, 0.0)
        for i in range(t.size):
            qT = _qmul(_conj(_quat_euler(al[i], be[i], ga[i])), q03)
            got[i] += h[i] * _ylm_from_quat(l, m, qT) + \
                (-1.0) ** l * np.conj(h[i]) * _ylm_from_quat(l, -m, qT)
    assert np.max(np.abs(got - want)) <= 1e-12 * np.max(np.abs(want))


def _difference_weights(eps, K):
    """C_m (m = -H .. H) of the summation-by-parts form used by the mixed TDI
    tile tables: y(c + eps) = y_c + sum_m C_m (y_{c+m+1} - y_{c+m})."""
    H = (K - 2) // 2
    w = response.lagrange_weights(eps, K - 1)
    C = np.zeros(K - 1)
    for mi in range(K - 1):
        m = mi - H
        for k in range(K):
            o = k - H
            if m >= 0 and o > m:
                C[mi] += w[k]
            if m < 0 and o <= m:
                C[mi] -= w[k]
    return C


def test_combined_pair_fir_equals_the_sum_of_its_terms():
    """The mixed TDI kernel's per-(channel, link) FIR: the difference weights of
    the pair's terms added at offsets bo - H - min(bo - H) into G, applied to dy
    from row s + min(bo - H), plus each term's centre sample, give the signed
    sum of the terms' Lagrange interpolations."""
    K, H = 32, 15
    rng = np.random.default_rng(4)
    t = np.arange(400)
    y = np.sin(0.05 * t) + 0.3 * np.cos(0.013 * t + 1.0) + 0.01 * rng.normal(size=t.size)
    dy = np.append(np.diff(y), 0.0)
    bos = [-2, -5, -9, -12]
    sgs = [1.0, -1.0, 1.0, -1.0]
    epss = rng.uniform(0.0, 1.0, 4)
    bmin = min(b - H for b in bos)
    ntap = max(b - H for b in bos) - bmin + K - 1
    G = np.zeros(ntap)
    for b, sg, e in zip(bos, sgs, epss):
        o = b - H - bmin
        G[o:o + K - 1] += sg * _difference_weights(e, K)
    for s in range(150, 250, 7):
        got = sum(sg * y[s + b] for b, sg in zip(bos, sgs))
        got += float(np.dot(G, dy[s + bmin:s + bmin + ntap]))
        want = 0.0
        for b, sg, e in zip(bos, sgs, epss):
            w = response.lagrange_weights(e, K - 1)
            c = s + b
            want += sg * float(np.dot(w, y[c - H:c - H + K]))
        assert abs(got - want) <= 1e-12, (s, got, want)


def _prime_stage(A, R, L, tw):
    """fft.cu's prime-radix stage: the stage twiddles in place, then the R-point
    DFT by conjugate pairs u_q = y_q + y_{R-q}, v_q = y_q - y_{R-q}."""
    m = A.size
    nb, stride = m // R, m // (L * R)
    y = A.copy()
    for i in range(m):
        q, j = divmod(i, nb)
        k = j % L
        if q > 0 and k > 0:
            y[i] *= tw[q * k * stride]
    B = np.zeros(m, dtype=np.complex128)
    h = (R - 1) // 2
    for j in range(nb):
        k = j % L
        base = (j - k) * R + k
        for s in range(h + 1):
            U = V = 0j
            for q in range(1, h + 1):
                a, b = y[j + q * nb], y[j + (R - q) * nb]
                w = tw[(q * s * nb) % m]
                U += w.real * (a + b)
                V += w.imag * (a - b)
            B[base + s * L] = y[j] + U + 1j * V
            if s > 0:
                B[base + (R - s) * L] = y[j] + U - 1j * V
    return B


def _stockham(x, radices):
    """The pass kernels' Stockham stages in numpy: stage (R, L) reads
    A[j + q nb], applies W_m^{q (k stride + s nb)} (k = j mod L: the stage
    twiddle times W_R^{q s}) and writes B[(j - k) R + k + s L]; a prime radix
    R >= 11 goes through _prime_stage."""
    m = x.size
    tw = np.exp(-2j * np.pi * np.arange(m) / m)
    A = x.astype(np.complex128)
    L = 1
    for R in radices:
        if R >= 11:
            A = _prime_stage(A, R, L, tw)
            L *= R
            continue
        nb, stride = m // R, m // (L * R)
        B = np.zeros(m, dtype=np.complex128)
        for j in range(nb):
            k = j % L
            base = (j - k) * R + k
            for s in range(R):
                e = k * stride + s * nb
                q = np.arange(R)
                B[base + s * L] = np.sum(A[j + q * nb] * tw[(q * e) % m])
        A = B
        L *= R
    return A


@pytest.mark.parametrize("radices", [(8, 3, 5), (61,), (2, 61), (61, 3, 2), (4, 2, 3, 61),
                                     (8, 2, 61), (11,), (3, 127)])
def test_stockham_stages_with_a_prime_radix_are_the_dft(radices):
    """The stage order and twiddle indices of fft.cu, including the direct
    prime-radix stage that lengths with a factor in [11, 127] use (the 61-day
    window at 5 s), against numpy's FFT."""
    m = int(np.prod(radices))
    x = np.random.default_rng(m).standard_normal(m) + 1j * np.random.default_rng(m + 1).standard_normal(m)
    assert np.max(np.abs(_stockham(x, radices) - np.fft.fft(x))) <= 1e-12 * np.sqrt(m) * np.max(np.abs(x)) * m


def _expand_weights_f32(xs, i):
    """het_expand_kernel's FP32 cubic weights of sample i from node indices xs
    [4], in the kernel's order: den_q = prod_{t != q} (x_q - x_t) over t
    ascending, 1 / den_q, then (e1 e23) / den_0, (e0 e23) / den_1,
    (e01 e3) / den_2, (e01 e2) / den_3 with e_q = i - x_q."""
    f = np.float32
    x = [f(v) for v in xs]
    dinv = []
    for q in range(4):
        den = f(1)
        for t in range(4):
            if t != q:
                den = f(den * f(x[q] - x[t]))
        dinv.append(f(f(1) / den))
    xi = f(i)
    e = [f(xi - x[q]) for q in range(4)]
    e01, e23 = f(e[0] * e[1]), f(e[2] * e[3])
    return np.array([f(f(e[1] * e23) * dinv[0]), f(f(e[0] * e23) * dinv[1]),
                     f(f(e01 * e[3]) * dinv[2]), f(f(e01 * e[2]) * dinv[3])], dtype=np.float64)


@pytest.mark.parametrize("xs", [(0, 1, 2, 3), (0, 50, 100, 150), (1000, 1050, 5000, 13640),
                                (20000, 28640, 37280, 45920), (5000, 13640, 13641, 13642)])
def test_expansion_weights_in_fp32_stay_within_rounding(xs):
    """The heterodyne expansion's Lagrange-form weights in FP32 (node indices
    are exact integers below 2^24, so e_q and the node differences are exact):
    every weight within a few FP32 roundings of the FP64 Lagrange weight, for
    uniform spacing, the 250 s start taper, a taper-to-chirp step and the
    12 h cap, and dense nodes after a long interval (weights up to ~1e3, a
    spacing the node rule avoids: its chirp spacing has shrunk to about one
    sample where the dense window starts)."""
    xs64 = np.array(xs, dtype=np.float64)
    for i in range(xs[0], xs[3] + 1, max(1, (xs[3] - xs[0]) // 997)):
        w64 = np.array([np.prod([(i - xs64[t]) / (xs64[q] - xs64[t]) for t in range(4) if t != q])
                        for q in range(4)])
        w32 = _expand_weights_f32(xs, i)
        # the cubic reproduces constants (to FP64 rounding of weights that
        # reach ~1e3 where dense nodes follow a long interval)
        assert abs(np.sum(w64) - 1.0) <= 1e-14 * np.sum(np.abs(w64))
        # each weight is five or six correctly rounded FP32 operations on exact inputs
        assert np.all(np.abs(w32 - w64) <= 8 * 2.0 ** -24 * np.abs(w64) + 1e-30), (i, w32, w64)
