"""Pins of the oracle's coloured noise: the likelihood's inner product inverts
the synthesis exactly ((n|n) = sum of the band's squared normals), nothing
leaks out of band, and the noise is real and stationary in distribution
(its sample PSD matches S over many realisations)."""
import numpy as np

from oracle import likelihood, noise


def _setup(n=8640, dt=5.0, gen=20):
    return n, dt, 1e-4, 0.02, gen


def test_inner_product_of_the_noise_is_the_sum_of_squared_normals():
    n, dt, flo, fhi, gen = _setup()
    nb = n // 2 + 1
    z = np.random.default_rng(1).normal(size=(3, 2, nb))
    x = noise.noise_aet(z, n, dt, flo, fhi, gen)
    f = likelihood.freqs(n, dt)
    mask = likelihood.band(n, dt, flo, fhi)
    s_ae, s_t = likelihood.psd_aet(np.where(f > 0, f, 1.0), gen)
    df = 1.0 / (n * dt)
    for c in range(3):
        xf = likelihood.dft(x[c], dt)
        got = likelihood.inner(xf, xf, s_t if c == 2 else s_ae, df, mask)
        want = float(np.sum(z[c, 0][mask] ** 2 + z[c, 1][mask] ** 2))
        assert abs(got - want) <= 1e-9 * want
        assert np.max(np.abs(xf[~mask])) <= 1e-12 * np.max(np.abs(xf[mask]))
    # zero-noise logL at the truth becomes -1/2 (n|n)
    assert likelihood.loglike(np.zeros((3, n)), -x, dt, flo, fhi, gen) < 0


def test_sample_psd_matches_the_model():
    n, dt, flo, fhi, gen = _setup(n=4320, gen=15)
    nb = n // 2 + 1
    rng = np.random.default_rng(2)
    f = likelihood.freqs(n, dt)
    mask = likelihood.band(n, dt, flo, fhi)
    s_ae, _ = likelihood.psd_aet(np.where(f > 0, f, 1.0), gen)
    acc = np.zeros(nb)
    R = 200
    for _ in range(R):
        x = noise.noise_aet(rng.normal(size=(3, 2, nb)), n, dt, flo, fhi, gen)
        acc += np.abs(likelihood.dft(x[0], dt)) ** 2
    # one-sided PSD estimate S = 2 |dt N_k|^2 / (n dt), averaged over realisations
    est = 2.0 * acc / R / (n * dt)
    ratio = est[mask] / s_ae[mask]
    assert abs(np.mean(ratio) - 1.0) < 0.02
