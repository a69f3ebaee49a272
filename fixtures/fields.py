"""Seeded Gaussian random fields by random Fourier features (Rahimi & Recht, 2007).

g(x) = sqrt(2/M) * sum_m cos(w_m . x + phi_m) with w_m ~ N(0, ell^-2 I) and
phi_m ~ U[0, 2 pi) has zero mean, unit variance and covariance exp(-|x-y|^2 / (2 ell^2))
as M grows. A lognormal coefficient is a = exp(sigma * g).
"""

import numpy as np


def gaussian_field(coords, ell, rng, modes=512, chunk=1 << 15):
    coords = np.asarray(coords, dtype=np.float64)
    n, d = coords.shape
    omega = rng.standard_normal((modes, d)) / float(ell)
    phase = rng.uniform(0.0, 2.0 * np.pi, modes)
    g = np.empty(n)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        g[s:e] = np.cos(coords[s:e] @ omega.T + phase).sum(axis=1)
    return g * np.sqrt(2.0 / modes)


def lognormal_field(coords, ell, sigma, rng, modes=512):
    return np.exp(float(sigma) * gaussian_field(coords, ell, rng, modes))
