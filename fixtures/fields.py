"""Seeded Gaussian random fields by random Fourier features (Rahimi & Recht, 2007).

g(x) = sqrt(2/M) * sum_m cos(w_m . x + phi_m) with w_m ~ N(0, ell^-2 I) and
phi_m ~ U[0, 2 pi) has zero mean, unit variance and covariance exp(-|x-y|^2 / (2 ell^2))
as M grows. A lognormal coefficient is a = exp(sigma * g).

On a full box grid (the nodes of ``grid_coords(shape)``) the same sum is evaluated as
Re sum_m e^{i phi_m} prod_t e^{i w_mt x_t}: the per-axis factors take only shape[t]
values, so the last axis becomes one complex matrix product (identical field up to
rounding, about 1e-13 relative).
"""

import numpy as np


def _draw(rng, modes, d, ell):
    omega = rng.standard_normal((modes, d)) / float(ell)
    phase = rng.uniform(0.0, 2.0 * np.pi, modes)
    return omega, phase


def gaussian_field(coords, ell, rng, modes=512, chunk=1 << 15):
    coords = np.asarray(coords, dtype=np.float64)
    n, d = coords.shape
    omega, phase = _draw(rng, modes, d, ell)
    g = np.empty(n)
    for s in range(0, n, chunk):
        e = min(n, s + chunk)
        g[s:e] = np.cos(coords[s:e] @ omega.T + phase).sum(axis=1)
    return g * np.sqrt(2.0 / modes)


def gaussian_grid_field(shape, ell, rng, modes=512):
    """gaussian_field(grid_coords(shape), ell, rng, modes) for a full box grid (x fastest)."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    omega, phase = _draw(rng, modes, d, ell)
    # acc[m, x_0, ..., x_{d-2}] = e^{i phi_m} prod_{t < d-1} e^{i w_mt x_t}
    acc = np.exp(1j * phase).reshape(modes, *([1] * (d - 1)))
    for t in range(d - 1):
        f = np.exp(1j * np.outer(omega[:, t], np.arange(shape[t])))
        acc = acc * f.reshape((modes,) + (1,) * t + (shape[t],) + (1,) * (d - 2 - t))
    last = np.exp(1j * np.outer(omega[:, d - 1], np.arange(shape[d - 1])))   # (M, n_last)
    g = (acc.reshape(modes, -1).T @ last).real                                 # (prod, n_last)
    # rows: x_0..x_{d-2} in C order over acc's axes; nodes are x fastest (Fortran order)
    g = g.reshape(*shape[:-1], shape[-1])
    return g.reshape(-1, order="F") * np.sqrt(2.0 / modes)


def lognormal_field(coords, ell, sigma, rng, modes=512):
    return np.exp(float(sigma) * gaussian_field(coords, ell, rng, modes))


def lognormal_grid_field(shape, ell, sigma, rng, modes=512):
    return np.exp(float(sigma) * gaussian_grid_field(shape, ell, rng, modes))
