"""Inputs of the learned sketch proposal (no method arithmetic).

* ``node_attributes``: the raw per-interface-node input of the sketch network, read off
  the grid, the coefficient field and the partition: normalized coordinates, the log
  coefficient at the node and at its 2 * dim grid neighbours (clamped at the boundary),
  and per axis a 0/1 flag telling whether the node lies on a separator plane orthogonal
  to that axis (its two neighbours along the axis belong to different parts).
  Rows are in the interface order of Gamma-sized vectors (increasing node index).
* ``init_params``: seeded Glorot-uniform initial weights and zero biases, as one flat
  vector in the layout both implementations read (W1, b1, W2, b2, W3, b3; weights
  row-major, input dimension first).
* ``training_field``: the seeded lognormal coefficient fields of the learned-sketch
  workload (2D 5-point, correlation length and sigma drawn per seed).
"""

import numpy as np

from .fields import lognormal_grid_field
from .grids import diffusion_matrix, grid_coords
from .partition import nd_partition
from .seeds import rng_for


def node_attributes(shape, coef, part):
    """(n_gamma, 4 * dim + 1) float64 raw attributes of the interface nodes."""
    shape = tuple(int(x) for x in shape)
    dim = len(shape)
    # node numbering of the grids: x fastest (Fortran order)
    la = np.log(np.asarray(coef, dtype=np.float64)).reshape(shape, order="F")
    P = np.asarray(part).reshape(shape, order="F")
    gam = np.nonzero(np.asarray(part).ravel() < 0)[0]
    idx = np.unravel_index(gam, shape, order="F")
    cols = [(idx[a] + 1.0) / (shape[a] + 1.0) for a in range(dim)]
    cols.append(la[idx])
    for a in range(dim):
        for d in (-1, 1):
            j = list(idx)
            j[a] = np.clip(idx[a] + d, 0, shape[a] - 1)
            cols.append(la[tuple(j)])
    for a in range(dim):
        lo = list(idx)
        hi = list(idx)
        lo[a] = np.clip(idx[a] - 1, 0, shape[a] - 1)
        hi[a] = np.clip(idx[a] + 1, 0, shape[a] - 1)
        cols.append((P[tuple(lo)] != P[tuple(hi)]).astype(np.float64))
    return np.ascontiguousarray(np.stack(cols, axis=1))


def net_dims(d_raw, n_coord, n_freq, hidden, s_out):
    """Layer sizes (d0, hidden, hidden, s_out) of the network; d0 counts the embedding."""
    d0 = 2 * n_freq * n_coord + (d_raw - n_coord)
    return d0, hidden, hidden, s_out


def num_params(d_raw, n_coord, n_freq, hidden, s_out):
    d0, h1, h2, so = net_dims(d_raw, n_coord, n_freq, hidden, s_out)
    return d0 * h1 + h1 + h1 * h2 + h2 + h2 * so + so


def init_params(seed_index, d_raw, n_coord, n_freq, hidden, s_out, config=3):
    """Flat float64 vector of initial parameters (Glorot uniform weights, zero biases)."""
    rng = rng_for(config, seed_index, "net_init")
    d0, h1, h2, so = net_dims(d_raw, n_coord, n_freq, hidden, s_out)
    parts = []
    for a, b in ((d0, h1), (h1, h2), (h2, so)):
        lim = np.sqrt(6.0 / (a + b))
        parts.append(rng.uniform(-lim, lim, size=a * b))
        parts.append(np.zeros(b))
    return np.concatenate(parts)


def training_field(index, shape=(256, 256), ell_range=(4.0, 16.0), sigma_range=(1.0, 3.0),
                   config=3, ell_scale=1.0):
    """Coefficient field ``index`` of the learned-sketch family: lognormal with
    ell ~ U(ell_range) cells (times ell_scale) and sigma ~ U(sigma_range)."""
    rng = rng_for(config, index, "train")
    ell = float(rng.uniform(*ell_range)) * ell_scale
    sigma = float(rng.uniform(*sigma_range))
    coef = lognormal_grid_field(shape, ell, sigma, rng)
    return coef, dict(ell=ell, sigma=sigma)


def training_problem(index, shape=(256, 256), nsub=16, **kw):
    """(A, part, coef, attrs) of training field ``index`` on ``shape`` with ``nsub`` parts."""
    coef, meta = training_field(index, shape, **kw)
    A = diffusion_matrix(shape, coef)
    part, _ = nd_partition(shape, nsub)
    return A, part, coef, node_attributes(shape, coef, part), meta
