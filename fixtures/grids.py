"""Cell-centred finite-difference diffusion operators on structured grids.

Unknowns sit at the ``prod(shape)`` interior nodes of a box grid (Dirichlet boundary
nodes eliminated); node index = x + nx*(y + ny*z) (x fastest). The operator is the
unscaled 2*d+1 point stencil of -div(K a grad u):

* interior face between nodes i, j along axis t: coefficient s_t * 2 a_i a_j / (a_i + a_j)
  (harmonic mean of the node coefficients), contributing -c to A[i,j] and +c to both
  diagonals;
* boundary face of node i along axis t: s_t * a_i added to A[i,i].

``s_t`` is a per-axis scale (axis anisotropy, or the diagonal entries K_xx, K_yy of a
rotated anisotropy tensor, whose mixed term a 5-point stencil cannot represent).
The result is symmetric, irreducibly diagonally dominant with positive diagonal, hence SPD.
"""

import numpy as np
import scipy.sparse as sp


def grid_coords(shape):
    """(n, d) integer coordinates of the nodes, x fastest."""
    n = int(np.prod(shape))
    idx = np.unravel_index(np.arange(n, dtype=np.int64), shape, order="F")
    return np.stack(idx, axis=1).astype(np.int64)


def diffusion_matrix(shape, coef=None, axis_scale=None):
    """SPD scipy CSR matrix (float64, sorted indices) of the stencil above."""
    shape = tuple(int(s) for s in shape)
    d = len(shape)
    n = int(np.prod(shape))
    a = np.ones(n) if coef is None else np.asarray(coef, dtype=np.float64).reshape(n)
    scale = np.ones(d) if axis_scale is None else np.asarray(axis_scale, dtype=np.float64)
    coords = grid_coords(shape)
    diag = np.zeros(n)
    rows, cols, vals = [], [], []
    stride = 1
    for t in range(d):
        c = coords[:, t]
        # interior faces (i, i + stride) along axis t
        i = np.nonzero(c < shape[t] - 1)[0]
        j = i + stride
        k = scale[t] * 2.0 * a[i] * a[j] / (a[i] + a[j])
        rows += [i, j]
        cols += [j, i]
        vals += [-k, -k]
        np.add.at(diag, i, k)
        np.add.at(diag, j, k)
        # boundary faces (to the eliminated Dirichlet nodes)
        lo = np.nonzero(c == 0)[0]
        hi = np.nonzero(c == shape[t] - 1)[0]
        np.add.at(diag, lo, scale[t] * a[lo])
        np.add.at(diag, hi, scale[t] * a[hi])
        stride *= shape[t]
    rows.append(np.arange(n))
    cols.append(np.arange(n))
    vals.append(diag)
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A
