"""Geometric nested dissection of a box grid into the DBBD form of §2.3, eq. (perm_A).

The paper obtains the doubly bordered block diagonal form with a graph partitioner
(METIS); for structured grids a geometric recursive coordinate bisection gives the same
kind of partition: split the longest axis (ties to the lowest axis) of the current box at
m = floor((lo + hi) / 2); the plane coordinate == m joins the separator (interface)
Gamma; recurse depth-first on the two halves; the boxes left after log2(nsub) levels are
the interior subdomains, numbered in depth-first order.

``interior_nd_order`` gives a fill-reducing elimination order for each interior block by
the same bisection continued inside the subdomain box (children first, separator last),
which is the ordering a caller would normally hand to a sparse direct solver.
"""

import numpy as np


def _split_axis(lo, hi):
    ext = [h - l + 1 for l, h in zip(lo, hi)]
    return int(np.argmax(ext))  # argmax returns the lowest axis on ties


def nd_partition(shape, nsub):
    """part[i] in [0, nsub) for interior nodes, -1 for the separator Gamma.

    Returns (part, boxes) where boxes[b] = (lo, hi) inclusive bounds of subdomain b.
    """
    levels = int(round(np.log2(nsub)))
    if 1 << levels != nsub:
        raise ValueError("nsub must be a power of two")
    shape = tuple(int(s) for s in shape)
    n = int(np.prod(shape))
    part = np.full(n, -1, dtype=np.int32)
    grid = part.reshape(shape, order="F")   # view: grid[x, y, ...] is node x + nx*(y + ...)
    boxes = []

    def rec(lo, hi, depth):
        if any(h < l for l, h in zip(lo, hi)):
            raise ValueError("grid too small for the requested number of subdomains")
        if depth == levels:
            b = len(boxes)
            boxes.append((tuple(lo), tuple(hi)))
            grid[tuple(slice(l, h + 1) for l, h in zip(lo, hi))] = b
            return
        ax = _split_axis(lo, hi)
        m = (lo[ax] + hi[ax]) // 2
        left_hi = list(hi)
        left_hi[ax] = m - 1
        right_lo = list(lo)
        right_lo[ax] = m + 1
        rec(list(lo), left_hi, depth + 1)
        rec(right_lo, list(hi), depth + 1)

    rec([0] * len(shape), [s - 1 for s in shape], 0)
    return part, boxes


def _box_nd_order(lo, hi, shape, leaf):
    """Global node ids of the box in nested-dissection order (halves first, plane last)."""
    ext = [h - l + 1 for l, h in zip(lo, hi)]
    if any(e <= 0 for e in ext):
        return np.zeros(0, dtype=np.int64)
    if int(np.prod(ext)) <= leaf:
        rng = [np.arange(l, h + 1) for l, h in zip(lo, hi)]
        grid = np.meshgrid(*rng, indexing="ij")
        # x fastest inside the leaf box
        pts = np.stack([g.ravel(order="F") for g in grid], axis=1)
        strides = np.cumprod([1] + list(shape[:-1]))
        return (pts * strides).sum(axis=1).astype(np.int64)
    ax = _split_axis(lo, hi)
    m = (lo[ax] + hi[ax]) // 2
    left_hi = list(hi)
    left_hi[ax] = m - 1
    right_lo = list(lo)
    right_lo[ax] = m + 1
    sep_lo = list(lo)
    sep_hi = list(hi)
    sep_lo[ax] = sep_hi[ax] = m
    return np.concatenate([
        _box_nd_order(list(lo), left_hi, shape, leaf),
        _box_nd_order(right_lo, list(hi), shape, leaf),
        _box_nd_order(sep_lo, sep_hi, shape, 1 << 62),  # separator: one dense block
    ])


def interior_nd_order(shape, boxes, leaf=16):
    """Concatenated nested-dissection orders of all subdomain boxes (block by block)."""
    shape = tuple(int(s) for s in shape)
    return np.concatenate([_box_nd_order(list(lo), list(hi), shape, leaf) for lo, hi in boxes])


def interface_partition(A_G, coords, nblocks):
    """A DBBD partition of the interface matrix A_Gamma itself (its own §2.3 eq. (perm_A)
    form), for the recursive treatment of A_Gamma.

    Recursive coordinate bisection of the interface nodes' coordinates (median split of the
    widest axis, depth-first numbering) gives nblocks boxes; every edge of A_Gamma that joins
    two boxes puts its endpoint in the higher-numbered box on the second-level separator
    (label -1), so no edge is left between interior nodes of different boxes.
    Returns part2 (int32, n_Gamma entries in A_Gamma's row order).
    """
    import scipy.sparse as sp
    levels = int(round(np.log2(nblocks)))
    if 1 << levels != nblocks:
        raise ValueError("nblocks must be a power of two")
    coords = np.asarray(coords, dtype=np.float64)
    n = coords.shape[0]
    box = np.zeros(n, dtype=np.int32)

    def rec(idx, depth, label):
        if depth == levels:
            box[idx] = label
            return label + 1
        c = coords[idx]
        ax = int(np.argmax(c.max(axis=0) - c.min(axis=0)))
        order = idx[np.argsort(c[:, ax], kind="stable")]
        h = len(order) // 2
        label = rec(order[:h], depth + 1, label)
        return rec(order[h:], depth + 1, label)

    rec(np.arange(n), 0, 0)
    C = sp.coo_matrix(A_G)
    cut = box[C.row] != box[C.col]
    hi = np.where(box[C.row[cut]] > box[C.col[cut]], C.row[cut], C.col[cut])
    part = box.copy()
    part[hi] = -1
    return part
