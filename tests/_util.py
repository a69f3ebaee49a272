"""Shared helpers of the test-suite (inputs only; no method arithmetic)."""

import numpy as np
import pytest

import fixtures as F


def tiny_problem(shape=(10, 9), nsub=2, lognormal=(3.0, 1.5), seed=0):
    coef = None
    if lognormal is not None:
        rng = np.random.default_rng(seed)
        coef = F.lognormal_field(F.grid_coords(shape), lognormal[0], lognormal[1], rng)
    A = F.diffusion_matrix(shape, coef)
    part, boxes = F.nd_partition(shape, nsub)
    perm = F.interior_nd_order(shape, boxes)
    return A, part, perm


def lib_or_build():
    """The loaded CUDA library, building it in-tree when missing (nvcc cross-compiles)."""
    import paper_2101_12164_gb300 as N
    from paper_2101_12164_gb300 import build as B
    try:
        B.build()
    except Exception as e:  # pragma: no cover - only without nvcc
        pytest.skip("cannot build libnsp.so: %s" % e)
    return N


def torch_cuda():
    import torch
    return torch
