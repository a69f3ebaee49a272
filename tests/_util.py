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


def colwise_err(a, ref):
    """Entry-wise error of a against ref, column by column: the largest over columns j of
    max_i |a_ij - ref_ij| / max_i |ref_ij| (a vector is one column). Unlike a Frobenius
    ratio over a whole block, a few wrong rows or one wrong small column cannot hide here."""
    a = np.asarray(a, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    assert a.shape == ref.shape, (a.shape, ref.shape)
    if ref.ndim == 1:
        a, ref = a[:, None], ref[:, None]
    a = a.reshape(a.shape[0], -1)
    ref = ref.reshape(ref.shape[0], -1)
    scale = np.maximum(np.abs(ref).max(axis=0), 1e-300)
    return float((np.abs(a - ref).max(axis=0) / scale).max())


def operator_err(Z1, S1, Z2, S2):
    """|| Z1 diag(S1) Z1^T - Z2 diag(S2) Z2^T ||_F / || Z2 diag(S2) Z2^T ||_F through k x k
    Grams (the Nyström factor as an operator: eigenvector signs and rotations inside
    clusters are arbitrary)."""
    Z1, Z2 = np.asarray(Z1, np.float64), np.asarray(Z2, np.float64)
    S1, S2 = np.asarray(S1, np.float64), np.asarray(S2, np.float64)
    G11, G22, G12 = Z1.T @ Z1, Z2.T @ Z2, Z1.T @ Z2
    M11, M22 = S1[:, None] * G11, S2[:, None] * G22     # diag(S) Z^T Z
    n11, n22 = np.sum(M11 * M11.T), np.sum(M22 * M22.T)
    n12 = np.sum((S1[:, None] * G12) * (G12 * S2[None, :]))
    return float(np.sqrt(max(n11 + n22 - 2.0 * n12, 0.0) / n22))


def max_principal_angle(U1, U2):
    """Largest principal angle (radians) between span(U1) and span(U2) (orthonormalized)."""
    Q1, _ = np.linalg.qr(np.asarray(U1, np.float64))
    Q2, _ = np.linalg.qr(np.asarray(U2, np.float64))
    sv = np.linalg.svd(Q1.T @ Q2, compute_uv=False)
    return float(np.arccos(np.clip(sv.min(), -1.0, 1.0)))
