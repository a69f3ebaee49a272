"""The dense products of the inner block PCG on the tcgen05 tensor cores (nsp_gram,
nsp_block_update) against float64 products of the same float32 inputs, entry by entry.

Error model of 3xTF32 (x = x_hi + x_lo, products x_hi y_hi + x_hi y_lo + x_lo y_hi, FP32
accumulation): each product carries a relative error of about 2^-21 (the dropped x_lo y_lo
and the TF32 truncation of the low parts), the FP32 sums about 2^-24 per addition. The bound
per entry used here, 2^-16 sqrt(sum_i p_i^2) + 2^-22 sum_i |p_i| over the products p_i of the
entry, holds these with margin, while one TF32 product per pair (2^-11 relative, the error
of an unsplit TF32 product) exceeds it by more than ten times on the cases of up to 10^4
rows; a wrong descriptor or layout gives O(1) errors.
"""

import numpy as np
import pytest

from ._util import lib_or_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    return lib_or_build()


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


def _bound(P_abs_sum, P_sq_sum):
    return 2.0 ** -16 * np.sqrt(P_sq_sum) + 2.0 ** -22 * P_abs_sum


@pytest.mark.parametrize("n,s1,s2", [(1000, 7, 13), (5000, 80, 80), (70001, 160, 160),
                                     (3, 256, 256), (40000, 129, 33), (300000, 160, 160)])
def test_gram_matches_float64(N, torch, n, s1, s2):
    rng = np.random.default_rng(n + s1)
    X = rng.standard_normal((n, s1)).astype(np.float32)
    Y = rng.standard_normal((n, s2)).astype(np.float32)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    Cd = torch.empty(s1, s2, dtype=torch.float64, device="cuda")
    N.nsp_gram(Xd, Yd, Cd)
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    ref = X64.T @ Y64
    bound = _bound(np.abs(X64).T @ np.abs(Y64), (X64 ** 2).T @ (Y64 ** 2))
    err = np.abs(Cd.cpu().numpy() - ref)
    assert np.all(err <= bound), float((err / bound).max())
    # an unsplit TF32 product would be far outside the bound (where the bound is not yet
    # dominated by its FP32-accumulation term, which grows linearly with n)
    if 1000 <= n <= 10000:
        assert float(np.median(2.0 ** -11 * np.sqrt((X64 ** 2).T @ (Y64 ** 2)) / bound)) > 10


@pytest.mark.parametrize("n,s1,s2,beta,inplace", [(1000, 80, 80, 0.0, False),
                                                  (70001, 160, 160, 1.0, True),
                                                  (257, 13, 7, -0.5, False),
                                                  (300000, 160, 64, 1.0, False),
                                                  (5, 256, 256, 1.0, True)])
def test_block_update_matches_float64(N, torch, n, s1, s2, beta, inplace):
    rng = np.random.default_rng(n + s2)
    A = rng.standard_normal((n, s1)).astype(np.float32)
    M = rng.standard_normal((s1, s2))
    Cin = rng.standard_normal((n, s2)).astype(np.float32)
    scale = -1.5
    Ad = torch.tensor(A, device="cuda")
    Md = torch.tensor(M, dtype=torch.float64, device="cuda")
    Cd = torch.tensor(Cin, device="cuda")
    Od = Cd if inplace else torch.empty(n, s2, dtype=torch.float32, device="cuda")
    N.nsp_block_update(Ad, Md, Od, scale=scale, Cin=Cd if beta != 0.0 else None, beta=beta)
    A64, M32 = A.astype(np.float64), M.astype(np.float32).astype(np.float64)
    ref = scale * (A64 @ M32) + (beta * Cin.astype(np.float64) if beta != 0.0 else 0.0)
    bound = abs(scale) * _bound(np.abs(A64) @ np.abs(M32), (A64 ** 2) @ (M32 ** 2)) \
        + 2.0 ** -23 * (np.abs(ref) + abs(beta) * np.abs(Cin))
    err = np.abs(Od.cpu().numpy().astype(np.float64) - ref)
    assert np.all(err <= bound), float((err / bound).max())


def test_block_pcg_with_tensor_core_products_matches_simt(N, torch, monkeypatch):
    # the same FP32 build with the Grams and block updates on the SIMT pipes (NSP_TC=0):
    # same inner iteration count, E and Y within the FP32 level of the block PCG
    import fixtures as F
    from ._util import colwise_err, tiny_problem
    A, part, _ = tiny_problem((37, 29), 4, (5.0, 2.0), seed=7)
    G = np.random.default_rng(3).standard_normal((int((part < 0).sum()), 10))
    outs = []
    for tc in ("1", "0"):
        monkeypatch.setenv("NSP_TC", tc)
        h = N.nsp_build(A, part, 4, k=6, p=4, precision="fp32", sketch=G, keep_intermediates=True)
        outs.append((h.info()["it_inner"], h.get_intermediate(1), h.get_intermediate(2)))
        h.destroy()
    assert outs[0][0] == outs[1][0]
    assert colwise_err(outs[0][1], outs[1][1]) < 1e-4
    assert colwise_err(outs[0][2], outs[1][2]) < 1e-4


@pytest.mark.parametrize("n,s1,s2", [(1000, 7, 13), (70001, 160, 160), (300000, 128, 128)])
def test_compensated_gram_matches_exact_sums(N, torch, n, s1, s2):
    # the Nyström core's Grams: products of FP32 values are exact in FP64 and the reference
    # sums them in FP64 (typically ~sqrt(n) 2^-53 sum |p| off); the compensated FP32 kernel,
    # typically ~sqrt(rows per chunk) 2^-48 sum |p| off, must be within 2^-36 sum |p|, while
    # plain FP32 sums of these rows are ~sqrt(n) 2^-24 ~ 2^-16 sum |p| off
    rng = np.random.default_rng(n + 3 * s1)
    X = rng.standard_normal((n, s1)).astype(np.float32)
    Y = rng.standard_normal((n, s2)).astype(np.float32)
    Xd, Yd = torch.tensor(X, device="cuda"), torch.tensor(Y, device="cuda")
    Cd = torch.empty(s1, s2, dtype=torch.float64, device="cuda")
    N.nsp_gram(Xd, Yd, Cd, compensated=True)
    X64, Y64 = X.astype(np.float64), Y.astype(np.float64)
    ref = X64.T @ Y64
    absum = np.abs(X64).T @ np.abs(Y64)
    err = np.abs(Cd.cpu().numpy() - ref)
    assert np.all(err <= 2.0 ** -36 * absum + 1e-300), float((err / absum).max())
