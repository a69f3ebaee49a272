"""The variant M1 of §4.1 (eq. (prec1S)) on the GPU.

M1 = A_G^{-1} + Zb Sigma Zb^T comes from the Nyström approximation of R^{-T} A_GI S_I^{-1}
A_IG R^{-1} with A_G = R^T R. The GPU takes R from its own factorization of A_G (its
fill-reducing order), the oracle a dense Cholesky factor in the natural order, so the two M1
are different preconditioners in general. They coincide where the Nyström approximation is
exact: with a sketch of n_Gamma columns and exact inner solves, R^{-T} B R^{-1} = Ub Lambda
Ub^T exactly and M1 = A_G^{-1} + R^{-1} Ub Lambda (I - Lambda)^{-1} Ub^T R^{-T} =
S_Gamma^{-1} for any R. That identity pins the GPU form (both half sweeps, the sketch
R^{-1} G, the core on (G, R^{-T} Y), Zb = R^{-1} Ub) entry by entry on interfaces where
A_GI S_I^{-1} A_IG has full rank (the oracle's own M1 meets it at rounding level there); at
ordinary k the outer iteration counts are compared with the oracle's M1.
"""

import numpy as np
import pytest

import oracle as O

from ._util import colwise_err, lib_or_build, tiny_problem

pytestmark = pytest.mark.gpu

CASES = {
    "tiny2d": dict(shape=(13, 11), nsub=2, lognormal=(3.0, 1.5)),
    "tiny3d": dict(shape=(9, 8, 7), nsub=4, lognormal=(2.0, 1.5)),
    "ragged2d": dict(shape=(37, 29), nsub=4, lognormal=(5.0, 2.0)),
    # one separator plane: every interface unknown couples to interior ones, so
    # A_GI S_I^{-1} A_IG has full rank and one block-PCG iteration on n_Gamma columns is exact
    "plane3d": dict(shape=(9, 8, 7), nsub=2, lognormal=(2.0, 1.5)),
    "plane3d_b": dict(shape=(11, 10, 9), nsub=2, lognormal=(3.0, 1.5)),
}


@pytest.fixture(scope="module")
def N():
    return lib_or_build()


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


def _case(name):
    c = CASES[name]
    A, part, _ = tiny_problem(c["shape"], c["nsub"], c["lognormal"], seed=7)
    return A, part, c["nsub"]


@pytest.mark.parametrize("name", ["tiny2d", "plane3d", "plane3d_b"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_m1_with_exact_nystrom_is_schur_inverse(N, torch, name, prec):
    # n_Gamma sketch columns: the first block-PCG iteration spans the whole space and meets
    # the inner tolerance, the Nyström core has full rank
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    nG = D.n_G
    assert nG <= 256
    G = np.random.default_rng(11).standard_normal((nG, nG))
    h = N.nsp_build(A, part, nsub, k=nG, p=0, precision=prec, sketch=G, variant="m1",
                    eps_inner=1e-9, drop_tol=1e-14 if prec == "fp64" else 1e-7)
    S = D.dense_S_gamma()
    rng = np.random.default_rng(12)
    # a transposed half sweep anywhere (R^{-T} for R^{-1} or back) leaves errors near 1e-2
    tol = 1e-7 if prec == "fp64" else 3e-3
    for _ in range(2):
        r = rng.standard_normal(nG)
        rd = torch.tensor(r, dtype=torch.float64, device="cuda")
        zd = torch.empty_like(rd)
        h.apply(rd, zd)
        err = colwise_err(zd.cpu().numpy(), np.linalg.solve(S, r))
        assert err < tol, err
    h.destroy()


@pytest.mark.parametrize("name", ["tiny3d", "ragged2d"])
@pytest.mark.parametrize("prec,form", [("fp64", "schur"), ("fp32", "full")])
def test_m1_solve_iterations_match_oracle(N, torch, name, prec, form):
    # different R on the two sides: the same sketch, tolerance and outer rtol give iteration
    # counts within a few of each other, and the GPU reaches the rtol
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    G = np.random.default_rng(13).standard_normal((D.n_G, k + p))
    b = A @ np.random.default_rng(14).standard_normal(A.shape[0])
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=G, outer_form=form,
                    variant="m1")
    M, _ = O.build_m1(D, G, k, 0.1)
    _, it_ref, _ = O.solve(D, M.apply, b, rtol=1e-8)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=1e-8, maxit=500)
    assert O.relative_residual(A, xd.cpu().numpy(), b) < 1e-7
    assert abs(inf["it_pcg"] - it_ref) <= 3, (inf["it_pcg"], it_ref)
    h.destroy()


def test_m1_power_iterations_refused(N):
    A, part, nsub = _case("tiny2d")
    with pytest.raises(N.NspError) as e:
        N.nsp_build(A, part, nsub, k=4, p=2, variant="m1", q=1)
    assert e.value.status == 9   # NSP_ERR_UNSUPPORTED
