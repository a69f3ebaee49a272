"""Parity of the M_{2A-DEF} variant (§4.3, adapted deflation) with the FP64 oracle.

The handle is built with variant="m2_adef" from the same explicit sketch G as the oracle.
Both sides deflate span(A_G^{-1} U) with E = Z^T S_G Z; the GPU forms S_G Z in the handle's
precision, so FP64 handles agree at rounding level and FP32 handles at the level of the
FP32 S_G apply (the same bounds as the M2 apply tests). The outer PCG reaches the tolerance
in the oracle's iteration count +-2.
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


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_m2adef_matches_oracle(N, torch, name, prec):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    dtol = 1e-12 if prec == "fp64" else 1e-6
    G = np.random.default_rng(5).standard_normal((D.n_G, k + p))
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=G, drop_tol=dtol,
                    variant="m2_adef")
    M, _ = O.build_m2(D, G, k, 0.1, drop_tol=dtol, variant="M2_ADEF")
    rng = np.random.default_rng(6)
    tol = 1e-7 if prec == "fp64" else 1e-2
    for _ in range(2):
        r = rng.standard_normal(D.n_G)
        rd = torch.tensor(r, dtype=torch.float64, device="cuda")
        zd = torch.empty_like(rd)
        h.apply(rd, zd)
        err = colwise_err(zd.cpu().numpy(), M.apply(r))
        assert err < tol, err
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,form", [("fp64", "schur"), ("fp32", "full")])
def test_solve_parity_m2adef(N, torch, name, prec, form):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    G = np.random.default_rng(8).standard_normal((D.n_G, k + p))
    b = A @ np.random.default_rng(9).standard_normal(A.shape[0])
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=G, outer_form=form,
                    variant="m2_adef")
    M, _ = O.build_m2(D, G, k, 0.1, variant="M2_ADEF")
    _, it_ref, _ = O.solve(D, M.apply, b, rtol=1e-8)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=1e-8, maxit=500)
    assert O.relative_residual(A, xd.cpu().numpy(), b) < 1e-7
    assert abs(inf["it_pcg"] - it_ref) <= 2, (inf["it_pcg"], it_ref)
    h.destroy()


def test_m2adef_exact_with_full_interface_basis(N, torch):
    # k = n_Gamma and tight inner solves: span(Z) holds every deflated direction, so
    # M_{2A-DEF} S_G = I and the outer PCG stops after one or two iterations
    A, part, nsub = _case("tiny2d")
    D = O.DBBD(A, part, nsub)
    G = np.random.default_rng(10).standard_normal((D.n_G, D.n_G))
    b = A @ np.random.default_rng(11).standard_normal(A.shape[0])
    h = N.nsp_build(A, part, nsub, k=D.n_G, p=0, precision="fp64", sketch=G,
                    eps_inner=1e-13, eps_trunc_rel=1e-12, outer_form="schur",
                    variant="m2_adef")
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=1e-10, maxit=50)
    assert inf["it_pcg"] <= 3, inf["it_pcg"]
    assert O.relative_residual(A, xd.cpu().numpy(), b) < 1e-9
    h.destroy()


def test_m2adef_refused_on_batched_handles(N):
    A, part, nsub = _case("tiny2d")
    with pytest.raises(N.NspError) as e:
        N.nsp_build_batched([(A, part, nsub)], k=4, p=2, variant="m2_adef")
    assert e.value.status == 9   # NSP_ERR_UNSUPPORTED
