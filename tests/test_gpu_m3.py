"""Parity of the variants M3 and M_{3A-DEF} (§4.3) with the FP64 oracle.

M3 approximates S_I^{-1} by Nyström from an interior sketch G_I (n_interior x s): both sides
take the same explicit G_I, solve S_I X = G_I by block PCG preconditioned by A_I to the inner
tolerance, form V Sigma V^T by Algorithm 1 steps 3-8 and Zh = A_G^{-1} A_GI V. FP64 handles
stop after the oracle's number of inner iterations and apply M3 at rounding level; FP32
handles apply it at the FP32 level; both reach the outer tolerance in the oracle's iteration
count +-2.
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
@pytest.mark.parametrize("variant", ["m3", "m3_adef"])
def test_apply_m3_matches_oracle(N, torch, name, prec, variant):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    dtol = 1e-12 if prec == "fp64" else 1e-6
    GI = np.random.default_rng(5).standard_normal((D.n_I, k + p))
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=GI, drop_tol=dtol,
                    variant=variant)
    M, info = O.build_m3(D, GI, k, 0.1, drop_tol=dtol, variant=variant.upper())
    if prec == "fp64":
        assert h.info()["it_inner"] == info["it_inner"]
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
def test_solve_parity_m3(N, torch, name, prec, form):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    GI = np.random.default_rng(8).standard_normal((D.n_I, k + p))
    b = A @ np.random.default_rng(9).standard_normal(A.shape[0])
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=GI, outer_form=form,
                    variant="m3")
    M, _ = O.build_m3(D, GI, k, 0.1)
    _, it_ref, _ = O.solve(D, M.apply, b, rtol=1e-8)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=1e-8, maxit=500)
    assert O.relative_residual(A, xd.cpu().numpy(), b) < 1e-7
    assert abs(inf["it_pcg"] - it_ref) <= 2, (inf["it_pcg"], it_ref)
    h.destroy()


def test_m3_requests_refused(N):
    A, part, nsub = _case("tiny2d")
    with pytest.raises(N.NspError) as e:
        N.nsp_build(A, part, nsub, k=4, p=2, variant="m3", q=1)
    assert e.value.status == 9   # NSP_ERR_UNSUPPORTED
    h = N.nsp_build(A, part, nsub, k=4, p=2, variant="m3", keep_intermediates=True)
    with pytest.raises(N.NspError):
        h.get_intermediate(0)
    h.destroy()
    with pytest.raises(N.NspError) as e:
        N.nsp_build_batched([(A, part, nsub)], k=4, p=2, variant="m3")
    assert e.value.status == 9
