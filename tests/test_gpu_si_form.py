"""Parity of the S_I inner form (Algorithm 2 steps 2-4 as the paper writes them) with the
FP64 oracle: F = A_IG G, block PCG on S_I X = F preconditioned by A_I (§5 setup), Y = A_GI X.

Same sketch on both sides. FP64 handles stop after the same number of inner iterations as
the oracle's S_I form and give its Y, Sigma and Z Sigma Z^T at rounding level; FP32 handles
stop within one iteration of it and reach the outer tolerance in its iteration count +-2.
"""

import numpy as np
import pytest

import oracle as O

from ._util import colwise_err, lib_or_build, operator_err, tiny_problem

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
def test_si_build_parity_fp64(N, name):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    G = np.random.default_rng(3).standard_normal((D.n_G, k + p))
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision="fp64", sketch=G, drop_tol=1e-12,
                    keep_intermediates=True, inner_form="s_i")
    M, info = O.build_m2(D, G, k, 0.1, form="S_I", drop_tol=1e-12)
    gi = h.info()
    assert gi["it_inner"] == info["it_inner"]
    assert gi["rank"] == len(M.Sigma)
    assert colwise_err(h.get_intermediate(2), info["Y"]) < 1e-7
    Z, S = h.get_basis()
    assert np.allclose(S, M.Sigma, rtol=1e-8)
    assert operator_err(Z, S, M.Z, M.Sigma) < 1e-7
    with pytest.raises(N.NspError):
        h.get_intermediate(1)          # X has n_interior rows in this form
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,form", [("fp64", "schur"), ("fp32", "full")])
def test_si_solve_parity(N, torch, name, prec, form):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    G = np.random.default_rng(8).standard_normal((D.n_G, k + p))
    b = A @ np.random.default_rng(9).standard_normal(A.shape[0])
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=G, outer_form=form,
                    inner_form="s_i")
    M, info = O.build_m2(D, G, k, 0.1, form="S_I")
    _, it_ref, _ = O.solve(D, M.apply, b, rtol=1e-8)
    assert abs(h.info()["it_inner"] - info["it_inner"]) <= 1
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=1e-8, maxit=500)
    assert O.relative_residual(A, xd.cpu().numpy(), b) < 1e-7
    assert abs(inf["it_pcg"] - it_ref) <= 2, (inf["it_pcg"], it_ref)
    h.destroy()


def test_si_form_refused_on_batched_handles(N):
    A, part, nsub = _case("tiny2d")
    with pytest.raises(N.NspError) as e:
        N.nsp_build_batched([(A, part, nsub)], k=4, p=2, inner_form="s_i")
    assert e.value.status == 9   # NSP_ERR_UNSUPPORTED
