"""Parity of the q-power iteration Nyström build (§2.1 eq. (power)) with the FP64 oracle.

Both sides start from the same explicit sketch Omega, apply B = A_GI S_I^{-1} A_IG by the
inner block PCG q + 1 times and orthonormalize the columns between applications by a
thresholded Cholesky-QR with the same drop rule. FP64 handles take the same number of inner
iterations in every pass and give the same low-rank term Z Sigma Z^T at rounding level; FP32
handles reach the outer tolerance in the oracle's iteration count +-2.
"""

import numpy as np
import pytest

import oracle as O

from ._util import lib_or_build, operator_err, tiny_problem

pytestmark = pytest.mark.gpu

CASES = {
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
@pytest.mark.parametrize("q", [1, 2])
def test_power_build_parity_fp64(N, name, q):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    G = np.random.default_rng(3).standard_normal((D.n_G, k + p))
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision="fp64", sketch=G, drop_tol=1e-12,
                    keep_intermediates=True, q=q)
    M, info = O.build_m2(D, G, k, 0.1, drop_tol=1e-12, q=q)
    gi = h.info()
    assert gi["it_power"] == sum(info["it_power"])
    assert gi["it_inner"] == info["it_inner"]
    assert gi["rank"] == len(M.Sigma)
    # the final sketch spans the oracle's (orthonormal bases of the same subspace)
    Gg = h.get_intermediate(0)
    Go = info["G"]
    assert np.linalg.norm(Gg @ (Gg.T @ Go) - Go) < 1e-6 * np.sqrt(Go.shape[1])
    Z, S = h.get_basis()
    assert np.allclose(S, M.Sigma, rtol=1e-6)
    assert operator_err(Z, S, M.Z, M.Sigma) < 1e-6
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,form", [("fp64", "schur"), ("fp32", "full")])
def test_power_solve_parity(N, torch, name, prec, form):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    G = np.random.default_rng(8).standard_normal((D.n_G, k + p))
    b = A @ np.random.default_rng(9).standard_normal(A.shape[0])
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=G, outer_form=form, q=1)
    M, _ = O.build_m2(D, G, k, 0.1, q=1)
    _, it_ref, _ = O.solve(D, M.apply, b, rtol=1e-8)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=1e-8, maxit=500)
    assert O.relative_residual(A, xd.cpu().numpy(), b) < 1e-7
    assert abs(inf["it_pcg"] - it_ref) <= 2, (inf["it_pcg"], it_ref)
    h.destroy()


def test_power_iteration_requests_refused(N):
    A, part, nsub = _case("tiny3d")
    with pytest.raises(N.NspError) as e:
        N.nsp_build(A, part, nsub, k=4, p=2, q=-1)
    assert e.value.status == 1   # NSP_ERR_INVALID_ARG
    with pytest.raises(N.NspError) as e:
        N.nsp_build_batched([(A, part, nsub)], k=4, p=2, q=1)
    assert e.value.status == 9   # NSP_ERR_UNSUPPORTED
