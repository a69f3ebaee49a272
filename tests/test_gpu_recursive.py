"""The recursive treatment of A_Gamma on the GPU (concluding section; the reading is the
oracle's ``recursive_gamma``): A_Gamma split by a DBBD partition of its own, A_Gamma^{-1}
replaced by the block elimination of §2.3 eq. (A_LDLT) for that split with the split's M2 as
the Schur solve, in every place the build and the preconditioner use A_Gamma^{-1}.

Entry-wise against the oracle: the nested inverse itself (nsp_factor_solve(1, ...)), and the
recursive M2. Pinned to the plain definition: with a nested sketch of full width the nested
inverse is A_Gamma^{-1} and the recursive M2 is the plain M2. Outer iterations against the
oracle's recursive M2 at the paper's loose tolerances.
"""

import numpy as np
import pytest

import fixtures as F
import oracle as O

from ._util import colwise_err, lib_or_build, tiny_problem

pytestmark = pytest.mark.gpu

CASES = {
    "plane3d": ((9, 8, 7), 2, 2),
    "cross3d": ((12, 11, 9), 4, 4),
    "plane3d_b": ((13, 12, 11), 2, 4),
}


@pytest.fixture(scope="module")
def N():
    return lib_or_build()


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


def _case(name, seed=3):
    shape, nsub, nsub2 = CASES[name]
    A, part, _ = tiny_problem(shape, nsub, (3.0, 1.5), seed=seed)
    D = O.DBBD(A, part, nsub)
    part2 = F.interface_partition(D.A_G, F.grid_coords(shape)[D.gamma], nsub2)
    d2 = O.DBBD(D.A_G, part2, nsub2)
    return A, part, nsub, D, part2, nsub2, d2


def _nested(d2, full=False, seed=21):
    k2 = d2.n_G if full else max(2, d2.n_G // 4)
    p2 = 0 if full else 3
    G2 = np.random.default_rng(seed).standard_normal((d2.n_G, k2 + p2))
    return k2, p2, G2


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("s", [1, 7, 32])
def test_nested_inverse_matches_oracle_fp64(N, torch, name, s):
    A, part, nsub, D, part2, nsub2, d2 = _case(name)
    k2, p2, G2 = _nested(d2)
    Dr, _ = O.recursive_gamma(D, part2, nsub2, G2, k2, eps_inner=1e-10)
    h = N.nsp_build(A, part, nsub, k=4, p=2, precision="fp64", drop_tol=1e-14,
                    gamma_part=part2, gamma_nblocks=nsub2, gamma_k=k2, gamma_p=p2,
                    gamma_sketch=G2, gamma_eps_inner=1e-10)
    inf = h.info()
    assert inf["n_gamma2"] == d2.n_G and inf["rank_gamma"] == k2 and inf["it_inner_gamma"] > 0
    B = np.random.default_rng(30 + s).standard_normal((D.n_G, s))
    Bd = torch.tensor(B, dtype=torch.float64, device="cuda")
    Xd = torch.empty_like(Bd)
    h.factor_solve(1, Bd, Xd)
    torch.cuda.synchronize()
    X = Xd.cpu().numpy().reshape(D.n_G, s)
    ref = Dr.solve_G(B).reshape(D.n_G, s)
    assert colwise_err(X, ref) < 1e-8
    # the nested approximation is active: not A_Gamma^{-1}
    assert colwise_err(X, D.solve_G(B).reshape(D.n_G, s)) > 1e-6
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_full_width_nested_sketch_gives_the_exact_inverse(N, torch, name, prec):
    A, part, nsub, D, part2, nsub2, d2 = _case(name)
    k2, p2, G2 = _nested(d2, full=True)
    fp64 = prec == "fp64"
    h = N.nsp_build(A, part, nsub, k=4, p=2, precision=prec,
                    drop_tol=1e-14 if fp64 else 1e-7,
                    gamma_part=part2, gamma_nblocks=nsub2, gamma_k=k2, gamma_p=p2,
                    gamma_sketch=G2, gamma_eps_inner=1e-10 if fp64 else 1e-5)
    dt = torch.float64 if fp64 else torch.float32
    B = np.random.default_rng(40).standard_normal((D.n_G, 5))
    Bd = torch.tensor(B, dtype=dt, device="cuda")
    Xd = torch.empty_like(Bd)
    h.factor_solve(1, Bd, Xd)
    torch.cuda.synchronize()
    err = colwise_err(Xd.double().cpu().numpy(), D.solve_G(B))
    assert err < (1e-7 if fp64 else 5e-3), err
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
def test_recursive_m2_matches_oracle_fp64(N, torch, name):
    A, part, nsub, D, part2, nsub2, d2 = _case(name)
    k2, p2, G2 = _nested(d2)
    k, p = 5, 3
    G = np.random.default_rng(22).standard_normal((D.n_G, k + p))
    Dr, _ = O.recursive_gamma(D, part2, nsub2, G2, k2, eps_inner=1e-10)
    M, _ = O.build_m2(Dr, G, k, eps_inner=1e-10)
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision="fp64", sketch=G, eps_inner=1e-10,
                    drop_tol=1e-14, gamma_part=part2, gamma_nblocks=nsub2, gamma_k=k2,
                    gamma_p=p2, gamma_sketch=G2, gamma_eps_inner=1e-10)
    rng = np.random.default_rng(23)
    for _ in range(2):
        r = rng.standard_normal(D.n_G)
        rd = torch.tensor(r, dtype=torch.float64, device="cuda")
        zd = torch.empty_like(rd)
        h.apply(rd, zd)
        assert colwise_err(zd.cpu().numpy(), M.apply(r)) < 1e-7
    h.destroy()


def test_full_width_nested_sketch_gives_the_plain_m2(N, torch):
    A, part, nsub, D, part2, nsub2, d2 = _case("cross3d")
    k2, p2, G2 = _nested(d2, full=True)
    k, p = 6, 2
    G = np.random.default_rng(24).standard_normal((D.n_G, k + p))
    M, _ = O.build_m2(D, G, k, eps_inner=1e-10)            # plain M2: A_Gamma factorized
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision="fp64", sketch=G, eps_inner=1e-10,
                    drop_tol=1e-14, gamma_part=part2, gamma_nblocks=nsub2, gamma_k=k2,
                    gamma_p=p2, gamma_sketch=G2, gamma_eps_inner=1e-12)
    r = np.random.default_rng(25).standard_normal(D.n_G)
    rd = torch.tensor(r, dtype=torch.float64, device="cuda")
    zd = torch.empty_like(rd)
    h.apply(rd, zd)
    assert colwise_err(zd.cpu().numpy(), M.apply(r)) < 1e-7
    h.destroy()


@pytest.mark.parametrize("name", ["cross3d", "plane3d_b"])
@pytest.mark.parametrize("prec,form", [("fp64", "schur"), ("fp32", "full")])
def test_recursive_solve_iterations_match_oracle(N, torch, name, prec, form):
    A, part, nsub, D, part2, nsub2, d2 = _case(name)
    k2, p2, G2 = _nested(d2)
    k, p = 6, 4
    G = np.random.default_rng(26).standard_normal((D.n_G, k + p))
    b = A @ np.random.default_rng(27).standard_normal(A.shape[0])
    Dr, _ = O.recursive_gamma(D, part2, nsub2, G2, k2, eps_inner=0.1)
    M, _ = O.build_m2(Dr, G, k, eps_inner=0.1)
    _, it_ref, _ = O.solve(Dr, M.apply, b, rtol=1e-8)
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=G, outer_form=form,
                    gamma_part=part2, gamma_nblocks=nsub2, gamma_k=k2, gamma_p=p2,
                    gamma_sketch=G2, gamma_eps_inner=0.1)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=1e-8, maxit=500)
    assert O.relative_residual(A, xd.cpu().numpy(), b) < 1e-7
    assert abs(inf["it_pcg"] - it_ref) <= 3, (inf["it_pcg"], it_ref)
    # rebuild with doubled values keeps the split and halves the solution
    h.rebuild(torch.tensor(2.0 * A.data, dtype=torch.float64, device="cuda"), sketch=G, k=k,
              p=p, precision=prec, outer_form=form, gamma_k=k2, gamma_p=p2, gamma_sketch=G2,
              gamma_eps_inner=0.1)
    x2 = torch.zeros_like(bd)
    h.solve(bd, x2, rtol=1e-8, maxit=500)
    assert colwise_err(2.0 * x2.cpu().numpy(), xd.cpu().numpy()) < 1e-6
    h.destroy()


def test_recursive_refusals(N):
    A, part, nsub, D, part2, nsub2, d2 = _case("plane3d")
    with pytest.raises(N.NspError) as e:      # G2 smaller than gamma_k + gamma_p
        N.nsp_build(A, part, nsub, k=4, p=2, gamma_part=part2, gamma_nblocks=nsub2,
                    gamma_k=d2.n_G, gamma_p=1)
    assert e.value.status == 1
    bad = part2.copy()
    g2 = np.nonzero(bad < 0)[0]
    bad[g2] = 0                               # no second-level interface
    with pytest.raises(N.NspError) as e:
        N.nsp_build(A, part, nsub, k=4, p=2, gamma_part=bad, gamma_nblocks=nsub2,
                    gamma_k=2, gamma_p=1)
    assert e.value.status in (1, 2)           # INVALID_ARG or NOT_DBBD
    h = N.nsp_build(A, part, nsub, k=4, p=2, gamma_part=part2, gamma_nblocks=nsub2,
                    gamma_k=2, gamma_p=1)
    with pytest.raises(N.NspError) as e:      # the A_Gamma block is not factorized
        h.get_factor(nsub, D.n_G)
    assert e.value.status == 9
    h.destroy()
