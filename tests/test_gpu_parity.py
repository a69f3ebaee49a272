"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, step by step.

Every comparison is entry-wise, column by column (``colwise_err``: the largest
|gpu - oracle| of a column over that column's largest |oracle| entry), except the Nyström
factor, which is compared as an operator (eigenvector signs and rotations inside clusters are
arbitrary). Tolerances: FP64 handles at rounding level (the two sides factorize with
different orderings, so agreement is to a few hundred ulps times the condition number of
the operation); FP32 handles at the FP32 level, c * kappa * 2^-24 with the bounds written in
each test. The case "cluster3d" (a 20^3 grid in two subdomains) has fronts of more than 192
rows, so its factorization takes the clustered path (a cluster of CTAs per front); the
factor test checks that such a front exists.
"""

import numpy as np
import pytest

import fixtures as F
import oracle as O
from oracle import philox

from ._util import colwise_err, lib_or_build, operator_err, tiny_problem

pytestmark = pytest.mark.gpu

CASES = {
    "tiny2d": dict(shape=(13, 11), nsub=2, lognormal=(3.0, 1.5)),
    "tiny3d": dict(shape=(9, 8, 7), nsub=4, lognormal=(2.0, 1.5)),
    "ragged2d": dict(shape=(37, 29), nsub=4, lognormal=(5.0, 2.0)),
    "cluster3d": dict(shape=(20, 20, 20), nsub=2, lognormal=(4.0, 1.5)),
}
BIG_FRONT = 192   # fronts with at least this many rows are factorized by a CTA cluster


@pytest.fixture(scope="module")
def N():
    return lib_or_build()


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


def _case(name):
    c = CASES[name]
    A, part, perm = tiny_problem(c["shape"], c["nsub"], c["lognormal"], seed=7)
    return A, part, c["nsub"]


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_factor_entries_match_dense_cholesky(N, name, prec):
    A, part, nsub = _case(name)
    h = N.nsp_build(A, part, nsub, k=4, p=2, precision=prec)
    tol = 1e-10 if prec == "fp64" else 1e-4
    sizes = [int((part == b).sum()) for b in range(nsub)] + [int((part < 0).sum())]
    biggest = 0
    for b, nb in enumerate(sizes):
        order, L = h.get_factor(b, nb)
        ref = np.linalg.cholesky(A[order][:, order].toarray())
        err = colwise_err(L, ref)
        assert err < tol, (b, err)
        # rows of the largest front: the structural column count of L (first column of a
        # supernode = its front's rows)
        biggest = max(biggest, int((L != 0).sum(axis=0).max()))
    if name == "cluster3d":
        assert biggest >= BIG_FRONT, biggest
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("s", [1, 3, 16, 26, 80])
def test_factor_solves_match_oracle(N, torch, name, prec, s):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    h = N.nsp_build(A, part, nsub, k=4, p=2, precision=prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    rng = np.random.default_rng(s)
    tol = 1e-10 if prec == "fp64" else 5e-4
    for which, n, ref_solve in ((0, D.n_I, D.solve_I), (1, D.n_G, D.solve_G)):
        B = rng.standard_normal((n, s))
        Bd = torch.tensor(B, dtype=dt, device="cuda")
        Xd = torch.empty_like(Bd)
        h.factor_solve(which, Bd, Xd)
        torch.cuda.synchronize()
        X = Xd.double().cpu().numpy()
        ref = ref_solve(B.astype(np.float32).astype(np.float64) if prec == "fp32" else B)
        err = colwise_err(X.reshape(n, s), ref.reshape(n, s))
        assert err < tol, (which, err)
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("s", [1, 5, 16, 80])
def test_schur_apply_matches_oracle(N, torch, name, prec, s):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    h = N.nsp_build(A, part, nsub, k=4, p=2, precision=prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    X = np.random.default_rng(100 + s).standard_normal((D.n_G, s))
    Xd = torch.tensor(X, dtype=dt, device="cuda")
    Yd = torch.empty_like(Xd)
    h.schur_apply(Xd, Yd)
    torch.cuda.synchronize()
    ref = D.apply_S_gamma(X.astype(np.float32).astype(np.float64) if prec == "fp32" else X)
    tol = 1e-9 if prec == "fp64" else 1e-3
    err = colwise_err(Yd.double().cpu().numpy(), ref)
    assert err < tol, err
    h.destroy()


@pytest.mark.parametrize("sched", ["resident", "global", "smem"])
@pytest.mark.parametrize("name", ["tiny3d", "ragged2d", "cluster3d"])
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("s", [1, 7, 80, 160])
def test_both_sweep_schedulers_match_oracle(N, torch, monkeypatch, sched, name, prec, s):
    # the block-resident sweep (one CTA per block), the dependency-driven persistent sweep and
    # the sweeps without dependency waits ("smem": for one right-hand side each block's
    # vectors in shared memory, for several one CTA per block and 32-column slice, widths
    # that are not a multiple of 4 falling back to the block-resident sweep) compute the same
    # A_I^{-1} B, A_G^{-1} B and S_Gamma X; each is forced here (the autotuner keeps only the
    # fastest)
    monkeypatch.setenv("NSP_SWEEP", sched)
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    h = N.nsp_build(A, part, nsub, k=4, p=2, precision=prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    cast = (lambda M: M) if prec == "fp64" else (lambda M: M.astype(np.float32).astype(np.float64))
    tol = 1e-10 if prec == "fp64" else 5e-4
    B = cast(np.random.default_rng(40 + s).standard_normal((D.n_I, s)))
    Bd = torch.tensor(B, dtype=dt, device="cuda")
    Xd = torch.empty_like(Bd)
    h.factor_solve(0, Bd, Xd)
    X = cast(np.random.default_rng(50 + s).standard_normal((D.n_G, s)))
    Xg = torch.tensor(X, dtype=dt, device="cuda")
    Yg = torch.empty_like(Xg)
    h.schur_apply(Xg, Yg)
    Zg = torch.empty_like(Xg)
    h.factor_solve(1, Xg, Zg)
    torch.cuda.synchronize()
    err = colwise_err(Xd.double().cpu().numpy().reshape(D.n_I, s), D.solve_I(B))
    assert err < tol, err
    err = colwise_err(Zg.double().cpu().numpy().reshape(D.n_G, s), D.solve_G(X))
    assert err < tol, err
    err = colwise_err(Yg.double().cpu().numpy().reshape(D.n_G, s), D.apply_S_gamma(X))
    assert err < (1e-9 if prec == "fp64" else 1e-3), err
    h.destroy()


def test_gaussian_sketch_matches_oracle_generator(N, torch):
    n = 100003
    out = torch.empty(n, dtype=torch.float64, device="cuda")
    N.nsp_gaussian(987654321123, n, out)
    torch.cuda.synchronize()
    ref = philox.gaussian(987654321123, n)
    assert np.allclose(out.cpu().numpy(), ref, rtol=1e-12, atol=1e-12)


@pytest.mark.parametrize("name", ["tiny3d", "ragged2d"])
def test_build_parity_fp64(N, name):
    # same sketch on both sides: block PCG iterations equal, E, Y, Sigma and M2 agree
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    G = np.random.default_rng(3).standard_normal((D.n_G, k + p))
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision="fp64", sketch=G, drop_tol=1e-12,
                    keep_intermediates=True)
    M, info = O.build_m2(D, G, k, 0.1, form="S_gamma", drop_tol=1e-12)
    gi = h.info()
    assert gi["it_inner"] == info["it_inner"]
    assert gi["rank"] == len(info["eig_T"][:k])
    assert np.allclose(h.get_intermediate(0), G)
    assert colwise_err(h.get_intermediate(1), info["X"]) < 1e-7
    assert colwise_err(h.get_intermediate(2), info["Y"]) < 1e-7
    Z, S = h.get_basis()
    assert np.allclose(S, info["eig_T"][:k], rtol=1e-8)
    # M2 as an operator: Z Sigma Z^T (signs/rotations of eigenvectors are arbitrary)
    assert operator_err(Z, S, M.Z, M.Sigma) < 1e-7
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_apply_m2_matches_oracle(N, torch, name, prec):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    G = np.random.default_rng(5).standard_normal((D.n_G, k + p))
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=G,
                    drop_tol=1e-12 if prec == "fp64" else 1e-6)
    M, _ = O.build_m2(D, G, k, 0.1, drop_tol=1e-12 if prec == "fp64" else 1e-6)
    r = np.random.default_rng(6).standard_normal(D.n_G)
    rd = torch.tensor(r, dtype=torch.float64, device="cuda")
    zd = torch.empty_like(rd)
    h.apply(rd, zd)
    tol = 1e-7 if prec == "fp64" else 5e-3
    err = colwise_err(zd.cpu().numpy(), M.apply(r))
    assert err < tol, err
    h.destroy()


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("prec,form", [("fp64", "schur"), ("fp32", "full"), ("fp64", "full")])
def test_solve_parity(N, torch, name, prec, form):
    A, part, nsub = _case(name)
    D = O.DBBD(A, part, nsub)
    k, p = 6, 4
    G = np.random.default_rng(8).standard_normal((D.n_G, k + p))
    x_star = np.random.default_rng(9).standard_normal(A.shape[0])
    b = A @ x_star
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=G, outer_form=form)
    M, _ = O.build_m2(D, G, k, 0.1)
    c = {}
    x_ref, it_ref, _ = O.solve(D, M.apply, b, rtol=1e-8, coeffs=c)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=1e-8, maxit=500)
    x = xd.cpu().numpy()
    assert O.relative_residual(A, x, b) < 1e-8 * 10
    assert abs(inf["it_pcg"] - it_ref) <= 2, (inf["it_pcg"], it_ref)
    # condition estimate of M2 S_Gamma from the outer PCG's Lanczos coefficients (both sides
    # stop at 1e-8, where the extreme Ritz values have converged)
    lmin, lmax, kappa = O.kappa_estimate(c["alpha"], c["beta"])
    ktol = 1e-6 if (prec == "fp64" and inf["it_pcg"] == it_ref) else 5e-2
    assert abs(inf["kappa_est"] - kappa) <= ktol * kappa, (inf["kappa_est"], kappa)
    assert abs(inf["lambda_max_est"] - lmax) <= ktol * lmax
    # the residual tolerance leaves x free up to kappa(A) * 1e-8 relative, on both sides:
    # the GPU solution is entry-wise as close to the exact x* as the oracle's (within 10x)
    assert colwise_err(x, x_star) <= 10 * max(colwise_err(x_ref, x_star), 1e-10)
    # host buffers go through the same entry point
    xh = np.zeros_like(b)
    inf2 = h.solve(np.ascontiguousarray(b), xh, rtol=1e-8, maxit=500)
    assert np.allclose(xh, x, rtol=1e-12, atol=1e-12)
    h.destroy()


def test_not_spd_block_reported(N):
    A, part, nsub = _case("tiny2d")
    B = A.tolil()
    i = int(np.nonzero(part == 1)[0][3])
    B[i, i] = -abs(B[i, i])
    with pytest.raises(N.NspError) as e:
        N.nsp_build(B.tocsr(), part, nsub, k=4, p=2, precision="fp64")
    assert e.value.status == 3


def test_singular_c_matches_oracle(N):
    # A separator three nodes thick: its middle column touches no interior node, so A_IG has
    # zero columns, rank(A_GI S_I^{-1} A_IG) <= 18 < s = 24 and C = G^T Y is singular: step 7
    # must drop eigenvalues (the EVD path of the Nyström core, not the Cholesky shortcut).
    shape = (21, 9)
    A = F.diffusion_matrix(shape)
    ix = np.arange(A.shape[0]) % shape[0]          # x fastest
    part = np.where(ix < 9, 0, np.where(ix > 11, 1, -1)).astype(np.int32)
    D = O.DBBD(A, part, 2)
    k, p = 12, 12
    G = np.random.default_rng(21).standard_normal((D.n_G, k + p))
    M, info = O.build_m2(D, G, k, 0.1, form="S_gamma", drop_tol=1e-12)
    assert info["rank_C"] < k + p
    h = N.nsp_build(A, part, 2, k=k, p=p, precision="fp64", sketch=G, drop_tol=1e-12)
    gi = h.info()
    assert gi["it_inner"] == info["it_inner"]
    assert gi["rank"] == len(info["eig_T"][:k])
    Z, S = h.get_basis()
    assert np.allclose(S, info["eig_T"][:gi["rank"]], rtol=1e-8)
    assert operator_err(Z, S, M.Z, M.Sigma) < 1e-7
    h.destroy()
