"""Pins of the FP64 oracle against what the paper and the mathematics fix.

None of these checks re-types the oracle's own formula: each compares the oracle with an
independent characterisation (closed forms, block inverses of A, textbook identities,
finite termination, the Nyström definition, spectral inclusions stated in the paper).
"""

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

import fixtures as F
import oracle as O


def tiny(shape=(8, 8), nsub=2, lognormal=None, seed=0):
    coef = None
    if lognormal is not None:
        rng = np.random.default_rng(seed)
        coef = F.lognormal_field(F.grid_coords(shape), lognormal[0], lognormal[1], rng)
    A = F.diffusion_matrix(shape, coef)
    part, _ = F.nd_partition(shape, nsub)
    return A, part


# ---------------------------------------------------------------- fixtures
@pytest.mark.parametrize("N", [5, 9, 12])
def test_poisson2d_closed_form_eigenvalues(N):
    A = F.diffusion_matrix((N, N)).toarray()
    i = np.arange(1, N + 1)
    lam = (4 - 2 * np.cos(i[:, None] * np.pi / (N + 1))
           - 2 * np.cos(i[None, :] * np.pi / (N + 1))).ravel()
    assert np.allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(lam), atol=1e-12)


def test_poisson3d_closed_form_eigenvalues():
    N = 5
    A = F.diffusion_matrix((N, N, N)).toarray()
    c = 2 - 2 * np.cos(np.arange(1, N + 1) * np.pi / (N + 1))
    lam = (c[:, None, None] + c[None, :, None] + c[None, None, :]).ravel()
    assert np.allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(lam), atol=1e-12)


def test_diffusion_is_spd_and_symmetric():
    A, _ = tiny((7, 6, 5), 2, lognormal=(2.0, 2.0))
    D = A.toarray()
    assert np.allclose(D, D.T)
    assert np.linalg.eigvalsh(D).min() > 0
    assert A.has_sorted_indices


def test_partition_is_dbbd_and_config0_sizes():
    P = F.make_problem(0)
    assert P.n == 4096 and P.n_gamma == 127
    assert sorted(int((P.part == b).sum()) for b in range(4)) == [961, 992, 992, 1024]
    coo = P.A.tocoo()
    pr, pc = P.part[coo.row], P.part[coo.col]
    both = (pr >= 0) & (pc >= 0)
    assert np.all(pr[both] == pc[both])          # no coupling between subdomains
    # the interior order lists every interior node once, block by block
    assert np.array_equal(np.sort(P.perm), np.nonzero(P.part >= 0)[0])
    assert np.all(np.diff(P.part[P.perm]) >= 0)


def test_dbbd_rejects_coupled_blocks():
    A, part = tiny((6, 6), 2)
    part = part.copy()
    part[part < 0] = 0      # separator merged into block 0 -> blocks 0 and 1 couple
    with pytest.raises(O.NotDBBD):
        O.DBBD(A, part, 2)


# ---------------------------------------------------------------- Schur complements
def test_schur_gamma_is_inverse_of_gamma_block_of_Ainv():
    A, part = tiny((9, 8), 4, lognormal=(3.0, 1.5))
    D = O.DBBD(A, part)
    Ainv = np.linalg.inv(A.toarray())
    S = D.dense_S_gamma()
    assert np.allclose(S @ Ainv[np.ix_(D.gamma, D.gamma)], np.eye(D.n_G), atol=1e-10)
    # block elimination (eq. A_LDLT): A [x_I; x_G] = [0; f]  =>  S_Gamma x_G = f
    f = np.random.default_rng(1).standard_normal(D.n_G)
    rhs = np.zeros(D.n)
    rhs[D.gamma] = f
    x = np.linalg.solve(A.toarray(), rhs)
    assert np.allclose(D.apply_S_gamma(x[D.gamma]), f, atol=1e-10)


def test_schur_interior_is_inverse_of_interior_block_of_Ainv():
    A, part = tiny((8, 7), 2, lognormal=(3.0, 1.0))
    D = O.DBBD(A, part)
    Ainv = np.linalg.inv(A.toarray())
    SI = D.dense_S_I()
    assert np.allclose(SI @ Ainv[np.ix_(D.interior, D.interior)], np.eye(D.n_I), atol=1e-10)


def test_smw_identity():
    A, part = tiny((8, 8), 2, lognormal=(2.0, 1.0))
    D = O.DBBD(A, part)
    AGinv = np.linalg.inv(D.A_G.toarray())
    lhs = np.linalg.inv(D.dense_S_gamma())
    rhs = AGinv + AGinv @ D.A_GI.toarray() @ np.linalg.inv(D.dense_S_I()) @ D.A_IG.toarray() @ AGinv
    assert np.allclose(lhs, rhs, rtol=1e-9, atol=1e-12)


def test_first_level_spectrum_and_eigen_map():
    # lambda(A_G^{-1} S_G) in (0, 1] (§2.3) and the map lambda -> 1/lambda - 1 (§4.1)
    A, part = tiny((9, 9), 4, lognormal=(3.0, 1.0))
    D = O.DBBD(A, part)
    S = D.dense_S_gamma()
    AG = D.A_G.toarray()
    lam = sla.eigh(S, AG, eigvals_only=True)
    assert lam.min() > 0 and lam.max() <= 1 + 1e-12
    B = D.A_GI.toarray() @ np.linalg.inv(D.dense_S_I()) @ D.A_IG.toarray()
    mu = np.sort(sla.eigh(B, AG, eigvals_only=True))
    assert np.allclose(mu, np.sort(1.0 / lam - 1.0), rtol=1e-8, atol=1e-8)


# ---------------------------------------------------------------- (block) CG
def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Q * ev) @ Q.T


def test_pcg_finite_termination_and_error_bound():
    # in exact arithmetic CG ends after (number of distinct eigenvalues) steps; with 6
    # well separated eigenvalues this survives rounding
    n = 30
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    A6 = (Q * np.repeat([1.0, 2.0, 5.0, 9.0, 20.0, 50.0], 5)) @ Q.T
    xs = rng.standard_normal(n)
    x, it, hist = O.pcg(lambda v: A6 @ v, lambda v: v, A6 @ xs, rtol=1e-11, maxit=200)
    assert it <= 7
    assert np.allclose(x, xs, atol=1e-8)
    # CG error bound of the introduction (eq. k-th_error_cg) at every step
    A = _spd(n, 3, cond=50.0)
    b = A @ xs
    lam = np.linalg.eigvalsh(A)
    kappa = lam.max() / lam.min()
    rate = (np.sqrt(kappa) - 1) / (np.sqrt(kappa) + 1)
    e0 = np.sqrt(xs @ A @ xs)
    for k in range(1, 15):
        xk, _, _ = O.pcg(lambda v: A @ v, lambda v: v, b, rtol=0.0, maxit=k)
        ek = np.sqrt((xs - xk) @ A @ (xs - xk))
        assert ek <= 2 * e0 * rate ** k * (1 + 1e-10)


def test_block_pcg_finite_termination():
    n, s = 24, 4
    A = _spd(n, 5, cond=1e2)
    B = np.random.default_rng(6).standard_normal((n, s))
    X, it, hist = O.block_pcg(lambda V: A @ V, lambda V: V, B, tol=1e-10, maxit=100)
    assert it <= int(np.ceil(n / s)) + 2
    assert np.linalg.norm(A @ X - B) / np.linalg.norm(B) < 1e-9


def test_block_pcg_single_column_is_pcg():
    n = 40
    A = _spd(n, 7, cond=1e3)
    Minv = np.diag(1.0 / np.diag(A))
    b = np.random.default_rng(8).standard_normal(n)
    for k in (1, 3, 7, 12):
        xb, itb, _ = O.block_pcg(lambda V: A @ V, lambda V: Minv @ V, b[:, None], tol=0.0,
                                 maxit=k)
        x, it, _ = O.pcg(lambda v: A @ v, lambda v: Minv @ v, b, rtol=0.0, maxit=k)
        assert itb == it == k
        assert np.allclose(xb[:, 0], x, rtol=1e-9, atol=1e-12)


def test_block_pcg_breakdown_free_on_duplicate_columns():
    n = 30
    A = _spd(n, 9, cond=1e2)
    b = np.random.default_rng(10).standard_normal((n, 2))
    B = np.concatenate([b, b, 2 * b[:, :1]], axis=1)      # rank 2, 5 columns
    X, it, _ = O.block_pcg(lambda V: A @ V, lambda V: V, B, tol=1e-10, maxit=100)
    assert np.all(np.isfinite(X))
    assert np.linalg.norm(A @ X - B) / np.linalg.norm(B) < 1e-9
    assert O.orth(B).shape[1] == 2


def test_pcg_matches_scipy_cg():
    A, part = tiny((10, 10), 2, lognormal=(3.0, 1.0))
    b = np.random.default_rng(11).standard_normal(A.shape[0])
    x, it, _ = O.pcg(lambda v: A @ v, lambda v: v, b, rtol=1e-12, maxit=1000)
    xr = spla.spsolve(sp.csc_matrix(A), b)
    assert np.allclose(x, xr, rtol=1e-8, atol=1e-10)


# ---------------------------------------------------------------- Nyström (§2.1, Alg. 1)
def test_nystrom_core_matches_definition():
    # Nystrom approximation of eq. (NystromApprox): B G (G^T B G)^+ (B G)^T
    rng = np.random.default_rng(12)
    n, s = 40, 10
    Bm = _spd(n, 13, cond=1e6)
    G = rng.standard_normal((n, s))
    Y = Bm @ G
    U, Sig, info = O.nystrom_core(G, Y, k=s, eps_rel=1e-14)
    ref = Y @ np.linalg.pinv(G.T @ Y) @ Y.T
    assert np.allclose((U * Sig) @ U.T, ref, rtol=1e-7, atol=1e-8 * np.abs(ref).max())
    assert np.allclose(U.T @ U, np.eye(U.shape[1]), atol=1e-10)
    assert np.all(np.diff(Sig) <= 0)


def test_nystrom_exact_for_low_rank():
    rng = np.random.default_rng(14)
    n, r, s = 50, 6, 10
    V = np.linalg.qr(rng.standard_normal((n, r)))[0]
    ev = np.array([50.0, 20.0, 9.0, 4.0, 2.0, 1.0])
    Bm = (V * ev) @ V.T
    G = rng.standard_normal((n, s))
    U, Sig, info = O.nystrom_core(G, Bm @ G, k=8)
    assert U.shape[1] == r                      # rank min(r, k) (§2.1)
    assert np.allclose(Sig, ev, rtol=1e-9)
    assert np.allclose((U * Sig) @ U.T, Bm, atol=1e-9)
    # k < r: exact top-k eigenvectors
    U3, S3, _ = O.nystrom_core(G, Bm @ G, k=3)
    assert np.allclose(np.abs(U3.T @ V[:, :3]), np.eye(3), atol=1e-9)


# ---------------------------------------------------------------- M2 (§4.3, Alg. 2)
def _small_problem():
    A, part = tiny((12, 12), 2, lognormal=(4.0, 1.0), seed=3)
    return A, part, O.DBBD(A, part)


@pytest.mark.parametrize("form", ["S_gamma", "S_I"])
def test_m2_exact_when_rank_captured(form):
    # n_Gamma = 12, s = 14 >= rank(A_GI S_I^{-1} A_IG): M2 = S_Gamma^{-1}, PCG in 1 step
    A, part, D = _small_problem()
    s = D.n_G + 2
    G = np.random.default_rng(15).standard_normal((D.n_G, s))
    M, info = O.build_m2(D, G, k=s, eps_inner=1e-14, form=form, eps_rel=1e-13)
    Sinv = np.linalg.inv(D.dense_S_gamma())
    assert np.allclose(M.dense(), Sinv, rtol=1e-7, atol=1e-9 * np.abs(Sinv).max())
    b = np.random.default_rng(16).standard_normal(D.n)
    x, it, _ = O.solve(D, M.apply, b, rtol=1e-10)
    assert it <= 2
    assert O.relative_residual(A, x, b) < 1e-9


def test_m2_spectral_inclusion_and_monotone_in_k():
    # 0 <= B_k <= B  =>  A_G^{-1} <= M2 <= S_G^{-1}: Lambda(M2 S) in [lambda_min(A_G^{-1}S), 1]
    A, part = tiny((14, 14), 4, lognormal=(3.0, 1.5), seed=4)
    D = O.DBBD(A, part)
    S = D.dense_S_gamma()
    lam1 = sla.eigh(S, D.A_G.toarray(), eigvals_only=True).min()
    G = np.random.default_rng(17).standard_normal((D.n_G, D.n_G))
    prev = lam1 * (1 - 1e-9)
    for k in (2, 5, 10, 20):
        M, _ = O.build_m2(D, G[:, :k + 4], k=k, eps_inner=1e-14)
        mu = np.linalg.eigvals(M.dense() @ S).real
        assert mu.min() >= lam1 * (1 - 1e-7) and mu.max() <= 1 + 1e-7
        assert mu.min() >= prev * (1 - 1e-7)
        prev = mu.min()


def test_forms_agree_for_exact_inner_solves():
    A, part, D = _small_problem()
    G = np.random.default_rng(18).standard_normal((D.n_G, 6))
    _, a = O.build_m2(D, G, k=4, eps_inner=1e-14, form="S_gamma")
    _, b = O.build_m2(D, G, k=4, eps_inner=1e-14, form="S_I")
    _, c = O.build_m2(D, G, k=4, eps_inner=1e-14, form="S_gamma_naive")
    assert np.allclose(a["Y"], b["Y"], rtol=1e-8, atol=1e-10)
    assert np.allclose(c["Y"], b["Y"], rtol=1e-6, atol=1e-8)


def test_solve_and_full_space_form_on_config0():
    P = F.make_problem(0)
    D = O.DBBD(P.A, P.part, P.nsub)
    G = F.make_sketch(D.n_G, P.s, 0)
    _, b = F.make_rhs(P, 0)
    M, info = O.build_m2(D, G, P.k, P.eps_inner)
    x, it, _ = O.solve(D, M.apply, b, rtol=1e-8)
    x2, it2, _ = O.solve_full_space(D, M.apply, b, rtol=1e-8)
    x1, it1, _ = O.solve(D, D.solve_G, b, rtol=1e-8)
    assert O.relative_residual(P.A, x, b) < 1e-7
    assert abs(it - it2) <= 1
    assert it < it1                                       # two-level beats S1
    assert np.allclose(x, spla.spsolve(sp.csc_matrix(P.A), b), rtol=1e-6, atol=1e-7)


# ---------------------------------------------------------------- M_{2A-DEF} (§4.3)
def _rgamma_definition(D, U):
    # eq. (deflation_comp_from_low_rank) and eq. (our_two_level_preconditioner) written with
    # the dense Cholesky factor A_G = R^T R and the transformed basis Ub = R^{-T} U
    R = np.linalg.cholesky(D.A_G.toarray()).T
    Ri = np.linalg.inv(R)
    S = D.dense_S_gamma()
    Sh = Ri.T @ S @ Ri
    Ub = Ri.T @ U
    E = Ub.T @ Sh @ Ub
    Q = Ub @ np.linalg.solve(E, Ub.T)
    Pdef = np.eye(D.n_G) - Q @ Sh + Q
    return Ri @ Pdef @ Ri.T


def test_m2adef_equals_rgamma_form_of_the_paper():
    A, part = tiny((14, 14), 4, lognormal=(3.0, 1.5), seed=5)
    D = O.DBBD(A, part)
    G = np.random.default_rng(21).standard_normal((D.n_G, 9))
    M, info = O.build_m2(D, G, k=6, eps_inner=0.1, variant="M2_ADEF")
    ref = _rgamma_definition(D, info["U"])
    assert np.allclose(M.dense(), ref, rtol=1e-9, atol=1e-11 * np.abs(ref).max())


def test_m2adef_deflation_identity():
    # Z^T S_G M = Z^T for any basis Z: the correction is S_G-orthogonal to span(Z)
    A, part = tiny((12, 12), 2, lognormal=(4.0, 1.0), seed=6)
    D = O.DBBD(A, part)
    Z = np.random.default_rng(22).standard_normal((D.n_G, 4))
    M = O.M2ADEF(D, Z)
    S = D.dense_S_gamma()
    assert np.allclose(Z.T @ S @ M.dense(), Z.T, rtol=1e-9, atol=1e-9 * np.abs(Z).max())


def test_m2adef_moves_deflated_eigenvalues_to_one():
    # Z = k exact generalized eigenvectors of (S_G, A_G) for the smallest eigenvalues:
    # Lambda(M S_G) = {1 (k times)} and the other n_G - k eigenvalues unchanged
    A, part = tiny((14, 14), 4, lognormal=(3.0, 1.5), seed=7)
    D = O.DBBD(A, part)
    S = D.dense_S_gamma()
    lam, V = sla.eigh(S, D.A_G.toarray())
    k = 5
    mu = np.sort(np.linalg.eigvals(O.M2ADEF(D, V[:, :k]).dense() @ S).real)
    want = np.sort(np.concatenate([np.ones(k), lam[k:]]))
    assert np.allclose(mu, want, rtol=1e-8, atol=1e-9)


def test_m2adef_exact_when_rank_captured():
    A, part, D = _small_problem()
    s = D.n_G + 2
    G = np.random.default_rng(23).standard_normal((D.n_G, s))
    M, _ = O.build_m2(D, G, k=s, eps_inner=1e-14, eps_rel=1e-13, variant="M2_ADEF")
    Sinv = np.linalg.inv(D.dense_S_gamma())
    assert np.allclose(M.dense(), Sinv, rtol=1e-7, atol=1e-9 * np.abs(Sinv).max())
    b = np.random.default_rng(24).standard_normal(D.n)
    x, it, _ = O.solve(D, M.apply, b, rtol=1e-10)
    assert it <= 2
    assert O.relative_residual(A, x, b) < 1e-9


def test_m2adef_iterations_close_to_m2_on_config0():
    # Table (compare_variations): M2 and M_{2A-DEF} need nearly the same outer iterations
    P = F.make_problem(0)
    D = O.DBBD(P.A, P.part, P.nsub)
    G = F.make_sketch(D.n_G, P.s, 0)
    _, b = F.make_rhs(P, 0)
    M2, _ = O.build_m2(D, G, P.k, P.eps_inner)
    Ma, _ = O.build_m2(D, G, P.k, P.eps_inner, variant="M2_ADEF")
    x2, it2, _ = O.solve(D, M2.apply, b, rtol=1e-8)
    xa, ita, _ = O.solve(D, Ma.apply, b, rtol=1e-8)
    assert O.relative_residual(P.A, xa, b) < 1e-7
    assert abs(ita - it2) <= 2


# ---------------------------------------------------------------- power iteration (§2.1)
def _dense_B(A, D):
    # the matrix Algorithm 2 approximates, B = A_GI S_I^{-1} A_IG (§4.3 eq.
    # (internal_term_lr_approximation_1)), with S_I^{-1} the interior block of A^{-1}
    Ainv = np.linalg.inv(A.toarray())
    SIinv = Ainv[np.ix_(D.interior, D.interior)]
    return D.A_GI.toarray() @ SIinv @ D.A_IG.toarray()


@pytest.mark.parametrize("q", [1, 2])
def test_power_nystrom_matches_definition(q):
    # eq. (NystromApprox) with eq. (power), G = B^q Omega formed without orthonormalization
    A, part = tiny((12, 12), 2, lognormal=(4.0, 1.0), seed=8)
    D = O.DBBD(A, part)
    B = _dense_B(A, D)
    s = 5
    Om = np.random.default_rng(31).standard_normal((D.n_G, s))
    G = np.linalg.matrix_power(B, q) @ Om
    BG = B @ G
    ref = BG @ np.linalg.solve(G.T @ BG, BG.T)
    M, info = O.build_m2(D, Om, k=s, eps_inner=1e-14, eps_rel=1e-13, q=q)
    got = (info["U"] * M.Sigma) @ info["U"].T
    assert len(info["it_power"]) == q
    assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref)


def test_power_iteration_sharpens_the_approximation():
    A, part = tiny((14, 14), 4, lognormal=(3.0, 1.5), seed=9)
    D = O.DBBD(A, part)
    B = _dense_B(A, D)
    Om = np.random.default_rng(32).standard_normal((D.n_G, 8))
    err = []
    for q in (0, 1, 2):
        M, info = O.build_m2(D, Om, k=6, eps_inner=1e-14, eps_rel=1e-13, q=q)
        err.append(np.linalg.norm(B - (info["U"] * M.Sigma) @ info["U"].T, 2))
    assert err[2] < err[0] and err[1] < err[0]
    # the rank-6 truncation can do no better than the best rank-6 approximation
    lam = np.sort(np.linalg.eigvalsh(B))[::-1]
    assert min(err) >= lam[6] * (1 - 1e-8)


# ---------------------------------------------------------------- M3 (§4.3)
def _dense_SIinv(A, D):
    Ainv = np.linalg.inv(A.toarray())
    return Ainv[np.ix_(D.interior, D.interior)]


def test_m3_nystrom_of_SIinv_matches_definition():
    # k = s, exact solves: V Sigma V^T = F (G^T F)^{-1} F^T with F = S_I^{-1} G (eq. (NystromApprox))
    A, part = tiny((12, 12), 2, lognormal=(4.0, 1.0), seed=10)
    D = O.DBBD(A, part)
    B = _dense_SIinv(A, D)
    G = np.random.default_rng(41).standard_normal((D.n_I, 7))
    F = B @ G
    ref = F @ np.linalg.solve(G.T @ F, F.T)
    M, info = O.build_m3(D, G, k=7, eps_inner=1e-14, eps_rel=1e-13)
    got = (info["V"] * M.Sigma) @ info["V"].T
    assert np.linalg.norm(got - ref) <= 1e-7 * np.linalg.norm(ref)
    # Zh = A_G^{-1} A_GI V, independent dense products
    Zh = np.linalg.solve(D.A_G.toarray(), D.A_GI.toarray() @ info["V"])
    assert np.allclose(M.Z, Zh, rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("variant", ["M3", "M3_ADEF"])
def test_m3_exact_when_sketch_spans_interior(variant):
    # s = n_I: V Sigma V^T = S_I^{-1}, so by SMW (§4.1 eq. (S-1)) M3 = S_Gamma^{-1}
    A, part = tiny((6, 6), 2, lognormal=(3.0, 1.0), seed=11)
    D = O.DBBD(A, part)
    G = np.random.default_rng(42).standard_normal((D.n_I, D.n_I))
    M, _ = O.build_m3(D, G, k=D.n_I, eps_inner=1e-14, eps_rel=1e-14, variant=variant)
    Sinv = np.linalg.inv(D.dense_S_gamma())
    assert np.allclose(M.dense(), Sinv, rtol=1e-6, atol=1e-8 * np.abs(Sinv).max())
    b = np.random.default_rng(43).standard_normal(D.n)
    x, it, _ = O.solve(D, M.apply, b, rtol=1e-10)
    assert it <= 2
    assert O.relative_residual(A, x, b) < 1e-9


def test_m3_spectral_inclusion():
    # 0 <= V Sigma V^T <= S_I^{-1} for exact solves => A_G^{-1} <= M3 <= S_G^{-1}
    A, part = tiny((14, 14), 4, lognormal=(3.0, 1.5), seed=12)
    D = O.DBBD(A, part)
    S = D.dense_S_gamma()
    lam1 = sla.eigh(S, D.A_G.toarray(), eigvals_only=True).min()
    G = np.random.default_rng(44).standard_normal((D.n_I, 20))
    M, _ = O.build_m3(D, G, k=12, eps_inner=1e-14)
    mu = np.linalg.eigvals(M.dense() @ S).real
    assert mu.min() >= lam1 * (1 - 1e-7) and mu.max() <= 1 + 1e-7
    assert mu.min() > lam1 * (1 + 1e-6)          # and it does improve on S1


def test_kept_columns_drops_exactly_the_dependent_columns():
    # the drop rule shared by the block-PCG orthonormalization and the A-DEF basis: a column
    # is dropped iff it lies in the span of the columns kept before it (brute-force ranks)
    rng = np.random.default_rng(51)
    a, b, c = rng.standard_normal((3, 40))
    W = np.stack([a, b, a + 2 * b, np.zeros(40), c, 3 * c - b], axis=1)
    keep = O.kept_columns(W.T @ W, 1e-12)
    assert keep == [0, 1, 4]
    for j in range(W.shape[1]):
        prev = [i for i in keep if i < j]
        grows = np.linalg.matrix_rank(W[:, prev + [j]]) > np.linalg.matrix_rank(W[:, prev]) \
            if prev else np.linalg.norm(W[:, j]) > 0
        assert (j in keep) == bool(grows), j


# ---------------------------------------------------------------- Proposition 4.1 (§4.2)
def test_expected_effective_condition_within_proposition_4_1():
    # I - H = R^{-T} S_G R^{-1} (A_G = R^T R); the oracle's Nyström (Algorithm 1, q = 0, no
    # truncation) of B = R^{-T} A_GI S_I^{-1} A_IG R^{-1} = (I - H)^{-1} - I (eq. (Rt_S-1_R))
    # gives U (n_G x (k+p)); P = I - (I-H) U E^{-1} U^T. Over 60 seeds the mean sqrt of the
    # effective condition number of P (I-H) stays below eq. (tight_bound), with lambda_1..k the
    # k smallest eigenvalues of I - H (so that gamma_{t,k} <= 1) and E(c) of eq. (constant).
    A, part = tiny((14, 14), 4, lognormal=(3.0, 1.5), seed=13)
    D = O.DBBD(A, part)
    n = D.n_G
    R = np.linalg.cholesky(D.A_G.toarray()).T
    Ri = np.linalg.inv(R)
    IH = Ri.T @ D.dense_S_gamma() @ Ri
    IH = 0.5 * (IH + IH.T)
    lam = np.sort(np.linalg.eigvalsh(IH))            # lam[i-1] = lambda_i, increasing
    k, p = min(4, int(np.sum(lam <= 0.5))), 4          # the proposition assumes lambda_k <= 1/2
    assert k >= 2 and lam[k - 1] <= 0.5
    B = np.linalg.inv(IH) - np.eye(n)
    B = 0.5 * (B + B.T)
    Ec = np.sqrt(k / (p - 1)) + np.e * np.sqrt((k + p) * (n - k)) / p
    gam = lambda t: (1 / lam[k] - 1) / (1 / lam[t - 1] - 1)
    bound = np.sqrt(2) * min(max(Ec * np.sqrt(2 * t) * np.sqrt(gam(t)), 1.0)
                             * np.sqrt(lam[-1] / lam[t]) for t in range(1, k + 1))
    vals = []
    for seed in range(60):
        G = np.random.default_rng(1000 + seed).standard_normal((n, k + p))
        U, _, _ = O.nystrom_core(G, B @ G, k + p, eps_rel=1e-13)
        E = U.T @ IH @ U
        P = np.eye(n) - IH @ U @ np.linalg.solve(E, U.T)
        mu = np.sort(np.abs(np.linalg.eigvals(P @ IH)))[U.shape[1]:]   # drop the deflated zeros
        vals.append(np.sqrt(mu[-1] / mu[0]))
    assert np.mean(vals) <= bound
    # the bound is loose here (about 16); what the Nyström basis must also do is align with the
    # smallest eigenvectors of I - H: deflating it cuts sqrt(kappa) well below the first
    # level's (a basis of the largest ones, from Nyström of I - H itself, would not)
    assert np.max(vals) <= np.sqrt(lam[-1] / lam[0]) * (1 + 1e-8)
    assert np.mean(vals) < 0.8 * np.sqrt(lam[-1] / lam[0])


# ---------------------------------------------------------------- paper trends (§5), config 0
def test_block_cg_beats_per_column_cg_and_loose_inner_tolerance_is_harmless():
    # §5.1: block CG on the k + p right-hand sides needs fewer iterations than CG on each
    # column; §5.2: it_PCG is flat for eps_{S_I} in [0.01, 0.3]
    P = F.make_problem(0)
    D = O.DBBD(P.A, P.part, P.nsub)
    G = F.make_sketch(D.n_G, P.s, 0)
    _, b = F.make_rhs(P, 0)
    Fh = D.A_GI @ D.solve_I(D.A_IG @ G)
    _, it_block, _ = O.block_pcg(D.apply_S_gamma, D.solve_G, Fh, 0.1)
    it_cols = [O.pcg(D.apply_S_gamma, D.solve_G, Fh[:, j], rtol=0.1)[1]
               for j in range(Fh.shape[1])]
    assert it_block < max(it_cols)
    its = []
    for eps in (0.01, 0.1, 0.3):
        M, _ = O.build_m2(D, G, P.k, eps)
        its.append(O.solve(D, M.apply, b, rtol=1e-8)[1])
    assert max(its) - min(its) <= 2, its


# ---------------------------------------------------------------- M1 (§4.1)
def test_m1_without_truncation_is_m2_on_the_transformed_sketch():
    # k = s, exact solves: F (G^T F)^+ F^T with F = R^{-T} Y and G^T F = (R^{-1} G)^T Y, so
    # R^{-1} Ub Sigma Ub^T R^{-T} = A_G^{-1} Y C^+ Y^T A_G^{-1}: M1(G) = M2(R^{-1} G)
    A, part = tiny((14, 14), 4, lognormal=(3.0, 1.5), seed=14)
    D = O.DBBD(A, part)
    G = np.random.default_rng(61).standard_normal((D.n_G, 7))
    M1, info = O.build_m1(D, G, k=7, eps_inner=1e-14, eps_rel=1e-13)
    Gp = np.linalg.solve(np.linalg.cholesky(D.A_G.toarray()).T, G)
    M2, _ = O.build_m2(D, Gp, k=7, eps_inner=1e-14, eps_rel=1e-13)
    ref = M2.dense()
    assert np.allclose(M1.dense(), ref, rtol=1e-7, atol=1e-9 * np.abs(ref).max())
    # eq. (Rt_S-1_R): R S_G^{-1} R^T = I + R^{-T} A_GI S_I^{-1} A_IG R^{-1}; Ub Sigma Ub^T is its
    # Nyström approximation, so it never exceeds R S_G^{-1} R^T - I
    R = info["R"]
    B = R @ np.linalg.inv(D.dense_S_gamma()) @ R.T - np.eye(D.n_G)
    Bk = (info["U"] * M1.Sigma) @ info["U"].T
    assert np.linalg.eigvalsh(0.5 * (B - Bk + (B - Bk).T)).min() > -1e-8 * np.abs(B).max()


def test_m1_exact_when_rank_captured_and_spectral_inclusion():
    A, part, D = _small_problem()
    s = D.n_G + 2
    G = np.random.default_rng(62).standard_normal((D.n_G, s))
    M, _ = O.build_m1(D, G, k=s, eps_inner=1e-14, eps_rel=1e-13)
    Sinv = np.linalg.inv(D.dense_S_gamma())
    assert np.allclose(M.dense(), Sinv, rtol=1e-7, atol=1e-9 * np.abs(Sinv).max())
    A2, part2 = tiny((14, 14), 4, lognormal=(3.0, 1.5), seed=4)
    D2 = O.DBBD(A2, part2)
    S = D2.dense_S_gamma()
    lam1 = sla.eigh(S, D2.A_G.toarray(), eigvals_only=True).min()
    G2 = np.random.default_rng(63).standard_normal((D2.n_G, 9))
    M2, _ = O.build_m1(D2, G2, k=5, eps_inner=1e-14)
    mu = np.linalg.eigvals(M2.dense() @ S).real
    assert mu.min() >= lam1 * (1 - 1e-7) and mu.max() <= 1 + 1e-7
