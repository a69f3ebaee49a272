"""Pins of the oracle's condition estimate from the outer PCG (oracle.lanczos_tridiagonal,
oracle.kappa_estimate).

What fixes it independently of the code: CG and Lanczos build the same Krylov basis, so the
tridiagonal formed from PCG's coefficients has the Ritz values of the preconditioned
operator M A; after n steps on an n x n system these are exactly its eigenvalues (a dense
eigen-decomposition gives them), and before that the extreme Ritz values lie inside the
spectrum and move outward as steps are added (Cauchy interlacing of nested tridiagonals).
On the 64 x 64 Poisson case (4 subdomains) the estimate from the outer PCG with M2 and with
the first level S1 = A_Gamma is compared with the dense spectrum of M S_Gamma, whose
eigenvalues lie in (0, 1] for S1 (§4.1).
"""

import numpy as np
import pytest
import scipy.linalg as sla

import fixtures as F
import oracle as O


def _spd(n, eigs, seed):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, n)))
    return (Q * eigs) @ Q.T


def test_full_run_gives_the_spectrum_identity_preconditioner():
    # few, well separated eigenvalues: n steps in floating point keep the basis orthogonal
    lam = np.array([1.0, 1.7, 2.9, 4.2, 6.0, 8.5, 11.0, 15.0])
    A = _spd(8, lam, 1)
    f = np.random.default_rng(2).standard_normal(8)
    c = {}
    O.pcg(lambda v: A @ v, lambda r: r.copy(), f, rtol=0.0, maxit=8, coeffs=c)
    assert len(c["alpha"]) == 8 and len(c["beta"]) >= 7
    ritz = np.linalg.eigvalsh(O.lanczos_tridiagonal(c["alpha"], c["beta"]))
    assert np.allclose(ritz, np.sort(lam), rtol=1e-8)
    lmin, lmax, kappa = O.kappa_estimate(c["alpha"], c["beta"])
    assert np.isclose(kappa, lam.max() / lam.min(), rtol=1e-8)


def test_full_run_gives_the_preconditioned_spectrum():
    n = 8
    A = _spd(n, np.geomspace(1.0, 30.0, n), 3)
    M = _spd(n, np.geomspace(0.5, 2.0, n), 4)
    f = np.random.default_rng(5).standard_normal(n)
    c = {}
    O.pcg(lambda v: A @ v, lambda r: M @ r, f, rtol=0.0, maxit=n, coeffs=c)
    ritz = np.linalg.eigvalsh(O.lanczos_tridiagonal(c["alpha"], c["beta"]))
    # eigenvalues of M A = those of the generalized problem A v = lambda M^{-1} v
    ref = sla.eigh(A, np.linalg.inv(M), eigvals_only=True)
    assert np.allclose(ritz, ref, rtol=1e-7)


def test_partial_runs_interlace_inside_the_spectrum():
    lam = np.geomspace(1.0, 1e4, 40)
    A = _spd(40, lam, 6)
    f = np.random.default_rng(7).standard_normal(40)
    c = {}
    O.pcg(lambda v: A @ v, lambda r: r.copy(), f, rtol=0.0, maxit=25, coeffs=c)
    prev = None
    for m in range(2, 26):
        e = np.linalg.eigvalsh(O.lanczos_tridiagonal(c["alpha"][:m], c["beta"][:m - 1]))
        assert e[0] >= lam[0] * (1 - 1e-10) and e[-1] <= lam[-1] * (1 + 1e-10)
        if prev is not None:     # extremes move outward (interlacing)
            assert e[0] <= prev[0] * (1 + 1e-10) and e[-1] >= prev[-1] * (1 - 1e-10)
        prev = e


@pytest.mark.parametrize("prec", ["M2", "S1"])
def test_outer_pcg_estimate_on_poisson_matches_dense_spectrum(prec):
    P = F.make_problem(0)
    D = O.DBBD(P.A, P.part, P.nsub)
    G = F.make_sketch(D.n_G, P.s, 0)
    _, b = F.make_rhs(P, 0)
    if prec == "M2":
        M, _ = O.build_m2(D, G, P.k, P.eps_inner)
        apply_M, dense_M = M.apply, M.dense()
    else:
        apply_M, dense_M = D.solve_G, D.solve_G(np.eye(D.n_G))
    c = {}
    _, it, _ = O.solve(D, apply_M, b, rtol=P.rtol, coeffs=c)
    assert len(c["alpha"]) == it
    lmin, lmax, kappa = O.kappa_estimate(c["alpha"], c["beta"])
    S = D.dense_S_gamma()
    ev = np.sort(np.linalg.eigvals(dense_M @ S).real)
    # extreme Ritz values after a run to 1e-8 are converged to a few parts in 1e3
    assert lmin >= ev[0] * (1 - 1e-8) and lmax <= ev[-1] * (1 + 1e-8)
    assert np.isclose(lmax, ev[-1], rtol=1e-3), (lmax, ev[-1])
    assert np.isclose(lmin, ev[0], rtol=1e-2), (lmin, ev[0])
    assert np.isclose(kappa, ev[-1] / ev[0], rtol=1e-2)
    if prec == "S1":
        assert ev[-1] <= 1.0 + 1e-10   # lambda(A_G^{-1} S_G) in (0, 1] (§4.1)
