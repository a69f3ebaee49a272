"""Pins of the oracle's recursive treatment of A_Gamma (concluding section; the reading is in
``oracle.recursive_gamma``): A_Gamma gets a DBBD split of its own and A_Gamma^{-1} becomes the
block elimination of §2.3 eq. (A_LDLT) for that split with the split's M2 as its Schur solve.

What fixes it, independently of its own code:
* with a nested sketch of full width and exact inner solves, the nested M2 is S_C^{-1} (the
  Nyström approximation is exact), so the nested inverse is A_Gamma^{-1} itself (a sparse
  direct solve);
* at any nested rank the nested M2 lies below S_C^{-1} in the Loewner order (Nyström
  approximations underestimate, exact inner solves), and the block elimination is a
  congruence, so A_Gamma~^{-1} is symmetric with the eigenvalues of A_Gamma~^{-1} A_Gamma in
  (0, 1]; a dropped or sign-flipped coupling term breaks the symmetry or the bound;
* with the exact nested inverse the recursive M2 is the plain M2 of Algorithm 2.
"""

import numpy as np
import pytest

import fixtures as F
import oracle as O

from ._util import tiny_problem


def _split(shape, nsub, nsub2, seed=3):
    A, part, _ = tiny_problem(shape, nsub, (3.0, 1.5), seed=seed)
    D = O.DBBD(A, part, nsub)
    coords = F.grid_coords(shape)[D.gamma]
    part2 = F.interface_partition(D.A_G, coords, nsub2)
    return A, D, part2


CASES = [((9, 8, 7), 2, 2), ((12, 11, 9), 4, 4), ((13, 12, 11), 2, 4)]


@pytest.mark.parametrize("shape,nsub,nsub2", CASES)
def test_interface_partition_is_dbbd_of_a_gamma(shape, nsub, nsub2):
    _, D, part2 = _split(shape, nsub, nsub2)
    d2 = O.DBBD(D.A_G, part2, nsub2)          # raises NotDBBD if two blocks couple
    assert d2.n_G > 0 and all(len(b) > 0 for b in d2.blocks)
    assert d2.n_G < D.n_G // 2


@pytest.mark.parametrize("shape,nsub,nsub2", CASES)
def test_nested_inverse_is_exact_at_full_nested_rank(shape, nsub, nsub2):
    _, D, part2 = _split(shape, nsub, nsub2)
    d2 = O.DBBD(D.A_G, part2, nsub2)
    n2 = d2.n_G
    G2 = np.random.default_rng(5).standard_normal((n2, n2))
    Dr, info = O.recursive_gamma(D, part2, nsub2, G2, n2, eps_inner=1e-13)
    B = np.random.default_rng(6).standard_normal((D.n_G, 3))
    X = Dr.solve_G(B)
    ref = D.solve_G(B)
    assert np.abs(X - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("shape,nsub,nsub2", CASES)
def test_nested_inverse_is_spd_and_below_the_exact_inverse(shape, nsub, nsub2):
    _, D, part2 = _split(shape, nsub, nsub2)
    d2 = O.DBBD(D.A_G, part2, nsub2)
    k2 = max(2, d2.n_G // 4)
    G2 = np.random.default_rng(7).standard_normal((d2.n_G, k2 + 2))
    Dr, _ = O.recursive_gamma(D, part2, nsub2, G2, k2, eps_inner=1e-13)
    Minv = Dr.solve_G(np.eye(D.n_G))
    assert np.abs(Minv - Minv.T).max() <= 1e-10 * np.abs(Minv).max()
    AG = D.A_G.toarray()
    # eigenvalues of A_Gamma~^{-1} A_Gamma: positive, at most 1, and not all 1 (the nested
    # approximation is active)
    ev = np.linalg.eigvals(Minv @ AG).real
    assert ev.min() > 0.0
    assert ev.max() <= 1.0 + 1e-8
    assert ev.min() < 1.0 - 1e-3


@pytest.mark.parametrize("shape,nsub,nsub2", CASES[:2])
def test_recursive_m2_is_plain_m2_with_exact_nested_inverse(shape, nsub, nsub2):
    _, D, part2 = _split(shape, nsub, nsub2)
    d2 = O.DBBD(D.A_G, part2, nsub2)
    G2 = np.random.default_rng(8).standard_normal((d2.n_G, d2.n_G))
    Dr, _ = O.recursive_gamma(D, part2, nsub2, G2, d2.n_G, eps_inner=1e-13)
    k, p = 5, 3
    G = np.random.default_rng(9).standard_normal((D.n_G, k + p))
    M, _ = O.build_m2(D, G, k, eps_inner=1e-12)
    Mr, _ = O.build_m2(Dr, G, k, eps_inner=1e-12)
    R = np.random.default_rng(10).standard_normal((D.n_G, 4))
    a, b = M.apply(R), Mr.apply(R)
    assert np.abs(a - b).max() <= 1e-7 * np.abs(a).max()


def test_recursive_m2_outer_pcg_converges():
    A, D, part2 = _split((12, 11, 9), 4, 4)
    d2 = O.DBBD(D.A_G, part2, 4)
    k2 = max(2, d2.n_G // 4)
    G2 = np.random.default_rng(11).standard_normal((d2.n_G, k2 + 2))
    Dr, _ = O.recursive_gamma(D, part2, 4, G2, k2)
    G = np.random.default_rng(12).standard_normal((D.n_G, 8))
    Mr, _ = O.build_m2(Dr, G, 6)
    b = A @ np.random.default_rng(13).standard_normal(A.shape[0])
    x, it, _ = O.solve(Dr, Mr.apply, b, rtol=1e-8)
    assert O.relative_residual(A, x, b) < 1e-7
    # the nested approximation costs iterations over the plain M2 with the same sketch
    M, _ = O.build_m2(D, G, 6)
    _, it0, _ = O.solve(D, M.apply, b, rtol=1e-8)
    assert it >= it0
