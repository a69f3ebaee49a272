"""Edge cases of the CUDA path against the oracle: the widest sketch block, a single
interior block, a one-node block, ragged block sizes, a zero right-hand side, and the
requests the method cannot serve (s above the supported width, k + p above n_Gamma,
no interface)."""

import numpy as np
import pytest

import fixtures as F
import oracle as O

from ._util import lib_or_build, operator_err, tiny_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    return lib_or_build()


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


def _parity(N, torch, A, part, nsub, k, p, prec="fp64", its_tol=2):
    D = O.DBBD(A, part, nsub)
    G = np.random.default_rng(7).standard_normal((D.n_G, k + p))
    b = A @ np.random.default_rng(8).standard_normal(A.shape[0])
    h = N.nsp_build(A, part, nsub, k=k, p=p, precision=prec, sketch=G)
    M, info = O.build_m2(D, G, k, 0.1)
    _, it_ref, _ = O.solve(D, M.apply, b, rtol=1e-8)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=1e-8, maxit=500)
    assert O.relative_residual(A, xd.cpu().numpy(), b) < 1e-7
    if prec == "fp64":
        assert inf["it_inner"] == info["it_inner"]
    assert abs(inf["it_pcg"] - it_ref) <= its_tol, (inf["it_pcg"], it_ref)
    return h, D, M


def test_widest_sketch_block(N, torch):
    # s = k + p = 256, the widest block of the sweeps and of the s x s core
    A, part, _ = tiny_problem((80, 80), 16, (3.0, 1.0), seed=2)
    h, D, M = _parity(N, torch, A, part, 16, 200, 56)
    Z, S = h.get_basis()
    # 256-column inner block PCG and Nyström core in FP64 on both sides, with different
    # factor orderings and Cholesky-QR variants (equal in exact arithmetic): the eigenvalues
    # agree to 1e-7; the tail of the 200 kept eigenvalues is clustered (relative gaps ~1e-2),
    # so the eigenvectors carry rounding of order eps * cond / gap: 1e-5 as an operator
    assert np.allclose(S, M.Sigma, rtol=1e-7)
    assert operator_err(Z, S, M.Z, M.Sigma) < 1e-5
    h.destroy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_core_widths_with_shared_memory_factor(N, torch, prec):
    # s = 136 (88 < s <= 160): the s x s Cholesky factor of the block-PCG steps and the FP32
    # Jacobi matrices of the Nyström core live in shared memory, the other s x s buffers in
    # global memory
    A, part, _ = tiny_problem((70, 70), 16, (3.0, 1.0), seed=4)
    h, D, M = _parity(N, torch, A, part, 16, 120, 16, prec=prec)
    Z, S = h.get_basis()
    if prec == "fp64":
        assert np.allclose(S, M.Sigma, rtol=1e-7)
        assert operator_err(Z, S, M.Z, M.Sigma) < 1e-5
    else:
        assert np.allclose(S, M.Sigma, rtol=1e-2)
    h.destroy()


def test_single_interior_block(N, torch):
    shape = (18, 14)
    A = F.diffusion_matrix(shape)
    ix = np.arange(A.shape[0]) % shape[0]
    part = np.where(ix < 12, 0, -1).astype(np.int32)
    h, _, _ = _parity(N, torch, A, part, 1, 4, 4)
    h.destroy()


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_one_node_block_and_ragged_blocks(N, torch, prec):
    # block 1 is a single node inside a ring of interface nodes; block 0 is the rest
    shape = (15, 15)
    A = F.diffusion_matrix(shape)
    ix = np.arange(A.shape[0]) % shape[0]
    iy = np.arange(A.shape[0]) // shape[0]
    part = np.zeros(A.shape[0], dtype=np.int32)
    ring = (np.abs(ix - 7) <= 1) & (np.abs(iy - 7) <= 1)
    part[ring] = -1
    part[(ix == 7) & (iy == 7)] = 1
    part[ix == 12] = -1           # a second interface line
    part[ix > 12] = 2             # a thin third block (2 columns)
    h, _, _ = _parity(N, torch, A, part, 3, 3, 3, prec=prec)
    h.destroy()


def test_zero_right_hand_side(N, torch):
    A, part, _ = tiny_problem((13, 11), 2, (3.0, 1.5), seed=7)
    h = N.nsp_build(A, part, 2, k=4, p=2, precision="fp32")
    bd = torch.zeros(A.shape[0], dtype=torch.float64, device="cuda")
    xd = torch.full_like(bd, 5.0)
    inf = h.solve(bd, xd)
    assert inf["it_pcg"] == 0
    assert torch.count_nonzero(xd) == 0
    h.destroy()


def test_requests_the_method_cannot_serve(N):
    A, part, _ = tiny_problem((13, 11), 2, (3.0, 1.5), seed=7)
    n_gamma = int((part < 0).sum())
    with pytest.raises(N.NspError) as e:
        N.nsp_build(A, part, 2, k=n_gamma, p=1, precision="fp64")     # k + p > n_Gamma
    assert e.value.status == 1
    B, part2, _ = tiny_problem((60, 60), 16, None, seed=0)
    with pytest.raises(N.NspError) as e:
        N.nsp_build(B, part2, 16, k=200, p=57, precision="fp64")      # s = 257
    assert e.value.status == 9
    # no interface at all: a single block, no Schur complement to approximate
    with pytest.raises(N.NspError) as e:
        N.nsp_build(A, np.zeros(A.shape[0], dtype=np.int32), 1, k=2, p=1, precision="fp64")
    assert e.value.status in (1, 2)
