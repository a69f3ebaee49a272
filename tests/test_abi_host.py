"""C-ABI checks that need no GPU: every declared symbol is exported, and the host-only
analysis (validation, DBBD check, orderings, symbolic factorization) behaves."""

import ctypes
import os
import re

import numpy as np
import pytest
import scipy.sparse as sp

import fixtures as F

from ._util import lib_or_build, tiny_problem

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "nsp.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(nsp_[a-z_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    N = lib_or_build()
    names = declared_functions()
    assert len(names) >= 15
    L = ctypes.CDLL(N.LIB_PATH)
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing
    assert set(N.EXPORTS) == set(names)


def test_status_strings():
    N = lib_or_build()
    for code in range(10):
        assert N.lib().nsp_status_string(code)


def _dense_nnz_chol(A, order):
    M = A[order][:, order].toarray()
    L = np.linalg.cholesky(M)
    return int((np.abs(L) > 0).sum())


@pytest.mark.parametrize("shape,nsub", [((12, 11), 2), ((9, 8, 7), 4), ((20, 20), 4)])
def test_symbolic_counts_match_dense_cholesky(shape, nsub):
    # with the caller's elimination order, nnz(L) of every interior block equals the nonzero
    # count of the dense Cholesky factor of the permuted block (no cancellation in SPD
    # diffusion matrices with positive weights)
    N = lib_or_build()
    A, part, perm = tiny_problem(shape, nsub)
    info = N.nsp_analyze(A, part, nsub, perm)
    ref = 0
    for b in range(nsub):
        order = [g for g in perm if part[g] == b]
        ref += _dense_nnz_chol(A, order)
    assert info["nnz_L_interior"] == ref
    assert info["n_gamma"] == int((part < 0).sum())
    assert info["n_interior"] + info["n_gamma"] == A.shape[0]
    # nnz(L_G) is at least the lower triangle of A_G and at most dense
    G = np.nonzero(part < 0)[0]
    AG = A[G][:, G]
    assert (AG.nnz + len(G)) // 2 <= info["nnz_L_gamma"] <= len(G) * (len(G) + 1) // 2


def test_library_ordering_without_perm_is_valid():
    N = lib_or_build()
    A, part, _ = tiny_problem((16, 16), 4)
    info = N.nsp_analyze(A, part, 4, None)
    dense = sum(int((part == b).sum()) * (int((part == b).sum()) + 1) // 2 for b in range(4))
    assert 0 < info["nnz_L_interior"] < dense


def _expect(N, code, A, part, nsub, perm=None):
    with pytest.raises(N.NspError) as e:
        N.nsp_analyze(A, part, nsub, perm)
    assert e.value.status == code


def test_rejects_malformed_inputs():
    N = lib_or_build()
    A, part, perm = tiny_problem((8, 8), 2)
    # coupled blocks -> NOT_DBBD
    bad = part.copy()
    bad[bad < 0] = 0
    _expect(N, 2, A, bad, 2)
    # asymmetric pattern
    B = A.tolil()
    B[0, 5] = 1.0
    _expect(N, 1, B.tocsr(), part, 2)
    # missing diagonal
    C = A.tolil()
    C[3, 3] = 0.0
    C = C.tocsr()
    C.eliminate_zeros()
    _expect(N, 1, C, part, 2)
    # part out of range
    bad = part.copy()
    bad[0] = 7
    _expect(N, 1, A, bad, 2)
    # perm that is not a permutation of the interior unknowns
    _expect(N, 1, A, part, 2, perm[:-1].tolist() + [perm[0]])
    # empty interface
    _expect(N, 1, A, np.zeros_like(part), 1)


def test_short_sketch_refused_before_the_library_reads_it():
    import paper_2101_12164_gb300 as N
    A, part, _ = tiny_problem((9, 8), 2, None)
    n_g, n_i = int((part < 0).sum()), int((part >= 0).sum())
    with pytest.raises(ValueError):
        N.nsp_build(A, part, 2, k=4, p=2, sketch=np.zeros((n_g, 5)))
    with pytest.raises(ValueError):      # M3 reads an interior sketch
        N.nsp_build(A, part, 2, k=4, p=2, sketch=np.zeros((n_g, 6)), variant="m3")
    with pytest.raises(ValueError):
        N.nsp_build_batched([(A, part, 2), (A, part, 2)], k=4, p=2,
                            sketch=np.zeros((n_g, 6)))
    with pytest.raises(ValueError):      # the nested sketch of the recursive A_Gamma
        N.nsp_build(A, part, 2, k=4, p=2, gamma_part=np.array([0, 0, 0, -1, 1, 1, 1, 1]),
                    gamma_nblocks=2, gamma_k=1, gamma_p=1, gamma_sketch=np.zeros(1))
    N._check_sketch(dict(k=4, p=2, sketch=np.zeros((n_i, 6)), variant="m3"), n_g, n_i)
    N._check_sketch(dict(k=4, p=2, sketch=np.zeros((n_g, 6))), n_g, n_i)


def _build_status(N, A, part, nsub, batched=False, **fields):
    keep = []
    csr = N._csr_struct(A, keep)
    ps = N._part_struct(part, nsub, None, keep)
    prm = N.make_params(k=4, p=2, stream=0)
    for f, v in fields.items():
        setattr(prm, f, v)
    h = ctypes.c_void_p()
    if batched:
        csrs, parts = (N.nsp_csr * 1)(csr), (N.nsp_partition * 1)(ps)
        st = N.lib().nsp_build_batched(1, csrs, parts, ctypes.byref(prm), ctypes.byref(h))
    else:
        st = N.lib().nsp_build(ctypes.byref(csr), ctypes.byref(ps), ctypes.byref(prm),
                               ctypes.byref(h))
    if st == 0:
        N.lib().nsp_destroy(h)
    return st


def test_parameters_checked_on_the_host_before_device_work():
    # these statuses come back without a GPU: the checks run before any allocation
    N = lib_or_build()
    A, part, _ = tiny_problem((9, 8), 2, None)
    bad = [dict(k=0), dict(p=-1), dict(variant=7), dict(q=-1), dict(q=17),
           dict(inner_form=3), dict(precision=5)]
    for f in bad:
        assert _build_status(N, A, part, 2, **f) == 1, f          # NSP_ERR_INVALID_ARG
    assert _build_status(N, A, part, 2, k=200, p=100) == 9         # NSP_ERR_UNSUPPORTED
    for f in (dict(variant=1), dict(variant=2), dict(q=1), dict(k=60, p=40)):
        assert _build_status(N, A, part, 2, batched=True, **f) == 9, f
    # valid requests pass the checks (then build, or fail later at the device on a CPU machine)
    for f in (dict(), dict(variant=3), dict(q=2), dict(inner_form=1)):
        assert _build_status(N, A, part, 2, **f) not in (1, 9), f
    # the recursive A_G: gamma_levels in {0, 1}; a split is required; M2, S_Gamma form, q = 0;
    # single handles only
    gp = np.zeros(int((part < 0).sum()), dtype=np.int32)
    g = dict(gamma_levels=1, gamma_nblocks=1, gamma_part=N._ptr(gp))
    assert _build_status(N, A, part, 2, gamma_levels=2) == 1
    assert _build_status(N, A, part, 2, gamma_levels=1) == 1                 # no split
    assert _build_status(N, A, part, 2, **dict(g, gamma_nblocks=0)) == 1
    assert _build_status(N, A, part, 2, **dict(g, gamma_k=0)) == 1
    assert _build_status(N, A, part, 2, **dict(g, gamma_k=200, gamma_p=100)) == 9
    for f in (dict(variant=1), dict(variant=2), dict(variant=4), dict(inner_form=1), dict(q=1)):
        assert _build_status(N, A, part, 2, **dict(g, **f)) == 9, f
    assert _build_status(N, A, part, 2, batched=True, **g) == 9
    gv = np.array([0, 0, 0, -1, 1, 1, 1, 1], dtype=np.int32)   # the 8-node interface line
    assert gv.size == gp.size
    assert _build_status(N, A, part, 2, gamma_levels=1, gamma_nblocks=2, gamma_part=N._ptr(gv),
                         gamma_k=1, gamma_p=0) not in (1, 9)
