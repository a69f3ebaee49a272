"""Batched handles (nsp_build_batched / nsp_solve_batched): many independent systems in one
handle, every quantity of Algorithm 2 and of the outer PCG per matrix.

Each matrix of a batch must behave as if it had been built and solved alone: the block
PCG stops after the same number of iterations as the oracle's for that matrix (same
sketch), the low-rank term Z Sigma Z^T matches the oracle's M2, and the outer PCG reaches
the tolerance in the oracle's iteration count (+-2). The batch mixes sizes, 2D and 3D
problems and contrast levels, so matrices stop at different iterations.
"""

import numpy as np
import pytest

import oracle as O

from ._util import colwise_err, lib_or_build, operator_err, tiny_problem

pytestmark = pytest.mark.gpu

BATCH = [
    dict(shape=(13, 11), nsub=2, lognormal=(3.0, 1.5)),
    dict(shape=(9, 8, 7), nsub=4, lognormal=(2.0, 1.5)),
    dict(shape=(37, 29), nsub=4, lognormal=(5.0, 2.0)),
    dict(shape=(21, 19), nsub=4, lognormal=None),
    dict(shape=(10, 9, 8), nsub=2, lognormal=(4.0, 1.0)),
]
K, PO = 6, 4


@pytest.fixture(scope="module")
def N():
    return lib_or_build()


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


@pytest.fixture(scope="module")
def batch():
    mats, dbbd, sketches, xs, bs = [], [], [], [], []
    for i, c in enumerate(BATCH):
        A, part, _ = tiny_problem(c["shape"], c["nsub"], c["lognormal"], seed=20 + i)
        D = O.DBBD(A, part, c["nsub"])
        mats.append((A, part, c["nsub"]))
        dbbd.append(D)
        sketches.append(np.random.default_rng(100 + i).standard_normal((D.n_G, K + PO)))
        x = np.random.default_rng(200 + i).standard_normal(A.shape[0])
        xs.append(x)
        bs.append(A @ x)
    refs = []
    for D, G, b in zip(dbbd, sketches, bs):
        M, info = O.build_m2(D, G, K, 0.1, form="S_gamma", drop_tol=1e-12)
        _, it, _ = O.solve(D, M.apply, b, rtol=1e-8)
        refs.append((M, info, it))
    return dict(mats=mats, dbbd=dbbd, G=sketches, b=bs, refs=refs)


def _offsets(sizes):
    return np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_batched_build_and_solve_match_oracle_per_matrix(N, torch, batch, prec):
    G = np.concatenate(batch["G"], axis=0)
    h = N.nsp_build_batched(batch["mats"], k=K, p=PO, precision=prec, sketch=G,
                            drop_tol=1e-12 if prec == "fp64" else 1e-6)
    b = np.concatenate(batch["b"])
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    infos = h.solve_batched(bd, xd, rtol=1e-8, maxit=500)
    x = xd.cpu().numpy()
    noff = _offsets([A.shape[0] for A, _, _ in batch["mats"]])
    goff = _offsets([D.n_G for D in batch["dbbd"]])
    Z, S = h.get_basis()
    for m, ((A, _, _), (M, info, it_ref)) in enumerate(zip(batch["mats"], batch["refs"])):
        inf = infos[m]
        xm = x[noff[m]:noff[m + 1]]
        assert O.relative_residual(A, xm, batch["b"][m]) < 1e-7, m
        assert inf["final_residual"] < 1e-7
        assert abs(inf["it_pcg"] - it_ref) <= 2, (m, inf["it_pcg"], it_ref)
        if prec == "fp64":
            assert inf["it_inner"] == info["it_inner"], (m, inf["it_inner"], info["it_inner"])
            assert inf["rank"] == len(info["eig_T"][:K])
            Zm = Z[goff[m]:goff[m + 1]]
            r = inf["rank"]
            assert np.allclose(S[m, :r], info["eig_T"][:r], rtol=1e-8)
            assert np.all(S[m, r:] == 0)
            assert operator_err(Zm, S[m], M.Z, M.Sigma) < 1e-7, m
        else:
            assert abs(inf["it_inner"] - info["it_inner"]) <= 1
    # host buffers go through the same entry point
    xh = np.zeros_like(b)
    infos_h = h.solve_batched(b, xh, rtol=1e-8, maxit=500)
    assert [i["it_pcg"] for i in infos_h] == [i["it_pcg"] for i in infos]
    assert np.allclose(xh, x, rtol=0, atol=1e-12 * np.abs(x).max())
    h.destroy()


def test_batched_equals_single_handles(N, torch, batch):
    # the batch's arithmetic per matrix is the single handle's (same sketch, FP64)
    G = np.concatenate(batch["G"], axis=0)
    h = N.nsp_build_batched(batch["mats"], k=K, p=PO, precision="fp64", sketch=G)
    b = np.concatenate(batch["b"])
    x = np.zeros_like(b)
    infos = h.solve_batched(b, x, rtol=1e-10, maxit=500)
    noff = _offsets([A.shape[0] for A, _, _ in batch["mats"]])
    for m, (A, part, nsub) in enumerate(batch["mats"]):
        h1 = N.nsp_build(A, part, nsub, k=K, p=PO, precision="fp64", sketch=batch["G"][m],
                         outer_form="full")
        x1 = np.zeros(A.shape[0])
        i1 = h1.solve(batch["b"][m], x1, rtol=1e-10, maxit=500)
        assert i1["it_inner"] == infos[m]["it_inner"]
        assert i1["rank"] == infos[m]["rank"]
        assert abs(i1["it_pcg"] - infos[m]["it_pcg"]) <= 1
        assert colwise_err(x[noff[m]:noff[m + 1]], x1) < 1e-7
        h1.destroy()
    h.destroy()


def test_batched_apply_matches_oracle_m2(N, torch, batch):
    G = np.concatenate(batch["G"], axis=0)
    h = N.nsp_build_batched(batch["mats"], k=K, p=PO, precision="fp64", sketch=G)
    rs = [np.random.default_rng(300 + m).standard_normal(D.n_G) for m, D in enumerate(batch["dbbd"])]
    rd = torch.tensor(np.concatenate(rs), dtype=torch.float64, device="cuda")
    zd = torch.empty_like(rd)
    h.apply(rd, zd)
    z = zd.cpu().numpy()
    goff = _offsets([D.n_G for D in batch["dbbd"]])
    for m, (M, _, _) in enumerate(batch["refs"]):
        assert colwise_err(z[goff[m]:goff[m + 1]], M.apply(rs[m])) < 1e-7, m
    h.destroy()


def test_batched_zero_rhs_and_rebuild(N, torch, batch):
    # a matrix with b = 0 stops at once with x = 0 while the others iterate; a rebuild with
    # every value doubled halves the solution
    mats = batch["mats"][:3]
    G = np.concatenate(batch["G"][:3], axis=0)
    h = N.nsp_build_batched(mats, k=K, p=PO, precision="fp64", sketch=G)
    bs = [batch["b"][0], np.zeros(mats[1][0].shape[0]), batch["b"][2]]
    b = np.concatenate(bs)
    x = np.zeros_like(b)
    infos = h.solve_batched(b, x, rtol=1e-9, maxit=500)
    n0, n1 = mats[0][0].shape[0], mats[1][0].shape[0]
    assert infos[1]["it_pcg"] == 0
    assert np.all(x[n0:n0 + n1] == 0)
    assert infos[0]["it_pcg"] > 0 and infos[2]["it_pcg"] > 0
    vals = np.concatenate([A.data for A, _, _ in mats]) * 2.0
    h.rebuild(vals, on_device=False)
    x2 = np.zeros_like(b)
    h.solve_batched(b, x2, rtol=1e-9, maxit=500)
    assert colwise_err(x2, 0.5 * x) < 1e-6
    h.destroy()


def test_batched_handle_refuses_single_solve(N, batch):
    h = N.nsp_build_batched(batch["mats"][:2], k=K, p=PO, precision="fp64")
    n = sum(A.shape[0] for A, _, _ in batch["mats"][:2])
    with pytest.raises(N.NspError) as e:
        h.solve(np.ones(n), np.zeros(n))
    assert e.value.status == 1
    h.destroy()
