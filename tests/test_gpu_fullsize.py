"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

The 64^3 lognormal workload (n = 262,144, 32 blocks, k = 64, p = 16, FP32 inner solves) and
two matrices of the 64-matrix anisotropic batch are too large for element-by-element oracle
comparison of every output, so these tests check sampled outputs the oracle computes one by
one, and properties that hold at any size:
* S_Gamma applied to two sampled columns, and A_I^{-1} applied to one, against the oracle's
  sparse-direct results (FP32 tolerance);
* the outer solve reaches ||b - A x|| / ||b|| <= 1e-8 and the oracle's outer iteration count
  within +-2 (the oracle runs the same Algorithm 2 with the same sketch in FP64), also for
  M_{2A-DEF}, M3 and the S_I inner form.
"""

import numpy as np
import pytest

import fixtures as F
import oracle as O

from ._util import lib_or_build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def N():
    return lib_or_build()


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


@pytest.fixture(scope="module")
def cfg1():
    P = F.make_problem(1, 0)
    D = O.DBBD(P.A, P.part, P.nsub)
    return P, D


def _rel(a, b):
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def test_fullsize_schur_and_interior_solves_sampled(N, torch, cfg1):
    P, D = cfg1
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, precision="fp32")
    s = P.s
    rng = np.random.default_rng(31)
    X = rng.standard_normal((P.n_gamma, s)).astype(np.float32)
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.empty_like(Xd)
    h.schur_apply(Xd, Yd)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy()
    for j in (0, s - 1):
        ref = D.apply_S_gamma(X[:, j].astype(np.float64))
        assert _rel(Y[:, j].astype(np.float64), ref) < 2e-4, j
    # A_I^{-1} on one column (interior order of the C ABI = the oracle's block order)
    b = rng.standard_normal(D.n_I)
    bd = torch.tensor(b.astype(np.float32), device="cuda")
    xd = torch.empty_like(bd)
    h.factor_solve(0, bd, xd)
    torch.cuda.synchronize()
    assert _rel(xd.double().cpu().numpy(), D.solve_I(b)) < 2e-4
    h.destroy()


def test_fullsize_solve_matches_oracle_iterations(N, torch, cfg1):
    P, D = cfg1
    G = F.make_sketch(P.n_gamma, P.s, 1, 0)
    _, b = F.make_rhs(P, 1, 0)
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                    precision="fp32", sketch=G)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=P.rtol, maxit=500)
    x = xd.cpu().numpy()
    assert O.relative_residual(P.A, x, b) < 1e-8
    M, info = O.build_m2(D, G, P.k, P.eps_inner)
    _, it_ref, _ = O.solve(D, M.apply, b, rtol=P.rtol)
    assert abs(inf["it_inner"] - info["it_inner"]) <= 1, (inf["it_inner"], info["it_inner"])
    assert abs(inf["it_pcg"] - it_ref) <= 2, (inf["it_pcg"], it_ref)
    h.destroy()


@pytest.mark.parametrize("variant,form", [("m2_adef", "s_gamma"), ("m2", "s_i"), ("m3", "s_gamma")])
def test_fullsize_variants_match_oracle_iterations(N, torch, cfg1, variant, form):
    # the §4.3 variants and the S_I inner form at the benchmark size, same sketch both sides
    # (M3: an interior sketch of n_interior x s)
    P, D = cfg1
    _, b = F.make_rhs(P, 1, 0)
    if variant == "m3":
        G = np.random.default_rng(77).standard_normal((D.n_I, P.s))
        M, info = O.build_m3(D, G, P.k, P.eps_inner)
    else:
        G = F.make_sketch(P.n_gamma, P.s, 1, 0)
        M, info = O.build_m2(D, G, P.k, P.eps_inner, form="S_I" if form == "s_i" else "S_gamma",
                             variant="M2_ADEF" if variant == "m2_adef" else "M2")
    _, it_ref, _ = O.solve(D, M.apply, b, rtol=P.rtol)
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                    precision="fp32", sketch=G, variant=variant, inner_form=form)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=P.rtol, maxit=500)
    assert O.relative_residual(P.A, xd.cpu().numpy(), b) < 1e-8
    assert abs(inf["it_inner"] - info["it_inner"]) <= 1, (inf["it_inner"], info["it_inner"])
    assert abs(inf["it_pcg"] - it_ref) <= 2, (inf["it_pcg"], it_ref)
    h.destroy()


def test_fullsize_batch_sampled_matrices(N, torch):
    specs = F.batched_problem_specs()
    probs = [F.problem_from_spec(sp) for sp in specs]
    bs = [F.make_rhs(Pm, 2, i)[1] for i, Pm in enumerate(probs)]
    Gs = [F.make_sketch(Pm.n_gamma, Pm.s, 2, i) for i, Pm in enumerate(probs)]
    k, p = probs[0].k, probs[0].p
    h = N.nsp_build_batched([(Pm.A, Pm.part, Pm.nsub) for Pm in probs], k=k, p=p,
                            eps_inner=probs[0].eps_inner, precision="fp32",
                            sketch=np.concatenate(Gs, axis=0))
    b = np.concatenate(bs)
    x = np.zeros_like(b)
    infos = h.solve_batched(b, x, rtol=1e-8, maxit=1000)
    off = np.concatenate([[0], np.cumsum([Pm.n for Pm in probs])])
    for m in range(len(probs)):
        xm = x[off[m]:off[m + 1]]
        assert O.relative_residual(probs[m].A, xm, bs[m]) < 1e-8, m
    # two sampled matrices against the oracle (smallest and largest of the batch)
    sizes = [Pm.n for Pm in probs]
    for m in (int(np.argmin(sizes)), int(np.argmax(sizes))):
        Pm = probs[m]
        D = O.DBBD(Pm.A, Pm.part, Pm.nsub)
        M, info = O.build_m2(D, Gs[m], k, Pm.eps_inner)
        _, it_ref, _ = O.solve(D, M.apply, bs[m], rtol=1e-8)
        assert abs(infos[m]["it_inner"] - info["it_inner"]) <= 1, m
        assert abs(infos[m]["it_pcg"] - it_ref) <= 2, (m, infos[m]["it_pcg"], it_ref)
    h.destroy()
