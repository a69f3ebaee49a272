"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

Workloads: the 64^3 lognormal problem (n = 262,144, 32 blocks, k = 64, p = 16), the 128^3
anisotropic problem (n = 2,097,152, 256 blocks, k = 128, p = 32; the bench workload) and two
matrices of the 64-matrix anisotropic batch, all with FP32 factors and inner solves.

* 64^3: every column of S_Gamma X (80 columns) and a 16-column block of A_I^{-1} B against
  the oracle's sparse-direct results, entry-wise per column; Algorithm 2 and the outer solve
  with the same sketch as the oracle: inner iterations within 1, outer within 2, residual
  <= 1e-8, the Nyström factor Z Sigma Z^T as an operator, the largest principal angle between
  the two bases U, the condition estimate of M2 S_Gamma, and the solution against the
  oracle's.
* 128^3: the oracle takes about twenty minutes there, so its outputs are stored at seeded
  sample rows by tests/golden/make_golden.py (calls only oracle/); the same quantities are
  compared on those rows.

The error bounds used here and reported by bench.py (FP32 inner solves against the FP64
oracle with the same sketch): S_Gamma and A_I^{-1} entries 1e-3 of the column maximum; the
Nyström term as an operator 5e-3 and its sampled entries 1e-2; the largest principal angle
between the bases 0.1 rad; the condition estimate 5 %; the solution as close to the exact x*
as the oracle's within a factor 10.
"""

import json
import os

import numpy as np
import pytest

import fixtures as F
import oracle as O

from ._util import colwise_err, lib_or_build, max_principal_angle, operator_err

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def test_fullsize_schur_and_interior_solves(N, torch, cfg1):
    P, D = cfg1
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, precision="fp32")
    s = P.s
    X = F.make_probe(P.n_gamma, s, 1, 0).astype(np.float32)
    Xd = torch.tensor(X, device="cuda")
    Yd = torch.empty_like(Xd)
    h.schur_apply(Xd, Yd)
    torch.cuda.synchronize()
    ref = D.apply_S_gamma(X.astype(np.float64))
    assert colwise_err(Yd.cpu().numpy(), ref) < 1e-3
    # A_I^{-1} on a 16-column block (interior order of the C ABI = the oracle's block order)
    B = F.make_probe(D.n_I, 16, 1, 1).astype(np.float32)
    Bd = torch.tensor(B, device="cuda")
    Xi = torch.empty_like(Bd)
    h.factor_solve(0, Bd, Xi)
    torch.cuda.synchronize()
    assert colwise_err(Xi.cpu().numpy(), D.solve_I(B.astype(np.float64))) < 1e-3
    h.destroy()


def test_fullsize_build_and_solve_match_oracle(N, torch, cfg1):
    P, D = cfg1
    G = F.make_sketch(P.n_gamma, P.s, 1, 0)
    x_star, b = F.make_rhs(P, 1, 0)
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                    precision="fp32", sketch=G, keep_intermediates=True)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=P.rtol, maxit=500)
    x = xd.cpu().numpy()
    assert O.relative_residual(P.A, x, b) < 1e-8
    M, info = O.build_m2(D, G, P.k, P.eps_inner)
    c = {}
    x_ref, it_ref, _ = O.solve(D, M.apply, b, rtol=P.rtol, coeffs=c)
    assert abs(inf["it_inner"] - info["it_inner"]) <= 1, (inf["it_inner"], info["it_inner"])
    assert abs(inf["it_pcg"] - it_ref) <= 2, (inf["it_pcg"], it_ref)
    # the Nyström factor against the FP64 oracle's with the same sketch
    Z, S = h.get_basis()
    assert operator_err(Z, S, M.Z, M.Sigma) < 5e-3
    U = h.get_intermediate(3)
    U_ref = M.Z.copy()                       # Z = A_G^{-1} U: recover U = A_G Z
    U_ref = D.A_G @ U_ref
    assert max_principal_angle(U, U_ref) < 0.1
    # the condition estimate of M2 S_Gamma and the solution
    _, _, kappa = O.kappa_estimate(c["alpha"], c["beta"])
    assert abs(inf["kappa_est"] - kappa) <= 5e-2 * kappa, (inf["kappa_est"], kappa)
    assert colwise_err(x, x_star) <= 10 * max(colwise_err(x_ref, x_star), 1e-10)
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


def test_fullsize_m1_solves_like_m2(N, torch, cfg1):
    # M1 (§4.1) at the benchmark size: the oracle's M1 needs a dense factor of A_G (n_Gamma
    # in the tens of thousands here), so this checks the GPU form against the outer
    # tolerance and against M2 from the same sketch, which §5 finds about as effective
    P, D = cfg1
    _, b = F.make_rhs(P, 1, 0)
    G = F.make_sketch(P.n_gamma, P.s, 1, 0)
    its = {}
    for variant in ("m2", "m1"):
        h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                        precision="fp32", sketch=G, variant=variant)
        bd = torch.tensor(b, dtype=torch.float64, device="cuda")
        xd = torch.zeros_like(bd)
        its[variant] = h.solve(bd, xd, rtol=P.rtol, maxit=500)["it_pcg"]
        assert O.relative_residual(P.A, xd.cpu().numpy(), b) < 1e-8
        h.destroy()
    assert its["m1"] <= its["m2"] + 5, its


def test_fullsize_recursive_gamma_solves(N, torch, cfg1):
    # the recursive A_G (concluding section; reading of the oracle's recursive_gamma) at the
    # benchmark size: A_G split into 16 blocks by the interface nodes' coordinates, M2' of
    # rank 32. Entry-wise parity is on the small cases (test_gpu_recursive.py); here the outer
    # tolerance is reached and the weaker A_G^{-1} costs a few outer iterations over M2
    P, D = cfg1
    _, b = F.make_rhs(P, 1, 0)
    G = F.make_sketch(P.n_gamma, P.s, 1, 0)
    part2 = F.interface_partition(D.A_G, P.coords[D.gamma], 16)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    its = {}
    for rec in (False, True):
        kw = dict(gamma_part=part2, gamma_nblocks=16, gamma_k=32, gamma_p=16) if rec else {}
        h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                        precision="fp32", sketch=G, **kw)
        xd = torch.zeros_like(bd)
        inf = h.solve(bd, xd, rtol=P.rtol, maxit=500)
        its[rec] = inf["it_pcg"]
        assert O.relative_residual(P.A, xd.cpu().numpy(), b) < 1e-8
        if rec:
            inf2 = h.info()
            assert inf2["n_gamma2"] == int((part2 < 0).sum())
            assert inf2["rank_gamma"] == 32 and inf2["it_inner_gamma"] >= 1
        h.destroy()
    assert its[True] <= its[False] + 10, its


# ------------------------------------------------------------------ 128^3 (stored oracle)
@pytest.fixture(scope="module")
def cfg4():
    with open(os.path.join(GOLDEN, "aniso3d_128.json")) as f:
        gold = json.load(f)
    P = F.make_problem(4, 0)
    return P, gold


def _sampled_err(full, gold_block, rows):
    full = np.asarray(full, dtype=np.float64).reshape(full.shape[0], -1)
    ref = np.asarray(gold_block["values"], dtype=np.float64)
    scale = np.asarray(gold_block["colmax"], dtype=np.float64)
    return float((np.abs(full[rows] - ref).max(axis=0) / scale).max())


def test_fullsize128_schur_and_interior_sampled(N, torch, cfg4):
    P, gold = cfg4
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, precision="fp32")
    inf = h.info()
    assert (inf["n_gamma"], inf["n_interior"]) == (gold["n_gamma"], gold["n_interior"])
    X = F.make_probe(gold["n_gamma"], 2, 4, 0)
    Xd = torch.tensor(X, dtype=torch.float32, device="cuda")
    Yd = torch.empty_like(Xd)
    h.schur_apply(Xd, Yd)
    B = F.make_probe(gold["n_interior"], 2, 4, 1)
    Bd = torch.tensor(B, dtype=torch.float32, device="cuda")
    Xi = torch.empty_like(Bd)
    h.factor_solve(0, Bd, Xi)
    torch.cuda.synchronize()
    assert _sampled_err(Yd.cpu().numpy(), gold["schur"], gold["rows_gamma"]) < 1e-3
    assert _sampled_err(Xi.cpu().numpy(), gold["interior"], gold["rows_interior"]) < 1e-3
    h.destroy()


@pytest.mark.parametrize("sched", ["global", "resident", "smem"])
def test_fullsize128_single_vector_schedulers(N, torch, cfg4, monkeypatch, sched):
    # one right-hand side at a time through each single-vector scheduler (the outer solve's
    # interior sweeps), against the stored oracle columns of A_I^{-1} B
    monkeypatch.setenv("NSP_SWEEP", sched)
    P, gold = cfg4
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, precision="fp32")
    B = F.make_probe(gold["n_interior"], 2, 4, 1)
    for j in range(B.shape[1]):
        Bd = torch.tensor(np.ascontiguousarray(B[:, j]), dtype=torch.float32, device="cuda")
        Xi = torch.empty_like(Bd)
        h.factor_solve(0, Bd, Xi)
        torch.cuda.synchronize()
        ref = {"values": [r[j:j + 1] for r in gold["interior"]["values"]],
               "colmax": gold["interior"]["colmax"][j:j + 1]}
        err = _sampled_err(Xi.cpu().numpy().reshape(-1, 1), ref, gold["rows_interior"])
        assert err < 1e-3, (j, err)
    h.destroy()


def test_fullsize128_build_and_solve_match_oracle(N, torch, cfg4):
    P, gold = cfg4
    G = F.make_sketch(gold["n_gamma"], P.s, 4, 0)
    x_star, b = F.make_rhs(P, 4, 0)
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                    precision="fp32", sketch=G)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=P.rtol, maxit=500)
    x = xd.cpu().numpy()
    g = gold["build"]
    assert O.relative_residual(P.A, x, b) < 1e-8
    assert abs(inf["it_inner"] - g["it_inner"]) <= 1, (inf["it_inner"], g["it_inner"])
    assert abs(inf["it_pcg"] - gold["solve"]["it_pcg"]) <= 2, (inf["it_pcg"], gold["solve"])
    Z, S = h.get_basis()
    assert inf["rank"] == g["rank"]
    assert np.allclose(S, g["sigma"], rtol=1e-2)
    V = F.make_probe(gold["n_gamma"], 4, 4, 2)
    assert _sampled_err((Z * S) @ (Z.T @ V), g["nystrom_term"], gold["rows_gamma"]) < 1e-2
    Vd = torch.tensor(V[:, 0], dtype=torch.float64, device="cuda")
    Md = torch.empty_like(Vd)
    h.apply(Vd, Md)
    torch.cuda.synchronize()
    m2_ref = {"values": [r[:1] for r in g["m2_apply"]["values"]],
              "colmax": g["m2_apply"]["colmax"][:1]}
    assert _sampled_err(Md.cpu().numpy(), m2_ref, gold["rows_gamma"]) < 1e-2
    assert abs(inf["kappa_est"] - gold["solve"]["kappa"]) <= 5e-2 * gold["solve"]["kappa"]
    err_x = float(np.linalg.norm(x - x_star) / np.linalg.norm(x_star))
    assert err_x <= 10 * max(gold["solve"]["err_vs_xstar"], 1e-10), err_x
    h.destroy()


@pytest.mark.parametrize("variant", ["m2_adef", "m3"])
def test_fullsize128_variants_solve(N, torch, cfg4, variant):
    # the §4.3 variants at the 128^3 size (k = 128: the k x k Grams of M_2A-DEF and the
    # interior sketch of M3 run at widths the M2 build does not use): the outer solve
    # reaches 1e-8 (no stored oracle run for these)
    P, gold = cfg4
    _, b = F.make_rhs(P, 4, 0)
    h = N.nsp_build(P.A, P.part, P.nsub, k=P.k, p=P.p, eps_inner=P.eps_inner,
                    precision="fp32", variant=variant)
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    xd = torch.zeros_like(bd)
    inf = h.solve(bd, xd, rtol=P.rtol, maxit=500)
    assert O.relative_residual(P.A, xd.cpu().numpy(), b) < 1e-8
    assert inf["it_pcg"] > 0
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
