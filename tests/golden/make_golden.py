"""Write the stored expected values of the full-size parity tests (calls only oracle/ and
the seeded input generators of fixtures/).

    python tests/golden/make_golden.py 4      # aniso3d_128 -> tests/golden/aniso3d_128.json

The 128^3 workload (n = 2,097,152, 256 subdomains, k = 128, p = 32) takes the FP64 oracle
about twenty minutes on one core (SuperLU factorizations, the 160-column inner block PCG,
the outer PCG), too long to repeat inside a test, so the outputs that the GPU tests compare
are stored here at seeded sample rows:
  schur     : S_Gamma X for a seeded 2-column X (§2.3 eq. (schur_complement));
  interior  : A_I^{-1} B for a seeded 2-column B;
  build     : Algorithm 2 with the seeded sketch G: inner iterations, rank, Sigma, and the
              Nyström term Z Sigma Z^T V and the whole M2 V for a seeded 4-column V;
  solve     : outer PCG iterations, the condition estimate from its coefficients, x at
              sample rows, and the errors of x against the known x*.
Each sampled block also stores its column-wise max |value| over ALL rows (the scale of the
entry-wise comparison).
"""

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import fixtures as F  # noqa: E402
import oracle as O  # noqa: E402

NSAMPLE = 2048


def _sampled(Y, rows):
    Y = np.asarray(Y, dtype=np.float64).reshape(Y.shape[0], -1)
    return {"values": Y[rows].tolist(), "colmax": np.abs(Y).max(axis=0).tolist()}


def make(config):
    t_all = time.perf_counter()
    P = F.make_problem(config, 0)
    x_star, b = F.make_rhs(P, config, 0)
    t0 = time.perf_counter()
    D = O.DBBD(P.A, P.part, P.nsub)
    t_dbbd = time.perf_counter() - t0
    rows_g = F.sample_rows(D.n_G, NSAMPLE, config, 0)
    rows_i = F.sample_rows(D.n_I, NSAMPLE, config, 1)
    rows_x = F.sample_rows(P.n, NSAMPLE, config, 2)
    out = {"workload": P.name, "n": int(P.n), "n_gamma": int(D.n_G), "n_interior": int(D.n_I),
           "nsub": int(P.nsub), "k": int(P.k), "p": int(P.p), "eps_inner": P.eps_inner,
           "rtol": P.rtol, "nsample": NSAMPLE,
           "rows_gamma": rows_g.tolist(), "rows_interior": rows_i.tolist(),
           "rows_full": rows_x.tolist()}
    X = F.make_probe(D.n_G, 2, config, 0)
    out["schur"] = _sampled(D.apply_S_gamma(X), rows_g)
    B = F.make_probe(D.n_I, 2, config, 1)
    out["interior"] = _sampled(D.solve_I(B), rows_i)
    G = F.make_sketch(D.n_G, P.s, config, 0)
    t0 = time.perf_counter()
    M, info = O.build_m2(D, G, P.k, P.eps_inner)
    t_build = time.perf_counter() - t0
    V = F.make_probe(D.n_G, 4, config, 2)
    out["build"] = {"it_inner": int(info["it_inner"]), "rank": int(len(M.Sigma)),
                    "sigma": [float(v) for v in M.Sigma],
                    "nystrom_term": _sampled((M.Z * M.Sigma) @ (M.Z.T @ V), rows_g),
                    "m2_apply": _sampled(M.apply(V), rows_g)}
    c = {}
    t0 = time.perf_counter()
    x, it, hist = O.solve(D, M.apply, b, rtol=P.rtol, coeffs=c)
    t_solve = time.perf_counter() - t0
    lmin, lmax, kappa = O.kappa_estimate(c["alpha"], c["beta"])
    out["solve"] = {"it_pcg": int(it), "lambda_min": lmin, "lambda_max": lmax,
                    "kappa": kappa, "x": _sampled(x, rows_x),
                    "residual": O.relative_residual(P.A, x, b),
                    "err_vs_xstar": float(np.linalg.norm(x - x_star) / np.linalg.norm(x_star))}
    out["oracle_seconds"] = {"dbbd_factor": t_dbbd, "build_m2": t_build, "solve": t_solve,
                             "total": time.perf_counter() - t_all}
    path = os.path.join(HERE, "%s.json" % P.name)
    with open(path, "w") as f:
        json.dump(out, f)
    return path


if __name__ == "__main__":
    print(make(int(sys.argv[1]) if len(sys.argv) > 1 else 4))
