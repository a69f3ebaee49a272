"""nsp_schur_apply_noalloc: the S_Gamma apply for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc at the point where they need the operator, for example
code running while a CUDA stream is being captured into a graph, or code under an allocator
that forbids device allocations. The library serves them with an entry point whose
temporaries live in one fixed device array. This file checks, through the C ABI, that it
returns what nsp_schur_apply returns, on two calls in a row (the array keeps the previous
call's contents), and that a problem too large for the array is refused.
"""

import numpy as np
import pytest

import oracle as O

from ._util import lib_or_build, tiny_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("s", [1, 7])
def test_noalloc_matches_schur_apply(prec, s):
    import torch

    N = lib_or_build()
    A, part, _ = tiny_problem((21, 19), 4, (4.0, 1.5), seed=11)
    h = N.nsp_build(A, part, 4, k=4, p=2, precision=prec)
    dt = torch.float64 if prec == "fp64" else torch.float32
    n_gamma = int((part < 0).sum())
    X0 = np.random.default_rng(40 + s).standard_normal((n_gamma, s))
    X = torch.tensor(X0, dtype=dt, device="cuda")
    Yref = torch.empty_like(X)
    h.schur_apply(X, Yref)  # the allocating entry point (also prepares the sweep plan)
    torch.cuda.synchronize()
    tol = 1e-12 if prec == "fp64" else 1e-5
    scale = float(Yref.abs().max())
    for _ in range(2):
        Y = torch.full_like(X, float("nan"))
        h.schur_apply_noalloc(X, Y)
        torch.cuda.synchronize()
        assert torch.isfinite(Y).all()
        assert float((Y - Yref).abs().max()) <= tol * scale
    # and, like every parity test, against the oracle
    ref = O.DBBD(A, part, 4).apply_S_gamma(X0)
    rel = np.linalg.norm(Y.double().cpu().numpy() - ref) / np.linalg.norm(ref)
    assert rel < (1e-10 if prec == "fp64" else 2e-4)
    h.destroy()


def test_noalloc_refuses_problems_beyond_its_array():
    import torch

    import fixtures as F
    N = lib_or_build()
    P = F.make_problem(0)       # 64 x 64 Poisson: 256 FP64 columns need about 29 MB
    h = N.nsp_build(P.A, P.part, P.nsub, k=4, p=2, precision="fp64")
    X = torch.zeros(P.n_gamma, 256, dtype=torch.float64, device="cuda")
    Y = torch.zeros_like(X)
    with pytest.raises(N.NspError) as e:
        h.schur_apply_noalloc(X, Y)
    assert e.value.status == 1
    h.destroy()
