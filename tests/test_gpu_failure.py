"""Failure detection of the persistent sweeps without any GPU fault.

Every dependency wait inside a sweep is bounded; when one runs out the sweep raises its abort
flag, every CTA skips its remaining items, the kernel returns and a device timeout is recorded
for the host. nsp_check_timeout_path makes all waits of one sweep unreachable on purpose (a
counter target no launch will reach) with a short bound, and reports what the sweep recorded.
The handle must then keep working and give the same results as before.
"""

import numpy as np
import pytest

from ._util import lib_or_build, tiny_problem

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_unreachable_wait_times_out_and_handle_recovers(prec):
    import torch
    N = lib_or_build()
    A, part, _ = tiny_problem((21, 19), 4, (4.0, 1.5), seed=11)
    h = N.nsp_build(A, part, 4, k=4, p=2, precision=prec)
    b = A @ np.random.default_rng(3).standard_normal(A.shape[0])
    bd = torch.tensor(b, dtype=torch.float64, device="cuda")
    x0 = torch.zeros_like(bd)
    i0 = h.solve(bd, x0, rtol=1e-10)
    assert h.check_timeout_path(1 << 12) == 6          # NSP_ERR_TIMEOUT
    x1 = torch.zeros_like(bd)
    i1 = h.solve(bd, x1, rtol=1e-10)
    assert i1["it_pcg"] == i0["it_pcg"]
    assert torch.equal(x0, x1)
    # and again: the check leaves the plan in a clean state each time
    assert h.check_timeout_path(1 << 10) == 6
    x2 = torch.zeros_like(bd)
    h.solve(bd, x2, rtol=1e-10)
    assert torch.equal(x0, x2)
    h.destroy()
