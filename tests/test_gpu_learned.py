"""The learned sketch proposal on the GPU (nsp_net_*): parity with the FP64 oracle of
oracle/sketch_net.py, the BF16 inference kernel, the Gaussian fallback flag, and what the
trained network gains over the Gaussian sketch on held-out fields.
"""

import numpy as np
import pytest

import fixtures.learned as FL
from oracle import sketch_net as SN

from ._util import colwise_err, lib_or_build

pytestmark = pytest.mark.gpu

D_RAW, N_COORD, N_FREQ, HIDDEN = 9, 2, 4, 16


@pytest.fixture(scope="module")
def N():
    return lib_or_build()


@pytest.fixture(scope="module")
def torch():
    import torch as T
    return T


def _case(s_out=12, n=150, k=5, seed=0):
    rng = np.random.default_rng(seed)
    theta = FL.init_params(seed, D_RAW, N_COORD, N_FREQ, HIDDEN, s_out)
    theta += 0.05 * rng.standard_normal(theta.size)   # non-zero biases too
    attrs = rng.uniform(0.0, 1.0, (n, D_RAW))
    attrs[:, 2:7] = rng.normal(0.0, 2.0, (n, 5))       # log-coefficient-like attributes
    U, _ = np.linalg.qr(rng.standard_normal((n, k)))
    return theta, attrs, U


SHAPE = lambda s: (D_RAW, N_COORD, N_FREQ, HIDDEN, s)  # noqa: E731


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-11), ("fp32", 1e-4)])
def test_forward_matches_oracle(N, torch, prec, tol):
    theta, attrs, _ = _case()
    net = N.SketchNet(theta, D_RAW, N_COORD, N_FREQ, HIDDEN, 12, precision=prec)
    G = torch.empty(attrs.shape[0], 12, dtype=torch.float64, device="cuda")
    net.forward(torch.tensor(attrs, device="cuda"), G)
    ref, _ = SN.forward(theta, attrs, SHAPE(12))
    assert colwise_err(G.cpu().numpy(), ref) < tol
    # host arrays go through the same call
    Gh = np.zeros((attrs.shape[0], 12))
    net.forward(attrs, Gh)
    assert np.array_equal(Gh, G.cpu().numpy())
    net.destroy()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("fp32", 5e-3)])
@pytest.mark.parametrize("mu", [0.0, 0.02])
def test_loss_and_gradient_match_oracle(N, torch, prec, tol, mu):
    theta, attrs, U = _case(seed=1)
    net = N.SketchNet(theta, D_RAW, N_COORD, N_FREQ, HIDDEN, 12, precision=prec, mu=mu)
    L = net.loss_grad(torch.tensor(attrs, device="cuda"), torch.tensor(U, device="cuda"))
    Lref, gref = SN.loss_and_grad(theta, attrs, U, SHAPE(12), mu)
    assert abs(L - Lref) <= tol * abs(Lref)
    assert colwise_err(net.grad(), gref) < tol
    # gradients accumulate over calls until the Adam step clears them
    net.loss_grad(attrs, U, want_loss=False)
    assert colwise_err(net.grad(), 2 * gref) < tol
    net.destroy()


def test_adam_matches_oracle(N, torch):
    theta, attrs, U = _case(seed=2)
    net = N.SketchNet(theta, D_RAW, N_COORD, N_FREQ, HIDDEN, 12, precision="fp64", mu=0.01)
    th, m, v = theta.copy(), np.zeros_like(theta), np.zeros_like(theta)
    for t in range(1, 4):
        net.loss_grad(attrs, U, want_loss=False)
        net.adam_step(3e-3)
        _, g = SN.loss_and_grad(th, attrs, U, SHAPE(12), 0.01)
        th, m, v = SN.adam_step(th, g, m, v, t, 3e-3)
    assert colwise_err(net.params(), th) < 1e-10
    assert colwise_err(net.get(2), m) < 1e-10 and colwise_err(net.get(3), v) < 1e-10
    assert np.all(net.grad() == 0)
    net.destroy()


def test_bf16_sketch_orthonormal_and_rank_flag(N, torch):
    theta, attrs, _ = _case(seed=3)
    net = N.SketchNet(theta, D_RAW, N_COORD, N_FREQ, HIDDEN, 12, precision="fp32")
    ad = torch.tensor(attrs, device="cuda")
    ref, _ = SN.forward(theta, attrs, SHAPE(12))
    # raw output: BF16 embedding and hidden layers (8-bit significands), FP32 output layer;
    # the oracle emulating the same roundings differs by 0.3 % on this case
    Graw = torch.empty(attrs.shape[0], 12, dtype=torch.float64, device="cuda")
    net.sketch(ad, Graw, check=False)
    err_raw = colwise_err(Graw.cpu().numpy(), ref)
    G = torch.empty_like(Graw)
    assert net.sketch(ad, G)
    Gh = G.cpu().numpy()
    err_range = float(np.linalg.norm(ref - Gh @ (Gh.T @ ref)) / np.linalg.norm(ref))
    print("bf16 inference: raw error", err_raw, "range error", err_range)
    assert err_raw < 3e-2
    # the checked proposal is returned orthonormalized, with the range of the raw output
    assert np.abs(Gh.T @ Gh - np.eye(12)).max() < 1e-10
    assert err_range < 1e-2
    # a network whose output layer is zero proposes a rank-deficient block
    z = theta.copy()
    nw3 = HIDDEN * 12 + 12
    z[-nw3:] = 0.0
    net.set_params(z)
    assert not net.sketch(attrs, np.zeros((attrs.shape[0], 12)))
    net.destroy()


def test_shape_validation(N):
    theta, _, _ = _case()
    with pytest.raises(ValueError):
        N.SketchNet(theta[:-1], D_RAW, N_COORD, N_FREQ, HIDDEN, 12)
    with pytest.raises(N.NspError):
        N.SketchNet(np.zeros(10), D_RAW, N_COORD, N_FREQ, 0, 12)


def test_trained_sketch_gains_over_gaussian(N, torch):
    """Train on 48 seeded 64 x 64 lognormal fields (4 parts, k = 12, p = 4) against the
    method's own FP64 bases, evaluate on 12 held-out fields: the learned block is much
    closer to the target subspace (projector loss), the inner block PCG needs fewer
    iterations, and the outer PCG needs no more iterations on average."""
    from paper_2101_12164_gb300 import learned as LR
    shape, nsub, k, p = (64, 64), 4, 12, 4
    s = k + p
    kw = dict(ell_scale=64 / 256.0)
    train = LR.make_dataset(range(48), shape, nsub, s, kw)
    test = LR.make_dataset(range(10000, 10012), shape, nsub, s, kw)
    d_raw = train[0]["attrs"].shape[1]
    theta0 = FL.init_params(0, d_raw, 2, 8, 64, s)
    net = N.SketchNet(theta0, d_raw, 2, 8, 64, s, precision="fp32", mu=1e-2)
    hist = LR.train(net, train, epochs=150, lr=1e-3, log_every=50)
    assert hist[-1][1] < 0.5 * hist[0][1]
    rows = LR.evaluate(net, test, k, p)
    lossL, lossG = [], []
    for d in test:
        G = torch.empty(d["attrs"].shape[0], s, dtype=torch.float64, device="cuda")
        assert net.sketch(d["attrs"], G)
        U = d["U"].cpu().numpy()
        lossL.append(LR.sketch_loss(G.cpu().numpy(), U))
        lossG.append(LR.sketch_loss(np.random.default_rng(d["index"]).standard_normal(G.shape), U))
    inner = {m: np.mean([r[m]["it_inner"] for r in rows]) for m in ("gauss", "learned")}
    outer = {m: np.mean([r[m]["it_pcg"] for r in rows]) for m in ("gauss", "learned")}
    print("projector loss", np.mean(lossL), np.mean(lossG), "inner", inner, "outer", outer)
    assert np.mean(lossL) < 0.5 * np.mean(lossG)
    assert inner["learned"] < inner["gauss"]
    assert outer["learned"] <= outer["gauss"] + 0.5
    for r in rows:
        assert r["learned"]["final_residual"] < 1e-7
    net.destroy()
