"""Training and evaluation driver of the learned sketch proposal (runs on the GPU).

Every arithmetic step runs in the library's kernels (nsp_net_* for the network, nsp_build /
nsp_solve for the method); this module only moves arrays and loops over fields.

* Targets: for each field, the method's own FP64 Nyström basis computed with tight settings
  (FP64 factors, inner tolerance 1e-6, sketch width 2 s_out), i.e. the orthonormal U of
  Algorithm 2 step 10 with s_out columns (nsp_get_intermediate(3)).
* Training: one Adam step per field (batch of one), fields in a seeded random order each
  epoch, cosine learning-rate decay.
* Evaluation on held-out fields: M2 built with the Gaussian sketch and with the learned one
  (Gaussian fallback when the learned block is rank-deficient), both with the same k, p and
  precision; reported per field: inner block-PCG iterations, outer PCG iterations,
  build + solve time, and the projector loss of each sketch against the target basis.

``python -m paper_2101_12164_gb300.learned`` runs the 256^2 lognormal workload (16 parts,
k = 48, p = 8) and prints one JSON line.
"""

import argparse
import json
import time

import numpy as np

from . import SketchNet, nsp_build

ATTR_SHAPE = dict(n_coord=2, n_freq=8, hidden=64)


def target_basis(A, part, nsub, s_out, seed):
    """FP64 Nyström basis U (n_gamma x s_out, orthonormal) of the method with tight settings."""
    h = nsp_build(A, part, nsub, k=s_out, p=s_out, eps_inner=1e-6, precision="fp64", seed=seed,
                  keep_intermediates=True)
    try:
        inf = h.info()
        if inf["rank"] < s_out:
            raise RuntimeError("target basis has rank %d < %d" % (inf["rank"], s_out))
        return h.get_intermediate(3)
    finally:
        h.destroy()


def make_dataset(indices, shape, nsub, s_out, field_kw, device="cuda"):
    """[(attrs_dev, U_dev, A, part)] for the given field indices."""
    import torch

    import fixtures.learned as FL
    out = []
    for i in indices:
        A, part, coef, attrs, meta = FL.training_problem(i, shape, nsub, **field_kw)
        U = target_basis(A, part, nsub, s_out, seed=7919 + i)
        out.append(dict(index=i, A=A, part=part, meta=meta,
                        attrs=torch.tensor(attrs, dtype=torch.float64, device=device),
                        U=torch.tensor(U, dtype=torch.float64, device=device)))
    return out


def train(net, data, epochs, lr, seed=0, log_every=0):
    rng = np.random.default_rng(seed)
    total = epochs * len(data)
    step = 0
    hist = []
    for ep in range(epochs):
        order = rng.permutation(len(data))
        want = log_every and (ep % log_every == 0 or ep == epochs - 1)
        losses = []
        for j in order:
            d = data[j]
            L = net.loss_grad(d["attrs"], d["U"], want_loss=bool(want))
            if want:
                losses.append(L)
            lr_t = lr * 0.5 * (1.0 + np.cos(np.pi * step / total))
            net.adam_step(lr_t)
            step += 1
        if want:
            hist.append((ep, float(np.mean(losses))))
    return hist


def evaluate(net, data, k, p, precision="fp32", seed=0, rtol=1e-8):
    """Per held-out field: Gaussian vs learned sketch (inner its, outer its, ms)."""
    import torch
    rows = []
    for d in data:
        A, part = d["A"], d["part"]
        nsub = int(part.max()) + 1
        n_gamma = d["attrs"].shape[0]
        G = torch.empty(n_gamma, k + p, dtype=torch.float64, device="cuda")
        full = net.sketch(d["attrs"], G)
        b = A @ np.random.default_rng(seed + d["index"]).standard_normal(A.shape[0])
        bd = torch.tensor(b, dtype=torch.float64, device="cuda")
        row = dict(index=d["index"], full_rank=full)
        for name, kw in (("gauss", dict(seed=1000 + d["index"])),
                         ("learned", dict(sketch=G) if full else dict(seed=1000 + d["index"]))):
            xd = torch.zeros_like(bd)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            h = nsp_build(A, part, nsub, k=k, p=p, precision=precision, **kw)
            inf = h.solve(bd, xd, rtol=rtol, maxit=1000)
            torch.cuda.synchronize()
            ms = (time.perf_counter() - t0) * 1e3
            row[name] = dict(it_inner=inf["it_inner"], it_pcg=inf["it_pcg"], ms=ms,
                             final_residual=inf["final_residual"], rank=inf["rank"])
            h.destroy()
        rows.append(row)
    return rows


def sketch_loss(G, U):
    """||(I - Pi_G) U||_F^2 of a sketch against a target, on the host (reporting only)."""
    Q, _ = np.linalg.qr(np.asarray(G))
    U = np.asarray(U)
    return float(np.linalg.norm(U - Q @ (Q.T @ U)) ** 2)


def main():
    import torch

    import fixtures.learned as FL
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", type=int, default=256)
    ap.add_argument("--nsub", type=int, default=16)
    ap.add_argument("--k", type=int, default=48)
    ap.add_argument("--p", type=int, default=8)
    ap.add_argument("--train", type=int, default=512)
    ap.add_argument("--test", type=int, default=64)
    ap.add_argument("--epochs", type=int, default=60)
    ap.add_argument("--lr", type=float, default=1e-3)
    ap.add_argument("--mu", type=float, default=1e-2)
    args = ap.parse_args()
    shape = (args.grid, args.grid)
    s_out = args.k + args.p
    kw = dict(ell_scale=args.grid / 256.0)
    t0 = time.perf_counter()
    train_set = make_dataset(range(args.train), shape, args.nsub, s_out, kw)
    test_set = make_dataset(range(10000, 10000 + args.test), shape, args.nsub, s_out, kw)
    t_data = time.perf_counter() - t0
    d_raw = train_set[0]["attrs"].shape[1]
    theta0 = FL.init_params(0, d_raw, ATTR_SHAPE["n_coord"], ATTR_SHAPE["n_freq"],
                            ATTR_SHAPE["hidden"], s_out)
    net = SketchNet(theta0, d_raw, s_out=s_out, precision="fp32", mu=args.mu, **ATTR_SHAPE)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hist = train(net, train_set, args.epochs, args.lr, log_every=max(1, args.epochs // 6))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    rows = evaluate(net, test_set, args.k, args.p)
    losses = []
    for d in test_set:
        G = torch.empty(d["attrs"].shape[0], s_out, dtype=torch.float64, device="cuda")
        net.sketch(d["attrs"], G)
        Gg = np.random.default_rng(5 + d["index"]).standard_normal(G.shape)
        U = d["U"].cpu().numpy()
        losses.append((sketch_loss(G.cpu().numpy(), U), sketch_loss(Gg, U)))
    out = {
        "workload": "lognormal2d_%d: 2D 5-point lognormal (ell U[4,16] cells, sigma U[1,3]), "
                    "%d parts, k=%d, p=%d" % (args.grid, args.nsub, args.k, args.p),
        "train_fields": args.train, "test_fields": args.test, "epochs": args.epochs,
        "data_s": t_data, "train_s": t_train, "loss_history": hist,
        "test_projector_loss": {"learned": float(np.mean([a for a, _ in losses])),
                                "gauss": float(np.mean([b for _, b in losses]))},
        "mean": {name: {key: float(np.mean([r[name][key] for r in rows]))
                        for key in ("it_inner", "it_pcg", "ms")}
                 for name in ("gauss", "learned")},
        "fallbacks": int(sum(not r["full_rank"] for r in rows)),
        "rows": rows,
    }
    print(json.dumps(out))
    net.destroy()


if __name__ == "__main__":
    main()
