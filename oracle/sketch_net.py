"""FP64 CPU oracle of the learned sketch proposal (TEST INFRASTRUCTURE, like nsp_oracle).

The paper draws the sketch G of Algorithm 2 step 1 at random; its angle bound (§4.2,
Proposition 4.1 with eq. (tight_bound)) shows that the Nyström factor is better when
range(G) is closer to the dominant eigenvectors of the operator being approximated. The
learned proposal replaces G by the output of a small network phi evaluated at every
interface node; it is trained to minimise the projector loss against bases the method
itself computes. This module defines that network, the loss and their exact gradients in
plain numpy float64, in the order the computation is written below; it shares no code
with the CUDA path.

Network (per interface node i, raw attributes a_i in R^{d_raw}, the first n_coord of them
coordinates in (0, 1)):
  embedding  e_i = [sin(pi j a_ic), cos(pi j a_ic) for c < n_coord, j = 1..F] ++ a_i[n_coord:]
  layer 1    h1 = tanh(e W1 + b1)
  layer 2    h2 = tanh(h1 W2 + b2)
  output     g  = h2 W3 + b3                 (one row of G, s = k + p columns)
Loss for a target U (n x k, orthonormal columns), with M = G^T G (s x s):
  L(G) = || U - G M^{-1} G^T U ||_F^2  +  mu || M / n - I ||_F^2
The first term is ||(I - Pi_G) U||_F^2, Pi_G the orthogonal projector onto range(G); the
second keeps G well conditioned (L is otherwise invariant under G -> G T, and its
gradient grows with cond(M)). With W = M^{-1} G^T U and R = U - G W:
  dL/dG = -2 R W^T + (4 mu / n) G (M / n - I).
Parameters are one flat vector [W1, b1, W2, b2, W3, b3] (weights row-major, input
dimension first). Training uses Adam (Kingma & Ba 2015) with bias correction.
"""

import numpy as np


def dims(d_raw, n_coord, n_freq, hidden, s_out):
    d0 = 2 * n_freq * n_coord + (d_raw - n_coord)
    return d0, hidden, hidden, s_out


def unpack(theta, shape):
    d0, h1, h2, so = dims(*shape)
    out, o = [], 0
    for a, b in ((d0, h1), (h1, h2), (h2, so)):
        out.append(theta[o:o + a * b].reshape(a, b))
        o += a * b
        out.append(theta[o:o + b])
        o += b
    assert o == theta.size
    return out


def embed(attrs, n_coord, n_freq):
    """e_i: sines and cosines of pi j x for every coordinate x, then the other attributes."""
    attrs = np.asarray(attrs, dtype=np.float64)
    cols = []
    for c in range(n_coord):
        for j in range(1, n_freq + 1):
            cols.append(np.sin(np.pi * j * attrs[:, c]))
            cols.append(np.cos(np.pi * j * attrs[:, c]))
    return np.concatenate([np.stack(cols, axis=1), attrs[:, n_coord:]], axis=1)


def forward(theta, attrs, shape):
    """G (n x s) and the activations kept for the backward pass."""
    d_raw, n_coord, n_freq, hidden, s_out = shape
    W1, b1, W2, b2, W3, b3 = unpack(theta, shape)
    e = embed(attrs, n_coord, n_freq)
    h1 = np.tanh(e @ W1 + b1)
    h2 = np.tanh(h1 @ W2 + b2)
    G = h2 @ W3 + b3
    return G, (e, h1, h2)


def projector_loss(G, U, mu):
    """(L, dL/dG) of the loss above."""
    n, s = G.shape
    M = G.T @ G
    W = np.linalg.solve(M, G.T @ U)
    R = U - G @ W
    E = M / n - np.eye(s)
    L = float((R * R).sum() + mu * (E * E).sum())
    dG = -2.0 * R @ W.T + (4.0 * mu / n) * G @ E
    return L, dG


def loss_and_grad(theta, attrs, U, shape, mu):
    """(L, dL/dtheta) by the chain rule through the three layers."""
    G, (e, h1, h2) = forward(theta, attrs, shape)
    L, dG = projector_loss(G, U, mu)
    W1, b1, W2, b2, W3, b3 = unpack(theta, shape)
    dW3 = h2.T @ dG
    db3 = dG.sum(axis=0)
    dz2 = (dG @ W3.T) * (1.0 - h2 * h2)
    dW2 = h1.T @ dz2
    db2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2.T) * (1.0 - h1 * h1)
    dW1 = e.T @ dz1
    db1 = dz1.sum(axis=0)
    grad = np.concatenate([dW1.ravel(), db1, dW2.ravel(), db2, dW3.ravel(), db3])
    return L, grad


def adam_step(theta, grad, m, v, t, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (t = 1 for the first step); returns (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** t)
    vh = v / (1.0 - beta2 ** t)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
