"""Per-element MLP that predicts a stage solve's initial Krylov guess.

Not in the paper (a learned addition around its GMRES, which still tests
the result: the solve converges to the same tolerance from any guess).

Network: x (3 nb features of one element) -> Linear(3nb, 256) -> ReLU ->
Linear(256, 256) -> ReLU -> Linear(256, nb).  Weights W (out x in) and
biases b, FP64 here.  Loss: mean over samples and outputs of
(y_pred - y_true)^2 / 2.  Optimiser: Adam (Kingma & Ba 2015) with bias
correction.

Features of element e for ROW stage i (all divided by the stage scale
s = ||b||_2 / sqrt(N), the state by its own RMS): [b_e / s, Y_{i-1,e} / s,
U_e / rms(U)]; target Y_{i,e} / s.

Pins (tests/test_oracle_mlp.py): backward against central finite
differences of the loss; Adam's first step equals lr * sign(g) (bias
correction); a linear target is learned.
"""
from __future__ import annotations

import numpy as np


def init_params(sizes, seed):
    """He-uniform weights, zero biases: list of (W, b)."""
    rng = np.random.default_rng(seed)
    params = []
    for fan_in, fan_out in zip(sizes[:-1], sizes[1:]):
        lim = np.sqrt(6.0 / fan_in)
        params.append((rng.uniform(-lim, lim, (fan_out, fan_in)), np.zeros(fan_out)))
    return params


def forward(params, X):
    """Returns the output and the pre-activations / activations of every layer."""
    acts = [X]
    pre = []
    h = X
    for li, (W, b) in enumerate(params):
        z = h @ W.T + b
        pre.append(z)
        h = np.maximum(z, 0.0) if li < len(params) - 1 else z
        acts.append(h)
    return h, pre, acts


def loss(params, X, Y):
    out, _, _ = forward(params, X)
    return 0.5 * np.mean((out - Y) ** 2)


def backward(params, X, Y):
    """Gradients of ``loss`` with respect to every W and b."""
    out, pre, acts = forward(params, X)
    g = (out - Y) / out.size
    grads = [None] * len(params)
    for li in range(len(params) - 1, -1, -1):
        W, _ = params[li]
        gW = g.T @ acts[li]
        gb = g.sum(axis=0)
        grads[li] = (gW, gb)
        if li > 0:
            g = (g @ W) * (pre[li - 1] > 0.0)
    return grads


class Adam:
    def __init__(self, params, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        self.lr, self.b1, self.b2, self.eps = lr, beta1, beta2, eps
        self.t = 0
        self.m = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]
        self.v = [(np.zeros_like(W), np.zeros_like(b)) for W, b in params]

    def step(self, params, grads):
        self.t += 1
        out = []
        for li, ((W, b), (gW, gb)) in enumerate(zip(params, grads)):
            new = []
            for k, (p, g) in enumerate(((W, gW), (b, gb))):
                m = self.b1 * self.m[li][k] + (1 - self.b1) * g
                v = self.b2 * self.v[li][k] + (1 - self.b2) * g * g
                self.m[li] = tuple(m if kk == k else self.m[li][kk] for kk in range(2))
                self.v[li] = tuple(v if kk == k else self.v[li][kk] for kk in range(2))
                mh = m / (1 - self.b1 ** self.t)
                vh = v / (1 - self.b2 ** self.t)
                new.append(p - self.lr * mh / (np.sqrt(vh) + self.eps))
            out.append(tuple(new))
        return out


def stage_features(b, Yprev, U):
    """(Ne, 3 nb) features and the stage scale s for one ROW stage solve;
    b, Yprev, U are (Ne, 4, Np)."""
    ne = b.shape[0]
    s = np.linalg.norm(b) / np.sqrt(b.size)
    s = s if s > 0 else 1.0
    su = np.sqrt(np.mean(U * U))
    X = np.concatenate([b.reshape(ne, -1) / s, Yprev.reshape(ne, -1) / s, U.reshape(ne, -1) / su], axis=1)
    return X, s
