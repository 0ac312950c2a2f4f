"""CPU oracle for the learned proposal: MADE network, Adam training, independent MH.

TEST INFRASTRUCTURE ONLY.  Not part of the paper: the build adds a masked
autoregressive MLP (MADE: Germain, Gregor, Murray, Larochelle, ICML 2015) trained
by maximum likelihood on the plain sampler's bitstrings, and uses it as the
proposal of an independent Metropolis-Hastings chain whose target is
p(x) = |<x|psi>|^2 (amplitudes from the boundary-MPS contraction).

Network (natural variable order 1..n, hidden width h, three hidden layers):
  h1 = relu((W1 * M1) x + b1), h2 = relu((W2 * M2) h1 + b2), h3 = relu((W3 * M3) h2 + b3),
  l  = (W4 * M4) h3 + b4,  g(x_i = 1 | x_<i) = sigmoid(l_i).
Degrees: inputs i+1; hidden unit k of every layer 1 + (k mod (n-1)); outputs i+1.
Masks: hidden M[k, j] = [deg_out(k) >= deg_in(j)], output M4[i, k] = [i+1 > deg(k)].
log g(x) = sum_i x_i log s(l_i) + (1 - x_i) log s(-l_i).
Parameters are packed (float) as W1[h,n], b1[h], W2[h,h], b2[h], W3[h,h], b3[h],
W4[n,h], b4[n] -- the layout the library's tns_made_* calls use.
"""
from __future__ import annotations

import numpy as np

from . import philox


def degrees(n: int, h: int):
    d_in = np.arange(1, n + 1)
    d_h = 1 + (np.arange(h) % max(1, n - 1))
    return d_in, d_h


def masks(n: int, h: int):
    d_in, d_h = degrees(n, h)
    M1 = (d_h[:, None] >= d_in[None, :]).astype(np.float64)
    M2 = (d_h[:, None] >= d_h[None, :]).astype(np.float64)
    M4 = (d_in[:, None] > d_h[None, :]).astype(np.float64)
    return M1, M2, M2.copy(), M4


def shapes(n: int, h: int):
    return [(h, n), (h,), (h, h), (h,), (h, h), (h,), (n, h), (n,)]


def unpack(theta: np.ndarray, n: int, h: int):
    out, off = [], 0
    for s in shapes(n, h):
        sz = int(np.prod(s))
        out.append(np.asarray(theta[off:off + sz], dtype=np.float64).reshape(s))
        off += sz
    return out


def pack(parts) -> np.ndarray:
    return np.concatenate([np.asarray(p, dtype=np.float64).ravel() for p in parts])


def n_params(n: int, h: int) -> int:
    return int(sum(np.prod(s) for s in shapes(n, h)))


def softplus(z):
    return np.logaddexp(0.0, z)


def forward(theta, x, n, h):
    """Logits l [B, n] and the cached activations for the backward pass."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, n, h)
    M1, M2, M3, M4 = masks(n, h)
    x = np.asarray(x, dtype=np.float64)
    z1 = x @ (W1 * M1).T + b1
    a1 = np.maximum(z1, 0)
    z2 = a1 @ (W2 * M2).T + b2
    a2 = np.maximum(z2, 0)
    z3 = a2 @ (W3 * M3).T + b3
    a3 = np.maximum(z3, 0)
    logits = a3 @ (W4 * M4).T + b4
    return logits, (x, z1, a1, z2, a2, z3, a3)


def log_prob(theta, x, n, h):
    """log g(x) per row."""
    l, _ = forward(theta, x, n, h)
    s = 2.0 * np.asarray(x, dtype=np.float64) - 1.0
    return -np.sum(softplus(-s * l), axis=1)


def loss_and_grad(theta, x, n, h):
    """Mean negative log-likelihood over the batch and its gradient (packed)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = unpack(theta, n, h)
    M1, M2, M3, M4 = masks(n, h)
    l, (x, z1, a1, z2, a2, z3, a3) = forward(theta, x, n, h)
    B = x.shape[0]
    s = 2.0 * x - 1.0
    loss = float(np.mean(np.sum(softplus(-s * l), axis=1)))
    dl = (1.0 / (1.0 + np.exp(-l)) - x) / B                  # d loss / d logits
    gW4 = (dl.T @ a3) * M4
    gb4 = dl.sum(axis=0)
    d3 = (dl @ (W4 * M4)) * (z3 > 0)
    gW3 = (d3.T @ a2) * M3
    gb3 = d3.sum(axis=0)
    d2 = (d3 @ (W3 * M3)) * (z2 > 0)
    gW2 = (d2.T @ a1) * M2
    gb2 = d2.sum(axis=0)
    d1 = (d2 @ (W2 * M2)) * (z1 > 0)
    gW1 = (d1.T @ x) * M1
    gb1 = d1.sum(axis=0)
    return loss, pack([gW1, gb1, gW2, gb2, gW3, gb3, gW4, gb4])


class Adam:
    """Adam (Kingma & Ba 2015) with bias correction."""

    def __init__(self, size, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8):
        self.m = np.zeros(size)
        self.v = np.zeros(size)
        self.t = 0
        self.lr, self.b1, self.b2, self.eps = lr, b1, b2, eps

    def step(self, theta, g):
        self.t += 1
        self.m = self.b1 * self.m + (1 - self.b1) * g
        self.v = self.b2 * self.v + (1 - self.b2) * g * g
        mh = self.m / (1 - self.b1 ** self.t)
        vh = self.v / (1 - self.b2 ** self.t)
        return theta - self.lr * mh / (np.sqrt(vh) + self.eps)


def train(theta, data, n, h, batch, epochs, lr=1e-3, orders=None):
    """Mini-batch Adam on the mean NLL; orders[e] is the data permutation of epoch e."""
    opt = Adam(theta.size, lr=lr)
    losses = []
    for e in range(epochs):
        order = np.arange(len(data)) if orders is None else orders[e]
        tot, cnt = 0.0, 0
        for i in range(0, len(data), batch):
            xb = data[order[i:i + batch]]
            loss, g = loss_and_grad(theta, xb, n, h)
            theta = opt.step(theta, g)
            tot += loss * len(xb)
            cnt += len(xb)
        losses.append(tot / cnt)
    return theta, losses


def sample(theta, n_samples, n, h, seed, sample_offset=0):
    """Ancestral sampling; qubit i of proposal s uses Philox counter (s lo, s hi, i, 1):
    x_i = 1 iff u >= g(x_i = 0 | x_<i).  Returns bits and log g."""
    x = np.zeros((n_samples, n))
    k0, k1 = philox.split_seed(seed)
    sid = np.arange(sample_offset, sample_offset + n_samples, dtype=np.uint64)
    for i in range(n):
        l, _ = forward(theta, x, n, h)
        w0, w1, _, _ = philox.philox4x32_10(sid & philox.MASK, sid >> np.uint64(32), np.full_like(sid, i),
                                            np.ones_like(sid), k0, k1)
        u = philox.u53(w0, w1)
        p0 = 1.0 / (1.0 + np.exp(l[:, i]))
        x[:, i] = (u >= p0).astype(np.float64)
    return x.astype(np.uint8), log_prob(theta, x, n, h)


def mh_independent(logp_prop, logg_prop, logp0, logg0, seed):
    """Independent Metropolis-Hastings over precomputed proposals.

    Chain c at step t proposes proposal (c, t); accept iff u < exp(lp' - lp + lg - lg')
    with u from Philox counter (c, t, 0, 2), key seed (u53 in [0, 1)).  Returns
    state[c, t] = index t' of the proposal the chain holds after step t (-1 for its
    initial state) and the number of acceptances per chain.
    """
    C, T = logp_prop.shape
    k0, k1 = philox.split_seed(seed)
    state = np.full((C, T), -1, dtype=np.int64)
    acc = np.zeros(C, dtype=np.int64)
    for c in range(C):
        lp, lg, cur = float(logp0[c]), float(logg0[c]), -1
        for t in range(T):
            w0, w1, _, _ = philox.philox4x32_10(c, t, 0, 2, k0, k1)
            u = float(philox.u53(w0, w1))
            a = (logp_prop[c, t] - lp) + (lg - logg_prop[c, t])
            if np.log(u) < a if u > 0 else True:
                lp, lg, cur = float(logp_prop[c, t]), float(logg_prop[c, t]), t
                acc[c] += 1
            state[c, t] = cur
    return state, acc
