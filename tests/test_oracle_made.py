"""Pins of the learned-proposal oracle (MADE, Adam, independent MH) against definitions."""
import itertools

import numpy as np
import pytest

import workloads as w
from oracle import made


def _theta(n, h, seed=3):
    rng = np.random.default_rng(seed)
    return rng.normal(scale=0.5, size=made.n_params(n, h))


def test_autoregressive_distribution_is_normalised():
    """sum_x g(x) = 1 by enumeration: holds only if every mask respects the variable order."""
    n, h = 8, 16
    theta = _theta(n, h)
    xs = np.array(list(itertools.product([0, 1], repeat=n)), dtype=np.float64)
    assert abs(np.exp(made.log_prob(theta, xs, n, h)).sum() - 1.0) < 1e-12


def test_output_i_ignores_inputs_at_or_after_i():
    n, h = 6, 12
    theta = _theta(n, h)
    x = np.zeros((1, n))
    base, _ = made.forward(theta, x, n, h)
    for j in range(n):
        x2 = x.copy()
        x2[0, j] = 1
        l2, _ = made.forward(theta, x2, n, h)
        assert np.allclose(l2[0, : j + 1], base[0, : j + 1])


def test_gradient_matches_finite_differences():
    n, h = 6, 10
    theta = _theta(n, h, seed=5)
    rng = np.random.default_rng(1)
    x = rng.integers(0, 2, size=(7, n)).astype(np.float64)
    _, g = made.loss_and_grad(theta, x, n, h)
    for idx in rng.choice(theta.size, size=40, replace=False):
        e = np.zeros_like(theta)
        e[idx] = 1e-6
        fd = (made.loss_and_grad(theta + e, x, n, h)[0] - made.loss_and_grad(theta - e, x, n, h)[0]) / 2e-6
        assert abs(fd - g[idx]) < 1e-6 * max(1.0, abs(fd))


def test_adam_first_step_closed_form():
    """Bias-corrected first Adam step is -lr * g / (|g| + eps) per coordinate."""
    opt = made.Adam(3, lr=0.1)
    th = np.array([1.0, -2.0, 0.5])
    g = np.array([0.3, -4.0, 0.0])
    out = opt.step(th, g)
    assert np.allclose(out, th - 0.1 * g / (np.abs(g) + 1e-8))


def test_ancestral_sampling_frequencies_and_logprob():
    n, h = 4, 8
    theta = _theta(n, h, seed=9)
    xs, lg = made.sample(theta, 20000, n, h, seed=12)
    assert np.allclose(lg, made.log_prob(theta, xs, n, h))
    allx = np.array(list(itertools.product([0, 1], repeat=n)))
    p = np.exp(made.log_prob(theta, allx, n, h))
    idx = (xs * (2 ** np.arange(n - 1, -1, -1))).sum(axis=1)
    freq = np.bincount(idx, minlength=2 ** n) / len(xs)
    assert np.all(np.abs(freq - p) < 4 * np.sqrt(p * (1 - p) / len(xs)) + 1e-4)


def test_mh_accepts_everything_when_proposal_is_target():
    rng = np.random.default_rng(0)
    lp = rng.normal(size=(4, 50))
    state, acc = made.mh_independent(lp, lp, np.zeros(4), np.zeros(4), seed=3)
    assert (acc == 50).all() and (state[:, -1] == 49).all()


def test_mh_stationary_distribution_is_target():
    """Independent MH with a non-matching proposal converges to p (16 states)."""
    rng = np.random.default_rng(4)
    logp = rng.normal(size=16)
    logg = rng.normal(scale=0.3, size=16)
    g = np.exp(logg) / np.exp(logg).sum()
    C, T = 64, 3000
    props = rng.choice(16, size=(C, T), p=g)
    x0 = rng.choice(16, size=C, p=g)
    state, acc = made.mh_independent(logp[props], logg[props], logp[x0], logg[x0], seed=5)
    held = np.where(state >= 0, np.take_along_axis(props, np.maximum(state, 0), axis=1), x0[:, None])
    freq = np.bincount(held[:, 500:].ravel(), minlength=16) / held[:, 500:].size
    p = np.exp(logp) / np.exp(logp).sum()
    assert np.abs(freq - p).max() < 0.02


def test_init_and_training_reduce_loss():
    n, h = 8, 16
    theta = w.made_init(n, h, seed=7).astype(np.float64)
    rng = np.random.default_rng(2)
    data = (rng.random((512, n)) < np.linspace(0.1, 0.9, n)).astype(np.float64)
    th2, losses = made.train(theta, data, n, h, batch=64, epochs=5, lr=1e-2,
                             orders=w.epoch_orders(len(data), 5))
    assert losses[-1] < losses[0]
