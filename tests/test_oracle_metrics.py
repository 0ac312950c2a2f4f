"""Pins of the oracle's sample-quality metrics (oracle/metrics.py) against closed forms."""
import numpy as np

from oracle import metrics


def test_marginals_from_statevector_bell_and_product():
    # (|00> + |11>)/sqrt2: <n_i> = 1/2, <n_0 n_1> = 1/2
    psi = np.zeros((2, 2), dtype=complex)
    psi[0, 0] = psi[1, 1] = 1 / np.sqrt(2)
    one, two = metrics.marginals_from_statevector(psi)
    assert np.allclose(one, [0.5, 0.5]) and np.isclose(two[0, 1], 0.5) and np.isclose(two[1, 0], 0.5)
    # product |0>|1>|+>: <n> = (0, 1, 1/2), <n_1 n_2> = 1/2, unnormalised input
    plus = np.array([1, 1]) / np.sqrt(2)
    psi = 3.0 * np.einsum("a,b,c->abc", [1, 0], [0, 1], plus)
    one, two = metrics.marginals_from_statevector(psi)
    assert np.allclose(one, [0, 1, 0.5])
    assert np.isclose(two[1, 2], 0.5) and np.isclose(two[0, 1], 0.0) and np.allclose(np.diag(two), one)


def test_marginals_from_samples_counts():
    bits = np.array([[1, 0, 1], [1, 1, 0], [0, 0, 1], [1, 0, 1]])
    one, two = metrics.marginals_from_samples(bits)
    assert np.allclose(one, [0.75, 0.25, 0.75])
    assert np.isclose(two[0, 2], 0.5) and np.isclose(two[0, 1], 0.25) and np.isclose(two[1, 2], 0.0)


def test_sector_fraction():
    bits = np.array([[1, 0, 1], [1, 1, 0], [0, 0, 1], [1, 1, 1]])
    assert metrics.sector_fraction(bits, 2) == 0.5


def test_importance_estimate_and_ratio_identities():
    rng = np.random.default_rng(0)
    vals = rng.normal(size=1000)
    lp = rng.normal(size=1000)
    # q = p: weights 1, plain mean; ratios 1; KLD 0
    assert np.isclose(metrics.importance_estimate(vals, lp, lp), vals.mean())
    assert np.allclose(metrics.p_over_q(lp, lp), 1.0)
    assert metrics.kld(lp, lp) == 0.0
    # q = p e^{-c}: constant weights cancel in the self-normalised estimate
    assert np.isclose(metrics.importance_estimate(vals, lp + 3.0, lp), vals.mean())
    # two-point check: weights (1, 3) on values (0, 1) -> 3/4
    assert np.isclose(metrics.importance_estimate([0.0, 1.0], np.log([1.0, 3.0]), [0.0, 0.0]), 0.75)


def test_self_normalised_estimate_converges_to_target_mean():
    """Draw from q = uniform over 8 states, weight by p/q: the estimate of E_p[f]
    converges to the exact value (law of large numbers, 5 sigma)."""
    rng = np.random.default_rng(1)
    p = rng.random(8)
    p /= p.sum()
    f = np.arange(8, dtype=float)
    x = rng.integers(0, 8, size=200000)
    est = metrics.importance_estimate(f[x], np.log(p[x]), np.full(x.size, np.log(1 / 8)))
    exact = float(p @ f)
    w = 8 * p[x]
    sd = np.sqrt(np.mean(w ** 2 * (f[x] - exact) ** 2) / x.size)
    assert abs(est - exact) < 5 * sd
