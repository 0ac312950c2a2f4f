"""Sample-quality metrics of the paper (Appendix and Methods), plain numpy.

TEST INFRASTRUCTURE ONLY.

* p/q ratios and their mean, an unbiased estimator of <psi|psi> (Methods,
  "Sampling from Tensor Network States");
* sample KLD = E_q[log q - log p] (Eq. kld);
* fraction of samples in the initial U(1) sector (Results, Heisenberg / LUCJ);
* single- and two-site marginals from samples or from a statevector;
* self-normalised importance-sampling estimate of a diagonal observable
  (Appendix; the printed normalisation is ambiguous, read as sum w O / sum w).
"""
from __future__ import annotations

import numpy as np


def p_over_q(log_p, log_q):
    return np.exp(np.asarray(log_p) - np.asarray(log_q))


def kld(log_q, log_p) -> float:
    return float(np.mean(np.asarray(log_q) - np.asarray(log_p)))


def sector_fraction(bits, n_ones: int) -> float:
    return float(np.mean(np.asarray(bits).sum(axis=1) == n_ones))


def marginals_from_samples(bits):
    b = np.asarray(bits, dtype=np.float64)
    one = b.mean(axis=0)
    two = (b.T @ b) / b.shape[0]
    return one, two


def marginals_from_statevector(psi):
    p = np.abs(psi) ** 2
    p = p / p.sum()
    n = p.ndim
    one = np.array([p.sum(axis=tuple(a for a in range(n) if a != q))[1] for q in range(n)])
    two = np.zeros((n, n))
    for i in range(n):
        for j in range(n):
            if i == j:
                two[i, j] = one[i]
            else:
                axes = tuple(a for a in range(n) if a not in (i, j))
                pij = p.sum(axis=axes)
                two[i, j] = pij[1, 1]
    return one, two


def importance_estimate(values, log_p, log_q) -> float:
    w = p_over_q(log_p, log_q)
    return float(np.sum(w * np.asarray(values)) / np.sum(w))
