"""Pins of the oracle's one-site variational MPS-MPO fitting (oracle/bmps.fit_compress),
the paper's compressor: monotone overlap, never worse than its zip-up initial guess,
exact at full rank, and bounded by the Schmidt spectrum of the exact product."""
import numpy as np
import pytest

from oracle import bmps


def _random_problem(W, dm, dw, seed):
    rng = np.random.default_rng(seed)
    rnd = lambda *s: rng.normal(size=s) + 1j * rng.normal(size=s)
    mps = [rnd(1 if j == 0 else dm, 2, 1, 1 if j == W - 1 else dm) for j in range(W)]
    mpo = [rnd(1 if j == 0 else dw, 2, 2, 1 if j == W - 1 else dw) for j in range(W)]
    return mps, mpo


def _dense_product(mps, mpo):
    v = None
    for m, w in zip(mps, mpo):
        p = bmps._product_site(m, w)
        a, l, y, xp, A, r = p.shape
        p2 = p.reshape(a * l, y * xp, A * r)
        v = p2[0] if v is None else np.tensordot(v, p2, axes=([-1], [0]))
    return v.reshape(-1)


def _dense_mps(Y, log_norm):
    v = None
    for y in Y:
        k, yy, xp, kp = y.shape
        y2 = y.reshape(k, yy * xp, kp)
        v = y2[0] if v is None else np.tensordot(v, y2, axes=([-1], [0]))
    return v.reshape(-1) * np.exp(log_norm)


def _fidelity(v, ex):
    return abs(np.vdot(v, ex)) ** 2 / (np.vdot(v, v).real * np.vdot(ex, ex).real)


@pytest.mark.parametrize("R,seed", [(2, 0), (4, 1), (6, 2)])
def test_fit_overlap_is_monotone_and_beats_its_initial_guess(R, seed):
    mps, mpo = _random_problem(6, 4, 3, seed)
    ex = _dense_product(mps, mpo)
    Yz, lz = bmps.zip_compress(mps, mpo, R, 1, 0, 0)
    hist = []
    Yf, lf = bmps.fit_compress(mps, mpo, R, 1, 0, 0, sweeps=3, history=hist)
    assert all(b >= a * (1 - 1e-12) for a, b in zip(hist, hist[1:]))
    fz, ff = _fidelity(_dense_mps(Yz, lz), ex), _fidelity(_dense_mps(Yf, lf), ex)
    assert ff >= fz - 1e-12
    # no MPS of bond R can exceed the kept Schmidt weight of the exact product at any cut
    d = 2                                             # output physical dimension per site
    for cut in range(1, 6):
        s = np.linalg.svd(ex.reshape(d ** cut, -1), compute_uv=False) ** 2
        assert ff <= s[:R].sum() / s.sum() + 1e-12


def test_fit_is_exact_at_full_rank_including_the_norm():
    mps, mpo = _random_problem(5, 3, 2, 7)
    ex = _dense_product(mps, mpo)
    Yf, lf = bmps.fit_compress(mps, mpo, 64, 1, 0, 0, sweeps=2)
    v = _dense_mps(Yf, lf)
    assert np.linalg.norm(v - ex) <= 1e-12 * np.linalg.norm(ex)
