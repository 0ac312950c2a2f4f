"""Pins of the oracle's direct (sample-free) marginals, oracle/bmps.direct_marginals:
brute-force statevector marginals of the same TNS when the boundary rank covers the
environments, including a transposed (ladder) grid with empty cells."""
import numpy as np
import pytest

import workloads as w
from oracle import bmps, metrics
from oracle.tns import GridTNS


def _state(lat, bits, groups, chi):
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in groups:
        t.apply_group(g, chi)
        t.bp(500, 1e-12)
    return t


@pytest.mark.parametrize("kind", ["su4_3x3", "heis_4x4_truncated", "ladder"])
def test_direct_marginals_equal_bruteforce(kind):
    if kind == "su4_3x3":
        lat = w.square(3, 3)
        bits = w.domain_wall_bits(lat)
        t = _state(lat, bits, w.random_su4_circuit(lat, 1, seed=5), 16)
    elif kind == "heis_4x4_truncated":
        lat = w.square(4, 4)
        bits = w.domain_wall_bits(lat)
        t = _state(lat, bits, w.heisenberg_circuit(lat, 2, 0.2), 4)     # chi = 4 truncates
    else:
        lat = w.ladder(4)
        groups, bits = w.lucj_like_circuit(lat, reps=1, seed=3)
        t = _state(lat, bits, groups, 16)
    one, two = bmps.direct_marginals(t, 256)
    o_ref, t_ref = metrics.marginals_from_statevector(t.statevector_bruteforce())
    assert np.abs(one - o_ref).max() < 1e-10
    mask = ~np.isnan(two)
    assert mask.sum() >= len(one)
    assert np.abs(two[mask] - t_ref[mask]).max() < 1e-10
    assert np.allclose(np.diag(two), one)


def test_first_site_marginal_equals_first_sampler_conditional():
    """The first qubit of the first row has no prefix: its sampler conditional q(0)
    is 1 - <n> (two different contraction orders of the same network)."""
    lat = w.square(3, 3)
    bits = w.domain_wall_bits(lat)
    t = _state(lat, bits, w.random_su4_circuit(lat, 1, seed=9), 16)
    one, _ = bmps.direct_marginals(t, 64)
    _, _, q0 = bmps.sample(t, 64, 1, seed=3)
    q = int(t.cell_qubit[0, 0])
    assert abs(q0[0, q] - (1.0 - one[q])) < 1e-10


def test_certification_at_exact_rank_and_unbiased_mean_ratio():
    """Exact sampling: p/q = 1 for every sample, KLD 0.  Truncated sampling: the mean of
    p/q estimates sum_x p(x) = 1 (Methods) within 4 standard errors."""
    lat = w.square(3, 3)
    bits = w.domain_wall_bits(lat)
    t = _state(lat, bits, w.random_su4_circuit(lat, 1, seed=4), 16)
    xs, lq, _ = bmps.sample(t, 64, 30, seed=2)
    c = bmps.certify(t, xs, lq, 64)
    assert np.allclose(c["ratio"], 1.0, atol=1e-9) and abs(c["kld"]) < 1e-9
    xs, lq, _ = bmps.sample(t, 2, 300, seed=3)
    c = bmps.certify(t, xs, lq, 64)
    r = c["ratio"]
    assert abs(r.mean() - 1.0) < 4 * r.std() / np.sqrt(r.size)
    assert c["kld"] > -0.05 and sum(c["hist"][0]) == r.size


def test_projected_norms_agree_with_row_transfers_and_bruteforce():
    """Two independent contractions of the same marginals: the norm of the projected
    state (any pair of rows) and the row transfer between top and bottom environments
    (same row); both against brute force."""
    lat = w.square(3, 3)
    bits = w.domain_wall_bits(lat)
    t = _state(lat, bits, w.random_su4_circuit(lat, 1, seed=11), 16)
    one, two = bmps.direct_marginals(t, 64)
    o_ref, t_ref = metrics.marginals_from_statevector(t.statevector_bruteforce())
    q_same = [int(t.cell_qubit[1, 0]), int(t.cell_qubit[1, 2])]
    q_cross = [int(t.cell_qubit[0, 1]), int(t.cell_qubit[2, 2])]
    assert abs(bmps.projected_marginal(t, 64, [q_same[0]]) - one[q_same[0]]) < 1e-10
    assert abs(bmps.projected_marginal(t, 64, q_same) - two[q_same[0], q_same[1]]) < 1e-10
    assert abs(bmps.projected_marginal(t, 64, q_cross) - t_ref[q_cross[0], q_cross[1]]) < 1e-10
    assert np.isnan(two[q_cross[0], q_cross[1]])
