"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms, the exact statevector, brute-force
contraction, and exactness limits stated in the paper.
"""
import os

import numpy as np
import pytest
import scipy.linalg

import workloads as w
from oracle import bmps, metrics, philox
from oracle import statevector as sv
from oracle.tns import GridTNS

X = np.array([[0, 1], [1, 0]], dtype=complex)
Y = np.array([[0, -1j], [1j, 0]], dtype=complex)
Z = np.diag([1.0, -1.0]).astype(complex)


# ---------------------------------------------------------------- Philox
def test_philox_known_answers(golden_dir):
    """Philox4x32-10 reproduces the published known-answer vectors (Salmon et al. SC'11)."""
    rows = [l.split() for l in open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) if l[0] != "#"]
    assert len(rows) == 3
    for r in rows:
        v = [int(x, 16) for x in r]
        out = philox.philox4x32_10(*v[:6])
        assert [int(o) for o in out] == v[6:]


def test_uniforms_in_range_and_decorrelated():
    u = philox.draw_uniforms(20250711, np.arange(4096), 3)
    assert (u >= 0).all() and (u < 1).all()
    assert abs(u.mean() - 0.5) < 4 * np.sqrt(1 / 12 / 4096)
    om = philox.test_matrix(5, philox.STAGE_SAMPLE, 2, 3, 64, 40)
    assert om.shape == (64, 40)
    assert np.abs(om.real).max() <= 1 and np.abs(om.imag).max() <= 1
    assert not np.allclose(om, philox.test_matrix(5, philox.STAGE_SAMPLE, 2, 4, 64, 40))


# ---------------------------------------------------------------- gates
@pytest.mark.parametrize("dt", [0.1, 0.2, 0.7])
def test_heisenberg_gate_closed_form(dt):
    """exp(-i dt (XX+YY+ZZ)) from the closed form equals the matrix exponential (Eq. Heisenberg)."""
    Hb = np.kron(X, X) + np.kron(Y, Y) + np.kron(Z, Z)
    U = w.heisenberg_gate(dt)
    assert np.abs(U - scipy.linalg.expm(-1j * dt * Hb)).max() < 1e-14
    assert np.abs(U.conj().T @ U - np.eye(4)).max() < 1e-14


def test_disordered_heisenberg_circuit():
    """One coupling per bond in [0.8, 1.2], every gate exp(-i J_e dt (XX+YY+ZZ)) by the
    matrix exponential, the same coupling on a bond in every layer, the uniform
    circuit's colour order, and the same draw for the same seed."""
    lat = w.square(4, 4)
    dt = 0.2
    groups = w.disordered_heisenberg_circuit(lat, 2, dt, seed=3)
    again = w.disordered_heisenberg_circuit(lat, 2, dt, seed=3)
    uni = w.heisenberg_circuit(lat, 2, dt)
    Hb = np.kron(X, X) + np.kron(Y, Y) + np.kron(Z, Z)
    assert len(groups) == len(uni)
    per_bond = {}
    for g, gu, ga in zip(groups, uni, again):
        assert [(a, b) for a, b, _ in g] == [(a, b) for a, b, _ in gu]
        for (a, b, U), (_, _, Ua) in zip(g, ga):
            assert np.array_equal(U, Ua)
            J = -np.angle(U[0, 0]) / dt          # |00> is an eigenvector with phase e^{-i J dt}
            assert 0.8 <= J <= 1.2
            assert np.abs(U - scipy.linalg.expm(-1j * J * dt * Hb)).max() < 1e-13
            if (a, b) in per_bond:
                assert np.array_equal(per_bond[(a, b)], U)
            per_bond[(a, b)] = U
    assert len(per_bond) == len(lat.edges)
    assert len({round(float(-np.angle(U[0, 0]) / dt), 12) for U in per_bond.values()}) == len(per_bond)


def test_givens_is_xx_plus_yy_rotation():
    th = 1.234
    U = w.givens_gate(th)
    ref = scipy.linalg.expm(-1j * th / 4 * (np.kron(X, X) + np.kron(Y, Y)))
    assert np.abs(U - ref).max() < 1e-14


# ---------------------------------------------------------------- lattices
def test_lattice_sizes():
    hh = w.heavy_hex()
    assert hh.n_qubits == 164 and hh.n_edges == 188
    assert hh.n_edges - hh.n_qubits + 1 == 25            # 25 primitive loops (Results)
    deg = np.bincount(hh.edges.ravel())
    assert set(deg) == {2, 3} and len(hh.colors) == 3
    sq = w.square(10, 10)
    assert sq.n_edges == 180 and len(sq.colors) == 4
    ld = w.ladder(26)
    assert ld.n_qubits == 52 and ld.n_edges == 76


# ---------------------------------------------------------------- statevector
def test_statevector_gate_matches_kron():
    rng = np.random.default_rng(0)
    psi = rng.normal(size=(2, 2, 2)) + 1j * rng.normal(size=(2, 2, 2))
    U = scipy.linalg.expm(-1j * (rng.normal(size=(4, 4)) + rng.normal(size=(4, 4)).T))
    out = sv.apply_gate(psi, 0, 2, U)
    # q0=0 high bit, q1=2: reorder to (0,2,1) so the gate acts on the first two axes
    ref = (U @ np.transpose(psi, (0, 2, 1)).reshape(4, 2)).reshape(2, 2, 2)
    assert np.abs(out - np.transpose(ref, (0, 2, 1))).max() < 1e-14


# ---------------------------------------------------------------- simple update
@pytest.mark.parametrize("H,W,L,chi,kind", [
    (2, 2, 2, 16, "su4"), (2, 3, 2, 16, "su4"), (3, 3, 1, 4, "heis"), (4, 4, 1, 4, "heis"),
    (1, 5, 3, 8, "su4"),
])
def test_untruncated_simple_update_is_exact(H, W, L, chi, kind):
    """eps_i = 0 implies |psi_i> = G_i |psi_{i-1}> (Methods, after Eq. 1); checked to 1e-10."""
    lat = w.square(H, W)
    bits = w.domain_wall_bits(lat)
    groups = w.random_su4_circuit(lat, L, seed=5) if kind == "su4" else w.heisenberg_circuit(lat, L, 0.2)
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in groups:
        t.apply_group(g, chi)
        t.bp(500, 1e-12)
    assert max(t.eps) < 1e-14
    psi = sv.run(bits, groups)
    assert np.abs(t.statevector_bruteforce() - psi).max() < 1e-10


def test_one_qubit_gates_exact():
    lat = w.ladder(3)
    groups, bits = w.lucj_like_circuit(lat, reps=1, seed=3)
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in groups:
        t.apply_group(g, 64)
        t.bp(500, 1e-12)
    assert np.abs(t.statevector_bruteforce() - sv.run(bits, groups)).max() < 1e-10


def _tree_lattice(H, W):
    """Comb: every horizontal bond plus the vertical bonds of column 0 (a tree)."""
    grid = np.array([(r, c) for r in range(H) for c in range(W)], dtype=np.int32)
    edges = [(r * W + c, r * W + c + 1) for r in range(H) for c in range(W - 1)]
    edges += [(r * W, (r + 1) * W) for r in range(H - 1)]
    return w.Lattice("comb", grid, np.array(edges, dtype=np.int32), [[i] for i in range(len(edges))])


@pytest.mark.parametrize("shape", [(1, 6), (3, 3)])
def test_discarded_weight_exact_on_trees(shape):
    """Without loops BP is exact, so <psi|psi> = prod_i (1 - eps_i) (Eqs. 1-2 and the remark after them)."""
    H, W = shape
    lat = w.square(H, W) if H == 1 else _tree_lattice(H, W)
    bits = (np.arange(lat.n_qubits) % 2).astype(np.uint8)
    rng = np.random.default_rng(11)
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for _ in range(4):
        for (a, b) in lat.edges:
            z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
            U, _ = np.linalg.qr(z)
            t.apply_2q(int(a), int(b), U, chi=2)
            t.bp(500, 1e-13)
    assert max(t.eps) > 1e-3                      # truncation really happened
    nrm = np.sum(np.abs(t.statevector_bruteforce()) ** 2)
    assert abs(nrm - np.exp(t.log_fidelity)) < 1e-10


def test_bp_messages_are_exact_environments_on_tree():
    """On a tree the BP fixed point equals the exact environment of the cut bond (Methods, BP on trees).

    The message into (0,0) from (0,1) must equal the contraction of the branch
    {(0,1), (0,2)} of <psi|psi> with the cut bond left open.
    """
    lat = _tree_lattice(3, 3)
    t = GridTNS(lat.grid_rc, lat.edges, np.zeros(9, dtype=np.uint8))
    rng = np.random.default_rng(2)
    for _ in range(2):
        for (a, b) in lat.edges:
            z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
            t.apply_2q(int(a), int(b), np.linalg.qr(z)[0], chi=4)
    t.bp(500, 1e-14)
    a1 = t.T[0][1][:, 0, :, 0, :]          # s, l, r
    a2 = t.T[0][2][:, 0, :, 0, 0]          # s, l
    V = np.einsum("skj,tj->kst", a1, a2)
    env = np.einsum("kst,Kst->kK", V, V.conj())
    env /= np.linalg.norm(env)
    assert np.abs(env - t.msg[(0, 0, 4)]).max() < 1e-10


# ---------------------------------------------------------------- boundary MPS
def _state(H, W, L, chi, seed=None):
    lat = w.square(H, W)
    bits = w.domain_wall_bits(lat)
    groups = w.heisenberg_circuit(lat, L, 0.2) if seed is None else w.random_su4_circuit(lat, L, seed)
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in groups:
        t.apply_group(g, chi)
        t.bp(500, 1e-12)
    return lat, bits, groups, t


@pytest.mark.parametrize("exact", [False, True])
def test_truncate_full_rank_equals_svd(exact):
    rng = np.random.default_rng(4)
    T = rng.normal(size=(40, 12)) + 1j * rng.normal(size=(40, 12))
    K, C = bmps.truncate(T, 12, lambda n, k: None, exact=exact)
    assert np.abs(K @ C - T).max() < 1e-12
    assert np.abs(K.conj().T @ K - np.eye(12)).max() < 1e-12


def test_truncate_randomized_matches_optimal_rank_r():
    """With a decaying spectrum the range finder reaches the optimal (Eckart-Young) error."""
    rng = np.random.default_rng(5)
    U, _ = np.linalg.qr(rng.normal(size=(300, 120)) + 1j * rng.normal(size=(300, 120)))
    V, _ = np.linalg.qr(rng.normal(size=(200, 120)) + 1j * rng.normal(size=(200, 120)))
    s = 0.7 ** np.arange(120)
    T = (U * s) @ V.conj().T
    R = 20
    K, C = bmps.truncate(T, R, lambda n, k: philox.test_matrix(1, 0, 0, 0, n, k))
    err = np.linalg.norm(T - K @ C)
    opt = np.sqrt(np.sum(s[R:] ** 2))
    assert err < opt * (1 + 1e-6)
    Ke, Ce = bmps.truncate(T, R, None, exact=True)
    # subspace-iteration error ~ (s_{R+p}/s_R)^3 relative to s_R (HMT 2011, Cor. 10.10)
    assert np.abs(K @ C - Ke @ Ce).max() < 1e-6
    # the phase convention makes K itself agree with the exact SVD basis; the leading
    # singular vectors (far from the cut) agree to high accuracy
    assert np.abs(K[:, :10] - Ke[:, :10]).max() < 1e-7
    assert np.abs(K - Ke).max() < 1e-3


def test_truncate_flat_spectrum_converges_to_exact_svd():
    """Flat spectrum at the cut, shaped like the 10x10 chi_b = 64 zip matrices (power law
    sigma_i = (1 + 5.5 i / R)^-1.5: sigma_{R+1}/sigma_R = 0.96, sigma_2R/sigma_R = 0.39,
    sigma_R/sigma_1 = 0.063).  With k = 2R columns and q subspace iterations the angle
    between the kept subspace and the exact top-R singular subspace is about
    (sigma_{k+1}/sigma_R)^(2q+1) (Halko, Martinsson, Tropp 2011, Sec. 10), checked
    against LAPACK's SVD at q = 3 and q = 4; one iteration fewer fails the bound."""
    rng = np.random.default_rng(11)
    M, N, R = 512, 256, 32
    U, _ = np.linalg.qr(rng.normal(size=(M, N)) + 1j * rng.normal(size=(M, N)))
    V, _ = np.linalg.qr(rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))
    s = (1.0 + np.arange(N) * 5.5 / R) ** -1.5
    T = (U * s) @ V.conj().T
    Ke, Ce = bmps.truncate(T, R, None, exact=True)
    opt = np.sqrt(np.sum(s[R:] ** 2))
    assert abs(np.linalg.norm(T - Ke @ Ce) / opt - 1) < 1e-12          # Eckart-Young
    om = lambda n, k: philox.test_matrix(1, 0, 0, 0, n, k)
    for q in (3, 4):
        K, C = bmps.truncate(T, R, om, power_iters=q, oversample=R)
        pred = (s[2 * R] / s[R - 1]) ** (2 * q + 1)
        angle = np.linalg.norm(U[:, :R] - K @ (K.conj().T @ U[:, :R]), 2)
        assert angle < 1.5 * pred
        assert np.linalg.norm(K @ C - Ke @ Ce) / np.linalg.norm(T) < 0.1 * pred
        assert np.linalg.norm(T - K @ C) / opt - 1 < pred ** 2
    K, C = bmps.truncate(T, R, om, power_iters=2, oversample=R)
    angle = np.linalg.norm(U[:, :R] - K @ (K.conj().T @ U[:, :R]), 2)
    assert angle > 3 * (s[2 * R] / s[R - 1]) ** 7


@pytest.mark.parametrize("H,W,L,chi", [(3, 3, 1, 4), (4, 4, 1, 4), (2, 4, 2, 16)])
def test_sampler_exact_when_R_large(H, W, L, chi):
    """R -> infinity is exact (Appendix): q(x) = |<x|psi>|^2 / <psi|psi> for every sample."""
    lat, bits, groups, t = _state(H, W, L, chi)
    p = np.abs(sv.run(bits, groups)) ** 2
    E, log_norm = bmps.norm_envs(t, 256, 7)
    assert abs(np.exp(log_norm) - p.sum()) < 1e-10
    xs, logq, _ = bmps.sample(t, 256, 24, seed=3, env=E)
    for x, lq in zip(xs, logq):
        assert abs(np.exp(lq) - p[tuple(x)] / p.sum()) < 1e-10
    assert set(xs.sum(axis=1)) == {int(bits.sum())}           # U(1) sector (Results)


def test_conditionals_sum_to_one_by_enumeration():
    """Forced-path replay over all 2^n bitstrings: sum_x q(x) = 1 even when truncated."""
    lat, bits, groups, t = _state(2, 3, 2, 2, seed=9)
    assert max(t.eps) > 1e-4
    E, _ = bmps.norm_envs(t, 2, 7)
    allx = np.array([[(i >> q) & 1 for q in range(6)] for i in range(64)], dtype=np.uint8)
    _, logq, _ = bmps.sample(t, 2, 0, seed=1, forced=allx, env=E)
    assert abs(np.exp(logq).sum() - 1.0) < 1e-12


def test_replay_reproduces_draws():
    lat, bits, groups, t = _state(3, 3, 2, 4, seed=2)
    E, _ = bmps.norm_envs(t, 8, 7)
    xs, lq, q0 = bmps.sample(t, 8, 16, seed=44, env=E)
    _, lq2, q02 = bmps.sample(t, 8, 0, seed=44, forced=xs, env=E)
    assert np.abs(lq - lq2).max() < 1e-12 and np.abs(q0 - q02).max() < 1e-12
    u = np.stack([philox.draw_uniforms(44, i, np.arange(9)) for i in range(16)])
    assert ((u >= q0) == (xs == 1)).all()                     # x = 1 iff u >= q(0|prefix)


@pytest.mark.parametrize("H,W,L,chi", [(3, 3, 2, 4), (4, 3, 1, 4)])
def test_amplitude_matches_bruteforce(H, W, L, chi):
    lat, bits, groups, t = _state(H, W, L, chi, seed=6)
    rng = np.random.default_rng(1)
    for _ in range(5):
        x = rng.integers(0, 2, size=lat.n_qubits)
        la, ph = bmps.amplitude(t, 256, x, 3)
        ref = t.amplitude_bruteforce(x)
        assert abs(np.exp(la + 1j * ph) - ref) < 1e-10 * max(1.0, abs(ref))


def test_mean_ratio_estimates_norm_when_truncated():
    """E_{x~q}[p/q] = <psi|psi> (Methods): within 4 standard errors on 400 samples."""
    lat, bits, groups, t = _state(3, 3, 3, 2)
    p = np.abs(t.statevector_bruteforce()) ** 2
    xs, logq, _ = bmps.sample(t, 2, 400, seed=8)
    r = metrics.p_over_q(np.log(p[tuple(xs.T)]), logq)
    assert abs(r.mean() - p.sum()) < 4 * r.std() / np.sqrt(len(r)) + 1e-12
    assert metrics.kld(logq, np.log(p[tuple(xs.T)] / p.sum())) > -0.05


def test_heavy_hex_embedding_sampler_exact_small():
    """Empty grid cells (dimension-1 tensors) do not change the sampled distribution."""
    lat = w.heavy_hex(2, 3)
    bits = w.domain_wall_bits(lat)
    groups = w.heisenberg_circuit(lat, 1, 0.2)
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in groups:
        t.apply_group(g, 16)
        t.bp(500, 1e-12)
    p = np.abs(sv.run(bits, groups)) ** 2
    xs, logq, _ = bmps.sample(t, 64, 12, seed=2)
    for x, lq in zip(xs, logq):
        assert abs(np.exp(lq) - p[tuple(x)] / p.sum()) < 1e-10
