"""GPU parity of the hot path, through the C ABI, against the CPU oracle.

The sampler comparisons use a shared state: the oracle builds it, writes a TNSF
fixture, and the library loads the same tensors (truncated singular vectors are
only fixed up to gauge, so two independently built states are the same state but
not the same tensors).  States the library builds itself are checked through
their amplitudes against the oracle's statevector, never read by the oracle.  Tolerances: 1e-9 on probabilities in the FP64
path, 1e-4 on conditionals in the mixed path (FP32 contractions against an
FP64 oracle; the marginal bar of 1e-3 with a 10x margin).
"""
import os

import numpy as np
import pytest

import workloads as w
from oracle import bmps, fixture
from oracle import statevector as sv
from oracle.tns import GridTNS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_11424_gb300 as p
    from paper_2507_11424_gb300 import build
    build.build()
    p.load()
    return p


def gpu_state(pkg, lat, bits, groups, chi, prec="fp64", chi_max=None):
    st = pkg.TNSState(lat.grid_rc, lat.edges, bits, chi_max=chi_max or chi, prec=prec)
    eps = []
    for g in groups:
        eps.extend(st.apply_gate_layer(g, chi=chi))
        st.bp_gauge(500, 1e-12)
    return st, np.array(eps)


def oracle_state(lat, bits, groups, chi):
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in groups:
        t.apply_group(g, chi)
        t.bp(500, 1e-12)
    return t


def to_gpu(pkg, t, tmp_path, prec="fp64", name="s.tnsf"):
    """Load the oracle's state into the library (TNSF file written by the oracle)."""
    p = str(tmp_path / name)
    fixture.save(t, p)
    st = pkg.TNSState.load_file(p)
    st.n = t.n
    st.set_precision(prec)
    return st


def all_bits(n):
    """Every bitstring of n qubits, qubit 0 the most significant (statevector order)."""
    return ((np.arange(2 ** n)[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1).astype(np.uint8)


def gpu_statevector(st, n, chi_b=256):
    """<x|psi> for every x from the library's amplitudes (exact when chi_b covers the boundary)."""
    import torch
    la, ph = st.amplitude(chi_b, torch.tensor(all_bits(n), device="cuda"))
    return np.exp(la.cpu().numpy() + 1j * ph.cpu().numpy())


# ------------------------------------------------------------ gate layer / BP
@pytest.mark.parametrize("H,W,L,chi,kind", [(2, 3, 2, 16, "su4"), (3, 3, 1, 4, "heis"), (4, 4, 1, 4, "heis"),
                                            (1, 5, 3, 8, "su4")])
def test_untruncated_gate_layers_exact(pkg, tmp_path, H, W, L, chi, kind):
    lat = w.square(H, W)
    bits = w.domain_wall_bits(lat)
    groups = w.random_su4_circuit(lat, L, seed=5) if kind == "su4" else w.heisenberg_circuit(lat, L, 0.2)
    st, eps = gpu_state(pkg, lat, bits, groups, chi)
    assert eps.max() < 1e-14
    assert np.abs(gpu_statevector(st, lat.n_qubits) - sv.run(bits, groups).reshape(-1)).max() < 1e-10


def test_one_qubit_gates_and_ladder_orientation(pkg, tmp_path):
    lat = w.ladder(4)
    groups, bits = w.lucj_like_circuit(lat, reps=1, seed=3)
    st, _ = gpu_state(pkg, lat, bits, groups, 64)
    assert st.query()["transposed"]
    assert np.abs(gpu_statevector(st, lat.n_qubits) - sv.run(bits, groups).reshape(-1)).max() < 1e-10


def test_truncated_gate_errors_match_oracle(pkg, tmp_path):
    """Config-1 circuit (4x4, 4 layers, chi = 4): per-gate eps (Eq. 1) and log f (Eq. 2)."""
    lat = w.square(4, 4)
    bits = w.domain_wall_bits(lat)
    groups = w.heisenberg_circuit(lat, 4, 0.2)
    st, eps = gpu_state(pkg, lat, bits, groups, 4)
    t = oracle_state(lat, bits, groups, 4)
    assert eps.max() > 1e-3
    assert np.abs(eps - np.array(t.eps)).max() < 1e-8
    assert abs(st.log_fidelity() - t.log_fidelity) < 1e-8
    # the two states agree as states (gauge-invariant): compare statevectors
    assert np.abs(gpu_statevector(st, 16) - t.statevector_bruteforce().reshape(-1)).max() < 1e-7


def test_bp_reports_iterations_and_converges(pkg):
    lat = w.square(3, 3)
    bits = w.domain_wall_bits(lat)
    st, _ = gpu_state(pkg, lat, bits, w.heisenberg_circuit(lat, 2, 0.2)[:5], 4)
    it, res = st.bp_gauge(500, 1e-12)
    assert res < 1e-12 and it >= 1
    from paper_2507_11424_gb300 import TNSError
    st.apply_gate_layer(w.heisenberg_circuit(lat, 1, 0.2)[0], chi=4)
    with pytest.raises(TNSError) as ei:
        st.bp_gauge(1, 1e-30, strict=True)
    assert ei.value.code == 4          # TNS_ERR_NOT_CONVERGED, state still usable
    st.bp_gauge(500, 1e-12)


def test_mixed_bp_reaches_the_fp64_fixed_point(pkg):
    """Mixed-path BP (complex64 message contractions on the tensor cores, FP64
    Hermitisation and normalisation) against FP64 BP on the same circuit: 6x6 square
    lattice, 3 Heisenberg layers at chi = 16 (the third truncates), so the message contractions of the
    interior cells are large enough for the tensor cores.  The BP fixed point sets the
    gauge of every truncated gate, so per-gate truncation errors (Eq. 1) and log f
    (Eq. 2) agree to the FP32 rounding floor of the mixed messages; the device time,
    bytes and flops of the last call are reported."""
    lat = w.square(6, 6)
    bits = w.domain_wall_bits(lat)
    groups = w.heisenberg_circuit(lat, 3, 0.2)
    st64, eps64 = gpu_state(pkg, lat, bits, groups, 16, prec="fp64")
    st32, eps32 = gpu_state(pkg, lat, bits, groups, 16, prec="mixed")
    assert eps64.max() > 1e-4
    assert np.abs(eps32 - eps64).max() < 2e-5, np.abs(eps32 - eps64).max()
    assert abs(st32.log_fidelity() - st64.log_fidelity()) < 1e-4, (st32.log_fidelity(), st64.log_fidelity())
    # a fresh gate group, then a full mixed BP run from the stale messages
    st32.apply_gate_layer(w.heisenberg_circuit(lat, 1, 0.2)[0], chi=16)
    it, res = st32.bp_gauge(200, 1e-10)
    assert it >= 2 and res < 1e-3
    stats = st32.bp_stats()
    assert stats["ms"] > 0 and stats["bytes"] > 0 and stats["flops"] > 0
    st32.close()
    st64.close()


def test_invalid_gate_layers_rejected(pkg):
    from paper_2507_11424_gb300 import TNSError
    lat = w.square(3, 3)
    st = pkg.TNSState(lat.grid_rc, lat.edges, np.zeros(9, np.uint8), chi_max=4)
    U = w.heisenberg_gate(0.2)
    for grp in ([(0, 1, U), (1, 2, U)], [(0, 4, U)], [(0, 9, U)]):
        with pytest.raises(TNSError) as ei:
            st.apply_gate_layer(grp, chi=4)
        assert ei.value.code == 1
    with pytest.raises(TNSError):
        st.apply_gate_layer([(0, 1, U)], chi=8)          # chi > chi_max


# ------------------------------------------------------------ sampler
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
@pytest.mark.parametrize("shape", [(3, 3), (4, 4), (2, 5)])
def test_sampler_exact_when_R_large(pkg, shape, prec, tol):
    """R beyond the exact rank: q(x) = |<x|psi>|^2 / <psi|psi> (Appendix) for every sample."""
    lat = w.square(*shape)
    bits = w.domain_wall_bits(lat)
    groups = w.heisenberg_circuit(lat, 1, 0.2)
    st, _ = gpu_state(pkg, lat, bits, groups, 4, prec=prec)
    p = np.abs(sv.run(bits, groups)) ** 2
    xs, logq = st.sample(chi_b=256, n=37, seed=11)
    xs, logq = xs.cpu().numpy(), logq.cpu().numpy()
    assert (xs.sum(axis=1) == bits.sum()).all()                      # U(1) sector
    ref = np.log(p[tuple(xs.T)] / p.sum())
    assert np.abs(logq - ref).max() < tol


@pytest.mark.parametrize("prec,tol,tc", [("fp64", 1e-9, False), ("mixed", 1e-4, False), ("mixed", 1e-4, True)])
def test_sampler_matches_oracle_config1(pkg, tmp_path, prec, tol, tc):
    """Config 1 (4x4, L=4, chi=4, chi_b=16): conditionals along the GPU's draws equal the oracle's."""
    lat = w.square(4, 4)
    bits = w.domain_wall_bits(lat)
    t = oracle_state(lat, bits, w.heisenberg_circuit(lat, 4, 0.2), 4)
    st = to_gpu(pkg, t, tmp_path, prec)
    st.set_tensor_cores(tc)
    seed, n = 20250711, 48
    xs, logq, cond = st.sample(chi_b=16, n=n, seed=seed, cond=True)
    xs, logq, cond = xs.cpu().numpy(), logq.cpu().numpy(), cond.cpu().numpy()
    cut = bmps.ORTH_SHIFT
    _, lq_o, q0_o = bmps.sample(t, 16, 0, seed, forced=xs, gram_cut=cut)
    assert np.abs(cond - q0_o).max() < tol
    assert np.abs(logq - lq_o).max() < 20 * tol
    # the oracle's own draws with the same Philox stream give the same bits,
    # except where the uniform falls within the tolerance of the conditional
    xo, lqo, q0o = bmps.sample(t, 16, n, seed, gram_cut=cut)
    u = np.stack([__import__("oracle.philox", fromlist=["x"]).draw_uniforms(seed, i, np.arange(16)) for i in range(n)])
    close = np.abs(u - q0o) < 1e-3
    rows_ok = (xo == xs) | close.any(axis=1, keepdims=True)
    assert rows_ok.all()
    # replay entry point reproduces the conditionals
    import torch
    lq_r, cond_r = st.sample_replay(16, torch.tensor(xs, device="cuda"), seed)
    assert np.abs(cond_r.cpu().numpy() - cond).max() < 1e-12


def test_amplitude_matches_bruteforce(pkg, tmp_path):
    import torch
    lat = w.square(3, 4)
    bits = w.domain_wall_bits(lat)
    t = oracle_state(lat, bits, w.random_su4_circuit(lat, 1, seed=6), 4)
    st = to_gpu(pkg, t, tmp_path)
    rng = np.random.default_rng(3)
    xs = rng.integers(0, 2, size=(40, lat.n_qubits)).astype(np.uint8)
    for prec, tol in (("fp64", 1e-10), ("mixed", 1e-4)):
        st.set_precision(prec)
        la, ph = st.amplitude(256, torch.tensor(xs, device="cuda"))
        amp = np.exp(la.cpu().numpy() + 1j * ph.cpu().numpy())
        ref = np.array([t.amplitude_bruteforce(x) for x in xs])
        assert np.abs(amp - ref).max() < tol * np.abs(ref).max()


def test_amplitude_truncated_matches_oracle(pkg, tmp_path):
    import torch
    lat = w.square(4, 4)
    bits = w.domain_wall_bits(lat)
    t = oracle_state(lat, bits, w.heisenberg_circuit(lat, 4, 0.2), 4)
    st = to_gpu(pkg, t, tmp_path)
    xs, _ = st.sample(chi_b=16, n=12, seed=3)
    la, ph = st.amplitude(8, xs)
    la = la.cpu().numpy()
    for i, x in enumerate(xs.cpu().numpy()):
        lo, po = bmps.amplitude(t, 8, x, 0)
        assert abs(la[i] - lo) < 1e-9


def test_log_norm_matches_oracle(pkg, tmp_path):
    lat = w.square(4, 4)
    bits = w.domain_wall_bits(lat)
    t = oracle_state(lat, bits, w.heisenberg_circuit(lat, 4, 0.2), 4)
    st = to_gpu(pkg, t, tmp_path)
    # (R = 256 still truncates here: the exact boundary rank at row 1 is up to 16^3)
    for R in (4, 16, 64, 256):
        _, ln_o = bmps.norm_envs(t, R)
        assert abs(st.log_norm(R) - ln_o) < 1e-9


def test_heavy_hex_cells_and_edge_cases(pkg, tmp_path):
    """Empty grid cells (dimension-1 tensors), zero samples, a single sample."""
    lat = w.heavy_hex(2, 3)
    bits = w.domain_wall_bits(lat)
    groups = w.heisenberg_circuit(lat, 1, 0.2)
    st, _ = gpu_state(pkg, lat, bits, groups, 16)
    p = np.abs(sv.run(bits, groups)) ** 2
    xs, logq = st.sample(chi_b=64, n=1, seed=2)
    x = xs.cpu().numpy()[0]
    assert abs(logq.cpu().numpy()[0] - np.log(p[tuple(x)] / p.sum())) < 1e-9
    xs0, lq0 = st.sample(chi_b=64, n=0, seed=2)
    assert xs0.shape[0] == 0


def test_save_load_roundtrip(pkg, tmp_path):
    lat = w.square(3, 3)
    bits = w.domain_wall_bits(lat)
    st, _ = gpu_state(pkg, lat, bits, w.heisenberg_circuit(lat, 2, 0.2), 4)
    path = str(tmp_path / "a.tnsf")
    st.save(path)
    st2 = pkg.TNSState.load_file(path)
    st2.n = 9
    st2.set_precision("fp64")
    a, la = st.sample(16, 8, 5)
    b, lb = st2.sample(16, 8, 5)
    assert (a.cpu().numpy() == b.cpu().numpy()).all()
    assert np.abs(la.cpu().numpy() - lb.cpu().numpy()).max() < 1e-12
    # the format is shared with the oracle: an oracle-written file loads into the
    # library, and the library writes it back unchanged
    t = oracle_state(lat, bits, w.heisenberg_circuit(lat, 2, 0.2), 4)
    st3 = to_gpu(pkg, t, tmp_path, name="b.tnsf")
    st3.save(str(tmp_path / "c.tnsf"))
    back = fixture.load(str(tmp_path / "c.tnsf"))
    assert (back.H, back.W, back.n, back.transposed) == (t.H, t.W, t.n, t.transposed)
    assert back.log_fidelity == t.log_fidelity
    for r in range(t.H):
        for c in range(t.W):
            assert np.array_equal(back.T[r][c], t.T[r][c])
    assert back.msg.keys() == t.msg.keys()
    assert all(np.array_equal(back.msg[k], t.msg[k]) for k in t.msg)


def test_tensor_core_path_matches_cuda_cores(pkg, tmp_path):
    """Mixed path with environment GEMMs on tcgen05 vs on CUDA cores, and vs the oracle (5x5, chi = 8)."""
    lat = w.square(5, 5)
    bits = w.domain_wall_bits(lat)
    t = oracle_state(lat, bits, w.heisenberg_circuit(lat, 3, 0.2), 8)
    st = to_gpu(pkg, t, tmp_path, "mixed")
    R, seed, n = 32, 77, 16
    st.profile(True)
    st.set_tensor_cores(True)
    xs, lq1, c1 = st.sample(R, n, seed, cond=True)
    prof = st.profile_read()
    assert prof["env_gemm"]["launches"] > 0 and prof["tc_prep"]["launches"] > 0   # tensor cores really ran
    st.set_tensor_cores(False)
    xs2, lq2, c2 = st.sample(R, n, seed, cond=True)
    assert np.abs(c1.cpu().numpy() - c2.cpu().numpy()).max() < 1e-4
    _, lq_o, q0_o = bmps.sample(t, R, 0, seed, forced=xs.cpu().numpy(), gram_cut=bmps.ORTH_SHIFT)
    assert np.abs(c1.cpu().numpy() - q0_o).max() < 1e-4


@pytest.mark.parametrize("prec", ["mixed", "fp64"])
def test_graph_replay_equals_eager(pkg, tmp_path, prec):
    """The sampler's per-chunk CUDA graph (captured on the second call of a shape,
    replayed after) gives the same bits, log q and conditionals as eager launches,
    for new seeds, new output buffers, replays and ragged last chunks."""
    import torch
    lat = w.square(4, 4)
    bits = w.domain_wall_bits(lat)
    t = oracle_state(lat, bits, w.heisenberg_circuit(lat, 4, 0.2), 4)
    st_g = to_gpu(pkg, t, tmp_path, prec, "g.tnsf")
    st_e = to_gpu(pkg, t, tmp_path, prec, "e.tnsf")
    st_e.set_graphs(False)
    for seed, n in ((5, 24), (6, 24), (7, 24), (8, 24), (9, 10)):
        a = st_g.sample(16, n, seed, cond=True)
        b = st_e.sample(16, n, seed, cond=True)
        for x, y in zip(a, b):
            assert torch.equal(x, y)
        ra = st_g.sample_replay(16, a[0], seed)
        rb = st_e.sample_replay(16, a[0], seed)
        assert torch.equal(ra[1], rb[1]) and torch.equal(ra[1], a[2])
    # a replayed graph counts the kernels it launches
    assert st_g.launch_count() == st_e.launch_count()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sample_range_is_a_slice_of_the_stream(pkg, tmp_path, prec):
    """tns_sample_range(first, n) returns rows first .. first + n - 1 of the stream that
    tns_sample draws with the same seed (the sharding rule of the multi-device sampler),
    whatever the chunk it is drawn in: bit for bit in the FP64 path; in the mixed path
    the same bits, with conditionals and log q equal to FP32 rounding (a contraction
    whose rows span the chunk's samples can take the tensor cores or the CUDA cores
    depending on the chunk's size)."""
    import torch
    lat = w.square(4, 4)
    bits = w.domain_wall_bits(lat)
    t = oracle_state(lat, bits, w.heisenberg_circuit(lat, 4, 0.2), 4)
    st = to_gpu(pkg, t, tmp_path, prec, "r.tnsf")
    full = st.sample(16, 20, 99, cond=True)
    for first, n in ((0, 7), (7, 6), (13, 7), (19, 1)):
        part = st.sample(16, n, 99, cond=True, first=first)
        xs, lq, cq = part
        assert torch.equal(xs, full[0][first:first + n])
        if prec == "fp64":
            assert torch.equal(lq, full[1][first:first + n]) and torch.equal(cq, full[2][first:first + n])
        else:
            assert (lq - full[1][first:first + n]).abs().max().item() < 1e-5
            assert (cq - full[2][first:first + n]).abs().max().item() < 1e-6
    with pytest.raises(pkg.TNSError):
        st.sample(16, 2, 99, first=-1)
    st.close()
