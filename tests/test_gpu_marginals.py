"""Sampled marginals against exact ones, within shot noise (GPU).

The 4x4 workload (domain-wall Heisenberg quench, 4 layers, dt = 0.2, chi = 4) is
built by the CPU oracle and loaded into the library.  At boundary rank 256 every
boundary bond of the 4x4 grid is kept, so the sampler draws from
p(x) = |<x|psi>|^2 / <psi|psi> exactly (Appendix, "Sampling from a Tensor Network
State"); p itself comes from the oracle's brute-force contraction of the TNS.
16384 draws in the mixed path must reproduce every one-site marginal <n_i> and
every two-site marginal <n_i n_j> within the shot-noise band
|p_hat - p| <= z sqrt(p (1 - p) / N), with z the two-sided 3-sigma level
Bonferroni-adjusted over all 16 + 120 marginals.
"""
import numpy as np
import pytest

import workloads as w
from oracle import fixture
from oracle.tns import GridTNS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_11424_gb300 as p
    from paper_2507_11424_gb300 import build
    build.build()
    p.load()
    return p


def test_sampled_marginals_within_shot_noise(pkg, tmp_path):
    from scipy.stats import norm
    cfg = w.CONFIGS["sq4x4"]
    lat = w.make_lattice(cfg["lattice"])
    bits = w.domain_wall_bits(lat)
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in w.heisenberg_circuit(lat, cfg["layers"], cfg["dt"]):
        t.apply_group(g, cfg["chi"])
        t.bp(500, 1e-12)
    psi = t.statevector_bruteforce().reshape(-1)
    p = np.abs(psi) ** 2
    p /= p.sum()
    n = lat.n_qubits
    allx = ((np.arange(2 ** n)[:, None] >> (n - 1 - np.arange(n))[None, :]) & 1).astype(np.float64)
    one = p @ allx
    two = allx.T @ (p[:, None] * allx)

    path = str(tmp_path / "cfg1.tnsf")
    fixture.save(t, path)
    st = pkg.TNSState.load_file(path)
    st.n = n
    st.set_precision("mixed")
    N = 16384
    xs, _ = st.sample(256, N, seed=20250711)
    x = xs.cpu().numpy().astype(np.float64)
    one_hat = x.mean(0)
    two_hat = x.T @ x / N
    iu = np.triu_indices(n, 1)
    m = n + iu[0].size
    z = norm.ppf(1 - 0.0027 / (2 * m))
    band1 = z * np.sqrt(one * (1 - one) / N) + 1e-12
    band2 = z * np.sqrt(two[iu] * (1 - two[iu]) / N) + 1e-12
    assert np.all(np.abs(one_hat - one) <= band1), np.max(np.abs(one_hat - one) / band1)
    assert np.all(np.abs(two_hat[iu] - two[iu]) <= band2), np.max(np.abs(two_hat[iu] - two[iu]) / band2)
    # the U(1) charge of the domain wall is conserved by every gate: each draw keeps it
    assert np.all(x.sum(1) == bits.sum())
    st.close()


@pytest.mark.parametrize("H,W,L,chi,R,kind,prec,tol", [(4, 4, 4, 4, 16, "heis", "fp64", 1e-9),
                                                       (4, 4, 4, 4, 16, "heis", "mixed", 1e-4),
                                                       (4, 4, 2, 4, 8, "su4", "fp64", 1e-9),
                                                       (5, 4, 2, 4, 8, "heis", "fp64", 1e-9),
                                                       (3, 3, 1, 4, 64, "heis", "fp64", 1e-10)])
def test_direct_marginals_match_oracle(pkg, tmp_path, H, W, L, chi, R, kind, prec, tol):
    """tns_direct_marginals against oracle/bmps.direct_marginals on the same (oracle-built)
    state and rank: every one-site and same-row two-site marginal, truncated and exact."""
    from oracle import bmps
    lat = w.square(H, W)
    bits = w.domain_wall_bits(lat)
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    groups = w.heisenberg_circuit(lat, L, 0.2) if kind == "heis" else w.random_su4_circuit(lat, L, seed=5)
    for g in groups:
        t.apply_group(g, chi)
        t.bp(500, 1e-12)
    one_o, two_o = bmps.direct_marginals(t, R)
    path = str(tmp_path / "dm.tnsf")
    fixture.save(t, path)
    st = pkg.TNSState.load_file(path)
    st.n = t.n
    st.set_precision(prec)
    one, two = st.direct_marginals(R)
    assert np.abs(one - one_o).max() < tol
    mask = ~np.isnan(two_o)
    assert np.array_equal(mask, ~np.isnan(two))
    assert np.abs(two[mask] - two_o[mask]).max() < tol
    st.close()


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-9), ("mixed", 1e-4)])
def test_certification_matches_oracle(pkg, tmp_path, prec, tol):
    """tns_certify against oracle/bmps.certify: the oracle draws 24 samples at rank 8
    from its own 4x4 state (chi = 4, 4 layers); both certify them at rank 16 (log p,
    mean p/q, KL estimate).  The oracle's bits and log q are the input to both."""
    import torch
    from oracle import bmps
    lat = w.square(4, 4)
    bits0 = w.domain_wall_bits(lat)
    t = GridTNS(lat.grid_rc, lat.edges, bits0)
    for g in w.heisenberg_circuit(lat, 4, 0.2):
        t.apply_group(g, 4)
        t.bp(500, 1e-12)
    xs, logq, _ = bmps.sample(t, 8, 24, seed=31)
    ref = bmps.certify(t, xs, logq, 16)
    path = str(tmp_path / "cert.tnsf")
    fixture.save(t, path)
    st = pkg.TNSState.load_file(path)
    st.n = t.n
    st.set_precision(prec)
    logp, stats = st.certify(16, torch.tensor(xs, device="cuda"), torch.tensor(logq, device="cuda"))
    assert np.abs(logp.cpu().numpy() - ref["log_p"]).max() < tol * 10
    assert abs(stats["mean_ratio"] - ref["mean_ratio"]) < tol * 10
    assert abs(stats["kld"] - ref["kld"]) < tol * 10
    assert stats["n_finite"] == 24
    st.close()
