"""GPU learned proposal (MADE, Adam, ancestral sampling) and independent MH, through
the C ABI, against the CPU oracle in oracle/made.py.

Tolerances come from the arithmetic.  GEMM operands (masked weights, activations,
back-propagated errors) are rounded to BF16 (relative 2^-9) and accumulated in
FP32.  bf16_grad below rounds at the same points; with it, at n = 100, h = 256
and the initial weights, logit errors reach 3.3e-3 and log g errors 9.2e-3
against FP64, so log g is held to 3e-2.  The gradient is more sensitive: on the
correlated test data the rounding of the forward weights and activations alone
moves it by 1.9% and 1.5% (2.2% together; the rounding of the error signals adds
0.1%), so it is held to 1e-3 against the rounding model and 3e-2 against FP64.
"""
import numpy as np
import pytest

import workloads as w
from oracle import made, philox
from oracle import statevector as sv

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_11424_gb300 as p
    from paper_2507_11424_gb300 import build
    build.build()
    p.load()
    return p


def markov_bits(n_rows, n, stay=0.85, seed=3):
    """Correlated bitstrings: x_0 ~ Bernoulli(1/2), x_i = x_{i-1} with probability `stay`."""
    rng = np.random.default_rng(seed)
    x = np.zeros((n_rows, n), dtype=np.uint8)
    x[:, 0] = rng.random(n_rows) < 0.5
    flip = rng.random((n_rows, n)) >= stay
    for i in range(1, n):
        x[:, i] = x[:, i - 1] ^ flip[:, i]
    return x


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bf16(a):
    """Round to the nearest BF16 (ties to even), returned as float64."""
    u = np.asarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def bf16_grad(theta, x, n, h):
    """Mean-NLL gradient with BF16 operands at the library's rounding points (FP64 sums)."""
    W1, b1, W2, b2, W3, b3, W4, b4 = made.unpack(theta, n, h)
    Ws = [bf16(W * M) for W, M in zip((W1, W2, W3, W4), made.masks(n, h))]
    x = np.asarray(x, dtype=np.float64)
    B = x.shape[0]
    z1 = x @ Ws[0].T + b1
    a1 = bf16(np.maximum(z1, 0))
    z2 = a1 @ Ws[1].T + b2
    a2 = bf16(np.maximum(z2, 0))
    z3 = a2 @ Ws[2].T + b3
    a3 = bf16(np.maximum(z3, 0))
    l = a3 @ Ws[3].T + b4
    dl = (1 / (1 + np.exp(-l)) - x) / B
    d3 = (bf16(dl) @ Ws[3]) * (z3 > 0)
    d2 = (bf16(d3) @ Ws[2]) * (z2 > 0)
    d1 = (bf16(d2) @ Ws[1]) * (z1 > 0)
    M1, M2, M3, M4 = made.masks(n, h)
    return made.pack([(bf16(d1).T @ x) * M1, d1.sum(0), (bf16(d2).T @ a1) * M2, d2.sum(0),
                      (bf16(d3).T @ a2) * M3, d3.sum(0), (bf16(dl).T @ a3) * M4, dl.sum(0)])


@pytest.mark.parametrize("n,h,rows", [(100, 256, 1000), (20, 64, 77), (7, 5, 3)])
def test_logprob_matches_oracle(pkg, n, h, rows):
    theta = w.made_init(n, h, seed=7)
    x = markov_bits(rows, n)
    m = pkg.MADE(n, h, theta)
    got = m.log_prob(dev(x)).cpu().numpy()
    ref = made.log_prob(theta.astype(np.float64), x, n, h)
    assert np.abs(got - ref).max() <= 3e-2


def test_params_roundtrip(pkg):
    theta = w.made_init(12, 32, seed=7)
    m = pkg.MADE(12, 32, theta)
    assert np.array_equal(m.params(), theta)


@pytest.mark.parametrize("n,h,rows", [(100, 256, 1024), (20, 64, 300)])
def test_gradient_matches_oracle(pkg, n, h, rows):
    theta = w.made_init(n, h, seed=7)
    x = markov_bits(rows, n, seed=5)
    m = pkg.MADE(n, h, theta)
    loss, g = m.grad(dev(x))
    loss_ref, g_ref = made.loss_and_grad(theta.astype(np.float64), x, n, h)
    assert abs(loss - loss_ref) <= 3e-2 / 10 + 1e-3 * abs(loss_ref)
    assert np.linalg.norm(g - g_ref) <= 3e-2 * np.linalg.norm(g_ref)
    g_bf = bf16_grad(theta.astype(np.float64), x, n, h)
    assert np.linalg.norm(g - g_bf) <= 1e-3 * np.linalg.norm(g_bf)
    # masked-out weights have exactly zero gradient
    M = made.masks(n, h)
    off = 0
    for k, s in enumerate(made.shapes(n, h)):
        sz = int(np.prod(s))
        if k % 2 == 0:
            blockg = g[off:off + sz].reshape(s)
            assert np.all(blockg[M[k // 2] == 0] == 0)
        off += sz
    assert np.array_equal(m.params(), theta)   # grad leaves the parameters alone


def test_training_matches_oracle_and_learns(pkg):
    n, h, rows, batch, epochs, lr = 20, 64, 2048, 64, 5, 1e-2
    theta = w.made_init(n, h, seed=7)
    x = markov_bits(rows, n, seed=9)
    orders = w.epoch_orders(rows, epochs, seed=7)
    m = pkg.MADE(n, h, theta)
    losses = m.train(dev(x), batch, epochs, lr=lr, orders=orders)
    th_ref, losses_ref = made.train(theta.astype(np.float64), x, n, h, batch, epochs, lr=lr, orders=orders)
    # BF16 gradients steer a slightly different trajectory: the rounding model drifts by <= 0.7% here
    assert np.all(np.abs(losses - np.array(losses_ref)) <= 2e-2 * np.abs(losses_ref))
    # the Markov source has entropy ln 2 + (n-1) H(0.15) = 8.72 nats; uniform bits 13.86
    assert losses[-1] < losses[0] - 3.0
    held = markov_bits(512, n, seed=10)
    lp = m.log_prob(dev(held)).cpu().numpy()
    lp_ref = made.log_prob(th_ref, held, n, h)
    assert abs(lp.mean() - lp_ref.mean()) <= 2e-2 * abs(lp_ref.mean())
    # an Adam step moves a parameter by at most lr (1 - b1) / sqrt(1 - b2) = 3.17 lr (Kingma & Ba, Sec. 2.1)
    steps = epochs * (rows // batch)
    assert np.abs(m.params() - theta).max() <= 3.17 * lr * steps


def test_train_ragged_batches_and_natural_order(pkg):
    n, h, rows, batch = 9, 16, 1000, 384     # 384 + 384 + 232
    theta = w.made_init(n, h, seed=7)
    x = markov_bits(rows, n, seed=2)
    m = pkg.MADE(n, h, theta)
    losses = m.train(dev(x), batch, 2, lr=1e-3)
    _, losses_ref = made.train(theta.astype(np.float64), x, n, h, batch, 2, lr=1e-3)
    assert np.all(np.abs(losses - np.array(losses_ref)) <= 1e-2 * np.abs(losses_ref))


def test_ancestral_sampling(pkg):
    """Bits follow the Philox rule on the network's own conditionals: re-deriving
    each decision with the oracle's FP64 conditionals along the GPU bits may only
    disagree where the uniform lies within the BF16 error of q0."""
    n, h, N, seed = 30, 64, 4096, 20250711
    theta = w.made_init(n, h, seed=7)
    m = pkg.MADE(n, h, theta)
    x = markov_bits(2048, n, seed=4)
    m.train(dev(x), 256, 2, lr=3e-3, orders=w.epoch_orders(2048, 2, seed=7))
    th = m.params().astype(np.float64)
    bits_d, logg_d = m.sample(N, seed)
    bits, logg = bits_d.cpu().numpy(), logg_d.cpu().numpy()
    assert set(np.unique(bits)) <= {0, 1}
    l, _ = made.forward(th, bits.astype(np.float64), n, h)   # teacher-forced logits
    q0 = 1.0 / (1.0 + np.exp(l))
    k0, k1 = philox.split_seed(seed)
    sid = np.arange(N, dtype=np.uint64)
    mism = 0
    for i in range(n):
        w0, w1, _, _ = philox.philox4x32_10(sid & philox.MASK, sid >> np.uint64(32), np.full_like(sid, i),
                                            np.ones_like(sid), k0, k1)
        u = philox.u53(w0, w1)
        dec = (u >= q0[:, i]).astype(np.uint8)
        bad = dec != bits[:, i]
        assert np.all(np.abs(u[bad] - q0[bad, i]) < 1e-2)
        mism += int(bad.sum())
    assert mism <= 1e-3 * N * n
    # log g of the draw equals the library's own log g of the same bits (same logits)
    assert np.array_equal(logg, m.log_prob(bits_d).cpu().numpy())
    assert np.abs(logg - made.log_prob(th, bits, n, h)).max() <= 3e-2 + 1e-3 * np.abs(logg).max()
    # sample offsets: the draw for proposal s depends only on (seed, s)
    b2, _ = m.sample(N // 2 + 5, seed)
    assert np.array_equal(b2.cpu().numpy(), bits[: N // 2 + 5])


def test_mh_matches_oracle(pkg):
    rng = np.random.default_rng(0)
    C, T, seed = 300, 257, 99
    lpp, lgp = rng.normal(size=(C, T)) * 2, rng.normal(size=(C, T)) * 2
    lp0, lg0 = rng.normal(size=C), rng.normal(size=C)
    st, acc = pkg.mh_independent(dev(lpp), dev(lgp), dev(lp0), dev(lg0), seed)
    st_ref, acc_ref = made.mh_independent(lpp, lgp, lp0, lg0, seed)
    assert np.array_equal(st.cpu().numpy(), st_ref)
    assert np.array_equal(acc.cpu().numpy(), acc_ref)
    # with g = p every independent proposal is accepted
    st, acc = pkg.mh_independent(dev(lpp), dev(lpp), dev(lp0), dev(lp0), seed)
    assert np.all(acc.cpu().numpy() == T)
    assert np.array_equal(st.cpu().numpy(), np.tile(np.arange(T, dtype=np.int32), (C, 1)))


def test_mh_edge_cases(pkg):
    import torch
    e = torch.zeros(0, dtype=torch.float64, device="cuda")
    st, acc = pkg.mh_independent(e.reshape(0, 5), e.reshape(0, 5), e, e, 1)
    assert st.shape == (0, 5) and acc.shape == (0,)
    z = torch.zeros(4, dtype=torch.float64, device="cuda")
    st, acc = pkg.mh_independent(z.reshape(4, 1)[:, :0], z.reshape(4, 1)[:, :0], z, z, 1)
    assert st.shape == (4, 0) and np.all(acc.cpu().numpy() == 0)


def test_learned_mh_corrects_a_poor_proposal(pkg):
    """16 qubits (4x4, one layer of random two-qubit gates, no truncation).  The
    untrained MADE is a poor proposal; independent MH with target |<x|psi>|^2 from
    the library's amplitudes recovers the exact single-site marginals, which the
    raw proposals miss by many standard errors."""
    lat = w.square(4, 4)
    bits0 = w.domain_wall_bits(lat)
    groups = w.random_su4_circuit(lat, 1, seed=5)
    st = pkg.TNSState(lat.grid_rc, lat.edges, bits0, chi_max=16, prec="fp64")
    for g in groups:
        st.apply_gate_layer(g, chi=16)
        st.bp_gauge(500, 1e-12)
    n, h, chi_b = lat.n_qubits, 32, 64      # chi_b = 64 keeps every boundary bond of the 4x4 grid exact
    allx = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    la, _ = st.amplitude(chi_b, dev(allx))
    p = np.exp(2 * la.cpu().numpy())
    p /= p.sum()
    exact = p @ allx
    psi = sv.run(bits0, groups).reshape(-1)
    assert np.abs(np.sort(p) - np.sort(np.abs(psi) ** 2)).max() < 1e-10   # same distribution as the circuit

    Cn, T = 512, 128
    m = pkg.MADE(n, h, w.made_init(n, h, seed=7))
    prop, lg = m.sample(Cn * T, seed=5)
    lp = 2 * st.amplitude(chi_b, prop)[0]
    sb, _ = st.sample(chi_b, Cn, seed=7)           # chain starts: exact plain-sampler draws
    lg0 = m.log_prob(sb)
    lp0 = 2 * st.amplitude(chi_b, sb)[0]
    state, acc = pkg.mh_independent(lp.reshape(Cn, T), lg.reshape(Cn, T), lp0, lg0, seed=8)
    state = state.cpu().numpy()
    propn, sbn = prop.cpu().numpy().reshape(Cn, T, n), sb.cpu().numpy()
    held = np.take_along_axis(propn, np.maximum(state, 0)[..., None], 1)
    chain = np.where(state[..., None] >= 0, held, sbn[:, None, :])
    est = chain.reshape(-1, n).mean(0)
    raw = propn.reshape(-1, n).mean(0)
    rate = acc.cpu().numpy().mean() / T
    assert 0.05 < rate < 0.95
    # correlated chain: inflate the binomial variance by (1 + rho) / (1 - rho) <= 2 / rate
    se = np.sqrt(exact * (1 - exact) / (Cn * T) * 2 / rate)
    assert np.all(np.abs(est - exact) <= 5 * se)
    assert np.abs(raw - exact).max() > 20 * np.sqrt(0.25 / (Cn * T))


def test_trained_proposal_gains_over_untrained(pkg):
    """What training buys: the MADE fitted to the plain sampler's draws (the method
    without the network) against the same network untrained, on the 16-qubit state
    above, at equal cost (the same number of proposals, chains and steps).  Trained:
    smaller KL(p || g), a higher MH acceptance rate, and chain marginals closer to
    the exact ones."""
    lat = w.square(4, 4)
    bits0 = w.domain_wall_bits(lat)
    groups = w.random_su4_circuit(lat, 1, seed=5)
    st = pkg.TNSState(lat.grid_rc, lat.edges, bits0, chi_max=16, prec="mixed")
    for g in groups:
        st.apply_gate_layer(g, chi=16)
        st.bp_gauge(500, 1e-12)
    n, h, chi_b = lat.n_qubits, 32, 64
    allx = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    la, _ = st.amplitude(chi_b, dev(allx))
    lp_all = 2 * la.cpu().numpy()
    p = np.exp(lp_all - lp_all.max())
    p /= p.sum()
    exact = p @ allx

    train, _ = st.sample(chi_b, 8192, seed=11)           # the plain sampler's draws
    theta0 = w.made_init(n, h, seed=7)
    trained, untrained = pkg.MADE(n, h, theta0), pkg.MADE(n, h, theta0)
    losses = trained.train(train, 256, 15, lr=3e-3, orders=w.epoch_orders(8192, 15, seed=3))
    assert losses[-1] < losses[0]

    def kl(m):
        lg = m.log_prob(dev(allx)).cpu().numpy()
        keep = p > 0
        return float(np.sum(p[keep] * (np.log(p[keep]) - lg[keep])))

    Cn, T = 256, 64
    sb, _ = st.sample(chi_b, Cn, seed=7)
    lp0 = 2 * st.amplitude(chi_b, sb)[0]
    res = {}
    for name, m in (("trained", trained), ("untrained", untrained)):
        prop, lg = m.sample(Cn * T, seed=5)
        lp = 2 * st.amplitude(chi_b, prop)[0]
        state, acc = pkg.mh_independent(lp.reshape(Cn, T), lg.reshape(Cn, T), lp0, m.log_prob(sb), seed=8)
        state = state.cpu().numpy()
        propn, sbn = prop.cpu().numpy().reshape(Cn, T, n), sb.cpu().numpy()
        held = np.take_along_axis(propn, np.maximum(state, 0)[..., None], 1)
        chain = np.where(state[..., None] >= 0, held, sbn[:, None, :])
        res[name] = dict(kl=kl(m), rate=acc.cpu().numpy().mean() / T,
                         err=np.abs(chain.reshape(-1, n).mean(0) - exact).max())
    t, u = res["trained"], res["untrained"]
    assert t["kl"] < 0.5 * u["kl"], res
    assert t["rate"] > 1.5 * u["rate"] and t["rate"] > 0.3, res
    assert t["err"] < u["err"], res
