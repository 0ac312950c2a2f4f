"""The other workload shapes on the GPU: heavy-hex lattices (ragged degrees 2/3,
empty grid cells, boundary along the transposed short side) and LUCJ-like ladders
(two registers, boundary of length 2, one-qubit phase layers).

Reduced instances of the same constructions as the full-size workloads, built by
the CPU oracle and loaded into the library; the library draws samples and the
oracle replays them with the same settings (range-finder test matrices keyed by
the same seed): every conditional to 1e-8 in the FP64 path and 5e-4 in the mixed
path (half the metric's 1e-3 bar; FP32 orthonormalisation at shift 1e-5 and FP32
Jacobi give ~1e-4 here).  The full-size shapes are timed by bench.py --config heavyhex164 / ladder52.
"""
import numpy as np
import pytest

import workloads as w
from oracle import bmps, fixture
from oracle.tns import GridTNS

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import paper_2507_11424_gb300 as p
    from paper_2507_11424_gb300 import build
    build.build()
    p.load()
    return p


def _oracle_state(kind):
    if kind == "heavy_hex":
        lat = w.heavy_hex(4, 6)
        bits = w.domain_wall_bits(lat)
        groups = w.heisenberg_circuit(lat, 3, 0.2)
        chi, R = 8, 32
    else:
        lat = w.ladder(10)
        groups, bits = w.lucj_like_circuit(lat, reps=1, seed=11424)
        chi, R = 16, 64
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in groups:
        t.apply_group(g, chi)
        t.bp(200, 1e-12)
    return t, R


@pytest.mark.parametrize("kind", ["heavy_hex", "ladder"])
@pytest.mark.parametrize("prec,tol", [("fp64", 1e-8), ("mixed", 5e-4)])
def test_shape_conditionals_match_oracle(pkg, tmp_path, kind, prec, tol):
    t, R = _oracle_state(kind)
    path = str(tmp_path / f"{kind}.tnsf")
    fixture.save(t, path)
    st = pkg.TNSState.load_file(path)
    st.n = t.n
    st.set_precision(prec)
    seed = 424242
    xs, logq, cond = st.sample(R, 6, seed, cond=True)
    xs, logq, cond = xs.cpu().numpy(), logq.cpu().numpy(), cond.cpu().numpy()
    _, lq_o, q0_o = bmps.sample(t, R, 0, seed, forced=xs)
    assert np.abs(cond - q0_o).max() < tol
    assert np.abs(logq - lq_o).max() < 50 * tol
    st.close()
