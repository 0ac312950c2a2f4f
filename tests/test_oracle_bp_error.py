"""Pins of the oracle's BP loop error (oracle/bp_error.py): on a lattice that is one
loop the transfer matrix's trace is the norm <psi|psi> by brute force; product
states have eps = 0; 0 <= eps <= 1 - 1/chi^2 (Results); the spectrum does not depend
on where the loop is cut or on its orientation."""
import numpy as np
import pytest

import workloads as w
from oracle import bp_error as be
from oracle.tns import GridTNS


def _state(H, W, layers, chi, seed):
    lat = w.square(H, W)
    bits = w.domain_wall_bits(lat)
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in w.random_su4_circuit(lat, layers, seed=seed):
        t.apply_group(g, chi)
        t.bp(500, 1e-12)
    return t


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_single_loop_trace_is_the_norm(seed):
    t = _state(2, 2, 3, 16, seed)
    psi = t.statevector_bruteforce()
    T = be.loop_transfer(t, be.plaquettes(t)[0])
    assert abs(np.trace(T) - np.vdot(psi, psi).real) < 1e-12 * abs(np.vdot(psi, psi))


def test_product_state_has_no_loop_error():
    lat = w.square(3, 3)
    t = GridTNS(lat.grid_rc, lat.edges, w.domain_wall_bits(lat))
    t.bp(10, 1e-12)
    eps, errs = be.bp_error(t)
    assert eps == 0.0 and len(errs) == 4


def test_bounds_and_cut_invariance():
    t = _state(3, 3, 2, 4, 7)
    eps, errs = be.bp_error(t)
    chi = max(t.T[r][c].shape[leg] for r in range(3) for c in range(3) for leg in (1, 2, 3, 4))
    assert all(0.0 <= e <= 1 - 1 / chi ** 2 + 1e-12 for e in errs)
    cyc = be.plaquettes(t)[0]
    ref = np.sort(np.abs(np.linalg.eigvals(be.loop_transfer(t, cyc))))
    for k in range(1, 4):
        rot = cyc[k:] + cyc[:k]
        assert np.allclose(np.sort(np.abs(np.linalg.eigvals(be.loop_transfer(t, rot)))), ref, atol=1e-12 * ref.max())
    rev = np.sort(np.abs(np.linalg.eigvals(be.loop_transfer(t, cyc[::-1]))))
    assert np.allclose(rev, ref, atol=1e-12 * ref.max())
