"""Exact statevector simulation (<= ~22 qubits) used to pin the tensor-network oracle.

TEST INFRASTRUCTURE ONLY.  The exact state |psi_m> = prod_i G_i |psi_0> that the
paper's truncated simulation approximates (Methods, Eqs. 1-2).  Qubit q is bit q
of the basis-state tuple; the array is stored with axis q for qubit q.
"""
from __future__ import annotations

import numpy as np


def product_state(bits) -> np.ndarray:
    n = len(bits)
    psi = np.zeros((2,) * n, dtype=np.complex128)
    psi[tuple(int(b) for b in bits)] = 1.0
    return psi


def apply_gate(psi: np.ndarray, q0: int, q1: int, U: np.ndarray) -> np.ndarray:
    """Apply a 1- or 2-qubit gate (U[2*o0+o1, 2*i0+i1], q0 the high bit)."""
    n = psi.ndim
    if q1 < 0:
        out = np.tensordot(U, psi, axes=([1], [q0]))         # new axis 0 = q0
        return np.moveaxis(out, 0, q0)
    U4 = U.reshape(2, 2, 2, 2)
    out = np.tensordot(U4, psi, axes=([2, 3], [q0, q1]))      # axes: o0, o1, rest...
    rest = [a for a in range(n) if a not in (q0, q1)]
    order = [0] * n
    order[q0] = 0
    order[q1] = 1
    for pos, a in enumerate(rest):
        order[a] = 2 + pos
    return np.transpose(out, order)


def run(bits, groups) -> np.ndarray:
    psi = product_state(bits)
    for grp in groups:
        for (a, b, U) in grp:
            psi = apply_gate(psi, a, b, U)
    return psi


def probabilities(psi: np.ndarray) -> np.ndarray:
    return np.abs(psi) ** 2


def conditional(psi: np.ndarray, order, prefix_bits) -> float:
    """P(x_{order[k]} = 0 | x_{order[:k]} = prefix) for k = len(prefix_bits)."""
    p = probabilities(psi)
    idx = [slice(None)] * p.ndim
    for q, b in zip(order, prefix_bits):
        idx[q] = int(b)
    sub = p[tuple(idx)]
    k = len(prefix_bits)
    q = order[k]
    remaining = [a for a in range(p.ndim) if a not in order[:k]]
    axis = remaining.index(q)
    m = sub.sum(axis=tuple(a for a in range(sub.ndim) if a != axis))
    return float(m[0] / m.sum())
