"""Synthetic circuits shaped like the paper's workloads (seeded input generators).

A circuit is a list of *groups*; each group is a list of gates acting on
disjoint qubits (one edge colour, or one layer of single-qubit gates), matching
the paper's schedule of re-running belief propagation between groups of
non-overlapping gates (Methods, "Quantum Circuit Simulation").

A gate is ``(q0, q1, U)`` with ``U`` a 4x4 complex128 matrix indexed
``U[2*o0 + o1, 2*i0 + i1]`` (q0 is the high bit), or ``(q0, -1, U)`` with a
2x2 single-qubit ``U``.  Nothing here performs any step of the tensor-network
method; these are the workload definitions both implementations read.
"""
from __future__ import annotations

import numpy as np

from .lattices import Lattice

I2 = np.eye(2, dtype=np.complex128)
SWAP = np.array([[1, 0, 0, 0], [0, 0, 1, 0], [0, 1, 0, 0], [0, 0, 0, 1]], dtype=np.complex128)


def heisenberg_gate(dt: float, J: float = 1.0) -> np.ndarray:
    """exp(-i J dt (XX + YY + ZZ)) for one bond (Eqs. HeisenbergProp).

    Uses XX+YY+ZZ = 2 SWAP - I, so the gate is
    e^{i J dt} (cos(2 J dt) I - i sin(2 J dt) SWAP).
    """
    a = J * dt
    return np.exp(1j * a) * (np.cos(2 * a) * np.eye(4) - 1j * np.sin(2 * a) * SWAP)


def givens_gate(theta: float) -> np.ndarray:
    """Particle-number preserving XX+YY rotation exp(-i theta/4 (XX+YY))."""
    c, s = np.cos(theta / 2), np.sin(theta / 2)
    U = np.eye(4, dtype=np.complex128)
    U[1, 1] = c
    U[2, 2] = c
    U[1, 2] = -1j * s
    U[2, 1] = -1j * s
    return U


def phase_gate(phi: float) -> np.ndarray:
    return np.diag([1.0, np.exp(1j * phi)]).astype(np.complex128)


def cphase_gate(phi: float) -> np.ndarray:
    return np.diag([1.0, 1.0, 1.0, np.exp(1j * phi)]).astype(np.complex128)


def domain_wall_bits(lat: Lattice) -> np.ndarray:
    """Left half of the grid embedding in |0>, right half in |1>."""
    cols = lat.grid_rc[:, 1]
    split = (int(cols.max()) + 1) / 2.0
    return (cols >= split).astype(np.uint8)


def heisenberg_circuit(lat: Lattice, layers: int, dt: float, J: float = 1.0) -> list:
    """First-order Trotter circuit over the lattice's edge colouring (Eq. HeisenbergProp)."""
    U = heisenberg_gate(dt, J)
    groups = []
    for _ in range(layers):
        for col in lat.colors:
            groups.append([(int(lat.edges[e][0]), int(lat.edges[e][1]), U) for e in col])
    return groups


def disordered_heisenberg_circuit(lat: Lattice, layers: int, dt: float, seed: int, spread: float = 0.2) -> list:
    """The Trotter circuit of heisenberg_circuit with one coupling J_e per bond, drawn
    once from U[1 - spread, 1 + spread] (seeded, PCG64).  Random couplings remove the
    lattice symmetries of the uniform quench, whose truncations meet exactly degenerate
    singular values (so the truncated state depends on rounding); here every cut is
    generic and the state is reproducible across platforms."""
    rng = np.random.Generator(np.random.PCG64(seed))
    J = rng.uniform(1.0 - spread, 1.0 + spread, size=len(lat.edges))
    gates = [heisenberg_gate(dt, float(j)) for j in J]
    groups = []
    for _ in range(layers):
        for col in lat.colors:
            groups.append([(int(lat.edges[e][0]), int(lat.edges[e][1]), gates[e]) for e in col])
    return groups


def lucj_like_circuit(lat: Lattice, reps: int = 3, seed: int = 11424) -> tuple[list, np.ndarray]:
    """LUCJ-shaped ladder circuit (synthetic stand-in for the IBM LUCJ circuits).

    Two registers (ladder rows).  Each repetition: a depth-n brick network of
    Givens (XX+YY) rotations in each register with angles U[0, 2pi), a phase gate
    on every site with phases U[0, 2pi), and a controlled phase on every rung with
    phases U[0, pi).  A final Givens network closes the circuit.  Initial state:
    the first half of each register filled (|1>).
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    n = lat.n_qubits // 2

    def givens_network():
        gs = []
        for depth in range(n):
            start = depth % 2
            grp = []
            for reg in range(2):
                for i in range(start, n - 1, 2):
                    grp.append((reg * n + i, reg * n + i + 1, givens_gate(rng.uniform(0, 2 * np.pi))))
            gs.append(grp)
        return gs

    groups = []
    for _ in range(reps):
        groups.extend(givens_network())
        groups.append([(q, -1, phase_gate(rng.uniform(0, 2 * np.pi))) for q in range(2 * n)])
        groups.append([(i, n + i, cphase_gate(rng.uniform(0, np.pi))) for i in range(n)])
    groups.extend(givens_network())
    bits = np.zeros(2 * n, dtype=np.uint8)
    for reg in range(2):
        bits[reg * n: reg * n + (n + 1) // 2] = 1
    return groups, bits


def random_su4_circuit(lat: Lattice, layers: int, seed: int) -> list:
    """Haar-ish random two-qubit gates over the colouring (test workload only)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    groups = []
    for _ in range(layers):
        for col in lat.colors:
            grp = []
            for e in col:
                z = rng.normal(size=(4, 4)) + 1j * rng.normal(size=(4, 4))
                q, r = np.linalg.qr(z)
                q = q * (np.diag(r) / np.abs(np.diag(r)))
                grp.append((int(lat.edges[e][0]), int(lat.edges[e][1]), q))
            groups.append(grp)
    return groups


def flatten_group(group: list) -> tuple[np.ndarray, np.ndarray]:
    """Pack a group into the C-ABI arrays: sites int32 [g,2], mats float64 [g,16,2]."""
    g = len(group)
    sites = np.full((g, 2), -1, dtype=np.int32)
    mats = np.zeros((g, 16, 2), dtype=np.float64)
    for i, (a, b, U) in enumerate(group):
        sites[i, 0] = a
        sites[i, 1] = b
        flat = np.asarray(U, dtype=np.complex128).reshape(-1)
        mats[i, : flat.size, 0] = flat.real
        mats[i, : flat.size, 1] = flat.imag
    return sites, mats
