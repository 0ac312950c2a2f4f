"""Seeded synthetic workloads shared by the CPU oracle and the GB300 library.

Lattices (grid embeddings of square, heavy-hex and ladder processors) and the
circuits applied to them.  This package holds input definitions only; it does
not implement any step of the tensor-network simulation or sampling method.
"""
from .lattices import Lattice, square, heavy_hex, ladder, edge_index  # noqa: F401
from .circuits import (  # noqa: F401
    heisenberg_gate, givens_gate, phase_gate, cphase_gate, domain_wall_bits,
    heisenberg_circuit, disordered_heisenberg_circuit, lucj_like_circuit, random_su4_circuit, flatten_group,
)

from .made_init import made_init, epoch_orders  # noqa: F401

# Named configurations (sizes of the paper-shaped synthetic workloads).
CONFIGS = {
    "sq4x4": dict(lattice=("square", 4, 4), layers=4, dt=0.2, chi=4, chi_b=16, n_samples=1024),
    "sq10x10": dict(lattice=("square", 10, 10), layers=7, dt=0.2, chi=16, chi_b=64, n_samples=16384),
    "heavyhex164": dict(lattice=("heavy_hex", 6, 12), layers=20, dt=0.2, chi=32, chi_b=128, n_samples=32768),
    "ladder52": dict(lattice=("ladder", 26), reps=3, chi=64, chi_b=256, n_samples=4096),
}


def make_lattice(spec) -> Lattice:
    kind = spec[0]
    if kind == "square":
        return square(spec[1], spec[2])
    if kind == "heavy_hex":
        return heavy_hex(spec[1], spec[2])
    if kind == "ladder":
        return ladder(spec[1])
    raise ValueError(kind)
