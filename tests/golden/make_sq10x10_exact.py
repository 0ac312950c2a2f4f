"""Write the oracle's full-size reference draws for the 10x10 workload shape.

Calls only ``oracle/`` and ``workloads/``.  The state is a 10x10 square-lattice
domain-wall Heisenberg quench (7 Trotter layers, dt = 0.2) with one coupling per
bond drawn from U[0.8, 1.2] (``workloads.disordered_heisenberg_circuit``, seed
``J_SEED``), built by the oracle's BP-gauged simple update at chi = 16 with a fixed
number of BP sweeps after every gate group (``BP_SWEEPS``; the GPU test rebuilds the
same state with the same function, ``build_state``).  The couplings are disordered
because the uniform quench's truncations meet exactly degenerate singular values
(its lattice symmetries), where the kept basis, and hence the whole later state,
depends on the rounding of the host's LAPACK: a 1e-13 change of the gates moves its
per-gate truncation errors by 2e-6, so a state rebuilt on another machine is not the
state the reference was computed on.  With disordered couplings the same change moves
them by 7e-15.  The shapes (bond dimensions 16, boundary rank 64) and the launch
configuration are those of the uniform workload.  The oracle then samples it at boundary rank
chi_b = 64 with every truncation an exact truncated SVD (``exact=True``: the
plain definition of the compressor, Methods and Appendix "Sampling from a Tensor
Network State"), norm environments included, and stores per sample the drawn
bits, q(x_q = 0 | prefix) for every qubit, and log q(x).  Output:
``sq10x10_disordered_chib64_exact.npz`` next to this file (a few tens of KB).

    python tests/golden/make_sq10x10_exact.py [n_samples] [--save-envs PATH]

(--save-envs also pickles the exact norm environments, for studies of the
compressor; the test does not use them.)

Several CPU hours at most; the sampling seed is 20250711 (samples 0..n-1).
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402
from oracle import bmps  # noqa: E402
from oracle.tns import GridTNS  # noqa: E402

BP_SWEEPS = 4
SEED = 20250711
J_SEED = 2507
OUT = os.path.join(HERE, "sq10x10_disordered_chib64_exact.npz")


def build_state():
    """The oracle's 10x10 state: every gate group by simple update at chi = 16, then
    BP_SWEEPS parallel BP sweeps (warm started from the previous messages)."""
    cfg = w.CONFIGS["sq10x10"]
    lat = w.make_lattice(cfg["lattice"])
    bits = w.domain_wall_bits(lat)
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in w.disordered_heisenberg_circuit(lat, cfg["layers"], cfg["dt"], seed=J_SEED):
        t.apply_group(g, cfg["chi"])
        t.bp(BP_SWEEPS, 1e-10)
    return t, cfg, bits


def main():
    args = [a for a in sys.argv[1:] if not a.startswith("--")]
    n = int(args[0]) if args else 16
    env_path = sys.argv[sys.argv.index("--save-envs") + 1] if "--save-envs" in sys.argv else None
    t0 = time.time()
    t, cfg, bits0 = build_state()
    print(f"state {time.time() - t0:.0f} s, log f = {t.log_fidelity:.12f}", flush=True)
    R = cfg["chi_b"]
    E, log_norm = bmps.norm_envs(t, R, exact=True)
    print(f"environments {time.time() - t0:.0f} s, log <psi|psi> = {log_norm:.12f}", flush=True)
    if env_path:
        import pickle
        with open(env_path, "wb") as f:
            pickle.dump(E, f)
    bits = np.zeros((n, t.n), dtype=np.uint8)
    q0 = np.zeros((n, t.n))
    logq = np.zeros(n)
    for i in range(n):
        b, lq, q = bmps.sample(t, R, 1, SEED, sample_offset=i, env=E, exact=True)
        bits[i], logq[i], q0[i] = b[0], lq[0], q[0]
        print(f"sample {i} {time.time() - t0:.0f} s", flush=True)
        np.savez(OUT, bits=bits[: i + 1], q0=q0[: i + 1], logq=logq[: i + 1], log_norm=log_norm,
                 log_fidelity=t.log_fidelity, seed=SEED, chi_b=R, bp_sweeps=BP_SWEEPS, j_seed=J_SEED,
                 sector=int(bits0.sum()))


if __name__ == "__main__":
    main()
