"""TNSF fixture files: the oracle's own reader/writer of the library's state format.

TEST INFRASTRUCTURE ONLY.  Both implementations read and write this format so
that the sampler can be compared on one shared tensor-network state (the
truncated singular vectors of a simple update are only fixed up to gauge, so
two independently built states are equal as states but not as tensors).

Layout (little endian): "TNSF", u32 version=1, u32 H, W, n, transposed,
f64 log_fidelity, n x (u32 row, u32 col) cells of the qubits (oriented grid),
H*W x 4 u32 edge flags (u, l, d, r), then per cell (row-major) 5 u32 dims
(p, u, l, d, r) and the complex128 entries in [s][u][l][d][r] order, then per
cell and leg with an edge: u32 D and the D x D complex128 message into that
cell across that leg.
"""
from __future__ import annotations

import struct

import numpy as np

from .tns import GridTNS


def save(t: GridTNS, path: str) -> None:
    with open(path, "wb") as f:
        f.write(b"TNSF")
        f.write(struct.pack("<5I", 1, t.H, t.W, t.n, int(t.transposed)))
        f.write(struct.pack("<d", t.log_fidelity))
        for (r, c) in t.qubit_cell:
            f.write(struct.pack("<2I", r, c))
        for r in range(t.H):
            for c in range(t.W):
                f.write(struct.pack("<4I", *[int(t.has_edge(r, c, leg)) for leg in (1, 2, 3, 4)]))
        for r in range(t.H):
            for c in range(t.W):
                a = np.ascontiguousarray(t.T[r][c], dtype=np.complex128)
                f.write(struct.pack("<5I", *a.shape))
                f.write(a.tobytes())
        for r in range(t.H):
            for c in range(t.W):
                for leg in (1, 2, 3, 4):
                    if t.has_edge(r, c, leg):
                        m = np.ascontiguousarray(t.msg[(r, c, leg)], dtype=np.complex128)
                        f.write(struct.pack("<I", m.shape[0]))
                        f.write(m.tobytes())


def load(path: str) -> GridTNS:
    with open(path, "rb") as f:
        buf = f.read()
    if buf[:4] != b"TNSF":
        raise ValueError("not a TNSF file")
    off = 4
    ver, H, W, n, tr = struct.unpack_from("<5I", buf, off)
    off += 20
    if ver != 1:
        raise ValueError("unsupported TNSF version")
    (logf,) = struct.unpack_from("<d", buf, off)
    off += 8
    cells = []
    for _ in range(n):
        cells.append(struct.unpack_from("<2I", buf, off))
        off += 8
    t = GridTNS.__new__(GridTNS)
    t.H, t.W, t.n, t.transposed = H, W, n, bool(tr)
    t.qubit_cell = [tuple(map(int, x)) for x in cells]
    t.cell_qubit = -np.ones((H, W), dtype=np.int64)
    for q, (r, c) in enumerate(t.qubit_cell):
        t.cell_qubit[r, c] = q
    t.edge = {}
    for r in range(H):
        for c in range(W):
            flags = struct.unpack_from("<4I", buf, off)
            off += 16
            for leg, fl in zip((1, 2, 3, 4), flags):
                if fl:
                    t.edge[(r, c, leg)] = True
    t.T = [[None] * W for _ in range(H)]
    for r in range(H):
        for c in range(W):
            shape = struct.unpack_from("<5I", buf, off)
            off += 20
            cnt = int(np.prod(shape))
            t.T[r][c] = np.frombuffer(buf, dtype=np.complex128, count=cnt, offset=off).reshape(shape).copy()
            off += 16 * cnt
    t.msg = {}
    for r in range(H):
        for c in range(W):
            for leg in (1, 2, 3, 4):
                if (r, c, leg) in t.edge:
                    (D,) = struct.unpack_from("<I", buf, off)
                    off += 4
                    t.msg[(r, c, leg)] = np.frombuffer(buf, dtype=np.complex128, count=D * D,
                                                       offset=off).reshape(D, D).copy()
                    off += 16 * D * D
    t.log_fidelity = logf
    t.eps = []
    return t
