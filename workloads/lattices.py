"""Processor-shaped lattices embedded on a 2D grid (seeded input generators).

Each lattice is returned as a plain description that both the CPU oracle and
the C-ABI library consume:

* ``grid_rc``  int32 [n_qubits, 2]   (row, col) grid cell of every qubit,
* ``edges``    int32 [n_edges, 2]    qubit pairs joined by a tensor-network bond,
* ``colors``   list of lists of edge indices; every list is a matching
                (no qubit twice), i.e. one group of non-overlapping gates.

Every edge joins two grid cells that are nearest neighbours on the grid, so a
boundary-MPS sweep over grid rows sees a line of partitions (the paper's
"partitions whose quotient graph is a line", Methods, boundary-MPS section).
Nothing in this module performs any step of the tensor-network method.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class Lattice:
    name: str
    grid_rc: np.ndarray            # [n, 2] int32
    edges: np.ndarray              # [m, 2] int32
    colors: list = field(default_factory=list)   # list[list[int]] edge ids

    @property
    def n_qubits(self) -> int:
        return int(self.grid_rc.shape[0])

    @property
    def n_edges(self) -> int:
        return int(self.edges.shape[0])

    def check(self) -> None:
        """Validate the embedding: unique cells, grid-adjacent edges, proper colouring."""
        cells = {tuple(map(int, rc)) for rc in self.grid_rc}
        assert len(cells) == self.n_qubits, "two qubits share a grid cell"
        seen = set()
        for a, b in self.edges:
            ra, ca = self.grid_rc[a]
            rb, cb = self.grid_rc[b]
            assert abs(int(ra) - int(rb)) + abs(int(ca) - int(cb)) == 1, "edge not grid-adjacent"
            key = (min(a, b), max(a, b))
            assert key not in seen, "duplicate edge"
            seen.add(key)
        covered = []
        for grp in self.colors:
            used = set()
            for e in grp:
                a, b = map(int, self.edges[e])
                assert a not in used and b not in used, "colour class is not a matching"
                used.update((a, b))
            covered.extend(grp)
        if self.colors:
            assert sorted(covered) == list(range(self.n_edges)), "colouring misses edges"


def square(H: int, W: int) -> Lattice:
    """H x W square lattice (the Willow-like z=4 geometry, Methods).

    Qubit q = r*W + c.  Colours in the order H-even, H-odd, V-even, V-odd, where
    even/odd is the column (row) index of the left (top) site of the edge.
    """
    grid = np.array([(r, c) for r in range(H) for c in range(W)], dtype=np.int32)
    edges, groups = [], {"he": [], "ho": [], "ve": [], "vo": []}
    for r in range(H):
        for c in range(W):
            q = r * W + c
            if c + 1 < W:
                groups["he" if c % 2 == 0 else "ho"].append(len(edges))
                edges.append((q, q + 1))
            if r + 1 < H:
                groups["ve" if r % 2 == 0 else "vo"].append(len(edges))
                edges.append((q, q + W))
    colors = [g for g in (groups["he"], groups["ho"], groups["ve"], groups["vo"]) if g]
    lat = Lattice(f"square{H}x{W}", grid, np.array(edges, dtype=np.int32).reshape(-1, 2), colors)
    lat.check()
    return lat


def _bipartite_edge_coloring(n: int, edges: list[tuple[int, int]], n_colors: int) -> list[int]:
    """Proper edge colouring of a bipartite graph with max degree <= n_colors.

    Standard alternating-path (Koenig) construction: colour edges in order; when
    the two endpoints have no common free colour, flip the alternating a/b path
    starting at the second endpoint.  Deterministic given the edge order.
    """
    col_at = [dict() for _ in range(n)]      # vertex -> {colour: edge}
    color = [-1] * len(edges)

    def free(v):
        return [c for c in range(n_colors) if c not in col_at[v]]

    for e, (u, v) in enumerate(edges):
        fu, fv = free(u), free(v)
        common = [c for c in fu if c in fv]
        if common:
            c = common[0]
        else:
            a, b = fu[0], fv[0]
            # walk the path from v alternating colours a, b, b-edges then a-edges...
            path, x, want = [], v, a
            while want in col_at[x]:
                pe = col_at[x][want]
                path.append(pe)
                p, q = edges[pe]
                x = q if p == x else p
                want = b if want == a else a
            for pe in path:                      # swap a <-> b along the path
                p, q = edges[pe]
                old = color[pe]
                del col_at[p][old]
                del col_at[q][old]
            for pe in path:
                p, q = edges[pe]
                new = b if color[pe] == a else a
                color[pe] = new
                col_at[p][new] = pe
                col_at[q][new] = pe
            c = a
        color[e] = c
        col_at[u][c] = e
        col_at[v][c] = e
    return color


def heavy_hex(rows: int = 6, cols: int = 12, prune: bool = True) -> Lattice:
    """Heavy-hex lattice: brick-wall honeycomb with a bridge qubit on every edge.

    Honeycomb vertices (r, c), r < rows, c < cols; horizontal edges (r,c)-(r,c+1);
    vertical edge (r,c)-(r+1,c) iff (r + c) is even.  Degree-1 vertices (and their
    single edge) are removed when ``prune``; 6x12 then gives 70 vertices + 94
    bridges = 164 qubits with 25 primitive loops (the 164-qubit heavy-hex device
    of the Results section).  Grid embedding: vertex (r,c) -> (2r, 2c); the
    bridge of a horizontal edge -> (2r, 2c+1); of a vertical edge -> (2r+1, 2c).
    """
    verts = [(r, c) for r in range(rows) for c in range(cols)]
    hon = []
    for r in range(rows):
        for c in range(cols):
            if c + 1 < cols:
                hon.append(((r, c), (r, c + 1)))
            if r + 1 < rows and (r + c) % 2 == 0:
                hon.append(((r, c), (r + 1, c)))
    if prune:
        while True:
            deg = {v: 0 for v in verts}
            for a, b in hon:
                deg[a] += 1
                deg[b] += 1
            ones = {v for v in verts if deg[v] <= 1}
            if not ones:
                break
            verts = [v for v in verts if v not in ones]
            hon = [(a, b) for a, b in hon if a not in ones and b not in ones]
    cells, index = [], {}
    for (r, c) in verts:
        index[("v", r, c)] = len(cells)
        cells.append((2 * r, 2 * c))
    edges = []
    for (a, b) in hon:
        (ra, ca), (rb, cb) = a, b
        if ra == rb:
            cell = (2 * ra, 2 * ca + 1)
        else:
            cell = (2 * ra + 1, 2 * ca)
        bi = len(cells)
        cells.append(cell)
        edges.append((index[("v",) + a], bi))
        edges.append((bi, index[("v",) + b]))
    # sort qubits by grid cell (row-major) for a readable numbering
    order = sorted(range(len(cells)), key=lambda i: cells[i])
    new_of = {old: new for new, old in enumerate(order)}
    grid = np.array([cells[o] for o in order], dtype=np.int32)
    edges = sorted((min(new_of[a], new_of[b]), max(new_of[a], new_of[b])) for a, b in edges)
    color = _bipartite_edge_coloring(len(cells), edges, 3)
    colors = [[e for e in range(len(edges)) if color[e] == k] for k in range(3)]
    lat = Lattice(f"heavyhex{rows}x{cols}", grid, np.array(edges, dtype=np.int32), colors)
    lat.check()
    return lat


def ladder(n_per_register: int = 26) -> Lattice:
    """Two registers of ``n_per_register`` qubits (rows 0 and 1) joined by rungs.

    Qubit q = reg * n + i.  Colours: intra-register even bonds, odd bonds, rungs.
    """
    n = n_per_register
    grid = np.array([(reg, i) for reg in range(2) for i in range(n)], dtype=np.int32)
    edges, even, odd, rungs = [], [], [], []
    for reg in range(2):
        for i in range(n - 1):
            (even if i % 2 == 0 else odd).append(len(edges))
            edges.append((reg * n + i, reg * n + i + 1))
    for i in range(n):
        rungs.append(len(edges))
        edges.append((i, n + i))
    lat = Lattice(f"ladder2x{n}", grid, np.array(edges, dtype=np.int32), [even, odd, rungs])
    lat.check()
    return lat


def edge_index(lat: Lattice) -> dict:
    """Map an unordered qubit pair to its edge id."""
    return {(min(int(a), int(b)), max(int(a), int(b))): e for e, (a, b) in enumerate(lat.edges)}
