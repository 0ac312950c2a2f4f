"""CPU oracle for the tensor-network state: lattice, BP messages, gauged simple update.

TEST INFRASTRUCTURE ONLY: imported by tests/, the smoke check and the timed CPU
baseline, never by the product path.  Plain complex128 numpy/LAPACK, written
from the paper's Methods and Appendix; slow and direct on purpose.

Data layout (shared *format* with the library's fixture files, not code):
the lattice lives on an H x W grid (transposed at build time when W > H so
that the boundary MPS of the sampler runs along the shorter side).  Every grid
cell holds a tensor psi[s, u, l, d, r] (physical, up, left, down, right); cells
with no qubit have physical dimension 1, and legs without an edge have
dimension 1.  Messages are stored per receiving cell and leg:
msg[(r, c, leg)][k, kbar] is the message from the neighbour across ``leg`` into
cell (r, c); legs are 1=u, 2=l, 3=d, 4=r (the tensor axes).
"""
from __future__ import annotations

import numpy as np

LEG_U, LEG_L, LEG_D, LEG_R = 1, 2, 3, 4
OPP = {LEG_U: LEG_D, LEG_D: LEG_U, LEG_L: LEG_R, LEG_R: LEG_L}
STEP = {LEG_U: (-1, 0), LEG_D: (1, 0), LEG_L: (0, -1), LEG_R: (0, 1)}


def apply_leg(t: np.ndarray, leg: int, M: np.ndarray) -> np.ndarray:
    """t'[.. j ..] = sum_o t[.. o ..] M[o, j] on axis ``leg``."""
    return np.moveaxis(np.tensordot(t, M, axes=([leg], [0])), -1, leg)


class GridTNS:
    """Processor-shaped TNS: one tensor per qubit, bonds on the coupling graph (Methods)."""

    def __init__(self, grid_rc, edges, bits):
        rc = np.asarray(grid_rc, dtype=np.int64).copy()
        H0, W0 = rc.max(axis=0) + 1
        self.transposed = bool(W0 > H0)
        if self.transposed:
            rc = rc[:, ::-1].copy()
        self.H, self.W = (int(x) for x in rc.max(axis=0) + 1)
        self.n = rc.shape[0]
        self.qubit_cell = [tuple(map(int, x)) for x in rc]
        self.cell_qubit = -np.ones((self.H, self.W), dtype=np.int64)
        for q, (r, c) in enumerate(self.qubit_cell):
            self.cell_qubit[r, c] = q
        self.edge = {}                     # (r, c, leg) -> True
        for a, b in np.asarray(edges):
            (ra, ca), (rb, cb) = self.qubit_cell[int(a)], self.qubit_cell[int(b)]
            leg = {(-1, 0): LEG_U, (1, 0): LEG_D, (0, -1): LEG_L, (0, 1): LEG_R}[(rb - ra, cb - ca)]
            self.edge[(ra, ca, leg)] = True
            self.edge[(rb, cb, OPP[leg])] = True
        self.T = [[None] * self.W for _ in range(self.H)]
        for r in range(self.H):
            for c in range(self.W):
                q = self.cell_qubit[r, c]
                if q < 0:
                    t = np.ones((1, 1, 1, 1, 1), dtype=np.complex128)
                else:
                    t = np.zeros((2, 1, 1, 1, 1), dtype=np.complex128)
                    t[int(bits[q]), 0, 0, 0, 0] = 1.0
                self.T[r][c] = t
        self.msg = {key: np.ones((1, 1), dtype=np.complex128) for key in self.edge}
        self.log_fidelity = 0.0
        self.eps = []

    # -- geometry helpers -------------------------------------------------
    def has_edge(self, r, c, leg) -> bool:
        return (r, c, leg) in self.edge

    def nbr(self, r, c, leg):
        dr, dc = STEP[leg]
        return r + dr, c + dc

    def legs(self, r, c):
        return [leg for leg in (LEG_U, LEG_L, LEG_D, LEG_R) if self.has_edge(r, c, leg)]

    def bond_dim(self, r, c, leg) -> int:
        return self.T[r][c].shape[leg]

    def copy(self) -> "GridTNS":
        out = GridTNS.__new__(GridTNS)
        out.__dict__.update(self.__dict__)
        out.T = [[t.copy() for t in row] for row in self.T]
        out.msg = {k: v.copy() for k, v in self.msg.items()}
        out.eps = list(self.eps)
        return out

    # -- belief propagation (Appendix, "Applying Gates"; Fig. 8c) ----------
    def message_out(self, r, c, leg) -> np.ndarray:
        """m_{v -> v'} = psi_v psi_v^* contracted with all incoming messages but v' -> v.

        Hermitised and normalised to unit Frobenius norm (the paper's normalisation
        condition "the norm of a message tensor is 1").
        """
        t = self.T[r][c]
        X = t
        for l2 in self.legs(r, c):
            if l2 != leg:
                X = apply_leg(X, l2, self.msg[(r, c, l2)])
        axes = [a for a in range(5) if a != leg]
        M = np.tensordot(X, t.conj(), axes=(axes, axes))
        M = 0.5 * (M + M.conj().T)
        return M / np.linalg.norm(M)

    def bp(self, max_iter: int = 500, tol: float = 1e-12):
        """Parallel-schedule BP to a fixed point; returns (iterations, residual, converged)."""
        resid = np.inf
        for it in range(1, max_iter + 1):
            new = {}
            for (r, c, leg) in self.edge:
                nr, nc = self.nbr(r, c, leg)
                new[(nr, nc, OPP[leg])] = self.message_out(r, c, leg)
            resid = max(np.linalg.norm(new[k] - self.msg[k]) for k in new) if new else 0.0
            self.msg = new
            if resid < tol:
                return it, resid, True
        return max_iter, resid, False

    # -- gate application (Methods; Appendix Fig. 8d) ---------------------
    def _gauge(self, r, c, skip_leg):
        """sqrt / inverse-sqrt of every incoming message except across ``skip_leg``."""
        X, Xi = {}, {}
        for leg in self.legs(r, c):
            if leg == skip_leg:
                continue
            m = self.msg[(r, c, leg)]
            lam, V = np.linalg.eigh(0.5 * (m + m.conj().T))
            lam = np.maximum(lam, 1e-12 * lam.max())
            X[leg] = (V * np.sqrt(lam)) @ V.conj().T
            Xi[leg] = (V / np.sqrt(lam)) @ V.conj().T
        return X, Xi

    def apply_1q(self, q: int, U: np.ndarray) -> None:
        """One-qubit gates are contracted exactly into the physical leg (no truncation)."""
        r, c = self.qubit_cell[q]
        self.T[r][c] = np.tensordot(U, self.T[r][c], axes=([1], [0]))

    def apply_2q(self, q0: int, q1: int, U: np.ndarray, chi: int, cutoff: float = 1e-14) -> float:
        """BP-gauged simple update of a two-qubit gate; returns the gate error eps (Eq. 1).

        Gauge the two sites with the square roots of their incoming messages,
        reduce each to an R factor by QR, apply the gate to R_A R_B, truncate the
        SVD to chi (keeping singular values above cutoff * sigma_1), split sqrt(S)
        symmetrically, and ungauge with the inverse square roots.  The state is not
        renormalised.  The bond messages become diag(S)/|S|, the exact BP update
        of the new bond given the other incoming messages.
        """
        (ra, ca), (rb, cb) = self.qubit_cell[q0], self.qubit_cell[q1]
        j = {(-1, 0): LEG_U, (1, 0): LEG_D, (0, -1): LEG_L, (0, 1): LEG_R}[(rb - ra, cb - ca)]
        jb = OPP[j]
        if not self.has_edge(ra, ca, j):
            raise ValueError("gate on a pair without a bond")
        Xa, Xai = self._gauge(ra, ca, j)
        Xb, Xbi = self._gauge(rb, cb, jb)
        ta, tb = self.T[ra][ca], self.T[rb][cb]
        for leg, M in Xa.items():
            ta = apply_leg(ta, leg, M)
        for leg, M in Xb.items():
            tb = apply_leg(tb, leg, M)

        def reduce(t, leg):
            others = [a for a in range(1, 5) if a != leg]
            perm = others + [0, leg]
            tp = np.transpose(t, perm)
            oshape = tp.shape[:3]
            A = tp.reshape(int(np.prod(oshape)), -1)
            Q, R = np.linalg.qr(A, mode="reduced")
            return Q, R.reshape(R.shape[0], t.shape[0], t.shape[leg]), oshape, perm

        Qa, Ra, osa, perma = reduce(ta, j)
        Qb, Rb, osb, permb = reduce(tb, jb)
        P = np.einsum("asb,ctb->asct", Ra, Rb)
        theta = np.einsum("xyst,asct->axcy", U.reshape(2, 2, 2, 2), P)
        r1, r2 = theta.shape[0], theta.shape[2]
        Um, sv, Vh = np.linalg.svd(theta.reshape(r1 * 2, r2 * 2), full_matrices=False)
        keep = int(np.count_nonzero(sv > cutoff * sv[0])) if sv[0] > 0 else 1
        k = max(1, min(chi, keep))
        eps = float(np.sum(sv[k:] ** 2) / np.sum(sv ** 2)) if sv[0] > 0 else 0.0
        sq = np.sqrt(sv[:k])
        Ua = (Um[:, :k] * sq).reshape(r1, 2, k)
        Vb = (Vh[:k, :].T * sq).reshape(r2, 2, k)
        na = np.tensordot(Qa, Ua, axes=([1], [0])).reshape(*osa, 2, k)
        nb = np.tensordot(Qb, Vb, axes=([1], [0])).reshape(*osb, 2, k)
        na = np.transpose(na, np.argsort(perma))
        nb = np.transpose(nb, np.argsort(permb))
        for leg, M in Xai.items():
            na = apply_leg(na, leg, M)
        for leg, M in Xbi.items():
            nb = apply_leg(nb, leg, M)
        self.T[ra][ca], self.T[rb][cb] = na, nb
        m = np.diag(sv[:k]).astype(np.complex128)
        m /= np.linalg.norm(m)
        self.msg[(ra, ca, j)] = m.copy()
        self.msg[(rb, cb, jb)] = m.copy()
        self.eps.append(eps)
        self.log_fidelity += float(np.log1p(-eps)) if eps < 1 else -np.inf
        return eps

    def apply_group(self, group, chi: int, cutoff: float = 1e-14) -> list:
        eps = []
        for (a, b, U) in group:
            if b < 0:
                self.apply_1q(a, U)
                eps.append(0.0)
            else:
                eps.append(self.apply_2q(a, b, U, chi, cutoff))
        return eps

    # -- brute-force contraction for small lattices (pins) -----------------
    def _labelled(self, bits=None):
        """Every cell tensor with index labels; physical legs projected when bits given."""
        items = []
        for r in range(self.H):
            for c in range(self.W):
                t = self.T[r][c]
                q = int(self.cell_qubit[r, c])
                if q < 0:
                    t, labels = t[0], []
                elif bits is not None:
                    t, labels = t[int(bits[q])], []
                else:
                    labels = [("p", q)]
                labels = labels + [("v", r - 1, c), ("h", r, c - 1), ("v", r, c), ("h", r, c)]
                items.append((t, labels))
        return items

    @staticmethod
    def _contract(a, b):
        ta, la = a
        tb, lb = b
        shared = [x for x in la if x in lb]
        out = np.tensordot(ta, tb, axes=([la.index(x) for x in shared], [lb.index(x) for x in shared]))
        lo = [x for x in la if x not in shared] + [x for x in lb if x not in shared]
        return out, lo

    def _contract_all(self, items):
        """Contract cell by cell in row-major order; leftover open labels have dim 1."""
        acc = (np.ones(()), [])
        for it in items:
            acc = self._contract(acc, it)
        t, labels = acc
        keep = [i for i, x in enumerate(labels) if x[0] == "p"]
        drop = [i for i, x in enumerate(labels) if x[0] != "p"]
        t = np.transpose(t, keep + drop).reshape([t.shape[i] for i in keep])
        return t, [labels[i] for i in keep]

    def amplitude_bruteforce(self, bits) -> complex:
        """<x|psi> by exact contraction of the projected network (small lattices)."""
        t, _ = self._contract_all(self._labelled(bits))
        return complex(np.asarray(t).reshape(()))

    def statevector_bruteforce(self) -> np.ndarray:
        """Full 2^n statevector of the TNS by exact contraction (small lattices only)."""
        t, labels = self._contract_all(self._labelled(None))
        order = [labels.index(("p", q)) for q in range(self.n)]
        return np.transpose(t, order)
