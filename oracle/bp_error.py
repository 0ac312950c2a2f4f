"""BP loop error of the norm network (Results, Eqs. avBPError and loopBPerror;
Appendix "Computing the BP Error"), plain numpy.

TEST INFRASTRUCTURE ONLY.  For a loop v_1 -> v_2 -> ... -> v_L -> v_1 of grid cells
joined by bonds, every site's double-layer tensor psi_v psi_v^* gets the incoming
BP messages on its legs off the loop; the bond (v_L, v_1) is cut open, and the
product of the sites' (in, in-bar) x (out, out-bar) matrices is the loop's transfer
matrix.  With its eigenvalues lambda_1, lambda_2, ... sorted by modulus,
eps_l = 1 - |lambda_1| / sum_i |lambda_i|, and eps is the mean over the loops.
Primitive loops of a square grid are its plaquettes.
"""
from __future__ import annotations

import numpy as np

from .tns import LEG_D, LEG_L, LEG_R, LEG_U, apply_leg


def _leg_towards(a, b):
    dr, dc = b[0] - a[0], b[1] - a[1]
    return {(-1, 0): LEG_U, (1, 0): LEG_D, (0, -1): LEG_L, (0, 1): LEG_R}[(dr, dc)]


def site_matrix(tns, cell, leg_in, leg_out):
    """D[(i, ibar), (o, obar)] = sum psi[.. i .. o ..] (messages on the other legs) conj psi[.. ibar .. obar ..]."""
    r, c = cell
    t = tns.T[r][c]
    X = t
    for leg in tns.legs(r, c):
        if leg not in (leg_in, leg_out):
            X = apply_leg(X, leg, tns.msg[(r, c, leg)])
    others = [a for a in range(5) if a not in (leg_in, leg_out)]
    D = np.tensordot(X, t.conj(), axes=(others, others))           # i, o, ibar, obar (sorted leg order)
    i_first = leg_in < leg_out
    if not i_first:                                                 # axes came out as o, i, obar, ibar
        D = np.transpose(D, (1, 0, 3, 2))
    di, do = t.shape[leg_in], t.shape[leg_out]
    return np.transpose(D, (0, 2, 1, 3)).reshape(di * di, do * do)


def loop_transfer(tns, cells):
    """Transfer matrix of the loop cells[0] -> cells[1] -> ... -> cells[-1] -> cells[0],
    cut open on the bond (cells[-1], cells[0])."""
    L = len(cells)
    T = None
    for k in range(L):
        prev, cur, nxt = cells[k - 1], cells[k], cells[(k + 1) % L]
        D = site_matrix(tns, cur, _leg_towards(cur, prev), _leg_towards(cur, nxt))
        T = D if T is None else T @ D
    return T


def loop_error(tns, cells) -> float:
    lam = np.linalg.eigvals(loop_transfer(tns, cells))
    a = np.sort(np.abs(lam))[::-1]
    return float(1.0 - a[0] / a.sum()) if a.sum() > 0 else 0.0


def plaquettes(tns):
    """Square plaquettes whose four bonds all exist, as cell cycles."""
    out = []
    for r in range(tns.H - 1):
        for c in range(tns.W - 1):
            cyc = [(r, c), (r, c + 1), (r + 1, c + 1), (r + 1, c)]
            if all(tns.has_edge(*a, _leg_towards(a, b)) for a, b in zip(cyc, cyc[1:] + cyc[:1])):
                out.append(cyc)
    return out


def bp_error(tns, loops=None):
    """(mean eps, per-loop eps) over the given loops (default: the plaquettes)."""
    loops = plaquettes(tns) if loops is None else loops
    errs = [loop_error(tns, cyc) for cyc in loops]
    return (float(np.mean(errs)) if errs else 0.0), errs
