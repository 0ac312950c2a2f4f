"""CPU oracle for the generalized boundary-MPS contraction and the TNS sampler.

TEST INFRASTRUCTURE ONLY.  complex128 numpy/LAPACK, one sample at a time,
following the paper's Appendix "Sampling from a Tensor Network State" (Fig. 7):

* partitions are the grid rows b = 0..H-1 (the grid is oriented so that rows
  are the long direction and the boundary MPS runs along the short side);
* the norm network is contracted once from the bottom, giving the stored
  environments E_{b+1} ("M_{b+1 -> b}" in the paper), each an MPS of rank R;
* each sample sweeps the rows top to bottom: the row is absorbed into the
  sample's boundary MPS m_b and compressed to rank R ("fit"), the row's qubits
  are drawn one by one from their one-site conditional marginals, and the
  projected row becomes m_{b+1};
* q(x) is the product of the conditionals.

The MPS-MPO compression is a zip-up sweep whose per-site truncated SVD (the
"QR and truncated SVD" of the method) has two forms here.  ``exact=True`` is the
plain definition: LAPACK's SVD of the site matrix, keep the top R singular
vectors.  The default follows the library's computation of the same truncation,
a randomized range finder (Halko, Martinsson, Tropp 2011, Alg. 4.4: a shared
Philox test matrix with R + OVERSAMPLE columns, POWER_ITERS subspace iterations
with an orthonormalisation after every application, then an SVD of the
projected matrix), whose kept subspace converges to the exact one like
(sigma_{k+1} / sigma_R)^(2q+1); when R + oversampling covers the full column
dimension the test matrix is the identity and the step is exact.  Tests compare
the library with both: the randomized form pins the implementation to rounding,
the exact form bounds how far the method's result is from the definition.  ``fit_sweeps > 0`` follows the zip with the
paper's one-site variational fitting (``fit_compress``; Methods and Fig. 7c),
which only raises the overlap with the exact MPS-MPO product.

``direct_marginals`` gives sample-free one-site and same-row two-site marginals
from the norm network (top and bottom environments around each row);
``projected_marginal`` gives <prod n_q> for any set of qubits as the norm of the
projected state over the norm of the state.

Index conventions (logical order j = 0..W-1 along the sweep direction):
  MPS site  m[a, Xc, Xp, a']   (Xc contracted with the MPO, Xp passed through)
  MPO site  w[l, Xc, Y, r]
  output    out[k, Y, Xp, k']
Rows alternate direction (even rows left-to-right, odd rows right-to-left) so
every zip starts at the orthogonality centre the previous one left behind.
"""
from __future__ import annotations

import numpy as np

from . import philox

# Range-finder settings of the truncated SVD (the library's defaults): k = R + OVERSAMPLE
# columns and POWER_ITERS subspace iterations in the sampler and amplitude zips,
# ENV_POWER_ITERS in the norm-environment zips.  Read at call time.
OVERSAMPLE = 48
POWER_ITERS = 3
ENV_POWER_ITERS = 6
# Shift of the Cholesky orthonormalisation of a range-finder basis, relative to
# the largest diagonal entry of its Gram matrix: it only regularises
# rank-deficient bases (orth(Y) is an orthonormal basis of range(Y)).
ORTH_SHIFT = 1e-14


# ---------------------------------------------------------------- small helpers
def fix_phase(U: np.ndarray) -> np.ndarray:
    """Deterministic column phases: make sum_i u_i / sqrt(i+1) real positive.

    Falls back to the largest-magnitude entry when that sum vanishes.  Applied to
    the columns of the compressed site tensor K (rows = (k, y, xp)), so the
    convention does not depend on any internal basis.  Both the oracle and the
    library use it so that the boundary MPS handed from row to row is the same
    tensor, not just the same state.
    """
    U = U.copy()
    w = 1.0 / np.sqrt(np.arange(U.shape[0]) + 1.0)
    for j in range(U.shape[1]):
        c = np.dot(w, U[:, j])
        if abs(c) > 1e-8:
            U[:, j] *= np.conj(c) / abs(c)
        else:
            i = int(np.argmax(np.abs(U[:, j])))
            if abs(U[i, j]) > 0:
                U[:, j] *= np.conj(U[i, j]) / abs(U[i, j])
    return U


def eigh_desc(A: np.ndarray):
    lam, V = np.linalg.eigh(0.5 * (A + A.conj().T))
    return lam[::-1], V[:, ::-1]


def orth(Y: np.ndarray, shift: float) -> np.ndarray:
    """Orthonormal basis Q = Y L^{-H} of range(Y), with L L^H = Y^H Y + shift * max_i G_ii * I.

    The shift keeps the Cholesky factorisation defined for rank-deficient Y and
    damps directions whose Gram eigenvalue is below shift * max_i G_ii.
    """
    G = Y.conj().T @ Y
    m = float(np.max(np.real(np.diag(G)))) if G.size else 0.0
    if m <= 0:
        return np.zeros_like(Y)
    L = np.linalg.cholesky(G + shift * m * np.eye(G.shape[0]))
    return np.linalg.solve(L, Y.conj().T).conj().T          # Y L^{-H}


def truncate(T: np.ndarray, R: int, omega, gram_cut: float = ORTH_SHIFT, exact: bool = False,
             power_iters: int | None = None, oversample: int | None = None):
    """Rank-R factorisation T ~ K C with K having orthonormal columns (the "QR + truncated SVD").

    Randomized range finder with subspace iteration, orthonormalising after every
    application (Halko, Martinsson, Tropp 2011, Alg. 4.4): Y = T Omega, then
    ``power_iters`` times Y = T orth(T^H orth(Y)); Omega = I (and no iteration)
    when k = R + p >= N, which makes the step an exact truncated SVD.  Then
    Q = orth(Y), B = Q^H T, B B^H = U_B S^2 U_B^H, K = Q U_B[:, :R], C = K^H T.
    Column phases of K follow ``fix_phase``.  ``gram_cut`` is the orthonormalisation
    shift.  ``power_iters`` / ``oversample`` default to POWER_ITERS / OVERSAMPLE.
    Returns K (M x Rk), C (Rk x N), Rk = min(R, M, N).
    """
    power_iters = POWER_ITERS if power_iters is None else power_iters
    oversample = OVERSAMPLE if oversample is None else oversample
    M, N = T.shape
    Rk = min(R, M, N)
    K = np.zeros((M, Rk), dtype=np.complex128)
    if exact:
        U, s, Vh = np.linalg.svd(T, full_matrices=False)
        n = min(Rk, s.size)
        K[:, :n] = fix_phase(U[:, :n])
        return K, K.conj().T @ T
    kk = min(R + oversample, M, N)
    if kk == N:
        Y = T
    else:
        Y = T @ omega(N, kk)
        for _ in range(power_iters):
            Z = orth(T.conj().T @ orth(Y, gram_cut), gram_cut)
            Y = T @ Z
    Q = orth(Y, gram_cut)
    B = Q.conj().T @ T
    mu, UB = eigh_desc(B @ B.conj().T)
    n = min(Rk, UB.shape[1])
    K[:, :n] = fix_phase(Q @ UB[:, :n])
    return K, K.conj().T @ T


def zip_compress(mps, mpo, R, seed, stage, row, exact=False, gram_cut=ORTH_SHIFT, power_iters=None):
    """Zip-up MPS-MPO compression to rank R along the given (logical) site order.

    T_j[(k, y, xp), (a', r)] = sum C_{j-1}[k, a, l] m_j[a, xc, xp, a'] w_j[l, xc, y, r];
    T_j = K_j C_j by ``truncate``; the last site keeps T / |T|.  Returns the output
    MPS (sites out[k, y, xp, k']) and log|T_last| (the output's norm, since all
    other sites are isometries).
    """
    W = len(mps)
    C = np.ones((1, 1, 1), dtype=np.complex128)
    out = []
    log_scale = 0.0
    for j in range(W):
        m, w = mps[j], mpo[j]
        X = np.tensordot(C, m, axes=([1], [0]))            # k, l, xc, xp, a'
        T = np.tensordot(X, w, axes=([1, 2], [0, 1]))      # k, xp, a', y, r
        T = np.transpose(T, (0, 3, 1, 2, 4))               # k, y, xp, a', r
        k, y, xp, ap, r = T.shape
        Tm = T.reshape(k * y * xp, ap * r)
        if j == W - 1:
            nrm = np.linalg.norm(Tm)
            log_scale = float(np.log(nrm)) if nrm > 0 else -np.inf
            out.append((Tm / nrm if nrm > 0 else Tm).reshape(k, y, xp, 1))
            break
        omega = lambda n, kk, _j=j: philox.test_matrix(seed, stage, row, _j, n, kk)
        K, Cn = truncate(Tm, R, omega, gram_cut=gram_cut, exact=exact, power_iters=power_iters)
        out.append(K.reshape(k, y, xp, K.shape[1]))
        C = Cn.reshape(Cn.shape[0], ap, r)
    return out, log_scale


def compress(mps, mpo, R, seed, stage, row, exact=False, gram_cut=ORTH_SHIFT, fit_sweeps=0, power_iters=None):
    """The zip-up compression, followed by ``fit_sweeps`` sweeps of one-site
    variational fitting when fit_sweeps > 0 (the paper's compressor)."""
    if fit_sweeps > 0:
        return fit_compress(mps, mpo, R, seed, stage, row, sweeps=fit_sweeps, exact=exact, gram_cut=gram_cut,
                            power_iters=power_iters)
    return zip_compress(mps, mpo, R, seed, stage, row, exact=exact, gram_cut=gram_cut, power_iters=power_iters)


def mirror_mps(mps):
    """Reverse the site order of an MPS (swap each site's bond axes)."""
    return [np.swapaxes(x, 0, x.ndim - 1) for x in reversed(mps)]


def row_tensors(tns, b, reverse):
    """Row b's site tensors psi[s,u,l,d,r] in logical order (l<->r swapped if reversed)."""
    row = [tns.T[b][c] for c in range(tns.W)]
    if reverse:
        row = [np.transpose(t, (0, 1, 4, 3, 2)) for t in reversed(row)]
    return row


def row_cells(tns, b, reverse):
    cs = list(range(tns.W))
    return list(reversed(cs)) if reverse else cs


# ---------------------------------------------------------- norm environments
ENV_SEED = 0


def norm_envs(tns, R, seed=ENV_SEED, gram_cut=ORTH_SHIFT, exact=False, fit_sweeps=0):
    """Bottom environments E[b] of <psi|psi> for b = 1..H (E[H] trivial).

    E[b] is stored in column order with sites E[b][c][e, d, dbar, e'] on the
    vertical bonds between rows b-1 and b.  Built once, independent of the
    number of samples: absorb the ket row (zip left-to-right, compress to R),
    then the bra row (zip right-to-left, compress to R).  The range-finder test
    matrices of the environments are keyed with ENV_SEED, independent of the
    sampling seed.  Returns (E, log_norm) where log_norm is log <psi|psi> from the
    last (b = 0) step.
    """
    H, W = tns.H, tns.W
    E = {H: [np.ones((1, 1, 1, 1), dtype=np.complex128) for _ in range(W)]}
    log_norm = 0.0
    for b in range(H - 1, -1, -1):
        row = row_tensors(tns, b, reverse=False)
        m = [x for x in E[b + 1]]                                   # e, d, dbar, e'
        mpo = []
        for t in row:                                                # ket: Xc = d, Y = (s, u)
            s, u, l, d, r = t.shape
            mpo.append(np.transpose(t, (2, 3, 0, 1, 4)).reshape(l, d, s * u, r))
        Z, ls1 = compress(m, mpo, R, seed, philox.STAGE_ENV_KET, b, exact=exact, gram_cut=gram_cut,
                          fit_sweeps=fit_sweeps, power_iters=ENV_POWER_ITERS)
        # Z_j: k, (s,u), dbar, k' -> bra input: Xc = (s, dbar), Xp = u
        mz, mpo2 = [], []
        for zj, t in zip(Z, row):
            s, u, l, d, r = t.shape
            k, _, db, kp = zj.shape
            z5 = zj.reshape(k, s, u, db, kp)
            mz.append(np.transpose(z5, (0, 1, 3, 2, 4)).reshape(k, s * db, u, kp))
            mpo2.append(np.transpose(t.conj(), (2, 0, 3, 1, 4)).reshape(l, s * d, u, r))
        mz, mpo2 = mirror_mps(mz), list(reversed([np.transpose(w, (3, 1, 2, 0)) for w in mpo2]))
        Eb, ls2 = compress(mz, mpo2, R, seed, philox.STAGE_ENV_BRA, b, exact=exact, gram_cut=gram_cut,
                           fit_sweeps=fit_sweeps, power_iters=ENV_POWER_ITERS)
        Eb = mirror_mps(Eb)                                          # back to column order
        E[b] = [np.transpose(x, (0, 2, 1, 3)) for x in Eb]           # e, u(ket), ubar, e'
        log_norm += ls1 + ls2
    total = np.prod([x.reshape(()) for x in E[0]])
    log_norm += float(np.log(abs(total))) if abs(total) > 0 else -np.inf
    return E, log_norm


# ------------------------------------------------------------------- sampler
def sample_row(m, row, Eb, R, seed, b, uniforms=None, forced=None, gram_cut=ORTH_SHIFT, exact=False, fit_sweeps=0):
    """One partition: absorb + compress, right environments, draw left to right.

    m: MPS m[a, u, 1, a'] in this row's logical order; row: psi sites in logical
    order; Eb: env sites [e, d, dbar, e'] in logical order.  Either ``uniforms``
    (draw: x = 1 iff u >= q(0|prefix)) or ``forced`` bits (replay) is given.
    Returns (bits, q0 per site, sum log q(x_j|prefix), m_next in logical order).
    """
    W = len(row)
    mpo = []
    for t in row:
        s, u, l, d, r = t.shape
        mpo.append(np.transpose(t, (2, 1, 0, 3, 4)).reshape(l, u, s * d, r))
    Kp, _ = compress(m, mpo, R, seed, philox.STAGE_SAMPLE, b, exact=exact, gram_cut=gram_cut, fit_sweeps=fit_sweeps)
    K = [Kp[j].reshape(Kp[j].shape[0], row[j].shape[0], row[j].shape[3], Kp[j].shape[3]) for j in range(W)]
    F = [None] * (W + 1)
    F[W] = np.ones((1, 1, 1), dtype=np.complex128)
    for j in range(W - 1, 0, -1):
        # F_j[a, e, A] = sum K[a,s,d,b] E[e,d,f,g] conj K[A,s,f,B] F_{j+1}[b,g,B]
        X = np.tensordot(K[j], F[j + 1], axes=([3], [0]))             # a, s, d, g, B
        X = np.tensordot(X, Eb[j], axes=([2, 3], [1, 3]))             # a, s, B, e, f
        Fj = np.tensordot(X, K[j].conj(), axes=([1, 2, 4], [1, 3, 2]))  # a, e, A
        F[j] = Fj / np.linalg.norm(Fj)
    L = np.ones((1, 1, 1), dtype=np.complex128)
    bits = np.zeros(W, dtype=np.int64)
    q0s = np.ones(W)
    logq = 0.0
    m_next = []
    for j in range(W):
        X = np.tensordot(L, K[j], axes=([0], [0]))                    # e, A, s, d, b
        X = np.tensordot(X, Eb[j], axes=([0, 3], [0, 1]))             # A, s, b, f, g
        G = np.einsum("Asbfg,AsfB->sbgB", X, K[j].conj())             # s, b, g, B
        rho = np.real(np.tensordot(G, F[j + 1], axes=([1, 2, 3], [0, 1, 2])))
        rho = np.maximum(rho, 0.0)
        tot = float(rho.sum())
        if row[j].shape[0] == 1:
            x, q0 = 0, 1.0
        else:
            q0 = float(rho[0] / tot) if tot > 0 else 0.5
            x = int(forced[j]) if forced is not None else int(uniforms[j] >= q0)
            qx = q0 if x == 0 else 1.0 - q0
            logq += float(np.log(qx)) if qx > 0 else -np.inf
        bits[j] = x
        q0s[j] = q0
        L = G[x] / (tot if tot > 0 else 1.0)
        m_next.append(K[j][:, x, :, :][:, :, None, :])                 # a, d, 1, a'
    return bits, q0s, logq, m_next


def sample(tns, R, n_samples, seed, sample_offset=0, forced=None, env=None, gram_cut=ORTH_SHIFT, exact=False,
           fit_sweeps=0):
    """Draw samples (or replay ``forced`` bitstrings); returns bits [n, n_qubits], log q, q0.

    q0[n, qubit] is the conditional probability of 0 that the draw of that qubit used.
    """
    H, W = tns.H, tns.W
    E = env if env is not None else norm_envs(tns, R, ENV_SEED, gram_cut=gram_cut, exact=exact,
                                              fit_sweeps=fit_sweeps)[0]
    n = n_samples if forced is None else forced.shape[0]
    bits_out = np.zeros((n, tns.n), dtype=np.uint8)
    q0_out = np.ones((n, tns.n))
    logq = np.zeros(n)
    for i in range(n):
        sid = sample_offset + i
        m = [np.ones((1, 1, 1, 1), dtype=np.complex128) for _ in range(W)]
        for b in range(H):
            rev = (b % 2 == 1)
            cells = row_cells(tns, b, rev)
            row = row_tensors(tns, b, rev)
            Eb = E[b + 1] if not rev else mirror_mps(E[b + 1])
            qubits = [int(tns.cell_qubit[b, c]) for c in cells]
            uni = fb = None
            if forced is None:
                uni = philox.draw_uniforms(seed, sid, np.array([max(q, 0) for q in qubits]))
            else:
                fb = [int(forced[i, q]) if q >= 0 else 0 for q in qubits]
            xb, q0b, lq, m_next = sample_row(m, row, Eb, R, seed, b, uniforms=uni, forced=fb,
                                             gram_cut=gram_cut, exact=exact, fit_sweeps=fit_sweeps)
            logq[i] += lq
            for j, q in enumerate(qubits):
                if q >= 0:
                    bits_out[i, q] = xb[j]
                    q0_out[i, q] = q0b[j]
            m = mirror_mps(m_next)
    return bits_out, logq, q0_out


def amplitude(tns, R, bits, seed, gram_cut=ORTH_SHIFT, exact=False, fit_sweeps=0):
    """<x|psi> by single-layer boundary MPS over projected rows; returns (log|a|, phase)."""
    H, W = tns.H, tns.W
    m = [np.ones((1, 1, 1, 1), dtype=np.complex128) for _ in range(W)]
    log_abs = 0.0
    out = None
    for b in range(H):
        rev = (b % 2 == 1)
        cells = row_cells(tns, b, rev)
        row = row_tensors(tns, b, rev)
        mpo = []
        for c, t in zip(cells, row):
            q = int(tns.cell_qubit[b, c])
            tp = t[int(bits[q]) if q >= 0 else 0]                       # u, l, d, r
            mpo.append(np.transpose(tp, (1, 0, 2, 3)))                   # l, u, d, r
        out, ls = compress(m, mpo, R, seed, philox.STAGE_AMPLITUDE, b, exact=exact, gram_cut=gram_cut,
                           fit_sweeps=fit_sweeps)
        if not np.isfinite(ls):
            return -np.inf, 0.0
        log_abs += ls
        m = mirror_mps(out)
    z = np.prod([x.reshape(()) for x in out])
    if abs(z) == 0:
        return -np.inf, 0.0
    return log_abs + float(np.log(abs(z))), float(np.angle(z))


# ------------------------------------------------------- direct marginals
class _Flipped:
    """The same TNS read upside down: row b -> H-1-b, up and down legs exchanged."""

    def __init__(self, tns):
        self.H, self.W = tns.H, tns.W
        self.T = [[np.transpose(tns.T[tns.H - 1 - b][c], (0, 3, 2, 1, 4)) for c in range(tns.W)]
                  for b in range(tns.H)]


def _grow_left(L, U, t, o, D):
    """L'[e', r, rb, f'] = sum L[e, l, lb, f] U[e, u, ub, e'] t[s, u, l, d, r] o[s, s']
    conj t[s', ub, lb, db, rb] D[f, d, db, f']: one site of a row of the norm network
    between its top (U) and bottom (D) environments, absorbed from the left."""
    X = np.tensordot(L, U, axes=([0], [0]))                    # l, lb, f, u, ub, e'
    X = np.tensordot(X, t, axes=([0, 3], [2, 1]))              # lb, f, ub, e', s, d, r
    tb = np.tensordot(o, t.conj(), axes=([1], [0]))            # s, ub, lb, db, rb
    X = np.tensordot(X, tb, axes=([0, 2, 4], [2, 1, 0]))       # f, e', d, r, db, rb
    return np.tensordot(X, D, axes=([0, 2, 4], [0, 1, 2]))     # e', r, rb, f'


def _grow_right(Rt, U, t, o, D):
    """The same site absorbed from the right: R'[e, l, lb, f] from R[e', r, rb, f']."""
    X = np.tensordot(U, Rt, axes=([3], [0]))                   # e, u, ub, r, rb, f'
    X = np.tensordot(X, t, axes=([1, 3], [1, 4]))              # e, ub, rb, f', s, l, d
    tb = np.tensordot(o, t.conj(), axes=([1], [0]))            # s, ub, lb, db, rb
    X = np.tensordot(X, tb, axes=([1, 2, 4], [1, 4, 0]))       # e, f', l, d, lb, db
    return np.tensordot(X, D, axes=([1, 3, 5], [3, 1, 2]))     # e, l, lb, f


def direct_marginals(tns, R, gram_cut=ORTH_SHIFT, exact=False, pairs=True):
    """Sample-free marginals <n_q> = <psi|P1_q|psi>/<psi|psi> for every qubit and
    <n_q n_q'> for every pair in the same grid row (NaN for pairs in different
    rows, and for all pairs when ``pairs`` is False), by boundary-MPS contraction of
    the norm network <psi|psi>.

    Row b is contracted exactly between its top environment (rows 0..b-1, the
    bottom environments of the upside-down TNS) and its bottom environment E[b+1]
    (rows b+1..H-1), both compressed to rank R as in norm_envs, one site at a time
    from the left and from the right, with the projector P1 = |1><1| inserted on
    the physical legs of the marginal's qubits.  Exact when R covers the
    environments' ranks.  Returns (one [n], two [n, n]).
    """
    H, W = tns.H, tns.W
    E, _ = norm_envs(tns, R, gram_cut=gram_cut, exact=exact)
    Ef, _ = norm_envs(_Flipped(tns), R, gram_cut=gram_cut, exact=exact)
    n = int((tns.cell_qubit >= 0).sum())
    one = np.full(n, np.nan)
    two = np.full((n, n), np.nan)
    P1 = np.diag([0.0, 1.0]).astype(np.complex128)
    for b in range(H):
        U = Ef[H - b]                 # sites [e, u, ubar, e'] on row b's up legs (flipped: down legs)
        D = E[b + 1]                  # sites [f, d, dbar, f'] on row b's down legs
        T = tns.T[b]
        ident = [np.eye(T[c].shape[0], dtype=np.complex128) for c in range(W)]
        left = [np.ones((1, 1, 1, 1), dtype=np.complex128)]
        for c in range(W):
            left.append(_grow_left(left[c], U[c], T[c], ident[c], D[c]))
        right = [None] * (W + 1)
        right[W] = np.ones((1, 1, 1, 1), dtype=np.complex128)
        for c in range(W - 1, -1, -1):
            right[c] = _grow_right(right[c + 1], U[c], T[c], ident[c], D[c])
        # A truncated environment makes the contracted values slightly complex; the ratio
        # of real parts is the one the sampler's conditionals use (q = Re rho_0 /
        # Re(rho_0 + rho_1)), so marginals and conditionals are the same functional.
        norm = float(np.real(left[W].reshape(()).item()))
        qs = [(c, int(tns.cell_qubit[b, c])) for c in range(W) if tns.cell_qubit[b, c] >= 0]
        for i, (ci, qi) in enumerate(qs):
            v = _grow_left(left[ci], U[ci], T[ci], P1, D[ci])
            one[qi] = float(np.real(np.sum(v * right[ci + 1]))) / norm
            two[qi, qi] = one[qi]
            if not pairs:
                continue
            for c in range(ci + 1, W):
                q = int(tns.cell_qubit[b, c])
                if q >= 0:
                    val = float(np.real(np.sum(_grow_left(v, U[c], T[c], P1, D[c]) * right[c + 1]))) / norm
                    two[qi, q] = two[q, qi] = val
                v = _grow_left(v, U[c], T[c], ident[c], D[c])
    return one, two


# ------------------------------------------------- one-site variational fitting
def _product_site(m, w):
    """P[a, l, y, xp, a', r] = sum_xc m[a, xc, xp, a'] w[l, xc, y, r] (exact MPS-MPO site)."""
    return np.einsum("acpA,lcyr->alypAr", m, w)


def fit_compress(mps, mpo, R, seed, stage, row, sweeps=2, exact=False, gram_cut=ORTH_SHIFT, history=None,
                 power_iters=None):
    """MPS-MPO compression to rank R by one-site variational fitting (Methods and
    Appendix "Sampling...": maximise the overlap of the output MPS with the exact
    MPS-MPO product by sweeping through the output's sites and replacing each with
    the derivative of the overlap with respect to it; Verstraete, Murg, Cirac 2008).

    The initial guess is the zip-up result (``zip_compress``), so the bond dimensions
    are those of the zip; each sweep goes right to left then left to right, keeping
    the output in mixed canonical form around the updated site (QR / LQ of the
    update; the triangular factor is dropped because the neighbour is recomputed
    from the environments).  Returns the output in the zip's convention (sites
    out[k, y, xp, k'], left-isometric except the last, which carries unit norm) and
    log of the output's norm.  ``history`` (a list) receives the overlap
    |<Y|P>| / |Y| after every local update.
    """
    W = len(mps)
    Y, _ = zip_compress(mps, mpo, R, seed, stage, row, exact=exact, gram_cut=gram_cut, power_iters=power_iters)
    P = [_product_site(m, w) for m, w in zip(mps, mpo)]
    one = np.ones((1, 1, 1), dtype=np.complex128)

    def grow_left(Lj, j):          # L_{j+1}[k', a', r]
        return np.einsum("kal,kypK,alypAr->KAr", Lj, Y[j].conj(), P[j], optimize=True)

    def grow_right(Rj1, j):        # R_j[k, a, l]
        return np.einsum("kypK,alypAr,KAr->kal", Y[j].conj(), P[j], Rj1, optimize=True)

    def update(Lj, Rj1, j):        # derivative of <Y|P> w.r.t. conj(Y_j)
        return np.einsum("kal,alypAr,KAr->kypK", Lj, P[j], Rj1, optimize=True)

    log_norm = 0.0
    for _ in range(sweeps):
        # left environments for the current (left-canonical) guess
        L = [one]
        for j in range(W - 1):
            L.append(grow_left(L[j], j))
        Rn = [None] * (W + 1)
        Rn[W] = one
        for j in range(W - 1, 0, -1):            # right to left
            Yj = update(L[j], Rn[j + 1], j)
            if history is not None:
                history.append(float(np.linalg.norm(Yj)))
            k, y, xp, kp = Yj.shape
            q, _r = np.linalg.qr(Yj.reshape(k, y * xp * kp).T)       # Yj = r^T q^T: rows of q^T orthonormal
            Y[j] = q.T.reshape(q.shape[1], y, xp, kp)
            Rn[j] = grow_right(Rn[j + 1], j)
        L = [one]
        for j in range(W):                       # left to right
            Yj = update(L[j], Rn[j + 1], j)
            if history is not None:
                history.append(float(np.linalg.norm(Yj)))
            if j == W - 1:
                nrm = float(np.linalg.norm(Yj))
                log_norm = float(np.log(nrm)) if nrm > 0 else -np.inf
                Y[j] = Yj / nrm if nrm > 0 else Yj
                break
            k, y, xp, kp = Yj.shape
            q, _r = np.linalg.qr(Yj.reshape(k * y * xp, kp))
            Y[j] = q.reshape(k, y, xp, q.shape[1])
            L.append(grow_left(L[j], j))
    return Y, log_norm


# --------------------------------------------------------- sample certification
def certify(tns, bits, logq, R_cert, seed=0, bins=20):
    """p(x) of sampled bitstrings by an independent amplitude contraction at rank
    R_cert (e.g. twice the sampling rank; Methods "p(x) = |<x|psi>|^2" and the
    verification step of the Appendix), normalised by <psi|psi> at the same rank.

    Returns dict(log_p, ratio = p/q, mean_ratio (an estimator of 1), kld =
    E_q[log q - log p], hist = (counts, edges) of log10(p/q)).
    """
    _, log_norm = norm_envs(tns, R_cert)
    log_p = np.array([2.0 * amplitude(tns, R_cert, x, seed)[0] - log_norm for x in np.asarray(bits)])
    logq = np.asarray(logq, dtype=np.float64)
    ratio = np.exp(log_p - logq)
    finite = np.isfinite(log_p)
    lr = np.log10(ratio[finite & (ratio > 0)])
    hist = np.histogram(lr, bins=bins) if lr.size else (np.zeros(bins, dtype=np.int64), np.linspace(0, 1, bins + 1))
    return dict(log_p=log_p, ratio=ratio, mean_ratio=float(ratio.mean()), kld=float(np.mean(logq - log_p)),
                hist=hist)


def projected_marginal(tns, R, qubits, gram_cut=ORTH_SHIFT, exact=False):
    """<prod_q n_q> = |prod_q P1_q psi|^2 / |psi|^2 for the given qubits (any rows): the
    norm network of the state with those qubits' physical index fixed to 1, over
    the norm network of the state (both at boundary rank R)."""
    class _Proj:
        pass
    proj = _Proj()
    proj.H, proj.W = tns.H, tns.W
    proj.T = [[t for t in row] for row in tns.T]
    for q in qubits:
        r, c = (int(x) for x in np.argwhere(tns.cell_qubit == q)[0])
        t = tns.T[r][c].copy()
        t[0] = 0.0
        proj.T[r][c] = t
    _, ln_p = norm_envs(proj, R, gram_cut=gram_cut, exact=exact)
    _, ln = norm_envs(tns, R, gram_cut=gram_cut, exact=exact)
    return float(np.exp(ln_p - ln)) if np.isfinite(ln_p) else 0.0
