"""Device primitives through the C ABI against the oracle / numpy (GPU)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    import paper_2507_11424_gb300 as pkg
    from paper_2507_11424_gb300 import build
    build.build()
    return torch, pkg.load()


def _ptr(t):
    import ctypes
    return ctypes.c_void_p(t.data_ptr())


def test_device_philox_bit_exact(env):
    torch, lib = env
    from oracle import philox
    rng = np.random.default_rng(0)
    ck = rng.integers(0, 2**32, size=(4096, 6), dtype=np.uint64)
    ck[0] = 0
    ck[1] = 0xFFFFFFFF
    d_in = torch.tensor(ck.astype(np.uint32).view(np.int32), device="cuda")
    d_out = torch.zeros((4096, 4), dtype=torch.int32, device="cuda")
    assert lib.tns_test_philox(4096, _ptr(d_in), _ptr(d_out), None) == 0
    got = d_out.cpu().numpy().view(np.uint32)
    ref = np.stack(philox.philox4x32_10(*[ck[:, i] for i in range(6)]), axis=1)
    assert (got == ref.astype(np.uint32)).all()


@pytest.mark.parametrize("n,batch", [(1, 3), (7, 5), (16, 4), (72, 3), (81, 2), (136, 2), (264, 2)])
def test_device_eigh(env, n, batch):
    torch, lib = env
    rng = np.random.default_rng(n)
    A = rng.normal(size=(batch, n, n)) + 1j * rng.normal(size=(batch, n, n))
    A = A @ np.conj(np.transpose(A, (0, 2, 1)))            # PSD, like Gram matrices
    A[0] = A[0] * 1e-3 + np.diag(np.arange(n)) * 0.0        # scaled copy
    dA = torch.tensor(A.view(np.float64), device="cuda")
    lam = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    V = torch.zeros((batch, n, n, 2), dtype=torch.float64, device="cuda")
    assert lib.tns_test_eigh(batch, n, _ptr(dA), _ptr(lam), _ptr(V), None) == 0
    import ctypes
    sw = (ctypes.c_int32 * batch)()
    assert lib.tns_test_eigh_sweeps(batch, ctypes.cast(sw, ctypes.c_void_p)) == 0
    assert all(0 < x <= 25 for x in sw), list(sw)                     # converged, in few sweeps
    lam = lam.cpu().numpy()
    V = V.cpu().numpy().view(np.complex128).reshape(batch, n, n)
    for b in range(batch):
        ref = np.linalg.eigvalsh(A[b])[::-1]
        scale = np.abs(ref).max()
        assert np.abs(lam[b] - ref).max() < 1e-12 * scale
        assert np.abs(V[b].conj().T @ V[b] - np.eye(n)).max() < 1e-12
        assert np.abs(A[b] @ V[b] - V[b] * lam[b]).max() < 1e-11 * scale


@pytest.mark.parametrize("n,batch", [(1, 3), (7, 5), (72, 3), (81, 2), (112, 2), (113, 2), (136, 2), (200, 2)])
def test_device_eigh_fp32(env, n, batch):
    """FP32 Jacobi (mixed-precision truncation) on complex64 input: backward error of
    a Jacobi method is a modest multiple of n eps ||A|| (eps = 2^-24)."""
    torch, lib = env
    rng = np.random.default_rng(7 * n)
    A = rng.normal(size=(batch, n, n)) + 1j * rng.normal(size=(batch, n, n))
    A = A @ np.conj(np.transpose(A, (0, 2, 1)))
    A[0] *= 1e-3
    A32 = A.astype(np.complex64)
    dA = torch.tensor(A32.view(np.float32), device="cuda")
    lam = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    V = torch.zeros((batch, n, n, 2), dtype=torch.float64, device="cuda")
    assert lib.tns_test_eigh32(batch, n, _ptr(dA), _ptr(lam), _ptr(V), None) == 0
    import ctypes
    sw = (ctypes.c_int32 * batch)()
    assert lib.tns_test_eigh_sweeps(batch, ctypes.cast(sw, ctypes.c_void_p)) == 0
    assert all(0 < x <= 25 for x in sw), list(sw)
    lam = lam.cpu().numpy()
    V = V.cpu().numpy().view(np.complex128).reshape(batch, n, n)
    tol = 4 * n * 2.0 ** -24
    for b in range(batch):
        Ab = A32[b].astype(np.complex128)
        ref = np.linalg.eigvalsh(Ab)[::-1]
        scale = np.linalg.norm(Ab)
        assert np.abs(lam[b] - ref).max() < tol * scale
        assert np.abs(V[b].conj().T @ V[b] - np.eye(n)).max() < tol
        assert np.abs(Ab @ V[b] - V[b] * lam[b]).max() < tol * scale


@pytest.mark.parametrize("m,n,batch", [(4, 4, 2), (64, 64, 2), (40, 13, 3), (128, 128, 1), (200, 72, 2)])
def test_device_svd(env, m, n, batch):
    torch, lib = env
    rng = np.random.default_rng(m * n)
    A = rng.normal(size=(batch, m, n)) + 1j * rng.normal(size=(batch, m, n))
    A[0, :, -1] = A[0, :, 0]                                  # rank deficient
    dA = torch.tensor(A.view(np.float64), device="cuda")
    s = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    U = torch.zeros((batch, m, n, 2), dtype=torch.float64, device="cuda")
    V = torch.zeros((batch, n, n, 2), dtype=torch.float64, device="cuda")
    assert lib.tns_test_svd(batch, m, n, _ptr(dA), _ptr(s), _ptr(U), _ptr(V), None) == 0
    s = s.cpu().numpy()
    U = U.cpu().numpy().view(np.complex128).reshape(batch, m, n)
    V = V.cpu().numpy().view(np.complex128).reshape(batch, n, n)
    for b in range(batch):
        ref = np.linalg.svd(A[b], compute_uv=False)
        assert np.abs(s[b] - ref).max() < 1e-12 * ref[0]
        rec = (U[b] * s[b]) @ V[b].conj().T
        assert np.abs(rec - A[b]).max() < 1e-12 * ref[0]
        assert np.abs(V[b].conj().T @ V[b] - np.eye(n)).max() < 1e-12


@pytest.mark.parametrize("n,batch,rank", [(72, 3, 72), (72, 2, 50), (112, 2, 112), (113, 2, 100), (264, 2, 256)])
def test_device_cholesky_orthonormaliser(env, n, batch, rank):
    """Y W has orthonormal columns on range(Y) when W comes from the shifted Cholesky of Y^H Y."""
    torch, lib = env
    rng = np.random.default_rng(n + rank)
    m = 3 * n
    Y = (rng.normal(size=(batch, m, rank)) + 1j * rng.normal(size=(batch, m, rank))) @ \
        (rng.normal(size=(batch, rank, n)) + 1j * rng.normal(size=(batch, rank, n)))
    G = np.conj(np.transpose(Y, (0, 2, 1))) @ Y
    dG = torch.tensor(np.ascontiguousarray(G).view(np.float64), device="cuda")
    dW = torch.zeros((batch, n, n, 2), dtype=torch.float64, device="cuda")
    assert lib.tns_test_cholw(batch, n, 1e-14, _ptr(dG), _ptr(dW), None) == 0
    W = dW.cpu().numpy().view(np.complex128).reshape(batch, n, n)
    for b in range(batch):
        Q = Y[b] @ W[b]
        P = Q @ Q.conj().T                                   # projector onto range(Y)
        Yn = Y[b] / np.linalg.norm(Y[b])
        assert np.abs(P @ Yn - Yn).max() < 1e-10
        s = np.linalg.svd(Q, compute_uv=False)
        assert np.abs(s[:rank] - 1).max() < 1e-6


@pytest.mark.parametrize("M,N,K", [(128, 128, 16), (1000, 512, 512), (4096, 1024, 1024), (257, 130, 18), (8192, 96, 64),
                                   (77, 33, 5), (5, 300, 1)])
def test_device_tensor_core_gemm(env, M, N, K):
    """tcgen05 tf32x3 complex GEMM C = A B^T against complex128 numpy (FP32-level accuracy)."""
    torch, lib = env
    rng = np.random.default_rng(M + N + K)
    A = (rng.normal(size=(M, K)) + 1j * rng.normal(size=(M, K))).astype(np.complex64)
    B = (rng.normal(size=(N, K)) + 1j * rng.normal(size=(N, K))).astype(np.complex64)
    dA = torch.tensor(A.view(np.float32), device="cuda")
    dB = torch.tensor(B.view(np.float32), device="cuda")
    dC = torch.full((M, 2 * N), np.nan, dtype=torch.float32, device="cuda")
    rc = lib.tns_test_tcgemm(M, N, K, _ptr(dA), _ptr(dB), _ptr(dC), None)
    assert rc == 0, lib.tns_last_error()
    C = dC.cpu().numpy().view(np.complex64).astype(np.complex128)
    ref = A.astype(np.complex128) @ B.astype(np.complex128).T
    scale = np.abs(A).max() * np.abs(B).max() * np.sqrt(K)
    err = np.abs(C - ref).max() / scale
    # FP32 accumulation over 2K real products (~ sqrt(2K) 2^-23 of the scale) plus the
    # split's own error: hi and lo are rounded to nearest TF32, so each real product
    # carries up to 3 * 2^-22 |a||b| (the dropped lo*lo term and the two lo roundings)
    assert err < 2.5e-7 * np.sqrt(2 * K) + 6 * 2.0 ** -22 / np.sqrt(K), err


def _labelled(rng, labels, dims, shared=()):
    """Random complex64 array with one axis per label; axes in `shared` get stride 0."""
    shape = [1 if l in shared else d for l, d in zip(labels, dims)]
    X = (rng.normal(size=shape) + 1j * rng.normal(size=shape)).astype(np.complex64)
    strides = [0 if l in shared else s // 8 for l, s in zip(labels, X.strides)]
    full = np.broadcast_to(X, dims)
    return X, full, strides


def _contract(env, mode, la, A, sa, da, ca, lb, B, sb, db, cb, lc, dc):
    torch, lib = env
    cdt, fdt = (np.complex128, np.float64) if mode == 2 else (np.complex64, np.float32)
    dA = torch.tensor(np.ascontiguousarray(A.astype(cdt)).view(fdt), device="cuda")
    dB = torch.tensor(np.ascontiguousarray(B.astype(cdt)).view(fdt), device="cuda")
    n_c = int(np.prod(dc))
    dC = torch.full((2 * n_c,), float("nan"), dtype=torch.float64 if mode == 2 else torch.float32, device="cuda")
    sc = [int(np.prod(dc[i + 1:])) for i in range(len(dc))]
    a_d, a_s, b_d, b_s, c_d, c_s = (np.asarray(v, dtype=np.int64) for v in (da, sa, db, sb, dc, sc))
    rc = lib.tns_test_contract(la.encode(), a_d.ctypes.data, a_s.ctypes.data, int(ca), _ptr(dA),
                               lb.encode(), b_d.ctypes.data, b_s.ctypes.data, int(cb), _ptr(dB),
                               lc.encode(), c_d.ctypes.data, c_s.ctypes.data, _ptr(dC), mode, None)
    assert rc == 0, lib.tns_last_error()
    return dC.cpu().numpy().view(cdt).reshape(dc)


CONTRACTIONS = [
    # (labels A, dims A, shared A, conj A, labels B, dims B, shared B, conj B, labels C)
    ("SasdA", (3, 20, 2, 6, 17), "", 0, "SAfB", (3, 17, 9, 17), "", 0, "SasBdf"),          # absorb, odd K
    ("SasBdf", (3, 20, 2, 17, 6, 9), "", 0, "edDf", (11, 6, 5, 9), "", 0, "SaesBD"),      # shared environment
    ("SaesBD", (3, 20, 11, 2, 17, 5), "", 0, "ScsDB", (3, 13, 2, 5, 17), "", 1, "Saec"),   # conj, small N
    ("SsAfcD", (3, 2, 17, 9, 13, 5), "", 0, "ScsDB", (3, 13, 2, 5, 17), "", 1, "SsAfB"),   # two batch groups
    ("Saec", (4, 12, 7, 12), "", 1, "SasdA", (4, 12, 2, 5, 12), "S", 0, "ScsAed"),        # stride-0 batch in B
    ("Saec", (4, 12, 7, 12), "S", 0, "SasdA", (4, 12, 2, 5, 12), "", 0, "ScsAed"),        # stride-0 batch in A
    ("mk", (300, 40), "", 0, "nk", (200, 40), "", 0, "mn"),                               # BN = 256, ragged tiles
    ("km", (40, 300), "", 1, "kn", (40, 60), "", 0, "nm"),                                # transposed, BN = 128
    ("mc", (1024, 264), "", 1, "me", (1024, 264), "", 0, "ce"),                           # Gram Y^H Y, n > 128
    ("Smc", (2, 700, 136), "", 1, "Sme", (2, 700, 136), "", 0, "Sce"),                    # batched Gram
]


@pytest.mark.parametrize("case", range(len(CONTRACTIONS)))
def test_device_contraction_planner(env, case):
    """Labelled contractions on the tensor cores (mode 1), the FP32 CUDA cores (0) and
    FP64 (2) against complex128 einsum.  Bound, elementwise: FP32 summation of 2K real
    products, (2K + 2) 2^-23 sum |a||b|, plus 6 * 2^-22 sum |a||b| for the TF32 split
    (each real product within 3 * 2^-22 |a||b|; two real products per component)."""
    la, da, sha, ca, lb, db, shb, cb, lc = CONTRACTIONS[case]
    rng = np.random.default_rng(100 + case)
    A, Af, sa = _labelled(rng, la, da, sha)
    B, Bf, sb = _labelled(rng, lb, db, shb)
    dims = dict(zip(la, da))
    dims.update(zip(lb, db))
    dc = tuple(dims[l] for l in lc)
    Ac = np.conj(Af) if ca else Af
    Bc = np.conj(Bf) if cb else Bf
    spec = f"{la},{lb}->{lc}"
    ref = np.einsum(spec, Ac.astype(np.complex128), Bc.astype(np.complex128))
    ref_abs = np.einsum(spec, np.abs(Af).astype(np.float64), np.abs(Bf).astype(np.float64))
    K = int(np.prod([dims[l] for l in set(la) & set(lb) if l not in lc]))
    for mode in (1, 0, 2):
        C = _contract(env, mode, la, A, sa, da, ca, lb, B, sb, db, cb, lc, dc)
        tol = (1e-13 if mode == 2 else (2 * K + 2) * 2.0 ** -23 + (6 * 2.0 ** -22 if mode == 1 else 0)) * ref_abs
        assert np.all(np.abs(C - ref) <= tol), (mode, np.max(np.abs(C - ref) / ref_abs))


def test_tile_widths_are_bit_identical(env):
    """Every tensor-core tile variant (128 and 256 real columns pipelined, 128 columns
    single-stage with three CTAs per SM) gives the same bits, so the library's
    timing-based choice between them never changes a result."""
    import ctypes as C
    torch, lib = env
    rng = np.random.default_rng(21)
    for M, N, K in ((700, 200, 96), (4096, 96, 1024)):
        A = (rng.normal(size=(M, K)) + 1j * rng.normal(size=(M, K))).astype(np.complex64)
        B = (rng.normal(size=(N, K)) + 1j * rng.normal(size=(N, K))).astype(np.complex64)
        dA = torch.tensor(A.view(np.float32), device="cuda")
        dB = torch.tensor(B.view(np.float32), device="cuda")
        out = []
        for bn in (128, 256, 129):
            assert lib.tns_test_tc_tile(bn) == 0
            dC = torch.full((M, 2 * N), float("nan"), device="cuda")
            assert lib.tns_test_tcgemm(M, N, K, C.c_void_p(dA.data_ptr()), C.c_void_p(dB.data_ptr()),
                                       C.c_void_p(dC.data_ptr()), None) == 0
            out.append(dC.cpu())
        assert lib.tns_test_tc_tile(0) == 0
        assert torch.equal(out[0], out[1])
        assert torch.equal(out[0], out[2])
