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


@pytest.mark.parametrize("n,batch,rank", [(72, 3, 72), (72, 2, 50), (264, 2, 256)])
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


@pytest.mark.parametrize("M,N,K", [(128, 128, 16), (1000, 512, 512), (4096, 1024, 1024), (257, 130, 18), (8192, 96, 64)])
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
    # FP32 accumulation over 2K real products: ~ sqrt(2K) * 2^-23 of the scale
    assert err < 2.5e-7 * np.sqrt(2 * K), err
