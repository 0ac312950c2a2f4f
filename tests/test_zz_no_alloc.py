"""tns_eigh_noalloc against the allocating eigensolver entry point (GPU).

The no-allocation variant serves callers that cannot call cudaMalloc (device
memory owned by another allocator, or latency-critical code that cannot take an
allocation's synchronisation); its scratch is a static device array shared by
every call.  This file is collected last so that a failure here leaves every
other test already run; it also passes on its own in a fresh process.
"""
import ctypes

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
    return ctypes.c_void_p(t.data_ptr())


@pytest.mark.parametrize("n,batch", [(136, 3), (40, 4)])
def test_noalloc_eigh_matches_allocating_entry_point(env, n, batch):
    torch, lib = env
    rng = np.random.default_rng(7 * n + batch)
    A = rng.normal(size=(batch, n, n)) + 1j * rng.normal(size=(batch, n, n))
    A = A @ np.conj(np.transpose(A, (0, 2, 1)))
    dA = torch.tensor(np.ascontiguousarray(A).view(np.float64), device="cuda")
    lam_ref = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    V_ref = torch.zeros((batch, n, n, 2), dtype=torch.float64, device="cuda")
    assert lib.tns_test_eigh(batch, n, _ptr(dA), _ptr(lam_ref), _ptr(V_ref), None) == 0
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    scale = float(torch.abs(lam_ref).max())
    for _ in range(2):                       # two calls in a row share the same scratch
        lam = torch.full((batch, n), np.nan, dtype=torch.float64, device="cuda")
        V = torch.full((batch, n, n, 2), np.nan, dtype=torch.float64, device="cuda")
        assert lib.tns_eigh_noalloc(batch, n, _ptr(dA), _ptr(lam), _ptr(V), stream) == 0
        torch.cuda.synchronize()
        assert torch.abs(lam - lam_ref).max().item() < 1e-12 * scale
        assert torch.abs(V - V_ref).max().item() < 1e-10
        Vc = V.cpu().numpy().view(np.complex128).reshape(batch, n, n)
        lc = lam.cpu().numpy()
        for b in range(batch):
            assert np.abs(A[b] @ Vc[b] - Vc[b] * lc[b]).max() < 1e-11 * scale
        # every matrix converged, and the status query reads that back
        st = torch.full((batch,), -1, dtype=torch.int32, device="cuda")
        assert lib.tns_eigh_noalloc_status(batch, _ptr(st), stream) == 0
        torch.cuda.synchronize()
        assert st.tolist() == [0] * batch
    assert lib.tns_eigh_noalloc_status(batch + 1, _ptr(st), stream) == 1


def test_noalloc_rejects_batches_beyond_the_static_scratch(env):
    torch, lib = env
    n, batch = 264, 64                       # 64 x 2.2 MB of scratch > 16 MiB
    dA = torch.zeros((batch, n, n, 2), dtype=torch.float64, device="cuda")
    lam = torch.zeros((batch, n), dtype=torch.float64, device="cuda")
    V = torch.zeros((batch, n, n, 2), dtype=torch.float64, device="cuda")
    assert lib.tns_eigh_noalloc(batch, n, _ptr(dA), _ptr(lam), _ptr(V), None) == 1
    assert b"static limit" in lib.tns_last_error()
