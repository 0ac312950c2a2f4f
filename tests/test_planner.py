"""Host-side decisions of the tensor-core contraction planner (tile-class and operand
roles per shape), through tns_test_plan: no device is touched.  Shapes are the
sampler's contractions at the 10x10, chi = 16, chi_b = 64 workload with 128 samples."""
import ctypes

import numpy as np
import pytest

S, R, CHI, P = 128, 64, 16, 2


@pytest.fixture(scope="module")
def lib():
    from paper_2507_11424_gb300 import _native, build
    build.build()
    return _native.open_library(_native.LIB_PATH)


def view(labels, dims, shared=""):
    st, acc = [], 1
    for l, d in zip(reversed(labels), reversed(dims)):
        st.append(0 if l in shared else acc)
        acc *= 1 if l in shared else d
    return labels, list(dims), list(reversed(st))


def plan(lib, A, B, C, conj_a=0, conj_b=0):
    arr = lambda v: (ctypes.c_int64 * len(v))(*v)
    out = (ctypes.c_int64 * 11)()
    rc = lib.tns_test_plan(A[0].encode(), arr(A[1]), arr(A[2]), conj_a, B[0].encode(), arr(B[1]), arr(B[2]), conj_b,
                           C[0].encode(), arr(C[1]), arr(C[2]), out)
    assert rc == 0
    keys = ["tc", "swapped", "a_in_place", "a_shared", "b_shared", "merged", "tile_n", "M", "N", "K", "batch"]
    return dict(zip(keys, list(out)))


def test_environment_contraction_reads_A_in_place_with_wide_tiles(lib):
    # T2[S][a][e][s][B][D] = sum_{d,f} T1[S][a][s][B][d][f] E[e][D][d][f]
    d = plan(lib, view("SasBdf", (S, R, P, R, CHI, R)), view("eDdf", (R, CHI, CHI, R)),
             view("SaesBD", (S, R, R, P, R, CHI)))
    assert d["tc"] == 1 and d["swapped"] == 0 and d["a_in_place"] == 1 and d["tile_n"] == 256
    assert (d["M"], d["N"], d["K"], d["batch"]) == (S * R * P * R, R * CHI, CHI * R, 1)


def test_sweep_contraction_with_narrow_output_uses_half_tiles(lib):
    # F[S][a][e][c] = sum_{s,B,D} T2[S][a][e][s][B][D] conj K'[S][c][s][D][B]
    d = plan(lib, view("SaesBD", (S, R, R, P, R, CHI)), view("ScsDB", (S, R, P, CHI, R)),
             view("Saec", (S, R, R, R)), conj_b=1)
    assert d["tc"] == 1 and d["swapped"] == 0 and d["a_in_place"] == 1 and d["tile_n"] == 128
    assert (d["M"], d["N"], d["K"], d["batch"]) == (R * R, R, P * R * CHI, S)


def test_two_batch_groups(lib):
    # G[S][s][A][f][B] = sum_{c,D} U2[S][s][A][f][c][D] conj K'[S][c][s][D][B]
    d = plan(lib, view("SsAfcD", (S, P, R, R, R, CHI)), view("ScsDB", (S, R, P, CHI, R)),
             view("SsAfB", (S, P, R, R, R)), conj_b=1)
    assert d["tc"] == 1 and d["a_in_place"] == 1 and d["batch"] == S * P and d["tile_n"] == 128


def test_path_choice_is_per_batch_entry(lib):
    """Tensor cores or CUDA cores by the MACs of one batch entry (at least 2^18), never by
    the batch count: the two paths round differently, and a sample's result must not
    depend on the size of the chunk it is drawn in."""
    n = 72
    for batch in (1, 7, S):
        d = plan(lib, view("Smc", (batch, 2048, n)), view("Sme", (batch, 2048, n)), view("Sce", (batch, n, n)),
                 conj_a=1)
        assert d["tc"] == 1 and d["tile_n"] == 256 and d["a_in_place"] == 0  # conjugated A is gathered
        d = plan(lib, view("Smc", (batch, 32, 64)), view("Sme", (batch, 32, 64)), view("Sce", (batch, 64, 64)),
                 conj_a=1)
        assert d["tc"] == 0 and d["M"] * d["N"] * d["K"] < 2 ** 18
    # the operand roles do not follow the batch count either
    roles = {plan(lib, view("Smk", (b, 4096, 512)), view("Snk", (b, 256, 512), shared="S"),
                  view("Smn", (b, 4096, 256)))["swapped"] for b in (2, 7, S)}
    assert len(roles) == 1


def test_shared_operand_goes_to_the_expanded_side_and_rows_merge(lib):
    # A batched, B shared through a stride-0 batch axis: one launch over all rows
    d = plan(lib, view("Smk", (S, 4096, 512)), view("Snk", (S, 256, 512), shared="S"), view("Smn", (S, 4096, 256)))
    assert d["tc"] == 1 and d["b_shared"] == 1 and d["merged"] == 1 and d["swapped"] == 0
    # the shared operand given as A: roles swap so that it is expanded once
    d = plan(lib, view("Snk", (S, 256, 512), shared="S"), view("Smk", (S, 4096, 512)), view("Snm", (S, 256, 4096)))
    assert d["tc"] == 1 and d["swapped"] == 1 and d["b_shared"] == 1 and d["merged"] == 1


def test_both_operands_shared_is_not_a_tensor_core_batch(lib):
    d = plan(lib, view("Smk", (S, 1024, 512), shared="S"), view("Snk", (S, 512, 512), shared="S"),
             view("Smn", (S, 1024, 512)))
    assert d["tc"] == 0


def test_empty_and_inconsistent_views(lib):
    d = plan(lib, view("mk", (0, 8)), view("nk", (8, 8)), view("mn", (0, 8)))
    assert d["tc"] == 0 and d["M"] == 0
    arr = lambda v: (ctypes.c_int64 * len(v))(*v)
    out = (ctypes.c_int64 * 11)()
    rc = lib.tns_test_plan(b"mk", arr([4, 8]), arr([8, 1]), 0, b"nk", arr([8, 9]), arr([9, 1]), 0,
                           b"mn", arr([4, 8]), arr([8, 1]), out)
    assert rc == 1                                                 # k = 8 vs 9
