"""Run one tensor-core complex contraction of a given shape (profiling case).

    python -m paper_2507_11424_gb300.tc_case --M 32768 --N 1024 --K 1024 --reps 2

C = A B^T with A complex64 [M][K] and B complex64 [N][K] random, through
tns_test_tcgemm (the library's TF32x3 tcgen05 path: B expansion, then the GEMM
kernel).  Prints the mean time per call measured with CUDA events and the
algorithmic rate 8 M N K / t.
"""
from __future__ import annotations

import argparse
import ctypes as C
import json


def main():
    import torch
    from . import build, _native
    ap = argparse.ArgumentParser()
    ap.add_argument("--M", type=int, default=32768)
    ap.add_argument("--N", type=int, default=1024)
    ap.add_argument("--K", type=int, default=1024)
    ap.add_argument("--reps", type=int, default=2)
    a = ap.parse_args()
    build.build()
    lib = _native.load()
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((a.M, 2 * a.K), device="cuda", generator=g)
    B = torch.randn((a.N, 2 * a.K), device="cuda", generator=g)
    Cm = torch.empty((a.M, 2 * a.N), device="cuda")
    times = []
    for _ in range(a.reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc = lib.tns_test_tcgemm(a.M, a.N, a.K, C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                                 C.c_void_p(Cm.data_ptr()), None)
        e1.record()
        torch.cuda.synchronize()
        if rc != 0:
            raise SystemExit(f"tns_test_tcgemm failed: {lib.tns_last_error().decode()}")
        times.append(e0.elapsed_time(e1))
    ms = sum(times[1:]) / max(1, len(times) - 1) if len(times) > 1 else times[0]
    print(json.dumps({"M": a.M, "N": a.N, "K": a.K, "ms_per_call": ms,
                      "tflops": 8.0 * a.M * a.N * a.K / (ms / 1e3) / 1e12}))


if __name__ == "__main__":
    main()
