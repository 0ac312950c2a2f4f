"""Benchmark: boundary-MPS sampling throughput on one GB300 (samples/s).

Workload: the 10x10 square-lattice domain-wall Heisenberg quench (7 Trotter
layers, dt = 0.2, chi = 16) sampled with boundary rank chi_b = 64 in the
mixed-precision path.  The state is built by the library (gate layers + BP)
before timing; the norm environments are built once (cached in the state) and
reported separately.  A step is one tns_sample call over a batch of samples:
absorb + zip-up compression of every row, right environments, and the fused
marginal/draw/project sweep for every qubit.  The working set of a step is far
larger than the 129 MB L2, so no flush is needed between steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--batch B] [--impl gb300|reference]

Under torchrun (N > 1) every rank holds its own replica of the state and draws
its own samples (independent seeds): weak scaling, no collective on the data
path.  --impl reference times the CPU oracle (plain numpy complex128) instead.
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "samples/s at <=1e-3 marginal error vs plain sampler; boundary-MPS TFLOP/s"
CONFIG = "sq10x10"
WORKLOADS = {
    "sq10x10": "square 10x10 domain-wall Heisenberg quench, 7 layers dt=0.2, chi=16, chi_b=64",
    "sq4x4": "square 4x4 domain-wall Heisenberg quench, 4 layers dt=0.2, chi=4, chi_b=16",
    "heavyhex164": "heavy-hex 164 qubits (6x12 brick-wall honeycomb with bridges, degrees 2/3) domain-wall "
                   "Heisenberg quench, 20 layers dt=0.2, chi=32, chi_b=128",
    "ladder52": "2x26 ladder LUCJ-like circuit (Givens networks, phases, rung controlled phases; 3 repetitions), "
                "chi=64, chi_b=256",
}
WORKLOAD = WORKLOADS[CONFIG]
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
FP32_PEAK_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12   # 80.5 TFLOP/s SIMT FP32
TF32_PER_BF16 = 1.1 / 2.25          # nominal dense tf32 : bf16 tensor throughput
# DRAM traffic of the tensor-core GEMM kernel from one ncu capture of a smaller case of the
# same contraction (A 32768 x 1024 complex64 read once, B 1024 x 1024, C 32768 x 1024; the
# `--gemm-case 32768,1024,1024` mode of this script): dram read + write bytes and the case's
# algorithmic flop.  Traffic grows with the rows processed, so a launch's traffic is scaled
# by its flop.
TC_CAPTURE_BYTES = 401.568768e6 + 243.923456e6
TC_CAPTURE_FLOP = 8.0 * 32768 * 1024 * 1024


def tensor_peak():
    """Measured bf16 dense burst peak scaled to tf32, divided by the 3 MMA passes of the split product."""
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        bf16, src = float(pk["bf16_tflops"]), "measured"
    except Exception:
        bf16, src = 1900.0, "fallback"
    return bf16 * TF32_PER_BF16 / 3.0, src, bf16


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=None, help="samples per step (default 128; 1024 at 4x4)")
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--config", default=CONFIG, choices=sorted(WORKLOADS),
                    help="workload (the 10x10 square lattice is the headline; the others are the other paper shapes)")
    ap.add_argument("--mode", default="plain", choices=["plain", "learned"],
                    help="plain: the boundary-MPS sampler; learned: MADE proposal + independent MH on the same state")
    ap.add_argument("--train-samples", type=int, default=32768)
    ap.add_argument("--train-chib", type=int, default=16,
                    help="boundary rank of the plain-sampler draws the network is trained on")
    ap.add_argument("--proposals", type=int, default=8192)
    ap.add_argument("--chains", type=int, default=128)
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--compression", default=None, metavar="P,Q,QENV",
                    help="range-finder oversampling, subspace iterations, environment iterations (library defaults)")
    ap.add_argument("--plain-samples", type=int, default=4,
                    help="samples the plain FP64 sampler replays for its rate and the marginal error (0 = skip)")
    ap.add_argument("--cpu-budget", type=float, default=30.0)
    ap.add_argument("--gemm-case", default=None, metavar="M,N,K",
                    help="time one tensor-core complex GEMM C = A B^T of this shape instead (profiling case)")
    ap.add_argument("--gemm-reps", type=int, default=2)
    ap.add_argument("--state-cache", default=None,
                    help="TNSF file: load the state from it when present, else build it and save it there")
    return ap.parse_args()


SAMPLING_SEED = 20250711


def shard_first(rank: int, world: int, step: int, batch: int) -> int:
    """First stream index of a rank's samples at a step: the ranks split one sample
    stream (one seed) into disjoint, contiguous ranges, step after step, so the job's
    samples are the 1-GPU stream's first (step + 1) * world * batch samples."""
    return (step * world + rank) * batch


def max_over_ranks(x: float, world: int, device: str = "cuda") -> float:
    """The slowest rank's value (the job's time); identity on one rank."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world: int, batch: int, steps: int, seconds: float) -> float:
    """Whole-job samples/s: every rank draws `batch` samples per step."""
    return world * batch * steps / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(name: str | None = None):
    """(config dict, lattice, initial bits, gate groups) of a named workload."""
    import workloads as w
    cfg = w.CONFIGS[name or CONFIG]
    lat = w.make_lattice(cfg["lattice"])
    if "reps" in cfg:
        groups, bits = w.lucj_like_circuit(lat, reps=cfg["reps"], seed=11424)
    else:
        bits = w.domain_wall_bits(lat)
        groups = w.heisenberg_circuit(lat, cfg["layers"], cfg["dt"])
    return cfg, lat, bits, groups


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait(timeout=10)
        self.f.close()
        rows = [l.split(",") for l in open(self.path) if l.strip()]
        sm = [float(r[1]) for r in rows if len(r) >= 9 and r[1].strip().replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if len(r) >= 9 and r[2].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in rows:
            if len(r) < 9:
                continue
            for nm, v in zip(names, r[5:9]):
                if "Active" in v and "Not" not in v:
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle
def _oracle_sampler_worker(path, R, seed, budget, q):
    """Time the CPU oracle on the same state: norm environments, then samples until the budget."""
    import numpy as np
    from oracle import bmps, fixture
    t = fixture.load(path)
    t0 = time.time()
    E, _ = bmps.norm_envs(t, R, gram_cut=bmps.ORTH_SHIFT)
    env_s = time.time() - t0
    rows_done, t1 = 0, None
    H = t.H
    # one sample, row by row, until the budget is spent (a bounded sample of the workload).
    # Row 0 starts from the trivial boundary (rank 1) and is far cheaper than the rest: it
    # runs untimed, and the timed rows (from row 1, at full boundary rank) set the rate.
    m = [np.ones((1, 1, 1, 1), dtype=np.complex128) for _ in range(t.W)]
    for b in range(H):
        if b == 1:
            t1 = time.time()
        rev = (b % 2 == 1)
        cells = bmps.row_cells(t, b, rev)
        row = bmps.row_tensors(t, b, rev)
        Eb = E[b + 1] if not rev else bmps.mirror_mps(E[b + 1])
        from oracle import philox
        qubits = [int(t.cell_qubit[b, c]) for c in cells]
        uni = philox.draw_uniforms(seed, 0, np.array([max(x, 0) for x in qubits]))
        _, _, _, m_next = bmps.sample_row(m, row, Eb, R, seed, b, uniforms=uni, gram_cut=bmps.ORTH_SHIFT)
        m = bmps.mirror_mps(m_next)
        if t1 is None:
            continue
        rows_done += 1
        if time.time() - t1 > budget:
            break
    q.put(dict(env_s=env_s, rows=rows_done, H=H, sample_s=time.time() - t1 if t1 else 0.0,
               threads=os.cpu_count()))


def start_cpu_baseline(st, R, budget):
    path = os.path.join(tempfile.gettempdir(), f"bench_state_{os.getpid()}.tnsf")
    st.save(path)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    p = ctx.Process(target=_oracle_sampler_worker, args=(path, R, 7, budget, q), daemon=True)
    p.start()
    return p, q, path


def finish_cpu_baseline(p, q, path, timeout):
    res = None
    try:
        res = q.get(timeout=timeout)
    except Exception:
        pass
    if p.is_alive():
        p.terminate()
    try:
        os.unlink(path)
    except OSError:
        pass
    if not res:
        return None
    frac = res["rows"] / res["H"]
    return {"value": frac / res["sample_s"] if res["sample_s"] > 0 else None, "unit": "samples/s",
            "cores": res["threads"], "kind": "oracle",
            "sample": (f"CPU oracle (numpy complex128) on the same state: rows 1..{res['rows']} of {res['H']} "
                       f"of one sample (full boundary rank; row 0, rank 1, untimed) in {res['sample_s']:.1f} s, "
                       f"scaled by rows to samples/s; its norm environments took {res['env_s']:.1f} s (setup, "
                       f"excluded as on the GPU)")}


# ---------------------------------------------------------------- GPU arm
def plain_sampler(st, R, args, seed):
    """The plain FP64 sampler on the same state: its rate, and the marginal error of the
    mixed path against it.

    The mixed path draws `--plain-samples` samples with their conditionals; the FP64 path
    (every contraction and factorisation in FP64) then replays the same bitstrings
    (forced-path replay, the same work as drawing them) and is timed with CUDA events
    after a one-sample warm-up.  The marginal error is max / mean |q_mixed - q_fp64| over
    every conditional q(x_v = 0 | prefix) of those samples.
    """
    import torch
    n = args.plain_samples
    xs, _, cond_m = st.sample(R, n, seed, cond=True)
    st.set_precision("fp64")
    try:
        t0 = time.time()
        st.log_norm(R)                            # FP64 norm environments (setup, as for the mixed path)
        env_s = time.time() - t0
        st.sample_replay(R, xs[:1], seed)         # warm-up
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, cond_p = st.sample_replay(R, xs, seed)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
    finally:
        st.set_precision(args.prec)
    d = (cond_m - cond_p).abs()
    return {"samples_per_s": n / (ms / 1e3), "samples": n, "ms": ms, "env_build_s": round(env_s, 2),
            "marginal_err_max": float(d.max()), "marginal_err_mean": float(d.mean()),
            "what": ("TNS_PREC_FP64 replay of the mixed path's bitstrings (same work as drawing them), CUDA events; "
                     "marginal error = |q_mixed - q_fp64| over every conditional of those samples")}


def build_state(pkg, lat, bits, groups, chi, prec):
    """The state through the library (gate layers, then BP after every layer), with
    the BP measurements summed over the build: device time and algorithmic bytes and
    flops from tns_bp_stats, and wall time of the gate layers."""
    import torch
    st = pkg.TNSState(lat.grid_rc, lat.edges, bits, chi_max=chi, prec=prec)
    bp = {"calls": 0, "iters": 0, "ms": 0.0, "bytes": 0.0, "flops": 0.0, "gates_s": 0.0, "max_residual": 0.0}
    for g in groups:
        t0 = time.time()
        st.apply_gate_layer(g, chi=chi)
        torch.cuda.synchronize()
        bp["gates_s"] += time.time() - t0
        it, res = st.bp_gauge(300, 1e-10)
        s = st.bp_stats()
        bp["calls"] += 1
        bp["iters"] += it
        bp["max_residual"] = max(bp["max_residual"], res)
        for k in ("ms", "bytes", "flops"):
            bp[k] += s[k]
    return st, bp


def bp_report(bp, prec):
    """BP over the state build: achieved GB/s (algorithmic bytes / device time) against
    the measured HBM copy rate, and the message contractions' TFLOP/s."""
    if not bp or bp["ms"] <= 0:
        return None
    try:
        hbm = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"])
        src = "measured"
    except Exception:
        hbm, src = 6800.0, "fallback"
    gbs = bp["bytes"] / (bp["ms"] / 1e3) / 1e9
    return {"calls": bp["calls"], "iterations": bp["iters"], "device_s": round(bp["ms"] / 1e3, 3),
            "ms_per_iteration": round(bp["ms"] / max(1, bp["iters"]), 3),
            "achieved_gbs": round(gbs, 1), "hbm_peak_gbs": hbm, "hbm_frac": round(gbs / hbm, 4),
            "peak_note": f"{src} HBM copy rate",
            "tflops": round(bp["flops"] / (bp["ms"] / 1e3) / 1e12, 3), "max_final_residual": bp["max_residual"],
            "gates_wall_s": round(bp["gates_s"], 2),
            "precision": ("complex64 contractions (TF32x3 tensor cores / FP32), FP64 normalisation" if prec == "mixed"
                          else "FP64")}


def run_gpu(args):
    import torch
    import paper_2507_11424_gb300 as pkg
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg, lat, bits, groups = workload()
    chi, R, B = cfg["chi"], cfg["chi_b"], args.batch
    t0 = time.time()
    bp = None
    if args.state_cache and os.path.exists(args.state_cache):
        st = pkg.TNSState.load_file(args.state_cache)
        st.n = lat.n_qubits
        st.set_precision(args.prec)
    else:
        st, bp = build_state(pkg, lat, bits, groups, chi, args.prec)
        if args.state_cache:
            st.save(args.state_cache)
    torch.cuda.synchronize()
    build_s = time.time() - t0
    if args.compression:
        st.set_compression(*(int(x) for x in args.compression.split(",")))
    t0 = time.time()
    log_norm = st.log_norm(R)
    torch.cuda.synchronize()
    env_s = time.time() - t0
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = start_cpu_baseline(st, R, args.cpu_budget)
    n_sites = lat.n_qubits
    bits_d = torch.zeros((B, n_sites), dtype=torch.uint8, device="cuda")
    logq_d = torch.zeros(B, dtype=torch.float64, device="cuda")
    seed = SAMPLING_SEED
    step_no = 0

    def draw():
        nonlocal step_no
        st.sample(R, B, seed, out=(bits_d, logq_d, None), first=shard_first(rank, world, step_no, B))
        step_no += 1

    for i in range(args.warmup):
        draw()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = Clocks(local)
    clocks.start()
    launches0 = st.launch_count()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    for k in range(args.steps):
        draw()
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1)
    launches = st.launch_count() - launches0
    clk = clocks.stop()
    # one more step with per-class kernel timing (CUDA events around every launch on the
    # library's stream; launches are eager while timing is on): the class breakdown and
    # the dominant kernel's achieved rate for the roofline
    st.profile(True)
    draw()
    torch.cuda.synchronize()
    prof = st.profile_read()
    st.profile(False)
    prof_steps = 1
    ms = max_over_ranks(ms, world)
    value = job_rate(world, B, args.steps, ms / 1e3)
    # end to end through the public API: host-visible results every step
    bits_h = torch.empty((B, n_sites), dtype=torch.uint8, pin_memory=True)
    logq_h = torch.empty(B, dtype=torch.float64, pin_memory=True)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.time()
    for k in range(args.steps):
        draw()
        bits_h.copy_(bits_d, non_blocking=True)
        logq_h.copy_(logq_d, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    e2e_s = time.time() - t0
    e2e_s = max_over_ranks(e2e_s, world)
    sector = float((bits_h.numpy().sum(axis=1) == int(bits.sum())).mean())
    plain = plain_sampler(st, R, args, seed) if args.prec == "mixed" and args.plain_samples > 0 else None
    env = prof["env_gemm"]
    achieved = env["flops"] / (env["ms"] / 1e3) / 1e12 if env["ms"] > 0 else None
    total_flops = sum(v["flops"] for v in prof.values())
    if args.prec == "mixed" and prof["tc_prep"]["launches"] > 0:
        peak, src, bf16 = tensor_peak()
        per_launch_flop = env["flops"] / env["launches"] if env["launches"] else 0.0
        roofline = {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                    "frac": achieved / peak if achieved else None,
                    "traffic": TC_CAPTURE_BYTES * per_launch_flop / TC_CAPTURE_FLOP,
                    "traffic_note": "bytes per average launch, scaled by flop from the ncu capture of the "
                                    "32768 x 1024 x 1024 case",
                    "kernel": "tc_gemm_tf32x3_kernel (environment contraction, tcgen05 kind::tf32, 3-pass split)",
                    "peak_note": (f"{src} bf16 dense burst {bf16} TFLOP/s x {TF32_PER_BF16:.3f} (nominal tf32/bf16) "
                                  "/ 3 MMA passes per product; achieved counts 8 flop per complex MAC once")}
    else:
        roofline = {"bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_PEAK_TFLOPS if achieved else None, "traffic": None,
                    "kernel": "env_gemm on CUDA cores (SIMT complex contraction)",
                    "peak_note": "152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz"}
    # the oracle first builds its norm environments (a few minutes of setup), then times rows
    cpu_res = finish_cpu_baseline(*cpu, timeout=args.cpu_budget + 900.0) if cpu else None
    out = {
        "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64" if args.prec == "mixed" else "c128", "data": "synthetic",
        "config": {"workload": WORKLOAD, "samples_per_step": B, "precision_path": args.prec, "l2": "working set > L2, no flush",
                   "compression": args.compression or "48,3,6 (library defaults: oversampling, subspace iterations, "
                                                      "environment iterations)",
                   "cuda_graphs": "per-chunk launch sequence replayed from a graph after warm-up",
                   "parallelism": f"replicas x{world}, one sample stream sharded by index"},
        "e2e": {"value": job_rate(world, B, args.steps, e2e_s), "unit": "samples/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": B * n_sites + 8 * B},
        "roofline": roofline,
        "cpu_baseline": cpu_res,
        "clocks": clk,
        "gpu_launches": launches,
        "boundary_mps_tflops": total_flops * args.steps / prof_steps / (ms / 1e3) / 1e12,
        "profile_steps": prof_steps,
        "profile": {k: {"ms": round(v["ms"], 2), "launches": v["launches"],
                        "tflops": round(v["flops"] / (v["ms"] / 1e3) / 1e12, 2) if v["ms"] > 0 and v["flops"] else None}
                    for k, v in prof.items() if v["launches"]},
        "plain_fp64": plain,
        "state_build_s": round(build_s, 2), "bp": bp_report(bp, args.prec),
        "env_build_s": round(env_s, 3), "log_norm": log_norm,
        "log_fidelity": st.log_fidelity(), "sector_fraction": sector,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    st.close()
    if world > 1:
        torch.distributed.destroy_process_group()


# ---------------------------------------------------------------- learned proposal
def marginals(bits):
    """One-site means and same-sample two-site means <x_i x_j> of a [N][n] bit array."""
    import numpy as np
    x = np.asarray(bits, dtype=np.float64)
    return x.mean(0), (x.T @ x) / x.shape[0]


def run_learned(args):
    """The learned-proposal sampler on the 10x10 state (independent MH with a MADE proposal).

    Steps, on one GPU, all through the library: (1) plain-sampler draws at boundary rank
    --train-chib as training data; (2) MADE training (4 weight layers, hidden 256, BF16
    tensor-core GEMMs, Adam, 20 epochs); (3) --proposals ancestral proposals and their
    log g; (4) log p = 2 log|<x|psi>| at chi_b = 64 for every proposal (tns_amplitude);
    (5) --chains independent MH chains over the proposals, started from plain-sampler
    draws.  Timed (CUDA events): the sampling stage (3)-(5) against the plain mixed
    sampler at chi_b = 64 drawing the reference samples on the same state; training
    (1)-(2) is reported separately (paid once per state).  Marginal quality: TVD-style
    maximum distance of one- and two-site marginals of the chain states from the plain
    sampler's, with the plain sampler's shot noise beside it.
    """
    import numpy as np
    import torch
    import paper_2507_11424_gb300 as pkg
    import workloads as w
    torch.cuda.set_device(0)
    cfg, lat, bits, groups = workload()
    chi, R, n = cfg["chi"], cfg["chi_b"], lat.n_qubits
    t0 = time.time()
    if args.state_cache and os.path.exists(args.state_cache):
        st = pkg.TNSState.load_file(args.state_cache)
        st.n = n
        st.set_precision("mixed")
    else:
        st, _ = build_state(pkg, lat, bits, groups, chi, "mixed")
        if args.state_cache:
            st.save(args.state_cache)
    build_s = time.time() - t0

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        out = fn()
        e1.record()
        torch.cuda.synchronize()
        return out, e0.elapsed_time(e1) / 1e3

    st.log_norm(R)
    st.log_norm(args.train_chib)
    # plain sampler at chi_b = 64: the reference draws and the rate to beat
    (ref_bits, _), plain_s = timed(lambda: st.sample(R, args.batch, 424242))
    plain_rate = args.batch / plain_s
    # (1)-(2) training data and training
    (train_bits, _), data_s = timed(lambda: st.sample(args.train_chib, args.train_samples, 777))
    h, epochs = 256, 20
    m = pkg.MADE(n, h, w.made_init(n, h, seed=7))
    losses, train_s = timed(lambda: m.train(train_bits, 1024, epochs, lr=1e-3,
                                            orders=w.epoch_orders(args.train_samples, epochs, seed=3)))
    # (3)-(5) the learned sampler
    Cn = args.chains
    T = args.proposals // Cn

    def learned():
        prop, lg = m.sample(Cn * T, seed=5)
        lp = 2 * st.amplitude(R, prop)[0]
        lp0 = 2 * st.amplitude(R, ref_bits[:Cn])[0]
        state, acc = pkg.mh_independent(lp.reshape(Cn, T), lg.reshape(Cn, T), lp0, m.log_prob(ref_bits[:Cn]), seed=8)
        return prop, state, acc

    (prop, state, acc), learn_s = timed(learned)
    state = state.cpu().numpy()
    propn, starts = prop.cpu().numpy().reshape(Cn, T, n), ref_bits[:Cn].cpu().numpy()
    held = np.take_along_axis(propn, np.maximum(state, 0)[..., None], 1)
    chain = np.where(state[..., None] >= 0, held, starts[:, None, :]).reshape(-1, n)
    rate = float(acc.cpu().numpy().mean() / T)
    m1_ref, m2_ref = marginals(ref_bits.cpu().numpy())
    m1, m2 = marginals(chain)
    m1_prop, m2_prop = marginals(propn.reshape(-1, n))
    out = {
        "metric": "learned-proposal samples/s vs plain sampler (independent MH, MADE proposal)",
        "mode": "learned", "config": {"workload": WORKLOAD, "chi_b": R, "train_chi_b": args.train_chib,
                                      "train_samples": args.train_samples, "proposals": Cn * T, "chains": Cn,
                                      "steps": T, "made": f"n={n}, hidden={h}, 4 weight layers, BF16 tcgen05"},
        "learned_chain_states_per_s": Cn * T / learn_s,
        "learned_accepted_per_s": float(acc.cpu().numpy().sum()) / learn_s,
        "acceptance": rate,
        "plain_samples_per_s": plain_rate,
        "plain_reference_samples": args.batch,
        "train": {"data_s": round(data_s, 2), "train_s": round(train_s, 2), "loss_first": float(losses[0]),
                  "loss_last": float(losses[-1])},
        "marginals_vs_plain": {
            "one_site_max_abs": float(np.abs(m1 - m1_ref).max()),
            "two_site_max_abs": float(np.abs(m2 - m2_ref).max()),
            "raw_proposals_one_site_max_abs": float(np.abs(m1_prop - m1_ref).max()),
            "plain_shot_noise_1sigma": float(np.sqrt(0.25 / args.batch)),
        },
        "state_build_s": round(build_s, 2),
    }
    print(json.dumps(out), flush=True)
    m.close()
    st.close()


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The CPU oracle as the reference implementation, on the same workload and metric.

    The oracle applies the same circuit by its simple update; BP runs at most
    two sweeps per gate group (the oracle's BP costs seconds per sweep here, and
    the sampler's cost depends only on the bond dimensions, which saturate at
    chi either way).  A step is one row of one sample (a bounded sample of the
    workload); samples/s = (1/H) / seconds per step.
    """
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import numpy as np
    from oracle import bmps, philox
    from oracle.tns import GridTNS
    cfg, lat, bits, groups = workload()
    chi, R = cfg["chi"], cfg["chi_b"]
    t = GridTNS(lat.grid_rc, lat.edges, bits)
    for g in groups:
        t.apply_group(g, chi)
        t.bp(2, 1e-10)
    E, _ = bmps.norm_envs(t, R, gram_cut=bmps.ORTH_SHIFT)
    H = t.H
    m = [np.ones((1, 1, 1, 1), dtype=np.complex128) for _ in range(t.W)]
    times = []
    for k in range(args.warmup + args.steps):
        b = k % H
        if b == 0:
            m = [np.ones((1, 1, 1, 1), dtype=np.complex128) for _ in range(t.W)]
        rev = (b % 2 == 1)
        cells = bmps.row_cells(t, b, rev)
        row = bmps.row_tensors(t, b, rev)
        Eb = E[b + 1] if not rev else bmps.mirror_mps(E[b + 1])
        qubits = [int(t.cell_qubit[b, c]) for c in cells]
        uni = philox.draw_uniforms(7, k // H, np.array([max(x, 0) for x in qubits]))
        t0 = time.time()
        _, _, _, m_next = bmps.sample_row(m, row, Eb, R, 7, b, uniforms=uni, gram_cut=bmps.ORTH_SHIFT)
        times.append(time.time() - t0)
        m = bmps.mirror_mps(m_next)
    step = sum(times[args.warmup:]) / max(1, args.steps)
    value = (1.0 / H) / step
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": "samples/s", "n_gpus": world,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
           "config": {"workload": WORKLOAD, "samples_per_step": args.batch, "parallelism": f"replicas x{world}",
                      "step": "one row of one sample (the oracle's rate is scaled to samples/s)"},
           "cpu_baseline": {"value": value, "unit": "samples/s", "cores": os.cpu_count(), "kind": "oracle",
                            "sample": f"one row of one sample per step ({args.steps} timed steps), scaled by 1/{H}"},
           "e2e": {"value": value, "unit": "samples/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_gemm_case(args):
    """One tensor-core complex contraction C = A B^T (A complex64 [M][K], B [N][K], random)
    through tns_test_tcgemm (B expansion, then the GEMM kernel), timed with CUDA events;
    prints the mean time per call after the first and the algorithmic rate 8 M N K / t."""
    import ctypes as C
    import torch
    from paper_2507_11424_gb300 import build, _native
    M, N, K = (int(x) for x in args.gemm_case.split(","))
    build.build()
    lib = _native.load()
    g = torch.Generator(device="cuda").manual_seed(0)
    A = torch.randn((M, 2 * K), device="cuda", generator=g)
    B = torch.randn((N, 2 * K), device="cuda", generator=g)
    Cm = torch.empty((M, 2 * N), device="cuda")
    times = []
    for _ in range(max(1, args.gemm_reps)):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc = lib.tns_test_tcgemm(M, N, K, C.c_void_p(A.data_ptr()), C.c_void_p(B.data_ptr()),
                                 C.c_void_p(Cm.data_ptr()), None)
        e1.record()
        torch.cuda.synchronize()
        if rc != 0:
            raise SystemExit(f"tns_test_tcgemm failed: {lib.tns_last_error().decode()}")
        times.append(e0.elapsed_time(e1))
    ms = sum(times[1:]) / (len(times) - 1) if len(times) > 1 else times[0]
    print(json.dumps({"gemm_case": [M, N, K], "ms_per_call": ms, "tflops": 8.0 * M * N * K / (ms / 1e3) / 1e12}))


def main():
    global CONFIG, WORKLOAD
    args = parse()
    CONFIG, WORKLOAD = args.config, WORKLOADS[args.config]
    if args.batch is None:
        args.batch = 1024 if args.config == "sq4x4" else 128
    if args.gemm_case:
        run_gemm_case(args)
        return
    if args.mode == "learned" and args.impl != "reference":
        run_learned(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
