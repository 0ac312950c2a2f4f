"""GB300-native boundary-MPS sampler for 2D tensor-network states (arXiv 2507.11424).

Python view of the C ABI in ``include/tns.h``.  torch supplies device memory and
the CUDA stream; every computation runs in the sm_103a kernels of libtns.so.

    st = TNSState(lat.grid_rc, lat.edges, bits, chi_max=16)
    for group in circuit:
        st.apply_gate_layer(group, chi=16)
        st.bp_gauge()
    bits, logq = st.sample(chi_b=64, n=1024, seed=1)
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _native
from ._native import PREC, TNSError, check, load  # noqa: F401

__all__ = ["TNSState", "MADE", "mh_independent", "TNSError", "load", "pack_group"]


def _torch():
    import torch
    return torch


def _stream_handle(stream):
    torch = _torch()
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


def pack_group(group):
    """Gate list [(q0, q1 or -1, U), ...] -> (sites int32 [g,2], mats float64 [g,16,2])."""
    g = len(group)
    sites = np.full((g, 2), -1, dtype=np.int32)
    mats = np.zeros((g, 16, 2), dtype=np.float64)
    for i, (a, b, U) in enumerate(group):
        sites[i] = (a, b)
        flat = np.asarray(U, dtype=np.complex128).reshape(-1)
        mats[i, : flat.size, 0] = flat.real
        mats[i, : flat.size, 1] = flat.imag
    return sites, mats


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


class TNSState:
    """Owner of a library state (one processor-shaped TNS on the current GPU)."""

    def __init__(self, grid_rc=None, edges=None, bits=None, chi_max: int = 16, prec: str = "mixed",
                 stream=None, _handle=None):
        self.lib = load()
        self._h = C.c_void_p()
        if _handle is not None:
            self._h = _handle
            return
        grid = np.ascontiguousarray(np.asarray(grid_rc, dtype=np.int32).reshape(-1, 2))
        ed = np.ascontiguousarray(np.asarray(edges, dtype=np.int32).reshape(-1, 2))
        b = np.ascontiguousarray(np.asarray(bits, dtype=np.uint8).reshape(-1))
        self.n = grid.shape[0]
        check(self.lib.tns_build_lattice(grid.shape[0], _ptr(grid), ed.shape[0], _ptr(ed), _ptr(b), int(chi_max),
                                         PREC[prec], _stream_handle(stream), C.byref(self._h)), "tns_build_lattice")

    @classmethod
    def load_file(cls, path: str, stream=None) -> "TNSState":
        lib = load()
        h = C.c_void_p()
        check(lib.tns_load(path.encode(), _stream_handle(stream), C.byref(h)), "tns_load")
        st = cls(_handle=h)
        st.n = None
        return st

    def close(self):
        if self._h:
            self.lib.tns_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---------------------------------------------------------------- circuit
    def apply_gate_layer(self, group, chi: int, cutoff: float = 1e-14) -> np.ndarray:
        sites, mats = group if isinstance(group, tuple) else pack_group(group)
        sites = np.ascontiguousarray(sites, dtype=np.int32)
        mats = np.ascontiguousarray(mats, dtype=np.float64)
        eps = np.zeros(sites.shape[0], dtype=np.float64)
        check(self.lib.tns_apply_gate_layer(self._h, sites.shape[0], _ptr(sites), _ptr(mats), int(chi),
                                            float(cutoff), _ptr(eps)), "tns_apply_gate_layer")
        return eps

    def bp_gauge(self, max_iter: int = 500, tol: float = 1e-12, strict: bool = False):
        it = C.c_int32()
        res = C.c_double()
        allow = () if strict else (_native.TNS_ERR_NOT_CONVERGED,)
        check(self.lib.tns_bp_gauge(self._h, int(max_iter), float(tol), C.byref(it), C.byref(res)),
              "tns_bp_gauge", allow)
        return it.value, res.value

    def bp_stats(self) -> dict:
        """Device time, algorithmic bytes and flops of the last bp_gauge call."""
        ms, by, fl = C.c_double(), C.c_double(), C.c_double()
        check(self.lib.tns_bp_stats(self._h, C.byref(ms), C.byref(by), C.byref(fl)), "tns_bp_stats")
        return {"ms": ms.value, "bytes": by.value, "flops": fl.value}

    def log_fidelity(self) -> float:
        v = C.c_double()
        check(self.lib.tns_log_fidelity(self._h, C.byref(v)), "tns_log_fidelity")
        return v.value

    def log_norm(self, chi_b: int) -> float:
        v = C.c_double()
        check(self.lib.tns_log_norm(self._h, int(chi_b), C.byref(v)), "tns_log_norm")
        return v.value

    def direct_marginals(self, chi_b: int, pairs: bool = True):
        """(one [n], two [n, n] or None): <n_q> and same-row <n_q n_q'> by boundary-MPS contraction."""
        if self.n is None:
            raise ValueError("number of qubits unknown: set .n after load_file")
        n = self.n
        one = np.zeros(n, dtype=np.float64)
        two = np.zeros((n, n), dtype=np.float64) if pairs else None
        check(self.lib.tns_direct_marginals(self._h, int(chi_b), _ptr(one), _ptr(two) if pairs else None),
              "tns_direct_marginals")
        return one, two

    def set_precision(self, prec: str):
        check(self.lib.tns_set_precision(self._h, PREC[prec]), "tns_set_precision")

    def query(self):
        H, W, tr, chi = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        check(self.lib.tns_query(self._h, C.byref(H), C.byref(W), C.byref(tr), C.byref(chi)), "tns_query")
        return dict(H=H.value, W=W.value, transposed=bool(tr.value), chi=chi.value)

    def save(self, path: str):
        check(self.lib.tns_save(self._h, path.encode()), "tns_save")

    def launch_count(self) -> int:
        v = C.c_int64()
        check(self.lib.tns_launch_count(self._h, C.byref(v)), "tns_launch_count")
        return v.value

    PROFILE_CLASSES = ("env_gemm", "sweep_gemm", "zip_gemm", "eigh", "marginal", "tc_prep", "tc_prep_sweep",
                       "tc_prep_zip", "zip_simt", "sweep_simt")

    def set_compression(self, oversample: int, power_iters: int, env_power_iters: int):
        """Range-finder settings of the truncated SVDs (see tns_set_compression)."""
        check(self.lib.tns_set_compression(self._h, int(oversample), int(power_iters), int(env_power_iters)),
              "tns_set_compression")

    def set_graphs(self, enable: bool):
        """Replay the sampler's per-chunk launch sequence from CUDA graphs (see tns_set_graphs)."""
        check(self.lib.tns_set_graphs(self._h, 1 if enable else 0), "tns_set_graphs")

    def set_tensor_cores(self, enable: bool):
        check(self.lib.tns_set_tensor_cores(self._h, 1 if enable else 0), "tns_set_tensor_cores")

    def profile(self, enable: bool = True):
        check(self.lib.tns_profile_enable(self._h, 1 if enable else 0), "tns_profile_enable")

    def profile_read(self):
        out = {}
        for i, name in enumerate(self.PROFILE_CLASSES):
            ms, n, fl = C.c_double(), C.c_int64(), C.c_double()
            check(self.lib.tns_profile_read(self._h, i, C.byref(ms), C.byref(n), C.byref(fl)), "tns_profile_read")
            out[name] = dict(ms=ms.value, launches=n.value, flops=fl.value)
        return out

    # ---------------------------------------------------------------- sampling
    def sample(self, chi_b: int, n: int, seed: int, n_sites: int | None = None, cond: bool = False, out=None,
               first: int = 0):
        """Draw n samples; returns torch CUDA tensors (bits uint8 [n, n_sites], logq f64 [n][, cond]).
        first > 0 draws samples first .. first + n - 1 of the seed's stream (tns_sample_range)."""
        torch = _torch()
        ns = n_sites or self.n
        if out is None:
            bits = torch.zeros((n, ns), dtype=torch.uint8, device="cuda")
            logq = torch.zeros(n, dtype=torch.float64, device="cuda")
            cnd = torch.zeros((n, ns), dtype=torch.float64, device="cuda") if cond else None
        else:
            bits, logq, cnd = out
        ptrs = (C.c_void_p(bits.data_ptr()), C.c_void_p(logq.data_ptr()),
                C.c_void_p(cnd.data_ptr()) if cnd is not None else None)
        sd = C.c_uint64(int(seed) & (2**64 - 1))
        if first:
            check(self.lib.tns_sample_range(self._h, int(chi_b), int(first), int(n), sd, *ptrs), "tns_sample_range")
        else:
            check(self.lib.tns_sample(self._h, int(chi_b), int(n), sd, *ptrs), "tns_sample")
        return (bits, logq, cnd) if cond else (bits, logq)

    def sample_replay(self, chi_b: int, bits, seed: int = 0):
        torch = _torch()
        n, ns = bits.shape
        logq = torch.zeros(n, dtype=torch.float64, device="cuda")
        cnd = torch.zeros((n, ns), dtype=torch.float64, device="cuda")
        check(self.lib.tns_sample_replay(self._h, int(chi_b), int(n), C.c_uint64(int(seed) & (2**64 - 1)),
                                         C.c_void_p(bits.data_ptr()), C.c_void_p(logq.data_ptr()),
                                         C.c_void_p(cnd.data_ptr())), "tns_sample_replay")
        return logq, cnd

    def certify(self, chi_b: int, bits, logq):
        """(log p [n] device tensor, dict of p/q statistics) at certification rank chi_b (tns_certify)."""
        torch = _torch()
        n = bits.shape[0]
        logp = torch.zeros(n, dtype=torch.float64, device="cuda")
        st = np.zeros(5, dtype=np.float64)
        check(self.lib.tns_certify(self._h, int(chi_b), int(n), C.c_void_p(bits.data_ptr()),
                                   C.c_void_p(logq.data_ptr()), C.c_void_p(logp.data_ptr()), _ptr(st)), "tns_certify")
        return logp, dict(mean_ratio=st[0], mean_ratio_se=st[1], kld=st[2], n_finite=int(st[3]), log_norm=st[4])

    def amplitude(self, chi_b: int, bits):
        torch = _torch()
        n = bits.shape[0]
        la = torch.zeros(n, dtype=torch.float64, device="cuda")
        ph = torch.zeros(n, dtype=torch.float64, device="cuda")
        check(self.lib.tns_amplitude(self._h, int(chi_b), int(n), C.c_void_p(bits.data_ptr()),
                                     C.c_void_p(la.data_ptr()), C.c_void_p(ph.data_ptr())), "tns_amplitude")
        return la, ph


class MADE:
    """Learned autoregressive proposal (tns_made_* in include/tns.h), on the current GPU."""

    def __init__(self, n_sites: int, hidden: int, params, stream=None):
        self.lib = load()
        self.n, self.h = int(n_sites), int(hidden)
        p = np.ascontiguousarray(np.asarray(params, dtype=np.float32).reshape(-1))
        if p.size != self.n_params(self.n, self.h):
            raise ValueError(f"expected {self.n_params(self.n, self.h)} parameters, got {p.size}")
        self._h = C.c_void_p()
        check(self.lib.tns_made_create(self.n, self.h, _ptr(p), _stream_handle(stream), C.byref(self._h)),
              "tns_made_create")

    @staticmethod
    def n_params(n: int, h: int) -> int:
        return 2 * h * n + 2 * h * h + 3 * h + n

    def close(self):
        if self._h:
            self.lib.tns_made_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self) -> np.ndarray:
        out = np.zeros(self.n_params(self.n, self.h), dtype=np.float32)
        check(self.lib.tns_made_params(self._h, _ptr(out)), "tns_made_params")
        return out

    def train(self, bits, batch: int, epochs: int, lr: float = 1e-3, orders=None) -> np.ndarray:
        """Adam on the mean NLL of the rows of bits (torch uint8 CUDA [n, n_sites]); per-epoch losses."""
        n = int(bits.shape[0])
        losses = np.zeros(max(epochs, 1), dtype=np.float64)
        od = None
        if orders is not None:
            od = np.ascontiguousarray(np.asarray(orders, dtype=np.int32).reshape(epochs, n))
        check(self.lib.tns_made_train(self._h, C.c_void_p(bits.data_ptr()), n, int(batch), int(epochs),
                                      _ptr(od) if od is not None else None, float(lr), _ptr(losses)),
              "tns_made_train")
        return losses[:epochs]

    def grad(self, bits):
        g = np.zeros(self.n_params(self.n, self.h), dtype=np.float32)
        loss = C.c_double()
        check(self.lib.tns_made_grad(self._h, C.c_void_p(bits.data_ptr()), int(bits.shape[0]), _ptr(g),
                                     C.byref(loss)), "tns_made_grad")
        return loss.value, g

    def log_prob(self, bits):
        torch = _torch()
        out = torch.zeros(int(bits.shape[0]), dtype=torch.float64, device="cuda")
        check(self.lib.tns_made_logprob(self._h, C.c_void_p(bits.data_ptr()), int(bits.shape[0]),
                                        C.c_void_p(out.data_ptr())), "tns_made_logprob")
        return out

    def sample(self, n: int, seed: int):
        torch = _torch()
        bits = torch.zeros((n, self.n), dtype=torch.uint8, device="cuda")
        logg = torch.zeros(n, dtype=torch.float64, device="cuda")
        check(self.lib.tns_made_sample(self._h, int(n), C.c_uint64(int(seed) & (2**64 - 1)),
                                       C.c_void_p(bits.data_ptr()), C.c_void_p(logg.data_ptr())), "tns_made_sample")
        return bits, logg


def mh_independent(logp_prop, logg_prop, logp0, logg0, seed: int, stream=None):
    """Independent MH chains over precomputed proposals (torch float64 CUDA tensors
    [C, T], [C, T], [C], [C]); returns (state int32 [C, T], accepted int64 [C])."""
    torch = _torch()
    Cn, T = logp_prop.shape
    tensors = [t.contiguous() for t in (logp_prop, logg_prop, logp0, logg0)]
    state = torch.empty((Cn, T), dtype=torch.int32, device="cuda")
    acc = torch.empty(Cn, dtype=torch.int64, device="cuda")
    check(load().tns_mh_independent(int(Cn), int(T), *[C.c_void_p(t.data_ptr()) for t in tensors],
                                    C.c_uint64(int(seed) & (2**64 - 1)), C.c_void_p(state.data_ptr()),
                                    C.c_void_p(acc.data_ptr()), _stream_handle(stream)), "tns_mh_independent")
    return state, acc
