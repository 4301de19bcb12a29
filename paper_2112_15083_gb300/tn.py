"""Thin Python binding of libtn (include/tn.h): argument marshalling only.

Every computation runs inside libtn's CUDA kernels.  PyTorch is used for device
buffers and the current CUDA stream.  The names mirror the C entry points without
the ``tn_`` prefix.  If the shared library is missing this module raises at import
of ``lib()``; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libtn.so")

TN_OK, TN_EINVAL, TN_ENOMEM, TN_ETIMEOUT, TN_EDEVICE, TN_EUNSUPPORTED = 0, -1, -2, -3, -4, -5
PREC_C64, PREC_BF16X2, PREC_FP16X2 = 0, 1, 2
DEVICE_BUFFERS = 1

EXPORTED = [
    "tn_plan_opts_default", "tn_circuit_load", "tn_circuit_destroy", "tn_plan", "tn_plan_destroy",
    "tn_plan_get_info", "tn_plan_sliced_edges", "tn_partial_norms", "tn_slice_cut", "tn_select",
    "tn_contract", "tn_xeb", "tn_spoof", "tn_sample", "tn_rejection_sample", "tn_draw_batches", "tn_strerror", "tn_last_error",
    "tn_plan_host", "tn_sliced_vertex_select", "tn_sample_step", "tn_trace_enable", "tn_trace_read",
    "tn_slice_cut_noalloc", "tn_plan_estimate", "tn_plan_sync", "tn_server_opts_default", "tn_server_create",
    "tn_server_submit", "tn_server_query", "tn_server_wait", "tn_server_get_stats", "tn_server_destroy",
    "tn_plan_test_stall", "tn_job_create", "tn_job_run", "tn_job_get_info", "tn_job_amplitudes", "tn_job_finish", "tn_job_destroy",
]

REQ_STATUS = {0: "queued", 1: "planning", 2: "planned", 3: "active", 4: "done", 5: "failed", 6: "rejected"}


class ServerOpts(ctypes.Structure):
    _fields_ = [
        ("hbm_budget_bytes", ctypes.c_double), ("max_active", ctypes.c_int32), ("planner_threads", ctypes.c_int32),
        ("log2_batches", ctypes.c_int32), ("max_log2_batches", ctypes.c_int32), ("order_trials", ctypes.c_int32),
        ("max_request_seconds", ctypes.c_double),
        ("assumed_flops", ctypes.c_double), ("assumed_flops_c64", ctypes.c_double), ("device", ctypes.c_int32),
    ]


class RequestInfo(ctypes.Structure):
    _fields_ = [
        ("status", ctypes.c_int32), ("error", ctypes.c_int32), ("F", ctypes.c_double), ("steps", ctypes.c_int64),
        ("accepted", ctypes.c_int64), ("n_slices", ctypes.c_int64), ("est_bytes", ctypes.c_int64),
        ("flops", ctypes.c_double), ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
        ("t_done", ctypes.c_double),
    ]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_int64) for k in ("submitted", "queued", "planning", "planned", "active", "done",
                                                "failed", "rejected")] + [
        ("bytes_in_use", ctypes.c_double), ("time_s", ctypes.c_double)]


class TnError(RuntimeError):
    def __init__(self, code, where):
        self.code = code
        L = lib()
        msg = L.tn_last_error().decode(errors="replace")
        super().__init__("%s: %s (%d): %s" % (where, L.tn_strerror(code).decode(), code, msg))


class Edge(ctypes.Structure):
    _fields_ = [("qubit", ctypes.c_int32), ("segment", ctypes.c_int32)]


ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class PlanOpts(ctypes.Structure):
    _fields_ = [
        ("precision", ctypes.c_int32),
        ("log2_batches", ctypes.c_int32),
        ("order_seed", ctypes.c_uint64),
        ("order_trials", ctypes.c_int32),
        ("n_auto_sliced", ctypes.c_int32),
        ("max_log2_tensor", ctypes.c_int32),
        ("hbm_budget_bytes", ctypes.c_double),
        ("max_norm_flops", ctypes.c_double),
        ("autotune", ctypes.c_int32),
        ("fuse_root_sum", ctypes.c_int32),
        ("job_groups", ctypes.c_int32),
        ("anneal_iters", ctypes.c_int32),
        ("parallel_search", ctypes.c_int32),
        ("stream", ctypes.c_void_p),
        ("alloc", ALLOC_FN),
        ("free", FREE_FN),
        ("alloc_ctx", ctypes.c_void_p),
    ]


class PlanInfo(ctypes.Structure):
    _fields_ = [
        ("n_qubits", ctypes.c_int32), ("n_open", ctypes.c_int32), ("n_closed", ctypes.c_int32),
        ("log2_batches", ctypes.c_int32), ("n_leaves", ctypes.c_int32), ("n_steps", ctypes.c_int32),
        ("n_sliced", ctypes.c_int32), ("log2_max_tensor", ctypes.c_int32),
        ("flops_per_slice", ctypes.c_double), ("flops_all_slices", ctypes.c_double),
    ]


class StepTrace(ctypes.Structure):
    _fields_ = [
        ("step", ctypes.c_int32), ("launches", ctypes.c_int32), ("ms", ctypes.c_double),
        ("flops_per_launch", ctypes.c_double), ("bytes_per_launch", ctypes.c_double),
        ("nbat", ctypes.c_int32), ("nm", ctypes.c_int32), ("nn", ctypes.c_int32), ("nk", ctypes.c_int32),
        ("nver", ctypes.c_int64), ("kernel", ctypes.c_int32), ("gathers", ctypes.c_int32),
        ("in_place", ctypes.c_int32),
    ]


class JobInfo(ctypes.Structure):
    _fields_ = [
        ("n_slices", ctypes.c_int64), ("F", ctypes.c_double), ("chunk_slices", ctypes.c_int64),
        ("n_chunks", ctypes.c_int64), ("groups", ctypes.c_int64), ("T", ctypes.c_int64),
        ("chunks_done", ctypes.c_int64), ("flops_done", ctypes.c_double), ("flops_chunk", ctypes.c_double),
    ]


class SampleStats(ctypes.Structure):
    _fields_ = [
        ("F", ctypes.c_double), ("eps_hat", ctypes.c_double), ("steps", ctypes.c_int64),
        ("accepted", ctypes.c_int64), ("n_slices", ctypes.c_int64), ("flops", ctypes.c_double),
    ]


_lib = None


def lib():
    """Load libtn.so (built by paper_2112_15083_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtn.so is not built (run paper_2112_15083_gb300.build.build())")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64, u64, dbl = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
        L.tn_plan_opts_default.argtypes = [ctypes.POINTER(PlanOpts)]
        L.tn_plan_opts_default.restype = None
        L.tn_circuit_load.argtypes = [ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(vp)]
        L.tn_circuit_destroy.argtypes = [vp]
        L.tn_circuit_destroy.restype = None
        L.tn_plan.argtypes = [vp, vp, i32, vp, i32, vp, i32, ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
        L.tn_plan_destroy.argtypes = [vp]
        L.tn_plan_destroy.restype = None
        L.tn_plan_get_info.argtypes = [vp, ctypes.POINTER(PlanInfo)]
        L.tn_plan_sliced_edges.argtypes = [vp, vp, i32, ctypes.POINTER(i32)]
        L.tn_partial_norms.argtypes = [vp, dbl, vp, ctypes.POINTER(i32), vp, i64]
        L.tn_slice_cut.argtypes = [vp, i32, dbl, vp, vp, ctypes.POINTER(i32), ctypes.POINTER(dbl)]
        L.tn_select.argtypes = [vp, dbl, vp, i64, ctypes.POINTER(i64), ctypes.POINTER(dbl)]
        L.tn_contract.argtypes = [vp, vp, i64, vp, i64, vp, i32]
        L.tn_xeb.argtypes = [vp, vp, i64, vp, i64, ctypes.POINTER(dbl), vp]
        L.tn_spoof.argtypes = [vp, vp, i64, u64, i64, vp, vp]
        L.tn_sample.argtypes = [vp, dbl, i64, u64, dbl, vp, i32, ctypes.POINTER(SampleStats)]
        L.tn_rejection_sample.argtypes = [vp, i64, i32, dbl, u64, u64, vp, vp, vp]
        L.tn_draw_batches.argtypes = [u64, u64, i64, i32, vp, vp]
        L.tn_plan_host.argtypes = [vp, vp, i32, vp, i32, vp, i32, ctypes.POINTER(PlanOpts),
                                   ctypes.POINTER(PlanInfo), vp, i32, vp, i32]
        L.tn_sliced_vertex_select.argtypes = [vp, vp, i32, i32, vp, ctypes.POINTER(i32)]
        L.tn_sample_step.argtypes = [vp, vp, i64, dbl, u64, u64, dbl, i32, vp, vp, i32]
        L.tn_trace_enable.argtypes = [vp, i32]
        L.tn_trace_read.argtypes = [vp, ctypes.POINTER(StepTrace), i32, ctypes.POINTER(i32)]
        L.tn_plan_estimate.argtypes = [vp, vp, i64, ctypes.POINTER(i64), ctypes.POINTER(dbl), ctypes.POINTER(dbl)]
        L.tn_plan_sync.argtypes = [vp]
        L.tn_server_opts_default.argtypes = [ctypes.POINTER(ServerOpts)]
        L.tn_server_opts_default.restype = None
        L.tn_server_create.argtypes = [ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]
        L.tn_server_submit.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, vp, i32, i32, i32, dbl, i64, u64, dbl,
                                       ctypes.POINTER(i64)]
        L.tn_server_query.argtypes = [vp, i64, ctypes.POINTER(RequestInfo)]
        L.tn_server_wait.argtypes = [vp, i64, dbl, vp, i64, ctypes.POINTER(RequestInfo)]
        L.tn_server_get_stats.argtypes = [vp, ctypes.POINTER(ServerStats)]
        L.tn_server_destroy.argtypes = [vp]
        L.tn_server_destroy.restype = None
        L.tn_slice_cut_noalloc.argtypes = [vp, i32, dbl, vp, vp, ctypes.POINTER(i32), ctypes.POINTER(dbl)]
        L.tn_plan_test_stall.argtypes = [vp, i64]
        L.tn_job_create.argtypes = [vp, dbl, i64, u64, dbl, i64, ctypes.POINTER(vp), ctypes.POINTER(JobInfo)]
        L.tn_job_run.argtypes = [vp, i64, i64]
        L.tn_job_get_info.argtypes = [vp, ctypes.POINTER(JobInfo)]
        L.tn_job_amplitudes.argtypes = [vp, i64, vp]
        L.tn_job_finish.argtypes = [vp, vp, i32, ctypes.POINTER(SampleStats)]
        L.tn_job_destroy.argtypes = [vp]
        L.tn_job_destroy.restype = None
        L.tn_strerror.argtypes = [ctypes.c_int]
        L.tn_strerror.restype = ctypes.c_char_p
        L.tn_last_error.argtypes = []
        L.tn_last_error.restype = ctypes.c_char_p
        for name in EXPORTED:
            if name not in ("tn_plan_opts_default", "tn_circuit_destroy", "tn_plan_destroy",
                            "tn_strerror", "tn_last_error", "tn_server_opts_default", "tn_server_destroy",
                            "tn_job_destroy"):
                getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(rc, where):
    if rc != TN_OK:
        raise TnError(rc, where)


def _np_ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


def _stream_ptr(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ctypes.c_void_p(int(stream))


# ------------------------------------------------------------------ torch allocator

class _TorchAllocator:
    """Device memory for the plan's arenas from PyTorch's caching allocator."""

    def __init__(self, device):
        import torch
        self.torch = torch
        self.device = device
        self.alloc = ALLOC_FN(self._alloc)
        self.free = FREE_FN(self._free)

    def _alloc(self, nbytes, stream, ctx):
        try:
            return self.torch.cuda.caching_allocator_alloc(int(nbytes), self.device, stream or 0)
        except Exception:
            return None

    def _free(self, ptr, nbytes, stream, ctx):
        try:
            self.torch.cuda.caching_allocator_delete(ptr)
        except Exception:
            pass


# ------------------------------------------------------------------ objects

class Circuit:
    def __init__(self, buf: bytes):
        self.h = ctypes.c_void_p()
        _check(lib().tn_circuit_load(buf, len(buf), ctypes.byref(self.h)), "tn_circuit_load")

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.tn_circuit_destroy(self.h)
            self.h = None


def circuit_load(buf: bytes) -> Circuit:
    return Circuit(buf)


class Plan:
    def __init__(self, circuit: Circuit, open_qubits, sliced=None, order=None, precision=PREC_C64,
                 log2_batches=8, order_seed=0, order_trials=64, n_auto_sliced=0,
                 hbm_budget_bytes=0.0, stream=None, use_torch_allocator=True, max_norm_flops=0.0,
                 autotune=None, max_log2_tensor=0, fuse_root_sum=False, job_groups=1, anneal_iters=0,
                 parallel_search=False):
        L = lib()
        o = PlanOpts()
        L.tn_plan_opts_default(ctypes.byref(o))
        o.precision = precision
        o.log2_batches = log2_batches
        o.order_seed = order_seed
        o.order_trials = order_trials
        o.n_auto_sliced = n_auto_sliced
        o.max_log2_tensor = max_log2_tensor
        if hbm_budget_bytes:
            o.hbm_budget_bytes = hbm_budget_bytes
        if max_norm_flops:
            o.max_norm_flops = max_norm_flops
        if autotune is not None:
            o.autotune = int(autotune)
        o.fuse_root_sum = int(bool(fuse_root_sum))
        o.job_groups = int(job_groups)
        o.anneal_iters = int(anneal_iters)
        o.parallel_search = int(bool(parallel_search))
        o.stream = _stream_ptr(stream)
        self._alloc = None
        if use_torch_allocator:
            import torch
            self._alloc = _TorchAllocator(torch.cuda.current_device())
            o.alloc = self._alloc.alloc
            o.free = self._alloc.free
        self.opts = o
        self.stream = o.stream
        openq = np.ascontiguousarray(np.asarray(open_qubits, dtype=np.int32))
        self.open_qubits = [int(x) for x in openq]
        if sliced is not None:
            arr = (Edge * max(1, len(sliced)))(*[Edge(int(q), int(s)) for (q, s) in sliced])
            sl_ptr, n_sl = ctypes.cast(arr, ctypes.c_void_p), len(sliced)
        else:
            sl_ptr, n_sl = None, 0
        if order is not None:
            ordarr = np.ascontiguousarray(np.asarray(order, dtype=np.int32).reshape(-1))
            ord_ptr, n_ord = _np_ptr(ordarr), ordarr.size // 2
        else:
            ord_ptr, n_ord = None, 0
        self.h = ctypes.c_void_p()
        self._circuit = circuit
        rc = L.tn_plan(circuit.h, ord_ptr, n_ord, sl_ptr, n_sl, _np_ptr(openq), openq.size,
                       ctypes.byref(o), ctypes.byref(self.h))
        _check(rc, "tn_plan")

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.tn_plan_destroy(self.h)
            self.h = None

    # ---- queries
    def info(self) -> dict:
        inf = PlanInfo()
        _check(lib().tn_plan_get_info(self.h, ctypes.byref(inf)), "tn_plan_get_info")
        return {k: getattr(inf, k) for k, _ in PlanInfo._fields_}

    def sliced_edges(self) -> list:
        n = ctypes.c_int32()
        _check(lib().tn_plan_sliced_edges(self.h, None, 0, ctypes.byref(n)), "tn_plan_sliced_edges")
        arr = (Edge * max(1, n.value))()
        _check(lib().tn_plan_sliced_edges(self.h, ctypes.cast(arr, ctypes.c_void_p), n.value, ctypes.byref(n)),
               "tn_plan_sliced_edges")
        return [(arr[i].qubit, arr[i].segment) for i in range(n.value)]

    # ---- selection
    def partial_norms(self, f: float):
        import math
        k0 = int(math.ceil(3.0 - math.log2(f)))
        S = np.zeros(max(1, k0), dtype=np.int32)
        R = np.zeros(1 << max(0, min(k0, 20)), dtype=np.float64)
        k = ctypes.c_int32()
        _check(lib().tn_partial_norms(self.h, f, _np_ptr(S), ctypes.byref(k), _np_ptr(R), R.size),
               "tn_partial_norms")
        return S[: k.value].copy(), R[: 1 << k.value].copy()

    def select(self, f: float):
        n = ctypes.c_int64()
        F = ctypes.c_double()
        _check(lib().tn_select(self.h, f, None, 0, ctypes.byref(n), ctypes.byref(F)), "tn_select")
        out = np.zeros(max(1, n.value), dtype=np.uint64)
        _check(lib().tn_select(self.h, f, _np_ptr(out), out.size, ctypes.byref(n), ctypes.byref(F)), "tn_select")
        return out[: n.value], F.value

    # ---- contraction
    def contract(self, slices, closed_bits, out=None):
        """Host path: numpy in, complex128 numpy (n_batches, 2^n_open) out.
        Device path: pass torch CUDA tensors (closed_bits int64/uint64, out complex128)."""
        sl = np.ascontiguousarray(np.asarray(slices, dtype=np.uint64))
        L = lib()
        na = 1 << len(self.open_qubits)
        try:
            import torch
            is_dev = isinstance(closed_bits, torch.Tensor) and closed_bits.is_cuda
        except ImportError:
            is_dev = False
        if is_dev:
            nb = closed_bits.numel()
            if out is None:
                out = torch.empty((nb, na), dtype=torch.complex128, device=closed_bits.device)
            rc = L.tn_contract(self.h, _np_ptr(sl), sl.size, ctypes.c_void_p(closed_bits.data_ptr()), nb,
                               ctypes.c_void_p(out.data_ptr()), DEVICE_BUFFERS)
            _check(rc, "tn_contract")
            return out
        cb = np.ascontiguousarray(np.asarray(closed_bits, dtype=np.uint64).reshape(-1))
        nb = max(1, cb.size)
        if cb.size == 0:
            cb = np.zeros(1, dtype=np.uint64)
        res = np.zeros((nb, na), dtype=np.complex128) if out is None else out
        rc = L.tn_contract(self.h, _np_ptr(sl), sl.size, _np_ptr(cb), nb, _np_ptr(res), 0)
        _check(rc, "tn_contract")
        return res

    def xeb(self, slices, bitstrings, return_amplitudes=False):
        """Linear XEB (Eq. 1) of the given bitstrings from their amplitudes summed over the
        slice set; with return_amplitudes, also those amplitudes (complex128 numpy)."""
        sl = np.ascontiguousarray(np.asarray(slices, dtype=np.uint64))
        bs = np.ascontiguousarray(np.asarray(bitstrings, dtype=np.uint64).reshape(-1))
        amps = np.zeros(bs.size, dtype=np.complex128) if return_amplitudes else None
        x = ctypes.c_double()
        rc = lib().tn_xeb(self.h, _np_ptr(sl), sl.size, _np_ptr(bs), bs.size, ctypes.byref(x),
                          _np_ptr(amps) if amps is not None else None)
        _check(rc, "tn_xeb")
        return (x.value, amps) if return_amplitudes else x.value

    def spoof(self, slices, closed_pattern: int, N: int, return_probs=False):
        """XEB spoofing: the N strings of the batch closed_pattern with the largest |a|^2
        over the slice set, in ascending in-batch index order (uint64 numpy); with
        return_probs, also their |a|^2."""
        sl = np.ascontiguousarray(np.asarray(slices, dtype=np.uint64))
        bits = np.zeros(N, dtype=np.uint64)
        pr = np.zeros(N, dtype=np.float64) if return_probs else None
        rc = lib().tn_spoof(self.h, _np_ptr(sl), sl.size, int(closed_pattern), int(N), _np_ptr(bits),
                            _np_ptr(pr) if pr is not None else None)
        _check(rc, "tn_spoof")
        return (bits, pr) if return_probs else bits

    def sample_step(self, slices, F: float, seed: int, t0: int, alpha: float = 2.0, reuse_stem: bool = False,
                    accept=None, bits=None):
        """One batch group on the device.  accept / bits: torch CUDA tensors (uint8, int64)
        for the asynchronous device path, or None for host numpy outputs (synchronous)."""
        sl = np.ascontiguousarray(np.asarray(slices, dtype=np.uint64))
        L = lib()
        if accept is not None:
            rc = L.tn_sample_step(self.h, _np_ptr(sl), sl.size, F, seed, t0, alpha, int(reuse_stem),
                                  ctypes.c_void_p(accept.data_ptr()), ctypes.c_void_p(bits.data_ptr()),
                                  DEVICE_BUFFERS)
            _check(rc, "tn_sample_step")
            return accept, bits
        T = 1 << self.info()["log2_batches"]
        acc = np.zeros(T, dtype=np.uint8)
        b = np.zeros(T, dtype=np.uint64)
        rc = L.tn_sample_step(self.h, _np_ptr(sl), sl.size, F, seed, t0, alpha, int(reuse_stem), _np_ptr(acc),
                              _np_ptr(b), 0)
        _check(rc, "tn_sample_step")
        return acc, b

    def estimate(self, slices):
        """Host-only (device bytes, FLOPs of the first batch group, FLOPs of later groups)."""
        sl = np.ascontiguousarray(np.asarray(slices, dtype=np.uint64))
        b = ctypes.c_int64()
        f1 = ctypes.c_double()
        f2 = ctypes.c_double()
        _check(lib().tn_plan_estimate(self.h, _np_ptr(sl), sl.size, ctypes.byref(b), ctypes.byref(f1), ctypes.byref(f2)),
               "tn_plan_estimate")
        return b.value, f1.value, f2.value

    def trace(self, on: bool = True):
        _check(lib().tn_trace_enable(self.h, int(on)), "tn_trace_enable")

    def trace_read(self) -> list:
        n = ctypes.c_int32()
        _check(lib().tn_trace_read(self.h, None, 0, ctypes.byref(n)), "tn_trace_read")
        arr = (StepTrace * max(1, n.value))()
        _check(lib().tn_trace_read(self.h, arr, n.value, ctypes.byref(n)), "tn_trace_read")
        return [{k: getattr(arr[i], k) for k, _ in StepTrace._fields_} for i in range(n.value)]

    def test_stall(self, cycles: int):
        """Tests only: make the tensor-core launches' first wait run out (tn_plan_test_stall)."""
        _check(lib().tn_plan_test_stall(self.h, int(cycles)), "tn_plan_test_stall")

    def job(self, f_target: float, N: int, seed: int, alpha: float = 2.0, max_chunk_slices: int = 0) -> "Job":
        return Job(self, f_target, N, seed, alpha, max_chunk_slices)

    def sample(self, f_target: float, N: int, seed: int, alpha: float = 2.0):
        out = np.zeros(max(1, N), dtype=np.uint64)
        st = SampleStats()
        rc = lib().tn_sample(self.h, f_target, N, seed, alpha, _np_ptr(out), 0, ctypes.byref(st))
        _check(rc, "tn_sample")
        return out[:N], {k: getattr(st, k) for k, _ in SampleStats._fields_}


JOB_PARTIAL = 2


class Job:
    """A chunked sampling job (tn_job_*): the retained slices in chunks, every chunk
    contracted for all of the job's batch groups and summed in FP64, then one accept /
    pick pass over all batches."""

    def __init__(self, plan: "Plan", f_target: float, N: int, seed: int, alpha: float = 2.0,
                 max_chunk_slices: int = 0):
        self.h = ctypes.c_void_p()
        self._plan = plan
        self.N = int(N)
        inf = JobInfo()
        _check(lib().tn_job_create(plan.h, f_target, int(N), int(seed), alpha, int(max_chunk_slices),
                                   ctypes.byref(self.h), ctypes.byref(inf)), "tn_job_create")

    def __del__(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.tn_job_destroy(self.h)
            self.h = None

    def info(self) -> dict:
        inf = JobInfo()
        _check(lib().tn_job_get_info(self.h, ctypes.byref(inf)), "tn_job_get_info")
        return {k: getattr(inf, k) for k, _ in JobInfo._fields_}

    def run(self, first: int = 0, count: int | None = None):
        if count is None:
            count = self.info()["n_chunks"] - first
        _check(lib().tn_job_run(self.h, int(first), int(count)), "tn_job_run")

    def amplitudes(self, g: int) -> np.ndarray:
        T = self.info()["T"]
        out = np.zeros((T, 64), dtype=np.complex128)
        _check(lib().tn_job_amplitudes(self.h, int(g), _np_ptr(out)), "tn_job_amplitudes")
        return out

    def finish(self, partial: bool = False):
        out = np.zeros(self.N, dtype=np.uint64)
        st = SampleStats()
        _check(lib().tn_job_finish(self.h, _np_ptr(out), JOB_PARTIAL if partial else 0, ctypes.byref(st)),
               "tn_job_finish")
        return out, {k: getattr(st, k) for k, _ in SampleStats._fields_}


def plan_host(circuit: Circuit, open_qubits, sliced=None, order=None, log2_batches=8, order_seed=0,
              order_trials=64, n_auto_sliced=0, precision=PREC_C64, max_log2_tensor=0, hbm_budget_bytes=0.0,
              job_groups=1, anneal_iters=0, parallel_search=False):
    """Host-only planning (no GPU): (info dict, steps array (n_steps, 7), sliced edges).
    Step row: batch, m, n, k bits, log2 versions of C, A, B."""
    L = lib()
    o = PlanOpts()
    L.tn_plan_opts_default(ctypes.byref(o))
    o.precision = precision
    o.log2_batches = log2_batches
    o.order_seed = order_seed
    o.order_trials = order_trials
    o.n_auto_sliced = n_auto_sliced
    o.max_log2_tensor = max_log2_tensor
    if hbm_budget_bytes:
        o.hbm_budget_bytes = hbm_budget_bytes
    o.job_groups = int(job_groups)
    o.anneal_iters = int(anneal_iters)
    o.parallel_search = int(bool(parallel_search))
    openq = np.ascontiguousarray(np.asarray(open_qubits, dtype=np.int32))
    if sliced is not None:
        arr = (Edge * max(1, len(sliced)))(*[Edge(int(q), int(s)) for (q, s) in sliced])
        sl_ptr, n_sl = ctypes.cast(arr, ctypes.c_void_p), len(sliced)
    else:
        sl_ptr, n_sl = None, 0
    if order is not None:
        ordarr = np.ascontiguousarray(np.asarray(order, dtype=np.int32).reshape(-1))
        ord_ptr, n_ord = _np_ptr(ordarr), ordarr.size // 2
    else:
        ord_ptr, n_ord = None, 0
    inf = PlanInfo()
    steps = np.zeros((4096, 7), dtype=np.int32)
    sl_out = (Edge * 64)()
    rc = L.tn_plan_host(circuit.h, ord_ptr, n_ord, sl_ptr, n_sl, _np_ptr(openq), openq.size, ctypes.byref(o),
                        ctypes.byref(inf), _np_ptr(steps), 4096, ctypes.cast(sl_out, ctypes.c_void_p), 64)
    _check(rc, "tn_plan_host")
    info = {k: getattr(inf, k) for k, _ in PlanInfo._fields_}
    return info, steps[: info["n_steps"]].copy(), [(sl_out[i].qubit, sl_out[i].segment) for i in range(info["n_sliced"])]


def sliced_vertex_select(circuit: Circuit, I, k: int):
    """Alg. 2 on the host: positions into I of the selected S."""
    arr = (Edge * max(1, len(I)))(*[Edge(int(q), int(s)) for (q, s) in I])
    out = np.zeros(max(1, len(I)), dtype=np.int32)
    kk = ctypes.c_int32()
    _check(lib().tn_sliced_vertex_select(circuit.h, ctypes.cast(arr, ctypes.c_void_p), len(I), k, _np_ptr(out),
                                         ctypes.byref(kk)), "tn_sliced_vertex_select")
    return out[: kk.value].copy()


def plan(circuit, open_qubits, **kw) -> Plan:
    return Plan(circuit, open_qubits, **kw)


def slice_cut(R, f: float, stream=None):
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float64))
    k = int(np.log2(R.size))
    assert R.size == 1 << k
    X = np.zeros(R.size, dtype=np.int32)
    n = ctypes.c_int32()
    F = ctypes.c_double()
    _check(lib().tn_slice_cut(_np_ptr(R), k, f, _stream_ptr(stream), _np_ptr(X), ctypes.byref(n), ctypes.byref(F)),
           "tn_slice_cut")
    return X[: n.value].copy(), F.value


def slice_cut_noalloc(R, f: float, stream=None):
    """tn_slice_cut_noalloc: the slice cut with its device scratch in libtn's static array
    (no device allocation; k <= 12)."""
    R = np.ascontiguousarray(np.asarray(R, dtype=np.float64))
    k = int(np.log2(R.size))
    assert R.size == 1 << k
    X = np.zeros(R.size, dtype=np.int32)
    n = ctypes.c_int32()
    F = ctypes.c_double()
    _check(lib().tn_slice_cut_noalloc(_np_ptr(R), k, f, _stream_ptr(stream), _np_ptr(X), ctypes.byref(n),
                                      ctypes.byref(F)), "tn_slice_cut_noalloc")
    return X[: n.value].copy(), F.value


def rejection_sample(p, b_bits: int, alpha: float, seed: int, t0: int = 0, stream=None):
    """p: torch CUDA float64 tensor (T, 64).  Returns (accept uint8, pick int32) CUDA tensors."""
    import torch
    assert p.is_cuda and p.dtype == torch.float64 and p.shape[-1] == 64
    p = p.contiguous()
    T = p.shape[0]
    acc = torch.empty(T, dtype=torch.uint8, device=p.device)
    pick = torch.empty(T, dtype=torch.int32, device=p.device)
    _check(lib().tn_rejection_sample(ctypes.c_void_p(p.data_ptr()), T, b_bits, alpha, seed, t0,
                                     ctypes.c_void_p(acc.data_ptr()), ctypes.c_void_p(pick.data_ptr()),
                                     _stream_ptr(stream)), "tn_rejection_sample")
    return acc, pick


def draw_batches(seed: int, t0: int, T: int, b_bits: int, device="cuda", stream=None):
    import torch
    j = torch.empty(T, dtype=torch.int64, device=device)
    _check(lib().tn_draw_batches(seed, t0, T, b_bits, ctypes.c_void_p(j.data_ptr()), _stream_ptr(stream)),
           "tn_draw_batches")
    return j


class Server:
    """Continuous-batching sampling server (tn_server_*)."""

    def __init__(self, hbm_budget_bytes=150e9, max_active=8, planner_threads=2, log2_batches=8, order_trials=64,
                 max_request_seconds=600.0, assumed_flops=3e14, assumed_flops_c64=3e13, device=0,
                 max_log2_batches=14):
        L = lib()
        o = ServerOpts()
        L.tn_server_opts_default(ctypes.byref(o))
        o.hbm_budget_bytes = hbm_budget_bytes
        o.max_active = max_active
        o.planner_threads = planner_threads
        o.log2_batches = log2_batches
        o.max_log2_batches = max_log2_batches
        o.order_trials = order_trials
        o.max_request_seconds = max_request_seconds
        o.assumed_flops = assumed_flops
        o.assumed_flops_c64 = assumed_flops_c64
        o.device = device
        self.h = ctypes.c_void_p()
        _check(L.tn_server_create(ctypes.byref(o), ctypes.byref(self.h)), "tn_server_create")

    def submit(self, circuit_bytes: bytes, open_qubits, N: int, f: float = 1.0, seed: int = 0, alpha: float = 2.0,
               precision=PREC_C64, n_sliced=0) -> int:
        openq = np.ascontiguousarray(np.asarray(open_qubits, dtype=np.int32))
        rid = ctypes.c_int64()
        _check(lib().tn_server_submit(self.h, circuit_bytes, len(circuit_bytes), _np_ptr(openq), openq.size, precision,
                                      n_sliced, f, N, seed, alpha, ctypes.byref(rid)), "tn_server_submit")
        return rid.value

    @staticmethod
    def _info(inf):
        d = {k: getattr(inf, k) for k, _ in RequestInfo._fields_}
        d["status"] = REQ_STATUS.get(d["status"], d["status"])
        return d

    def query(self, rid: int) -> dict:
        inf = RequestInfo()
        _check(lib().tn_server_query(self.h, rid, ctypes.byref(inf)), "tn_server_query")
        return self._info(inf)

    def wait(self, rid: int, N: int, timeout: float = 0.0):
        """(bitstrings or None, info dict); bitstrings only when the request succeeded."""
        out = np.zeros(max(1, N), dtype=np.uint64)
        inf = RequestInfo()
        rc = lib().tn_server_wait(self.h, rid, timeout, _np_ptr(out), N, ctypes.byref(inf))
        info = self._info(inf)
        info["rc"] = rc
        return (out[:N] if rc == TN_OK else None), info

    def stats(self) -> dict:
        st = ServerStats()
        _check(lib().tn_server_get_stats(self.h, ctypes.byref(st)), "tn_server_get_stats")
        return {k: getattr(st, k) for k, _ in ServerStats._fields_}

    def close(self):
        if getattr(self, "h", None) and self.h.value and _lib is not None:
            _lib.tn_server_destroy(self.h)
            self.h = None

    def __del__(self):
        self.close()
