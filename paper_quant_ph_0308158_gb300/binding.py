"""Thin Python binding of libqsim.so (include/qsim.h): argument marshalling only.

Every step of the simulation runs in the library's CUDA kernels.  There is
no CPU fallback: if the library is missing or cannot load, constructing a
``Simulator`` raises ``QsimError``.

    sim = Simulator(M=16, dtype=np.complex128)      # state + scratch from torch
    sim.load_state(k1)                              # numpy, 2^M amplitudes
    sim.apply(steps)                                # workloads.STEP_DTYPE array
    k2 = sim.read_state()
    p, norm = sim.probabilities(with_norm=True)     # FP64
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from .workloads import STEP_DTYPE

QSIM_OK = 0
QSIM_EINVAL = -1
QSIM_ENOMEM = -2
QSIM_ECUDA = -3
QSIM_ETIMEOUT = -4
QSIM_EBUSY = -5
QSIM_ENOTFOUND = -6

QSIM_C64 = 0
QSIM_C128 = 1

STRATEGY = {"auto": 0, "sweep": 1, "tile": 2, "gather": 3, "inplace": 4}
PASS_KIND = {1: "sweep", 2: "tile", 3: "gather"}
KERNEL = {1: "sweep_kernel", 2: "tile_kernel", 3: "gather_affine_kernel",
          4: "gather_sliced_kernel", 5: "qsim_jit_gather", 6: "probs_kernel",
          7: "gather_coset_kernel", 8: "qsim_jit_closed"}

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "_lib", "libqsim.so")

# every symbol include/qsim.h declares
EXPORTS = (
    "qsim_create", "qsim_create_with_buffers", "qsim_destroy", "qsim_load_state",
    "qsim_read_state", "qsim_state_device", "qsim_apply_circuit",
    "qsim_apply_circuit_probabilities", "qsim_apply_circuit_probabilities_async", "qsim_autotune",
    "qsim_set_strategy",
    "qsim_set_canonicalize", "qsim_set_profiling", "qsim_get_pass_times", "qsim_set_jit",
    "qsim_set_wait_test", "qsim_set_coset", "qsim_gather_rows", "qsim_plan_circuit_ex",
    "qsim_batch_create_ex", "qsim_apply_circuit_product",
    "qsim_jit_precompile",
    "qsim_get_plan_stats", "qsim_synchronize", "qsim_probabilities",
    "qsim_probabilities_device", "qsim_plan_circuit", "qsim_last_error", "qsim_version",
    "qsim_probabilities_noalloc", "qsim_load_product_state", "qsim_row_array",
    "qsim_load_state_async", "qsim_probabilities_async", "qsim_batch_create", "qsim_batch_destroy",
    "qsim_batch_load_state", "qsim_batch_read_state", "qsim_batch_state_device", "qsim_batch_run",
    "qsim_batch_run_plain", "qsim_batch_synchronize", "qsim_batch_info", "qsim_server_create",
    "qsim_server_submit", "qsim_server_poll", "qsim_server_release", "qsim_server_wait_all",
    "qsim_server_get_stats", "qsim_server_destroy", "qsim_server_drain", "qsim_server_set_backfill",
    "qsim_server_set_paused", "qsim_server_set_tracing", "qsim_server_get_trace",
    "qsim_server_set_copy_streams", "qsim_server_set_upload_chunk", "qsim_server_set_eviction",
)


class QsimError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__("qsim error %d: %s" % (code, msg))
        self.code = code


class PlanStats(ctypes.Structure):
    _fields_ = [("steps_in", ctypes.c_uint64), ("steps_cancelled", ctypes.c_uint64),
                ("passes", ctypes.c_uint64), ("sweep_passes", ctypes.c_uint64),
                ("tile_passes", ctypes.c_uint64), ("gather_passes", ctypes.c_uint64),
                ("algorithmic_bytes", ctypes.c_double), ("full_pass_equiv", ctypes.c_double),
                ("est_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class PlanOptions(ctypes.Structure):
    _fields_ = [("strategy", ctypes.c_int), ("tile_bits", ctypes.c_int), ("low_bits", ctypes.c_int),
                ("scratch_available", ctypes.c_int), ("jit", ctypes.c_int), ("coset", ctypes.c_int),
                ("coset_run_bits", ctypes.c_int), ("canonicalize", ctypes.c_int),
                ("closed_known", ctypes.c_int), ("closed_delta", ctypes.c_uint64)]


class BatchStats(ctypes.Structure):
    _fields_ = [("circuits", ctypes.c_uint64), ("levels", ctypes.c_uint64),
                ("items", ctypes.c_uint64), ("passes", ctypes.c_uint64),
                ("amplitude_steps", ctypes.c_uint64), ("algorithmic_bytes", ctypes.c_double),
                ("arena_bytes", ctypes.c_uint64), ("stream", ctypes.c_void_p),
                ("coset_passes", ctypes.c_uint64), ("affine_passes", ctypes.c_uint64),
                ("sliced_passes", ctypes.c_uint64), ("sweep_passes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("admitted", ctypes.c_uint64),
                ("completed", ctypes.c_uint64), ("rounds", ctypes.c_uint64),
                ("launches", ctypes.c_uint64), ("active", ctypes.c_uint64),
                ("waiting", ctypes.c_uint64), ("budget_bytes", ctypes.c_uint64),
                ("in_use_bytes", ctypes.c_uint64), ("peak_in_use_bytes", ctypes.c_uint64),
                ("host_in_use_bytes", ctypes.c_uint64), ("amplitude_steps", ctypes.c_double),
                ("backfilled", ctypes.c_uint64), ("h2d_bytes", ctypes.c_uint64),
                ("d2h_bytes", ctypes.c_uint64), ("h2d_busy_ms", ctypes.c_double),
                ("d2h_busy_ms", ctypes.c_double), ("compute_busy_ms", ctypes.c_double),
                ("issue_ms", ctypes.c_double), ("issue_ms_max", ctypes.c_double),
                ("evicted", ctypes.c_uint64), ("swapped_in", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class BatchOptions(ctypes.Structure):
    _fields_ = [("coset_min_qubits", ctypes.c_uint32)]


class TuneResult(ctypes.Structure):
    _fields_ = [("strategy", ctypes.c_int), ("tile_bits", ctypes.c_int), ("low_bits", ctypes.c_int),
                ("jit", ctypes.c_int), ("ms", ctypes.c_double), ("passes", ctypes.c_uint64)]


class ServerTraceRecord(ctypes.Structure):
    _fields_ = [("id", ctypes.c_uint64), ("M", ctypes.c_uint32), ("passes", ctypes.c_uint32),
                ("L", ctypes.c_uint64), ("submit_ms", ctypes.c_double), ("admit_ms", ctypes.c_double),
                ("upload_start_ms", ctypes.c_double), ("upload_end_ms", ctypes.c_double),
                ("compute_start_ms", ctypes.c_double), ("compute_end_ms", ctypes.c_double),
                ("download_start_ms", ctypes.c_double), ("download_end_ms", ctypes.c_double),
                ("done_ms", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def lib_path() -> str:
    return _LIB_PATH


def load() -> ctypes.CDLL:
    """Load libqsim.so (built by ``paper_quant_ph_0308158_gb300.build``)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise QsimError(QSIM_EINVAL, "libqsim.so is not built (%s); run "
                            "paper_quant_ph_0308158_gb300.build.build()" % _LIB_PATH)
        L = ctypes.CDLL(_LIB_PATH)
        p, i, u32, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_uint32, ctypes.c_size_t
        pp = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "qsim_create": ([u32, i, pp], i),
            "qsim_create_with_buffers": ([u32, i, p, p, p, pp], i),
            "qsim_destroy": ([p], None),
            "qsim_load_state": ([p, p, sz], i),
            "qsim_read_state": ([p, p, sz], i),
            "qsim_state_device": ([p], p),
            "qsim_apply_circuit": ([p, p, sz], i),
            "qsim_apply_circuit_probabilities": ([p, p, sz, p], i),
            "qsim_apply_circuit_probabilities_async": ([p, p, sz, p, sz], i),
            "qsim_autotune": ([p, p, sz, i, p, sz, ctypes.POINTER(sz)], i),
            "qsim_set_strategy": ([p, i, i, i], i),
            "qsim_set_canonicalize": ([p, i], i),
            "qsim_set_profiling": ([p, i], i),
            "qsim_set_jit": ([p, i], i),
            "qsim_set_wait_test": ([p, u32], i),
            "qsim_set_coset": ([p, i, i, i], i),
            "qsim_apply_circuit_product": ([p, p, p, sz, p], i),
            "qsim_gather_rows": ([p, p, p, u32, i, p, i, p], i),
            "qsim_plan_circuit_ex": ([u32, i, p, sz, ctypes.POINTER(PlanOptions), ctypes.POINTER(PlanStats),
                                      p, p, p, p, sz], i),
            "qsim_jit_precompile": ([u32, i, p, sz, i, ctypes.POINTER(ctypes.c_double)], i),
            "qsim_get_pass_times": ([p, p, p, p, sz, ctypes.POINTER(sz)], i),
            "qsim_get_plan_stats": ([p, ctypes.POINTER(PlanStats)], i),
            "qsim_synchronize": ([p], i),
            "qsim_probabilities": ([p, p, sz, ctypes.POINTER(ctypes.c_double)], i),
            "qsim_probabilities_device": ([p, p, ctypes.POINTER(ctypes.c_double)], i),
            "qsim_plan_circuit": ([u32, i, p, sz, i, i, i, i, ctypes.POINTER(PlanStats), p, p, p, sz], i),
            "qsim_probabilities_noalloc": ([p, u32, i, p, p, p], i),
            "qsim_load_product_state": ([p, p], i),
            "qsim_row_array": ([p, p, sz, p], i),
            "qsim_load_state_async": ([p, p, sz], i),
            "qsim_probabilities_async": ([p, p, sz], i),
            "qsim_batch_create": ([sz, p, i, p, p, pp], i),
            "qsim_batch_create_ex": ([sz, p, i, p, p, ctypes.POINTER(BatchOptions), pp], i),
            "qsim_batch_destroy": ([p], None),
            "qsim_batch_load_state": ([p, sz, p, sz], i),
            "qsim_batch_read_state": ([p, sz, p, sz], i),
            "qsim_batch_state_device": ([p, sz], p),
            "qsim_batch_run": ([p], i),
            "qsim_batch_run_plain": ([p], i),
            "qsim_batch_synchronize": ([p], i),
            "qsim_batch_info": ([p, ctypes.POINTER(BatchStats)], i),
            "qsim_server_create": ([sz, sz, i, pp], i),
            "qsim_server_submit": ([p, u32, p, p, sz, ctypes.POINTER(ctypes.c_uint64)], i),
            "qsim_server_poll": ([p, ctypes.c_uint64, ctypes.POINTER(i), ctypes.POINTER(ctypes.c_double),
                                  ctypes.POINTER(ctypes.POINTER(ctypes.c_double))], i),
            "qsim_server_release": ([p, ctypes.c_uint64], i),
            "qsim_server_drain": ([p, p, p, sz, ctypes.POINTER(sz)], i),
            "qsim_server_wait_all": ([p, ctypes.c_double], i),
            "qsim_server_get_stats": ([p, ctypes.POINTER(ServerStats)], i),
            "qsim_server_set_backfill": ([p, ctypes.c_double], i),
            "qsim_server_set_paused": ([p, i], i),
            "qsim_server_set_copy_streams": ([p, i], i),
            "qsim_server_set_upload_chunk": ([p, sz], i),
            "qsim_server_set_eviction": ([p, ctypes.c_double], i),
            "qsim_server_set_tracing": ([p, i], i),
            "qsim_server_get_trace": ([p, p, sz, ctypes.POINTER(sz)], i),
            "qsim_server_destroy": ([p], None),
            "qsim_last_error": ([], ctypes.c_char_p),
            "qsim_version": ([], ctypes.c_char_p),
        }
        for name, (args, res) in sig.items():
            f = getattr(L, name)
            f.argtypes = args
            f.restype = res
        _lib = L
        return L


def _check(rc: int):
    if rc != QSIM_OK:
        msg = load().qsim_last_error()
        raise QsimError(rc, msg.decode() if msg else "")


def dtype_code(dtype) -> int:
    dt = np.dtype(dtype)
    if dt == np.complex64:
        return QSIM_C64
    if dt == np.complex128:
        return QSIM_C128
    raise QsimError(QSIM_EINVAL, "dtype must be complex64 or complex128")


def as_steps(steps) -> np.ndarray:
    s = np.ascontiguousarray(steps)
    if s.dtype != STEP_DTYPE:
        raise QsimError(QSIM_EINVAL, "steps must be a workloads.STEP_DTYPE array")
    return s


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def plan_circuit(M: int, dtype, steps, strategy: str = "auto", tile_bits: int = 0,
                 low_bits: int = 0, scratch: bool = True) -> dict:
    """Host-only planning (no GPU): pass kinds, pass boundaries, applied order."""
    L = load()
    s = as_steps(steps)
    cap = max(len(s), 1)
    order = np.zeros(cap, dtype=np.uint64)
    ends = np.zeros(cap, dtype=np.uint64)
    kinds = np.zeros(cap, dtype=np.uint32)
    st = PlanStats()
    _check(L.qsim_plan_circuit(M, dtype_code(dtype), _ptr(s), len(s), STRATEGY[strategy],
                               tile_bits, low_bits, int(scratch), ctypes.byref(st),
                               _ptr(order), _ptr(ends), _ptr(kinds), cap))
    n_pass = int(st.passes)
    n_ord = int(st.steps_in - st.steps_cancelled)
    return dict(stats=st.as_dict(), order=order[:n_ord].copy(), pass_ends=ends[:n_pass].copy(),
                kinds=[PASS_KIND[int(k)] for k in kinds[:n_pass]])


VARIANT = {1: "sweep", 2: "tile", 3: "affine", 4: "sliced", 5: "compiled", 7: "coset", 8: "closed"}


def plan_circuit_ex(M: int, dtype, steps, strategy: str = "auto", tile_bits: int = 0,
                    low_bits: int = 0, scratch: bool = True, jit: bool = False, coset: bool = True,
                    coset_run_bits: int = 0, canonicalize: bool = True,
                    closed_delta: int | None = None) -> dict:
    """Host-only planning with every switch: per pass its kernel variant and
    the cost model's estimated time (ms)."""
    L = load()
    s = as_steps(steps)
    cap = max(len(s), 1)
    order = np.zeros(cap, dtype=np.uint64)
    ends = np.zeros(cap, dtype=np.uint64)
    var = np.zeros(cap, dtype=np.uint32)
    est = np.zeros(cap, dtype=np.float64)
    st = PlanStats()
    o = PlanOptions(STRATEGY[strategy], tile_bits, low_bits, int(scratch), int(jit), int(coset),
                    coset_run_bits, int(canonicalize), int(closed_delta is not None),
                    int(closed_delta or 0))
    _check(L.qsim_plan_circuit_ex(M, dtype_code(dtype), _ptr(s), len(s), ctypes.byref(o),
                                  ctypes.byref(st), _ptr(order), _ptr(ends), _ptr(var), _ptr(est), cap))
    n_pass = int(st.passes)
    n_ord = int(st.steps_in - st.steps_cancelled)
    return dict(stats=st.as_dict(), order=order[:n_ord].copy(), pass_ends=ends[:n_pass].copy(),
                variants=[VARIANT[int(k)] for k in var[:n_pass]], est_ms=est[:n_pass].copy())


class Simulator:
    """A 2^M-amplitude state on the current CUDA device.

    ``buffers="torch"`` (default) takes the state and scratch buffers from the
    PyTorch caching allocator and runs on torch's current stream;
    ``buffers="library"`` lets libqsim allocate them (cudaMalloc) on its own
    stream.  ``scratch=False`` keeps every pass in place.
    """

    def __init__(self, M: int, dtype=np.complex128, buffers: str = "torch",
                 scratch: bool = True):
        self.M = int(M)
        self.dtype = np.dtype(dtype)
        self.n = 1 << self.M
        self._lib = load()
        self._ctx = ctypes.c_void_p()
        self._tensors = []
        code = dtype_code(self.dtype)
        if buffers == "torch":
            import torch
            tdt = torch.complex64 if code == QSIM_C64 else torch.complex128
            st = torch.empty(self.n, dtype=tdt, device="cuda")
            st.zero_()
            sc = torch.empty(self.n, dtype=tdt, device="cuda") if scratch else None
            self._tensors = [st, sc]
            stream = torch.cuda.current_stream().cuda_stream
            _check(self._lib.qsim_create_with_buffers(
                self.M, code, ctypes.c_void_p(st.data_ptr()),
                ctypes.c_void_p(sc.data_ptr() if sc is not None else 0),
                ctypes.c_void_p(stream), ctypes.byref(self._ctx)))
        elif buffers == "library":
            _check(self._lib.qsim_create(self.M, code, ctypes.byref(self._ctx)))
            if not scratch:
                self.set_strategy("inplace")
        else:
            raise QsimError(QSIM_EINVAL, "buffers must be 'torch' or 'library'")

    # -- lifetime ---------------------------------------------------------------
    def close(self):
        if self._ctx:
            self._lib.qsim_destroy(self._ctx)
            self._ctx = ctypes.c_void_p()
        self._tensors = []

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- state ------------------------------------------------------------------
    def load_state(self, k1: np.ndarray):
        a = np.ascontiguousarray(k1, dtype=self.dtype)
        if a.shape != (self.n,):
            raise QsimError(QSIM_EINVAL, "state must have 2^M amplitudes")
        _check(self._lib.qsim_load_state(self._ctx, _ptr(a), self.n))

    def load_state_async(self, k1: np.ndarray):
        """Queue the copy-in of k1 (keep it alive and unchanged, ideally pinned,
        until synchronize())."""
        if k1.dtype != self.dtype or k1.shape != (self.n,) or not k1.flags.c_contiguous:
            raise QsimError(QSIM_EINVAL, "state must be a contiguous array of 2^M amplitudes")
        _check(self._lib.qsim_load_state_async(self._ctx, _ptr(k1), self.n))

    def probabilities_async(self, out: np.ndarray):
        """Queue probabilities into out (2^M float64, kept alive until synchronize())."""
        if out.dtype != np.float64 or out.shape != (self.n,) or not out.flags.c_contiguous:
            raise QsimError(QSIM_EINVAL, "out must be a contiguous float64 array of 2^M entries")
        _check(self._lib.qsim_probabilities_async(self._ctx, _ptr(out), self.n))

    def load_product_state(self, qubits: np.ndarray):
        """Product state of App. 1 from M qubit pairs: qubits[b] = (q_b(0), q_b(1))
        as a complex (M, 2) array; b = 0 is the paper's a(1)."""
        q = np.ascontiguousarray(qubits, dtype=np.complex128)
        if q.shape != (self.M, 2):
            raise QsimError(QSIM_EINVAL, "qubits must be a complex (M, 2) array")
        _check(self._lib.qsim_load_product_state(self._ctx, _ptr(q)))

    def read_state(self, out: np.ndarray | None = None) -> np.ndarray:
        if out is None:
            out = np.empty(self.n, dtype=self.dtype)
        _check(self._lib.qsim_read_state(self._ctx, _ptr(out), self.n))
        return out

    def state_ptr(self) -> int:
        return int(self._lib.qsim_state_device(self._ctx) or 0)

    def state_tensor(self):
        """The torch tensor that currently holds the state (torch buffers only)."""
        ptr = self.state_ptr()
        for t in self._tensors:
            if t is not None and t.data_ptr() == ptr:
                return t
        raise QsimError(QSIM_EINVAL, "state is not in a torch-owned buffer")

    # -- circuits -----------------------------------------------------------------
    def set_strategy(self, strategy: str = "auto", tile_bits: int = 0, low_bits: int = 0):
        _check(self._lib.qsim_set_strategy(self._ctx, STRATEGY[strategy], tile_bits, low_bits))

    def set_jit(self, enable: bool):
        _check(self._lib.qsim_set_jit(self._ctx, int(bool(enable))))

    def set_coset(self, enable: bool, run_bits: int = 0, stage_kib: int = 0):
        """Affine gathers through coset-blocked tiles (default) or direct reads."""
        _check(self._lib.qsim_set_coset(self._ctx, int(bool(enable)), run_bits, stage_kib))

    def set_wait_test(self, poll_limit: int):
        """Arm the next tile pass to give up its pipeline waits (testing)."""
        _check(self._lib.qsim_set_wait_test(self._ctx, poll_limit))

    def set_canonicalize(self, enable: bool):
        _check(self._lib.qsim_set_canonicalize(self._ctx, int(bool(enable))))

    def apply(self, steps):
        s = as_steps(steps)
        _check(self._lib.qsim_apply_circuit(self._ctx, _ptr(s), len(s)))

    def apply_product(self, qubits: np.ndarray, steps, out_ptr: int = 0):
        """Apply steps to the App. 1 product state of qubits (M x 2 complex),
        the first tile pass computing its inputs (probabilities to out_ptr if
        non-zero)."""
        q = np.ascontiguousarray(qubits, dtype=np.complex128)
        if q.shape != (self.M, 2):
            raise QsimError(QSIM_EINVAL, "qubits must be a complex (M, 2) array")
        s = as_steps(steps)
        _check(self._lib.qsim_apply_circuit_product(self._ctx, _ptr(q), _ptr(s), len(s),
                                                    ctypes.c_void_p(out_ptr or None)))

    def apply_probabilities(self, steps, out_ptr: int):
        """apply(steps), then FP64 probabilities into device memory at out_ptr
        (2^M doubles), written by the last pass where its kernel can."""
        s = as_steps(steps)
        _check(self._lib.qsim_apply_circuit_probabilities(self._ctx, _ptr(s), len(s),
                                                          ctypes.c_void_p(out_ptr)))

    def apply_probabilities_async(self, steps, out: np.ndarray):
        """apply(steps), then FP64 probabilities into out (2^M float64, pinned
        for speed), queued: valid after synchronize()."""
        if out.dtype != np.float64 or out.shape != (self.n,) or not out.flags.c_contiguous:
            raise QsimError(QSIM_EINVAL, "out must be a contiguous float64 array of 2^M entries")
        s = as_steps(steps)
        _check(self._lib.qsim_apply_circuit_probabilities_async(self._ctx, _ptr(s), len(s), _ptr(out),
                                                                self.n))

    def autotune(self, steps, reps: int = 2) -> list:
        """Time candidate plans on this context's state (left unchanged) and keep
        the fastest; returns the candidates fastest first as dicts."""
        s = as_steps(steps)
        buf = (TuneResult * 64)()
        n = ctypes.c_size_t(0)
        _check(self._lib.qsim_autotune(self._ctx, _ptr(s), len(s), int(reps), buf, 64,
                                       ctypes.byref(n)))
        names = {v: k for k, v in STRATEGY.items()}
        return [{"strategy": names[r.strategy], "tile_bits": r.tile_bits, "low_bits": r.low_bits,
                 "jit": bool(r.jit), "ms": r.ms, "passes": int(r.passes)}
                for r in buf[:min(n.value, 64)]]

    def set_profiling(self, enable: bool):
        _check(self._lib.qsim_set_profiling(self._ctx, int(bool(enable))))

    def pass_times(self):
        """[(kernel, ms, algorithmic bytes)] for every pass recorded since the
        last call (profiling must be on); clears the record."""
        n = ctypes.c_size_t(0)
        _check(self._lib.qsim_get_pass_times(self._ctx, None, None, None, 0, ctypes.byref(n)))
        k = int(n.value)
        ms = np.zeros(max(k, 1), np.float64)
        kinds = np.zeros(max(k, 1), np.uint32)
        by = np.zeros(max(k, 1), np.float64)
        _check(self._lib.qsim_get_pass_times(self._ctx, _ptr(ms), _ptr(kinds), _ptr(by), k,
                                             ctypes.byref(n)))
        return [(KERNEL[int(kinds[i])], float(ms[i]), float(by[i])) for i in range(k)]

    def row_array(self, steps, out_ptr: int):
        """x(i) for every row (Sec. 2h product) into device memory at out_ptr
        (2^M uint64)."""
        s = as_steps(steps)
        _check(self._lib.qsim_row_array(self._ctx, _ptr(s), len(s), ctypes.c_void_p(out_ptr)))

    def plan_stats(self) -> dict:
        st = PlanStats()
        _check(self._lib.qsim_get_plan_stats(self._ctx, ctypes.byref(st)))
        return st.as_dict()

    def synchronize(self):
        _check(self._lib.qsim_synchronize(self._ctx))

    # -- post-processing --------------------------------------------------------------
    def probabilities(self, with_norm: bool = False, out: np.ndarray | None = None):
        """FP64 probabilities in host memory (``out``: optional float64 buffer,
        e.g. pinned, of 2^M entries)."""
        p = np.empty(self.n, dtype=np.float64) if out is None else out
        if p.dtype != np.float64 or p.shape != (self.n,) or not p.flags.c_contiguous:
            raise QsimError(QSIM_EINVAL, "out must be a contiguous float64 array of 2^M entries")
        norm = ctypes.c_double(0.0)
        _check(self._lib.qsim_probabilities(self._ctx, _ptr(p), self.n,
                                            ctypes.byref(norm) if with_norm else None))
        return (p, norm.value) if with_norm else p

    def probabilities_device(self, out_ptr: int, with_norm: bool = False):
        """FP64 probabilities into device memory at out_ptr (2^M doubles)."""
        norm = ctypes.c_double(0.0)
        _check(self._lib.qsim_probabilities_device(self._ctx, ctypes.c_void_p(out_ptr),
                                                   ctypes.byref(norm) if with_norm else None))
        return norm.value if with_norm else None


def jit_precompile(M: int, dtype, steps, canonicalize: bool = True) -> float:
    """Compile the circuit-specialised kernels of a circuit; returns compile ms."""
    s = as_steps(steps)
    ms = ctypes.c_double(0.0)
    _check(load().qsim_jit_precompile(M, dtype_code(dtype), _ptr(s), len(s), int(canonicalize),
                                      ctypes.byref(ms)))
    return ms.value


class Batch:
    """Independent circuits run together: ``run()`` replays one captured graph
    of persistent launches; ``run_plain()`` launches one kernel per circuit
    pass.  circuits: list of (M, steps)."""

    def __init__(self, circuits, dtype=np.complex64, coset_min_qubits: int | None = None):
        self._lib = load()
        self.dtype = np.dtype(dtype)
        self.M = [int(m) for m, _ in circuits]
        self._steps = [as_steps(s) for _, s in circuits]
        n = len(circuits)
        Ms = (ctypes.c_uint32 * n)(*self.M)
        ptrs = (ctypes.c_void_p * n)(*[s.ctypes.data if len(s) else 0 for s in self._steps])
        Ls = (ctypes.c_size_t * n)(*[len(s) for s in self._steps])
        self._b = ctypes.c_void_p()
        opts = None if coset_min_qubits is None else ctypes.byref(BatchOptions(coset_min_qubits))
        _check(self._lib.qsim_batch_create_ex(n, ctypes.cast(Ms, ctypes.c_void_p), dtype_code(self.dtype),
                                              ctypes.cast(ptrs, ctypes.c_void_p),
                                              ctypes.cast(Ls, ctypes.c_void_p), opts, ctypes.byref(self._b)))

    def close(self):
        if self._b:
            self._lib.qsim_batch_destroy(self._b)
            self._b = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def load_state(self, i: int, k: np.ndarray):
        a = np.ascontiguousarray(k, dtype=self.dtype)
        _check(self._lib.qsim_batch_load_state(self._b, i, _ptr(a), a.shape[0]))

    def read_state(self, i: int) -> np.ndarray:
        out = np.empty(1 << self.M[i], dtype=self.dtype)
        _check(self._lib.qsim_batch_read_state(self._b, i, _ptr(out), out.shape[0]))
        return out

    def state_ptr(self, i: int) -> int:
        return int(self._lib.qsim_batch_state_device(self._b, i) or 0)

    def run(self):
        _check(self._lib.qsim_batch_run(self._b))

    def run_plain(self):
        _check(self._lib.qsim_batch_run_plain(self._b))

    def synchronize(self):
        _check(self._lib.qsim_batch_synchronize(self._b))

    def info(self) -> dict:
        st = BatchStats()
        _check(self._lib.qsim_batch_info(self._b, ctypes.byref(st)))
        return st.as_dict()


class Server:
    """Continuous-batching request loop (qsim_server_*).  ``submit`` returns a
    request id; ``poll`` returns (done, latency_ms, probabilities view)."""

    def __init__(self, hbm_budget_bytes: int, host_result_bytes: int, dtype=np.complex128):
        self._lib = load()
        self.dtype = np.dtype(dtype)
        self._s = ctypes.c_void_p()
        self._keep = {}
        _check(self._lib.qsim_server_create(int(hbm_budget_bytes), int(host_result_bytes),
                                            dtype_code(self.dtype), ctypes.byref(self._s)))

    def close(self):
        if self._s:
            self._lib.qsim_server_destroy(self._s)
            self._s = ctypes.c_void_p()
        self._keep = {}

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_backfill(self, max_head_wait_ms: float):
        """Backfill admission while the oldest waiting request has waited less
        than max_head_wait_ms (negative: strict FIFO)."""
        _check(self._lib.qsim_server_set_backfill(self._s, float(max_head_wait_ms)))

    def set_copy_streams(self, n: int):
        """Copies in and out on two overlapping streams (2) or one stream (1)."""
        _check(self._lib.qsim_server_set_copy_streams(self._s, int(n)))

    def set_eviction(self, evict_after_ms: float):
        """Swap running requests out to host memory for a head that waited
        this long (negative: off)."""
        _check(self._lib.qsim_server_set_eviction(self._s, float(evict_after_ms)))

    def set_upload_chunk(self, nbytes: int):
        _check(self._lib.qsim_server_set_upload_chunk(self._s, nbytes))

    def set_paused(self, paused: bool):
        """Pause or resume admission (admitted requests keep running)."""
        _check(self._lib.qsim_server_set_paused(self._s, int(bool(paused))))

    def set_tracing(self, enable: bool):
        """Record a timeline per finished request (see trace())."""
        _check(self._lib.qsim_server_set_tracing(self._s, int(bool(enable))))

    def trace(self) -> np.ndarray:
        """Timelines recorded since the last call, as a structured array with
        the fields of qsim_server_trace_record (milliseconds)."""
        rows = []
        while True:
            buf = (ServerTraceRecord * 4096)()
            n = ctypes.c_size_t(0)
            _check(self._lib.qsim_server_get_trace(self._s, buf, 4096, ctypes.byref(n)))
            rows.extend(buf[:n.value])
            if n.value < 4096:
                break
        dt = np.dtype([(f, np.uint64 if t in (ctypes.c_uint64,) else
                        np.uint32 if t is ctypes.c_uint32 else np.float64)
                       for f, t in ServerTraceRecord._fields_])
        return np.array([tuple(getattr(r, f) for f, _ in ServerTraceRecord._fields_) for r in rows],
                        dtype=dt)

    def submit(self, M: int, k1: np.ndarray, steps) -> int:
        """k1 must stay alive and unchanged until the request is done (kept here)."""
        a = np.ascontiguousarray(k1)
        if a.dtype != self.dtype or a.shape != (1 << M,):
            raise QsimError(QSIM_EINVAL, "state must be 2^M amplitudes of the server dtype")
        s = as_steps(steps)
        rid = ctypes.c_uint64(0)
        _check(self._lib.qsim_server_submit(self._s, M, _ptr(a), _ptr(s), len(s), ctypes.byref(rid)))
        self._keep[rid.value] = (a, M)
        return rid.value

    def poll(self, rid: int, copy: bool = True):
        done = ctypes.c_int(0)
        lat = ctypes.c_double(0.0)
        pp = ctypes.POINTER(ctypes.c_double)()
        _check(self._lib.qsim_server_poll(self._s, rid, ctypes.byref(done), ctypes.byref(lat),
                                          ctypes.byref(pp)))
        if not done.value:
            return False, None, None
        M = self._keep[rid][1]
        probs = np.ctypeslib.as_array(pp, shape=(1 << M,))
        return True, lat.value, (probs.copy() if copy else probs)

    def drain(self, cap: int = 4096):
        """[(request id, latency ms)] of requests finished since the last drain."""
        ids = np.zeros(cap, dtype=np.uint64)
        lat = np.zeros(cap, dtype=np.float64)
        n = ctypes.c_size_t(0)
        _check(self._lib.qsim_server_drain(self._s, _ptr(ids), _ptr(lat), cap, ctypes.byref(n)))
        return [(int(ids[i]), float(lat[i])) for i in range(n.value)]

    def release(self, rid: int):
        _check(self._lib.qsim_server_release(self._s, rid))
        self._keep.pop(rid, None)

    def wait_all(self, timeout_s: float = 600.0):
        _check(self._lib.qsim_server_wait_all(self._s, timeout_s))

    def stats(self) -> dict:
        st = ServerStats()
        _check(self._lib.qsim_server_get_stats(self._s, ctypes.byref(st)))
        return st.as_dict()


def gather_rows(d_in: int, d_out: int, d_rows: int, M: int, dtype, d_probs: int = 0,
                loads_in_flight: int = 0, stream: int = 0):
    """k2(i) = k1(x(i)) for a stored row array (device pointers, no context)."""
    L = load()
    _check(L.qsim_gather_rows(ctypes.c_void_p(d_in), ctypes.c_void_p(d_out), ctypes.c_void_p(d_rows),
                              M, dtype_code(dtype), ctypes.c_void_p(d_probs or None), loads_in_flight,
                              ctypes.c_void_p(stream or None)))


def version() -> str:
    return load().qsim_version().decode()
