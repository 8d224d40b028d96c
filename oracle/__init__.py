"""CPU oracle for reversible wiring-diagram simulation -- TEST INFRASTRUCTURE.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline / reference
legs of ``bench.py`` may import this package.  The CUDA library never links
or calls it, and this package imports nothing from the CUDA library's
package: both sides meet only through numpy arrays built by the seeded
input generators.

The arithmetic lives in ``qsim_oracle.c`` (plain C, FP64 complex, compiled
with ``-ffp-contract=off``); this module compiles it with gcc on first use
and marshals numpy arrays through ctypes.  Every routine cites the passage
of Burger's paper (Sec. 2a-2i, Sec. 4) that it restates.

Functions take a state as a 1-D complex numpy array of length 2^M and a
circuit as a structured numpy array with fields (target u4, reserved u4,
ctrl_mask u8, ctrl_pol u8), steps[0] acting first.  complex64 states are
widened to complex128 exactly; outputs are returned as complex128 and can be
narrowed back exactly because amplitudes are only moved.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qsim_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")

STEP_DTYPE = np.dtype(
    [("target", "<u4"), ("reserved", "<u4"), ("ctrl_mask", "<u8"), ("ctrl_pol", "<u8")]
)

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile qsim_oracle.c into oracle/_build/liboracle.so (gcc, -O2)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
           "-fno-fast-math", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        p = ctypes.c_void_p
        u32, sz, i32 = ctypes.c_uint32, ctypes.c_size_t, ctypes.c_int
        lib.oracle_validate.argtypes = [u32, p, sz]
        lib.oracle_validate.restype = i32
        lib.oracle_step_row_array.argtypes = [u32, p, p]
        lib.oracle_step_row_array.restype = i32
        lib.oracle_paper_product.argtypes = [u32, p, sz, p]
        lib.oracle_paper_product.restype = i32
        lib.oracle_gather_map.argtypes = [u32, p, sz, p]
        lib.oracle_gather_map.restype = i32
        lib.oracle_gather.argtypes = [u32, p, p, p]
        lib.oracle_gather.restype = i32
        lib.oracle_apply_circuit.argtypes = [u32, p, p, sz]
        lib.oracle_apply_circuit.restype = i32
        lib.oracle_source_rows.argtypes = [u32, p, sz, p, sz, p]
        lib.oracle_source_rows.restype = i32
        lib.oracle_product_state.argtypes = [u32, p, p]
        lib.oracle_product_state.restype = i32
        lib.oracle_probabilities.argtypes = [p, sz, p]
        lib.oracle_probabilities.restype = None
        lib.oracle_sum.argtypes = [p, sz]
        lib.oracle_sum.restype = ctypes.c_double
        _lib = lib
        return lib


def _steps(steps) -> np.ndarray:
    s = np.ascontiguousarray(steps)
    if s.dtype != STEP_DTYPE:
        raise TypeError("steps must be a numpy array of oracle.STEP_DTYPE")
    return s


def _ptr(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data) if a.size else ctypes.c_void_p(0)


def _check(rc: int, what: str):
    if rc != 0:
        raise ValueError("oracle: invalid arguments to %s" % what)


def validate(M: int, steps) -> bool:
    """True when every step is a valid wiring-diagram step on M wires."""
    s = _steps(steps)
    return _load().oracle_validate(M, _ptr(s), len(s)) == 0


def apply_circuit(M: int, k1: np.ndarray, steps) -> np.ndarray:
    """k2 = U_L ... U_1 k1, one step at a time (plain definition, Sec. 2a/2d)."""
    s = _steps(steps)
    k = np.array(k1, dtype=np.complex128, copy=True)
    if k.shape != (1 << M,):
        raise ValueError("state length must be 2^M")
    _check(_load().oracle_apply_circuit(M, _ptr(k), _ptr(s), len(s)), "apply_circuit")
    return k


def apply_circuit_inplace(M: int, k: np.ndarray, steps) -> np.ndarray:
    """apply_circuit on a complex128 state the caller owns, in place (no copy):
    the same C loop, for timing the oracle on states too large to copy."""
    s = _steps(steps)
    if k.dtype != np.complex128 or k.shape != (1 << M,) or not k.flags.c_contiguous:
        raise ValueError("state must be a contiguous complex128 array of length 2^M")
    _check(_load().oracle_apply_circuit(M, _ptr(k), _ptr(s), len(s)), "apply_circuit")
    return k


def step_row_array(M: int, step) -> np.ndarray:
    """Row array y(i) of one step, built by the +/-2^(goto-1) toggles (Sec. 2b-2d)."""
    s = _steps(np.asarray([step], dtype=STEP_DTYPE) if np.ndim(step) == 0 else step)
    y = np.empty(1 << M, dtype=np.int64)
    _check(_load().oracle_step_row_array(M, _ptr(s), _ptr(y)), "step_row_array")
    return y


def paper_product(M: int, steps) -> np.ndarray:
    """x after the literal Sec. 2h rule x(i) <- y(x(i)), steps in the order given."""
    s = _steps(steps)
    x = np.empty(1 << M, dtype=np.int64)
    _check(_load().oracle_paper_product(M, _ptr(s), len(s), _ptr(x)), "paper_product")
    return x


def gather_map(M: int, steps) -> np.ndarray:
    """x with k2(i) = k1(x(i)) equal to the circuit (Sec. 2h rule, last step first)."""
    s = _steps(steps)
    x = np.empty(1 << M, dtype=np.int64)
    _check(_load().oracle_gather_map(M, _ptr(s), len(s), _ptr(x)), "gather_map")
    return x


def gather(M: int, k1: np.ndarray, x: np.ndarray) -> np.ndarray:
    """k2(i) = k1(x(i)) (Sec. 2b closing formula)."""
    k = np.ascontiguousarray(k1, dtype=np.complex128)
    xx = np.ascontiguousarray(x, dtype=np.int64)
    out = np.empty_like(k)
    _check(_load().oracle_gather(M, _ptr(k), _ptr(xx), _ptr(out)), "gather")
    return out


def sparse_matrix_method(M: int, k1: np.ndarray, steps) -> np.ndarray:
    """The paper's summarised algorithm end to end: product, then gather."""
    return gather(M, k1, gather_map(M, steps))


def source_rows(M: int, steps, rows) -> np.ndarray:
    """x(i) for selected output rows only (k2(i) = k1(x(i))), any M <= 63."""
    s = _steps(steps)
    r = np.ascontiguousarray(rows, dtype=np.uint64)
    out = np.empty_like(r)
    _check(_load().oracle_source_rows(M, _ptr(s), len(s), _ptr(r), len(r), _ptr(out)),
           "source_rows")
    return out


def sample_outputs(M: int, k1_lookup, steps, rows) -> np.ndarray:
    """k2 at selected rows: k1_lookup(source rows) gathers the input values."""
    src = source_rows(M, steps, rows)
    return np.asarray(k1_lookup(src.astype(np.int64)), dtype=np.complex128)


def product_state(M: int, qubits) -> np.ndarray:
    """k1 from M qubits (App. 1): qubits[b] = (q_{b+1}(0), q_{b+1}(1))."""
    q = np.ascontiguousarray(qubits, dtype=np.complex128)
    if q.shape != (M, 2):
        raise ValueError("qubits must be a complex (M, 2) array")
    k = np.empty(1 << M, dtype=np.complex128)
    _check(_load().oracle_product_state(M, _ptr(q), _ptr(k)), "product_state")
    return k


def probabilities(k: np.ndarray) -> np.ndarray:
    """|k(i)|^2 in FP64, re*re + im*im without fused multiply-add."""
    kk = np.ascontiguousarray(k, dtype=np.complex128)
    p = np.empty(kk.shape[0], dtype=np.float64)
    _load().oracle_probabilities(_ptr(kk), kk.shape[0], _ptr(p))
    return p


def fsum_pairwise(v: np.ndarray) -> float:
    """Pairwise FP64 sum (used for the norm)."""
    vv = np.ascontiguousarray(v, dtype=np.float64)
    return float(_load().oracle_sum(_ptr(vv), vv.shape[0]))
