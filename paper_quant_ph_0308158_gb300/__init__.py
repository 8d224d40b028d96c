"""GB300-native engine for reversible wiring-diagram state-vector simulation.

Burger's sparse-matrix method (a wiring diagram of NOT / controlled-NOT /
Toffoli / multi-controlled NOT steps, each a symmetric permutation matrix,
applied to a 2^M-amplitude state) runs in hand-written sm_103a kernels behind
the C ABI of ``include/qsim.h``; this package holds that library's sources
(``csrc/``), its build script, a thin ctypes binding and the seeded workload
generators.  Importing the package does not load the library; ``Simulator``
and ``load()`` do, and raise ``QsimError`` when it is missing.
"""
from .binding import (QsimError, Simulator, Batch, Server, load, plan_circuit, version,  # noqa: F401
                      jit_precompile, gather_rows, plan_circuit_ex, EXPORTS, STRATEGY)
from .workloads import STEP_DTYPE, make_steps  # noqa: F401

__all__ = ["QsimError", "Simulator", "Batch", "Server", "load", "plan_circuit", "version", "jit_precompile", "gather_rows", "plan_circuit_ex", "EXPORTS",
           "STRATEGY", "STEP_DTYPE", "make_steps"]
