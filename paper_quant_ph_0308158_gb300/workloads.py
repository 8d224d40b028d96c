"""Seeded synthetic inputs: states and wiring diagrams.

This module only draws random numbers and writes step lists; it applies no
step and computes nothing the simulator computes.  Tests feed the same
arrays to the CUDA library and to the CPU oracle, so both sides see
identical inputs.

Step arrays use ``STEP_DTYPE`` (24 bytes: target u4, reserved u4,
ctrl_mask u8, ctrl_pol u8), index bit b standing for the paper's address
wire a(b+1) (Sec. 2b).  A step with ctrl_mask == 0 is an unconditional NOT
(Sec. 2e).

Workloads (the paper's own example circuits are in Sec. 2b, 2h and Sec. 4):

* ``cnot_circuit``      -- L controlled-NOTs, control and target distinct
                           uniform bits.
* ``mixed_circuit``     -- 10% NOT, 50% CNOT, 30% Toffoli, 10% NOT with 3-5
                           controls; bits distinct within a step, controls
                           on |1>.
* ``adder_circuit``     -- ripple-carry adder of two n-bit registers with
                           carry-in and carry-out (majority / un-majority
                           ladder of Cuccaro, Draper, Kutin and Moulton,
                           quant-ph/0410184), CNOT/Toffoli only, with the
                           2n+2 lines placed on address bits by a seeded
                           permutation.
* ``parity_circuit``    -- the Sec. 4 test program: CNOTs from a(2)..a(M)
                           onto a(1).
* ``random_state``      -- magnitudes U[0,1), phases U[0,2pi), unit norm.
* ``alternating_state`` -- the paper's (1,-1,1,-1,...)/sqrt(2^M) input.
"""
from __future__ import annotations

import math
import os
from concurrent.futures import ThreadPoolExecutor

import numpy as np

STEP_DTYPE = np.dtype(
    [("target", "<u4"), ("reserved", "<u4"), ("ctrl_mask", "<u8"), ("ctrl_pol", "<u8")]
)

# Amplitudes generated per independent random stream; chunk c of a state
# with seed s is drawn from SeedSequence([s, c]), so any chunk can be
# regenerated alone and chunks can be drawn in parallel.
STATE_CHUNK_LOG2 = 20


def make_steps(rows) -> np.ndarray:
    """Step array from (target, ctrl_mask, ctrl_pol) tuples."""
    a = np.zeros(len(rows), dtype=STEP_DTYPE)
    for i, (t, c, p) in enumerate(rows):
        a[i] = (t, 0, c, p)
    return a


def _bits_to_mask(bits) -> int:
    m = 0
    for b in bits:
        m |= 1 << int(b)
    return m


# ----------------------------------------------------------------------------
# states
# ----------------------------------------------------------------------------

def _chunk_amps(seed: int, chunk: int, n: int) -> np.ndarray:
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([seed, chunk])))
    r = rng.random(n)
    phi = rng.random(n) * (2.0 * math.pi)
    a = np.empty(n, dtype=np.complex128)
    a.real = r * np.cos(phi)
    a.imag = r * np.sin(phi)
    return a


def _threads() -> int:
    return max(1, min(32, os.cpu_count() or 1))


def random_state(M: int, dtype=np.complex128, seed: int = 0, out: np.ndarray | None = None
                 ) -> np.ndarray:
    """Seeded state of 2^M amplitudes r*exp(i*phi), r ~ U[0,1), phi ~ U[0,2pi),
    normalised to unit norm in FP64 and then cast to ``dtype``.

    Built in chunks of 2^20 amplitudes on a thread pool: the norm is the
    exactly rounded sum (math.fsum) of per-chunk FP64 sums, then every chunk
    is regenerated, scaled and cast.  ``out`` may be a preallocated (e.g.
    pinned) buffer of the right length and dtype.
    """
    dtype = np.dtype(dtype)
    n = 1 << M
    cn = 1 << min(M, STATE_CHUNK_LOG2)
    nchunks = n // cn
    if out is None:
        out = np.empty(n, dtype=dtype)
    elif out.shape != (n,) or out.dtype != dtype:
        raise ValueError("out has the wrong shape or dtype")

    def norm_part(c):
        a = _chunk_amps(seed, c, cn)
        return float(np.sum(a.real * a.real + a.imag * a.imag))

    with ThreadPoolExecutor(_threads()) as ex:
        parts = list(ex.map(norm_part, range(nchunks)))
        scale = 1.0 / math.sqrt(math.fsum(parts))

        def fill(c):
            a = _chunk_amps(seed, c, cn)
            a *= scale
            out[c * cn:(c + 1) * cn] = a.astype(dtype, copy=False)

        list(ex.map(fill, range(nchunks)))
    return out


def alternating_state(M: int, dtype=np.complex128, out: np.ndarray | None = None) -> np.ndarray:
    """(1, -1, 1, -1, ...)/sqrt(2^M): the input of the paper's Sec. 2b example
    and of its Sec. 4 computational example (``out``: optional preallocated,
    e.g. pinned, buffer)."""
    n = 1 << M
    a = np.empty(n, dtype=dtype) if out is None else out
    if a.shape != (n,) or a.dtype != np.dtype(dtype):
        raise ValueError("out has the wrong shape or dtype")
    s = 1.0 / math.sqrt(n)
    a[0::2] = s
    a[1::2] = -s
    return a


# ----------------------------------------------------------------------------
# circuits
# ----------------------------------------------------------------------------

def _distinct_bits(rng, L: int, M: int, k: int) -> np.ndarray:
    """(L, k) array: each row k distinct uniform bits of [0, M) in random order."""
    keys = rng.random((L, M))
    return np.argsort(keys, axis=1)[:, :k].astype(np.int64)


def _masks(bits: np.ndarray, counts: np.ndarray) -> np.ndarray:
    """OR of 1<<bits[i, j] over j < counts[i]."""
    L, k = bits.shape
    m = np.zeros(L, dtype=np.uint64)
    for j in range(k):
        use = counts > j
        m[use] |= np.left_shift(np.uint64(1), bits[use, j].astype(np.uint64))
    return m


def cnot_circuit(M: int, L: int, seed: int) -> np.ndarray:
    """L controlled-NOTs with control and target two distinct uniform bits."""
    rng = np.random.Generator(np.random.PCG64(seed))
    bits = _distinct_bits(rng, L, M, 2)
    a = np.zeros(L, dtype=STEP_DTYPE)
    a["target"] = bits[:, 0]
    m = np.left_shift(np.uint64(1), bits[:, 1].astype(np.uint64))
    a["ctrl_mask"] = m
    a["ctrl_pol"] = m
    return a


def mixed_circuit(M: int, L: int, seed: int) -> np.ndarray:
    """10% NOT, 50% CNOT, 30% Toffoli, 10% NOT with 3-5 controls (uniform);
    all bits of a step distinct and uniform; controls on |1>."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kinds = rng.choice(4, size=L, p=[0.1, 0.5, 0.3, 0.1])
    many = rng.integers(3, 6, size=L)
    nc = np.choose(kinds, [np.zeros(L, np.int64), np.ones(L, np.int64),
                           np.full(L, 2, np.int64), many])
    nc = np.minimum(nc, M - 1)
    k = int(min(6, M))
    bits = _distinct_bits(rng, L, M, k)
    a = np.zeros(L, dtype=STEP_DTYPE)
    a["target"] = bits[:, 0]
    m = _masks(bits[:, 1:], nc)
    a["ctrl_mask"] = m
    a["ctrl_pol"] = m
    return a


def local_mixed_circuit(M: int, L: int, seed: int, target_bits: int = 12) -> np.ndarray:
    """The mixed gate set (10% NOT, 50% CNOT, 30% Toffoli, 10% NOT with 3-5
    controls) with every target among the lowest ``target_bits`` address
    bits and the controls anywhere: arithmetic on a low register."""
    rng = np.random.Generator(np.random.PCG64(seed))
    kinds = rng.choice(4, size=L, p=[0.1, 0.5, 0.3, 0.1])
    many = rng.integers(3, 6, size=L)
    nc = np.choose(kinds, [np.zeros(L, np.int64), np.ones(L, np.int64),
                           np.full(L, 2, np.int64), many])
    nc = np.minimum(nc, M - 1)
    tgt = rng.integers(0, target_bits, size=L)
    keys = rng.random((L, M))
    keys[np.arange(L), tgt] = 2.0  # the target is never a control
    ctl = np.argsort(keys, axis=1)[:, :5]
    a = np.zeros(L, dtype=STEP_DTYPE)
    a["target"] = tgt
    m = _masks(ctl, nc)
    a["ctrl_mask"] = m
    a["ctrl_pol"] = m
    return a


def random_circuit(M: int, L: int, seed: int, max_controls: int = 4,
                   polarity: bool = True) -> np.ndarray:
    """General random steps for property tests: 0..max_controls controls,
    random polarity when ``polarity`` is set."""
    rng = np.random.Generator(np.random.PCG64(seed))
    mc = min(max_controls, M - 1)
    nc = rng.integers(0, mc + 1, size=L)
    bits = _distinct_bits(rng, L, M, mc + 1)
    a = np.zeros(L, dtype=STEP_DTYPE)
    a["target"] = bits[:, 0]
    m = _masks(bits[:, 1:], nc)
    a["ctrl_mask"] = m
    if polarity:
        r = rng.integers(0, 1 << 62, size=L, dtype=np.int64).astype(np.uint64)
        a["ctrl_pol"] = m & r
    else:
        a["ctrl_pol"] = m
    return a


def parity_circuit(M: int) -> np.ndarray:
    """Sec. 4 test program: controlled-NOTs from a(j), j = 2..M, onto a(1)."""
    return make_steps([(0, 1 << (j - 1), 1 << (j - 1)) for j in range(2, M + 1)])


def adder_lines(n: int):
    """Logical line numbers of the ripple-carry adder: carry-in 0, then a_i at
    1 + 2i and b_i at 2 + 2i (interleaved), carry-out 2n + 1."""
    cin = 0
    a = [1 + 2 * i for i in range(n)]
    b = [2 + 2 * i for i in range(n)]
    cout = 2 * n + 1
    return cin, a, b, cout


def adder_steps_logical(n: int):
    """One addition b <- a + b + c_in (mod 2^n), carry-out line XOR carry,
    as (target line, [control lines]) pairs: 6n + 1 steps.

    Majority gate on (c, b, a): CNOT a->b, CNOT a->c, Toffoli (c, b)->a.
    Un-majority on (c, b, a): Toffoli (c, b)->a, CNOT a->c, CNOT c->b.
    The carry ripples up through a_0..a_{n-1}; the top carry is copied onto
    the carry-out line; the un-majority ladder runs back down, leaving the
    sum in b and restoring a and c_in.
    """
    cin, a, b, cout = adder_lines(n)
    ops = []

    def maj(c, bb, aa):
        ops.extend([(bb, [aa]), (c, [aa]), (aa, [c, bb])])

    def uma(c, bb, aa):
        ops.extend([(aa, [c, bb]), (c, [aa]), (bb, [c])])

    carries = [cin] + a[:-1]
    for i in range(n):
        maj(carries[i], b[i], a[i])
    ops.append((cout, [a[n - 1]]))
    for i in reversed(range(n)):
        uma(carries[i], b[i], a[i])
    return ops


def adder_circuit(n: int = 15, additions_per_unit: int = 2, repeats: int = 8,
                  seed: int = 3, M: int | None = None):
    """Ripple-carry adder circuit on M = 2n + 2 address bits (or more).

    A unit is ``additions_per_unit`` successive additions; the unit repeats
    ``repeats`` times.  Logical lines are placed on address bits by a seeded
    permutation so that targets span low and high bits.  Returns
    ``(steps, line_to_bit)``.
    """
    lines = 2 * n + 2
    if M is None:
        M = lines
    if M < lines:
        raise ValueError("adder needs M >= 2n + 2")
    rng = np.random.Generator(np.random.PCG64(seed))
    line_to_bit = [int(b) for b in rng.permutation(M)[:lines]]
    one = adder_steps_logical(n)
    rows = []
    for _ in range(repeats):
        for _ in range(additions_per_unit):
            for tgt, ctl in one:
                m = _bits_to_mask(line_to_bit[c] for c in ctl)
                rows.append((line_to_bit[tgt], m, m))
    return make_steps(rows), line_to_bit


# ----------------------------------------------------------------------------
# named workloads
# ----------------------------------------------------------------------------

def config_small_cnot(seed: int = 1):
    """M=16 complex128, L=64 CNOTs (distinct uniform control/target)."""
    return dict(name="M16_c128_cnot64", M=16, dtype=np.complex128,
                steps=cnot_circuit(16, 64, seed), state_seed=seed)


def config_cnot(M: int = 28, seed: int = 2, L: int = 1000, dtype=np.complex128):
    """L controlled-NOTs (distinct uniform control/target) on a 2^M state."""
    tag = "c128" if np.dtype(dtype) == np.complex128 else "c64"
    return dict(name="M%d_%s_cnot%d" % (M, tag, L), M=M, dtype=dtype,
                steps=cnot_circuit(M, L, seed), state_seed=seed)


def config_mixed(M: int = 28, seed: int = 2, L: int = 1000, dtype=np.complex128):
    """L steps of the NOT/CNOT/Toffoli/MCX mix on a 2^M state."""
    tag = "c128" if np.dtype(dtype) == np.complex128 else "c64"
    return dict(name="M%d_%s_mix%d" % (M, tag, L), M=M, dtype=dtype,
                steps=mixed_circuit(M, L, seed), state_seed=seed)


def config_hybrid(M: int = 28, seed: int = 6, dtype=np.complex128):
    """A circuit whose best plan mixes strategies per segment: 300 steps of
    the mixed gate set on a 12-bit low register (controls anywhere; tile
    passes keep them local), then a linear layer of 1000 random CNOTs over
    all bits (one coset gather)."""
    tag = "c128" if np.dtype(dtype) == np.complex128 else "c64"
    steps = np.concatenate([local_mixed_circuit(M, 300, seed, 12), cnot_circuit(M, 1000, seed + 1)])
    return dict(name="M%d_%s_hybrid300x1000" % (M, tag), M=M, dtype=dtype, steps=steps,
                state_seed=seed)


def config_mixed_m28(seed: int = 2, L: int = 1000):
    """M=28 complex128 (4 GiB), L=1000 steps of the NOT/CNOT/Toffoli/MCX mix."""
    return config_mixed(28, seed, L)


def config_adder_m32(seed: int = 3):
    """M=32 complex64 (32 GiB, in place): ripple-carry adder of two 15-bit
    registers plus carry-in/out, two additions per unit, unit repeated 8x."""
    steps, l2b = adder_circuit(15, 2, 8, seed)
    return dict(name="M32_c64_adder15x16", M=32, dtype=np.complex64,
                steps=steps, state_seed=seed, line_to_bit=l2b)


def config_adder(n: int = 13, seed: int = 3):
    """Ripple-carry adder on M = 2n + 2 bits, complex64, in place (the M = 32
    workload scaled down: n = 13 gives M = 28, a 2 GiB state)."""
    steps, l2b = adder_circuit(n, 2, 8, seed)
    M = 2 * n + 2
    return dict(name="M%d_c64_adder%dx16" % (M, n), M=M, dtype=np.complex64,
                steps=steps, state_seed=seed, line_to_bit=l2b)


def sec4_qubits(M: int) -> np.ndarray:
    """The Sec. 4 input (1, -1, 1, -1, ...)/sqrt(2^M) as M qubits (App. 1):
    (1, -1)/sqrt(2) on a(1) and (1, 1)/sqrt(2) on every other wire."""
    s = 1.0 / math.sqrt(2.0)
    q = np.empty((M, 2), dtype=np.complex128)
    q[0] = (s, -s)
    q[1:] = (s, s)
    return q


def config_parity(M: int = 32):
    """Sec. 4 computational example: the parity of a(2)..a(M) onto a(1) on the
    alternating input, generated on the device from its qubits (App. 1)."""
    return dict(name="M%d_c64_parity_sec4" % M, M=M, dtype=np.complex64,
                steps=parity_circuit(M), state_seed=None, qubits=sec4_qubits(M))


def batch_specs(n: int = 4096, seed: int = 4, mix: str = "cnot",
                m_range=(10, 22), l_range=(50, 2000)):
    """Independent circuits for the batched run: M ~ U{10..22},
    L ~ U{50..2000}; ``mix`` is "cnot" (CNOT-only) or "mixed"."""
    rng = np.random.Generator(np.random.PCG64(seed))
    Ms = rng.integers(m_range[0], m_range[1] + 1, size=n)
    Ls = rng.integers(l_range[0], l_range[1] + 1, size=n)
    out = []
    for i in range(n):
        cs = int(seed * 1_000_003 + i)
        M, L = int(Ms[i]), int(Ls[i])
        steps = cnot_circuit(M, L, cs) if mix == "cnot" else mixed_circuit(M, L, cs)
        out.append(dict(M=M, L=L, steps=steps, state_seed=cs))
    return out


def serving_requests(n: int = 20000, rate: float = 200.0, seed: int = 5,
                     m_range=(12, 30), l_range=(100, 5000), mix: str = "cnot"):
    """Poisson arrivals at ``rate`` req/s with M ~ U{12..30}, L ~ U{100..5000}.
    Returns dicts with arrival time (s), M, L, steps and state seed."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate, size=n)
    t = np.cumsum(gaps)
    Ms = rng.integers(m_range[0], m_range[1] + 1, size=n)
    Ls = rng.integers(l_range[0], l_range[1] + 1, size=n)
    out = []
    for i in range(n):
        cs = int(seed * 1_000_003 + i)
        M, L = int(Ms[i]), int(Ls[i])
        steps = cnot_circuit(M, L, cs) if mix == "cnot" else mixed_circuit(M, L, cs)
        out.append(dict(arrival=float(t[i]), M=M, L=L, steps=steps, state_seed=cs))
    return out
