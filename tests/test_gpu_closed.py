"""Closed tile passes (qsim_jit_closed) against the CPU oracle.

When a circuit's net row map changes only a few address bits (found exactly
on the device as the OR over every row of x(i) ^ i), every output's source
lies in the same coset of those bits, so one in-place pass over tiles holding
those bits applies the whole circuit: each tile is loaded, each output's
source x(i) is evaluated from the compiled step list (Sec. 2h product per
row), and the tile is written back (Sec. 2b gather).  States must match the
oracle bit for bit.
"""
import numpy as np
import pytest

import oracle
from paper_quant_ph_0308158_gb300 import Simulator, workloads as W
from tests.helpers import assert_probs_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_quant_ph_0308158_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def uncompute_circuit(M, s, L1, L2, seed):
    """C1 + C2 + reverse(C1): C1 reads and writes only bits outside a set S of
    s bits, C2 writes only S (controls anywhere), so the net map changes only
    bits of S and every step of C1 is undone."""
    rng = np.random.default_rng(seed)
    S = sorted(int(x) for x in rng.choice(M, size=s, replace=False))
    out = [b for b in range(M) if b not in S]
    rows1 = []
    for _ in range(L1):
        t, *c = (int(x) for x in rng.choice(out, size=3, replace=False))
        nc = int(rng.integers(0, 3))
        m = sum(1 << x for x in c[:nc])
        rows1.append((t, m, m & int(rng.integers(0, 1 << 40))))
    rows2 = []
    for _ in range(L2):
        t = int(rng.choice(S))
        c = [int(x) for x in rng.choice([b for b in range(M) if b != t], size=3, replace=False)]
        nc = int(rng.integers(0, 4))
        m = sum(1 << x for x in c[:nc])
        rows2.append((t, m, m))
    return W.make_steps(rows1 + rows2 + rows1[::-1]), sum(1 << b for b in S)


def _run_closed(M, dtype, steps, k1, probs=None):
    with Simulator(M, dtype, scratch=False) as sim:
        sim.set_strategy("inplace")
        sim.set_canonicalize(False)
        sim.set_jit(True)
        sim.set_profiling(True)
        sim.load_state(k1)
        if probs is None:
            sim.apply(steps)
        else:
            sim.apply_probabilities(steps, probs.data_ptr())
        kernels = [k for k, _, _ in sim.pass_times()]
        return sim.read_state(), kernels


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("M,s,L1,L2,seed", [(12, 4, 30, 40, 1), (14, 7, 60, 120, 2), (17, 9, 100, 300, 3),
                                            (20, 11, 150, 500, 4), (22, 12, 200, 400, 5)])
def test_closed_pass_bit_exact(dtype, M, s, L1, L2, seed):
    steps, _ = uncompute_circuit(M, s, L1, L2, seed)
    k1 = W.random_state(M, dtype, seed)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    got, kernels = _run_closed(M, dtype, steps, k1)
    np.testing.assert_array_equal(got, want)
    if M > (14 if dtype == np.complex64 else 13):
        assert kernels == ["qsim_jit_closed"]
    else:  # one ordinary tile holds the whole state: a single tile pass does it
        assert len(kernels) == 1


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_closed_pass_writes_probabilities(cuda, dtype):
    torch = cuda
    M = 19
    steps, _ = uncompute_circuit(M, 10, 120, 300, 9)
    k1 = W.random_state(M, dtype, 9)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    p = torch.full((1 << M,), -1.0, dtype=torch.float64, device="cuda")
    got, kernels = _run_closed(M, dtype, steps, k1, probs=p)
    np.testing.assert_array_equal(got, want)
    # the closed pass writes the probabilities beside the amplitudes it stores
    assert kernels == ["qsim_jit_closed"]
    want_p = oracle.probabilities(want)
    if dtype == np.complex64:
        np.testing.assert_array_equal(p.cpu().numpy().view(np.uint64), want_p.view(np.uint64))
    else:
        assert_probs_close(p.cpu().numpy(), want_p)


def test_no_whole_circuit_closed_pass_when_every_bit_changes():
    """A random circuit changes every bit: no single closed pass; its tile
    segments (whose steps change only tile bits) may still run as closed
    passes over their own tiles.  Exact either way."""
    M = 16
    steps = W.mixed_circuit(M, 200, 12)
    k1 = W.random_state(M, np.complex64, 12)
    want = oracle.apply_circuit(M, k1, steps).astype(np.complex64)
    got, kernels = _run_closed(M, np.complex64, steps, k1)
    np.testing.assert_array_equal(got, want)
    assert len(kernels) > 1


def test_adder_m28_closed_full_state():
    """The ripple-carry adder at M = 28 (two 13-bit registers): its net map
    changes b_4..b_12 and the carry-out only, one closed pass in place;
    every amplitude against the oracle."""
    cfg = W.config_adder(13)
    M, steps = cfg["M"], cfg["steps"]
    k1 = W.random_state(M, np.complex64, cfg["state_seed"])
    want = oracle.apply_circuit(M, k1, steps).astype(np.complex64)
    got, kernels = _run_closed(M, np.complex64, steps, k1)
    np.testing.assert_array_equal(got, want)
    assert kernels == ["qsim_jit_closed"]
