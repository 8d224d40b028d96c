"""Coset-blocked affine gather (gather_coset_kernel) against the CPU oracle.

NOT/CNOT-only segments are one GF(2) affine map x(i) = A i ^ b (the Sec. 2h
product of such steps, gathered as in Sec. 2b).  The coset kernel cuts the
output space into cosets of S = span(low r bits, A^-1 of the low r bits), so
every read and write is an aligned run of 2^r amplitudes.  States must match
the oracle bit for bit for every run length r, tile group size and M,
including maps that keep the low bits among themselves (d = 0, the Sec. 4
parity program) and sizes below one run.
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


def _run(M, dtype, steps, k1, run_bits=0, coset=True, probs=None):
    with Simulator(M, dtype) as sim:
        sim.set_strategy("gather")
        sim.set_canonicalize(False)
        sim.set_coset(coset, run_bits)
        sim.set_profiling(True)
        sim.load_state(k1)
        if probs is None:
            sim.apply(steps)
        else:
            sim.apply_probabilities(steps, probs.data_ptr())
        kernels = [k for k, _, _ in sim.pass_times()]
        return sim.read_state(), kernels


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("M,L,seed", [(1, 3, 1), (2, 9, 2), (4, 30, 3), (6, 70, 4), (9, 200, 5),
                                      (12, 500, 6), (15, 1000, 7), (19, 1000, 8), (22, 1500, 9)])
@pytest.mark.parametrize("run_bits", [0, 1, 3, 5, 7])
def test_coset_gather_bit_exact(dtype, M, L, seed, run_bits):
    if M == 1:  # NOT only
        steps = W.make_steps([(0, 0, 0)] * L)
    else:
        steps = np.concatenate([W.cnot_circuit(M, L, seed), W.make_steps([(M - 1, 0, 0), (0, 0, 0)])])
    k1 = W.random_state(M, dtype, seed)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    got, kernels = _run(M, dtype, steps, k1, run_bits)
    np.testing.assert_array_equal(got, want)
    assert kernels == ["gather_coset_kernel"]


@pytest.mark.parametrize("M", [12, 20])
def test_coset_gather_low_bits_closed_map(M):
    """The Sec. 4 parity program maps the low bits among themselves (no
    coset bits, d = 0): one run per tile, many tiles per stage."""
    k1 = W.alternating_state(M, np.complex64)
    steps = W.parity_circuit(M)
    want = oracle.apply_circuit(M, k1, steps).astype(np.complex64)
    got, _ = _run(M, np.complex64, steps, k1)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_coset_gather_writes_probabilities(cuda, dtype):
    torch = cuda
    M = 18
    steps = W.cnot_circuit(M, 700, 31)
    k1 = W.random_state(M, dtype, 31)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    p = torch.full((1 << M,), -1.0, dtype=torch.float64, device="cuda")
    got, kernels = _run(M, dtype, steps, k1, probs=p)
    np.testing.assert_array_equal(got, want)
    assert kernels == ["gather_coset_kernel"]
    want_p = oracle.probabilities(want)
    if dtype == np.complex64:
        np.testing.assert_array_equal(p.cpu().numpy().view(np.uint64), want_p.view(np.uint64))
    else:
        assert_probs_close(p.cpu().numpy(), want_p)


def test_cnot_m28_workload_sampled(cuda):
    """The M = 28 complex128 1000-CNOT workload: sampled rows against the
    oracle's single-row evaluation, coset pass against the direct affine
    pass over the whole state."""
    torch = cuda
    cfg = W.config_cnot(28)
    M, steps = cfg["M"], cfg["steps"]
    k1 = W.random_state(M, np.complex128, cfg["state_seed"])
    rng = np.random.default_rng(28)
    rows = rng.integers(0, 1 << M, size=1 << 20, dtype=np.uint64)
    rows[:2] = [0, (1 << M) - 1]
    src = oracle.source_rows(M, steps, rows).astype(np.int64)
    ridx = torch.from_numpy(rows.astype(np.int64)).cuda()
    outs = []
    for coset in (True, False):
        with Simulator(M, np.complex128) as sim:
            sim.set_canonicalize(False)
            sim.set_coset(coset)
            sim.load_state(k1)
            sim.apply(steps)
            sim.synchronize()
            t = sim.state_tensor()
            np.testing.assert_array_equal(t[ridx].cpu().numpy(), k1[src])
            outs.append(t.clone())
    assert bool((outs[0].view(torch.int64) == outs[1].view(torch.int64)).all())


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("U", [0, 4, 16])
def test_gather_by_stored_row_array(cuda, dtype, U):
    """qsim_gather_rows with the row array of a circuit (qsim_row_array)
    reproduces the circuit (Sec. 2b gather of the Sec. 2h product), with
    probabilities, for every loads-in-flight setting; rows beyond 2^M wrap."""
    torch = cuda
    from paper_quant_ph_0308158_gb300 import gather_rows
    M = 17
    steps = W.mixed_circuit(M, 300, 44)
    k1 = W.random_state(M, dtype, 44)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    tdt = torch.complex64 if dtype == np.complex64 else torch.complex128
    rows = torch.empty(1 << M, dtype=torch.int64, device="cuda")
    with Simulator(M, dtype) as sim:
        sim.row_array(steps, rows.data_ptr())
        sim.synchronize()
    np.testing.assert_array_equal(rows.cpu().numpy(), oracle.gather_map(M, steps))
    d_in = torch.from_numpy(k1).to("cuda")
    d_out = torch.empty(1 << M, dtype=tdt, device="cuda")
    p = torch.empty(1 << M, dtype=torch.float64, device="cuda")
    rows += torch.randint(0, 4, (1 << M,), device="cuda") << M  # taken modulo 2^M
    gather_rows(d_in.data_ptr(), d_out.data_ptr(), rows.data_ptr(), M, dtype, p.data_ptr(), U,
                torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(d_out.cpu().numpy(), want)
    want_p = oracle.probabilities(want)
    assert_probs_close(p.cpu().numpy(), want_p)
