"""Host buffers for the state and the probabilities (qsim_host_alloc) and
copies out of several contexts queued on one stream (qsim_set_copy_stream)."""
import ctypes

import numpy as np
import pytest

import oracle
from paper_quant_ph_0308158_gb300 import HostBuffer, QsimError, Simulator, load, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("nbytes", [1 << 20, (5 << 30) // 2])
def test_host_buffer_round_trip(cuda, nbytes):
    """A small (one 2 MiB-rounded chunk) and a multi-chunk buffer (2.5 GiB:
    three 1 GiB chunks moved into one range): every byte written on the host
    reaches the device and comes back."""
    torch = cuda
    n = nbytes // 8
    buf = HostBuffer((n,), np.float64)
    a = buf.array
    assert a.shape == (n,) and a.ctypes.data % (2 << 20) == 0
    a[:] = np.arange(n, dtype=np.float64)
    d = torch.from_numpy(a).to("cuda", non_blocking=True)
    torch.cuda.synchronize()
    assert float(d[-1].item()) == float(n - 1) and float(d[n // 3].item()) == float(n // 3)
    d.mul_(-1.0)
    torch.from_numpy(a).copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    idx = np.random.default_rng(1).integers(0, n, size=1 << 16)
    np.testing.assert_array_equal(a[idx], -idx.astype(np.float64))
    assert a[0] == 0.0 and a[-1] == -(n - 1)
    del d, a
    buf.close()
    buf.close()  # idempotent


def test_host_alloc_rejects_bad_arguments(cuda):
    lib = load()
    p = ctypes.c_void_p()
    assert lib.qsim_host_alloc(0, ctypes.byref(p)) == -1
    assert lib.qsim_host_alloc(1 << 20, None) == -1
    x = np.zeros(16)
    assert lib.qsim_host_free(ctypes.c_void_p(x.ctypes.data)) == -1  # not ours
    assert lib.qsim_host_free(None) == 0
    assert lib.qsim_host_alloc(1 << 62, ctypes.byref(p)) == -2  # more than the host has


def test_shared_copy_stream_two_contexts(cuda):
    """Two contexts whose probabilities go out on one caller stream, then on
    their private streams again: every result equals the oracle's."""
    torch = cuda
    M = 20
    cs = torch.cuda.Stream()
    steps = [W.cnot_circuit(M, 40, 1), W.mixed_circuit(M, 60, 2)]
    k1 = [W.random_state(M, np.complex64, 3), W.random_state(M, np.complex64, 4)]
    want = [oracle.probabilities(oracle.apply_circuit(M, k1[i], steps[i]).astype(np.complex64))
            for i in range(2)]
    outs = HostBuffer((2, 1 << M), np.float64)
    sims = [Simulator(M, np.complex64) for _ in range(2)]
    try:
        for shared in (True, False):
            for i, sm in enumerate(sims):
                sm.set_copy_stream(cs.cuda_stream if shared else 0)
                sm.load_state(k1[i])
            outs.array[:] = -1.0
            for i, sm in enumerate(sims):
                sm.apply_probabilities_async(steps[i], outs.array[i])
            for sm in sims:
                sm.synchronize()
            for i in range(2):
                np.testing.assert_array_equal(outs.array[i].view(np.uint64), want[i].view(np.uint64))
    finally:
        for sm in sims:
            sm.close()
        outs.close()
