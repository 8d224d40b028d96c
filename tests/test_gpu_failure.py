"""Failure handling on the GPU without a fault: the tile pipeline's bounded
waits.

Every mbarrier wait in the tile pass gives up after a bounded number of
polls, sets the context's error flag and returns.  The testing hook
qsim_set_wait_test makes the next tile pass's producer warp leave before it
issues any copy, with a short poll limit, so that every consumer wait runs
out with nothing in flight.  The test checks that the library reports
QSIM_ETIMEOUT, that the stalled pass changed no amplitude, and that the
context then applies circuits bit-exactly again.
"""
import numpy as np
import pytest

import oracle
from paper_quant_ph_0308158_gb300 import QsimError, Simulator, workloads as W
from paper_quant_ph_0308158_gb300.binding import QSIM_EINVAL, QSIM_ETIMEOUT

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_quant_ph_0308158_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_bounded_wait_gives_up_and_context_recovers(dtype):
    M = 16
    steps = W.mixed_circuit(M, 60, 5)
    k1 = W.random_state(M, dtype, 5)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    with Simulator(M, dtype) as sim:
        sim.set_strategy("tile")
        sim.set_canonicalize(False)
        sim.load_state(k1)
        # one tile pass (both targets are low bits), armed to stall
        single = W.make_steps([(0, 1 << 3, 1 << 3), (2, 0, 0)])
        sim.set_wait_test(1000)
        sim.apply(single)
        assert sim.plan_stats()["tile_passes"] == 1
        with pytest.raises(QsimError) as ei:
            sim.synchronize()
        assert ei.value.code == QSIM_ETIMEOUT
        # the stalled pass moved nothing; the flag was cleared by the report
        np.testing.assert_array_equal(sim.read_state(), k1)
        sim.synchronize()
        # the hook was one-shot: the same context now runs circuits exactly
        sim.apply(steps)
        np.testing.assert_array_equal(sim.read_state(), want)


def test_wait_test_rejects_bad_limits():
    with Simulator(8, np.complex128) as sim:
        for bad in (0, (1 << 20) + 1):
            with pytest.raises(QsimError) as ei:
                sim.set_wait_test(bad)
            assert ei.value.code == QSIM_EINVAL
