"""qsim_probabilities_noalloc: probabilities and norm without allocating.

The entry point serves callers that cannot allocate device memory when they
need a result (GPU memory wholly reserved by another allocator, a plug-in
held to a fixed budget, a loop that must not enter the allocator).  Its only
scratch is a fixed device array inside the library, so this test checks,
through the C ABI, that two calls in a row on different states give the same
probabilities and norm as the context-based qsim_probabilities_device (and
as the CPU oracle), and that out-of-range sizes are refused.  The file name
makes pytest collect it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_quant_ph_0308158_gb300 import Simulator, load, workloads as W
from tests.helpers import assert_probs_close

pytestmark = pytest.mark.gpu

NORM_RTOL = 1e-12


@pytest.fixture(scope="module")
def torch():
    import torch as t
    assert t.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_quant_ph_0308158_gb300 import build
    build.build()
    t.cuda.set_device(0)
    # memory PyTorch still caches from earlier tests goes back to the device:
    # the first launch of the library's code in this context loads its module
    t.cuda.empty_cache()
    return t


def _noalloc(torch, state_t, M, dtype_code):
    lib = load()
    n = 1 << M
    probs = torch.empty(n, dtype=torch.float64, device="cuda")
    norm = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = lib.qsim_probabilities_noalloc(
        ctypes.c_void_p(state_t.data_ptr()), M, dtype_code, ctypes.c_void_p(probs.data_ptr()),
        ctypes.c_void_p(norm.data_ptr()), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, lib.qsim_last_error()
    torch.cuda.synchronize()
    return probs.cpu().numpy(), float(norm.item())


def _existing(torch, k, M, dtype):
    with Simulator(M, dtype) as sim:
        sim.load_state(k)
        probs = torch.empty(1 << M, dtype=torch.float64, device="cuda")
        norm = sim.probabilities_device(probs.data_ptr(), with_norm=True)
        torch.cuda.synchronize()
        return probs.cpu().numpy(), norm


@pytest.mark.parametrize("dtype,code,M", [(np.complex128, 1, 18), (np.complex64, 0, 21)])
def test_noalloc_matches_existing_entry_point_twice(torch, dtype, code, M):
    tdt = torch.complex128 if code == 1 else torch.complex64
    for seed in (101, 202):  # two calls in a row, different states
        k = W.random_state(M, dtype, seed)
        st = torch.from_numpy(k).to("cuda")
        p_new, n_new = _noalloc(torch, st, M, code)
        p_old, n_old = _existing(torch, k, M, dtype)
        np.testing.assert_array_equal(p_new, p_old)
        assert abs(n_new - n_old) <= NORM_RTOL * abs(n_old)
        p_ref = oracle.probabilities(k)
        assert_probs_close(p_new, p_ref)
        assert abs(n_new - oracle.fsum_pairwise(p_ref)) <= NORM_RTOL * n_old
        assert st.dtype == tdt


def test_noalloc_norm_only_and_rejections(torch):
    lib = load()
    M = 12
    k = W.random_state(M, np.complex128, 5)
    st = torch.from_numpy(k).to("cuda")
    norm = torch.zeros(1, dtype=torch.float64, device="cuda")
    s = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert lib.qsim_probabilities_noalloc(ctypes.c_void_p(st.data_ptr()), M, 1, None,
                                          ctypes.c_void_p(norm.data_ptr()), s) == 0
    torch.cuda.synchronize()
    assert abs(norm.item() - oracle.fsum_pairwise(oracle.probabilities(k))) <= NORM_RTOL
    # sizes beyond the maximum and bad arguments are refused before any launch
    for bad_M in (0, 35, 64):
        rc = lib.qsim_probabilities_noalloc(ctypes.c_void_p(st.data_ptr()), bad_M, 1, None,
                                            ctypes.c_void_p(norm.data_ptr()), s)
        assert rc == -1 and b"M must be in" in lib.qsim_last_error()
    assert lib.qsim_probabilities_noalloc(ctypes.c_void_p(st.data_ptr()), M, 7, None,
                                          ctypes.c_void_p(norm.data_ptr()), s) == -1
    assert lib.qsim_probabilities_noalloc(None, M, 1, None, ctypes.c_void_p(norm.data_ptr()), s) == -1
