"""Shared assertions for the GPU tests."""
import numpy as np

# FP64 probabilities: the contract is 1e-12 relative to the CPU oracle.  For
# complex128 the kernel evaluates re*re + im*im with one fused multiply-add,
# so it may differ from the oracle's two separately rounded products by one
# unit in the last place (complex64 squares are exact, so there the results
# are identical); anything beyond two units is a real error.
PROB_RTOL = 1e-12


def assert_probs_close(got, want):
    got = np.asarray(got, dtype=np.float64)
    want = np.asarray(want, dtype=np.float64)
    np.testing.assert_allclose(got, want, rtol=PROB_RTOL, atol=0)
    ulps = np.abs(got - want) / np.spacing(np.abs(want))
    assert float(np.max(ulps, initial=0.0)) <= 2.0, "probabilities differ by more than 2 ulp"
