"""The seeded synthetic inputs match the workloads they stand for: gate mix,
distinct bits, controls on |1>, state distribution and norm, adder size,
Sec. 4 program, batch and serving streams.  No GPU needed."""
import math

import numpy as np
import pytest

import oracle
from paper_quant_ph_0308158_gb300 import workloads as W


def _popcount(m):
    return np.array([bin(int(x)).count("1") for x in m])


def test_mixed_circuit_gate_mix_and_distinct_bits():
    M, L = 28, 20000
    s = W.mixed_circuit(M, L, seed=2)
    nc = _popcount(s["ctrl_mask"])
    frac = [np.mean(nc == 0), np.mean(nc == 1), np.mean(nc == 2), np.mean(nc >= 3)]
    for got, want in zip(frac, [0.1, 0.5, 0.3, 0.1]):
        assert abs(got - want) < 0.015
    assert set(np.unique(nc[nc >= 3])) == {3, 4, 5}
    assert np.all(s["ctrl_pol"] == s["ctrl_mask"])  # controls on |1>
    assert np.all(((s["ctrl_mask"] >> s["target"].astype(np.uint64)) & np.uint64(1)) == 0)
    assert oracle.validate(M, s)
    # targets and controls spread over all address bits
    t = np.bincount(s["target"], minlength=M) / L
    assert t.min() > 0.5 / M and t.max() < 1.5 / M


def test_cnot_circuit_distinct_uniform_bits():
    M, L = 16, 64000
    s = W.cnot_circuit(M, L, seed=1)
    assert np.all(_popcount(s["ctrl_mask"]) == 1)
    assert np.all(s["ctrl_pol"] == s["ctrl_mask"])
    ctrl = np.log2(s["ctrl_mask"].astype(np.float64)).astype(int)
    assert np.all(ctrl != s["target"])
    pairs = np.bincount(ctrl * M + s["target"], minlength=M * M).reshape(M, M)
    off = pairs[~np.eye(M, dtype=bool)]
    assert off.min() > 0.6 * L / (M * (M - 1)) and off.max() < 1.4 * L / (M * (M - 1))


def test_random_state_distribution_and_norm():
    M = 18
    k = W.random_state(M, np.complex128, seed=7)
    assert abs(oracle.fsum_pairwise(oracle.probabilities(k)) - 1.0) < 1e-12
    # magnitudes before normalising: the norm is about sqrt(2^M / 3), E[r^2] = 1/3
    r = np.abs(k) * math.sqrt((1 << M) / 3.0)
    assert 0.98 < r.max() < 1.02 and r.min() < 1e-3
    assert abs(np.mean(r) - 0.5) < 0.01  # uniform in [0, 1)
    assert abs(np.mean(r < 0.25) - 0.25) < 0.01
    phase = np.angle(k) % (2 * math.pi)
    hist = np.histogram(phase, bins=16, range=(0, 2 * math.pi))[0] / k.size
    assert np.all(np.abs(hist - 1 / 16) < 0.004)  # phases uniform in [0, 2 pi)
    # same seed, same state; complex64 is the rounded complex128 state
    np.testing.assert_array_equal(k, W.random_state(M, np.complex128, seed=7))
    np.testing.assert_array_equal(W.random_state(M, np.complex64, seed=7), k.astype(np.complex64))


def test_adder_workload_size_and_bit_placement():
    cfg = W.config_adder_m32()
    assert cfg["M"] == 32 and cfg["dtype"] == np.complex64
    assert len(cfg["steps"]) == 2 * (6 * 15 + 1) * 8  # two additions of 91 steps, 8 units
    assert oracle.validate(32, cfg["steps"])
    t = np.unique(cfg["steps"]["target"])
    assert t.min() < 8 and t.max() > 24  # targets span low and high address bits
    nc = _popcount(cfg["steps"]["ctrl_mask"])
    assert set(np.unique(nc)) == {1, 2}  # CNOT and Toffoli only


def test_sec4_parity_program_and_input():
    M = 12
    s = W.parity_circuit(M)
    assert len(s) == M - 1 and np.all(s["target"] == 0)
    assert sorted(int(m).bit_length() - 1 for m in s["ctrl_mask"]) == list(range(1, M))
    k = oracle.product_state(M, W.sec4_qubits(M))
    np.testing.assert_allclose(k, W.alternating_state(M), rtol=1e-14, atol=0)


@pytest.mark.parametrize("mix", ["cnot", "mixed"])
def test_batch_specs_ranges(mix):
    specs = W.batch_specs(n=512, mix=mix)
    Ms = np.array([s["M"] for s in specs])
    Ls = np.array([s["L"] for s in specs])
    assert Ms.min() >= 10 and Ms.max() <= 22 and len(np.unique(Ms)) == 13
    assert Ls.min() >= 50 and Ls.max() <= 2000
    for s in specs[:20]:
        assert len(s["steps"]) == s["L"] and oracle.validate(s["M"], s["steps"])


def test_serving_stream_is_poisson_with_the_stated_ranges():
    specs = W.serving_requests(n=4000, rate=200.0, seed=5)
    t = np.array([s["arrival"] for s in specs])
    gaps = np.diff(np.concatenate([[0.0], t]))
    assert np.all(gaps > 0)
    assert abs(np.mean(gaps) - 1 / 200) < 0.0004
    assert abs(np.std(gaps) / np.mean(gaps) - 1.0) < 0.05  # exponential: cv = 1
    Ms = np.array([s["M"] for s in specs])
    Ls = np.array([s["L"] for s in specs])
    assert Ms.min() == 12 and Ms.max() == 30
    assert Ls.min() >= 100 and Ls.max() <= 5000
    assert all(np.all(_popcount(s["steps"]["ctrl_mask"]) == 1) for s in specs[:50])
