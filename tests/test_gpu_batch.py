"""Batches of independent circuits (qsim_batch_*) against the CPU oracle:
the graph-replayed persistent launches and the one-launch-per-pass path
must both give every circuit's state bit for bit, over several runs."""
import numpy as np
import pytest

import oracle
from paper_quant_ph_0308158_gb300 import Batch, QsimError, workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_quant_ph_0308158_gb300 import build
    build.build()
    torch.cuda.set_device(0)


def _circuits(seed, n, m_lo, m_hi, l_lo, l_hi, kind):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        M = int(rng.integers(m_lo, m_hi + 1))
        L = int(rng.integers(l_lo, l_hi + 1))
        if kind == "cnot":
            st = W.cnot_circuit(M, L, seed * 1000 + i)
        elif kind == "mixed":
            st = W.mixed_circuit(M, L, seed * 1000 + i)
        else:
            st = W.random_circuit(M, L, seed * 1000 + i, max_controls=min(9, M - 1))
        out.append((M, st))
    return out


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("kind", ["cnot", "mixed", "random"])
def test_batch_runs_match_the_oracle(dtype, kind):
    circs = _circuits({"cnot": 1, "mixed": 2, "random": 3}[kind], 23, 2, 15, 1, 400, kind)
    states = [W.random_state(M, dtype, 100 + i) for i, (M, _) in enumerate(circs)]
    want = [s.astype(np.complex128) for s in states]
    with Batch(circs, dtype) as b:
        info = b.info()
        assert info["circuits"] == len(circs) and info["levels"] >= 1
        for i, s in enumerate(states):
            b.load_state(i, s)
        for run in range(3):  # graph (even), graph (odd), one launch per pass
            if run < 2:
                b.run()
            else:
                b.run_plain()
            b.synchronize()
            for i, (M, st) in enumerate(circs):
                want[i] = oracle.apply_circuit(M, want[i], st)
                np.testing.assert_array_equal(b.read_state(i), want[i].astype(dtype),
                                              err_msg="circuit %d run %d" % (i, run))


def test_batch_with_several_levels():
    # one circuit longer than a gather pass holds, one with a nine-control step
    M = 12
    long = W.mixed_circuit(M, 5000, 7)
    many = np.concatenate([W.mixed_circuit(M, 30, 8), W.make_steps([(0, 0b1111111110, 0b1111111110)]),
                           W.mixed_circuit(M, 30, 9)])
    circs = [(M, long), (M, many), (9, W.cnot_circuit(9, 50, 1))]
    states = [W.random_state(m, np.complex128, 7 + i) for i, (m, _) in enumerate(circs)]
    with Batch(circs, np.complex128) as b:
        assert b.info()["levels"] >= 2
        for i, s in enumerate(states):
            b.load_state(i, s)
        for run in range(2):
            b.run()
            b.synchronize()
        for i, (m, st) in enumerate(circs):
            w = oracle.apply_circuit(m, oracle.apply_circuit(m, states[i], st), st)
            np.testing.assert_array_equal(b.read_state(i), w)


def test_batch_rejects_invalid_circuits():
    bad = W.make_steps([(0, 1, 1)])  # target is its own control
    with pytest.raises(QsimError) as e:
        Batch([(4, W.cnot_circuit(4, 5, 1)), (4, bad)], np.complex64)
    assert "circuit 1" in str(e.value)


@pytest.mark.parametrize("kind", ["cnot", "mixed"])
@pytest.mark.parametrize("coset_min", [10, 18])
def test_batch_at_workload_sizes_sampled(kind, coset_min):
    """Circuits of the batched workload's sizes (M up to 22, L up to 2000,
    complex64), NOT/CNOT circuits read in coset-tile order from M >=
    coset_min: sampled rows of every circuit against the oracle's single-row
    evaluation, after a graph run and after a plain run."""
    rng = np.random.default_rng(44)
    specs = [(22, 2000), (21, 1500), (20, 60), (18, 900), (17, 50), (14, 1200), (11, 700), (10, 50)]
    circs = []
    for i, (M, L) in enumerate(specs):
        st = W.cnot_circuit(M, L, 4400 + i) if kind == "cnot" else W.mixed_circuit(M, L, 4400 + i)
        circs.append((M, st))
    states = [W.random_state(M, np.complex64, 900 + i) for i, (M, _) in enumerate(circs)]
    with Batch(circs, np.complex64, coset_min_qubits=coset_min) as b:
        info = b.info()
        n_cnot_big = sum(1 for M, _ in specs if M >= coset_min) if kind == "cnot" else 0
        assert info["coset_passes"] == n_cnot_big
        for i, s in enumerate(states):
            b.load_state(i, s)
        for run in range(2):
            b.run() if run == 0 else b.run_plain()
            b.synchronize()
            for i, (M, st) in enumerate(circs):
                rows = rng.integers(0, 1 << M, size=min(1 << M, 1 << 14), dtype=np.uint64)
                full = np.concatenate([st] * (run + 1))
                src = oracle.source_rows(M, full, rows).astype(np.int64)
                got = b.read_state(i)[rows.astype(np.int64)]
                np.testing.assert_array_equal(got, states[i][src], err_msg="circuit %d run %d" % (i, run))
