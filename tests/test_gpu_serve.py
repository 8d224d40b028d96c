"""The serving loop (qsim_server_*): requests admitted under an HBM budget,
run together in rounds, results identical to the CPU oracle and to the same
request served alone."""
import threading
import time

import numpy as np
import pytest

import oracle
from paper_quant_ph_0308158_gb300 import QsimError, Server, workloads as W
from tests.helpers import assert_probs_close

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_quant_ph_0308158_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    torch.cuda.empty_cache()  # the servers below take their budgets with cudaMalloc


def _requests(n, seed, m_lo=4, m_hi=16):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(n):
        M = int(rng.integers(m_lo, m_hi + 1))
        kind = int(rng.integers(3))
        L = int(rng.integers(0, 600)) if i % 7 else 4500  # some need two gather passes
        if kind == 0:
            st = W.cnot_circuit(M, L, 5000 + i)
        elif kind == 1:
            st = W.mixed_circuit(M, L, 5000 + i)
        else:
            st = W.random_circuit(M, L, 5000 + i, max_controls=min(9, M - 1))
        k1 = W.random_state(M, np.complex128, 7000 + i)
        out.append((M, k1, st))
    return out


def _expected(M, k1, st):
    return oracle.probabilities(oracle.apply_circuit(M, k1, st))


def test_served_results_match_the_oracle_and_the_request_alone():
    reqs = _requests(40, 1)
    # a budget that holds only a few of the largest requests at once
    with Server(24 << 20, 64 << 20, np.complex128) as srv:
        ids = []
        for i, (M, k1, st) in enumerate(reqs):  # arrivals spread over time
            ids.append(srv.submit(M, k1, st))
            if i % 5 == 4:
                time.sleep(0.002)
        srv.wait_all(300)
        stats = srv.stats()
        assert stats["completed"] == len(reqs) and stats["rounds"] >= 2
        assert stats["peak_in_use_bytes"] <= 24 << 20
        mixed = {}
        for rid, (M, k1, st) in zip(ids, reqs):
            done, lat, p = srv.poll(rid)
            assert done and lat > 0
            mixed[rid] = p
            assert_probs_close(p, _expected(M, k1, st))
            srv.release(rid)
        assert srv.stats()["in_use_bytes"] == 0 and srv.stats()["host_in_use_bytes"] == 0
    # the same requests served one at a time give the same bits
    with Server(24 << 20, 64 << 20, np.complex128) as srv:
        for rid, (M, k1, st) in list(zip(ids, reqs))[:8]:
            r = srv.submit(M, k1, st)
            srv.wait_all(60)
            done, _, p = srv.poll(r)
            assert done
            np.testing.assert_array_equal(p, mixed[rid])
            srv.release(r)


def test_concurrent_submitters():
    reqs = _requests(24, 2, 6, 14)
    with Server(64 << 20, 64 << 20, np.complex128) as srv:
        ids = [None] * len(reqs)

        def worker(lo):
            for j in range(lo, len(reqs), 3):
                M, k1, st = reqs[j]
                ids[j] = srv.submit(M, k1, st)

        th = [threading.Thread(target=worker, args=(t,)) for t in range(3)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        srv.wait_all(300)
        for rid, (M, k1, st) in zip(ids, reqs):
            done, _, p = srv.poll(rid)
            assert done
            assert_probs_close(p, _expected(M, k1, st))
            srv.release(rid)


def test_admission_rejections():
    with Server(1 << 20, 1 << 20, np.complex128) as srv:
        big = W.random_state(16, np.complex128, 1)  # 2^16 * 40 bytes > 1 MiB
        with pytest.raises(QsimError) as e:
            srv.submit(16, big, W.cnot_circuit(16, 4, 1))
        assert e.value.code == -5
        with pytest.raises(QsimError) as e:
            srv.submit(4, W.random_state(4, np.complex128, 1), W.make_steps([(0, 1, 1)]))
        assert e.value.code == -1
        with pytest.raises(QsimError):
            srv.poll(12345)


def _dev_bytes(M, amp=16):
    """Device memory the server reserves for a one-pass request without plan
    tables: the input state and a buffer for the probabilities."""
    a = lambda x: (x + 255) // 256 * 256
    return a((1 << M) * amp) + a((1 << M) * 8)


@pytest.mark.parametrize("backfill_ms", [1e9, -1.0])
def test_backfill_admission(backfill_ms):
    """A request that does not fit while an earlier one runs is passed by
    smaller requests that do (backfill), unless backfill is off; every result
    still matches the oracle."""
    big = [(16, W.random_state(16, np.complex128, 40 + i), W.cnot_circuit(16, 3000, 40 + i))
           for i in range(2)]
    small = [(8, W.random_state(8, np.complex128, 50 + i), W.mixed_circuit(8, 200, 50 + i))
             for i in range(8)]
    budget = _dev_bytes(16) * 3 // 2  # one large request at a time, the small ones beside it
    with Server(budget, 64 << 20, np.complex128) as srv:
        srv.set_backfill(backfill_ms)
        srv.set_paused(True)
        ids = [srv.submit(*r) for r in big + small]  # queue: big, big, small x 8
        srv.set_paused(False)
        srv.wait_all(300)
        st = srv.stats()
        if backfill_ms > 0:
            assert st["backfilled"] >= 1
        else:
            assert st["backfilled"] == 0
        assert st["completed"] == len(ids) and st["peak_in_use_bytes"] <= budget
        for rid, (M, k1, steps) in zip(ids, big + small):
            done, _, p = srv.poll(rid)
            assert done
            assert_probs_close(p, _expected(M, k1, steps))
            srv.release(rid)
        assert st["h2d_bytes"] == sum((1 << M) * 16 for M, _, _ in big + small)
        assert st["d2h_bytes"] == sum((1 << M) * 8 for M, _, _ in big + small)
        assert st["h2d_busy_ms"] > 0 and st["d2h_busy_ms"] > 0 and st["compute_busy_ms"] > 0


def test_trace_records_each_request_in_order():
    reqs = _requests(12, 9, 6, 14)
    with Server(64 << 20, 64 << 20, np.complex128) as srv:
        srv.set_tracing(True)
        ids = [srv.submit(M, k1, st) for M, k1, st in reqs]
        srv.wait_all(300)
        tr = srv.trace()
        assert sorted(tr["id"].tolist()) == sorted(ids)
        for rec in tr:
            assert rec["submit_ms"] <= rec["admit_ms"] <= rec["done_ms"]
            assert 0 <= rec["upload_start_ms"] <= rec["upload_end_ms"]
            assert rec["upload_end_ms"] <= rec["download_start_ms"] <= rec["download_end_ms"]
            if rec["passes"]:
                assert rec["upload_end_ms"] <= rec["compute_start_ms"] <= rec["compute_end_ms"]
                assert rec["compute_end_ms"] <= rec["download_start_ms"]
        assert len(srv.trace()) == 0  # moved out
        for rid in ids:
            srv.release(rid)


def test_served_large_requests_alone_and_in_the_mix():
    """Requests of the serving workload's larger sizes (M = 24, 26, 28:
    states of 0.25-4 GiB, multi-GB device blocks and 64-bit offsets) mixed
    with small ones: sampled probabilities against the oracle's single-row
    evaluation, and each large result bit-identical when served alone."""
    rng = np.random.default_rng(2428)
    big = []
    for i, (M, L) in enumerate([(24, 2600), (26, 1800), (28, 1200)]):
        st = W.cnot_circuit(M, L, 8800 + i) if i != 1 else W.mixed_circuit(M, L, 8800 + i)
        big.append((M, W.random_state(M, np.complex128, 8900 + i), st))
    small = _requests(10, 5, 8, 16)
    reqs = big[:1] + small[:5] + big[1:] + small[5:]
    with Server(24 << 30, 8 << 30, np.complex128) as srv:
        ids = [srv.submit(M, k1, st) for (M, k1, st) in reqs]
        srv.wait_all(600)
        assert srv.stats()["completed"] == len(reqs)
        mixed = {}
        for rid, (M, k1, st) in zip(ids, reqs):
            done, _, p = srv.poll(rid)
            assert done
            if M >= 24:
                rows = rng.integers(0, 1 << M, size=1 << 16, dtype=np.uint64)
                rows[:2] = [0, (1 << M) - 1]
                src = oracle.source_rows(M, st, rows).astype(np.int64)
                assert_probs_close(p[rows.astype(np.int64)], oracle.probabilities(k1[src]))
                mixed[M] = p.copy()
            else:
                assert_probs_close(p, _expected(M, k1, st))
            srv.release(rid)
    for M, k1, st in big:
        with Server(24 << 30, 8 << 30, np.complex128) as srv:
            r = srv.submit(M, k1, st)
            srv.wait_all(300)
            done, _, p = srv.poll(r)
            assert done
            np.testing.assert_array_equal(p, mixed[M])
            srv.release(r)


def test_eviction_makes_room_for_the_head_and_results_stay_exact():
    """Long-running requests fill the HBM budget; a larger request arrives.
    With eviction on, running requests are swapped out to host memory between
    their passes, the newcomer is admitted, and the evicted requests come back
    and finish: every result equals the oracle's and the same requests served
    without eviction, bit for bit."""
    Ms, Mb = 20, 22
    smalls = [(Ms, W.random_state(Ms, np.complex128, 40 + i), W.mixed_circuit(Ms, 400000, 40 + i))
              for i in range(6)]
    big = (Mb, W.random_state(Mb, np.complex128, 77), W.cnot_circuit(Mb, 800, 77))
    reqs = smalls + [big]

    def serve(evict):
        out = {}
        with Server(256 << 20, 512 << 20, np.complex128) as srv:
            srv.set_backfill(-1)
            if evict:
                srv.set_eviction(0.0)
            ids = [srv.submit(M, k1, st) for (M, k1, st) in smalls]
            deadline = time.time() + 60
            while srv.stats()["active"] < len(smalls) and time.time() < deadline:
                time.sleep(0.001)
            ids.append(srv.submit(*big))
            srv.wait_all(600)
            st = srv.stats()
            assert st["completed"] == len(reqs)
            for rid, (M, k1, steps) in zip(ids, reqs):
                done, _, p = srv.poll(rid)
                assert done
                out[rid] = p.copy()
                srv.release(rid)
            assert srv.stats()["host_in_use_bytes"] == 0 and srv.stats()["in_use_bytes"] == 0
        return [out[i] for i in ids], st

    with_ev, st = serve(True)
    assert st["evicted"] >= 1 and st["swapped_in"] == st["evicted"]
    without, st0 = serve(False)
    assert st0["evicted"] == 0
    for a, b in zip(with_ev, without):
        np.testing.assert_array_equal(a, b)
    rng = np.random.default_rng(4040)
    for p, (M, k1, steps) in zip(with_ev, reqs):  # sampled rows: the circuits are long
        rows = rng.integers(0, 1 << M, size=1 << 10, dtype=np.uint64)
        src = oracle.source_rows(M, steps, rows).astype(np.int64)
        assert_probs_close(p[rows.astype(np.int64)], oracle.probabilities(k1[src]))
