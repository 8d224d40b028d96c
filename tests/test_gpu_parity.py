"""GPU parity: the CUDA library through its C ABI against the CPU oracle.

Amplitudes are only moved, so states must match bit for bit; FP64
probabilities match the oracle within 1e-12 relative and two units in the
last place (bit for bit for complex64, whose squares are exact), and the norm
within 1e-12 relative (summation order differs).
Small cases compare every amplitude; the full-size workloads compare sampled
output rows (the oracle evaluates them one at a time) plus permutation
invariants of the whole state computed on the device.
"""
import math

import numpy as np
import pytest

import oracle
from paper_quant_ph_0308158_gb300 import QsimError, Simulator, workloads as W
from tests.helpers import assert_probs_close

pytestmark = pytest.mark.gpu

NORM_RTOL = 1e-12


@pytest.fixture(scope="module", autouse=True)
def cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_quant_ph_0308158_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    return torch


def run(M, dtype, steps, k1, strategy="auto", tile_bits=0, low_bits=0, buffers="torch"):
    with Simulator(M, dtype, buffers=buffers) as sim:
        sim.set_strategy(strategy, tile_bits, low_bits)
        sim.load_state(k1)
        sim.apply(steps)
        out = sim.read_state()
        stats = sim.plan_stats()
    return out, stats


STRATS = ["auto", "sweep", "tile", "gather", "inplace"]


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("strategy", STRATS)
@pytest.mark.parametrize("M,L,seed", [(1, 7, 1), (2, 20, 2), (5, 90, 3), (9, 300, 4),
                                      (12, 333, 5), (14, 260, 6), (17, 200, 7)])
def test_random_circuits_bit_exact(dtype, strategy, M, L, seed):
    steps = W.random_circuit(M, L, seed, max_controls=min(8, M - 1))
    k1 = W.random_state(M, dtype, seed)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    got, _ = run(M, dtype, steps, k1, strategy)
    np.testing.assert_array_equal(got, want)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("k,l", [(6, 1), (8, 3), (10, 4), (11, 5), (12, 2), (13, 5), (14, 4)])
def test_tile_geometries(dtype, k, l):
    M = 18
    steps = W.mixed_circuit(M, 400, 11)
    k1 = W.random_state(M, dtype, 11)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    if np.dtype(dtype).itemsize * (1 << k) > 128 * 1024:
        pytest.skip("tile larger than shared memory")
    got, st = run(M, dtype, steps, k1, "tile", k, l)
    assert st["tile_passes"] == st["passes"] >= 1
    np.testing.assert_array_equal(got, want)


def test_sec2b_worked_example_on_gpu():
    M = 3
    k1 = W.alternating_state(M)
    steps = W.make_steps([(0, 2, 2)])
    want = np.array([1, -1, -1, 1, 1, -1, -1, 1]) / math.sqrt(8)
    for s in STRATS:
        got, _ = run(M, np.complex128, steps, k1, s)
        np.testing.assert_array_equal(got, want.astype(np.complex128))


@pytest.mark.parametrize("M", [20, 26])
def test_sec4_parity_program_closed_form_on_gpu(M):
    k1 = W.alternating_state(M, np.complex64)
    steps = W.parity_circuit(M)
    i = np.arange(1 << M, dtype=np.uint64)
    par = np.zeros_like(i)
    for b in range(M):
        par ^= (i >> np.uint64(b)) & np.uint64(1)
    want = (np.where(par, -1.0, 1.0) / math.sqrt(1 << M)).astype(np.complex64)
    for s in ("auto", "tile", "gather"):
        got, _ = run(M, np.complex64, steps, k1, s)
        np.testing.assert_array_equal(got, want)


def test_edge_cases():
    M = 10
    k1 = W.random_state(M, np.complex128, 3)
    # empty circuit
    got, st = run(M, np.complex128, W.make_steps([]), k1)
    np.testing.assert_array_equal(got, k1)
    assert st["passes"] == 0
    # one NOT on the top bit: contiguous half exchange
    got, _ = run(M, np.complex128, W.make_steps([(M - 1, 0, 0)]), k1, "sweep")
    np.testing.assert_array_equal(got, np.concatenate([k1[512:], k1[:512]]))
    # the maximum number of controls, both polarities
    full = (1 << M) - 1
    for pol in (full & ~1, 0b1010101010 & ~1):
        steps = W.make_steps([(0, full & ~1, pol)])
        want = oracle.apply_circuit(M, k1, steps)
        for s in STRATS:
            got, _ = run(M, np.complex128, steps, k1, s)
            np.testing.assert_array_equal(got, want)
    # adjacent equal steps cancel to the identity, and apply when asked to
    steps = W.make_steps([(3, 1, 1), (3, 1, 1)])
    got, st = run(M, np.complex128, steps, k1)
    np.testing.assert_array_equal(got, k1)
    assert st["steps_cancelled"] == 2
    with Simulator(M, np.complex128) as sim:
        sim.set_canonicalize(False)
        sim.load_state(k1)
        sim.apply(steps)
        np.testing.assert_array_equal(sim.read_state(), k1)
        assert sim.plan_stats()["steps_cancelled"] == 0


def test_invalid_circuit_leaves_state_untouched():
    M = 8
    k1 = W.random_state(M, np.complex64, 2)
    with Simulator(M, np.complex64) as sim:
        sim.load_state(k1)
        bad = W.make_steps([(0, 2, 2), (1, 2, 2)])
        with pytest.raises(QsimError) as e:
            sim.apply(bad)
        assert e.value.code == -1
        np.testing.assert_array_equal(sim.read_state(), k1)
        with pytest.raises(QsimError):
            sim.load_state(k1[:-1])


def test_library_buffers_and_repeated_applies():
    M = 15
    steps = W.mixed_circuit(M, 300, 9)
    k1 = W.random_state(M, np.complex128, 9)
    want = oracle.apply_circuit(M, oracle.apply_circuit(M, k1, steps), steps)
    for buffers in ("torch", "library"):
        with Simulator(M, np.complex128, buffers=buffers) as sim:
            sim.load_state(k1)
            sim.apply(steps)
            sim.apply(steps)
            np.testing.assert_array_equal(sim.read_state(), want)
    with Simulator(M, np.complex128, buffers="library", scratch=False) as sim:
        sim.load_state(k1)
        sim.apply(steps)
        assert sim.plan_stats()["gather_passes"] == 0


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("M", [1, 7, 16, 25])
def test_probabilities_fp64(dtype, M):
    k1 = W.random_state(M, dtype, M)
    steps = W.random_circuit(M, 50, M)
    want_state = oracle.apply_circuit(M, k1, steps)
    want = oracle.probabilities(want_state)
    with Simulator(M, dtype) as sim:
        sim.load_state(k1)
        sim.apply(steps)
        p, norm = sim.probabilities(with_norm=True)
    assert_probs_close(p, want)
    ref = oracle.fsum_pairwise(want)
    assert abs(norm - ref) <= NORM_RTOL * ref
    assert abs(norm - 1.0) < 1e-6 if dtype == np.complex64 else abs(norm - 1.0) < 1e-12


def test_complex64_probabilities_bit_identical_including_special_values():
    """complex64 squares are exact in FP64, so the only rounding is the sum:
    the device must agree with the oracle bit for bit, also for zeros of
    either sign, subnormals, the largest and smallest normals, infinities
    and NaNs (a state of 'arbitrary magnitude', Sec. 1)."""
    M = 14
    f32 = np.finfo(np.float32)
    special = np.array([0.0, -0.0, 1.0, -1.5, f32.max, -f32.max, f32.tiny, -f32.tiny,
                        f32.smallest_subnormal, 3 * f32.smallest_subnormal,
                        np.float32(1e-40), np.inf, -np.inf, np.nan, 2.0 ** -75, 2.0 ** 63],
                       dtype=np.float32)
    rng = np.random.default_rng(11)
    parts = rng.standard_normal(2 << M).astype(np.float32)
    parts *= np.exp2(rng.integers(-140, 120, size=parts.size)).astype(np.float32)
    parts[rng.integers(0, parts.size, size=4096)] = rng.choice(special, size=4096)
    k1 = parts.view(np.complex64)

    def same(got, want):
        np.testing.assert_array_equal(got.view(np.uint64)[~np.isnan(want)],
                                      want.view(np.uint64)[~np.isnan(want)])
        assert np.array_equal(np.isnan(got), np.isnan(want))

    with Simulator(M, np.complex64) as sim:
        sim.load_state(k1)
        same(sim.probabilities(), oracle.probabilities(k1))
    # the same arithmetic where a tile or compiled-gather pass writes them
    import torch
    steps = W.random_circuit(M, 64, 12, max_controls=3)
    want = oracle.probabilities(oracle.apply_circuit(M, k1, steps).astype(np.complex64))
    for strategy, jit in (("tile", False), ("gather", True), ("gather", False)):
        out = torch.empty(1 << M, dtype=torch.float64, device="cuda")
        with Simulator(M, np.complex64) as sim:
            sim.set_strategy(strategy)
            sim.set_jit(jit)
            sim.load_state(k1)
            sim.apply_probabilities(steps, out.data_ptr())
            sim.synchronize()
        same(out.cpu().numpy(), want)


# ----------------------------------------------------------------------------
# full-size workloads
# ----------------------------------------------------------------------------

def _device_hash(t):
    """Order-independent sums over the state's 64-bit words (wrapping)."""
    import torch
    w = t.view(torch.int64)
    return int(w.sum().item()), int((w * (w | 1)).sum().item())


def test_small_cnot_workload_full_state():
    cfg = W.config_small_cnot()
    M, steps = cfg["M"], cfg["steps"]
    for k1 in (W.random_state(M, np.complex128, cfg["state_seed"]), W.alternating_state(M)):
        want = oracle.apply_circuit(M, k1, steps)
        for s in STRATS:
            got, _ = run(M, np.complex128, steps, k1, s)
            np.testing.assert_array_equal(got, want)


def _sampled_check(cfg, strategy, rows=1 << 20, jit=False, probs=False):
    """Run a full-size workload through the C ABI and compare sampled output
    rows bit for bit with the oracle's single-row evaluation k2(i) = k1(x(i))
    (Sec. 2h product, Sec. 2b gather), plus order-independent sums of the
    whole state before and after.  With probs the circuit runs through
    qsim_apply_circuit_probabilities, as the benchmark does, and the sampled
    FP64 probabilities are compared with the oracle's.  Returns the plan
    statistics and the kernels that ran."""
    import torch
    M, dtype, steps = cfg["M"], cfg["dtype"], cfg["steps"]
    k1 = W.random_state(M, dtype, cfg["state_seed"])
    rng = np.random.default_rng(12345)
    r = rng.integers(0, 1 << M, size=rows, dtype=np.uint64)
    r[:4] = [0, 1, (1 << M) - 2, (1 << M) - 1]
    src = oracle.source_rows(M, steps, r).astype(np.int64)
    want = k1[src]
    ridx = torch.from_numpy(r.astype(np.int64)).cuda()
    with Simulator(M, dtype, scratch=(strategy != "inplace")) as sim:
        sim.set_strategy(strategy)
        sim.set_canonicalize(False)
        sim.set_jit(jit)
        sim.set_profiling(True)
        sim.load_state(k1)
        h0 = _device_hash(sim.state_tensor())
        p_dev = None
        if probs:
            p_dev = torch.full((1 << M,), -1.0, dtype=torch.float64, device="cuda")
            sim.apply_probabilities(steps, p_dev.data_ptr())
        else:
            sim.apply(steps)
        sim.synchronize()
        kernels = [k for k, _, _ in sim.pass_times()]
        t = sim.state_tensor()
        got = t[ridx].cpu().numpy()
        h1 = _device_hash(t)
        got_p = p_dev[ridx].cpu().numpy() if probs else None
        stats = sim.plan_stats()
        del p_dev
    np.testing.assert_array_equal(got, want)
    assert h0 == h1
    if probs:
        want_p = oracle.probabilities(want)
        if np.dtype(dtype) == np.complex64:  # exact squares: identical bits
            np.testing.assert_array_equal(got_p.view(np.uint64), want_p.view(np.uint64))
        else:
            assert_probs_close(got_p, want_p)
    return stats, kernels


def test_mixed_m28_workload_sampled():
    """M=28 complex128, 1000 mixed steps, bit-sliced interpreter
    (gather_sliced_kernel: compiled kernels off)."""
    st, kernels = _sampled_check(W.config_mixed_m28(), "auto")
    assert st["gather_passes"] >= 1
    assert "gather_sliced_kernel" in kernels


def test_mixed_m28_benchmarked_launch_sampled():
    """The benchmarked launch of the M=28 complex128 1000-step mixed workload:
    compiled gather (qsim_jit_gather), no cancellation, probabilities written
    by the same pass -- sampled rows bit-exact, probabilities within 1e-12
    and 2 ulp of the oracle's."""
    st, kernels = _sampled_check(W.config_mixed_m28(), "auto", jit=True, probs=True)
    assert st["passes"] == 1 and st["gather_passes"] == 1
    assert kernels == ["qsim_jit_gather"]


def test_mixed_m28_workload_inplace_sampled():
    st, _ = _sampled_check(W.config_mixed_m28(), "inplace")
    assert st["gather_passes"] == 0


def test_adder_m32_workload_sampled():
    """M=32 complex64 (32 GiB) adder, in place, tile passes (compiled kernels
    off), the last one also writing the FP64 probabilities (bit-exact for
    complex64, whose squares are exact)."""
    st, kernels = _sampled_check(W.config_adder_m32(), "inplace", rows=1 << 18, probs=True)
    assert st["gather_passes"] == 0 and st["passes"] >= 1
    assert set(kernels) <= {"tile_kernel", "sweep_kernel"} and kernels[-1] == "tile_kernel"


def test_adder_m32_benchmarked_closed_pass_sampled():
    """M=32 complex64 adder in place as benchmarked: compiled kernels on, so
    the whole circuit is one closed tile pass (its net map changes only
    b_4..b_14 and the carry-out), which also writes the probabilities."""
    st, kernels = _sampled_check(W.config_adder_m32(), "inplace", rows=1 << 20, jit=True, probs=True)
    assert st["passes"] == 1 and kernels == ["qsim_jit_closed"]


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
def test_hybrid_plan_full_state(dtype):
    """A plan that mixes strategies per segment (tile passes, then a coset
    gather): every amplitude against the oracle."""
    cfg = W.config_hybrid(18, dtype=dtype)
    M, steps = cfg["M"], cfg["steps"]
    k1 = W.random_state(M, dtype, cfg["state_seed"])
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    with Simulator(M, dtype) as sim:
        sim.set_canonicalize(False)
        sim.set_profiling(True)
        sim.load_state(k1)
        sim.apply(steps)
        got = sim.read_state()
        kernels = [k for k, _, _ in sim.pass_times()]
    np.testing.assert_array_equal(got, want)
    assert len(kernels) >= 2 and kernels[-1] == "gather_coset_kernel"


def test_hybrid_m28_workload_sampled():
    """The M=28 complex128 hybrid workload as benchmarked (closed passes over
    the register's tile, one coset gather writing the probabilities)."""
    st, kernels = _sampled_check(W.config_hybrid(), "auto", jit=True, probs=True)
    assert st["tile_passes"] >= 1 and st["gather_passes"] == 1
    assert kernels[-1] == "gather_coset_kernel" and "qsim_jit_closed" in kernels


def test_sec4_parity_m32_from_qubits_with_probabilities(cuda):
    """The Sec. 4 example at M = 32 as the benchmark runs it: the alternating
    input generated from its qubits (App. 1), the parity program in place,
    probabilities written by the pass.  Closed form: k2(i) =
    (-1)^popcount(i) / 2^16 for every row (checked on the device, plus sampled
    rows against the oracle's single-row evaluation), p(i) = 2^-32 exactly."""
    torch = cuda
    M = 32
    cfg = W.config_parity(M)
    steps = cfg["steps"]
    probs = torch.empty(1 << M, dtype=torch.float64, device="cuda")
    with Simulator(M, np.complex64, scratch=False) as sim:
        sim.set_strategy("inplace")
        sim.load_product_state(cfg["qubits"])
        sim.apply_probabilities(steps, probs.data_ptr())
        sim.synchronize()
        assert sim.plan_stats()["passes"] == 1
        st = sim.state_tensor().view(torch.float32).view(-1, 2)
        assert bool((st[:, 1] == 0).all())
        re = st[:, 0]
        assert bool((re.abs() == 2.0 ** -16).all())
        # the sign is the parity of the row: spot-check blocks and random rows
        rng = np.random.default_rng(32)
        rows = np.concatenate([np.arange(4096, dtype=np.uint64),
                               rng.integers(0, 1 << M, size=1 << 16, dtype=np.uint64)])
        got = re[torch.from_numpy(rows.astype(np.int64)).cuda()].cpu().numpy()
        src = oracle.source_rows(M, steps, rows)  # k2(i) = k1(x(i)), k1 alternating
        want = np.where((src & 1).astype(bool), -1.0, 1.0) * 2.0 ** -16
        np.testing.assert_array_equal(got, want.astype(np.float32))
        par = np.zeros_like(rows)
        for b in range(M):
            par ^= (rows >> np.uint64(b)) & np.uint64(1)
        np.testing.assert_array_equal(got, np.where(par.astype(bool), -1.0, 1.0).astype(np.float32) * 2.0 ** -16)
        assert bool((probs == 2.0 ** -32).all())


# ----------------------------------------------------------------------------
# circuit-specialised (compiled) gather kernels and 64-bit indices
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("M,L,seed", [(10, 40, 1), (13, 300, 2), (17, 257, 3), (20, 1000, 4)])
def test_compiled_gather_bit_exact(dtype, M, L, seed):
    steps = W.random_circuit(M, L, seed, max_controls=min(8, M - 1))
    k1 = W.random_state(M, dtype, seed)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    with Simulator(M, dtype) as sim:
        sim.set_strategy("gather")
        sim.set_jit(True)
        sim.set_profiling(True)
        sim.load_state(k1)
        sim.apply(steps)
        got = sim.read_state()
        kernels = {k for k, _, _ in sim.pass_times()}
    np.testing.assert_array_equal(got, want)
    assert "qsim_jit_gather" in kernels


# (strategy, jit, circuit) -> kernel of the last pass, which writes the probabilities
FUSED_CASES = [
    ("tile", False, "mixed", "tile_kernel"),
    ("inplace", False, "mixed", "tile_kernel"),
    ("gather", False, "cnot", "gather_coset_kernel"),
    ("gather", "nocoset", "cnot", "gather_affine_kernel"),
    ("gather", False, "mixed", "gather_sliced_kernel"),
    ("gather", True, "mixed", "qsim_jit_gather"),
    ("sweep", False, "mixed", "probs_kernel"),  # a sweep cannot: separate pass
]


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("strategy,jit,mix,kernel", FUSED_CASES)
@pytest.mark.parametrize("M", [10, 17])  # compiled gathers start at M = 10
def test_apply_circuit_probabilities(cuda, dtype, strategy, jit, mix, kernel, M):
    """Probabilities written by the last pass equal the separate probability
    pass bit for bit and the oracle's within the contract; the state is
    bit-exact."""
    torch = cuda
    L = 120
    seed = 70 + M
    if mix == "cnot":
        steps = W.cnot_circuit(M, L, seed)
    else:
        steps = W.random_circuit(M, L, seed, max_controls=min(5, M - 1))
    k1 = W.random_state(M, dtype, seed)
    want_state = oracle.apply_circuit(M, k1, steps)
    want_p = oracle.probabilities(want_state.astype(dtype))
    fused = torch.full((1 << M,), -1.0, dtype=torch.float64, device="cuda")
    plain = torch.empty(1 << M, dtype=torch.float64, device="cuda")
    with Simulator(M, dtype) as sim:
        sim.set_strategy(strategy)
        sim.set_jit(jit is True)
        sim.set_coset(jit != "nocoset")
        sim.set_canonicalize(False)
        sim.set_profiling(True)
        sim.load_state(k1)
        sim.apply_probabilities(steps, fused.data_ptr())
        kernels = [k for k, _, _ in sim.pass_times()]
        got_state = sim.read_state()
        sim.probabilities_device(plain.data_ptr())
        sim.synchronize()
    np.testing.assert_array_equal(got_state, want_state.astype(dtype))
    assert kernels[-1] == kernel
    assert kernels.count("probs_kernel") == (1 if kernel == "probs_kernel" else 0)
    f = fused.cpu().numpy()
    np.testing.assert_array_equal(f.view(np.uint64), plain.cpu().numpy().view(np.uint64))
    if dtype == np.complex64:
        np.testing.assert_array_equal(f.view(np.uint64), want_p.view(np.uint64))
    else:
        assert_probs_close(f, want_p)


def test_apply_circuit_probabilities_idle_tiles_and_empty_circuit(cuda):
    """A tile pass whose steps fire on a few tiles only must still write the
    probabilities of every tile; an empty circuit runs the probability pass."""
    torch = cuda
    M = 18
    # Toffoli and 3-control steps on low targets controlled by the top bits:
    # most tiles have no active step
    steps = W.make_steps([(0, (1 << 17) | (1 << 16), (1 << 17) | (1 << 16)),
                          (3, (1 << 17) | (1 << 16) | (1 << 15), (1 << 17) | (1 << 16) | (1 << 15)),
                          (1, 1 << 17, 0)])
    for dtype in (np.complex64, np.complex128):
        k1 = W.random_state(M, dtype, 5)
        want_state = oracle.apply_circuit(M, k1, steps).astype(dtype)
        want_p = oracle.probabilities(want_state)
        for circuit, strategy in ((steps, "tile"), (steps[:0], "auto")):
            out = torch.full((1 << M,), -1.0, dtype=torch.float64, device="cuda")
            with Simulator(M, dtype) as sim:
                sim.set_strategy(strategy)
                sim.load_state(k1)
                sim.apply_probabilities(circuit, out.data_ptr())
                sim.synchronize()
                state = sim.read_state()
            ref_state = want_state if len(circuit) else k1
            ref_p = want_p if len(circuit) else oracle.probabilities(k1)
            np.testing.assert_array_equal(state, ref_state)
            assert_probs_close(out.cpu().numpy(), ref_p)


def test_apply_circuit_probabilities_rejects_bad_output(cuda):
    torch = cuda
    with Simulator(8, np.complex128) as sim:
        buf = torch.empty(257, dtype=torch.float64, device="cuda")
        with pytest.raises(QsimError):
            sim.apply_probabilities(W.cnot_circuit(8, 4, 1), 0)
        with pytest.raises(QsimError):
            sim.apply_probabilities(W.cnot_circuit(8, 4, 1), buf.data_ptr() + 4)


def test_complex64_probabilities_any_8_byte_offset(cuda):
    """complex64 probabilities into a buffer on a 16-byte boundary and one 8
    bytes past it (the 16-byte pair stores are used only where both buffers
    allow them): bit-identical to the oracle either way, nothing written
    outside the 2^M entries."""
    torch = cuda
    for M in (1, 5, 16):
        k1 = W.random_state(M, np.complex64, 21 + M)
        want = oracle.probabilities(k1)
        buf = torch.full((2 + (1 << M) + 2,), -1.0, dtype=torch.float64, device="cuda")
        for off in (2, 1):   # 16-byte and 8-byte aligned starts
            buf.fill_(-1.0)
            with Simulator(M, np.complex64) as sim:
                sim.load_state(k1)
                sim.apply_probabilities(W.make_steps([]), buf.data_ptr() + 8 * off)
                sim.synchronize()
            got = buf.cpu().numpy()
            np.testing.assert_array_equal(got[off:off + (1 << M)].view(np.uint64), want.view(np.uint64))
            assert (got[:off] == -1.0).all() and (got[off + (1 << M):] == -1.0).all()


def test_wide_indices_m33():
    """M = 33 complex64 (64 GiB + 64 GiB scratch): 64-bit index paths of the
    compiled, bit-sliced, affine, tile and sweep kernels, checked on sampled
    rows and by running the reversed circuit back to the input."""
    import torch
    M, dtype = 33, np.complex64
    steps = W.mixed_circuit(M, 300, 33)
    cnots = W.cnot_circuit(M, 100, 34)
    k1 = W.random_state(M, dtype, 33)
    rng = np.random.default_rng(33)
    rows = rng.integers(0, 1 << M, size=1 << 17, dtype=np.uint64)
    rows[:2] = [(1 << M) - 1, 1 << 32]
    ridx = torch.from_numpy(rows.astype(np.int64)).cuda()
    with Simulator(M, dtype) as sim:
        sim.set_canonicalize(False)
        sim.load_state(k1)
        sim.set_strategy("gather")
        sim.set_jit(True)
        sim.apply(steps)                           # compiled gather
        sim.synchronize()
        src = oracle.source_rows(M, steps, rows).astype(np.int64)
        np.testing.assert_array_equal(sim.state_tensor()[ridx].cpu().numpy(), k1[src])
        sim.set_jit(False)
        sim.apply(cnots)                           # coset-blocked affine gather
        sim.set_coset(False)
        sim.apply(np.concatenate([cnots[::-1], cnots]))  # identity, direct affine gather
        sim.set_coset(True)
        sim.synchronize()
        both = np.concatenate([steps, cnots])
        src = oracle.source_rows(M, both, rows).astype(np.int64)
        np.testing.assert_array_equal(sim.state_tensor()[ridx].cpu().numpy(), k1[src])
        sim.apply(both[::-1][:150].copy())         # bit-sliced gather (cnots + 50 steps)
        sim.set_strategy("inplace")
        sim.apply(both[::-1][150:].copy())         # tile / sweep passes, in place
        sim.synchronize()
        np.testing.assert_array_equal(sim.state_tensor()[ridx].cpu().numpy(), k1[rows.astype(np.int64)])


# ----------------------------------------------------------------------------
# App. 1: the input generated on the device from M qubits
# ----------------------------------------------------------------------------

# The device multiplies (high-bit partial product) x (low-bit partial product)
# while the oracle multiplies the factors one by one from the top: at most
# M complex products, each correctly rounded per real operation, so the two
# differ by far less than 1e-13 of |k1(i)| in FP64.
PRODUCT_RTOL = 1e-13


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("M", [1, 5, 10, 11, 16, 23])
def test_product_state_input(dtype, M):
    rng = np.random.default_rng(100 + M)
    q = rng.normal(size=(M, 2)) + 1j * rng.normal(size=(M, 2))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    want = oracle.product_state(M, q)
    with Simulator(M, dtype) as sim:
        sim.load_product_state(q)
        got = sim.read_state().astype(np.complex128)
    if dtype == np.complex128:
        assert np.all(np.abs(got - want) <= PRODUCT_RTOL * np.abs(want) + 1e-300)
    else:  # rounded once to complex64 at the end: within one float ulp per part
        w = want.astype(np.complex64).astype(np.complex128)
        tol = np.spacing(np.abs(w.real).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(got.real - w.real) <= tol)
        tol = np.spacing(np.abs(w.imag).astype(np.float32)).astype(np.float64)
        assert np.all(np.abs(got.imag - w.imag) <= tol)


def test_product_state_exact_cases_and_sec4_input():
    # integer components: every product is exact on both sides
    M = 12
    rng = np.random.default_rng(5)
    q = rng.integers(-2, 3, size=(M, 2)) + 1j * rng.integers(-2, 3, size=(M, 2))
    with Simulator(M, np.complex128) as sim:
        sim.load_product_state(q)
        np.testing.assert_array_equal(sim.read_state(), oracle.product_state(M, q))
    # Sec. 4: (1, -1, 1, -1, ...)/sqrt(2^M) is the product of (1, -1)/sqrt2 on
    # a(1) and (1, 1)/sqrt2 elsewhere (1/sqrt2 is itself rounded, so the
    # product carries M rounding errors of the factor)
    M = 16
    q = W.sec4_qubits(M)
    with Simulator(M, np.complex128) as sim:
        sim.load_product_state(q)
        got = sim.read_state()
    np.testing.assert_allclose(got, W.alternating_state(M), rtol=PRODUCT_RTOL, atol=0)
    np.testing.assert_allclose(got, oracle.product_state(M, q), rtol=PRODUCT_RTOL, atol=0)


# ----------------------------------------------------------------------------
# the row array of the product (Sec. 2h), kept as "information about the unitary"
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("M,L,seed", [(1, 3, 1), (3, 10, 2), (12, 500, 3), (20, 300, 4)])
def test_row_array_equals_the_sec2h_product(M, L, seed):
    import torch
    steps = W.random_circuit(M, L, seed, max_controls=min(8, M - 1))
    rows = torch.empty(1 << M, dtype=torch.int64, device="cuda")
    with Simulator(M, np.complex64) as sim:
        sim.row_array(steps, rows.data_ptr())
        sim.synchronize()
    np.testing.assert_array_equal(rows.cpu().numpy(), oracle.gather_map(M, steps))


def test_row_array_rejects_steps_beyond_eight_controls():
    import torch
    M = 12
    rows = torch.empty(1 << M, dtype=torch.int64, device="cuda")
    with Simulator(M, np.complex64) as sim:
        with pytest.raises(QsimError) as e:
            sim.row_array(W.make_steps([(0, 0b1111111110, 0b1111111110)]), rows.data_ptr())
        assert "more than 8 controls" in str(e.value)


def test_async_load_and_probabilities_on_two_contexts():
    """The copy-in / copy-out calls queued without waiting, alternating two
    contexts on two streams as the end-to-end benchmark does."""
    import torch
    M = 18
    steps = W.mixed_circuit(M, 300, 21)
    states = [W.random_state(M, np.complex128, 21 + i) for i in range(4)]
    want = [oracle.probabilities(oracle.apply_circuit(M, k, steps)) for k in states]
    s2 = torch.cuda.Stream()
    with Simulator(M, np.complex128) as a:
        with torch.cuda.stream(s2):
            b = Simulator(M, np.complex128)
        sims = (a, b)
        outs = [np.zeros(1 << M) for _ in range(8)]
        for i in range(8):  # separate probability pass, then fused into the circuit's pass
            sm = sims[i & 1]
            if i >= 2:
                sm.synchronize()
            sm.load_state_async(states[i % 4])
            if i < 4:
                sm.apply(steps)
                sm.probabilities_async(outs[i])
            else:
                sm.apply_probabilities_async(steps, outs[i])
        for sm in sims:
            sm.synchronize()
        b.close()
    for i in range(8):
        assert_probs_close(outs[i], want[i % 4])
    # back-to-back asynchronous reads on one context reuse its buffer safely
    with Simulator(M, np.complex128) as a:
        r = [np.zeros(1 << M) for _ in range(3)]
        a.load_state(states[0])
        a.probabilities_async(r[0])
        a.apply_probabilities_async(steps, r[1])
        a.apply_probabilities_async(steps[::-1], r[2])
        a.synchronize()
    assert_probs_close(r[0], oracle.probabilities(states[0]))
    assert_probs_close(r[1], want[0])
    assert_probs_close(r[2], oracle.probabilities(states[0]))


# ----------------------------------------------------------------------------
# autotuning
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("dtype,M,L,scratch", [(np.complex128, 18, 300, True),
                                               (np.complex64, 20, 200, False),
                                               (np.complex128, 12, 40, True)])
def test_autotune_keeps_the_state_and_picks_a_working_plan(dtype, M, L, scratch):
    steps = W.mixed_circuit(M, L, seed=M)
    k1 = W.random_state(M, dtype, M)
    want = oracle.apply_circuit(M, k1, steps).astype(dtype)
    with Simulator(M, dtype, scratch=scratch) as sim:
        sim.load_state(k1)
        res = sim.autotune(steps, reps=1)
        np.testing.assert_array_equal(sim.read_state(), k1)  # forward + reverse = identity
        ran = [r for r in res if r["ms"] >= 0]
        assert ran and ran == sorted(ran, key=lambda r: r["ms"])
        assert any(r["strategy"] == "tile" for r in ran)
        assert scratch == any(r["strategy"] == "gather" for r in res)
        sim.apply(steps)  # with the plan the tuner kept
        np.testing.assert_array_equal(sim.read_state(), want)
        with pytest.raises(QsimError):
            sim.autotune(steps, reps=0)


# ----------------------------------------------------------------------------
# App. 1 input fused into the first pass (qsim_apply_circuit_product)
# ----------------------------------------------------------------------------

def _assert_close_to_product(got, want, dtype):
    """complex128: within 1e-13 of |k| (as the product-state input);
    complex64: per part within one float ulp of the oracle's value rounded to
    float, plus 2^-42 |k| for the float-float arithmetic: the FP64 partial
    products are split into float-float (2^-48 relative each), the tile's
    factor times the high-bit product and that times the low-bit product are
    float-float complex products (each within about 2^-45 of |k|, as a part
    of a complex product can cancel), so three stages stay under 2^-43."""
    got = got.astype(np.complex128)
    if dtype == np.complex128:
        assert np.all(np.abs(got - want) <= PRODUCT_RTOL * np.abs(want) + 1e-300)
        return
    w = want.astype(np.complex64).astype(np.complex128)
    slack = 2.0 ** -42 * np.abs(want)
    for g, ww in ((got.real, w.real), (got.imag, w.imag)):
        tol = np.spacing(np.abs(ww).astype(np.float32)).astype(np.float64) + slack
        assert np.all(np.abs(g - ww) <= tol)


@pytest.mark.parametrize("dtype", [np.complex64, np.complex128])
@pytest.mark.parametrize("M,seed", [(12, 1), (16, 2), (20, 3), (23, 4)])
def test_product_input_fused_into_the_first_tile_pass(cuda, dtype, M, seed):
    torch = cuda
    rng = np.random.default_rng(300 + M)
    q = rng.normal(size=(M, 2)) + 1j * rng.normal(size=(M, 2))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    steps = np.concatenate([W.local_mixed_circuit(M, 150, seed, min(10, M)),
                            W.mixed_circuit(M, 100, seed)])
    want = oracle.apply_circuit(M, oracle.product_state(M, q), steps)
    p = torch.full((1 << M,), -1.0, dtype=torch.float64, device="cuda")
    with Simulator(M, dtype, scratch=False) as sim:
        sim.set_strategy("inplace")
        sim.set_canonicalize(False)
        sim.set_profiling(True)
        sim.load_state(W.random_state(M, dtype, 9))  # overwritten by the product input
        sim.apply_product(q, steps, p.data_ptr())
        kernels = [k for k, _, _ in sim.pass_times()]
        got = sim.read_state()
    assert kernels[0] == "tile_kernel"
    if kernels[-1] != "probs_kernel":  # a plan ending in a sweep needs the separate pass
        assert "probs_kernel" not in kernels
    _assert_close_to_product(got, want, dtype)
    # the probabilities are those of the amplitudes stored
    assert_probs_close(p.cpu().numpy(), oracle.probabilities(got))


def test_product_input_falls_back_when_the_plan_starts_with_a_gather():
    M = 14
    rng = np.random.default_rng(14)
    q = rng.normal(size=(M, 2)) + 1j * rng.normal(size=(M, 2))
    steps = W.mixed_circuit(M, 400, 14)
    want = oracle.apply_circuit(M, oracle.product_state(M, q), steps)
    with Simulator(M, np.complex128) as sim:
        sim.set_strategy("gather")
        sim.set_profiling(True)
        sim.apply_product(q, steps)
        kernels = [k for k, _, _ in sim.pass_times()]
        got = sim.read_state()
    assert kernels[0] != "tile_kernel"
    _assert_close_to_product(got, want, np.complex128)


@pytest.mark.parametrize("jit", [False, True])
def test_sec4_parity_m32_fused_product_input(cuda, jit):
    """The Sec. 4 example at M = 32 from its qubits (App. 1): with compiled
    kernels off, the input is generated inside the one tile pass; with them on
    (as benchmarked: AUTO with a scratch buffer), the planner writes the input
    with the product-state kernel and runs one closed pass.  Every amplitude
    (-1)^popcount(i) / 2^16 exactly (checked on the device), every
    probability exactly 2^-32."""
    torch = cuda
    M = 32
    cfg = W.config_parity(M)
    probs = torch.empty(1 << M, dtype=torch.float64, device="cuda")
    with Simulator(M, np.complex64, scratch=jit) as sim:
        sim.set_strategy("auto" if jit else "inplace")
        sim.set_jit(jit)
        sim.set_canonicalize(False)
        sim.set_profiling(True)
        sim.apply_product(cfg["qubits"], cfg["steps"], probs.data_ptr())
        sim.synchronize()
        assert [k for k, _, _ in sim.pass_times()] == (["qsim_jit_closed"] if jit else ["tile_kernel"])
        st = sim.state_tensor().view(torch.float32).view(-1, 2)
        assert bool((st[:, 1] == 0).all())
        re = st[:, 0]
        assert bool((re.abs() == 2.0 ** -16).all())
        rng = np.random.default_rng(3232)
        rows = rng.integers(0, 1 << M, size=1 << 16, dtype=np.uint64)
        got = re[torch.from_numpy(rows.astype(np.int64)).cuda()].cpu().numpy()
        par = np.zeros_like(rows)
        for b in range(M):
            par ^= (rows >> np.uint64(b)) & np.uint64(1)
        np.testing.assert_array_equal(got, np.where(par.astype(bool), -1.0, 1.0).astype(np.float32) * 2.0 ** -16)
        assert bool((probs == 2.0 ** -32).all())
