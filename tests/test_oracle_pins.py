"""Pins for the CPU oracle: values the paper prints, closed forms, textbook
constructions and invariants -- none of them re-types the oracle's loop.

Paper: J. R. Burger, "New approaches to quantum computer simulation in a
classical supercomputer".  Each test names the passage it pins.
"""
import math

import numpy as np
import pytest

import oracle
from paper_quant_ph_0308158_gb300 import workloads as W
from tests import golden_io


# ----------------------------------------------------------------------------
# values printed in the paper
# ----------------------------------------------------------------------------

def test_sec2b_worked_example_all_oracle_routes():
    """Sec. 2b: alternating input through 'a(2) controls a(1)' (printed k2)."""
    g = golden_io.read("sec2b_worked_example.txt")
    M, steps = g["M"], g["steps"]
    s = 1.0 / math.sqrt(2 ** M)
    k1 = (g["k1"] * s).astype(np.complex128)
    want = (g["k2"] * s).astype(np.complex128)
    np.testing.assert_array_equal(oracle.apply_circuit(M, k1, steps), want)
    np.testing.assert_array_equal(oracle.sparse_matrix_method(M, k1, steps), want)
    rows = np.arange(2 ** M, dtype=np.uint64)
    np.testing.assert_array_equal(k1[oracle.source_rows(M, steps, rows).astype(np.int64)], want)
    y = oracle.step_row_array(M, steps[0])
    np.testing.assert_array_equal(y, g["y"].astype(np.int64))
    inter = [(i, int(y[i])) for i in range(2 ** M) if y[i] > i]
    assert inter == g["interchanges"]


def test_sec2h_figure2_running_products():
    """Sec. 2h: row arrays of H1, H2, H3 and the running product x(i)=y(x(i))."""
    g = golden_io.read("sec2h_figure2_products.txt")
    M, steps = g["M"], g["steps"]
    for s in range(3):
        y = oracle.step_row_array(M, steps[s])
        np.testing.assert_array_equal(y[:4] + 1, g["y%d" % (s + 1)].astype(np.int64))
        x = oracle.paper_product(M, steps[: s + 1])
        np.testing.assert_array_equal(x[:4] + 1, g["x%d" % (s + 1)].astype(np.int64))
    x = oracle.paper_product(M, steps)
    inter = [(i, int(x[i])) for i in range(2 ** M) if x[i] > i]
    assert inter == g["interchanges"]


def test_sec2_block_rules():
    """Sec. 2b (from=3, goto=1), 2c (quadruples, +/-2), 2e (NOT), 2f (from<goto)."""
    g = golden_io.read("sec2_block_rules.txt")
    M = g["M"]
    for t, c, p, *y in g["case"]:
        st = W.make_steps([(t, c, p)])
        np.testing.assert_array_equal(oracle.step_row_array(M, st[0]), np.array(y))


def test_figure2_circuit_equals_negative_polarity_cnot():
    """NOT a(2); a(2) controls a(1); NOT a(2) acts as 'a(2)=0 controls a(1)'."""
    g = golden_io.read("sec2h_figure2_products.txt")
    neg = W.make_steps([(0, 2, 0)])
    for M in (3, 6):
        k = W.random_state(M, np.complex128, seed=11)
        np.testing.assert_array_equal(oracle.apply_circuit(M, k, g["steps"]),
                                      oracle.apply_circuit(M, k, neg))


# ----------------------------------------------------------------------------
# composition order (reading of Sec. 2h) -- pinned by the definition
# ----------------------------------------------------------------------------

def test_product_order_reading_non_palindromic():
    """k2 = U_2 U_1 k1 for 'a(1) controls a(2)' then 'a(2) controls a(1)'.

    The textbook matrix product decides: the literal Sec. 2h rule in circuit
    order gives the inverse map; fed last-to-first it gives the circuit."""
    M = 2
    steps = W.make_steps([(1, 1, 1), (0, 2, 2)])
    k1 = np.array([1, 2, 3, 4], dtype=np.complex128)
    U = _dense_circuit(M, steps)
    want = U @ k1
    np.testing.assert_array_equal(oracle.apply_circuit(M, k1, steps), want)
    np.testing.assert_array_equal(oracle.gather(M, k1, oracle.gather_map(M, steps)), want)
    literal = oracle.gather(M, k1, oracle.paper_product(M, steps))
    assert not np.array_equal(literal, want)
    np.testing.assert_array_equal(literal, np.linalg.inv(U).real @ k1)


# ----------------------------------------------------------------------------
# Sec. 4 computational example: closed form
# ----------------------------------------------------------------------------

def _popcount(a):
    a = np.asarray(a, dtype=np.uint64)
    c = np.zeros(a.shape, dtype=np.uint64)
    for b in range(64):
        c += (a >> np.uint64(b)) & np.uint64(1)
    return c


@pytest.mark.parametrize("M", [3, 8, 14])
def test_sec4_parity_program_closed_form(M):
    """CNOTs a(j)->a(1), j=2..M, on (1,-1,...)/sqrt(2^M) give (-1)^popcount(i)/sqrt(2^M)."""
    k1 = W.alternating_state(M)
    steps = W.parity_circuit(M)
    i = np.arange(2 ** M, dtype=np.uint64)
    want = np.where(_popcount(i) & np.uint64(1), -1.0, 1.0) / math.sqrt(2 ** M)
    np.testing.assert_array_equal(oracle.apply_circuit(M, k1, steps), want.astype(np.complex128))
    np.testing.assert_array_equal(oracle.sparse_matrix_method(M, k1, steps),
                                  want.astype(np.complex128))


@pytest.mark.parametrize("M", [32, 40])
def test_sec4_parity_program_sampled_rows(M):
    """Same closed form at M = 32 and 40, one output row at a time."""
    rng = np.random.default_rng(M)
    rows = rng.integers(0, 2 ** M, size=20000, dtype=np.uint64)
    src = oracle.source_rows(M, W.parity_circuit(M), rows)
    # input (-1)^(bit 0 of src) must equal (-1)^popcount(row)
    np.testing.assert_array_equal(src & np.uint64(1), _popcount(rows) & np.uint64(1))
    # the program only changes bit 0
    np.testing.assert_array_equal(src >> np.uint64(1), rows >> np.uint64(1))


# ----------------------------------------------------------------------------
# textbook dense matrices (Kronecker products of projectors and X)
# ----------------------------------------------------------------------------

def _dense_step(M, t, C, P):
    """U = I - kron(...) with (I - X) on the target, |p><p| on each control."""
    I2 = np.eye(2)
    IX = np.array([[1.0, -1.0], [-1.0, 1.0]])
    P0 = np.array([[1.0, 0.0], [0.0, 0.0]])
    P1 = np.array([[0.0, 0.0], [0.0, 1.0]])
    K = np.ones((1, 1))
    for b in reversed(range(M)):  # kron order: a(M) ... a(1)
        if b == t:
            f = IX
        elif (C >> b) & 1:
            f = P1 if (P >> b) & 1 else P0
        else:
            f = I2
        K = np.kron(K, f)
    return np.eye(2 ** M) - K


def _dense_circuit(M, steps):
    U = np.eye(2 ** M)
    for s in steps:
        U = _dense_step(M, int(s["target"]), int(s["ctrl_mask"]), int(s["ctrl_pol"])) @ U
    return U


@pytest.mark.parametrize("M,L,seed", [(1, 3, 1), (2, 6, 2), (4, 20, 3), (6, 40, 4), (7, 30, 5)])
def test_dense_matrix_products(M, L, seed):
    """Oracle = textbook product U_L ... U_1 of Kronecker-built step matrices."""
    steps = W.random_circuit(M, L, seed, max_controls=3)
    k1 = W.random_state(M, np.complex128, seed)
    U = _dense_circuit(M, steps)
    want = U.astype(np.complex128) @ k1
    np.testing.assert_array_equal(oracle.apply_circuit(M, k1, steps), want)
    np.testing.assert_array_equal(oracle.sparse_matrix_method(M, k1, steps), want)
    # every step matrix is symmetric with one unit entry per row (Sec. 2a)
    for s in steps[:5]:
        Us = _dense_step(M, int(s["target"]), int(s["ctrl_mask"]), int(s["ctrl_pol"]))
        np.testing.assert_array_equal(Us, Us.T)
        np.testing.assert_array_equal((Us != 0).sum(axis=1), np.ones(2 ** M))
        y = oracle.step_row_array(M, s)
        np.testing.assert_array_equal(np.argmax(Us, axis=1), y)


# ----------------------------------------------------------------------------
# invariants
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("M,seed", [(5, 1), (10, 2), (12, 3)])
def test_involution_reverse_multiset_norm(M, seed):
    steps = W.random_circuit(M, 80, seed)
    k1 = W.random_state(M, np.complex128, seed)
    k2 = oracle.apply_circuit(M, k1, steps)
    # each step undoes itself, so the reversed circuit undoes the circuit
    np.testing.assert_array_equal(oracle.apply_circuit(M, k2, steps[::-1].copy()), k1)
    one = steps[:1]
    np.testing.assert_array_equal(oracle.apply_circuit(M, oracle.apply_circuit(M, k1, one), one), k1)
    # a permutation: same multiset of amplitudes, same norm
    np.testing.assert_array_equal(np.sort_complex(k2), np.sort_complex(k1))
    assert abs(np.vdot(k2, k2).real - 1.0) < 1e-12


@pytest.mark.parametrize("M,seed", [(9, 1), (12, 2)])
def test_source_rows_matches_full_state(M, seed):
    steps = W.random_circuit(M, 60, seed)
    k1 = W.random_state(M, np.complex128, seed)
    k2 = oracle.apply_circuit(M, k1, steps)
    rows = np.arange(2 ** M, dtype=np.uint64)
    src = oracle.source_rows(M, steps, rows).astype(np.int64)
    np.testing.assert_array_equal(k1[src], k2)
    np.testing.assert_array_equal(src, oracle.gather_map(M, steps))


def test_cnot_circuits_equal_their_gf2_affine_map():
    """CNOT/NOT circuits (any polarity) are the affine map A i + b over GF(2)."""
    M = 12
    rng = np.random.default_rng(7)
    rows = []
    for _ in range(200):
        if rng.random() < 0.15:
            rows.append((int(rng.integers(M)), 0, 0))
        else:
            c, t = rng.choice(M, 2, replace=False)
            rows.append((int(t), 1 << int(c), int(rng.integers(2)) << int(c)))
    steps = W.make_steps(rows)
    A = [1 << b for b in range(M)]  # output bit t = parity(A[t] & i) ^ bvec[t]
    bvec = [0] * M
    for t, c, p in rows:
        if c == 0:
            bvec[t] ^= 1
        else:
            cb = c.bit_length() - 1
            A[t] ^= A[cb]
            bvec[t] ^= bvec[cb] ^ (0 if p else 1)
    i = np.arange(2 ** M, dtype=np.uint64)
    f = np.zeros_like(i)
    for t in range(M):
        bit = (_popcount(i & np.uint64(A[t])) & np.uint64(1)) ^ np.uint64(bvec[t])
        f |= bit << np.uint64(t)
    k1 = W.random_state(M, np.complex128, 3)
    k2 = oracle.apply_circuit(M, k1, steps)
    np.testing.assert_array_equal(k2[f.astype(np.int64)], k1)


# ----------------------------------------------------------------------------
# ripple-carry adder workload: arithmetic closed form
# ----------------------------------------------------------------------------

def _adder_forward(idx, n, l2b, times):
    """b <- a + b + cin (mod 2^n), cout ^= carry, applied ``times`` times."""
    cin_l, a_l, b_l, cout_l = W.adder_lines(n)
    idx = np.asarray(idx, dtype=np.uint64)

    def get(line):
        return (idx >> np.uint64(l2b[line])) & np.uint64(1)

    a = sum(get(a_l[i]) << np.uint64(i) for i in range(n))
    b = sum(get(b_l[i]) << np.uint64(i) for i in range(n))
    cin = get(cin_l)
    cout = get(cout_l)
    for _ in range(times):
        s = a + b + cin
        b = s & np.uint64((1 << n) - 1)
        cout = cout ^ (s >> np.uint64(n))
    out = idx.copy()
    for i in range(n):
        out &= ~np.uint64(1 << l2b[b_l[i]])
        out |= ((b >> np.uint64(i)) & np.uint64(1)) << np.uint64(l2b[b_l[i]])
    out &= ~np.uint64(1 << l2b[cout_l])
    out |= cout << np.uint64(l2b[cout_l])
    return out


def test_adder_small_full_state():
    n, reps = 3, 2
    steps, l2b = W.adder_circuit(n, 2, reps, seed=9)
    M = 2 * n + 2
    assert len(steps) == (6 * n + 1) * 2 * reps
    k1 = W.random_state(M, np.complex128, 5)
    k2 = oracle.apply_circuit(M, k1, steps)
    i = np.arange(2 ** M, dtype=np.uint64)
    f = _adder_forward(i, n, l2b, 2 * reps)
    np.testing.assert_array_equal(k2[f.astype(np.int64)], k1)


def test_adder_m32_sampled_rows():
    """The M=32 adder workload: sampled output rows map back by the closed form."""
    cfg = W.config_adder_m32()
    steps, l2b, M = cfg["steps"], cfg["line_to_bit"], cfg["M"]
    assert M == 32 and len(steps) == 1456
    rows = np.random.default_rng(1).integers(0, 2 ** 32, size=100000, dtype=np.uint64)
    src = oracle.source_rows(M, steps, rows)
    np.testing.assert_array_equal(_adder_forward(src, 15, l2b, 16), rows)


# ----------------------------------------------------------------------------
# probabilities and norm
# ----------------------------------------------------------------------------

def test_probabilities_pins():
    M = 10
    alt = oracle.probabilities(W.alternating_state(M))
    np.testing.assert_array_equal(alt, np.full(2 ** M, 1.0 / 2 ** M))
    k = W.random_state(16, np.complex128, 4)
    p = oracle.probabilities(k)
    assert np.all(p >= 0)
    # |z|^2 from numpy's hypot-based abs agrees to a few ulp
    np.testing.assert_allclose(p, np.abs(k) ** 2, rtol=1e-15, atol=0)
    assert abs(oracle.fsum_pairwise(p) - math.fsum(p)) <= 1e-15
    assert abs(math.fsum(p) - 1.0) < 1e-13
    # a permutation of the state permutes its probabilities
    steps = W.random_circuit(16, 30, 5)
    p2 = oracle.probabilities(oracle.apply_circuit(16, k, steps))
    np.testing.assert_array_equal(p2, p[oracle.gather_map(16, steps)])


def test_pairwise_sum_error_bound():
    v = np.random.default_rng(3).random(1 << 20)
    exact = math.fsum(v)
    assert abs(oracle.fsum_pairwise(v) - exact) <= 1e-13 * exact


# ----------------------------------------------------------------------------
# validation
# ----------------------------------------------------------------------------

def test_validation_rejects_invalid_steps():
    M = 4
    assert oracle.validate(M, W.make_steps([(0, 2, 2), (3, 0, 0)]))
    assert not oracle.validate(M, W.make_steps([(4, 0, 0)]))        # no such wire
    assert not oracle.validate(M, W.make_steps([(1, 2, 2)]))        # target is a control
    assert not oracle.validate(M, W.make_steps([(0, 2, 6)]))        # polarity off the mask
    assert not oracle.validate(M, W.make_steps([(0, 16, 16)]))      # control wire absent
    with pytest.raises(ValueError):
        oracle.apply_circuit(M, np.zeros(16, np.complex128), W.make_steps([(4, 0, 0)]))


# ----------------------------------------------------------------------------
# App. 1: product-state input
# ----------------------------------------------------------------------------

def test_app1_product_state_example_and_kron():
    """k1 = q_M (x) ... (x) q_1; e.g. k1(5) = q3(1) q2(0) q1(1) (App. 1)."""
    M = 3
    # distinct primes make every product identify its factors; integers keep it exact
    q = np.array([[2, 3], [5, 7], [11, 13]], dtype=np.complex128)  # q1, q2, q3
    k = oracle.product_state(M, q)
    assert k[5] == q[2][1] * q[1][0] * q[0][1] == 13 * 5 * 3
    ref = np.kron(q[2], np.kron(q[1], q[0]))  # library Kronecker product
    np.testing.assert_array_equal(k, ref)
    # complex integer components stay exact as well
    rng = np.random.default_rng(0)
    qi = rng.integers(-4, 5, size=(6, 2)) + 1j * rng.integers(-4, 5, size=(6, 2))
    ref = qi[5]
    for b in range(4, -1, -1):
        ref = np.kron(ref, qi[b])
    np.testing.assert_array_equal(oracle.product_state(6, qi), ref)


def test_app1_product_state_norm_and_random_qubits():
    M = 12
    rng = np.random.default_rng(1)
    q = rng.normal(size=(M, 2)) + 1j * rng.normal(size=(M, 2))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    k = oracle.product_state(M, q)
    ref = q[M - 1]
    for b in range(M - 2, -1, -1):
        ref = np.kron(ref, q[b])
    np.testing.assert_allclose(k, ref, rtol=1e-14, atol=1e-17)
    assert abs(oracle.fsum_pairwise(oracle.probabilities(k)) - 1.0) < 1e-13
