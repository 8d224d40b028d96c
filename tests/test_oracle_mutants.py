"""Planted mistakes in the CPU oracle must be caught by its pins.

Each mutant is a one-token change of ``oracle/qsim_oracle.c`` (a dropped
term, a wrong sign, a reversed order, a transposed operand).  The mutated
source is compiled into a temporary library, swapped in for the real one,
and the pin tests of ``test_oracle_pins`` are run against it: at least one
of them has to fail.  None of the mutants writes out of bounds.
"""
import ctypes
import os
import subprocess

import pytest

import oracle
from tests import test_oracle_pins as pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "qsim_oracle.c")

MUTANTS = {
    "source_rows_sign": ("i -= half; /* lower half of the sub-matrix */",
                         "i += 0; /* lower half of the sub-matrix */"),
    "source_rows_order": ("for (size_t s = L; s-- > 0;) {",
                          "for (size_t s = 0; s < L; ++s) {"),
    "polarity_dropped": ("return (i & s->ctrl_mask) == s->ctrl_pol;",
                         "return (i & s->ctrl_mask) == s->ctrl_mask;"),
    "gather_map_not_reversed": ("rev[s] = steps[L - 1 - s];", "rev[s] = steps[s];"),
    "apply_swaps_each_pair_twice": (
        "if (i & half) continue; /* visit upper-half rows only */\n"
        "            if (!toggled(st, i)) continue;\n"
        "            ocplx tmp = k[i];\n"
        "            k[i] = k[i + half];\n"
        "            k[i + half] = tmp;",
        "if (!toggled(st, i)) continue;\n"
        "            ocplx tmp = k[i];\n"
        "            k[i] = k[i ^ half];\n"
        "            k[i ^ half] = tmp;"),
    "row_array_lower_half_untouched": ("y[upper + half] = y[upper + half] - half;",
                                       "y[upper + half] = y[upper + half];"),
    "gather_transposed": ("for (int64_t i = 0; i < n; ++i) k2[i] = k1[x[i]];",
                          "for (int64_t i = 0; i < n; ++i) k2[x[i]] = k1[i];"),
    "probability_term_dropped": ("p[i] = a + b;", "p[i] = a;"),
    "product_bits_reversed": ("const ocplx f = q[2 * b + ((i >> b) & 1u)];",
                              "const ocplx f = q[2 * b + ((i >> (M - 1 - b)) & 1u)];"),
    "product_conjugate_term": ("const double im = acc.re * f.im + acc.im * f.re;",
                               "const double im = acc.re * f.im - acc.im * f.re;"),
    "control_test_inverted": ("if (!toggled(st, i)) continue;\n            ocplx tmp",
                              "if (toggled(st, i)) continue;\n            ocplx tmp"),
}

PINS = [
    (pins.test_sec2b_worked_example_all_oracle_routes, {}),
    (pins.test_sec2h_figure2_running_products, {}),
    (pins.test_sec2_block_rules, {}),
    (pins.test_figure2_circuit_equals_negative_polarity_cnot, {}),
    (pins.test_product_order_reading_non_palindromic, {}),
    (pins.test_sec4_parity_program_closed_form, {"M": 8}),
    (pins.test_sec4_parity_program_sampled_rows, {"M": 32}),
    (pins.test_dense_matrix_products, {"M": 6, "L": 40, "seed": 4}),
    (pins.test_involution_reverse_multiset_norm, {"M": 10, "seed": 2}),
    (pins.test_source_rows_matches_full_state, {"M": 9, "seed": 1}),
    (pins.test_cnot_circuits_equal_their_gf2_affine_map, {}),
    (pins.test_adder_small_full_state, {}),
    (pins.test_probabilities_pins, {}),
    (pins.test_app1_product_state_example_and_kron, {}),
    (pins.test_app1_product_state_norm_and_random_qubits, {}),
]


def _build_mutant(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation anchor for %s not unique" % name
    path = tmp_path / ("m_%s.c" % name)
    path.write_text(src.replace(old, new))
    so = tmp_path / ("m_%s.so" % name)
    subprocess.run(["gcc", "-O1", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                    "-o", str(so), str(path)], check=True)
    return str(so)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(name, tmp_path, monkeypatch):
    old, new = MUTANTS[name]
    so = _build_mutant(tmp_path, name, old, new)
    real = oracle._load()
    lib = ctypes.CDLL(so)
    for fn in ("oracle_validate", "oracle_step_row_array", "oracle_paper_product",
               "oracle_gather_map", "oracle_gather", "oracle_apply_circuit",
               "oracle_source_rows", "oracle_product_state", "oracle_probabilities", "oracle_sum"):
        f, g = getattr(lib, fn), getattr(real, fn)
        f.argtypes, f.restype = g.argtypes, g.restype
    monkeypatch.setattr(oracle, "_lib", lib)
    caught = []
    for fn, kw in PINS:
        try:
            fn(**kw)
        except (AssertionError, ValueError):
            caught.append(fn.__name__)
    assert caught, "mutant %s passed every pin" % name


def test_unmutated_oracle_passes_the_same_pins():
    for fn, kw in PINS:
        fn(**kw)
