"""Host-side tests of libqsim.so that need no GPU: the library loads, exports
every symbol of include/qsim.h, and its planner (validation, cancellation,
commutation-aware segmentation) preserves the circuit -- checked by applying
the planner's step order with the CPU oracle."""
import os
import re

import numpy as np
import pytest

import oracle
import paper_quant_ph_0308158_gb300 as pkg
from paper_quant_ph_0308158_gb300 import QsimError, plan_circuit, workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_quant_ph_0308158_gb300 import build
    build.build()


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "qsim.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(qsim_[a-z_0-9]+)\s*\(", src)))


def test_library_exports_every_declared_symbol():
    lib = pkg.load()
    names = _declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), "libqsim.so does not export %s" % n
    assert sorted(pkg.EXPORTS) == names
    assert "sm_103a" in pkg.version()


def test_step_record_layout_matches_header():
    assert W.STEP_DTYPE.itemsize == 24
    assert W.STEP_DTYPE.fields["ctrl_mask"][1] == 8


def test_struct_layouts_match_the_binding(tmp_path):
    """Every public struct of include/qsim.h has the size and field offsets
    the ctypes binding assumes (compiled with the host C compiler)."""
    import ctypes
    import subprocess
    from paper_quant_ph_0308158_gb300 import binding as B
    structs = {"qsim_plan_stats": B.PlanStats, "qsim_batch_stats": B.BatchStats,
               "qsim_server_stats": B.ServerStats, "qsim_server_trace_record": B.ServerTraceRecord,
               "qsim_tune_result": B.TuneResult, "qsim_plan_options": B.PlanOptions,
               "qsim_batch_options": B.BatchOptions}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "qsim.h"', "int main(void) {"]
    for cname, py in structs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f, _ in py._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f, cname, f))
    for f in W.STEP_DTYPE.names:
        lines.append('printf("qsim_step %s %%zu\\n", offsetof(qsim_step, %s));' % (f, f))
    lines.append('printf("qsim_step size %zu\\n", sizeof(qsim_step));')
    lines.append("return 0; }")
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n"):
        if line:
            a, b, c = line.split()
            got[(a, b)] = int(c)
    assert got[("qsim_step", "size")] == W.STEP_DTYPE.itemsize
    for f in W.STEP_DTYPE.names:
        assert got[("qsim_step", f)] == W.STEP_DTYPE.fields[f][1], f
    for cname, py in structs.items():
        assert got[(cname, "size")] == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert got[(cname, f)] == getattr(py, f).offset, (cname, f)



@pytest.mark.parametrize("strategy", ["auto", "sweep", "tile", "gather", "inplace"])
@pytest.mark.parametrize("M,L,seed", [(6, 200, 1), (10, 400, 2), (13, 300, 3)])
def test_planned_order_preserves_the_circuit(strategy, M, L, seed):
    steps = W.random_circuit(M, L, seed, max_controls=4)
    # small tiles force many passes and much reordering
    plan = plan_circuit(M, np.complex128, steps, strategy, tile_bits=6, low_bits=2)
    k1 = W.random_state(M, np.complex128, seed)
    want = oracle.apply_circuit(M, k1, steps)
    got = oracle.apply_circuit(M, k1, steps[plan["order"].astype(np.int64)])
    np.testing.assert_array_equal(got, want)
    assert plan["stats"]["passes"] == len(plan["kinds"])
    assert int(plan["pass_ends"][-1]) == len(plan["order"])
    if strategy == "sweep":
        assert set(plan["kinds"]) == {"sweep"} and len(plan["kinds"]) == len(plan["order"])
    if strategy == "tile":
        assert set(plan["kinds"]) == {"tile"}
    if strategy == "inplace":
        assert "gather" not in plan["kinds"]


def test_tile_passes_respect_the_tile_width():
    M, k, l = 16, 8, 3
    steps = W.mixed_circuit(M, 500, 4)
    plan = plan_circuit(M, np.complex64, steps, "tile", tile_bits=k, low_bits=l)
    start = 0
    for end in plan["pass_ends"]:
        seg = steps[plan["order"][start:int(end)].astype(np.int64)]
        high = {int(t) for t in seg["target"] if t >= l}
        assert len(high) <= k - l
        start = int(end)
    # lookahead merges more than a plain in-order split would
    naive = 0
    cur = set()
    for t in steps["target"]:
        if t >= l and t not in cur:
            if len(cur) == k - l:
                naive += 1
                cur = set()
            cur.add(int(t))
    naive += 1
    assert len(plan["pass_ends"]) <= naive


def test_tile_geometry_without_high_bits_falls_back_to_sweeps():
    """A forced tile width equal to the run length leaves no tile bit above
    the low ones: steps with higher targets must become sweeps (the planner
    once looped on them) and the plan must still be the circuit."""
    M = 22
    steps = W.random_circuit(M, 142, 291, max_controls=3)
    r = plan_circuit(M, np.complex128, steps, strategy="tile", tile_bits=6, low_bits=6, scratch=False)
    assert "sweep" in r["kinds"] and "tile" in r["kinds"]
    order = r["order"]
    assert sorted(order.tolist()) == list(range(len(steps)))
    k1 = W.random_state(14, np.complex128, 1)
    small = W.random_circuit(14, 80, 5, max_controls=3)
    rs = plan_circuit(14, np.complex128, small, strategy="tile", tile_bits=6, low_bits=6, scratch=False)
    np.testing.assert_array_equal(oracle.apply_circuit(14, k1, small[rs["order"]]),
                                  oracle.apply_circuit(14, k1, small))


def test_cnot_only_circuit_is_one_affine_gather_pass():
    steps = W.cnot_circuit(16, 64, 1)
    plan = plan_circuit(16, np.complex128, steps, "gather")
    assert plan["kinds"] == ["gather"]
    plan = plan_circuit(16, np.complex128, steps, "auto")
    assert plan["kinds"] == ["gather"]


def test_many_controls_fall_back_to_sweeps_inside_gather_plans():
    M = 12
    many = W.make_steps([(0, 0b1111111110, 0b1010101110)])  # nine controls
    steps = np.concatenate([W.mixed_circuit(M, 10, 1), many, W.mixed_circuit(M, 10, 2)])
    plan = plan_circuit(M, np.complex128, steps, "gather")
    assert "sweep" in plan["kinds"] and "gather" in plan["kinds"]


def test_adjacent_equal_steps_cancel():
    a = W.make_steps([(0, 2, 2), (3, 0, 0), (3, 0, 0), (0, 2, 2)])
    plan = plan_circuit(4, np.complex128, a, "auto")
    assert plan["stats"]["steps_cancelled"] == 4 and plan["stats"]["passes"] == 0


@pytest.mark.parametrize("bad,why", [
    ((4, 0, 0), "target bit >= M"),
    ((1, 2, 2), "target bit is also a control"),
    ((0, 2, 6), "polarity bit outside the control mask"),
    ((0, 16, 16), "control bit >= M"),
])
def test_invalid_steps_are_rejected(bad, why):
    steps = W.make_steps([(0, 0, 0), bad])
    with pytest.raises(QsimError) as e:
        plan_circuit(4, np.complex128, steps)
    assert e.value.code == -1 and why in str(e.value) and "step 1" in str(e.value)


def test_bad_arguments():
    steps = W.make_steps([(0, 0, 0)])
    with pytest.raises(QsimError):
        plan_circuit(0, np.complex128, steps)
    with pytest.raises(QsimError):
        plan_circuit(35, np.complex128, steps)
    with pytest.raises(QsimError):
        plan_circuit(4, np.float32, steps)
    with pytest.raises(QsimError):
        plan_circuit(4, np.complex128, steps, "gather", scratch=False)


def test_workload_plans_have_expected_shape():
    cfg = W.config_mixed_m28()
    plan = plan_circuit(cfg["M"], cfg["dtype"], cfg["steps"], "auto")
    assert plan["kinds"] == ["gather"]       # one bit-sliced pass for 1000 steps
    plan = plan_circuit(cfg["M"], cfg["dtype"], cfg["steps"], "inplace")
    assert "gather" not in plan["kinds"] and plan["stats"]["passes"] < 250
    cfg = W.config_adder_m32()
    plan = plan_circuit(cfg["M"], cfg["dtype"], cfg["steps"], "inplace")
    assert plan["stats"]["steps_cancelled"] == 0
    assert plan["stats"]["tile_passes"] >= 1


def test_jit_precompile_on_the_host():
    from paper_quant_ph_0308158_gb300 import jit_precompile
    steps = W.mixed_circuit(14, 100, 3)
    ms = jit_precompile(14, np.complex128, steps)
    assert ms >= 0.0
    # a second call finds the compiled kernel cached
    assert jit_precompile(14, np.complex128, steps) == ms
    plan = plan_circuit(14, np.complex128, steps, "gather")
    assert plan["kinds"] == ["gather"]
