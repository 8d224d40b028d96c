"""Host checks of the planner's pass encodings: compiles the programs in
tests/native/ (which include the planner's source) with the host compiler
and runs them.  No GPU.

- tile_plan_check: tile layouts (tensor-map copies in bounds, aligned, moving
  the amplitudes the local order names) and per-tile step encodings;
- gather_plan_check: affine tables, bit-sliced descriptors, compiled step
  lists and sweep pair enumeration, each evaluated on sampled rows against
  the circuit's own steps;
- arena_check: the serving budget's first-fit allocator (coverage, no
  overlap, merged free blocks, counters)."""
import os
import resource
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _limit_memory():
    resource.setrlimit(resource.RLIMIT_AS, (4 << 30, 4 << 30))


@pytest.mark.parametrize("program", ["tile_plan_check", "gather_plan_check", "arena_check"])
def test_planner_encodings(tmp_path, program):
    exe = tmp_path / program
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(exe),
                    os.path.join(ROOT, "tests", "native", program + ".cpp")], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300,
                       preexec_fn=_limit_memory)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok:"), r.stdout


def test_c_program_builds_against_the_abi(tmp_path):
    """A plain C program compiles against include/qsim.h and links against
    libqsim.so (it is run by the GPU test below)."""
    from paper_quant_ph_0308158_gb300 import build
    lib = build.build()
    exe = tmp_path / "c_abi_usage"
    subprocess.run(["gcc", "-std=c11", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    "-o", str(exe), os.path.join(ROOT, "tests", "native", "c_abi_usage.c"),
                    "-L", os.path.dirname(lib), "-lqsim", "-Wl,-rpath," + os.path.dirname(lib), "-lm"],
                   check=True)
    assert exe.exists()


@pytest.mark.gpu
def test_c_program_runs_the_figure2_circuit(tmp_path):
    from paper_quant_ph_0308158_gb300 import build
    lib = build.build()
    exe = tmp_path / "c_abi_usage"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    os.path.join(ROOT, "tests", "native", "c_abi_usage.c"), "-L", os.path.dirname(lib),
                    "-lqsim", "-Wl,-rpath," + os.path.dirname(lib), "-lm"], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "ok", r.stdout + r.stderr
