"""Host checks built from tests/native/ with the host compiler (no GPU unless
marked): the planner's pass encodings, the serving allocator, the
compiled-gather generator's bit-plane code, and a plain C program against
the C ABI.

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


def _eval_generated_planes(src: str, M: int, my: int):
    """Evaluate the plane set-up and step lines of a generated compiled
    gather for the 32 outputs my .. my+31 of one thread; returns the planes."""
    import re
    planes = {}
    mask = 0xFFFFFFFF
    for line in src.splitlines():
        line = line.strip()
        m = re.fullmatch(r"u32 p(\d+) = (0x[0-9a-f]+)u;", line)
        if m:
            planes[int(m.group(1))] = int(m.group(2), 16)
            continue
        m = re.fullmatch(r"u32 p(\d+) = 0u - \(u32\)\(\(my >> (\d+)\) & 1ull\);", line)
        if m:
            planes[int(m.group(1))] = mask if (my >> int(m.group(2))) & 1 else 0
            continue
        m = re.fullmatch(r"p(\d+) = ~p(\d+);", line)
        if m:
            planes[int(m.group(1))] = ~planes[int(m.group(2))] & mask
            continue
        m = re.fullmatch(r"p(\d+) \^= (.+);", line)
        if m:
            acc = mask
            for term in m.group(2).split(" & "):
                neg = term.startswith("~")
                v = planes[int(term.lstrip("~p"))]
                acc &= (~v & mask) if neg else v
            planes[int(m.group(1))] ^= acc
    return planes


@pytest.mark.parametrize("M,L,seed", [(1, 5, 1), (4, 40, 2), (9, 200, 3), (20, 400, 4), (32, 300, 5)])
def test_compiled_gather_source_evaluates_the_inverse_circuit(tmp_path, M, L, seed):
    """The generated kernel's bit-plane code, evaluated on the host, gives
    every output row its source row x(i): the steps last to first, controls
    on |0> complemented, the low five planes as fixed lane patterns."""
    import numpy as np
    from paper_quant_ph_0308158_gb300 import workloads as W
    cuda_inc = "/usr/local/cuda/include"
    exe = tmp_path / "jit_source_dump"
    subprocess.run(["g++", "-O1", "-std=c++17", "-I", cuda_inc, "-x", "c++", "-o", str(exe),
                    os.path.join(ROOT, "tests", "native", "jit_source_dump.cpp"),
                    "-L/usr/local/cuda/lib64", "-lcudart", "-ldl"], check=True)
    steps = W.random_circuit(M, L, seed, max_controls=min(6, M - 1)) if M > 1 else \
        W.make_steps([(0, 0, 0)] * L)
    text = "%d 16 %d\n" % (M, L) + "".join(
        "%d %d %d\n" % (int(s["target"]), int(s["ctrl_mask"]), int(s["ctrl_pol"])) for s in steps)
    env = dict(os.environ, LD_LIBRARY_PATH="/usr/local/cuda/lib64:" + os.environ.get("LD_LIBRARY_PATH", ""))
    src = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True, env=env).stdout
    rng = np.random.default_rng(seed)
    n = 1 << M
    for my in {0, max(0, n - 32)} | {int(x) * 32 for x in rng.integers(0, max(1, n // 32), size=8)}:
        planes = _eval_generated_planes(src, M, my)
        for j in range(min(32, n - my)):
            i = my + j
            x = i
            for s in steps[::-1]:
                if (x & int(s["ctrl_mask"])) == int(s["ctrl_pol"]):
                    x ^= 1 << int(s["target"])
            got = sum(((planes[b] >> j) & 1) << b for b in range(M))
            assert got == x, (M, i)
