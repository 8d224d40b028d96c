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
  overlap, merged free blocks, counters);
- prob_math_check: the complex64 probability arithmetic against the FPU;
- ff_math_check: the float-float products of the App. 1 input against long
  double products;
- closed_source_dump: the generated closed tile pass, evaluated on the host
  and compiled with NVRTC."""
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


def test_probability_arithmetic_matches_the_fpu(tmp_path):
    """The complex64 probability, squared exactly in integer arithmetic and
    summed by one FP64 add (prob_math.cuh compiled for the host), equals the
    host FPU's
    (double)re*re + (double)im*im bit for bit on 28 million pairs: random
    patterns, every exponent alignment of the add, and special values."""
    exe = tmp_path / "prob_math_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe),
                    os.path.join(ROOT, "tests", "native", "prob_math_check.cpp")], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok:"), r.stdout + r.stderr


def test_float_float_products_within_their_bounds(tmp_path):
    """The float-float complex arithmetic of the App. 1 input (ff_math.cuh
    compiled for the host, every operation one correctly rounded step): FP64
    splits within 2^-48, single products within 2^-43 of |a||b|, the device's
    two product chains within 2^-41 of |k| and rounding to within one float
    ulp of the exact product, on six million cases."""
    exe = tmp_path / "ff_math_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe),
                    os.path.join(ROOT, "tests", "native", "ff_math_check.cpp")], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.startswith("ok:"), r.stdout + r.stderr


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


def _closed_dump(tmp_path, M, amp, steps, delta, compile_=False):
    exe = tmp_path / "closed_source_dump"
    if not exe.exists():
        subprocess.run(["g++", "-O1", "-std=c++17", "-I", "/usr/local/cuda/include", "-x", "c++", "-o", str(exe),
                        os.path.join(ROOT, "tests", "native", "closed_source_dump.cpp"),
                        "-L/usr/local/cuda/lib64", "-lcudart", "-ldl"], check=True)
    text = "%d %d %d %d\n" % (M, amp, len(steps), delta) + "".join(
        "%d %d %d\n" % (int(s["target"]), int(s["ctrl_mask"]), int(s["ctrl_pol"])) for s in steps)
    env = dict(os.environ, LD_LIBRARY_PATH="/usr/local/cuda/lib64:" + os.environ.get("LD_LIBRARY_PATH", ""))
    r = subprocess.run([str(exe)] + (["--compile"] if compile_ else []), input=text, capture_output=True,
                       text=True, env=env, timeout=300)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr
    return r.stdout


def _eval_closed(src: str, M: int, base: int, tid: int):
    """Evaluate the generated closed kernel's plane set-up, steps and local
    source read-out for thread tid of the tile at 'base'; returns the 32
    local source indices."""
    import re
    mask = 0xFFFFFFFF
    planes, r = {}, {}
    j0 = tid * 32
    for line in src.splitlines():
        line = line.strip()
        m = re.fullmatch(r"u32 p(\d+) = (0x[0-9a-f]+)u;", line)
        if m:
            planes[int(m.group(1))] = int(m.group(2), 16)
            continue
        m = re.fullmatch(r"u32 p(\d+) = 0u - \(\(j0 >> (\d+)\) & 1u\);", line)
        if m:
            planes[int(m.group(1))] = mask if (j0 >> int(m.group(2))) & 1 else 0
            continue
        m = re.fullmatch(r"u32 p(\d+) = 0u - \(u32\)\(\(base >> (\d+)\) & 1ull\);", line)
        if m:
            planes[int(m.group(1))] = mask if (base >> int(m.group(2))) & 1 else 0
            continue
        m = re.fullmatch(r"p(\d+) = ~p(\d+);", line)
        if m:
            planes[int(m.group(1))] = ~planes[int(m.group(2))] & mask
            continue
        m = re.fullmatch(r"p(\d+) \^= (.+);", line)
        if m:
            acc = mask
            for term in m.group(2).split(" & "):
                v = planes[int(term.lstrip("~p"))]
                acc &= (~v & mask) if term.startswith("~") else v
            planes[int(m.group(1))] ^= acc
            continue
        m = re.fullmatch(r"r\[(\d+)\] = (p(\d+)|0u);", line)
        if m:
            r[int(m.group(1))] = planes[int(m.group(3))] if m.group(3) else 0
    return [sum(((r[q] >> u) & 1) << q for q in range(32)) for u in range(32)]


@pytest.mark.parametrize("amp", [8, 16])
def test_closed_pass_source_finds_every_source_in_its_tile(tmp_path, amp):
    """The generated closed tile pass for the M=32 ripple-carry adder (its
    net map changes only b_4..b_14 and the carry-out: 16 additions of a leave
    b's low four bits alone), evaluated on the host for sampled tiles and
    threads: each output's source, read from the tile's local order, is the
    oracle's x(i).  The source also compiles with NVRTC for sm_103a."""
    import numpy as np
    import oracle
    from paper_quant_ph_0308158_gb300 import workloads as W
    cfg = W.config_adder_m32()
    l2b = cfg["line_to_bit"]
    cin, a, b, cout = W.adder_lines(15)
    delta = 0
    for x in b[4:] + [cout]:
        delta |= 1 << l2b[x]
    out = _closed_dump(tmp_path, 32, amp, cfg["steps"], delta, compile_=(amp == 8))
    lay = [l for l in out.splitlines() if l.startswith("@LAYOUT")][0].split()[1:]
    outs = [int(x) for x in [l for l in out.splitlines() if l.startswith("@OUT")][0].split()[1:]]
    l, k = int(lay[0]), int(lay[1])
    lb = list(range(l)) + [int(x) for x in lay[2:]]
    assert len(lb) == k and (delta & ~sum(1 << x for x in lb)) == 0
    if amp == 8:
        assert "compiled" in out.splitlines()[-1]

    def deposit(v, bits):
        return sum(((v >> q) & 1) << bit for q, bit in enumerate(bits))

    rng = np.random.default_rng(amp)
    rows, srcs = [], []
    for _ in range(6):
        t = int(rng.integers(0, 1 << len(outs)))
        base = deposit(t, outs)
        for tid in rng.integers(0, (1 << k) // 32, size=3):
            loc = _eval_closed(out, 32, base, int(tid))
            for u in range(32):
                rows.append(base | deposit(int(tid) * 32 + u, lb))
                srcs.append(base | deposit(loc[u], lb))
    want = oracle.source_rows(32, cfg["steps"], np.array(rows, dtype=np.uint64))
    np.testing.assert_array_equal(np.array(srcs, dtype=np.uint64), want)
