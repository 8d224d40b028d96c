"""Host check of the tile planner's layouts and step encodings: compiles
tests/native/tile_plan_check.cpp (which includes the planner's source) with
the host compiler and runs it.  No GPU."""
import os
import resource
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _limit_memory():
    resource.setrlimit(resource.RLIMIT_AS, (4 << 30, 4 << 30))


def test_tile_layouts_and_step_encodings(tmp_path):
    exe = tmp_path / "tile_plan_check"
    subprocess.run(["g++", "-O2", "-std=c++17", "-o", str(exe),
                    os.path.join(ROOT, "tests", "native", "tile_plan_check.cpp")], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300,
                       preexec_fn=_limit_memory)
    assert r.returncode == 0, r.stdout + r.stderr
    assert r.stdout.startswith("ok:"), r.stdout
