"""Reader for the small text fixtures under tests/golden/ (paper values)."""
import os

import numpy as np

from paper_quant_ph_0308158_gb300.workloads import make_steps

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def read(name):
    """Parse 'key v1 v2 ...' lines; 'step' and 'case' lines accumulate."""
    out = {"step": [], "case": []}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *vals = line.split()
            if key in ("step", "case"):
                out[key].append([int(v) for v in vals])
            elif key == "interchanges":
                out[key] = [tuple(int(x) for x in v.split(",")) for v in vals]
            elif key == "M":
                out[key] = int(vals[0])
            else:
                out[key] = np.array([float(v) for v in vals])
    if out["step"]:
        out["steps"] = make_steps([tuple(s) for s in out["step"]])
    return out
