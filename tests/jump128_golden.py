"""Reader of tests/golden/jump128_rkl2_ptl.txt (written by tests/golden/make_jump128.py from the
float64 oracle): the cycle schedule and the sampled final state of the precision-stress run."""
from __future__ import annotations

import os

import numpy as np

PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "jump128_rkl2_ptl.txt")


def load(path: str = PATH) -> dict:
    dt_c, s, k, idx, val = [], [], [], [], []
    dt_e = None
    with open(path) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            if t[0] == "dt_E":
                dt_e = float(t[1])
            elif t[0] == "cycle":
                dt_c.append(float(t[2]))
                s.append(int(t[3]))
                k.append(int(t[4]))
            elif t[0] == "sample":
                idx.append(int(t[1]))
                val.append(float(t[2]))
    return {"dt_E": dt_e, "dt_c": dt_c, "s": s, "k": k, "idx": np.array(idx, dtype=np.int64),
            "u": np.array(val, dtype=np.float64)}
