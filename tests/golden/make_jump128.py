"""Writes jump128_rkl2_ptl.txt: the float64 oracle's RKL2 + PTL advance of the precision-stress
workload (128 x 256 x 512 shell, q = 1.05; temperature rising from 0.01 to 1 over three radial
cells at r = 1.02, 5 % noise; dt = 1e5 dt_E), given as its cycle schedule and the final state at
seeded sample points: 2048 anywhere in the shell and 2048 in the radial band of the jump.

It calls only oracle/ and synth/ (the input recipe).  Run from the repository root:
    python tests/golden/make_jump128.py        (about ten minutes on one core)
"""
from __future__ import annotations

import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle.advance import sts_advance  # noqa: E402
from oracle.geometry import Shell  # noqa: E402
from oracle.tc import TCOperator  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "jump128_rkl2_ptl.txt")
SAMPLE_SEED = 20240301


def sample_points(grid) -> np.ndarray:
    """Flat indices (phi, theta, r order, r fastest) of the sample points."""
    rng = np.random.default_rng(SAMPLE_SEED)
    n_r, n_t, n_p = len(grid.r_face) - 1, len(grid.t_face) - 1, grid.n_phi
    anywhere = rng.integers(0, n_r * n_t * n_p, 2048)
    i_jump = int(np.searchsorted(grid.r_face, 1.02) - 1)
    i = rng.integers(max(0, i_jump - 4), min(n_r, i_jump + 5), 2048)
    j = rng.integers(0, n_t, 2048)
    k = rng.integers(0, n_p, 2048)
    band = (k * n_t + j) * n_r + i
    return np.concatenate([anywhere, band]).astype(np.int64)


def main() -> None:
    wl = synth.WORKLOADS["jump128"]
    g = synth.make_grid(wl["n_r"], wl["n_t"], wl["n_p"], wl["q"])
    inp = synth.tc_inputs(g, wl["seed"], noise=wl["noise"], profile="jump")
    op = TCOperator.spherical(Shell(g.r_face, g.t_face, g.n_phi), inp.T, inp.n, inp.B)
    dt_e = op.dt_explicit()
    t0 = time.time()
    u, log = sts_advance(op, inp.T.reshape(-1), wl["ratio"] * dt_e, scheme="rkl2", use_ptl=True)
    idx = sample_points(g)
    with open(OUT, "w") as f:
        f.write("# float64 oracle, RKL2 + PTL (floor 1 dt_E), jump128 workload: "
                f"{wl['n_r']}x{wl['n_t']}x{wl['n_p']}, q={wl['q']}, seed={wl['seed']}, noise={wl['noise']}, "
                f"dt = {wl['ratio']:g} dt_E\n")
        f.write(f"# written by tests/golden/make_jump128.py in {time.time() - t0:.0f} s\n")
        f.write(f"dt_E {dt_e!r}\n")
        for c in range(log.cycles):
            f.write(f"cycle {c} {log.dt_c[c]!r} {log.s[c]} {log.k[c]}\n")
        for q in idx:
            f.write(f"sample {int(q)} {float(u[q])!r}\n")


if __name__ == "__main__":
    main()
