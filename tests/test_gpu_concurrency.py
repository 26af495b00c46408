"""Separate contexts are independent: two contexts on their own streams, driven from two host
threads at once (RKL2 + PTL cycles, floor speculation included), give bit-identical results and
schedules to the same calls made one after the other."""
import concurrent.futures

import numpy as np
import pytest

from gpu_common import gpu_ctx, tc_problem, to_dev, to_host, visc_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01004_gb300.build import build
    build()


def _setup(torch):
    import paper_2403_01004_gb300 as pb
    from synth import device
    out = []
    for kind, (g, inp, op, u) in (("tc", tc_problem(64, 40, 48, noise=0.05)), ("visc", visc_problem(40, 32, 24))):
        s = torch.cuda.Stream()
        fields = device.tc_fields(inp) if kind == "tc" else device.visc_fields(inp)
        ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, kind, fields, "fp32", stream=s)
        out.append((ctx, s, u, 200.0 * op.dt_explicit()))
    return out


def test_two_contexts_from_two_threads_match_sequential():
    import torch
    import paper_2403_01004_gb300 as pb
    probs = _setup(torch)

    def run(ctx, s, u, dt):
        with torch.cuda.stream(s):
            x = to_dev(u, ctx)
        s.synchronize()
        st = pb.rkl2_advance(ctx, x, dt, use_ptl=True)
        return to_host(x), st["dt_cycle"], st["work_cycle"], st["k_cycle"]

    seq = [run(*p) for p in probs]
    for _ in range(3):
        with concurrent.futures.ThreadPoolExecutor(2) as pool:
            par = [f.result() for f in [pool.submit(run, *p) for p in probs]]
        for (xa, da, wa, ka), (xb, db, wb, kb) in zip(seq, par):
            assert da == db and wa == wb and ka == kb
            np.testing.assert_array_equal(xa, xb)
