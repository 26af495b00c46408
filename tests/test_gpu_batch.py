"""Batched super time stepping (one persistent graph launch over many problems) against the
oracle and against the one-problem path, for uneven grid sizes and stage counts."""
import numpy as np
import pytest

from gpu_common import TOL, gpu_ctx, rel_l2, tc_problem, to_dev, to_host
from oracle.advance import sts_advance

pytestmark = pytest.mark.gpu

SHAPES = [(16, 16, 16), (40, 21, 13), (32, 32, 64), (64, 24, 20), (16, 32, 32), (24, 16, 12)]
# non-integer ratios: 4r and 6r stay off the stage-count boundaries, where a last-bit
# difference between the two sides' dt_E would flip s
RATIOS = [10.3, 1000.7, 75.2, 301.7, 10003.1, 33.3]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01004_gb300.build import build
    build()


def _problems():
    out = []
    rng = np.random.default_rng(11)
    for b, (shape, ratio) in enumerate(zip(SHAPES, RATIOS)):
        m = rng.normal(size=3)
        m /= np.linalg.norm(m)
        g, inp, op, u = tc_problem(*shape, seed=1000 + b, noise=0.05, m=m)
        out.append((g, inp, op, u, ratio * op.dt_explicit()))
    return out


@pytest.mark.parametrize("scheme", ["rkl2", "rkg2"])
def test_batched_matches_oracle_and_single_path(scheme):
    import paper_2403_01004_gb300 as pb
    probs = _problems()
    ctxs = [gpu_ctx("tc", g, inp, "fp32") for g, inp, _, _, _ in probs]
    us = [to_dev(u, c) for c, (_, _, _, u, _) in zip(ctxs, probs)]
    u_in = [to_host(x) for x in us]
    dts = [dt for *_, dt in probs]
    batch = pb.pb_batch_create(ctxs)
    st = pb.pb_batch_rkl2_advance(batch, us, dts, scheme=scheme)
    for p, (g, inp, op, _, dt) in enumerate(probs):
        uo, log = sts_advance(op, u_in[p], dt, scheme, use_ptl=False)
        assert st[p]["total_stages"] == log.s[0]
        assert rel_l2(to_host(us[p]), uo) <= TOL["fp32"], (p, rel_l2(to_host(us[p]), uo))
        single = to_dev(u_in[p], ctxs[p])
        pb.rkl2_advance(ctxs[p], single, dt, scheme=scheme, use_ptl=False)
        # two float32 kernels (different contraction of the same formulas): each within the
        # float32 tolerance of the oracle, so within that tolerance of each other
        assert rel_l2(to_host(us[p]), to_host(single)) <= TOL["fp32"]
    # a second launch reuses the captured graph and continues from the new states
    before = [to_host(x) for x in us]
    pb.pb_batch_rkl2_advance(batch, us, dts, scheme=scheme)
    for p, (g, inp, op, _, dt) in enumerate(probs):
        uo, _ = sts_advance(op, before[p], dt, scheme, use_ptl=False)
        assert rel_l2(to_host(us[p]), uo) <= TOL["fp32"]


def test_autotune_keeps_states_and_result():
    import paper_2403_01004_gb300 as pb
    probs = _problems()
    ctxs = [gpu_ctx("tc", g, inp, "fp32") for g, inp, _, _, _ in probs]
    us = [to_dev(u, c) for c, (_, _, _, u, _) in zip(ctxs, probs)]
    u_in = [to_host(x) for x in us]
    dts = [dt for *_, dt in probs]
    batch = pb.pb_batch_create(ctxs)
    tune, ms = pb.pb_autotune(batch, us, dts)
    assert tune["kchunk"] in (4, 8, 16, 32, 64) and tune["blocks_per_sm"] in (2, 4, 6, 8) and ms > 0
    for p in range(len(us)):
        np.testing.assert_array_equal(to_host(us[p]), u_in[p])     # untouched by the tuner
    pb.pb_batch_rkl2_advance(batch, us, dts)
    for p, (g, inp, op, _, dt) in enumerate(probs):
        uo, _ = sts_advance(op, u_in[p], dt, "rkl2", use_ptl=False)
        assert rel_l2(to_host(us[p]), uo) <= TOL["fp32"]
