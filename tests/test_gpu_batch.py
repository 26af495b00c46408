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


def _config2(n=64):
    """The batched workload's problems (synth.batched_problems): grids from 16^3 to 128 x 128 x
    256, dt/dt_E log-uniform in [10, 1e4], tilted dipoles."""
    import synth
    from oracle.geometry import Shell
    from oracle.tc import TCOperator
    out = []
    for pr in synth.batched_problems()[:n]:
        g = synth.make_grid(pr["n_r"], pr["n_t"], pr["n_p"], pr["q"])
        inp = synth.tc_inputs(g, pr["seed"], m=pr["m"])
        out.append((pr, g, inp))
    return out


@pytest.mark.parametrize("tma", [True, False])
def test_config2_batched_equals_single_problem_bit_for_bit(monkeypatch, tma):
    """All 64 problems of the batched workload in one launch with the 32 x 8 tile (small_tiles = 0)
    against each problem advanced alone by the one-problem kernel of the same tile: the TMA ring
    (the batch marches its tiles with the same per-tile function and maps of the same boxes) or,
    with PB_DISABLE_TMA=1 for every context, the register tile.  Same tile arithmetic and the same
    stage coefficients, so the states agree bit for bit; the phi chunking differs (the batch's
    kchunk) and must not matter."""
    import paper_2403_01004_gb300 as pb
    from synth import device
    import torch
    monkeypatch.setenv("PB_DISABLE_TMA", "0" if tma else "1")
    probs = _config2()
    ctxs = [pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", device.tc_fields(inp), "fp32") for _, g, inp in probs]
    u0 = [torch.from_numpy(inp.T.reshape(-1)).to("cuda", torch.float32) for _, _, inp in probs]
    dts = [pr["ratio"] * pb.parabolic_dt_explicit(c) for (pr, _, _), c in zip(probs, ctxs)]
    us = [u.clone() for u in u0]
    batch = pb.pb_batch_create(ctxs, tune=dict(kchunk=8, blocks_per_sm=4, small_tiles=0))
    st = pb.pb_batch_rkl2_advance(batch, us, dts)
    for p, ((pr, g, inp), dt) in enumerate(zip(probs, dts)):
        ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", device.tc_fields(inp), "fp32")
        x = u0[p].clone()
        s1 = pb.rkl2_advance(ctx, x, dt, use_ptl=False)
        assert s1["total_stages"] == st[p]["total_stages"]
        assert torch.equal(x, us[p]), (p, pr["n_r"], pr["n_t"], pr["n_p"], float((x - us[p]).abs().max()))
        ctx.close()
    stages = [x["total_stages"] for x in st]
    assert min(stages) <= 10 and max(stages) >= 150        # the workload's spread of stage counts


def test_config2_batched_against_the_oracle():
    """The batched workload in its tuned launch (small tiles included) against the oracle on every
    problem small enough for it (points x stages <= 4e6): each within the float32 tolerance."""
    import paper_2403_01004_gb300 as pb
    from oracle.geometry import Shell
    from oracle.tc import TCOperator
    from synth import device
    import torch
    probs = _config2()
    ctxs = [pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", device.tc_fields(inp), "fp32") for _, g, inp in probs]
    us = [torch.from_numpy(inp.T.reshape(-1)).to("cuda", torch.float32) for _, _, inp in probs]
    u_in = [u.to(torch.float64).cpu().numpy() for u in us]
    dts = [pr["ratio"] * pb.parabolic_dt_explicit(c) for (pr, _, _), c in zip(probs, ctxs)]
    batch = pb.pb_batch_create(ctxs)
    st = pb.pb_batch_rkl2_advance(batch, us, dts)
    checked = 0
    for p, (pr, g, inp) in enumerate(probs):
        n = g.n_r * g.n_theta * g.n_phi
        if n * st[p]["total_stages"] > 4e6:
            continue
        op = TCOperator.spherical(Shell(g.r_face, g.t_face, g.n_phi), inp.T, inp.n, inp.B)
        uo, log = sts_advance(op, u_in[p], dts[p], "rkl2", use_ptl=False)
        assert log.s[0] == st[p]["total_stages"]
        got = us[p].to(torch.float64).cpu().numpy()
        assert rel_l2(got, uo) <= TOL["fp32"], (p, rel_l2(got, uo))
        checked += 1
    assert checked >= 8
