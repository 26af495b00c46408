"""Non-linear conduction with the diffusivity re-lagged every cycle (rkl2_advance_relag) against the
oracle's sts_advance_relag on the same seeded shell: the float64 path reproduces the oracle's
schedule (cycle lengths, stage counts, PTL location per cycle) and state to 1e-12; float32
replays the oracle's schedule to 1e-5; energy is conserved."""
import numpy as np
import pytest

import synth
from gpu_common import TOL, rel_l2, to_dev, to_host
from oracle.advance import sts_advance_relag
from oracle.geometry import Shell
from oracle.tc import TCOperator

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def prob():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01004_gb300.build import build
    build()
    g = synth.make_grid(32, 32, 64, 1.05)
    inp = synth.tc_inputs(g, synth.SEED_BASE + 3, noise=0.05)
    sh = Shell(g.r_face, g.t_face, g.n_phi)
    mk = lambda T0: TCOperator.spherical(sh, np.reshape(T0, g.shape), inp.n, inp.B)
    u = inp.T.reshape(-1).copy()
    dt = 100.0 * mk(u).dt_explicit()
    uo, log, dtE = sts_advance_relag(mk, u, dt)
    return g, inp, u, dt, uo, log, dtE, mk


def _ctx(g, inp, prec):
    import paper_2403_01004_gb300 as pb
    from synth import device
    fields = device.tc_fields(inp)
    return pb, pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", fields, prec), fields


@pytest.mark.parametrize("scheme", ["rkl2", "rkg2"])
def test_relag_fp64_matches_oracle(prob, scheme):
    g, inp, u, dt, uo, log, dtE, mk = prob
    if scheme == "rkg2":
        uo, log, dtE = sts_advance_relag(mk, u, dt, scheme="rkg2")
    pb, ctx, fields = _ctx(g, inp, "fp64")
    ud = to_dev(u, ctx)
    st = pb.rkl2_advance_relag(ctx, ud, dt, fields, scheme=scheme)
    assert log.cycles > 3
    assert st["cycles"] == log.cycles
    assert st["work_cycle"] == log.s
    assert st["k_cycle"] == log.k
    np.testing.assert_allclose(st["dt_cycle"], log.dt_c, rtol=1e-11)
    assert st["dt_explicit"] == pytest.approx(dtE, rel=1e-12)
    got = to_host(ud)
    assert rel_l2(got, uo) <= TOL["fp64"], rel_l2(got, uo)
    w = mk(u).w
    assert np.sum(got / w) == pytest.approx(np.sum(u / w), rel=1e-12)


def test_relag_fp32_on_the_oracle_schedule(prob):
    g, inp, u, dt, uo, log, dtE, mk = prob
    pb, ctx, fields = _ctx(g, inp, "fp32")
    ud = to_dev(u, ctx)
    u_in = to_host(ud)
    uo32, log32, _ = sts_advance_relag(mk, u_in, dt, forced=log.dt_c)
    st = pb.rkl2_advance_relag(ctx, ud, 0.0, fields, forced=log.dt_c)
    assert st["work_cycle"] == log32.s
    assert rel_l2(to_host(ud), uo32) <= TOL["fp32"], rel_l2(to_host(ud), uo32)


def test_relag_refuses_viscosity():
    import paper_2403_01004_gb300 as pb
    from synth import device
    g = synth.make_grid(12, 10, 8, 1.05)
    vi = synth.visc_inputs(g, 1)
    ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "visc", device.visc_fields(vi), "fp64")
    v = to_dev(device.visc_state(vi), ctx)
    inp = synth.tc_inputs(g, 1)
    with pytest.raises(ValueError):
        pb.rkl2_advance_relag(ctx, v, 1.0, device.tc_fields(inp))
