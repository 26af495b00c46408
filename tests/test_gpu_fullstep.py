"""The benchmark's whole step at full size: the 256 x 256 x 512 shell advanced over dt = 1e3 dt_E by
RKL2 under PTL cycling, each operator on its own (conduction on T; viscosity on the three staggered
velocity components), exactly as bench.py times it: the context precision's own PTL decisions,
the speculated floor cycles and the second state buffer included.

The float64 oracle cannot run a multi-cycle step on 33.5M points in a test's time, so the check is
a chain.  (1) The float32 (and bfloat16-storage) step against the float64 GPU path replaying the
same cycle schedule: the precision's error alone, held to the stated tolerances (1e-5, 1e-2).
(2) The float64 GPU path against the oracle: its first cycle of the step at sampled points on
windows of the grid (after s stages a point depends only on points within s cells), to 1e-12.
The float64 path's agreement with the oracle over a whole multi-cycle step at full size is the
jump128 test.  (3) The float64 step's own PTL schedule against the float32 one's."""
import numpy as np
import pytest

import synth
from gpu_common import TOL, rel_l2, to_host
from oracle.geometry import Shell
from oracle.sts import rkl2_coefficients, sts_step
from oracle.tc import TCOperator

pytestmark = pytest.mark.gpu

N_R, N_T, N_P = 256, 256, 512
RATIO = 1e3


@pytest.fixture(scope="module")
def full():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01004_gb300 as pb
    from paper_2403_01004_gb300.build import build
    from synth import device
    build()
    g = synth.make_grid(N_R, N_T, N_P, 1.01)
    tc = synth.tc_inputs(g, synth.SEED_BASE + 1)
    vi = synth.visc_inputs(g, synth.SEED_BASE + 1)
    fields = {"tc": device.tc_fields(tc), "visc": device.visc_fields(vi)}
    states = {"tc": torch.from_numpy(tc.T.reshape(-1)).cuda(),
              "visc": torch.from_numpy(device.visc_state(vi)).cuda()}
    return pb, torch, g, tc, fields, states, {}


def _step(full, kind, prec, forced=None):
    pb, torch, g, tc, fields, states, cache = full
    key = (kind, prec, None if forced is None else tuple(forced))
    if key in cache:
        return cache[key]
    ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, kind, fields[kind], prec)
    x = states[kind].to(ctx.dtype).clone()
    dt = RATIO * pb.parabolic_dt_explicit(ctx)
    st = pb.rkl2_advance(ctx, x, dt if forced is None else 0.0, use_ptl=True, forced=forced)
    ctx.close()
    cache[key] = (st, x.to(torch.float64))
    return cache[key]


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_full_step_against_float64_on_the_same_schedule(full, kind, prec):
    st, x = _step(full, kind, prec)
    assert st["status"] == 0 and st["cycles"] == len(st["dt_cycle"])
    st64, x64 = _step(full, kind, "fp64", forced=st["dt_cycle"])
    assert st64["work_cycle"] == st["work_cycle"]
    e = rel_l2(to_host(x), to_host(x64))
    print(f"shell256 {kind} step, {prec}: {st['cycles']} cycles, {st['total_stages']} stages; "
          f"relative L2 against float64 on the same schedule {e:.3e}")
    assert e <= TOL[prec], e


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_float64_step_schedule(full, kind):
    """The float64 step's own PTL decisions against the float32 step's: the same number of
    cycles and stages (the decisions compare |F| and Eq. 5's bounds, which the two precisions
    resolve alike on this workload)."""
    st32, _ = _step(full, kind, "fp32")
    st64, _ = _step(full, kind, "fp64")
    print(f"shell256 {kind}: float64 {st64['cycles']} cycles / {st64['total_stages']} stages, "
          f"float32 {st32['cycles']} / {st32['total_stages']}")
    assert st64["cycles"] == st32["cycles"]
    assert st64["total_stages"] == st32["total_stages"]


def test_float64_first_cycle_against_the_oracle(full):
    """The float64 step's first conduction cycle, replayed alone, at sampled points (r
    boundaries, poles, phi wrap) against the oracle's stages on windows of margin s + 1."""
    pb, torch, g, tc, fields, states, _ = full
    st64, _ = _step(full, "tc", "fp64")
    dt_c = st64["dt_cycle"][0]
    ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", fields["tc"], "fp64")
    x = states["tc"].clone()
    st = pb.rkl2_advance(ctx, x, 0.0, forced=[dt_c])
    ctx.close()
    s = st["work_cycle"][0]
    co = rkl2_coefficients(s)
    xh = to_host(x).reshape(N_P, N_T, N_R)
    uh = tc.T
    m = s + 1
    for (k, j, i) in [(0, 0, 0), (N_P - 1, N_T - 1, N_R - 1), (37, 128, 3), (300, 1, 200), (129, 254, 90)]:
        i0, i1 = max(0, i - m), min(N_R, i + m + 1)
        j0, j1 = max(0, j - m), min(N_T, j + m + 1)
        ks = [(k + d) % N_P for d in range(-m, m + 1)]
        sl = lambda a: a[ks][:, j0:j1, i0:i1]
        sh = Shell(g.r_face[i0:i1 + 1], g.t_face[j0:j1 + 1], len(ks), dphi=2 * np.pi / N_P)
        op = TCOperator.spherical(sh, sl(tc.T), sl(tc.n), [sl(b) for b in tc.B])
        uw = sl(uh).reshape(-1)
        xo = sts_step(op.apply, uw, op.apply(uw), dt_c, co).reshape(op.shape)
        ref = xo[m, j - j0, i - i0]
        assert abs(xh[k, j, i] - ref) <= TOL["fp64"] * max(abs(ref), np.abs(uh).mean()), ((k, j, i), xh[k, j, i], ref)
