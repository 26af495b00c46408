"""Precision stress at full size: the 128 x 256 x 512 shell with the temperature jump at r = 1.02
(three radial cells wide, 5 % noise), advanced over dt = 1e5 dt_E by RKL2 + PTL.  The float64
oracle's run (schedule and sampled final state) is stored in tests/golden/jump128_rkl2_ptl.txt.

Float64 reproduces the oracle's PTL schedule and state (1e-12).  Float32, bfloat16 storage and
float64 storage with the float32 stencil (fp64s) replay that schedule, so the comparison measures
the arithmetic alone, and are held to the stated tolerances: float32 1e-5, bfloat16 storage 1e-2
(fp64s, whose stencil is float32, to 1e-5), on both the uniform samples (their relative L2
estimates the full-grid error) and the samples in the radial band of the jump.  The last cycle
has s = 632 stages: the double-float stage recurrence keeps its arithmetic from accumulating
rounding over them, so what remains is the storage rounding of the stage values (float32) and,
for bfloat16 storage, the rounding of the records and of the state handed back.  Run with their
own PTL, float32 and bfloat16 storage finish the step in a schedule close to the oracle's and
stay within the same tolerances."""
import numpy as np
import pytest

import synth
from gpu_common import TOL
from jump128_golden import load

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2403_01004_gb300 as pb
    from paper_2403_01004_gb300.build import build
    from synth import device
    build()
    wl = synth.WORKLOADS["jump128"]
    g = synth.make_grid(wl["n_r"], wl["n_t"], wl["n_p"], wl["q"])
    inp = synth.tc_inputs(g, wl["seed"], noise=wl["noise"], profile="jump")
    return pb, torch, g, inp, device.tc_fields(inp), wl, load()


def _run(setup, prec, **kw):
    pb, torch, g, inp, fields, wl, gold = setup
    ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", fields, prec)
    dtype = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16, "fp64s": torch.float64}[prec]
    u = torch.from_numpy(inp.T.reshape(-1)).to("cuda", dtype)
    dt_e = pb.parabolic_dt_explicit(ctx)
    st = pb.rkl2_advance(ctx, u, wl["ratio"] * dt_e, **kw)
    got = u[torch.from_numpy(gold["idx"]).to("cuda")].to(torch.float64).cpu().numpy()
    ctx.close()
    return st, got, dt_e


def _errors(got, gold):
    """Relative L2 over the uniform samples (full-grid estimate) and over the jump band."""
    u, b = slice(0, 2048), slice(2048, 4096)
    rel = lambda s: float(np.linalg.norm(got[s] - gold["u"][s]) / np.linalg.norm(gold["u"][s]))
    return rel(u), rel(b)


def test_fp64_reproduces_the_oracle_schedule_and_state(setup):
    gold = setup[-1]
    st, got, dt_e = _run(setup, "fp64", use_ptl=True)
    assert dt_e == pytest.approx(gold["dt_E"], rel=1e-13)
    assert st["cycles"] == len(gold["dt_c"])
    assert st["work_cycle"] == gold["s"]
    assert st["k_cycle"] == gold["k"]
    np.testing.assert_allclose(st["dt_cycle"], gold["dt_c"], rtol=1e-10)
    e_all, e_band = _errors(got, gold)
    assert e_all <= TOL["fp64"] and e_band <= TOL["fp64"], (e_all, e_band)


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64s"])
def test_reduced_precision_on_the_oracle_schedule(setup, prec):
    gold = setup[-1]
    st, got, _ = _run(setup, prec, forced=gold["dt_c"])
    if prec != "bf16":
        # bfloat16 storage takes its stage counts from its own dt_E, the bound of the operator on
        # its rounded records (up to 2^-8 away from the float64 one)
        assert st["work_cycle"] == gold["s"]
    e_all, e_band = _errors(got, gold)
    print(f"jump128 {prec} on the oracle schedule: relative L2 {e_all:.3e} (uniform), {e_band:.3e} (jump band)")
    assert np.isfinite(got).all()
    tol = TOL["fp32" if prec == "fp64s" else prec]
    assert e_all <= tol and e_band <= tol, (e_all, e_band, tol)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_reduced_precision_with_its_own_ptl(setup, prec):
    """The reduced-precision run takes its own PTL decisions: it must finish the step (no cycle
    cap) in about the oracle's number of cycles and land within the same tolerance."""
    gold = setup[-1]
    st, got, _ = _run(setup, prec, use_ptl=True, max_cycles=400, raise_on_error=False)
    assert st["status"] == 0, st["status"]
    e_all, e_band = _errors(got, gold)
    print(f"jump128 {prec} own PTL: {st['cycles']} cycles, {st['total_stages']} stages; relative L2 "
          f"{e_all:.3e} (uniform), {e_band:.3e} (jump band)")
    assert st["cycles"] <= 2 * len(gold["dt_c"])
    assert e_all <= TOL[prec] and e_band <= TOL[prec], (e_all, e_band)
