"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Tolerances (relative L2 of the result against the oracle): FP64 1e-12, FP32 1e-5, BF16 storage
1e-2.  Operator applications (F = L u) are compared in the max norm relative to max |F|, with
tolerances derived from the storage rounding of u amplified by the cancellation in the
differences of neighbouring values (about 100x for 1% noise): FP64 1e-12, FP32 1e-4,
BF16 3e-1 (BF16 only resolves 0.4% of a value)."""
import math

import numpy as np
import pytest

from gpu_common import TOL, gpu_ctx, rel_l2, rel_max, tc_problem, to_dev, to_host, visc_problem
from oracle.advance import be_advance, sts_advance
from oracle.pcg import be_solve
from oracle.ptl import ptl

pytestmark = pytest.mark.gpu

APPLY_TOL = {"fp64": 1e-12, "fp32": 1e-4, "bf16": 3e-1}
# several tiles in r (32) and theta (8), ragged tails, phi chunking with wrap
SHAPES = [(40, 21, 13), (32, 32, 64), (2, 2, 3), (67, 9, 5)]


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01004_gb300.build import build
    build()


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_tc_apply(shape, prec):
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(*shape, noise=0.2, m=np.array([0.6, 0.0, 0.8]))
    ctx = gpu_ctx("tc", g, inp, prec)
    ud = to_dev(u, ctx)
    F = to_host(pb.parabolic_apply(ctx, ud))
    Fo = op.apply(to_host(ud))      # oracle on the same (rounded) input
    assert rel_max(F, Fo) <= APPLY_TOL[prec], rel_max(F, Fo)
    assert pb.parabolic_dt_explicit(ctx) == pytest.approx(op.dt_explicit(), rel=1e-13 if prec == "fp64" else 1e-13)


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_visc_apply(shape, prec):
    import paper_2403_01004_gb300 as pb
    g, vi, op, v = visc_problem(*shape)
    ctx = gpu_ctx("visc", g, vi, prec)
    vd = to_dev(v, ctx)
    F = to_host(pb.parabolic_apply(ctx, vd))
    Fo = op.apply(to_host(vd))
    assert rel_max(F, Fo) <= APPLY_TOL[prec], rel_max(F, Fo)
    assert pb.parabolic_dt_explicit(ctx) == pytest.approx(op.dt_explicit(), rel=1e-13)


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_ptl_fp64(kind):
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(32, 32, 64) if kind == "tc" else visc_problem(24, 20, 16)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    dtp, k, fmax = pb.ptl_compute(ctx, to_dev(u, ctx))
    dto, ko, fo = ptl(op, u, op.apply(u))
    assert k == ko
    assert dtp == pytest.approx(dto, rel=1e-11)
    assert fmax == pytest.approx(fo, rel=1e-12)


def _sts_compare(kind, shape, scheme, prec, use_ptl=True, forced=None, ratio=100.0):
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(*shape) if kind == "tc" else visc_problem(*shape)
    ctx = gpu_ctx(kind, g, inp, prec)
    dt = ratio * op.dt_explicit()
    ud = to_dev(u, ctx)
    u_in = to_host(ud)
    st = pb.rkl2_advance(ctx, ud, dt, scheme=scheme, use_ptl=use_ptl, forced=forced)
    uo, log = sts_advance(op, u_in, dt, scheme, use_ptl=use_ptl, forced=forced)
    return st, log, to_host(ud), uo, op, u_in


@pytest.mark.parametrize("scheme", ["rkl2", "rkg2"])
@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_sts_ptl_fp64_matches_oracle_schedule_and_state(kind, scheme):
    shape = (32, 32, 64) if kind == "tc" else (24, 20, 16)
    st, log, ug, uo, op, u_in = _sts_compare(kind, shape, scheme, "fp64")
    assert st["cycles"] == log.cycles
    assert st["work_cycle"] == log.s
    assert st["k_cycle"] == log.k
    np.testing.assert_allclose(st["dt_cycle"], log.dt_c, rtol=1e-11)
    assert rel_l2(ug, uo) <= TOL["fp64"], rel_l2(ug, uo)
    M = 1.0 / op.w
    assert (M * ug).sum() == pytest.approx((M * u_in).sum(), rel=1e-13)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_sts_reduced_precision_forced_schedule(kind, prec):
    """The schedule is taken from the oracle's FP64 PTL run and replayed on both sides, so the
    comparison isolates the arithmetic precision from the (discontinuous) cycle decisions."""
    if kind == "visc" and prec == "bf16":
        pytest.skip("bf16 storage targets the conduction workload")
    shape = (32, 32, 64) if kind == "tc" else (24, 20, 16)
    g, inp, op, u = tc_problem(*shape) if kind == "tc" else visc_problem(*shape)
    _, log = sts_advance(op, u, 100.0 * op.dt_explicit(), "rkl2", use_ptl=True)
    st, log2, ug, uo, _, _ = _sts_compare(kind, shape, "rkl2", prec, forced=log.dt_c)
    assert st["work_cycle"] == log2.s
    assert rel_l2(ug, uo) <= TOL[prec], rel_l2(ug, uo)


def test_sts_no_ptl_single_cycle_fp64():
    st, log, ug, uo, _, _ = _sts_compare("tc", (40, 21, 13), "rkl2", "fp64", use_ptl=False)
    assert st["cycles"] == 1 and st["work_cycle"] == log.s == [20]
    assert rel_l2(ug, uo) <= TOL["fp64"]


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_be_fixed_iterations_fp64(kind):
    """Exactly N PCG iterations on both sides: isolates the kernels from the stopping test."""
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(32, 32, 64) if kind == "tc" else visc_problem(24, 20, 16)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    dt = 100.0 * op.dt_explicit()
    ud = to_dev(u, ctx)
    st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, fixed_iters=25)
    res = be_solve(op, u, dt, 0.0, 0, fixed_iters=25)
    assert st["total_iters"] == 25
    assert rel_l2(to_host(ud), res.x) <= TOL["fp64"], rel_l2(to_host(ud), res.x)


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_be_ptl_fp64_converged(kind):
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(32, 32, 64) if kind == "tc" else visc_problem(24, 20, 16)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    dt = 100.0 * op.dt_explicit()
    ud = to_dev(u, ctx)
    st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=True, rtol=1e-10)
    uo, log = be_advance(op, u, dt, use_ptl=True, rtol=1e-10)
    assert st["cycles"] == log.cycles
    np.testing.assert_allclose(st["dt_cycle"], log.dt_c, rtol=1e-9)
    # both solves meet rtol; iteration counts agree to within one per solve
    assert all(abs(a - b) <= 1 for a, b in zip(st["work_cycle"], log.iters))
    assert rel_l2(to_host(ud), uo) <= 1e-8


def test_be_fp32_fixed_iterations():
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(32, 32, 64)
    ctx = gpu_ctx("tc", g, inp, "fp32")
    dt = 100.0 * op.dt_explicit()
    ud = to_dev(u, ctx)
    pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, fixed_iters=20)
    res = be_solve(op, to_host(to_dev(u, ctx)), dt, 0.0, 0, fixed_iters=20)
    assert rel_l2(to_host(ud), res.x) <= TOL["fp32"], rel_l2(to_host(ud), res.x)


def test_errors_nonfinite_maxcycles_noconverge():
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(16, 12, 8)
    ctx = gpu_ctx("tc", g, inp, "fp64")
    dt = 100.0 * op.dt_explicit()
    bad = u.copy()
    bad[37] = np.nan
    ud = to_dev(bad, ctx)
    st = pb.rkl2_advance(ctx, ud, dt, raise_on_error=False)
    assert st["status"] == pb.PB_ENONFINITE
    ud = to_dev(u, ctx)
    st = pb.rkl2_advance(ctx, ud, dt, max_cycles=2, raise_on_error=False)
    assert st["status"] == pb.PB_EMAXCYCLES and st["cycles"] == 2
    ud = to_dev(u, ctx)
    st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, max_iter=3, raise_on_error=False)
    assert st["status"] == pb.PB_ENOCONVERGE
    np.testing.assert_array_equal(to_host(ud), u)        # state restored to the cycle start
    st = pb.rkl2_advance(ctx, ud, 0.0)
    assert st["cycles"] == 0
    np.testing.assert_array_equal(to_host(ud), u)


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_tma_and_fallback_kernels_agree(prec, monkeypatch):
    """The TMA pipeline (aligned rows) and the register-prefetch kernel compute the same stages."""
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(64, 24, 20, noise=0.1)
    dt = 50.0 * op.dt_explicit()
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("PB_DISABLE_TMA", flag)
        ctx = gpu_ctx("tc", g, inp, prec)
        ud = to_dev(u, ctx)
        pb.rkl2_advance(ctx, ud, dt, use_ptl=True)
        outs.append(to_host(ud))
    assert rel_l2(outs[0], outs[1]) <= {"fp64": 1e-14, "fp32": 1e-6, "bf16": 1e-2}[prec]


@pytest.mark.parametrize("prec", ["fp64", "fp32", "mixed"])
def test_pcg_tma_and_fallback_kernels_agree(prec, monkeypatch):
    """The PCG product through the TMA kernel (p assembled on chip from r, D^-1 and p_old) and
    through the register-prefetch kernel give the same iterates; ragged theta tail."""
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(64, 21, 20, noise=0.1)
    dt = 200.0 * op.dt_explicit()
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("PB_DISABLE_TMA", flag)
        ctx = gpu_ctx("tc", g, inp, "fp64" if prec == "mixed" else prec)
        ud = to_dev(u, ctx)
        if prec == "mixed":
            st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, rtol=1e-10, mixed=True)
            assert st["final_rel_residual"] <= 1e-10
        else:
            st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, fixed_iters=30)
            assert st["total_iters"] == 30
        outs.append(to_host(ud))
    assert rel_l2(outs[0], outs[1]) <= {"fp64": 1e-13, "fp32": 1e-5, "mixed": 1e-9}[prec]


def _be_state_bound(op, u, dt_cycles, x_a, x_b, rtol_a, rtol_b):
    """M-norm distance of two Backward Euler runs over the same cycles whose solves stopped at
    relative residuals rtol_a and rtol_b, and the bound the stopping test guarantees for it.

    With M = diag(1/w) and L = w A self-adjoint and negative semi-definite in the M inner product,
    one BE step (I - dt L)^-1 does not grow the M-norm, and a solve stopped at ||r|| <= rtol ||b||
    is off by S^-1 r with ||S^-1 r||_M <= sqrt(max w) ||r||_2.  Summed over the cycles (b = M u of
    each cycle, from the oracle's states; 1 % slack for the two sides' b and float64 rounding)."""
    M = 1.0 / op.w
    sw = math.sqrt(float(op.w.max()))
    bound, cur = 0.0, np.array(u, dtype=np.float64)
    for dt_c in dt_cycles:
        bound += 1.01 * sw * (rtol_a + rtol_b) * float(np.linalg.norm(M * cur))
        cur = be_solve(op, cur, dt_c, 1e-13, 100000).x
    d = np.asarray(x_a, dtype=np.float64) - np.asarray(x_b, dtype=np.float64)
    return float(np.sqrt(np.sum(M * d * d))), bound


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_be_mixed_precision_refinement(kind):
    """Float64 context, float32 PCG corrections with float64 residuals: the true residual meets
    rtol, and the state is within the distance of the oracle's converged BE that the two
    stopping tests allow.  The oracle's PTL schedule is replayed on both sides: the solves
    differ at the 1e-11 level, which can move a (discontinuous) PTL decision."""
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(32, 32, 64) if kind == "tc" else visc_problem(24, 20, 16)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    dt = 100.0 * op.dt_explicit()
    _, log = be_advance(op, u, dt, use_ptl=True, rtol=1e-12)
    uo, _ = be_advance(op, u, dt, forced=log.dt_c, rtol=1e-12)
    ud = to_dev(u, ctx)
    st = pb.be_pcg_advance(ctx, ud, dt, forced=log.dt_c, rtol=1e-10, mixed=True)
    assert st["cycles"] == log.cycles
    assert st["final_rel_residual"] <= 1e-10
    diff, bound = _be_state_bound(op, u, log.dt_c, to_host(ud), uo, 1e-10, 1e-12)
    assert diff <= bound, (diff, bound)
    # one cycle: the oracle's own residual of the GPU solution meets the stopping test
    ud = to_dev(u, ctx)
    st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, rtol=1e-10, mixed=True)
    x = to_host(ud)
    b = u / op.w
    res = b - (x / op.w - dt * op.apply_A(x))
    assert np.linalg.norm(res) <= 1.001e-10 * np.linalg.norm(b), np.linalg.norm(res) / np.linalg.norm(b)
    # and driven by its own PTL decisions it still meets the tolerance in every cycle
    ud = to_dev(u, ctx)
    st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=True, rtol=1e-10, mixed=True)
    assert st["final_rel_residual"] <= 1e-10 and abs(st["cycles"] - log.cycles) <= 2
