"""GPU parity: the CUDA path through the C ABI against the FP64 oracle on the same seeded inputs.

Tolerances (relative L2 of the result against the oracle): FP64 1e-12, FP32 1e-5, BF16 storage
1e-2.  Operator applications (F = L u, the oracle on the same rounded u) are compared in the max
norm relative to max |F|: FP64 1e-12; FP32 1e-4 (float32 rounding of the records and of the
arithmetic, amplified by the cancellation in the differences of neighbouring values); BF16
storage 3e-2 (the records rounded to bfloat16, 2^-9 relative, a few per point, and F handed back
in bfloat16)."""
import math

import numpy as np
import pytest

from gpu_common import TOL, gpu_ctx, rel_l2, rel_max, tc_problem, to_dev, to_host, visc_problem
from oracle.advance import be_advance, sts_advance
from oracle.pcg import be_solve
from oracle.ptl import ptl, ptl_full

pytestmark = pytest.mark.gpu

APPLY_TOL = {"fp64": 1e-12, "fp32": 1e-4, "bf16": 3e-2}
# dt_E is the Gershgorin bound of the operator the context applies: bfloat16 storage bounds the
# operator on its rounded records (each 2^-9 relative at most from the float64 one)
DTE_TOL = {"fp64": 1e-13, "fp32": 1e-13, "bf16": 8e-3}
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
    assert pb.parabolic_dt_explicit(ctx) == pytest.approx(op.dt_explicit(), rel=DTE_TOL[prec])


@pytest.mark.parametrize("shape", SHAPES)
@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
def test_visc_apply(shape, prec):
    import paper_2403_01004_gb300 as pb
    g, vi, op, v = visc_problem(*shape)
    ctx = gpu_ctx("visc", g, vi, prec)
    vd = to_dev(v, ctx)
    F = to_host(pb.parabolic_apply(ctx, vd))
    Fo = op.apply(to_host(vd))
    assert rel_max(F, Fo) <= APPLY_TOL[prec], rel_max(F, Fo)
    assert pb.parabolic_dt_explicit(ctx) == pytest.approx(op.dt_explicit(), rel=DTE_TOL[prec])


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


def _sts_compare(kind, shape, scheme, prec, use_ptl=True, forced=None, ratio=100.0, ptl_mode="fmax"):
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(*shape) if kind == "tc" else visc_problem(*shape)
    ctx = gpu_ctx(kind, g, inp, prec)
    dt = ratio * op.dt_explicit()
    ud = to_dev(u, ctx)
    u_in = to_host(ud)
    st = pb.rkl2_advance(ctx, ud, dt, scheme=scheme, use_ptl=use_ptl, forced=forced, ptl_mode=ptl_mode,
                         record_full=True)
    uo, log = sts_advance(op, u_in, dt, scheme, use_ptl=use_ptl, forced=forced, ptl_mode=ptl_mode)
    return st, log, to_host(ud), uo, op, u_in


def _ptl_full_interval(op, u, F, eps):
    """Range of the full-grid PTL when every F and u entry may be off by eps times its max norm
    (the float64 apply tolerance): a pair's bound b = -du/dF moves, to first order, by at most
    b (2 eps |F|_inf / |dF| + 2 eps |u|_inf / |du|); the minimum then lies between the smallest
    lower end and the smallest upper end.  Pairs as in the oracle: (i, i + e_d), phi periodic."""
    fi, ui = np.abs(F).max(), np.abs(u).max()
    lo, hi = math.inf, math.inf
    for shape, off in zip(op.shapes, getattr(op, "offsets", [0])):
        n = int(np.prod(shape))
        U, G = u[off:off + n].reshape(shape), F[off:off + n].reshape(shape)
        for ua, ub, ga, gb in ((U[:, :, :-1], U[:, :, 1:], G[:, :, :-1], G[:, :, 1:]),
                               (U[:, :-1], U[:, 1:], G[:, :-1], G[:, 1:]),
                               (U, np.roll(U, -1, 0), G, np.roll(G, -1, 0))):
            du, dF = ua - ub, ga - gb
            ok = (du != 0) & (dF != 0) & (du * dF < 0)
            if ok.any():
                b = -du[ok] / dF[ok]
                db = b * (2 * eps * fi / np.abs(dF[ok]) + 2 * eps * ui / np.abs(du[ok]))
                lo, hi = min(lo, float((b - db).min())), min(hi, float((b + db).min()))
    return lo, hi


PTL_FULL_SHAPES = {"tc": [(40, 21, 13), (32, 32, 64), (67, 9, 5), (2, 2, 3)], "visc": [(24, 20, 16), (9, 7, 5)]}


@pytest.mark.parametrize("kind,shape", [(k, s) for k, v in PTL_FULL_SHAPES.items() for s in v])
def test_ptl_full_fp64(kind, shape):
    """Eq. 4 over every pair of face neighbours: the float64 bound agrees with the oracle's (F
    differs in the last bits: different summation order) and the pair is the oracle's; never
    above the F_max-localised value."""
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(*shape, noise=0.05) if kind == "tc" else visc_problem(*shape)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    ud = to_dev(u, ctx)
    dt, cell, d = pb.ptl_full_compute(ctx, ud)
    dto, keyo = ptl_full(op, u, op.apply(u))
    assert 3 * cell + d == keyo
    assert dt == pytest.approx(dto, rel=1e-10)
    assert dt <= pb.ptl_compute(ctx, ud)[0]


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_ptl_full_fp32(kind):
    """Float32 state and arithmetic: the bound is within 1e-3 of the oracle's on the same
    (rounded) state, and the GPU's pair is one whose float64 bound is that close to the minimum
    (near-equal bounds may swap under float32 rounding of F)."""
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(40, 21, 13, noise=0.05) if kind == "tc" else visc_problem(24, 20, 16)
    ctx = gpu_ctx(kind, g, inp, "fp32")
    ud = to_dev(u, ctx)
    ur = to_host(ud)
    F = op.apply(ur)
    dt, cell, d = pb.ptl_full_compute(ctx, ud)
    dto, keyo = ptl_full(op, ur, F)
    assert dt == pytest.approx(dto, rel=1e-3)
    comp = int(np.searchsorted(getattr(op, "offsets", [0, op.n]), cell, side="right") - 1)
    n_p, n_t, n_r = op.shapes[comp]
    off = int(getattr(op, "offsets", [0])[comp])
    loc = cell - off
    k, rem = divmod(loc, n_t * n_r)
    j, i = divmod(rem, n_r)
    nb = [cell + 1, cell + n_r, off + (((k + 1) % n_p) * n_t + j) * n_r + i][d]
    assert -(ur[cell] - ur[nb]) / (F[cell] - F[nb]) == pytest.approx(dto, rel=1e-3)


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_cycles_under_full_grid_ptl_fp64(kind):
    """STS and BE cycled by the unlocalised PTL: the float64 schedule is the oracle's, with the
    Eq. 5 value recorded beside it; the state agrees with the oracle's."""
    import paper_2403_01004_gb300 as pb
    shape = (32, 32, 64) if kind == "tc" else (24, 20, 16)
    st, log, ug, uo, op, u_in = _sts_compare(kind, shape, "rkl2", "fp64", ptl_mode="full")
    assert st["cycles"] == log.cycles
    assert st["work_cycle"] == log.s
    np.testing.assert_allclose(st["dt_cycle"], log.dt_c, rtol=1e-10)
    assert st["dt_ptl_cycle"] == st["dt_full_cycle"]
    _check_full_values(op, u_in, log.dt_c, st["dt_full_cycle"])
    assert rel_l2(ug, uo) <= TOL["fp64"], rel_l2(ug, uo)
    g, inp, op, u = tc_problem(*shape) if kind == "tc" else visc_problem(*shape)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    dt = 100.0 * op.dt_explicit()
    ud = to_dev(u, ctx)
    stb = pb.be_pcg_advance(ctx, ud, dt, use_ptl=True, rtol=1e-10, ptl_mode="full")
    ub, logb = be_advance(op, u, dt, use_ptl=True, rtol=1e-10, ptl_mode="full")
    assert stb["cycles"] == logb.cycles
    np.testing.assert_allclose(stb["dt_cycle"], logb.dt_c, rtol=1e-9)


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_full_grid_ptl_recorded_beside_fmax_fp64(kind):
    """record_full under the default mode: the cycles are the Eq. 5 schedule, and each recorded
    full-grid value is the oracle's ptl_full of the oracle's state before that cycle."""
    shape = (32, 32, 64) if kind == "tc" else (24, 20, 16)
    st, log, ug, uo, op, u_in = _sts_compare(kind, shape, "rkl2", "fp64")
    assert st["cycles"] == log.cycles
    _check_full_values(op, u_in, log.dt_c, st["dt_full_cycle"])
    assert all(f <= p * (1 + 1e-12) for f, p in zip(st["dt_full_cycle"], st["dt_ptl_cycle"]))


def _check_full_values(op, u0, dt_cycles, got):
    """Each recorded full-grid value lies in the rounding interval of the oracle's state before
    that cycle (float64 apply tolerance, 1e-12 of the max norm)."""
    cur = np.array(u0, dtype=np.float64)
    for c, dt_c in enumerate(dt_cycles):
        F = op.apply(cur)
        lo, hi = _ptl_full_interval(op, cur, F, TOL["fp64"])
        assert lo <= got[c] <= hi, (c, lo, got[c], hi, ptl_full(op, cur, F)[0])
        cur, _ = sts_advance(op, cur, dt_c, "rkl2", forced=[dt_c])


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


@pytest.mark.parametrize("prec", ["fp32", "bf16", "fp64s"])
@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_sts_reduced_precision_forced_schedule(kind, prec):
    """The schedule is taken from the oracle's FP64 PTL run and replayed on both sides, so the
    comparison isolates the arithmetic precision from the (discontinuous) cycle decisions.
    fp64s (float64 storage, float32 stencil) is held to the float32 tolerance: its stencil
    arithmetic is float32."""
    shape = (32, 32, 64) if kind == "tc" else (24, 20, 16)
    g, inp, op, u = tc_problem(*shape) if kind == "tc" else visc_problem(*shape)
    _, log = sts_advance(op, u, 100.0 * op.dt_explicit(), "rkl2", use_ptl=True)
    st, log2, ug, uo, _, _ = _sts_compare(kind, shape, "rkl2", prec, forced=log.dt_c)
    if prec != "bf16":      # bfloat16 storage: stage counts from its own dt_E (rounded records)
        assert st["work_cycle"] == log2.s
    tol = TOL["fp32" if prec == "fp64s" else prec]
    assert rel_l2(ug, uo) <= tol, rel_l2(ug, uo)


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


def test_fp64_storage_refuses_pcg():
    """Float64 storage with a float32 stencil cannot reach the PCG tolerances: BE is refused."""
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(16, 12, 8)
    ctx = gpu_ctx("tc", g, inp, "fp64s")
    st = pb.be_pcg_advance(ctx, to_dev(u, ctx), 10.0 * op.dt_explicit(), raise_on_error=False)
    assert st["status"] == pb.PB_ENOTSUP


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


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16", "fp64s"])
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
    # same arithmetic, compiled in two kernels (the compiler may contract the corner sums
    # differently); bfloat16 storage rounds the two float32 results once at the end
    assert rel_l2(outs[0], outs[1]) <= {"fp64": 1e-14, "fp32": 1e-6, "bf16": 1e-3, "fp64s": 1e-6}[prec]


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


def test_be_mixed_double_float_residual(monkeypatch):
    """Mixed-precision BE on conduction drives its refinements with the double-float residual and
    accepts a stop only on the float64 one: against float64 residuals throughout
    (PB_MIXED_FP64_RESIDUAL=1) both runs meet the tolerance, take the oracle's PTL schedule within
    the same slack, and differ by no more than their stopping tests allow."""
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(32, 32, 64)
    dt = 100.0 * op.dt_explicit()
    _, log = be_advance(op, u, dt, use_ptl=True, rtol=1e-12)
    res = {}
    for flag in ("1", "0"):
        monkeypatch.setenv("PB_MIXED_FP64_RESIDUAL", flag)
        ctx = gpu_ctx("tc", g, inp, "fp64")
        ud = to_dev(u, ctx)
        st = pb.be_pcg_advance(ctx, ud, dt, forced=log.dt_c, rtol=1e-10, mixed=True)
        assert st["final_rel_residual"] <= 1e-10
        res[flag] = (to_host(ud), st)
        ctx.close()
    (x64, s64), (xdf, sdf) = res["1"], res["0"]
    assert sdf["cycles"] == s64["cycles"] == log.cycles
    diff, bound = _be_state_bound(op, u, log.dt_c, xdf, x64, 1e-10, 1e-10)
    assert diff <= bound, (diff, bound)
    # the double-float run's last state passes the float64 test in the oracle too
    ctx = gpu_ctx("tc", g, inp, "fp64")
    ud = to_dev(u, ctx)
    pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, rtol=1e-10, mixed=True)
    xo = to_host(ud)
    b = u / op.w
    r = b - (xo / op.w - dt * op.apply_A(xo))
    assert np.linalg.norm(r) <= 1.001e-10 * np.linalg.norm(b)
    ctx.close()


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_be_mixed_after_coefficient_update(kind):
    """parabolic_update also refreshes the float32 shadow (and the double-float records) of
    mixed-precision BE: a context that solved with one operator and was then updated to another
    solves exactly as a fresh context built on the second one (same iterations, same state)."""
    import paper_2403_01004_gb300 as pb
    import synth
    from synth import device
    shape = (32, 32, 64) if kind == "tc" else (24, 20, 16)
    g, inp, op, u = tc_problem(*shape) if kind == "tc" else visc_problem(*shape)
    inp2 = synth.tc_inputs(g, synth.SEED_BASE + 7, noise=0.05) if kind == "tc" else synth.visc_inputs(g, synth.SEED_BASE + 7)
    fields2 = device.tc_fields(inp2) if kind == "tc" else device.visc_fields(inp2)
    fresh = gpu_ctx(kind, g, inp2, "fp64")
    dt = 100.0 * pb.parabolic_dt_explicit(fresh)
    x_fresh = to_dev(u, fresh)
    st_fresh = pb.be_pcg_advance(fresh, x_fresh, dt, use_ptl=False, rtol=1e-10, mixed=True)
    upd = gpu_ctx(kind, g, inp, "fp64")
    pb.be_pcg_advance(upd, to_dev(u, upd), 100.0 * pb.parabolic_dt_explicit(upd), use_ptl=False, rtol=1e-10,
                      mixed=True)          # builds the shadow on the first operator
    pb.parabolic_update(upd, fields2)
    assert pb.parabolic_dt_explicit(upd) == pb.parabolic_dt_explicit(fresh)
    x_upd = to_dev(u, upd)
    st_upd = pb.be_pcg_advance(upd, x_upd, dt, use_ptl=False, rtol=1e-10, mixed=True)
    assert st_upd["total_iters"] == st_fresh["total_iters"]
    np.testing.assert_array_equal(to_host(x_upd), to_host(x_fresh))
    fresh.close()
    upd.close()


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_async_advance_replays_from_a_cuda_graph(kind):
    """rkl2_advance_async (a forced schedule, enqueued only) captured in a CUDA graph and replayed
    gives the synchronous call's result bit for bit; the PTL is refused by the graph-only form."""
    import torch
    import paper_2403_01004_gb300 as pb
    from synth import device
    g, inp, op, u = tc_problem(40, 21, 13) if kind == "tc" else visc_problem(24, 20, 16)
    s = torch.cuda.Stream()
    fields = device.tc_fields(inp) if kind == "tc" else device.visc_fields(inp)
    ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, kind, fields, "fp32", stream=s)
    _, log = sts_advance(op, u, 50.0 * op.dt_explicit(), "rkl2", use_ptl=True)
    sched = list(log.dt_c)
    ref = to_dev(u, ctx)
    torch.cuda.synchronize()
    pb.rkl2_advance(ctx, ref, sum(sched), forced=sched)
    x = to_dev(u, ctx)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        pb.rkl2_advance_async(ctx, x, 0.0, forced=sched)
    for _ in range(2):
        x.copy_(to_dev(u, ctx))
        torch.cuda.synchronize()
        graph.replay()
        torch.cuda.synchronize()
        np.testing.assert_array_equal(to_host(x), to_host(ref))
    with pytest.raises(pb.ParabolicError):
        pb.rkl2_advance_async(ctx, x, 50.0 * op.dt_explicit())      # one cycle under the PTL
