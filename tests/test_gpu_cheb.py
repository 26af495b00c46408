"""The Chebyshev-preconditioned Backward Euler PCG (precond="chebyshev") through the C ABI against
the oracle's be_solve / be_advance with the same polynomial preconditioner: exactly N iterations
on both sides (float64 1e-12, float32 1e-5), the PTL-cycled solve to rtol 1e-10 (same schedule,
iteration counts within one, states within the two stopping tests), the TMA and register-path
kernels against each other, and mixed precision with Chebyshev inner solves."""
import numpy as np
import pytest

from gpu_common import TOL, gpu_ctx, rel_l2, tc_problem, to_dev, to_host, visc_problem
from oracle.advance import be_advance
from oracle.pcg import be_solve

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01004_gb300.build import build
    build()


def _problem(kind):
    return tc_problem(40, 21, 13, noise=0.05) if kind == "tc" else visc_problem(24, 20, 16)


@pytest.mark.parametrize("degree", [2, 3, 5])
@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_cheb_fixed_iterations_fp64(kind, degree):
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = _problem(kind)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    dt = 300.0 * op.dt_explicit()
    ud = to_dev(u, ctx)
    st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, fixed_iters=20, precond="chebyshev", pc_degree=degree)
    res = be_solve(op, u, dt, 0.0, 0, fixed_iters=20, precond="chebyshev", degree=degree)
    assert st["total_iters"] == 20
    assert rel_l2(to_host(ud), res.x) <= TOL["fp64"], rel_l2(to_host(ud), res.x)


def test_cheb_fixed_iterations_fp32():
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = _problem("tc")
    ctx = gpu_ctx("tc", g, inp, "fp32")
    dt = 300.0 * op.dt_explicit()
    ud = to_dev(u, ctx)
    pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, fixed_iters=15, precond="chebyshev", pc_degree=3)
    res = be_solve(op, to_host(to_dev(u, ctx)), dt, 0.0, 0, fixed_iters=15, precond="chebyshev", degree=3)
    assert rel_l2(to_host(ud), res.x) <= TOL["fp32"], rel_l2(to_host(ud), res.x)


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_cheb_ptl_converged_fp64(kind):
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = _problem(kind)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    dt = 100.0 * op.dt_explicit()
    ud = to_dev(u, ctx)
    st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=True, rtol=1e-10, precond="chebyshev", pc_degree=3)
    uo, log = be_advance(op, u, dt, use_ptl=True, rtol=1e-10, precond="chebyshev", degree=3)
    st_j = pb.be_pcg_advance(ctx, to_dev(u, ctx), dt, use_ptl=True, rtol=1e-10)
    assert st["cycles"] == log.cycles
    np.testing.assert_allclose(st["dt_cycle"], log.dt_c, rtol=1e-9)
    assert all(abs(a - b) <= 1 for a, b in zip(st["work_cycle"], log.iters))
    assert st["total_iters"] < st_j["total_iters"]
    assert rel_l2(to_host(ud), uo) <= 1e-8


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_cheb_tma_and_register_kernels_agree(prec, monkeypatch):
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(64, 21, 20, noise=0.1)
    dt = 200.0 * op.dt_explicit()
    outs = []
    for flag in ("0", "1"):
        monkeypatch.setenv("PB_DISABLE_TMA", flag)
        ctx = gpu_ctx("tc", g, inp, prec)
        ud = to_dev(u, ctx)
        pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, fixed_iters=12, precond="chebyshev", pc_degree=4)
        outs.append(to_host(ud))
    assert rel_l2(outs[0], outs[1]) <= {"fp64": 1e-13, "fp32": 1e-6}[prec]


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_cheb_mixed_precision_meets_the_float64_tolerance(kind):
    """Mixed precision with Chebyshev inner solves: the oracle's true residual of the GPU solution
    meets rtol, as with point-Jacobi inner solves, in fewer inner iterations."""
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = _problem(kind)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    dt = 300.0 * op.dt_explicit()
    ud = to_dev(u, ctx)
    st = pb.be_pcg_advance(ctx, ud, dt, use_ptl=False, rtol=1e-10, mixed=True, precond="chebyshev", pc_degree=3)
    st_j = pb.be_pcg_advance(ctx, to_dev(u, ctx), dt, use_ptl=False, rtol=1e-10, mixed=True)
    x = to_host(ud)
    M = 1.0 / op.w
    b = M * u
    res = np.linalg.norm(b - (M * x - dt * op.apply_A(x))) / np.linalg.norm(b)
    assert res <= 1e-10, res
    assert st["total_iters"] < st_j["total_iters"]
