"""Parity at the benchmark's full size (the 256 x 256 x 512 shell, float32, the launch
configuration bench.py times), on sampled outputs the oracle computes on windows of the grid.

The stencil couples a point to its neighbours one cell away, so after m stages a point depends
only on points within m cells: a window with margin m + 1 around a point reproduces the
full-grid result there exactly (the window's own edges, closed with zero flux or periodically,
only disturb points within m cells of them).  Windows cover the r boundaries, the poles and the
phi wrap."""
import numpy as np
import pytest

import synth
from gpu_common import TOL, to_dev, to_host
from oracle.geometry import Shell
from oracle.ptl import ptl
from oracle.sts import rkl2_coefficients, sts_step
from oracle.tc import TCOperator

pytestmark = pytest.mark.gpu

N_R, N_T, N_P = 256, 256, 512


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
    inp = synth.tc_inputs(g, synth.SEED_BASE + 1)
    ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", device.tc_fields(inp), "fp32")
    u = to_dev(inp.T.reshape(-1), ctx)
    return pb, g, inp, ctx, u


def _window(g, inp, center, m):
    """Oracle operator on the window of half-width m around center = (k, j, i), with the index
    ranges clipped at the r and theta boundaries (there the window edge is the true boundary)
    and phi taken modulo n_phi."""
    k, j, i = center
    i0, i1 = max(0, i - m), min(N_R, i + m + 1)
    j0, j1 = max(0, j - m), min(N_T, j + m + 1)
    ks = [(k + d) % N_P for d in range(-m, m + 1)]
    sl = lambda a: a[ks][:, j0:j1, i0:i1]
    sh = Shell(g.r_face[i0:i1 + 1], g.t_face[j0:j1 + 1], len(ks), dphi=2 * np.pi / N_P)
    op = TCOperator.spherical(sh, sl(inp.T), sl(inp.n), [sl(b) for b in inp.B])
    local = (m, j - j0, i - i0)
    return op, sl, local


CENTERS = [(0, 0, 0), (511, 255, 255), (37, 128, 3), (300, 1, 200), (129, 254, 90), (256, 100, 128)]


def test_apply_at_full_size(full):
    pb, g, inp, ctx, u = full
    F = to_host(pb.parabolic_apply(ctx, u)).reshape(N_P, N_T, N_R)
    uh = to_host(u).reshape(N_P, N_T, N_R)
    for c in CENTERS:
        op, sl, (lk, lj, li) = _window(g, inp, c, 2)
        Fo = op.apply(sl(uh).reshape(-1)).reshape(op.shape)
        got, ref = F[c], Fo[lk, lj, li]
        scale = np.abs(Fo[lk - 1:lk + 2]).max()
        assert abs(got - ref) <= 1e-4 * scale, (c, got, ref)


def test_ptl_decision_at_full_size(full):
    pb, g, inp, ctx, u = full
    dtp, k, fmax = pb.ptl_compute(ctx, u)
    F = to_host(pb.parabolic_apply(ctx, u))
    # k is the first maximiser of |F| and fmax its magnitude (the decision in float32)
    assert int(np.argmax(np.abs(F))) == k and fmax == pytest.approx(float(np.abs(F[k])), rel=1e-7)
    # Eq. 5 at k from the oracle's float64 F on a window around k
    kk = np.unravel_index(k, (N_P, N_T, N_R))
    op, sl, local = _window(g, inp, kk, 3)
    uw = sl(to_host(u).reshape(N_P, N_T, N_R)).reshape(-1)
    Fw = op.apply(uw)
    kl = int(np.ravel_multi_index(local, op.shape))
    ref_fmax = abs(Fw[kl])
    assert fmax == pytest.approx(ref_fmax, rel=1e-4)
    # the oracle's Eq. 5 restricted to k (its own argmax over the window need not be k)
    best = np.inf
    for j in op.neighbors(kl):
        du, dF = uw[kl] - uw[j], Fw[kl] - Fw[j]
        if du != 0 and dF != 0 and du * dF < 0:
            best = min(best, -du / dF)
    assert dtp == pytest.approx(best, rel=1e-3)


def test_one_cycle_at_full_size(full):
    """One RKL2 cycle of 30 dt_E (s = 11 stages) on the whole grid, checked at sampled points
    against the oracle's stages on windows of margin 12."""
    pb, g, inp, ctx, u = full
    dt = 30.0 * pb.parabolic_dt_explicit(ctx)
    uh0 = to_host(u).reshape(N_P, N_T, N_R)
    x = u.clone()
    st = pb.rkl2_advance(ctx, x, dt, use_ptl=False)
    s = st["work_cycle"][0]
    assert s == 11
    xh = to_host(x).reshape(N_P, N_T, N_R)
    co = rkl2_coefficients(s)
    for c in CENTERS[:4]:
        op, sl, local = _window(g, inp, c, s + 1)
        uw = sl(uh0).reshape(-1)
        xo = sts_step(op.apply, uw, op.apply(uw), dt, co).reshape(op.shape)
        got, ref = xh[c], xo[local]
        assert abs(got - ref) <= TOL["fp32"] * max(abs(ref), np.abs(uh0).mean()), (c, got, ref)
