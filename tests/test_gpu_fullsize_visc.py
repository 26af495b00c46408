"""Viscosity parity at the benchmark's full size (the 256 x 256 x 512 shell, float32, the launch
configuration bench.py times), on sampled outputs the oracle computes on windows.

Each velocity component lives on its own staggered grid and the operator does not couple the
components, so a window of one component is the same operator on a sub-shell whose face arrays
are sliced to give that component's points (v_r at r faces a+1..b, so r_face[a:b+2]; v_theta
likewise in theta; phi windows keep the full dphi).  After m stages a point depends only on
points within m cells, so a window of margin m + 1 reproduces the full-grid result there."""
import numpy as np
import pytest

import synth
from gpu_common import TOL, to_host
from oracle.geometry import Shell
from oracle.sts import rkl2_coefficients, sts_step
from oracle.visc import ViscOperator, staggered_axes

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
    vi = synth.visc_inputs(g, synth.SEED_BASE + 1)
    ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "visc", device.visc_fields(vi), "fp32")
    v = torch.from_numpy(device.visc_state(vi)).to("cuda", torch.float32)
    return pb, g, vi, ctx, v


def _shape(comp):
    """(n_phi, n_theta, n_r) of velocity component comp."""
    return (N_P, N_T - 1 if comp == 1 else N_T, N_R - 1 if comp == 0 else N_R)


def _offsets():
    sizes = [int(np.prod(_shape(c))) for c in range(3)]
    return np.concatenate([[0], np.cumsum(sizes)]).astype(int)


def _window(g, vi, comp, center, m):
    """Oracle operator of component `comp` on the window of half-width m around center = (k, j, i)
    of that component's index space; returns (op, its component block, slicer, local index)."""
    n_p, n_t, n_r = _shape(comp)
    k, j, i = center
    i0, i1 = max(0, i - m), min(n_r, i + m + 1)
    j0, j1 = max(0, j - m), min(n_t, j + m + 1)
    ks = [(k + d) % n_p for d in range(-m, m + 1)]
    rf = g.r_face[i0:i1 + 2] if comp == 0 else g.r_face[i0:i1 + 1]
    tf = g.t_face[j0:j1 + 2] if comp == 1 else g.t_face[j0:j1 + 1]
    sh = Shell(rf, tf, len(ks), dphi=2 * np.pi / N_P)
    sl = lambda a: a[ks][:, j0:j1, i0:i1]
    rho, nu = [], []
    for c in range(3):
        (pr, _), (pt, _), pp = staggered_axes(sh, c)
        shp = (len(pp), len(pt), len(pr))
        rho.append(sl(vi.rho[c]) if c == comp else np.ones(shp))
        nu.append(sl(vi.nu[c]) if c == comp else np.ones(shp))
    op = ViscOperator.spherical(sh, rho, nu)
    assert op.shapes[comp] == sl(vi.rho[comp]).shape
    return op, comp, sl, (m, j - j0, i - i0)


def _apply_comp(op, comp, uw):
    """F of one component of the window operator (the others held at zero)."""
    u = np.zeros(op.n)
    u[op.offsets[comp]:op.offsets[comp + 1]] = uw.reshape(-1)
    return op.apply(u)[op.offsets[comp]:op.offsets[comp + 1]].reshape(op.shapes[comp])


CENTERS = [(0, 0, 0), (511, 254, 254), (37, 128, 3), (300, 1, 200), (129, 253, 90), (256, 100, 128)]


def _split(x):
    off = _offsets()
    return [x[off[c]:off[c + 1]].reshape(_shape(c)) for c in range(3)]


def test_visc_apply_at_full_size(full):
    pb, g, vi, ctx, v = full
    F = _split(to_host(pb.parabolic_apply(ctx, v)))
    vh = _split(to_host(v))
    for comp in range(3):
        for c in CENTERS:
            op, _, sl, loc = _window(g, vi, comp, c, 2)
            Fo = _apply_comp(op, comp, sl(vh[comp]))
            got, ref = F[comp][c], Fo[loc]
            scale = np.abs(Fo[loc[0] - 1:loc[0] + 2]).max()
            assert abs(got - ref) <= 1e-4 * scale, (comp, c, got, ref)


def test_visc_one_cycle_at_full_size(full):
    """One unsplit RKL2 cycle of 20 dt_E (s = 9) on all three components, checked at sampled
    points of each against the oracle's stages on windows of margin s + 1."""
    pb, g, vi, ctx, v = full
    dt = 20.0 * pb.parabolic_dt_explicit(ctx)
    vh0 = _split(to_host(v))
    x = v.clone()
    st = pb.rkl2_advance(ctx, x, dt, use_ptl=False)
    s = st["work_cycle"][0]
    assert s == 9
    xh = _split(to_host(x))
    co = rkl2_coefficients(s)
    for comp in range(3):
        for c in CENTERS[:3]:
            op, _, sl, loc = _window(g, vi, comp, c, s + 1)
            uw = sl(vh0[comp])
            F = lambda w: _apply_comp(op, comp, w.reshape(op.shapes[comp])).reshape(-1)
            xo = sts_step(F, uw.reshape(-1), F(uw.reshape(-1)), dt, co).reshape(op.shapes[comp])
            got, ref = xh[comp][c], xo[loc]
            assert abs(got - ref) <= TOL["fp32"] * max(abs(ref), np.abs(vh0[comp]).mean()), (comp, c, got, ref)
