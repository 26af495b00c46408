"""pb_ptl_noalloc: the PTL entry point for callers that cannot allocate device memory (a host code
that owns a fixed device arena for a whole run, or that cannot take the device synchronisation of
cudaMalloc / cudaFree inside its time-step loop).  It keeps its scratch in a fixed device array
inside the library; this test calls it through the C ABI, twice in a row, and checks each result
against ptl_compute of a context built on the same inputs.  The records it needs are packed here
from the oracle's float64 coefficients, so the two sides agree to rounding."""
import ctypes

import numpy as np
import pytest

from gpu_common import gpu_ctx, rel_max, tc_problem, to_dev, to_host, visc_problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01004_gb300.build import build
    build()
    import paper_2403_01004_gb300 as pb
    return pb.load_library()


def _records(op, kind):
    """Coef4 records {a, b, c, w} per point from the oracle operator (flat, r fastest)."""
    if kind == "tc":
        a = op.ahat.reshape(3, -1)
        return np.ascontiguousarray(np.stack([a[0], a[1], a[2], op.w], axis=1))
    parts = []
    for comp in range(3):
        cr, ct, cp = (x.reshape(-1) for x in op.c[comp])
        parts.append(np.stack([cr, ct, cp, op.w_list[comp].reshape(-1)], axis=1))
    return np.ascontiguousarray(np.concatenate(parts))


@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_ptl_noalloc_matches_ptl_compute_twice(lib, kind):
    import torch
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(40, 21, 13, noise=0.2) if kind == "tc" else visc_problem(24, 20, 16)
    ctx = gpu_ctx(kind, g, inp, "fp64")
    rec = torch.from_numpy(_records(op, kind)).cuda()
    rng = np.random.default_rng(7)
    for call in range(2):
        state = u if call == 0 else u * (1.0 + 0.05 * rng.uniform(-1, 1, u.size))
        ud = to_dev(state, ctx)
        F = torch.empty_like(ud)
        dt, k, fm = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
        kcode = pb.PB_TC_ANISO if kind == "tc" else pb.PB_VISC_ISO
        rc = lib.pb_ptl_noalloc(kcode, g.n_r, g.n_theta, g.n_phi, pb.PB_FP64, ctypes.c_void_p(rec.data_ptr()),
                                ctypes.c_void_p(ud.data_ptr()), ctypes.c_void_p(F.data_ptr()), ctypes.byref(dt),
                                ctypes.byref(k), ctypes.byref(fm), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
        assert rc == pb.PB_OK
        dt_ref, k_ref, fm_ref = pb.ptl_compute(ctx, ud)
        assert k.value == k_ref
        assert dt.value == pytest.approx(dt_ref, rel=1e-11)
        assert fm.value == pytest.approx(fm_ref, rel=1e-12)
        assert rel_max(to_host(F), to_host(pb.parabolic_apply(ctx, ud))) <= 1e-12


def test_ptl_noalloc_rejects_bad_sizes(lib):
    import paper_2403_01004_gb300 as pb
    dt = ctypes.c_double()
    rc = lib.pb_ptl_noalloc(pb.PB_TC_ANISO, 1, 8, 8, pb.PB_FP64, ctypes.c_void_p(16), ctypes.c_void_p(32),
                            ctypes.c_void_p(64), ctypes.byref(dt), None, None, None)
    assert rc == pb.PB_EINVAL
    # more (r, theta) tiles than the fixed scratch holds partials for (65,520): rejected before
    # any device work, so the dummy pointers are never touched
    rc = lib.pb_ptl_noalloc(pb.PB_TC_ANISO, 32 * 300, 8 * 300, 4, pb.PB_FP64, ctypes.c_void_p(16),
                            ctypes.c_void_p(32), ctypes.c_void_p(64), ctypes.byref(dt), None, None, None)
    assert rc == pb.PB_EINVAL
