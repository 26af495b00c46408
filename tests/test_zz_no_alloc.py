"""pb_ptl_noalloc: the PTL entry point for callers that cannot allocate device memory (a host code
that owns a fixed device arena for a whole run, or that cannot take the device synchronisation of
cudaMalloc / cudaFree inside its time-step loop).  It keeps its scratch in a fixed device array
inside the library.  This test calls it through the C ABI, twice in a row, in each precision, and
checks each result against the float64 oracle's F and Eq. 5 evaluated on the same (rounded)
records and state, and against ptl_compute of a context built on the same inputs.  The records
are packed here from the oracle's float64 coefficients and rounded to the precision's record type,
and both sides read exactly those values.  It also checks that the calls leave the device's free
memory and PyTorch's allocator unchanged."""
import ctypes

import numpy as np
import pytest

from gpu_common import gpu_ctx, rel_max, tc_problem, to_dev, to_host, visc_problem
from oracle.ptl import ptl
from oracle.tc import TCOperator
from oracle.visc import ViscOperator

pytestmark = pytest.mark.gpu

# F tolerance (max norm relative to max |F|): float64 arithmetic, float32 arithmetic with the
# cancellation of neighbour differences at 20 % noise (as the float32 apply tests)
F_TOL = {"fp64": 1e-12, "fp32": 1e-4, "bf16": 1e-4}
DT_TOL = {"fp64": 1e-11, "fp32": 1e-3, "bf16": 1e-3}


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


def _rounded_operator(op, kind, rec64):
    """The oracle operator on the records exactly as the library reads them."""
    if kind == "tc":
        ahat = np.stack([rec64[:, 0], rec64[:, 1], rec64[:, 2]]).reshape(op.ahat.shape)
        return TCOperator(ahat, rec64[:, 3].reshape(op.w3.shape), periodic=op.periodic)
    c_list, w_list = [], []
    for comp in range(3):
        lo, hi = op.offsets[comp], op.offsets[comp + 1]
        shp = op.shapes[comp]
        c_list.append(tuple(rec64[lo:hi, x].reshape(shp) for x in range(3)))
        w_list.append(rec64[lo:hi, 3].reshape(shp))
    return ViscOperator(c_list, w_list, periodic=op.periodic)


def _call(lib, pb, kind, g, prec_code, rec, ud, F):
    import torch
    dt, k, fm = ctypes.c_double(), ctypes.c_int64(), ctypes.c_double()
    kcode = pb.PB_TC_ANISO if kind == "tc" else pb.PB_VISC_ISO
    rc = lib.pb_ptl_noalloc(kcode, g.n_r, g.n_theta, g.n_phi, prec_code, ctypes.c_void_p(rec.data_ptr()),
                            ctypes.c_void_p(ud.data_ptr()), ctypes.c_void_p(F.data_ptr()), ctypes.byref(dt),
                            ctypes.byref(k), ctypes.byref(fm), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    return rc, dt.value, k.value, fm.value


@pytest.mark.parametrize("prec", ["fp64", "fp32", "bf16"])
@pytest.mark.parametrize("kind", ["tc", "visc"])
def test_ptl_noalloc_matches_oracle_and_ptl_compute_twice(lib, kind, prec):
    import torch
    import paper_2403_01004_gb300 as pb
    g, inp, op, u = tc_problem(40, 21, 13, noise=0.2) if kind == "tc" else visc_problem(24, 20, 16)
    ctx = gpu_ctx(kind, g, inp, prec)
    rec_t = {"fp64": torch.float64, "fp32": torch.float32, "bf16": torch.bfloat16}[prec]
    f_t = torch.float64 if prec == "fp64" else torch.float32
    rec = torch.from_numpy(_records(op, kind)).to(torch.float32 if prec != "fp64" else torch.float64).to(rec_t).cuda()
    op_r = _rounded_operator(op, kind, rec.to(torch.float64).cpu().numpy())
    rng = np.random.default_rng(7)
    mem = lambda: (torch.cuda.mem_get_info()[0], torch.cuda.memory_allocated())
    for call in range(3):
        state = u if call == 0 else u * (1.0 + 0.05 * rng.uniform(-1, 1, u.size))
        ud = to_dev(state, ctx)                     # the state in the precision's storage type
        F = torch.empty(ud.numel(), dtype=f_t, device="cuda")
        torch.cuda.synchronize()
        before = mem()
        rc, dt, k, fm = _call(lib, pb, kind, g, pb.PRECISIONS[prec], rec, ud, F)
        assert rc == pb.PB_OK
        torch.cuda.synchronize()
        if call >= 1:
            # the first call may load the library's module (and its fixed array) into the
            # context; every later call allocates nothing
            assert mem() == before
        # against the oracle on the same records and state
        us = to_host(ud)
        Fo = op_r.apply(us)
        assert rel_max(to_host(F), Fo) <= F_TOL[prec], rel_max(to_host(F), Fo)
        dto, ko, fo = ptl(op_r, us, Fo)
        # k attains max |F| to the F tolerance (equal to the oracle's unless two are that close)
        assert abs(Fo[k]) >= fo * (1.0 - 2.0 * F_TOL[prec]), (k, ko)
        if k == ko:
            assert dt == pytest.approx(dto, rel=DT_TOL[prec])
        assert fm == pytest.approx(fo, rel=2.0 * F_TOL[prec])
        # against the context's PTL pass (same arithmetic; its records were rounded on the device)
        dt_ref, k_ref, fm_ref = pb.ptl_compute(ctx, ud)
        if prec == "fp64":
            assert k == k_ref
            assert dt == pytest.approx(dt_ref, rel=1e-11)
            assert fm == pytest.approx(fm_ref, rel=1e-12)
        else:
            assert fm == pytest.approx(fm_ref, rel=2.0 * F_TOL[prec])
            if k == k_ref:
                assert dt == pytest.approx(dt_ref, rel=DT_TOL[prec])


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
