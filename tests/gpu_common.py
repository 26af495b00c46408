"""Shared helpers of the GPU parity tests: build the same seeded problem for the oracle and for
the library, and compare."""
import numpy as np

import synth
from oracle.geometry import Shell
from oracle.tc import TCOperator
from oracle.visc import ViscOperator
from synth import device

TOL = {"fp64": 1e-12, "fp32": 1e-5, "bf16": 1e-2}


def rel_l2(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


def rel_max(a, b) -> float:
    a = np.asarray(a, dtype=np.float64).reshape(-1)
    b = np.asarray(b, dtype=np.float64).reshape(-1)
    return float(np.abs(a - b).max() / np.abs(b).max())


def tc_problem(n_r, n_t, n_p, q=1.05, seed=synth.SEED_BASE, noise=0.01, m=None, profile="exp"):
    g = synth.make_grid(n_r, n_t, n_p, q)
    inp = synth.tc_inputs(g, seed, noise=noise, m=m, profile=profile)
    op = TCOperator.spherical(Shell(g.r_face, g.t_face, g.n_phi), inp.T, inp.n, inp.B)
    return g, inp, op, inp.T.reshape(-1).copy()


def visc_problem(n_r, n_t, n_p, q=1.05, seed=synth.SEED_BASE):
    g = synth.make_grid(n_r, n_t, n_p, q)
    vi = synth.visc_inputs(g, seed)
    op = ViscOperator.spherical(Shell(g.r_face, g.t_face, g.n_phi), vi.rho, vi.nu)
    return g, vi, op, device.visc_state(vi)


def gpu_ctx(kind, g, inp, precision):
    import paper_2403_01004_gb300 as pb
    fields = device.tc_fields(inp) if kind == "tc" else device.visc_fields(inp)
    return pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, kind, fields, precision)


def to_dev(a, ctx):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to("cuda").to(ctx.dtype).contiguous()


def to_host(t):
    import torch
    return t.detach().to(torch.float64).cpu().numpy()
