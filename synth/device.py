"""Moves `synth` inputs to CUDA tensors in the layout the library's C ABI expects (no arithmetic
of the method: only copies and concatenation)."""
from __future__ import annotations

import numpy as np


def tc_fields(inp, device="cuda"):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
    return {"T0": t(inp.T), "n": t(inp.n), "B": [t(b) for b in inp.B]}


def visc_fields(vi, device="cuda"):
    import torch
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).to(device)
    return {"rho": [t(a) for a in vi.rho], "nu": [t(a) for a in vi.nu]}


def visc_state(vi) -> np.ndarray:
    """The three velocity components back to back, each flattened with r fastest."""
    return np.concatenate([np.asarray(a, dtype=np.float64).reshape(-1) for a in vi.v])
