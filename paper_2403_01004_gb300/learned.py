"""Training data and training for the learned PCG initial guess.

The samples are Backward Euler solves made by this library (PC1 PCG to rtol 1e-10) on
seeded random conduction profiles; each gives the network's features of the pre-step state
and the target (x - u^n)/S.  Only orchestration lives here: features, solves, crops, forward,
backward and the optimiser all run in the library's kernels."""
from __future__ import annotations

import torch

import synth
from synth import device

from . import Model, be_pcg_advance, parabolic_dt_explicit, parabolic_setup, pb_guess_features, pb_model_train


def generate(n_samples: int, shape=(48, 48, 96), q: float = 1.05, ratio: float = 1e4, seed: int = 7,
             rtol: float = 1e-10):
    """Returns (feats (N, n_phi, n_theta, n_r, 16) bf16, targets (N, n_phi, n_theta, n_r) f32,
    total PCG iterations of the solves)."""
    n_r, n_t, n_p = shape
    g = synth.make_grid(n_r, n_t, n_p, q)
    feats = torch.empty((n_samples, n_p, n_t, n_r, 16), dtype=torch.bfloat16, device="cuda")
    targets = torch.empty((n_samples, n_p, n_t, n_r), dtype=torch.float32, device="cuda")
    iters = 0
    for i in range(n_samples):
        inp = synth.tc_random_inputs(g, seed * 100003 + i)
        ctx = parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", device.tc_fields(inp), "fp64")
        u = torch.from_numpy(inp.T.reshape(-1)).cuda()
        dt = ratio * parabolic_dt_explicit(ctx)
        x = u.clone()
        st = be_pcg_advance(ctx, x, dt, use_ptl=False, rtol=rtol, mixed=True)
        iters += st["total_iters"]
        f, t, _ = pb_guess_features(ctx, u, dt, x)
        feats[i].copy_(f.view(n_p, n_t, n_r, 16))
        targets[i].copy_(t.view(n_p, n_t, n_r))
        ctx.close()
    return feats, targets, iters


def train(feats, targets, steps: int = 400, batch: int = 8, crop: int = 24, border: int = 4, lr: float = 2e-3,
          seed: int = 0, model: Model | None = None) -> tuple:
    """Trains (or continues) a model on the samples; returns (model, final loss)."""
    model = model or Model(seed)
    N, D, H, W = targets.shape
    loss = pb_model_train(model, feats, targets, (N, D, H, W), steps, batch, crop, border, lr, seed)
    return model, loss


def time_forward(D: int, H: int, W: int, reps: int = 5, seed: int = 0) -> float:
    """Best-of-reps milliseconds of one network forward (four conv layers) on a D x H x W grid of
    seeded random features (phi wrapping), after one untimed forward."""
    from . import pb_model_forward
    gen = torch.Generator(device="cpu").manual_seed(seed)
    feats = torch.zeros(D * H * W, 16)
    feats[:, :6] = torch.randn(D * H * W, 6, generator=gen)
    feats = feats.to("cuda", torch.bfloat16).reshape(-1)
    model = Model(seed)
    pb_model_forward(model, feats, (1, D, H, W), wrap_d=True)
    best = float("inf")
    for _ in range(reps):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        pb_model_forward(model, feats, (1, D, H, W), wrap_d=True)
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    model.close()
    return best


if __name__ == "__main__":
    # python -m paper_2403_01004_gb300.learned D H W [reps]: times the network forward
    import sys
    D, H, W = (int(a) for a in sys.argv[1:4])
    reps = int(sys.argv[4]) if len(sys.argv) > 4 else 5
    from .build import build
    build()
    print(f"forward {D}x{H}x{W}: {time_forward(D, H, W, reps):.3f} ms (best of {reps})")
