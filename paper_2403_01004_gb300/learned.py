"""Training for the learned PCG initial guess.

The samples are Backward Euler solves made by this library (its features of the pre-step state
and the target increment (x - u^n)/S, smoothed as learned_guess smooths the network output);
they come from the caller (bench.py makes them from seeded random profiles).  Only
orchestration lives here: features, solves, crops, forward, backward and the optimiser all run in
the library's kernels."""
from __future__ import annotations

import torch

from . import Model, pb_model_train


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
