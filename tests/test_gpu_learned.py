"""The learned PCG warm start: the network's forward pass and gradients against the FP64
oracle (oracle/convnet.py), training on the library's own BE solves, and what the trained
guess gains over the method without it (PCG still reaches the same tolerance from it, and the
previous-step state stays the fallback and the judge).

Tolerances: activations are stored in bfloat16 (relative rounding 2^-9) after each of the four
layers and the backward gradients too, so the forward output is compared at 1e-2 and the
gradients at 5e-2 relative L2 per layer (a few roundings of 2^-9, amplified by cancellation in
the sums over 27 x 16 terms)."""
import numpy as np
import pytest

from oracle import convnet

pytestmark = pytest.mark.gpu
NW = 27 * 16 * 16


@pytest.fixture(scope="module", autouse=True)
def built():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2403_01004_gb300.build import build
    build()


def _random_params(rng):
    import torch
    import paper_2403_01004_gb300 as pb
    params = np.zeros(pb.Model.num_params(), np.float32)
    for l in range(4):
        base = l * (NW + 16)
        W = rng.normal(scale=0.15, size=(27, 16, 16)).astype(np.float32)
        if l == 0:
            W[:, 6:, :] = 0.0
        if l == 3:
            W[:, :, 1:] = 0.0
        b = rng.normal(scale=0.05, size=16).astype(np.float32)
        if l == 3:
            b[1:] = 0.0
        params[base:base + NW] = torch.from_numpy(W).bfloat16().float().numpy().reshape(-1)   # bf16 weights
        params[base + NW:base + NW + 16] = b
    return params


def _oracle_params(params):
    ps = []
    for l in range(4):
        base = l * (NW + 16)
        W = params[base:base + NW].reshape(3, 3, 3, 16, 16).astype(np.float64)   # [phi][theta][r][ci][co]
        ps.append((np.transpose(W, (4, 3, 0, 1, 2)), params[base + NW:base + NW + 16].astype(np.float64)))
    return ps


def test_forward_and_gradients_match_oracle():
    import torch
    import paper_2403_01004_gb300 as pb
    rng = np.random.default_rng(3)
    params = _random_params(rng)
    model = pb.Model(1)
    model.set_params(params)
    np.testing.assert_array_equal(model.get_params(), params)
    S_, D, H, W = 2, 6, 8, 12
    f = np.zeros((S_, D, H, W, 16), np.float32)
    f[..., :6] = rng.normal(size=(S_, D, H, W, 6))
    fb = torch.from_numpy(f).bfloat16().cuda()
    f = fb.float().cpu().numpy()
    y = pb.pb_model_forward(model, fb.reshape(-1), (S_, D, H, W)).cpu().numpy().reshape(S_, D, H, W)
    ps = _oracle_params(params)
    t = rng.normal(size=(S_, D, H, W)).astype(np.float32)
    mask = np.zeros_like(t)
    mask[:, 1:-1, 1:-1, 1:-1] = 1.0
    L, g = pb.pb_model_grad(model, fb.reshape(-1), torch.from_numpy(t).cuda().reshape(-1),
                            torch.from_numpy(mask).cuda().reshape(-1), (S_, D, H, W))
    go, Lo = None, 0.0
    for s in range(S_):
        yo, cache = convnet.forward(ps, np.transpose(f[s], (3, 0, 1, 2)).astype(np.float64))
        assert np.linalg.norm(y[s] - yo[0]) / np.linalg.norm(yo[0]) <= 1e-2
        # the padded last layer has 16 outputs, of which only channel 0 is the prediction
        r = (yo[0] - t[s]) * mask[s]
        Lo += float((r * r).sum())
        dy = np.zeros_like(yo)
        dy[0] = 2.0 * r / mask.sum()
        grads, _ = convnet.backward(ps, cache, dy)
        go = grads if go is None else [(a[0] + b[0], a[1] + b[1]) for a, b in zip(go, grads)]
    assert L == pytest.approx(Lo / mask.sum(), rel=2e-2)
    for l in range(4):
        base = l * (NW + 16)
        gw = g[base:base + NW].reshape(3, 3, 3, 16, 16)
        gwo = np.transpose(go[l][0], (2, 3, 4, 1, 0))
        assert np.linalg.norm(gw - gwo) / np.linalg.norm(gwo) <= 5e-2, l
        gb, gbo = g[base + NW:base + NW + 16], go[l][1]
        assert np.linalg.norm(gb - gbo) / np.linalg.norm(gbo) <= 5e-2, l


def test_training_and_what_the_guess_gains(capsys):
    """Trained on 600 library-made solves (64^3 seeded random profiles, 1e4 dt_E), the network's
    smoothed prediction fits the smoothed targets better than the zero increment, and as a PCG
    initial guess it beats the zero guess and lands within 3 % of the previous-step guess (raw,
    unjudged), which the judge never does worse than.  A larger gain is not available at rtol
    1e-10 here: the smoothed targets are dominated by scales far beyond the network's 9-point
    receptive field (at 1e4 dt_E the diffusion length is about 100 cells), even the exact
    increment, smoothed, saves only about 15 % of the iterations, and grid-scale error in a guess
    costs far more than that."""
    import torch
    import bench
    import paper_2403_01004_gb300 as pb
    import synth
    from paper_2403_01004_gb300 import learned
    from synth import device
    feats, targ, _ = bench.learned_training_data(pb, torch, 600, shape=(64, 64, 64), seed=7)
    N, D, H, W = targ.shape
    model = pb.Model(0)
    learned.train(feats, targ, steps=3000, batch=16, crop=24, border=4, lr=2e-3, seed=1, model=model)
    # mean squared error over the training samples (4 points in from every face), against the
    # untrained model, which predicts a zero increment
    y = pb.pb_model_forward(model, feats.reshape(-1), (N, D, H, W)).view(N, D, H, W)
    y = pb.pb_guess_smooth(y.reshape(-1).contiguous(), (N, D, H, W)).view(N, D, H, W)
    inner = (slice(None), slice(4, -4), slice(4, -4), slice(4, -4))
    mse = float(((y - targ)[inner] ** 2).mean())
    base = float((targ[inner] ** 2).mean())
    with capsys.disabled():
        print(f"\nsmoothed-target MSE {mse:.3e} against {base:.3e} for the zero increment")
    assert mse < base, (mse, base)
    rows = []
    for k in range(3):
        g = synth.make_grid(32, 32, 64, 1.05)
        inp = synth.tc_random_inputs(g, 999 + k)
        ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", device.tc_fields(inp), "fp64")
        u = torch.from_numpy(inp.T.reshape(-1)).cuda()
        dt = 1e4 * pb.parabolic_dt_explicit(ctx)
        res = {}
        for name in ("previous", "zero", "learned", "learned+judge"):
            x = u.clone()
            x0 = None
            if name == "zero":
                x0 = torch.zeros_like(u)
            elif name.startswith("learned"):
                x0 = pb.learned_guess(ctx, model, u, dt)
            st = pb.be_pcg_advance(ctx, x, dt, use_ptl=False, rtol=1e-10, x0=x0,
                                   judge_guess=(name == "learned+judge"), mixed=True)
            assert st["final_rel_residual"] <= 1e-10          # the same tolerance from every guess
            res[name] = st["total_iters"]
        rows.append(res)
        assert res["learned"] < res["zero"]
        assert res["learned"] <= 1.03 * res["previous"] + 1
        assert res["learned+judge"] <= res["previous"] + 2
    with capsys.disabled():
        print("\nPCG iterations to rtol 1e-10 (zero / previous-step / learned / learned judged):",
              [(r["zero"], r["previous"], r["learned"], r["learned+judge"]) for r in rows])


_CONV_CASE = r"""
import sys, numpy as np, torch
sys.path.insert(0, {tests!r})
import paper_2403_01004_gb300 as pb
from test_gpu_learned import _random_params
rng = np.random.default_rng(11)
params = _random_params(rng)
model = pb.Model(1)
model.set_params(params)
S_, D, H, W = 2, 5, 19, 13
f = np.zeros((S_, D, H, W, 16), np.float32)
f[..., :6] = rng.normal(size=(S_, D, H, W, 6))
fb = torch.from_numpy(f).bfloat16().cuda().reshape(-1)
y0 = pb.pb_model_forward(model, fb, (S_, D, H, W), wrap_d=False).cpu().numpy()
y1 = pb.pb_model_forward(model, fb, (S_, D, H, W), wrap_d=True).cpu().numpy()
t = torch.from_numpy(rng.normal(size=(S_, D, H, W)).astype(np.float32)).cuda().reshape(-1)
mask = torch.ones(S_ * D * H * W, dtype=torch.float32, device="cuda")
L, g = pb.pb_model_grad(model, fb, t, mask, (S_, D, H, W))
np.savez({out!r}, y0=y0, y1=y1, L=L, g=g)
"""


def test_tensor_core_layers_match_cuda_core_layers(tmp_path):
    """The tcgen05 conv layers (the default) against the CUDA-core kernel of the same layers,
    selected by PB_CONV_CUDA_CORES=1 in a second process: forward outputs (with and without the
    phi wrap) and all gradients on a shape ragged in every tile dimension (2 x 5 x 19 x 13 against
    output tiles of 2 x 16 x 8) agree to the rounding of their different summation orders (both
    accumulate in float32; activations are rounded to bfloat16 between layers)."""
    import os
    import subprocess
    import sys
    tests = os.path.dirname(os.path.abspath(__file__))
    res = {}
    for name, env in (("tc", {}), ("cuda_cores", {"PB_CONV_CUDA_CORES": "1"})):
        out = str(tmp_path / f"{name}.npz")
        code = _CONV_CASE.format(tests=tests, out=out)
        r = subprocess.run([sys.executable, "-c", code], env={**os.environ, **env}, capture_output=True, text=True,
                           timeout=600)
        assert r.returncode == 0, r.stderr[-2000:]
        res[name] = np.load(out)
    a, b = res["tc"], res["cuda_cores"]
    for key in ("y0", "y1"):
        assert np.linalg.norm(a[key] - b[key]) <= 5e-3 * np.linalg.norm(b[key]), key
    assert not np.allclose(a["y0"], a["y1"])        # the wrap changes the d-boundary points
    assert float(a["L"]) == pytest.approx(float(b["L"]), rel=5e-3)
    assert np.linalg.norm(a["g"] - b["g"]) <= 2e-2 * np.linalg.norm(b["g"])
