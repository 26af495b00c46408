#!/usr/bin/env python
"""Benchmark of one parabolic step on the production-shaped shell (arXiv:2403.01004 hot path).

Workload "shell256": a 256(r) x 256(theta) x 512(phi) spherical shell (33.5M cells, radial
stretch 1.01, dipole field, T = (0.01 + 0.99 exp(-(r-1)/2))(1 + 1% noise), n = exp(-(r-1)/0.5))
carrying thermal conduction on T and artificial viscosity on the three staggered velocity
components (v ~ N(0, 0.1), nu = 1e-3 r^2, rho = n).  One step = for each operator: set up the
frozen coefficients and dt_E from the lagged fields, then advance over dt = 1e3 dt_E with RKL2
under PTL cycling, float32 storage and arithmetic with float64 reductions.  Inputs are seeded
synthetic stand-ins for the paper's MAS states.

value: point-stage updates per second (cells x stages, the PTL / y0 pass counted as stage 1)
summed over both operators, with inputs resident in HBM.  e2e: the same through the C ABI with
host buffers (pinned host -> device copies of every input field and device -> host copies of
both results inside the timed region).  The working set (about 4 GB) is far above the 129 MB L2,
so no flush is needed between steps.

--impl reference times the FP64 CPU oracle (the plain NumPy restatement of the method) on a
bounded window of the same workload and reports the same metric.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "parabolic-step time & point-updates/s (RKL2, PCG) vs FP64 plain; % HBM roof"
UNIT = "point-stage updates/s"
WORKLOADS = {
    "shell256": dict(n_r=256, n_t=256, n_p=512, q=1.01, ratio=1000.0, seed_off=1),
    "shell128": dict(n_r=128, n_t=128, n_p=256, q=1.01, ratio=1000.0, seed_off=1),   # small smoke size
}


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="shell256", choices=sorted(WORKLOADS))
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "bf16"])
    ap.add_argument("--scheme", default="rkl2", choices=["rkl2", "rkg2"])
    ap.add_argument("--no-fp64", action="store_true", help="skip the FP64 plain comparison step")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-pcg", action="store_true")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-launch sub-benchmark")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-guess sub-benchmark")
    ap.add_argument("--no-rkg2", action="store_true", help="skip the RKG2 comparison step")
    ap.add_argument("--no-ptl-study", action="store_true", help="skip the F_max vs full-grid PTL study")
    ap.add_argument("--no-stress", action="store_true", help="skip the jump128 precision-stress probe")
    ap.add_argument("--no-fig1", action="store_true", help="skip the Fig. 1 reproduction on the periodic box")
    return ap.parse_args()


# ---- inputs ----------------------------------------------------------------------------------
def make_inputs(wl):
    import numpy as np
    import synth
    g = synth.make_grid(wl["n_r"], wl["n_t"], wl["n_p"], wl["q"])
    seed = synth.SEED_BASE + wl["seed_off"]
    tc = synth.tc_inputs(g, seed)
    vi = synth.visc_inputs(g, seed)
    return g, tc, vi


# ---- clocks ------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,pci.bus_id,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, bus_id: str | None):
        self.bus_id = (bus_id or "").lower()
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-lms", "200", "-f", self.path], stdout=subprocess.DEVNULL,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as fh:
                for line in fh:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) < 10:
                        continue
                    if self.bus_id and self.bus_id not in parts[1].lower() and parts[1].lower() not in self.bus_id:
                        continue
                    rows.append(parts)
            os.unlink(self.path)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}

        def num(x):
            try:
                return float(x.split()[0])
            except Exception:
                return None
        sm = [num(r[2]) for r in rows if num(r[2]) is not None]
        smax = [num(r[3]) for r in rows if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ---- multi-rank aggregation ----------------------------------------------------------------------
def reduce_timing(units: float, ms: float, device="cuda"):
    """Whole-job units (sum over ranks) and the slowest rank's time (max over ranks); each rank
    runs an independent replica, so no data crosses ranks except these two numbers."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return units, ms
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(u.item()), float(t.item())


# ---- our implementation --------------------------------------------------------------------
def run_ours(args):
    import numpy as np
    import torch

    import paper_2403_01004_gb300 as pb
    from paper_2403_01004_gb300.build import build
    from synth import device

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        build()
    if world > 1:
        torch.distributed.barrier()
    pb.load_library()
    wl = WORKLOADS[args.workload]
    g, tc, vi = make_inputs(wl)
    dtype = {"fp32": torch.float32, "fp64": torch.float64, "bf16": torch.bfloat16}[args.precision]

    # host (pinned) copies of every input of a step, and their device counterparts
    def pinned(a, dt=torch.float64):
        return torch.from_numpy(np.ascontiguousarray(a)).to(dt).pin_memory()
    h_tc = {"T0": pinned(tc.T), "n": pinned(tc.n), "B": [pinned(b) for b in tc.B]}
    h_vi = {"rho": [pinned(a) for a in vi.rho], "nu": [pinned(a) for a in vi.nu]}
    h_u = pinned(tc.T.reshape(-1), dtype)
    h_v = pinned(device.visc_state(vi), dtype)
    d_tc = {"T0": h_tc["T0"].cuda(), "n": h_tc["n"].cuda(), "B": [b.cuda() for b in h_tc["B"]]}
    d_vi = {"rho": [a.cuda() for a in h_vi["rho"]], "nu": [a.cuda() for a in h_vi["nu"]]}
    d_u0, d_v0 = h_u.cuda(), h_v.cuda()
    u, v = torch.empty_like(d_u0), torch.empty_like(d_v0)
    out_u, out_v = torch.empty_like(h_u).pin_memory(), torch.empty_like(h_v).pin_memory()

    ctx_tc = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", d_tc, args.precision)
    ctx_v = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "visc", d_vi, args.precision)
    n_tc, n_v = ctx_tc.n, ctx_v.n
    stats = {}

    def step_tc(tc_fields, u_src):
        u.copy_(u_src)
        pb.parabolic_update(ctx_tc, tc_fields)
        dt = wl["ratio"] * pb.parabolic_dt_explicit(ctx_tc)
        stats["tc"] = pb.rkl2_advance(ctx_tc, u, dt, scheme=args.scheme, use_ptl=True)
        return n_tc * stats["tc"]["total_stages"]

    def step_visc(vi_fields, v_src):
        v.copy_(v_src)
        pb.parabolic_update(ctx_v, vi_fields)
        dt = wl["ratio"] * pb.parabolic_dt_explicit(ctx_v)
        stats["visc"] = pb.rkl2_advance(ctx_v, v, dt, scheme=args.scheme, use_ptl=True)
        return n_v * stats["visc"]["total_stages"]

    def step(tc_fields, vi_fields, u_src, v_src):
        return step_tc(tc_fields, u_src) + step_visc(vi_fields, v_src)

    # end to end: every input from pinned host memory and both results back, inside the timed
    # region, pipelined as a user advancing many steps would.  An operator's inputs are consumed
    # by its coefficient update and the copy of its initial state, so the next step's inputs of
    # that operator travel on a copy stream while its super steps run, and each result travels
    # back while the next operator (or the next step) computes.  The first step of a timed run
    # copies its own inputs (the viscosity inputs while conduction computes), the last prefetches
    # none; the last result is waited for inside the timed region.
    copy_stream = torch.cuda.Stream()
    e2e_state = {"left": 0, "tc_ready": None, "v_ready": None, "u_out": None, "v_out": None}

    def on_copy_stream(after, copies):
        """Runs copies on the copy stream after event `after` of the main stream; returns the
        event that marks their completion."""
        copy_stream.wait_event(after)
        with torch.cuda.stream(copy_stream):
            copies()
            ev = torch.cuda.Event()
            ev.record(copy_stream)
        return ev

    def copy_tc_in():
        for k in ("T0", "n"):
            d_tc[k].copy_(h_tc[k], non_blocking=True)
        for a in range(3):
            d_tc["B"][a].copy_(h_tc["B"][a], non_blocking=True)
        d_u0.copy_(h_u, non_blocking=True)

    def copy_visc_in():
        for a in range(3):
            d_vi["rho"][a].copy_(h_vi["rho"][a], non_blocking=True)
            d_vi["nu"][a].copy_(h_vi["nu"][a], non_blocking=True)
        d_v0.copy_(h_v, non_blocking=True)

    def marker(stream_):
        ev = torch.cuda.Event()
        ev.record(stream_)
        return ev

    def e2e_step():
        main = torch.cuda.current_stream()
        e2e_state["left"] -= 1
        more = e2e_state["left"] > 0
        now = marker(main)
        ev_tc = e2e_state["tc_ready"] or on_copy_stream(now, copy_tc_in)
        ev_v = e2e_state["v_ready"] or on_copy_stream(now, copy_visc_in)
        # conduction: its inputs are consumed by the update and the state copy
        main.wait_event(ev_tc)
        if e2e_state["u_out"] is not None:
            main.wait_event(e2e_state["u_out"])       # the previous result has left u
        u.copy_(d_u0)
        pb.parabolic_update(ctx_tc, d_tc)
        dt = wl["ratio"] * pb.parabolic_dt_explicit(ctx_tc)
        e2e_state["tc_ready"] = on_copy_stream(marker(main), copy_tc_in) if more else None
        stats["tc"] = pb.rkl2_advance(ctx_tc, u, dt, scheme=args.scheme, use_ptl=True)
        units = n_tc * stats["tc"]["total_stages"]
        e2e_state["u_out"] = on_copy_stream(marker(main), lambda: out_u.copy_(u, non_blocking=True))
        # viscosity, the same way
        main.wait_event(ev_v)
        if e2e_state["v_out"] is not None:
            main.wait_event(e2e_state["v_out"])
        v.copy_(d_v0)
        pb.parabolic_update(ctx_v, d_vi)
        dt = wl["ratio"] * pb.parabolic_dt_explicit(ctx_v)
        e2e_state["v_ready"] = on_copy_stream(marker(main), copy_visc_in) if more else None
        stats["visc"] = pb.rkl2_advance(ctx_v, v, dt, scheme=args.scheme, use_ptl=True)
        units += n_v * stats["visc"]["total_stages"]
        e2e_state["v_out"] = on_copy_stream(marker(main), lambda: out_v.copy_(v, non_blocking=True))
        if not more:
            main.wait_stream(copy_stream)
        return units

    stream = torch.cuda.current_stream()

    def timed(fn, k):
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.perf_counter()
        ev0.record(stream)
        units = 0
        for _ in range(k):
            units += fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        ms = ev0.elapsed_time(ev1)
        units, ms = reduce_timing(units, ms)
        if world > 1:
            torch.distributed.barrier()
        return units, ms, wall

    for _ in range(args.warmup):
        step(d_tc, d_vi, d_u0, d_v0)
    # timed region: device-resident inputs, per-kernel CUDA-event accounting on
    pb.pb_profile_enable(ctx_tc, True)
    pb.pb_profile_enable(ctx_v, True)
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    clocks = ClockSampler(getattr(props, "pci_bus_id", None))
    clocks.start()
    units, ms, wall = timed(lambda: step(d_tc, d_vi, d_u0, d_v0), args.steps)
    clk = clocks.stop()
    prof = pb.pb_profile_read(ctx_tc) + pb.pb_profile_read(ctx_v)
    pb.pb_profile_enable(ctx_tc, False)
    pb.pb_profile_enable(ctx_v, False)
    step_stats = {k: dict(cycles=v_["cycles"], stages=v_["total_stages"]) for k, v_ in stats.items()}
    value = units / (ms / 1e3)
    # the timed step's results and cycle schedules (every step starts from the same inputs)
    result = {"tc": u.clone(), "visc": v.clone()}
    schedule = {k: list(v_["dt_cycle"]) for k, v_ in stats.items()}
    launches = sum(p["launches"] for p in prof)

    e2e = None
    if not args.no_e2e:
        e2e_state["left"] = 1
        e2e_step()
        e2e_state.update(left=args.steps, u_out=None, v_out=None)
        units_e, ms_e, _ = timed(e2e_step, args.steps)
        h2d = sum(t.numel() * t.element_size() for t in [h_tc["T0"], h_tc["n"], *h_tc["B"], *h_vi["rho"], *h_vi["nu"], h_u, h_v])
        d2h = out_u.numel() * out_u.element_size() + out_v.numel() * out_v.element_size()
        # every step starts from the same inputs: the results copied back must equal the device-
        # resident run's bit for bit (a check that no copy overtook its consumer)
        same = bool(torch.equal(out_u.to(result["tc"].device), result["tc"]) and
                    torch.equal(out_v.to(result["visc"].device), result["visc"]))
        e2e = {"value": units_e / (ms_e / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
               "d2h_bytes_per_step": d2h, "ms_per_step": ms_e / args.steps, "results_equal_device_run": same}

    # dominant kernel class of the timed region and its roofline against measured HBM bandwidth
    dom = max(prof, key=lambda p: p["total_ms"])
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    per_launch_ms = dom["total_ms"] / max(1, dom["timed_launches"])
    per_launch_bytes = dom["bytes"] / max(1, dom["launches"])
    achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9
    traffic = traffic_for(dom["name"], args)
    roofline = {"bound": "hbm", "kernel": dom["name"], "achieved": round(achieved, 1), "peak": peak,
                "peak_source": peak_src, "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "alg_bytes_per_launch": per_launch_bytes,
                "ms_per_launch": round(per_launch_ms, 4)}
    kernels = kernel_table(prof)

    extra = {}
    if not args.no_fp64 and args.precision != "fp64":
        extra["fp64_plain"], extra["accuracy"] = fp64_probe(pb, torch, g, d_tc, d_vi, d_u0, d_v0, wl, args, value,
                                                            result, schedule)
        extra["accuracy"]["oracle_first_cycle"] = oracle_first_cycle_probe(pb, torch, g, tc, ctx_tc, d_u0,
                                                                           schedule["tc"][0], args)
    if not args.no_rkg2 and args.scheme == "rkl2":
        # the paper's own scheme (Appendix A) on the same step: same kernels, its coefficients
        # and odd stage counts; its stronger high-mode damping changes the PTL schedule
        prev = args.scheme
        args.scheme = "rkg2"
        step(d_tc, d_vi, d_u0, d_v0)
        units_g, ms_g, _ = timed(lambda: step(d_tc, d_vi, d_u0, d_v0), 1)
        args.scheme = prev
        extra["rkg2_step"] = {"value": units_g / (ms_g / 1e3), "unit": UNIT, "ms_per_step": ms_g,
                              "step": {k: dict(cycles=v_["cycles"], stages=v_["total_stages"]) for k, v_ in stats.items()}}
    # time per step decides the comparison of the schemes (point-stage updates/s rewards a
    # schedule of many short cycles); both schemes' steps, with each operator's cycles and stages
    step_time = {args.scheme: {"ms": ms / args.steps, **step_stats}}
    if "rkg2_step" in extra:
        step_time["rkg2"] = {"ms": extra["rkg2_step"]["ms_per_step"], **extra["rkg2_step"]["step"]}
    if "fp64_plain" in extra:
        step_time[f"{args.scheme}_fp64_plain"] = {"ms": extra["fp64_plain"]["ms_per_step"], **extra["fp64_plain"]["step"]}
    if not args.no_ptl_study:
        extra["ptl_study"] = ptl_study_probe(pb, torch, ctx_tc, ctx_v, d_u0, d_v0, wl)
    if not args.no_stress:
        extra["precision_stress"] = precision_stress_probe(pb, torch)
    if not args.no_fig1:
        extra["fig1"] = fig1_probe(pb, torch)
    if not args.no_pcg:
        extra["pcg"] = pcg_probe(pb, torch, g, d_tc, d_u0, wl)
    if not args.no_batch:
        extra["batched"] = batched_probe(pb, torch)
    if not args.no_learned:
        extra["learned_guess"] = learned_probe(pb, torch)
    cpu = None
    if rank == 0 and not args.no_cpu:
        cpu = cpu_baseline(g, tc, vi, wl, step_stats, n_tc, n_v)
        cpu["cpu_model"] = cpu_model()
        extra["cpu_baseline_all_cores"] = cpu_baseline_all_cores(g, tc, vi, step_stats, n_tc, n_v)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "step_time": step_time,
        "accuracy": extra.pop("accuracy", None), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp32": "f32", "fp64": "f64", "bf16": "bf16-storage/f32"}[args.precision],
        "data": "synthetic (seeded dipole shell; stand-in for the paper's MAS Test 2 state)",
        "config": arm_config(args, wl, world),
        "clocks": clk, "e2e": e2e, "gpu_launches": launches, "roofline": roofline,
        "cpu_baseline": cpu, "step": step_stats, "kernels": kernels, "wall_s_timed": round(wall, 3),
        **extra,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def kernel_table(prof):
    """Per kernel class: launches, event-timed total, share, and algorithmic GB/s per launch."""
    total = max(1e-9, sum(q["total_ms"] for q in prof))
    return [{"name": p["name"], "launches": p["launches"], "ms": round(p["total_ms"], 3),
             "share": round(p["total_ms"] / total, 4),
             "GB/s": round(p["bytes"] / max(1, p["launches"]) / (p["total_ms"] / max(1, p["timed_launches"]) / 1e3) / 1e9, 1)
             if p["total_ms"] > 0 else None} for p in sorted(prof, key=lambda p: -p["total_ms"])]


KERNEL_SOURCES = ("common.cuh", "prof.h", "reduce.cuh", "march.cuh", "march_tma.cuh", "tma.cuh",
                  "epilogues.cuh", "ops_impl.cuh", "dfloat.cuh")


def source_hash() -> str:
    """Hash of the files that define the stencil kernels and their launch configuration."""
    import hashlib
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2403_01004_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(f.encode())
            h.update(fh.read())
    return h.hexdigest()[:16]


def traffic_for(kernel: str, args):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on the current
    kernel sources for this workload and precision; otherwise None."""
    path = os.path.join(ROOT, "profiles", "dram_traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    if d.get("source_sha") != source_hash():
        return None
    e = d.get("kernels", {}).get(f"{args.workload}/{args.precision}/{kernel}")
    return e


def pcg_probe(pb, torch, g, d_tc, d_u0, wl):
    """Backward Euler + PCG on the same conduction problem, float64 state, to rtol 1e-10: one
    cycle of dt = 1e3 dt_E with plain float64 PCG and with mixed precision (float64 residuals,
    float32 corrections), and the whole step under PTL cycling (mixed); each with point-Jacobi
    (PC1) and with the Chebyshev polynomial preconditioner of degree m (m - 1 extra stencil
    passes per iteration)."""
    ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", d_tc, "fp64")
    u0 = d_u0.to(torch.float64)
    dt = wl["ratio"] * pb.parabolic_dt_explicit(ctx)
    out = {"what": "BE + PC1 PCG, shell256 conduction, float64 state, rtol 1e-10"}
    cheb = lambda m: dict(precond="chebyshev", pc_degree=m)
    for name, kw in (("one_cycle_fp64", dict(use_ptl=False)), ("one_cycle_mixed", dict(use_ptl=False, mixed=True)),
                     ("ptl_step_mixed", dict(use_ptl=True, mixed=True)),
                     ("one_cycle_fp64_cheb3", dict(use_ptl=False, **cheb(3))),
                     ("one_cycle_mixed_cheb2", dict(use_ptl=False, mixed=True, **cheb(2))),
                     ("one_cycle_mixed_cheb3", dict(use_ptl=False, mixed=True, **cheb(3))),
                     ("one_cycle_mixed_cheb4", dict(use_ptl=False, mixed=True, **cheb(4))),
                     ("ptl_step_mixed_cheb3", dict(use_ptl=True, mixed=True, **cheb(3)))):
        u = u0.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st = pb.be_pcg_advance(ctx, u, dt, rtol=1e-10, **kw)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[name] = {"ms": ms, "cycles": st["cycles"], "iterations": st["total_iters"],
                     "rel_residual": st["final_rel_residual"],
                     "point_iterations_per_s": ctx.n * st["total_iters"] / (ms / 1e3)}
        # per kernel class (a separate, event-timed run of the same solve)
        u = u0.clone()
        pb.pb_profile_enable(ctx, True)
        pb.be_pcg_advance(ctx, u, dt, rtol=1e-10, **kw)
        torch.cuda.synchronize()
        out[name]["kernels"] = kernel_table(pb.pb_profile_read(ctx))
        pb.pb_profile_enable(ctx, False)
    ctx.close()
    return out


def batched_probe(pb, torch, reps=3):
    """The batched workload: 64 conduction problems (n_r, n_theta in {16..128}, n_phi in
    {n_theta, 2 n_theta}, dt/dt_E log-uniform in [10, 1e4], tilted dipoles), float32, advanced by
    one autotuned persistent graph launch, against the same problems advanced one by one."""
    import synth
    from synth import device
    probs = synth.batched_problems()
    ctxs, u0s, dts = [], [], []
    for pr in probs:
        g = synth.make_grid(pr["n_r"], pr["n_t"], pr["n_p"], pr["q"])
        inp = synth.tc_inputs(g, pr["seed"], m=pr["m"])
        ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", device.tc_fields(inp), "fp32")
        ctxs.append(ctx)
        u0s.append(torch.from_numpy(inp.T.reshape(-1)).to("cuda", torch.float32))
        dts.append(pr["ratio"] * pb.parabolic_dt_explicit(ctx))
    us = [u.clone() for u in u0s]
    batch = pb.pb_batch_create(ctxs)
    tune, tune_ms = pb.pb_autotune(batch, us, dts)
    st = pb.pb_batch_rkl2_advance(batch, us, dts)
    units = sum(c.n * x["total_stages"] for c, x in zip(ctxs, st))

    def timed(fn):
        best = 1e30
        for _ in range(reps):
            for u, u0 in zip(us, u0s):
                u.copy_(u0)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best

    ms_b = timed(lambda: pb.pb_batch_rkl2_advance(batch, us, dts))
    ms_s = timed(lambda: [pb.rkl2_advance(c, u, dt, use_ptl=False) for c, u, dt in zip(ctxs, us, dts)])
    stages = [x["total_stages"] for x in st]
    batch.close()
    for c in ctxs:
        c.close()
    return {"what": "64 float32 conduction problems, one RKL2 cycle each (dt/dt_E log-uniform 10..1e4)",
            "cells": int(sum(c.n for c in ctxs)), "stages_min_max": [min(stages), max(stages)],
            "point_stages": int(units), "tune": tune,
            "batched_ms": ms_b, "batched_value": units / (ms_b / 1e3),
            "separate_launches_ms": ms_s, "separate_value": units / (ms_s / 1e3),
            "speedup_vs_separate": ms_s / ms_b, "unit": UNIT}


def learned_training_data(pb, torch, n_samples: int, shape=(64, 64, 64), q: float = 1.05, ratio: float = 1e4,
                          seed: int = 7, rtol: float = 1e-10):
    """Training samples for the learned guess, made by the library: Backward Euler solves (mixed
    precision PCG to rtol) of seeded random conduction profiles on an n_r x n_theta x n_phi shell,
    each giving the network's features of the pre-step state and the target (x - u^n)/S smoothed
    as learned_guess smooths the network output.  Returns (feats (N, n_phi, n_theta, n_r, 16) bf16,
    targets (N, n_phi, n_theta, n_r) f32, total PCG iterations of the solves)."""
    import synth
    from synth import device
    n_r, n_t, n_p = shape
    g = synth.make_grid(n_r, n_t, n_p, q)
    feats = torch.empty((n_samples, n_p, n_t, n_r, 16), dtype=torch.bfloat16, device="cuda")
    targets = torch.empty((n_samples, n_p, n_t, n_r), dtype=torch.float32, device="cuda")
    iters = 0
    for i in range(n_samples):
        inp = synth.tc_random_inputs(g, seed * 100003 + i)
        ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", device.tc_fields(inp), "fp64")
        u = torch.from_numpy(inp.T.reshape(-1)).cuda()
        dt = ratio * pb.parabolic_dt_explicit(ctx)
        x = u.clone()
        st = pb.be_pcg_advance(ctx, x, dt, use_ptl=False, rtol=rtol, mixed=True)
        iters += st["total_iters"]
        f, t, _ = pb.pb_guess_features(ctx, u, dt, x)
        feats[i].copy_(f.view(n_p, n_t, n_r, 16))
        targets[i].copy_(pb.pb_guess_smooth(t, (1, n_p, n_t, n_r)).view(n_p, n_t, n_r))
        ctx.close()
    return feats, targets, iters


def learned_probe(pb, torch):
    """The learned-guess workload: BE conduction on the 192 x 192 x 384 shell at dt = 1e4 dt_E,
    PCG (mixed precision) to rtol 1e-10 from the zero, previous-step and learned (raw and judged)
    guesses.  The network is trained first on 2000 solves this library makes on 64 x 64 x 64
    seeded random profiles (targets smoothed as the guess smooths the network output)."""
    import synth
    from paper_2403_01004_gb300 import learned
    from synth import device
    n_train, train_shape, steps = 2000, (64, 64, 64), 6000
    t0 = time.perf_counter()
    feats, targ, gen_iters = learned_training_data(pb, torch, n_train, shape=train_shape, seed=7)
    torch.cuda.synchronize()
    t_gen = time.perf_counter() - t0
    t0 = time.perf_counter()
    model, loss = learned.train(feats, targ, steps=steps, batch=16, crop=24, border=4, lr=2e-3, seed=1)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del feats, targ
    wl = synth.WORKLOADS["shell192"]
    g = synth.make_grid(wl["n_r"], wl["n_t"], wl["n_p"], wl["q"])
    inp = synth.tc_inputs(g, wl["seed"])
    ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", device.tc_fields(inp), "fp64")
    u = torch.from_numpy(inp.T.reshape(-1)).cuda()
    dt = wl["ratio"] * pb.parabolic_dt_explicit(ctx)
    out = {}
    for name in ("zero", "previous", "learned_raw", "learned_judged"):
        x = u.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        x0 = None
        if name == "zero":
            x0 = torch.zeros_like(u)
        elif name.startswith("learned"):
            x0 = pb.learned_guess(ctx, model, u, dt)
        st = pb.be_pcg_advance(ctx, x, dt, use_ptl=False, rtol=1e-10, x0=x0, judge_guess=(name == "learned_judged"),
                               mixed=True)
        e1.record()
        torch.cuda.synchronize()
        out[name] = {"iterations": st["total_iters"], "ms": e0.elapsed_time(e1),
                     "rel_residual": st["final_rel_residual"], "started_from_guess": bool(st["guess_used"])}

    def best_ms(fn, reps=5):
        ts = []
        for _ in range(reps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            fn()
            e1.record()
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        return min(ts)

    # the guess alone (features, four conv layers, x0) and the four tensor-core conv layers alone;
    # per point a layer reads 16 bf16 channels and writes 16 (plus the 16 pre-activations of
    # layers 1-3, the float32 output of layer 4), and does 27 x 16 x 16 multiply-adds
    feats, _, _ = pb.pb_guess_features(ctx, u, dt)
    shape = (1, g.n_phi, g.n_theta, g.n_r)
    ms_guess = best_ms(lambda: pb.learned_guess(ctx, model, u, dt))
    ms_net = best_ms(lambda: pb.pb_model_forward(model, feats, shape, wrap_d=True))
    pts = ctx.n
    flops = 4 * 2 * 27 * 16 * 16 * pts
    layer_bytes = pts * (3 * (32 + 64) + (32 + 4))
    out["guess_ms"] = ms_guess
    out["network"] = {"ms": ms_net, "layers": 4, "points": pts, "TFLOP/s": flops / (ms_net / 1e3) / 1e12,
                      "alg_GB/s": layer_bytes / (ms_net / 1e3) / 1e9,
                      "note": "pb_model_forward: 4 tcgen05 conv layers (27 MMAs of 128 x 16 x 16 per 128 points), "
                              "plus a device copy of the input features and of the output"}
    ctx.close()
    model.close()
    return {"what": "BE + PC1 PCG (mixed precision, rtol 1e-10), 192x192x384 shell, dt = 1e4 dt_E, one solve per guess",
            "training": {"samples": n_train, "sample_grid": "x".join(map(str, train_shape)),
                         "solve_iterations": gen_iters, "generate_s": round(t_gen, 2), "steps": steps,
                         "batch": 16, "crop": 24, "train_s": round(t_train, 2), "last_batch_loss": loss},
            **out}


def ptl_study_probe(pb, torch, ctx_tc, ctx_v, d_u0, d_v0, wl):
    """The F_max localisation of Eq. 5 against the full-grid PTL (Eq. 4 over every pair of face
    neighbours) on the step's own states: both values before every cycle of the Eq. 5 step, the
    same step cycled by the full-grid value instead, and the full-grid pass's own rate."""
    import numpy as np
    out = {"what": "RKL2 step of each operator (dt = %g dt_E), float32: Eq. 5 (F_max) vs Eq. 4 over all "
                   "pairs (full), both evaluated before every cycle of the Eq. 5-driven step" % wl["ratio"]}
    for name, ctx, src in (("tc", ctx_tc, d_u0), ("visc", ctx_v, d_v0)):
        dte = pb.parabolic_dt_explicit(ctx)
        dt = wl["ratio"] * dte
        x = src.clone()
        st = pb.rkl2_advance(ctx, x, dt, use_ptl=True, record_full=True, stats_capacity=8192)
        fm = np.array(st["dt_ptl_cycle"], dtype=np.float64)
        fu = np.array(st["dt_full_cycle"], dtype=np.float64)
        ok = np.isfinite(fm) & np.isfinite(fu) & (fm > 0)
        r = fu[ok] / fm[ok]
        rec = {"cycles": st["cycles"], "stages": st["total_stages"],
               "full_below_fmax_by_0.1pct": float(np.mean(r < 0.999)) if r.size else None,
               "full_below_half_fmax": float(np.mean(r < 0.5)) if r.size else None,
               "ratio_full_over_fmax": {"min": float(r.min()), "median": float(np.median(r)), "max": float(r.max())}
               if r.size else None,
               "fmax_over_dtE": {"first": float(fm[0] / dte), "median": float(np.median(fm[ok]) / dte)},
               "full_over_dtE": {"first": float(fu[0] / dte), "median": float(np.median(fu[ok]) / dte)}}
        x = src.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        st2 = pb.rkl2_advance(ctx, x, dt, use_ptl=True, ptl_mode="full", raise_on_error=False)
        e1.record()
        torch.cuda.synchronize()
        rec["cycled_by_full"] = {"status": st2["status"], "cycles": st2["cycles"], "stages": st2["total_stages"],
                                 "ms": e0.elapsed_time(e1)}
        out[name] = rec
    # the full-grid pass alone (after its PTL pass), event-timed per launch
    pb.pb_profile_enable(ctx_tc, True)
    for _ in range(5):
        pb.ptl_full_compute(ctx_tc, d_u0)
    torch.cuda.synchronize()
    prof = {p["name"]: p for p in pb.pb_profile_read(ctx_tc)}
    pb.pb_profile_enable(ctx_tc, False)
    p = prof.get("tc.ptl_full")
    if p and p["timed_launches"]:
        ms = p["total_ms"] / p["timed_launches"]
        out["ptl_full_pass"] = {"ms_per_launch": round(ms, 4), "alg_bytes": p["bytes"] / p["launches"],
                                "GB/s": round(p["bytes"] / p["launches"] / (ms / 1e3) / 1e9, 1)}
    return out


def fig1_probe(pb, torch, n_phi=256, ratio=500.0):
    """Fig. 1 on the GPU.  Middle / right: the 1-D second-order heat equation at 500 explicit
    steps is the periodic conduction box 3 x 3 x n_phi with the field along phi (dt_E = 1/2 for
    states constant in r and theta); one step from a delta plane carries every mode, and the FFT
    along phi gives each mode's amplification, z_m = -1000 sin^2(pi m / n_phi).  Left: the
    estimated speedup over explicit Euler, (dt / dt_E) / s, from the library's stage counts."""
    import numpy as np
    from scipy.special import eval_gegenbauer, eval_legendre

    def closed(scheme, s, z):
        if scheme == "rkl2":
            b = (s * s + s - 2.0) / (2.0 * s * (s + 1.0))
            return (1 - b) + b * eval_legendre(s, 1.0 + 4.0 / (s * s + s - 2.0) * z)
        b = 4.0 * (s - 1.0) * (s + 4.0) / (3.0 * s * (s + 1.0) * (s + 2.0) * (s + 3.0))
        return 1.0 - b * (s + 1.0) * (s + 2.0) / 2.0 + b * eval_gegenbauer(s, 1.5, 1.0 + 6.0 / ((s + 4.0) * (s - 1.0)) * z)

    shape = (n_phi, 3, 3)
    ones = torch.ones(shape, dtype=torch.float64, device="cuda")
    fields = {"T0": ones, "n": ones, "B": [0 * ones, 0 * ones, ones]}
    ctx = pb.parabolic_setup_box(3, 3, n_phi, "tc", fields, "fp64", C=1.0)
    dt_e = pb.parabolic_dt_explicit(ctx)
    m = np.arange(n_phi)
    z = ratio * dt_e * (-4.0 * np.sin(np.pi * m / n_phi) ** 2)
    high = np.abs(z) > 0.5 * np.abs(z).max()
    out = {"what": "1-D heat equation (box 3x3x%d, field along phi), one step of %g dt_E from a delta plane; "
                   "amplification per Fourier mode" % (n_phi, ratio), "dt_E": dt_e, "z_min": float(z.min())}
    for scheme in ("rkl2", "rkg2", "be"):
        u = torch.zeros(shape, dtype=torch.float64, device="cuda")
        u[0] = 1.0
        u = u.reshape(-1)
        if scheme == "be":
            st = pb.be_pcg_advance(ctx, u, ratio * dt_e, use_ptl=False, rtol=1e-14, max_iter=20000)
            ref, s = 1.0 / (1.0 - z), None
        else:
            st = pb.rkl2_advance(ctx, u, ratio * dt_e, scheme=scheme, use_ptl=False)
            s = st["work_cycle"][0]
            ref = closed(scheme, s, z)
        amp = np.fft.fft(u.reshape(shape)[:, 1, 1].cpu().numpy()).real
        out[scheme] = {"stages": s, "pcg_iterations": st["total_iters"] if scheme == "be" else None,
                       "max_abs_amp_high_modes": float(np.abs(amp[high]).max()),
                       "spread_high_modes": float(np.ptp(amp[high])),
                       "max_dev_from_closed_form": float(np.abs(amp - ref).max())}
    out["exact_max_high_modes"] = float(np.exp(z[high]).max())
    speed = {}
    for r in (10.0, 30.0, 100.0, 300.0, 1000.0, 3000.0, 1e4, 3e4, 1e5):
        row = {}
        for scheme in ("rkl2", "rkg2"):
            u = torch.zeros(shape[0] * 9, dtype=torch.float64, device="cuda")
            st = pb.rkl2_advance(ctx, u, r * dt_e, scheme=scheme, use_ptl=False)
            row[scheme] = round(r / st["work_cycle"][0], 3)
        speed["%g" % r] = row
    out["estimated_speedup_vs_euler"] = speed
    ctx.close()
    return out


def precision_stress_probe(pb, torch, bf16_cap=5000):
    """The jump128 workload (128 x 256 x 512 shell, temperature jump at r = 1.02 over three radial
    cells, 5 % noise; RKL2 + PTL over dt = 1e5 dt_E) in float64, float32, bfloat16 storage and
    float64 storage with the float32 stencil (fp64s):
    each precision's own PTL schedule (cycles, stages, time; bfloat16 capped at bf16_cap cycles),
    and its error against the float64 oracle's sampled final state when it replays the oracle's
    schedule (tests/golden/jump128_rkl2_ptl.txt, written by the oracle-only script beside it)."""
    import importlib.util
    import numpy as np
    import synth
    from synth import device
    spec = importlib.util.spec_from_file_location("jump128_golden", os.path.join(ROOT, "tests", "jump128_golden.py"))
    golden = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(golden)
    if not os.path.exists(golden.PATH):
        return {"unavailable": "tests/golden/jump128_rkl2_ptl.txt missing"}
    gold = golden.load()
    wl = synth.WORKLOADS["jump128"]
    g = synth.make_grid(wl["n_r"], wl["n_t"], wl["n_p"], wl["q"])
    inp = synth.tc_inputs(g, wl["seed"], noise=wl["noise"], profile="jump")
    fields = device.tc_fields(inp)
    idx = torch.from_numpy(gold["idx"]).to("cuda")
    out = {"what": "jump128: 128x256x512 shell, T jump at r = 1.02 (3 cells), RKL2 + PTL over 1e5 dt_E",
           "oracle": {"cycles": len(gold["dt_c"]), "stages": int(sum(gold["s"]))}}
    for prec, dtype in (("fp64", torch.float64), ("fp32", torch.float32), ("bf16", torch.bfloat16),
                        ("fp64s", torch.float64)):
        ctx = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", fields, prec)
        dt = wl["ratio"] * pb.parabolic_dt_explicit(ctx)
        rec = {}
        for mode in ("own_ptl", "oracle_schedule"):
            u = torch.from_numpy(inp.T.reshape(-1)).to("cuda", dtype)
            kw = dict(use_ptl=True, max_cycles=bf16_cap) if mode == "own_ptl" else dict(forced=gold["dt_c"])
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            st = pb.rkl2_advance(ctx, u, dt, raise_on_error=False, **kw)
            e1.record()
            torch.cuda.synchronize()
            got = u[idx].to(torch.float64).cpu().numpy()
            rel = lambda sl: float(np.linalg.norm(got[sl] - gold["u"][sl]) / np.linalg.norm(gold["u"][sl]))
            rec[mode] = {"status": pb.load_library().pb_status_string(st["status"]).decode(),
                         "cycles": st["cycles"], "stages": st["total_stages"], "ms": round(e0.elapsed_time(e1), 2),
                         "rel_l2_vs_oracle_uniform_samples": rel(slice(0, 2048)),
                         "rel_l2_vs_oracle_jump_band": rel(slice(2048, 4096))}
        out[prec] = rec
        ctx.close()
    return out


def fp64_probe(pb, torch, g, d_tc, d_vi, d_u0, d_v0, wl, args, value32, result, schedule):
    """The same step with float64 storage and arithmetic (the plain FP64 GPU path), timed once,
    and the error of the timed step's results against it: relative L2 against the float64 run of
    the timed step's own cycle schedule (the precision alone), and against the float64 step with
    its own PTL decisions (precision and schedule together)."""
    c1 = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "tc", d_tc, "fp64")
    c2 = pb.parabolic_setup(g.r_face, g.t_face, g.n_phi, "visc", d_vi, "fp64")
    u = d_u0.to(torch.float64)
    v = d_v0.to(torch.float64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    s1 = pb.rkl2_advance(c1, u, wl["ratio"] * pb.parabolic_dt_explicit(c1), scheme=args.scheme)
    s2 = pb.rkl2_advance(c2, v, wl["ratio"] * pb.parabolic_dt_explicit(c2), scheme=args.scheme)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    units = c1.n * s1["total_stages"] + c2.n * s2["total_stages"]
    val = units / (ms / 1e3)

    def rel(a, b):
        a = a.to(torch.float64)
        return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

    acc = {"what": f"relative L2 of the timed {args.precision} step's results against the float64 GPU path",
           "tolerance": {"fp32": 1e-5, "bf16": 1e-2}.get(args.precision)}
    own = {"tc": (s1, u), "visc": (s2, v)}
    for name, ctx, x0 in (("tc", c1, d_u0), ("visc", c2, d_v0)):
        st64, x64 = own[name]
        same = list(st64["dt_cycle"]) == schedule[name] or (
            len(st64["dt_cycle"]) == len(schedule[name]) and
            all(abs(a - b) <= 1e-12 * abs(b) for a, b in zip(st64["dt_cycle"], schedule[name])))
        xf = x0.to(torch.float64)
        pb.rkl2_advance(ctx, xf, 0.0, scheme=args.scheme, forced=schedule[name])
        acc[name] = {"same_schedule_rel_l2": rel(result[name], xf),
                     "own_ptl_rel_l2": rel(result[name], x64),
                     "schedules_equal": bool(same), "cycles": len(schedule[name]), "cycles_fp64": st64["cycles"]}
    c1.close()
    c2.close()
    return ({"value": val, "unit": UNIT, "ms_per_step": ms, "speedup_of_main": value32 / val,
             "step": {"tc": dict(cycles=s1["cycles"], stages=s1["total_stages"]),
                      "visc": dict(cycles=s2["cycles"], stages=s2["total_stages"])}}, acc)


def oracle_first_cycle_probe(pb, torch, g, tc, ctx, d_u0, dt_c, args):
    """The timed step's first conduction cycle (its own length and stage count) at sampled points
    against the float64 oracle's stages on windows of the grid: after s stages a point depends
    only on points within s cells, so a window of margin s + 1 reproduces the full-grid result
    there (windows on the r boundaries, the poles and the phi wrap)."""
    from oracle.geometry import Shell
    from oracle.sts import rkl2_coefficients, rkg2_coefficients, sts_step
    from oracle.tc import TCOperator
    n_r, n_t, n_p = g.n_r, g.n_theta, g.n_phi
    x = d_u0.clone()
    st = pb.rkl2_advance(ctx, x, 0.0, scheme=args.scheme, forced=[dt_c])
    s = st["work_cycle"][0]
    co = (rkl2_coefficients if args.scheme == "rkl2" else rkg2_coefficients)(s)
    xh = x.to(torch.float64).cpu().numpy().reshape(n_p, n_t, n_r)
    uh = d_u0.to(torch.float64).cpu().numpy().reshape(n_p, n_t, n_r)
    m = s + 1
    got, ref = [], []
    for (k, j, i) in [(0, 0, 0), (n_p - 1, n_t - 1, n_r - 1), (37, n_t // 2, 3), (n_p // 2, 1, n_r * 3 // 4)]:
        i0, i1 = max(0, i - m), min(n_r, i + m + 1)
        j0, j1 = max(0, j - m), min(n_t, j + m + 1)
        ks = [(k + d) % n_p for d in range(-m, m + 1)]
        sl = lambda a: a[ks][:, j0:j1, i0:i1]
        sh = Shell(g.r_face[i0:i1 + 1], g.t_face[j0:j1 + 1], len(ks), dphi=2 * np.pi / n_p)
        op = TCOperator.spherical(sh, sl(tc.T), sl(tc.n), [sl(b) for b in tc.B])
        uw = sl(uh).reshape(-1)
        xo = sts_step(op.apply, uw, op.apply(uw), dt_c, co).reshape(op.shape)
        got.append(xh[k, j, i])
        ref.append(xo[m, j - j0, i - i0])
    got, ref = np.array(got), np.array(ref)
    return {"what": "first conduction cycle of the step at 4 sampled points (boundaries, poles, wrap) "
                    "against the float64 oracle on windows", "stages": s,
            "rel_l2": float(np.linalg.norm(got - ref) / np.linalg.norm(ref))}


# ---- CPU oracle -------------------------------------------------------------------------------
def oracle_rates(g, tc, vi, budget_s: float):
    """Point-stage rate of the oracle's conduction and viscosity stages on a window of the
    workload: 256 x 256 x 8 cells (full r and theta, 8 phi planes)."""
    import numpy as np
    from oracle.geometry import Shell
    from oracle.sts import rkl2_coefficients, sts_step
    from oracle.tc import TCOperator
    from oracle.visc import ViscOperator
    import synth

    kw = 8
    sh = Shell(g.r_face, g.t_face, kw, dphi=2 * np.pi / g.n_phi)
    op = TCOperator.spherical(sh, tc.T[:kw], tc.n[:kw], [b[:kw] for b in tc.B])
    u = tc.T[:kw].reshape(-1).copy()
    vop = ViscOperator.spherical(sh, [a[:kw] for a in vi.rho], [a[:kw] for a in vi.nu])
    v = np.concatenate([a[:kw].reshape(-1) for a in vi.v])
    out = {}
    for name, o, x in (("tc", op, u), ("visc", vop, v)):
        s = 4
        t0 = time.perf_counter()
        stages = 0
        while time.perf_counter() - t0 < budget_s / 2:
            y0 = o.apply(x)
            sts_step(o.apply, x, y0, 1e-9, rkl2_coefficients(s))
            stages += s
        out[name] = (o.n * stages / (time.perf_counter() - t0), o.n, stages)
    return out


def _window_rates(args):
    """One process's share of the all-cores oracle timing: the conduction and viscosity stage
    rates on its own 8-plane phi window (arrays sliced by the parent)."""
    r_face, t_face, n_phi, T, n, B, rho, nu, v, budget_s = args
    import numpy as np
    from oracle.geometry import Shell
    from oracle.sts import rkl2_coefficients, sts_step
    from oracle.tc import TCOperator
    from oracle.visc import ViscOperator
    kw = T.shape[0]
    sh = Shell(r_face, t_face, kw, dphi=2 * np.pi / n_phi)
    ops = (("tc", TCOperator.spherical(sh, T, n, B), T.reshape(-1).copy()),
           ("visc", ViscOperator.spherical(sh, rho, nu), np.concatenate([a.reshape(-1) for a in v])))
    out = {}
    for name, o, x in ops:
        s, stages = 4, 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < budget_s / 2:
            sts_step(o.apply, x, o.apply(x), 1e-9, rkl2_coefficients(s))
            stages += s
        out[name] = o.n * stages / (time.perf_counter() - t0)
    return out


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def cpu_baseline_all_cores(g, tc, vi, step_stats, n_tc, n_v, budget_s=8.0):
    """The oracle on every host core at once: one spawned process per core, each timing its own
    8-plane phi window of the workload; the per-core rates add up."""
    import multiprocessing as mp
    ncores = os.cpu_count() or 1
    kw = 8
    jobs = []
    for w in range(ncores):
        ks = [(kw * w + d) % g.n_phi for d in range(kw)]
        sl = lambda a: np.ascontiguousarray(a[ks])
        jobs.append((g.r_face, g.t_face, g.n_phi, sl(tc.T), sl(tc.n), [sl(b) for b in tc.B],
                     [sl(a) for a in vi.rho], [sl(a) for a in vi.nu], [sl(a) for a in vi.v], budget_s))
    with mp.get_context("spawn").Pool(ncores) as pool:
        res = pool.map(_window_rates, jobs)
    r_tc = sum(r["tc"] for r in res)
    r_v = sum(r["visc"] for r in res)
    st = step_stats
    t_est = n_tc * st["tc"]["stages"] / r_tc + n_v * st["visc"]["stages"] / r_v
    return {"value": (n_tc * st["tc"]["stages"] + n_v * st["visc"]["stages"]) / t_est, "unit": UNIT,
            "cores": ncores, "cpu_model": cpu_model(), "kind": "oracle",
            "sample": f"{ncores} spawned processes, each the NumPy float64 oracle on its own 256x256x8 phi "
                      f"window (~{budget_s:.0f} s); per-core rates summed, combined in the step's stage mix",
            "tc_point_stages_per_s": r_tc, "visc_point_stages_per_s": r_v}


def cpu_baseline(g, tc, vi, wl, step_stats, n_tc, n_v, budget_s=16.0):
    rates = oracle_rates(g, tc, vi, budget_s)
    st = step_stats
    t_est = n_tc * st["tc"]["stages"] / rates["tc"][0] + n_v * st["visc"]["stages"] / rates["visc"][0]
    value = (n_tc * st["tc"]["stages"] + n_v * st["visc"]["stages"]) / t_est
    return {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": (f"NumPy float64 oracle stages on a 256x256x8 phi window of the workload "
                       f"(conduction {rates['tc'][2]} stages, viscosity {rates['visc'][2]} stages, ~{budget_s:.0f} s); "
                       f"rates combined in the step's own conduction / viscosity stage mix"),
            "tc_point_stages_per_s": rates["tc"][0], "visc_point_stages_per_s": rates["visc"][0]}


def arm_config(args, wl, world):
    """The workload description both arms print."""
    return {"workload": f"{args.workload}: {wl['n_r']}x{wl['n_t']}x{wl['n_p']} shell, thermal conduction + "
                        f"3-component viscosity, {args.scheme.upper()} + PTL, dt = {wl['ratio']:g} dt_E per operator",
            "precision": args.precision, "scheme": args.scheme, "parallelism": f"replicas x{world}",
            "l2": "working set ~4 GB >> 129 MB L2: no flush needed"}


def run_reference(args):
    """The oracle as the reference arm: each step is a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    wl = WORKLOADS[args.workload]
    g, tc, vi = make_inputs(wl)
    # the stage mix of the GPU step (measured on GB300 for this workload), used to weight the
    # conduction and viscosity rates exactly as the main arm's metric does
    mix = {"tc": {"stages": 178}, "visc": {"stages": 2002}}
    n_tc = g.size
    n_v = (g.n_r - 1) * g.n_theta * g.n_phi + g.n_r * (g.n_theta - 1) * g.n_phi + g.size
    for _ in range(args.warmup):
        oracle_rates(g, tc, vi, 2.0)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(g, tc, vi, wl, mix, n_tc, n_v, budget_s=8.0)["value"])
    wall = time.perf_counter() - t0
    value = statistics.median(vals)
    cpu = {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": "per step: NumPy float64 oracle stages on a 256x256x8 phi window (~8 s), "
                     "conduction / viscosity rates weighted by the GPU step's stage mix"}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": arm_config(args, wl, int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": cpu, "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                                         "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    a = parse_args()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
