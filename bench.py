#!/usr/bin/env python
"""Benchmark of the FEM harmonic-inpainting data optimisation on GB300.

One step = the whole hot path on one seeded image.  Default (configuration
4, the largest): an 8193 x 8193 image with texture; create the two-triangle
mesh, spatial optimisation (top-k 1 % of triangles per round, newest-vertex
bisection, FP32 CG inside float-float iterative refinement, until 2 % of the
pixels are vertices), g = f at the mask vertices, 50 tonal CG iterations on
the normal equations through forward and adjoint solves.  value = image
Mpixel per second of whole-step time, inputs resident in HBM; e2e = the same
through the public API with the image copied from pinned host memory and the
result (mesh + g) copied back inside the timed region.  The plain FP64 GPU
path is timed on the same workload after the timed region (fp64_path).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank optimises its own image (seed + rank):
replicas, no collective on the data path; the barrier and the max over
ranks of the timed region are the only communication.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpixel/s FEM inpaint+tonal opt at 1e-6 rel err vs FP64"
# FP32 CG and FP32 pixel work; float-float (a pair of FP32, about 48 bits)
# for the refinement residuals and the per-pixel error sums; FP64 per
# triangle, per vertex and in the CG scalars
DTYPE_MIXED = "fp32+float-float+fp64"
UNIT = "Mpixel/s"
L2_FLUSH_BYTES = 512 << 20


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=4, choices=[1, 2, 3, 4, 6, 7],
                    help="1: 257^2 FP64, one triangle per round to 5%%, one solve + errors; 2: 1025^2 "
                         "spatial (1%% per round, 3%%) + tonal; 3: 2049^2 at 4%% + tonal; 4 (default): 8193^2 "
                         "textured at 2%% + 50 tonal iterations; 6: 1024^2 at 4%% + tonal (Table 2's size); "
                         "7: 4896 x 3264 textured at 2%% + 50 tonal iterations (Fig. 3's size); the serving "
                         "workload (5) is --serve")
    ap.add_argument("--n", type=int, default=None)
    ap.add_argument("--density", type=float, default=None)
    ap.add_argument("--frac", type=float, default=None)
    ap.add_argument("--tonal-tol", type=float, default=None)
    ap.add_argument("--precision", default=None, choices=["fp32ir", "fp64"])
    ap.add_argument("--inner-tol", type=float, default=None,
                    help="relative tolerance of the tonal inner solves (default: the library's 1e-11; 1e-13 in "
                         "configuration 4, whose 50th outer iterate is sensitive to the inner solves' accuracy)")
    ap.add_argument("--seed", type=int, default=None)
    ap.add_argument("--fast-keys", type=int, default=-1, choices=[-1, 0, 1, 2],
                    help="selection keys: -1 the library's choice by image size, 0 exact, 1 FP32 intervals + exact "
                         "band (incremental FP32 pass after the first round), 2 as 1 with a full FP32 pass every round")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-check", action="store_true", help="skip the FP64 accuracy check after timing")
    ap.add_argument("--no-fp64-timing", action="store_true", help="skip timing the plain FP64 GPU path")
    ap.add_argument("--ncu-step", action="store_true",
                    help="for ncu launch lists: one warm-up step, then exactly one step, no timing output")
    ap.add_argument("--serve", action="store_true",
                    help="configuration 5: serving with continuous batching (closed loop, then Poisson arrivals)")
    ap.add_argument("--requests", type=int, default=512)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--solve-micro", action="store_true",
                    help="time the Laplace solve alone on the refined mesh (FP32-IR and FP64), 20 solves each")
    ap.add_argument("--pass-micro", default=None,
                    help="comma-separated round counts: time the error pass over all squares (k_sq, FP32 with "
                         "error intervals) on the mesh after each number of spatial rounds, 10 passes each")
    ap.add_argument("--mesh-file", default=None,
                    help="with --pass-micro and one round count: import the mesh from this .npz file if it "
                         "exists, else refine and save it there (so that a profiler run launches few kernels "
                         "before the pass)")
    a = ap.parse_args()
    preset = PRESETS[a.config]
    for k, v in preset.items():
        if getattr(a, k, None) is None:
            setattr(a, k, v)
    return a


# seeded workloads (seed = configuration index - 1)
PRESETS = {
    1: dict(n=257, density=0.05, frac=0.0, seed=0, texture=False, tonal="none", tonal_tol=0.0, tonal_iters=0,
            precision="fp64", inner_tol=1e-11),
    2: dict(n=1025, density=0.03, frac=0.01, seed=1, texture=False, tonal="tol", tonal_tol=1e-8, tonal_iters=0,
            precision="fp32ir", inner_tol=1e-11),
    3: dict(n=2049, density=0.04, frac=0.01, seed=2, texture=False, tonal="tol", tonal_tol=1e-8, tonal_iters=0,
            precision="fp32ir", inner_tol=1e-11),
    4: dict(n=8193, density=0.02, frac=0.01, seed=3, texture=True, tonal="iters", tonal_tol=0.0, tonal_iters=50,
            precision="fp32ir", inner_tol=1e-13),
    # (5 is the serving workload, bench.py --serve)
    # the paper's own image sizes (general sizes in the smallest (2^L+1)^2
    # domain): Table 2's largest, 1024 x 1024 at 4 %, and the 4896 x 3264
    # photograph size of Fig. 3 (textured synthetic stand-in) at 2 %
    6: dict(n=1024, h=1024, density=0.04, frac=0.01, seed=4, texture=False, tonal="tol", tonal_tol=1e-8,
            tonal_iters=0, precision="fp32ir", inner_tol=1e-11),
    7: dict(n=4896, h=3264, density=0.02, frac=0.01, seed=5, texture=True, tonal="iters", tonal_tol=0.0,
            tonal_iters=50, precision="fp32ir", inner_tol=1e-13),
}


def image_hw(a):
    """(height, width) of the workload's image."""
    return (getattr(a, "h", None) or a.n), a.n


def make_workload_image(a, seed):
    import numpy as np
    import seeded_inputs
    H, W = image_hw(a)
    if H == W:
        return seeded_inputs.make_image(W, seed, texture=a.texture)
    return np.ascontiguousarray(seeded_inputs.make_image(max(W, H), seed, texture=a.texture)[:H, :W])


def workload_name(a):
    H, W = image_hw(a)
    sp = (f"{W}x{H} seeded image{' with texture' if a.texture else ''}: spatial optimisation "
          f"({'one triangle' if a.frac == 0 else f'top-k {a.frac:.0%} of triangles'} per round, NVB, to "
          f"{a.density:.0%} vertex density)")
    if a.tonal == "none":
        return sp + " + one Laplace solve + per-triangle errors"
    if a.tonal == "iters":
        return sp + f" + {a.tonal_iters} tonal CG iterations on B^T B g = B^T f"
    return sp + f" + tonal optimisation (CG on B^T B g = B^T f, tol {a.tonal_tol:g})"


def config(a, world):
    H, W = image_hw(a)
    return {"workload": workload_name(a), "config_index": a.config, "image": f"{W}x{H}", "density": a.density,
            "topk_frac": a.frac, "tonal": a.tonal, "tonal_tol": a.tonal_tol, "tonal_iters": a.tonal_iters,
            "inner_tol": a.inner_tol, "fast_keys": {-1: "auto", 0: "exact", 1: "fp32_band", 2: "fp32_band_full_pass"}[getattr(a, "fast_keys", -1)],
            "precision": a.precision, "seed": a.seed, "l2_flush": True,
            "parallelism": f"replicas{world}" if world > 1 else "single"}


# ------------------------------------------------------------------ helpers
def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, device) -> float:
    """The largest value over all ranks (the timed region's total); the only
    collective of the multi-GPU run, which otherwise runs independent replicas."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_seed(base_seed: int, rank: int) -> int:
    """Each rank optimises its own seeded image (replicas, weak scaling)."""
    return base_seed + rank


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev: int):
        self.dev = dev
        self.lines = []
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                      stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.p = None

    def _read(self):
        for line in self.p.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def traffic_record(family):
    """Per-launch DRAM bytes of the dominant kernel from a committed ncu
    summary, used only while the kernel source it was taken from is unchanged."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(p):
        return None
    import hashlib
    with open(p) as fh:
        rec = json.load(fh).get(family)
    if not rec:
        return None
    for name, want in rec.get("sources", {}).items():
        src = os.path.join(ROOT, "paper_2105_01586_gb300", "csrc", name)
        h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] if os.path.exists(src) else None
        if h != want:
            return None
    return rec["dram_bytes_per_launch"] if rec.get("sources") else None


# --------------------------------------------------------------- our arm
def run_ours(a, world, rank, local):
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_01586_gb300 as fem
    import seeded_inputs

    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n = a.n
    H, W = image_hw(a)
    P = W * H
    f_np = make_workload_image(a, replica_seed(a.seed, rank))
    f = torch.from_numpy(f_np).to(dev)
    prec = fem.FEM_PREC_FP64 if a.precision == "fp64" else fem.FEM_PREC_FP32_IR
    p = fem.params(topk_frac=a.frac, tonal_tol=a.tonal_tol, precision=prec, inner_tol=a.inner_tol,
                   fast_keys=a.fast_keys)
    if a.tonal == "iters":
        p.tonal_maxit = a.tonal_iters
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def run(f_dev, pp):
        mesh = fem.Mesh(W, H)
        mesh.spatial_refine(f_dev, a.density, pp)
        st_sp = mesh.stats()
        g = mesh.g_from_f(f_dev)
        if a.tonal == "none":
            # one Laplace solve and the per-triangle errors of the final mesh
            uv = torch.empty(mesh.V, dtype=torch.float64, device=f_dev.device)
            fem.fem_inpaint(mesh.h, g, None, uv, pp)
            err = torch.empty(mesh.T, dtype=torch.float64, device=f_dev.device)
            fem.fem_triangle_errors(mesh.h, uv, f_dev, err)
        else:
            fem.fem_tonal_opt(mesh.h, f_dev, g, pp, allow_not_converged=(a.tonal == "iters"))
        return mesh, g, st_sp

    def step(f_dev, keep=False, pp=None):
        mesh, g, _ = run(f_dev, pp or p)
        if keep:
            return mesh, g
        mesh.close()
        return None

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    if a.solve_micro:
        print(json.dumps(solve_micro(fem, torch, f, n, a)), flush=True)
        return
    if a.pass_micro:
        for line in pass_micro(fem, torch, f, n, a):
            print(json.dumps(line), flush=True)
        return

    if a.ncu_step:
        step(f)
        torch.cuda.synchronize(dev)
        n0 = fem.fem_launch_count()
        step(f)
        torch.cuda.synchronize(dev)
        print(json.dumps({"ncu_step_launches": fem.fem_launch_count() - n0, "warmup_launches": n0}), flush=True)
        return

    for _ in range(a.warmup):
        step(f)
    # which kernel family dominates (one profiled step, all families)
    fem.fem_profile_enable(True)
    step(f)
    prof_all = fem.fem_profile_read()
    fem.fem_profile_enable(False)
    # The roofline is reported for the step's top kernel among the three
    # with a per-unit algorithmic byte model: the square-tiled error pass
    # ("raster_pass", k_sq over all squares), the component solve ("cg",
    # k_solve_comp) or the system build ("assembly", k_build_system).
    # Refinement and top-k are chains of short kernels.
    dom = max(("raster_pass", "cg", "assembly"), key=lambda k: prof_all[k]["ms"])

    def steps_timed(k=None, pp=None):
        times = []
        for _ in range(a.steps if k is None else k):
            flush.zero_()
            torch.cuda.synchronize(dev)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(f, pp=pp)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        return times

    # timed region: K steps, L2 flushed between steps (outside the events),
    # no per-kernel events (an event between two kernels ends the launch
    # overlap of programmatic dependent launch and would slow the step)
    barrier()
    clk = ClockSampler(local)
    clk.start()
    launches0 = fem.fem_launch_count()
    times = steps_timed()
    launches = fem.fem_launch_count() - launches0
    clocks = clk.stop()
    total_ms = max_over_ranks(sum(times), dev)
    barrier()
    ms_per_step = total_ms / a.steps
    value = world * P / 1e6 / (ms_per_step / 1e3)

    # roofline region: the same K steps again, with the dominant family's
    # launches bracketed by events on the launching stream
    fem.fem_profile_enable(dom)
    prof_times = steps_timed()
    prof = fem.fem_profile_read()[dom]
    fem.fem_profile_enable(False)

    # the plain FP64 GPU path on the same workload (same parameters but the
    # precision), timed the same way after the timed region
    fp64_path = None
    if not a.no_fp64_timing and a.precision != "fp64":
        p64t = fem.params(topk_frac=a.frac, tonal_tol=a.tonal_tol, precision=fem.FEM_PREC_FP64,
                          inner_tol=a.inner_tol, fast_keys=a.fast_keys)
        if a.tonal == "iters":
            p64t.tonal_maxit = a.tonal_iters
        step(f, pp=p64t)
        k64 = max(1, min(a.steps, 3))
        t64 = steps_timed(k64, p64t)
        ms64 = sum(t64) / k64
        fp64_path = {"ms_per_step": round(ms64, 3), "value": round(P / 1e6 / (ms64 / 1e3), 4), "unit": UNIT,
                     "steps": k64, "mixed_precision_speedup": round(ms64 / ms_per_step, 4)}

    # end to end through the public API: pinned host image in, mesh + g out
    f_host = torch.from_numpy(f_np).pin_memory()
    e2e_times = []
    h2d = d2h = 0
    for _ in range(max(1, min(a.steps, 3))):
        flush.zero_()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        f_dev = f_host.to(dev, non_blocking=True)
        mesh, g = step(f_dev, keep=True)
        g_host = g.cpu()
        xy, tri, mk = mesh.export()
        torch.cuda.synchronize(dev)
        e2e_times.append((time.perf_counter() - t0) * 1e3)
        h2d = f_host.numel() * 4
        d2h = g_host.numel() * 4 + xy.nbytes + tri.nbytes + mk.nbytes
        mesh.close()
    e2e_ms = statistics.mean(e2e_times)
    e2e = {"value": round(world * P / 1e6 / (e2e_ms / 1e3), 4), "unit": UNIT, "h2d_bytes_per_step": h2d,
           "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3)}

    # accuracy vs the plain FP64 GPU path (outside the timed region): same
    # mesh expected; g compared at tight tolerance, or after the same number
    # of tonal iterations when the workload fixes the iteration count
    mem0 = torch.cuda.mem_get_info(dev)[0]
    mesh, g, st_sp = run(f, p)
    mem1 = torch.cuda.mem_get_info(dev)[0]
    st = mesh.stats()
    info = mesh.info
    extra = {"V": info[0], "T": info[1], "nmask": info[2], "rounds": st_sp["rounds"],
             "min_topk_margin": st_sp["min_margin"], "cg_iters_spatial": st_sp["cg_iters"],
             "solves_spatial": st_sp["solves"], "hbm_bytes_in_use_after_step": int(mem0 - mem1)}
    if a.tonal != "none":
        extra.update({"tonal_iters": st["tonal_iters"], "tonal_relres": st["tonal_relres"],
                      "cg_iters_tonal": st["cg_iters"], "solves_tonal": st["solves"]})
    gxy, gtri, gmk = mesh.export()
    gpu_info = {"xy": gxy, "tri": gtri, "mask": gmk, "rounds": st_sp["rounds"],
                "tonal_iters": st.get("tonal_iters", 0) if a.tonal != "none" else 0}
    if not a.no_check and a.precision != "fp64":
        p64 = fem.params(topk_frac=a.frac, precision=fem.FEM_PREC_FP64, tonal_tol=1e-12, inner_tol=1e-13,
                         tonal_maxit=20000)
        if a.tonal == "iters":
            p64.tonal_maxit = a.tonal_iters
            p64.tonal_tol = 0.0
        s2, g64, _ = run(f, p64)
        extra["mesh_equal_fp64"] = bool(all(np.array_equal(x, y) for x, y in zip((gxy, gtri, gmk), s2.export())))
        if a.tonal != "none":
            rel = float(torch.linalg.vector_norm(g.double() - g64.double()) / torch.linalg.vector_norm(g64.double()))
            extra["rel_err_vs_fp64"] = rel
        s2.close()
    mesh.close()
    if a.tonal == "none":
        extra["note"] = "per-triangle errors via fem_triangle_errors after one FP64 solve"

    peak, peak_kind = measured_peaks()
    per_launch_bytes = prof["bytes"] / max(1, prof["launches"])
    per_launch_ms = prof["ms"] / max(1, prof["launches"])
    achieved = per_launch_bytes / (per_launch_ms / 1e3) / 1e9 if per_launch_ms > 0 else 0.0
    roofline = {"bound": "hbm", "kernel_family": dom, "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4), "traffic": traffic_record(dom), "peak_kind": peak_kind,
                "region": f"{a.steps} steps after the timed region, the family's launches bracketed by events",
                "launches_in_region": prof["launches"], "ms_in_region": round(prof["ms"], 3),
                "share_of_step": round(prof["ms"] / sum(prof_times), 4),
                "family_ms_one_step": {k: round(v["ms"], 3) for k, v in prof_all.items()}}
    # the three families with a byte model, from the one profiled step
    fams = {}
    for k in ("raster_pass", "cg", "assembly"):
        v = prof_all[k]
        gbs = v["bytes"] / (v["ms"] / 1e3) / 1e9 if v["ms"] > 0 else 0.0
        fams[k] = {"ms": round(v["ms"], 3), "launches": v["launches"], "achieved": round(gbs, 2),
                   "frac": round(gbs / peak, 4)}
    roofline["families_one_step"] = fams

    line = {"metric": METRIC, "value": round(value, 4), "unit": UNIT, "n_gpus": world, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": round(ms_per_step, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if a.precision == "fp64" else DTYPE_MIXED,
            "data": "synthetic", "config": config(a, world), "roofline": roofline, "e2e": e2e, "clocks": clocks,
            "gpu_launches": int(launches)}
    if fp64_path:
        line["fp64_path"] = fp64_path
    line.update(extra)
    if rank == 0 and world == 1 and not a.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(a, f_np, gpu_info)
        line["cpu_baseline_openmp"] = cpu_baseline_openmp(a, f_np, gpu_info)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def pass_micro(fem, torch, f, n, a):
    """The error pass alone (the kernel that reads every pixel once per
    round) on the meshes the spatial optimisation reaches after the given
    numbers of rounds: device time per pass from CUDA events around the
    kernel, algorithmic bytes (4 B per pixel, 32 B per triangle, 16 B per
    vertex) per second, and the fraction of the measured HBM bandwidth."""
    peak, _ = measured_peaks()
    out = []
    import numpy as np
    for rounds in [int(x) for x in str(a.pass_micro).split(",")]:
        mesh = fem.Mesh(n)
        if a.mesh_file and os.path.exists(a.mesh_file):
            z = np.load(a.mesh_file)
            mesh.import_(z["xy"], z["tri"], z["mask"])
        else:
            # exact keys in the loop, so that the fast pass runs only below
            mesh.spatial_refine(f, a.density, fem.params(topk_frac=a.frac, max_rounds=rounds, fast_keys=0))
            if a.mesh_file:
                xy, tri, mk = mesh.export()
                np.savez(a.mesh_file, xy=xy, tri=tri, mask=mk)
        g = mesh.g_from_f(f)
        _, uv = mesh.inpaint(g, want_uv=True)
        for _ in range(3):
            mesh.triangle_error_bounds(uv, f)
        torch.cuda.synchronize()
        fem.fem_profile_enable("raster_pass")
        for _ in range(10):
            mesh.triangle_error_bounds(uv, f)
        prof = fem.fem_profile_read()["raster_pass"]
        fem.fem_profile_enable(False)
        us = 1e3 * prof["ms"] / max(1, prof["launches"])
        gbs = prof["bytes"] / max(1, prof["launches"]) / (us * 1e-6) / 1e9 if us > 0 else 0.0
        V, T, K = mesh.info
        out.append({"pass_micro": True, "rounds": rounds, "V": V, "T": T, "us_per_pass": round(us, 2),
                    "gbs": round(gbs, 1), "frac": round(gbs / peak, 4)})
        mesh.close()
    return out


def solve_micro(fem, torch, f, n, a):
    """Laplace solves on the mesh of the spatial optimisation, with g = f at
    the mask perturbed each call so that every solve iterates from the
    previous solution.  Wall time per fem_inpaint call (host timer, includes
    the launch and the result read-back) and CG iterations."""
    import numpy as np
    mesh = fem.Mesh(n)
    mesh.spatial_refine(f, a.density, fem.params(topk_frac=a.frac))
    g = mesh.g_from_f(f)
    out = {"nU": mesh.V - mesh.nmask, "V": mesh.V}
    for name, prec in (("fp32ir", fem.FEM_PREC_FP32_IR), ("fp64", fem.FEM_PREC_FP64)):
        p = fem.params(precision=prec)
        for _ in range(3):
            fem.fem_inpaint(mesh.h, g, None, None, p)
        times, its = [], []
        idx = torch.arange(g.numel(), device=g.device, dtype=torch.float32)
        for k in range(20):
            gg = (g + 1e-3 * torch.sin(idx * (k + 1))).contiguous()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fem.fem_inpaint(mesh.h, gg, None, None, p)
            torch.cuda.synchronize()
            times.append(time.perf_counter() - t0)
            its.append(mesh.stats()["cg_iters"])
        out[name] = {"ms_per_solve": round(1e3 * float(np.median(times)), 4), "cg_iters": float(np.median(its))}
    mesh.close()
    return out


# ------------------------------------------------------- the oracle on CPU
def oracle_job(a, f_np, tonal_iters=None):
    """The oracle on the whole workload of configurations 1-2; tonal_iters
    caps the tonal outer iterations (None: run to the tolerance).  Returns
    (spatial s, tonal-or-solve s, outer iterations, rounds)."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    om, log = oracle.spatial(f_np, a.density, a.frac)
    t1 = time.perf_counter()
    if a.tonal == "none":
        v, _, _ = oracle.solve(om, oracle.g_from_f(om, f_np))
        oracle.raster(om, v, f_np)
        return t1 - t0, time.perf_counter() - t1, 0, len(log)
    g, st = oracle.tonal(om, f_np, tol=a.tonal_tol if a.tonal == "tol" else 0.0,
                         maxit=tonal_iters or (a.tonal_iters if a.tonal == "iters" else 100000), inner_tol=a.inner_tol,
                         allow_not_converged=True)
    return t1 - t0, time.perf_counter() - t1, st["iters"], len(log)


# Whole-job counts of the sampled workloads: spatial rounds and tonal outer
# iterations.  The spatial optimisation is deterministic and its meshes are
# the same on every correct implementation (bit-exact topology), so the round
# count is a property of the seeded workload; the 8193^2 workload fixes 50
# tonal iterations.
JOB_COUNTS = {3: (362, 63), 4: (541, 50)}


def oracle_sample(a, f_np, tonal_mesh=None, rounds=2):
    """A bounded sample of the oracle's work on the workload: the first
    `rounds` spatial rounds from the two-triangle mesh, then one tonal outer
    iteration (tonal(maxit=1): the set-up passes B^T f, B g0, B^T r and one
    iteration) on `tonal_mesh` (default: the mesh the sample reached).
    Returns (seconds per round, seconds of tonal(maxit=1), total seconds)."""
    import oracle
    t0 = time.perf_counter()
    om, _ = oracle.spatial(f_np, a.density, a.frac, max_rounds=rounds)
    t1 = time.perf_counter()
    oracle.tonal(tonal_mesh if tonal_mesh is not None else om, f_np, tol=0.0, maxit=1, inner_tol=a.inner_tol,
                 allow_not_converged=True)
    t2 = time.perf_counter()
    return (t1 - t0) / rounds, t2 - t1, t2 - t0


def project_job(t_round, t_tonal1, rounds, iters):
    """Whole-job seconds from a sample: every round costs a sampled round, and
    the tonal run costs its set-up plus `iters` iterations, where tonal(maxit=1)
    is three set-up applications of B or B^T and one iteration of two (each a
    pixel pass plus a solve), so one application costs t_tonal1 / 5."""
    return t_round * rounds + t_tonal1 / 5.0 * (3 + 2 * iters)


def cpu_baseline(a, f_np, gpu):
    """The oracle on the host cores.  Configurations 1-2: the whole workload,
    once.  Larger images: a bounded sample (oracle_sample: the first spatial
    rounds, and one tonal iteration on the GPU's final mesh) scaled to the
    whole job by the GPU run's round and iteration counts (project_job).  The
    sampled rounds run on the smallest meshes of the loop, so the estimate is
    a lower bound on the oracle's time."""
    import oracle
    H, W = image_hw(a)
    P = W * H
    if max(W, H) <= 1025:
        ts, tt, it, rounds = oracle_job(a, f_np)
        what = "tonal" if a.tonal != "none" else "solve + errors"
        return {"value": round(P / 1e6 / (ts + tt), 6), "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"one full run of the workload by the FP64 C oracle (single thread): spatial {rounds} "
                          f"rounds {ts:.1f} s + {what} ({it} outer iterations) {tt:.1f} s"}
    R = 4
    N = 3
    while N < max(W, H):
        N = 2 * N - 1
    om = oracle.Mesh(N, gpu["xy"][:, 0].copy(), gpu["xy"][:, 1].copy(), gpu["mask"].copy(), gpu["tri"][:, 0].copy(),
                     gpu["tri"][:, 1].copy(), gpu["tri"][:, 2].copy(), W, H)
    t_round, t_tonal1, _ = oracle_sample(a, f_np, tonal_mesh=om, rounds=R)
    est = project_job(t_round, t_tonal1, gpu["rounds"], gpu["tonal_iters"])
    return {"value": round(P / 1e6 / est, 6), "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"bounded sample by the FP64 C oracle (single thread): the first {R} spatial rounds "
                      f"({t_round:.2f} s each, scaled to {gpu['rounds']} rounds) + one tonal iteration with its "
                      f"set-up on the GPU's final mesh ({t_tonal1:.2f} s, scaled to {gpu['tonal_iters']} "
                      f"iterations); estimated {est:.0f} s for the job (a lower bound: the sampled rounds run on "
                      f"the loop's smallest meshes)"}


def cpu_baseline_openmp(a, f_np, gpu):
    """The same measurement as cpu_baseline with the oracle's OpenMP build on
    all host cores (raster and A_UU x parallel, bit-identical results)."""
    import oracle
    try:
        oracle.build(openmp=True)
        cores = oracle.use_openmp(True)
    except Exception as e:  # noqa: BLE001
        return {"unavailable": f"OpenMP build of the oracle failed: {e}"}
    try:
        out = cpu_baseline(a, f_np, gpu)
    finally:
        oracle.use_openmp(False)
    out["cores"] = cores
    out["kind"] = "oracle_openmp"
    out["sample"] = out["sample"].replace("(single thread)", f"(OpenMP build, {cores} threads)")
    return out


def run_reference(a, world, rank):
    """The oracle as the reference arm, on the same workload.  Configurations
    1-2: each step runs the whole job (spatial optimisation and tonal
    optimisation to the tolerance).  Configurations 3-4 (hours on one core):
    each step runs a bounded sample of the job (oracle_sample: 2 spatial rounds
    and one tonal iteration), ms_per_step is that sample's wall time, and value
    is the whole job's throughput projected from it (project_job with the
    workload's round and iteration counts, JOB_COUNTS)."""
    if rank != 0:
        return
    H, W = image_hw(a)
    f_np = make_workload_image(a, a.seed)
    P = W * H
    base = {"metric": METRIC, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config(a, 1), "impl": "reference"}
    if a.config in (1, 2, 6):
        for _ in range(a.warmup):
            oracle_job(a, f_np)
        times, its, rounds = [], 0, 0
        for _ in range(a.steps):
            ts, tt, its, rounds = oracle_job(a, f_np)
            times.append(ts + tt)
        ms = 1e3 * statistics.mean(times)
        value = P / 1e6 / (ms / 1e3)
        sample = (f"each step the whole job by the FP64 C oracle (single thread): spatial optimisation "
                  f"({rounds} rounds) + " + (f"tonal optimisation ({its} outer iterations)" if a.tonal != "none"
                                              else "one solve + per-triangle errors"))
        extra = {}
    else:
        if a.config not in JOB_COUNTS:
            print(json.dumps({"impl": "reference", "unavailable": f"no recorded round count for configuration {a.config}"}))
            return
        rounds, iters = JOB_COUNTS[a.config]
        for _ in range(a.warmup):
            oracle_sample(a, f_np)
        samples = [oracle_sample(a, f_np) for _ in range(a.steps)]
        ms = 1e3 * statistics.mean(x[2] for x in samples)
        t_round = statistics.median(x[0] for x in samples)
        t_tonal1 = statistics.median(x[1] for x in samples)
        est = project_job(t_round, t_tonal1, rounds, iters)
        value = P / 1e6 / est
        sample = (f"each step a bounded sample by the FP64 C oracle (single thread): the first 2 spatial rounds "
                  f"({t_round:.2f} s each) + one tonal iteration with its set-up ({t_tonal1:.2f} s); value "
                  f"projected to the whole job ({rounds} rounds, {iters} tonal iterations): {est:.0f} s, a lower "
                  f"bound (the sampled rounds run on the loop's smallest meshes)")
        extra = {"projection": {"job_seconds": round(est, 1), "rounds": rounds, "tonal_iters": iters,
                                "sample_seconds_per_step": round(ms / 1e3, 3)}}
    line = dict(base)
    line.update({"value": round(value, 6), "ms_per_step": round(ms, 3),
                 "cpu_baseline": {"value": round(value, 6), "unit": UNIT, "kind": "oracle", "cores": 1,
                                  "sample": sample},
                 "e2e": {"value": round(value, 6), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}})
    line.update(extra)
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------ serving
def _make_image_job(args):
    import seeded_inputs
    n, seed = args
    return n, seed, seeded_inputs.make_image(n, seed)


def run_serving(a, world, rank):
    """Configuration 5: requests with side drawn from {257, 513, 1025, 2049}
    and density from U[2 %, 10 %], each a spatial + tonal optimisation of a
    seeded image, served by fem_server (continuous batching, admission by
    device memory).  Closed loop first (all requests at once) for the
    saturated throughput, then Poisson arrivals at 0.8x and 0.5x of it."""
    import numpy as np
    from concurrent.futures import ProcessPoolExecutor
    import multiprocessing as mp
    if rank != 0:
        return
    R = a.requests
    rng = np.random.default_rng(4)
    sides = rng.choice([257, 513, 1025, 2049], size=R)
    dens = rng.uniform(0.02, 0.10, size=R)
    pool_n = 8
    jobs = [(int(n), int(n) * 1000 + j) for n in (257, 513, 1025, 2049) for j in range(pool_n)]
    with ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4), mp_context=mp.get_context("spawn")) as ex:
        images = {(n, sd): img for n, sd, img in ex.map(_make_image_job, jobs)}

    def image(i):
        n = int(sides[i])
        return images[(n, n * 1000 + i % pool_n)]

    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_2105_01586_gb300 as fem
    from paper_2105_01586_gb300.serving import Server
    torch.cuda.init()
    p = fem.params(tonal_tol=1e-6)
    mpx = float(np.sum(sides.astype(np.float64) ** 2)) / 1e6

    def run(arrivals):
        with Server(slots=a.slots) as sv:
            t0 = time.perf_counter()
            ids = []
            for i in range(R):
                if arrivals is not None:
                    dt = arrivals[i] - (time.perf_counter() - t0)
                    if dt > 0:
                        time.sleep(dt)
                ids.append(sv.submit(image(i), float(dens[i]), p))
            res = []
            for rid in ids:
                sv.wait(rid)
                res.append(sv.result(rid))
                sv.release(rid)
        lat = np.array([r["t_end"] - r["t_submit"] for r in res]) * 1e3
        span = max(r["t_end"] for r in res) - min(r["t_submit"] for r in res)
        bad = sum(1 for r in res if r["status"] not in (0, 4))
        ratio = np.array([r["mem_measured"] / r["mem_estimate"] for r in res if r["mem_estimate"] > 0])
        return {"requests": R, "makespan_s": round(span, 3), "mpixel_per_s": round(mpx / span, 3),
                "requests_per_s": round(R / span, 3), "p50_ms": round(float(np.percentile(lat, 50)), 2),
                "p99_ms": round(float(np.percentile(lat, 99)), 2), "failed": bad,
                "mem_measured_over_estimate": {"median": round(float(np.median(ratio)), 4),
                                               "max": round(float(ratio.max()), 4)} if ratio.size else None}

    # warm-up: one request of each size
    with Server(slots=4) as sv:
        for n in (257, 513, 1025, 2049):
            rid = sv.submit(images[(n, n * 1000)], 0.05, p)
            sv.wait(rid)
    closed = run(None)
    lam = closed["requests_per_s"]
    out = {"closed_loop": closed}
    for load in (0.8, 0.5):
        arr = np.cumsum(np.random.default_rng(7).exponential(1.0 / (load * lam), size=R))
        out[f"poisson_{load}"] = run(arr)
    main = out["poisson_0.8"]
    line = {"metric": "serving Mpixel/s and p50/p99 latency (Poisson arrivals at 0.8x saturated throughput)",
            "value": main["mpixel_per_s"], "unit": "Mpixel/s", "p50_ms": main["p50_ms"], "p99_ms": main["p99_ms"],
            "n_gpus": 1, "higher_is_better": True, "dtype": DTYPE_MIXED, "data": "synthetic",
            "config": {"workload": f"{R} requests, side from {{257,513,1025,2049}}, density U[2%,10%], spatial + "
                                   f"tonal (tol 1e-6) each", "slots": a.slots, "config_index": 5},
            "runs": out}
    print(json.dumps(line), flush=True)


def main():
    a = parse()
    world, rank, local = dist_setup()
    if a.warmup < 3:
        a.warmup = 3
    if a.impl == "reference":
        run_reference(a, world, rank)
    elif a.serve:
        run_serving(a, world, rank)
    else:
        run_ours(a, world, rank, local)


if __name__ == "__main__":
    main()
