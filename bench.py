"""Benchmark of the FFT Lippmann-Schwinger iteration on GB300.

Workload (one "step"): the paper's square array of squares at 25 % volume
fraction on an 8192 x 8192 grid, inclusion conductivities sigma_1 in
{0.01, 0.1, 10, 100, 1e4}, each solved to a relative sigma_* change of 1e-6
(three consecutive iterates) with the basic Moulinec-Suquet scheme and with the
accelerated scheme (Eyre-Milton in the substituted space H'') using the
paper's pole-interval estimate [alpha, beta] = [1/4, 4]; FP32 fields (real
sigma_1: the packed real layout, two half-spectrum planes), FP64 reductions,
trigonometric Green symbol.  Inputs are synthetic and already
resident on the device for `value`; `e2e` repeats the step through the C ABI
from a pinned host mask to pinned host copies of every field E.

Prints one JSON line (rank 0).  `--impl reference` times the FP64 CPU oracle
instead on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from synth import SIGMA1_SWEEP_2D, square_array_mask  # noqa: E402

METRIC = "voxel-iters/s; time-to-1e-6 σ* accelerated vs basic MS; % HBM roofline"
UNIT = "voxel-iters/s"
SCHEMES = ("ms", "em", "em_sub")       # basic MS vs Eyre-Milton vs accelerated (EM in H'')
ALPHA_BETA = (0.25, 4.0)          # the Moulinec-Suquet estimate quoted in the paper
TOL = 1e-6
FRACTION = 0.25
# Lanczos extreme nodes lie inside the weighted spectrum, so the estimated slit
# is a little short; widening it only slows convergence slightly (section
# "Estimating the parameters alpha and beta"), a short one can diverge.
HULL_MARGIN = 0.05


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="ours", choices=("ours", "reference"))
    p.add_argument("--n", type=int, default=8192)
    p.add_argument("--green", default="trig", choices=("trig", "fd"))
    p.add_argument("--sigmas", default=",".join(str(s) for s in SIGMA1_SWEEP_2D))
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--pass-reps", type=int, default=20)
    p.add_argument("--workload", default="square2d",
                   choices=("square2d", "lattice64", "cube3d", "sweep", "adjoint", "fig5", "passes", "cufft",
                            "precision"),
                   help="square2d (default): the headline 2-D square-array sweep; the others measure the "
                        "64^2 FP64 lattice, the 3-D cubic arrays, the batched complex-sigma_1 sweep and the "
                        "adjoint (gradient) configuration, one JSON line each")
    p.add_argument("--sweep-sigmas", type=int, default=16, help="sweep: sigma_1 values per microstructure per step")
    p.add_argument("--fd-voxels", type=int, default=64, help="adjoint: voxels checked by central differences")
    p.add_argument("--fig-iters", type=int, default=600, help="fig5: iteration cap per curve")
    p.add_argument("--dim", type=int, default=2, choices=(2, 3), help="passes: 2-D or 3-D square array")
    p.add_argument("--plot-dir", default=None,
                   help="fig5: also write the two convergence plots (SVG) and their data (JSON) here")
    return p.parse_args()


def workload_config(args, sigmas):
    return {
        "workload": f"2D square array of squares (f=0.25), {args.n}x{args.n}, sigma1 in {list(sigmas)}, "
                    f"MS vs EM vs EM-in-H'' (alpha,beta)=(1/4,4), rel. sigma* change {TOL:g} x3, "
                    f"{args.green} Green symbol",
        "n": args.n, "d": 2, "sigma1": list(sigmas), "schemes": list(SCHEMES), "alpha_beta": list(ALPHA_BETA),
        "tol": TOL, "green": args.green, "fields": "FP32 (packed real layout: two half-spectrum planes), FP64 reductions",
        "l2": f"inputs larger than L2: every pass streams the state "
              f"({2 * (args.n // 2 + 4) * args.n * 8 / 1e9:.2f} GB of half-spectrum planes) against a 129 MB L2",
    }


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(name)
        os.unlink(self.path)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(smax)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# roofline helpers
# ---------------------------------------------------------------------------
def algorithmic_bytes(kind, scheme, N, d=2, fraction=FRACTION, cbytes=8, packed=False):
    """Bytes a pass must move per launch (FP32 fields, 1-byte mask).

    Complex layout: each of the d components is a complex plane (cbytes per
    voxel).  Packed real layout (2-D, real coefficients): the d = 2 real
    components share one complex plane, so the field costs cbytes per voxel.
    row pass: read + write the Q field and read the mask (1 B); the substituted
    schemes also read + write S (and T) on phase-1 voxels only.
    strided pass: read + write the Q field.
    """
    per_field = cbytes if packed else d * cbytes
    if kind == "row":
        extra = {"ms": 0, "em": 0, "ms_sub": 2, "em_sub": 4}[scheme] * per_field * fraction
        return N * (2 * per_field + 1 + extra)
    return N * 2 * per_field


def kernel_source_hash():
    h = hashlib.sha256()
    for p in sorted(glob.glob(os.path.join(ROOT, "paper_2001_08289_gb300", "csrc", "*"))):
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


def ncu_traffic(kernel, workload_key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel sources (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(path):
        return None
    data = json.load(open(path))
    if data.get("source_hash") != kernel_source_hash():
        return None
    ent = data.get("kernels", {}).get(f"{kernel}|{workload_key}")
    return None if ent is None else ent.get("dram_bytes_per_launch")


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, its FFTs on every host core
# ---------------------------------------------------------------------------
def oracle_sample(n, sigmas, schemes=("ms",), updates=1):
    """`updates` iterations (sigma_k evaluation + update) of each scheme on the
    n x n square array; returns (voxel-iterations, seconds)."""
    from oracle import schemes as S

    mask = square_array_mask(n)
    vox = 0
    t0 = time.perf_counter()
    for s1 in sigmas:
        for sch in schemes:
            pb = S.Problem(mask, s1, np.array([1.0, 0.0]), "trig")
            sc = S.make_scheme(pb, sch, *ALPHA_BETA)
            st = sc.init_state()
            for _ in range(updates):
                sc.observe(st)
                st = sc.update(st)
                vox += mask.size
    return vox, time.perf_counter() - t0


def oracle_cores():
    from oracle import fourier

    return int(fourier.WORKERS)


def cpu_baseline_block(n=8192, updates=5):
    vox, dt = oracle_sample(n, (10.0,), updates=updates)
    return {"value": vox / dt, "unit": UNIT, "cores": oracle_cores(), "kind": "oracle",
            "sample": f"{updates} MS iterations (sigma_k evaluation + update) at sigma1=10 on the {n}x{n} square "
                      f"array, FP64 numpy oracle with scipy.fft on {oracle_cores()} threads, {dt:.1f} s"}


def run_reference(args, sigmas):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = args.n
    s1 = sigmas[len(sigmas) // 2]
    for _ in range(args.warmup):
        oracle_sample(min(n, 2048), (s1,))       # warm-up: imports, FFT plans, page-in
    vox, dt = 0, 0.0
    for _ in range(args.steps):
        v, t = oracle_sample(n, (s1,))
        vox += v
        dt += t
    value = vox / dt
    sample = (f"per step: one MS iteration (sigma_k evaluation + update) at sigma1={s1} on the {n}x{n} square "
              f"array (FP64 numpy oracle, scipy.fft on {oracle_cores()} threads)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex)",
            "data": "synthetic", "config": workload_config(args, sigmas),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle_cores(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def combine_ranks(elapsed: float, units: float, device="cpu"):
    """Replicas: the job's time is the slowest rank's, its work the sum over ranks.
    Needs an initialised process group (nccl on the GPUs, gloo in the CPU tests)."""
    import torch
    import torch.distributed as dist

    t = torch.tensor([elapsed], dtype=torch.float64, device=device)
    u = torch.tensor([units], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t[0]), float(u[0])


# ---------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------
def run_ours(args, sigmas):
    import torch

    import paper_2001_08289_gb300 as L
    from paper_2001_08289_gb300 import build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0 or world == 1:
        build.build()
    if world > 1:
        dist.barrier()
    L.load_library()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.Stream(device=dev)
    n = args.n
    N = n * n
    mask_np = square_array_mask(n)
    mask_dev = torch.from_numpy(mask_np).to(dev)
    grid = L.Grid(mask_dev, stream=stream.cuda_stream)
    e = [1.0, 0.0]
    kw = dict(precision="fp32", green=args.green, tol=TOL, max_iter=500, alpha=ALPHA_BETA[0], beta=ALPHA_BETA[1])

    layout = {"packed": False}

    def step(g):
        out = []
        for s1 in sigmas:
            for sch in SCHEMES:
                r = g.solve(s1, e, scheme=sch, **kw)
                layout["packed"] = r.packed
                out.append((s1, sch, r.iterations, r.status, r.sigma_star, r.solve_ms, r.kernel_launches,
                            r.hist_sigma))
                r.free()
        return out

    # reference sigma_* per sigma_1 for the true-error counts (untimed): EM in H'' with
    # FP32 fields run far past the tolerance; FP64 fields are limited to x lines of
    # 4096 points, so the reference is the median of the last 20 iterates, and their
    # spread is its own uncertainty
    refs = {}
    for s1 in sigmas:
        r = grid.solve(s1, e, scheme="em_sub", **dict(kw, tol=0.0, max_iter=200))
        tail = r.hist_sigma[-20:]
        refs[s1] = (complex(np.median(tail.real), np.median(tail.imag)),
                    float(np.abs(tail - np.median(tail.real)).max() / abs(np.median(tail.real))))
        r.free()
    for _ in range(args.warmup):
        step(grid)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[0]) if \
        os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0].isdigit() else local
    clocks = ClockSampler(gpu_index)
    clocks.start()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    ev0.record(stream)
    results = []
    for _ in range(args.steps):
        results.append(step(grid))
    ev1.record(stream)
    torch.cuda.synchronize()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    clk = clocks.stop()
    vox = sum(it * N for stp in results for (_, _, it, *_) in stp)
    launches = sum(stp_i[6] for stp in results for stp_i in stp)
    if world > 1:
        elapsed, vox = combine_ranks(elapsed, vox, dev)
    value = vox / elapsed

    # per-solve summary of the last timed step: iterations and time to the stop rule,
    # and (from the sigma_k history) to a true relative error of 1e-6 against a long
    # reference run; a solve that hit its iteration cap gives a lower bound only
    last = results[-1]
    per = {}
    for (s1, sch, it, st, sig, ms, _, hist) in last:
        ref, ref_spread = refs[s1]
        err = np.abs(hist - ref) / abs(ref)
        below = np.nonzero(err > TOL)[0]
        hit = None if (below.size and below[-1] == len(err) - 1) else (int(below[-1]) + 1 if below.size else 0)
        per.setdefault(str(s1), {})[sch] = {
            "iters": it, "status": st, "capped": st == 3, "ms": round(ms, 3), "sigma_star": [sig.real, sig.imag],
            "iters_to_true_1e-6": hit,
            "ms_to_true_1e-6": None if hit is None else round(ms * (hit + 1) / (it + 1), 3)}
    speed = {}
    for k, v in per.items():
        for other in ("ms", "em"):
            key = f"{other}_over_em_sub"
            if other in v and "em_sub" in v:
                r = round(v[other]["ms"] / v["em_sub"]["ms"], 3)
                speed.setdefault(key, {})[k] = r if not v[other]["capped"] else f">= {r} ({other} capped at 500)"
    # pass timing with CUDA events on the grid's stream
    passes = {}
    peak, peak_kind = measured_peaks()
    for sch in ("ms", "em_sub"):
        grid.prepare(10.0, e, scheme=sch, precision="fp32", green=args.green, tol=0.0, max_iter=100000,
                     alpha=ALPHA_BETA[0], beta=ALPHA_BETA[1])
        for kind, name in ((0, "row"), (1, "col")):
            with torch.cuda.stream(stream):
                grid.launch_passes(kind, 3)
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record(stream)
                grid.launch_passes(kind, args.pass_reps)
                b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b) / args.pass_reps
            byt = algorithmic_bytes(name, sch, N, packed=layout["packed"])
            passes[f"{name}_pass|{sch}"] = {"ms": round(ms, 4), "alg_bytes": int(byt),
                                            "GBps": round(byt / ms / 1e6, 1),
                                            "frac_of_measured_hbm": round(byt / ms / 1e6 / peak, 4)}
    dom = max(("row_pass|ms", "col_pass|ms"), key=lambda k: passes[k]["ms"])
    kname = dom.split("|")[0]
    wl = f"{n}x{n}_ms_fp32_{'packed' if layout['packed'] else 'complex'}"
    roof = {"bound": "hbm", "kernel": kname, "achieved": passes[dom]["GBps"], "peak": peak, "unit": "GB/s",
            "frac": passes[dom]["frac_of_measured_hbm"], "traffic": ncu_traffic(kname, wl),
            "peak_source": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)" if peak_kind == "measured" else "fallback",
            "per_launch_alg_bytes": passes[dom]["alg_bytes"], "per_launch_ms": passes[dom]["ms"]}

    # the arithmetic ceiling beside the HBM one: the passes' FFT flops (5 n log2 n per
    # complex line transform, forward and inverse) against the FP32 FMA rate measured
    # on this GPU now (plain and paired fma.rn.f32x2 forms)
    fma_plain = L.lsfft_fma_peak(False, 3)
    fma_paired = L.lsfft_fma_peak(True, 3)
    fma_peak = max(fma_plain, fma_paired)
    lines = {"row_pass": n if layout["packed"] else 2 * n, "col_pass": (n + 2) if layout["packed"] else 2 * n}
    alu = {"fp32_fma_tflops_measured": round(fma_plain, 2), "fp32_fma_paired_tflops_measured": round(fma_paired, 2),
           "flops_convention": "5 n log2 n per complex line transform, two transforms per line per pass"}
    for kn in ("row_pass", "col_pass"):
        fl = 2 * lines[kn] * 5.0 * n * math.log2(n)
        tf = fl / (passes[f"{kn}|ms"]["ms"] * 1e-3) / 1e12
        alu[kn] = {"fft_flops_per_launch": int(fl), "achieved_tflops": round(tf, 2), "frac": round(tf / fma_peak, 4)}

    # comparison only: the same MS update written with torch.fft (cuFFT), per update
    cufft = cufft_ms_update(n, green=args.green)
    ours_ms = passes["row_pass|ms"]["ms"] + passes["col_pass|ms"]["ms"]
    cufft["ours_ms_per_update"] = round(ours_ms, 4)
    cufft["speedup_ours_vs_cufft"] = round(cufft["ms_per_update"] / ours_ms, 2)

    # end to end through the C ABI: pinned host mask in, pinned host fields out.
    # Each solve's field goes to one of three pinned host buffers on a copy stream
    # (lsfft_copy_field_async) while the next solves run; up to two copies are in
    # flight, so a copy slowed down by the passes beside it does not hold up a short
    # next solve.  A result is freed once its copy has completed, and every copy has
    # landed before the clock stops.
    e2e = None
    if not args.no_e2e:
        depth = 2
        mask_pin = torch.from_numpy(mask_np).pin_memory()
        host_E = [torch.empty((2, n, n), dtype=torch.complex64).pin_memory() for _ in range(depth + 1)]
        copy_stream = torch.cuda.Stream(device=dev)
        h2d = mask_pin.numel()
        d2h = 0
        e2e_vox = 0
        copies = 0
        pending = []   # (result, event recorded after its copy)
        # this box's device-to-host rate into pinned memory, for context (untimed)
        probe = torch.empty((2, n, n), dtype=torch.complex64, device=dev)
        with torch.cuda.stream(copy_stream):
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            host_E[0].copy_(probe, non_blocking=True)
            c0.record(copy_stream)
            host_E[0].copy_(probe, non_blocking=True)
            c1.record(copy_stream)
        copy_stream.synchronize()
        d2h_gbps = probe.numel() * 8 / (c0.elapsed_time(c1) * 1e6)
        del probe
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h = L.lsfft_create_grid(2, (n, n), mask_pin.numpy(), stream.cuda_stream)
            for s1 in sigmas:
                for sch in SCHEMES:
                    st, ptr = L.lsfft_solve(h, s1, e, L.make_opts(scheme=sch, **kw))
                    if len(pending) >= depth:
                        old_ptr, old_ev = pending.pop(0)
                        old_ev.synchronize()
                        L.lsfft_free_result(old_ptr)
                    L.lsfft_copy_field_async(ptr, host_E[copies % (depth + 1)].data_ptr(), False,
                                             copy_stream.cuda_stream)
                    ev = torch.cuda.Event()
                    ev.record(copy_stream)
                    pending.append((ptr, ev))
                    copies += 1
                    r = ptr.contents
                    e2e_vox += r.iters * N
                    if _ == 0:
                        d2h += host_E[0].numel() * 8 + 4 * 8 * r.hist_len + 16
            L.lsfft_destroy_grid(h)
        copy_stream.synchronize()
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        for old_ptr, _ in pending:
            L.lsfft_free_result(old_ptr)
        e2e = {"value": e2e_vox / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "d2h_gbps_pinned": round(d2h_gbps, 1),
               "note": "lsfft_create_grid from pinned host mask, lsfft_solve per (sigma1, scheme), "
                       "lsfft_copy_field_async of every E to pinned host memory on a copy stream (up to two copies "
                       "in flight, overlapping the next solves), host wall clock until the last copy has landed"}
    grid.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if layout["packed"] else "c64",
            "data": "synthetic", "layout": "packed real (E_x + i E_y in one complex plane)" if layout["packed"]
            else "complex component planes",
            "config": workload_config(args, sigmas), "roofline": roof, "alu_ceiling": alu,
            "gpu_launches": int(launches),
            "clocks": clk, "e2e": e2e,
            "time_to_tol": {"per_sigma1": per, "time_ratio": speed,
                            "true_error_reference": {str(k): {"sigma_star": [v[0].real, v[0].imag], "spread": v[1]}
                                                     for k, v in refs.items()},
                            "note": "iters_to_true_1e-6: first iterate from which |sigma_k - ref|/|ref| stays "
                                    "<= 1e-6, ref = median of the last 20 of 200 EM-in-H'' iterates (FP32 fields, "
                                    "FP64 reductions); 'capped' solves stopped at max_iter = 500"},
            "passes": passes, "cufft_comparison": cufft}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_block(args.n)
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------------------------
# further workloads (one JSON line each; not the driver's default)
# ---------------------------------------------------------------------------
def _gpu_setup():
    import torch

    import paper_2001_08289_gb300 as L
    from paper_2001_08289_gb300 import build

    torch.cuda.set_device(0)
    build.build()
    L.load_library()
    return torch, L


def _line(metric, value, unit, args, config, **extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic",
            "workload_kind": args.workload, "config": config}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_lattice64(args):
    """The 64^2 lattice: the 64^2 square array, sigma_1 = 10, FP64, stop at relative change
    1e-10; MS, EM and both substituted schemes with [alpha, beta] from the oracle's
    dense pole computation on the same grid (weight cutoffs 1e-10 and 1e-3, both
    Green symbols; stored in tests/golden/dense_pole_hulls_64.json by a script that
    calls only the oracle), with the GPU Lanczos hull reported beside them.
    Microseconds per iteration and iterations per scheme (latency-bound: not a
    roofline case)."""
    torch, L = _gpu_setup()
    mask = square_array_mask(64)
    e = [1.0, 0.0]
    fixture = json.load(open(os.path.join(ROOT, "tests", "golden", "dense_pole_hulls_64.json")))["hulls"]
    out, lanczos = {}, {}

    def timed(g, **kw):
        for _ in range(args.warmup):
            g.solve(10.0, e, **kw).free()
        ms, its, sig = [], [], None
        for _ in range(args.steps):
            r = g.solve(10.0, e, **kw)
            ms.append(r.solve_ms)
            its.append(r.iterations)
            sig = r.sigma_star
            r.free()
        return {"iters": its[-1], "solve_ms": round(float(np.median(ms)), 4),
                "us_per_iter": round(1e3 * float(np.median(ms)) / its[-1], 2), "sigma_star": sig.real}

    with L.Grid(mask) as g:
        for green, cut in (("trig", 1e-3), ("fd", 1e-10)):
            a, b, _, _ = g.lanczos_hull(e, green=green, precision="fp64", steps=200, cutoff=cut)
            lanczos[green] = {"cutoff": cut, "alpha": a, "beta": b}
        for green in ("trig", "fd"):
            base = dict(precision="fp64", green=green, tol=1e-10, max_iter=4000)
            for sch in ("ms", "em"):
                out[f"{green}|{sch}"] = timed(g, scheme=sch, **base)
            for cutoff in ("1e-10", "0.001"):
                h = fixture[f"{green}|{cutoff}"]
                for sch in ("ms_sub", "em_sub"):
                    out[f"{green}|{sch}|dense poles {cutoff}"] = timed(g, scheme=sch, alpha=h["alpha"],
                                                                       beta=h["beta"], **base)
            for sch in ("ms_sub", "em_sub"):
                out[f"{green}|{sch}|lanczos"] = timed(g, scheme=sch, alpha=lanczos[green]["alpha"],
                                                      beta=lanczos[green]["beta"], **base)
    tot_vox = sum(v["iters"] for v in out.values()) * mask.size
    tot_s = sum(v["solve_ms"] for v in out.values()) / 1e3
    us = sorted(v["us_per_iter"] for v in out.values())
    _line("voxel-iters/s (64^2 FP64 lattice)", tot_vox / tot_s, UNIT, args,
          {"workload": "64x64 square array, sigma1=10, FP64, stop 1e-10; alpha, beta of the substituted schemes "
                       "from the oracle's dense poles (cutoffs 1e-10 and 1e-3) and from GPU Lanczos",
           "dense_pole_hulls": fixture, "lanczos_hulls": lanczos},
          dtype="c128", per_scheme=out, us_per_iter_median=us[len(us) // 2])


def run_cube3d(args):
    """3-D cubic array of cubes of side n/2 (f = 1/8), sigma_1 in {5, 50, 500}, FP32,
    MS vs EM in H'' with alpha, beta from GPU Lanczos: voxel-iters/s and pass roofline."""
    from synth import SIGMA1_SWEEP_3D

    torch, L = _gpu_setup()
    n = args.n if args.n <= 512 else 256
    mask = square_array_mask(n, d=3)
    N = mask.size
    e = [1.0, 0.0, 0.0]
    stream = torch.cuda.Stream()
    per = {}
    # The forward-difference symbol: its weighted poles fill a clean interval, as the
    # substitution assumes; the trigonometric symbol has tiny-weight poles far outside
    # any truncated hull, on which EM in H'' diverges for large sigma_1 (the oracle
    # shows the same).
    green = "fd"
    with L.Grid(mask, stream=stream.cuda_stream) as g:
        a, b, _, _ = g.lanczos_hull(e, green=green, precision="fp32", steps=60, cutoff=1e-8)
        a, b = a * (1 - HULL_MARGIN), b * (1 + HULL_MARGIN)
        kws = {sch: dict(scheme=sch, precision="fp32", green=green, tol=TOL, max_iter=400, alpha=a, beta=b)
               for sch in SCHEMES}
        for _ in range(args.warmup):
            for s1 in SIGMA1_SWEEP_3D:
                for sch in SCHEMES:
                    g.solve(s1, e, **kws[sch]).free()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev0.record(stream)
        vox = 0
        for _ in range(args.steps):
            for s1 in SIGMA1_SWEEP_3D:
                for sch in SCHEMES:
                    r = g.solve(s1, e, **kws[sch])
                    vox += r.iterations * N
                    per.setdefault(str(s1), {})[sch] = {"iters": r.iterations, "status": r.status,
                                                        "ms": round(r.solve_ms, 3), "sigma_star": r.sigma_star.real}
                    r.free()
        ev1.record(stream)
        torch.cuda.synchronize()
        elapsed = ev0.elapsed_time(ev1) / 1e3
        peak, _ = measured_peaks()
        passes = {}
        for sch in SCHEMES:
            g.prepare(50.0, e, **dict(kws[sch], tol=0.0, max_iter=100000))
            for kind, name, nbytes in ((0, "row", N * (2 * 24 + 1 + (4 * 24 * 0.125 if sch == "em_sub" else 0))),
                                       (1, "strided_x3", 3 * N * 2 * 24)):
                with torch.cuda.stream(stream):
                    g.launch_passes(kind, 2)
                    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    t0.record(stream)
                    g.launch_passes(kind, args.pass_reps)
                    t1.record(stream)
                torch.cuda.synchronize()
                ms = t0.elapsed_time(t1) / args.pass_reps
                passes[f"{name}|{sch}"] = {"ms": round(ms, 4), "alg_bytes": int(nbytes),
                                           "GBps": round(nbytes / ms / 1e6, 1),
                                           "frac_of_measured_hbm": round(nbytes / ms / 1e6 / peak, 4)}
    _line(METRIC, vox / elapsed, UNIT, args,
          {"workload": f"3D cubic array of cubes (f=1/8), {n}^3, sigma1 in {list(SIGMA1_SWEEP_3D)}, MS vs "
                       f"EM-in-H'' with Lanczos (alpha,beta)=({a:.4g},{b:.4g}) widened by {HULL_MARGIN:g}, "
                       f"tol {TOL:g}, fd Green symbol",
           "n": n, "d": 3}, dtype="c64", ms_per_step=1e3 * elapsed / args.steps, time_to_tol=per, passes=passes)


def run_sweep(args):
    """Batched complex-sigma_1 sweep: 32 RSA-disk microstructures (n in 128..1024, 8
    each), sigma_1 = r e^{i theta}, EM in H'' with per-microstructure Lanczos
    alpha, beta; all solves of a step run in one persistent launch
    (lsfft_solve_sweep).  The same jobs through the host-scheduled batch
    (lsfft_solve_batch, one stream per grid) are timed once for comparison."""
    from synth import complex_sigma_ray, rsa_disk_mask

    torch, L = _gpu_setup()
    sizes = [128] * 8 + [256] * 8 + [512] * 8 + [1024] * 8
    grids, hulls, vox_n = [], [], []
    for s, n in enumerate(sizes):
        m, info = rsa_disk_mask(n, seed=s)
        g = L.Grid(m)
        a, b, _, _ = g.lanczos_hull([1.0, 0.0], green="fd", precision="fp32", steps=60, cutoff=1e-6)
        grids.append(g)
        hulls.append((a * (1 - HULL_MARGIN), b * (1 + HULL_MARGIN)))
        vox_n.append(m.size)
    allsig = complex_sigma_ray(count=512, seed=1000)

    host_scheduled = False

    def step(k):
        sig = allsig[(k * args.sweep_sigmas) % 512:][:args.sweep_sigmas]
        jobs = []
        for g, (a, b) in zip(grids, hulls):
            for s1 in sig:
                # EM in H'' where it is stable against rounding (rate < limit), else plain EM
                rate, limit = L.lsfft_substitution_rates(s1, a, b)
                sch = "em_sub" if rate < 0.98 * limit else "em"
                jobs.append((g, s1, [1.0, 0.0], dict(scheme=sch, green="fd", tol=TOL, max_iter=400, alpha=a, beta=b)))
        out = (L.solve_batch if host_scheduled else L.solve_sweep)(jobs)
        vox = sum(r.iterations * jobs[i][0].N for i, r in enumerate(out) if not isinstance(r, Exception))
        st = [(jobs[i][3]["scheme"], getattr(r, "status", -1)) for i, r in enumerate(out)]
        for r in out:
            if not isinstance(r, Exception):
                r.free()
        return vox, len(jobs), st

    host_scheduled = True   # comparison: one timed step of the host-scheduled batch
    step(0)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    hv, hn, _ = step(1)
    torch.cuda.synchronize()
    host_rate = hv / (time.perf_counter() - t0)
    host_scheduled = False

    for k in range(args.warmup):
        step(k)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    vox = solves = 0
    statuses = []
    for k in range(args.steps):
        v, nj, st = step(args.warmup + k)
        vox += v
        solves += nj
        statuses += st
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    for g in grids:
        g.close()
    _line("voxel-iters/s (batched complex-sigma1 sweep)", vox / dt, UNIT, args,
          {"workload": f"32 RSA-disk microstructures (n=128..1024, 8 each), {args.sweep_sigmas} complex sigma1 "
                       f"per microstructure per step from the r e^(i theta) ray (seed 1000), EM-in-H'' with "
                       f"per-microstructure Lanczos alpha,beta (fd, cutoff 1e-6) widened by {HULL_MARGIN:g} "
                       f"(plain EM where EM-in-H'' is not rounding-stable), tol {TOL:g}, FP32, at most 400 "
                       f"iterations",
           "solves_per_step": solves // max(args.steps, 1)},
          dtype="c64", solves_per_s=solves / dt, ms_per_step=1e3 * dt / args.steps, gpu_launches_per_step=1,
          status_counts={f"{sch}:{st}": statuses.count((sch, st)) for sch, st in sorted(set(statuses))},
          host_scheduled_batch_voxel_iters_per_s=host_rate,
          executor="one persistent launch per step (lsfft_solve_sweep): device work queue over (solve, pass, item)")


def run_adjoint(args):
    """128^3 Bernoulli(0.2) voxels after one periodic 3x3x3 majority filter,
    sigma = 1 + 19 chi: forward solve plus gradient, and central differences
    (step 1e-3) of the variational energy estimate at random voxels, FP64."""
    from synth import bernoulli_majority_mask

    torch, L = _gpu_setup()
    n = 128
    mask = bernoulli_majority_mask(n, p=0.2, seed=5)
    sig = 1.0 + 19.0 * mask.astype(np.float64)
    e = [1.0, 0.0, 0.0]
    opts = dict(scheme="em", precision="fp64", green="fd", tol=1e-15, max_iter=3000)
    rng = np.random.default_rng(6)
    with L.Grid(mask) as g:
        g.set_sigma_field(sig, sigma0=np.sqrt(20.0))
        grad = torch.empty(mask.shape, dtype=torch.complex128, device="cuda")
        times = []
        for k in range(args.warmup + args.steps):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r = g.solve(1.0, e, **opts)
            d1, en = g.gradient(r, e, grad.data_ptr())
            torch.cuda.synchronize()
            if k >= args.warmup:
                times.append(time.perf_counter() - t0)
            its = r.iterations
            r.free()
        gf = grad.cpu().numpy().real
        # voxels: half inside the (sparse) inclusions, half anywhere
        inc = np.argwhere(mask)
        picks = [tuple(v) for v in inc[rng.permutation(len(inc))[:args.fd_voxels // 2]]]
        picks += [tuple(rng.integers(0, n, 3)) for _ in range(args.fd_voxels - len(picks))]
        errs = []
        h = 1e-3
        for v in picks:
            vals = []
            for sgn in (1, -1):
                sp = sig.copy()
                sp[v] += sgn * h
                g.set_sigma_field(sp, sigma0=np.sqrt(20.0))
                rr = g.solve(1.0, e, **opts)
                vals.append(g.gradient(rr, e)[1].real)
                rr.free()
            fd = (vals[0] - vals[1]) / (2 * h)
            errs.append(abs(fd - gf[v]) / abs(gf[v]))
    _line("forward+gradient wall time (128^3 adjoint configuration)", float(np.median(times)), "s", args,
          {"workload": "128^3 Bernoulli(0.2) voxels (seed 5) after one periodic 3x3x3 majority filter (>=14/27), "
                       "sigma = 1 + 19 chi, EM FP64 tol 1e-15, fd Green symbol",
           "inclusion_fraction": float(mask.mean())}, dtype="c128", higher_is_better=False, iterations=its,
          dsigma_dsigma1=d1.real, energy_sigma_star=en.real, fd_voxels=len(picks), fd_max_rel_err=max(errs),
          fd_median_rel_err=float(np.median(errs)))


def cufft_ms_update(n, green="trig", iters=30, s1=10.0):
    """Comparison only: the Moulinec-Suquet update on the n x n square array written
    with torch.fft (cuFFT real-to-complex transforms) and torch elementwise kernels,
    FP32, sigma_1 = 10: tau = (sigma/sigma_0 - 1) E, E^ = -Gamma tau^ (zero mode N e,
    Nyquist lines zero for the trig symbol), E = inverse FFT, and <sigma E> per
    update.  Fixed iteration count, CUDA events.  Returns a dict."""
    import torch

    dev = torch.device("cuda", torch.cuda.current_device())
    mask = torch.from_numpy(square_array_mask(n)).to(dev)
    s0 = (s1 + 1.0) / 2
    a = torch.where(mask != 0, torch.tensor(s1 / s0 - 1, device=dev), torch.tensor(1 / s0 - 1, device=dev))
    sig = torch.where(mask != 0, torch.tensor(s1, device=dev), torch.tensor(1.0, device=dev))
    ky = torch.fft.fftfreq(n, d=1.0 / n, device=dev).round().view(n, 1)
    kx = torch.arange(n // 2 + 1, device=dev, dtype=torch.float32).view(1, n // 2 + 1)
    if green == "trig":
        ux, uy = kx.to(torch.complex64), ky.to(torch.complex64)
        nyq = (ky == -(n // 2)) | (kx == n // 2)
    else:
        ux = torch.exp(2j * math.pi * kx / n) - 1
        uy = torch.exp(2j * math.pi * ky / n) - 1
        nyq = torch.zeros_like(kx * ky, dtype=torch.bool)
    k2 = (ux.abs() ** 2 + uy.abs() ** 2)
    inv = torch.where((k2 > 0) & ~nyq, 1.0 / k2.clamp(min=1e-30), torch.zeros_like(k2))
    E = torch.zeros((2, n, n), device=dev, dtype=torch.float32)
    E[0] = 1.0

    def update(E):
        T = torch.fft.rfft2(a * E)
        proj = (ux.conj() * T[0] + uy.conj() * T[1]) * inv
        Eh = torch.stack((-ux * proj, -uy * proj))
        Eh[0, 0, 0] = n * n * 1.0
        Eh[1, 0, 0] = 0.0
        E = torch.fft.irfft2(Eh, s=(n, n))
        return E, (sig * E[0]).mean()

    for _ in range(3):
        E, sk = update(E)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record()
    for _ in range(iters):
        E, sk = update(E)
    t1.record()
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1) / iters
    return {"ms_per_update": round(ms, 4), "voxel_iters_per_s": n * n / (ms / 1e3), "sigma_k": float(sk),
            "what": f"MS update, sigma1={s1}, {n}x{n}, torch.fft.rfft2/irfft2 (cuFFT) + torch elementwise kernels, "
                    f"FP32, {green} symbol; comparison only, not the library's path"}


def run_cufft(args):
    """Comparison only: the same Moulinec-Suquet update with torch.fft (cuFFT)."""
    torch, L = _gpu_setup()
    c = cufft_ms_update(args.n, green=args.green)
    _line("voxel-iters/s (torch.fft / cuFFT comparison, MS update)", c["voxel_iters_per_s"], UNIT, args,
          {"workload": c["what"], "n": args.n}, dtype="f32", ms_per_update=c["ms_per_update"], sigma_k=c["sigma_k"])


def run_precision(args):
    """FP32 fields with FP64 reductions against an all-FP64 GPU run on the 2048^2
    square array (sigma_1 in the 2-D sweep, MS and EM in H'' on [1/4, 4], trig):
    sigma_* and E differences, and the iterations and wall time until sigma_k is
    within 1e-6 of the FP64 run's converged value (time to a true tolerance)."""
    torch, L = _gpu_setup()
    n = args.n if args.n <= 4096 else 2048
    mask = square_array_mask(n)
    e = [1.0, 0.0]
    out = {}
    with L.Grid(mask) as g:
        for s1 in (0.01, 0.1, 10.0, 100.0, 1e4):
            ref = g.solve(s1, e, scheme="em_sub", precision="fp64", tol=1e-12, max_iter=2000, alpha=0.25, beta=4.0)
            s_ref = ref.sigma_star
            E_ref = ref.field_numpy()
            ref.free()
            for sch in SCHEMES:
                row = {}
                for prec in ("fp32", "fp64"):
                    r = g.solve(s1, e, scheme=sch, precision=prec, tol=TOL, max_iter=500, alpha=0.25, beta=4.0)
                    err = np.abs(r.hist_sigma - s_ref) / abs(s_ref)
                    hit = int(np.argmax(err <= 1e-6)) if np.any(err <= 1e-6) else None
                    Ef = r.field_numpy().astype(np.complex128)
                    row[prec] = {"iters": r.iterations, "status": r.status, "ms": round(r.solve_ms, 3),
                                 "rel_err_sigma_vs_fp64_converged": float(abs(r.sigma_star - s_ref) / abs(s_ref)),
                                 "rel_l2_E_vs_fp64_converged": float(np.linalg.norm(Ef - E_ref) / np.linalg.norm(E_ref)),
                                 "iters_to_true_1e-6": hit,
                                 "ms_to_true_1e-6": None if hit is None else round(r.solve_ms * (hit + 1) / (r.iterations + 1), 3)}
                    r.free()
                out[f"{s1:g}|{sch}"] = row
    _line("sigma_* and E agreement of FP32 fields with an all-FP64 run; time to a true 1e-6", n * n, "voxels", args,
          {"workload": f"{n}x{n} square array, sigma1 in [0.01, 0.1, 10, 100, 1e4], MS and EM in H'' on [1/4, 4], "
                       "trig symbol, stop at relative change 1e-6; reference: EM in H'' in FP64 to 1e-12", "n": n},
          dtype="f32 and f64", results=out)


def run_passes(args):
    """Pass timing alone (the unit the profiles capture): after one lsfft_prepare per
    scheme, `--pass-reps` launches of the row pass, then of the strided pass(es), on
    the square array at sigma_1 = 10, FP32, trig symbol; CUDA events on the grid's
    stream.  `--dim 3` uses the n^3 cubic array (n <= 512)."""
    torch, L = _gpu_setup()
    d = args.dim
    n = args.n if d == 2 else min(args.n, 512)
    mask = square_array_mask(n, d=d)
    N = mask.size
    e = [1.0] + [0.0] * (d - 1)
    stream = torch.cuda.Stream()
    peak, _ = measured_peaks()
    frac = 0.25 if d == 2 else 0.125
    out = {}
    with L.Grid(mask, stream=stream.cuda_stream) as g:
        for sch in SCHEMES:
            g.prepare(10.0, e, scheme=sch, precision="fp32", green=args.green, tol=0.0, max_iter=100000,
                      alpha=ALPHA_BETA[0], beta=ALPHA_BETA[1])
            packed = d == 2
            for kind, name in ((0, "row"), (1, "col")):
                with torch.cuda.stream(stream):
                    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    a.record(stream)
                    g.launch_passes(kind, args.pass_reps)
                    b.record(stream)
                torch.cuda.synchronize()
                ms = a.elapsed_time(b) / args.pass_reps
                byt = algorithmic_bytes(name, sch, N, d=d, fraction=frac, packed=packed)
                if name == "col" and d == 3:
                    byt *= 3
                out[f"{name}|{sch}"] = {"ms": round(ms, 4), "alg_bytes": int(byt), "GBps": round(byt / ms / 1e6, 1),
                                        "frac_of_measured_hbm": round(byt / ms / 1e6 / peak, 4)}
    _line("pass time (row pass / strided pass)", out["col|ms"]["ms"], "ms", args,
          {"workload": f"square array {'x'.join([str(n)] * d)}, sigma1 = 10, FP32, {args.green} symbol, "
                       f"{args.pass_reps} launches per pass kind after lsfft_prepare", "n": n, "d": d},
          dtype="f32" if d == 2 else "c64", higher_is_better=False, passes=out)


def write_convergence_svg(path, title, curves, floor=1e-12, width=640, height=420):
    """A log-scale line plot of error against iteration, as plain SVG text.
    curves: {label: (list of errors, colour, dash)}."""
    ml, mr, mt, mb = 70, 170, 40, 50
    pw, ph = width - ml - mr, height - mt - mb
    kmax = max(len(c[0]) for c in curves.values()) - 1
    lo, hi = math.floor(math.log10(floor)), 0
    X = lambda k: ml + pw * k / max(kmax, 1)
    Y = lambda v: mt + ph * (hi - math.log10(max(v, floor))) / (hi - lo)
    out = [f'<svg xmlns="http://www.w3.org/2000/svg" width="{width}" height="{height}" '
           f'font-family="sans-serif" font-size="12">',
           f'<rect width="{width}" height="{height}" fill="white"/>',
           f'<text x="{ml}" y="22" font-size="14">{title}</text>',
           f'<rect x="{ml}" y="{mt}" width="{pw}" height="{ph}" fill="none" stroke="black"/>']
    for dec in range(lo, hi + 1, 2):
        y = Y(10.0 ** dec)
        out.append(f'<line x1="{ml}" y1="{y:.1f}" x2="{ml + pw}" y2="{y:.1f}" stroke="#ddd"/>')
        out.append(f'<text x="{ml - 8}" y="{y + 4:.1f}" text-anchor="end">1e{dec}</text>')
    step = max(1, int(round(kmax / 8 / 5.0)) * 5)
    for k in range(0, kmax + 1, step):
        out.append(f'<text x="{X(k):.1f}" y="{mt + ph + 18}" text-anchor="middle">{k}</text>')
    out.append(f'<text x="{ml + pw / 2}" y="{height - 10}" text-anchor="middle">iteration k</text>')
    out.append(f'<text x="16" y="{mt + ph / 2}" transform="rotate(-90 16 {mt + ph / 2})" text-anchor="middle">'
               f'|sigma_k - sigma_*| / sigma_*</text>')
    for i, (label, (ys, colour, dash)) in enumerate(curves.items()):
        pts = " ".join(f"{X(k):.1f},{Y(v):.1f}" for k, v in enumerate(ys))
        da = f' stroke-dasharray="{dash}"' if dash else ""
        out.append(f'<polyline points="{pts}" fill="none" stroke="{colour}" stroke-width="1.6"{da}/>')
        ly = mt + 16 + 18 * i
        out.append(f'<line x1="{ml + pw + 12}" y1="{ly}" x2="{ml + pw + 36}" y2="{ly}" stroke="{colour}" '
                   f'stroke-width="1.6"{da}/>')
        out.append(f'<text x="{ml + pw + 42}" y="{ly + 4}">{label}</text>')
    out.append("</svg>")
    with open(path, "w") as f:
        f.write("\n".join(out) + "\n")


def run_fig5(args):
    """The Moulinec-Suquet experiment of the section on their numerical example:
    square array of squares at 25 %, sigma_1 = 0 (insulating squares), sigma_2 = 1,
    pole interval estimate [1/4, 4]; convergence of sigma_k for MS against MS in
    H'' (their first figure) and for EM against EM in H'' (their second).  The
    curves are the relative distance of sigma_k to the converged discrete value and
    to Obnosov's continuum value sqrt(1/3) (Eq. J47a), per iteration, FP64.

    EM with the reference sqrt(sigma_1 sigma_2) is undefined at sigma_1 = 0; its
    curve uses the per-voxel mode with the reference 1/2 (the MS reference)."""
    torch, L = _gpu_setup()
    n = args.n if args.n <= 4096 else 2048
    mask = square_array_mask(n)
    e = [1.0, 0.0]
    obn = math.sqrt(1.0 / 3.0)
    out = {}
    t0 = time.perf_counter()
    vox = 0
    with L.Grid(mask) as g:
        for green in ("fd", "trig"):
            ref = g.solve(0.0, e, scheme="em_sub", precision="fp64", green=green, tol=1e-13, max_iter=4000,
                          alpha=0.25, beta=4.0)
            s_ref = ref.sigma_star.real
            ref.free()
            for sch in ("ms", "ms_sub", "em", "em_sub"):
                kw = dict(scheme=sch, precision="fp64", green=green, tol=1e-11, max_iter=args.fig_iters,
                          alpha=0.25, beta=4.0)
                if sch == "em":
                    g.set_sigma_field(1.0 - mask.astype(np.float64), sigma0=0.5)
                    r = g.solve(1.0, e, **kw)
                    g.set_sigma_field(None)
                else:
                    r = g.solve(0.0, e, **kw)
                vox += r.iterations * mask.size
                h = r.hist_sigma.real
                err = np.abs(h - s_ref) / s_ref
                first = {f"1e-{p}": (int(np.argmax(err < 10.0 ** -p)) if np.any(err < 10.0 ** -p) else None)
                         for p in range(2, 11, 2)}
                out[f"{green}|{sch}"] = {
                    "iters": r.iterations, "status": r.status, "sigma_star": r.sigma_star.real,
                    "rel_err_vs_obnosov": abs(r.sigma_star.real - obn) / obn, "discrete_limit": s_ref,
                    "first_iter_below": first,
                    "curve_rel_err_vs_limit": [float(f"{x:.3g}") for x in err[:200]]}
                r.free()
    dt = time.perf_counter() - t0
    if args.plot_dir:
        os.makedirs(args.plot_dir, exist_ok=True)
        style = {"fd": ("", ""), "trig": ("4,3", " (trig)")}
        for fig, pair in (("fig5b_ms_vs_ms_sub", ("ms", "ms_sub")), ("fig5c_em_vs_em_sub", ("em", "em_sub"))):
            curves = {}
            for green in ("fd", "trig"):
                dash, suffix = style[green]
                for sch, colour in zip(pair, ("#1f4e9c", "#c0392b")):
                    name = {"ms": "MS", "ms_sub": "MS in H''", "em": "EM (ref. 1/2)", "em_sub": "EM in H''"}[sch]
                    curves[name + suffix] = (out[f"{green}|{sch}"]["curve_rel_err_vs_limit"][:80], colour, dash)
            write_convergence_svg(os.path.join(args.plot_dir, f"{fig}_square{n}_sigma1_0.svg"),
                                  f"sigma_1 = 0, [alpha, beta] = [1/4, 4], {n}x{n} square array, FP64", curves)
        with open(os.path.join(args.plot_dir, f"fig5_square{n}_sigma1_0_curves.json"), "w") as f:
            json.dump({k: {kk: vv for kk, vv in v.items()} for k, v in out.items()}, f, indent=0)
    _line("iterations to a relative sigma_* error (sigma_1 = 0 experiment)", vox / dt, UNIT, args,
          {"workload": f"{n}x{n} square array of squares (f = 1/4), sigma_1 = 0, sigma_2 = 1, e = (1, 0), "
                       "[alpha, beta] = [1/4, 4], FP64, fd and trig Green symbols; EM with reference 1/2 "
                       "through the per-voxel mode", "n": n, "obnosov_sigma_star": obn},
          dtype="c128", curves=out)


def main():
    args = parse()
    sigmas = tuple(float(s) for s in args.sigmas.split(","))
    if args.impl == "reference":
        run_reference(args, sigmas)
    elif args.workload == "square2d":
        run_ours(args, sigmas)
    else:
        {"lattice64": run_lattice64, "cube3d": run_cube3d, "sweep": run_sweep, "adjoint": run_adjoint,
         "fig5": run_fig5, "passes": run_passes, "cufft": run_cufft, "precision": run_precision}[
            args.workload](args)


if __name__ == "__main__":
    main()
