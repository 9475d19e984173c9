"""Benchmark of the FFT Lippmann-Schwinger iteration on GB300.

Workload (one "step"): the paper's square array of squares at 25 % volume
fraction on an 8192 x 8192 grid, inclusion conductivities sigma_1 in
{0.01, 0.1, 10, 100, 1e4}, each solved to a relative sigma_* change of 1e-6
(three consecutive iterates) with the basic Moulinec-Suquet scheme and with the
accelerated scheme (Eyre-Milton in the substituted space H'') using the
paper's pole-interval estimate [alpha, beta] = [1/4, 4]; complex FP32 fields,
FP64 reductions, trigonometric Green symbol.  Inputs are synthetic and already
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
SCHEMES = ("ms", "em_sub")
ALPHA_BETA = (0.25, 4.0)          # the Moulinec-Suquet estimate quoted in the paper
TOL = 1e-6
FRACTION = 0.25


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
    return p.parse_args()


def workload_config(args, sigmas):
    return {
        "workload": f"2D square array of squares (f=0.25), {args.n}x{args.n}, sigma1 in {list(sigmas)}, "
                    f"MS vs EM-in-H'' (alpha,beta)=(1/4,4), rel. sigma* change {TOL:g} x3, {args.green} Green symbol",
        "n": args.n, "d": 2, "sigma1": list(sigmas), "schemes": list(SCHEMES), "alpha_beta": list(ALPHA_BETA),
        "tol": TOL, "green": args.green, "fields": "complex FP32, FP64 reductions",
        "l2": "inputs larger than L2 (state 1 GiB per field at 8192^2)",
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
# CPU baseline: the FP64 oracle as it stands (single-threaded numpy FFTs)
# ---------------------------------------------------------------------------
def oracle_sample(n, sigmas, schemes=SCHEMES, updates=1):
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


def cpu_baseline_block(n=4096):
    vox, dt = oracle_sample(n, (10.0,))
    return {"value": vox / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one update (+ sigma_k evaluation) of MS and of EM-in-H'' at sigma1=10 on a {n}x{n} "
                      f"square array, FP64 numpy (single-threaded FFT), {dt:.1f} s"}


def run_reference(args, sigmas):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n = 2048
    for _ in range(args.warmup):
        oracle_sample(n, (sigmas[len(sigmas) // 2],))
    vox, dt = 0, 0.0
    for _ in range(args.steps):
        v, t = oracle_sample(n, (sigmas[len(sigmas) // 2],))
        vox += v
        dt += t
    value = vox / dt
    sample = (f"per step: one update of MS and of EM-in-H'' at sigma1={sigmas[len(sigmas) // 2]} on a {n}x{n} "
              f"square array (FP64 numpy oracle, single-threaded)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64 (complex)",
            "data": "synthetic", "config": workload_config(args, sigmas),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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
                out.append((s1, sch, r.iterations, r.status, r.sigma_star, r.solve_ms, r.kernel_launches))
                r.free()
        return out

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
    vox = sum(it * N for stp in results for (_, _, it, _, _, _, _) in stp)
    launches = sum(kl for stp in results for (*_, kl) in stp)
    if world > 1:
        t = torch.tensor([elapsed, vox], dtype=torch.float64, device=dev)
        tmax = t.clone()
        dist.all_reduce(tmax[0:1], op=dist.ReduceOp.MAX)
        dist.all_reduce(t[1:2], op=dist.ReduceOp.SUM)
        elapsed, vox = float(tmax[0]), float(t[1])
    value = vox / elapsed

    # per-solve summary of the last timed step: iterations and time to the stop rule
    last = results[-1]
    per = {}
    for (s1, sch, it, st, sig, ms, _) in last:
        per.setdefault(str(s1), {})[sch] = {"iters": it, "status": st, "ms": round(ms, 3),
                                            "sigma_star": [sig.real, sig.imag]}
    speed = {k: round(v["ms"]["ms"] / v["em_sub"]["ms"], 3) if "ms" in v and "em_sub" in v else None
             for k, v in per.items()}
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

    # end to end through the C ABI: pinned host mask in, pinned host fields out
    e2e = None
    if not args.no_e2e:
        mask_pin = torch.from_numpy(mask_np).pin_memory()
        host_E = torch.empty((2, n, n), dtype=torch.complex64).pin_memory()
        h2d = mask_pin.numel()
        d2h = 0
        e2e_vox = 0
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            h = L.lsfft_create_grid(2, (n, n), mask_pin.numpy(), stream.cuda_stream)
            for s1 in sigmas:
                for sch in SCHEMES:
                    st, ptr = L.lsfft_solve(h, s1, e, L.make_opts(scheme=sch, **kw))
                    L.lsfft_copy_field(ptr, host_E.data_ptr(), False)
                    r = ptr.contents
                    e2e_vox += r.iters * N
                    if _ == 0:
                        d2h += host_E.numel() * 8 + 4 * 8 * r.hist_len + 16
                    L.lsfft_free_result(ptr)
            L.lsfft_destroy_grid(h)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        e2e = {"value": e2e_vox / dt, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "note": "lsfft_create_grid from pinned host mask, lsfft_solve per (sigma1, scheme), "
                       "lsfft_copy_field of every E to pinned host memory, host wall clock"}
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
            "config": workload_config(args, sigmas), "roofline": roof, "gpu_launches": int(launches),
            "clocks": clk, "e2e": e2e, "time_to_tol": {"per_sigma1": per, "ms_over_em_sub_time_ratio": speed},
            "passes": passes}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_block()
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    sigmas = tuple(float(s) for s in args.sigmas.split(","))
    if args.impl == "reference":
        run_reference(args, sigmas)
    else:
        run_ours(args, sigmas)


if __name__ == "__main__":
    main()
