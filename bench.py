"""Benchmark: GLUP/s of the 3D 7-point Jacobi and lexicographic Gauss-Seidel
smoothers on the 400^3 FP64 grid (100 sweeps each), through the C ABI.

One step = 100 Jacobi sweeps + 100 Gauss-Seidel sweeps on two resident
400^3 FP64 grids (halo U[0,1) seed 1, interior U[0,1) seed 2) + the FP64
residual norm of each result.  value = lattice-site updates of the step / its
device time (GLUP/s), timed with CUDA events on the launching stream over
exactly --steps steps after --warmup untimed steps.  Each grid (512.6 MB) is
about four times the 129 MB L2, so no flush is needed between steps.

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

N = 400
SWEEPS = 100
# the launch configuration timed for the headline (tests/test_gpu_parity.py checks it at full size)
HEADLINE = {
    "jacobi": {"nt": 1, "tile": (32, 8, 0)},
    "gs": {"nt": 1, "tile": (16, 16, 16)},
}
NT_SWEEP = [1, 2, 4, 8, 16]
METRIC = "GLUP/s at 400^3 FP64 (Jacobi, GS) vs HBM roofline; batched/served vs plain, p99"
FP64_OPS_PER_LUP = 6  # 5 adds + 1 multiply per Laplace site update (Sec. 3 listings)


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as fh:
            return json.load(fh), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# FP64 ALU peak derived from the unit counts and clock: 152 SMs x 2 FP64 lanes per
# clock x 2070 MHz = 629.3 G FP64 operations/s (the 1.25 TFLOP/s datasheet figure
# counts an FMA as two).  Each add or multiply of the site update is one operation.
FP64_ALU_PEAK_TOPS = 152 * 2 * 2.070e9 / 1e12


class ClockSampler:
    """nvidia-smi samples every 200 ms while running (SM clock, reasons)."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.lines: list[str] = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=5)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _traffic_from_profiles(kernel: str):
    """Per-launch DRAM bytes of `kernel` from profiles/dram_traffic.txt, if recorded
    for the current source of the kernel's translation unit (else None)."""
    import hashlib

    path = os.path.join(ROOT, "profiles", "dram_traffic.txt")
    if not os.path.exists(path):
        return None
    rec = {}
    with open(path) as fh:
        for ln in fh:
            ln = ln.strip()
            if not ln or ln.startswith("#"):
                continue
            parts = ln.split()
            if len(parts) >= 4:
                rec[parts[0]] = (parts[1], parts[2], float(parts[3]))
    if kernel not in rec:
        return None
    src, digest, bytes_per_launch = rec[kernel]
    try:
        with open(os.path.join(ROOT, src), "rb") as fh:
            cur = hashlib.sha256(fh.read()).hexdigest()[:16]
    except OSError:
        return None
    return bytes_per_launch if cur == digest else None


# ------------------------------------------------------------------ oracle --
def _oracle_sample(n: int, sweeps: int):
    """Time the CPU oracle (as it stands) on the 400^3 grid for `sweeps` Jacobi and
    `sweeps` Gauss-Seidel sweeps.  Returns (GLUP/s, seconds, LUP)."""
    import oracle
    from paper_1004_1741_gb300 import workloads

    u0 = workloads.laplace_cube(n)
    t0 = time.perf_counter()
    oracle.jacobi(u0, None, 1.0, sweeps)
    oracle.gs_lex(u0, None, 1.0, sweeps)
    dt = time.perf_counter() - t0
    lup = 2.0 * sweeps * n ** 3
    return lup / dt / 1e9, dt, lup


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle.build as ob

    ob.build()
    n = N
    for _ in range(args.warmup):
        _oracle_sample(n, 1)
    times = []
    lup = 0.0
    for _ in range(args.steps):
        _, dt, lup = _oracle_sample(n, 1)
        times.append(dt)
    tot = sum(times)
    value = lup * args.steps / tot / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "jacobi+gs 400^3 fp64, 1 sweep each per step (bounded sample of the 100-sweep "
                               "workload)", "n": n, "sweeps_per_step": 1},
        "cpu_baseline": {"value": value, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
                         "sample": "400^3 FP64, 1 Jacobi + 1 Gauss-Seidel sweep per step, serial C oracle"},
        "e2e": {"value": value, "unit": "GLUP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- GPU --
def run_gpu(args):
    import torch

    from paper_1004_1741_gb300 import capi, workloads

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist  # noqa: F811

        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    ctx = capi.Context(local)

    u_host = workloads.laplace_cube(N)
    uj = torch.from_numpy(u_host).to(dev)
    ug = uj.clone()
    lup_step = 2.0 * SWEEPS * N ** 3
    cj, cg = HEADLINE["jacobi"], HEADLINE["gs"]
    ev = {k: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for k in ("j", "g")}
    acc = {"j": 0.0, "g": 0.0}

    def step(timed: bool):
        if timed:
            ev["j"][0].record(stream)
        capi.stencil_jacobi(ctx, uj, None, 1.0, SWEEPS, nt=cj["nt"], tile=cj["tile"], stream=stream)
        if timed:
            ev["j"][1].record(stream)
            ev["g"][0].record(stream)
        capi.stencil_gs_lex(ctx, ug, None, 1.0, SWEEPS, nt=cg["nt"], tile=cg["tile"], stream=stream)
        if timed:
            ev["g"][1].record(stream)
        rj = capi.residual_norm(ctx, uj, None, 1.0, stream=stream)
        rg = capi.residual_norm(ctx, ug, None, 1.0, stream=stream)
        if timed:
            acc["j"] += ev["j"][0].elapsed_time(ev["j"][1])
            acc["g"] += ev["g"][0].elapsed_time(ev["g"][1])
        return rj, rg

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clocks = ClockSampler(local)
    clocks.start()
    launches0 = ctx.kernel_launches
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        step(True)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    launches = ctx.kernel_launches - launches0
    clk = clocks.stop()
    if dist:
        tmax = torch.tensor([ms], device=dev)
        dist.all_reduce(tmax, op=dist.ReduceOp.MAX)
        ms = float(tmax.item())
        dist.barrier()
    value = world * lup_step * args.steps / (ms / 1e3) / 1e9

    # per-smoother GLUP/s over the timed region
    lup_one = SWEEPS * N ** 3 * args.steps
    glups = {"jacobi": lup_one / (acc["j"] / 1e3) / 1e9, "gs": lup_one / (acc["g"] / 1e3) / 1e9}

    # roofline of the dominant kernel (the smoother call that took longer)
    dom = "gs" if acc["g"] >= acc["j"] else "jacobi"
    kern = "gs_task_kernel" if dom == "gs" else "jacobi_zmarch_kernel"
    nlaunch = (args.steps and (launch_counts(ctx, dom, cj if dom == "jacobi" else cg))) or 1
    dur_s = (acc["g"] if dom == "gs" else acc["j"]) / 1e3 / (args.steps * nlaunch)
    flops_per_launch = FP64_OPS_PER_LUP * SWEEPS * N ** 3 / nlaunch
    achieved = flops_per_launch / dur_s / 1e12
    traffic = _traffic_from_profiles(kern)
    roofline = {"bound": "alu", "achieved": achieved, "peak": FP64_ALU_PEAK_TOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_ALU_PEAK_TOPS, "traffic": traffic, "kernel": kern,
                "peak_source": "derived: 152 SM x 2 FP64 lanes/clk x 2070 MHz (1.25 TFLOP/s FMA-counted datasheet)"}
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    hbm_bound = {str(nt): hbm * nt / 16.0 for nt in NT_SWEEP}

    details = {"glups": glups, "hbm_roofline_glups_fp64": hbm_bound, "hbm_gbs": hbm, "hbm_source": src,
               "fp64_alu_roofline_glups": FP64_ALU_PEAK_TOPS * 1e12 / FP64_OPS_PER_LUP / 1e9,
               "frac_of_min_roofline": {k: v / min(hbm / 16.0 * HEADLINE[k]["nt"],
                                                   FP64_ALU_PEAK_TOPS * 1e3 / FP64_OPS_PER_LUP)
                                        for k, v in glups.items()}}

    # temporal depth sweep (one 100-sweep run per nt and smoother, after the timed region)
    if not args.skip_nt_sweep:
        details["nt_sweep"] = nt_sweep(ctx, capi, torch, uj, ug, stream)

    # end to end through the public API: pinned host -> device, run, device -> host
    e2e = None
    if not args.skip_e2e:
        e2e = run_e2e(ctx, capi, torch, u_host, dev, stream, args)

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        g, dt, lup = _oracle_sample(N, 2)
        cpu = {"value": g, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "sample": "400^3 FP64, 2 Jacobi + 2 Gauss-Seidel sweeps (%.0f MLUP, %.1f s), serial C oracle"
                         % (lup / 1e6, dt)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "jacobi+gs 400^3 fp64, 100 sweeps each + residual norms", "n": N,
                       "sweeps": SWEEPS, "jacobi": {"nt": cj["nt"], "tile": list(cj["tile"])},
                       "gs": {"nt": cg["nt"], "tile": list(cg["tile"])}, "parallelism": "replicas" if world > 1 else "1gpu",
                       "l2": "inputs larger than L2 (2 x 512.6 MB vs 129 MB); no flush"},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches, "clocks": clk,
            "details": details,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def launch_counts(ctx, smoother, cfg):
    """Kernel launches of one 100-sweep call of `smoother` (from the library's own counter)."""
    import torch

    from paper_1004_1741_gb300 import capi

    u = torch.zeros((N + 2,) * 3, dtype=torch.float64, device="cuda")
    before = ctx.kernel_launches
    fn = capi.stencil_jacobi if smoother == "jacobi" else capi.stencil_gs_lex
    fn(ctx, u, None, 1.0, SWEEPS, nt=cfg["nt"], tile=cfg["tile"])
    torch.cuda.synchronize()
    n = ctx.kernel_launches - before
    del u
    return n


def nt_sweep(ctx, capi, torch, uj, ug, stream):
    out = {}
    for name, fn, u, cfg in (("jacobi", capi.stencil_jacobi, uj, HEADLINE["jacobi"]),
                             ("gs", capi.stencil_gs_lex, ug, HEADLINE["gs"])):
        res = {}
        for nt in NT_SWEEP:
            try:
                tile = cfg["tile"] if nt == 1 else (0, 0, 0)
                fn(ctx, u, None, 1.0, SWEEPS, nt=nt, tile=tile, stream=stream)  # warm
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn(ctx, u, None, 1.0, SWEEPS, nt=nt, tile=tile, stream=stream)
                b.record(stream)
                torch.cuda.synchronize()
                t = a.elapsed_time(b) / 1e3
                res[str(nt)] = {"glups": SWEEPS * N ** 3 / t / 1e9, "ms": t * 1e3,
                                "alg_bytes_per_lup": 16.0 / nt}
            except capi.StencilError as e:
                res[str(nt)] = {"unsupported": str(e)}
        out[name] = res
    return out


def run_e2e(ctx, capi, torch, u_host, dev, stream, args):
    hj = torch.from_numpy(u_host).pin_memory()
    hg = hj.clone().pin_memory()
    oj = torch.empty_like(hj).pin_memory()
    og = torch.empty_like(hg).pin_memory()
    dj = torch.empty(hj.shape, dtype=torch.float64, device=dev)
    dg = torch.empty_like(dj)
    cj, cg = HEADLINE["jacobi"], HEADLINE["gs"]

    def step():
        dj.copy_(hj, non_blocking=True)
        dg.copy_(hg, non_blocking=True)
        capi.stencil_jacobi(ctx, dj, None, 1.0, SWEEPS, nt=cj["nt"], tile=cj["tile"], stream=stream)
        capi.stencil_gs_lex(ctx, dg, None, 1.0, SWEEPS, nt=cg["nt"], tile=cg["tile"], stream=stream)
        capi.residual_norm(ctx, dj, None, 1.0, stream=stream)
        capi.residual_norm(ctx, dg, None, 1.0, stream=stream)
        oj.copy_(dj, non_blocking=True)
        og.copy_(dg, non_blocking=True)

    step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 3))
    a.record(stream)
    for _ in range(steps):
        step()
    b.record(stream)
    torch.cuda.synchronize()
    t = a.elapsed_time(b) / 1e3
    nbytes = hj.numel() * 8 * 2
    return {"value": 2.0 * SWEEPS * N ** 3 * steps / t / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": steps}


def run_case(args):
    """One smoother on an n^3 FP64 grid (halo seed 1, interior seed 2), --repeat calls
    of --sweeps sweeps: the small case for profiler captures."""
    import torch

    from paper_1004_1741_gb300 import capi, workloads

    ctx = capi.Context(0)
    u = torch.from_numpy(workloads.laplace_cube(args.n)).to("cuda")
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    u = u.to(dt)
    fn = capi.stencil_jacobi if args.case == "jacobi" else capi.stencil_gs_lex
    tile = tuple(int(x) for x in args.tile.split(",")) if args.tile else (0, 0, 0)
    for _ in range(args.repeat):
        fn(ctx, u, None, 1.0, args.sweeps, nt=args.nt, tile=tile)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "n": args.n, "sweeps": args.sweeps, "nt": args.nt, "repeat": args.repeat,
                      "launches": ctx.kernel_launches}))
    ctx.close()
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--skip-nt-sweep", action="store_true")
    ap.add_argument("--skip-e2e", action="store_true")
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--case", choices=["jacobi", "gs"], help="run one smoother only (profiling case)")
    ap.add_argument("--n", type=int, default=320)
    ap.add_argument("--sweeps", type=int, default=8)
    ap.add_argument("--nt", type=int, default=1)
    ap.add_argument("--tile", default="")
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--repeat", type=int, default=1)
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
