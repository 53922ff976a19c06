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
# the launch configuration timed for the headline (tests/test_gpu_parity.py checks it at full size);
# int_adds: the fixed integer-pipe additions measured fastest on this positive data (the library's
# default, the adaptive form, pays a warp vote per update for data of both signs)
HEADLINE = {
    "jacobi": {"nt": 1, "tile": (32, 4, 0), "variant": 0, "int_adds": 3},
    "gs": {"nt": 1, "tile": (8, 16, 0), "variant": 5, "int_adds": 3},
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


# The roofline the bench reports divides by rates measured in the same run
# (measured_peaks: the library's throughput probes).  For context it also gives the
# figure derived from unit counts and clocks: the FP64 pipe at 152 SMs x 2 FP64 lanes
# per clock x 2070 MHz = 629.3 G FP64 operations/s (the 1.25 TFLOP/s datasheet figure
# counts an FMA as two); each add or multiply of the site update is one operation.
FP64_ALU_PEAK_TOPS = 152 * 2 * 2.070e9 / 1e12
# The kernels also run binary64 additions on the integer ALU pipe (64 lanes per clock
# per SM, ncu sm__inst_executed_pipe_alu.avg.peak_sustained = 2 warp instructions per
# cycle), each costing INT_ADD_ALU_INSTR ALU warp instructions per warp of additions
# (ncu: the Jacobi z-march executes 20.0 ALU warp instructions per warp of sites with
# no integer additions and 103.4 with three, one symmetric and two ordered).  With the
# multiply on the FP64 pipe and the five additions split freely, the two pipes together
# retire at most (2 + 64 / INT_ADD_ALU_INSTR) operations per clock per SM: the bound
# reported below.
INT_ADD_ALU_INSTR = (103.4 - 20.0) / 3
FP64_COMBINED_PEAK_TOPS = 152 * (2 + 64 / INT_ADD_ALU_INSTR) * 2.070e9 / 1e12


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
def reduce_max_over_ranks(x: float, dist, device) -> float:
    """Max of x over the ranks of the process group (x itself when dist is None).
    The timed region of a multi-GPU run is the slowest rank's."""
    if dist is None:
        return float(x)
    import torch

    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_glups(lup_per_rank: float, world: int, ms_max: float) -> float:
    """Whole-job throughput: updates of all ranks over the slowest rank's time."""
    return world * lup_per_rank / (ms_max / 1e3) / 1e9


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


def _omp_sample(n: int, sweeps: int):
    """Time the all-core CPU baseline (oracle/stencil_omp.c: Jacobi over planes, pipeline-parallel
    Gauss-Seidel, the oracle's bits) on the 400^3 grid for `sweeps` sweeps of each smoother.
    Returns (GLUP/s, seconds, LUP, threads)."""
    import oracle
    from paper_1004_1741_gb300 import workloads

    u0 = workloads.laplace_cube(n)
    oracle.gs_lex_omp(u0[:34, :34, :34].copy(), None, 1.0, 1)  # load the library, start the thread pool
    t0 = time.perf_counter()
    oracle.jacobi_omp(u0, None, 1.0, sweeps)
    oracle.gs_lex_omp(u0, None, 1.0, sweeps)
    dt = time.perf_counter() - t0
    lup = 2.0 * sweeps * n ** 3
    return lup / dt / 1e9, dt, lup, oracle.omp_threads()


def _batched_oracle_sample(count: int = 256, subset: int = 16, sweeps: int = 2):
    """Time the serial CPU oracle on the first `subset` grids of the 256-grid Poisson batch, `sweeps`
    Jacobi and `sweeps` Gauss-Seidel sweeps each; the rate stands for the whole batch (the grids are
    drawn i.i.d.).  Returns (GLUP/s Jacobi, GLUP/s Gauss-Seidel, seconds, LUP per smoother)."""
    import oracle
    from paper_1004_1741_gb300 import workloads

    cases = workloads.batched_poisson(count)[:subset]
    lup = float(sum(c.nx * c.ny * c.nz for c in cases)) * sweeps
    t0 = time.perf_counter()
    for c in cases:
        oracle.jacobi(c.u, c.f, c.h, sweeps)
    t1 = time.perf_counter()
    for c in cases:
        oracle.gs_lex(c.u, c.f, c.h, sweeps)
    t2 = time.perf_counter()
    return lup / (t1 - t0) / 1e9, lup / (t2 - t1) / 1e9, t2 - t0, lup


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
        capi.stencil_jacobi(ctx, uj, None, 1.0, SWEEPS, nt=cj["nt"], tile=cj["tile"], variant=cj["variant"],
                            int_adds=cj["int_adds"], stream=stream)
        if timed:
            ev["j"][1].record(stream)
            ev["g"][0].record(stream)
        capi.stencil_gs_lex(ctx, ug, None, 1.0, SWEEPS, nt=cg["nt"], tile=cg["tile"], variant=cg["variant"],
                            int_adds=cg["int_adds"], stream=stream)
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
    ms = reduce_max_over_ranks(ms, dist, dev)
    if dist:
        dist.barrier()
    value = whole_job_glups(lup_step * args.steps, world, ms)

    # per-smoother GLUP/s over the timed region
    lup_one = SWEEPS * N ** 3 * args.steps
    glups = {"jacobi": lup_one / (acc["j"] / 1e3) / 1e9, "gs": lup_one / (acc["g"] / 1e3) / 1e9}

    # roofline of the dominant kernel (the smoother call that took longer)
    dom = "gs" if acc["g"] >= acc["j"] else "jacobi"
    kern = ({4: "gs_column_kernel", 5: "dataflow_column_kernel"}.get(cg["variant"], "gs_direct_kernel")
            if dom == "gs" else "jacobi_zmarch_kernel")
    nlaunch = (args.steps and (launch_counts(ctx, dom, cj if dom == "jacobi" else cg))) or 1
    dur_s = (acc["g"] if dom == "gs" else acc["j"]) / 1e3 / (args.steps * nlaunch)
    flops_per_launch = FP64_OPS_PER_LUP * SWEEPS * N ** 3 / nlaunch
    achieved = flops_per_launch / dur_s / 1e12
    traffic = _traffic_from_profiles(kern)
    peaks, src = _peaks()
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    # the pipes' peaks measured in this run (throughput probes, after the timed region)
    probe = measured_peaks(capi, local)
    fp64_tops = probe["fp64_ops_per_s"] / 1e12
    comb_tops = (probe["fp64_ops_per_s"] + probe["int_add_f64_per_s"]) / 1e12
    roofline = {"bound": "alu", "achieved": achieved, "peak": comb_tops, "unit": "TFLOP/s",
                "frac": achieved / comb_tops, "traffic": traffic, "kernel": kern,
                "peak_source": "measured in this run (stencil_probe_throughput): FP64 additions/s %.3e + binary64 "
                               "additions/s on the integer pipes %.3e, both from independent chains at 32 warps per "
                               "SM; achieved counts the 6 algorithmic FP64 operations of a site update (5 adds, "
                               "1 multiply)" % (probe["fp64_ops_per_s"], probe["int_add_f64_per_s"]),
                "frac_of_fp64_pipe_only": achieved / fp64_tops,
                "hbm": {"achieved_gbs": 16.0 * SWEEPS * N ** 3 / nlaunch / dur_s / 1e9, "peak_gbs": hbm,
                        "peak_source": src + " (MEASURED_PEAKS.json copy)",
                        "frac": 16.0 * SWEEPS * N ** 3 / nlaunch / dur_s / 1e9 / hbm},
                "derived_peak_unit_counts": FP64_COMBINED_PEAK_TOPS}
    hbm_bound = {str(nt): hbm * nt / 16.0 for nt in NT_SWEEP}

    details = {"glups": glups, "hbm_roofline_glups_fp64": hbm_bound, "hbm_gbs": hbm, "hbm_source": src,
               "probe": probe,
               "fp64_pipe_roofline_glups": fp64_tops * 1e12 / FP64_OPS_PER_LUP / 1e9,
               "fp64_plus_int_roofline_glups": comb_tops * 1e12 / FP64_OPS_PER_LUP / 1e9,
               "frac_of_min_roofline": {k: v / min(hbm / 16.0 * HEADLINE[k]["nt"],
                                                   comb_tops * 1e3 / FP64_OPS_PER_LUP)
                                        for k, v in glups.items()}}

    # temporal depth sweep (one 100-sweep run per nt and smoother, after the timed region)
    if not args.skip_nt_sweep:
        details["nt_sweep"] = nt_sweep(ctx, capi, torch, uj, ug, stream)

    if not args.skip_batched:
        details["batched_256"] = batched_compare(ctx, capi, torch, dev, stream)

    # end to end through the public API: pinned host -> device, run, device -> host
    e2e = None
    if not args.skip_e2e:
        e2e = run_e2e(ctx, capi, torch, u_host, dev, stream, args)

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        g, dt, lup = _oracle_sample(N, 2)
        cpu = {"value": g, "unit": "GLUP/s", "cores": 1, "kind": "oracle",
               "sample": "400^3 FP64, 2 Jacobi + 2 Gauss-Seidel sweeps (%.0f MLUP, %.1f s), serial C oracle"
                         % (lup / 1e6, dt)}
        if "batched_256" in details:
            gj, gg, dtb, lupb = _batched_oracle_sample()
            details["batched_256"]["cpu_oracle"] = {
                "jacobi_glups": gj, "gs_glups": gg, "cores": 1, "kind": "oracle",
                "sample": "the first 16 of the 256 grids, 2 Jacobi + 2 Gauss-Seidel sweeps each (%.0f MLUP per "
                          "smoother, %.1f s), serial C oracle; the rate stands for the whole batch" % (lupb / 1e6, dtb)}
        g2, dt2, lup2, thr = _omp_sample(N, 8)
        cpu_all = {"value": g2, "unit": "GLUP/s", "cores": thr, "nproc": os.cpu_count(), "kind": "openmp",
                   "sample": "400^3 FP64, 8 Jacobi (planes split among threads) + 8 pipeline-parallel Gauss-Seidel "
                             "sweeps (%.0f MLUP, %.1f s), the oracle's arithmetic on all host cores, bit-exact with "
                             "it" % (lup2 / 1e6, dt2)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "GLUP/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "jacobi+gs 400^3 fp64, 100 sweeps each + residual norms", "n": N,
                       "sweeps": SWEEPS,
                       "jacobi": {"nt": cj["nt"], "tile": list(cj["tile"]), "variant": cj["variant"],
                                  "int_adds": cj["int_adds"]},
                       "gs": {"nt": cg["nt"], "tile": list(cg["tile"]), "variant": cg["variant"],
                              "int_adds": cg["int_adds"]}, "parallelism": "replicas" if world > 1 else "1gpu",
                       "l2": "inputs larger than L2 (2 x 512.6 MB vs 129 MB); no flush"},
            "roofline": roofline, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
            "gpu_launches": launches, "clocks": clk,
            "details": details,
        }
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()
    return 0


def measured_peaks(capi, device: int) -> dict:
    """Throughput probes on a context of their own (its workspace, including 2 GiB for the copy probe, is
    released afterwards): whole-GPU FP64, FP32, integer-ALU and integer-pipe binary64-addition rates and the
    copy kernel's DRAM bandwidth."""
    c = capi.Context(device)
    try:
        return capi.stencil_probe_throughput(c, copy_bytes=2 << 30)
    finally:
        c.close()


def launch_counts(ctx, smoother, cfg):
    """Kernel launches of one 100-sweep call of `smoother` (from the library's own counter)."""
    import torch

    from paper_1004_1741_gb300 import capi

    u = torch.zeros((N + 2,) * 3, dtype=torch.float64, device="cuda")
    before = ctx.kernel_launches
    fn = capi.stencil_jacobi if smoother == "jacobi" else capi.stencil_gs_lex
    fn(ctx, u, None, 1.0, SWEEPS, nt=cfg["nt"], tile=cfg["tile"], variant=cfg["variant"])
    torch.cuda.synchronize()
    n = ctx.kernel_launches - before
    del u
    return n


def _nt_cfg(name, nt):
    """Launch parameters of one point of the temporal-depth sweep: the FP64 headline configuration at nt = 1;
    Gauss-Seidel at nt = 2..4 (and FP32 at nt = 1) as the persistent column march with nt sweeps per task
    (8x8 columns FP64 with two integer-pipe additions, 16x8 FP32); deeper blocking, Jacobi at nt > 1 and FP32
    Jacobi the library defaults."""
    base = HEADLINE["gs" if name.startswith("gs") else "jacobi"]
    f32 = name.endswith("f32")
    if name.startswith("gs") and nt <= 4:
        if nt == 1 and not f32:
            return dict(tile=base["tile"], variant=base["variant"], int_adds=base["int_adds"])
        return dict(tile=(16, 8, 0) if f32 else (8, 8, 0), variant=5, int_adds=-1 if f32 else 2)
    if nt == 1 and not f32:
        return dict(tile=base["tile"], variant=base["variant"], int_adds=base["int_adds"])
    return dict(tile=(0, 0, 0), variant=0, int_adds=-1)


def nt_sweep(ctx, capi, torch, uj, ug, stream):
    out = {}
    for name, fn, u in (("jacobi", capi.stencil_jacobi, uj), ("gs", capi.stencil_gs_lex, ug),
                        ("jacobi_f32", capi.stencil_jacobi, uj.float()), ("gs_f32", capi.stencil_gs_lex, ug.float())):
        res = {}
        for nt in NT_SWEEP:
            cfg = _nt_cfg(name, nt)
            try:
                fn(ctx, u, None, 1.0, SWEEPS, nt=nt, stream=stream, **cfg)  # warm
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn(ctx, u, None, 1.0, SWEEPS, nt=nt, stream=stream, **cfg)
                b.record(stream)
                torch.cuda.synchronize()
                t = a.elapsed_time(b) / 1e3
                res[str(nt)] = {"glups": SWEEPS * N ** 3 / t / 1e9, "ms": t * 1e3,
                                "alg_bytes_per_lup": (8.0 if u.dtype == torch.float32 else 16.0) / nt,
                                "variant": cfg["variant"], "tile": list(cfg["tile"])}
            except capi.StencilError as e:
                res[str(nt)] = {"unsupported": str(e)}
        out[name] = res
    return out


def batched_compare(ctx, capi, torch, dev, stream, count=256):
    """256 uneven Poisson grids (extents multiples of 16 in [32,192], seed 3): the
    plain per-grid loop of single-grid calls vs one batched call with the library defaults
    and with the parameters the whole-batch autotuner picks, 50 Jacobi and 20 Gauss-Seidel
    sweeps, FP64; speedup = plain / the faster batched."""
    from paper_1004_1741_gb300 import workloads

    cases = workloads.batched_poisson(count)
    us = [torch.from_numpy(c.u).to(dev) for c in cases]
    fs = [torch.from_numpy(c.f).to(dev) for c in cases]
    hs = [c.h for c in cases]
    saved = [u.clone() for u in us]
    sites = float(sum(c.nx * c.ny * c.nz for c in cases))
    out = {"grids": count, "sites": sites}

    def timed(fn):
        for u, s0 in zip(us, saved):
            u.copy_(s0)
        fn()  # warm (tables, plans, graphs)
        for u, s0 in zip(us, saved):
            u.copy_(s0)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / 1e3

    for name, sm, sweeps, single in (("jacobi", capi.STENCIL_JACOBI, 50, capi.stencil_jacobi),
                                     ("gs", capi.STENCIL_GS, 20, capi.stencil_gs_lex)):
        t_plain = timed(lambda: [single(ctx, u, f, h, sweeps, stream=stream) for u, f, h in zip(us, fs, hs)])
        t_batch = timed(lambda: capi.stencil_batched(ctx, us, fs, hs, [sweeps] * count, sm, stream=stream))
        # the whole-batch autotuner: candidates timed on copies of these grids, as the batched call runs them
        params, tune_glups = capi.stencil_autotune_batched(ctx, us, fs, hs, [sweeps] * count, sm, stream=stream)
        t_tuned = timed(lambda: capi.stencil_batched(ctx, us, fs, hs, [sweeps] * count, sm, stream=stream, **params))
        lup = sites * sweeps
        out[name] = {"sweeps": sweeps, "plain_glups": lup / t_plain / 1e9, "batched_glups": lup / t_batch / 1e9,
                     "autotuned": {"params": {k: (list(v) if isinstance(v, tuple) else v) for k, v in params.items()},
                                   "tuner_glups": tune_glups, "batched_glups": lup / t_tuned / 1e9},
                     "speedup": t_plain / min(t_batch, t_tuned)}
    del us, fs, saved
    torch.cuda.empty_cache()
    return out


def run_e2e(ctx, capi, torch, u_host, dev, stream, args):
    """The headline step end to end through the C ABI: every step copies both grids in from pinned host
    memory, runs the two smoothers, computes both residual norms and copies both grids back.  The steps are
    pipelined over two sets of device grids and three streams: step k+1's grids are copied in while step k
    computes (issued after step k's Jacobi call, before its blocking persistent Gauss-Seidel call), and step
    k's results are copied out while step k+1 computes (the kernels themselves run one after the other on the
    compute stream, as in the device-timed step).  Timed from the first copy in to the last copy out."""
    import numpy as np

    hj = torch.from_numpy(u_host).pin_memory()
    hg = hj.clone().pin_memory()
    oj = torch.empty_like(hj).pin_memory()
    og = torch.empty_like(hg).pin_memory()
    dj = [torch.empty(hj.shape, dtype=torch.float64, device=dev) for _ in range(2)]
    dg = [torch.empty_like(dj[0]) for _ in range(2)]
    cj, cg = HEADLINE["jacobi"], HEADLINE["gs"]
    s_in, s_out = torch.cuda.Stream(device=dev), torch.cuda.Stream(device=dev)
    s_run = stream
    ev_in = [torch.cuda.Event() for _ in range(2)]
    ev_run = [torch.cuda.Event() for _ in range(2)]
    ev_out = [torch.cuda.Event() for _ in range(2)]
    used = [False, False]

    def copy_in(k):
        b = k % 2
        with torch.cuda.stream(s_in):
            if used[b]:
                s_in.wait_event(ev_out[b])  # buffer b's previous results have been copied out
            dj[b].copy_(hj, non_blocking=True)
            dg[b].copy_(hg, non_blocking=True)
            ev_in[b].record(s_in)

    def run(k, prefetch):
        b = k % 2
        s_run.wait_event(ev_in[b])
        capi.stencil_jacobi(ctx, dj[b], None, 1.0, SWEEPS, nt=cj["nt"], tile=cj["tile"], variant=cj["variant"],
                            int_adds=cj["int_adds"], stream=s_run)
        if prefetch:  # the next step's grids go in now: the persistent Gauss-Seidel call returns when it is done
            copy_in(k + 1)
        capi.stencil_gs_lex(ctx, dg[b], None, 1.0, SWEEPS, nt=cg["nt"], tile=cg["tile"], variant=cg["variant"],
                            int_adds=cg["int_adds"], stream=s_run)
        capi.residual_norm(ctx, dj[b], None, 1.0, stream=s_run)
        capi.residual_norm(ctx, dg[b], None, 1.0, stream=s_run)
        ev_run[b].record(s_run)
        with torch.cuda.stream(s_out):
            s_out.wait_event(ev_run[b])
            oj.copy_(dj[b], non_blocking=True)
            og.copy_(dg[b], non_blocking=True)
            ev_out[b].record(s_out)
        used[b] = True

    copy_in(0)  # warm-up: workspace, plans, graphs
    for k in range(2):
        run(k, k == 0)
    torch.cuda.synchronize()
    a, b_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    steps = max(1, min(args.steps, 10))
    a.record(s_in)
    copy_in(0)
    for k in range(steps):
        run(k, k + 1 < steps)
    s_in.wait_stream(s_out)
    b_.record(s_in)
    torch.cuda.synchronize()
    t = a.elapsed_time(b_) / 1e3
    nbytes = hj.numel() * 8 * 2
    last = (steps - 1) % 2
    if not (np.array_equal(oj.numpy(), dj[last].cpu().numpy()) and np.array_equal(og.numpy(), dg[last].cpu().numpy())):
        raise RuntimeError("e2e: the grids read back differ from the device grids")
    return {"value": 2.0 * SWEEPS * N ** 3 * steps / t / 1e9, "unit": "GLUP/s", "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes, "steps": steps, "streams": 3, "pipelined": "2 sets of device grids"}


def run_case(args):
    """One smoother on an n^3 grid (halo seed 1, interior seed 2, or zero with --zero-u; --poisson
    adds f ~ N(0,1)):
    one untimed call (workspace, plans, graphs), then --repeat calls of --sweeps sweeps timed
    with CUDA events: the small case for profiler captures and single-configuration timings."""
    import numpy as np
    import torch

    from paper_1004_1741_gb300 import capi, workloads

    ctx = capi.Context(0)
    if args.case == "mg":  # --sweeps V-cycles of the multigrid solve on the sine-mode problem (FP64)
        prob = workloads.sine_modes_problem(args.n, seed=4)
        f = torch.from_numpy(prob.f).to("cuda")
        u = torch.zeros_like(f)
        sm = capi.STENCIL_GS if args.variant == 0 else capi.STENCIL_JACOBI
        for _ in range(args.repeat):
            capi.stencil_mg_solve(ctx, u, f, prob.h, sm, rtol=0.0, max_cycles=args.sweeps)
        torch.cuda.synchronize()
        print(json.dumps({"case": "mg", "n": args.n, "cycles": args.sweeps, "launches": ctx.kernel_launches}))
        ctx.close()
        return 0
    u = torch.from_numpy(workloads.laplace_cube(args.n)).to("cuda")
    if args.zero_u:
        u.zero_()
    dt = torch.float32 if args.dtype == "f32" else torch.float64
    u = u.to(dt)
    f = None
    if args.poisson:  # f ~ N(0,1) on the interior (seed 1), h = 1/(n+1)
        rng = np.random.default_rng(1)
        fh = np.zeros(u.shape)
        fh[1:-1, 1:-1, 1:-1] = rng.standard_normal((args.n,) * 3)
        f = torch.from_numpy(fh).to("cuda").to(dt)
    h = 1.0 / (args.n + 1) if args.poisson else 1.0
    fn = capi.stencil_jacobi if args.case == "jacobi" else capi.stencil_gs_lex
    tile = tuple(int(x) for x in args.tile.split(",")) if args.tile else (0, 0, 0)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    fn(ctx, u, f, h, args.sweeps, nt=args.nt, tile=tile, variant=args.variant, int_adds=args.int_adds)
    torch.cuda.synchronize()
    n0 = ctx.kernel_launches
    a.record()
    for _ in range(args.repeat):
        fn(ctx, u, f, h, args.sweeps, nt=args.nt, tile=tile, variant=args.variant, int_adds=args.int_adds)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    print(json.dumps({"case": args.case, "n": args.n, "sweeps": args.sweeps, "nt": args.nt, "repeat": args.repeat,
                      "variant": args.variant, "int_adds": args.int_adds, "dtype": args.dtype,
                      "poisson": bool(args.poisson), "zero_u": bool(args.zero_u),
                      "launches": ctx.kernel_launches - n0, "ms": ms,
                      "glups": args.n ** 3 * args.sweeps * args.repeat / ms / 1e6,
                      "workspace_mb": ctx.workspace_bytes / 1e6}))
    ctx.close()
    return 0


def run_suite_mixed(args):
    """Mixed precision against FP64 at equal final residual on the sine-mode Poisson problem
    (8 modes + N(0,1e-3) noise, seed 4).

    Main comparison: time to ||r||/||f|| <= 1e-10 at 511^3 (the largest cube below 512 whose
    multigrid levels nest) of the FP64 multigrid V(2,2) solve against the defect correction with
    FP32 V(2,2) cycles inside (FP64 residual and update), per smoother, with the largest
    difference of the two solutions.  Context: at 512^3 the plain FP64 sweeps run a fixed budget
    and the defect correction with plain FP32 sweeps inside runs until the same residual (plain
    smoothers need ~10^6 sweeps for 1e-10 at this size)."""
    import torch

    from paper_1004_1741_gb300 import capi, workloads

    nmg = args.n if args.n != 320 else 511
    rtol = 1e-10
    dev = torch.device("cuda", 0)
    ctx = capi.Context(0)
    prob = workloads.sine_modes_problem(nmg, seed=4)
    f = torch.from_numpy(prob.f).to(dev)
    mg = {}
    for name, sm in (("gs", capi.STENCIL_GS), ("jacobi", capi.STENCIL_JACOBI), ("gs_rb", capi.STENCIL_GS_RB)):
        def run_f64(u):
            return capi.stencil_mg_solve(ctx, u, f, prob.h, sm, nu1=2, nu2=2, ncoarse=20, rtol=rtol, max_cycles=60)

        def run_mixed(u):
            return capi.stencil_solve_mixed_mg(ctx, u, f, prob.h, sm, nu1=2, nu2=2, ncoarse=20, rtol=rtol,
                                               max_outer=60, inner_cycles=args.inner)
        out = {}
        for label, fn in (("fp64_mg", run_f64), ("mixed_mg", run_mixed)):
            u = torch.zeros_like(f)
            fn(u)  # warm-up: workspace, task tables, plans
            times = []
            for _ in range(max(1, args.repeat)):
                u.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                rel, iters, ok = fn(u)
                torch.cuda.synchronize()
                times.append(time.perf_counter() - t0)
            out[label] = {"iters": iters, "rel": rel, "reached": ok, "s": min(times), "s_all": times,
                          "u": u}
        a, b = out["fp64_mg"].pop("u"), out["mixed_mg"].pop("u")
        umax = float(a.abs().max().item())
        mg[name] = {**out, "inner_cycles": args.inner,
                    "speedup_at_equal_residual": out["fp64_mg"]["s"] / out["mixed_mg"]["s"],
                    "max_abs_diff_u_over_max_u": float((a - b).abs().max().item()) / umax}
        del a, b
    del f
    torch.cuda.empty_cache()
    # context: plain sweeps at 512^3, equal residual after a fixed FP64 budget
    n = 512
    prob = workloads.sine_modes_problem(n, seed=4)
    f = torch.from_numpy(prob.f).to(dev)
    plain = {}
    for name, sm in (("jacobi", capi.STENCIL_JACOBI), ("gs", capi.STENCIL_GS)):
        budget, check = 200, 20
        u = torch.zeros_like(f)
        capi.stencil_solve_f64(ctx, u, f, prob.h, sm, 0.0, check, check)  # warm
        u.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rel64, sw, _ = capi.stencil_solve_f64(ctx, u, f, prob.h, sm, 0.0, budget, check)
        torch.cuda.synchronize()
        t64 = time.perf_counter() - t0
        u2 = torch.zeros_like(f)
        capi.stencil_solve_mixed(ctx, u2, f, prob.h, sm, 0.5, 1, check)  # warm
        u2.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        relm, outer, ok = capi.stencil_solve_mixed(ctx, u2, f, prob.h, sm, rel64, 10 * budget // check, check)
        torch.cuda.synchronize()
        tm = time.perf_counter() - t0
        plain[name] = {"fp64": {"sweeps": sw, "rel": rel64, "s": t64},
                       "mixed": {"outer": outer, "inner_sweeps": check, "rel": relm, "reached": ok, "s": tm},
                       "speedup_at_equal_residual": t64 / tm,
                       "max_abs_diff_u_over_max_u": float((u2 - u).abs().max().item()) / float(u.abs().max().item())}
    line = {"suite": "mixed",
            "metric": "time to ||r||/||f|| <= 1e-10, %d^3 Poisson: FP64 multigrid vs FP32 multigrid inside FP64 "
                      "defect correction" % nmg, "n": nmg, "rtol": rtol, "unit": "s", "data": "synthetic",
            "multigrid": mg,
            "context_plain_sweeps_512": {"metric": "time to equal relative residual after 200 FP64 sweeps",
                                         "results": plain}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_suite_mg(args):
    """Multigrid V-cycle solve of the sine-mode Poisson problem (8 modes + N(0,1e-3)
    noise, seed 4) at 511^3 (odd extents: 8 levels down to 1^3) to a relative
    residual of 1e-10 with each smoother, V(2,2), 20 coarsest sweeps; against the
    plain FP64 sweeps of the same smoother (which need ~10^6 sweeps for 1e-10 at
    this size: their time is projected from their measured GLUP/s) and the serial
    oracle's time per V-cycle on a bounded 127^3 sample."""
    import torch

    import oracle
    from paper_1004_1741_gb300 import capi, workloads

    n = args.n if args.n != 320 else 511
    prob = workloads.sine_modes_problem(n, seed=4)
    dev = torch.device("cuda", 0)
    ctx = capi.Context(0)
    f = torch.from_numpy(prob.f).to(dev)
    res = {}
    for name, sm in (("gs", capi.STENCIL_GS), ("jacobi", capi.STENCIL_JACOBI), ("gs_rb", capi.STENCIL_GS_RB)):
        u = torch.zeros_like(f)
        capi.stencil_mg_solve(ctx, u, f, prob.h, sm, rtol=0.0, max_cycles=1)  # warm (workspace, tables)
        u.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rel, cycles, ok = capi.stencil_mg_solve(ctx, u, f, prob.h, sm, nu1=2, nu2=2, ncoarse=20, rtol=1e-10,
                                                max_cycles=60)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        abs_r, rel_check = capi.residual_norm(ctx, u, f, prob.h)
        res[name] = {"cycles": cycles, "rel": rel, "reached": ok, "s": t, "s_per_cycle": t / max(cycles, 1),
                     "rel_check": rel_check, "fine_sweep_equivalent_glups": n ** 3 * 4 * cycles / t / 1e9}
        if sm == capi.STENCIL_GS_RB:
            continue
        # plain sweeps of the same smoother for comparison (measured rate, projected count)
        u2 = torch.zeros_like(f)
        rel200, sw, _ = capi.stencil_solve_f64(ctx, u2, f, prob.h, sm, 0.0, 200, 100)
        u2.zero_()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        rel200, sw, _ = capi.stencil_solve_f64(ctx, u2, f, prob.h, sm, 0.0, 200, 100)
        torch.cuda.synchronize()
        t_sw = time.perf_counter() - t1
        res[name]["plain_sweeps"] = {"sweeps": sw, "rel_after": rel200, "s": t_sw, "glups": n ** 3 * sw / t_sw / 1e9}
    # CPU oracle: one V-cycle on a 127^3 sample of the same problem family
    small = workloads.sine_modes_problem(127, seed=4)
    t0 = time.perf_counter()
    oracle.mg_solve(small.f * 0.0, small.f, small.h, oracle.MG_GS, 2, 2, 20, 32, 0.0, 1)
    t_cpu = time.perf_counter() - t0
    line = {"suite": "mg", "metric": "time to relative residual 1e-10, %d^3 Poisson, multigrid V(2,2)" % n,
            "n": n, "unit": "s", "data": "synthetic", "results": res,
            "cpu_oracle": {"n": 127, "smoother": "gs", "s_per_cycle": t_cpu, "cores": 1, "kind": "oracle"}}
    print(json.dumps(line), flush=True)
    ctx.close()
    return 0


def run_suite_served(args):
    """Served stream: Poisson arrivals of smoothing and solve requests (sides log-uniform in [32, 384],
    rounded to multiples of 16, solve requests one less so that their multigrid levels nest; 10-200 sweeps,
    or a solve to 1e-8 capped at 2000 fine-grid sweeps; FP64/FP32 smoothing), 150 GB HBM budget, for a range
    of arrival rates; p50/p99 latency, GLUP/s, admitted/cancelled per rate.  At most --slots requests are on
    the device at once; --grace seconds after the end of the arrival window the requests never admitted are
    cancelled (counted) and the admitted ones drain.  Host inputs and result buffers are page-locked.  Solve
    requests run red-black multigrid V(2,2) cycles in FP64, or with --solve mixed FP32 cycles inside FP64
    defect correction (in both arms).  Beside it, the same streams served one request at a time through the plain
    single-grid calls (copy in, smooth or multigrid-solve, copy out), first come first served: the per-request
    baseline."""
    import numpy as np
    import torch

    from paper_1004_1741_gb300 import capi, workloads

    rates = [float(x) for x in args.rates.split(",")]
    window = args.window
    pool = {}

    def pinned(a):
        """a copy of a in page-locked host memory (the copies of both arms run at the link's rate)"""
        t = torch.empty(a.shape, dtype=torch.float64 if a.dtype == np.float64 else torch.float32, pin_memory=True)
        out = t.numpy()
        out[...] = a
        keep.append(t)
        return out

    keep = []

    def inputs(nn, dt):
        key = (nn, dt)
        if key not in pool:
            rng = np.random.default_rng(nn)
            u = rng.random((nn + 2,) * 3)
            u[1:-1, 1:-1, 1:-1] = 0.0
            fz = np.zeros_like(u)
            fz[1:-1, 1:-1, 1:-1] = rng.standard_normal((nn,) * 3)
            pool[key] = (pinned(u.astype(dt)), pinned(fz.astype(dt)))
        return pool[key]

    def shape(r):
        nn = max(32, min(384, 16 * round(r.n / 16)))
        if r.kind == "solve":
            nn -= 1
        dt = np.float64 if (r.dtype == "f64" or r.kind == "solve") else np.float32
        return nn, dt

    mixed = args.solve == "mixed"  # solve requests: FP32 multigrid cycles inside FP64 defect correction
    kinds = {"jacobi": capi.STENCIL_REQ_JACOBI, "gs": capi.STENCIL_REQ_GS,
             "solve": capi.STENCIL_REQ_SOLVE_MIXED if mixed else capi.STENCIL_REQ_SOLVE}
    outs = {}

    def pct(lat, q):
        return lat[min(len(lat) - 1, int(q * (len(lat) - 1) + 0.5))] if lat else None

    def prepare(reqs):
        """the stream's host buffers, page-locked before the clock starts: inputs per shape, and one
        result buffer per shape (what the copy back costs, without a buffer per request; the values
        are not used)"""
        for r in reqs:
            if r.arrival_s > window:
                break
            nn, dt = shape(r)
            u, _ = inputs(nn, dt)
            if (nn, dt) not in outs:
                outs[(nn, dt)] = pinned(np.empty_like(u))

    def served(reqs):
        prepare(reqs)
        with capi.Server(0, hbm_budget_bytes=150 * 10 ** 9, sweeps_per_round=args.quantum,
                         max_active=args.slots) as srv:
            t0 = time.perf_counter()
            tickets, late = [], []
            for r in reqs:
                if r.arrival_s > window:
                    break
                now = time.perf_counter() - t0
                if r.arrival_s > now:
                    time.sleep(r.arrival_s - now)
                nn, dt = shape(r)
                u, fz = inputs(nn, dt)
                late.append(time.perf_counter() - t0 - r.arrival_s)  # the server's latency starts at submit
                tickets.append(srv.submit(kinds[r.kind], u, fz, 1.0 / (nn + 1), r.sweeps, rtol=r.rtol,
                                          u_out=outs[(nn, dt)]))
            t_arr = time.perf_counter() - t0
            time.sleep(args.grace)  # requests that arrived just before the window closed get admitted
            for t in tickets:  # then what was never admitted is cancelled, admitted work drains
                srv.cancel(t)
            results = [srv.wait(t, args.drain) for t in tickets]
            t_end = time.perf_counter() - t0
            st = srv.stats()
        if any(r is None for r in results):
            raise RuntimeError("served requests did not drain within %.0f s" % args.drain)
        ok = (capi.STENCIL_OK, capi.STENCIL_ERR_NOT_CONVERGED)
        # latency from the scheduled arrival, like the one-at-a-time baseline's
        lat = sorted(r["latency_s"] + lt for r, lt in zip(results, late) if r["status"] in ok)
        done = [r for r in results if r["status"] in ok]
        # the last result's completion, from the stream's start (the grace wait and the drain's polling
        # are not work)
        t_last = max([reqs[i].arrival_s + lt + r["latency_s"] for i, (r, lt) in enumerate(zip(results, late))
                      if r["status"] in ok] or [t_end])
        return {"submitted": len(tickets), "completed": len(done),
                "cancelled": sum(1 for r in results if r["status"] == capi.STENCIL_ERR_CANCELLED),
                "solves_converged": sum(1 for r in results if r["status"] == capi.STENCIL_OK and r["rel_residual"] >= 0),
                "p50_s": pct(lat, 0.5), "p99_s": pct(lat, 0.99), "glups_busy": st["glups"],
                "smoothing_glups": st["smooth_lup"] / st["smooth_s"] / 1e9 if st["smooth_s"] > 0 else None,
                "solve_cycles": st["solve_cycles"], "solve_s": st["solve_s"], "smoothing_s": st["smooth_s"],
                "copy_gb": st["copy_bytes"] / 1e9, "copy_s": st["copy_s"],
                "glups_wall": st["lup_total"] / t_last / 1e9, "lup": st["lup_total"], "busy_s": st["busy_s"],
                "wall_s": t_last, "arrival_window_s": t_arr, "hbm_peak_gb": st["hbm_peak"] / 1e9,
                "launches": st["launches"]}

    def plain(reqs):
        """The same arrivals, one request at a time (FIFO) through the single-grid calls."""
        ctx = capi.Context(0)
        dev = torch.device("cuda", 0)
        prepare(reqs)
        t0 = time.perf_counter()
        lat, lup, n = [], 0.0, 0
        t_smooth, lup_smooth, t_copy = 0.0, 0.0, 0.0
        for r in reqs:
            if r.arrival_s > window:
                break
            now = time.perf_counter() - t0
            if r.arrival_s > now:
                time.sleep(r.arrival_s - now)
            nn, dt = shape(r)
            uh, fh = inputs(nn, dt)
            tc = time.perf_counter()
            u = torch.from_numpy(uh).to(dev)
            f = torch.from_numpy(fh).to(dev)
            torch.cuda.synchronize()
            t_copy += time.perf_counter() - tc
            h = 1.0 / (nn + 1)
            if r.kind == "solve":
                cyc = 0
                solve = capi.stencil_solve_mixed_mg if mixed else capi.stencil_mg_solve
                cap = {"max_outer": r.sweeps // 4} if mixed else {"max_cycles": r.sweeps // 4}
                rel, cyc, _ = solve(ctx, u, f, h, capi.STENCIL_GS_RB, nu1=2, nu2=2, ncoarse=args.quantum,
                                    rtol=r.rtol, **cap)
                lup += 4.0 * cyc * nn ** 3
            else:
                torch.cuda.synchronize()
                ts = time.perf_counter()
                (capi.stencil_jacobi if r.kind == "jacobi" else capi.stencil_gs_lex)(ctx, u, f, h, r.sweeps)
                torch.cuda.synchronize()
                t_smooth += time.perf_counter() - ts
                lup += float(r.sweeps) * nn ** 3
                lup_smooth += float(r.sweeps) * nn ** 3
            torch.cuda.synchronize()
            tc = time.perf_counter()
            torch.from_numpy(outs[(nn, dt)]).copy_(u)
            t_copy += time.perf_counter() - tc
            lat.append(time.perf_counter() - t0 - r.arrival_s)
            n += 1
        t_end = time.perf_counter() - t0
        ctx.close()
        lat.sort()
        return {"completed": n, "p50_s": pct(lat, 0.5), "p99_s": pct(lat, 0.99), "glups_wall": lup / t_end / 1e9,
                "smoothing_glups": lup_smooth / t_smooth / 1e9 if t_smooth > 0 else None, "copy_s": t_copy,
                "wall_s": t_end}

    out = []
    for rate in rates:
        reqs = workloads.served_stream(rate, max(1, int(rate * window * 1.2)), seed=5)
        row = {"rate_hz": rate, "served": served(reqs)}
        if rate <= args.plain_max_rate:
            row["plain_per_request"] = plain(reqs)
        out.append(row)
    line = {"suite": "served", "metric": "p50/p99 latency and GLUP/s vs arrival rate (continuous batching), beside "
                                         "the same streams served one request at a time",
            "unit": "s", "data": "synthetic", "window_s": window, "slots": args.slots,
            "sweeps_per_round": args.quantum, "solve": args.solve, "results": out}
    print(json.dumps(line), flush=True)
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
    ap.add_argument("--skip-batched", action="store_true")
    ap.add_argument("--case", choices=["jacobi", "gs", "mg"],
                    help="run one smoother (or the multigrid solve: --variant 0 GS, 1 Jacobi) only (profiling case)")
    ap.add_argument("--n", type=int, default=320)
    ap.add_argument("--sweeps", type=int, default=8)
    ap.add_argument("--nt", type=int, default=1)
    ap.add_argument("--tile", default="")
    ap.add_argument("--dtype", choices=["f64", "f32"], default="f64")
    ap.add_argument("--variant", type=int, default=0, help="kernel variant of the profiling case")
    ap.add_argument("--int-adds", type=int, default=-1, help="integer-pipe additions of the profiling case")
    ap.add_argument("--poisson", action="store_true", help="profiling case with f ~ N(0,1) instead of f = 0")
    ap.add_argument("--zero-u", action="store_true",
                    help="profiling case from u = 0 (halo too): with --poisson the iterates take both signs")
    ap.add_argument("--repeat", type=int, default=1)
    ap.add_argument("--inner", type=int, default=1, help="FP32 V-cycles per outer iteration (--suite mixed)")
    ap.add_argument("--suite", choices=["mixed", "served", "mg"], help="a secondary workload instead of the headline")
    ap.add_argument("--rates", default="2,5,10,25,50,100,200,500,2000")
    ap.add_argument("--plain-max-rate", type=float, default=500.0,
                    help="--suite served: rates up to this also run the one-request-at-a-time baseline")
    ap.add_argument("--window", type=float, default=3.0)
    ap.add_argument("--drain", type=float, default=60.0)
    ap.add_argument("--grace", type=float, default=0.5,
                    help="--suite served: seconds after the window before unadmitted requests are cancelled")
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--quantum", type=int, default=50, help="--suite served: sweeps per request and round")
    ap.add_argument("--solve", choices=["f64", "mixed"], default="f64",
                    help="--suite served: solve requests as FP64 multigrid or FP32 multigrid in FP64 defect correction")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.suite == "mixed":
        return run_suite_mixed(args)
    if args.suite == "served":
        return run_suite_served(args)
    if args.suite == "mg":
        return run_suite_mg(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
