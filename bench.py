"""Benchmark: cell-updates/s of the explicit shallow-water step on GB300.

Default workload: 10,001,406 triangles (3163 x 1581 jittered grid over
100 km x 50 km), bed of 8 random sinusoids, per-cell Manning n, radial dam
break, cells and edges in Morton order, FP32 state with compensated face
sums and an FP64 mass integral; one step = one explicit Euler step of the
whole mesh (all face fluxes, updates, friction and the CFL reduction).

Prints ONE JSON line (rank 0). Under torchrun with N > 1 every rank runs an
independent replica on its own GPU (the single-mesh step has no exchange on
one GPU per rank here), and `value` is the sum over ranks divided by the
slowest rank's time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "cell-updates/s"
UNIT = "cell-updates/s"
HBM_FALLBACK_GBS = 6800.0
L2_BYTES = 129 * 1024 * 1024

# Algorithmic bytes per cell-update: each cell reads h, hu, hv, z, 1/area and
# n, each edge's nx, ny, l and two int32 endpoints once (1.5 edges per cell),
# and each cell writes h, hu, hv once: (12.5 + [n]) words + 12 bytes.
def alg_bytes_per_cell(word: int, per_cell_n: bool) -> float:
    return (12.5 + (1.0 if per_cell_n else 0.0)) * word + 12.0


WORKLOADS = {
    "sinusoid_10m": dict(fn="sinusoid_case", kw={}, per_cell_n=True, seed=3,
                         desc="10,001,406 triangles, 8-sinusoid bed, per-cell n, radial dam break"),
    "humps_1m": dict(fn="humps_case", kw={}, per_cell_n=False, seed=2,
                     desc="1,000,000 triangles, 3 Gaussian humps, n=0.03, wet/dry"),
}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d.get("hbm_gbs", HBM_FALLBACK_GBS)), "measured"
    return HBM_FALLBACK_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.out = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.out, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
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
        self.out.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 8:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[0]) for r in rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[4 + k] == "Active"})
        loaded = [s for s in sm if mx and s > 0.5 * max(mx)] or sm
        return {"sm_mhz": statistics.median(loaded) if loaded else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


def job_rate(local_cells: int, local_seconds: float, dist=None, device=None):
    """Whole-job rate over replicas: every rank's cell-updates over the slowest
    rank's time (max over ranks). Without a process group, the local rate.
    Returns (cells_per_second, slowest_seconds, total_cells)."""
    if dist is None:
        return local_cells / local_seconds, local_seconds, local_cells
    import torch
    t = torch.tensor([float(local_seconds)], dtype=torch.float64, device=device)
    c = torch.tensor([float(local_cells)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return c.item() / t.item(), t.item(), int(c.item())


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_case(name: str):
    from paper_1807_00672_gb300 import inputs
    w = WORKLOADS[name]
    return getattr(inputs, w["fn"])(**w["kw"])


def small_case(name: str, cells: int):
    """The same workload recipe at a reduced size (bounded oracle samples)."""
    from paper_1807_00672_gb300 import inputs
    w = WORKLOADS[name]
    full = getattr(inputs, w["fn"])
    if name == "sinusoid_10m":
        ny = max(4, int(round(math.sqrt(cells / 4.0))))
        scale = (2 * ny) / 3163.0
        return full(nx=2 * ny, ny=ny, lx=100_000.0 * scale, ly=50_000.0 * scale)
    ny = max(4, int(round(math.sqrt(cells / 4.0))))
    scale = (2 * ny) / 1000.0
    return full(nx=2 * ny, ny=ny, lx=10_000.0 * scale, ly=5_000.0 * scale)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rate(case, steps: int, warmup: int, threads: int = 1):
    """Cell-updates/s of the FP64 oracle on `case`, its edge and cell loops
    on `threads` host threads (the results do not depend on it)."""
    import oracle
    oracle.set_threads(threads)
    try:
        o = oracle.state_from_case(case)
        if warmup:
            o.run(warmup)
        t0 = time.perf_counter()
        o.run(steps)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_threads(1)
    return o.mesh.T * steps / dt, dt


def run_reference(args, ws, rank):
    """The FP64 CPU oracle as it stands, timed on this host's cores."""
    if rank != 0:
        return
    case = small_case(args.workload, args.ref_cells)
    t_cells = case.mesh.n_tris
    cores = host_cores()
    rate, secs = oracle_rate(case, args.steps, args.warmup, cores)
    sample = (f"same recipe as {args.workload} at {t_cells} triangles, {args.steps} steps "
              f"after {args.warmup} warm-up steps, FP64 oracle, edge and cell loops on "
              f"{cores} host threads")
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": args.workload, "triangles_sampled": t_cells},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="sinusoid_10m")
    ap.add_argument("--precision", choices=["f32", "f64"], default="f32")
    ap.add_argument("--kernel", choices=["auto", "tiled", "edge"], default="auto")
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--stages", type=int, default=0)
    ap.add_argument("--cpt", type=int, default=0, help="cells per thread of the tiled kernel")
    ap.add_argument("--halo-schedule", type=int, default=0,
                    help="tiled kernel variant: 0 default, 1 early halo gather, 2 pipelined")
    ap.add_argument("--fp64-steps", type=int, default=50)
    ap.add_argument("--e2e-steps", type=int, default=0, help="solver steps per e2e call (0 = --steps)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the fp64, error and ensemble legs")
    ap.add_argument("--no-ensemble", action="store_true", help="skip the ensemble leg")
    ap.add_argument("--ensemble-steps", type=int, default=200)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg")
    ap.add_argument("--adjoint-steps", type=int, default=500)
    ap.add_argument("--adjoint-checkpoint", type=int, default=50)
    ap.add_argument("--no-water-drop", action="store_true", help="skip the water-drop leg")
    ap.add_argument("--adjoint-profile", action="store_true",
                    help="only record 4 steps of the workload and run one gradient (a short "
                         "command to profile the adjoint kernel under ncu); prints the tape info")
    ap.add_argument("--water-drop-test", type=int, default=4, help="Table 2 grid size (1-5)")
    ap.add_argument("--no-error", action="store_true",
                    help="skip the FP32-vs-oracle error legs at full size")
    ap.add_argument("--error-steps", type=int, default=1000,
                    help="steps of the 10M workload's FP32-vs-oracle error leg")
    ap.add_argument("--humps-steps", type=int, default=500)
    ap.add_argument("--ref-cells", type=int, default=25_000)
    ap.add_argument("--cpu-cells", type=int, default=1_000_000)
    ap.add_argument("--cpu-steps", type=int, default=150)
    args = ap.parse_args()
    ws, rank, local = dist_env()

    if args.impl == "reference":
        run_reference(args, ws, rank)
        return

    import torch
    from paper_1807_00672_gb300 import build, swe

    dist = None
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    if rank == 0:
        build.build()
    if dist is not None:
        dist.barrier()
    dev = torch.device("cuda", torch.cuda.current_device())

    case = make_case(args.workload)
    if args.adjoint_profile:
        mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=args.precision, tile=args.tile)
        st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
        tape = swe.Tape(st, 4, 4, [5, 100])
        r = tape.grad(g_h=np.random.default_rng(0).standard_normal(mesh.T))
        print(json.dumps({"adjoint_profile": tape.info(),
                          "finite": bool(all(np.isfinite(v).all() for v in r.values()))}))
        return
    stream = torch.cuda.Stream(device=dev)
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=args.precision, kernel=args.kernel,
                    tile=args.tile, stages=args.stages, cells_per_thread=args.cpt,
                    halo_schedule=args.halo_schedule, stream=ctypes_stream(stream))
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    T = mesh.T
    kernels_per_step = 2 if args.kernel == "edge" else 1

    # warm-up: the step graph is captured and uploaded first (swe_run with 0
    # steps takes none), then exactly --warmup steps run
    warm = args.warmup
    st.run(0)
    st.run(warm)
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    st.run(args.steps, sync=False)
    ev1.record(stream)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    ms = ev0.elapsed_time(ev1)
    clocks = sampler.stop() if sampler else None
    st.sync()
    value, secs_max, _ = job_rate(T * args.steps, ms * 1e-3, dist, dev)
    ms = secs_max * 1e3

    # Dominant kernel. With the tiled kernel every launch in the timed region
    # is one step of k_tiled_step, so its average launch duration over the
    # timed region is the region's CUDA-event time over its launch count.
    # Single launches bracketed by events (which add launch latency and lose
    # the overlap between consecutive steps) are reported beside it.
    per_launch = []
    for _ in range(min(args.steps, 200)):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.run(1, sync=False)
        b.record(stream)
        per_launch.append((a, b))
    torch.cuda.synchronize()
    st.sync()
    isolated_ms = statistics.mean(a.elapsed_time(b) for a, b in per_launch)
    kern_ms = ms / args.steps if args.kernel != "edge" else isolated_ms
    word = 4 if args.precision == "f32" else 8
    balg = alg_bytes_per_cell(word, WORKLOADS[args.workload]["per_cell_n"])
    peak, peak_kind = measured_peaks()
    achieved = balg * T / (kern_ms * 1e-3) / 1e9
    traffic = profiled_traffic(args)

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": warm, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {
            "workload": args.workload, "desc": WORKLOADS[args.workload]["desc"],
            "triangles": T, "edges": mesh.E, "precision": args.precision,
            "kernel": args.kernel, "tile": args.tile or (512 if args.precision == "f32" and (args.cpt or 2) == 2 else 256), "stages": args.stages or 2,
            "cells_per_thread": args.cpt or 2,
            "order": "morton", "seed": WORKLOADS[args.workload]["seed"],
            "l2": f"inputs larger than L2: {mesh.device_bytes() / 1e6:.0f} MB of mesh + "
                  f"{6 * word * T / 1e6:.0f} MB of state vs 129 MB L2",
            "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
        },
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "k_tiled_step" if args.kernel != "edge" else "k_edge_flux+k_cell_update",
                     "alg_bytes_per_cell": balg, "kernel_ms": kern_ms,
                     "kernel_ms_basis": ("timed region / launches in it" if args.kernel != "edge"
                                         else "single launches between CUDA events"),
                     "isolated_launch_ms": isolated_ms,
                     "peak_source": f"{peak_kind} HBM copy bandwidth"},
        "gpu_launches": args.steps * kernels_per_step,
        "clocks": clocks,
    }

    # e2e through the C ABI with pinned host buffers: H2D of (h, hu, hv),
    # the steps, D2H of (h, hu, hv), on the wall clock. An FP32 state's
    # fields travel as FP32 arrays (swe_state_set_f32 / swe_copy_out_f32:
    # exactly the values the state holds); the FP64-array calls
    # (swe_state_set / swe_copy_out) are timed beside them. One untimed call
    # first, then the median of three.
    e2e_steps = args.e2e_steps or args.steps

    def e2e_call(word):
        ht = torch.float32 if word == 4 else torch.float64
        hp = [torch.from_numpy(np.ascontiguousarray(a)).to(ht).pin_memory()
              for a in (case.h, case.hu, case.hv)]
        ho = [torch.empty(T, dtype=ht).pin_memory() for _ in range(3)]
        times = []
        for rep in range(4):
            torch.cuda.synchronize()
            if dist is not None:
                dist.barrier()
            t0 = time.perf_counter()
            swe_set_ptrs(st, hp)
            st.run(e2e_steps, sync=False)
            swe_copy_ptrs(st, ho)
            t1 = time.perf_counter()
            if rep:
                times.append(t1 - t0)
        rate, _, _ = job_rate(T * e2e_steps, float(np.median(times)), dist, dev)
        return rate, 3 * word * T

    host_word = 4 if args.precision == "f32" else 8
    e2e_value, nbytes = e2e_call(host_word)
    out["e2e"] = {"value": e2e_value, "unit": UNIT,
                  "h2d_bytes_per_step": nbytes / e2e_steps, "d2h_bytes_per_step": nbytes / e2e_steps,
                  "steps_per_call": e2e_steps, "h2d_bytes_per_call": nbytes,
                  "d2h_bytes_per_call": nbytes, "timing": "median of 3 calls after 1 untimed call",
                  "path": (f"swe_state_set{'_f32' if host_word == 4 else ''} (pinned host, "
                           f"{'FP32' if host_word == 4 else 'FP64'} arrays) + swe_run + "
                           f"swe_copy_out{'_f32' if host_word == 4 else ''} (pinned host)")}
    if host_word == 4:
        v64, b64 = e2e_call(8)
        out["e2e"]["fp64_host_arrays"] = {"value": v64, "unit": UNIT, "h2d_bytes_per_call": b64,
                                          "d2h_bytes_per_call": b64,
                                          "path": "swe_state_set + swe_run + swe_copy_out"}

    # The adjoint leg runs first among the extras: its backward/forward
    # ratio compares two timings of the same run, taken before the long
    # FP64 and ensemble legs. The extras are single-GPU measurements: with
    # several ranks (replicas) they are skipped, so the other GPUs are not
    # held while rank 0 runs them.
    if ws > 1:
        args.no_extras = True
    errors = {}
    if rank == 0 and not args.no_extras and not args.no_adjoint:
        out["adjoint"] = adjoint_leg(args, stream, errors)
    if rank == 0 and not args.no_extras:
        out["fp64"] = fp64_leg(case, args, stream, ws)
        if args.precision == "f32":
            out["compensated_depth"] = compensated_leg(case, args, stream)
        out["humps_1m"] = humps_leg(args, stream, errors)
    if rank == 0 and not args.no_extras and not args.no_ensemble:
        out["ensemble"] = ensemble_leg(args, stream, errors)
    if rank == 0 and not args.no_extras and not args.no_water_drop:
        out["water_drop"] = water_drop_leg(args, stream)
    if rank == 0 and not args.no_extras and not args.no_error:
        errors["stoker_2500"] = stoker_error(args)
        if args.workload == "sinusoid_10m":
            errors["sinusoid_10m"] = fp32_error(case, mesh, steps=args.error_steps)
    if errors:
        out["error"] = errors
    st.close()
    mesh.close()
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        # the FP64 oracle on the same recipe: about 10-20 s single-threaded
        # (the paper's one-core comparison), then the same sample with its
        # edge and cell loops on every host core
        small = small_case(args.workload, args.cpu_cells)
        k = args.cpu_steps
        rate1, secs1 = oracle_rate(small, k, 1, 1)
        cores = host_cores()
        rate, secs = oracle_rate(small, k, 1, cores)
        out["cpu_baseline"] = {
            "value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"FP64 oracle, edge and cell loops on {cores} host threads, {k} steps of "
                      f"the same recipe at {small.mesh.n_tris} triangles ({secs:.1f} s)",
            "single_thread": {"value": rate1, "cores": 1, "seconds": secs1}}
    if rank == 0:
        out["summary"] = summary(out)
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


def ctypes_stream(stream):
    import ctypes
    return ctypes.c_void_p(stream.cuda_stream)


def swe_set_ptrs(st, tensors):
    """swe_state_set (float64 tensors) or swe_state_set_f32 (float32)."""
    import ctypes
    import torch
    from paper_1807_00672_gb300 import swe
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in tensors]
    name = "swe_state_set_f32" if tensors[0].dtype == torch.float32 else "swe_state_set"
    swe._check(getattr(swe.lib(), name)(st._h, *ptrs), name)


def swe_copy_ptrs(st, tensors):
    """swe_copy_out (float64 tensors) or swe_copy_out_f32 (float32)."""
    import ctypes
    import torch
    from paper_1807_00672_gb300 import swe
    ptrs = [ctypes.c_void_p(t.data_ptr()) for t in tensors]
    name = "swe_copy_out_f32" if tensors[0].dtype == torch.float32 else "swe_copy_out"
    swe._check(getattr(swe.lib(), name)(st._h, *ptrs, None, None), name)


def fp64_leg(case, args, stream, ws):
    """The FP64 path on the same mesh: cell-updates/s and HBM fraction."""
    import torch
    from paper_1807_00672_gb300 import swe
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f64", kernel=args.kernel,
                    tile=args.tile, stream=ctypes_stream(stream))
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    st.run(0)
    st.run(3)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    st.run(args.fp64_steps, sync=False)
    b.record(stream)
    torch.cuda.synchronize()
    st.sync()
    ms = a.elapsed_time(b) / args.fp64_steps
    balg = alg_bytes_per_cell(8, WORKLOADS[args.workload]["per_cell_n"])
    peak, kind = measured_peaks()
    achieved = balg * mesh.T / (ms * 1e-3) / 1e9
    st.close()
    mesh.close()
    out = {"value": mesh.T / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
           "steps": args.fp64_steps, "hbm_frac": achieved / peak, "achieved_gbs": achieved,
           "alg_bytes_per_cell": balg}
    # The FP64 step is bound by FP64 arithmetic: its executed flops per cell
    # (ncu count of the kernel, profiles/fp64_ops.txt) against the measured
    # FP64 fused multiply-add rate (and the nominal 1.25 TFLOP/s).
    fpc = profiled_fp64_flops(args)
    ipc = profiled_fp64_flops(args, field=3)
    rate = swe.fp64_fma_rate(ctypes_stream(stream))
    alu = {"bound": "alu", "unit": "TFLOP/s", "peak": rate, "peak_source": "measured DFMA rate",
           "peak_nominal": 1.25, "flops_per_cell": fpc}
    if fpc is not None:
        alu["achieved"] = fpc * mesh.T / (ms * 1e-3) / 1e12
        alu["frac"] = alu["achieved"] / rate
    if ipc is not None:
        # The FP64 pipe issues one DADD, DMUL or DFMA per slot; its slot rate
        # is the measured DFMA rate / 2. DADD and DMUL count one flop for a
        # whole slot, so for a pipe-bound kernel the instruction fraction is
        # the measure of how busy the FP64 units are kept.
        alu["fp64_inst_per_cell"] = ipc
        alu["pipe_frac"] = ipc * mesh.T / (ms * 1e-3) / (rate * 1e12 / 2.0)
    out["alu"] = alu
    return out


def ensemble_leg(args, stream, errors):
    """256 independent dam-break scenarios of log-uniform size (5k-500k
    triangles, 26.6M in all) in one mesh, FP32: the kernel shape comes from
    the autotuner (measured on every 8th scenario), then the whole ensemble
    is timed over --ensemble-steps steps replayed from CUDA graphs."""
    import torch
    from paper_1807_00672_gb300 import autotune, inputs, swe
    t0 = time.perf_counter()
    cases = inputs.ensemble_cases()
    total = sum(c.mesh.n_tris for c in cases)
    tuned = autotune.tune(cases[::8], "f32", key_cells=total, key_scenarios=len(cases),
                          use_cache=False)
    mesh = swe.Mesh.ensemble([(c.mesh.xy, c.mesh.tri) for c in cases], precision="f32",
                             tile=tuned["tile"], cells_per_thread=tuned["cells_per_thread"],
                             stages=tuned["stages"], halo_schedule=tuned["halo_schedule"],
                             stream=ctypes_stream(stream))
    cat = lambda name: np.concatenate([getattr(c, name) for c in cases])
    st = swe.State(mesh, cat("h"), cat("hu"), cat("hv"), cat("z"), cat("n"))
    setup_s = time.perf_counter() - t0
    st.run(16)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    k = args.ensemble_steps
    a.record(stream)
    st.run(k, sync=False)
    b.record(stream)
    torch.cuda.synchronize()
    st.sync()
    ms = a.elapsed_time(b) / k
    balg = alg_bytes_per_cell(4, False)  # n is constant within a scenario
    peak, kind = measured_peaks()
    achieved = balg * mesh.T / (ms * 1e-3) / 1e9
    steps = {st.scenario(i)["steps"] for i in (0, len(cases) - 1)}
    res = {"value": mesh.T / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": k,
           "scenarios": len(cases), "triangles": mesh.T,
           "triangles_min_max": [min(mesh.scenario_cells), max(mesh.scenario_cells)],
           "hbm_frac": achieved / peak, "achieved_gbs": achieved, "alg_bytes_per_cell": balg,
           "peak_source": f"{kind} HBM copy bandwidth",
           "shape": {"tile": tuned["tile"], "cells_per_thread": tuned["cells_per_thread"],
                     "stages": tuned["stages"], "halo_schedule": tuned["halo_schedule"],
                     "autotuned_on": f"{len(cases[::8])} scenarios"},
           "autotune_trials": sum(1 for t in tuned["trials"] if "sec_per_step" in t),
           "setup_s": setup_s, "scenario_steps": sorted(steps)}
    errors["ensemble_256"] = ensemble_error(cases, mesh, st, args.ensemble_steps)
    st.close()
    mesh.close()
    return res


def ensemble_error(cases, mesh, st, steps, every=16):
    """FP32 error of the ensemble against the FP64 oracle on every 16th
    scenario, at one simulated time for all: the smallest time the sampled
    scenarios reach in `steps` oracle steps. The ensemble restarts from its
    initial state and advances every scenario to that time (each on its own
    CFL steps); each sampled scenario's oracle advances to it as well."""
    sample = list(range(0, len(cases), every))
    t_end = min(_oracle_to(cases[i], steps=steps)[2] for i in sample)
    cat = lambda name: np.concatenate([getattr(c, name) for c in cases])
    st.set(cat("h"), cat("hu"), cat("hv"))
    m0 = {i: st.scenario(i)["mass"] for i in sample}
    st.advance(t_end)
    got = st.fields()
    per = []
    for i in sample:
        o, k, _, _ = _oracle_to(cases[i], t_end=t_end)
        a, n = mesh.scenario_offsets[i], mesh.scenario_cells[i]
        e = _rel_errors([f[a:a + n] for f in got], (o.h, o.hu, o.hv), o.mesh.cells()["area"])
        info = st.scenario(i)
        e["mass_rel_drift_fp32"] = abs(info["mass"] - m0[i]) / m0[i]
        e["steps_oracle"], e["steps_fp32"] = int(k), int(info["steps"])
        per.append(e)
    res = {"scenarios_sampled": len(sample), "t": t_end, "vs": "FP64 oracle at the same simulated time"}
    for key in per[0]:
        if key.startswith(("l1_", "linf_", "mass_")):
            res[key] = max(p[key] for p in per)  # worst sampled scenario
    res["steps_oracle_min_max"] = [min(p["steps_oracle"] for p in per), max(p["steps_oracle"] for p in per)]
    return res


# Algorithmic bytes per cell of one adjoint step: reads U^n (h, hu, hv, z),
# U^{n+1} (h, hu, hv), lambda^{n+1} (4 words), area, g n^2 and the running
# dL/d(g n^2), the edge geometry and endpoints once (1.5 edges per cell);
# writes lambda^n (4 words) and dL/d(g n^2): 23.5 words + 12 bytes.
def adjoint_bytes_per_cell(word: int) -> float:
    return 23.5 * word + 12.0


def adjoint_leg(args, stream, errors):
    """Gradient of the calibration loss (1,000,000 triangles fully wet, 64
    gauges, L = sum over steps and gauges of (h - h_obs)^2, observations from
    the same run with a perturbed Manning n) with respect to n, z and the
    initial state, through --adjoint-steps steps with checkpoints every
    --adjoint-checkpoint steps. Reports the device times of the plain forward
    run, the recorded forward and the backward (recompute + adjoint), their
    ratio, and the FP32 gradient's distance to the FP64 one."""
    import torch
    from paper_1807_00672_gb300 import inputs, swe
    N, K = args.adjoint_steps, args.adjoint_checkpoint
    case = inputs.make_config("calibration_1m")
    gauges = inputs.gauge_cells(case, 64, seed=5, radius=1_500.0)
    n_obs = inputs.perturbed_manning(case, seed=5)
    # Gradient meshes use 256-cell tiles: the adjoint kernel runs on the
    # forward's tiles, and at 512 cells its shared memory allows half as many
    # blocks per SM (the forward itself is within 2 % of its 512-cell speed).
    tile = 256
    res = {"workload": "calibration_1m", "triangles": case.mesh.n_tris, "steps": N,
           "checkpoint_every": K, "gauges": int(gauges.shape[0]), "tile": tile}
    grads, tapes, resids = {}, {}, {}
    for prec in ("f32", "f64"):
        mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec, tile=tile,
                        stream=ctypes_stream(stream))
        obs_st = swe.State(mesh, case.h, case.hu, case.hv, case.z, n_obs)
        obs_tape = swe.Tape(obs_st, N, K, gauges)
        obs = obs_tape.gauge_h.copy()
        obs_tape.close()
        obs_st.close()
        # plain forward: N steps replayed from graphs
        st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
        st.run(16)
        st.set(case.h, case.hu, case.hv)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.run(N, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        st.sync()
        fwd_ms = a.elapsed_time(b)
        st.set(case.h, case.hu, case.hv)
        tape = swe.Tape(st, N, K, gauges)
        resid = tape.gauge_h - obs
        g = 2.0 * resid
        tape.grad(g_gauge=g)  # warm-up
        r = tape.grad(g_gauge=g)
        info = tape.info()
        grads[prec] = r
        resids[prec] = resid
        word = 4 if prec == "f32" else 8
        bwd = info["grad_ms"]
        adj_step = max(bwd - (N - (N + K - 1) // K) * fwd_ms / N, 1e-9) / N
        peak, kind = measured_peaks()
        res[prec] = {
            "loss": float((resid ** 2).sum()), "forward_ms": fwd_ms,
            "recorded_forward_ms": info["record_ms"], "backward_ms": bwd,
            "backward_over_forward": bwd / fwd_ms,
            "adjoint_step_ms_est": adj_step,
            "adjoint_hbm_frac_est": adjoint_bytes_per_cell(word) * mesh.T / (adj_step * 1e-3) / 1e9 / peak,
            "tape_bytes": info["bytes"],
            "finite": bool(all(np.isfinite(v).all() for v in r.values()))}
        if prec == "f32":
            tapes["f32"] = (mesh, st, tape)  # kept for the seeded run below
            errors["calibration_1m"] = fp32_error(case, mesh, steps=N)
        else:
            tape.close()
            st.close()
            mesh.close()
    # Where the FP32 gradient's distance to the FP64 one comes from: the FP32
    # adjoint seeded with the FP64 run's residuals isolates the adjoint's own
    # error from that of the FP32 forward's gauge depths (the misfits are
    # about 1e-5 m on 3 m of water, near FP32's resolution of the depth).
    mesh32, st32, tape32 = tapes["f32"]
    seeded = tape32.grad(g_gauge=2.0 * resids["f64"])
    tape32.close()
    st32.close()
    mesh32.close()
    for k in ("n", "z", "h"):
        ref = grads["f64"][k]
        den = np.abs(ref).max()
        res[f"f32_vs_f64_rel_{k}"] = float(np.abs(grads["f32"][k] - ref).max() / den)
        res[f"f32_adjoint_f64_seeds_rel_{k}"] = float(np.abs(seeded[k] - ref).max() / den)
    res["misfit_rms_m"] = float(np.sqrt((resids["f64"] ** 2).mean()))
    res["fp32_gauge_depth_err_max_m"] = float(np.abs(resids["f32"] - resids["f64"]).max())
    res["adjoint_alg_bytes_per_cell"] = {"f32": adjoint_bytes_per_cell(4), "f64": adjoint_bytes_per_cell(8)}
    res["peak_source"] = f"{kind} HBM copy bandwidth"
    res["note"] = ("backward = recompute of each checkpoint segment's inner steps with the forward "
                   "kernel + one adjoint launch per step; adjoint step time estimated as (backward - "
                   "recomputed steps x forward step) / steps")
    return res


def water_drop_leg(args, stream):
    """The paper's water drop (Sec. 3) to its longest end time T_s = 2,400 s
    on the grid of Table 2's test --water-drop-test (4: 1,057,058 triangles),
    FP32 and FP64, through swe_advance (graph-replayed steps, exact end
    time): steps, wall time, cell-updates/s, mass drift, and the FP32 free
    surface's L1 / Linf distance to the FP64 one at T_s."""
    import torch
    from paper_1807_00672_gb300 import inputs, swe
    n = inputs.WATER_DROP_N[args.water_drop_test]
    case = inputs.water_drop_case(n)
    res = {"table2_test": args.water_drop_test, "triangles": case.mesh.n_tris, "t_end": 2400.0}
    fields = {}
    for prec in ("f32", "f64", "f32_compensated"):
        comp = prec == "f32_compensated"
        mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f32" if comp else prec,
                        compensated_depth=comp, stream=ctypes_stream(stream))
        st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
        m0 = st.mass
        st.run(16)  # capture the step graph
        st.set(case.h, case.hu, case.hv)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k = st.advance(2400.0)
        secs = time.perf_counter() - t0
        h, _, _ = st.fields()
        fields[prec] = h
        res[prec] = {"steps": k, "seconds": secs, "value": mesh.T * k / secs, "unit": UNIT,
                     "t": st.t, "mass_rel_drift": abs(st.mass - m0) / m0}
        st.close()
        mesh.close()
    eta64 = fields["f64"] - 10.0
    for key in ("f32", "f32_compensated"):
        eta32 = fields[key] - 10.0
        res[f"{key}_vs_f64_linf_eta"] = float(np.abs(eta32 - eta64).max() / np.abs(eta64).max())
        res[f"{key}_vs_f64_l1_eta"] = float(np.abs(eta32 - eta64).sum() / np.abs(eta64).sum())
    return res


def _rel_errors(got, ref, area):
    """Per field (h, hu, hv): L1 = sum area |d| / sum area |ref| and
    Linf = max |d| / max |ref|."""
    res = {}
    for name, g, r in zip(("h", "hu", "hv"), got, ref):
        d = np.abs(np.asarray(g) - r)
        den = float((area * np.abs(r)).sum())
        res[f"l1_{name}"] = float((area * d).sum()) / den if den > 0 else float(d.max())
        mx = float(np.abs(r).max())
        res[f"linf_{name}"] = float(d.max()) / mx if mx > 0 else float(d.max())
    return res


def _oracle_to(case, steps=None, t_end=None):
    """The FP64 oracle on every host core: `steps` CFL steps, or steps to
    t_end. Returns (state, steps taken, end time, seconds)."""
    import oracle
    oracle.set_threads(host_cores())
    try:
        t0 = time.perf_counter()
        o = oracle.state_from_case(case)
        if t_end is None:
            o.run(steps)
            k = steps
        else:
            k = o.advance(t_end)
        return o, k, o.t, time.perf_counter() - t0
    finally:
        oracle.set_threads(1)


def fp32_error(case, mesh=None, steps=None, t_end=None, stream=None):
    """The FP32 path against the FP64 oracle at one simulated time: the
    oracle runs `steps` CFL steps (or to t_end) from the initial state, and
    the FP32 state advances to the time the oracle reached (swe_advance: the
    last step is clamped to it), each with its own CFL time steps. Returns
    L1 / Linf of h, hu, hv, the FP64-integrated mass drift of the FP32 state
    and both step counts. `mesh`: an FP32 mesh of the case to reuse."""
    from paper_1807_00672_gb300 import swe
    o, k_ref, t_end, secs = _oracle_to(case, steps, t_end)
    own = mesh is None
    if own:
        mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f32",
                        stream=None if stream is None else ctypes_stream(stream))
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    m0 = st.mass
    k = st.advance(t_end)
    got = st.fields()
    m1 = st.mass
    res = {"triangles": int(case.mesh.n_tris), "t": t_end, "steps_oracle": int(k_ref),
           "steps_fp32": int(k), "vs": "FP64 oracle at the same simulated time"}
    res.update(_rel_errors(got, (o.h, o.hu, o.hv), o.mesh.cells()["area"]))
    res["mass_rel_drift_fp32"] = abs(m1 - m0) / m0
    res["oracle_s"] = round(secs, 2)
    st.close()
    if own:
        mesh.close()
    # the same against FP32 with a per-cell depth residual (compensated_depth)
    cm = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f32", compensated_depth=True,
                  stream=None if stream is None else ctypes_stream(stream))
    cs = swe.State(cm, case.h, case.hu, case.hv, case.z, case.n)
    m0 = cs.mass
    kc = cs.advance(t_end)
    comp = {"steps_fp32": int(kc)}
    comp.update(_rel_errors(cs.fields(), (o.h, o.hu, o.hv), o.mesh.cells()["area"]))
    comp["mass_rel_drift_fp32"] = abs(cs.mass - m0) / m0
    res["compensated_depth"] = comp
    cs.close()
    cm.close()
    return res


def stoker_error(args):
    """The 2,500-triangle dam break to T_s = 2 s (FP64 workload): the FP64
    path's largest per-field error against the oracle (max |d| / max |ref|)
    and the FP32 path's L1 / Linf."""
    from paper_1807_00672_gb300 import inputs, swe
    case = inputs.stoker_case()
    o, k_ref, t, _ = _oracle_to(case, t_end=2.0)
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f64")
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    k = st.advance(2.0)
    got = st.fields()
    res = {"triangles": mesh.T, "t": 2.0, "steps_oracle": int(k_ref), "steps_fp64": int(k)}
    res["fp64_max_rel"] = {n: float(np.abs(g - r).max() / np.abs(r).max())
                           for n, g, r in zip(("h", "hu", "hv"), got, (o.h, o.hu, o.hv))}
    st.close()
    mesh.close()
    res["fp32"] = fp32_error(case, t_end=2.0)
    return res


def humps_leg(args, stream, errors):
    """The 1,000,000-triangle workload (three Gaussian humps, n = 0.03,
    wet/dry fronts): FP32 and FP64 cell-updates/s over graph-replayed steps
    timed with CUDA events, with the HBM fraction at 62 and 112 algorithmic
    bytes per cell (scalar n); and the FP32 error against the oracle after
    --humps-steps steps (into `errors`)."""
    import torch
    from paper_1807_00672_gb300 import swe
    case = make_case("humps_1m")
    peak, kind = measured_peaks()
    res = {"triangles": case.mesh.n_tris}
    for prec, k in (("f32", args.humps_steps), ("f64", 100)):
        mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision=prec, stream=ctypes_stream(stream))
        st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
        st.run(0)
        st.run(3)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        st.run(k, sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        st.sync()
        ms = a.elapsed_time(b) / k
        balg = alg_bytes_per_cell(4 if prec == "f32" else 8, False)
        achieved = balg * mesh.T / (ms * 1e-3) / 1e9
        res[prec] = {"value": mesh.T / (ms * 1e-3), "ms_per_step": ms, "steps": k,
                     "hbm_frac": achieved / peak, "alg_bytes_per_cell": balg}
        st.close()
        if prec == "f32":
            errors["humps_1m"] = fp32_error(case, mesh, steps=args.humps_steps)
        mesh.close()
    res["peak_source"] = f"{kind} HBM copy bandwidth"
    return res


def compensated_leg(case, args, stream, steps=200):
    """The FP32 step of the same workload with a per-cell depth residual
    (compensated_depth): cell-updates/s over `steps` graph-replayed steps
    (CUDA events) and the HBM fraction at the algorithmic bytes plus the
    residual's read and write (8 B per cell)."""
    import torch
    from paper_1807_00672_gb300 import swe
    peak, kind = measured_peaks()
    mesh = swe.Mesh(case.mesh.xy, case.mesh.tri, precision="f32", compensated_depth=True,
                    stream=ctypes_stream(stream))
    st = swe.State(mesh, case.h, case.hu, case.hv, case.z, case.n)
    st.run(0)
    st.run(max(3, args.warmup))
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    st.run(steps, sync=False)
    b.record(stream)
    torch.cuda.synchronize()
    st.sync()
    ms = a.elapsed_time(b) / steps
    balg = alg_bytes_per_cell(4, WORKLOADS[args.workload]["per_cell_n"]) + 8
    res = {"value": mesh.T / (ms * 1e-3), "unit": UNIT, "ms_per_step": ms, "steps": steps,
           "alg_bytes_per_cell": balg, "hbm_frac": balg * mesh.T / (ms * 1e-3) / 1e9 / peak,
           "peak_source": f"{kind} HBM copy bandwidth"}
    st.close()
    mesh.close()
    return res


def summary(out):
    """The headline figures again, compact, at the end of the line."""
    r = lambda x: None if x is None else float(f"{x:.4g}")
    main_key = f"{out['dtype']}_{out['config']['workload']}"
    s = {main_key: {"value": r(out["value"]), "hbm_frac": r(out["roofline"]["frac"])},
         "e2e": r(out["e2e"]["value"])}
    if "fp64_host_arrays" in out["e2e"]:
        s["e2e_fp64_host_arrays"] = r(out["e2e"]["fp64_host_arrays"]["value"])
    if "fp64" in out:
        s["fp64_10m"] = {"value": r(out["fp64"]["value"]), "hbm_frac": r(out["fp64"]["hbm_frac"]),
                         "alu_frac": r(out["fp64"]["alu"].get("frac")),
                         "fp64_pipe_frac": r(out["fp64"]["alu"].get("pipe_frac"))}
    if "humps_1m" in out:
        s["humps_1m"] = {p: {"value": r(out["humps_1m"][p]["value"]),
                             "hbm_frac": r(out["humps_1m"][p]["hbm_frac"])} for p in ("f32", "f64")}
    if "ensemble" in out:
        s["ensemble"] = {"value": r(out["ensemble"]["value"]), "hbm_frac": r(out["ensemble"]["hbm_frac"])}
    if "adjoint" in out:
        a = out["adjoint"]
        s["adjoint_backward_over_forward"] = {p: r(a[p]["backward_over_forward"])
                                              for p in ("f32", "f64") if p in a}
        s["adjoint_hbm_frac_est"] = {p: r(a[p].get("adjoint_hbm_frac_est"))
                                     for p in ("f32", "f64") if p in a}
        s["adjoint_f32_vs_f64_rel_n"] = {"own_seeds": r(a.get("f32_vs_f64_rel_n")),
                                         "f64_seeds": r(a.get("f32_adjoint_f64_seeds_rel_n"))}
    if "error" in out:
        e = {}
        for cfg, v in out["error"].items():
            v = v.get("fp32", v)
            e[cfg] = {"l1_h": r(v.get("l1_h")), "linf_h": r(v.get("linf_h")),
                      "l1_hu": r(v.get("l1_hu")), "mass": r(v.get("mass_rel_drift_fp32"))}
            c = v.get("compensated_depth")
            if c:
                e[cfg]["compensated_depth"] = {"l1_h": r(c.get("l1_h")),
                                               "mass": r(c.get("mass_rel_drift_fp32"))}
        s["fp32_error_vs_oracle"] = e
    if "compensated_depth" in out:
        c = out["compensated_depth"]
        s["f32_compensated_depth"] = {"value": r(c["value"]), "hbm_frac": r(c["hbm_frac"])}
    if "water_drop" in out:
        w = out["water_drop"]
        s["water_drop_mass_drift"] = {k: r(w[k]["mass_rel_drift"])
                                      for k in ("f32", "f32_compensated", "f64") if k in w}
    return s


def kernel_source_digest():
    """First 16 hex digits of the sha256 of the step kernel's source with its
    // comments, trailing blanks and empty lines removed: the key under which
    profiles/traffic.txt and profiles/fp64_ops.txt hold counter values, so
    that they stay valid across comment edits and lapse on code changes."""
    import hashlib
    src = os.path.join(ROOT, "paper_1807_00672_gb300", "csrc", "swe_kernels.cuh")
    lines = []
    for line in open(src, encoding="utf-8"):
        code = line.split("//", 1)[0].rstrip()
        if code:
            lines.append(code)
    return hashlib.sha256("\n".join(lines).encode()).hexdigest()[:16]


def profiled_traffic(args):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the kernel source as it is now (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(path) or args.precision != "f32" or args.kernel == "edge":
        return None
    if args.tile not in (0, 512) or args.cpt not in (0, 2) or args.stages not in (0, 2):
        return None  # the capture is of the default shape
    digest = kernel_source_digest()
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 4 and parts[0] == args.workload and parts[1] == digest:
                return float(parts[2])
    return None


def profiled_fp64_flops(args, field: int = 2):
    """FP64 flops (field 2) or FP64 pipe instructions (field 3) per cell of the
    FP64 step from the committed ncu count, if it was taken on the kernel
    source as it is now and on the default shape."""
    path = os.path.join(ROOT, "profiles", "fp64_ops.txt")
    if not os.path.exists(path) or args.kernel == "edge" or args.tile not in (0, 256):
        return None
    digest = kernel_source_digest()
    with open(path) as f:
        for line in f:
            parts = line.split()
            if len(parts) >= 5 and parts[0] == args.workload and parts[1] == digest:
                try:
                    return float(parts[field])
                except ValueError:
                    return None
    return None


if __name__ == "__main__":
    main()
