#!/usr/bin/env python3
"""Throughput of the fused D3Q27 cumulant LBM + actuator-line time step.

Workload: the single-rotor case, 256x128x128 cells, velocity inlet 0.05 lu
with 1 % seeded white noise, zero-gradient outlet, periodic y/z, one
three-bladed rotor (D = 32 cells at (64, 64, 64), 40 Gaussian-spread elements
per blade, eps = 2, TSR 6, synthetic polars), FP32 PDF storage.  A step is one
launch of the fused stream-collide kernel, which also evaluates the actuator
line of the next step.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
the host cores instead (rank 0 only).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MLUPS & % HBM roofline per GB300 (fused LBM+ALM step) vs plain FP32 at stated accuracy"
WORKLOAD = "single_turbine_256x128x128"
DIAG_EVERY = 100  # FP64 mass/momentum sums fused into every 100th step


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5000)
    p.add_argument("--warmup", type=int, default=50)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--storage", choices=["fp32", "bf16", "fp16"], default="fp32")
    p.add_argument("--collision", choices=["cumulant", "srt_smag"], default="cumulant")
    p.add_argument("--tile", type=str, default="auto",
                   help="CTA tile XxY, XxYxZ or XxYxZxS (S = 1: rows staged in shared memory; S = 2: one cell "
                        "per thread where the bulk kernel would take two), or 'auto' (the library's autotuner, cached)")
    p.add_argument("--workload", choices=["single", "batch16", "periodic", "precision", "warmstart", "tilesweep"],
                   default="single",
                   help="single: the 256x128x128 rotor case; batch16: 16 seeded rotor lattices stepped by "
                        "the same two launches; precision: 512x256x256 rotor, FP32 vs BF16 vs FP16 storage, mean wake profiles; "
                        "warmstart: 3x3 farm, steps to a settled mean from a cold vs a surrogate warm start; "
                        "tilesweep: the single-rotor workload at every tile candidate of the tuner; "
                        "periodic: the 256x128x128 lattice periodic, without rotor or inlet, from a seeded "
                        "near-equilibrium state (with --inplace: one PDF array, AA pattern)")
    p.add_argument("--inplace", action="store_true", help="one PDF array (AA pattern), periodic or single workload")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-bf16", action="store_true", help="skip the BF16-storage record of the default line")
    p.add_argument("--kernel", choices=["gauss", "roma"], default="gauss",
                   help="force regularisation of the single-rotor workload: the Gaussian (eps = 2) or Roma's "
                        "three-point delta")
    args = p.parse_args()
    if args.inplace and args.workload not in ("periodic", "single"):
        p.error("--inplace applies to --workload periodic and single")
    if args.inplace and (args.steps % 2 or args.warmup % 2):
        p.error("--inplace needs even --steps and --warmup (the state is read at even step counts)")
    if args.kernel != "gauss" and args.workload != "single":
        p.error("--kernel applies to --workload single")
    return args


def tile_label(tile):
    """'XxYxZ' of a (tile_x, tile_y, tile_z, form) tuple, with ' staged' for rows
    staged in shared memory and ' single' for one cell per thread where the
    bulk kernel would pair cells."""
    return "x".join(str(v) for v in tile[:3]) + {0: "", 1: " staged", 2: " single"}.get(int(tile[3]), "")


def dist_info():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def reduce_max(values, dist=None, device="cpu"):
    """The maximum over ranks of each value (every rank receives it): the job's
    time is the slowest rank's."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def job_mlups(world, cells, steps, elapsed_ms):
    """Whole-job throughput of `world` replicas, each advancing `cells` cells by
    `steps` steps, in the slowest rank's time."""
    return world * cells * steps / (elapsed_ms * 1e-3) / 1e6


# DRAM bytes per time step (dram__bytes_read.sum + dram__bytes_write.sum over
# the step's three launches: the rotor tiles, the actuator line and the rest)
# of the single-rotor workload at the tiles the tuner picks from, each from one
# ncu capture of one step of
# `bench.py --steps 8 --warmup 4 --storage <fp32|bf16> --tile <tile> --no-e2e
# --no-cpu-baseline --no-bf16` (-k regex:"k_step|k_bulk|k_alm" -s 10 -c 3), keyed
# by (workload, storage, collision, tile).  The in-place periodic lattice's entry
# is the mean of an odd and an even step (one launch each) of
# `bench.py --workload periodic --inplace --storage bf16 --steps 8 --warmup 4
# --tile 32x8x1 --no-e2e --no-cpu-baseline` (-k regex:k_step_aa -s 6 -c 2).
# They hold for the kernel source whose comment-free SHA-256 is recorded and are
# reported as null once the code changes.
NCU_TRAFFIC = {
    "kernel_sha256": "6ebab0dd9a536cc2e9684873cb7fb185ede20d11c30b304df7945fa70312fa5f",
    "bytes": {
        ("single_turbine_256x128x128", "fp32", "cumulant", "32x4x1"): 464981504 + 385692416,
        ("single_turbine_256x128x128", "fp32", "cumulant", "32x8x1"): 464846080 + 386084096,
        ("single_turbine_256x128x128", "fp32", "cumulant", "64x1x1"): 460046080 + 370189056,
        ("single_turbine_256x128x128", "fp32", "cumulant", "64x2x1"): 459883264 + 369536000,
        ("single_turbine_256x128x128", "fp32", "cumulant", "32x2x1"): 465237760 + 385448704,
        ("single_turbine_256x128x128", "fp32", "cumulant", "64x4x1"): 459782912 + 369896704,
        ("single_turbine_256x128x128", "fp32", "cumulant", "128x1x1"): 459787520 + 369744640,
        ("single_turbine_256x128x128", "fp32", "cumulant", "128x2x1"): 459758080 + 369656320,
        ("single_turbine_256x128x128", "bf16", "cumulant", "32x4x1"): 243667968 + 176583168,
        ("single_turbine_256x128x128", "bf16", "cumulant", "32x8x1"): 243569920 + 176768512,
        ("single_turbine_256x128x128", "bf16", "cumulant", "64x1x1"): 236081152 + 163854848,
        ("single_turbine_256x128x128", "bf16", "cumulant", "64x2x1"): 236033536 + 163473408,
        ("single_turbine_256x128x128", "bf16", "cumulant", "32x2x1"): 243940864 + 176277248,
        ("single_turbine_256x128x128", "bf16", "cumulant", "64x4x1"): 235862016 + 163803904,
        ("single_turbine_256x128x128", "bf16", "cumulant", "128x1x1"): 235836416 + 163271168,
        ("single_turbine_256x128x128", "bf16", "cumulant", "128x2x1"): 235859456 + 162748160,
        ("periodic_256x128x128_inplace", "bf16", "cumulant", "32x8x1"): 226669440 + 169525376,
    },
}


def strip_c_comments(src):
    """C/C++ source with its // and /* */ comments removed (string and
    character literals kept), trailing blanks dropped and blank lines removed:
    what the compiler sees, so that a comment edit keeps the hash."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            out.append(" ")
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    lines = (l.rstrip() for l in "".join(out).split("\n"))
    return "\n".join(l for l in lines if l)


def kernel_source_sha256():
    """SHA-256 of the step kernel's source (lbm_kernels.cu + lbm_internal.h)
    without comments."""
    h = hashlib.sha256()
    for f in ("lbm_kernels.cu", "lbm_internal.h"):
        with open(os.path.join(ROOT, "paper_2402_13171_gb300", "csrc", f), encoding="utf-8") as fp:
            h.update(strip_c_comments(fp.read()).encode())
    return h.hexdigest()


def measured_traffic(workload, storage, collision, tile):
    if NCU_TRAFFIC["kernel_sha256"] != kernel_source_sha256():
        return None
    return NCU_TRAFFIC["bytes"].get((workload, storage, collision, tile))


def bytes_per_cell_update(q=27, force_components=0, elem_bytes=4):
    """Algorithmic bytes of one cell update: q loads and q stores of the
    storage type, plus a dense force field if one is read (Sec. 4.3 counts 3
    components; the fused gather here reads none)."""
    return (2 * q + force_components) * elem_bytes


def max_mlups(bandwidth_gbs, bytes_per_cell):
    """Bandwidth-bound ceiling of the update rate, P_max = b_S / n_b (Sec. 4.3)."""
    return bandwidth_gbs * 1e9 / bytes_per_cell / 1e6


def lightspeed(bandwidth_gbs, flops_per_cell, peak_gflops, bytes_per_cell):
    """l = min(1, B_m / B_c) with machine balance b_S / P_peak and code balance
    n_b / n_f (Sec. 4.3): below 1 the kernel is bandwidth-bound."""
    return min(1.0, bandwidth_gbs * flops_per_cell / (peak_gflops * bytes_per_cell))


def achieved_gbs(bytes_per_cell, cells, seconds):
    return bytes_per_cell * cells / seconds / 1e9


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        import tempfile
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"lbm_bench_clocks_{os.getpid()}_{index}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        with open(self.path) as f:
            return self.summarise(f)

    @staticmethod
    def summarise(lines):
        """Median SM clock, maximum clock and the throttle reasons seen in
        nvidia-smi CSV lines of the query Q (malformed lines are skipped)."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample_run(steps_hint, budget_s):
    """The FP64 oracle on the host cores: full rotor + inflow setup of the
    workload, stream-collide restricted to a slab of z planes through the rotor
    (a bounded sample).  Returns (seconds per step, cells per step, threads)."""
    import oracle as O
    from paper_2402_13171_gb300 import inputs as I

    dom, turb = I.single_turbine_case()
    d = O.make_domain(dom["nx"], dom["ny"], dom["nz"], collision=dom["collision"], nu=dom["nu"], bc=dom["bc"],
                      u_ref=dom["u_ref"], noise_rel=dom["noise_rel"], seed=dom["seed"])
    s = O.Sim(d, [O.TurbineSpec(**turb)])
    s.init_fields()
    planes = 8
    z0 = 56
    t = time.perf_counter()
    s.step_planes(z0, z0 + planes)
    per_plane = (time.perf_counter() - t) / planes
    planes = int(max(1, min(64, budget_s / max(1, steps_hint) / per_plane)))
    return s, z0, planes, dom["nx"] * dom["ny"] * planes, O.num_threads()


def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    s, z0, planes, cells, threads = oracle_sample_run(args.steps + args.warmup, 150.0)
    for _ in range(args.warmup):
        s.step_planes(z0, z0 + planes)
    t = time.perf_counter()
    for _ in range(args.steps):
        s.step_planes(z0, z0 + planes)
    dt = time.perf_counter() - t
    value = cells * args.steps / dt / 1e6
    sample = (f"FP64 C oracle, OpenMP; each step: blade kinematics, sampling, forces and Gaussian spreading of the "
              f"full rotor, then pull + cumulant collision on z planes [{z0}, {z0 + planes}) of the "
              f"256x128x128 lattice ({cells} cells)")
    line = {
        "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "collision": "cumulant", "sample_cells_per_step": cells},
        "impl": "reference",
        "cpu_baseline": {"value": value, "unit": "MLUPS", "cores": threads, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def accuracy_check(storage="fp32"):
    """Part of the CPU-baseline leg: scaled-down rotor case (48x32x32, D = 12,
    3 x 6 elements), 50 steps: max |u_gpu - u_oracle| (GPU in the given storage
    vs the FP64 oracle)."""
    import numpy as np
    import oracle as O
    from paper_2402_13171_gb300 import inputs as I
    from paper_2402_13171_gb300 import lbm

    dom, turb = I.single_turbine_case(48, 32, 32, diameter=12.0, elements_per_blade=6, seed=11)
    g = lbm.Lattice.create(dom["nx"], dom["ny"], dom["nz"], nu=dom["nu"], bc=dom["bc"], seed=dom["seed"],
                           storage=storage)
    g.set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
    g.add_turbine(**turb)
    g.step(50)
    _, ug = g.moments()
    d = O.make_domain(dom["nx"], dom["ny"], dom["nz"], nu=dom["nu"], bc=dom["bc"], u_ref=dom["u_ref"],
                      noise_rel=dom["noise_rel"], seed=dom["seed"])
    s = O.Sim(d, [O.TurbineSpec(**turb)])
    s.init_fields()
    s.step(50)
    _, uo = s.moments()
    g.destroy()
    return float(np.abs(ug - uo).max())


def run_ours(args):
    import numpy as np
    import torch

    from paper_2402_13171_gb300 import build as B
    from paper_2402_13171_gb300 import inputs as I
    from paper_2402_13171_gb300 import lbm

    rank, world, local = dist_info()
    B.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    tile = (0, 0, 0, 0) if args.tile == "auto" else tuple(int(v) for v in args.tile.split("x"))
    if args.workload == "single":
        dom, turb = I.single_turbine_case(kernel=args.kernel)
        dom["collision"] = args.collision
        lat = lbm.Lattice.create(dom["nx"], dom["ny"], dom["nz"], device=local, collision=args.collision,
                                 nu=dom["nu"], smag_c=dom["smag_c"], storage=args.storage, bc=dom["bc"],
                                 seed=dom["seed"], tile=tile, diag_every=DIAG_EVERY, inplace=args.inplace)
        lat.set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
        lat.add_turbine(**turb)
        lattices = [lat]
        workload = (WORKLOAD if args.kernel == "gauss" else WORKLOAD + "_roma") + ("_inplace" if args.inplace else "")
        extra = {"rotor": "3 blades x 40 elements, D=32 at (64,64,64), TSR 6, "
                          + ("Gaussian eps=2" if args.kernel == "gauss" else "Roma 3-point delta")}
    elif args.workload == "periodic":
        nx, ny, nz = 256, 128, 128
        lat = lbm.Lattice.create(nx, ny, nz, device=local, collision=args.collision, nu=1e-3, smag_c=0.1,
                                 storage=args.storage, bc=("periodic",) * 3, tile=tile, diag_every=DIAG_EVERY,
                                 inplace=args.inplace)
        rho0, u0, fneq0 = I.random_state(nx, ny, nz, seed=I.DEFAULT_SEED + 9, u_mean=(0.05, 0.0, 0.0), du=0.01,
                                         drho=0.005, fneq_amp=2e-4)
        lat.init_fields(rho0, u0, fneq0)
        del rho0, u0, fneq0
        lattices = [lat]
        workload = "periodic_256x128x128" + ("_inplace" if args.inplace else "")
        extra = {"scheme": "AA pattern, one PDF array" if args.inplace else "pull, two PDF arrays",
                 "pdf_bytes": 27 * nx * ny * nz * {"fp32": 4, "bf16": 2, "fp16": 2}[args.storage]
                 * (1 if args.inplace else 2)}
    else:
        cases = I.batch_instances(16)
        cfgs = [dict(nx=d["nx"], ny=d["ny"], nz=d["nz"], collision=args.collision, nu=d["nu"], smag_c=d["smag_c"],
                     storage=args.storage, bc=d["bc"], seed=d["seed"], tile=tile, diag_every=DIAG_EVERY)
                for d, _ in cases]
        lattices = lbm.batch_create(cfgs, device=local)
        for L, (d, t) in zip(lattices, cases):
            L.set_inflow(u_ref=d["u_ref"], noise_rel=d["noise_rel"])
            L.add_turbine(**t)
        lat = lattices[0]
        workload = "batch16_single_turbine_lattices"
        extra = {"lattices": [f"{d['nx']}x{d['ny']}x{d['nz']}" for d, _ in cases],
                 "rotor_diameters": [round(2 * t["radius"], 2) for _, t in cases]}
    if args.tile == "auto":
        cache = os.path.join(ROOT, "paper_2402_13171_gb300", "_build", "tune_cache.txt")
        lat.autotune(steps=20, cache=cache)
    tx_, ty_, tz_, st_ = lat.tile()
    tile_used = tile_label(lat.tile())
    bytes_per_cell, cells = lat.traffic_model()
    lat.step(args.warmup)
    lat.sync()
    launches_per_step = lat.launches_per_step()

    # ---- timed region: K steps, CUDA events on the launch stream, per-replay events inside
    clocks = ClockSampler(local)
    lat.set_profiling(True)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    clocks.start()
    time.sleep(0.3)
    e0.record(lat.stream)
    lat.step(args.steps)
    e1.record(lat.stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    lat.sync()
    elapsed_ms = e0.elapsed_time(e1)
    kernel_ms, timed_steps = lat.kernel_time()
    lat.set_profiling(False)
    elapsed_ms, kernel_ms = reduce_max([elapsed_ms, kernel_ms], dist, device="cuda")
    value = job_mlups(world, cells, args.steps, elapsed_ms)
    peak, peak_kind = load_peaks()
    achieved = achieved_gbs(bytes_per_cell, cells, kernel_ms * 1e-3)
    thrust, torque = lat.loads(0) if lat.turbines else (None, None)
    diag_sums, diag_step = lat.diagnostics()

    # ---- end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e and args.workload == "single":
        N = cells
        rho_h = torch.ones(N, dtype=torch.float64).pin_memory().numpy()
        u_h = torch.zeros(3 * N, dtype=torch.float64).pin_memory().numpy()
        u_h[:N] = dom["u_ref"][0]
        # each step's loads are written by the device straight into page-locked
        # memory (no copy on the stream) and read one step behind, so the host
        # never waits on the step it has just enqueued
        rho_o = torch.empty(N, dtype=torch.float64).pin_memory().numpy()
        u_o = torch.empty(3 * N, dtype=torch.float64).pin_memory().numpy()
        ring = torch.zeros((4, 1, 2), dtype=torch.float64).pin_memory()
        ring_np = ring.numpy()
        evs = [torch.cuda.Event(), torch.cuda.Event()]

        def e2e_pass(k):
            lat.init_fields(rho_h, u_h)
            lat.set_loads_sink(ring)
            s0 = lat.step_count()
            loads = None
            for i in range(k):
                lat.step(1)
                evs[i % 2].record(lat.stream)
                if i > 0:
                    evs[(i - 1) % 2].synchronize()
                    loads = ring_np[(s0 + i) % 4, 0].tolist()
            evs[(k - 1) % 2].synchronize()
            loads = ring_np[(s0 + k) % 4, 0].tolist()
            lat.moments(rho_o, u_o)
            return loads

        e2e_pass(min(args.warmup, args.steps))   # untimed: first-use staging allocations
        barrier()
        t = time.perf_counter()
        last_loads = e2e_pass(args.steps)
        barrier()
        dt = time.perf_counter() - t
        dt = reduce_max([dt], dist, device="cuda")[0]
        e2e = {"value": job_mlups(world, cells, args.steps, dt * 1e3), "unit": "MLUPS",
               "h2d_bytes_per_step": 32.0 * N / args.steps,
               "d2h_bytes_per_step": 16.0 + 32.0 * N / args.steps,
               "api": "lbm_init_fields(page-locked FP64 rho, u) + alm_set_loads_sink(page-locked ring) + K x "
                      "(lbm_step(1), read that step's thrust and torque from the ring one step behind) + "
                      "lbm_get_moments(into page-locked FP64 rho, u); after one untimed pass of the same calls",
               "last_loads": last_loads}

    # the same workload with BF16 offset storage (the precision pattern's
    # halved bytes), timed the same way on its own lattice
    bf16 = None
    if args.workload == "single" and args.storage == "fp32" and not args.inplace and not args.no_bf16:
        lat.destroy()
        lattices = []
        lb = lbm.Lattice.create(dom["nx"], dom["ny"], dom["nz"], device=local, collision=args.collision,
                                nu=dom["nu"], smag_c=dom["smag_c"], storage="bf16", bc=dom["bc"], seed=dom["seed"],
                                tile=tile, diag_every=DIAG_EVERY)
        lb.set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
        lb.add_turbine(**turb)
        if args.tile == "auto":
            lb.autotune(steps=20, cache=os.path.join(ROOT, "paper_2402_13171_gb300", "_build", "tune_cache.txt"))
        bpc16, _ = lb.traffic_model()
        lb.step(args.warmup)
        lb.sync()
        lb.set_profiling(True)
        barrier()
        e0.record(lb.stream)
        lb.step(args.steps)
        e1.record(lb.stream)
        torch.cuda.synchronize()
        lb.sync()
        ms16 = e0.elapsed_time(e1)
        k16, _ = lb.kernel_time()
        ms16, k16 = reduce_max([ms16, k16], dist, device="cuda")
        ach16 = achieved_gbs(bpc16, cells, k16 * 1e-3)
        tile16 = tile_label(lb.tile())
        bf16 = {"value": job_mlups(world, cells, args.steps, ms16), "unit": "MLUPS", "ms_per_step": ms16 / args.steps,
                "tile": tile16,
                "roofline": {"bound": "hbm", "achieved": ach16, "peak": peak, "unit": "GB/s", "frac": ach16 / peak,
                             "traffic": measured_traffic(workload, "bf16", args.collision, tile16),
                             "bytes_per_cell": bpc16, "kernel_ms": k16}}
        lb.destroy()

    acc = None
    cpu = None
    if rank == 0 and world == 1 and args.workload == "single" and not args.no_cpu_baseline:
        # the CPU-baseline leg: the oracle timed on the host cores, and the
        # accuracy of the GPU path against it on a scaled-down rotor case
        acc = accuracy_check()
        if bf16 is not None:
            bf16["max_du_vs_fp64_oracle"] = accuracy_check("bf16")
            bf16["accuracy_case"] = "48x32x32 rotor, 50 steps"
        if True:
            s, z0, planes, ccells, threads = oracle_sample_run(30, 20.0)
            nst = 5
            t = time.perf_counter()
            for _ in range(nst):
                s.step_planes(z0, z0 + planes)
            dt = time.perf_counter() - t
            cpu = {"value": ccells * nst / dt / 1e6, "unit": "MLUPS", "cores": threads, "kind": "oracle",
                   "sample": f"FP64 C oracle, {nst} steps of the full rotor + pull/cumulant collision on z planes "
                             f"[{z0}, {z0 + planes}) of the 256x128x128 lattice ({ccells} cells per step)"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": elapsed_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": workload, "cells": cells, "storage": args.storage, "collision": args.collision,
                       **extra,
                       "tile": tile_used, "tuned": args.tile == "auto", "diag_every": DIAG_EVERY,
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": f"no flush: PDF arrays {2 * bytes_per_cell / 2 * cells / 1e6:.0f} MB > 129 MB L2"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak,
                         "traffic": measured_traffic(workload, args.storage, args.collision, tile_used),
                         "kernel": "one time step: rotor tiles (k_step), actuator line (k_alm), fused "
                                   "stream-collide of the rest (k_bulk, k_bulk2 with 16-bit storage)",
                         "bytes_per_cell": bytes_per_cell, "kernel_ms": kernel_ms, "peak_kind": peak_kind},
            "e2e": e2e,
            "gpu_launches": args.steps * launches_per_step,
            "clocks": clk,
            "cpu_baseline": cpu,
            "accuracy": {"max_du_vs_fp64_oracle": acc, "case": "48x32x32 rotor, 50 steps"} if acc is not None else None,
            "loads": {"thrust": thrust, "torque": torque},
            "diagnostics": {"step": diag_step, "sum_drho": diag_sums[0], "momentum": list(diag_sums[1:])},
            "bf16": bf16,
            "paper_context": PAPER_CONTEXT,
        }
        print(json.dumps(line), flush=True)
    for L in lattices:
        L.destroy()
    if dist is not None:
        dist.destroy_process_group()


def run_precision(args):
    """The single rotor scaled to 512x256x256 (D = 64 at (128, 128, 128), 80
    elements per blade): the same seeded run with PDFs stored in FP32, BF16 and
    FP16.  Mean u_x/U profiles along y through the hub at 2D, 4D and 5D
    downstream (the farthest station at least 1D before the outlet; 8D does not
    fit), averaged over the last 40 % of the steps.  Errors of the 16-bit runs
    are L_inf and L2 (RMS) of the profile differences against FP32."""
    import numpy as np
    import torch

    from paper_2402_13171_gb300 import build as B
    from paper_2402_13171_gb300 import inputs as I
    from paper_2402_13171_gb300 import lbm

    B.build()
    torch.cuda.set_device(0)
    nx, ny, nz = 512, 256, 256
    D = 64.0
    hub = (128.0, 128.0, 128.0)
    stations = {"2D": 256, "4D": 384, "5D": 448}
    steps = args.steps
    avg_from = int(0.6 * steps)
    every = 20
    ys = np.arange(ny)
    px = np.concatenate([np.full(ny, x) for x in stations.values()])
    py = np.concatenate([ys] * len(stations))
    pz = np.full(px.size, int(hub[2]))
    out = {}
    # "fp32_twin": the FP32 run with the inflow noise drawn from another seed --
    # past the chaotic horizon its mean wake differs from the first FP32 run's by
    # the statistical floor of the comparison, which a storage error must exceed
    # to be seen
    for storage in ("fp32", "fp32_twin", "bf16", "fp16"):
        dom, turb = I.single_turbine_case(nx, ny, nz, diameter=D, hub=hub, elements_per_blade=80)
        seed = dom["seed"] + (1 if storage == "fp32_twin" else 0)
        lat = lbm.Lattice.create(nx, ny, nz, nu=dom["nu"], storage=storage.split("_")[0], bc=dom["bc"], seed=seed)
        lat.set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
        lat.add_turbine(**turb)
        lat.autotune(steps=10, cache=os.path.join(ROOT, "paper_2402_13171_gb300", "_build", "tune_cache.txt"))
        bpc, cells = lat.traffic_model()
        acc = np.zeros((px.size, 3))
        nsamp = 0
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        timed_ms = 0.0
        timed_steps = 0
        done = 0
        while done < steps:
            n = min(every, steps - done)
            e0.record(lat.stream)
            lat.step(n)
            e1.record(lat.stream)
            e1.synchronize()
            timed_ms += e0.elapsed_time(e1)
            timed_steps += n
            done += n
            if done >= avg_from:
                _, u = lat.probe(px, py, pz)
                acc += u
                nsamp += 1
        mean = acc / max(nsamp, 1) / dom["u_ref"][0]
        mlups = cells * timed_steps / (timed_ms * 1e-3) / 1e6
        out[storage] = {"mean_ux": mean[:, 0], "mlups": mlups,
                        "hbm_frac": bpc * cells * timed_steps / (timed_ms * 1e-3) / 1e9 / load_peaks()[0],
                        "tile": tile_label(lat.tile())}
        lat.destroy()
    errors = {}
    for storage in ("fp32_twin", "bf16", "fp16"):
        errors[storage] = {}
        for k, name in enumerate(stations):
            sl = slice(k * ny, (k + 1) * ny)
            d = out[storage]["mean_ux"][sl] - out["fp32"]["mean_ux"][sl]
            errors[storage][name] = {"linf": float(np.abs(d).max()), "l2": float(np.sqrt(np.mean(d ** 2)))}
    # storage errors as multiples of the FP32-vs-FP32 floor (1 = not separable from chaos)
    vs_floor = {st: {name: {m: errors[st][name][m] / max(errors["fp32_twin"][name][m], 1e-30) for m in ("linf", "l2")}
                     for name in stations} for st in ("bf16", "fp16")}
    crop = precision_crop_vs_oracle(args) if not args.no_cpu_baseline else None
    deficit = {name: float(1.0 - out["fp32"]["mean_ux"][k * ny:(k + 1) * ny].min()) for k, name in enumerate(stations)}
    line = {
        "metric": METRIC, "value": out["fp32"]["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": steps, "warmup": 0,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "precision_512x256x256", "cells": nx * ny * nz, "rotor": "D=64 at (128,128,128), "
                   "3 x 80 elements, eps=2, TSR 6", "average": f"steps {avg_from}..{steps}, every {every}"},
        "runs": {k: {"mlups": v["mlups"], "hbm_frac": v["hbm_frac"], "tile": v["tile"]} for k, v in out.items()},
        "max_wake_deficit_fp32": deficit,
        "profile_error_vs_fp32": errors,
        "profile_error_over_fp32_floor": vs_floor,
        "crop_128_vs_fp64_oracle": crop,
    }
    print(json.dumps(line), flush=True)


def precision_crop_vs_oracle(args, checkpoints=(40, 200, 1000)):
    """Before the flow turns chaotic the storage error is measured directly: the
    workload's rotor (D = 32, hub (32, 64, 64)) in a 128^3 inlet/outlet lattice,
    FP32, BF16 and FP16 storage against the FP64 oracle after 40, 200 and 1000
    steps (max and RMS |u - u_oracle| over the whole field, lattice units)."""
    import numpy as np

    import oracle as O
    from paper_2402_13171_gb300 import inputs as I
    from paper_2402_13171_gb300 import lbm

    O.build()
    dom, turb = I.single_turbine_case(128, 128, 128, diameter=32.0, hub=(32.0, 64.0, 64.0))
    d = O.make_domain(128, 128, 128, nu=dom["nu"], bc=dom["bc"], u_ref=dom["u_ref"], noise_rel=dom["noise_rel"],
                      seed=dom["seed"])
    sim = O.Sim(d, [O.TurbineSpec(**turb)])
    sim.init_fields()
    ref = {}
    t0 = time.perf_counter()
    for n in checkpoints:
        sim.step(n - sim.step_count)
        ref[n] = sim.moments()[1]
    oracle_s = time.perf_counter() - t0
    res = {"oracle_seconds": oracle_s, "threads": O.num_threads()}
    for storage in ("fp32", "bf16", "fp16"):
        g = lbm.Lattice.create(128, 128, 128, nu=dom["nu"], storage=storage, bc=dom["bc"], seed=dom["seed"])
        g.set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
        g.add_turbine(**turb)
        res[storage] = {}
        for n in checkpoints:
            g.step(n - g.step_count())
            du = np.abs(g.moments()[1] - ref[n])
            res[storage][str(n)] = {"max": float(du.max()), "rms": float(np.sqrt(np.mean(du ** 2)))}
        g.destroy()
    return res


def run_warmstart(args):
    """Learned warm start on the 3x3 farm: 1024x384x192 cells, rotors D = 48
    in rows x = 96, 336, 576 and columns y = 48, 192, 336 at hub height 96,
    seeded yaw in [0, 10] degrees, TSR 6; log-law inflow
    u(z) = 0.05 ln(z_c/0.1)/ln(96/0.1) with 1 % noise, free-slip top and
    bottom, periodic y.  The surrogate (6 -> 4 x 128 GELU -> 3, BF16 weights)
    is trained on the mean wakes of 64 single-rotor runs of this solver.  The
    farm runs --steps steps from the inflow profile (cold) and from the
    surrogate's superposed wakes (warm); the second halves of both give the
    converged mean of hub-plane u_x and its noise floor (median distance of a
    1000-step window mean to it); each run settles at its first window within
    k times the noise floor, k = 2, 3, 4."""
    import numpy as np
    import torch

    from paper_2402_13171_gb300 import build as B
    from paper_2402_13171_gb300 import inputs as I
    from paper_2402_13171_gb300 import lbm
    from paper_2402_13171_gb300 import surrogate as S

    B.build()
    torch.cuda.set_device(0)
    t = time.perf_counter()
    # training data: 64 runs shaped like the single-rotor workload (256x128x128,
    # D = 32 at (64, 64, 64)), wakes developed over one flow-through time
    X, T, runs = S.generate_wake_data(64, seed=31, shape=(256, 128, 128), D=32.0, spinup=6000, average=4000, every=40)
    t_data = time.perf_counter() - t
    net = S.WakeMLP(seed=4)
    net.set_data(X, T)
    t = time.perf_counter()
    loss = net.train(3000, batch=4096, lr=1e-3, seed=9)
    t_train = time.perf_counter() - t
    nx, ny, nz, D = 1024, 384, 192, 48.0
    rng = np.random.default_rng(2402131715)
    zc = np.arange(nz) + 0.5
    Uz = 0.05 * np.log(zc / 0.1) / np.log(96.0 / 0.1)
    u_hub = float(0.05 * np.log(96.5 / 0.1) / np.log(96.0 / 0.1))
    rotors = [dict(hub=(float(x), float(y), 96.0), D=D, tsr=6.0, yaw=float(np.radians(rng.uniform(0, 10))),
                   u_hub=u_hub) for x in (96, 336, 576) for y in (48, 192, 336)]
    cache = os.path.join(ROOT, "paper_2402_13171_gb300", "_build", "tune_cache.txt")
    result = {}
    wms = {}
    for mode in ("cold", "warm"):
        lat = lbm.Lattice.create(nx, ny, nz, nu=1e-3, bc=("inout", "periodic", "freeslip"), seed=2402131715)
        lat.set_inflow(u_ref=(0.05, 0.0, 0.0), kind=1, z0=0.1, z_ref=96.0, noise_rel=0.01)
        for r in rotors:
            lat.add_turbine(**I.single_turbine(nx, ny, nz, diameter=D, hub=r["hub"], elements_per_blade=40,
                                               tsr=r["tsr"], u_inf=u_hub, yaw=r["yaw"]))
        lat.autotune(steps=5, cache=cache)
        t = time.perf_counter()
        if mode == "warm":
            u0 = S.farm_initial_velocity(net, (nx, ny, nz), rotors, Uz, stride=4)
            lat.init_fields(None, u0, None)
            del u0
        t_init = time.perf_counter() - t
        wm = S.WindowMeans(lat, z=96, every=50, window=1000)
        t = time.perf_counter()
        wm.advance(args.steps)
        t_run = time.perf_counter() - t
        wms[mode] = wm
        result[mode] = {"steps_run": args.steps, "run_s": t_run, "init_s": t_init,
                        "mlups": nx * ny * nz * args.steps / t_run / 1e6}
        lat.destroy()
    ref, noise = S.converged_reference([wms["cold"], wms["warm"]], args.steps // 2)
    for mode in ("cold", "warm"):
        result[mode]["settled_at_step"] = {f"{k}x_noise": S.settle_step(wms[mode], ref, k * noise) for k in (2, 3, 4)}
        result[mode]["window_errors"] = [round(e, 4) for e in S.window_errors(wms[mode], ref)]
        # the workload's criterion: running mean changes by < 1e-3 (relative L2) over 1000 steps
        result[mode]["running_mean_converged_at_step"] = {
            str(tol): S.running_mean_settle_step(wms[mode], tol) for tol in (1e-3, 2e-3, 5e-3)}
        result[mode]["running_mean_changes"] = [(e, round(c, 6)) for e, c in S.running_mean_changes(wms[mode])]
    line = {
        "metric": METRIC, "value": result["cold"]["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
        "warmup": 0, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "warmstart_farm_1024x384x192", "rotors": 9, "D": D, "inflow": "log law, 1% noise",
                   "criterion": "first 1000-step window mean of hub-plane u_x within k x the noise floor "
                                "(relative L2) of the converged mean (second halves of both runs), k = 2, 3, 4; "
                                "and the workload's own: relative L2 change of the running mean of hub-plane u_x "
                                "over 1000 steps below 1e-3 (also 2e-3, 5e-3)",
                   "training_runs": "64 x 256x128x128, D = 32, TSR 4-8, yaw 0-10 deg, U 0.03-0.06, "
                                    "6000 steps spin-up + 4000 averaged",
                   "noise_floor": noise},
        "surrogate": {"params": net.n_params, "train_samples": int(X.shape[0]), "final_mse": loss,
                      "data_s": t_data, "train_s": t_train, "runs": len(runs)},
        "cold": result["cold"], "warm": result["warm"],
    }
    net.destroy()
    print(json.dumps(line), flush=True)


# The paper's own single-device figures (Sec. 4, table of estimated and measured
# kernel performance; FP32, 64 cells per rotor diameter, NewMexico rotor):
# context from other hardware, not a target.
PAPER_CONTEXT = {
    "NVIDIA A100-SXM-80GB": {"mlups_with_turbine": 1677.0, "mlups_without": 1866.5, "stream_copy_gbs": 1713.0,
                             "fraction_of_bandwidth_bound": 0.223, "bytes_per_cell": 228},
    "AMD EPYC 7763 (64 cores)": {"mlups_with_turbine": 202.1, "mlups_without": 204.0, "stream_copy_gbs": 105.2,
                                 "fraction_of_bandwidth_bound": 0.438, "bytes_per_cell": 228},
}

# The tuner's candidates (tile_x, tile_y, tile_z, load mode), as in lbm_autotune.
TILE_CANDIDATES = [(32, 4, 1, 0), (32, 2, 1, 0), (32, 8, 1, 0), (64, 2, 1, 0), (64, 1, 1, 0), (128, 1, 1, 0),
                   (32, 4, 2, 0), (32, 4, 4, 0), (32, 2, 4, 0), (32, 2, 8, 0), (64, 2, 4, 0), (32, 4, 8, 0),
                   (64, 1, 1, 1), (128, 1, 1, 1), (256, 1, 1, 1)]


def run_tilesweep(args):
    """The single-rotor workload at every tile candidate of the tuner: the
    device time per step (CUDA events over --steps steps after --warmup) and
    its fraction of the HBM roofline.  CUDA events only: DRAM bytes are taken
    by a separate capture of one step at one tile (`bench.py --tile ...` under
    ncu with -c 2)."""
    import torch

    from paper_2402_13171_gb300 import build as B
    from paper_2402_13171_gb300 import inputs as I
    from paper_2402_13171_gb300 import lbm

    B.build()
    torch.cuda.set_device(0)
    peak, peak_kind = load_peaks()
    rows = []
    for tile in TILE_CANDIDATES:
        dom, turb = I.single_turbine_case()
        lat = lbm.Lattice.create(dom["nx"], dom["ny"], dom["nz"], nu=dom["nu"], storage=args.storage, bc=dom["bc"],
                                 seed=dom["seed"], tile=tile, diag_every=DIAG_EVERY)
        lat.set_inflow(u_ref=dom["u_ref"], noise_rel=dom["noise_rel"])
        lat.add_turbine(**turb)
        lat.step(args.warmup)
        lat.sync()
        lat.set_profiling(True)
        lat.step(args.steps)
        lat.sync()
        ms, _ = lat.kernel_time()
        bpc, cells = lat.traffic_model()
        rows.append({"tile": tile_label(tile),
                     "kernel_ms": ms, "mlups": cells / ms / 1e3,
                     "frac": achieved_gbs(bpc, cells, ms * 1e-3) / peak})
        lat.destroy()
    best = max(rows, key=lambda r: r["mlups"])
    line = {"metric": METRIC, "value": best["mlups"], "unit": "MLUPS", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": WORKLOAD + "_tilesweep", "storage": args.storage,
                                            "peak_gbs": peak, "peak_kind": peak_kind},
            "tiles": rows}
    print(json.dumps(line), flush=True)


def main():
    args = parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "precision":
        run_precision(args)
    elif args.workload == "warmstart":
        run_warmstart(args)
    elif args.workload == "tilesweep":
        run_tilesweep(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
