#!/usr/bin/env python3
"""Throughput of the FDTD/PIC time step on one GB300 (or N replicas).

The default precision form is P32_U64 (FP32 fields with compensated
potential levels and float-float momenta, FP64 frame clock, gamma and power):
the form whose error after c2's 5000 steps stays within the stated field
(1e-4) and power (1e-3) tolerances.  P32 and P64 are timed beside it.

A step is one pass of the whole hot path over the c2 workload
(128x128x1024 cells, 2^21 macroparticles, rest-frame IR FEL shaped like the
paper's Example 1): potential update with Mur faces, E/B from the potentials,
gather + undulator + Boris push, deposit of J and rho, re-sort of the particles
into cell tiles, and the radiated-power sample.  Inputs live in HBM for the
whole run (state 0.8 GB > 129 MB L2, so no L2 flush is needed).

value  = cell-updates/s of the whole step, summed over ranks (weak scaling:
         every rank runs its own replica; the path has no exchange step);
e2e    = the same metric through the C ABI from host buffers: create (copy-in
         of the bunch), K steps, copy-out of the power record and particles.
--impl reference times the FP64 CPU oracle on the host cores instead.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("cell-updates/s + particle-pushes/s on 1 GB300 (FP32 vs FP64, % HBM roofline); "
          "jobs/h, p99")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="mithra", choices=["mithra", "reference"])
    ap.add_argument("--workload", default="c2")
    ap.add_argument("--precision", default="p32_u64", choices=["p32", "p32_u64", "p32_c", "p64"],
                    help="p32_u64 (default): FP32 fields with compensated levels and "
                         "float-float momenta, the form that meets the 1e-4 field and 1e-3 "
                         "power tolerance after the configured 5000 steps; p32: plain FP32 "
                         "state; p64: all FP64")
    ap.add_argument("--no-c3", action="store_true",
                    help="step mode: skip the c3 summary (256x256x2048 cells, 2^24 particles)")
    ap.add_argument("--c3-steps", type=int, default=60)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-p64", action="store_true")
    ap.add_argument("--mode", default="step", choices=["step", "batch", "serve", "precision"],
                    help="step: one simulation (c2); batch: 64 uneven simulations (c4); "
                         "serve: continuous batching of Poisson arrivals (c5); precision: "
                         "per-output error of the FP32 forms against P64 over the whole "
                         "grid after --steps steps (c2), with P64 checked against the "
                         "stored oracle checkpoints")
    ap.add_argument("--job-steps", type=int, default=100,
                    help="batch mode: steps timed per job (jobs of 1000 steps are scaled)")
    ap.add_argument("--plain-jobs", type=int, default=8,
                    help="batch mode: jobs run one by one in plain FP64")
    ap.add_argument("--duration", type=float, default=60.0, help="serve mode: seconds per run")
    ap.add_argument("--no-batch", action="store_true", help="step mode: skip the c4 summary")
    ap.add_argument("--no-serve", action="store_true", help="step mode: skip the c5 summary")
    ap.add_argument("--rate", type=float, default=20.0, help="serve mode: arrivals per second")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples every 200 ms while running."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid: str | None):
        self.uuid = uuid
        self.rows = []
        self.p = None
        self.t = None

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.uuid:
            cmd += ["-i", self.uuid]
        try:
            self.p = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                      text=True)
        except OSError:
            self.p = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.p.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def stop(self):
        if self.p is None:
            return
        time.sleep(0.25)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        if self.t:
            self.t.join(timeout=5)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for nm, v in zip(names, r[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "samples": len(self.rows), "reasons": sorted(reasons)}


# kernels behind one timed scope of the library's profiler: the potential
# update is the Mur boundary kernel plus the interior kernel, the re-sort scan
# two passes
KERNELS_PER_SCOPE = {"potential_step": 2, "scan_counts": 2}


PRECISIONS = {"p32": "P32", "p32_u64": "P32_U64", "p32_c": "P32_C", "p64": "P64"}

# DRAM bytes (read + write) per launch from one ncu capture (--set full, the
# c2 step in the bench's launch configuration) of the kernels as they are
# now, by (timed scope, precision, workload); a kernel changed since its
# capture must leave this table
NCU_TRAFFIC = {
    # k_mur_boundary<1, float, 1, 1> + k_potential_zloop_mur1<1, float>
    ("potential_step", "p32_u64", "c2"): 35241728 + 187392 + 725083904 + 634589184,
    # k_push_tiled<0, float, FF2, 1, 0>
    ("push", "p32_u64", "c2"): None,
    # k_mur_boundary<0, float, 1, 1> + k_potential_zloop_mur1<0, float>
    ("potential_step", "p32", "c2"): 28195072 + 39680 + 589268224 + 498427136,
    # k_push_tiled<0, float, float, 0, 0>
    ("push", "p32", "c2"): None,
}


def push_rates(kt: dict, n_particles: int, grid: dict, prec: str) -> dict | None:
    """The particle step's achieved bandwidth and deposit (atomic) rates per
    second of its CUDA-event duration: each particle deposits rho at 8
    vertices (two int32 shared-memory atomics each, hi and lo of the
    fixed-point block, in the FP32 forms) and J at 8 vertices (one FP32x4
    vector reduction in L2 each)."""
    if "push" not in kt or not kt["push"][1]:
        return None
    s = kt["push"][0] / kt["push"][1] / 1e3
    ab = algorithmic_bytes("push", grid, n_particles, prec)
    return {"avg_launch_ms": s * 1e3, "achieved_gbs": ab / s / 1e9,
            "charge_vertex_deposits_per_s": 8 * n_particles / s,
            "current_vertex_deposits_per_s": 8 * n_particles / s,
            "shared_int32_atomics_per_s": (16 * n_particles / s) if prec != "p64" else None,
            "l2_vector_reductions_per_s": (8 * n_particles / s) if prec != "p64" else None}


def algorithmic_bytes(kernel: str, grid: dict, n_particles: int, prec: str,
                      source_vertices: int | None = None) -> float:
    """Algorithmic bytes per launch (the minimum a kernel must move).
    source_vertices: the vertices whose sources the potential update reads
    (the vertices of the tiles the particle step marked; None: every
    interior vertex)."""
    r = 8 if prec == "p64" else 4                      # field and fraction values
    um = 4 if prec in ("p32", "p32_c") else 8          # momenta
    lo = prec in ("p32_c", "p32_u64")                  # compensated potential levels
    interior = (grid["nx"] - 2) * (grid["ny"] - 2) * (grid["nz"] - 2)
    if kernel == "potential_step":
        # every vertex of the grid (the interior by the update, the boundary
        # by Mur in increment form, which also reads and writes the
        # vertex's level and increment): read psi^n and the increment, write
        # psi^{n+1} and the new increment, 4 x 4 values, plus 2 x 8 bytes
        # for the bfloat16 lo parts of compensated levels; and the 4 source
        # values of every vertex of a marked tile (the zeroing stores of the
        # sources the last deposit touched are not counted)
        sv = interior if source_vertices is None else min(source_vertices, interior)
        return all_cells(grid) * (4 * 4 * r + (16 if lo else 0)) + sv * 4 * r
    if kernel == "push":
        # read the slot's position, read and write cell + 3 fractions + 3
        # momenta + original index; write key and rank
        return n_particles * (4 + 2 * (8 + 3 * r + 3 * um) + 8)
    if kernel == "slot_map":
        # the re-sort's slot map: read key, rank and offset, write the slot's
        # position
        return n_particles * 16
    if kernel == "scan_counts":
        ntiles = -(-grid["nx"] // 8) * -(-grid["ny"] // 8) * -(-grid["nz"] // 8)
        return ntiles * 12
    if kernel == "power":
        return (grid["nx"] - 2) * (grid["ny"] - 2) * 14 * 4 * r
    return 0.0


def minimum_bytes(kernel: str, grid: dict, n_particles: int, prec: str) -> float:
    """The algorithmic minimum of a three-level potential update (read
    psi^n, psi^{n-1} and the source, write psi^{n+1}: 16 words per cell,
    plus the bfloat16 lo parts of compensated levels read and written); the
    increment form's extra read and write of the increment are not in it."""
    if kernel != "potential_step":
        return algorithmic_bytes(kernel, grid, n_particles, prec)
    r = 8 if prec == "p64" else 4
    lo = prec in ("p32_c", "p32_u64")
    return all_cells(grid) * (4 * 4 * r + (16 if lo else 0))


def max_over_ranks(x: float, world: int) -> float:
    """The largest value over the ranks (the slowest replica's time); the
    reduction runs on the process group's own device (CUDA for NCCL)."""
    if world <= 1:
        return x
    import torch
    dev = "cuda" if torch.distributed.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], device=dev, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def all_cells(g: dict) -> int:
    return g["nx"] * g["ny"] * g["nz"]


def interior_cells(g: dict) -> int:
    return (g["nx"] - 2) * (g["ny"] - 2) * (g["nz"] - 2)


def source_reads(sim, g: dict) -> dict:
    """The source tiles the simulation's next potential update reads, and
    their vertices (512 a tile, at most the interior)."""
    marked, everywhere = sim.source_tiles()
    verts = interior_cells(g) if everywhere else min(512 * marked, interior_cells(g))
    return {"marked_tiles": marked, "everywhere": everywhere, "vertices": verts}


def replica_bunch(workload: dict, rank: int) -> dict:
    """Each rank runs its own replica of the workload with its own seed."""
    from paper_1612_03310_gb300 import inputs
    return inputs.make_bunch(workload["bunch_spec"], workload["seed"] + rank)


def replica_totals(world: int, ncell: int, npart: int, n_sub: int, steps: int,
                   seconds: float) -> tuple:
    """Whole-job cell-updates/s and particle-pushes/s: every rank advanced its
    own replica by `steps` steps; `seconds` is the slowest rank's time."""
    return world * ncell * steps / seconds, world * npart * n_sub * steps / seconds


def run_gpu(args, rank, world):
    import torch
    from paper_1612_03310_gb300 import inputs, mithra

    dev = torch.cuda.current_device()
    w = inputs.workload(args.workload)
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    bunch = replica_bunch(w, rank)
    n_part = bunch["x"].size
    ncell = g["nx"] * g["ny"] * g["nz"]
    prec = getattr(mithra, PRECISIONS[args.precision])
    kp = g["nz"] - 16
    stream = torch.cuda.Stream()  # a dedicated stream: events bracket exactly our work
    torch.cuda.set_stream(stream)
    K, W = args.steps, args.warmup

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    from paper_1612_03310_gb300 import autotune
    tuning = autotune.tune(g, und, bunch, prec, stream=stream.cuda_stream)  # untimed
    sim = mithra.Simulation(g, und, bunch, precision=prec, stream=stream.cuda_stream)
    sim.set_tuning(**tuning)
    sim.set_power_sampling(kp, W + 2 * K)
    sim.step(W)
    sim.sync()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid)
    sampler.start()
    time.sleep(0.3)
    # the timed region: K steps as the library runs them (pairs of steps
    # replayed from a captured CUDA graph, no per-kernel events)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    # a second timed region of K steps launched one by one with a CUDA event
    # pair around every kernel scope on the simulation's stream: the
    # per-kernel durations of the roofline
    sim.profile(True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(K)
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    sampler.stop()
    ms_events = e0.elapsed_time(e1)
    kt = sim.kernel_times()
    sim.profile(False)
    power = sim.read_power()
    parts = sim.copy_particles()
    src_reads = source_reads(sim, g)
    sim.close()
    ms = max_over_ranks(ms, world)
    rec = autotune.record(g, n_part, prec) or {}
    res = dict(ms=ms, ms_events=max_over_ranks(ms_events, world), kernel_times=kt,
               clocks=sampler.summary(), n_part=n_part, ncell=ncell,
               tuning=tuning, trials=[{k: (round(v, 4) if k == "ms" else v) for k, v in t.items()}
                                      for t in rec.get("trials", [])],
               grid=g, n_lost=parts["n_lost"], power_last=float(power[-1, 0]),
               source_reads=src_reads,
               launches=sum(n * KERNELS_PER_SCOPE.get(k, 1) for k, (_, n) in kt.items()))

    # the other precision forms on the same workload, shorter: P64 (plain
    # FP64) and P32_U64 (compensated FP32 levels, FP64 momenta: the form that
    # meets the field tolerance after the configured steps)
    def side_run(precision, steps):
        sim = mithra.Simulation(g, und, bunch, precision=precision, stream=stream.cuda_stream)
        sim.set_tuning(**autotune.tune(g, und, bunch, precision, stream=stream.cuda_stream))
        sim.set_power_sampling(kp, W + 2 * steps)
        sim.step(W)
        torch.cuda.synchronize()
        barrier()
        e0.record(stream)
        sim.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms_side = e0.elapsed_time(e1)
        sim.profile(True)           # per-kernel durations: a second region
        sim.step(steps)
        torch.cuda.synchronize()
        kts = sim.kernel_times()
        src = source_reads(sim, g)
        sim.close()
        ms_side = max_over_ranks(ms_side, world)
        return dict(ms=ms_side, steps=steps, kernel_times=kts, source_reads=src)

    if not args.no_p64 and prec != mithra.P64:
        res["p64"] = side_run(mithra.P64, max(20, K // 10))
    if not args.no_p64 and prec == mithra.P32:
        res["p32_u64"] = side_run(mithra.P32_U64, max(50, K // 4))
    if not args.no_p64 and prec == mithra.P32_U64:
        res["p32"] = side_run(mithra.P32, max(50, K // 4))

    # end to end through the C ABI from host buffers
    if not args.no_e2e:
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim = mithra.Simulation(g, und, bunch, precision=prec, stream=stream.cuda_stream)
        sim.set_tuning(**tuning)
        sim.set_power_sampling(kp, K)
        sim.step(K)
        rec = sim.read_power()
        out = sim.copy_particles()
        sim.close()
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        barrier()
        e2e_s = max_over_ranks(t1 - t0, world)
        res["e2e"] = dict(seconds=e2e_s, h2d=6 * 8 * n_part, d2h=rec.nbytes + 7 * 8 * n_part,
                          check=float(np.isfinite(out["x"]).all()))
    return res


def run_c3(args, peak: float) -> dict:
    """c3, the largest single-GPU workload (256x256x2048 cells, 2^24
    particles), in the bench's precision form: K3 steps as the library runs
    them (graph replays), then K3 more with per-kernel CUDA events for the
    roofline of its dominant kernel and of the potential update."""
    import torch
    from paper_1612_03310_gb300 import autotune, inputs, mithra
    w = inputs.workload("c3")
    g, und = dict(w["grid"], boundary=1), w["undulator"]
    bunch = inputs.make_bunch(w["bunch_spec"], w["seed"])
    n_part = bunch["x"].size
    ncell = g["nx"] * g["ny"] * g["nz"]
    prec = getattr(mithra, PRECISIONS[args.precision])
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    K3 = args.c3_steps
    tuning = autotune.tune(g, und, bunch, prec, stream=stream.cuda_stream)
    sim = mithra.Simulation(g, und, bunch, precision=prec, stream=stream.cuda_stream)
    sim.set_tuning(**tuning)
    sim.set_power_sampling(g["nz"] - 16, 5 + 2 * K3)
    sim.step(5)
    sim.sync()
    sampler = ClockSampler(None)
    sampler.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    sim.step(K3)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    sim.profile(True)
    sim.step(K3)
    sim.sync()
    sampler.stop()
    kt = sim.kernel_times()
    sim.profile(False)
    n_lost = sim.copy_particles()["n_lost"]
    src = source_reads(sim, g)
    sim.close()
    s = ms / 1e3
    dom = max(kt, key=lambda k: kt[k][0])
    dom_ms = kt[dom][0] / max(kt[dom][1], 1)
    ab = algorithmic_bytes(dom, g, n_part, args.precision, src["vertices"])
    st_ms = kt["potential_step"][0] / max(kt["potential_step"][1], 1)
    st_b = algorithmic_bytes("potential_step", g, n_part, args.precision, src["vertices"])
    total = sum(v[0] for v in kt.values())
    return {"workload": inputs.describe("c3"), "precision": args.precision, "steps": K3,
            "ms_per_step": ms / K3, "cell_updates_per_s": ncell * K3 / s,
            "particle_pushes_per_s": n_part * K3 / s,
            "roofline": {"bound": "hbm", "kernel": dom, "achieved": ab / (dom_ms / 1e3) / 1e9,
                         "peak": peak, "unit": "GB/s",
                         "frac": ab / (dom_ms / 1e3) / 1e9 / peak,
                         "algorithmic_bytes_per_launch": ab, "avg_launch_ms": dom_ms,
                         "traffic": None},
            "stencil": {"avg_launch_ms": st_ms, "achieved_gbs": st_b / (st_ms / 1e3) / 1e9,
                        "frac": st_b / (st_ms / 1e3) / 1e9 / peak,
                        "cell_updates_per_s": ncell / (st_ms / 1e3),
                        "bytes_per_cell": st_b / all_cells(g), "source_reads": src},
            "kernel_share": {k: round(v[0] / total, 4) for k, v in kt.items()},
            "tuning": tuning, "clocks": sampler.summary(), "n_lost": n_lost}


def cpu_oracle_rate(workload: str, budget_s: float, max_steps: int | None = None,
                    warmup: int = 0):
    """Times the FP64 oracle on the host cores on the same workload, as many
    whole steps as fit in budget_s (at least one, at most max_steps), after
    `warmup` untimed steps."""
    sys.path.insert(0, os.path.join(ROOT, "oracle"))
    import oracle
    from paper_1612_03310_gb300 import inputs
    oracle.build()
    w = inputs.workload(workload)
    bunch = inputs.make_bunch(w["bunch_spec"], w["seed"])
    o = oracle.OracleSim(w["grid"], w["undulator"], bunch)
    g = w["grid"]
    ncell = g["nx"] * g["ny"] * g["nz"]
    if warmup > 0:
        o.step(warmup)
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if max_steps is not None and steps >= max_steps:
            break
        if el + el / steps > budget_s:
            break
    el = time.perf_counter() - t0
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dict(cell_updates_per_s=ncell * steps / el, pushes_per_s=bunch["x"].size * steps / el,
                steps=steps, seconds=el, cores=cores,
                sample=f"{steps} whole FP64 oracle steps of {workload} "
                       f"({g['nx']}x{g['ny']}x{g['nz']} cells, {bunch['x'].size} particles); "
                       f"the particle loop is serial, the grid loops use OpenMP")


def _time_steps(stream, stepper, K: int) -> float:
    """ms per step of K steps of stepper (CUDA events on stream)."""
    import torch
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(stream)
    stepper(K)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / K


def _batch_arm(jobs, prec, mode, K, stream, kp_frac=None):
    """A batch of jobs in precision prec and batch mode ("auto", True fused,
    False per member): ms per batched step over K steps (after 4 untimed
    ones), the form the graph took, and with kp_frac each job's power record
    at plane kp_frac * nz and its final E_x."""
    from paper_1612_03310_gb300 import inputs, mithra
    sims = []
    for j in jobs:
        g = dict(j["grid"], boundary=1)
        sim = mithra.Simulation(g, j["undulator"], inputs.make_bunch(j["bunch_spec"], j["seed"]),
                                precision=prec)
        kp = int(kp_frac * g["nz"]) if kp_frac else g["nz"] - 8
        sim.set_power_sampling(kp, K + 8)
        sims.append(sim)
    b = mithra.Batch(stream=stream.cuda_stream)
    for sim in sims:
        b.add(sim)
    b.set_mode(mode)
    b.step(4)
    b.sync()
    ms = _time_steps(stream, b.step, K)
    out = dict(ms=ms, fused=b.fused())
    if kp_frac:
        out["power"] = [sim.read_power()[:, 0] for sim in sims]
        out["Ex"] = [sim.copy_field("Ex") for sim in sims]
    b.close()
    for sim in sims:
        sim.close()
    return out


def _plain_arm(jobs, prec, K, stream, kp_frac=None):
    """The same jobs one after another, each a plain simulation stepped alone:
    ms per job of K steps, and the power records and final E_x."""
    from paper_1612_03310_gb300 import inputs, mithra
    total = 0.0
    power, ex = [], []
    for j in jobs:
        g = dict(j["grid"], boundary=1)
        sim = mithra.Simulation(g, j["undulator"], inputs.make_bunch(j["bunch_spec"], j["seed"]),
                                precision=prec, stream=stream.cuda_stream)
        kp = int(kp_frac * g["nz"]) if kp_frac else g["nz"] - 8
        sim.set_power_sampling(kp, K + 8)
        sim.step(4)
        sim.sync()
        total += _time_steps(stream, sim.step, K) * K
        if kp_frac:
            power.append(sim.read_power()[:, 0])
            ex.append(sim.copy_field("Ex"))
        sim.close()
    return dict(ms_per_job=total / len(jobs), power=power, Ex=ex)


def run_batch(args, K: int | None = None, plain_jobs: int | None = None) -> dict:
    """c4: 64 design-sweep simulations of uneven size advanced together, in
    jobs/h of 1000-step jobs (K timed steps, scaled), against the same jobs
    run one after another as plain simulations (P32, to isolate what batching
    buys, and P64, the plain FP64 form).  The tolerance-meeting form P32_U64
    is timed batched as well, and its per-job power (on a plane the radiation
    reaches within the run) and E_x are compared with P64 job by job.  A
    second case, 256 tiny jobs, is where the fused batched form (one launch
    per phase for all members) pays over one launch sequence per member."""
    import torch
    from paper_1612_03310_gb300 import inputs, mithra
    jobs = inputs.batch_jobs(64, steps=1000)
    K = args.job_steps if K is None else K
    n_plain = args.plain_jobs if plain_jobs is None else plain_jobs
    scale = 1000.0 / K
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    jh = lambda ms_per_step, n: 3600.0 * n / (ms_per_step * 1000.0 / 1e3)  # noqa: E731
    auto = _batch_arm(jobs, mithra.P32, "auto", K, stream)
    fused = _batch_arm(jobs, mithra.P32, True, max(10, K // 5), stream)
    member = _batch_arm(jobs, mithra.P32, False, max(10, K // 5), stream)
    kpf = 0.8  # 0.05 nz ahead of the bunch head: radiation arrives within the run
    u64 = _batch_arm(jobs[:n_plain], mithra.P32_U64, "auto", K, stream, kp_frac=kpf)
    u64_all = _batch_arm(jobs, mithra.P32_U64, "auto", max(10, K // 5), stream)
    plain32 = _plain_arm(jobs[:n_plain], mithra.P32, K, stream)
    plain64 = _plain_arm(jobs[:n_plain], mithra.P64, K, stream, kp_frac=kpf)
    perr, ferr = [], []
    for k in range(n_plain):
        p64, p32 = plain64["power"][k], u64["power"][k]
        m = np.abs(p64).max()
        if m > 0:
            perr.append(float(np.abs(p32 - p64).max() / m))
        e64 = plain64["Ex"][k]
        ferr.append(float(np.linalg.norm(u64["Ex"][k] - e64) / np.linalg.norm(e64)))
    cells = sum(j["grid"]["nx"] * j["grid"]["ny"] * j["grid"]["nz"] for j in jobs)
    parts = sum(j["bunch_spec"]["n"] for j in jobs)
    per_job_plain64 = plain64["ms_per_job"] * scale / 1e3
    per_job_plain32 = plain32["ms_per_job"] * scale / 1e3
    # tiny jobs: 256 of 32 x 32 x 128 cells and 2000 particles
    tiny = inputs.uniform_jobs(256, 32, 128, 2000)
    t_auto = _batch_arm(tiny, mithra.P32, "auto", K, stream)
    t_member = _batch_arm(tiny, mithra.P32, False, K, stream)
    t_plain = _plain_arm(tiny[:16], mithra.P32, K, stream)
    return {"metric": "jobs/h, 64 uneven simulations of 1000 steps (c4)", "impl": "mithra",
            "mode": "batch", "value": jh(auto["ms"], len(jobs)), "unit": "jobs/h",
            "higher_is_better": True, "n_gpus": 1, "steps": K, "ms_per_step": auto["ms"],
            "form": "fused" if auto["fused"] else "per member",
            "fused_jobs_per_h": jh(fused["ms"], len(jobs)),
            "per_member_jobs_per_h": jh(member["ms"], len(jobs)),
            "plain_p32_jobs_per_h": 3600.0 / per_job_plain32,
            "plain_p64_jobs_per_h": 3600.0 / per_job_plain64,
            "speedup_vs_plain_p32": jh(auto["ms"], len(jobs)) * per_job_plain32 / 3600.0,
            "speedup_vs_plain": jh(auto["ms"], len(jobs)) * per_job_plain64 / 3600.0,
            "p32_u64_jobs_per_h": jh(u64_all["ms"], len(jobs)),
            "p32_u64_speedup_vs_plain_p64": jh(u64_all["ms"], len(jobs)) * per_job_plain64 / 3600,
            "cell_updates_per_s": cells / (auto["ms"] / 1e3),
            "particle_pushes_per_s": parts / (auto["ms"] / 1e3),
            "accuracy_p32_u64_vs_p64": {
                "power_max_rel": max(perr) if perr else None, "jobs_with_power": len(perr),
                "Ex_rel_l2_max": max(ferr), "jobs": n_plain,
                "note": f"{K} steps, power through the plane at 0.8 nz (0.05 nz ahead of the "
                        f"bunch head), the first {n_plain} jobs, batched P32_U64 against each "
                        f"job run alone in P64"},
            "tiny": {"jobs": len(tiny), "grid": "32x32x128", "particles": 2000,
                     "form": "fused" if t_auto["fused"] else "per member",
                     "jobs_per_h": jh(t_auto["ms"], len(tiny)),
                     "per_member_jobs_per_h": jh(t_member["ms"], len(tiny)),
                     "plain_p32_jobs_per_h": 3600.0 / (t_plain["ms_per_job"] * scale / 1e3)},
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"c4: 64 grids 48^2x192..128^2x768, {cells} cells, "
                                   f"{parts} particles, 64-512 particles per cell column",
                       "timed": f"{K} steps per arm (fused/per-member/all-P32_U64 arms "
                                f"{max(10, K // 5)}), jobs/h scaled to 1000 steps",
                       "plain": f"{n_plain} jobs one after another, P32 and P64"}}


def run_serve(args, duration: float | None = None) -> dict:
    """c5: Poisson arrivals of design-sweep jobs served by continuous
    batching, at the configured rate and at half of the measured capacity."""
    import torch
    from paper_1612_03310_gb300 import mithra, serve, inputs
    free, _ = torch.cuda.mem_get_info()
    budget = int(0.85 * free)
    dur = args.duration if duration is None else duration
    prec = getattr(mithra, PRECISIONS[args.precision])
    out = {}
    runs = [("rate", args.rate)]
    for name, rate in runs:
        jobs = inputs.serve_jobs(int(rate * dur) + 1, rate)
        srv = serve.Server(budget, tick_steps=64, precision=prec)
        st = srv.run(jobs, time_limit=dur)
        st.pop("done")
        st.pop("not_done", None)
        out[name] = dict(st, offered_rate=rate)
    # capacity in jobs/s: the cell updates the GPU served per second over the
    # cell updates of a mean job of the stream
    all_jobs = inputs.serve_jobs(int(args.rate * dur) + 1, args.rate)
    mean_cells = float(np.mean([j["grid"]["nx"] * j["grid"]["ny"] * j["grid"]["nz"] * j["steps"]
                                for j in all_jobs]))
    cap = out["rate"]["served_cell_updates_per_s"] / mean_cells
    half = max(0.05, 0.5 * cap)
    jobs = inputs.serve_jobs(int(half * dur) + 1, half, seed=6)
    srv = serve.Server(budget, tick_steps=64, precision=prec)
    st = srv.run(jobs, time_limit=dur + 120.0)
    st.pop("done")
    st.pop("not_done", None)
    out["half_capacity"] = dict(st, offered_rate=half)
    r = out["rate"]
    out["capacity_jobs_per_s"] = cap
    return {"metric": "jobs/h and p50/p99 latency, continuous batching (c5)", "impl": "mithra",
            "mode": "serve", "value": r["jobs_per_hour"], "unit": "jobs/h",
            "higher_is_better": True, "n_gpus": 1, "p50_s": r["p50_s"], "p99_s": r["p99_s"],
            "dtype": "f32", "data": "synthetic", "runs": out, "precision": args.precision,
            "config": {"workload": "c5: Poisson arrivals, grids 32^2x128..160^2x1024, "
                                   "1e3-4e6 particles, 500-5000 steps",
                       "duration_s": dur, "hbm_budget": budget}}


PRECISION_FIELDS = ["Ex", "Ey", "Ez", "Bx", "By", "Bz", "Ax", "Ay", "Az", "phi",
                    "Jx", "Jy", "Jz", "rho"]


def run_precision(args) -> dict:
    """Per-output error of the FP32 forms on c2 after K steps: P32, P32_C and
    P32_U64 against P64 over the whole grid (every field, relative L2), the power at
    every step, every particle.  P64 itself is held against the FP64 oracle's
    stored checkpoints (plane fields and power) at the steps they cover."""
    import glob
    from paper_1612_03310_gb300 import inputs, mithra
    w = inputs.workload(args.workload)
    g = dict(w["grid"], boundary=1)
    P = inputs.make_bunch(w["bunch_spec"], w["seed"])
    K = args.steps
    kp = g["nz"] - 16
    here = os.path.dirname(os.path.abspath(__file__))
    cks = {}
    for path in glob.glob(os.path.join(here, "tests", "golden", f"{args.workload}_reference_*.npz")):
        d = np.load(path)
        cks[int(d["steps"])] = d
    sims = {}
    for nm in ("P64", "P32", "P32_C", "P32_U64"):
        sims[nm] = mithra.Simulation(g, w["undulator"], P, precision=getattr(mithra, nm))
        sims[nm].set_power_sampling(kp, K)
    out = {"metric": f"per-output error after {K} steps, {args.workload}", "impl": "mithra",
           "mode": "precision", "steps": K, "data": "synthetic",
           "config": {"workload": inputs.describe(args.workload)}}
    oracle_check = {}
    done = 0
    for stop in sorted([s for s in cks if s <= K]) + [K]:
        if stop > done:
            for sim in sims.values():
                sim.step(stop - done)
            done = stop
        if stop in cks and stop not in oracle_check:
            d = cks[stop]
            k0 = int(d["plane_k"])
            e = {}
            for f in PRECISION_FIELDS:
                a = sims["P64"].copy_field(f)[k0]
                b = d["plane_" + f].astype(np.float64)
                e[f] = float(np.linalg.norm(a - b) / np.linalg.norm(b))
            pr = d["power"][:stop, 0]
            pg = sims["P64"].read_power()[:stop, 0]
            e["power"] = float(np.abs(pg - pr).max() / np.abs(pr).max())
            oracle_check[stop] = {k: float("%.3g" % v) for k, v in e.items()}
    ref_fields = {}
    res = {"P32": {}, "P32_C": {}, "P32_U64": {}}
    for f in PRECISION_FIELDS:
        ref = sims["P64"].copy_field(f)
        nr = float(np.linalg.norm(ref))
        for nm in res:
            a = sims[nm].copy_field(f)
            res[nm][f] = float(np.linalg.norm(a - ref) / nr) if nr > 0 else float(np.linalg.norm(a))
        ref_fields[f] = nr
    pw = sims["P64"].read_power()[:, 0]
    parts = sims["P64"].copy_particles()
    for nm in res:
        p = sims[nm].read_power()[:, 0]
        res[nm]["power"] = float(np.abs(p - pw).max() / np.abs(pw).max())
        q = sims[nm].copy_particles()
        res[nm]["position_cells"] = max(
            float(np.abs((q[k] - parts[k]) / g[dk]).max()) for k, dk in
            (("x", "dx"), ("y", "dy"), ("z", "dz")))
        us = float(np.abs(parts["uz"]).max())
        res[nm]["momentum_rel"] = max(float(np.abs(q[k] - parts[k]).max())
                                      for k in ("ux", "uy", "uz")) / us
        res[nm] = {k: float("%.3g" % v) for k, v in res[nm].items()}
        res[nm]["n_lost"] = int(q["n_lost"])
    for sim in sims.values():
        sim.close()
    out["errors_vs_p64"] = res
    out["p64_vs_oracle_checkpoints"] = oracle_check
    out["tolerances"] = {"fields": 1e-4, "power": 1e-3}
    return out


def main():
    args = parse()
    if args.mode in ("batch", "serve", "precision") and args.impl == "mithra":
        import torch
        torch.cuda.set_device(0)
        from paper_1612_03310_gb300 import build_lib
        build_lib.build()
        run = {"batch": run_batch, "serve": run_serve, "precision": run_precision}[args.mode]
        print(json.dumps(run(args)))
        return
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    from paper_1612_03310_gb300 import inputs
    w = inputs.workload(args.workload)
    g = w["grid"]
    cfg = {"workload": inputs.describe(args.workload), "grid": [g["nx"], g["ny"], g["nz"]],
           "particles": w["bunch_spec"]["n"], "precision": args.precision,
           "l2": "state 0.8 GB per replica > 129 MB L2 (no flush needed)",
           "parallelism": f"replicas x{world}"}

    if args.impl == "reference":
        if rank != 0:
            return
        os.environ.setdefault("OMP_NUM_THREADS", str(os.cpu_count() or 1))
        budget = 120.0
        # one untimed warm-up step at most (the oracle has no caches to
        # warm beyond first touch), then up to K timed steps within the budget
        wu = min(args.warmup, 1)
        r = cpu_oracle_rate(args.workload, budget, max_steps=max(args.steps, 1), warmup=wu)
        line = {"impl": "reference", "metric": METRIC, "value": r["cell_updates_per_s"],
                "unit": "cell-updates/s", "n_gpus": 0, "steps": r["steps"],
                "warmup": wu, "ms_per_step": 1e3 * r["seconds"] / r["steps"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "config": cfg,
                "particle_pushes_per_s": r["pushes_per_s"],
                "cpu_baseline": {"value": r["cell_updates_per_s"], "unit": "cell-updates/s",
                                 "cores": r["cores"], "kind": "oracle", "sample": r["sample"]},
                "e2e": {"value": r["cell_updates_per_s"], "unit": "cell-updates/s",
                        "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    import torch
    if world > 1:
        torch.cuda.set_device(local)
        torch.distributed.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    from paper_1612_03310_gb300 import build_lib
    if rank == 0:
        build_lib.build()
    if world > 1:
        torch.distributed.barrier()
    res = run_gpu(args, rank, world)
    if rank != 0:
        torch.distributed.destroy_process_group()
        return

    K = args.steps
    s = res["ms"] / 1e3
    ncell, npart = res["ncell"], res["n_part"]
    value, pushes = replica_totals(world, ncell, npart, g.get("n_sub", 1), K, s)
    peak, peak_kind = peaks()
    kt = res["kernel_times"]
    dom = max(kt, key=lambda k: kt[k][0])
    avg_ms = kt[dom][0] / max(kt[dom][1], 1)
    sv = res["source_reads"]["vertices"]
    ab = algorithmic_bytes(dom, res["grid"], npart, args.precision, sv)
    achieved = ab / (avg_ms / 1e3) / 1e9
    stencil_ms = kt["potential_step"][0] / max(kt["potential_step"][1], 1)
    stencil_b = algorithmic_bytes("potential_step", res["grid"], npart, args.precision, sv)
    stencil_gbs = stencil_b / (stencil_ms / 1e3) / 1e9
    stencil_min_gbs = minimum_bytes("potential_step", res["grid"], npart, args.precision) / (
        stencil_ms / 1e3) / 1e9
    total_kernel_ms = sum(v[0] for v in kt.values())
    line = {
        "metric": METRIC, "value": value, "unit": "cell-updates/s", "n_gpus": world,
        "steps": K, "warmup": args.warmup, "ms_per_step": res["ms"] / K,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "p64" else "f32", "data": "synthetic",
        "config": cfg,
        "particle_pushes_per_s": pushes,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak, "peak_kind": peak_kind,
                     "algorithmic_bytes_per_launch": ab, "avg_launch_ms": avg_ms,
                     "traffic": NCU_TRAFFIC.get((dom, args.precision, args.workload))},
        "stencil": {"kernel": "potential_step", "avg_launch_ms": stencil_ms,
                    "achieved_gbs": stencil_gbs, "frac": stencil_gbs / peak,
                    "bytes_per_cell": stencil_b / all_cells(g),
                    "bytes_model": "every vertex of the grid (interior by the update, boundary "
                                   "by Mur in increment form): read psi^n and D, write "
                                   "psi^{n+1} and D (16 B each in FP32, plus 8 B lo parts read "
                                   "and written for compensated levels), plus the 4 source "
                                   "values of every vertex of the marked source tiles",
                    "source_reads": res["source_reads"],
                    "frac_at_minimum_bytes": stencil_min_gbs / peak,
                    "minimum_bytes_per_cell": minimum_bytes("potential_step", res["grid"], npart,
                                                            args.precision) / all_cells(g),
                    "cell_updates_per_s": ncell / (stencil_ms / 1e3)},
        "push": push_rates(kt, npart, res["grid"], args.precision),
        "kernel_share": {k: round(v[0] / total_kernel_ms, 4) for k, v in kt.items()},
        "kernel_timing": {"region": "a second timed region of the same K steps launched one "
                                    "by one, a CUDA event pair around every kernel scope on the "
                                    "simulation's stream",
                          "ms_per_step": res["ms_events"] / K},
        "clocks": res["clocks"],
        "gpu_launches": res["launches"],
        "tuning": res["tuning"],
        "tuning_trials": res.get("trials"),
        "n_lost": res["n_lost"],
    }
    for side in ("p64", "p32_u64", "p32"):
        if side not in res:
            continue
        p = res[side]
        kts = p["kernel_times"]
        sts = kts["potential_step"][0] / max(kts["potential_step"][1], 1)
        line[side] = {"ms_per_step": p["ms"] / p["steps"], "steps": p["steps"],
                      "cell_updates_per_s": world * ncell * p["steps"] / (p["ms"] / 1e3),
                      "particle_pushes_per_s": world * npart * p["steps"] / (p["ms"] / 1e3),
                      "stencil_gbs": algorithmic_bytes("potential_step", res["grid"], npart,
                                                       side, p["source_reads"]["vertices"])
                      / (sts / 1e3) / 1e9,
                      "kernel_ms_per_launch": {k: v[0] / max(v[1], 1) for k, v in kts.items()
                                               if v[1]}}
    if "e2e" in res:
        e = res["e2e"]
        line["e2e"] = {"value": world * ncell * K / e["seconds"], "unit": "cell-updates/s",
                       "h2d_bytes_per_step": e["h2d"] / K, "d2h_bytes_per_step": e["d2h"] / K,
                       "seconds": e["seconds"]}
    if world == 1 and not args.no_c3:
        line["c3"] = run_c3(args, peak)
    if world == 1 and not args.no_batch:
        bt = run_batch(args, K=100, plain_jobs=4)
        line["batch"] = {k: v for k, v in bt.items()
                         if k not in ("metric", "impl", "mode", "higher_is_better", "n_gpus",
                                      "dtype", "data")}
    if world == 1 and not args.no_serve:
        sv = run_serve(args, duration=20.0)
        line["serve"] = {"jobs_per_h": sv["value"], "p50_s": sv["p50_s"], "p99_s": sv["p99_s"],
                         "precision": sv["precision"], "runs": sv["runs"],
                         "config": sv["config"]}
    if world == 1 and not args.no_cpu_baseline:
        r = cpu_oracle_rate(args.workload, 20.0)
        line["cpu_baseline"] = {"value": r["cell_updates_per_s"], "unit": "cell-updates/s",
                                "cores": r["cores"], "kind": "oracle", "sample": r["sample"],
                                "particle_pushes_per_s": r["pushes_per_s"]}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
