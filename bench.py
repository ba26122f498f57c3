#!/usr/bin/env python3
"""Throughput benchmark of the explicit mass-spring step on one GB300.

Workload (default): the 256^3 throughput lattice -- 16,777,216 masses,
216,338,940 26-neighbourhood springs (k ~ U[5e3, 5e4] N/m per spring,
c = 0.05 N s/m, bottom layer anchored, v ~ N(0, 1e-3) m/s, dt = 5e-5 s,
gravity on, no contact).  A bench "step" is one explicit time step over the
whole lattice (every spring and every mass updated once).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Under torchrun with N > 1 every rank runs its
own independent lattice (weak scaling, no data-path collective); the time is
the max over ranks.  --impl reference times the CPU oracle on the host cores
over a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "element updates/s (springs+masses) & %HBM roofline; batched robot-sim-s/s"
UNIT = "elements/s"
FALLBACK_HBM_GBS = 6800.0
# algorithmic bytes of one step: per mass read x, v (24 B) + write x, v
# (24 B) + inverse mass (4 B); per spring, general-graph model G: i, j, k, L0
# (16 B); lattice model L (topology and rest lengths from the grid): k (4 B).
# A kernel is graded on the model its layout is entitled to.
BYTES_PER_MASS = 52
BYTES_PER_SPRING = {"G": 16, "L": 4}
KERNEL_NAMES = ["", "gather", "tiled", "persistent", "lattice"]
STEP_KERNELS = {1: "k_step", 2: "k_step_tiled", 4: "k_step_lattice"}
STEP_SOURCES = {1: "ms_step.cu", 2: "ms_step.cu", 4: "ms_lattice.cu"}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def kernel_traffic(kernel_src: str, kname: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        with open(kernel_src, "rb") as f:
            h = hashlib.sha256(f.read()).hexdigest()[:16]
        ent = d.get(kname)
        if ent and ent.get("source_sha256_16") == h:
            return ent
    except Exception:
        pass
    return None


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap,clocks.mem")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                mem = float(parts[7]) if len(parts) > 7 else float("nan")
                rows.append((float(parts[0]), float(parts[1]), parts[3:7], mem))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for _, _, flags, _ in rows for q, f in enumerate(flags) if f.lower() == "active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows), "mem_mhz": statistics.median(r[3] for r in rows)}


def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Replicas:
    """N independent replicas launched by torchrun (one per GPU): no data-path
    collective; only a barrier around each timed region and the max over
    ranks of its duration, so `value` counts the work of all ranks over the
    slowest rank's time.  backend: "nccl" on GPUs, "gloo" for host tests."""

    def __init__(self, world: int, backend: str = "nccl"):
        self.world = world
        self.dist = None
        self.device = "cuda" if backend == "nccl" else "cpu"
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.dist = dist

    def barrier(self):
        if self.dist:
            self.dist.barrier()

    def max(self, x: float) -> float:
        if not self.dist:
            return float(x)
        import torch
        t = torch.tensor([float(x)], dtype=torch.float64, device=self.device)
        self.dist.all_reduce(t, op=self.dist.ReduceOp.MAX)
        return float(t.item())

    def throughput(self, units_per_rank: float, seconds: float) -> float:
        """whole-job units per second: every rank's units over the max time"""
        return self.world * units_per_rank / self.max(seconds)

    def close(self):
        if self.dist:
            self.dist.destroy_process_group()
            self.dist = None


def lattice_workload(n: int):
    s = synth.throughput_lattice(n=n)
    p = synth.throughput_params()
    return s, p


def byte_model(kernel_id: int) -> str:
    return "L" if kernel_id == 4 else "G"


def workload_config(n, N, S, model="L"):
    return {"workload": f"lattice{n} ({n}^3 masses, 26-neighbourhood springs, k~U[5e3,5e4], c=0.05, "
                        f"anchored bottom layer, v~N(0,1e-3), dt=5e-5, gravity, no contact)",
            "n_masses": N, "n_springs": S, "elements_per_step": N + S,
            "l2": "working set > L2 (no flush needed)",
            "byte_model": f"{model} ({BYTES_PER_MASS} B/mass + {BYTES_PER_SPRING[model]} B/spring)"}


# ------------------------------------------------------------------ oracle
def host_threads() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def time_oracle(side: int, threads: int, max_seconds: float, max_steps: int = 10000, warmup: int = 0):
    """Run the FP64 oracle on a side^3 lattice with the workload's parameters:
    `warmup` untimed steps, then one timed call of as many steps as fit in
    max_seconds (estimated from one calibration step), at most max_steps.
    threads = 1 is the serial oracle (ora_run), more is its mass-partitioned
    variant (ora_run_threads, bit-identical results).  Returns (elements/s,
    steps, seconds, threads used, N, S)."""
    import oracle
    s, p = lattice_workload(side)
    ar = oracle._Arrays(s)
    x, v = s["x"], s["v"]
    used = 1

    def run(n0, n, x, v):
        nonlocal used
        if threads == 1:
            return oracle.run(s, p, n, n0=n0, x=x, v=v, arrays=ar)
        x, v, used = oracle.run_threads(s, p, n, threads, n0=n0, x=x, v=v, arrays=ar)
        return x, v

    n0 = 0
    if warmup > 0:
        x, v = run(n0, warmup, x, v)
        n0 += warmup
    steps = max_steps
    if max_seconds < 1e8:
        t0 = time.perf_counter()
        x, v = run(n0, 1, x, v)
        n0 += 1
        steps = int(max(1, min(max_steps, max_seconds / max(time.perf_counter() - t0, 1e-6))))
    t0 = time.perf_counter()
    x, v = run(n0, steps, x, v)
    el = time.perf_counter() - t0
    N, S = s["x"].shape[0], s["ij"].shape[0]
    return steps * (N + S) / el, steps, el, used, N, S


def oracle_baseline(max_seconds: float = 15.0):
    """cpu_baseline: the FP64 oracle on the host cores -- on every core the
    process may use (a 64^3 sample) and, beside it, single-threaded (a 40^3
    sample); about max_seconds in all."""
    T = host_threads()
    v_all, st_all, el_all, used, N64, S64 = time_oracle(64, T, max_seconds / 2)
    v_one, st_one, el_one, _, N40, S40 = time_oracle(40, 1, max_seconds / 2)
    return {"value": v_all, "unit": UNIT, "cores": used, "kind": "oracle",
            "sample": f"64^3 lattice ({N64} masses, {S64} springs) with the workload's parameters, {st_all} steps "
                      f"in {el_all:.1f} s, FP64, {used} threads (masses partitioned, serial summation order)",
            "host_cpus": T,
            "single_thread": {"value": v_one, "unit": UNIT, "cores": 1,
                              "sample": f"40^3 lattice ({N40} masses, {S40} springs), {st_one} steps in {el_one:.1f} s"}}


def run_reference(args, world, rank):
    """Reference arm: the FP64 oracle as it stands on the host cores (all the
    process may use), one oracle step per bench step on a bounded sample of
    the workload (a ref_side^3 lattice with the workload's parameters)."""
    if rank != 0:
        return 0
    side = args.ref_side
    T = host_threads()
    val, steps, el, used, Ns, Ss = time_oracle(side, T, max_seconds=1e9, max_steps=args.steps, warmup=args.warmup)
    n = args.n
    N = n ** 3
    S = synth.lattice_spring_count(n, n, n)
    sample = (f"{side}^3 lattice ({Ns} masses, {Ss} springs) with the workload's parameters, "
              f"{steps} timed steps in {el:.2f} s, FP64, {used} threads")
    cfg = dict(workload_config(n, N, S), sample=f"each bench step = one oracle step of a {side}^3 sample "
                                                   f"({Ns + Ss} elements)")
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": steps, "warmup": args.warmup,
            "ms_per_step": el / steps * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded)",
            "config": cfg,
            "extrapolated_ms_per_step_at_workload": (N + S) / val * 1e3,
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": used, "kind": "oracle", "sample": sample,
                             "host_cpus": T},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ ours
def run_ours(args, world, rank, local):
    import torch
    import paper_2207_09334_gb300 as ms

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (no CPU fallback)")
    torch.cuda.set_device(local)
    reps = Replicas(world)
    ms.load()
    n = args.n
    t0 = time.perf_counter()
    s, p = lattice_workload(n)
    if args.integrator in ("verlet", "rk4"):
        p = dict(p, mu=0.0, vel_damping=0.0)   # contact is off: the same physics
    launches_per_step = 4 if args.integrator == "rk4" else 1
    N, S = s["x"].shape[0], s["ij"].shape[0]
    t_gen = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    t0 = time.perf_counter()
    sim = ms.Sim(s, p, reorder=args.order, kernel=args.kernel, stream=stream, integrator=args.integrator)
    torch.cuda.synchronize()
    t_create = time.perf_counter() - t0
    info = sim.info()

    for _ in range(args.warmup):
        sim.step(1)
    sim.sync()

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    reps.barrier()
    torch.cuda.synchronize()
    with Clocks(local) as clk:
        ev[0].record(stream)
        for q in range(args.steps):
            sim.step(1)
            ev[q + 1].record(stream)
        torch.cuda.synchronize()
    reps.barrier()
    total_ms = ev[0].elapsed_time(ev[-1])
    per = [ev[q].elapsed_time(ev[q + 1]) for q in range(args.steps)]
    sim.sync()
    value = reps.throughput((N + S) * args.steps, total_ms * 1e-3)
    total_ms = reps.max(total_ms)
    ms_per_step = total_ms / args.steps

    # end to end through the public API with host buffers: upload the state
    # from pinned host memory, run the workload's 200 steps, read it back
    e2e_steps = args.e2e_sim_steps
    bytes_state = 2 * N * 3 * 4
    e2e = None
    if args.e2e_iters > 0:
        xh = torch.from_numpy(np.ascontiguousarray(s["x"])).pin_memory()
        vh = torch.from_numpy(np.ascontiguousarray(s["v"])).pin_memory()
        xo = torch.empty_like(xh).pin_memory(); vo = torch.empty_like(vh).pin_memory()
        e2e_times = []
        reps.barrier()
        try:
            for it in range(args.e2e_iters + 1):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                sim.set_state(xh, vh)
                sim.step(e2e_steps)
                sim.get_state(xo, vo)
                el = time.perf_counter() - t0
                if it > 0:
                    e2e_times.append(el)
            e2e_val = reps.throughput((N + S) * e2e_steps, statistics.median(e2e_times))
            e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": bytes_state,
                   "d2h_bytes_per_step": bytes_state,
                   "note": f"each e2e step = ms_set_state(pinned host) + ms_step({e2e_steps}) + ms_get_state(pinned host)"}
        except ms.MsError as err:
            # forward Euler (eq. 4) amplifies every undamped mode: on this lattice
            # the state leaves the finite range within the e2e leg's steps
            e2e = {"value": None, "unit": UNIT, "h2d_bytes_per_step": bytes_state, "d2h_bytes_per_step": bytes_state,
                   "note": f"not measured: {err}"}

    hbm, hbm_kind = peaks()
    model = byte_model(info["kernel"])
    alg_bytes = BYTES_PER_MASS * N + BYTES_PER_SPRING[model] * S
    kern_ms = statistics.mean(per) / launches_per_step
    achieved = alg_bytes / (kern_ms * 1e-3) / 1e9
    kname = STEP_KERNELS.get(info["kernel"], "k_step")
    tr = kernel_traffic(os.path.join(ROOT, "paper_2207_09334_gb300", "csrc", STEP_SOURCES.get(info["kernel"], "ms_step.cu")),
                        kname) if args.integrator == "symplectic_euler" else None   # the capture is of the default scheme
    traffic = None
    if tr is not None:
        traffic = tr["dram_bytes_per_launch_at_256"] * (N + S) / tr["elements_at_256"] if n != 256 else tr["dram_bytes_per_launch_at_256"]
    cpu = oracle_baseline(max_seconds=args.cpu_seconds) if (rank == 0 and world == 1 and args.cpu_seconds > 0) else None

    clocks = clk.summary()
    batched = screening = adjoint = None
    if args.batched and args.integrator == "symplectic_euler":
        sim.close()                                  # free the lattice before the population is built
        batched = measure_population(args, reps, local, args.sim_steps_per_bench_step, 1)
        screening = measure_screening(args, reps, local)
        adjoint = measure_adjoint(args, reps, local)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": dict(workload_config(n, N, S, model), parallelism=f"replicas x{world}" if world > 1 else "1 GPU",
                           setup_s={"generate": round(t_gen, 1), "create": round(t_create, 1)},
                           mass_order=args.order, kernel=KERNEL_NAMES[info["kernel"]],
                           integrator=args.integrator,
                           device_bytes=info["device_bytes"], records=info["n_records"]),
            "e2e": e2e,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic,
                         "kernel": kname, "peak_kind": f"{hbm_kind} (hbm_gbs)",
                         "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": kern_ms},
            "gpu_launches": args.steps * launches_per_step,
            "clocks": clocks}
    if cpu is not None:
        line["cpu_baseline"] = cpu
    if batched is not None:                       # each with its own timed region
        line["batched"] = batched
        line["surrogate_screening"] = screening
        line["adjoint"] = adjoint
    if rank == 0:
        print(json.dumps(line), flush=True)
    sim.close()
    reps.close()
    return 0


# ------------------------------------------------------------------ other workloads
# algorithmic bytes of one population step: the robots' state stays in shared
# memory for the whole launch, so a step reads only the merged spring records:
# two robot-local endpoints (2 x 2 B), k, L0, the actuation pair (alpha, beta)
# and c (5 x 4 B)
POP_BYTES_PER_RECORD = 24


def measure_population(args, reps, local, sim_steps, timed_launches, warm_launches=1):
    """Batched voxel-robot population (4096 robots by default): robot-sim-s/s
    of `timed_launches` persistent launches of `sim_steps` steps each (one
    CUDA-graph replay per launch), a side record of 100-step launches, the
    plain per-robot launch loop on a short sample, and the roofline of the
    population kernel against POP_BYTES_PER_RECORD per merged spring and step."""
    import torch
    import paper_2207_09334_gb300 as ms
    designs = synth.voxel_population(args.robots, seed=2)
    p = synth.voxel_params()
    t0 = time.perf_counter()
    pop = ms.Population(designs, synth.VOXEL_MATERIALS, synth.VOXEL_FREQ, synth.VOXEL_EDGE, synth.VOXEL_MASS, p)
    pop.autotune(sample_steps=50)
    inf = pop.info()
    t_create = time.perf_counter() - t0
    stream = torch.cuda.current_stream()

    def timed(nsteps, reps_n):
        for _ in range(warm_launches):
            pop.run(nsteps)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        reps.barrier()
        e0.record(stream)
        for _ in range(reps_n):
            pop.run(nsteps)
        e1.record(stream)
        torch.cuda.synchronize()
        reps.barrier()
        return reps.max(e0.elapsed_time(e1))

    with Clocks(local) as clk:
        ms_total = timed(sim_steps, timed_launches)
    sim_s = args.robots * sim_steps * p["dt"] * timed_launches
    value = reps.throughput(sim_s, ms_total * 1e-3)
    ms_100 = timed(100, 5)
    value_100 = reps.throughput(args.robots * 100 * p["dt"] * 5, ms_100 * 1e-3)
    # the plain per-robot loop on a short sample of steps
    L = args.loop_steps
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    pop.run_loop(L)
    torch.cuda.synchronize()
    loop_s = reps.max(time.perf_counter() - t0)
    loop_value = reps.world * args.robots * L * p["dt"] / loop_s
    travel = pop.com_travel()
    steps_per_s = sim_steps * timed_launches / (ms_total * 1e-3)
    hbm, hbm_kind = peaks()
    achieved = POP_BYTES_PER_RECORD * inf["n_records"] * steps_per_s / 1e9
    rec = {"value": value, "unit": "robot-sim-s/s", "ms_per_launch": ms_total / timed_launches,
           "sim_steps_per_launch": sim_steps, "launches": timed_launches,
           "config": {"workload": f"population of {args.robots} voxel robots (sides U{{3..12}}, seed 2), "
                                  f"{sim_steps} simulated steps (dt = 1e-4) per persistent launch",
                      "n_masses": inf["n_masses"], "n_springs_merged": inf["n_records"],
                      "block_robots": inf["n_block_items"], "warp_robots": inf["n_warp_items"],
                      "threads_per_cta": inf["threads"], "setup_s": round(t_create, 1)},
           "elements_per_s": (inf["n_masses"] + inf["n_records"]) * steps_per_s * reps.world,
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                        "traffic": None, "kernel": "k_batch", "peak_kind": f"{hbm_kind} (hbm_gbs)",
                        "algorithmic_bytes_per_step": POP_BYTES_PER_RECORD * inf["n_records"],
                        "byte_model": f"{POP_BYTES_PER_RECORD} B per merged spring per step (state in shared memory)"},
           "launches_of_100_steps": {"value": value_100, "unit": "robot-sim-s/s", "ms_per_launch": ms_100 / 5},
           "per_robot_loop": {"value": loop_value, "unit": "robot-sim-s/s", "sim_steps": L,
                              "speedup_of_batched": value / loop_value},
           "travel_mean_m": float(np.mean(travel)), "clocks": clk.summary(),
           "gpu_launches": 3 * timed_launches}
    pop.close()
    return rec


def measure_screening(args, reps, local, passes=3, warm=2):
    """The surrogate's screening rate (config 5's learned component): 2^20 raw
    8^3 material grids scored per bench pass by the tensor-core MLP (one-hot
    tiles built on chip), 65 536 designs per forward pass."""
    import torch
    import paper_2207_09334_gb300 as ms
    B, n_cand = args.screen_batch, args.candidates
    rng = np.random.default_rng(4)
    cand = torch.tensor(rng.integers(0, 4, size=(n_cand, 512)).astype(np.uint8), device="cuda")
    out = torch.empty(n_cand, device="cuda")
    stream = torch.cuda.current_stream()
    with ms.Surrogate(2048, 512, max_batch=max(B, 1024), seed=0) as net:
        def screen_once():
            for q in range(0, n_cand, B):
                net.forward_materials(cand[q:q + B], out[q:q + B])
        for _ in range(warm):
            screen_once()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        reps.barrier()
        e0.record(stream)
        for _ in range(passes):
            screen_once()
        e1.record(stream)
        torch.cuda.synchronize()
        reps.barrier()
        ms_total = reps.max(e0.elapsed_time(e1))
    flops = 2.0 * (2048 * 512 + 512 * 512 + 512) * n_cand * passes * reps.world
    return {"value": reps.world * n_cand * passes / (ms_total * 1e-3), "unit": "designs/s",
            "ms_per_pass": ms_total / passes, "tensor_tflops": flops / (ms_total * 1e-3) / 1e12,
            "config": {"workload": f"MLP 2048->512->512->1 (bf16, fp32 accumulate) scoring {n_cand} 8^3 designs per "
                                   f"pass, {B} per forward pass", "passes": passes}}


def measure_adjoint(args, reps, local, evals=2, warm=1):
    """The differentiable batch (config 4): 256 walkers of 8^3 voxels, loss =
    centre-of-mass x-travel after 2000 steps, gradients w.r.t. every voxel's
    phase and log-stiffness by the checkpointed adjoint."""
    import torch
    import paper_2207_09334_gb300 as ms
    designs = synth.walker_designs(args.walkers, seed=3)
    mats = [m for m, _ in designs]
    phase = torch.tensor(np.concatenate([p.ravel() for _, p in designs]), device="cuda")
    kmat = synth.VOXEL_MATERIALS[:, 0]
    logk = torch.tensor(np.concatenate([np.where(m > 0, np.log(np.maximum(kmat[m], 1.0)), 0.0).ravel()
                                        for m in mats]).astype(np.float32), device="cuda")
    nsteps = args.rollout_steps
    stream = torch.cuda.current_stream()
    with ms.Adjoint(mats, synth.VOXEL_MATERIALS, synth.VOXEL_FREQ, synth.VOXEL_EDGE, synth.VOXEL_MASS,
                    synth.voxel_params(), checkpoint_every=100, max_steps=nsteps) as adj:
        for _ in range(warm):
            adj.gradients(nsteps, phase, logk)
        torch.cuda.synchronize()
        threads = adj.threads
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        reps.barrier()
        e0.record(stream)
        for _ in range(evals):
            loss, gp, gk = adj.gradients(nsteps, phase, logk)
        e1.record(stream)
        torch.cuda.synchronize()
        reps.barrier()
        ms_total = reps.max(e0.elapsed_time(e1))
    return {"value": reps.world * args.walkers * nsteps * synth.voxel_params()["dt"] * evals / (ms_total * 1e-3),
            "unit": "robot-sim-s/s (forward + reverse)", "ms_per_evaluation": ms_total / evals,
            "config": {"workload": f"{args.walkers} walkers of 8^3 voxels (seed 3), {nsteps} steps, checkpoint every "
                                   "100; one evaluation = loss + gradient for all walkers", "evaluations": evals,
                       "threads_per_robot": threads},
            "mean_travel_m": float(loss.mean())}


def run_population(args, world, rank, local):
    """Batched voxel-robot population: robot-sim-seconds per second, one bench
    step = one persistent launch of --sim-steps-per-bench-step (5000) steps."""
    import torch
    import paper_2207_09334_gb300 as ms
    torch.cuda.set_device(local)
    ms.load()
    reps = Replicas(world)
    S = args.sim_steps_per_bench_step
    rec = measure_population(args, reps, local, S, args.steps, warm_launches=max(1, min(args.warmup, 3)))
    line = {"metric": "batched robot-sim-s/s", "value": rec["value"], "unit": "robot-sim-s/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": rec["ms_per_launch"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded)", "config": rec["config"], "elements_per_s": rec["elements_per_s"],
            "roofline": rec["roofline"], "launches_of_100_steps": rec["launches_of_100_steps"],
            "per_robot_loop": rec["per_robot_loop"], "gpu_launches": rec["gpu_launches"], "clocks": rec["clocks"],
            "travel_mean_m": rec["travel_mean_m"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    reps.close()
    return 0


def run_surrogate(args, world, rank, local):
    """Surrogate screening throughput: candidate designs scored per second by
    the tensor-core MLP (one-hot encode + forward), against the simulator's
    designs per second for the same 2 s rollouts."""
    import torch
    import paper_2207_09334_gb300 as ms
    torch.cuda.set_device(local)
    ms.load()
    B = args.screen_batch                       # rows per forward pass while screening
    n_cand = args.candidates
    rng = np.random.default_rng(4)
    cand = torch.tensor(rng.integers(0, 4, size=(n_cand, 512)).astype(np.uint8), device="cuda")
    net = ms.Surrogate(2048, 512, max_batch=max(B, 1024), seed=0)
    out = torch.empty(n_cand, device="cuda")
    stream = torch.cuda.current_stream()

    def screen_once():
        for s in range(0, n_cand, B):
            net.forward_materials(cand[s:s + B], out[s:s + B])
    reps = Replicas(world)
    for _ in range(args.warmup):
        screen_once()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    reps.barrier()
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            screen_once()
        e1.record(stream)
        torch.cuda.synchronize()
    reps.barrier()
    ms_total = e0.elapsed_time(e1)
    value = reps.throughput(n_cand * args.steps, ms_total * 1e-3)
    ms_total = reps.max(ms_total)
    flops = 2.0 * (2048 * 512 + 512 * 512 + 512) * n_cand * args.steps * world
    # training step throughput (forward + backward + Adam, batch 1024)
    TB = 1024
    tgt = torch.randn(TB, device="cuda")
    for _ in range(3):
        net.train_step(cand[:TB], tgt)
    torch.cuda.synchronize()
    e0.record(stream)
    for _ in range(20):
        net.train_step(cand[:TB], tgt)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1) / 20
    # the simulator's rate on the same kind of design (2 s rollout = 20000 steps), sampled
    side = 8
    nsim = args.sim_designs
    designs = [(m.reshape(side, side, side), synth.surrogate_phase_field(side))
               for m in rng.integers(0, 4, size=(nsim, 512)).astype(np.uint8)]
    with ms.Population(designs, synth.VOXEL_MATERIALS, synth.VOXEL_FREQ, synth.VOXEL_EDGE, synth.VOXEL_MASS,
                       synth.voxel_params()) as pop:
        pop.autotune(sample_steps=50)
        pop.run(200)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        pop.run(2000)
        torch.cuda.synchronize()
        sim_rate = nsim / ((time.perf_counter() - t0) * 10.0)      # 2000 of the 20000 steps
    line = {"metric": "designs screened/s", "value": value, "unit": "designs/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate)",
            "data": "synthetic (seeded)",
            "config": {"workload": f"MLP 2048->512->512->1 scoring {n_cand} one-hot 8^3 designs per bench step, "
                                   f"{B} designs per forward pass"},
            "tensor_tflops": flops / (ms_total * 1e-3) / 1e12,
            "train_step_ms_batch1024": train_ms,
            "simulator_designs_per_s_2s_rollout": sim_rate,
            "screen_speedup_vs_simulation": value / (world * sim_rate),
            "gpu_launches": args.steps * (2 * (n_cand // B) + 2 * (n_cand // B)),
            "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    net.close()
    reps.close()
    return 0


def run_screen(args, world, rank, local):
    """The surrogate screening pipeline end to end: label designs with 2 s
    batched rollouts, train the tensor-core MLP on them, report its held-out
    R^2 and mean absolute error against the simulator, screen a candidate
    population and re-simulate the predicted top 1 % against a random 1 %
    of the same candidates (the method without the surrogate)."""
    import torch
    import paper_2207_09334_gb300 as ms
    from paper_2207_09334_gb300 import screen
    torch.cuda.set_device(local)
    ms.load()
    rng = np.random.default_rng(4)
    side, nsteps = 8, 20000                        # 2 s rollouts at dt = 1e-4
    n_train, n_val, n_cand = args.train_designs, 2048, args.candidates
    sim_args = (synth.VOXEL_MATERIALS, synth.VOXEL_FREQ, synth.VOXEL_EDGE, synth.VOXEL_MASS, synth.voxel_params())
    # random materials kept to each design's largest face-connected body, so
    # that loose voxels are not simulated (and labelled) as separate bodies
    mats = synth.largest_components(rng.integers(0, 4, size=(n_train + n_val, side, side, side)).astype(np.uint8))
    t0 = time.perf_counter()
    y = screen.simulate_travel(mats, *sim_args, nsteps=nsteps)
    t_label = time.perf_counter() - t0
    t0 = time.perf_counter()
    net, mu, sd = screen.train(mats[:n_train], y[:n_train], epochs=10, batch=1024, lr=1e-3, seed=0)
    t_train = time.perf_counter() - t0
    cand = synth.largest_components(rng.integers(0, 4, size=(n_cand, side, side, side)).astype(np.uint8))
    with net:
        pv = screen.predict(net, mats[n_train:], mu, sd)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        top, _ = screen.screen(net, cand, mu, sd, top_frac=0.01)
        t_screen = time.perf_counter() - t0
    yv = y[n_train:]
    k = len(top)
    y_top = screen.simulate_travel(cand[top], *sim_args, nsteps=nsteps)
    y_rand = screen.simulate_travel(cand[rng.choice(n_cand, size=k, replace=False)], *sim_args, nsteps=nsteps)
    line = {"metric": "designs screened/s (surrogate pipeline)", "value": n_cand / t_screen, "unit": "designs/s",
            "n_gpus": world, "steps": 1, "warmup": 0, "ms_per_step": t_screen * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "bf16 (fp32 accumulate); sim f32",
            "data": "synthetic (seeded)",
            "config": {"workload": f"{n_train} training designs (8^3, 4 materials, seed 4) labelled by 2 s rollouts, "
                                   f"{n_val} held out, {n_cand} candidates screened, top 1 % re-simulated",
                       "train_designs": n_train, "candidates": n_cand},
            "surrogate_r2": float(screen.r2(pv, yv)),
            "surrogate_mae_m": float(np.mean(np.abs(pv - yv))), "label_std_m": float(yv.std()),
            "top1pct_mean_travel_m": float(y_top.mean()), "random1pct_mean_travel_m": float(y_rand.mean()),
            "top1pct_gain_in_random_std_errors": float((y_top.mean() - y_rand.mean()) / (y_rand.std() / np.sqrt(k))),
            "label_s": round(t_label, 1), "train_s": round(t_train, 2),
            "screen_wall_s": round(t_screen, 3), "note": "screening time includes the host-to-device copy of the candidates"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_cube(args, world, rank, local):
    """The small-system workload: the 10^3 soft cube (1000 masses, 10,476
    springs) dropped from 0.05 m onto the ground with friction, 10,000 steps,
    timed on each single-system kernel.  Small systems are bound by latency,
    not bandwidth; value is the persistent cluster kernel's rate."""
    import torch
    import paper_2207_09334_gb300 as ms
    torch.cuda.set_device(local)
    ms.load()
    s = synth.soft_cube()
    p = synth.soft_cube_params(contact=True)
    N, S = s["x"].shape[0], s["ij"].shape[0]
    nsteps = args.cube_steps
    stream = torch.cuda.current_stream()
    reps = Replicas(world)
    per_kernel = {}
    launches = 0
    for kernel in ("persistent", "tiled", "gather"):
        with ms.Sim(s, p, kernel=kernel, stream=stream) as sim:
            for _ in range(args.warmup):
                sim.step(100)
            sim.sync()
            sim.set_state(s["x"], s["v"])
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            reps.barrier()
            torch.cuda.synchronize()
            e0.record(stream)
            sim.step(nsteps)
            e1.record(stream)
            torch.cuda.synchronize()
            reps.barrier()
            ms_total = e0.elapsed_time(e1)
            x, _ = sim.get_state()
            per_kernel[kernel] = {"us_per_step": reps.max(ms_total) * 1e3 / nsteps,
                                  "elements_per_s": reps.throughput((N + S) * nsteps, ms_total * 1e-3),
                                  "com_z_final_m": float(x[:, 2].mean())}
            launches += 1 if kernel == "persistent" else nsteps
    best = per_kernel["persistent"]
    line = {"metric": "element updates/s (soft cube, 10^3 masses)", "value": best["elements_per_s"], "unit": "elements/s",
            "n_gpus": world, "steps": 1, "warmup": args.warmup, "ms_per_step": best["us_per_step"] * 1e-3 * nsteps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded)",
            "config": {"workload": f"10^3 soft cube (a = 0.01 m, k = 1e4, c = 0.1), dropped from 0.05 m, k_c = 1e5, "
                                   f"mu = 0.5, dt = 1e-4, {nsteps} steps per bench step",
                       "n_masses": N, "n_springs": S},
            "per_kernel": per_kernel, "gpu_launches": launches}
    if rank == 0:
        print(json.dumps(line), flush=True)
    reps.close()
    return 0


def run_sweep(args, world, rank, local):
    """Element update rate against system size (the paper's rate-vs-size
    experiment): throughput lattices of n^3 masses, the default kernel, the
    persistent kernel where the system fits it (a thread-block cluster up to
    8192 masses, then one cooperative launch while every tile is resident),
    and the lattice kernel where it is not already the default."""
    import torch
    import paper_2207_09334_gb300 as ms
    torch.cuda.set_device(local)
    ms.load()
    stream = torch.cuda.current_stream()
    reps = Replicas(world)
    rows = []
    for n in args.sweep_sizes:
        s, p = lattice_workload(n)
        N, S = s["x"].shape[0], s["ij"].shape[0]
        auto_kernel = None
        for kernel in ("auto", "persistent", "lattice"):
            try:
                sim = ms.Sim(s, p, kernel=None if kernel == "auto" else kernel, stream=stream)
            except ms.MsError:
                continue                            # the persistent kernel does not take this size
            if kernel == "auto":
                auto_kernel = sim.info()["kernel"]
            elif sim.info()["kernel"] == auto_kernel:
                sim.close()                         # already measured as the default
                continue
            with sim:
                steps = max(20, min(2000, int(2e9 // (N + S))))     # about 2e9 element updates per point
                sim.step(max(3, steps // 10))
                sim.sync()
                e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
                reps.barrier()
                torch.cuda.synchronize()
                e0.record(stream)
                sim.step(steps)                     # one call: the library launches the steps
                e1.record(stream)
                torch.cuda.synchronize()
                reps.barrier()
                t = e0.elapsed_time(e1) * 1e-3
                rows.append({"n": n, "masses": N, "springs": S, "kernel": KERNEL_NAMES[sim.info()["kernel"]],
                             "steps": steps, "us_per_step": reps.max(t) * 1e6 / steps,
                             "elements_per_s": reps.throughput((N + S) * steps, t)})
    best = max(r["elements_per_s"] for r in rows)
    line = {"metric": "element updates/s vs system size", "value": best, "unit": "elements/s", "n_gpus": world,
            "steps": None, "warmup": None, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded)",
            "config": {"workload": "throughput lattices n^3 (the 256^3 workload's parameters), default kernel and, where "
                                   "the system fits it, the persistent kernel", "sizes": list(args.sweep_sizes)},
            "points": rows}
    if rank == 0:
        print(json.dumps(line), flush=True)
    reps.close()
    return 0


def run_adjoint(args, world, rank, local):
    """Differentiable batch: 256 walkers of 8^3 voxels, loss = centre-of-mass
    x-travel after 2000 steps, gradients w.r.t. every voxel's phase and
    log-stiffness by the checkpointed adjoint (checkpoint every 100 steps)."""
    import torch
    import paper_2207_09334_gb300 as ms
    torch.cuda.set_device(local)
    ms.load()
    designs = synth.walker_designs(args.walkers, seed=3)
    mats = [m for m, _ in designs]
    phase = torch.tensor(np.concatenate([p.ravel() for _, p in designs]), device="cuda")
    kmat = synth.VOXEL_MATERIALS[:, 0]
    logk = torch.tensor(np.concatenate([np.where(m > 0, np.log(np.maximum(kmat[m], 1.0)), 0.0).ravel()
                                        for m in mats]).astype(np.float32), device="cuda")
    nsteps = args.rollout_steps
    adj = ms.Adjoint(mats, synth.VOXEL_MATERIALS, synth.VOXEL_FREQ, synth.VOXEL_EDGE, synth.VOXEL_MASS,
                     synth.voxel_params(), checkpoint_every=100, max_steps=nsteps)
    stream = torch.cuda.current_stream()
    reps = Replicas(world)
    for _ in range(args.warmup):
        adj.gradients(nsteps, phase, logk)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    reps.barrier()
    with Clocks(local) as clk:
        e0.record(stream)
        for _ in range(args.steps):
            loss, gp, gk = adj.gradients(nsteps, phase, logk)
        e1.record(stream)
        torch.cuda.synchronize()
    reps.barrier()
    ms_total = e0.elapsed_time(e1)
    value = reps.throughput(args.walkers * nsteps * synth.voxel_params()["dt"] * args.steps, ms_total * 1e-3)
    per = reps.max(ms_total) / args.steps
    line = {"metric": "differentiated robot-sim-s/s", "value": value, "unit": "robot-sim-s/s (forward + reverse)",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": per,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic (seeded)",
            "config": {"workload": f"{args.walkers} walkers of 8^3 voxels (seed 3), {nsteps} steps, checkpoint every 100; "
                                   "one bench step = one loss + gradient evaluation for all walkers",
                       "voxels": int(adj.n_voxels), "masses": int(adj.n_masses), "threads_per_robot": adj.threads},
            "mean_travel_m": float(loss.mean()), "grad_phase_rms": float(gp.pow(2).mean().sqrt()),
            "grad_logk_rms": float(gk.pow(2).mean().sqrt()),
            "gpu_launches": 5 * args.steps, "clocks": clk.summary()}
    if rank == 0:
        print(json.dumps(line), flush=True)
    adj.close()
    reps.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=256, help="lattice side (256 = the benchmark workload)")
    ap.add_argument("--order", default="auto", choices=["auto", "morton", "caller"], help="internal mass order")
    ap.add_argument("--kernel", default="auto", choices=["auto", "gather", "tiled", "lattice"])
    ap.add_argument("--integrator", default="symplectic_euler",
                    choices=["symplectic_euler", "forward_euler", "verlet", "rk4"],
                    help="lattice workload: step scheme (rk4 = 4 stage launches per step)")
    ap.add_argument("--e2e-sim-steps", type=int, default=200)
    ap.add_argument("--e2e-iters", type=int, default=3)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-side", type=int, default=64, help="reference arm: side of the sampled lattice")
    ap.add_argument("--workload", default="lattice",
                    choices=["lattice", "population", "surrogate", "adjoint", "screen", "cube", "sweep"])
    ap.add_argument("--cube-steps", type=int, default=10000, help="cube workload: steps per kernel")
    ap.add_argument("--sweep-sizes", type=int, nargs="+", default=[8, 10, 12, 16, 18, 20, 24, 32, 40, 48, 64, 96, 128, 192, 256],
                    help="sweep workload: lattice sides")
    ap.add_argument("--train-designs", type=int, default=16384, help="screen workload: labelled training designs (200000 = the full config)")
    ap.add_argument("--walkers", type=int, default=256)
    ap.add_argument("--rollout-steps", type=int, default=2000)
    ap.add_argument("--robots", type=int, default=4096)
    ap.add_argument("--sim-steps-per-bench-step", type=int, default=5000,
                    help="population workload: simulated steps per persistent launch (one bench step)")
    ap.add_argument("--batched", type=int, default=1,
                    help="lattice workload: add the records of the population (one 5000-step launch), the "
                         "surrogate's screening and the adjoint")
    ap.add_argument("--loop-steps", type=int, default=5)
    ap.add_argument("--candidates", type=int, default=1 << 20)
    ap.add_argument("--screen-batch", type=int, default=65536, help="designs per surrogate forward pass")
    ap.add_argument("--sim-designs", type=int, default=1024)
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "population":
        return run_population(args, world, rank, local)
    if args.workload == "surrogate":
        return run_surrogate(args, world, rank, local)
    if args.workload == "adjoint":
        return run_adjoint(args, world, rank, local)
    if args.workload == "screen":
        return run_screen(args, world, rank, local)
    if args.workload == "cube":
        return run_cube(args, world, rank, local)
    if args.workload == "sweep":
        return run_sweep(args, world, rank, local)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
