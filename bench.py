"""Benchmark of the relaxation hot path: particle-steps/s on the 3D cube-minus-sphere workload.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A step is one pass of the whole hot path (cell-list rebuild, pressure pass with the feature
boundary correction, controller, viscous update with projection) over every particle of the
instance.  Workload (headline): unit cube minus a centred sphere of radius 0.3, curve particles
on the 12 edges, surface particles on the 6 faces and the sphere, volume particles inside, 8
fixed corners, h = min(0.008 + 0.04 |d_sphere|, 0.05) scaled to ~1.2M particles, FP32 pair sums
with FP64 projection/reductions -- the largest single-GPU configuration.

* value:  particle-steps/s over K device-timed steps (CUDA events on the library's stream),
          L2 flushed (256 MiB write) between steps; inputs resident in HBM.
* e2e:    the same metric through the public C ABI from pinned host buffers: upload of the
          initial state, K steps each followed by the read-back of the controller report,
          read-back of the final positions -- all inside the host-timed region.
* roofline: the dominant kernel's achieved rate from its live CUDA-event times, taken in a
          second timed region (up to 1000 more steps, same L2 flush) whose step graph holds an
          event between the stages; the headline region runs the graph without them, so that
          its kernel-to-kernel edges keep their programmatic (early) launch.
* cpu_baseline / --impl reference: the FP64 CPU oracle on the host cores (bounded sample of
          the same workload).
* disk_2d: the 2D unit disk minus 3 seeded holes (h linear in the distance to the nearest hole,
          0.004-0.04 scaled to ~120k particles), device-timed steps with its own stage split.
* batched: 64 independent instances (half 2D disks with holes, half 3D cubes minus a sphere,
          particle counts log-uniform over 1k-200k, seeded), one batch per dimension on its own
          stream, each step one CUDA graph per batch; particle-steps/s over all instances.
* serving: a seeded Poisson stream of jobs of the same two kinds through the server (admitted
          by memory, retired on convergence or at the iteration limit), p50/p99 job latency and
          aggregate particle-steps/s, beside the same jobs served one at a time by the plain
          FP64 single-instance path (FIFO on the measured service times).
* init_sampling: the 1.2M cube's initial particles drawn on the device (target counts of
          Eqs. 10, 11 and rho_t-proportional sampling, Sec. 3.6), beside the host generator.
* method_presets: the comparison of Sec. 4.1 on its Square (Eq. 25 sizing): iterations to the
          Phase-One target and to the end for the improved method and the earlier method's two
          presets (velocities zeroed every step / every 100 steps, no feature-boundary sum), and
          the Cube (Eq. 28) and Sphere01 cases of Sec. 4 for the paper's iteration counts, each
          final state's mesh quality beside the paper's tables.
Multi-GPU (torchrun): every rank runs an independent replica (weak scaling, no collective on
the data path); value = particles of all ranks x K / max rank time.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "particle-steps/s"
WORKLOAD = "cube_sphere_3d_1.2M"
DISK_WORKLOAD = "disk_holes_2d_120k"
FLOP_PER_PAIR = 50.0       # FP32 operations per interacting pair of the pressure pass (see design notes)
# DRAM bytes (read + write) per particle of one launch of the dominant kernel (the 3D pressure
# pass): the ncu capture of this kernel on the headline's generator at 300,009 particles, 5 steps
# after the start (116.7 MB read + 179.6 MB written); its traffic grows with the particle count
# (own state, neighbour records missing L2, the hand-over list), so a launch on n particles moves
# n times this.  Set to None whenever the kernel changes until it has been captured again.
DOMINANT_DRAM_BYTES_PER_PARTICLE = (116.726272e6 + 179.580416e6) / 300_009
SM_COUNT, FP32_LANES, SM_MAX_MHZ = 152, 128, 2070.0
# one 3D step: one-pass scan, scatter, gather, pressure pass, controller, viscous pass, update
# (+ next keys)
KERNELS_PER_STEP = 7


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=1_200_000)
    ap.add_argument("--disk-n", type=int, default=120_000)
    ap.add_argument("--no-disk", action="store_true")
    ap.add_argument("--disk-steps", type=int, default=200)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--batch-steps", type=int, default=200)
    ap.add_argument("--serve-jobs", type=int, default=24, help="arrivals of the 50 jobs/s stream served")
    ap.add_argument("--serve-iters", type=int, default=3000, help="iteration limit of a served job")
    ap.add_argument("--serve-max-n", type=int, default=2_000_000)
    ap.add_argument("--serve-threshold", type=float, default=1e-2,
                    help="Phase-One/Two threshold of served jobs (the level the method reaches under this "
                         "build's readings; the paper's 5e-6 is never reached)")
    ap.add_argument("--serve-70-jobs", type=int, default=12)
    ap.add_argument("--fp64-subset-max-n", type=int, default=60_000)
    ap.add_argument("--fp64-subset-jobs", type=int, default=4)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-cube", action="store_true")
    ap.add_argument("--no-presets", action="store_true")
    ap.add_argument("--preset-iters", type=int, default=40_000)
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return d, "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def hbm_peak(peaks):
    for k in ("hbm_gbs", "hbm_GBs", "hbm_copy_gbs", "hbm"):
        if k in peaks and isinstance(peaks[k], (int, float)):
            return float(peaks[k])
    return 6800.0


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[0]))
                mx.append(float(r[1]))
            except Exception:
                continue
            for k, nm in enumerate(names):
                if len(r) > 4 + k and r[4 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


def replica_throughput(local_ms, particles, steps, device=None):
    """Replicas (one independent instance per rank, no collective on the data path): the job
    time is the slowest rank's, the throughput counts every rank's particles.  Returns
    (max ms over ranks, particle-steps/s of the whole job)."""
    import torch

    ws = 1
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        ws = torch.distributed.get_world_size()
        t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
        n = torch.tensor([float(particles)], dtype=torch.float64, device=device)
        torch.distributed.all_reduce(n, op=torch.distributed.ReduceOp.SUM)
        local_ms, total = float(t.item()), float(n.item())
    else:
        total = float(particles)
    return local_ms, total * steps / (local_ms / 1e3)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def make_workload(n):
    """The headline workload: the cube minus a sphere at n particles (seed 3), built in a worker
    process (spawn) so that the calling process has made no GPU call when it forks nothing."""
    return generate([(4, n, 3, 0.3)])[0]


def make_disk(n):
    from paper_2003_01061_gb300 import workloads as WL

    return WL.disk_holes(n_target=n, seed=2)


def _gen_problem(spec):
    """A job given by its problem alone (its particles are drawn on the device at admission)."""
    from paper_2003_01061_gb300 import workloads as WL

    kind, n, seed, r = spec
    if kind == 2:
        return WL.disk_holes(n_target=n, seed=seed, mc_samples=100_000, sample=False)
    return WL.cube_sphere(n_target=n, seed=seed, sphere_r=r, mc_samples=100_000, sample=False)


def generate_problems(specs):
    import multiprocessing as mp

    procs = max(1, min(16, (os.cpu_count() or 2) - 1, len(specs)))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_gen_problem, specs, chunksize=1)


def _gen_one(spec):
    from paper_2003_01061_gb300 import workloads as WL

    kind, n, seed, r = spec
    if kind == 2:
        return WL.disk_holes(n_target=n, seed=seed, mc_samples=100_000)
    if kind == 4:   # the single-instance 3D workload, with the generator's default integration
        return WL.cube_sphere(n_target=n, seed=seed, sphere_r=r)
    return WL.cube_sphere(n_target=n, seed=seed, sphere_r=r, mc_samples=100_000)


def _specs(n_items, seed, n_lo, n_hi, alternate, rate=None, frac_3d=0.5):
    """Seeded (kind, n, seed, sphere radius) per item (+ Poisson arrival times when rate)."""
    rng = np.random.default_rng(seed)
    t, out, times = 0.0, [], []
    for k in range(n_items):
        if rate:
            t += float(rng.exponential(1.0 / rate))
        n = int(round(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        s = int(rng.integers(1 << 30))
        kind = (2 if k % 2 == 0 else 3) if alternate else (3 if rng.random() < frac_3d else 2)
        out.append((kind, n, s, float(rng.uniform(0.2, 0.35))))
        times.append(t)
    return out, times


def generate(specs):
    """Workloads built in a process pool started with spawn (never forked after GPU use)."""
    import multiprocessing as mp

    procs = max(1, min(16, (os.cpu_count() or 2) - 1, len(specs)))
    with mp.get_context("spawn").Pool(procs) as pool:
        return pool.map(_gen_one, specs, chunksize=1)


# ----------------------------------------------------------------------------------------
# CPU oracle timing (the reference arm and the cpu_baseline leg)
# ----------------------------------------------------------------------------------------
def oracle_rate(w, budget_s=15.0, sample=None, steps=None):
    """Times the FP64 oracle's pressure pass + update on a fixed random sample of particles.

    Every sampled particle runs with its full neighbourhood.  Unsampled neighbours carry
    a_p = 0 in the viscous sum: with the sampled particle's own velocity nonzero every pair
    term is still evaluated, so the work per sampled particle is that of the full step.
    Returns (particle-steps/s, description, threads, per-step seconds list)."""
    from oracle import oracle as O

    o = O.Oracle(w)
    n = o.n
    a_all = np.zeros((n, 3))
    rng = np.random.default_rng(0)

    def one(sub):
        t0 = time.perf_counter()
        r = o.interact(sub=sub, use_grid=True)
        for g in range(o.G):
            o.ctrl.dt[g] = r["dta"][g] if np.isfinite(r["dta"][g]) else 0.0
            o.ctrl.reset[g] = 1
        a_all[sub] = r["a_p"]
        o.integrate(a_all, sub=sub, use_grid=True)
        return time.perf_counter() - t0

    if sample is None:
        probe = np.sort(rng.choice(n, min(n, 2048), replace=False))
        per = one(probe) / len(probe)
        sample = int(min(n, max(1024, budget_s / 3.0 / max(per, 1e-9))))
    sub = np.sort(rng.choice(n, sample, replace=False))
    nsteps = steps if steps is not None else 3
    times = [one(sub) for _ in range(nsteps)]
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    rate = sample * len(times) / sum(times)
    desc = (f"FP64 oracle pressure pass + viscous update of {sample} randomly sampled particles (of {n}) "
            f"with full neighbourhoods, {len(times)} steps")
    return rate, desc, threads, times


def run_reference(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return
    w = make_workload(args.n)
    n = len(w["x"])
    budget = 90.0
    per_step = budget / max(args.steps + args.warmup, 1)
    from oracle import oracle as O

    O.build()
    rate0, _, _, _ = oracle_rate(w, budget_s=min(per_step * 3, 10.0), steps=1)
    sample = int(min(n, max(512, rate0 * per_step)))
    oracle_rate(w, sample=sample, steps=max(args.warmup, 0) or 1)
    rate, desc, threads, times = oracle_rate(w, sample=sample, steps=args.steps)
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": METRIC, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times) * n / sample,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles": n, "dim": 3, "precision": "fp64 oracle"},
        "cpu_baseline": {"value": rate, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": desc},
        "e2e": {"value": rate, "unit": METRIC, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


# ----------------------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------------------
def run_ours(args):
    import torch

    ws, rank, local = dist_env()
    # batch and serving inputs, generated before the first GPU call
    batch_ws, serve_ws, serve_t = None, None, None
    # the headline workload (every rank runs its own replica of it)
    t0 = time.perf_counter()
    w = make_workload(args.n)
    gen_s = time.perf_counter() - t0
    disk_w = make_disk(args.disk_n) if (rank == 0 and not args.no_disk) else None
    preset_w = cube_case_w = None
    if rank == 0 and not args.no_presets:
        from paper_2003_01061_gb300 import workloads as WL

        preset_w = WL.square_radial(seed=6)
        cube_case_w = (WL.cube_radial(seed=7), WL.sphere01(seed=8), WL.sphere02(seed=9))
    if rank == 0 and not args.no_batch:
        specs, _ = _specs(64, 4, 1_000, 200_000, alternate=True)
        batch_ws = generate(specs)
    if rank == 0 and not args.no_serve:
        specs, serve_t = _specs(args.serve_jobs, 5, 1_000, args.serve_max_n, alternate=False, rate=50.0)
        serve_ws = generate_problems(specs)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2003_01061_gb300 import build as B
    from paper_2003_01061_gb300 import sphmesh as S

    B.build()
    n = len(w["x"])
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    head = timed_run(S, torch, w, stream, flush, args.steps, args.warmup, min(args.steps, 200),
                     barrier=ws > 1, clock_index=local)
    m = head.pop("mesh")
    total_ms = head["total_ms"]
    rep = m.report()
    total_ms, value = replica_throughput(total_ms, n, args.steps, dev)
    peaks, peak_src = measured_peaks()
    clocks = head["clocks"]
    roofline = roofline_of(head, n, peaks, peak_src, dim=3)
    head_err = oracle_error(S, m, w, with_oracle=not args.no_cpu_baseline) if rank == 0 else None
    e2e = None
    if not args.no_e2e:
        e2e = e2e_run(S, w, stream, args.steps)

    disk = None
    if disk_w is not None:
        dm = timed_run(S, torch, disk_w, stream, flush, args.disk_steps, 5, min(args.disk_steps, 200))
        dmesh = dm.pop("mesh")
        disk_err = oracle_error(S, dmesh, disk_w, with_oracle=not args.no_cpu_baseline)
        dmesh.close()
        disk = {"value": dm["value"], "unit": METRIC, "steps": args.disk_steps,
                "ms_per_step": dm["total_ms"] / args.disk_steps, "particles": len(disk_w["x"]),
                "stages_ms": dm["stages_ms"], "pairs_per_particle": dm["pairs_per_particle"],
                "roofline": roofline_of(dm, len(disk_w["x"]), peaks, peak_src, dim=2), "oracle_error": disk_err,
                "config": {"workload": DISK_WORKLOAD + ": unit disk minus 3 seeded holes, h linear in the "
                                       "distance to the nearest hole (0.004-0.04) scaled to ~120k particles "
                                       "(seed 2), FP32", "l2": "flushed between timed steps (256 MiB write)"}}

    presets = None
    if preset_w is not None:
        presets = presets_run(S, preset_w, args.preset_iters)
        presets["cube_case"] = case_3d_run(S, cube_case_w[0], "cube_table", {"improved": 7000, "fu2019": 28800})
        presets["sphere01_case"] = case_3d_run(S, cube_case_w[1], "sphere01_table", {"improved": 4600, "fu2019": 17000})
        presets["sphere02_case"] = case_3d_run(S, cube_case_w[2], "sphere02_table", {"improved": 3800})

    sampling = None
    if rank == 0 and not args.no_cube:
        sampling = sampling_run(S, w, gen_s, with_oracle=not args.no_cpu_baseline)

    batched = None
    if batch_ws is not None:
        batched = batched_run(S, torch, dev, batch_ws, args.batch_steps)
        batched["config"] = {"workload": "64 instances, half disk_holes_2d / half cube_sphere_3d, "
                                         "n log-uniform 1k-200k (seed 4)",
                             "l2": "working set larger than L2 (no flush)"}
    serving = None
    if serve_ws is not None:
        serving = serving_legs(S, serve_ws, serve_t, args)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        from oracle import oracle as O

        O.build()
        rate, desc, threads, times = oracle_rate(w, budget_s=15.0)
        cpu = {"value": rate, "unit": METRIC, "cores": threads, "kind": "oracle", "sample": desc}

    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles": n, "dim": 3, "groups": m.n_groups,
                   "description": "unit cube minus a centred sphere r=0.3: 12 edge curves, 6 faces + the sphere "
                                  "surface, volume, 8 fixed corners; h = min(0.008 + 0.04|d_sphere|, 0.05) scaled "
                                  "to 1.2M particles (seed 3)",
                   "precision": "fp32 pair sums, fp64 projection and reductions", "replicas": ws,
                   "l2": "flushed between timed steps (256 MiB write); the working set is also larger than L2",
                   "phase_at_end": int(rep.phase), "iteration_at_end": int(rep.iteration)},
        "roofline": roofline,
        "oracle_error": head_err,
        "stages_ms": head["stages_ms"],
        "stages_timing": {"steps": head["stage_steps"],
                          "ms_per_step_with_stage_events": head["staged_ms"] / head["stage_steps"]},
        "pairs_per_particle": head["pairs_per_particle"],
        "clocks": clocks,
        "gpu_launches": KERNELS_PER_STEP * args.steps,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "disk_2d": disk,
        "method_presets": presets,
        "init_sampling": sampling,
        "batched": batched,
        "serving": serving,
    }
    m.close()
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


def e2e_run(S, w, stream, steps):
    """Whole job through the public API from pinned host buffers (host-timed)."""
    import torch

    n = len(w["x"])
    x = torch.from_numpy(np.ascontiguousarray(w["x"])).pin_memory().numpy()
    g = torch.from_numpy(np.ascontiguousarray(w["group"], dtype=np.int32)).pin_memory().numpy()
    xo = torch.empty((n, 3), dtype=torch.float64).pin_memory().numpy()
    go = torch.empty(n, dtype=torch.int32).pin_memory().numpy()
    m = S.Mesh(w, precision=32, stream=stream.cuda_stream)
    m.set_state()
    m.step(2)
    S.sph_mesh_report(m.h)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S.sph_mesh_set_state(m.h, x, g)
    for _ in range(steps):
        S.sph_mesh_step(m.h, 1)
        S.sph_mesh_report(m.h)          # the step's result: controller state (E_sys, phase, dt)
    got = S.lib().sph_mesh_positions(m.h, xo.ctypes.data, go.ctypes.data, None, None, n, None)
    t1 = time.perf_counter()
    assert got == 0
    m.close()
    h2d = n * (3 * 8 + 4)
    d2h_report = S.C.sizeof(S.sph_report) if hasattr(S, "C") else 1280
    d2h = n * (3 * 8 + 4) / steps + d2h_report
    return {"value": n * steps / (t1 - t0), "unit": METRIC, "h2d_bytes_per_step": h2d / steps,
            "d2h_bytes_per_step": d2h, "wall_s": t1 - t0,
            "job": f"upload of {n} particles, {steps} steps each with a controller-report read, final download"}


def stages_per_step(times, steps):
    """ms per step of each stage from the library's per-stage (launches, total ms) over `steps`
    steps (a stage may launch several kernels per step: its time is not divided by them)."""
    return {k: v[1] / max(steps, 1) for k, v in times.items()}


def timed_run(S, torch, w, stream, flush, steps, warmup, stage_steps, barrier=False, clock_index=None):
    """One FP32 instance of w: `warmup` untimed steps (they also capture the step graph), then
    `steps` device-timed steps (CUDA events on the library's stream, the graph without stage
    events, L2 flushed between steps), then `stage_steps` more with an event between the
    stages for the per-kernel split (those events turn the kernel-to-kernel edges they sit on
    into ordinary ones, so they are kept out of the headline steps)."""
    m = S.Mesh(w, precision=32, stream=stream.cuda_stream)
    m.set_state()
    m.step(max(warmup, 1))
    m.sync()

    def timed_steps(n_steps):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(n_steps)]
        with torch.cuda.stream(stream):
            for k in range(n_steps):
                evs[k][0].record(stream)
                m.step(1)
                evs[k][1].record(stream)
                flush.zero_()       # 256 MiB write between timed steps evicts the 129 MB L2
        torch.cuda.synchronize()
        return float(sum(a.elapsed_time(b) for a, b in evs))

    clk = Clocks(clock_index) if clock_index is not None else None
    if clk:
        clk.__enter__()
        time.sleep(0.3)             # let the sampler start before the timed region
    if barrier:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    total_ms = timed_steps(steps)
    if barrier:
        torch.distributed.barrier()
    if clk:
        clk.__exit__(None, None, None)
    S.sph_mesh_set_timing(m.h, 1)
    m.step(1)                       # re-capture with the stage events
    m.sync()
    S.sph_mesh_set_timing(m.h, 1)   # zero the accumulators
    stage_steps = max(stage_steps, 1)
    staged_ms = timed_steps(stage_steps)
    stage = S.sph_mesh_kernel_times(m.h)
    S.sph_mesh_set_timing(m.h, 0)
    m.sync()
    cand, accd = S.sph_debug_pair_counts(m.h)
    n = len(w["x"])
    stages = stages_per_step(stage, stage_steps)
    return {"mesh": m, "total_ms": total_ms, "value": n * steps / (total_ms / 1e3), "staged_ms": staged_ms,
            "stage_steps": stage_steps, "stages_ms": stages, "accd": accd,
            "clocks": clk.summary() if clk else None,
            "pairs_per_particle": {"candidates": cand / n, "interacting": accd / n}}


def oracle_error(S, m, w, n_sample=2048, with_oracle=True):
    """The FP64-oracle error of the FP32 result: the pressure pass on the mesh's current state
    (after the timed steps), on the GPU and in the oracle on the same positions, velocities and h,
    compared on a random sample of particles as |a_p(GPU) - a_p(oracle)| / S_i (S_i: the sum of the
    magnitudes of the terms of particle i's force; the parity tolerance is 1e-5)."""
    if not with_oracle:
        return None
    from oracle import oracle as O

    O.build()
    st = m.positions()
    n = len(st["x"])
    got = S.sph_debug_interact(m.h, n, m.n_groups)
    rng = np.random.default_rng(11)
    sub = np.sort(rng.choice(n, min(n, n_sample), replace=False))
    ww = dict(w, group=st["group"])
    o = O.Oracle(ww, x=st["x"], v=st["v"], h=st["h"])
    ref = o.interact(sub=sub, use_grid=True)
    moving = o.gdim[st["group"][sub]] > 0
    err = np.linalg.norm(got["a_p"][sub] - ref["a_p"], axis=1)[moving] / np.maximum(ref["S"][moving], 1e-300)
    return {"quantity": f"a_p of {len(sub)} sampled particles, GPU FP32 pressure pass against the FP64 oracle "
                        f"on the state after the timed steps", "max_rel_to_S": float(err.max()),
            "median_rel_to_S": float(np.median(err)), "tolerance": 1e-5}


def algorithmic_bytes(kernel, dim):
    """HBM bytes per particle of one launch if every array were read or written exactly once
    (FP32 build; neighbour records served on chip):
      pressure pass: own record (offsets + h, meta), (v, h), own cell, a_p + V~ written;
      update: record, (v, h), a_p, stored cell + offset in, cell, offset, velocity, h, meta,
              index and next key out."""
    if kernel == "interact":
        return (16 if dim == 2 else 20) + 16 + 4 * dim + 16
    if kernel == "integrate":
        return (16 if dim == 2 else 20) + 16 + 16 + 8 * dim + (8 * dim + 4 * dim + 4 + 4 + 4 + 4)
    return 0


def roofline_of(run, n, peaks, peak_src, dim):
    """Roofline object of the dominant kernel from the live stage times of `run`: the pressure
    pass is bounded by the FP32 pipes (FLOP_PER_PAIR per interacting pair); its HBM fraction on
    algorithmic bytes is reported beside it."""
    stages = run["stages_ms"]
    dom = max(("interact", "integrate", "control"), key=lambda k: stages.get(k, 0.0))
    t_dom = stages[dom] / 1e3
    fp32_peak = SM_COUNT * FP32_LANES * 2 * SM_MAX_MHZ * 1e6 / 1e12       # TFLOP/s at the maximum SM clock
    achieved = FLOP_PER_PAIR * run["accd"] / t_dom / 1e12
    bpp = algorithmic_bytes(dom, dim)
    hbm_gbs = n * bpp / t_dom / 1e9
    return {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
            "frac": achieved / fp32_peak,
            "traffic": (DOMINANT_DRAM_BYTES_PER_PARTICLE * n
                        if (dom == "interact" and dim == 3 and DOMINANT_DRAM_BYTES_PER_PARTICLE) else None),
            "kernel": dom, "avg_launch_ms": stages[dom],
            "work": f"{FLOP_PER_PAIR:.0f} FP32 operations x {run['accd']} interacting pairs per launch",
            "peak_source": f"FP32: {SM_COUNT} SMs x {FP32_LANES} lanes x 2 x {SM_MAX_MHZ:.0f} MHz",
            "algorithmic_bytes_per_particle": bpp,
            "hbm_achieved_gbs": hbm_gbs, "hbm_peak_gbs": hbm_peak(peaks), "hbm_frac": hbm_gbs / hbm_peak(peaks),
            "hbm_peak_source": peak_src}


def mesh_quality_2d(w, x):
    """Quality of the Delaunay triangulation of final 2D positions with the measures of Sec. 4
    (G = 2 sqrt(3) S / (P H), angles); triangles whose centroid lies outside the domain are
    dropped.  Measurement only: the method never triangulates."""
    import math

    from scipy.spatial import Delaunay

    from paper_2003_01061_gb300 import workloads as WL

    tri = Delaunay(x[:, :2])
    P = x[tri.simplices][:, :, :2]
    cen = np.concatenate([P.mean(axis=1), np.zeros((len(P), 1))], axis=1)
    P = P[WL.domain_phi(w["domain"], cen) > 0]
    e = np.stack([np.linalg.norm(P[:, 1] - P[:, 2], axis=1), np.linalg.norm(P[:, 0] - P[:, 2], axis=1),
                  np.linalg.norm(P[:, 0] - P[:, 1], axis=1)], axis=1)
    u, v = P[:, 1] - P[:, 0], P[:, 2] - P[:, 0]
    area = 0.5 * np.abs(u[:, 0] * v[:, 1] - u[:, 1] * v[:, 0])
    G = 2 * math.sqrt(3) * area / (0.5 * e.sum(axis=1) * e.max(axis=1))
    ang = []
    for k in range(3):
        a, b, c = e[:, k], e[:, (k + 1) % 3], e[:, (k + 2) % 3]
        ang.append(np.degrees(np.arccos(np.clip((b * b + c * c - a * a) / (2 * b * c), -1, 1))))
    ang = np.stack(ang, 1)
    # radius ratio 2 r_in / r_circ (1 for the equilateral triangle)
    rr = 2.0 * (area / (0.5 * e.sum(axis=1))) / (e.prod(axis=1) / (4.0 * area))
    return {"G_avg": float(G.mean()), "G_min": float(G.min()), "theta_max": float(ang.max()),
            "theta_min": float(ang.min()), "theta_min_avg": float(ang.min(axis=1).mean()),
            "theta_lt30": int((ang.min(axis=1) < 30).sum()), "rr_min": float(rr.min()), "rr_avg": float(rr.mean()),
            "N_tri": int(len(P))}


def sampling_run(S, w, gen_s, with_oracle=True):
    """The initial particles of the 1.2M cube drawn on the device (Sec. 3.6: target counts of
    Eqs. 10, 11 + rho_t-proportional rejection sampling), host wall time including the copy of
    the positions to the host; beside it the host-side numpy generator of the benchmark inputs
    (Monte-Carlo counts + rejection sampling, in a worker process) and the oracle's sampler on
    a bounded sample of the volume particles (one core)."""
    d, z = S.domain_desc(w["domain"]), S.sizing_desc(w["sizing"])
    S.sph_feature_counts(d, z)                       # first use of the kernels (untimed)
    t0 = time.perf_counter()
    M, N = S.sph_feature_counts(d, z)
    t1 = time.perf_counter()
    x, g = S.sph_sample_particles(d, z, 1, N)
    t2 = time.perf_counter()
    n = int(N.sum())
    out = {"particles": n, "counts_s": t1 - t0, "sample_s": t2 - t1, "value": n / (t2 - t0),
           "unit": "particles/s", "numpy_generator_s": gen_s,
           "numpy_generator_particles": len(w["x"])}
    if with_oracle:
        from oracle import oracle as O

        O.build()
        m = 20_000
        t3 = time.perf_counter()
        O.sample_feature(w, 0, 1, m)
        dt = time.perf_counter() - t3
        out["oracle"] = {"value": m / dt, "unit": "particles/s", "cores": 1,
                         "sample": f"first {m} volume particles of the same problem and seed"}
    out["config"] = {"workload": "cube_sphere_3d_1.2M descriptors (seed 3): counts by the midpoint rule "
                                 "(256^3 volume cells), Philox4x32-10 seed 1"}
    return out


def mesh_quality_3d(w, x, within=None):
    """Quality of the Delaunay tetrahedralisation of final 3D positions with the measures of
    Sec. 4: dihedral angles and the radius ratio gamma = 3 r_in / r_circ; tetrahedra whose
    centroid lies outside the domain, and flat ones (volume below 1e-9 of the mean), are
    dropped.  within = (q, r): only the tetrahedra whose centroid lies within r of q are
    measured (for a patch of a large state, away from the patch's own hull).  Measurement
    only: the method never tetrahedralises."""
    from scipy.spatial import Delaunay

    from paper_2003_01061_gb300 import workloads as WL

    T = x[Delaunay(x).simplices]
    T = T[WL.domain_phi(w["domain"], T.mean(axis=1)) > 0]
    if within is not None:
        T = T[np.linalg.norm(T.mean(axis=1) - np.asarray(within[0]), axis=1) < within[1]]
    a, b, c = T[:, 1] - T[:, 0], T[:, 2] - T[:, 0], T[:, 3] - T[:, 0]
    trip = np.einsum("ij,ij->i", a, np.cross(b, c))
    vol = np.abs(trip) / 6.0
    keep = vol > 1e-9 * vol.mean()
    T, a, b, c, trip, vol = T[keep], a[keep], b[keep], c[keep], trip[keep], vol[keep]
    alpha = (np.einsum("ij,ij->i", a, a)[:, None] * np.cross(b, c) + np.einsum("ij,ij->i", b, b)[:, None] * np.cross(c, a)
             + np.einsum("ij,ij->i", c, c)[:, None] * np.cross(a, b))
    r_circ = np.linalg.norm(alpha, axis=1) / (2.0 * np.abs(trip))
    area = 0.0
    for f in ((1, 2, 3), (0, 2, 3), (0, 1, 3), (0, 1, 2)):
        area = area + 0.5 * np.linalg.norm(np.cross(T[:, f[1]] - T[:, f[0]], T[:, f[2]] - T[:, f[0]]), axis=1)
    gamma = 3.0 * (3.0 * vol / area) / r_circ
    dih = []
    for i, j, k, l in ((0, 1, 2, 3), (0, 2, 1, 3), (0, 3, 1, 2), (1, 2, 0, 3), (1, 3, 0, 2), (2, 3, 0, 1)):
        e = T[:, j] - T[:, i]
        e = e / np.linalg.norm(e, axis=1, keepdims=True)
        u, v = T[:, k] - T[:, i], T[:, l] - T[:, i]
        u = u - np.einsum("ij,ij->i", u, e)[:, None] * e
        v = v - np.einsum("ij,ij->i", v, e)[:, None] * e
        cosang = np.einsum("ij,ij->i", u, v) / (np.linalg.norm(u, axis=1) * np.linalg.norm(v, axis=1))
        dih.append(np.degrees(np.arccos(np.clip(cosang, -1, 1))))
    dih = np.stack(dih, 1)
    tmin = dih.min(axis=1)
    return {"theta_min": float(dih.min()), "theta_max": float(dih.max()), "gamma_min": float(gamma.min()),
            "gamma_avg": float(gamma.mean()), "theta_min_avg": float(tmin.mean()),
            "theta_lt10": int((tmin < 10).sum()), "theta_lt20": int((tmin < 20).sum()),
            "theta_lt30": int((tmin < 30).sum()), "theta_lt40": int((tmin < 40).sum()), "N_tet": int(len(T))}


def case_3d_run(S, w, table, iters):
    """A 3D case of Sec. 4 (the Cube of Eq. 28, Sphere01, Sphere02): the improved method and,
    where the paper's table has it, the earlier method (fu2019 preset) for the paper's iteration
    counts, from the same initial particles; the mesh quality of the final states beside the
    paper's table."""
    from paper_2003_01061_gb300 import workloads as WL

    out = {}
    for name, over in (("improved", {}), ("improved_threshold1e-2", {"threshold": 1e-2}), ("fu2019", {})):
        if name.split("_")[0] not in iters:
            continue
        m = S.Mesh(w, precision=32, params=dict(WL.method_preset(w["params"], name.split("_")[0]), **over))
        m.set_state()
        m.sync()
        t0 = time.perf_counter()
        ok, it = S.sph_mesh_run_until_converged(m.h, iters[name.split("_")[0]])
        wall = time.perf_counter() - t0
        r = m.report()
        out[name] = {"iters": int(it), "done": bool(ok), "wall_s": wall, "escapes": int(r.escapes),
                     "E_sys": float(r.E_sys), "phase": int(r.phase),
                     "quality": mesh_quality_3d(w, m.positions()["x"])}
        m.close()
    out["initial_quality"] = mesh_quality_3d(w, w["x"])
    with open(os.path.join(ROOT, "tests", "golden", "paper_cases.json")) as f:
        out["paper_table"] = json.load(f)[table]
    out["config"] = {"workload": f"{w['name']}: {len(w['x'])} particles, FP32, paper controller, "
                                 f"iterations as in the paper's table"}
    return out


def presets_run(S, w, max_iters):
    """The comparison of Sec. 4.1 (Square, Eq. 25): the same initial particles relaxed by the
    improved method and by the two presets of the earlier method, each until the end of
    Phase Two or max_iters steps.  Iterations to the Phase-One target (the start of the
    transition) and to the end, host wall time of the whole run."""
    from paper_2003_01061_gb300 import workloads as WL

    out = {}
    # the improved method also with Phase-One damping eps1 = 0.1 and 0.2 (Sec. 3.4.3 suggests
    # [0, 0.2] for ill-posed initial samplings; the earlier method has no damping)
    # and with a threshold the Phase-One oscillation reaches (1e-2), so that Phase Two runs
    runs = [("improved", "improved", {}), ("improved_eps0.1", "improved", {"eps1": 0.1}),
            ("improved_eps0.2", "improved", {"eps1": 0.2}), ("improved_threshold1e-2", "improved", {"threshold": 1e-2}),
            ("fu2019_v2", "fu2019_v2", {}), ("fu2019", "fu2019", {})]
    for label, name, over in runs:
        m = S.Mesh(w, precision=32, params=dict(WL.method_preset(w["params"], name), **over))
        m.set_state()
        m.sync()
        t0 = time.perf_counter()
        ok, iters = S.sph_mesh_run_until_converged(m.h, max_iters)
        wall = time.perf_counter() - t0
        r = m.report()
        phase_one = int(r.ramp_start) if r.phase in (S.RAMP, S.PHASE2, S.DONE) else None
        out[label] = {"phase_one_iters": phase_one, "iters": int(iters), "done": bool(ok), "wall_s": wall,
                      "escapes": int(r.escapes), "E_sys": float(r.E_sys),
                      "quality": mesh_quality_2d(w, m.positions()["x"])}
        m.close()
    out["initial_quality"] = mesh_quality_2d(w, w["x"])
    with open(os.path.join(ROOT, "tests", "golden", "paper_cases.json")) as f:
        out["paper_table"] = json.load(f)["square_table"]
    out["config"] = {"workload": f"square_radial_2d: [0,100]^2, Eq. 25 sizing (h 0.244-4.88), {len(w['x'])} "
                                 f"particles (seed 6), FP32, paper controller, max {max_iters} iterations"}
    return out


def batched_run(S, torch, dev, ws, steps):
    """All instances of each dimension in one batch; the two batches on two streams."""
    groups = [[w for w in ws if w["domain"]["D"] == d] for d in (2, 3)]
    streams = [torch.cuda.Stream(device=dev) for _ in groups]
    batches = []
    for g, st in zip(groups, streams):
        if not g:
            continue
        b = S.Batch(g, precision=32, stream=st.cuda_stream)
        for i in range(len(g)):
            b.set_state(i)
        # cell size chosen by the library's autotuner on the loaded state (untimed)
        b.tuned = S.sph_batch_autotune(b.h, 5)
        batches.append((b, st, sum(len(w["x"]) for w in g)))
    for b, _, _ in batches:
        b.step(3)
    for b, _, _ in batches:
        b.sync()
    torch.cuda.synchronize()
    start = torch.cuda.Event(enable_timing=True)
    start.record(torch.cuda.current_stream(dev))
    ends = []
    for b, st, _ in batches:
        st.wait_event(start)
    for b, st, _ in batches:
        b.step(steps)
    for b, st, _ in batches:
        e = torch.cuda.Event(enable_timing=True)
        e.record(st)
        ends.append(e)
    torch.cuda.synchronize()
    ms = max(start.elapsed_time(e) for e in ends)
    parts = sum(n for _, _, n in batches)
    out = {"value": parts * steps / (ms / 1e3), "unit": METRIC, "steps": steps, "ms_per_step": ms / steps,
           "instances": len(ws), "particles": parts,
           "per_dim": {}}
    # the per-stage split: a few more steps per batch with stage events (alone on the GPU)
    staged = min(steps, 20)
    for (b, _, n), d in zip(batches, (2, 3)):
        S.sph_batch_set_timing(b.h, 1)
        b.step(1)
        b.sync()
        S.sph_batch_set_timing(b.h, 1)
        b.step(staged)
        b.sync()
        t = S.sph_batch_kernel_times(b.h)
        _, slots, _ = S.sph_batch_size(b.h)
        out["per_dim"][f"{d}d"] = {"instances": b.n_inst, "particles": n, "slots": slots,
                                   "cells_per_support": b.tuned[0],
                                   "autotune_trial_ms": {"1": b.tuned[1][0], "2": b.tuned[1][1], "4": b.tuned[1][2]},
                                   "stages_ms": stages_per_step(t, staged),
                                   "stage_steps": staged}
        S.sph_batch_set_timing(b.h, 0)
        b.sync()
        b.close()
    return out


def serving_run(S, jobs, times, max_iters, threshold, precision=32, max_jobs=64, steps_per_poll=20):
    """Real-time arrivals into the server, every job given by its problem alone (its particles
    drawn on the device at admission, Sec. 3.6) with the paper's controller at `threshold`;
    jobs retire when their two-phase criterion converges (DONE) or at max_iters.  Per job:
    latency = finish - scheduled arrival, queueing = admission - scheduled arrival, service =
    finish - admission (all host clock)."""
    srv = S.Server(precision=precision, max_jobs=max_jobs, slot_capacity=(-1, -1), hbm_fraction=0.3,
                   steps_per_poll=steps_per_poll)
    prm = [dict(w["params"], threshold=threshold) for w in jobs]
    # warm the step graphs with one small job of each dimension (not counted)
    for D in sorted({w["domain"]["D"] for w in jobs}):
        i = next(i for i, w in enumerate(jobs) if w["domain"]["D"] == D)
        srv.submit_sampled(jobs[i], steps_per_poll, seed=12345, params=prm[i])
    srv.drain()
    ids, lag = [], []
    t0 = time.perf_counter()
    k = 0
    while True:
        now = time.perf_counter() - t0
        while k < len(jobs) and times[k] <= now:
            ids.append(srv.submit_sampled(jobs[k], max_iters, seed=k + 1, params=prm[k]))
            lag.append((time.perf_counter() - t0) - times[k])    # submission after the scheduled arrival
            k += 1
        st = srv.poll()
        if k == len(jobs) and st.running == 0 and st.queued == 0:
            break
        if st.running == 0 and st.queued == 0 and k < len(jobs):
            time.sleep(max(0.0, times[k] - (time.perf_counter() - t0)))
    wall = time.perf_counter() - t0
    lat, que, svc, work, iters, n_of, states = [], [], [], [], [], [], {}
    t_end = 0.0
    for i, jid in enumerate(ids):
        info, _ = srv.job(jid, with_result=False)
        lat.append(info.t_finish - info.t_submit + lag[i])
        que.append(info.t_admit - info.t_submit + lag[i])
        svc.append(info.t_finish - info.t_admit)
        work.append(float(info.n) * float(info.iterations))
        iters.append(int(info.iterations))
        n_of.append(int(info.n))
        states[int(info.state)] = states.get(int(info.state), 0) + 1
        t_end = max(t_end, times[i] + lat[-1])
    srv.close()
    lat, que, svc = np.array(lat), np.array(que), np.array(svc)
    pct = lambda a, q: float(np.percentile(a, q))
    return {"p50_s": pct(lat, 50), "p99_s": pct(lat, 99), "mean_s": float(lat.mean()),
            "queueing_p50_s": pct(que, 50), "queueing_p99_s": pct(que, 99),
            "service_p50_s": pct(svc, 50), "service_p99_s": pct(svc, 99),
            "value": float(sum(work)) / (t_end - times[0]), "unit": METRIC, "wall_s": wall, "jobs": len(jobs),
            "particle_steps": float(sum(work)), "mean_job_work": float(np.mean(work)),
            "iterations_p50": pct(np.array(iters), 50), "particles": n_of, "iterations": iters,
            "latency_s": lat.tolist(), "done": states.get(S.JOB_DONE, 0),
            "not_converged": states.get(S.JOB_NOT_CONVERGED, 0), "failed": states.get(S.JOB_FAILED, 0)}


def serving_legs(S, jobs, times, args):
    """cfg5: (1) the seeded Poisson stream at 50 jobs/s (first --serve-jobs arrivals), N
    log-uniform over 1k-2M, half 2D disks with holes / half 3D cubes minus a sphere; (2) the same
    job mix at 70 % of the capacity measured in (1); (3) the plain FP64 path serving one job at a
    time (a server with one slot, precision 64) on a subset of (1)'s arrivals, beside the FP32
    server's latencies for the same jobs in (1)."""
    thr, cap_it = args.serve_threshold, args.serve_iters
    out = serving_run(S, jobs, times, cap_it, thr)
    out["config"] = {"workload": f"first {len(jobs)} arrivals of a Poisson stream at 50 jobs/s (seed 5), 2D disks "
                                 f"with holes / 3D cubes minus a sphere with probability 1/2, n log-uniform "
                                 f"1k-{args.serve_max_n // 1000}k, particles drawn on the device at admission, "
                                 f"paper controller (sample every 20, window 10, ramp 200, reset period 100) with "
                                 f"threshold {thr:g}, at most {cap_it} iterations, 20 steps per scheduling round",
                     "threshold_reason": "the paper's 5e-6 is never reached under this build's readings of "
                                         "Eq. 24 and the integrator (see the design notes); at this threshold "
                                         "jobs retire on convergence"}
    # (2) the same mix at 70 % of the measured capacity
    cap = out["value"]
    rate70 = 0.7 * cap / out["mean_job_work"]
    k70 = min(args.serve_70_jobs, len(jobs))
    rng = np.random.default_rng(55)
    t70 = np.cumsum(rng.exponential(1.0 / rate70, k70)).tolist()
    r70 = serving_run(S, jobs[:k70], t70, cap_it, thr)
    r70["config"] = {"rate_jobs_per_s": rate70, "capacity_particle_steps_per_s": cap,
                     "workload": f"the first {k70} problems of (1), Poisson arrivals (seed 55) at 70 % of the "
                                 f"capacity measured in (1)"}
    out["at_70pct_capacity"] = r70
    # (3) the plain FP64 path, one job at a time, on a subset
    sub = [i for i, w in enumerate(jobs) if w.get("n_expected", 0) <= args.fp64_subset_max_n][:args.fp64_subset_jobs]
    if sub:
        r64 = serving_run(S, [jobs[i] for i in sub], [times[i] - times[sub[0]] for i in sub], cap_it, thr,
                          precision=64, max_jobs=1)
        r64["config"] = {"subset": f"arrivals {sub} of (1) (the first {len(sub)} with n <= "
                                   f"{args.fp64_subset_max_n}), same arrival times, one job at a time, FP64"}
        r64["fp32_server_same_jobs_in_the_mix"] = {
            "p50_s": float(np.percentile([out["latency_s"][i] for i in sub], 50)),
            "p99_s": float(np.percentile([out["latency_s"][i] for i in sub], 99))}
        # the same subset through the FP32 server alone (same arrivals, nothing else resident)
        r32 = serving_run(S, [jobs[i] for i in sub], [times[i] - times[sub[0]] for i in sub], cap_it, thr)
        r64["fp32_server_same_jobs_alone"] = {k: r32[k] for k in ("p50_s", "p99_s", "value", "done")}
        out["fp64_one_at_a_time"] = r64
    return out


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
