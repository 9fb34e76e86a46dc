"""Benchmark of the coupled EHD phase-field LB time step on GB300.

Workload: the reversed-electrowetting sessile drop on a 512 x 1024 lattice (periodic x,
electrode walls in y, drop radius 80, density / viscosity ratio 10, permittivity ratio
20, ramped wall potential, the paper's potential stopping rule at 1e-5), FP32 storage.
One benchmark step is one full coupled time step over every node (moments, the
potential sub-iteration loop to the tolerance, the fused g / l / f pass).  The run
starts mid-ramp (step 10000 of a 20000-step ramp) so the wall potential changes every
step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Metric: coupled-step MLUPS = nodes x steps / s / 1e6 (with K,
the mean number of potential sub-iterations per step).  N > 1 (torchrun): one
independent replica per GPU (the step does not shard), value summed over ranks with the
slowest rank's time.
"""
from __future__ import annotations

import argparse
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

from paper_2407_01654_gb300 import workloads as wl  # noqa: E402

METRIC = "coupled-step MLUPS"
UNIT = "MLUPS"
WORKLOAD = ("reversed-electrowetting sessile drop, 512x1024 lattice (r=80, rho/mu ratio 10, "
            "eps ratio 20, ramped potential), full coupled step, potential rule tol 1e-5")
# Steps the simulation makes before the warm-up (untimed): the seeded velocity and charge
# perturbation of the start state decays over the first steps, during which the potential
# loop needs several hundred sub-iterations per step; after it the sub-iteration count
# settles, so the timed window measures the workload's typical step whatever the requested
# window length.
SPINUP_STEPS = 300
# Fixed potential sub-iteration count of the like-for-like comparison with the CPU
# reference arm (the oracle's cost per step depends only on the number of sub-iterations,
# not on the state): the reference arm runs the oracle at this count, the GPU line reports
# its own throughput at this count next to the rule-driven value.
K_COMPARE = 5
# A second fixed count: the step's time at K_COMPARE and at K_HIGH sub-iterations gives the
# marginal cost of one sub-iteration and, with the profiled solve time, the solve's fixed
# cost (launch, loading the state, writing it back)
K_HIGH = 25
# The workload as both arms name it (identical in the GPU and the reference line).
CONFIG = {"workload": WORKLOAD, "nodes": 512 * 1024,
          "start": f"step 10000 of a 20000-step ramp, then {SPINUP_STEPS} untimed steps",
          "l2": "inputs larger than L2: the simulation state is about 175 MB and a step "
                "touches about 150 MB (L2 129 MB); steps run back to back, L2 not flushed"}
# algorithmic bytes per node (FP32 populations read once and written once per pass):
# coupled pass: 27 populations read + written (216 B) + 6 lagged quantities read + written
# (48 B) + the 8 converged potential populations its local field needs (32 B) + phi for
# the stencils (4 B, each value read once); potential sub-iteration: 8 populations read +
# written (64 B) + (a, q) read (8 B).
BYTES_COUPLED = 216 + 48 + 32 + 4
BYTES_POTENTIAL = 64 + 8
# FP32 operations per node and potential sub-iteration (collision: moments 18, eight
# relaxations with forcing and source 8 x 8; stream and stopping sums 14), counted from
# the kernel source with a fused multiply-add as 2
FLOPS_POTENTIAL = 96
# shared-memory bytes per node and potential sub-iteration of the on-chip loop: the 8
# post-collision populations stored (32 B) and the 8 streamed ones loaded (32 B); the ring
# and export band traffic on top of it is overhead, not counted
SMEM_BYTES_POTENTIAL = 64
# thread instructions per lattice node and potential sub-iteration of the two-step on-chip
# loop, the ring's redundant work included (ncu: 629.2 M warp instructions over 524 288
# nodes x 379 sub-iterations, profiles/k_poisson_resident_sessile512x1024.md); at four
# warp instructions per clock and SM they set the loop's issue floor
INSTR_POTENTIAL = 101.3
SM_MAX_MHZ = 2070.0


def workload(seed=0):
    p, f, info = wl.sessile_drop(seed=seed, start_step=10000)
    f = wl.perturbed(p, f, seed=seed + 1, u_amp=1e-3, q_amp=1e-4)
    return p, f, info


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# Kernel sources each kernel is built from; a recorded traffic figure is used only while
# the hash of these files is the one it was measured on.
KERNEL_FILES = {
    "k_poisson_resident": ("poisson_resident.cu", "ehd_internal.cuh"),
    "k_poisson_resident2": ("poisson_resident.cu", "ehd_internal.cuh"),
    "k_poisson_resident3": ("poisson_resident.cu", "ehd_internal.cuh"),
    "k_coupled": ("kernels.cu", "ehd_internal.cuh"),
    "k_poisson": ("poisson.cu", "ehd_internal.cuh"),
}
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# of the bench workload (summaries under profiles/, named for the kernel and workload)
RECORDED_TRAFFIC = {
    # one potential solve of the two-step loop (about 465 sub-iterations on the captured
    # spin-up step; the solve's DRAM traffic does not grow with them): 21.025 MB read,
    # 0.061 MB written
    "k_poisson_resident2": (21086208, "1c6301a0a7f42dfc"),
    # one coupled pass, caches flushed before the launch: 90.247 MB read, 16.017 MB written
    # back during the launch (the rest of its writes leave L2 later)
    "k_coupled": (106264064, "4546c81efd9134c5"),
}


def kernel_source_hash(kernel):
    h = hashlib.sha256()
    for name in KERNEL_FILES[kernel]:
        h.update(open(os.path.join(ROOT, "paper_2407_01654_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel):
    """DRAM bytes per launch from the recorded ncu capture, or None once the kernel's
    sources have changed since it was taken."""
    rec = RECORDED_TRAFFIC.get(kernel)
    if rec is None or rec[1] != kernel_source_hash(kernel):
        return None
    return rec[0]


class ClockSampler:
    """nvidia-smi clock / throttle samples while the timed region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index=0):
        self.idx = gpu_index
        self.proc = None
        # the raw samples are kept beside the run ($EHD_CLOCKS_DIR, else the temp folder)
        folder = os.environ.get("EHD_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(folder, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def count(self):
        """Samples written so far."""
        if self.proc is None or not os.path.exists(self.path):
            return 0
        self.fh.flush()
        n = 0
        for line in open(self.path):
            parts = line.split(",")
            if len(parts) >= 9:
                try:
                    float(parts[1])
                    n += 1
                except ValueError:
                    pass
        return n

    def keep_busy(self, work, target, limit_s=5.0):
        """Runs `work` (GPU work, synchronised) until `target` samples have been written or
        `limit_s` has passed: the samples then show the clocks under load."""
        import torch
        t0 = time.perf_counter()
        while self.proc is not None and self.count() < target and time.perf_counter() - t0 < limit_s:
            work()
            torch.cuda.synchronize()

    def summary(self):
        if self.proc is None or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"]}
        sms, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sms.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sms:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["no samples"]}
        return {"sm_mhz": float(np.median(sms)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sms)}


def reduce_max(value, device):
    """The largest `value` over the ranks of the default process group (the slowest rank's
    time); `device` is where the reduction tensor lives ("cuda" with NCCL, "cpu" with
    gloo)."""
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def oracle_steps(n_warm, n_timed):
    """The oracle (numpy FP64, elementwise operations, one thread) on the full workload
    lattice at K_COMPARE potential sub-iterations per step: n_warm untimed steps, then
    n_timed steps each timed on the host clock.  Returns the per-step seconds.  (The
    oracle's cost per step depends on the sub-iteration count, not on the state, so it
    starts from the workload's initial fields.)"""
    from oracle import ehd as orc
    p, f, _ = workload()
    sim = orc.Sim(dict(p, poisson_fixed_iter=K_COMPARE))
    sim.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    for _ in range(n_warm):
        sim.step(1)
    out = []
    for _ in range(n_timed):
        t0 = time.perf_counter()
        sim.step(1)
        out.append(time.perf_counter() - t0)
    return out


def cpu_threads():
    """Threads the oracle's numpy may use (its BLAS pool; the elementwise work is
    single-threaded)."""
    for var in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS"):
        if os.environ.get(var, "").isdigit():
            return int(os.environ[var])
    return 1


def cpu_baseline(n_timed=3):
    """The oracle as it stands on this host, a bounded sample: 3 full 512 x 1024 coupled
    steps at K_COMPARE sub-iterations after one untimed step (about 5 s on the GPU machine's
    host)."""
    secs = oracle_steps(1, n_timed)
    nodes = CONFIG["nodes"]
    v = nodes * len(secs) / sum(secs) / 1e6
    return {"value": v, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
            "poisson_iters_per_step": K_COMPARE,
            "sample": f"{n_timed} full 512x1024 coupled steps of the workload on the FP64 oracle "
                      f"(numpy, one thread) at {K_COMPARE} potential sub-iterations per step "
                      f"after one untimed step; {sum(secs) / len(secs):.2f} s per step",
            "seconds_per_step": sum(secs) / len(secs)}


def run_reference(args, rank, world):
    """The reference arm: the oracle on the host cores, on the GPU arm's workload and
    config, K_COMPARE sub-iterations per step, the requested warm-up and timed steps (each
    a real oracle step, timed on the host clock).  Under torchrun only rank 0 runs it."""
    if rank != 0:
        return
    secs = oracle_steps(args.warmup, args.steps)
    nodes = CONFIG["nodes"]
    total = sum(secs)
    v = nodes * args.steps / total / 1e6
    sample = (f"{args.steps} full 512x1024 coupled steps of the workload on the FP64 oracle "
              f"(numpy, one thread) at {K_COMPARE} potential sub-iterations per step after "
              f"{args.warmup} untimed steps")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": dict(CONFIG),
        "poisson_iters_mean": float(K_COMPARE),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": cpu_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_gpu(args, rank, world):
    import torch
    from paper_2407_01654_gb300 import build as ehd_build
    from paper_2407_01654_gb300 import ehd

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        ehd_build.build()
    if world > 1:
        torch.distributed.barrier()
    p, f, info = workload(seed=rank)
    nodes = p["nx"] * p["ny"]
    schedule = None
    if not args.no_tune:
        # launch schedule of the potential loop for this lattice shape (cached per device)
        from paper_2407_01654_gb300 import autotune
        schedule = autotune.tune(p, fields=f)
        p.update(schedule)
    stream = torch.cuda.current_stream()
    sim = ehd.Sim(p, stream=stream)
    sim.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    loop_kind = sim.loop_kind()
    resident = loop_kind in (2, 3, 4)
    rkernel = {3: "k_poisson_resident2", 4: "k_poisson_resident3"}.get(loop_kind, "k_poisson_resident")
    spin = sim.step(args.spinup)
    sim.step(args.warmup)
    # the state the timed steps start from: the per-kernel profile, the fixed-count
    # comparison and the end-to-end run below start from it too
    start_state = sim.save_state()

    def timed_steps(s, n):
        """n steps as step graphs, back to back, between two CUDA events on the stream the
        library uses (synchronised on both sides); returns the time in ms."""
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        s.step(n, stats=False)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1)

    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    # the timed region (K steps of well under 0.1 ms each) is shorter than one clock sample
    # interval, so the clocks are sampled while a copy of the simulation runs the same steps
    # right before and right after it
    load_sim = ehd.Sim(p, stream=stream)
    load_sim.load_state(start_state)
    with ClockSampler(dev) as clk:
        clk.keep_busy(lambda: load_sim.step(100, stats=False), 2)
        n_before = clk.count()
        step_ms = timed_steps(sim, args.steps)
        clk.keep_busy(lambda: load_sim.step(100, stats=False), n_before + 2)
    load_sim.close()
    wall = time.perf_counter() - wall0
    st = sim.read_stats()
    if st["status"] not in (0, 4):
        raise RuntimeError(f"timed steps failed with status {st['status']}")
    kt_total = st["poisson_iters_total"]
    launches = st["kernel_launches"]
    # per-kernel device times: the same steps again from the same state, with CUDA events
    # around every launch (the same kernels, queued from the host instead of a graph)
    sim.load_state(start_state)
    sim.profile(True)
    sim.step(args.steps, stats=False)
    prof = sim.profile_read()
    sim.profile(False)
    pst = sim.read_stats()
    prof_iters = pst["poisson_iters_total"]
    if prof_iters != kt_total:
        raise RuntimeError(f"profiled replay made {prof_iters} sub-iterations, timed steps "
                           f"{kt_total}")
    t_local = step_ms / 1e3
    t_max = reduce_max(t_local, "cuda") if world > 1 else t_local
    value = world * nodes * args.steps / t_max / 1e6
    kbar = kt_total / args.steps
    # the same steps with a fixed number of potential sub-iterations per step (the count the
    # reference arm runs the oracle at): a like-for-like throughput against that arm
    simk = ehd.Sim(dict(p, poisson_fixed_iter=K_COMPARE), stream=stream)
    simk.load_state(start_state)
    simk.step(2)
    simk.load_state(start_state)
    torch.cuda.synchronize()
    fixed_ms = timed_steps(simk, args.steps)
    stk = simk.read_stats()
    simk.close()
    fixed_k = {"poisson_iters_per_step": K_COMPARE,
               "value": nodes * args.steps / (fixed_ms / 1e3) / 1e6, "unit": UNIT,
               "ms_per_step": fixed_ms / args.steps,
               "sub_iterations": stk["poisson_iters_total"]}
    simh = ehd.Sim(dict(p, poisson_fixed_iter=K_HIGH), stream=stream)
    simh.load_state(start_state)
    simh.step(2)
    simh.load_state(start_state)
    torch.cuda.synchronize()
    high_ms = timed_steps(simh, args.steps)
    simh.close()
    # marginal cost of one sub-iteration inside the step (us)
    marginal_us = (high_ms - fixed_ms) / args.steps / (K_HIGH - K_COMPARE) * 1e3
    # e2e through the C ABI with host buffers, the same window: the start state loaded
    # from pinned host memory (ehd_load_state), the steps, all fields read back to host
    # arrays (ehd_read_fields, float32 copies converted to double).  The output arrays are
    # the caller's, allocated once before the window and reused, as the C ABI's
    # caller-owned output buffers allow (a fresh array per read would time the host's
    # first touch of its pages, not the library)
    e2e = None
    if rank == 0 and not args.no_e2e:
        pinned = torch.frombuffer(bytearray(start_state), dtype=torch.uint8).pin_memory()
        sim2 = ehd.Sim(p, stream=stream)
        sim2.load_state(pinned)
        sim2.step(2)
        bufs = {n: np.zeros((p["ny"], p["nx"])) for n in ehd.FIELDS}
        sim2.read_fields(out=bufs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2.load_state(pinned)
        st2 = sim2.step(args.steps)
        out = sim2.read_fields(out=bufs)
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        sim2.close()
        h2d = pinned.numel()
        d2h = len(out) * 4 * nodes + 80
        e2e = {"value": nodes * args.steps / te / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "what": "ehd_load_state(pinned host blob of the start state) + ehd_step(K) + "
                       f"ehd_read_fields(host double, {len(out)} fields; float32 copies) into "
                       "caller-owned arrays reused from read to read",
               "poisson_iters_mean": st2["poisson_iters_total"] / args.steps}
        assert np.isfinite(out["phi"]).all()

    # the same workload with the moving populations stored as FP16 deviations (a second
    # figure, one GPU only; the headline is FP32): the schedule tuned for that storage, its
    # own spin-up from the same start fields, a window of the same length
    fp16 = None
    if world == 1 and not args.no_fp16:
        p16 = dict(p, precision=1)
        if not args.no_tune:
            p16.update(autotune.tune(p16, fields=f))
        s16 = ehd.Sim(p16, stream=stream)
        s16.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
        s16.step(args.spinup)
        s16.step(args.warmup)
        ms16 = timed_steps(s16, args.steps)
        st16 = s16.read_stats()
        s16.close()
        if st16["status"] not in (0, 4):
            raise RuntimeError(f"FP16-storage steps failed with status {st16['status']}")
        fp16 = {"value": nodes * args.steps / (ms16 / 1e3) / 1e6, "unit": UNIT,
                "ms_per_step": ms16 / args.steps,
                "poisson_iters_mean": st16["poisson_iters_total"] / args.steps,
                "storage": "24 moving populations as FP16 deviations from the lattice "
                           "weights, rest populations, potential populations and arithmetic "
                           "FP32",
                "schedule": ({k: p16[k] for k in ("poisson_loop", "tile_rows")}
                             if not args.no_tune else "built-in")}

    if rank != 0:
        return
    peak, peak_kind = peaks()
    props = torch.cuda.get_device_properties(dev)
    # FP32 rate: SMs x 128 lanes x 2 (a multiply-add) x the maximum SM clock
    fp32_peak = props.multi_processor_count * 128 * 2 * SM_MAX_MHZ * 1e6 / 1e12
    nodes_f = float(nodes)
    kinds = {}
    for k in ("moments", "potential", "coupled"):
        d = prof[k]
        kinds[k] = {"ms_total": d["ms"], "launches": d["launches"],
                    "us_per_launch": d["ms"] / max(d["launches"], 1) * 1e3}
    kinds["potential"]["sub_iterations"] = prof_iters
    kinds["potential"]["us_per_sub_iteration"] = prof["potential"]["ms"] / max(prof_iters, 1) * 1e3
    kinds["potential_idle"] = {"ms_total": prof["potential_idle"]["ms"],
                               "launches": prof["potential_idle"]["launches"]}
    dom = max(("moments", "potential", "coupled"), key=lambda k: kinds[k]["ms_total"])
    # the coupled pass streams populations through HBM: its roofline is the HBM copy rate
    tc = kinds["coupled"]["us_per_launch"] * 1e-6
    roof_coupled = {"bound": "hbm", "kernel": "k_coupled", "achieved": BYTES_COUPLED * nodes_f / tc / 1e9,
                    "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs (copy)", "unit": "GB/s",
                    "frac": BYTES_COUPLED * nodes_f / tc / 1e9 / peak,
                    "traffic": recorded_traffic("k_coupled"), "bytes_per_node": BYTES_COUPLED,
                    "launch_us": tc * 1e6}
    t_it = kinds["potential"]["us_per_sub_iteration"] * 1e-6
    if resident:
        # on-chip loop: its per-node data movement is through shared memory (each
        # sub-iteration stores the 8 post-collision populations and loads the 8 streamed
        # ones), against the shared-memory bandwidth measured live on this GPU
        smem_peak = ehd.smem_bandwidth(stream.cuda_stream) / 1e9
        ach = SMEM_BYTES_POTENTIAL * nodes_f / t_it / 1e9
        roof_pot = {"bound": "smem", "kernel": rkernel, "achieved": ach, "peak": smem_peak,
                    "peak_kind": "measured live: ehd_diag_smem_bandwidth (loads + stores, all "
                                 "SMs)", "unit": "GB/s", "frac": ach / smem_peak,
                    "traffic": recorded_traffic(rkernel),
                    "traffic_is": "DRAM bytes per launch (one solve), ncu",
                    "bytes_per_node_iteration": SMEM_BYTES_POTENTIAL,
                    "sub_iteration_us": t_it * 1e6,
                    "sub_iterations_per_launch": prof_iters / max(kinds["potential"]["launches"], 1),
                    "launch_us": kinds["potential"]["us_per_launch"],
                    "hbm_streamed_equivalent": {
                        "bytes_per_node_iteration": BYTES_POTENTIAL,
                        "GBps": BYTES_POTENTIAL * nodes_f / t_it / 1e9,
                        "frac_of_copy_peak": BYTES_POTENTIAL * nodes_f / t_it / 1e9 / peak},
                    "fp32": {"flops_per_node_iteration": FLOPS_POTENTIAL,
                             "TFLOPs": FLOPS_POTENTIAL * nodes_f / t_it / 1e12,
                             "frac_of_derived_peak": FLOPS_POTENTIAL * nodes_f / t_it / 1e12 /
                             fp32_peak}}
        # per launch at the window's K the solve's fixed part (launch, loading h and the
        # coefficients, writing h back) weighs heavily; the marginal sub-iteration is the
        # loop's own rate
        mb = SMEM_BYTES_POTENTIAL * nodes_f / (marginal_us * 1e-6) / 1e9
        roof_pot["marginal"] = {
            "what": f"(step time at K={K_HIGH} - at K={K_COMPARE}) / {K_HIGH - K_COMPARE}, "
                    "fixed sub-iteration counts, the same state",
            "sub_iteration_us": marginal_us, "achieved": mb, "frac": mb / smem_peak,
            "hbm_streamed_equivalent_frac":
                BYTES_POTENTIAL * nodes_f / (marginal_us * 1e-6) / 1e9 / peak,
            "solve_fixed_us": kinds["potential"]["us_per_launch"] - kbar * marginal_us}
        if loop_kind == 3:
            # a cycle (two sub-iterations) of the two-step loop with its exchange alone:
            # band export, grid barrier, ring import, no arithmetic
            try:
                floor_us = ehd.grid_exchange_floor(p["nx"], p["ny"], stream.cuda_stream) * 1e6
                # instruction issue of a cycle on the busiest SM at the maximum SM clock
                nodes_per_sm = nodes_f / props.multi_processor_count
                issue_us = 2 * nodes_per_sm * INSTR_POTENTIAL / 32 / 4 / (SM_MAX_MHZ * 1e6) * 1e6
                roof_pot["sync_floor"] = {
                    "what": "ehd_diag_grid_exchange: the two-step loop's exchange without its "
                            "arithmetic (64x56 tiles, 896 threads, one cooperative launch)",
                    "us_per_cycle": floor_us, "cycle_us": 2 * marginal_us,
                    "frac_of_cycle": floor_us / (2 * marginal_us),
                    "issue_us_per_cycle": issue_us,
                    "design_floor_us_per_cycle": floor_us + issue_us,
                    "design_frac": (floor_us + issue_us) / (2 * marginal_us),
                    "design_floor_is": "the measured exchange plus the issue of "
                                       f"{INSTR_POTENTIAL} instructions per node and "
                                       "sub-iteration at 4 warp instructions per clock and SM"}
            except ehd.EhdError as e:
                roof_pot["sync_floor"] = {"unavailable": str(e)}
    else:
        roof_pot = {"bound": "hbm", "kernel": "k_poisson", "achieved": BYTES_POTENTIAL * nodes_f / t_it / 1e9,
                    "peak": peak, "peak_kind": f"{peak_kind} hbm_gbs (copy)", "unit": "GB/s",
                    "frac": BYTES_POTENTIAL * nodes_f / t_it / 1e9 / peak,
                    "traffic": recorded_traffic("k_poisson"), "bytes_per_node": BYTES_POTENTIAL,
                    "launch_us": t_it * 1e6}
    roof = roof_pot if dom == "potential" else roof_coupled
    # whole-step fraction with the method's algorithmic bytes B(K) per node
    step_bytes = BYTES_COUPLED + BYTES_POTENTIAL * kbar
    step_frac = value / world * 1e6 * step_bytes / (peak * 1e9)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": dict(CONFIG, start=f"step 10000 of a 20000-step ramp, then {args.spinup} "
                                    f"untimed steps"),
        "poisson_iters_mean": kbar,
        "run": {"parallelism": f"replicas x{world}", "contact_angle_deg": round(info["theta"], 2),
                "storage": "fp32 SoA populations",
                "spinup_poisson_iters_mean": spin["poisson_iters_total"] / max(args.spinup, 1),
                "potential_loop": {1: "streaming (one launch per sub-iteration, graph WHILE node)",
                                   2: "on chip (one cooperative launch per step)",
                                   3: "on chip, two sub-iterations per halo exchange (one "
                                      "cooperative launch per step)",
                                   4: "on chip, three sub-iterations per halo exchange (one "
                                      "cooperative launch per step)"}[loop_kind],
                "schedule": dict(schedule, autotuned=True) if schedule else "built-in",
                "device": {"name": props.name, "sms": props.multi_processor_count},
                "step_algorithmic_bytes_per_node": step_bytes,
                "step_hbm_roofline_frac": step_frac, "wall_s": wall},
        "roofline": roof,
        "roofline_hbm_kernel": roof_coupled,
        "fixed_k": fixed_k,
        "kernels": kinds,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    if fp16 is not None:
        line["fp16_storage"] = fp16
    line["clocks"] = clk.summary()
    line["clocks"]["window"] = ("nvidia-smi every 50 ms while a copy of the simulation ran the "
                                "same steps right before and right after the timed region")
    if world == 1 and not args.no_serve:
        line["serving"] = run_serving()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)


SERVE_CAPACITY = ("32 droplet-deformation requests (Sec. 7.1 set-up, the C5 mix of grids "
                  "64^2/128^2/256^2/512^2 with r = 0.156 N, (R, S, Ca_E) seeded as for the 256^2 "
                  "droplet), all arriving at once, each run for 3000 steps (droplets do not reach "
                  "the 1e-6 steadiness rule within practical caps: after 30 000 steps phi still "
                  "changes by about 1e-4 per 500 steps), 2 GB device-memory budget")
SERVE_STEADY = ("24 two-layer planar requests (Sec. 6.1 set-up, 4 x {32, 48, 64}, permittivity "
                "ratio log-uniform [2, 20], conductivity ratio log-uniform [0.05, 0.5], FP32), "
                "Poisson arrivals, steady when the relative change of phi and of u over a "
                "500-step window is below 1e-6 (u below 1e-6 lattice units counts as rest), "
                "capped at 60 000 steps; differs from C5 in the request type (planar layers "
                "instead of droplets, which do not become steady) and in the count (24, not 256)")


def serve_arm(backend, reqs, window):
    from paper_2407_01654_gb300 import serve
    serve.warm_up(backend)
    clock = serve.WallClock()
    done = serve.serve(backend, reqs, clock, window=window)
    summ = serve.summarize(done, clock.now())
    keys = ("requests", "steady", "capped", "wall_s", "sims_per_hour", "p50_latency_s",
            "p99_latency_s", "p50_admit_to_end_s", "p99_admit_to_end_s",
            "p50_admit_to_steady_s", "p99_admit_to_steady_s",
            "poisson_iters_per_step", "steps_total")
    return {k: summ[k] for k in keys}


def run_serving():
    """Continuous batching against one-at-a-time runs of the same requests on the same GPU.

    Arms: the batch with every request in FP32 (the equal-accuracy comparison); one at a
    time on the plain path (FP32, streaming potential loop, kernels queued from the host
    without graphs); one at a time on the library's best single-simulation path (FP32,
    on-chip loop, one graph per step); and, as a second figure, the batch with half the
    requests in FP16-deviation storage.  Two workloads: droplet requests for capacity
    (sims/hour of fixed-length requests) and planar-layer requests that become steady
    (time from admission to steady state)."""
    from paper_2407_01654_gb300 import autotune, ehd, serve
    out = {"capacity_workload": SERVE_CAPACITY, "steady_workload": SERVE_STEADY}

    def batch(cap, tol, schedule):
        b = ehd.Batch(2 << 30, max_slots=64, steady_tol=tol, step_cap=cap)
        b.set_schedule(**schedule)
        return b

    sample = [(r.params, r.fields) for r in
              serve.make_requests(8, seed=99, sizes=(64, 128, 256, 512), rate=0.0,
                                  fp16_fraction=0.0)]
    sched = autotune.tune_batch(sample)
    out["batch_schedule"] = dict(sched, autotuned=True)
    cap = {}
    for arm in ("batched_fp32", "batched_fp16_mix", "one_at_a_time_best", "one_at_a_time_plain"):
        reqs = serve.make_requests(32, seed=0, sizes=(64, 128, 256, 512), rate=0.0,
                                   fp16_fraction=0.5 if arm == "batched_fp16_mix" else 0.0)
        if arm.startswith("batched"):
            backend = batch(3000, 1e-12, sched)
        else:
            backend = serve.OneAtATime(1e-12, 3000, plain=arm.endswith("plain"))
        cap[arm] = serve_arm(backend, reqs, 500)
        if arm.startswith("batched"):
            cap[arm]["kernel_launches"] = backend.info()["kernel_launches"]
            backend.close()
    plain = cap["one_at_a_time_plain"]["sims_per_hour"]
    cap["ratio_batched_fp32_vs_plain"] = cap["batched_fp32"]["sims_per_hour"] / plain
    cap["ratio_batched_fp32_vs_best_single"] = (cap["batched_fp32"]["sims_per_hour"] /
                                                cap["one_at_a_time_best"]["sims_per_hour"])
    cap["ratio_batched_fp16_mix_vs_plain"] = cap["batched_fp16_mix"]["sims_per_hour"] / plain
    out["capacity"] = cap
    steady = {}
    for arm in ("batched_fp32", "one_at_a_time_plain"):
        reqs = serve.make_planar_requests(24, seed=1, rate=20.0)
        if arm == "batched_fp32":
            backend = batch(60000, 1e-6, {"tile_rows": 32, "steps_per_graph": 16})
        else:
            backend = serve.OneAtATime(1e-6, 60000, plain=True)
        steady[arm] = serve_arm(backend, reqs, 500)
        if arm == "batched_fp32":
            backend.close()
    steady["ratio_batched_fp32_vs_plain"] = (steady["batched_fp32"]["sims_per_hour"] /
                                             steady["one_at_a_time_plain"]["sims_per_hour"])
    out["steady"] = steady
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-fp16", action="store_true",
                    help="skip the second figure with FP16-deviation population storage")
    ap.add_argument("--spinup", type=int, default=SPINUP_STEPS,
                    help="untimed steps before the warm-up (the workload's start state); "
                         "profiling captures use fewer to keep the launches before them few")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if world > 1:
        import torch
        backend = "nccl" if args.impl == "gb300" else "gloo"
        if args.impl == "gb300":
            torch.cuda.set_device(int(os.environ.get("LOCAL_RANK", "0")))
        torch.distributed.init_process_group(backend)
    try:
        if args.impl == "reference":
            run_reference(args, rank, world)
        else:
            run_gpu(args, rank, world)
    finally:
        if world > 1:
            import torch
            torch.distributed.barrier()
            torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
