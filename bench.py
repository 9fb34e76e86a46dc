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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2407_01654_gb300 import workloads as wl  # noqa: E402

METRIC = "coupled-step MLUPS"
UNIT = "MLUPS"
WORKLOAD = ("reversed-electrowetting sessile drop, 512x1024 lattice (r=80, rho/mu ratio 10, "
            "eps ratio 20, ramped potential), full coupled step, potential rule tol 1e-5")
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
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
L2_FLUSH_BYTES = 512 << 20


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
    # one potential solve of the two-step loop (280 sub-iterations on the captured step):
    # 21.030 MB read, 0.076 MB written
    "k_poisson_resident2": (21106176, "419d0b415696813c"),
    # one coupled pass: 88.137 MB read, 20.969 MB written back during the launch (the
    # rest of its writes leave L2 later)
    "k_coupled": (109106688, "3bcd59efcd78de5f"),
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
        self.path = os.path.join(ROOT, "gpurun_out", f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
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


# Mean potential sub-iterations per step of this workload with the paper's stopping rule
# over the default benchmark window (20 warm-up steps, then 200 timed steps from step
# 10000), measured on the GPU; the reference arm scales the oracle's per-sub-iteration cost
# to it (the GPU arm's own cpu_baseline uses the K of its run).
WORKLOAD_K = 117.52


def reduce_max(value, device):
    """The largest `value` over the ranks of the default process group (the slowest rank's
    time); `device` is where the reduction tensor lives ("cuda" with NCCL, "cpu" with
    gloo)."""
    import torch
    t = torch.tensor([float(value)], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def oracle_step_costs(k1=4, k2=12):
    """One full coupled step of the workload on the oracle at k1 and at k2 fixed potential
    sub-iterations: returns (seconds of the single-pass parts, seconds per sub-iteration).
    The oracle is numpy FP64 with elementwise operations only (one thread)."""
    from oracle import ehd as orc
    p, f, _ = workload()
    sim = orc.Sim(dict(p, poisson_fixed_iter=1))
    sim.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    sim.P.poisson_fixed_iter = k1
    t0 = time.perf_counter()
    sim.step(1)
    t1 = time.perf_counter() - t0
    sim.P.poisson_fixed_iter = k2
    t0 = time.perf_counter()
    sim.step(1)
    t2 = time.perf_counter() - t0
    t_iter = max((t2 - t1) / (k2 - k1), 0.0)
    return max(t1 - k1 * t_iter, 0.0), t_iter


def cpu_baseline(kbar):
    t_pass, t_iter = oracle_step_costs()
    p, _, _ = workload()
    nodes = p["nx"] * p["ny"]
    step = t_pass + kbar * t_iter
    return {"value": nodes / step / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"one full 512x1024 coupled step at 4 and one at 12 fixed potential "
                      f"sub-iterations (numpy FP64, one thread): {t_pass:.2f} s of single-pass "
                      f"work + {t_iter * 1e3:.1f} ms per sub-iteration, scaled to this run's "
                      f"mean of {kbar:.1f} sub-iterations per step",
            "seconds_per_step": step}


def run_reference(args, rank, world):
    if rank != 0:
        return
    # warm-up: one step's worth of oracle work, not timed
    if args.warmup > 0:
        oracle_step_costs(1, 2)
    n = max(1, min(args.steps, 3))
    steps_s = []
    for _ in range(n):
        t_pass, t_iter = oracle_step_costs()
        steps_s.append(t_pass + WORKLOAD_K * t_iter)
    p, _, _ = workload()
    nodes = p["nx"] * p["ny"]
    step = float(np.mean(steps_s))
    v = nodes / step / 1e6
    sample = (f"{n} samples of one full 512x1024 coupled step at 4 and at 12 fixed potential "
              f"sub-iterations each (numpy FP64, one thread), scaled to the workload's mean of "
              f"{WORKLOAD_K} sub-iterations per step (requested {args.steps} steps / "
              f"{args.warmup} warm-up)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": world,
        "steps": n, "warmup": min(args.warmup, 1), "ms_per_step": step * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "nodes": nodes, "poisson_iters_mean": WORKLOAD_K,
                   "l2": "n/a (CPU)"},
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
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
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sim.step(args.warmup)
    # the state the timed steps start from: the per-kernel profile below replays exactly
    # these steps (same sub-iteration counts)
    start_state = sim.save_state()

    # timed region: K steps as step graphs, L2 flushed before each, CUDA events around
    # each step on the stream the library uses
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    wall0 = time.perf_counter()
    with ClockSampler(dev) as clk:
        for j in range(args.steps):
            flush.fill_(j & 0xff)
            starts[j].record(stream)
            sim.step(1, stats=False)
            ends[j].record(stream)
        torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    st = sim.read_stats()
    if st["status"] not in (0, 4):
        raise RuntimeError(f"timed steps failed with status {st['status']}")
    kt_total = st["poisson_iters_total"]
    launches = st["kernel_launches"]
    step_ms = sum(s.elapsed_time(e) for s, e in zip(starts, ends))
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
    # e2e through the C ABI with host buffers: set_fields (host -> device), the same
    # number of steps, read all fields back to the host
    e2e = None
    if rank == 0 and not args.no_e2e:
        host = {k: np.ascontiguousarray(v, dtype=np.float64) for k, v in f.items()}
        sim2 = ehd.Sim(p, stream=stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sim2.set_fields(host["phi"], host["q"], host["ux"], host["uy"])
        st2 = sim2.step(args.steps)
        out = sim2.read_fields()
        torch.cuda.synchronize()
        te = time.perf_counter() - t0
        sim2.close()
        h2d = 4 * 4 * nodes
        d2h = 8 * 4 * nodes + 80
        e2e = {"value": nodes * args.steps / te / 1e6, "unit": UNIT,
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "what": "ehd_set_fields(host double) + ehd_step(K) + ehd_read_fields(host double, "
                       "8 fields); float32 copies",
               # these steps start from the fresh state (the timed steps above start after
               # the warm-up), so their mean sub-iteration count is higher
               "poisson_iters_mean": st2["poisson_iters_total"] / args.steps}
        assert np.isfinite(out["phi"]).all()

    if rank != 0:
        return
    peak, peak_kind = peaks()
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
        # on-chip loop: FP32 arithmetic per node and sub-iteration against the FP32 rate
        fl = FLOPS_POTENTIAL * nodes_f / t_it / 1e12
        roof_pot = {"bound": "alu", "kernel": rkernel, "achieved": fl,
                    "peak": FP32_PEAK_TFLOPS, "peak_kind": "derived: 152 SMs x 128 FP32 lanes x "
                    "2 flop x 2.07 GHz", "unit": "TFLOP/s", "frac": fl / FP32_PEAK_TFLOPS,
                    "traffic": recorded_traffic(rkernel),
                    "flops_per_node_iteration": FLOPS_POTENTIAL,
                    "sub_iteration_us": t_it * 1e6,
                    "streamed_equivalent_GBps": BYTES_POTENTIAL * nodes_f / t_it / 1e9}
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
        "config": {"workload": WORKLOAD, "nodes": nodes, "parallelism": f"replicas x{world}",
                   "poisson_iters_mean": kbar, "contact_angle_deg": round(info["theta"], 2),
                   "storage": "fp32 SoA populations",
                   "potential_loop": {1: "streaming (one launch per sub-iteration, graph WHILE node)",
                                      2: "resident (on chip, one cooperative launch per step)",
                                      3: "resident, two sub-iterations per halo exchange (on chip, "
                                         "one cooperative launch per step)",
                                      4: "resident, three sub-iterations per halo exchange (on chip, "
                                         "one cooperative launch per step)"}[loop_kind],
                   "schedule": dict(schedule, autotuned=True) if schedule else "built-in",
                   "l2": "flushed between timed steps (512 MiB device write outside the events)",
                   "step_algorithmic_bytes_per_node": step_bytes,
                   "step_hbm_roofline_frac": step_frac, "wall_s": wall},
        "roofline": roof,
        "roofline_hbm_kernel": roof_coupled,
        "kernels": kinds,
        "gpu_launches": launches,
        "e2e": e2e,
    }
    line["clocks"] = clk.summary()
    if world == 1 and not args.no_serve:
        line["serving"] = run_serving()
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(kbar)
    print(json.dumps(line), flush=True)


SERVE_WORKLOAD = ("32 droplet-deformation requests (Sec. 7.1 set-up), grids drawn from "
                  "64^2/128^2/256^2/512^2 with r = 0.156 N, (R, S, Ca_E) seeded as for the "
                  "256^2 droplet, half with FP16-deviation storage in the batched arm; "
                  "arrivals 50/s (above both arms' capacity, so sims/hour is service "
                  "capacity); steady when the relative change of phi and u over 500 steps "
                  "is < 1e-6, capped at 3000 steps; 2 GB device-memory budget")


def run_serving():
    """Continuous-batching serving against one-at-a-time plain FP32 runs of the same
    requests on the same GPU (each arm warmed up before its clock starts)."""
    from paper_2407_01654_gb300 import ehd, serve
    out = {"workload": SERVE_WORKLOAD}
    for arm in ("batched", "one_at_a_time_plain"):
        reqs = serve.make_requests(32, seed=0, sizes=(64, 128, 256, 512), rate=50.0)
        if arm == "batched":
            from paper_2407_01654_gb300 import autotune
            sample = [(r.params, r.fields) for r in
                      serve.make_requests(8, seed=99, sizes=(64, 128, 256, 512), rate=0.0)]
            schedule = autotune.tune_batch(sample)
            out["batch_schedule"] = dict(schedule, autotuned=True)
            backend = ehd.Batch(2 << 30, max_slots=64, steady_tol=1e-6, step_cap=3000)
            backend.set_schedule(**schedule)
        else:
            backend = serve.OneAtATime(1e-6, 3000)
        serve.warm_up(backend)
        clock = serve.WallClock()
        done = serve.serve(backend, reqs, clock, window=500)
        summ = serve.summarize(done, clock.now())
        out[arm] = {k: summ[k] for k in ("requests", "steady", "capped", "wall_s", "sims_per_hour",
                                         "p50_latency_s", "p99_latency_s",
                                         "poisson_iters_per_step")}
        if arm == "batched":
            out[arm]["kernel_launches"] = backend.info()["kernel_launches"]
            backend.close()
    out["sims_per_hour_ratio"] = (out["batched"]["sims_per_hour"] /
                                  out["one_at_a_time_plain"]["sims_per_hour"])
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
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
