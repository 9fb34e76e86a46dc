"""Measurement: the FP64 oracle against the GPU path on the two 256^2 configurations --
the Gaussian charge bell (Sec. 6.2; fully periodic, single phase) and the leaky-dielectric
droplet (Sec. 7.1; walls, two phases) -- both at a fixed K = 10 potential sub-iterations
per step.  Prints one JSON object: the host (cores, CPU model), the oracle's MLUPS on one
thread over a bounded number of steps, and the GPU path's MLUPS over 1000 steps (CUDA
graph per step, inputs resident, device-timed with CUDA events).

    python tests/oracle_timing.py [--oracle-steps 20] [--gpu-steps 1000]

The oracle's time per step does not depend on the step index at a fixed K, so a short
sample gives its rate; the number of steps actually timed is part of the output.
"""
import argparse
import json
import os
import platform
import subprocess
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

K = 10


def configs(n):
    from paper_2407_01654_gb300 import workloads as wl
    p2, f2, _, _ = wl.gaussian_bell(n, poisson_fixed_iter=K)
    p3, f3, _ = wl.droplet(seed=0, N=n, poisson_fixed_iter=K)
    return {f"gaussian charge bell {n}x{n} (Sec. 6.2)": (p2, f2),
            f"leaky-dielectric droplet {n}x{n}, seed 0 (Sec. 7.1)": (p3, f3)}


def host_info():
    model = platform.processor() or ""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    return {"machine": platform.machine(), "cpu": model, "nproc": os.cpu_count()}


def time_oracle(p, f, steps):
    from oracle import ehd as orc
    sim = orc.Sim(dict(p))
    sim.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    sim.step(1)  # warm-up
    t0 = time.perf_counter()
    sim.step(steps)
    dt = time.perf_counter() - t0
    return p["nx"] * p["ny"] * steps / dt / 1e6, dt


def time_gpu(p, f, steps):
    import torch
    from paper_2407_01654_gb300 import ehd
    stream = torch.cuda.current_stream()
    sim = ehd.Sim(p, stream=stream)
    sim.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    sim.step(5)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    sim.step(steps, stats=False)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = t0.elapsed_time(t1)
    st = sim.read_stats()
    sim.close()
    if st["status"] not in (0, 4):
        raise RuntimeError(f"GPU steps failed with status {st['status']}")
    return p["nx"] * p["ny"] * steps / (ms * 1e-3) / 1e6


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--oracle-steps", type=int, default=20)
    ap.add_argument("--gpu-steps", type=int, default=1000)
    args = ap.parse_args()
    out = {"fixed_K": K, "host": host_info(), "configs": {}}
    gpu = False
    try:
        import torch
        gpu = torch.cuda.is_available()
    except ImportError:
        pass
    if gpu:
        from paper_2407_01654_gb300 import build
        build.build()
    for name, (p, f) in configs(args.n).items():
        mlups, dt = time_oracle(p, f, args.oracle_steps)
        row = {"oracle_mlups": mlups, "oracle_steps": args.oracle_steps,
               "oracle_seconds": dt, "oracle_threads": 1}
        if gpu:
            row["gpu_mlups"] = time_gpu(p, f, args.gpu_steps)
            row["gpu_steps"] = args.gpu_steps
        out["configs"][name] = row
        print(json.dumps({name: row}), file=sys.stderr, flush=True)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
