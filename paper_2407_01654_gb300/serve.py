"""Serving loop: simulation requests arrive over time, are admitted into a batch of
resident simulations as slots and device memory free up, advance together, and leave when
steady (or at the step cap).  Continuous batching: a request that arrives while others are
running is admitted at the next window boundary if it fits, without waiting for the batch
to drain.

The scheduler talks to a backend with four calls -- admit(params, fields, id) -> slot or
None, run(nsteps), poll() -> [slot status], retire(slot) -- and reads time from a clock,
so the policy can be exercised on the CPU with a fake backend and a fake clock.

    python -m paper_2407_01654_gb300.serve --requests 48 --budget-gb 2
"""
from __future__ import annotations

import argparse
import heapq
import json
import math
import time
from dataclasses import dataclass, field

import numpy as np

from . import workloads as wl


@dataclass
class Request:
    id: int
    arrival: float              # seconds after the start of the run
    params: dict
    fields: dict
    admitted: float = math.nan
    finished: float = math.nan
    steps: int = 0
    iters: int = 0
    steady: bool = False
    capped: bool = False
    failed: str = ""            # why the request ended without a result ("" if it did not)
    rel_change: tuple = (math.nan, math.nan)


def make_requests(n, seed=0, sizes=(64, 128, 256, 512), rate=1.0, fp16_fraction=0.5):
    """Droplet-deformation requests (Sec. 7.1 set-up): grid drawn uniformly from `sizes`
    with r = 0.156 N, (R, S, Ca_E) seeded as for the single-droplet workload, half of them
    with FP16-deviation storage; Poisson arrivals at `rate` per second."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        N = int(rng.choice(sizes))
        R, S, Ca = wl.droplet_ratios(seed * 100003 + i)
        p, f, _ = wl.droplet(N=N, r=0.156 * N, R=R, S=S, Ca=Ca,
                             precision=int(rng.uniform() < fp16_fraction))
        out.append(Request(id=i, arrival=t, params=p, fields=f))
    return out


def make_planar_requests(n, seed=0, heights=(32, 48, 64), rate=1.0, width=4):
    """Two-layer planar requests (the Sec. 6.1 set-up of workloads.planar_layers): width x
    height lattices with the height drawn from `heights`, permittivity ratio log-uniform on
    [2, 20] and conductivity ratio log-uniform on [0.05, 0.5] (seeded), FP32; Poisson
    arrivals at `rate` per second.  Unlike droplet requests these reach a steady state
    (charge relaxed, fluid at rest) within tens of thousands of steps."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate) if rate > 0 else 0.0
        ny = int(rng.choice(heights))
        eps_ratio = float(10.0 ** rng.uniform(math.log10(2.0), math.log10(20.0)))
        sigma_ratio = float(10.0 ** rng.uniform(math.log10(0.05), math.log10(0.5)))
        p, f = wl.planar_layers(nx=width, ny=ny, eps_ratio=eps_ratio, sigma_ratio=sigma_ratio,
                                sigma_v=0.02)
        out.append(Request(id=i, arrival=t, params=p, fields=f))
    return out


class WallClock:
    def __init__(self):
        self.t0 = time.perf_counter()

    def now(self):
        return time.perf_counter() - self.t0

    def sleep_until(self, t):
        d = t - self.now()
        if d > 0:
            time.sleep(d)


def serve(backend, requests, clock, window=500, on_finish=None):
    """Runs the requests through the backend; returns them with admission and finish
    times filled.  Admission is first fit over the queue in arrival order (a request that
    does not fit does not block smaller ones behind it).  A request whose admission fails
    (an error from the backend, e.g. an allocation that fails or bad parameters) or whose
    state turns non-finite ends as failed, and the others run on."""
    pending = sorted(requests, key=lambda r: r.arrival)
    queue = []
    live = {}
    done = []
    i = 0
    spent = {"admit": 0.0, "run": 0.0, "poll": 0.0, "retire": 0.0}
    serve.spent = spent
    while i < len(pending) or queue or live:
        now = clock.now()
        while i < len(pending) and pending[i].arrival <= now:
            queue.append(pending[i])
            i += 1
        still = []
        for r in queue:
            t0 = clock.now()
            try:
                slot = backend.admit(r.params, r.fields, r.id)
            except (RuntimeError, MemoryError, ValueError) as e:
                spent["admit"] += clock.now() - t0
                r.failed = f"admission: {e}"
                r.admitted = r.finished = clock.now()
                done.append(r)
                continue
            spent["admit"] += clock.now() - t0
            if slot is None:
                still.append(r)
            else:
                r.admitted = clock.now()
                live[slot] = r
        queue = still
        if not live:
            if i < len(pending):
                clock.sleep_until(pending[i].arrival)
                continue
            if queue:
                raise RuntimeError("a queued request can never be admitted (larger than the batch)")
            break
        t0 = clock.now()
        backend.run(window)
        t1 = clock.now()
        status = backend.poll()
        spent["run"] += t1 - t0
        spent["poll"] += clock.now() - t1
        for st in status:
            r = live.get(st["slot"])
            if r is None:
                continue
            r.steps = st["steps"]
            r.iters = st.get("poisson_iters", 0)
            r.rel_change = (st["rel_change_phi"], st["rel_change_u"])
            if st["steady"] or st["capped"] or st["status"] == 5:
                r.steady = bool(st["steady"]) and st["status"] != 5
                r.capped = bool(st["capped"]) and not r.steady
                if st["status"] == 5:
                    r.failed = "non-finite state"
                r.finished = clock.now()
                if on_finish is not None:
                    on_finish(backend, st["slot"], r)
                t0 = clock.now()
                backend.retire(st["slot"])
                spent["retire"] += clock.now() - t0
                del live[st["slot"]]
                done.append(r)
    return done


def summarize(done, wall):
    """Latencies and throughput over the requests that ran to an end (steady or capped);
    failed ones are counted apart.  Admit-to-steady percentiles cover the steady requests
    only (None when none became steady); admit-to-end covers every completed request."""
    ok = [r for r in done if not r.failed]
    lat = np.array([r.finished - r.arrival for r in ok])
    run = np.array([r.finished - r.admitted for r in ok])
    run_steady = np.array([r.finished - r.admitted for r in ok if r.steady])

    def pct(a, q):
        return float(np.percentile(a, q)) if len(a) else None

    return {
        "requests": len(done),
        "steady": int(sum(r.steady for r in done)),
        "capped": int(sum(r.capped for r in done)),
        "failed": int(sum(bool(r.failed) for r in done)),
        "wall_s": wall,
        "sims_per_hour": len(ok) / wall * 3600.0 if wall > 0 else math.nan,
        "p50_latency_s": pct(lat, 50),
        "p99_latency_s": pct(lat, 99),
        "p50_admit_to_end_s": pct(run, 50),
        "p99_admit_to_end_s": pct(run, 99),
        "p50_admit_to_steady_s": pct(run_steady, 50),
        "p99_admit_to_steady_s": pct(run_steady, 99),
        "steps_total": int(sum(r.steps for r in ok)),
        "node_steps_total": int(sum(r.steps * r.params["nx"] * r.params["ny"] for r in done)),
        "poisson_iters_per_step": (float(sum(r.iters for r in done)) /
                                   max(1, sum(r.steps for r in done))),
    }


class OneAtATime:
    """Backend that runs one request at a time on its own simulation (no batching).
    plain=True: the straightforward path -- FP32 populations, the streaming potential
    kernel, every kernel queued from the host (no graphs) and the stopping rule checked on
    the host.  plain=False: the library's best single-simulation path -- FP32 populations,
    the on-chip potential loop where it fits, one captured graph per step."""

    def __init__(self, steady_tol=1e-6, step_cap=300000, plain=True):
        from . import ehd
        self.ehd = ehd
        self.tol = steady_tol
        self.cap = step_cap
        self.plain = plain
        self.sim = None
        self.req = None
        self.steps = 0
        self.prev = None
        self.rel = (math.inf, math.inf)
        self.at_rest = False

    def admit(self, params, fields, rid):
        if self.sim is not None:
            return None
        p = dict(params)
        p["precision"] = 0
        if self.plain:
            p["poisson_loop"] = 1
        self.sim = self.ehd.Sim(p)
        if self.plain:
            self.sim.use_graphs(False)  # the host-driven loop, kernel by kernel
        self.sim.set_fields(fields["phi"], fields["q"], fields["ux"], fields["uy"])
        self.rid = rid
        self.steps = 0
        self.iters = 0
        self.prev = None
        self.rel = (math.inf, math.inf)
        self.at_rest = False
        return 0

    def _snap(self):
        F = self.sim.read_fields(("phi", "ux", "uy"))
        return F["phi"], np.stack([F["ux"], F["uy"]])

    def run(self, n):
        if self.sim is None:
            return 0
        st = self.sim.step(n, stats=True)
        self.iters += st.get("poisson_iters_total", 0)
        self.steps += n
        phi, u = self._snap()
        if self.prev is not None:
            p0, u0 = self.prev
            # the batch's rule: velocities below 1e-6 (lattice units) count as rest in the
            # denominator of u's relative change
            u_floor = math.sqrt(1e-12 * phi.size)
            self.rel = (float(np.linalg.norm(phi - p0) / max(np.linalg.norm(phi), 1e-300)),
                        float(np.linalg.norm(u - u0) / max(np.linalg.norm(u), u_floor)))
        self.prev = (phi, u)
        self.at_rest = bool(np.sqrt(np.mean(np.sum(u * u, axis=0))) < 1e-6)
        return 0

    def poll(self):
        if self.sim is None:
            return []
        # the batch's rule: phi's relative change below the tolerance, and u's too unless
        # the flow is at rest (RMS speed below 1e-6 lattice units)
        steady = self.rel[0] < self.tol and (self.rel[1] < self.tol or self.at_rest)
        return [dict(slot=0, live=1, request_id=self.rid, steps=self.steps, poisson_iters=self.iters,
                     steady=int(steady), capped=int(self.steps >= self.cap), status=0,
                     rel_change_phi=self.rel[0], rel_change_u=self.rel[1])]

    def retire(self, slot):
        self.sim.close()
        self.sim = None


def warm_up(backend):
    """One tiny request through the backend before any clock starts (device context,
    module loading, first graph instantiation)."""
    p, f, _ = wl.droplet(N=32, r=5.0, R=1.0, S=1.0, Ca=0.1)
    slot = backend.admit(p, f, -1)
    backend.run(2)
    backend.retire(slot)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--requests", type=int, default=48)
    ap.add_argument("--sizes", default="64,128,256,512")
    ap.add_argument("--rate", type=float, default=4.0)
    ap.add_argument("--budget-gb", type=float, default=2.0)
    ap.add_argument("--slots", type=int, default=64)
    ap.add_argument("--window", type=int, default=500)
    ap.add_argument("--tol", type=float, default=1e-6)
    ap.add_argument("--cap", type=int, default=20000)
    ap.add_argument("--baseline", action="store_true")
    ap.add_argument("--tune", action="store_true", help="autotune the batch schedule first")
    args = ap.parse_args()
    from . import ehd
    sizes = tuple(int(x) for x in args.sizes.split(","))
    reqs = make_requests(args.requests, sizes=sizes, rate=args.rate)
    b = ehd.Batch(int(args.budget_gb * (1 << 30)), max_slots=args.slots, steady_tol=args.tol,
                  step_cap=args.cap)
    if args.tune:
        from . import autotune
        sample = [(r.params, r.fields) for r in make_requests(8, seed=99, sizes=sizes, rate=0.0)]
        b.set_schedule(**autotune.tune_batch(sample, budget=int(args.budget_gb * (1 << 30))))
    warm_up(b)
    clock = WallClock()
    done = serve(b, reqs, clock, window=args.window)
    out = {"batched": summarize(done, clock.now())}
    out["batched"]["seconds_in"] = dict(serve.spent)
    if args.baseline:
        reqs = make_requests(args.requests, sizes=sizes, rate=args.rate)
        plain = OneAtATime(args.tol, args.cap)
        warm_up(plain)
        clock = WallClock()
        done = serve(plain, reqs, clock, window=args.window)
        out["one_at_a_time_plain"] = summarize(done, clock.now())
        out["one_at_a_time_plain"]["seconds_in"] = dict(serve.spent)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
