"""The serving scheduler's policy on the CPU, with a fake batch backend and a fake clock:
continuous admission, first-fit over the queue, retirement on steady or cap, latency
bookkeeping, and host-side fault cases (a request that can never fit, a cancelled or
capped request freeing its slot)."""
import math

import pytest

from paper_2407_01654_gb300 import serve


class FakeClock:
    def __init__(self):
        self.t = 0.0

    def now(self):
        return self.t

    def sleep_until(self, t):
        self.t = max(self.t, t)


class FakeBatch:
    """Capacity in nodes; a run of n steps costs n * (live nodes) * 1e-9 s + 1e-4 s; a
    request is steady after `need[id]` steps."""

    def __init__(self, clock, capacity, need, cap=10 ** 9, slots=8):
        self.clock, self.capacity, self.need, self.cap, self.slots = clock, capacity, need, cap, slots
        self.live = {}
        self.used = 0
        self.max_live = 0

    def admit(self, params, fields, rid):
        n = params["nx"] * params["ny"]
        if self.used + n > self.capacity or len(self.live) >= self.slots:
            return None
        slot = min(set(range(self.slots)) - set(self.live))
        self.live[slot] = [rid, n, 0]
        self.used += n
        self.max_live = max(self.max_live, len(self.live))
        return slot

    def run(self, steps):
        self.clock.t += steps * sum(v[1] for v in self.live.values()) * 1e-9 + 1e-4
        for v in self.live.values():
            v[2] += steps

    def poll(self):
        return [dict(slot=s, steps=v[2], steady=int(v[2] >= self.need[v[0]]),
                     capped=int(v[2] >= self.cap), status=0, rel_change_phi=0.0,
                     rel_change_u=0.0) for s, v in self.live.items()]

    def retire(self, slot):
        self.used -= self.live.pop(slot)[1]


def req(i, t, n):
    return serve.Request(id=i, arrival=t, params=dict(nx=n, ny=n), fields={})


def test_all_requests_finish_with_consistent_times():
    clock = FakeClock()
    reqs = [req(i, 0.01 * i, 64 if i % 2 else 128) for i in range(20)]
    be = FakeBatch(clock, capacity=4 * 128 * 128, need={i: 1000 + 500 * (i % 3) for i in range(20)})
    done = serve.serve(be, reqs, clock, window=500)
    assert len(done) == 20 and all(r.steady for r in done)
    for r in done:
        assert r.arrival <= r.admitted <= r.finished
        assert r.steps >= be.need[r.id]
    s = serve.summarize(done, clock.now())
    assert s["p50_latency_s"] <= s["p99_latency_s"] and s["sims_per_hour"] > 0
    assert be.max_live > 1  # requests overlapped on the device


def test_continuous_admission_while_others_run():
    """A request arriving while a long one runs is admitted before the long one ends."""
    clock = FakeClock()
    reqs = [req(0, 0.0, 128), req(1, 1e-3, 64)]
    be = FakeBatch(clock, capacity=10 ** 6, need={0: 100000, 1: 1000})
    done = {r.id: r for r in serve.serve(be, reqs, clock, window=500)}
    assert done[1].admitted < done[0].finished
    assert done[1].finished < done[0].finished


def test_first_fit_does_not_block_small_requests():
    """A request too large for the free space waits; a smaller one behind it is admitted."""
    clock = FakeClock()
    reqs = [req(0, 0.0, 100), req(1, 1e-4, 100), req(2, 2e-4, 10)]
    be = FakeBatch(clock, capacity=100 * 100 + 10 * 10, need={0: 5000, 1: 1000, 2: 1000})
    done = {r.id: r for r in serve.serve(be, reqs, clock, window=500)}
    assert done[2].admitted < done[0].finished          # the small one went past the big one
    assert done[1].admitted >= done[0].finished          # the big one waited for room


def test_capped_request_frees_its_slot():
    clock = FakeClock()
    reqs = [req(0, 0.0, 64), req(1, 0.0, 64)]
    be = FakeBatch(clock, capacity=64 * 64, need={0: 10 ** 9, 1: 1000}, cap=3000)
    done = {r.id: r for r in serve.serve(be, reqs, clock, window=500)}
    assert done[0].capped and not done[0].steady and done[0].steps >= 3000
    assert done[1].steady and done[1].admitted >= done[0].finished
    assert be.used == 0 and not be.live


def test_request_larger_than_the_batch_is_an_error():
    clock = FakeClock()
    be = FakeBatch(clock, capacity=64 * 64, need={0: 1000})
    with pytest.raises(RuntimeError):
        serve.serve(be, [req(0, 0.0, 128)], clock, window=500)


def test_request_generator_is_seeded():
    a = serve.make_requests(6, seed=3, sizes=(16, 32), rate=2.0)
    b = serve.make_requests(6, seed=3, sizes=(16, 32), rate=2.0)
    assert [r.arrival for r in a] == [r.arrival for r in b]
    assert [r.params["nx"] for r in a] == [r.params["nx"] for r in b]
    assert all(r.params["nx"] in (16, 32) for r in a)
    assert a[-1].arrival > a[0].arrival > 0


class FailingBatch(FakeBatch):
    """A FakeBatch whose admission of the ids in `bad_alloc` fails (a mocked allocation
    failure) and whose requests in `nan` report a non-finite state after their first
    window."""

    def __init__(self, clock, capacity, need, bad_alloc=(), nan=(), **kw):
        super().__init__(clock, capacity, need, **kw)
        self.bad_alloc, self.nan = set(bad_alloc), set(nan)

    def admit(self, params, fields, rid):
        if rid in self.bad_alloc:
            raise MemoryError("mocked allocation failure")
        return super().admit(params, fields, rid)

    def poll(self):
        out = super().poll()
        for st in out:
            if self.live[st["slot"]][0] in self.nan and st["steps"] > 0:
                st["status"] = 5
        return out


def test_failed_requests_free_their_slots():
    """A request whose admission fails and one whose state turns non-finite end as failed;
    the other requests run to steady as before and the failures' slots are freed."""
    clock = FakeClock()
    be = FailingBatch(clock, capacity=64 * 64 * 2, need={0: 1000, 1: 1000, 2: 1500, 3: 1000},
                      bad_alloc={1}, nan={2}, slots=2)
    reqs = [req(i, 0.0, 64) for i in range(4)]
    done = serve.serve(be, reqs, clock, window=500)
    by = {r.id: r for r in done}
    assert len(done) == 4 and not be.live and be.used == 0
    assert by[1].failed.startswith("admission") and by[2].failed == "non-finite state"
    assert by[0].steady and by[3].steady and not by[0].failed and not by[3].failed
    s = serve.summarize(done, clock.now())
    assert s["failed"] == 2 and s["steady"] == 2


def test_admit_to_steady_counts_steady_requests_only():
    """Capped requests end at their cap, not at steady state: their admit-to-end times do
    not enter the admit-to-steady percentiles."""
    p = {"nx": 8, "ny": 8}

    def done(i, admitted, finished, steady):
        return serve.Request(id=i, arrival=0.0, params=p, fields={}, admitted=admitted,
                             finished=finished, steps=10, steady=steady, capped=not steady)

    capped_only = [done(0, 0.0, 5.0, False), done(1, 1.0, 9.0, False)]
    s = serve.summarize(capped_only, 10.0)
    assert s["steady"] == 0 and s["capped"] == 2
    assert s["p50_admit_to_steady_s"] is None and s["p99_admit_to_steady_s"] is None
    assert s["p50_admit_to_end_s"] == pytest.approx(6.5)
    mixed = capped_only + [done(2, 2.0, 3.0, True), done(3, 2.0, 5.0, True)]
    s = serve.summarize(mixed, 10.0)
    assert s["p50_admit_to_steady_s"] == pytest.approx(2.0)
    assert s["p99_admit_to_steady_s"] == pytest.approx(2.98)
    assert s["p99_admit_to_end_s"] == pytest.approx(7.91)  # 5 + 0.97 (8 - 5)
