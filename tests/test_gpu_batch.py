"""The batch (serving) layer on the GPU: many simulations resident in one arena, one
shared cooperative launch for all potential loops, continuous admission."""
import numpy as np
import pytest

from paper_2407_01654_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "q", "varphi", "Ex", "Ey", "ux", "uy", "p")


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_01654_gb300 import build
    build.build()
    from paper_2407_01654_gb300 import ehd
    return ehd


def request(N, seed, **over):
    R, S, Ca = wl.droplet_ratios(seed)
    p, f, _ = wl.droplet(N=N, r=0.156 * N, R=R, S=S, Ca=Ca, **over)
    return p, wl.perturbed(p, f, seed=seed, u_amp=1e-3, q_amp=1e-4)


def test_alone_equals_in_mix(gpu):
    """A request gives bit-identical fields alone in a batch and in a mix of requests of
    other sizes and parameters admitted at different times (stopping rule on)."""
    pa, fa = request(96, 1)
    alone = gpu.Batch(256 << 20, max_slots=4)
    s = alone.admit(pa, fa, 1)
    for _ in range(4):
        alone.run(60)
    ref = alone.read_fields(s)
    mix = gpu.Batch(512 << 20, max_slots=8)
    pb, fb = request(64, 2)
    pc, fc = request(128, 3, precision=1)
    sb = mix.admit(pb, fb, 2)
    mix.run(60)                     # b runs alone for a while
    sa = mix.admit(pa, fa, 1)       # a joins while b is live
    sc = mix.admit(pc, fc, 3)
    for _ in range(3):
        mix.run(60)
    mix.retire(sb)                  # b leaves mid-way
    mix.run(60)
    got = mix.read_fields(sa)
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k


def test_batch_slot_matches_single_simulation(gpu):
    """With a fixed sub-iteration count a batch slot and a plain simulation run the same
    arithmetic: bitwise equal fields (their potential tilings differ)."""
    p, f = request(80, 4, poisson_fixed_iter=4)
    b = gpu.Batch(128 << 20, max_slots=2)
    s = b.admit(p, f, 0)
    b.run(50)
    g = gpu.Sim(p)
    g.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    g.step(50)
    got, ref = b.read_fields(s), g.read_fields()
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k


def test_batch_slots_match_oracle(gpu):
    """Each slot of a mixed batch against the FP64 oracle directly: an FP32 slot and an
    FP16-deviation slot of different sizes and parameters, admitted together, 100 steps at
    a fixed sub-iteration count.  FP32 slot: relative L2 <= 1e-5 per field (the chemical
    potential against its terms' scale, times the Laplacian's gain); FP16 slot: <= 5e-3
    per field, the bar of the FP16 storage parity test."""
    from oracle import ehd as orc
    from test_gpu_parity import FP16_BAR, GROUPS, MU_GAIN, TOL_FIXED, mu_error, rel
    pa, fa = request(64, 21, poisson_fixed_iter=3)
    pb, fb = request(48, 22, poisson_fixed_iter=3, precision=1)
    b = gpu.Batch(256 << 20, max_slots=4)
    sa = b.admit(pa, fa, 0)
    sb = b.admit(pb, fb, 1)
    assert sa is not None and sb is not None
    b.run(100)
    for slot, (p, f), bar in ((sa, (pa, fa), TOL_FIXED), (sb, (pb, fb), FP16_BAR)):
        o = orc.Sim(p)
        o.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
        o.step(100)
        fo, fg = o.fields(), b.read_fields(slot)
        errs = {g: rel(np.stack([fg[k] for k in ks]), np.stack([fo[k] for k in ks]))
                for g, ks in GROUPS.items()}
        errs["mu"] = mu_error(o.P, fo, fg) / MU_GAIN
        print("batch slot vs oracle", "fp16" if p["precision"] else "fp32",
              {k: f"{v:.2e}" for k, v in errs.items()})
        assert all(v <= bar for v in errs.values()), errs
    assert all(st["steps"] == 100 for st in b.poll())


def test_admission_refusals_and_retire(gpu):
    """Admission is refused (the batch unchanged) when the arena, the slot count or the
    on-chip tile capacity would overflow; retiring frees the room again."""
    p, f = request(128, 5)
    ws_small = gpu.Batch(2 << 20, max_slots=4)          # arena too small for the request
    assert ws_small.admit(p, f, 0) is None and ws_small.info()["live_slots"] == 0
    b = gpu.Batch(64 << 20, max_slots=2)
    base = b.info()["arena_used"]
    s0 = b.admit(p, f, 0)
    s1 = b.admit(p, f, 1)
    assert s0 is not None and s1 is not None
    assert b.admit(p, f, 2) is None                      # no free slot
    b.run(20)
    b.retire(s0)
    assert b.info()["live_slots"] == 1
    s2 = b.admit(p, f, 2)
    assert s2 == s0
    b.retire(s1)
    b.retire(s2)
    assert b.info()["arena_used"] == base and b.info()["tiles_used"] == 0
    big = gpu.Batch(16 << 30, max_slots=4)
    cap = big.info()["tile_capacity"]
    pb, fb = request(512, 6)
    admitted = [big.admit(pb, fb, i) for i in range(4)]  # 128 tiles each
    assert sum(a is not None for a in admitted) == cap // 128


def test_admission_normalises_the_potential_loop(gpu):
    """A batch runs every slot's potential loop on chip with one sub-iteration per
    exchange: requests asking for the two- or three-step loop are admitted (whatever the
    batch's tile height) and compute the same fields; one asking for the streaming loop
    is refused as an invalid argument, not as a full batch."""
    p, f = request(96, 7, poisson_fixed_iter=4)
    res = []
    for loop in (2, 3, 4):
        b = gpu.Batch(256 << 20, max_slots=2)
        s = b.admit({**p, "poisson_loop": loop}, f, 0)
        assert s is not None
        b.run(30)
        res.append(b.read_fields(s))
    for r in res[1:]:
        for k in FIELDS:
            assert np.array_equal(r[k], res[0][k]), k
    b = gpu.Batch(64 << 20, max_slots=2)
    with pytest.raises(gpu.EhdError) as e:
        b.admit({**p, "poisson_loop": 1}, f, 0)
    assert e.value.code == 1
    assert b.info()["live_slots"] == 0


def test_step_cap_and_steadiness(gpu):
    """Status reporting: channel flow started at its steady profile is steady (relative
    change of u over a window well below 1e-3); a droplet request that is still moving is
    not; every slot reports its step count, the cap and its request id."""
    ny, nu, g = 32, 0.1, 1e-6
    p = wl.make_params(nx=64, ny=ny, walls_y=1, mu_l=nu, mu_v=nu, body_gx=g)
    y = np.arange(ny, dtype=float)
    ua = np.repeat((g / (2 * nu) * (y + 0.5) * (ny - 0.5 - y))[:, None], 64, axis=1)
    z = np.zeros((ny, 64))
    b = gpu.Batch(64 << 20, max_slots=2, steady_tol=1e-3, step_cap=800)
    s = b.admit(p, dict(phi=z, q=z, ux=ua, uy=z), 7)
    pd, fd = request(64, 9)
    sd = b.admit(pd, fd, 8)
    b.run(400)
    b.run(400)
    st = {x["slot"]: x for x in b.poll()}
    assert st[s]["steps"] == 800 and st[s]["capped"] == 1 and st[s]["request_id"] == 7
    assert st[s]["steady"] == 1 and st[s]["rel_change_u"] < 1e-3
    assert st[sd]["steady"] == 0 and st[sd]["rel_change_u"] > 1e-3


def test_serving_loop_runs_requests(gpu):
    """End-to-end serving on a small stream of requests: every request finishes, admission
    overlaps them on the device, latencies are recorded."""
    from paper_2407_01654_gb300 import serve
    reqs = serve.make_requests(6, seed=11, sizes=(32, 64), rate=200.0)
    b = gpu.Batch(256 << 20, max_slots=8, steady_tol=1e-4, step_cap=1500)
    clock = serve.WallClock()
    done = serve.serve(b, reqs, clock, window=250)
    assert len(done) == 6
    s = serve.summarize(done, clock.now())
    assert s["sims_per_hour"] > 0 and s["p99_latency_s"] >= s["p50_latency_s"]
    assert all(r.arrival <= r.admitted <= r.finished for r in done)


@pytest.mark.parametrize("rows,spg", [(16, 8), (64, 32)])
def test_alone_equals_in_mix_other_schedules(gpu, rows, spg):
    """The alone-versus-mix guarantee holds for every batch schedule."""
    pa, fa = request(96, 1)
    alone = gpu.Batch(256 << 20, max_slots=4)
    assert alone.set_schedule(rows, spg)
    s = alone.admit(pa, fa, 1)
    for _ in range(3):
        alone.run(50)
    ref = alone.read_fields(s)
    mix = gpu.Batch(512 << 20, max_slots=8)
    assert mix.set_schedule(rows, spg)
    pb, fb = request(64, 2)
    pc, fc = request(128, 3, precision=1)
    sb = mix.admit(pb, fb, 2)
    mix.run(50)
    sa = mix.admit(pa, fa, 1)
    sc = mix.admit(pc, fc, 3)
    mix.run(50)
    mix.retire(sb)
    mix.run(100)
    got = mix.read_fields(sa)
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k
    assert mix.info()["tile_rows"] == rows and mix.info()["steps_per_graph"] == spg
    assert sc is not None


def test_schedules_compute_the_same_fields(gpu):
    """At a fixed sub-iteration count every tile height gives identical fields, and the
    schedule cannot change while a slot is live."""
    p, f = request(100, 4, poisson_fixed_iter=4)
    out = []
    for rows, spg in ((16, 8), (32, 16), (64, 32)):
        b = gpu.Batch(128 << 20, max_slots=2)
        assert b.set_schedule(rows, spg)
        s = b.admit(p, f, 0)
        assert not b.set_schedule(32, 16)
        b.run(37)
        out.append(b.read_fields(s))
        b.close()
    for k in FIELDS:
        assert np.array_equal(out[0][k], out[1][k]) and np.array_equal(out[1][k], out[2][k]), k


def test_tuned_batch_schedule(gpu, tmp_path, monkeypatch):
    from paper_2407_01654_gb300 import autotune
    monkeypatch.setenv("EHD_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    reqs = [request(n, i) for i, n in enumerate((64, 64, 128, 256))]
    best = autotune.tune_batch(reqs, steps=32, budget=512 << 20)
    assert best in autotune.batch_candidates()


def test_non_finite_request_is_refused_without_disturbing_the_batch(gpu):
    """A request with a NaN in phi is refused at admission (EHD_ERR_NONFINITE), its
    workspace given back; the requests already in the batch compute exactly what they
    compute without the attempt, and the serving loop records the request as failed."""
    from paper_2407_01654_gb300 import serve
    pa, fa = request(64, 5)
    ref_b = gpu.Batch(128 << 20, max_slots=4)
    s = ref_b.admit(pa, fa, 1)
    ref_b.run(100)
    ref = ref_b.read_fields(s)
    ref_b.close()

    b = gpu.Batch(128 << 20, max_slots=4)
    s = b.admit(pa, fa, 1)
    b.run(40)
    before = b.info()
    pn, fn = request(64, 6)
    fn = dict(fn)
    fn["phi"] = fn["phi"].copy()
    fn["phi"][10, 10] = np.nan
    with pytest.raises(gpu.EhdError) as err:
        b.admit(pn, fn, 2)
    assert err.value.code == 5
    after = b.info()
    for key in ("live_slots", "arena_used", "tiles_used"):
        assert after[key] == before[key], key
    b.run(60)
    got = b.read_fields(s)
    for k in FIELDS:
        assert np.array_equal(got[k], ref[k]), k
    b.close()

    # through the serving loop: the bad request ends as failed, the good one runs on
    reqs = [serve.Request(id=0, arrival=0.0, params=pa, fields=fa),
            serve.Request(id=1, arrival=0.0, params=pn, fields=fn)]
    be = gpu.Batch(128 << 20, max_slots=4, steady_tol=1e-30, step_cap=200)
    done = serve.serve(be, reqs, serve.WallClock(), window=100)
    by = {r.id: r for r in done}
    assert by[1].failed.startswith("admission") and by[0].capped and not by[0].failed
    be.close()
