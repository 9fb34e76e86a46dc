"""Autotuner on the GPU: every candidate schedule computes the same bits, and the tuned
schedule runs."""
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


def run(ehd, p, f, steps):
    s = ehd.Sim(p)
    s.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    s.step(steps)
    out = s.read_fields()
    loop = s.loop_kind()
    s.close()
    return out, loop


def test_every_schedule_computes_the_same_bits(gpu):
    """Ragged 150 x 70 sessile drop with a rising ramp, 6 sub-iterations per step: the
    streaming loop and the on-chip loops (one, two, three sub-iterations per exchange) at
    every tile height give identical fields."""
    from paper_2407_01654_gb300 import autotune
    p, f, _ = wl.sessile_drop(nx=150, ny=70, r=20.0, theta=70.0, ramp_steps=60, start_step=10,
                              poisson_fixed_iter=6)
    f = wl.perturbed(p, f, seed=3, u_amp=1e-3, q_amp=1e-4)
    ref, _ = run(gpu, p, f, 30)
    kinds = set()
    for ov in autotune.candidates(p):
        got, loop = run(gpu, {**p, **ov}, f, 30)
        kinds.add(loop)
        for k in FIELDS:
            assert np.array_equal(got[k], ref[k]), (ov, k)
    assert kinds == {1, 2, 3, 4}


def test_tuned_schedule_runs_with_the_stopping_rule(gpu, tmp_path, monkeypatch):
    from paper_2407_01654_gb300 import autotune
    monkeypatch.setenv("EHD_AUTOTUNE_CACHE", str(tmp_path / "tune.json"))
    p, f, _ = wl.sessile_drop(nx=256, ny=256, r=40.0, theta=80.0, ramp_steps=100,
                              start_step=50)
    ov = autotune.tune(p, steps=8)
    assert set(ov) == {"poisson_loop", "tile_rows"}
    s = gpu.Sim({**p, **ov})
    s.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    st = s.step(5)
    assert st["status"] == 0 and st["poisson_iters_total"] >= 5
    assert s.loop_kind() == ov["poisson_loop"]
    assert autotune.tune(p) == ov  # cached
