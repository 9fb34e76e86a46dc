"""Non-finite input is reported, not hidden: a NaN in phi passed to ehd_set_fields makes
the call (and every later step of that simulation) return EHD_ERR_NONFINITE, the
potential loop stops after one sub-iteration instead of running to its cap, the state
holds the bad value, and a fresh simulation on the same context afterwards computes
exactly what it computed before.  The fault is made on the host; nothing faults on the
GPU."""
import numpy as np
import pytest

from test_gpu_parity import ALL_FIELDS, droplet_box

pytestmark = pytest.mark.gpu

NONFINITE = 5


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_01654_gb300 import build
    build.build()
    from paper_2407_01654_gb300 import ehd
    return ehd


def clean_run(gpu, p, f):
    g = gpu.Sim(p)
    assert g.set_fields(f["phi"], f["q"], f["ux"], f["uy"]) == 0
    st = g.step(5)
    out = g.read_fields()
    g.close()
    return st, out


@pytest.mark.parametrize("loop", [pytest.param(1, id="stream"), pytest.param(3, id="resident2")])
@pytest.mark.parametrize("rule", [pytest.param(False, id="fixed"), pytest.param(True, id="rule")])
def test_nan_in_phi_is_reported(gpu, loop, rule):
    over = dict(poisson_loop=loop)
    if not rule:
        over["poisson_fixed_iter"] = 3
    p, f = droplet_box(64, 40, 9.0, seed=14, **over)
    st0, f0 = clean_run(gpu, p, f)
    assert st0["status"] == 0 and st0["nonfinite"] == 0

    bad = dict(f)
    bad["phi"] = f["phi"].copy()
    bad["phi"][17, 23] = np.nan
    g = gpu.Sim(p)
    assert g.set_fields(bad["phi"], bad["q"], bad["ux"], bad["uy"]) == NONFINITE
    phi = g.read_fields(("phi",))["phi"]
    assert np.isnan(phi[17, 23])
    far = np.ones_like(phi, dtype=bool)
    far[15:20, 21:26] = False
    assert np.isfinite(phi[far]).all()
    st = g.step(3)
    assert st["status"] == NONFINITE and st["nonfinite"] == 1 and st["step"] == 3
    # the loop gave up at once (a NaN can never meet the stopping rule)
    assert st["poisson_iters_max"] == 1 and st["not_converged_steps"] == 3
    it, _, code = g.solve_potential()
    assert code == NONFINITE and it == 1
    g.close()

    st1, f1 = clean_run(gpu, p, f)
    assert st1["status"] == 0 and st1["poisson_iters_total"] == st0["poisson_iters_total"]
    for k in ALL_FIELDS:
        assert np.array_equal(f0[k], f1[k]), k
