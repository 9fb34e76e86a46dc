"""The synchronisation floor of the two-step on-chip loop (ehd_diag_grid_exchange): the
loop's exchange alone (band export, grid barrier, ring import) costs less than a cycle of
the loop itself, and a lattice with more tiles than SMs is refused before any launch."""
import pytest

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ehd():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_01654_gb300 import build
    build.build()
    from paper_2407_01654_gb300 import ehd
    return ehd


def test_exchange_floor_is_below_a_loop_cycle(ehd):
    import numpy as np
    from paper_2407_01654_gb300 import workloads as wl
    floor = ehd.grid_exchange_floor(512, 1024)
    assert np.isfinite(floor) and 0.0 < floor < 20e-6
    # a cycle of the loop on the same lattice: two sub-iterations at a fixed count
    p, f, _ = wl.sessile_drop(seed=0)
    p.update(poisson_loop=3, tile_rows=56)
    times = {}
    for k in (4, 24):
        p["poisson_fixed_iter"] = k
        s = ehd.Sim(p)
        s.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
        s.step(3, stats=False)
        s.read_stats()
        import time
        t0 = time.perf_counter()
        s.step(40, stats=False)
        s.read_stats()
        times[k] = (time.perf_counter() - t0) / 40
        s.close()
    cycle = (times[24] - times[4]) / 10
    assert floor < cycle, (floor, cycle)


def test_more_tiles_than_sms_is_refused(ehd):
    import torch
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    # 64 x 56 tiles: a lattice with more of them than SMs cannot run one tile per SM
    nty = sms // 3 + 1
    with pytest.raises(ehd.EhdError):
        ehd.grid_exchange_floor(64 * 4, 56 * nty)
