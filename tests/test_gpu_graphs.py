"""ehd_step(n) launches runs of eight steps as one CUDA graph (the rest one graph per
step): the same bits and sub-iteration counts as one graph per step, whatever the copy the
run starts on, with the streaming loop's WHILE node and with the on-chip loop."""
import numpy as np
import pytest

from test_gpu_parity import ALL_FIELDS, droplet_box

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2407_01654_gb300 import build
    build.build()
    from paper_2407_01654_gb300 import ehd
    return ehd


def run(gpu, p, f, chunks):
    g = gpu.Sim(p)
    g.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    tot = 0
    for n in chunks:
        st = g.step(n)
        assert st["status"] == 0
        tot += st["poisson_iters_total"]
    out = g.read_fields()
    g.close()
    return tot, out


@pytest.mark.parametrize("loop", [pytest.param(1, id="stream"), pytest.param(3, id="resident2")])
def test_runs_of_steps_in_one_graph(gpu, loop):
    p, f = droplet_box(64, 48, 10.0, seed=12, poisson_loop=loop)
    ka, fa = run(gpu, p, f, [19])        # 8 + 8 + 3
    kb, fb = run(gpu, p, f, [1] * 19)    # one graph per step
    kc, fc = run(gpu, p, f, [3, 16])     # runs starting on the other population copy
    assert ka == kb == kc
    for k in ALL_FIELDS:
        assert np.array_equal(fa[k], fb[k]), k
        assert np.array_equal(fa[k], fc[k]), k


def test_read_fields_into_caller_owned_buffers(gpu):
    """Fields read into the caller's arrays (reused across two reads, as the end-to-end
    measurement does) equal the fields read into fresh arrays, bit for bit, host and
    device."""
    import torch
    p, f = droplet_box(64, 48, 10.0, seed=5, poisson_loop=3)
    g = gpu.Sim(p)
    g.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    bufs = {n: np.full((48, 64), np.nan) for n in gpu.FIELDS}
    dbufs = {n: torch.empty((48, 64), dtype=torch.float32, device="cuda") for n in gpu.FIELDS}
    for _ in range(2):
        g.step(3)
        fresh = g.read_fields()
        mine = g.read_fields(out=bufs)
        dev = g.read_fields(device=True, out=dbufs)
        for n in gpu.FIELDS:
            assert mine[n] is bufs[n] and dev[n] is dbufs[n]
            assert np.array_equal(fresh[n], bufs[n]), n
            assert np.array_equal(fresh[n], dbufs[n].cpu().numpy().astype(np.float64)), n
    g.close()
