"""Failure detection without a GPU fault: the on-chip potential loop's grid barrier waits
with a time limit.  A diagnostic makes the barrier's count unreachable for one solve; the
waits run out (2 s), the kernel returns early, the call reports EHD_ERR_TIMEOUT and the
CUDA context stays usable for the next simulation."""
import time

import numpy as np
import pytest

from paper_2407_01654_gb300 import workloads as wl

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


def run(ehd, p, f, steps):
    s = ehd.Sim(p)
    s.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    st = s.step(steps)
    out = s.read_fields()
    s.close()
    return st, out


@pytest.mark.parametrize("loop", [2, 3, 4], ids=["one-step", "two-step", "three-step"])
def test_barrier_timeout_is_reported_and_the_context_recovers(gpu, loop):
    """Each on-chip loop has its own grid barrier; each gives up within the limit."""
    p, f, _ = wl.droplet(N=96, r=15.0, R=3.0, S=0.5, Ca=0.2, poisson_fixed_iter=5,
                         poisson_loop=loop)
    st0, ref = run(gpu, p, f, 6)
    assert st0["status"] == 0
    s = gpu.Sim(p)
    assert s.loop_kind() == loop
    s.set_fields(f["phi"], f["q"], f["ux"], f["uy"])
    s.step(2)
    s.diag_expire_barrier()
    t0 = time.perf_counter()
    with pytest.raises(gpu.EhdError) as err:
        s.step(1)
    dt = time.perf_counter() - t0
    assert err.value.code == 9                # EHD_ERR_TIMEOUT
    assert 1.5 < dt < 30.0                    # the 2 s limit, not a hang
    s.close()
    st1, again = run(gpu, p, f, 6)            # same context: a fresh simulation is exact
    assert st1["status"] == 0
    for k in ref:
        assert np.array_equal(again[k], ref[k]), k


def test_streaming_loop_has_no_barrier_to_expire(gpu):
    p, f, _ = wl.droplet(N=64, r=10.0, R=3.0, S=0.5, Ca=0.2, poisson_loop=1)
    s = gpu.Sim(p)
    with pytest.raises(gpu.EhdError):
        s.diag_expire_barrier()
    s.close()
